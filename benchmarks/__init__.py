"""Measurement drivers (sweeps and workload timings) that the DESIGN and
profiles/ numbers come from; run as `python -m benchmarks.<name>`.  Not part
of the library: they call it through its public binding."""
