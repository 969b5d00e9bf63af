"""CPU model of the shared-memory operand layouts the tcgen05 reductions use
(csrc/reduce.cuh warp form, csrc/reduce_bench.cu block form): every store in
bounds, one slot per (thread, row), free of bank conflicts, and the 128-byte
swizzled K-major read pattern of every MMA (rows 128 bytes apart, 16-byte
chunk c of row r at chunk c ^ r inside 1024-byte atoms, atoms `sbo` bytes
apart along N) maps each (n, k) element back to the thread and row that
wrote it.  compute-sanitizer is not available, so the index arithmetic is
checked here before it runs on a GPU."""
import pytest


def swizzle(addr):
    return addr ^ (((addr >> 7) & 7) << 4)


def mma_reads(start, n_rows, sbo):
    """(n, k) -> byte address read by one K = 8 TF32 MMA with N = n_rows."""
    out = {}
    for n in range(n_rows):
        for kk in range(8):
            lin = start + (n // 8) * sbo + (n % 8) * 128 + (kk // 4) * 16 + (kk % 4) * 4
            out[(n, kk)] = swizzle(lin)
    return out


def groups(threads):
    w = threads // 32
    return 8 if w % 8 == 0 else 4 if w % 4 == 0 else 2 if w % 2 == 0 else 0


@pytest.mark.parametrize("threads", list(range(64, 1025, 64)))
def test_block_form_layout(threads):
    ng = groups(threads)
    assert ng
    size = 32 * threads
    owner = {}
    for tid in range(threads):
        w, lane = tid >> 5, tid & 31
        base = (w // ng) * (ng * 1024) + (w % ng) * 1024 + (lane & 3) * 4
        for r in range(8):
            a = base + r * 128 + (((lane >> 2) ^ r) << 4)
            assert 0 <= a < size and a not in owner
            owner[a] = (tid, r)
    for w in range(threads // 32):          # each per-row store of a warp: 32 distinct banks
        for r in range(8):
            banks = {((((w // ng) * ng * 1024 + (w % ng) * 1024 + (lane & 3) * 4
                        + r * 128 + (((lane >> 2) ^ r) << 4)) // 4) % 32) for lane in range(32)}
            assert len(banks) == 32
    seen = set()
    for s in range(threads // (8 * ng)):
        start = (s >> 2) * ng * 1024 + (s & 3) * 32
        for (n, kk), a in mma_reads(start, 8 * ng, 1024).items():
            tid, r = owner[a]
            w, lane = tid >> 5, tid & 31
            assert r == n % 8 and w % ng == n // 8 and 32 * (w // ng) + lane == 8 * s + kk
            seen.add((tid, r))
    assert len(seen) == 8 * threads


def test_warp_form_layout():
    """One warp's 2 KB B operand: rows 0-7 hi terms, 8-15 lo terms, K = lanes."""
    owner = {}
    for lane in range(32):
        cq = lane >> 2
        for c in range(8):
            for part in (0, 1):
                a = part * 1024 + c * 128 + ((cq ^ c) << 4) + (lane & 3) * 4
                assert 0 <= a < 2048 and a not in owner
                owner[a] = (lane, c + 8 * part)
    for c in range(8):
        for part in (0, 1):
            banks = {((part * 1024 + c * 128 + (((lane >> 2) ^ c) << 4) + (lane & 3) * 4) // 4) % 32
                     for lane in range(32)}
            assert len(banks) == 32
    seen = set()
    for s in range(4):                        # K = 32 lanes in four K = 8 slices
        for (n, kk), a in mma_reads(32 * s, 16, 1024).items():
            lane, row = owner[a]
            assert row == n and lane == 8 * s + kk
            seen.add((lane, row))
    assert len(seen) == 32 * 16


def test_ones_operand_stays_inside_its_buffer():
    """The all-ones A operand (128 x 8 TF32, no swizzle) is read with 128-byte
    strides both ways: every core matrix lies inside the 2304 bytes of ones,
    whichever stride the hardware applies along which dimension."""
    for lbo, sbo in ((128, 128),):
        top = max(g * sbo + k * lbo + 127 for g in range(16) for k in range(2))
        top2 = max(g * lbo + k * sbo + 127 for g in range(16) for k in range(2))
        assert max(top, top2) < 2304
