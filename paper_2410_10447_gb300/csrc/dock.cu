// Lamarckian GA around the fused local search (Sec. 2.1): initial
// population, one GA generation per launch, run-best and evaluation
// accounting, and the FP64 rescoring of every run's best genotype.
//
// The paper names the GA without its rules; the rules implemented here (and,
// independently, in the FP64 oracle) are:
//  - random words from Philox4x32-10 keyed by the seed, counter (individual,
//    generation, run, call); initial genotypes use generation 0xFFFFFFFF;
//  - individual 0 of a new generation is the previous generation's best;
//    every other child: two binary tournaments (lower energy wins, ties to
//    the lower index), two-point crossover with probability p_cross, per-gene
//    mutation with probability p_mut by a uniform offset in [-1, 1) times
//    mut_trans (translation genes) or mut_angle; torsions wrapped;
//  - each individual gets a local search of ls_iters evaluations (ADADELTA,
//    or a Solis-Wets search spending at most that many) with probability
//    ls_rate, otherwise one scoring evaluation;
//  - a run stops after max_gens generations or once its evaluation count
//    reaches max_evals;
//  - early stopping (optional): after every conv_every-th generation a run
//    stops once the population standard deviation of its conv_top lowest
//    energies is below conv_tol (double precision from the float energies).
#include <math.h>

#include "adgb_internal.cuh"
#include "philox.cuh"

namespace adgb {

namespace {

constexpr uint32_t INIT_GEN = 0xFFFFFFFFu;
constexpr float PI_F = 3.14159265358979f;

// word layout of child k in generation gen: 0-3 tournaments, 4 crossover?,
// 5-6 cut points, 7 local search?, 8+2j mutate gene j?, 9+2j its offset
enum { W_TOUR = 0, W_CROSS = 4, W_CUT = 5, W_LS = 7, W_MUT = 8 };

__global__ void init_pop_kernel(const RecDev rec, int T, uint64_t seed, int n_runs, int pop,
                                float *genes, int *iters) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_runs * pop) return;
    const int run = idx / pop, k = idx - run * pop, G = 6 + T;
    float *g = genes + (size_t)idx * G;
    const int n[3] = {rec.nx, rec.ny, rec.nz};
    for (int d = 0; d < 3; d++) {
        const float ext = (float)(n[d] - 1) * rec.h;
        g[d] = rec.lo[d] + ext * (0.2f + 0.6f * unit24(ga_word(seed, run, INIT_GEN, k, d)));
    }
    g[3] = 2.f * PI_F * unit24(ga_word(seed, run, INIT_GEN, k, 3)) - PI_F;
    g[4] = acosf(1.f - 2.f * unit24(ga_word(seed, run, INIT_GEN, k, 4)));
    g[5] = 2.f * PI_F * unit24(ga_word(seed, run, INIT_GEN, k, 5));
    for (int j = 0; j < T; j++)
        g[6 + j] = 2.f * PI_F * unit24(ga_word(seed, run, INIT_GEN, k, 6 + j)) - PI_F;
    iters[idx] = 1;
}

// lowest energy, ties to the lowest index, over a block
__device__ void block_argmin(float e, int k, float *s_e, int *s_k, float &best_e, int &best_k) {
    for (int off = 16; off > 0; off >>= 1) {
        const float oe = __shfl_xor_sync(0xffffffffu, e, off);
        const int ok = __shfl_xor_sync(0xffffffffu, k, off);
        if (oe < e || (oe == e && ok < k)) {
            e = oe;
            k = ok;
        }
    }
    const int w = threadIdx.x >> 5, W = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_e[w] = e;
        s_k[w] = k;
    }
    __syncthreads();
    best_e = s_e[0];
    best_k = s_k[0];
    for (int i = 1; i < W; i++)
        if (s_e[i] < best_e || (s_e[i] == best_e && s_k[i] < best_k)) {
            best_e = s_e[i];
            best_k = s_k[i];
        }
    __syncthreads();
}

__global__ void ga_kernel(int pop, int G, const float *go, const float *eo, const DockCfg d,
                          uint32_t gen, float *gn, int *iters, const int *done) {
    extern __shared__ float s_e[];  // [pop] energies, then argmin scratch
    float *s_we = s_e + pop;
    int *s_wk = reinterpret_cast<int *>(s_we + 32);
    const int run = blockIdx.x;
    const size_t base = (size_t)run * pop;
    float e = INFINITY;
    int kk = 0x7fffffff;
    for (int k = threadIdx.x; k < pop; k += blockDim.x) {
        const float v = eo[base + k];
        s_e[k] = v;
        if (v < e || (v == e && k < kk)) {
            e = v;
            kk = k;
        }
    }
    __syncthreads();
    float be;
    int bk;
    block_argmin(e, kk, s_we, s_wk, be, bk);
    if (bk < 0 || bk >= pop) bk = 0;
    const bool stop = done && done[run] != 0;
    for (int k = threadIdx.x; k < pop; k += blockDim.x) {
        float *child = gn + (base + k) * G;
        if (stop) {
            const float *src = go + (base + k) * G;
            for (int j = 0; j < G; j++) child[j] = src[j];
            iters[base + k] = 0;
            continue;
        }
        if (k == 0) {
            const float *src = go + (base + bk) * G;
            for (int j = 0; j < G; j++) child[j] = src[j];
        } else {
            int par[2];
            for (int t = 0; t < 2; t++) {
                const int a = index_below(ga_word(d.seed, run, gen, k, W_TOUR + 2 * t), pop);
                const int b = index_below(ga_word(d.seed, run, gen, k, W_TOUR + 2 * t + 1), pop);
                par[t] = (s_e[b] < s_e[a] || (s_e[b] == s_e[a] && b < a)) ? b : a;
            }
            const float *A = go + (base + par[0]) * G, *B = go + (base + par[1]) * G;
            int c1 = 0, c2 = 0;
            if (unit24(ga_word(d.seed, run, gen, k, W_CROSS)) < d.p_cross) {
                c1 = index_below(ga_word(d.seed, run, gen, k, W_CUT), G + 1);
                c2 = index_below(ga_word(d.seed, run, gen, k, W_CUT + 1), G + 1);
                if (c1 > c2) {
                    const int t = c1;
                    c1 = c2;
                    c2 = t;
                }
            }
            for (int j = 0; j < G; j++) {
                float v = (j >= c1 && j < c2) ? B[j] : A[j];
                if (unit24(ga_word(d.seed, run, gen, k, W_MUT + 2 * j)) < d.p_mut) {
                    const float off = 2.f * unit24(ga_word(d.seed, run, gen, k, W_MUT + 2 * j + 1)) - 1.f;
                    v += off * (j < 3 ? d.mut_trans : d.mut_angle);
                }
                if (j >= 6) v -= 2.f * PI_F * floorf((v + PI_F) * (0.5f / PI_F));
                child[j] = v;
            }
        }
        iters[base + k] = unit24(ga_word(d.seed, run, gen, k, W_LS)) < d.ls_rate ? d.ls_iters : 1;
    }
}

// A run evaluated in this pass (runs stopped before it have all iters 0).
__device__ __forceinline__ bool kk_eval_flag(const int *iters, size_t base, int pop) {
    return pop > 0 && iters[base] > 0;
}

// Sum of one double over the block (all threads get it).
__device__ double block_sum_f64(double v, double *s_d) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, W = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) s_d[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < W; i++) t += s_d[i];
    __syncthreads();
    return t;
}

// Early-stopping test of one run (whole block): the population standard
// deviation of the `top` lowest of e[0..pop) is below tol; never with a NaN
// energy in the population or a non-finite one among the lowest.  An
// energy's rank is the number of energies below it (ties by index), so the
// top set is the same multiset whatever the order; mean and spread in double.
__device__ bool run_converged(const float *e, int pop, int top, float tol, double *s_d) {
    double s = 0.0;
    int bad = 0;
    for (int k = threadIdx.x; k < pop; k += blockDim.x) {
        const float v = e[k];
        if (isnan(v)) bad = 1;
        int rank = 0;
        for (int j = 0; j < pop; j++) {
            const float u = e[j];
            rank += (u < v) || (u == v && j < k);
        }
        if (rank < top) {
            if (!isfinite(v)) bad = 1;
            s += (double)v;
        }
    }
    bad = __syncthreads_or(bad);
    const double mean = block_sum_f64(s, s_d) / top;
    double q = 0.0;
    for (int k = threadIdx.x; k < pop; k += blockDim.x) {
        const float v = e[k];
        int rank = 0;
        for (int j = 0; j < pop; j++) {
            const float u = e[j];
            rank += (u < v) || (u == v && j < k);
        }
        if (rank < top) q += ((double)v - mean) * ((double)v - mean);
    }
    const double var = block_sum_f64(q, s_d) / top;
    return !bad && var < (double)tol * (double)tol;
}

// ga_converged_dev: one block per run.
__global__ void conv_kernel(int pop, int top, float tol, const float *energy, int *converged) {
    __shared__ float s_e[1024];
    __shared__ double s_d[32];
    const int run = blockIdx.x;
    for (int k = threadIdx.x; k < pop; k += blockDim.x) s_e[k] = energy[(size_t)run * pop + k];
    __syncthreads();
    const bool c = run_converged(s_e, pop, top, tol, s_d);
    if (threadIdx.x == 0) converged[run] = c ? 1 : 0;
}

// After an evaluation pass: evaluation count, run best, stop flag (budget,
// or early stopping after every conv_every-th generation gen >= 1).
__global__ void best_kernel(int pop, int G, const float *genes, const float *energy,
                            const int *iters, float *best_genes, float *best_e,
                            long long *evals, int *done, long long max_evals, int gen,
                            int conv_every, int conv_top, float conv_tol) {
    __shared__ float s_we[32];
    __shared__ int s_wk[32];
    __shared__ long long s_n[32];
    __shared__ float s_e[1024];
    __shared__ double s_d[32];
    const int run = blockIdx.x;
    const size_t base = (size_t)run * pop;
    float e = INFINITY;
    int kk = 0x7fffffff;
    long long n = 0;
    for (int k = threadIdx.x; k < pop; k += blockDim.x) {
        const int it = iters[base + k];
        n += it;
        const float v = energy[base + k];
        if (it > 0 && (v < e || (v == e && k < kk))) {
            e = v;
            kk = k;
        }
    }
    for (int off = 16; off > 0; off >>= 1) n += __shfl_xor_sync(0xffffffffu, n, off);
    if ((threadIdx.x & 31) == 0) s_n[threadIdx.x >> 5] = n;
    float be;
    int bk;
    block_argmin(e, kk, s_we, s_wk, be, bk);
    if (threadIdx.x == 0) {
        long long tot = 0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); w++) tot += s_n[w];
        const long long ev = evals[run] + tot;
        evals[run] = ev;
        s_n[0] = (bk >= 0 && bk < pop && be < best_e[run]) ? 1 : 0;
        if (s_n[0]) best_e[run] = be;
        if (ev >= max_evals) done[run] = 1;
        s_wk[0] = bk;
    }
    __syncthreads();
    if (s_n[0]) {
        const int k = s_wk[0];
        for (int j = threadIdx.x; j < G; j += blockDim.x)
            best_genes[(size_t)run * G + j] = genes[(base + k) * G + j];
    }
    // the run is evaluated this generation (not stopped before it) and due a test
    if (conv_every > 0 && gen >= 1 && gen % conv_every == 0 && kk_eval_flag(iters, base, pop)) {
        for (int k = threadIdx.x; k < pop; k += blockDim.x) s_e[k] = energy[base + k];
        __syncthreads();
        const bool c = run_converged(s_e, pop, conv_top, conv_tol, s_d);
        if (threadIdx.x == 0 && c) done[run] = 1;
    }
}

__global__ void init_state_kernel(int n_runs, float *best_e, long long *evals, int *done) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n_runs) {
        best_e[r] = INFINITY;
        evals[r] = 0;
        done[r] = 0;
    }
}

// ------------------------------------------------------------ FP64 rescoring
// The force-field constants as exact decimals (the FP32 path uses their
// float roundings, which differ from these by up to 3e-8 relative).
constexpr double D_W_VDW = 0.1662, D_W_HB = 0.1209, D_W_EL = 0.1406, D_W_DS = 0.1322;
constexpr double D_ELEC = 332.06363, D_SIGMA = 3.6, D_QSOL = 0.01097, D_R_MIN = 0.5, D_W_OUT = 10.0;
constexpr double D_MS_A = -8.5525, D_MS_EPS0 = 78.4, D_MS_LAMBDA = 0.003627, D_MS_K = 7.7839;

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 dcross(D3 a, D3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ void drot(D3 &r, D3 c, D3 k, double s, double omc) {
    const D3 v = {r.x - c.x, r.y - c.y, r.z - c.z};
    const D3 kv = dcross(k, v), kkv = dcross(k, kv);
    r.x += s * kv.x + omc * kkv.x;
    r.y += s * kv.y + omc * kkv.y;
    r.z += s * kv.z + omc * kkv.z;
}

// Energy of one genotype in double precision (coordinates, grid terms and
// pair terms recomputed from the stored single-precision inputs).  One warp
// per genotype; coordinates in shared memory.
__global__ void rescore_fp64_kernel(const RecDev R, const LigDev L, int n, const float *genes,
                                    double *out) {
    extern __shared__ double s_x[];  // [warps][N][3]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pose = blockIdx.x * (blockDim.x >> 5) + warp;
    if (pose >= n) return;
    const int N = L.n_atoms, T = L.n_tors, G = 6 + T;
    double *X = s_x + (size_t)warp * N * 3;
    const float *g = genes + (size_t)pose * G;
    const double phi = g[3], th = g[4], al = g[5];
    const D3 u = {sin(th) * cos(phi), sin(th) * sin(phi), cos(th)};
    const double sa = sin(al), oca = 1.0 - cos(al);
    for (int i = lane; i < N; i += 32) {
        const float4 r4 = L.ref[i];
        D3 p = {r4.x, r4.y, r4.z};
        for (int k = L.frag[i]; k >= 0; k = L.tparent[k]) {
            const int4 ta = L.tatoms[k];
            const float4 a4 = L.ref[ta.x], b4 = L.ref[ta.y];
            D3 ax = {(double)b4.x - a4.x, (double)b4.y - a4.y, (double)b4.z - a4.z};
            const double l = sqrt(ax.x * ax.x + ax.y * ax.y + ax.z * ax.z);
            ax.x /= l;
            ax.y /= l;
            ax.z /= l;
            const double psi = g[6 + k];
            drot(p, D3{b4.x, b4.y, b4.z}, ax, sin(psi), 1.0 - cos(psi));
        }
        drot(p, D3{0.0, 0.0, 0.0}, u, sa, oca);
        X[3 * i] = p.x + g[0];
        X[3 * i + 1] = p.y + g[1];
        X[3 * i + 2] = p.z + g[2];
    }
    __syncwarp();
    double e = 0.0;
    const int nn[3] = {R.nx, R.ny, R.nz};
    for (int i = lane; i < N; i += 32) {
        const double q = L.ref[i].w, aq = fabs(q);
        const int t = L.type[i];
        double pc[3], f[3], pen = 0.0;
        int i0[3];
        for (int d = 0; d < 3; d++) {
            const double xv = X[3 * i + d];
            const double lo = R.lo[d], hi = (double)R.lo[d] + (double)(nn[d] - 1) * (double)R.h;
            pc[d] = xv < lo ? lo : (xv > hi ? hi : xv);
            pen += (xv - pc[d]) * (xv - pc[d]);
            const double uu = (pc[d] - lo) / (double)R.h;
            int c = (int)floor(uu);
            c = c < 0 ? 0 : (c > nn[d] - 2 ? nn[d] - 2 : c);
            i0[d] = c;
            f[d] = uu - c;
        }
        const size_t cell = ((size_t)i0[2] * (R.ny - 1) + i0[1]) * (R.nx - 1) + i0[0];
        const float *cp = R.cells + cell * (size_t)R.M * 8;
        double v = 0.0;
        for (int c = 0; c < 8; c++) {
            const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
            const double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) * (cz ? f[2] : 1.0 - f[2]);
            v += w * ((double)cp[8 * t + c] + q * (double)cp[8 * (R.M - 2) + c] +
                      aq * (double)cp[8 * (R.M - 1) + c]);
        }
        e += v + D_W_OUT * pen;
    }
    for (int p = lane; p < L.n_pairs; p += 32) {
        const uint32_t pr = L.pairs[p];
        const int i = pr & 255, j = (pr >> 8) & 255;
        const int ti = L.type[i], tj = L.type[j];
        const double dx = X[3 * i] - X[3 * j], dy = X[3 * i + 1] - X[3 * j + 1],
                     dz = X[3 * i + 2] - X[3 * j + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double rc = r > D_R_MIN ? r : D_R_MIN;
        const int hi = L.t_hb[ti], hj = L.t_hb[tj];
        double ev;
        if ((hi == 1 && hj == 2) || (hi == 2 && hj == 1)) {
            const double s = (double)L.hb_R / rc, s2 = s * s, s10 = s2 * s2 * s2 * s2 * s2;
            ev = D_W_HB * (double)L.hb_eps * (5.0 * s10 * s2 - 6.0 * s10);
        } else {
            const double Rij = 0.5 * ((double)L.t_R[ti] + (double)L.t_R[tj]);
            const double eij = sqrt((double)L.t_eps[ti] * (double)L.t_eps[tj]);
            const double s = Rij / rc, s2 = s * s, s6 = s2 * s2 * s2;
            ev = D_W_VDW * eij * (s6 * s6 - 2.0 * s6);
        }
        const double qi = L.ref[i].w, qj = L.ref[j].w;
        const double B = D_MS_EPS0 - D_MS_A;
        const double epsr = D_MS_A + B / (1.0 + D_MS_K * exp(-D_MS_LAMBDA * B * rc));
        const double eel = D_W_EL * D_ELEC * qi * qj / (rc * epsr);
        const double Si = (double)L.t_sol[ti] + D_QSOL * fabs(qi);
        const double Sj = (double)L.t_sol[tj] + D_QSOL * fabs(qj);
        const double sig = D_SIGMA;
        const double eds = D_W_DS * (Si * (double)L.t_vol[tj] + Sj * (double)L.t_vol[ti]) *
                           exp(-r * r / (2.0 * sig * sig));
        e += ev + eel + eds;
    }
    for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
    if (lane == 0) out[pose] = e;
}

// Raw Philox4x32-10 words: in [n][6] = (counter 0-3, key 0-1), out [n][4].
__global__ void philox_kernel(const uint32_t *in, int n, uint32_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t *c = in + (size_t)i * 6;
    const Philox4 o = philox4x32_10(c[0], c[1], c[2], c[3], c[4], c[5]);
    uint32_t *d = out + (size_t)i * 4;
    d[0] = o.x;
    d[1] = o.y;
    d[2] = o.z;
    d[3] = o.w;
}

}  // namespace

cudaError_t launch_philox(const uint32_t *in, int n, uint32_t *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    philox_kernel<<<(n + 255) / 256, 256, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

cudaError_t launch_init_population(const RecDev &rec, int n_tors, uint64_t seed, int n_runs, int pop,
                                   float *genes, int *iters, cudaStream_t s) {
    const int n = n_runs * pop;
    if (n == 0) return cudaSuccess;
    init_pop_kernel<<<(n + 127) / 128, 128, 0, s>>>(rec, n_tors, seed, n_runs, pop, genes, iters);
    return cudaGetLastError();
}

cudaError_t launch_ga_generation(const DockCfg &d, int G, int gen, const float *genes,
                                 const float *energy, float *genes_out, int *iters, cudaStream_t s) {
    const int gt = d.pop >= 1024 ? 1024 : ((d.pop + 31) / 32) * 32;
    const int gsm = (d.pop + 32) * 4 + 32 * 4;
    ga_kernel<<<d.n_runs, gt, gsm, s>>>(d.pop, G, genes, energy, d, (uint32_t)gen, genes_out, iters,
                                        nullptr);
    return cudaGetLastError();
}

// The steps of dock() one at a time, for the serving loop, which advances
// many jobs by one generation per tick.
cudaError_t launch_job_start(const RecDev &rec, int n_tors, const DockCfg &d, DockScratch &w,
                             cudaStream_t s) {
    const int n = d.n_runs * d.pop;
    init_state_kernel<<<(d.n_runs + 127) / 128, 128, 0, s>>>(d.n_runs, w.best_e, w.evals, w.done);
    init_pop_kernel<<<(n + 127) / 128, 128, 0, s>>>(rec, n_tors, d.seed, d.n_runs, d.pop,
                                                     w.genes[0], w.iters);
    return cudaGetLastError();
}

cudaError_t launch_job_ga(const DockCfg &d, int G, int gen, DockScratch &w, int cur, cudaStream_t s) {
    const int gt = d.pop >= 1024 ? 1024 : ((d.pop + 31) / 32) * 32;
    const int gsm = (d.pop + 32) * 4 + 32 * 4;
    ga_kernel<<<d.n_runs, gt, gsm, s>>>(d.pop, G, w.genes[cur], w.energy, d, (uint32_t)gen,
                                       w.genes[cur ^ 1], w.iters, w.done);
    return cudaGetLastError();
}

cudaError_t launch_job_best(const DockCfg &d, int G, int gen, DockScratch &w, int cur,
                            float *best_genes, cudaStream_t s) {
    best_kernel<<<d.n_runs, 128, 0, s>>>(d.pop, G, w.genes[cur], w.energy, w.iters, best_genes,
                                         w.best_e, w.evals, w.done, d.max_evals, gen, d.conv_every,
                                         d.conv_top, d.conv_tol);
    return cudaGetLastError();
}

cudaError_t launch_ga_converged(int n_runs, int pop, int top, float tol, const float *energy,
                                int *converged, cudaStream_t s) {
    conv_kernel<<<n_runs, 128, 0, s>>>(pop, top, tol, energy, converged);
    return cudaGetLastError();
}

cudaError_t launch_rescore_fp64(const RecDev &rec, const LigDev &lig, int n, const float *genes,
                                double *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int warps = 4;
    const int smem = warps * lig.n_atoms * 3 * (int)sizeof(double);
    rescore_fp64_kernel<<<(n + warps - 1) / warps, 32 * warps, smem, s>>>(rec, lig, n, genes, out);
    return cudaGetLastError();
}

// One local-search launch over every run's individuals (budgets in w.iters;
// the Solis-Wets search writes back the evaluations it spent).
cudaError_t launch_dock_ls(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg,
                           const DockCfg &d, float *genes, int gen, DockScratch &w,
                           cudaStream_t s) {
    const int n = d.n_runs * d.pop;
    if (d.ls_method == 1) {
        SwCfg c;
        c.max_evals = 0;
        c.max_succ = d.sw_max_succ;
        c.max_fail = d.sw_max_fail;
        c.resume = 0;
        c.rho0 = d.sw_rho0;
        c.rho_min = d.sw_rho_min;
        c.angle_scale = d.sw_angle_scale;
        c.seed = d.seed;
        c.call = (uint32_t)gen & 0xFFFFu;
        c.pose_base = 0;
        return launch_sw(rec, lig, cfg, c, genes, n, w.energy, w.iters, nullptr, s, w.iters);
    }
    return launch_eval(rec, lig, cfg, MODE_LS, genes, genes, n, 0, d.rho, d.eps, 0, w.energy,
                       nullptr, nullptr, s, w.iters);
}

cudaError_t launch_dock(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg, const DockCfg &d,
                        float *best_genes, double *best_energy, long long *evals_out,
                        DockScratch &w, cudaStream_t s) {
    const int G = 6 + lig.n_tors, n = d.n_runs * d.pop;
    cudaError_t e;
    init_state_kernel<<<(d.n_runs + 127) / 128, 128, 0, s>>>(d.n_runs, w.best_e, w.evals, w.done);
    init_pop_kernel<<<(n + 127) / 128, 128, 0, s>>>(rec, lig.n_tors, d.seed, d.n_runs, d.pop,
                                                     w.genes[0], w.iters);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    auto local_search = [&](float *genes, int gen) -> cudaError_t {
        return launch_dock_ls(rec, lig, cfg, d, genes, gen, w, s);
    };
    if ((e = local_search(w.genes[0], 0)) != cudaSuccess) return e;
    const int bt = 128;
    best_kernel<<<d.n_runs, bt, 0, s>>>(d.pop, G, w.genes[0], w.energy, w.iters, best_genes,
                                       w.best_e, w.evals, w.done, d.max_evals, 0, d.conv_every,
                                       d.conv_top, d.conv_tol);
    int cur = 0;
    const int gt = d.pop >= 1024 ? 1024 : ((d.pop + 31) / 32) * 32;
    const int gsm = (d.pop + 32) * 4 + 32 * 4;
    for (int gen = 1; gen <= d.max_gens; gen++) {
        ga_kernel<<<d.n_runs, gt, gsm, s>>>(d.pop, G, w.genes[cur], w.energy, d, (uint32_t)gen,
                                           w.genes[cur ^ 1], w.iters, w.done);
        cur ^= 1;
        if ((e = local_search(w.genes[cur], gen)) != cudaSuccess) return e;
        best_kernel<<<d.n_runs, bt, 0, s>>>(d.pop, G, w.genes[cur], w.energy, w.iters,
                                           best_genes, w.best_e, w.evals, w.done, d.max_evals,
                                           gen, d.conv_every, d.conv_top, d.conv_tol);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_rescore_fp64(rec, lig, d.n_runs, best_genes, best_energy, s)) != cudaSuccess)
        return e;
    if (evals_out)
        e = cudaMemcpyAsync(evals_out, w.evals, sizeof(long long) * d.n_runs,
                            cudaMemcpyDeviceToDevice, s);
    return e;
}

}  // namespace adgb
