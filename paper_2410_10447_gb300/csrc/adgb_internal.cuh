// Internal device layouts of the adgb library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adgb.h"  // include/ is on the include path

namespace adgb {

// Mehler-Solmajer distance-dependent dielectric eps(r) = A + B / (1 + k exp(-lambda B r)).
constexpr float MS_A = -8.5525f;
constexpr float MS_EPS0 = 78.4f;
constexpr float MS_B = MS_EPS0 - MS_A;
constexpr float MS_LAMBDA = 0.003627f;
constexpr float MS_K = 7.7839f;

constexpr int MAX_GENES = 6 + ADGB_MAX_TORS;
constexpr int PAIR_CHUNK = 1024;   // pairs per force-buffer chunk (fixed: a ligand's arithmetic
                                   // does not depend on the launch it runs in)
constexpr int TYPE_TAB = ADGB_MAX_TYPES * ADGB_MAX_TYPES;

// Receptor as the kernels see it.  cells[((iz*(ny-1)+iy)*(nx-1)+ix)][m][c]
// holds map m at corner c = cx + 2 cy + 4 cz of cell (ix, iy, iz): one atom
// reads three 32-byte runs (its type map, then e and d adjacent).
struct RecDev {
    int nx, ny, nz, M;      // points per axis, maps (types + e + d)
    float lo[3], hi[3];     // first and last grid point per axis
    float inv_h;            // 1 / spacing
    float h;                // spacing
    const float *cells;
};

// Ligand as the kernels see it.  Atoms are stored in an internal order in
// which every torsion's moving set is one contiguous range [start, end).
struct LigDev {
    int n_atoms, n_tors, n_pairs, n_types;
    const float4 *ref;        // [N] reference x, y, z and charge q
    const float2 *sv;         // [N] (w_ds * S_i, V_i), S_i = solpar + QSOL |q_i|
    const int *type;          // [N] map index
    const int *frag;          // [N] deepest torsion moving the atom, -1 = root fragment
    const int *tparent;       // [T] enclosing torsion, -1 = root
    const int4 *tatoms;       // [T] (a, b, start, end), internal indices
    const float4 *taxis;      // [T] unit bond axis a->b in the reference conformation
    const float4 *tbref;      // [T] reference position of b
    const uint32_t *pairs;    // [Np] i | j << 8 | (ti*16+tj) << 16 | hb << 24
    const float2 *tptab;      // [256] (A, B): E = A r^-12 - B r^-m, m = 10 if hb else 6
    const float4 *pconst;     // [Np] per pair, in pair order: (A, B, w_el 332.06 q_i q_j,
                              // w_ds (S_i V_j + S_j V_i))
    const int *perm;          // [N] internal index -> caller's index
    int n_chunks;             // ceil(Np / PAIR_CHUNK)
    const int *inc_off;       // [n_chunks][N+1]: atom i's pairs in chunk q are
                              // inc[inc_off[q*(N+1)+i] .. inc_off[q*(N+1)+i+1])
    const uint16_t *inc;      // [2 Np] (pair index - q*PAIR_CHUNK) << 1 | (atom is the pair's
                              // second atom), ordered by chunk and atom (within an atom's
                              // list, in the order that spreads reads over the banks)
    int n_rounds, r_lanes;    // matching rounds of the pair list and lanes a round (32 up to
                              // 32 atoms, else the atoms rounded up to 32; 0 rounds: none):
                              // in a round lane a computes at most one pair with atom a first
                              // and receives the forces of at most two pairs with atom a second
    const uint32_t *rword;    // [n_rounds][r_lanes] partner lane | force-source lanes << 8,
                              // << 16 | hb << 24 | source used << 25, << 26
    const float4 *rconst;     // [n_rounds][r_lanes] the pair's constants as in pconst (zeros:
                              // no pair)
    // the caller's per-type parameters, kept for the FP64 rescoring
    const float *t_R, *t_eps, *t_vol, *t_sol;
    const int *t_hb;
    float hb_R, hb_eps;
};

// Solis-Wets local search parameters as the kernels see them.
struct SwCfg {
    int max_evals, max_succ, max_fail, resume;
    float rho0, rho_min, angle_scale;
    uint64_t seed;
    uint32_t call;     // random-stream selector
    int pose_base;     // random-stream index of the first genotype
};

// Lamarckian GA parameters as the kernels see them.
struct DockCfg {
    int n_runs, pop, max_gens, ls_iters;
    long long max_evals;
    float ls_rate, rho, eps, p_cross, p_mut, mut_trans, mut_angle;
    uint64_t seed;
    int conv_every, conv_top;   // early stopping (conv_every = 0: off)
    float conv_tol;
    int ls_method;              // 0 ADADELTA, 1 Solis-Wets
    float sw_rho0, sw_rho_min, sw_angle_scale;
    int sw_max_succ, sw_max_fail;
};

// Device working set of one dock call.
struct DockScratch {
    float *genes[2];      // [runs * pop][G] current and next population
    float *energy;        // [runs * pop]
    int *iters;           // [runs * pop] evaluations of each individual this generation
    float *best_e;        // [runs]
    long long *evals;     // [runs]
    int *done;            // [runs]
};

// Shared-memory layout of one block of the scoring / local-search kernel:
// per-ligand constants once, then per-pose working arrays.  All offsets in
// bytes, 16-byte aligned.
struct SmemLayout {
    int ref, type, frag, tparent, tatoms, taxis, tbref, incoff;
    int spairs, sinc, pairs_in_smem;   // optional copies of the pair list and incidence lists
    int pose0, pose_stride;          // first pose block, bytes per pose
    // offsets inside one pose block
    int p_xyz, p_grad, p_genes, p_ggrad, p_sc, p_red, p_stage, p_force, p_tq, p_seg;
    int chunk;                       // pairs per force-buffer chunk
    int total;

    static __host__ __device__ inline int al16(int x) { return (x + 15) & ~15; }

    // mma_stage: room for the mma.sync reductions' per-warp staging tile.
    __host__ __device__ inline void make(int N, int T, int ppb, int warps_per_pose, int ch,
                                         int np = 0, bool stage_pairs = false,
                                         bool mma_stage = true) {
        const int nch = (np + PAIR_CHUNK - 1) / PAIR_CHUNK;
        int o = 0;
        ref = o;     o = al16(o + 16 * N);
        type = o;    o = al16(o + 4 * N);
        frag = o;    o = al16(o + 4 * N);
        tparent = o; o = al16(o + 4 * (T > 0 ? T : 1));
        tatoms = o;  o = al16(o + 16 * (T > 0 ? T : 1));
        taxis = o;   o = al16(o + 16 * (T > 0 ? T : 1));
        tbref = o;   o = al16(o + 16 * (T > 0 ? T : 1));
        incoff = o;  if (stage_pairs) o = al16(o + 4 * nch * (N + 1));
        pairs_in_smem = stage_pairs ? 1 : 0;
        spairs = o;  if (stage_pairs) o = al16(o + 4 * np);
        sinc = o;    if (stage_pairs) o = al16(o + 4 * np);
        pose0 = o;
        int q = 0;
        p_xyz = q;   q = al16(q + 16 * N);
        p_grad = q;  q = al16(q + 16 * N);
        p_genes = q; q = al16(q + 4 * MAX_GENES);
        p_ggrad = q; q = al16(q + 4 * MAX_GENES);
        p_sc = q;    q = al16(q + 8 * (ADGB_MAX_TORS + 4));
        p_red = q;   q = al16(q + 4 * 8 * warps_per_pose);
        p_stage = q; q = al16(q + (mma_stage ? 4 * 32 * 12 * warps_per_pose : 0));
        // pairs of a force-buffer chunk; at least a round's slots for the
        // block form of the matching rounds (one float4 a lane)
        chunk = ch > 0 ? ch : 1;
        const int lanes = N <= 32 ? 32 : (N + 31) / 32 * 32;
        if (chunk < lanes) chunk = lanes;
        p_force = q; q = al16(q + 16 * chunk);
        p_tq = q;    // (unused: no torsion prefix scans)
        p_seg = q;
        pose_stride = q;
        total = pose0 + ppb * pose_stride;
    }

    // Layout of one ligand for the multi-ligand kernel: the pair list and
    // incidence lists are staged when they take at most 24 KB, and the
    // pair-force buffer holds min(pairs, 1024) pairs.  It depends on the
    // ligand alone, so a genotype's arithmetic is the same whatever other
    // ligands share the launch.  The host sizes a launch's shared memory to
    // the largest such layout; the device recomputes it per work item.
    static __host__ __device__ inline SmemLayout choose(int N, int T, int np, int ppb,
                                                        int warps_per_pose, bool mma_stage) {
        SmemLayout l;
        const bool stage = 8 * np <= 24 * 1024;
        const int ch = np < PAIR_CHUNK ? (np > 1 ? np : 1) : PAIR_CHUNK;
        l.make(N, T, ppb, warps_per_pose, ch, np, stage, mma_stage);
        return l;
    }
};

// Shared-memory layout of the two-genotypes-a-warp kernel (ligands of at
// most 32 atoms): the ligand's constants once, then per warp the two
// genotypes' coordinates (atom i: [2i] genotype A, [2i+1] genotype B), genes
// (float2 per gene) and sin / (1 - cos) of every angle (float4: A's pair,
// B's pair) and a staging tile.  All offsets in bytes from the layout's base,
// 16-byte aligned.
struct PairSmem {
    int ref, type, frag, tparent, tatoms, taxis, tbref;
    int warp0, warp_stride;
    int w_xyz, w_genes, w_sc, w_stage;
    int total;

    static __host__ __device__ inline int al16(int x) { return (x + 15) & ~15; }

    // stage: room for the warp's 32 x 12-float staging tile (the mma.sync
    // reductions and the shuffle form's torsion sums; not the tcgen05 form)
    __host__ __device__ inline void make(int N, int T, int warps, bool stage) {
        const int Tn = T > 0 ? T : 1;
        int o = 0;
        ref = o;     o = al16(o + 16 * N);
        type = o;    o = al16(o + 4 * N);
        frag = o;    o = al16(o + 4 * N);
        tparent = o; o = al16(o + 4 * Tn);
        tatoms = o;  o = al16(o + 16 * Tn);
        taxis = o;   o = al16(o + 16 * Tn);
        tbref = o;   o = al16(o + 16 * Tn);
        warp0 = o;
        int q = 0;
        w_xyz = q;   q = al16(q + 32 * 32);
        w_genes = q; q = al16(q + 8 * MAX_GENES);
        w_sc = q;    q = al16(q + 16 * (ADGB_MAX_TORS + 4));
        w_stage = q; q = al16(q + (stage ? 4 * 32 * 12 : 0));
        warp_stride = q;
        total = warp0 + warps * warp_stride;
    }
};

// Whether a ligand runs two genotypes a warp: at most 32 atoms with the
// warp form of the matching rounds (or no pairs), at most 32 genes (one gene
// slot a lane), one warp a genotype.
__host__ __device__ inline bool pair_eligible(int n_atoms, int n_tors, int n_pairs, int n_rounds,
                                              int r_lanes, int tpp) {
    return tpp == 32 && n_atoms <= 32 && 6 + n_tors <= 32 &&
           (n_pairs == 0 || (n_rounds > 0 && r_lanes == 32));
}

// Threads a genotype by ligand size (one warp up to 32 atoms, two up to 56,
// else 128; measured on 3000 genotypes, see the local-search launch-shape
// sweep): the single-ligand calls and the serving loop's size classes alike.
__host__ __device__ inline int threads_for_atoms(int n_atoms) {
    return n_atoms <= 32 ? 32 : (n_atoms <= 56 ? 64 : 128);
}

// Reduction variants that stage each warp's values in shared memory for
// mma.sync.
__host__ __device__ inline bool uses_mma_stage(int variant) {
    return variant == ADGB_REDUCE_MMA_TF32X2 || variant == ADGB_REDUCE_MMA_BF16X3;
}

// Work item of the multi-ligand local-search kernel: up to poses-per-block
// genotypes of one ligand against one receptor.
struct WorkItem {
    int lig, rec;          // indices into the launch's ligand / receptor tables
    int count;             // genotypes in this item
    int gstride;           // floats between consecutive genotypes
    float *genes;          // first genotype (in: start, out: best)
    float *energy;         // first best energy
    const int *iters;      // per-genotype evaluation counts, or null
    int iters_all;         // evaluation count when iters is null
    int cost;              // ordering key (host side)
    float rho, eps;        // ADADELTA parameters of the item's search
};

// Launch configuration of the fused kernel.
struct EvalCfg {
    int tpp;        // threads per pose (32, 64, 128)
    int ppb;        // poses per block
    int variant;    // ADGB_REDUCE_*
    int chunk;      // pairs per force-buffer chunk
    int stage_pairs;  // copy the pair list and incidence lists to shared memory
    int paired;     // two genotypes a warp where the ligand is eligible (pair_eligible)
};

// Carveout hint for the two-genotypes-a-warp kernels of the shuffle and
// mma.sync forms: the smallest shared-memory share of the SM's unified L1 /
// shared memory that still holds as many blocks as the registers allow; the
// rest stays L1 for the grid gathers and the round tables (measured on the
// 32-atom ligand's local search: 505 -> 516M evaluations/s, L1 hit rate 69
// -> 74%; on the one-genotype and Solis-Wets kernels 1-2% slower, so they
// keep the default).  The tcgen05 form keeps the default too (no gain
// measured: its P and B operands take 30 KB a block).
template <typename K>
inline cudaError_t prefer_l1(K k, int smem, int threads) {
    int dev = 0, per_sm = 0, reserved = 0, regs_sm = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
    if (e == cudaSuccess && per_sm > 0) {
        const int regs_block = ((fa.numRegs * 32 + 255) / 256) * 256 * (threads / 32);
        const int blocks = regs_block > 0 ? max(1, regs_sm / regs_block) : 1;
        const long need = (long)blocks * (smem + (long)fa.sharedSizeBytes + reserved);
        const int pct = (int)max(1L, min(100L, (need * 100 + per_sm - 1) / per_sm));
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    }
    // a hint: a refusal leaves the default carveout and is not the launch's error
    if (e != cudaSuccess) (void)cudaGetLastError();
    return cudaSuccess;
}

// Host-side launchers (eval.cu, reduce_bench.cu).
cudaError_t launch_eval(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg,
                        int mode, const float *genes_in, float *genes_out, int n,
                        int iters, float rho, float eps, int resume, float *energy,
                        float *grad, float *state, cudaStream_t s,
                        const int *iters_per_pose = nullptr);
// Two genotypes a warp (pair_eligible ligands only; EvalCfg::paired).  A
// tensor-core completion wait that gives up is counted (tc_gave_up_async).
cudaError_t launch_eval_pair(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg, int mode,
                             const float *genes_in, float *genes_out, int n, int iters, float rho,
                             float eps, int resume, float *energy, float *grad, float *state,
                             cudaStream_t s, const int *iters_per_pose);
int pair_smem_bytes(int layout_bytes, int warps, int variant, int device);
// Measurement-only paired local search without the steps in `skip`
// (ls_ablation_dev); cudaErrorInvalidValue for masks or variants not built.
cudaError_t launch_pair_ablation(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg,
                                 float *genes, int n, int iters, float *energy, cudaStream_t s,
                                 int skip);
int pair_layout_bytes(int n_atoms, int n_tors, int ppb, int variant);
// Queues copies of the tensor-core give-up counts of the local-search kernels
// on the current device (dst[0]: one genotype a warp and Solis-Wets, dst[1]:
// two genotypes a warp; monotonic) into host memory dst.
cudaError_t tc_gave_up_async(unsigned int dst[2], cudaStream_t s);
cudaError_t pair_tc_gave_up_async(unsigned int *dst, cudaStream_t s);
int pair_items_grid(const EvalCfg &cfg, int budget, int device);
cudaError_t launch_eval_pair_items(const WorkItem *items, int n_items, const LigDev *ligs,
                                   const RecDev *recs, int *counter, const EvalCfg &cfg, int budget,
                                   int grid, cudaStream_t s);
// Shared-memory bytes of one ligand's layout in a multi-ligand launch of
// shape cfg (the launch's budget is the largest over its ligands).
int items_layout_bytes(const EvalCfg &cfg, int n_atoms, int n_tors, int n_pairs);
// Solis-Wets searches; budget [n] (evaluations each genotype may spend) or
// null for c.max_evals; evals [n] receives the evaluations spent (it may be
// the budget array itself).
cudaError_t launch_sw(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg, const SwCfg &c,
                      float *genes, int n, float *energy, int *evals, float *state, cudaStream_t s,
                      const int *budget = nullptr);
cudaError_t launch_dock(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg, const DockCfg &d,
                        float *best_genes, double *best_energy, long long *evals_out,
                        DockScratch &w, cudaStream_t s);
cudaError_t launch_rescore_fp64(const RecDev &rec, const LigDev &lig, int n, const float *genes,
                                double *out, cudaStream_t s);
cudaError_t launch_init_population(const RecDev &rec, int n_tors, uint64_t seed, int n_runs, int pop,
                                   float *genes, int *iters, cudaStream_t s);
cudaError_t launch_ga_generation(const DockCfg &d, int G, int gen, const float *genes,
                                 const float *energy, float *genes_out, int *iters, cudaStream_t s);
cudaError_t launch_job_start(const RecDev &rec, int n_tors, const DockCfg &d, DockScratch &w,
                             cudaStream_t s);
cudaError_t launch_job_ga(const DockCfg &d, int G, int gen, DockScratch &w, int cur, cudaStream_t s);
// The local searches of one LGA generation (ADADELTA or Solis-Wets per
// d.ls_method, per-individual budgets in w.iters; Solis-Wets writes back the
// evaluations it spent), as dock() runs them.
cudaError_t launch_dock_ls(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg,
                           const DockCfg &d, float *genes, int gen, DockScratch &w,
                           cudaStream_t s);
cudaError_t launch_job_best(const DockCfg &d, int G, int gen, DockScratch &w, int cur,
                            float *best_genes, cudaStream_t s);
cudaError_t launch_ga_converged(int n_runs, int pop, int top, float tol, const float *energy,
                                int *converged, cudaStream_t s);
cudaError_t launch_philox(const uint32_t *in, int n, uint32_t *out, cudaStream_t s);
cudaError_t launch_alu_bench(int kind, int n_blocks, int threads, int reps, float *out,
                             cudaStream_t s);
cudaError_t launch_l2_bench(int kind, const float *buf, long long n4, int cell4, int n_blocks,
                            int threads, int reps, float *out, cudaStream_t s);
cudaError_t launch_coords(const LigDev &lig, const float *genes, int n, float *xyz,
                          cudaStream_t s);
// Persistent multi-ligand local search over a device table of work items
// (counter zeroed by the launch itself, so the launch can be replayed).
cudaError_t launch_eval_items(const WorkItem *items, int n_items, const LigDev *ligs,
                              const RecDev *recs, int *counter, const EvalCfg &cfg, int budget,
                              int grid, cudaStream_t s);
int items_grid(const EvalCfg &cfg, int budget, int device);
cudaError_t launch_pack_grid(const float *maps, int nx, int ny, int nz, int M,
                             float *cells, cudaStream_t s);
cudaError_t launch_reduce4_bench(int variant, const float *in, int threads, int n_blocks,
                                 int reps, float *out, cudaStream_t s);

enum { MODE_SCORE = 0, MODE_LS = 1 };

}  // namespace adgb

#include <string>
#include <vector>

namespace adgb {

// Host image of a validated ligand's device blob; `rel` holds the blob
// offsets in its pointer fields until bind_ligand relocates them.
struct LigandBlob {
    std::vector<unsigned char> bytes;
    LigDev rel;
    int max_type = 0;
};
int make_ligand_blob(std::string *err, const adgb_ligand_desc *d, int pair_rounds, LigandBlob &out);
LigDev bind_ligand(const LigandBlob &b, const unsigned char *mem);
int dock_cfg_from_params(const adgb_dock_params *p, int default_variant, DockCfg &d, int &variant,
                         std::string *err);
int ctx_device(const adgb_ctx *c);
int ctx_default_variant(const adgb_ctx *c);
int ctx_receptor(adgb_ctx *c, int rid, RecDev *out, int *n_type_maps);
int ctx_pair_rounds(const adgb_ctx *c);
int ctx_genotypes_per_warp(const adgb_ctx *c);
void ctx_launch_opts(const adgb_ctx *c, int *tpp, int *ppb);
// The launch shape of a ligand (threads a genotype, genotypes a block, two
// genotypes a warp or one); tpp_opt / ppb_opt 0 = by ligand size.
EvalCfg launch_cfg(const LigDev &L, int tpp_opt, int ppb_opt, int variant, int genotypes_per_warp);

}  // namespace adgb
