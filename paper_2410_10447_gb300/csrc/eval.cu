// Fused scoring / ADADELTA local-search kernel (Sec. 2.1, Sec. 3): one pose
// group of TPP threads per genotype, several pose groups per block sharing
// the ligand's constants in shared memory.  One launch runs every
// genotype's whole local search; between evaluations nothing leaves the SM
// except the grid-map gathers.
//
// Per evaluation (group barrier = __syncwarp for TPP = 32, bar.sync with a
// per-group id otherwise):
//   1. gene owners publish the genes and sin / (1 - cos) of every angle;
//   2. each thread builds its atoms' coordinates (torsions deepest-first
//      about reference axes, then rotation, then translation) and their
//      trilinear grid energy and gradient;
//   3. threads stride over the pair list: four pair terms, each pair's force
//      written to its own slot of a per-pose force buffer, then every atom's
//      owner thread sums the forces of its pairs (no atomics; chunked when
//      the pair list exceeds the buffer);
//   4. per-thread partials of (E, sum g, torque) and the torsion gradients
//      (each torsion's moving set is one contiguous atom range);
//   5. one 8-wide reduce-and-broadcast (warp shuffles or tensor cores);
//   6. gene gradient, best tracking and the ADADELTA update by the threads
//      that own the genes.
#include <math.h>

#include <algorithm>

#include "adgb_internal.cuh"
#include "philox.cuh"
#include "reduce.cuh"

namespace adgb {

struct EvalArgs {
    RecDev rec;
    LigDev lig;
    SmemLayout L;
    const float *genes_in;
    float *genes_out;
    float *energy;
    float *grad;
    float *state;
    const int *iters_pp;  // per-genotype evaluation counts, or null (all `iters`)
    int n, iters, resume, mode;
    float rho, eps;
};

constexpr float INV_SIG2 = 1.0f / (ADGB_DS_SIGMA * ADGB_DS_SIGMA);
constexpr float HALF_INV_SIG2 = 0.5f / (ADGB_DS_SIGMA * ADGB_DS_SIGMA);
constexpr float RMIN2 = ADGB_R_MIN * ADGB_R_MIN;
constexpr float PI_F = 3.14159265358979f;
constexpr int SC_ROT = ADGB_MAX_TORS;  // sc[] slots after the torsions: phi, theta, alpha

template <int TPP>
__device__ __forceinline__ void group_sync(int group) {
    if constexpr (TPP == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(group + 1), "r"(TPP) : "memory");
    }
}

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// p += s (k x v) + omc (k x (k x v)), v = p - b: rotation by the angle with
// sin = s, 1 - cos = omc about the axis k through b.  Exact at s = omc = 0.
__device__ __forceinline__ void rotate_about(float3 &p, float4 k4, float4 b4, float2 c) {
    const float3 k = make_float3(k4.x, k4.y, k4.z);
    const float3 v = make_float3(p.x - b4.x, p.y - b4.y, p.z - b4.z);
    const float3 kv = cross3(k, v);
    const float3 kkv = cross3(k, kv);
    p.x += c.x * kv.x + c.y * kkv.x;
    p.y += c.x * kv.y + c.y * kkv.y;
    p.z += c.x * kv.z + c.y * kkv.z;
}

// Grid cell of a point: clamped onto the grid, cell origin index, fractional
// position, inside flags, and the out-of-grid penalty and its gradient.
struct CellPos {
    size_t cell;
    float f[3], gout[3], pen;
    bool ins[3];
};

__device__ __forceinline__ CellPos locate(const RecDev &R, float3 x) {
    const float xs[3] = {x.x, x.y, x.z};
    const int n[3] = {R.nx, R.ny, R.nz};
    CellPos c;
    c.pen = 0.f;
    int i0[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float xc = fminf(fmaxf(xs[d], R.lo[d]), R.hi[d]);
        c.ins[d] = xs[d] >= R.lo[d] && xs[d] <= R.hi[d];
        const float dd = xs[d] - xc;
        c.pen += dd * dd;
        c.gout[d] = 2.f * ADGB_W_OUT * dd;
        const float u = (xc - R.lo[d]) * R.inv_h;
        int k = (int)u;  // u >= 0
        k = k > n[d] - 2 ? n[d] - 2 : k;
        i0[d] = k;
        c.f[d] = u - (float)k;
    }
    c.cell = ((size_t)i0[2] * (R.ny - 1) + i0[1]) * (R.nx - 1) + i0[0];
    return c;
}

// Intermolecular term of one atom from its cell's corner values (type map
// t0/t1, e map e0/e1, d map d0/d1; corner c = cx + 2 cy + 4 cz): the type's
// map plus q times e plus |q| times d, trilinearly interpolated at the point
// clamped onto the grid; a point outside pays W_OUT times its squared
// distance to the grid.
__device__ __forceinline__ float inter_from_corners(const RecDev &R, const CellPos &c, float q,
                                                    float4 t0, float4 t1, float4 e0, float4 e1,
                                                    float4 d0, float4 d1, float3 &g) {
    const float aq = fabsf(q);
    const float w0 = t0.x + q * e0.x + aq * d0.x, w1 = t0.y + q * e0.y + aq * d0.y;
    const float w2 = t0.z + q * e0.z + aq * d0.z, w3 = t0.w + q * e0.w + aq * d0.w;
    const float w4 = t1.x + q * e1.x + aq * d1.x, w5 = t1.y + q * e1.y + aq * d1.y;
    const float w6 = t1.z + q * e1.z + aq * d1.z, w7 = t1.w + q * e1.w + aq * d1.w;
    const float fx = c.f[0], fy = c.f[1], fz = c.f[2];
    const float x00 = w1 - w0, x10 = w3 - w2, x01 = w5 - w4, x11 = w7 - w6;
    const float c00 = w0 + fx * x00, c10 = w2 + fx * x10;
    const float c01 = w4 + fx * x01, c11 = w6 + fx * x11;
    const float y0 = c10 - c00, y1 = c11 - c01;
    const float c0 = c00 + fy * y0, c1 = c01 + fy * y1;
    const float val = c0 + fz * (c1 - c0);
    const float dx0 = x00 + fy * (x10 - x00), dx1 = x01 + fy * (x11 - x01);
    const float dfx = dx0 + fz * (dx1 - dx0);
    const float dfy = y0 + fz * (y1 - y0);
    const float dfz = c1 - c0;
    g.x = (c.ins[0] ? dfx * R.inv_h : 0.f) + c.gout[0];
    g.y = (c.ins[1] ? dfy * R.inv_h : 0.f) + c.gout[1];
    g.z = (c.ins[2] ? dfz * R.inv_h : 0.f) + c.gout[2];
    return val + ADGB_W_OUT * c.pen;
}

__device__ __forceinline__ const float4 *cell_ptr(const RecDev &R, size_t cell) {
    return reinterpret_cast<const float4 *>(R.cells + cell * (size_t)R.M * 8);
}

// Grid term read straight from global memory (L2).
__device__ __forceinline__ float inter_atom(const RecDev &R, int t, float q, float3 x, float3 &g) {
    const CellPos c = locate(R, x);
    const float4 *cp = cell_ptr(R, c.cell);
    return inter_from_corners(R, c, q, __ldg(cp + 2 * t), __ldg(cp + 2 * t + 1),
                              __ldg(cp + 2 * (R.M - 2)), __ldg(cp + 2 * (R.M - 2) + 1),
                              __ldg(cp + 2 * (R.M - 1)), __ldg(cp + 2 * (R.M - 1) + 1), g);
}

// One intramolecular pair: 12-6 (12-10 for donor-acceptor pairs) with
// A r^-12 - B r^-m, Coulomb with the Mehler-Solmajer dielectric, and
// desolvation.  pc = (A, B, w_el 332.06 q_i q_j, w_ds (S_i V_j + S_j V_i)).
// Returns the energy; f = dE/dx_i (atom j gets -f).
__device__ __forceinline__ float pair_term(float4 xi, float4 xj, float4 pc, bool hb, float3 &f) {
    const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const bool live = r2 >= RMIN2;
    const float r2c = fmaxf(r2, RMIN2);
    const float rinv = rsqrtf(r2c);
    const float rc = r2c * rinv;
    const float r2i = rinv * rinv;
    const float r6i = r2i * r2i * r2i;
    const float r12i = r6i * r6i;
    const float rmi = hb ? r6i * r2i * r2i : r6i;
    const float m = hb ? 10.f : 6.f;
    const float evdw = pc.x * r12i - pc.y * rmi;
    const float dvdw = (-12.f * pc.x * r12i + m * pc.y * rmi) * rinv;
    // eps(r) = num / den with den = 1 + k e^{-lambda B r}, num = A den + B;
    // 1/eps = den^2 r and eps'/eps = B k lambda B e^{..} r with r = 1/(den num):
    // one reciprocal for the whole dielectric.
    const float C = pc.z;
    const float ex = __expf(-MS_LAMBDA * MS_B * rc);
    const float den = 1.f + MS_K * ex;
    const float num = MS_A * den + MS_B;
    const float rr = __fdividef(1.f, den * num);
    const float eel = C * rinv * (den * den * rr);
    const float del = -eel * (rinv + (MS_B * MS_K * MS_LAMBDA * MS_B) * ex * rr);
    const float eds = pc.w * __expf(-r2 * HALF_INV_SIG2);
    const float fr = live ? (dvdw + del) * rinv : 0.f;
    const float fd = -eds * INV_SIG2;
    f = make_float3((fr + fd) * dx, (fr + fd) * dy, (fr + fd) * dz);
    return evdw + eel + eds;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float3 xyz3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }

// Two pair terms (a, b), the same formulas as pair_term with the adds,
// multiplies and fused multiply-adds of both pairs in packed FP32x2
// instructions (one instruction, two IEEE round-to-nearest results);
// reciprocal square roots, exponentials, the reciprocal, compares and
// selects per pair.  Returns the two energies' sum; fa, fb = dE/dx_i of each
// pair (its first atom; the second gets the negative).
__device__ __forceinline__ float pair_term2(float3 ia, float3 ib, float3 xa, float3 xb, float4 pa,
                                            float4 pb, bool hba, bool hbb, float3 &fa, float3 &fb) {
    const float2 neg = f2s(-1.f);
    const float2 dx = __ffma2_rn(f2(xa.x, xb.x), neg, f2(ia.x, ib.x));   // x_i - x_j, exact
    const float2 dy = __ffma2_rn(f2(xa.y, xb.y), neg, f2(ia.y, ib.y));
    const float2 dz = __ffma2_rn(f2(xa.z, xb.z), neg, f2(ia.z, ib.z));
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    const bool la = r2.x >= RMIN2, lb = r2.y >= RMIN2;
    const float2 r2c = f2(fmaxf(r2.x, RMIN2), fmaxf(r2.y, RMIN2));
    const float2 rinv = f2(rsqrtf(r2c.x), rsqrtf(r2c.y));
    const float2 rc = __fmul2_rn(r2c, rinv);
    const float2 r2i = __fmul2_rn(rinv, rinv);
    const float2 r4i = __fmul2_rn(r2i, r2i);
    const float2 r6i = __fmul2_rn(r4i, r2i);
    const float2 r12i = __fmul2_rn(r6i, r6i);
    const float2 r10i = __fmul2_rn(r6i, r4i);
    const float2 rmi = f2(hba ? r10i.x : r6i.x, hbb ? r10i.y : r6i.y);
    const float2 m = f2(hba ? 10.f : 6.f, hbb ? 10.f : 6.f);
    const float2 t12 = __fmul2_rn(f2(pa.x, pb.x), r12i), tm = __fmul2_rn(f2(pa.y, pb.y), rmi);
    const float2 evdw = __ffma2_rn(tm, neg, t12);
    const float2 dvdw = __fmul2_rn(__ffma2_rn(m, tm, __fmul2_rn(f2s(-12.f), t12)), rinv);
    const float2 xa_ = __fmul2_rn(f2s(-MS_LAMBDA * MS_B), rc);
    const float2 ex = f2(__expf(xa_.x), __expf(xa_.y));
    const float2 den = __ffma2_rn(f2s(MS_K), ex, f2s(1.f));
    const float2 num = __ffma2_rn(f2s(MS_A), den, f2s(MS_B));
    const float2 dn = __fmul2_rn(den, num);
    const float2 rr = f2(__fdividef(1.f, dn.x), __fdividef(1.f, dn.y));
    const float2 eel =
        __fmul2_rn(__fmul2_rn(f2(pa.z, pb.z), rinv), __fmul2_rn(__fmul2_rn(den, den), rr));
    const float2 del = __fmul2_rn(__fmul2_rn(eel, neg),
                                  __ffma2_rn(f2s(MS_B * MS_K * MS_LAMBDA * MS_B),
                                             __fmul2_rn(ex, rr), rinv));
    const float2 xd = __fmul2_rn(r2, f2s(-HALF_INV_SIG2));
    const float2 eds = __fmul2_rn(f2(pa.w, pb.w), f2(__expf(xd.x), __expf(xd.y)));
    const float2 frr = __fmul2_rn(__fadd2_rn(dvdw, del), rinv);
    const float2 ft = __ffma2_rn(eds, f2s(-INV_SIG2), f2(la ? frr.x : 0.f, lb ? frr.y : 0.f));
    const float2 fx = __fmul2_rn(ft, dx), fy = __fmul2_rn(ft, dy), fz = __fmul2_rn(ft, dz);
    fa = make_float3(fx.x, fy.x, fz.x);
    fb = make_float3(fx.y, fy.y, fz.y);
    const float2 e = __fadd2_rn(__fadd2_rn(evdw, eel), eds);
    return e.x + e.y;
}

// ISSUED: the tcgen05 variant's MMAs were already issued (tc05_issue) and
// only the wait and the TMEM load remain.
template <int TPP, int VAR, bool ISSUED = false>
__device__ __forceinline__ void group_sum8(float v[8], float *red, float *stage, int group,
                                           int gt, Tc05Warp &tw) {
    if constexpr (VAR == ADGB_REDUCE_TCGEN05) {
        if constexpr (ISSUED)
            tc05_finish(v, tw);
        else
            warp_sum8_tc05(v, tw);
    } else {
        warp_sum8<VAR>(v, stage);
    }
    if constexpr (TPP > 32) {
        const int w = gt >> 5;
        if ((gt & 31) == 0) {
#pragma unroll
            for (int c = 0; c < 8; c++) red[w * 8 + c] = v[c];
        }
        group_sync<TPP>(group);
#pragma unroll
        for (int c = 0; c < 8; c++) {
            float s = red[c];
#pragma unroll
            for (int k = 1; k < TPP / 32; k++) s += red[k * 8 + c];
            v[c] = s;
        }
    }
}

// Blocks of at most 128 threads; ADGB_MIN_BLOCKS resident blocks per SM
// bound the registers (5 -> 96 registers a thread, no spills; 3000
// one-warp genotypes then run in a single wave of 20 warps an SM).
#ifndef ADGB_MIN_BLOCKS
#define ADGB_MIN_BLOCKS 5
#endif
// The persistent multi-ligand kernel keeps more live state (the work loop,
// the current ligand's layout): at 96 registers it spilled 24-124 bytes;
// 4 blocks an SM (128 registers, no spills) measured 1.8% faster on the
// uneven 512-ligand batch (46.1 -> 46.9M evaluations/s, same GPU).
#ifndef ADGB_ITEMS_MIN_BLOCKS
#define ADGB_ITEMS_MIN_BLOCKS 4
#endif

// ------------------------------------------------- tcgen05 block set-up
// The tcgen05 reduction's shared-memory region sits at the front of the
// (1024-byte aligned) dynamic shared memory, before the ligand layout: one
// 2 KB B operand per warp at [0, 8192), the all-ones A operand at
// [8192, 10496), one mbarrier per warp at [10496, 10528) and the TMEM base
// address at [10528, 10532).  A block holds at most 4 warps (128 threads).
// The A operand (128 x 8 TF32) is read with 128-byte strides both ways, so
// its core matrices overlap inside 2304 bytes of ones.
constexpr int TC_B = 0, TC_A = 8192, TC_MBAR = 10496, TC_SLOT = 10528;
constexpr int TC_REGION = 10560;

template <int VAR>
__host__ __device__ constexpr int tc_front() { return VAR == ADGB_REDUCE_TCGEN05 ? TC_REGION : 0; }

// The multi-ligand kernel keeps its current ligand's layout and work-item
// index in a 128-byte header before the ligand layout (after the tcgen05
// region for that variant): the layout read from shared memory instead of
// held in registers across the work loop.
constexpr int ITEMS_HDR = 128;
static_assert(sizeof(SmemLayout) <= ITEMS_HDR - 16, "items header too small");
template <int VAR>
__host__ __device__ constexpr int items_front() {
    return (VAR == ADGB_REDUCE_TCGEN05 ? TC_REGION : 0) + ITEMS_HDR;
}

__host__ __device__ constexpr int tc_ncols(int warps) {   // 16 D columns a warp
    return 16 * warps <= 32 ? 32 : (16 * warps <= 64 ? 64 : 128);
}

// Allocates the block's TMEM, writes the ones operand and fills `tw` (all
// threads; contains block barriers).  R is the front of the dynamic shared
// memory.
template <int VAR>
__device__ __forceinline__ void tc_begin(unsigned char *R, Tc05Warp &tw) {
    if constexpr (VAR == ADGB_REDUCE_TCGEN05) {
        uint64_t *mb = reinterpret_cast<uint64_t *>(R + TC_MBAR);
        uint32_t *slot = reinterpret_cast<uint32_t *>(R + TC_SLOT);
        const int w = threadIdx.x >> 5, W = blockDim.x >> 5;
        const uint32_t ncols = tc_ncols(W);
        const uint32_t rs = tc05::smem_u32(R);
        uint32_t *ones = reinterpret_cast<uint32_t *>(R + TC_A);
        for (int i = threadIdx.x; i < (TC_MBAR - TC_A) / 4; i += blockDim.x) ones[i] = 0x3F800000u;
        tc05::fence_proxy_async_smem();
        if (w == 0) {
            tc05::alloc(slot, ncols);
            tc05::relinquish();
        }
        if ((int)threadIdx.x < W) tc05::mbar_init(mb + threadIdx.x, 1);
        tc05::fence_before();
        __syncthreads();
        tc05::fence_after();
        const uint32_t taddr = *slot;
        tw.a_desc = tc05::desc_plain(rs + TC_A, 128, 128);
        tw.b_s = rs + TC_B + 2048u * w;
        tw.b = R + TC_B + 2048 * w;
        tw.mbar = mb + w;
        tw.d_col = taddr + 16u * w;
        tw.d_lane = tc05::lane_addr(taddr, w & 3, 16 * w);
        tw.taddr = taddr;
        tw.ncols = ncols;
        tw.phase = 0;
        tw.ok = (rs & 1023u) == 0;   // the swizzled B atoms need 1024-byte alignment
    }
}

// Releases the block's TMEM once every warp's MMAs have completed (all
// threads; a warp whose wait gave up first waits, bounded, once more).
template <int VAR>
__device__ __forceinline__ void tc_end(Tc05Warp &tw) {
    if constexpr (VAR == ADGB_REDUCE_TCGEN05) {
        if (!tw.ok && tw.phase > 0)
            (void)tc05::mbar_wait(tw.mbar, (tw.phase - 1) & 1, TC05_WAIT_LIMIT);
        tc05::fence_before();
        __syncthreads();
        tc05::fence_after();
        if ((threadIdx.x >> 5) == 0) tc05::dealloc(tw.taddr, tw.ncols);
    }
}

// Per-genotype inputs and outputs of search_pose (pointers at that genotype).
struct PoseIO {
    const float *genes_in;  // [G] start genotype (unused with resume)
    float *genes_out;       // [G] best genotype (local search)
    float *energy;          // [1] energy (score) or best energy (local search)
    float *grad;            // [G] gene gradient (score) or null
    float *state;           // [3][G] (Omega, E[g^2], E[d^2]) or null
    int iters, mode, resume;
    float rho, eps;
};

// Where the pair list and incidence lists are read from (shared or global).
struct StagedLig {
    const uint32_t *prs;
    const uint16_t *incl;
    const int *incoff;   // [n_chunks][N+1]
};

// Copies one ligand's constants into shared memory (all threads of the
// block; the caller synchronises before the first use).
__device__ __forceinline__ StagedLig stage_ligand(unsigned char *sm, const SmemLayout &L,
                                                  const LigDev &lig) {
    const int N = lig.n_atoms, T = lig.n_tors, NP = lig.n_pairs;
    float4 *s_ref = reinterpret_cast<float4 *>(sm + L.ref);
    int *s_type = reinterpret_cast<int *>(sm + L.type);
    int *s_frag = reinterpret_cast<int *>(sm + L.frag);
    int *s_tpar = reinterpret_cast<int *>(sm + L.tparent);
    int4 *s_tat = reinterpret_cast<int4 *>(sm + L.tatoms);
    float4 *s_tax = reinterpret_cast<float4 *>(sm + L.taxis);
    float4 *s_tb = reinterpret_cast<float4 *>(sm + L.tbref);
    // pair records, incidence lists and their offsets: shared memory when they fit
    const uint32_t *prs = lig.pairs;
    const uint16_t *incl = lig.inc;
    const int *incoff = lig.inc_off;
    if (L.pairs_in_smem) {
        uint32_t *sp = reinterpret_cast<uint32_t *>(sm + L.spairs);
        uint16_t *si = reinterpret_cast<uint16_t *>(sm + L.sinc);
        int *so = reinterpret_cast<int *>(sm + L.incoff);
        for (int p = threadIdx.x; p < NP; p += blockDim.x) sp[p] = lig.pairs[p];
        for (int p = threadIdx.x; p < 2 * NP; p += blockDim.x) si[p] = lig.inc[p];
        for (int p = threadIdx.x; p < lig.n_chunks * (N + 1); p += blockDim.x) so[p] = lig.inc_off[p];
        prs = sp;
        incl = si;
        incoff = so;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        s_ref[i] = lig.ref[i];
        s_type[i] = lig.type[i];
        s_frag[i] = lig.frag[i];
    }
    for (int k = threadIdx.x; k < T; k += blockDim.x) {
        s_tpar[k] = lig.tparent[k];
        s_tat[k] = lig.tatoms[k];
        s_tax[k] = lig.taxis[k];
        s_tb[k] = lig.tbref[k];
    }
    return {prs, incl, incoff};
}

// Whole evaluation loop of one genotype by one pose group (TPP threads).
// NGS: genes each lane holds (ceil(G / TPP) at most); the default covers
// the largest genotype.
template <int TPP, int VAR, int NGS = (MAX_GENES + TPP - 1) / TPP>
__device__ __forceinline__ void search_pose(unsigned char *sm, const SmemLayout &L,
                                            const LigDev &lig, const RecDev &rec,
                                            const StagedLig &sl, const int group, const int gt,
                                            const PoseIO &io, Tc05Warp &tw) {
    const int N = lig.n_atoms, T = lig.n_tors, G = 6 + T, NP = lig.n_pairs;
    float4 *s_ref = reinterpret_cast<float4 *>(sm + L.ref);
    int *s_type = reinterpret_cast<int *>(sm + L.type);
    int *s_frag = reinterpret_cast<int *>(sm + L.frag);
    int *s_tpar = reinterpret_cast<int *>(sm + L.tparent);
    int4 *s_tat = reinterpret_cast<int4 *>(sm + L.tatoms);
    float4 *s_tax = reinterpret_cast<float4 *>(sm + L.taxis);
    float4 *s_tb = reinterpret_cast<float4 *>(sm + L.tbref);
    const float4 *pconst = lig.pconst;
    const uint32_t *prs = sl.prs;
    const uint16_t *incl = sl.incl;
    unsigned char *P = sm + L.pose0 + group * L.pose_stride;
    float4 *xyz = reinterpret_cast<float4 *>(P + L.p_xyz);
    float4 *grd = reinterpret_cast<float4 *>(P + L.p_grad);
    float *genes_s = reinterpret_cast<float *>(P + L.p_genes);
    float *ggrad = reinterpret_cast<float *>(P + L.p_ggrad);
    float2 *sc = reinterpret_cast<float2 *>(P + L.p_sc);
    float *red = reinterpret_cast<float *>(P + L.p_red);
    float *stage = reinterpret_cast<float *>(P + L.p_stage) + (gt >> 5) * 32 * 12;
    float4 *fbuf = reinterpret_cast<float4 *>(P + L.p_force);
    constexpr int MAXA = ADGB_MAX_ATOMS / TPP;  // atoms owned per thread, at most

    constexpr int NG = NGS;
    float om[NG], eg2[NG], ed2[NG], best[NG];
#pragma unroll
    for (int r = 0; r < NG; r++) {
        const int j = gt + r * TPP;
        om[r] = eg2[r] = ed2[r] = 0.f;
        if (j < G) {
            if (io.resume) {
                const float *st = io.state;
                om[r] = st[j];
                eg2[r] = st[G + j];
                ed2[r] = st[2 * G + j];
            } else {
                om[r] = io.genes_in[j];
            }
        }
        best[r] = om[r];
    }
    float best_e = INFINITY;
    const int iters = io.iters;

    for (int it = 0; it < iters; it++) {
        // 1. publish genes, sin and 1 - cos of every angle (half-angle form:
        //    sin = 2 sh ch, 1 - cos = 2 sh^2, exact zero at a zero angle).  phi
        //    and theta are published as (sin, cos) of the full angle.  One
        //    sincosf per gene on every lane keeps the lanes converged.
#pragma unroll
        for (int r = 0; r < NG; r++) {
            const int j = gt + r * TPP;
            if (r * TPP < G) {
                const bool full = j == 3 || j == 4;
                float sh, ch;
                sincosf(full ? om[r] : 0.5f * om[r], &sh, &ch);
                if (j < G) {
                    genes_s[j] = om[r];
                    const float2 v = full ? make_float2(sh, ch)
                                          : make_float2(2.f * sh * ch, 2.f * sh * sh);
                    if (j >= 6) sc[j - 6] = v;
                    else if (j >= 3) sc[SC_ROT + j - 3] = v;
                }
            }
        }
        group_sync<TPP>(group);
        const float3 tr = make_float3(genes_s[0], genes_s[1], genes_s[2]);
        const float2 sphi = sc[SC_ROT], sth = sc[SC_ROT + 1], sal = sc[SC_ROT + 2];
        const float3 u = make_float3(sth.x * sphi.y, sth.x * sphi.x, sth.y);
        // R - I = sin(a) [u]x + (1 - cos(a)) (u u^T - I)
        const float s = sal.x, o = sal.y;
        const float m00 = o * (u.x * u.x - 1.f), m11 = o * (u.y * u.y - 1.f),
                    m22 = o * (u.z * u.z - 1.f);
        const float m01 = o * u.x * u.y - s * u.z, m10 = o * u.x * u.y + s * u.z;
        const float m02 = o * u.x * u.z + s * u.y, m20 = o * u.x * u.z - s * u.y;
        const float m12 = o * u.y * u.z - s * u.x, m21 = o * u.y * u.z + s * u.x;

        // 2. coordinates and intermolecular terms.  With matching rounds
        //    (lane a owns atom a: one warp and shuffles up to 32 atoms, else
        //    the pose's threads with atoms gt and gt + TPP, more lanes than
        //    threads, and slots in shared memory) the thread keeps its atoms'
        //    positions and gradients in registers.
        const bool rounds = TPP == 32 && lig.n_rounds > 0 && lig.r_lanes == 32;
        const bool brounds = TPP > 32 && lig.n_rounds > 0 && lig.r_lanes > TPP &&
                             lig.r_lanes <= 2 * TPP;
        float3 xo = make_float3(0.f, 0.f, 0.f), go = xo, xo1 = xo, go1 = xo;
        float e_part = 0.f;
        for (int i = gt; i < N; i += TPP) {
            const float4 r4 = s_ref[i];
            float3 p = make_float3(r4.x, r4.y, r4.z);
            for (int k = s_frag[i]; k >= 0; k = s_tpar[k]) rotate_about(p, s_tax[k], s_tb[k], sc[k]);
            float3 x;
            x.x = p.x + (m00 * p.x + m01 * p.y + m02 * p.z) + tr.x;
            x.y = p.y + (m10 * p.x + m11 * p.y + m12 * p.z) + tr.y;
            x.z = p.z + (m20 * p.x + m21 * p.y + m22 * p.z) + tr.z;
            xyz[i] = make_float4(x.x, x.y, x.z, r4.w);
            float3 g;
            e_part += inter_atom(rec, s_type[i], r4.w, x, g);
            if (rounds || (brounds && i == gt)) {
                xo = x;
                go = g;
            } else if (brounds) {
                xo1 = x;
                go1 = g;
            } else {
                grd[i] = make_float4(g.x, g.y, g.z, 0.f);
            }
        }
        group_sync<TPP>(group);

        // 3c. block form of the matching rounds: in each chunk of rounds every
        //     lane writes its pair's force to its slot of the round, then
        //     (after one barrier) takes the forces of the (at most two) pairs
        //     whose second atom is its own from the slots its words name.
        //     Every slot of a round is written (lanes without a pair write an
        //     exact zero), so an unused receive slot, weighted by zero, reads a
        //     finite value.
        if (brounds) {
            const int VP = lig.r_lanes, R = lig.n_rounds;
            const int RC = max(1, L.chunk / VP);   // rounds a chunk (slots: RC x VP float4)
            const bool has0 = gt < VP, has1 = gt + TPP < VP;
            const uint32_t *rw = lig.rword;
            const float4 *rcs = lig.rconst;
            auto take = [&](float3 &g, uint32_t w, const float4 *slot) {
                const float m1 = (w >> 25) & 1 ? 1.f : 0.f, m2 = (w >> 26) & 1 ? 1.f : 0.f;
                const float4 f1 = slot[(w >> 8) & 255], f2 = slot[(w >> 16) & 255];
                g.x -= m1 * f1.x + m2 * f2.x;
                g.y -= m1 * f1.y + m2 * f2.y;
                g.z -= m1 * f1.z + m2 * f2.z;
            };
            for (int r0 = 0; r0 < R; r0 += RC) {
                const int r1 = min(R, r0 + RC);
                for (int r = r0; r < r1; r++) {
                    float4 *slot = fbuf + (r - r0) * VP;
                    if (has1) {   // both atoms of the thread: packed arithmetic
                        const uint32_t wa = __ldg(rw + (size_t)r * VP + gt);
                        const uint32_t wb = __ldg(rw + (size_t)r * VP + gt + TPP);
                        float3 fa, fb;
                        e_part += pair_term2(xo, xo1, xyz3(xyz[wa & 255]), xyz3(xyz[wb & 255]),
                                             __ldg(rcs + (size_t)r * VP + gt),
                                             __ldg(rcs + (size_t)r * VP + gt + TPP),
                                             (wa >> 24) & 1, (wb >> 24) & 1, fa, fb);
                        go.x += fa.x;
                        go.y += fa.y;
                        go.z += fa.z;
                        go1.x += fb.x;
                        go1.y += fb.y;
                        go1.z += fb.z;
                        slot[gt] = make_float4(fa.x, fa.y, fa.z, 0.f);
                        slot[gt + TPP] = make_float4(fb.x, fb.y, fb.z, 0.f);
                    } else if (has0) {
                        const uint32_t w = __ldg(rw + (size_t)r * VP + gt);
                        float3 f;
                        e_part += pair_term(make_float4(xo.x, xo.y, xo.z, 0.f), xyz[w & 255],
                                            __ldg(rcs + (size_t)r * VP + gt), (w >> 24) & 1, f);
                        go.x += f.x;
                        go.y += f.y;
                        go.z += f.z;
                        slot[gt] = make_float4(f.x, f.y, f.z, 0.f);
                    }
                }
                group_sync<TPP>(group);
                for (int r = r0; r < r1; r++) {
                    const float4 *slot = fbuf + (r - r0) * VP;
                    if (has0) take(go, __ldg(rw + (size_t)r * VP + gt), slot);
                    if (has1) take(go1, __ldg(rw + (size_t)r * VP + gt + TPP), slot);
                }
                group_sync<TPP>(group);   // the slots are rewritten by the next chunk
            }
            if (gt < N) grd[gt] = make_float4(go.x, go.y, go.z, 0.f);
            if (gt + TPP < N) grd[gt + TPP] = make_float4(go1.x, go1.y, go1.z, 0.f);
            group_sync<TPP>(group);   // gradients visible to the torsion scans
        }

        // 3a. intramolecular pairs in matching rounds: the partner's position
        //     and the reaction forces of the (at most two) pairs whose second
        //     atom is the lane's come by shuffles, an unused receive slot
        //     weighted by zero; lanes without a pair compute an exact zero
        //     (zero constants, partner = itself).
        if (rounds) {
            const uint32_t *rw = lig.rword + gt;
            const float4 *rc = lig.rconst + gt;
            const int R = lig.n_rounds;
            auto partner = [&](uint32_t w) {
                const int pj = w & 31;
                return make_float3(__shfl_sync(0xffffffffu, xo.x, pj),
                                   __shfl_sync(0xffffffffu, xo.y, pj),
                                   __shfl_sync(0xffffffffu, xo.z, pj));
            };
            auto settle = [&](uint32_t w, float3 f) {  // own force in, received forces out
                const int s1 = (w >> 8) & 31, s2 = (w >> 16) & 31;
                const float m1 = (w >> 25) & 1 ? 1.f : 0.f, m2 = (w >> 26) & 1 ? 1.f : 0.f;
                go.x += f.x;
                go.y += f.y;
                go.z += f.z;
                go.x -= m1 * __shfl_sync(0xffffffffu, f.x, s1);
                go.y -= m1 * __shfl_sync(0xffffffffu, f.y, s1);
                go.z -= m1 * __shfl_sync(0xffffffffu, f.z, s1);
                go.x -= m2 * __shfl_sync(0xffffffffu, f.x, s2);
                go.y -= m2 * __shfl_sync(0xffffffffu, f.y, s2);
                go.z -= m2 * __shfl_sync(0xffffffffu, f.z, s2);
            };
            int r = 0;
#pragma unroll 2
            for (; r + 1 < R; r += 2) {  // two rounds at once, packed arithmetic
                const uint32_t wa = __ldg(rw + 32 * r), wb = __ldg(rw + 32 * (r + 1));
                const float4 pa = __ldg(rc + 32 * r), pb = __ldg(rc + 32 * (r + 1));
                const float3 xa = partner(wa), xb = partner(wb);
                float3 fa, fb;
                e_part += pair_term2(xo, xo, xa, xb, pa, pb, (wa >> 24) & 1, (wb >> 24) & 1, fa,
                                     fb);
                settle(wa, fa);
                settle(wb, fb);
            }
            if (r < R) {
                const uint32_t w = __ldg(rw + 32 * r);
                const float4 pc = __ldg(rc + 32 * r);
                const float3 xj = partner(w);
                float3 f;
                e_part += pair_term(make_float4(xo.x, xo.y, xo.z, 0.f),
                                    make_float4(xj.x, xj.y, xj.z, 0.f), pc, (w >> 24) & 1, f);
                settle(w, f);
            }
        }

        // 3b. otherwise, chunk by chunk (PAIR_CHUNK pairs): every
        //    pair's force goes to its own slot of the force buffer, then each
        //    atom's owner adds the forces of its pairs in the chunk (per-chunk
        //    incidence lists with known bounds).  No two threads ever write
        //    the same word.
        for (int q = 0; q < (rounds || brounds ? 0 : lig.n_chunks); q++) {
            const int c0 = q * PAIR_CHUNK, c1 = min(NP, c0 + PAIR_CHUNK);
            int p = c0 + gt;
            for (; p + TPP < c1; p += 2 * TPP) {  // pairs p and p + TPP, packed arithmetic
                const uint32_t pa = prs[p], pb = prs[p + TPP];
                float3 fa, fb;
                e_part += pair_term2(xyz3(xyz[pa & 255]), xyz3(xyz[pb & 255]),
                                     xyz3(xyz[(pa >> 8) & 255]), xyz3(xyz[(pb >> 8) & 255]),
                                     __ldg(pconst + p), __ldg(pconst + p + TPP), (pa >> 24) & 1,
                                     (pb >> 24) & 1, fa, fb);
                fbuf[p - c0] = make_float4(fa.x, fa.y, fa.z, 0.f);
                fbuf[p + TPP - c0] = make_float4(fb.x, fb.y, fb.z, 0.f);
            }
            if (p < c1) {
                const uint32_t pr = prs[p];
                const int i = pr & 255, j = (pr >> 8) & 255;
                float3 f;
                e_part += pair_term(xyz[i], xyz[j], __ldg(pconst + p), (pr >> 24) & 1, f);
                fbuf[p - c0] = make_float4(f.x, f.y, f.z, 0.f);
            }
            group_sync<TPP>(group);
            const int *off = sl.incoff + q * (N + 1);
#pragma unroll
            for (int m = 0; m < MAXA; m++) {
                const int i = gt + m * TPP;
                if (i < N) {
                    const int cb = off[i], ce = off[i + 1];
                    float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll 4
                    for (int c = cb; c < ce; c++) {
                        const uint32_t e = incl[c];
                        const float4 f = fbuf[e >> 1];
                        const float sg = (e & 1) ? -1.f : 1.f;
                        ax += sg * f.x;
                        ay += sg * f.y;
                        az += sg * f.z;
                    }
                    const float4 g = grd[i];
                    grd[i] = make_float4(g.x + ax, g.y + ay, g.z + az, 0.f);
                }
            }
            group_sync<TPP>(group);
        }

        // 4. partial sums of (E, sum g, torque about the centre); torsion gradients
        float v[8] = {e_part, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int i = gt; i < N; i += TPP) {
            const float4 g = rounds ? make_float4(go.x, go.y, go.z, 0.f) : grd[i];
            const float4 x = rounds ? make_float4(xo.x, xo.y, xo.z, 0.f) : xyz[i];
            const float3 d = make_float3(x.x - tr.x, x.y - tr.y, x.z - tr.z);
            const float3 c = make_float3(d.y * g.z - d.z * g.y, d.z * g.x - d.x * g.z,
                                         d.x * g.y - d.y * g.x);
            v[1] += g.x;
            v[2] += g.y;
            v[3] += g.z;
            v[4] += c.x;
            v[5] += c.y;
            v[6] += c.z;
        }
        // the tensor-core reduction of the partials runs while the torsion
        // sums below are computed
        if constexpr (VAR == ADGB_REDUCE_TCGEN05) tc05_issue(v, tw);
        if (N <= 32) {
            // one atom per lane of the group's first warp: each torsion's lane
            // sums its moving atoms (one contiguous range [s, e) of the
            // depth-first order) with the lever arm from the bond's atom b,
            // a . sum (x - x_b) x g, from the shared coordinates and gradients
            if (rounds && gt < N) grd[gt] = make_float4(go.x, go.y, go.z, 0.f);
            group_sync<TPP>(group);
            for (int k = gt; k < T; k += TPP) {
                const int4 ta = s_tat[k];
                float gk = 0.f;
                if (ta.w > ta.z) {
                    const float4 xa = xyz[ta.x], xb = xyz[ta.y];
                    float3 acc = make_float3(0.f, 0.f, 0.f);
                    for (int i = ta.z; i < ta.w; i++) {
                        const float4 g = grd[i], x = xyz[i];
                        const float3 d = make_float3(x.x - xb.x, x.y - xb.y, x.z - xb.z);
                        acc.x += d.y * g.z - d.z * g.y;
                        acc.y += d.z * g.x - d.x * g.z;
                        acc.z += d.x * g.y - d.y * g.x;
                    }
                    const float3 ax = make_float3(xb.x - xa.x, xb.y - xa.y, xb.z - xa.z);
                    const float il = rsqrtf(ax.x * ax.x + ax.y * ax.y + ax.z * ax.z);
                    gk = (ax.x * acc.x + ax.y * acc.y + ax.z * acc.z) * il;
                }
                ggrad[6 + k] = gk;
            }
        } else {
            // any N: each torsion's gradient as a direct sum over its moving
            // atoms (one contiguous range of the depth-first order) with the
            // lever arm from the bond's atom b, a . sum (x - x_b) x g: warp w of
            // the pose takes torsions w, w + W, ...; its lanes stride the
            // range, then a butterfly sums the lanes (a fixed order).  (A
            // difference of prefix sums over the whole order would cancel
            // every atom before the range: for large forces far more rounding
            // error than the torsion's own terms carry.)
            group_sync<TPP>(group);
            constexpr int W = TPP / 32;
            const int lane = gt & 31;
            for (int k0 = 0; k0 < T; k0 += W) {
                const int k = k0 + (gt >> 5);   // warp-uniform
                float3 acc = make_float3(0.f, 0.f, 0.f);
                int4 ta = make_int4(0, 0, 0, 0);
                float4 xb = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k < T) {
                    ta = s_tat[k];
                    xb = xyz[ta.y];
                    for (int i = ta.z + lane; i < ta.w; i += 32) {
                        const float4 g = grd[i], x = xyz[i];
                        const float3 d = make_float3(x.x - xb.x, x.y - xb.y, x.z - xb.z);
                        acc.x += d.y * g.z - d.z * g.y;
                        acc.y += d.z * g.x - d.x * g.z;
                        acc.z += d.x * g.y - d.y * g.x;
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
                    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, off);
                }
                if (k < T && lane == 0) {
                    float gk = 0.f;
                    if (ta.w > ta.z) {
                        const float4 xa = xyz[ta.x];
                        const float3 ax = make_float3(xb.x - xa.x, xb.y - xa.y, xb.z - xa.z);
                        const float il = rsqrtf(ax.x * ax.x + ax.y * ax.y + ax.z * ax.z);
                        gk = (ax.x * acc.x + ax.y * acc.y + ax.z * acc.z) * il;
                    }
                    ggrad[6 + k] = gk;
                }
            }
        }

        // 5. one reduce-and-broadcast of the 8-vector
        group_sum8<TPP, VAR, true>(v, red, stage, group, gt, tw);
        group_sync<TPP>(group);  // torsion gradients visible

        // 6. gene gradient, best tracking, ADADELTA
        const float E = v[0];
        float gj[NG];
#pragma unroll
        for (int r = 0; r < NG; r++) {
            const int j = gt + r * TPP;
            float g = 0.f;
            if (j < 3) {
                g = v[1 + j];
            } else if (j < 5) {
                // d u / d phi or d theta; angular velocity sin(a) du + (1-cos a) u x du
                const float3 du = j == 3 ? make_float3(-sth.x * sphi.x, sth.x * sphi.y, 0.f)
                                         : make_float3(sth.y * sphi.y, sth.y * sphi.x, -sth.x);
                const float3 uxd = cross3(u, du);
                const float3 w = make_float3(s * du.x + o * uxd.x, s * du.y + o * uxd.y,
                                             s * du.z + o * uxd.z);
                g = v[4] * w.x + v[5] * w.y + v[6] * w.z;
            } else if (j == 5) {
                g = v[4] * u.x + v[5] * u.y + v[6] * u.z;
            } else if (j < G) {
                g = ggrad[j];
            }
            gj[r] = g;
        }
        if (io.mode == MODE_SCORE) {
            if (gt == 0) io.energy[0] = E;
            if (io.grad) {
#pragma unroll
                for (int r = 0; r < NG; r++) {
                    const int j = gt + r * TPP;
                    if (j < G) io.grad[j] = gj[r];
                }
            }
            return;
        }
        if (E < best_e) {
            best_e = E;
#pragma unroll
            for (int r = 0; r < NG; r++) best[r] = om[r];
        }
#pragma unroll
        for (int r = 0; r < NG; r++) {
            const int j = gt + r * TPP;
            if (j < G) {
                const float g = gj[r];
                eg2[r] = io.rho * eg2[r] + (1.f - io.rho) * g * g;
                const float d = -sqrtf(ed2[r] + io.eps) * rsqrtf(eg2[r] + io.eps) * g;
                ed2[r] = io.rho * ed2[r] + (1.f - io.rho) * d * d;
                float w = om[r] + d;
                if (j >= 6) w -= 2.f * PI_F * floorf((w + PI_F) * (0.5f / PI_F));
                om[r] = w;
            }
        }
    }
    if (io.mode == MODE_SCORE) return;  // iters == 0 never reaches here in score mode
#pragma unroll
    for (int r = 0; r < NG; r++) {
        const int j = gt + r * TPP;
        if (j < G) {
            io.genes_out[j] = best[r];
            if (io.state) {
                float *st = io.state;
                st[j] = om[r];
                st[G + j] = eg2[r];
                st[2 * G + j] = ed2[r];
            }
        }
    }
    if (gt == 0) io.energy[0] = best_e;
}

// ---------------------------------------------------------------------------
// Solis-Wets local search (Solis and Wets, Math. Oper. Res. 6, 1981, as
// AutoDock's alternative to the gradient search; Sec. 2.1 names both local
// searches).  Energy only: no forces, gather, torsion scans or gene gradient,
// one reduction of E per evaluation.  Each step draws a deviate
// d = bias + rho * sigma_j * z (z standard normal, sigma_j = 1 A for the
// translation genes, angle_scale rad for the angles), tries x + d, then x - d;
// a success moves x and updates the bias (0.2 b + 0.4 d forward, b - 0.4 d
// backward), a failure halves the bias; max_succ successes in a row double
// rho, max_fail failures halve it.  A search ends after max_evals
// evaluations or when rho < rho_min.  x only ever moves to a lower energy,
// so the final x is the best seen.
// ---------------------------------------------------------------------------
struct SwArgs {
    RecDev rec;
    LigDev lig;
    SmemLayout L;
    float *genes;         // [n][G] in (start) / out (final = best)
    float *energy;        // [n] out
    int *evals;           // [n] out or null
    float *state;         // [n][2G + 5] (x, bias, rho, successes, failures, E, step) or null
    const int *budget;    // [n] evaluations each genotype may spend, or null (max_evals)
    int n, max_evals, max_succ, max_fail, resume;
    float rho0, rho_min, angle_scale;
    uint64_t seed;
    uint32_t call;        // random-stream selector (with the genotype index and the step)
    int pose_base;        // genotype index of genes[0] in the random stream
};

constexpr uint32_t SW_TAG = 0x53570000u;

// Standard normal number j of step `it` of genotype `pose`: Box-Muller on
// two 24-bit uniforms of one Philox4x32-10 output (u1 in (0, 1], u2 in [0, 1)).
__device__ __forceinline__ float sw_normal(uint64_t seed, uint32_t pose, uint32_t it,
                                           uint32_t call, int j) {
    const Philox4 o = philox4x32_10(pose, it, SW_TAG | (call & 0xFFFFu), (uint32_t)j >> 2,
                                    (uint32_t)seed, (uint32_t)(seed >> 32));
    const bool second = (j >> 1) & 1;
    const uint32_t a = second ? o.z : o.x, b = second ? o.w : o.y;
    const float u1 = (float)((a >> 8) + 1u) * (1.0f / 16777216.0f);
    const float u2 = (float)(b >> 8) * (1.0f / 16777216.0f);
    const float r = sqrtf(-2.f * logf(u1));
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    return (j & 1) ? r * sn : r * cs;
}

template <int TPP, int VAR>
__device__ __forceinline__ void search_pose_sw(unsigned char *sm, const SmemLayout &L,
                                               const LigDev &lig, const RecDev &rec,
                                               const StagedLig &sl, const int group, const int gt,
                                               const SwArgs &a, const int pose, Tc05Warp &tw) {
    const int N = lig.n_atoms, T = lig.n_tors, G = 6 + T, NP = lig.n_pairs;
    float4 *s_ref = reinterpret_cast<float4 *>(sm + L.ref);
    int *s_type = reinterpret_cast<int *>(sm + L.type);
    int *s_frag = reinterpret_cast<int *>(sm + L.frag);
    int *s_tpar = reinterpret_cast<int *>(sm + L.tparent);
    float4 *s_tax = reinterpret_cast<float4 *>(sm + L.taxis);
    float4 *s_tb = reinterpret_cast<float4 *>(sm + L.tbref);
    const float4 *pconst = lig.pconst;
    const uint32_t *prs = sl.prs;
    unsigned char *P = sm + L.pose0 + group * L.pose_stride;
    float4 *xyz = reinterpret_cast<float4 *>(P + L.p_xyz);
    float *genes_s = reinterpret_cast<float *>(P + L.p_genes);
    float2 *sc = reinterpret_cast<float2 *>(P + L.p_sc);
    float *red = reinterpret_cast<float *>(P + L.p_red);
    float *stage = reinterpret_cast<float *>(P + L.p_stage) + (gt >> 5) * 32 * 12;
    constexpr int NG = (MAX_GENES + TPP - 1) / TPP;

    // energy of the genotype held lane-wise in g[] (whole group)
    auto energy = [&](const float *g) -> float {
#pragma unroll
        for (int r = 0; r < NG; r++) {
            const int j = gt + r * TPP;
            if (r * TPP < G) {
                const bool full = j == 3 || j == 4;
                float sh, ch;
                sincosf(full ? g[r] : 0.5f * g[r], &sh, &ch);
                if (j < G) {
                    genes_s[j] = g[r];
                    const float2 v = full ? make_float2(sh, ch)
                                          : make_float2(2.f * sh * ch, 2.f * sh * sh);
                    if (j >= 6) sc[j - 6] = v;
                    else if (j >= 3) sc[SC_ROT + j - 3] = v;
                }
            }
        }
        group_sync<TPP>(group);
        const float3 tr = make_float3(genes_s[0], genes_s[1], genes_s[2]);
        const float2 sphi = sc[SC_ROT], sth = sc[SC_ROT + 1], sal = sc[SC_ROT + 2];
        const float3 u = make_float3(sth.x * sphi.y, sth.x * sphi.x, sth.y);
        const float s = sal.x, o = sal.y;
        const float m00 = o * (u.x * u.x - 1.f), m11 = o * (u.y * u.y - 1.f),
                    m22 = o * (u.z * u.z - 1.f);
        const float m01 = o * u.x * u.y - s * u.z, m10 = o * u.x * u.y + s * u.z;
        const float m02 = o * u.x * u.z + s * u.y, m20 = o * u.x * u.z - s * u.y;
        const float m12 = o * u.y * u.z - s * u.x, m21 = o * u.y * u.z + s * u.x;
        float e_part = 0.f;
        for (int i = gt; i < N; i += TPP) {
            const float4 r4 = s_ref[i];
            float3 p = make_float3(r4.x, r4.y, r4.z);
            for (int k = s_frag[i]; k >= 0; k = s_tpar[k]) rotate_about(p, s_tax[k], s_tb[k], sc[k]);
            float3 x;
            x.x = p.x + (m00 * p.x + m01 * p.y + m02 * p.z) + tr.x;
            x.y = p.y + (m10 * p.x + m11 * p.y + m12 * p.z) + tr.y;
            x.z = p.z + (m20 * p.x + m21 * p.y + m22 * p.z) + tr.z;
            xyz[i] = make_float4(x.x, x.y, x.z, r4.w);
            float3 gi;
            e_part += inter_atom(rec, s_type[i], r4.w, x, gi);
        }
        group_sync<TPP>(group);
        int p = gt;
        for (; p + TPP < NP; p += 2 * TPP) {  // pairs p and p + TPP, packed arithmetic
            const uint32_t pa = prs[p], pb = prs[p + TPP];
            float3 fa, fb;
            e_part += pair_term2(xyz3(xyz[pa & 255]), xyz3(xyz[pb & 255]),
                                 xyz3(xyz[(pa >> 8) & 255]), xyz3(xyz[(pb >> 8) & 255]),
                                 __ldg(pconst + p), __ldg(pconst + p + TPP), (pa >> 24) & 1,
                                 (pb >> 24) & 1, fa, fb);
        }
        if (p < NP) {
            const uint32_t pr = prs[p];
            float3 f;
            e_part += pair_term(xyz[pr & 255], xyz[(pr >> 8) & 255], __ldg(pconst + p),
                                (pr >> 24) & 1, f);
        }
        float v[8] = {e_part, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        group_sum8<TPP, VAR>(v, red, stage, group, gt, tw);
        group_sync<TPP>(group);   // every lane is done with genes_s, sc and xyz
        return v[0];
    };

    float *gio = a.genes + (size_t)pose * G;
    float *st = a.state ? a.state + (size_t)pose * (2 * G + 5) : nullptr;
    const int max_evals = a.budget ? a.budget[pose] : a.max_evals;
    float x[NG], bias[NG], y[NG], d[NG];
    float rho, Ex;
    int ns, nf, step, evals = 0;
#pragma unroll
    for (int r = 0; r < NG; r++) {
        const int j = gt + r * TPP;
        x[r] = bias[r] = 0.f;
        if (j < G) {
            x[r] = a.resume ? st[j] : gio[j];
            bias[r] = a.resume ? st[G + j] : 0.f;
        }
    }
    if (a.resume) {
        rho = st[2 * G];
        ns = (int)st[2 * G + 1];
        nf = (int)st[2 * G + 2];
        Ex = st[2 * G + 3];
        step = (int)st[2 * G + 4];
    } else {
        rho = a.rho0;
        ns = nf = step = 0;
        Ex = max_evals > 0 ? energy(x) : INFINITY;
        evals = max_evals > 0 ? 1 : 0;
    }
    const uint32_t id = (uint32_t)(a.pose_base + pose);
    while (evals < max_evals && rho >= a.rho_min) {
#pragma unroll
        for (int r = 0; r < NG; r++) {
            const int j = gt + r * TPP;
            d[r] = y[r] = 0.f;
            if (j < G) {
                const float z = sw_normal(a.seed, id, (uint32_t)step, a.call, j);
                d[r] = bias[r] + rho * (j < 3 ? 1.f : a.angle_scale) * z;
                float w = x[r] + d[r];
                if (j >= 6) w -= 2.f * PI_F * floorf((w + PI_F) * (0.5f / PI_F));
                y[r] = w;
            }
        }
        const float E1 = energy(y);
        evals++;
        bool ok = E1 < Ex;
        if (ok) {
            Ex = E1;
#pragma unroll
            for (int r = 0; r < NG; r++) {
                x[r] = y[r];
                bias[r] = 0.2f * bias[r] + 0.4f * d[r];
            }
        } else if (evals < max_evals) {
#pragma unroll
            for (int r = 0; r < NG; r++) {
                const int j = gt + r * TPP;
                float w = x[r] - d[r];
                if (j >= 6) w -= 2.f * PI_F * floorf((w + PI_F) * (0.5f / PI_F));
                y[r] = j < G ? w : 0.f;
            }
            const float E2 = energy(y);
            evals++;
            ok = E2 < Ex;
            if (ok) {
                Ex = E2;
#pragma unroll
                for (int r = 0; r < NG; r++) {
                    x[r] = y[r];
                    bias[r] = bias[r] - 0.4f * d[r];
                }
            }
        }
        if (!ok) {
#pragma unroll
            for (int r = 0; r < NG; r++) bias[r] *= 0.5f;
        }
        if (ok) {
            ns++;
            nf = 0;
        } else {
            nf++;
            ns = 0;
        }
        if (ns >= a.max_succ) {
            rho *= 2.f;
            ns = 0;
        }
        if (nf >= a.max_fail) {
            rho *= 0.5f;
            nf = 0;
        }
        step++;
    }
#pragma unroll
    for (int r = 0; r < NG; r++) {
        const int j = gt + r * TPP;
        if (j < G) {
            gio[j] = x[r];
            if (st) {
                st[j] = x[r];
                st[G + j] = bias[r];
            }
        }
    }
    group_sync<TPP>(group);   // every lane has read the budget before it is overwritten
    if (gt == 0) {
        a.energy[pose] = Ex;
        if (a.evals) a.evals[pose] = evals;
        if (st) {
            st[2 * G] = rho;
            st[2 * G + 1] = (float)ns;
            st[2 * G + 2] = (float)nf;
            st[2 * G + 3] = Ex;
            st[2 * G + 4] = (float)step;
        }
    }
}

template <int TPP, int VAR>
__global__ void __launch_bounds__(128, ADGB_MIN_BLOCKS) sw_kernel(const SwArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + tc_front<VAR>();
    const StagedLig sl = stage_ligand(sm, a.L, a.lig);
    Tc05Warp tw;
    tc_begin<VAR>(smem_raw, tw);
    __syncthreads();
    const int group = threadIdx.x / TPP, gt = threadIdx.x % TPP;
    const int pose = blockIdx.x * (blockDim.x / TPP) + group;
    if (pose < a.n) search_pose_sw<TPP, VAR>(sm, a.L, a.lig, a.rec, sl, group, gt, a, pose, tw);
    tc_end<VAR>(tw);
}

template <int TPP, int VAR, int NGS>
__device__ __forceinline__ void eval_one(const EvalArgs &a, const StagedLig &sl, unsigned char *sm,
                                         int group, int gt, int pose, Tc05Warp &tw) {
    const int G = 6 + a.lig.n_tors;
    PoseIO io;
    io.genes_in = a.genes_in ? a.genes_in + (size_t)pose * G : nullptr;
    io.genes_out = a.genes_out ? a.genes_out + (size_t)pose * G : nullptr;
    io.energy = a.energy + pose;
    io.grad = a.grad ? a.grad + (size_t)pose * G : nullptr;
    io.state = a.state ? a.state + (size_t)pose * 3 * G : nullptr;
    io.iters = a.mode == MODE_SCORE ? 1 : (a.iters_pp ? a.iters_pp[pose] : a.iters);
    io.mode = a.mode;
    io.resume = a.resume;
    io.rho = a.rho;
    io.eps = a.eps;
    search_pose<TPP, VAR, NGS>(sm, a.L, a.lig, a.rec, sl, group, gt, io, tw);
}

template <int TPP, int VAR, int NGS>
__global__ void __launch_bounds__(128, ADGB_MIN_BLOCKS) eval_kernel(const EvalArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + tc_front<VAR>();
    const StagedLig sl = stage_ligand(sm, a.L, a.lig);
    Tc05Warp tw;
    tc_begin<VAR>(smem_raw, tw);
    __syncthreads();
    const int group = threadIdx.x / TPP, gt = threadIdx.x % TPP;
    const int pose = blockIdx.x * (blockDim.x / TPP) + group;
    if (pose < a.n) eval_one<TPP, VAR, NGS>(a, sl, sm, group, gt, pose, tw);
    tc_end<VAR>(tw);
}

// Persistent multi-ligand local search: every block takes work items from a
// device counter until the table is exhausted; a block re-stages the ligand
// constants only when the item's ligand differs from its previous one.
// Items are ordered by decreasing cost on the host (longest first).
struct ItemsArgs {
    const WorkItem *items;
    const LigDev *ligs;
    const RecDev *recs;
    int *counter;
    int n_items, ppb, budget;
};

template <int TPP, int VAR>
__global__ void __launch_bounds__(128, ADGB_ITEMS_MIN_BLOCKS) eval_items_kernel(const ItemsArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + items_front<VAR>();
    int &s_item = *reinterpret_cast<int *>(sm - 16);
    SmemLayout &L = *reinterpret_cast<SmemLayout *>(sm - ITEMS_HDR);
    constexpr int NG_MAX = (MAX_GENES + TPP - 1) / TPP;
    const int group = threadIdx.x / TPP, gt = threadIdx.x % TPP;
    int cur_lig = -1;
    StagedLig sl;
    Tc05Warp tw;
    tc_begin<VAR>(smem_raw, tw);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= a.n_items) break;
        const WorkItem w = a.items[it];
        if (w.lig != cur_lig) {
            const LigDev &lg = a.ligs[w.lig];
            if (threadIdx.x == 0)
                L = SmemLayout::choose(lg.n_atoms, lg.n_tors, lg.n_pairs, a.ppb, TPP / 32,
                                       uses_mma_stage(VAR));
            __syncthreads();
            sl = stage_ligand(sm, L, lg);
            cur_lig = w.lig;
            __syncthreads();
        }
        if (group < w.count) {
            PoseIO io;
            io.genes_in = w.genes + (size_t)group * w.gstride;
            io.genes_out = w.genes + (size_t)group * w.gstride;
            io.energy = w.energy + group;
            io.grad = nullptr;
            io.state = nullptr;
            io.iters = w.iters ? w.iters[group] : w.iters_all;
            io.mode = MODE_LS;
            io.resume = 0;
            io.rho = w.rho;
            io.eps = w.eps;
            // same specialisation as the single-ligand launch, so that both
            // give bit-identical searches
            const LigDev &lg = a.ligs[w.lig];
            if (NG_MAX > 1 && 6 + lg.n_tors <= TPP)
                search_pose<TPP, VAR, 1>(sm, L, lg, a.recs[w.rec], sl, group, gt, io, tw);
            else
                search_pose<TPP, VAR, NG_MAX>(sm, L, lg, a.recs[w.rec], sl, group, gt, io, tw);
        }
        __syncthreads();  // the item is done before smem or s_item change
    }
    tc_end<VAR>(tw);
    // the last block out re-arms the counter so that the launch can be replayed
    if (threadIdx.x == 0) {
        __threadfence();
        const int done = atomicAdd(a.counter + 1, 1);
        if (done == (int)gridDim.x - 1) {
            a.counter[0] = 0;
            a.counter[1] = 0;
            __threadfence();
        }
    }
}

// Dynamic shared memory of an eval launch whose layout needs `layout_bytes`:
// the tcgen05 variant puts its region in front and pads the total so that
// no more blocks are resident on an SM than its 512 TMEM columns serve at
// once (tcgen05.alloc would otherwise wait for a resident block to finish).
int eval_smem_bytes(int layout_bytes, const EvalCfg &cfg, int device, bool items) {
    if (cfg.variant != ADGB_REDUCE_TCGEN05) return layout_bytes + (items ? ITEMS_HDR : 0);
    int total = TC_REGION + (items ? ITEMS_HDR : 0) + layout_bytes;
    int sm_smem = 0, reserved = 0;
    if (cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device) !=
            cudaSuccess)
        return -1;
    const int fit = 512 / tc_ncols(cfg.tpp * cfg.ppb / 32);
    const int floor_bytes = sm_smem / (fit + 1) - reserved + 16;
    return total < floor_bytes ? floor_bytes : total;
}

template <int TPP, int VAR>
static cudaError_t launch_items_t(const ItemsArgs &a, int smem, int grid, cudaStream_t s) {
    auto k = eval_items_kernel<TPP, VAR>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, TPP * a.ppb, smem, s>>>(a);
    return cudaGetLastError();
}

template <int TPP>
static cudaError_t launch_items_v(const ItemsArgs &a, int variant, int smem, int grid,
                                  cudaStream_t s) {
    switch (variant) {
        case ADGB_REDUCE_SHFL: return launch_items_t<TPP, ADGB_REDUCE_SHFL>(a, smem, grid, s);
        case ADGB_REDUCE_MMA_TF32X2:
            return launch_items_t<TPP, ADGB_REDUCE_MMA_TF32X2>(a, smem, grid, s);
        case ADGB_REDUCE_MMA_BF16X3:
            return launch_items_t<TPP, ADGB_REDUCE_MMA_BF16X3>(a, smem, grid, s);
        case ADGB_REDUCE_TCGEN05:
            return launch_items_t<TPP, ADGB_REDUCE_TCGEN05>(a, smem, grid, s);
    }
    return cudaErrorInvalidValue;
}

int items_layout_bytes(const EvalCfg &cfg, int n_atoms, int n_tors, int n_pairs) {
    if (cfg.paired) return pair_layout_bytes(n_atoms, n_tors, cfg.ppb, cfg.variant);
    return SmemLayout::choose(n_atoms, n_tors, n_pairs, cfg.ppb, cfg.tpp / 32,
                              uses_mma_stage(cfg.variant)).total;
}

cudaError_t launch_eval_items(const WorkItem *items, int n_items, const LigDev *ligs,
                              const RecDev *recs, int *counter, const EvalCfg &cfg, int budget,
                              int grid, cudaStream_t s) {
    if (cfg.paired)
        return launch_eval_pair_items(items, n_items, ligs, recs, counter, cfg, budget, grid, s);
    ItemsArgs a;
    a.items = items;
    a.ligs = ligs;
    a.recs = recs;
    a.counter = counter;
    a.n_items = n_items;
    a.ppb = cfg.ppb;
    a.budget = budget;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int smem = eval_smem_bytes(budget, cfg, dev, true);
    if (smem < 0) return cudaErrorInvalidValue;
    switch (cfg.tpp) {
        case 32: return launch_items_v<32>(a, cfg.variant, smem, grid, s);
        case 64: return launch_items_v<64>(a, cfg.variant, smem, grid, s);
        case 128: return launch_items_v<128>(a, cfg.variant, smem, grid, s);
    }
    return cudaErrorInvalidValue;
}

// Blocks an SM holds at once, from the kernel's registers and static shared
// memory and the device's limits (registers allocated per warp in units of
// 256), and for the tcgen05 variant the 512 TMEM columns.  Used for that
// variant's persistent launches: for those kernels the runtime's occupancy
// query was measured to report one block an SM, although the launch holds
// as many as registers and shared memory allow (ncu: 5 for 96 registers).
static int resident_blocks(const cudaFuncAttributes &fa, const cudaDeviceProp &prop,
                           const EvalCfg &cfg, int smem) {
    const int threads = cfg.tpp * cfg.ppb, warps = (threads + 31) / 32;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    int n = regs_warp > 0 ? prop.regsPerMultiprocessor / (regs_warp * warps) : 32;
    const int smem_block = (int)fa.sharedSizeBytes + smem + (int)prop.reservedSharedMemPerBlock;
    n = std::min(n, (int)prop.sharedMemPerMultiprocessor / std::max(smem_block, 1));
    n = std::min(n, prop.maxThreadsPerMultiProcessor / (warps * 32));
    n = std::min(n, prop.maxBlocksPerMultiProcessor);
    if (cfg.variant == ADGB_REDUCE_TCGEN05) n = std::min(n, 512 / tc_ncols(warps));
    return n;
}

// Resident blocks of the persistent launch: SMs x blocks an SM can hold.
int items_grid(const EvalCfg &cfg, int budget, int device) {
    if (cfg.paired) return pair_items_grid(cfg, budget, device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return 0;
    int per_sm = 0;
    const int smem = eval_smem_bytes(budget, cfg, device, true);
    if (smem < 0) return 0;
    cudaError_t e = cudaErrorInvalidValue;
#define ADGB_OCC(TPP, VAR)                                                                   \
    if (cfg.tpp == TPP && cfg.variant == VAR) {                                              \
        e = cudaFuncSetAttribute(eval_items_kernel<TPP, VAR>,                                \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);         \
        if (e == cudaSuccess && VAR == ADGB_REDUCE_TCGEN05) {                                \
            cudaFuncAttributes fa;                                                           \
            e = cudaFuncGetAttributes(&fa, eval_items_kernel<TPP, VAR>);                     \
            if (e == cudaSuccess) per_sm = resident_blocks(fa, prop, cfg, smem);             \
        } else if (e == cudaSuccess) {                                                       \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                               \
                &per_sm, eval_items_kernel<TPP, VAR>, TPP * cfg.ppb, smem);                  \
        }                                                                                    \
    }
    ADGB_OCC(32, 0) ADGB_OCC(32, 1) ADGB_OCC(32, 2) ADGB_OCC(32, 3)
    ADGB_OCC(64, 0) ADGB_OCC(64, 1) ADGB_OCC(64, 2) ADGB_OCC(64, 3)
    ADGB_OCC(128, 0) ADGB_OCC(128, 1) ADGB_OCC(128, 2) ADGB_OCC(128, 3)
#undef ADGB_OCC
    if (e != cudaSuccess || per_sm < 1) return 0;
    return per_sm * prop.multiProcessorCount;
}

// A genotype that fits one gene a lane runs the kernel built for that
// (fewer live registers); larger ones the general kernel.
template <int TPP, int VAR>
static cudaError_t launch_t(const EvalArgs &a, int ppb, int smem, cudaStream_t s) {
    constexpr int NG_MAX = (MAX_GENES + TPP - 1) / TPP;
    auto k = (NG_MAX > 1 && 6 + a.lig.n_tors <= TPP) ? eval_kernel<TPP, VAR, 1>
                                                      : eval_kernel<TPP, VAR, NG_MAX>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int blocks = (a.n + ppb - 1) / ppb;
    k<<<blocks, TPP * ppb, smem, s>>>(a);
    return cudaGetLastError();
}

template <int TPP>
static cudaError_t launch_v(const EvalArgs &a, int ppb, int variant, int smem, cudaStream_t s) {
    switch (variant) {
        case ADGB_REDUCE_SHFL: return launch_t<TPP, ADGB_REDUCE_SHFL>(a, ppb, smem, s);
        case ADGB_REDUCE_MMA_TF32X2:
            return launch_t<TPP, ADGB_REDUCE_MMA_TF32X2>(a, ppb, smem, s);
        case ADGB_REDUCE_MMA_BF16X3:
            return launch_t<TPP, ADGB_REDUCE_MMA_BF16X3>(a, ppb, smem, s);
        case ADGB_REDUCE_TCGEN05: return launch_t<TPP, ADGB_REDUCE_TCGEN05>(a, ppb, smem, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_eval(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg, int mode,
                        const float *genes_in, float *genes_out, int n, int iters, float rho,
                        float eps, int resume, float *energy, float *grad, float *state,
                        cudaStream_t s, const int *iters_per_pose) {
    if (n == 0) return cudaSuccess;
    if (cfg.paired &&
        pair_eligible(lig.n_atoms, lig.n_tors, lig.n_pairs, lig.n_rounds, lig.r_lanes, cfg.tpp))
        return launch_eval_pair(rec, lig, cfg, mode, genes_in, genes_out, n, iters, rho, eps,
                                resume, energy, grad, state, s, iters_per_pose);
    EvalArgs a;
    a.iters_pp = iters_per_pose;
    a.rec = rec;
    a.lig = lig;
    a.L.make(lig.n_atoms, lig.n_tors, cfg.ppb, cfg.tpp / 32, cfg.chunk, lig.n_pairs,
             cfg.stage_pairs != 0, uses_mma_stage(cfg.variant));
    a.genes_in = genes_in;
    a.genes_out = genes_out;
    a.energy = energy;
    a.grad = grad;
    a.state = state;
    a.n = n;
    a.iters = iters;
    a.resume = resume;
    a.mode = mode;
    a.rho = rho;
    a.eps = eps;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int smem = eval_smem_bytes(a.L.total, cfg, dev, false);
    if (smem < 0) return cudaErrorInvalidValue;
    switch (cfg.tpp) {
        case 32: return launch_v<32>(a, cfg.ppb, cfg.variant, smem, s);
        case 64: return launch_v<64>(a, cfg.ppb, cfg.variant, smem, s);
        case 128: return launch_v<128>(a, cfg.ppb, cfg.variant, smem, s);
    }
    return cudaErrorInvalidValue;
}

template <int TPP, int VAR>
static cudaError_t launch_sw_t(const SwArgs &a, int ppb, int smem, cudaStream_t s) {
    auto k = sw_kernel<TPP, VAR>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<(a.n + ppb - 1) / ppb, TPP * ppb, smem, s>>>(a);
    return cudaGetLastError();
}

template <int TPP>
static cudaError_t launch_sw_v(const SwArgs &a, int ppb, int variant, int smem, cudaStream_t s) {
    switch (variant) {
        case ADGB_REDUCE_SHFL: return launch_sw_t<TPP, ADGB_REDUCE_SHFL>(a, ppb, smem, s);
        case ADGB_REDUCE_MMA_TF32X2: return launch_sw_t<TPP, ADGB_REDUCE_MMA_TF32X2>(a, ppb, smem, s);
        case ADGB_REDUCE_MMA_BF16X3: return launch_sw_t<TPP, ADGB_REDUCE_MMA_BF16X3>(a, ppb, smem, s);
        case ADGB_REDUCE_TCGEN05: return launch_sw_t<TPP, ADGB_REDUCE_TCGEN05>(a, ppb, smem, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sw(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg, const SwCfg &c,
                      float *genes, int n, float *energy, int *evals, float *state, cudaStream_t s,
                      const int *budget) {
    if (n == 0) return cudaSuccess;
    SwArgs a;
    a.rec = rec;
    a.lig = lig;
    a.L.make(lig.n_atoms, lig.n_tors, cfg.ppb, cfg.tpp / 32, cfg.chunk, lig.n_pairs,
             cfg.stage_pairs != 0, uses_mma_stage(cfg.variant));
    a.genes = genes;
    a.energy = energy;
    a.evals = evals;
    a.state = state;
    a.budget = budget;
    a.n = n;
    a.max_evals = c.max_evals;
    a.max_succ = c.max_succ;
    a.max_fail = c.max_fail;
    a.resume = c.resume;
    a.rho0 = c.rho0;
    a.rho_min = c.rho_min;
    a.angle_scale = c.angle_scale;
    a.seed = c.seed;
    a.call = c.call;
    a.pose_base = c.pose_base;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int smem = eval_smem_bytes(a.L.total, cfg, dev, false);
    if (smem < 0) return cudaErrorInvalidValue;
    switch (cfg.tpp) {
        case 32: return launch_sw_v<32>(a, cfg.ppb, cfg.variant, smem, s);
        case 64: return launch_sw_v<64>(a, cfg.ppb, cfg.variant, smem, s);
        case 128: return launch_sw_v<128>(a, cfg.ppb, cfg.variant, smem, s);
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ pose -> coords
// One block per genotype: coordinates only, written in the caller's atom order.
__global__ void __launch_bounds__(128) coords_kernel(const LigDev lig, const float *genes,
                                                     int n, float *out) {
    __shared__ float2 sc[ADGB_MAX_TORS + 3];
    const int pose = blockIdx.x;
    const int N = lig.n_atoms, T = lig.n_tors, G = 6 + T;
    const float *gp = genes + (size_t)pose * G;
    for (int j = threadIdx.x; j < G; j += blockDim.x) {
        if (j == 3 || j == 4) {
            float s, c;
            sincosf(gp[j], &s, &c);
            sc[SC_ROT + j - 3] = make_float2(s, c);
        } else if (j >= 5) {
            float sh, ch;
            sincosf(0.5f * gp[j], &sh, &ch);
            const float2 v = make_float2(2.f * sh * ch, 2.f * sh * sh);
            if (j == 5) sc[SC_ROT + 2] = v;
            else sc[j - 6] = v;
        }
    }
    __syncthreads();
    const float2 sphi = sc[SC_ROT], sth = sc[SC_ROT + 1], sal = sc[SC_ROT + 2];
    const float3 u = make_float3(sth.x * sphi.y, sth.x * sphi.x, sth.y);
    const float s = sal.x, o = sal.y;
    const float m00 = o * (u.x * u.x - 1.f), m11 = o * (u.y * u.y - 1.f), m22 = o * (u.z * u.z - 1.f);
    const float m01 = o * u.x * u.y - s * u.z, m10 = o * u.x * u.y + s * u.z;
    const float m02 = o * u.x * u.z + s * u.y, m20 = o * u.x * u.z - s * u.y;
    const float m12 = o * u.y * u.z - s * u.x, m21 = o * u.y * u.z + s * u.x;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float4 r4 = lig.ref[i];
        float3 p = make_float3(r4.x, r4.y, r4.z);
        for (int k = lig.frag[i]; k >= 0; k = lig.tparent[k])
            rotate_about(p, lig.taxis[k], lig.tbref[k], sc[k]);
        float *o3 = out + ((size_t)pose * N + lig.perm[i]) * 3;
        o3[0] = p.x + (m00 * p.x + m01 * p.y + m02 * p.z) + gp[0];
        o3[1] = p.y + (m10 * p.x + m11 * p.y + m12 * p.z) + gp[1];
        o3[2] = p.z + (m20 * p.x + m21 * p.y + m22 * p.z) + gp[2];
    }
}

cudaError_t launch_coords(const LigDev &lig, const float *genes, int n, float *xyz,
                          cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    coords_kernel<<<n, 128, 0, s>>>(lig, genes, n, xyz);
    return cudaGetLastError();
}

// ------------------------------------------------------------- grid packing
// cells[cell][m][c] <- maps[m][z+cz][y+cy][x+cx], c = cx + 2 cy + 4 cz.
__global__ void pack_grid_kernel(const float *maps, int nx, int ny, int nz, int M,
                                 float *cells) {
    const long ncell = (long)(nx - 1) * (ny - 1) * (nz - 1);
    const long total = ncell * M;
    for (long w = blockIdx.x * (long)blockDim.x + threadIdx.x; w < total;
         w += (long)gridDim.x * blockDim.x) {
        const long cell = w / M;
        const int m = (int)(w - cell * M);
        const int ix = (int)(cell % (nx - 1));
        const int iy = (int)((cell / (nx - 1)) % (ny - 1));
        const int iz = (int)(cell / ((long)(nx - 1) * (ny - 1)));
        const float *src = maps + (size_t)m * nx * ny * nz;
        float v[8];
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
            v[c] = src[((size_t)(iz + cz) * ny + (iy + cy)) * nx + (ix + cx)];
        }
        float4 *dst = reinterpret_cast<float4 *>(cells + (size_t)w * 8);
        dst[0] = make_float4(v[0], v[1], v[2], v[3]);
        dst[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
}

cudaError_t launch_pack_grid(const float *maps, int nx, int ny, int nz, int M, float *cells,
                             cudaStream_t s) {
    pack_grid_kernel<<<152 * 8, 256, 0, s>>>(maps, nx, ny, nz, M, cells);
    return cudaGetLastError();
}

cudaError_t tc_gave_up_async(unsigned int dst[2], cudaStream_t s) {
    cudaError_t e = cudaMemcpyFromSymbolAsync(dst, g_tc_gave_up, sizeof(unsigned int), 0,
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = pair_tc_gave_up_async(dst + 1, s);
    return e;
}

}  // namespace adgb
