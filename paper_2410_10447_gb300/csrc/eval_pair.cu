// Fused scoring / ADADELTA local search with two genotypes a warp, for
// ligands of at most 32 atoms (Sec. 2.1, Sec. 3; Table 1's
// gpu_gradient_minAD).  Lane a owns internal atom a in both genotypes; every
// FP32 operation of the evaluation runs as one packed FP32x2 instruction
// (genotype A in .x, B in .y: two IEEE round-to-nearest results, so each
// genotype's arithmetic is the same whichever genotype shares its warp), and
// the ligand's round words, pair constants, torsion tree and address
// arithmetic are read and computed once for both.
//
// Per evaluation (no block barrier; __syncwarp only):
//   1. gene lanes publish both genotypes' genes and sin / (1 - cos) of every
//      angle;
//   2. each lane moves its atom (torsions deepest-first about reference axes,
//      rotation, translation) in both genotypes and interpolates its grid
//      terms (two cells: one per genotype);
//   3. intramolecular pairs in matching rounds: the partner's positions by
//      shuffles, one pair term for both genotypes with the same constants,
//      the reaction forces of (at most two) pairs by shuffles;
//   4. per-lane partials of (E, g, (x - t) x g);
//   5. reduce-and-broadcast (Sec. 3, 4.2) of the partials and the torsions'
//      segmented sums over their moving atoms:
//        shuffle / mma.sync: warp reduce-scatter of the 16 partials, each gene
//          lane fetching the totals it needs; torsion lanes sum their moving
//          range from a shared-memory copy of the partials;
//        tcgen05: ONE tensor-core product D = P . B^T a warp, B = the 32 lanes'
//          partials of both genotypes (TF32 hi and lo terms, K = the lanes),
//          P the ligand's 0/1 matrix whose row 6 + k is torsion k's moving-atom
//          mask and every other row all ones: lane j reads row j of D from
//          tensor memory, i.e. the totals (translation and rotation genes) or
//          its torsion's moving-set sums (torsion genes) - the block reduction
//          and the segmented torsion reduction in one MMA;
//   6. gene gradient, best tracking and ADADELTA by the gene lanes.
#include <math.h>

#include "adgb_internal.cuh"
#include "reduce.cuh"
#include "tcgen05.cuh"

namespace adgb {

namespace {

constexpr float P_INV_SIG2 = 1.0f / (ADGB_DS_SIGMA * ADGB_DS_SIGMA);
constexpr float P_HALF_INV_SIG2 = 0.5f / (ADGB_DS_SIGMA * ADGB_DS_SIGMA);
constexpr float P_RMIN2 = ADGB_R_MIN * ADGB_R_MIN;
constexpr float P_PI = 3.14159265358979f;
constexpr int P_ROT = ADGB_MAX_TORS;   // sc slots after the torsions: phi, theta, alpha
constexpr unsigned FULL = 0xffffffffu;

// Steps a measurement-only launch leaves out (ls_ablation_dev): the time a
// step takes is the difference to the whole evaluation.  0 in every
// production launch.
enum {
    SK_PAIRS = 1,    // the pair rounds
    SK_GRID = 2,     // the grid terms (copies and interpolation)
    SK_RED = 4,      // the reduce-and-broadcast (the lane's own partials instead)
    SK_TORS = 8,     // the torsions' moving-set sums (shuffle and mma.sync forms)
    SK_WALK = 16,    // the torsion-tree walk of the coordinates
    SK_GENE = 32,    // the gene-gradient formulas
    SK_SINCOS = 64,  // the sines and cosines of the angles (zero angles instead)
    SK_PAIRMATH = 128,  // the pair terms' arithmetic (the exchanges kept)
    SK_PAIRXCHG = 256,  // the pair rounds' shuffles (the arithmetic kept)
    // not a step left out but the other tensor-core design, measured through
    // the same entry: ONE MMA a block (N = 32 x warps, after a block barrier)
    // instead of one a warp; needs full blocks and equal iteration counts
    SK_BLOCKMMA = 512,
    // test form of the tcgen05 variant: the MMAs are not issued, so the first
    // completion wait of every warp gives up after a short limit (the failure
    // path: NaN sums, the give-up count, TMEM still freed)
    SK_NOISSUE = 1024,
};
constexpr int TC2_TEST_LIMIT = 64;   // mbarrier probes of SK_NOISSUE's waits

// ------------------------------------------------------- packed FP32x2
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc(-1.f), a); }

struct V2 {   // a 3-vector of both genotypes
    float2 x, y, z;
};

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(FULL, v.x, src), __shfl_sync(FULL, v.y, src));
}

// a x b of both genotypes
__device__ __forceinline__ V2 cross2(const V2 &a, const V2 &b) {
    V2 c;
    c.x = fma2(a.y, b.z, mul2(bc(-1.f), mul2(a.z, b.y)));
    c.y = fma2(a.z, b.x, mul2(bc(-1.f), mul2(a.x, b.z)));
    c.z = fma2(a.x, b.y, mul2(bc(-1.f), mul2(a.y, b.x)));
    return c;
}
__device__ __forceinline__ float2 dot2(const V2 &a, const V2 &b) {
    return fma2(a.z, b.z, fma2(a.y, b.y, mul2(a.x, b.x)));
}

// p += s (k x v) + omc (k x (k x v)), v = p - b, for both genotypes: the
// axis k and point b are the ligand's (shared), c = (s_A, omc_A, s_B, omc_B).
// Exact at zero angles.
__device__ __forceinline__ void rotate2(V2 &p, float4 k, float4 b, float4 c) {
    const V2 v = {sub2(p.x, bc(b.x)), sub2(p.y, bc(b.y)), sub2(p.z, bc(b.z))};
    V2 kv, kkv;
    kv.x = fma2(bc(k.y), v.z, mul2(bc(-k.z), v.y));
    kv.y = fma2(bc(k.z), v.x, mul2(bc(-k.x), v.z));
    kv.z = fma2(bc(k.x), v.y, mul2(bc(-k.y), v.x));
    kkv.x = fma2(bc(k.y), kv.z, mul2(bc(-k.z), kv.y));
    kkv.y = fma2(bc(k.z), kv.x, mul2(bc(-k.x), kv.z));
    kkv.z = fma2(bc(k.x), kv.y, mul2(bc(-k.y), kv.x));
    const float2 s = make_float2(c.x, c.z), o = make_float2(c.y, c.w);
    p.x = fma2(s, kv.x, fma2(o, kkv.x, p.x));
    p.y = fma2(s, kv.y, fma2(o, kkv.y, p.y));
    p.z = fma2(s, kv.z, fma2(o, kkv.z, p.z));
}

// Intermolecular term of one atom in one genotype: the point clamped onto
// the grid, its cell's corners of the type map and of the e and d maps
// (cell-major corner-packed: three 32-byte runs) loaded, map + q e + |q| d
// interpolated trilinearly with its gradient, plus W_OUT times the squared
// distance outside the grid.
struct GridAt {
    float f0, f1, f2;   // position inside the cell (fractions)
    float o0, o1, o2;   // distance outside the grid per axis (0 inside)
};

// Trilinear value and gradient of map + q e + |q| d from the cell's corners
// (t0/t1 type map, e0/e1 e map, d0/d1 d map; corner c = cx + 2 cy + 4 cz),
// plus the out-of-grid penalty.
__device__ __forceinline__ float grid_interp(const RecDev &R, float q, const GridAt &a, float4 t0,
                                             float4 t1, float4 e0, float4 e1, float4 d0,
                                             float4 d1, float &g0, float &g1, float &g2) {
    // corner weights, two adjacent corners an instruction
    const float2 aq = bc(fabsf(q)), qq = bc(q);
    const float2 w01 = fma2(aq, make_float2(d0.x, d0.y), fma2(qq, make_float2(e0.x, e0.y), make_float2(t0.x, t0.y)));
    const float2 w23 = fma2(aq, make_float2(d0.z, d0.w), fma2(qq, make_float2(e0.z, e0.w), make_float2(t0.z, t0.w)));
    const float2 w45 = fma2(aq, make_float2(d1.x, d1.y), fma2(qq, make_float2(e1.x, e1.y), make_float2(t1.x, t1.y)));
    const float2 w67 = fma2(aq, make_float2(d1.z, d1.w), fma2(qq, make_float2(e1.z, e1.w), make_float2(t1.z, t1.w)));
    const float fx = a.f0, fy = a.f1, fz = a.f2;
    const float x00 = w01.y - w01.x, x10 = w23.y - w23.x, x01 = w45.y - w45.x, x11 = w67.y - w67.x;
    const float c00 = w01.x + fx * x00, c10 = w23.x + fx * x10;
    const float c01 = w45.x + fx * x01, c11 = w67.x + fx * x11;
    const float y0 = c10 - c00, y1 = c11 - c01;
    const float c0 = c00 + fy * y0, c1 = c01 + fy * y1;
    const float val = c0 + fz * (c1 - c0);
    const float dx0 = x00 + fy * (x10 - x00), dx1 = x01 + fy * (x11 - x01);
    const float dfx = dx0 + fz * (dx1 - dx0);
    const float dfy = y0 + fz * (y1 - y0);
    const float dfz = c1 - c0;
    g0 = (a.o0 == 0.f ? dfx * R.inv_h : 0.f) + 2.f * ADGB_W_OUT * a.o0;
    g1 = (a.o1 == 0.f ? dfy * R.inv_h : 0.f) + 2.f * ADGB_W_OUT * a.o1;
    g2 = (a.o2 == 0.f ? dfz * R.inv_h : 0.f) + 2.f * ADGB_W_OUT * a.o2;
    const float pen = a.o0 * a.o0 + a.o1 * a.o1 + a.o2 * a.o2;
    return val + ADGB_W_OUT * pen;
}

// The atom's cell and corners, loaded into registers.
__device__ __forceinline__ float grid_direct(const RecDev &R, int t, float q, float x0, float x1,
                                             float x2, float &g0, float &g1, float &g2) {
    const float xs[3] = {x0, x1, x2};
    const int n[3] = {R.nx, R.ny, R.nz};
    float f[3], o[3];
    int i0[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float xc = fminf(fmaxf(xs[d], R.lo[d]), R.hi[d]);
        o[d] = xs[d] - xc;
        const float u = (xc - R.lo[d]) * R.inv_h;
        int k = (int)u;   // u >= 0
        k = k > n[d] - 2 ? n[d] - 2 : k;
        i0[d] = k;
        f[d] = u - (float)k;
    }
    const size_t cell = ((size_t)i0[2] * (R.ny - 1) + i0[1]) * (R.nx - 1) + i0[0];
    const float4 *cp = reinterpret_cast<const float4 *>(R.cells + cell * (size_t)R.M * 8);
    const GridAt a{f[0], f[1], f[2], o[0], o[1], o[2]};
    return grid_interp(R, q, a, __ldg(cp + 2 * t), __ldg(cp + 2 * t + 1), __ldg(cp + 2 * (R.M - 2)),
                       __ldg(cp + 2 * (R.M - 2) + 1), __ldg(cp + 2 * (R.M - 1)),
                       __ldg(cp + 2 * (R.M - 1) + 1), g0, g1, g2);
}

// 2^x by the special-function unit (the exponentials of the pair terms take
// log2(e) folded into their constants).
__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float P_LOG2E = 1.4426950408889634f;

// One intramolecular pair in both genotypes (the same pair constants
// pc = (A, B, w_el 332.06 q_i q_j, w_ds (S_i V_j + S_j V_i)) and H-bond flag):
// A r^-12 - B r^-m (m = 10 for donor-acceptor pairs, else 6) with r clamped
// at R_MIN (no force below), Coulomb over the Mehler-Solmajer dielectric
// (one reciprocal: 1/eps = den^2 rr r, eps'/eps = B k lambda B e rr), and the
// desolvation Gaussian.  d = x_i - x_j; returns both energies, f = dE/dx_i.
__device__ __forceinline__ float2 pair_both(const V2 &d, float4 pc, bool hb, V2 &f) {
    const float2 r2 = fma2(d.z, d.z, fma2(d.y, d.y, mul2(d.x, d.x)));
    const bool la = r2.x >= P_RMIN2, lb = r2.y >= P_RMIN2;
    const float2 r2c = make_float2(fmaxf(r2.x, P_RMIN2), fmaxf(r2.y, P_RMIN2));
    const float2 rinv = make_float2(rsqrtf(r2c.x), rsqrtf(r2c.y));
    const float2 rc = mul2(r2c, rinv);
    const float2 r2i = mul2(rinv, rinv);
    const float2 r4i = mul2(r2i, r2i);
    const float2 r6i = mul2(r4i, r2i);
    const float2 r12i = mul2(r6i, r6i);
    const float2 rmi = hb ? mul2(r6i, r4i) : r6i;
    const float2 t12 = mul2(bc(pc.x), r12i), tm = mul2(bc(pc.y), rmi);
    const float2 evdw = fma2(tm, bc(-1.f), t12);
    const float2 dvdw = mul2(fma2(bc(hb ? 10.f : 6.f), tm, mul2(bc(-12.f), t12)), rinv);
    const float2 xe = mul2(bc(-MS_LAMBDA * MS_B * P_LOG2E), rc);
    const float2 ex = make_float2(ex2a(xe.x), ex2a(xe.y));
    const float2 den = fma2(bc(MS_K), ex, bc(1.f));
    const float2 num = fma2(bc(MS_A), den, bc(MS_B));
    const float2 dn = mul2(den, num);
    const float2 rr = make_float2(__fdividef(1.f, dn.x), __fdividef(1.f, dn.y));
    const float2 eel = mul2(mul2(bc(pc.z), rinv), mul2(mul2(den, den), rr));
    const float2 del = mul2(mul2(eel, bc(-1.f)),
                            fma2(bc(MS_B * MS_K * MS_LAMBDA * MS_B), mul2(ex, rr), rinv));
    const float2 xd = mul2(r2, bc(-P_HALF_INV_SIG2 * P_LOG2E));
    const float2 eds = mul2(bc(pc.w), make_float2(ex2a(xd.x), ex2a(xd.y)));
    const float2 frr = mul2(add2(dvdw, del), rinv);
    const float2 ft = fma2(eds, bc(-P_INV_SIG2), make_float2(la ? frr.x : 0.f, lb ? frr.y : 0.f));
    f.x = mul2(ft, d.x);
    f.y = mul2(ft, d.y);
    f.z = mul2(ft, d.z);
    return add2(add2(evdw, eel), eds);
}

// ------------------------------------------------ tcgen05 (paired form)
// Region at the front of the (1024-byte aligned) dynamic shared memory:
// the block's P operand (128 x 32 TF32, 128-byte-swizzled K-major: rows
// 32 q + l, q = 0..3, all hold the ligand's 32-row pattern, so that every
// warp reads its rows from its own tensor-memory lane quadrant) at
// [0, 16384), one 4 KB B operand a warp (32 rows: (genotype, hi/lo, 8
// components), K = the 32 lanes) from 16384, then one mbarrier a warp and the
// tensor-memory base address.
constexpr int TC2_A = 0, TC2_B = 16384;
__host__ __device__ constexpr int tc2_mbar(int warps) { return TC2_B + 4096 * warps; }
__host__ __device__ constexpr int tc2_region(int warps) { return tc2_mbar(warps) + 64; }
__host__ __device__ constexpr int tc2_ncols(int warps) {   // 32 D columns a warp
    return warps <= 1 ? 32 : (warps <= 2 ? 64 : 128);
}

struct Tc2 {
    unsigned char *b;   // this warp's B operand (generic address)
    uint64_t *mbar;     // completion barrier of this warp's MMAs
    uint32_t a_s, b_s;  // shared-window addresses of P and of this warp's B
    uint32_t d_col;     // TMEM address of this warp's D columns (lane 0)
    uint32_t d_lane;    // the same columns in this warp's lane quadrant
    uint32_t taddr, ncols, phase;
    int ok;             // 0 once a completion wait gave up (sums NaN)
};

// Allocates the block's tensor memory and its mbarriers (all threads; block
// barriers inside).
__device__ __forceinline__ void tc2_begin(unsigned char *R, Tc2 &t) {
    const int w = threadIdx.x >> 5, W = blockDim.x >> 5;
    uint64_t *mb = reinterpret_cast<uint64_t *>(R + tc2_mbar(W));
    uint32_t *slot = reinterpret_cast<uint32_t *>(R + tc2_mbar(W) + 32);
    const uint32_t ncols = tc2_ncols(W);
    if (w == 0) {
        tc05::alloc(slot, ncols);
        tc05::relinquish();
    }
    if ((int)threadIdx.x < W) tc05::mbar_init(mb + threadIdx.x, 1);
    tc05::fence_before();
    __syncthreads();
    tc05::fence_after();
    const uint32_t rs = tc05::smem_u32(R);
    t.taddr = *slot;
    t.ncols = ncols;
    t.a_s = rs + TC2_A;
    t.b_s = rs + TC2_B + 4096u * w;
    t.b = R + TC2_B + 4096 * w;
    t.mbar = mb + w;
    t.d_col = t.taddr + 32u * w;
    t.d_lane = tc05::lane_addr(t.taddr, w & 3, 32 * w);
    t.phase = 0;
    t.ok = (rs & 1023u) == 0;   // swizzled atoms need 1024-byte alignment
}

// Writes the P operand of a ligand (all threads of the block; the caller
// synchronises the block before the first MMA).  Row l of the pattern is
// torsion l - 6's moving-atom mask for 6 <= l < 6 + T (its atoms are one
// contiguous internal range [start, end)), all ones otherwise.
__device__ __forceinline__ void tc2_write_pattern(unsigned char *R, const int4 *tatoms, int T) {
    uint32_t *a = reinterpret_cast<uint32_t *>(R + TC2_A);
    for (int idx = threadIdx.x; idx < 128 * 32; idx += blockDim.x) {
        const int m = idx >> 5, k = idx & 31, l = m & 31, r = m & 7;
        bool one = true;
        if (l >= 6 && l < 6 + T) {
            const int4 ta = tatoms[l - 6];
            one = k >= ta.z && k < ta.w;
        }
        a[((m >> 3) * 1024 + r * 128 + (((k >> 2) ^ r) << 4) + (k & 3) * 4) >> 2] =
            one ? 0x3F800000u : 0u;
    }
    tc05::fence_proxy_async_smem();
}

// Stages the lane's 16 partials (8 a genotype) as TF32 hi and lo terms into
// this warp's B operand and has one lane issue D = P . B^T (M = 128, N = 32,
// K = 32 lanes in four K = 8 MMAs) committed to the warp's mbarrier.  BLK
// (measurement form): after a block barrier that every warp takes each
// evaluation (also after a failed wait), thread 0 issues one product over
// all warps' B operands (contiguous: N = 32 x warps) into the same D
// columns, committed to warp 0's mbarrier, which every warp then waits on.
template <bool BLK = false, bool ISSUE = true>
__device__ __forceinline__ void tc2_issue(const float2 v[8], Tc2 &t) {
    if (!BLK && !t.ok) return;
    const int lane = threadIdx.x & 31, cq = lane >> 2;
    if (t.ok) {
        unsigned char *mine = t.b + (lane & 3) * 4;
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const uint32_t ha = to_tf32(v[c].x), hb = to_tf32(v[c].y);
            const uint32_t la = to_tf32(v[c].x - __uint_as_float(ha));
            const uint32_t lb = to_tf32(v[c].y - __uint_as_float(hb));
            const int off = c * 128 + ((cq ^ c) << 4);
            *reinterpret_cast<uint32_t *>(mine + off) = ha;          // row c
            *reinterpret_cast<uint32_t *>(mine + 1024 + off) = la;   // row 8 + c
            *reinterpret_cast<uint32_t *>(mine + 2048 + off) = hb;   // row 16 + c
            *reinterpret_cast<uint32_t *>(mine + 3072 + off) = lb;   // row 24 + c
        }
        tc05::fence_proxy_async_smem();
    }
    tc05::fence_before();
    if constexpr (BLK) {
        asm volatile("bar.sync 1, %0;" ::"r"(blockDim.x) : "memory");
    } else {
        __syncwarp();
    }
    if (ISSUE && (BLK ? (threadIdx.x == 0 && t.ok) : lane == 0)) {
        tc05::fence_after();
        const uint32_t idesc = tc05::idesc_tf32(128, BLK ? 32 * (blockDim.x >> 5) : 32);
#pragma unroll
        for (int s = 0; s < 4; s++)
            tc05::mma_tf32_ss(t.d_col, tc05::desc_sw128(t.a_s + 32u * s, 1024),
                              tc05::desc_sw128(t.b_s + 32u * s, 1024), idesc, s > 0);
        tc05::commit(t.mbar);
    }
}

__device__ __forceinline__ void ld32_wait(uint32_t taddr, float v[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Waits (bounded) for the warp's MMAs and reads row `lane` of D: s[c] = the
// pattern row's sums of component c for both genotypes.  A wait that gives
// up makes the sums NaN from then on (tc2_end counts it).
template <int LIMIT = TC05_WAIT_LIMIT>
__device__ __forceinline__ void tc2_finish(float2 s[8], Tc2 &t) {
    if (t.ok) {
        const bool done = __all_sync(FULL, tc05::mbar_wait(t.mbar, t.phase & 1, LIMIT));
        t.phase++;
        if (done) {
            tc05::fence_after();
            float d[32];
            ld32_wait(t.d_lane, d);
#pragma unroll
            for (int c = 0; c < 8; c++) s[c] = make_float2(d[c] + d[8 + c], d[16 + c] + d[24 + c]);
            tc05::fence_before();   // these reads precede the warp's next MMA
            return;
        }
        t.ok = 0;
    }
#pragma unroll
    for (int c = 0; c < 8; c++) s[c] = bc(__int_as_float(0x7fc00000));
}

// Releases the block's tensor memory once every warp's MMAs are complete;
// counts a warp whose waits gave up (or that never had a usable operand
// region) in the module's give-up count.
template <int LIMIT = TC05_WAIT_LIMIT>
__device__ __forceinline__ void tc2_end(Tc2 &t) {
    if (!t.ok && t.phase > 0) (void)tc05::mbar_wait(t.mbar, (t.phase - 1) & 1, LIMIT);
    if (!t.ok && (threadIdx.x & 31) == 0) atomicAdd(&g_tc_gave_up, 1u);
    tc05::fence_before();
    __syncthreads();
    tc05::fence_after();
    if ((threadIdx.x >> 5) == 0) tc05::dealloc(t.taddr, t.ncols);
}

// ------------------------------------------------- shuffle reductions
// Reduce-scatter of 16 values (8 a genotype) by recursive halving over the
// lane bits 4..1, then one butterfly: value m ends in lanes whose bits 4..1
// are m's bits 3..0, i.e. in lane 2m and 2m + 1.  Every value is summed along
// the same tree (only the operand order of some additions differs), so a
// genotype's totals do not depend on which half of the warp's pair it is.
__device__ __forceinline__ float reduce_scatter16(float v[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int lv = 0; lv < 4; lv++) {
        const int h = 8 >> lv, m = 16 >> lv;
        const bool up = lane & m;
#pragma unroll
        for (int k = 0; k < h; k++) {
            const float send = up ? v[k] : v[k + h];
            const float keep = up ? v[k + h] : v[k];
            v[k] = keep + __shfl_xor_sync(FULL, send, m);
        }
    }
    return v[0] + __shfl_xor_sync(FULL, v[0], 1);
}
// index m of value (genotype g, component c) after the halving: the lane bits
// taken, highest first, select m's bits 3..0; the upper half keeps the upper
// values, so m = 8 g + c with the genotype the highest bit.
__device__ __forceinline__ int holder(int g, int c) { return 2 * (8 * g + c); }

// Per-launch arguments.
struct PairArgs {
    RecDev rec;
    LigDev lig;
    PairSmem L;
    const float *genes_in;
    float *genes_out;
    float *energy;
    float *grad;
    float *state;
    const int *iters_pp;
    int n, iters, resume, mode, ppb;
    float rho, eps;
};

// Inputs and outputs of the warp's two genotypes (pointers at each one).
struct PairIO {
    const float *genes_in[2];
    float *genes_out[2];
    float *energy[2];
    float *grad[2];
    float *state[2];
    int iters[2];
    int nvalid;   // 1: the second genotype is a copy of the first, not written
    int mode, resume;
    float rho, eps;
};

// Copies one ligand's constants into the block's shared memory (all threads;
// the caller synchronises before the first use).
__device__ __forceinline__ void stage_pair_ligand(unsigned char *sm, const PairSmem &L,
                                                  const LigDev &lig) {
    const int N = lig.n_atoms, T = lig.n_tors;
    float4 *s_ref = reinterpret_cast<float4 *>(sm + L.ref);
    int *s_type = reinterpret_cast<int *>(sm + L.type);
    int *s_frag = reinterpret_cast<int *>(sm + L.frag);
    int *s_tpar = reinterpret_cast<int *>(sm + L.tparent);
    int4 *s_tat = reinterpret_cast<int4 *>(sm + L.tatoms);
    float4 *s_tax = reinterpret_cast<float4 *>(sm + L.taxis);
    float4 *s_tb = reinterpret_cast<float4 *>(sm + L.tbref);
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
}

// Whole evaluation loop of a warp's two genotypes.
template <int VAR, int SKIP = 0>
__device__ __forceinline__ void search_pair(unsigned char *sm, const PairSmem &L,
                                            const LigDev &lig, const RecDev &rec, const int warp,
                                            const PairIO &io, Tc2 &tw) {
    const int lane = threadIdx.x & 31;
    const int N = lig.n_atoms, T = lig.n_tors, G = 6 + T;
    const float4 *s_ref = reinterpret_cast<const float4 *>(sm + L.ref);
    const int *s_type = reinterpret_cast<const int *>(sm + L.type);
    const int *s_frag = reinterpret_cast<const int *>(sm + L.frag);
    const int *s_tpar = reinterpret_cast<const int *>(sm + L.tparent);
    const int4 *s_tat = reinterpret_cast<const int4 *>(sm + L.tatoms);
    const float4 *s_tax = reinterpret_cast<const float4 *>(sm + L.taxis);
    const float4 *s_tb = reinterpret_cast<const float4 *>(sm + L.tbref);
    unsigned char *W = sm + L.warp0 + warp * L.warp_stride;
    float4 *xyz = reinterpret_cast<float4 *>(W + L.w_xyz);      // [2 i + g]
    float2 *genes_s = reinterpret_cast<float2 *>(W + L.w_genes);
    float4 *sc = reinterpret_cast<float4 *>(W + L.w_sc);
    float *stage = reinterpret_cast<float *>(W + L.w_stage);

    // the lane's gene (j = lane) of both genotypes, and ADADELTA state
    const int j = lane;
    float2 om = bc(0.f), eg2 = bc(0.f), ed2 = bc(0.f);
    if (j < G) {
#pragma unroll
        for (int g = 0; g < 2; g++) {
            float o, a = 0.f, b = 0.f;
            if (io.resume) {
                const float *st = io.state[g];
                o = st[j];
                a = st[G + j];
                b = st[2 * G + j];
            } else {
                o = io.genes_in[g][j];
            }
            if (g == 0) {
                om.x = o; eg2.x = a; ed2.x = b;
            } else {
                om.y = o; eg2.y = a; ed2.y = b;
            }
        }
    }
    float2 best = om, best_e = bc(INFINITY);
    // the lane's atom constants
    const bool has_atom = lane < N;
    const float4 r4 = has_atom ? s_ref[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int a_type = has_atom ? s_type[lane] : 0;
    const int a_frag = has_atom ? s_frag[lane] : -1;
    // the lane's torsion (j = 6 + k): bond atoms and moving range
    const int tk = j - 6;
    const bool tors_lane = tk >= 0 && tk < T;
    const int4 ta = tors_lane ? s_tat[tk] : make_int4(0, 0, 0, 0);
    const int R = lig.n_rounds;
    const uint32_t *rw = lig.rword + lane;
    const float4 *rcs = lig.rconst + lane;
    const int iters = max(io.iters[0], io.iters[1]);

    for (int it = 0; it < iters; it++) {
        // 1. genes and sin / (1 - cos) of every angle (half-angle form: exact
        //    zero at a zero angle; phi and theta as (sin, cos) of the angle)
        {
            const bool full = j == 3 || j == 4;
            float sa, ca, sb, cb;
            if constexpr (SKIP & SK_SINCOS) {
                sa = 0.f; ca = 1.f; sb = 0.f; cb = 1.f;
            } else {
                sincosf(full ? om.x : 0.5f * om.x, &sa, &ca);
                sincosf(full ? om.y : 0.5f * om.y, &sb, &cb);
            }
            if (j < G) {
                genes_s[j] = om;
                const float4 v = full ? make_float4(sa, ca, sb, cb)
                                      : make_float4(2.f * sa * ca, 2.f * sa * sa, 2.f * sb * cb,
                                                    2.f * sb * sb);
                if (j >= 6) sc[j - 6] = v;
                else if (j >= 3) sc[P_ROT + j - 3] = v;
            }
        }
        __syncwarp();
        const V2 tr = {genes_s[0], genes_s[1], genes_s[2]};
        const float4 c_phi = sc[P_ROT], c_th = sc[P_ROT + 1], c_al = sc[P_ROT + 2];
        const float2 sphi = make_float2(c_phi.x, c_phi.z), cphi = make_float2(c_phi.y, c_phi.w);
        const float2 sth = make_float2(c_th.x, c_th.z), cth = make_float2(c_th.y, c_th.w);
        const float2 s = make_float2(c_al.x, c_al.z), o = make_float2(c_al.y, c_al.w);
        const V2 u = {mul2(sth, cphi), mul2(sth, sphi), cth};
        // R - I = sin(a) [u]x + (1 - cos(a)) (u u^T - I)
        const float2 m00 = mul2(o, fma2(u.x, u.x, bc(-1.f)));
        const float2 m11 = mul2(o, fma2(u.y, u.y, bc(-1.f)));
        const float2 m22 = mul2(o, fma2(u.z, u.z, bc(-1.f)));
        const float2 oxy = mul2(mul2(o, u.x), u.y), oxz = mul2(mul2(o, u.x), u.z);
        const float2 oyz = mul2(mul2(o, u.y), u.z);
        const float2 m01 = fma2(bc(-1.f), mul2(s, u.z), oxy), m10 = fma2(s, u.z, oxy);
        const float2 m02 = fma2(s, u.y, oxz), m20 = fma2(bc(-1.f), mul2(s, u.y), oxz);
        const float2 m12 = fma2(bc(-1.f), mul2(s, u.x), oyz), m21 = fma2(s, u.x, oyz);

        // 2. the lane's atom in both genotypes and its grid terms
        V2 xo = {bc(0.f), bc(0.f), bc(0.f)}, go = xo;
        float2 e_acc = bc(0.f);
        if (has_atom) {
            V2 p = {bc(r4.x), bc(r4.y), bc(r4.z)};
            if constexpr (!(SKIP & SK_WALK))
                for (int k = a_frag; k >= 0; k = s_tpar[k]) rotate2(p, s_tax[k], s_tb[k], sc[k]);
            xo.x = add2(add2(p.x, fma2(m02, p.z, fma2(m01, p.y, mul2(m00, p.x)))), tr.x);
            xo.y = add2(add2(p.y, fma2(m12, p.z, fma2(m11, p.y, mul2(m10, p.x)))), tr.y);
            xo.z = add2(add2(p.z, fma2(m22, p.z, fma2(m21, p.y, mul2(m20, p.x)))), tr.z);
            if constexpr (!(SKIP & SK_GRID)) {
                float ga0, ga1, ga2, gb0, gb1, gb2;
                const float ea = grid_direct(rec, a_type, r4.w, xo.x.x, xo.y.x, xo.z.x, ga0, ga1, ga2);
                const float eb = grid_direct(rec, a_type, r4.w, xo.x.y, xo.y.y, xo.z.y, gb0, gb1, gb2);
                e_acc = make_float2(ea, eb);
                go = {make_float2(ga0, gb0), make_float2(ga1, gb1), make_float2(ga2, gb2)};
            }
            xyz[2 * lane] = make_float4(xo.x.x, xo.y.x, xo.z.x, r4.w);
            xyz[2 * lane + 1] = make_float4(xo.x.y, xo.y.y, xo.z.y, r4.w);
        }

        // 3. pair terms in matching rounds, two rounds at a time as
        //    independent chains (lanes without a pair compute an exact zero:
        //    zero constants, partner = itself or atom 0); the partner's
        //    positions and the (at most two) received reaction forces by
        //    shuffles
        auto xch = [&](float2 v, int src) {
            if constexpr (SKIP & SK_PAIRXCHG) return v;
            else return shfl2(v, src);
        };
        auto settle = [&](uint32_t w, const V2 &f) {
            go.x = add2(go.x, f.x);
            go.y = add2(go.y, f.y);
            go.z = add2(go.z, f.z);
            const int s1 = (w >> 8) & 31, s2 = (w >> 16) & 31;
            const float2 m1 = bc((w >> 25) & 1 ? -1.f : 0.f), m2 = bc((w >> 26) & 1 ? -1.f : 0.f);
            go.x = fma2(m1, xch(f.x, s1), go.x);
            go.y = fma2(m1, xch(f.y, s1), go.y);
            go.z = fma2(m1, xch(f.z, s1), go.z);
            go.x = fma2(m2, xch(f.x, s2), go.x);
            go.y = fma2(m2, xch(f.y, s2), go.y);
            go.z = fma2(m2, xch(f.z, s2), go.z);
        };
        auto pterm = [&](const V2 &d, float4 pc, bool hb, V2 &f) -> float2 {
            if constexpr (SKIP & SK_PAIRMATH) {
                f = d;
                return mul2(bc(pc.x), d.x);
            } else {
                return pair_both(d, pc, hb, f);
            }
        };
        auto part = [&](float2 v, int src) {   // the partner's coordinate (or a stand-in)
            if constexpr (SKIP & SK_PAIRXCHG) return add2(v, bc(1.5f + (float)src));
            else return shfl2(v, src);
        };
        int r = (SKIP & SK_PAIRS) ? R : 0;
        auto two_rounds = [&](int r0) {
            const uint32_t wa = __ldg(rw + 32 * r0), wb = __ldg(rw + 32 * (r0 + 1));
            const float4 pa = __ldg(rcs + 32 * r0), pb = __ldg(rcs + 32 * (r0 + 1));
            const int ja = wa & 31, jb = wb & 31;
            const V2 da = {sub2(xo.x, part(xo.x, ja)), sub2(xo.y, part(xo.y, ja)),
                           sub2(xo.z, part(xo.z, ja))};
            const V2 db = {sub2(xo.x, part(xo.x, jb)), sub2(xo.y, part(xo.y, jb)),
                           sub2(xo.z, part(xo.z, jb))};
            V2 fa, fb;
            const float2 ea = pterm(da, pa, (wa >> 24) & 1, fa);
            const float2 eb = pterm(db, pb, (wb >> 24) & 1, fb);
            e_acc = add2(add2(e_acc, ea), eb);
            settle(wa, fa);
            settle(wb, fb);
        };
        // unrolled twice: four rounds' chains for the scheduler to interleave
        // (measured +1.6% shuffle, +2.8% tcgen05 form on the 32-atom ligand)
#pragma unroll 2
        for (; r + 1 < R; r += 2) two_rounds(r);
        if (r < R) {
            const uint32_t w = __ldg(rw + 32 * r);
            const float4 pc = __ldg(rcs + 32 * r);
            const int pj = w & 31;
            const V2 d = {sub2(xo.x, part(xo.x, pj)), sub2(xo.y, part(xo.y, pj)),
                          sub2(xo.z, part(xo.z, pj))};
            V2 f;
            e_acc = add2(e_acc, pterm(d, pc, (w >> 24) & 1, f));
            settle(w, f);
        }

        // 4. partials (E, g, (x - t) x g) of both genotypes
        const V2 dxt = {sub2(xo.x, tr.x), sub2(xo.y, tr.y), sub2(xo.z, tr.z)};
        const V2 tq = has_atom ? cross2(dxt, go) : V2{bc(0.f), bc(0.f), bc(0.f)};
        float2 v[8] = {e_acc, go.x, go.y, go.z, tq.x, tq.y, tq.z, bc(0.f)};

        // 5. sums the lane's gene needs: E, and (sum g, sum (x - t) x g) over
        //    all atoms (translation and rotation lanes) or over torsion
        //    j - 6's moving atoms (torsion lanes)
        float2 E;
        V2 Gs, Ts;
        if constexpr (SKIP & SK_RED) {
            E = v[0];
            Gs = {v[1], v[2], v[3]};
            Ts = {v[4], v[5], v[6]};
        } else if constexpr (VAR == ADGB_REDUCE_TCGEN05) {
            float2 S[8];
            tc2_issue<(SKIP & SK_BLOCKMMA) != 0, (SKIP & SK_NOISSUE) == 0>(v, tw);
            tc2_finish<(SKIP & SK_NOISSUE) ? TC2_TEST_LIMIT : TC05_WAIT_LIMIT>(S, tw);
            E = shfl2(S[0], 0);   // lane 0's pattern row is all ones
            Gs = {S[1], S[2], S[3]};
            Ts = {S[4], S[5], S[6]};
        } else {
            if constexpr (VAR == ADGB_REDUCE_SHFL) {
                // totals: reduce-scatter, then E and three values a lane (its
                // gradient component for j < 3, the torque otherwise)
                float t16[16];
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    t16[c] = v[c].x;
                    t16[8 + c] = v[c].y;
                }
                const float mine = reduce_scatter16(t16);
                E = make_float2(__shfl_sync(FULL, mine, holder(0, 0)),
                                __shfl_sync(FULL, mine, holder(1, 0)));
                float2 q3[3];
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    const int c = j < 3 ? 1 + j : 4 + q;
                    q3[q] = make_float2(__shfl_sync(FULL, mine, holder(0, c)),
                                        __shfl_sync(FULL, mine, holder(1, c)));
                }
                Gs = {q3[0], q3[0], q3[0]};   // lane j < 3 reads its own component
                Ts = {q3[0], q3[1], q3[2]};
            } else {
                float va[8], vb[8];
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    va[c] = v[c].x;
                    vb[c] = v[c].y;
                }
                warp_sum8<VAR>(va, stage);
                warp_sum8<VAR>(vb, stage);
                E = make_float2(va[0], vb[0]);
                Gs = {make_float2(va[1], vb[1]), make_float2(va[2], vb[2]), make_float2(va[3], vb[3])};
                Ts = {make_float2(va[4], vb[4]), make_float2(va[5], vb[5]), make_float2(va[6], vb[6])};
            }
            // torsion lanes sum their moving range [start, end) from a shared
            // copy of every lane's (g, torque) partials (12 floats a lane, in
            // the warp's staging tile)
            if constexpr (!(SKIP & SK_TORS)) {
            __syncwarp();
            {
                float4 *row = reinterpret_cast<float4 *>(stage + 12 * lane);
                row[0] = make_float4(v[1].x, v[1].y, v[2].x, v[2].y);
                row[1] = make_float4(v[3].x, v[3].y, v[4].x, v[4].y);
                row[2] = make_float4(v[5].x, v[5].y, v[6].x, v[6].y);
            }
            __syncwarp();
            if (tors_lane) {
                float2 gs[6] = {bc(0.f), bc(0.f), bc(0.f), bc(0.f), bc(0.f), bc(0.f)};
                for (int i = ta.z; i < ta.w; i++) {
                    const float4 *row = reinterpret_cast<const float4 *>(stage + 12 * i);
                    const float4 a0 = row[0], a1 = row[1], a2 = row[2];
                    gs[0] = add2(gs[0], make_float2(a0.x, a0.y));
                    gs[1] = add2(gs[1], make_float2(a0.z, a0.w));
                    gs[2] = add2(gs[2], make_float2(a1.x, a1.y));
                    gs[3] = add2(gs[3], make_float2(a1.z, a1.w));
                    gs[4] = add2(gs[4], make_float2(a2.x, a2.y));
                    gs[5] = add2(gs[5], make_float2(a2.z, a2.w));
                }
                Gs = {gs[0], gs[1], gs[2]};
                Ts = {gs[3], gs[4], gs[5]};
            }
            __syncwarp();   // the copy and the staging tile are rewritten next evaluation
            }
        }

        // 6. gene gradient, best tracking, ADADELTA
        // Every gene lane evaluates one formula, g = W . Tv, its role choosing
        // W and Tv (no divergent paths): rotation genes phi / theta take the
        // angular velocity w = sin(a) du + (1 - cos a) u x du of the axis
        // change du and the torque; alpha takes u and the torque; torsion k
        // takes the unit bond axis a -> b and sum (x - x_b) x g = sum (x - t) x g
        // - (x_b - t) x sum g over its moving atoms; translation gene j takes
        // sum g's component j.
        float2 gj;
        if constexpr (SKIP & SK_GENE) {
            gj = Gs.x;
        } else {
            const bool th = j == 4;
            V2 du;
            du.x = th ? mul2(cth, cphi) : mul2(bc(-1.f), mul2(sth, sphi));
            du.y = th ? mul2(cth, sphi) : mul2(sth, cphi);
            du.z = th ? mul2(bc(-1.f), sth) : bc(0.f);
            const V2 uxd = cross2(u, du);
            const V2 wv = {fma2(s, du.x, mul2(o, uxd.x)), fma2(s, du.y, mul2(o, uxd.y)),
                           fma2(s, du.z, mul2(o, uxd.z))};
            // the torsion lane's bond atoms (atom 0 for the other lanes)
            const int ia = tors_lane ? ta.x : 0, ib = tors_lane ? ta.y : 0;
            const float4 xa0 = xyz[2 * ia], xa1 = xyz[2 * ia + 1];
            const float4 xb0 = xyz[2 * ib], xb1 = xyz[2 * ib + 1];
            const V2 xb = {make_float2(xb0.x, xb1.x), make_float2(xb0.y, xb1.y),
                           make_float2(xb0.z, xb1.z)};
            const V2 ax = {sub2(xb.x, make_float2(xa0.x, xa1.x)), sub2(xb.y, make_float2(xa0.y, xa1.y)),
                           sub2(xb.z, make_float2(xa0.z, xa1.z))};
            const float2 l2 = dot2(ax, ax);
            const float2 il = tors_lane ? make_float2(rsqrtf(l2.x), rsqrtf(l2.y)) : bc(0.f);
            const V2 bt = {sub2(xb.x, tr.x), sub2(xb.y, tr.y), sub2(xb.z, tr.z)};
            const V2 bxg = cross2(bt, Gs);
            const V2 acc = {sub2(Ts.x, bxg.x), sub2(Ts.y, bxg.y), sub2(Ts.z, bxg.z)};
            const V2 Tv = tors_lane ? acc : Ts;
            const V2 Wv = tors_lane ? V2{mul2(ax.x, il), mul2(ax.y, il), mul2(ax.z, il)}
                                    : (j == 5 ? u : wv);
            gj = dot2(Tv, Wv);
            if (j < 3) gj = j == 0 ? Gs.x : (j == 1 ? Gs.y : Gs.z);
            if ((tors_lane && ta.w <= ta.z) || j >= G) gj = bc(0.f);
        }
        if (io.mode == MODE_SCORE) {
            if (lane == 0) {
                io.energy[0][0] = E.x;
                if (io.nvalid > 1) io.energy[1][0] = E.y;
            }
            if (j < G) {
                if (io.grad[0]) io.grad[0][j] = gj.x;
                if (io.nvalid > 1 && io.grad[1]) io.grad[1][j] = gj.y;
            }
            return;
        }
        const bool act_a = it < io.iters[0], act_b = it < io.iters[1];
        if (act_a && E.x < best_e.x) {
            best_e.x = E.x;
            best.x = om.x;
        }
        if (act_b && E.y < best_e.y) {
            best_e.y = E.y;
            best.y = om.y;
        }
        if (j < G) {
            const float2 rho = bc(io.rho), omr = bc(1.f - io.rho), ep = bc(io.eps);
            const float2 neg2 = fma2(rho, eg2, mul2(omr, mul2(gj, gj)));
            const float2 a2 = add2(ed2, ep), b2 = add2(neg2, ep);
            const float2 d = mul2(mul2(make_float2(-sqrtf(a2.x), -sqrtf(a2.y)),
                                       make_float2(rsqrtf(b2.x), rsqrtf(b2.y))), gj);
            const float2 ned2 = fma2(rho, ed2, mul2(omr, mul2(d, d)));
            float2 w = add2(om, d);
            if (j >= 6) {
                w.x -= 2.f * P_PI * floorf((w.x + P_PI) * (0.5f / P_PI));
                w.y -= 2.f * P_PI * floorf((w.y + P_PI) * (0.5f / P_PI));
            }
            if (act_a) {
                eg2.x = neg2.x;
                ed2.x = ned2.x;
                om.x = w.x;
            }
            if (act_b) {
                eg2.y = neg2.y;
                ed2.y = ned2.y;
                om.y = w.y;
            }
        }
        __syncwarp();   // genes_s, sc and xyz are rewritten next evaluation
    }
    if (io.mode == MODE_SCORE) return;
#pragma unroll
    for (int g = 0; g < 2; g++) {
        if (g >= io.nvalid) break;
        if (j < G) {
            io.genes_out[g][j] = g ? best.y : best.x;
            if (io.state[g]) {
                float *st = io.state[g];
                st[j] = g ? om.y : om.x;
                st[G + j] = g ? eg2.y : eg2.x;
                st[2 * G + j] = g ? ed2.y : ed2.x;
            }
        }
        if (lane == 0) io.energy[g][0] = g ? best_e.y : best_e.x;
    }
}

__device__ __forceinline__ PairIO pair_io(const PairArgs &a, int p0, int nvalid) {
    const int G = 6 + a.lig.n_tors;
    PairIO io;
#pragma unroll
    for (int g = 0; g < 2; g++) {
        const int p = p0 + (g < nvalid ? g : 0);
        io.genes_in[g] = a.genes_in ? a.genes_in + (size_t)p * G : nullptr;
        io.genes_out[g] = a.genes_out ? a.genes_out + (size_t)p * G : nullptr;
        io.energy[g] = a.energy + p;
        io.grad[g] = a.grad ? a.grad + (size_t)p * G : nullptr;
        io.state[g] = a.state ? a.state + (size_t)p * 3 * G : nullptr;
        io.iters[g] = a.mode == MODE_SCORE ? 1 : (a.iters_pp ? a.iters_pp[p] : a.iters);
    }
    io.nvalid = nvalid;
    io.mode = a.mode;
    io.resume = a.resume;
    io.rho = a.rho;
    io.eps = a.eps;
    return io;
}

template <int VAR, int SKIP = 0>
__global__ void __launch_bounds__(64, 5) eval_pair_kernel(const PairArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5;
    unsigned char *sm = smem_raw + (VAR == ADGB_REDUCE_TCGEN05 ? tc2_region(W) : 0);
    stage_pair_ligand(sm, a.L, a.lig);
    Tc2 tw;
    if constexpr (VAR == ADGB_REDUCE_TCGEN05) {
        tc2_write_pattern(smem_raw, a.lig.tatoms, a.lig.n_tors);
        tc2_begin(smem_raw, tw);
        if constexpr ((SKIP & SK_BLOCKMMA) != 0) tw.mbar -= warp;   // warp 0's barrier for all
    }
    __syncthreads();
    const int b0 = blockIdx.x * a.ppb;
    const int count = min(a.ppb, a.n - b0);
    const int p0 = b0 + 2 * warp, nvalid = min(2, count - 2 * warp);
    if (nvalid > 0)
        search_pair<VAR, SKIP>(sm, a.L, a.lig, a.rec, warp, pair_io(a, p0, nvalid), tw);
    if constexpr (VAR == ADGB_REDUCE_TCGEN05)
        tc2_end<(SKIP & SK_NOISSUE) ? TC2_TEST_LIMIT : TC05_WAIT_LIMIT>(tw);
}

// Persistent multi-ligand form (batches and serving): blocks take work items
// (up to ppb genotypes of one ligand, two a warp) from a device counter and
// re-stage the ligand (and the tensor-core pattern) only when it changes.
// The current ligand's layout and the item index sit in a 128-byte header
// after the tensor-core region.  Every ligand of the launch must be
// pair_eligible (the host splits the others off).
constexpr int PAIR_HDR = 128;
static_assert(sizeof(PairSmem) <= PAIR_HDR - 16, "paired items header too small");

struct PairItemsArgs {
    const WorkItem *items;
    const LigDev *ligs;
    const RecDev *recs;
    int *counter;
    int n_items, ppb;
};

template <int VAR>
__global__ void __launch_bounds__(64, 5) eval_pair_items_kernel(const PairItemsArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5;
    unsigned char *sm =
        smem_raw + (VAR == ADGB_REDUCE_TCGEN05 ? tc2_region(W) : 0) + PAIR_HDR;
    int &s_item = *reinterpret_cast<int *>(sm - 16);
    PairSmem &L = *reinterpret_cast<PairSmem *>(sm - PAIR_HDR);
    int cur_lig = -1;
    Tc2 tw;
    if constexpr (VAR == ADGB_REDUCE_TCGEN05) tc2_begin(smem_raw, tw);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= a.n_items) break;
        const WorkItem w = a.items[it];
        const LigDev &lg = a.ligs[w.lig];
        if (w.lig != cur_lig) {
            if (threadIdx.x == 0)
                L.make(lg.n_atoms, lg.n_tors, W, VAR != ADGB_REDUCE_TCGEN05);
            __syncthreads();
            stage_pair_ligand(sm, L, lg);
            if constexpr (VAR == ADGB_REDUCE_TCGEN05) tc2_write_pattern(smem_raw, lg.tatoms, lg.n_tors);
            cur_lig = w.lig;
            __syncthreads();
        }
        const int nvalid = min(2, w.count - 2 * warp);
        if (nvalid > 0) {
            PairIO io;
#pragma unroll
            for (int g = 0; g < 2; g++) {
                const int k = 2 * warp + (g < nvalid ? g : 0);
                io.genes_in[g] = w.genes + (size_t)k * w.gstride;
                io.genes_out[g] = w.genes + (size_t)k * w.gstride;
                io.energy[g] = w.energy + k;
                io.grad[g] = nullptr;
                io.state[g] = nullptr;
                io.iters[g] = w.iters ? w.iters[k] : w.iters_all;
            }
            io.nvalid = nvalid;
            io.mode = MODE_LS;
            io.resume = 0;
            io.rho = w.rho;
            io.eps = w.eps;
            search_pair<VAR>(sm, L, lg, a.recs[w.rec], warp, io, tw);
        }
        __syncthreads();   // the item is done before shared memory or s_item change
    }
    if constexpr (VAR == ADGB_REDUCE_TCGEN05) tc2_end(tw);
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

template <int VAR>
cudaError_t pair_items_occupancy(int threads, int smem, int device, int *per_sm) {
    auto k = eval_pair_items_kernel<VAR>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (VAR != ADGB_REDUCE_TCGEN05)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads, smem);
    // the runtime's occupancy query reports one block an SM for kernels that
    // allocate tensor memory; count from the kernel's resources instead
    cudaFuncAttributes fa;
    cudaDeviceProp prop;
    if ((e = cudaFuncGetAttributes(&fa, k)) != cudaSuccess) return e;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) return e;
    const int warps = threads / 32;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    int n = regs_warp > 0 ? prop.regsPerMultiprocessor / (regs_warp * warps) : 32;
    const int smem_block = (int)fa.sharedSizeBytes + smem + (int)prop.reservedSharedMemPerBlock;
    n = min(n, (int)prop.sharedMemPerMultiprocessor / max(smem_block, 1));
    n = min(n, prop.maxThreadsPerMultiProcessor / threads);
    n = min(n, prop.maxBlocksPerMultiProcessor);
    n = min(n, 512 / tc2_ncols(warps));
    *per_sm = n;
    return cudaSuccess;
}

template <int VAR>
cudaError_t launch_pair_items_t(const PairItemsArgs &a, int smem, int grid, cudaStream_t s) {
    auto k = eval_pair_items_kernel<VAR>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && VAR != ADGB_REDUCE_TCGEN05) e = prefer_l1(k, smem, 32 * ((a.ppb + 1) / 2));
    if (e != cudaSuccess) return e;
    k<<<grid, 32 * ((a.ppb + 1) / 2), smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Shared-memory bytes one ligand's layout needs in a paired launch of ppb
// genotypes a block (items header included).
int pair_layout_bytes(int n_atoms, int n_tors, int ppb, int variant) {
    PairSmem L;
    ppb = ppb < 1 ? 1 : (ppb > 4 ? 4 : ppb);
    L.make(n_atoms, n_tors, (ppb + 1) / 2, variant != ADGB_REDUCE_TCGEN05);
    return L.total + PAIR_HDR;
}

cudaError_t launch_eval_pair_items(const WorkItem *items, int n_items, const LigDev *ligs,
                                   const RecDev *recs, int *counter, const EvalCfg &cfg, int budget,
                                   int grid, cudaStream_t s) {
    PairItemsArgs a;
    a.items = items;
    a.ligs = ligs;
    a.recs = recs;
    a.counter = counter;
    a.n_items = n_items;
    a.ppb = cfg.ppb < 1 ? 1 : (cfg.ppb > 4 ? 4 : cfg.ppb);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int smem = pair_smem_bytes(budget, (a.ppb + 1) / 2, cfg.variant, dev);
    if (smem < 0) return cudaErrorInvalidValue;
    switch (cfg.variant) {
        case ADGB_REDUCE_SHFL: return launch_pair_items_t<ADGB_REDUCE_SHFL>(a, smem, grid, s);
        case ADGB_REDUCE_MMA_TF32X2: return launch_pair_items_t<ADGB_REDUCE_MMA_TF32X2>(a, smem, grid, s);
        case ADGB_REDUCE_MMA_BF16X3: return launch_pair_items_t<ADGB_REDUCE_MMA_BF16X3>(a, smem, grid, s);
        case ADGB_REDUCE_TCGEN05: return launch_pair_items_t<ADGB_REDUCE_TCGEN05>(a, smem, grid, s);
    }
    return cudaErrorInvalidValue;
}

// Resident blocks of a persistent paired launch: SMs x blocks an SM holds.
int pair_items_grid(const EvalCfg &cfg, int budget, int device) {
    const int ppb = cfg.ppb < 1 ? 1 : (cfg.ppb > 4 ? 4 : cfg.ppb);
    const int threads = 32 * ((ppb + 1) / 2);
    const int smem = pair_smem_bytes(budget, threads / 32, cfg.variant, device);
    if (smem < 0) return 0;
    int per_sm = 0, sms = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (cfg.variant) {
        case ADGB_REDUCE_SHFL: e = pair_items_occupancy<ADGB_REDUCE_SHFL>(threads, smem, device, &per_sm); break;
        case ADGB_REDUCE_MMA_TF32X2: e = pair_items_occupancy<ADGB_REDUCE_MMA_TF32X2>(threads, smem, device, &per_sm); break;
        case ADGB_REDUCE_MMA_BF16X3: e = pair_items_occupancy<ADGB_REDUCE_MMA_BF16X3>(threads, smem, device, &per_sm); break;
        case ADGB_REDUCE_TCGEN05: e = pair_items_occupancy<ADGB_REDUCE_TCGEN05>(threads, smem, device, &per_sm); break;
    }
    if (e != cudaSuccess || per_sm < 1) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return per_sm * sms;
}

// Dynamic shared memory of a paired launch: the tcgen05 variant puts its
// region in front and pads the total so that no more blocks are resident on
// an SM than its 512 tensor-memory columns serve.
int pair_smem_bytes(int layout_bytes, int warps, int variant, int device) {
    if (variant != ADGB_REDUCE_TCGEN05) return layout_bytes;
    const int total = tc2_region(warps) + layout_bytes;
    int sm_smem = 0, reserved = 0;
    if (cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device) !=
            cudaSuccess)
        return -1;
    const int fit = 512 / tc2_ncols(warps);
    const int floor_bytes = sm_smem / (fit + 1) - reserved + 16;
    return total < floor_bytes ? floor_bytes : total;
}

template <int VAR, int SKIP = 0>
static cudaError_t launch_pair_t(const PairArgs &a, int smem, cudaStream_t s) {
    auto k = eval_pair_kernel<VAR, SKIP>;
    const int warps = (a.ppb + 1) / 2;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && VAR != ADGB_REDUCE_TCGEN05) e = prefer_l1(k, smem, 32 * warps);
    if (e != cudaSuccess) return e;
    k<<<(a.n + a.ppb - 1) / a.ppb, 32 * warps, smem, s>>>(a);
    return cudaGetLastError();
}

template <int VAR>
static cudaError_t launch_ablation_t(const PairArgs &a, int smem, cudaStream_t s, int skip) {
    switch (skip) {
        case 0: return launch_pair_t<VAR, 0>(a, smem, s);
        case SK_PAIRS: return launch_pair_t<VAR, SK_PAIRS>(a, smem, s);
        case SK_GRID: return launch_pair_t<VAR, SK_GRID>(a, smem, s);
        case SK_RED | SK_TORS: return launch_pair_t<VAR, SK_RED | SK_TORS>(a, smem, s);
        case SK_TORS: return launch_pair_t<VAR, SK_TORS>(a, smem, s);
        case SK_WALK: return launch_pair_t<VAR, SK_WALK>(a, smem, s);
        case SK_GENE: return launch_pair_t<VAR, SK_GENE>(a, smem, s);
        case SK_SINCOS: return launch_pair_t<VAR, SK_SINCOS>(a, smem, s);
        case SK_PAIRS | SK_GRID: return launch_pair_t<VAR, SK_PAIRS | SK_GRID>(a, smem, s);
        case SK_PAIRMATH: return launch_pair_t<VAR, SK_PAIRMATH>(a, smem, s);
        case SK_PAIRXCHG: return launch_pair_t<VAR, SK_PAIRXCHG>(a, smem, s);
        case SK_BLOCKMMA:
            // every warp of every block must take the block barrier of each
            // evaluation: full blocks only (the iteration count is uniform here)
            if (VAR != ADGB_REDUCE_TCGEN05 || a.n % a.ppb != 0 || a.ppb % 2 != 0 || a.iters_pp)
                return cudaErrorInvalidValue;
            return launch_pair_t<VAR, SK_BLOCKMMA>(a, smem, s);
        case SK_NOISSUE:
            if (VAR != ADGB_REDUCE_TCGEN05) return cudaErrorInvalidValue;
            return launch_pair_t<VAR, SK_NOISSUE>(a, smem, s);
    }
    return cudaErrorInvalidValue;
}

// skip < 0: production launch; else a measurement-only launch without the
// steps in the mask (ls_ablation_dev).
static cudaError_t launch_pair_any(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg,
                                   int mode, const float *genes_in, float *genes_out, int n,
                                   int iters, float rho, float eps, int resume, float *energy,
                                   float *grad, float *state, cudaStream_t s,
                                   const int *iters_per_pose, int skip) {
    if (n == 0) return cudaSuccess;
    if (!pair_eligible(lig.n_atoms, lig.n_tors, lig.n_pairs, lig.n_rounds, lig.r_lanes, cfg.tpp))
        return cudaErrorInvalidValue;
    PairArgs a;
    a.rec = rec;
    a.lig = lig;
    a.ppb = cfg.ppb < 1 ? 1 : (cfg.ppb > 4 ? 4 : cfg.ppb);
    const int warps = (a.ppb + 1) / 2;
    a.L.make(lig.n_atoms, lig.n_tors, warps, cfg.variant != ADGB_REDUCE_TCGEN05);
    a.genes_in = genes_in;
    a.genes_out = genes_out;
    a.energy = energy;
    a.grad = grad;
    a.state = state;
    a.iters_pp = iters_per_pose;
    a.n = n;
    a.iters = iters;
    a.resume = resume;
    a.mode = mode;
    a.rho = rho;
    a.eps = eps;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int smem = pair_smem_bytes(a.L.total, warps, cfg.variant, dev);
    if (smem < 0) return cudaErrorInvalidValue;
    if (skip >= 0) {
        switch (cfg.variant) {
            case ADGB_REDUCE_SHFL: return launch_ablation_t<ADGB_REDUCE_SHFL>(a, smem, s, skip);
            case ADGB_REDUCE_TCGEN05: return launch_ablation_t<ADGB_REDUCE_TCGEN05>(a, smem, s, skip);
        }
        return cudaErrorInvalidValue;
    }
    switch (cfg.variant) {
        case ADGB_REDUCE_SHFL: return launch_pair_t<ADGB_REDUCE_SHFL>(a, smem, s);
        case ADGB_REDUCE_MMA_TF32X2: return launch_pair_t<ADGB_REDUCE_MMA_TF32X2>(a, smem, s);
        case ADGB_REDUCE_MMA_BF16X3: return launch_pair_t<ADGB_REDUCE_MMA_BF16X3>(a, smem, s);
        case ADGB_REDUCE_TCGEN05: return launch_pair_t<ADGB_REDUCE_TCGEN05>(a, smem, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_eval_pair(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg, int mode,
                             const float *genes_in, float *genes_out, int n, int iters, float rho,
                             float eps, int resume, float *energy, float *grad, float *state,
                             cudaStream_t s, const int *iters_per_pose) {
    return launch_pair_any(rec, lig, cfg, mode, genes_in, genes_out, n, iters, rho, eps, resume,
                           energy, grad, state, s, iters_per_pose, -1);
}

cudaError_t launch_pair_ablation(const RecDev &rec, const LigDev &lig, const EvalCfg &cfg,
                                 float *genes, int n, int iters, float *energy, cudaStream_t s,
                                 int skip) {
    if (skip < 0) return cudaErrorInvalidValue;
    return launch_pair_any(rec, lig, cfg, MODE_LS, genes, genes, n, iters, 0.8f, 1e-2f, 0, energy,
                           nullptr, nullptr, s, nullptr, skip);
}

cudaError_t pair_tc_gave_up_async(unsigned int *dst, cudaStream_t s) {
    return cudaMemcpyFromSymbolAsync(dst, g_tc_gave_up, sizeof(unsigned int), 0,
                                     cudaMemcpyDeviceToHost, s);
}

}  // namespace adgb
