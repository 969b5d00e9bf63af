// C ABI of the adgb library: contexts, uploads (with validation and the
// internal atom order), and the launches behind score_poses / local_search /
// pose_coords / reduce4_bench.  See include/adgb.h for the contract.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "adgb_internal.cuh"

using namespace adgb;

namespace {

struct Receptor {
    RecDev dev;
    float *cells = nullptr;
    int n_type_maps = 0;
};

struct Ligand {
    LigDev dev;
    void *mem = nullptr;
    int n_atoms = 0, n_tors = 0, n_types = 0, n_pairs = 0, max_type = 0;
};

}  // namespace

namespace {
// An uneven batch: items of (receptor, ligand, genotype count) run by one
// persistent multi-ligand launch replayed from a captured CUDA graph.
struct Batch {
    std::vector<int> rec_idx, lig_idx, n_poses;  // per item, indices into the tables
    std::vector<LigDev> ligs;                    // unique ligands
    std::vector<RecDev> recs;                    // unique receptors
    std::vector<int> lig_n, lig_t, lig_np;       // sizes of the unique ligands
    long long total = 0;
    LigDev *d_ligs = nullptr;
    RecDev *d_recs = nullptr;
    int *d_counter = nullptr;                    // [2], re-armed by the kernel
    WorkItem *d_items = nullptr;
    int items_cap = 0, n_items = 0;
    EvalCfg cfg{32, 4, 0, 1, 0};
    bool tuned = false;
    cudaGraphExec_t exec = nullptr;
    // what the captured graph was built for
    const float *k_genes = nullptr;
    const float *k_energy = nullptr;
    int k_iters = -1, k_tpp = 0, k_ppb = 0, k_var = -1, k_paired = -1, budget = 0, grid = 0;
    float k_rho = 0.f, k_eps = 0.f;
};
}  // namespace

struct adgb_ctx {
    int device = 0;
    adgb_options opts{};
    std::map<int, Receptor> recs;
    std::map<int, Ligand> ligs;
    std::map<int, Batch> batches;
    std::map<long long, EvalCfg> tune_table;  // autotuned launch shape by size bucket
    int next_id = 1;
    std::string err;
    cudaStream_t stream = nullptr;  // used by the host-pointer calls
    void *stage = nullptr;          // device staging for host-pointer calls
    size_t stage_bytes = 0;
    unsigned int tc_seen = 0;       // tensor-core give-up count already reported (device-wide)
};

namespace {

int fail(adgb_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int ferr(std::string *err, int code, const char *fmt, ...) {
    if (err) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        *err = buf;
    }
    return code;
}

int cuda_fail(adgb_ctx *c, cudaError_t e, const char *what) {
    return fail(c, ADGB_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
}

// The device's tensor-core give-up count (both local-search modules), read
// after everything queued on the context's stream.
cudaError_t tc_count(adgb_ctx *c, unsigned int *count) {
    unsigned int h[2] = {0, 0};
    cudaError_t e = tc_gave_up_async(h, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    *count = h[0] + h[1];
    return e;
}

// ADGB_EDEVICE if a tensor-core completion wait gave up (in any kernel on
// the device) since the context last reported one, else ADGB_OK.
int tc_report(adgb_ctx *c, const char *what) {
    unsigned int n = 0;
    const cudaError_t e = tc_count(c, &n);
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    if (n == c->tc_seen) return ADGB_OK;
    c->tc_seen = n;
    return fail(c, ADGB_EDEVICE,
                "%s: a tensor-core completion wait gave up; the results of this call and of "
                "asynchronous calls since the last report are not valid", what);
}

// End of a synchronous call: its CUDA status, then the tensor-core report.
int sync_done(adgb_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    return tc_report(c, what);
}

// Makes ctx's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite(float x) { return isfinite(x); }

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int stage_reserve(adgb_ctx *c, size_t bytes) {
    if (bytes <= c->stage_bytes) return ADGB_OK;
    if (c->stage) cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&c->stage, bytes);
    if (e != cudaSuccess) return fail(c, ADGB_ENOMEM, "staging allocation of %zu bytes: %s",
                                      bytes, cudaGetErrorString(e));
    c->stage_bytes = bytes;
    return ADGB_OK;
}

// ------------------------------------------------------------- ligand build
struct Bits {
    uint64_t w[4] = {0, 0, 0, 0};
    void set(int i) { w[i >> 6] |= 1ull << (i & 63); }
    bool has(int i) const { return (w[i >> 6] >> (i & 63)) & 1; }
    bool subset_of(const Bits &o) const {
        for (int k = 0; k < 4; k++)
            if (w[k] & ~o.w[k]) return false;
        return true;
    }
    bool meets(const Bits &o) const {
        for (int k = 0; k < 4; k++)
            if (w[k] & o.w[k]) return true;
        return false;
    }
};

struct HostLigand {
    int N, T, NP;
    std::vector<float4> ref;
    std::vector<float2> sv;
    std::vector<int> type, frag, tparent, perm;
    std::vector<int4> tatoms;
    std::vector<float4> taxis, tbref;
    std::vector<uint32_t> pairs;
    std::vector<float2> tptab;
    std::vector<float4> pconst;
    std::vector<int> inc_off;
    std::vector<uint16_t> inc;
    int R = 0, VP = 0;               // matching rounds, lanes a round
    std::vector<uint32_t> rword;     // [R][VP]
    std::vector<float4> rconst;      // [R][VP]
    std::vector<float> tR, teps, tvol, tsol;
    std::vector<int> thb;
    int max_type = 0;
};

// Matching rounds of the pair list: lane a owns atom a (lanes: 32 for
// ligands of at most 32 atoms, one warp a genotype, partner positions and
// reaction forces by warp shuffles; else the atoms rounded up to 32, a block
// of threads with at most two atoms each, forces through per-round slots in
// shared memory).  A round gives every lane at most one pair to compute (its
// atom first) and at most two pairs whose reaction force it receives (its
// atom second), so that no per-pair force buffer or incidence list is
// needed.  Rounds:
// R = max(ceil(pairs / atoms), ceil(max degree / 3)), the least for which
// an atom of the largest degree fits (one out, two in a round) and the
// atoms' lanes hold every pair; R grows only if no orientation below fits.
//   1. Orient the pairs with every atom's in- and out-degrees within one of
//      each other: join the odd-degree atoms to an extra vertex, walk closed
//      trails until every edge is used (a closed trail enters and leaves a
//      vertex equally often), orient along the walk, drop the extra edges.
//   2. While an atom has more than R out-edges, reverse a directed path
//      from it to an atom with fewer than R (breadth-first search); the
//      ends change by one, the inner atoms not at all.  In-degrees stay at
//      most 2R because the degree is at most 3R.
//   3. Split each atom's in-edges over two receive slots (at most R each)
//      and colour the edges of the bipartite graph (tails; slots) with R
//      colours (Konig's theorem): a colour a free at the tail and b free at
//      the slot; if a is taken at the slot, swap a and b along the
//      alternating path that starts there.  Colour = round.
// Word of lane l in round r: partner lane (bits 0-7; l itself without a
// pair, atom 0 for a lane past the last atom, so that every read is of a
// real atom), source lanes of the two received forces (bits 8-15 and 16-23),
// hb flag (bit 24), whether each receive slot is used (bits 25 and 26).  A
// lane without a pair has all-zero constants, which make the pair term
// exactly zero.
constexpr int ROUNDS_BLOCK_MIN_ATOMS = 112;

void build_rounds(HostLigand &h) {
    const int N = h.N, NP = h.NP, X = N;  // X: the extra vertex
    std::vector<int> ea(NP), eb(NP), deg(N, 0);
    std::vector<std::vector<int>> adj(N + 1);  // edge ids
    std::vector<int> ex_a, ex_b;
    for (int p = 0; p < NP; p++) {
        ea[p] = h.pairs[p] & 255;
        eb[p] = (h.pairs[p] >> 8) & 255;
        adj[ea[p]].push_back(p);
        adj[eb[p]].push_back(p);
        deg[ea[p]]++;
        deg[eb[p]]++;
    }
    for (int v = 0; v < N; v++)
        if (adj[v].size() & 1) {
            const int id = NP + (int)ex_a.size();
            ex_a.push_back(v);
            ex_b.push_back(X);
            adj[v].push_back(id);
            adj[X].push_back(id);
        }
    const int NE = NP + (int)ex_a.size();
    auto end_a = [&](int e) { return e < NP ? ea[e] : ex_a[e - NP]; };
    auto end_b = [&](int e) { return e < NP ? eb[e] : ex_b[e - NP]; };
    std::vector<char> used(NE, 0);
    std::vector<int> tail(NE, -1), head(NE, -1);
    std::vector<size_t> next(N + 1, 0);
    for (int s0 = 0; s0 <= N; s0++) {
        for (;;) {
            while (next[s0] < adj[s0].size() && used[adj[s0][next[s0]]]) next[s0]++;
            if (next[s0] == adj[s0].size()) break;
            int v = s0;
            for (;;) {  // a closed trail from s0 (every degree is even)
                while (next[v] < adj[v].size() && used[adj[v][next[v]]]) next[v]++;
                if (next[v] == adj[v].size()) break;
                const int e = adj[v][next[v]];
                used[e] = 1;
                const int w = end_a(e) == v ? end_b(e) : end_a(e);
                tail[e] = v;
                head[e] = w;
                v = w;
            }
        }
    }
    const int maxdeg = *std::max_element(deg.begin(), deg.end());
    int R = std::max((NP + N - 1) / N, (maxdeg + 2) / 3);
    std::vector<std::vector<int>> outs(N);  // edges leaving each atom
    auto rebuild_out = [&]() {
        for (auto &o : outs) o.clear();
        for (int p = 0; p < NP; p++) outs[tail[p]].push_back(p);
    };
    rebuild_out();
    for (int u = 0; u < N; u++) {
        while ((int)outs[u].size() > R) {
            // breadth-first search along out-edges for an atom below R
            std::vector<int> via(N, -1);
            std::vector<char> seen(N, 0);
            std::vector<int> queue(1, u);
            seen[u] = 1;
            int found = -1;
            for (size_t qi = 0; qi < queue.size() && found < 0; qi++) {
                for (int p : outs[queue[qi]]) {
                    const int y = head[p];
                    if (seen[y]) continue;
                    seen[y] = 1;
                    via[y] = p;
                    if ((int)outs[y].size() < R) {
                        found = y;
                        break;
                    }
                    queue.push_back(y);
                }
            }
            if (found < 0) {  // every atom reachable from u is full: widen
                R++;
                continue;
            }
            for (int x = found; x != u;) {
                const int p = via[x];
                const int t = tail[p];
                std::swap(tail[p], head[p]);
                // p now leaves head: move it between the two out-lists, each
                // kept in edge order (as rebuild_out leaves them)
                std::vector<int> &from = outs[t], &to = outs[tail[p]];
                from.erase(std::lower_bound(from.begin(), from.end(), p));
                to.insert(std::lower_bound(to.begin(), to.end(), p), p);
                x = t;
            }
        }
    }
    // receive slots: slot 2v + k, k = 0, 1; an atom's in-edges split in halves
    std::vector<int> slot(NP, -1), ind(N, 0);
    for (int p = 0; p < NP; p++) ind[head[p]]++;
    for (int v = 0; v < N; v++) R = std::max(R, (ind[v] + 1) / 2);
    std::vector<int> filled(N, 0);
    for (int p = 0; p < NP; p++) {
        const int v = head[p];
        slot[p] = 2 * v + (filled[v]++ < (ind[v] + 1) / 2 ? 0 : 1);
    }
    // at_t[u][c] / at_s[q][c]: the edge of colour c leaving atom u / in slot q
    std::vector<int> at_t((size_t)N * R, -1), at_s((size_t)2 * N * R, -1), col(NP, -1);
    for (int p = 0; p < NP; p++) {
        const int u = tail[p], q = slot[p];
        int a = 0, b = 0;
        while (at_t[(size_t)u * R + a] >= 0) a++;
        while (at_s[(size_t)q * R + b] >= 0) b++;
        if (at_s[(size_t)q * R + a] >= 0) {
            // path from q: q -a- t1 -b- q2 -a- t3 ... ; swap a and b along it
            std::vector<int> path;
            int v = q, c = a;
            bool on_slot = true;
            for (;;) {
                const int e = on_slot ? at_s[(size_t)v * R + c] : at_t[(size_t)v * R + c];
                if (e < 0) break;
                path.push_back(e);
                v = on_slot ? tail[e] : slot[e];
                on_slot = !on_slot;
                c = c == a ? b : a;
            }
            for (int e : path) {
                at_t[(size_t)tail[e] * R + col[e]] = -1;
                at_s[(size_t)slot[e] * R + col[e]] = -1;
            }
            for (int e : path) {
                col[e] = col[e] == a ? b : a;
                at_t[(size_t)tail[e] * R + col[e]] = e;
                at_s[(size_t)slot[e] * R + col[e]] = e;
            }
        }
        col[p] = a;
        at_t[(size_t)u * R + a] = p;
        at_s[(size_t)q * R + a] = p;
    }
    const int VP = N <= 32 ? 32 : (N + 31) / 32 * 32;
    h.R = R;
    h.VP = VP;
    h.rword.assign((size_t)R * VP, 0);
    h.rconst.assign((size_t)R * VP, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int r = 0; r < R; r++) {
        uint32_t *wd = &h.rword[(size_t)r * VP];
        for (int l = 0; l < VP; l++) {
            uint32_t w = (uint32_t)(l < N ? l : 0) | (uint32_t)l << 8 | (uint32_t)l << 16;
            if (l < N) {
                const int e = at_t[(size_t)l * R + r];
                if (e >= 0) {
                    // lane l computes the pair with its own atom first: the
                    // pair term is symmetric (swapping the atoms negates dx,
                    // dy, dz exactly and hence the force)
                    w = (w & ~255u) | (uint32_t)head[e] | ((h.pairs[e] >> 24) & 1u) << 24;
                    h.rconst[(size_t)r * VP + l] = h.pconst[e];
                }
                for (int k = 0; k < 2; k++) {
                    const int f = at_s[(size_t)(2 * l + k) * R + r];
                    if (f >= 0)
                        w = (w & ~(255u << (8 + 8 * k))) | (uint32_t)tail[f] << (8 + 8 * k) |
                            1u << (25 + k);
                }
            }
            wd[l] = w;
        }
    }
}

// Whether the kernels use the matching rounds of a ligand (mode as
// adgb_options.pair_rounds).
bool use_pair_rounds(const HostLigand &h, int mode) { return h.R > 0 && mode == 0; }

int build_ligand(std::string *err, const adgb_ligand_desc *d, HostLigand &h) {
    if (!d) return ferr(err, ADGB_EINVAL, "ligand: null descriptor");
    const int N = d->n_atoms, T = d->n_tors, NP = d->n_pairs, NT = d->n_types;
    if (N < 1 || N > ADGB_MAX_ATOMS) return ferr(err, ADGB_EINVAL, "ligand: n_atoms %d not in 1..%d", N, ADGB_MAX_ATOMS);
    if (NT < 1 || NT > ADGB_MAX_TYPES) return ferr(err, ADGB_EINVAL, "ligand: n_types %d not in 1..%d", NT, ADGB_MAX_TYPES);
    if (T < 0 || T > ADGB_MAX_TORS) return ferr(err, ADGB_EINVAL, "ligand: n_tors %d not in 0..%d", T, ADGB_MAX_TORS);
    if (NP < 0 || NP > ADGB_MAX_ATOMS * (ADGB_MAX_ATOMS - 1) / 2)
        return ferr(err, ADGB_EINVAL, "ligand: n_pairs %d not in 0..%d", NP,
                    ADGB_MAX_ATOMS * (ADGB_MAX_ATOMS - 1) / 2);
    if (!d->type || !d->charge || !d->xyz || !d->R || !d->eps || !d->vol || !d->solpar || !d->hb_role)
        return ferr(err, ADGB_EINVAL, "ligand: null per-atom or per-type array");
    if (T > 0 && (!d->tors_bond || !d->mov_off)) return ferr(err, ADGB_EINVAL, "ligand: null torsion arrays");
    if (NP > 0 && !d->pairs) return ferr(err, ADGB_EINVAL, "ligand: null pair list");
    if (!finite(d->hb_R) || d->hb_R <= 0 || !finite(d->hb_eps) || d->hb_eps < 0)
        return ferr(err, ADGB_EINVAL, "ligand: bad hydrogen-bond parameters");
    for (int t = 0; t < NT; t++) {
        if (!finite(d->R[t]) || d->R[t] <= 0 || !finite(d->eps[t]) || d->eps[t] < 0 ||
            !finite(d->vol[t]) || !finite(d->solpar[t]) || d->hb_role[t] < 0 || d->hb_role[t] > 2)
            return ferr(err, ADGB_EINVAL, "ligand: bad parameters of type %d", t);
    }
    for (int i = 0; i < N; i++) {
        if (d->type[i] < 0 || d->type[i] >= NT) return ferr(err, ADGB_EINVAL, "ligand: atom %d type %d out of range", i, d->type[i]);
        if (!finite(d->charge[i]) || !finite(d->xyz[3 * i]) || !finite(d->xyz[3 * i + 1]) || !finite(d->xyz[3 * i + 2]))
            return ferr(err, ADGB_EINVAL, "ligand: atom %d has a non-finite value", i);
    }
    // torsion moving sets
    std::vector<Bits> S(T);
    if (T > 0) {
        if (d->mov_off[0] != 0) return ferr(err, ADGB_EINVAL, "ligand: mov_off[0] != 0");
        for (int k = 0; k < T; k++)
            if (d->mov_off[k + 1] < d->mov_off[k]) return ferr(err, ADGB_EINVAL, "ligand: mov_off not monotone");
        if (d->mov_off[T] > 0 && !d->mov_atoms) return ferr(err, ADGB_EINVAL, "ligand: null mov_atoms");
    }
    for (int k = 0; k < T; k++) {
        const int a = d->tors_bond[2 * k], b = d->tors_bond[2 * k + 1];
        if (a < 0 || a >= N || b < 0 || b >= N || a == b) return ferr(err, ADGB_EINVAL, "ligand: torsion %d bond (%d,%d) invalid", k, a, b);
        const double dx = d->xyz[3 * b] - d->xyz[3 * a], dy = d->xyz[3 * b + 1] - d->xyz[3 * a + 1],
                     dz = d->xyz[3 * b + 2] - d->xyz[3 * a + 2];
        if (!(dx * dx + dy * dy + dz * dz > 0)) return ferr(err, ADGB_EINVAL, "ligand: torsion %d has a zero-length bond", k);
        for (int m = d->mov_off[k]; m < d->mov_off[k + 1]; m++) {
            const int i = d->mov_atoms[m];
            if (i < 0 || i >= N) return ferr(err, ADGB_EINVAL, "ligand: torsion %d moves atom %d out of range", k, i);
            if (S[k].has(i)) return ferr(err, ADGB_EINVAL, "ligand: torsion %d lists atom %d twice", k, i);
            if (i == a || i == b) return ferr(err, ADGB_EINVAL, "ligand: torsion %d moves its own bond atom %d", k, i);
            S[k].set(i);
        }
    }
    // laminar tree, listed root to leaf
    for (int k = 0; k < T; k++) {
        const int ak = d->tors_bond[2 * k], bk = d->tors_bond[2 * k + 1];
        for (int q = k + 1; q < T; q++) {
            const int aq = d->tors_bond[2 * q], bq = d->tors_bond[2 * q + 1];
            const bool inside = S[q].meets(S[k]) || S[k].has(aq) || S[k].has(bq);
            if (inside) {
                if (!S[q].subset_of(S[k]) || !S[k].has(bq) || !(S[k].has(aq) || aq == bk))
                    return ferr(err, ADGB_EINVAL, "ligand: torsions %d and %d are neither nested nor disjoint", k, q);
            } else if (S[q].has(ak) || S[q].has(bk)) {
                return ferr(err, ADGB_EINVAL, "ligand: torsion %d encloses %d but is listed after it", q, k);
            }
        }
    }
    std::vector<int> tparent(T, -1), frag(N, -1);
    for (int k = 0; k < T; k++) {
        const int bk = d->tors_bond[2 * k + 1];
        for (int q = k - 1; q >= 0; q--)
            if (S[q].has(bk)) { tparent[k] = q; break; }
    }
    for (int i = 0; i < N; i++)
        for (int k = T - 1; k >= 0; k--)
            if (S[k].has(i)) { frag[i] = k; break; }
    // depth-first order: a torsion's moving set becomes one contiguous range
    std::vector<std::vector<int>> kids(T + 1);  // index 0 = root
    for (int k = 0; k < T; k++) kids[tparent[k] + 1].push_back(k);
    std::vector<int> perm, start(T, 0), end(T, 0);
    perm.reserve(N);
    std::vector<std::pair<int, int>> stack;  // (node, next child)
    auto emit_own = [&](int node) {
        for (int i = 0; i < N; i++)
            if (frag[i] == node) perm.push_back(i);
    };
    emit_own(-1);
    stack.push_back({-1, 0});
    while (!stack.empty()) {
        auto &top = stack.back();
        const auto &ch = kids[top.first + 1];
        if (top.second < (int)ch.size()) {
            const int k = ch[top.second++];
            start[k] = (int)perm.size();
            emit_own(k);
            stack.push_back({k, 0});
        } else {
            if (top.first >= 0) end[top.first] = (int)perm.size();
            stack.pop_back();
        }
    }
    if ((int)perm.size() != N) return ferr(err, ADGB_EINVAL, "ligand: torsion tree does not cover the atoms once");
    std::vector<int> inv(N);
    for (int n = 0; n < N; n++) inv[perm[n]] = n;
    for (int k = 0; k < T; k++) {
        if (end[k] - start[k] != d->mov_off[k + 1] - d->mov_off[k])
            return ferr(err, ADGB_EINVAL, "ligand: torsion %d moving set is not a subtree", k);
        for (int m = d->mov_off[k]; m < d->mov_off[k + 1]; m++) {
            const int n = inv[d->mov_atoms[m]];
            if (n < start[k] || n >= end[k]) return ferr(err, ADGB_EINVAL, "ligand: torsion %d moving set is not a subtree", k);
        }
    }
    h.N = N;
    h.T = T;
    h.NP = NP;
    h.perm = perm;
    h.ref.resize(N);
    h.sv.resize(N);
    h.type.resize(N);
    h.frag.resize(N);
    for (int n = 0; n < N; n++) {
        const int i = perm[n], t = d->type[i];
        const float q = d->charge[i];
        h.ref[n] = make_float4(d->xyz[3 * i], d->xyz[3 * i + 1], d->xyz[3 * i + 2], q);
        const double S_i = (double)d->solpar[t] + (double)ADGB_QSOL * fabs((double)q);
        h.sv[n] = make_float2((float)((double)ADGB_W_DS * S_i), d->vol[t]);
        h.type[n] = t;
        h.frag[n] = frag[i];
        h.max_type = std::max(h.max_type, t);
    }
    h.tparent = tparent;
    h.tatoms.resize(T);
    h.taxis.resize(T);
    h.tbref.resize(T);
    for (int k = 0; k < T; k++) {
        const int a = d->tors_bond[2 * k], b = d->tors_bond[2 * k + 1];
        const double dx = (double)d->xyz[3 * b] - d->xyz[3 * a], dy = (double)d->xyz[3 * b + 1] - d->xyz[3 * a + 1],
                     dz = (double)d->xyz[3 * b + 2] - d->xyz[3 * a + 2];
        const double l = sqrt(dx * dx + dy * dy + dz * dz);
        h.tatoms[k] = make_int4(inv[a], inv[b], start[k], end[k]);
        h.taxis[k] = make_float4((float)(dx / l), (float)(dy / l), (float)(dz / l), 0.f);
        h.tbref[k] = make_float4(d->xyz[3 * b], d->xyz[3 * b + 1], d->xyz[3 * b + 2], 0.f);
    }
    h.pairs.resize(NP);
    for (int p = 0; p < NP; p++) {
        const int i = d->pairs[2 * p], j = d->pairs[2 * p + 1];
        if (i < 0 || i >= N || j < 0 || j >= N || i == j)
            return ferr(err, ADGB_EINVAL, "ligand: pair %d (%d,%d) invalid", p, i, j);
        const int ti = d->type[i], tj = d->type[j];
        const int ri = d->hb_role[ti], rj = d->hb_role[tj];
        const uint32_t hb = (ri == 1 && rj == 2) || (ri == 2 && rj == 1);
        h.pairs[p] = (uint32_t)inv[i] | (uint32_t)inv[j] << 8 |
                     (uint32_t)(ti * ADGB_MAX_TYPES + tj) << 16 | hb << 24;
    }
    // A pair list longer than one chunk is stored in a fixed pseudo-random
    // order (sorted by a 64-bit mix of the atom indices), so that every chunk
    // touches the atoms about evenly and no owner thread carries a chunk's
    // gather alone.  One chunk keeps the caller's order.
    if (NP > PAIR_CHUNK) {
        auto mix = [](uint64_t x) {   // splitmix64 finaliser
            x += 0x9E3779B97F4A7C15ull;
            x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
            x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
            return x ^ (x >> 31);
        };
        std::vector<std::pair<uint64_t, uint32_t>> keyed(NP);
        for (int p = 0; p < NP; p++) keyed[p] = {mix(h.pairs[p] & 0xffff), h.pairs[p]};
        std::sort(keyed.begin(), keyed.end());
        for (int p = 0; p < NP; p++) h.pairs[p] = keyed[p].second;
    }
    // Within every chunk the pairs are re-ordered for the shared-memory
    // banks: the pair loop gives consecutive pairs to consecutive lanes, and a
    // quarter-warp's 16-byte coordinate loads (or a half-warp's 8-byte
    // parameter loads) conflict when two lanes read different atoms (type
    // pairs) in the same bank group.  A greedy pass appends, from the next 64
    // pairs in line, the one that adds the fewest such collisions.
    // A candidate's collisions are counted from the pairs already placed in
    // its quarter-warp (16-byte atom coordinates: bank group = atom & 7) and
    // half-warp (8-byte atom parameters and type-pair terms: & 15): for each
    // index, the placed entries in its bank group less those of the same atom
    // (or type pair), kept as running counts that restart at every quarter /
    // half-warp boundary.
    for (int p0 = 0; p0 < NP; p0 += PAIR_CHUNK) {
        const int p1 = std::min(NP, p0 + PAIR_CHUNK);
        std::vector<uint32_t> rem(h.pairs.begin() + p0, h.pairs.begin() + p1), out;
        out.reserve(rem.size());
        constexpr int WIN = 64;
        int qi[8], qj[8], hi[16], hj[16], ht[16];          // placed entries a bank group
        int qsi[256], qsj[256], hsi[256], hsj[256], hst[256];   // placed entries an atom / type pair
        while (!rem.empty()) {
            const int pos = (int)out.size();
            if (pos % 16 == 0) {
                std::fill(hi, hi + 16, 0); std::fill(hj, hj + 16, 0); std::fill(ht, ht + 16, 0);
                std::fill(hsi, hsi + 256, 0); std::fill(hsj, hsj + 256, 0); std::fill(hst, hst + 256, 0);
            }
            if (pos % 8 == 0) {
                std::fill(qi, qi + 8, 0); std::fill(qj, qj + 8, 0);
                std::fill(qsi, qsi + 256, 0); std::fill(qsj, qsj + 256, 0);
            }
            int best = 0, best_c = INT32_MAX;
            const int lim = std::min<int>(WIN, (int)rem.size());
            for (int t = 0; t < lim && best_c > 0; t++) {
                const uint32_t c = rem[t];
                const int i = c & 255, j = (c >> 8) & 255, tp = (c >> 16) & 255;
                const int cost = 2 * (qi[i & 7] - qsi[i]) + 2 * (qj[j & 7] - qsj[j]) +
                                 (hi[i & 15] - hsi[i]) + (hj[j & 15] - hsj[j]) +
                                 (ht[tp & 15] - hst[tp]);
                if (cost < best_c) {
                    best_c = cost;
                    best = t;
                }
            }
            const uint32_t c = rem[best];
            const int i = c & 255, j = (c >> 8) & 255, tp = (c >> 16) & 255;
            qi[i & 7]++; qj[j & 7]++; qsi[i]++; qsj[j]++;
            hi[i & 15]++; hj[j & 15]++; ht[tp & 15]++; hsi[i]++; hsj[j]++; hst[tp]++;
            out.push_back(c);
            rem.erase(rem.begin() + best);
        }
        std::copy(out.begin(), out.end(), h.pairs.begin() + p0);
    }
    // incidence lists per chunk of PAIR_CHUNK pairs: for every chunk and atom
    // the chunk's pairs it belongs to as (chunk-local index, side).  Owners of
    // atoms i read their k-th entries together, lane i % 32; each list is
    // ordered so that the 8 lanes of a quarter-warp read force slots in
    // different 16-byte bank groups at every k where they can (greedy).
    {
        const int nch = (NP + PAIR_CHUNK - 1) / PAIR_CHUNK;
        h.inc_off.assign((size_t)nch * (N + 1), 0);
        h.inc.assign(2 * (size_t)NP, 0);
        int pos = 0;
        for (int q = 0; q < nch; q++) {
            const int p0 = q * PAIR_CHUNK, p1 = std::min(NP, p0 + PAIR_CHUNK);
            std::vector<std::vector<uint16_t>> lists(N);
            for (int p = p0; p < p1; p++) {
                lists[h.pairs[p] & 255].push_back((uint16_t)((p - p0) << 1));
                lists[(h.pairs[p] >> 8) & 255].push_back((uint16_t)(((p - p0) << 1) | 1));
            }
            std::vector<std::vector<uint16_t>> ordered(N);
            for (int a0 = 0; a0 < N; a0 += 8) {
                const int a1 = std::min(N, a0 + 8);
                for (;;) {
                    int order[8], n_left = 0;
                    for (int a = a0; a < a1; a++)
                        if (!lists[a].empty()) order[n_left++] = a;
                    if (!n_left) break;
                    std::sort(order, order + n_left, [&](int x, int y) {
                        return lists[x].size() != lists[y].size() ? lists[x].size() > lists[y].size() : x < y;
                    });
                    int used[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    for (int u = 0; u < n_left; u++) {
                        std::vector<uint16_t> &L = lists[order[u]];
                        int pick = 0, pick_c = INT32_MAX;
                        for (int t = 0; t < (int)L.size() && pick_c > 0; t++) {
                            const int c = used[(L[t] >> 1) & 7];
                            if (c < pick_c) {
                                pick_c = c;
                                pick = t;
                            }
                        }
                        used[(L[pick] >> 1) & 7]++;
                        ordered[order[u]].push_back(L[pick]);
                        L.erase(L.begin() + pick);
                    }
                }
            }
            for (int a = 0; a < N; a++) {
                h.inc_off[(size_t)q * (N + 1) + a] = pos;
                for (uint16_t e : ordered[a]) h.inc[pos++] = e;
            }
            h.inc_off[(size_t)q * (N + 1) + N] = pos;
        }
    }
    h.tR.assign(d->R, d->R + NT);
    h.teps.assign(d->eps, d->eps + NT);
    h.tvol.assign(d->vol, d->vol + NT);
    h.tsol.assign(d->solpar, d->solpar + NT);
    h.thb.assign(d->hb_role, d->hb_role + NT);
    h.tptab.assign(TYPE_TAB, make_float2(0.f, 0.f));
    for (int ti = 0; ti < NT; ti++)
        for (int tj = 0; tj < NT; tj++) {
            const int ri = d->hb_role[ti], rj = d->hb_role[tj];
            const bool hb = (ri == 1 && rj == 2) || (ri == 2 && rj == 1);
            double A, B;
            if (hb) {
                const double R = d->hb_R, e = d->hb_eps;
                A = ADGB_W_HB * 5.0 * e * pow(R, 12);
                B = ADGB_W_HB * 6.0 * e * pow(R, 10);
            } else {
                const double R = 0.5 * ((double)d->R[ti] + d->R[tj]);
                const double e = sqrt((double)d->eps[ti] * d->eps[tj]);
                A = ADGB_W_VDW * e * pow(R, 12);
                B = ADGB_W_VDW * 2.0 * e * pow(R, 6);
            }
            h.tptab[ti * ADGB_MAX_TYPES + tj] = make_float2((float)A, (float)B);
        }
    // per-pair constants in pair order: what the pair term needs besides the
    // two positions, so that the pair loop reads one contiguous record
    h.pconst.resize(NP);
    for (int p = 0; p < NP; p++) {
        const uint32_t c = h.pairs[p];
        const int i = c & 255, j = (c >> 8) & 255;
        const float2 ab = h.tptab[(c >> 16) & 255];
        const double qq = (double)ADGB_W_EL * (double)ADGB_ELEC_KCAL * (double)h.ref[i].w * (double)h.ref[j].w;
        const double ds = (double)h.sv[i].x * h.sv[j].y + (double)h.sv[j].x * h.sv[i].y;
        h.pconst[p] = make_float4(ab.x, ab.y, (float)qq, (float)ds);
    }
    // matching rounds where they were measured faster than the force buffer
    // (3000 genotypes, local search): up to 32 atoms (one warp, 1.12-1.28x)
    // and above 112 (two atoms a thread of 128: 1.1x at 128 atoms, 1.3x at
    // 192, 1.5x at 256); between, the rounds' idle lanes cost more than the
    // owner gather they save
    if (NP > 0 && (N <= 32 || N > ROUNDS_BLOCK_MIN_ATOMS)) build_rounds(h);
    return ADGB_OK;
}

}  // namespace

// The launch shape of a ligand (every single-ligand call, dock() and each
// served job take it, so that they compute the same bits).
EvalCfg adgb::launch_cfg(const LigDev &L, int tpp_opt, int ppb_opt, int variant,
                         int genotypes_per_warp) {
    EvalCfg cfg;
    cfg.variant = variant;
    // one warp a genotype up to 32 atoms (one atom a lane, matching rounds),
    // two warps up to 56, else 128 threads a genotype: measured on 3000
    // genotypes, 64 x 2 beats 128 x 1 by 10-17% from 40 to 56 atoms, 128 x 1
    // beats 64 x 2 from 64 atoms on (by 10% at 64, 15-20% at 80-128, more
    // with the matching rounds above 112)
    const int by_size = threads_for_atoms(L.n_atoms);
    cfg.tpp = tpp_opt > 0 ? tpp_opt : by_size;
    int ppb = ppb_opt > 0 ? ppb_opt : 128 / cfg.tpp;
    while (ppb > 1 && cfg.tpp * ppb > 128) ppb--;
    cfg.stage_pairs = 8 * L.n_pairs <= 24 * 1024;
    cfg.chunk = std::max(1, std::min(L.n_pairs, PAIR_CHUNK));
    // keep a block's shared memory within 100 KB so that two blocks fit an SM
    SmemLayout lay;
    for (;; ppb--) {
        lay.make(L.n_atoms, L.n_tors, ppb, cfg.tpp / 32, cfg.chunk, L.n_pairs, cfg.stage_pairs,
                 uses_mma_stage(variant));
        if (lay.total <= 100 * 1024 || ppb == 1) break;
    }
    cfg.ppb = ppb;
    cfg.paired = genotypes_per_warp == 0 &&
                 pair_eligible(L.n_atoms, L.n_tors, L.n_pairs, L.n_rounds, L.r_lanes, cfg.tpp);
    return cfg;
}

namespace {

EvalCfg pick_cfg(const adgb_ctx *c, const Ligand &L, int variant) {
    return launch_cfg(L.dev, c->opts.threads_per_pose, c->opts.poses_per_block, variant,
                      c->opts.genotypes_per_warp);
}

int check_variant(adgb_ctx *c, int &variant) {
    if (variant < 0) variant = c->opts.reduce_variant;
    if (variant < 0 || variant >= ADGB_REDUCE_N) return fail(c, ADGB_EINVAL, "unknown reduce variant %d", variant);
    return ADGB_OK;
}

int lookup(adgb_ctx *c, int rid, int lid, Receptor **R, Ligand **L) {
    if (R) {
        auto it = c->recs.find(rid);
        if (it == c->recs.end()) return fail(c, ADGB_ENOTFOUND, "unknown receptor id %d", rid);
        *R = &it->second;
    }
    auto jt = c->ligs.find(lid);
    if (jt == c->ligs.end()) return fail(c, ADGB_ENOTFOUND, "unknown ligand id %d", lid);
    *L = &jt->second;
    if (R && *R && jt->second.max_type >= (*R)->n_type_maps)
        return fail(c, ADGB_EINVAL, "ligand type %d has no map in receptor %d (%d type maps)",
                    jt->second.max_type, rid, (*R)->n_type_maps);
    return ADGB_OK;
}

}  // namespace


namespace adgb {

int make_ligand_blob(std::string *err, const adgb_ligand_desc *d, int pair_rounds, LigandBlob &out) {
    HostLigand h;
    int rc = build_ligand(err, d, h);
    if (rc) return rc;
    if (!use_pair_rounds(h, pair_rounds)) h.R = h.VP = 0;
    const int N = h.N, T = h.T, NP = h.NP, NT = d->n_types;
    const int Tz = T > 0 ? T : 1, NPz = NP > 0 ? NP : 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = al256(off + bytes); return o; };
    const size_t o_ref = take(16 * N), o_sv = take(8 * N), o_type = take(4 * N), o_frag = take(4 * N);
    const size_t o_tpar = take(4 * Tz), o_tat = take(16 * Tz), o_tax = take(16 * Tz), o_tb = take(16 * Tz);
    const size_t o_pairs = take(4 * NPz), o_tab = take(8 * TYPE_TAB), o_perm = take(4 * N);
    const size_t o_pconst = take(16 * NPz);
    const int NCH = (NP + PAIR_CHUNK - 1) / PAIR_CHUNK;
    const size_t o_incoff = take(4 * (size_t)(NCH > 0 ? NCH : 1) * (N + 1)), o_inc = take(2 * 2 * (size_t)NPz);
    const size_t RVz = h.R > 0 ? (size_t)h.R * h.VP : 1;
    const size_t o_rword = take(4 * RVz), o_rconst = take(16 * RVz);
    const size_t o_tR = take(4 * NT), o_teps = take(4 * NT), o_tvol = take(4 * NT),
                 o_tsol = take(4 * NT), o_thb = take(4 * NT);
    std::vector<unsigned char> &buf = out.bytes;
    buf.assign(off, 0);
    memcpy(&buf[o_ref], h.ref.data(), 16 * N);
    memcpy(&buf[o_sv], h.sv.data(), 8 * N);
    memcpy(&buf[o_type], h.type.data(), 4 * N);
    memcpy(&buf[o_frag], h.frag.data(), 4 * N);
    if (T) {
        memcpy(&buf[o_tpar], h.tparent.data(), 4 * T);
        memcpy(&buf[o_tat], h.tatoms.data(), 16 * T);
        memcpy(&buf[o_tax], h.taxis.data(), 16 * T);
        memcpy(&buf[o_tb], h.tbref.data(), 16 * T);
    }
    if (NP) memcpy(&buf[o_pairs], h.pairs.data(), 4 * NP);
    if (NP) memcpy(&buf[o_pconst], h.pconst.data(), 16 * (size_t)NP);
    memcpy(&buf[o_tab], h.tptab.data(), 8 * TYPE_TAB);
    memcpy(&buf[o_perm], h.perm.data(), 4 * N);
    if (NCH) memcpy(&buf[o_incoff], h.inc_off.data(), 4 * (size_t)NCH * (N + 1));
    if (NP) memcpy(&buf[o_inc], h.inc.data(), 2 * 2 * (size_t)NP);
    if (h.R) {
        memcpy(&buf[o_rword], h.rword.data(), 4 * (size_t)h.R * h.VP);
        memcpy(&buf[o_rconst], h.rconst.data(), 16 * (size_t)h.R * h.VP);
    }
    memcpy(&buf[o_tR], h.tR.data(), 4 * NT);
    memcpy(&buf[o_teps], h.teps.data(), 4 * NT);
    memcpy(&buf[o_tvol], h.tvol.data(), 4 * NT);
    memcpy(&buf[o_tsol], h.tsol.data(), 4 * NT);
    memcpy(&buf[o_thb], h.thb.data(), 4 * NT);
    LigDev &v = out.rel;
    v.n_atoms = N;
    v.n_tors = T;
    v.n_pairs = NP;
    v.n_types = NT;
    v.n_chunks = NCH;
    v.n_rounds = h.R;
    v.r_lanes = h.R ? h.VP : 0;
    // offsets travel in the pointer fields until bind_ligand relocates them
    auto at = [](size_t o) { return reinterpret_cast<const unsigned char *>((uintptr_t)o); };
    v.ref = reinterpret_cast<const float4 *>(at(o_ref));
    v.sv = reinterpret_cast<const float2 *>(at(o_sv));
    v.type = reinterpret_cast<const int *>(at(o_type));
    v.frag = reinterpret_cast<const int *>(at(o_frag));
    v.tparent = reinterpret_cast<const int *>(at(o_tpar));
    v.tatoms = reinterpret_cast<const int4 *>(at(o_tat));
    v.taxis = reinterpret_cast<const float4 *>(at(o_tax));
    v.tbref = reinterpret_cast<const float4 *>(at(o_tb));
    v.pairs = reinterpret_cast<const uint32_t *>(at(o_pairs));
    v.tptab = reinterpret_cast<const float2 *>(at(o_tab));
    v.pconst = reinterpret_cast<const float4 *>(at(o_pconst));
    v.perm = reinterpret_cast<const int *>(at(o_perm));
    v.inc_off = reinterpret_cast<const int *>(at(o_incoff));
    v.inc = reinterpret_cast<const uint16_t *>(at(o_inc));
    v.rword = reinterpret_cast<const uint32_t *>(at(o_rword));
    v.rconst = reinterpret_cast<const float4 *>(at(o_rconst));
    v.t_R = reinterpret_cast<const float *>(at(o_tR));
    v.t_eps = reinterpret_cast<const float *>(at(o_teps));
    v.t_vol = reinterpret_cast<const float *>(at(o_tvol));
    v.t_sol = reinterpret_cast<const float *>(at(o_tsol));
    v.t_hb = reinterpret_cast<const int *>(at(o_thb));
    v.hb_R = d->hb_R;
    v.hb_eps = d->hb_eps;
    out.max_type = h.max_type;
    return ADGB_OK;
}

LigDev bind_ligand(const LigandBlob &b, const unsigned char *mem) {
    LigDev v = b.rel;
    auto mv = [&](auto p) { return reinterpret_cast<decltype(p)>(mem + reinterpret_cast<uintptr_t>(p)); };
    v.ref = mv(v.ref);
    v.sv = mv(v.sv);
    v.type = mv(v.type);
    v.frag = mv(v.frag);
    v.tparent = mv(v.tparent);
    v.tatoms = mv(v.tatoms);
    v.taxis = mv(v.taxis);
    v.tbref = mv(v.tbref);
    v.pairs = mv(v.pairs);
    v.tptab = mv(v.tptab);
    v.pconst = mv(v.pconst);
    v.perm = mv(v.perm);
    v.inc_off = mv(v.inc_off);
    v.inc = mv(v.inc);
    v.rword = mv(v.rword);
    v.rconst = mv(v.rconst);
    v.t_R = mv(v.t_R);
    v.t_eps = mv(v.t_eps);
    v.t_vol = mv(v.t_vol);
    v.t_sol = mv(v.t_sol);
    v.t_hb = mv(v.t_hb);
    return v;
}

}  // namespace adgb

namespace adgb {

int dock_cfg_from_params(const adgb_dock_params *p, int default_variant, DockCfg &d, int &variant,
                         std::string *err) {
    if (!p) return ferr(err, ADGB_EINVAL, "dock: null parameters");
    if (p->n_runs < 1 || p->pop < 2 || p->pop > 1024 || p->max_gens < 0 || p->ls_iters < 1 ||
        p->max_evals < 0 || !(p->ls_rate >= 0.f && p->ls_rate <= 1.f) ||
        !(p->rho > 0.f && p->rho < 1.f) || !(p->eps > 0.f) || !(p->p_cross >= 0.f && p->p_cross <= 1.f) ||
        !(p->p_mut >= 0.f && p->p_mut <= 1.f) || !finite(p->mut_trans) || !finite(p->mut_angle) ||
        (long long)p->n_runs * p->pop > (1 << 26))
        return ferr(err, ADGB_EINVAL, "dock: bad parameters");
    if (p->conv_every < 0 ||
        (p->conv_every > 0 && (p->conv_top < 2 || p->conv_top > p->pop || !(p->conv_tol > 0.f) ||
                               !finite(p->conv_tol))))
        return ferr(err, ADGB_EINVAL, "dock: bad early-stopping parameters");
    if (p->ls_method < 0 || p->ls_method > 1 ||
        (p->ls_method == 1 &&
         (!(p->sw_rho0 > 0.f) || !finite(p->sw_rho0) || !(p->sw_rho_min >= 0.f) ||
          !finite(p->sw_rho_min) || p->sw_max_succ < 1 || p->sw_max_fail < 1 ||
          !(p->sw_angle_scale > 0.f) || !finite(p->sw_angle_scale))))
        return ferr(err, ADGB_EINVAL, "dock: bad local-search method parameters");
    variant = p->reduce_variant < 0 ? default_variant : p->reduce_variant;
    if (variant < 0 || variant >= ADGB_REDUCE_N) return ferr(err, ADGB_EINVAL, "unknown reduce variant %d", variant);
    d.n_runs = p->n_runs;
    d.pop = p->pop;
    d.max_gens = p->max_gens;
    d.ls_iters = p->ls_iters;
    d.max_evals = p->max_evals;
    d.ls_rate = p->ls_rate;
    d.rho = p->rho;
    d.eps = p->eps;
    d.p_cross = p->p_cross;
    d.p_mut = p->p_mut;
    d.mut_trans = p->mut_trans;
    d.mut_angle = p->mut_angle;
    d.seed = p->seed;
    d.conv_every = p->conv_every;
    d.conv_top = p->conv_top;
    d.conv_tol = p->conv_tol;
    d.ls_method = p->ls_method;
    d.sw_rho0 = p->sw_rho0;
    d.sw_rho_min = p->sw_rho_min;
    d.sw_max_succ = p->sw_max_succ;
    d.sw_max_fail = p->sw_max_fail;
    d.sw_angle_scale = p->sw_angle_scale;
    return ADGB_OK;
}

int ctx_device(const adgb_ctx *c) { return c->device; }
int ctx_default_variant(const adgb_ctx *c) { return c->opts.reduce_variant; }

int ctx_pair_rounds(const adgb_ctx *c) { return c->opts.pair_rounds; }
int ctx_genotypes_per_warp(const adgb_ctx *c) { return c->opts.genotypes_per_warp; }
void ctx_launch_opts(const adgb_ctx *c, int *tpp, int *ppb) {
    *tpp = c->opts.threads_per_pose;
    *ppb = c->opts.poses_per_block;
}

int ctx_receptor(adgb_ctx *c, int rid, RecDev *out, int *n_type_maps) {
    auto it = c->recs.find(rid);
    if (it == c->recs.end()) return ADGB_ENOTFOUND;
    *out = it->second.dev;
    *n_type_maps = it->second.n_type_maps;
    return ADGB_OK;
}

}  // namespace adgb

extern "C" {

int adgb_create(adgb_ctx **ctx, int device, const adgb_options *opts) {
    if (!ctx) return ADGB_EINVAL;
    *ctx = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return ADGB_EDEVICE;
    adgb_ctx *c = new (std::nothrow) adgb_ctx();
    if (!c) return ADGB_ENOMEM;
    c->device = device;
    if (opts) c->opts = *opts;
    if (c->opts.threads_per_pose != 0 && c->opts.threads_per_pose != 32 &&
        c->opts.threads_per_pose != 64 && c->opts.threads_per_pose != 128) {
        delete c;
        return ADGB_EINVAL;
    }
    if (c->opts.poses_per_block < 0 || c->opts.poses_per_block > 8 ||
        c->opts.reduce_variant < 0 || c->opts.reduce_variant >= ADGB_REDUCE_N ||
        c->opts.pair_rounds < 0 || c->opts.pair_rounds > 1 || c->opts.genotypes_per_warp < 0 ||
        c->opts.genotypes_per_warp > 1) {
        delete c;
        return ADGB_EINVAL;
    }
    DeviceGuard g(device);
    if (!g.ok || cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        tc_count(c, &c->tc_seen) != cudaSuccess) {
        if (c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return ADGB_EDEVICE;
    }
    *ctx = c;
    return ADGB_OK;
}

int adgb_destroy(adgb_ctx *c) {
    if (!c) return ADGB_EINVAL;
    {
        DeviceGuard g(c->device);
        for (auto &kv : c->batches) {
            Batch &b = kv.second;
            if (b.exec) cudaGraphExecDestroy(b.exec);
            cudaFree(b.d_ligs);
            cudaFree(b.d_recs);
            cudaFree(b.d_counter);
            cudaFree(b.d_items);
        }
        for (auto &kv : c->recs) cudaFree(kv.second.cells);
        for (auto &kv : c->ligs) cudaFree(kv.second.mem);
        if (c->stage) cudaFree(c->stage);
        if (c->stream) cudaStreamDestroy(c->stream);
    }
    delete c;
    return ADGB_OK;
}

const char *adgb_last_error(const adgb_ctx *c) { return c ? c->err.c_str() : "null context"; }

int upload_receptor_grids(adgb_ctx *c, const adgb_grid_desc *g, const float *maps, int *receptor_id) {
    if (!c) return ADGB_EINVAL;
    if (!g || !maps || !receptor_id) return fail(c, ADGB_EINVAL, "receptor: null argument");
    if (g->nx < 2 || g->ny < 2 || g->nz < 2 || !(g->spacing > 0) || !finite(g->spacing) ||
        g->n_type_maps < 1 || g->n_type_maps > 254 || !finite(g->origin[0]) ||
        !finite(g->origin[1]) || !finite(g->origin[2]))
        return fail(c, ADGB_EINVAL, "receptor: bad grid description");
    DeviceGuard dg(c->device);
    if (!dg.ok) return fail(c, ADGB_EDEVICE, "cannot select device %d", c->device);
    const int M = g->n_type_maps + 2;
    const size_t npts = (size_t)g->nx * g->ny * g->nz;
    const size_t ncell = (size_t)(g->nx - 1) * (g->ny - 1) * (g->nz - 1);
    float *plain = nullptr, *cells = nullptr;
    cudaError_t e = cudaMalloc(&plain, npts * M * sizeof(float));
    if (e != cudaSuccess) return fail(c, ADGB_ENOMEM, "receptor: %s", cudaGetErrorString(e));
    e = cudaMalloc(&cells, ncell * M * 8 * sizeof(float));
    if (e != cudaSuccess) {
        cudaFree(plain);
        return fail(c, ADGB_ENOMEM, "receptor: %s", cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(plain, maps, npts * M * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_pack_grid(plain, g->nx, g->ny, g->nz, M, cells, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(plain);
    if (e != cudaSuccess) {
        cudaFree(cells);
        return cuda_fail(c, e, "receptor upload");
    }
    Receptor R;
    R.cells = cells;
    R.n_type_maps = g->n_type_maps;
    R.dev.nx = g->nx;
    R.dev.ny = g->ny;
    R.dev.nz = g->nz;
    R.dev.M = M;
    const int n[3] = {g->nx, g->ny, g->nz};
    for (int d = 0; d < 3; d++) {
        R.dev.lo[d] = g->origin[d];
        R.dev.hi[d] = (float)((double)g->origin[d] + (double)(n[d] - 1) * g->spacing);
    }
    R.dev.inv_h = (float)(1.0 / (double)g->spacing);
    R.dev.h = g->spacing;
    R.dev.cells = cells;
    const int id = c->next_id++;
    c->recs[id] = R;
    *receptor_id = id;
    return ADGB_OK;
}

int release_receptor(adgb_ctx *c, int id) {
    if (!c) return ADGB_EINVAL;
    auto it = c->recs.find(id);
    if (it == c->recs.end()) return fail(c, ADGB_ENOTFOUND, "unknown receptor id %d", id);
    DeviceGuard g(c->device);
    cudaFree(it->second.cells);
    c->recs.erase(it);
    return ADGB_OK;
}

int upload_ligand_torsion_tree(adgb_ctx *c, const adgb_ligand_desc *d, int *ligand_id) {
    if (!c) return ADGB_EINVAL;
    if (!ligand_id) return fail(c, ADGB_EINVAL, "ligand: null id pointer");
    LigandBlob blob;
    int rc = make_ligand_blob(&c->err, d, c->opts.pair_rounds, blob);
    if (rc) return rc;
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, ADGB_EDEVICE, "cannot select device %d", c->device);
    unsigned char *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, blob.bytes.size());
    if (e != cudaSuccess) return fail(c, ADGB_ENOMEM, "ligand: %s", cudaGetErrorString(e));
    e = cudaMemcpy(mem, blob.bytes.data(), blob.bytes.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(mem);
        return cuda_fail(c, e, "ligand upload");
    }
    Ligand L;
    L.mem = mem;
    L.n_atoms = blob.rel.n_atoms;
    L.n_tors = blob.rel.n_tors;
    L.n_types = blob.rel.n_types;
    L.n_pairs = blob.rel.n_pairs;
    L.max_type = blob.max_type;
    L.dev = bind_ligand(blob, mem);
    const int id = c->next_id++;
    c->ligs[id] = L;
    *ligand_id = id;
    return ADGB_OK;
}

int validate_ligand_torsion_tree(const adgb_ligand_desc *d, char *msg, int msg_len) {
    std::string err;
    HostLigand h;
    const int rc = build_ligand(&err, d, h);
    if (msg && msg_len > 0) {
        strncpy(msg, err.c_str(), (size_t)msg_len - 1);
        msg[msg_len - 1] = 0;
    }
    return rc;
}

int ligand_pair_rounds(const adgb_ligand_desc *d, int *n_rounds, int *lanes, int *max_degree,
                       unsigned int *words, int words_cap, int *perm) {
    std::string err;
    HostLigand h;
    const int rc = build_ligand(&err, d, h);
    if (rc) return rc;
    std::vector<int> deg(h.N, 0);
    for (uint32_t c : h.pairs) {
        deg[c & 255]++;
        deg[(c >> 8) & 255]++;
    }
    if (n_rounds) *n_rounds = h.R;
    if (lanes) *lanes = h.VP;
    if (max_degree) *max_degree = h.N ? *std::max_element(deg.begin(), deg.end()) : 0;
    if (words) {
        if ((size_t)words_cap < (size_t)h.R * h.VP) return ADGB_EINVAL;
        std::copy(h.rword.begin(), h.rword.end(), words);
    }
    if (perm) std::copy(h.perm.begin(), h.perm.end(), perm);
    return ADGB_OK;
}

int release_ligand(adgb_ctx *c, int id) {
    if (!c) return ADGB_EINVAL;
    auto it = c->ligs.find(id);
    if (it == c->ligs.end()) return fail(c, ADGB_ENOTFOUND, "unknown ligand id %d", id);
    DeviceGuard g(c->device);
    cudaFree(it->second.mem);
    c->ligs.erase(it);
    return ADGB_OK;
}

int pose_coords_dev(adgb_ctx *c, int ligand_id, const float *genes_dev, int n, float *xyz_dev,
                    adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    if (n < 0 || (n > 0 && (!genes_dev || !xyz_dev))) return fail(c, ADGB_EINVAL, "pose_coords: bad arguments");
    Ligand *L = nullptr;
    int rc = lookup(c, 0, ligand_id, nullptr, &L);
    if (rc) return rc;
    DeviceGuard g(c->device);
    cudaError_t e = launch_coords(L->dev, genes_dev, n, xyz_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "pose_coords");
}

int pose_coords(adgb_ctx *c, int ligand_id, const float *genes, int n, float *xyz) {
    if (!c) return ADGB_EINVAL;
    if (n < 0 || (n > 0 && (!genes || !xyz))) return fail(c, ADGB_EINVAL, "pose_coords: bad arguments");
    Ligand *L = nullptr;
    int rc = lookup(c, 0, ligand_id, nullptr, &L);
    if (rc || n == 0) return rc;
    DeviceGuard g(c->device);
    const size_t G = 6 + L->n_tors, bg = al256(4 * G * n), bx = 4 * 3 * (size_t)L->n_atoms * n;
    if ((rc = stage_reserve(c, bg + bx))) return rc;
    float *dg = (float *)c->stage, *dx = (float *)((char *)c->stage + bg);
    cudaError_t e = cudaMemcpyAsync(dg, genes, 4 * G * n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_coords(L->dev, dg, n, dx, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(xyz, dx, bx, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "pose_coords");
}

int score_poses_dev(adgb_ctx *c, int receptor_id, int ligand_id, const float *genes_dev, int n,
                    float *energy_dev, float *grad_dev, int variant, adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    if (n < 0 || (n > 0 && (!genes_dev || !energy_dev))) return fail(c, ADGB_EINVAL, "score_poses: bad arguments");
    int rc = check_variant(c, variant);
    if (rc) return rc;
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    if ((rc = lookup(c, receptor_id, ligand_id, &R, &L))) return rc;
    DeviceGuard g(c->device);
    cudaError_t e = launch_eval(R->dev, L->dev, pick_cfg(c, *L, variant), MODE_SCORE, genes_dev,
                                nullptr, n, 1, 0.f, 0.f, 0, energy_dev, grad_dev, nullptr,
                                (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "score_poses");
}

int score_poses(adgb_ctx *c, int receptor_id, int ligand_id, const float *genes, int n,
                float *energy, float *grad, int variant) {
    if (!c) return ADGB_EINVAL;
    if (n < 0 || (n > 0 && (!genes || !energy))) return fail(c, ADGB_EINVAL, "score_poses: bad arguments");
    int rc = check_variant(c, variant);
    if (rc) return rc;
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    if ((rc = lookup(c, receptor_id, ligand_id, &R, &L)) || n == 0) return rc;
    DeviceGuard g(c->device);
    const size_t G = 6 + L->n_tors, bg = al256(4 * G * n), be = al256(4 * (size_t)n);
    if ((rc = stage_reserve(c, 2 * bg + be))) return rc;
    float *dg = (float *)c->stage, *de = (float *)((char *)c->stage + bg);
    float *dgr = (float *)((char *)c->stage + bg + be);
    cudaError_t e = cudaMemcpyAsync(dg, genes, 4 * G * n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_eval(R->dev, L->dev, pick_cfg(c, *L, variant), MODE_SCORE, dg, nullptr, n, 1,
                        0.f, 0.f, 0, de, grad ? dgr : nullptr, nullptr, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(energy, de, 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, dgr, 4 * G * n, cudaMemcpyDeviceToHost, c->stream);
    return sync_done(c, e, "score_poses");
}

static int check_ls(adgb_ctx *c, const adgb_ls_params *p, int &variant) {
    if (!p) return fail(c, ADGB_EINVAL, "local_search: null parameters");
    if (p->iters < 0 || !(p->rho > 0.f && p->rho < 1.f) || !(p->eps > 0.f) || !finite(p->eps))
        return fail(c, ADGB_EINVAL, "local_search: bad parameters");
    if (p->flags & ~ADGB_LS_RESUME) return fail(c, ADGB_EINVAL, "local_search: unknown flags");
    variant = p->reduce_variant;
    return check_variant(c, variant);
}

int local_search_dev(adgb_ctx *c, int receptor_id, int ligand_id, float *genes_dev, int n,
                     const adgb_ls_params *p, float *best_energy_dev, float *state_dev,
                     adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    int variant, rc = check_ls(c, p, variant);
    if (rc) return rc;
    const bool resume = p->flags & ADGB_LS_RESUME;
    if (n < 0 || (n > 0 && (!genes_dev || !best_energy_dev || (resume && !state_dev))))
        return fail(c, ADGB_EINVAL, "local_search: bad arguments");
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    if ((rc = lookup(c, receptor_id, ligand_id, &R, &L))) return rc;
    DeviceGuard g(c->device);
    cudaError_t e = launch_eval(R->dev, L->dev, pick_cfg(c, *L, variant), MODE_LS, genes_dev,
                                genes_dev, n, p->iters, p->rho, p->eps, resume, best_energy_dev,
                                nullptr, state_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "local_search");
}

int local_search(adgb_ctx *c, int receptor_id, int ligand_id, float *genes, int n,
                 const adgb_ls_params *p, float *best_energy, float *state) {
    if (!c) return ADGB_EINVAL;
    int variant, rc = check_ls(c, p, variant);
    if (rc) return rc;
    const bool resume = p->flags & ADGB_LS_RESUME;
    if (n < 0 || (n > 0 && (!genes || !best_energy || (resume && !state))))
        return fail(c, ADGB_EINVAL, "local_search: bad arguments");
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    if ((rc = lookup(c, receptor_id, ligand_id, &R, &L)) || n == 0) return rc;
    DeviceGuard g(c->device);
    const size_t G = 6 + L->n_tors, bg = al256(4 * G * n), be = al256(4 * (size_t)n);
    const size_t bs = state ? al256(4 * 3 * G * n) : 0;
    if ((rc = stage_reserve(c, bg + be + bs))) return rc;
    float *dg = (float *)c->stage, *de = (float *)((char *)c->stage + bg);
    float *ds = state ? (float *)((char *)c->stage + bg + be) : nullptr;
    cudaError_t e = cudaMemcpyAsync(dg, genes, 4 * G * n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && resume) e = cudaMemcpyAsync(ds, state, 4 * 3 * G * n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_eval(R->dev, L->dev, pick_cfg(c, *L, variant), MODE_LS, dg, dg, n, p->iters,
                        p->rho, p->eps, resume, de, nullptr, ds, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(genes, dg, 4 * G * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(best_energy, de, 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && state) e = cudaMemcpyAsync(state, ds, 4 * 3 * G * n, cudaMemcpyDeviceToHost, c->stream);
    return sync_done(c, e, "local_search");
}

static int check_sw(adgb_ctx *c, const adgb_sw_params *p, int &variant, SwCfg &w) {
    if (!p) return fail(c, ADGB_EINVAL, "local_search_sw: null parameters");
    if (p->max_evals < 1 || !(p->rho0 > 0.f) || !finite(p->rho0) || !(p->rho_min >= 0.f) ||
        !finite(p->rho_min) || p->max_succ < 1 || p->max_fail < 1 || !(p->angle_scale > 0.f) ||
        !finite(p->angle_scale) || p->call < 0 || p->call > 0xFFFF)
        return fail(c, ADGB_EINVAL, "local_search_sw: bad parameters");
    variant = p->reduce_variant;
    int rc = check_variant(c, variant);
    if (rc) return rc;
    w.max_evals = p->max_evals;
    w.max_succ = p->max_succ;
    w.max_fail = p->max_fail;
    w.resume = (p->flags & ADGB_LS_RESUME) ? 1 : 0;
    w.rho0 = p->rho0;
    w.rho_min = p->rho_min;
    w.angle_scale = p->angle_scale;
    w.seed = p->seed;
    w.call = (uint32_t)p->call;
    w.pose_base = 0;
    return ADGB_OK;
}

int local_search_sw_dev(adgb_ctx *c, int receptor_id, int ligand_id, float *genes_dev, int n,
                        const adgb_sw_params *p, float *energy_dev, int *evals_dev,
                        float *state_dev, adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    int variant;
    SwCfg w;
    int rc = check_sw(c, p, variant, w);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!genes_dev || !energy_dev || (w.resume && !state_dev))))
        return fail(c, ADGB_EINVAL, "local_search_sw: bad arguments");
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    if ((rc = lookup(c, receptor_id, ligand_id, &R, &L))) return rc;
    DeviceGuard g(c->device);
    cudaError_t e = launch_sw(R->dev, L->dev, pick_cfg(c, *L, variant), w, genes_dev, n, energy_dev,
                              evals_dev, state_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "local_search_sw");
}

int local_search_sw(adgb_ctx *c, int receptor_id, int ligand_id, float *genes, int n,
                    const adgb_sw_params *p, float *energy, int *evals, float *state) {
    if (!c) return ADGB_EINVAL;
    int variant;
    SwCfg w;
    int rc = check_sw(c, p, variant, w);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!genes || !energy || (w.resume && !state))))
        return fail(c, ADGB_EINVAL, "local_search_sw: bad arguments");
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    if ((rc = lookup(c, receptor_id, ligand_id, &R, &L)) || n == 0) return rc;
    DeviceGuard g(c->device);
    const size_t G = 6 + L->n_tors, SW = 2 * G + 5;
    const size_t bg = al256(4 * G * n), be = al256(4 * (size_t)n), bv = al256(4 * (size_t)n);
    const size_t bs = state ? al256(4 * SW * n) : 0;
    if ((rc = stage_reserve(c, bg + be + bv + bs))) return rc;
    char *base = (char *)c->stage;
    float *dg = (float *)base, *de = (float *)(base + bg);
    int *dv = (int *)(base + bg + be);
    float *ds = state ? (float *)(base + bg + be + bv) : nullptr;
    cudaError_t e = cudaMemcpyAsync(dg, genes, 4 * G * n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && w.resume) e = cudaMemcpyAsync(ds, state, 4 * SW * n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_sw(R->dev, L->dev, pick_cfg(c, *L, variant), w, dg, n, de, dv, ds, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(genes, dg, 4 * G * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(energy, de, 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && evals) e = cudaMemcpyAsync(evals, dv, 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && state) e = cudaMemcpyAsync(state, ds, 4 * SW * n, cudaMemcpyDeviceToHost, c->stream);
    return sync_done(c, e, "local_search_sw");
}

static int check_dock(adgb_ctx *c, const adgb_dock_params *p, int &variant, DockCfg &d) {
    return dock_cfg_from_params(p, c->opts.reduce_variant, d, variant, &c->err);
}

// stream-ordered working set of one dock call
static cudaError_t dock_scratch(DockScratch &w, void **mem, int n, int G, int runs, cudaStream_t s) {
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = al256(off + b); return o; };
    const size_t og0 = take(4 * (size_t)n * G), og1 = take(4 * (size_t)n * G), oe = take(4 * (size_t)n),
                 oi = take(4 * (size_t)n), ob = take(4 * (size_t)runs), ov = take(8 * (size_t)runs),
                 od = take(4 * (size_t)runs);
    cudaError_t e = cudaMallocAsync(mem, off, s);
    if (e != cudaSuccess) return e;
    char *m = (char *)*mem;
    w.genes[0] = (float *)(m + og0);
    w.genes[1] = (float *)(m + og1);
    w.energy = (float *)(m + oe);
    w.iters = (int *)(m + oi);
    w.best_e = (float *)(m + ob);
    w.evals = (long long *)(m + ov);
    w.done = (int *)(m + od);
    return cudaSuccess;
}

int dock_dev(adgb_ctx *c, int receptor_id, int ligand_id, const adgb_dock_params *p,
             float *best_genes_dev, double *best_energy_dev, long long *evals_dev,
             adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    int variant;
    DockCfg d;
    int rc = check_dock(c, p, variant, d);
    if (rc) return rc;
    if (!best_genes_dev || !best_energy_dev) return fail(c, ADGB_EINVAL, "dock: null output");
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    if ((rc = lookup(c, receptor_id, ligand_id, &R, &L))) return rc;
    DeviceGuard g(c->device);
    const cudaStream_t s = (cudaStream_t)stream;
    DockScratch w;
    void *mem = nullptr;
    cudaError_t e = dock_scratch(w, &mem, d.n_runs * d.pop, 6 + L->n_tors, d.n_runs, s);
    if (e != cudaSuccess) return fail(c, ADGB_ENOMEM, "dock: %s", cudaGetErrorString(e));
    e = launch_dock(R->dev, L->dev, pick_cfg(c, *L, variant), d, best_genes_dev, best_energy_dev,
                    evals_dev, w, s);
    cudaFreeAsync(mem, s);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "dock");
}

int dock(adgb_ctx *c, int receptor_id, int ligand_id, const adgb_dock_params *p, float *best_genes,
         double *best_energy, long long *evals) {
    if (!c) return ADGB_EINVAL;
    int variant;
    DockCfg d;
    int rc = check_dock(c, p, variant, d);
    if (rc) return rc;
    if (!best_genes || !best_energy) return fail(c, ADGB_EINVAL, "dock: null output");
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    if ((rc = lookup(c, receptor_id, ligand_id, &R, &L))) return rc;
    DeviceGuard g(c->device);
    const int G = 6 + L->n_tors;
    const size_t bg = al256(4 * (size_t)d.n_runs * G), be = al256(8 * (size_t)d.n_runs);
    if ((rc = stage_reserve(c, bg + 2 * be))) return rc;
    float *dg = (float *)c->stage;
    double *de = (double *)((char *)c->stage + bg);
    long long *dv = (long long *)((char *)c->stage + bg + be);
    DockScratch w;
    void *mem = nullptr;
    cudaError_t e = dock_scratch(w, &mem, d.n_runs * d.pop, G, d.n_runs, c->stream);
    if (e != cudaSuccess) return fail(c, ADGB_ENOMEM, "dock: %s", cudaGetErrorString(e));
    e = launch_dock(R->dev, L->dev, pick_cfg(c, *L, variant), d, dg, de, dv, w, c->stream);
    cudaFreeAsync(mem, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(best_genes, dg, 4 * (size_t)d.n_runs * G, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(best_energy, de, 8 * (size_t)d.n_runs, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && evals) e = cudaMemcpyAsync(evals, dv, 8 * (size_t)d.n_runs, cudaMemcpyDeviceToHost, c->stream);
    return sync_done(c, e, "dock");
}

int ga_init_population_dev(adgb_ctx *c, int receptor_id, int ligand_id, unsigned long long seed,
                           int n_runs, int pop, float *genes_dev, adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    if (n_runs < 0 || pop < 0 || (n_runs * (long long)pop > 0 && !genes_dev))
        return fail(c, ADGB_EINVAL, "ga_init_population: bad arguments");
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    int rc = lookup(c, receptor_id, ligand_id, &R, &L);
    if (rc) return rc;
    DeviceGuard g(c->device);
    const int n = n_runs * pop;
    int *iters = nullptr;
    cudaError_t e = cudaMallocAsync(&iters, 4 * (size_t)(n > 0 ? n : 1), (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(c, ADGB_ENOMEM, "ga_init_population: %s", cudaGetErrorString(e));
    e = launch_init_population(R->dev, L->n_tors, seed, n_runs, pop, genes_dev, iters, (cudaStream_t)stream);
    cudaFreeAsync(iters, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "ga_init_population");
}

int ga_generation_dev(adgb_ctx *c, int ligand_id, const adgb_dock_params *p, int generation,
                      const float *genes_dev, const float *energy_dev, float *genes_out_dev,
                      int *iters_out_dev, adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    int variant;
    DockCfg d;
    int rc = check_dock(c, p, variant, d);
    if (rc) return rc;
    if (generation < 1 || !genes_dev || !energy_dev || !genes_out_dev || !iters_out_dev)
        return fail(c, ADGB_EINVAL, "ga_generation: bad arguments");
    Ligand *L = nullptr;
    if ((rc = lookup(c, 0, ligand_id, nullptr, &L))) return rc;
    DeviceGuard g(c->device);
    cudaError_t e = launch_ga_generation(d, 6 + L->n_tors, generation, genes_dev, energy_dev,
                                         genes_out_dev, iters_out_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "ga_generation");
}

int ga_converged_dev(adgb_ctx *c, const adgb_dock_params *p, const float *energy_dev,
                     int *converged_dev, adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    if (!p || !energy_dev || !converged_dev || p->n_runs < 1 || p->pop < 2 || p->pop > 1024 ||
        p->conv_top < 2 || p->conv_top > p->pop || !(p->conv_tol > 0.f) || !finite(p->conv_tol))
        return fail(c, ADGB_EINVAL, "ga_converged: bad arguments");
    DeviceGuard g(c->device);
    cudaError_t e = launch_ga_converged(p->n_runs, p->pop, p->conv_top, p->conv_tol, energy_dev,
                                        converged_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "ga_converged");
}

int rescore_fp64_dev(adgb_ctx *c, int receptor_id, int ligand_id, const float *genes_dev, int n,
                     double *energy_dev, adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    if (n < 0 || (n > 0 && (!genes_dev || !energy_dev))) return fail(c, ADGB_EINVAL, "rescore_fp64: bad arguments");
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    int rc = lookup(c, receptor_id, ligand_id, &R, &L);
    if (rc) return rc;
    DeviceGuard g(c->device);
    cudaError_t e = launch_rescore_fp64(R->dev, L->dev, n, genes_dev, energy_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "rescore_fp64");
}

int reduce4_bench_dev(adgb_ctx *c, int variant, const float *in_dev, int threads, int n_blocks,
                      int reps, float *out_dev, adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    const bool known = variant == ADGB_REDUCE_SHFL || variant == ADGB_REDUCE_MMA_TF32X2 ||
                       variant == ADGB_REDUCE_MMA_BF16X3 || variant == ADGB_REDUCE4_PAPER_FS ||
                       variant == ADGB_REDUCE4_PAPER_HALF || variant == ADGB_REDUCE4_TCGEN05_TF32X2 ||
                       variant == ADGB_REDUCE4_TCGEN05_WAIT_SELFTEST;
    if (!known) return fail(c, ADGB_EINVAL, "reduce4_bench: unknown variant %d", variant);
    if (threads < 32 || threads > 1024 || threads % 32 || n_blocks < 1 || reps < 1 || !in_dev || !out_dev)
        return fail(c, ADGB_EINVAL, "reduce4_bench: bad arguments");
    if ((variant == ADGB_REDUCE4_TCGEN05_TF32X2 || variant == ADGB_REDUCE4_TCGEN05_WAIT_SELFTEST) &&
        threads % 64)
        return fail(c, ADGB_EINVAL, "reduce4_bench: the tcgen05 form needs a multiple of 64 threads");
    DeviceGuard g(c->device);
    cudaError_t e = launch_reduce4_bench(variant, in_dev, threads, n_blocks, reps, out_dev,
                                         (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "reduce4_bench");
}

int alu_bench_dev(adgb_ctx *c, int kind, int n_blocks, int threads, int reps, float *out_dev,
                  adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    if (kind < 0 || kind > 3 || n_blocks < 1 || threads < 32 || threads > 256 || threads % 32 ||
        reps < 1 || !out_dev)
        return fail(c, ADGB_EINVAL, "alu_bench: bad arguments");
    DeviceGuard g(c->device);
    cudaError_t e = launch_alu_bench(kind, n_blocks, threads, reps, out_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "alu_bench");
}

int l2_bench_dev(adgb_ctx *c, int kind, const float *buf_dev, long long n_float4, int cell_float4,
                 int n_blocks, int threads, int reps, float *out_dev, adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    if ((kind != 0 && kind != 1) || !buf_dev || !out_dev || n_float4 < 1 || n_blocks < 1 ||
        threads < 32 || threads > 256 || threads % 32 || reps < 1 ||
        (reinterpret_cast<uintptr_t>(buf_dev) & 15))
        return fail(c, ADGB_EINVAL, "l2_bench: bad arguments");
    if (kind == 1 && (cell_float4 < 6 || cell_float4 % 2 || n_float4 < cell_float4 ||
                      n_float4 / cell_float4 > 0xffffffffLL))
        return fail(c, ADGB_EINVAL, "l2_bench: bad cell size");
    DeviceGuard g(c->device);
    cudaError_t e = launch_l2_bench(kind, buf_dev, n_float4, cell_float4, n_blocks, threads, reps,
                                    out_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "l2_bench");
}

int ls_ablation_dev(adgb_ctx *c, int receptor_id, int ligand_id, float *genes_dev, int n, int iters,
                    int variant, int skip_mask, float *best_energy_dev, adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    if (n < 0 || iters < 0 || skip_mask < 0 || (n > 0 && (!genes_dev || !best_energy_dev)))
        return fail(c, ADGB_EINVAL, "ls_ablation: bad arguments");
    if (variant != ADGB_REDUCE_SHFL && variant != ADGB_REDUCE_TCGEN05)
        return fail(c, ADGB_EINVAL, "ls_ablation: variant %d not built (shuffle and tcgen05 only)", variant);
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    int rc = lookup(c, receptor_id, ligand_id, &R, &L);
    if (rc) return rc;
    EvalCfg cfg = pick_cfg(c, *L, variant);
    if (!pair_eligible(L->n_atoms, L->n_tors, L->n_pairs, L->dev.n_rounds, L->dev.r_lanes, cfg.tpp))
        return fail(c, ADGB_EINVAL, "ls_ablation: the ligand does not run two genotypes a warp");
    DeviceGuard g(c->device);
    cudaError_t e = launch_pair_ablation(R->dev, L->dev, cfg, genes_dev, n, iters, best_energy_dev,
                                         (cudaStream_t)stream, skip_mask);
    if (e == cudaErrorInvalidValue) return fail(c, ADGB_EINVAL, "ls_ablation: mask %d not built", skip_mask);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "ls_ablation");
}

int device_status(adgb_ctx *c) {
    if (!c) return ADGB_EINVAL;
    DeviceGuard g(c->device);
    return tc_report(c, "device_status");
}

int philox4x32_10_dev(adgb_ctx *c, const unsigned int *in_dev, int n, unsigned int *out_dev,
                      adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    if (n < 0 || (n > 0 && (!in_dev || !out_dev))) return fail(c, ADGB_EINVAL, "philox4x32_10: bad arguments");
    DeviceGuard g(c->device);
    cudaError_t e = launch_philox(in_dev, n, out_dev, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "philox4x32_10");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// dock_noalloc_dev: dock_dev without any device allocation.
//
// Some callers cannot allocate device memory when they call the library:
// host programs that reserve the whole GPU memory budget up front and forbid
// libraries to allocate, and latency-critical serving paths where an
// allocation (which may synchronise the device, and may fail under memory
// pressure) is not acceptable in the middle of a request.  For them the dock
// working set lives in one fixed device array compiled into the library.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr size_t NOALLOC_BYTES = 4u << 20;  // 4 MiB, held on every device that loads the library
static __device__ __align__(256) unsigned char g_dock_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_dock_scratch on the current device (the host-side
// symbol is only a stand-in for it).  Looked up again on every call made
// outside a stream capture, so that a device reset (which reloads the module
// and may move the array) never leaves a stale address; a call made during a
// capture uses the address of the last uncaptured call on that device.
cudaError_t noalloc_base(int device, cudaStream_t s, void **out) {
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_noalloc_ptr[device]) {
        if (cap != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dock_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[device] = p;
    }
    *out = g_noalloc_ptr[device];
    return cudaSuccess;
}

// Same partition as the allocating path: two populations, energies, counts,
// run bests, evaluation counters, stop flags.
size_t noalloc_layout(DockScratch *w, unsigned char *base, int n, int G, int runs) {
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = al256(off + b); return o; };
    const size_t og0 = take(4 * (size_t)n * G), og1 = take(4 * (size_t)n * G), oe = take(4 * (size_t)n),
                 oi = take(4 * (size_t)n), ob = take(4 * (size_t)runs), ov = take(8 * (size_t)runs),
                 od = take(4 * (size_t)runs);
    if (w && base) {
        w->genes[0] = (float *)(base + og0);
        w->genes[1] = (float *)(base + og1);
        w->energy = (float *)(base + oe);
        w->iters = (int *)(base + oi);
        w->best_e = (float *)(base + ob);
        w->evals = (long long *)(base + ov);
        w->done = (int *)(base + od);
    }
    return off;
}

}  // namespace

extern "C" int dock_noalloc_dev(adgb_ctx *c, int receptor_id, int ligand_id,
                                const adgb_dock_params *p, float *best_genes_dev,
                                double *best_energy_dev, long long *evals_dev,
                                adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    int variant;
    DockCfg d;
    int rc = check_dock(c, p, variant, d);
    if (rc) return rc;
    if (!best_genes_dev || !best_energy_dev) return fail(c, ADGB_EINVAL, "dock_noalloc: null output");
    Receptor *R = nullptr;
    Ligand *L = nullptr;
    if ((rc = lookup(c, receptor_id, ligand_id, &R, &L))) return rc;
    const int G = 6 + L->n_tors;
    const size_t need = noalloc_layout(nullptr, nullptr, d.n_runs * d.pop, G, d.n_runs);
    if (need > NOALLOC_BYTES)
        return fail(c, ADGB_EINVAL,
                    "dock_noalloc: working set of %zu bytes (%d runs x %d individuals, %d genes) "
                    "exceeds the fixed %zu-byte array",
                    need, d.n_runs, d.pop, G, NOALLOC_BYTES);
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, ADGB_EDEVICE, "cannot select device %d", c->device);
    void *base = nullptr;
    cudaError_t e = noalloc_base(c->device, (cudaStream_t)stream, &base);
    if (e != cudaSuccess) return cuda_fail(c, e, "dock_noalloc: scratch address");
    DockScratch w;
    noalloc_layout(&w, (unsigned char *)base, d.n_runs * d.pop, G, d.n_runs);
    e = launch_dock(R->dev, L->dev, pick_cfg(c, *L, variant), d, best_genes_dev, best_energy_dev,
                    evals_dev, w, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "dock_noalloc");
}


// ---------------------------------------------------------------------------
// Uneven batches (one persistent multi-ligand launch, graph-captured, tuned)
// ---------------------------------------------------------------------------
namespace {

int batch_budget(const Batch &b, const EvalCfg &cfg) {
    int budget = 1024;
    for (size_t u = 0; u < b.ligs.size(); u++)
        budget = std::max(budget, items_layout_bytes(cfg, b.lig_n[u], b.lig_t[u], b.lig_np[u]));
    return budget;
}

// Two genotypes a warp only when every ligand of the batch qualifies (one
// launch shape serves the whole batch).
bool batch_pairable(const Batch &b, const EvalCfg &cfg) {
    for (const LigDev &l : b.ligs)
        if (!pair_eligible(l.n_atoms, l.n_tors, l.n_pairs, l.n_rounds, l.r_lanes, cfg.tpp)) return false;
    return true;
}

// Items of ppb genotypes of one ligand, longest (most work) first.
std::vector<WorkItem> batch_items(const Batch &b, const EvalCfg &cfg, float *genes, float *energy,
                                  int iters, float rho, float eps) {
    std::vector<WorkItem> items;
    long long row = 0;
    for (size_t i = 0; i < b.n_poses.size(); i++) {
        const int u = b.lig_idx[i];
        const int cost = (int)std::min<long long>(INT32_MAX, (long long)(b.lig_np[u] + 8 * b.lig_n[u] + 64));
        for (int k = 0; k < b.n_poses[i]; k += cfg.ppb) {
            WorkItem w;
            w.lig = u;
            w.rec = b.rec_idx[i];
            w.count = std::min(cfg.ppb, b.n_poses[i] - k);
            w.gstride = 6 + ADGB_MAX_TORS;
            w.genes = genes + (row + k) * (long long)(6 + ADGB_MAX_TORS);
            w.energy = energy + row + k;
            w.iters = nullptr;
            w.iters_all = iters;
            w.cost = cost;
            w.rho = rho;
            w.eps = eps;
            items.push_back(w);
        }
        row += b.n_poses[i];
    }
    std::stable_sort(items.begin(), items.end(), [](const WorkItem &x, const WorkItem &y) {
        return x.cost > y.cost || (x.cost == y.cost && x.lig < y.lig);
    });
    return items;
}

cudaError_t upload_items(Batch &b, const std::vector<WorkItem> &items, cudaStream_t s) {
    if ((int)items.size() > b.items_cap) {
        if (b.d_items) cudaFree(b.d_items);
        b.d_items = nullptr;
        cudaError_t e = cudaMalloc(&b.d_items, sizeof(WorkItem) * std::max<size_t>(items.size(), 1));
        if (e != cudaSuccess) return e;
        b.items_cap = (int)items.size();
    }
    b.n_items = (int)items.size();
    cudaError_t e = cudaMemcpyAsync(b.d_items, items.data(), sizeof(WorkItem) * items.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

long long tune_key(const Batch &b) {
    int n = 0, np = 0;
    for (size_t u = 0; u < b.ligs.size(); u++) {
        n = std::max(n, b.lig_n[u]);
        np = std::max(np, b.lig_np[u]);
    }
    return ((long long)((n + 31) / 32) << 32) | (long long)((np + 511) / 512);
}

}  // namespace

extern "C" int batch_create(adgb_ctx *c, int n_items, const int *receptor_ids, const int *ligand_ids,
                            const int *n_poses, int *batch_id) {
    if (!c) return ADGB_EINVAL;
    if (n_items < 1 || !receptor_ids || !ligand_ids || !n_poses || !batch_id)
        return fail(c, ADGB_EINVAL, "batch_create: bad arguments");
    Batch b;
    std::map<int, int> lmap, rmap;
    for (int i = 0; i < n_items; i++) {
        if (n_poses[i] < 0) return fail(c, ADGB_EINVAL, "batch_create: item %d has %d genotypes", i, n_poses[i]);
        Receptor *R = nullptr;
        Ligand *L = nullptr;
        int rc = lookup(c, receptor_ids[i], ligand_ids[i], &R, &L);
        if (rc) return rc;
        if (!lmap.count(ligand_ids[i])) {
            lmap[ligand_ids[i]] = (int)b.ligs.size();
            b.ligs.push_back(L->dev);
            b.lig_n.push_back(L->n_atoms);
            b.lig_t.push_back(L->n_tors);
            b.lig_np.push_back(L->n_pairs);
        }
        if (!rmap.count(receptor_ids[i])) {
            rmap[receptor_ids[i]] = (int)b.recs.size();
            b.recs.push_back(R->dev);
        }
        b.lig_idx.push_back(lmap[ligand_ids[i]]);
        b.rec_idx.push_back(rmap[receptor_ids[i]]);
        b.n_poses.push_back(n_poses[i]);
        b.total += n_poses[i];
    }
    DeviceGuard g(c->device);
    cudaError_t e = cudaMalloc(&b.d_ligs, sizeof(LigDev) * b.ligs.size());
    if (e == cudaSuccess) e = cudaMalloc(&b.d_recs, sizeof(RecDev) * b.recs.size());
    if (e == cudaSuccess) e = cudaMalloc(&b.d_counter, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(b.d_ligs, b.ligs.data(), sizeof(LigDev) * b.ligs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b.d_recs, b.recs.data(), sizeof(RecDev) * b.recs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b.d_counter, 0, 2 * sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(b.d_ligs);
        cudaFree(b.d_recs);
        cudaFree(b.d_counter);
        return fail(c, ADGB_ENOMEM, "batch_create: %s", cudaGetErrorString(e));
    }
    b.cfg.variant = c->opts.reduce_variant;
    b.cfg.paired = c->opts.genotypes_per_warp == 0;
    if (c->opts.threads_per_pose > 0) {   // the context's launch shape, until tuned
        b.cfg.tpp = c->opts.threads_per_pose;
        b.cfg.ppb = c->opts.poses_per_block > 0 ? c->opts.poses_per_block : 128 / b.cfg.tpp;
    }
    auto it = c->tune_table.find(tune_key(b));
    if (it != c->tune_table.end()) {
        b.cfg = it->second;
        b.tuned = true;
    }
    const int id = c->next_id++;
    c->batches[id] = std::move(b);
    *batch_id = id;
    return ADGB_OK;
}

extern "C" int batch_release(adgb_ctx *c, int batch_id) {
    if (!c) return ADGB_EINVAL;
    auto it = c->batches.find(batch_id);
    if (it == c->batches.end()) return fail(c, ADGB_ENOTFOUND, "unknown batch id %d", batch_id);
    DeviceGuard g(c->device);
    Batch &b = it->second;
    if (b.exec) cudaGraphExecDestroy(b.exec);
    cudaFree(b.d_ligs);
    cudaFree(b.d_recs);
    cudaFree(b.d_counter);
    cudaFree(b.d_items);
    c->batches.erase(it);
    return ADGB_OK;
}

extern "C" int batch_local_search_dev(adgb_ctx *c, int batch_id, float *genes_dev,
                                      const adgb_ls_params *p, float *best_energy_dev,
                                      adgb_stream stream) {
    if (!c) return ADGB_EINVAL;
    int variant, rc = check_ls(c, p, variant);
    if (rc) return rc;
    if (p->flags & ADGB_LS_RESUME) return fail(c, ADGB_EINVAL, "batch_local_search: resume is not supported");
    auto it = c->batches.find(batch_id);
    if (it == c->batches.end()) return fail(c, ADGB_ENOTFOUND, "unknown batch id %d", batch_id);
    Batch &b = it->second;
    if (b.total > 0 && (!genes_dev || !best_energy_dev)) return fail(c, ADGB_EINVAL, "batch_local_search: null buffers");
    if (b.total == 0) return ADGB_OK;
    DeviceGuard g(c->device);
    EvalCfg cfg = b.cfg;
    if (!b.tuned || p->reduce_variant >= 0) cfg.variant = variant;
    cfg.paired = cfg.paired && batch_pairable(b, cfg);
    cudaError_t e = cudaSuccess;
    const bool same = b.exec && b.k_genes == genes_dev && b.k_energy == best_energy_dev &&
                      b.k_iters == p->iters && b.k_rho == p->rho && b.k_eps == p->eps &&
                      b.k_tpp == cfg.tpp && b.k_ppb == cfg.ppb && b.k_var == cfg.variant &&
                      b.k_paired == cfg.paired;
    if (!same) {
        if (b.exec) cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
        b.budget = batch_budget(b, cfg);
        b.grid = items_grid(cfg, b.budget, c->device);
        if (b.grid < 1) return fail(c, ADGB_EINVAL, "batch_local_search: launch shape does not fit an SM");
        e = upload_items(b, batch_items(b, cfg, genes_dev, best_energy_dev, p->iters, p->rho, p->eps),
                         c->stream);
        cudaGraph_t graph = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = launch_eval_items(b.d_items, b.n_items, b.d_ligs, b.d_recs, b.d_counter,
                                               cfg, b.budget, b.grid, c->stream);
            e = cudaStreamEndCapture(c->stream, &graph);
            if (el != cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(c, e, "batch_local_search: graph capture");
        b.k_genes = genes_dev;
        b.k_energy = best_energy_dev;
        b.k_iters = p->iters;
        b.k_rho = p->rho;
        b.k_eps = p->eps;
        b.k_tpp = cfg.tpp;
        b.k_ppb = cfg.ppb;
        b.k_var = cfg.variant;
        b.k_paired = cfg.paired;
    }
    e = cudaGraphLaunch(b.exec, (cudaStream_t)stream);
    return e == cudaSuccess ? ADGB_OK : cuda_fail(c, e, "batch_local_search: graph launch");
}

extern "C" int batch_autotune(adgb_ctx *c, int batch_id, const float *genes_dev, int iters,
                              adgb_options *chosen) {
    if (!c) return ADGB_EINVAL;
    auto it = c->batches.find(batch_id);
    if (it == c->batches.end()) return fail(c, ADGB_ENOTFOUND, "unknown batch id %d", batch_id);
    Batch &b = it->second;
    if (iters < 1 || (b.total > 0 && !genes_dev)) return fail(c, ADGB_EINVAL, "batch_autotune: bad arguments");
    DeviceGuard g(c->device);
    // one genotype a warp (the last field 0) and, where every ligand of the
    // batch qualifies, two genotypes a warp
    const EvalCfg all[] = {{32, 4, ADGB_REDUCE_SHFL, 1, 0, 0}, {32, 4, ADGB_REDUCE_MMA_TF32X2, 1, 0, 0},
                           {32, 4, ADGB_REDUCE_MMA_BF16X3, 1, 0, 0}, {32, 4, ADGB_REDUCE_TCGEN05, 1, 0, 0},
                           {32, 2, ADGB_REDUCE_SHFL, 1, 0, 0}, {64, 2, ADGB_REDUCE_SHFL, 1, 0, 0},
                           {128, 1, ADGB_REDUCE_SHFL, 1, 0, 0},
                           {32, 4, ADGB_REDUCE_SHFL, 1, 0, 1}, {32, 8, ADGB_REDUCE_SHFL, 1, 0, 1},
                           {32, 4, ADGB_REDUCE_TCGEN05, 1, 0, 1}, {32, 8, ADGB_REDUCE_TCGEN05, 1, 0, 1}};
    std::vector<EvalCfg> cands;
    for (const EvalCfg &cf : all)
        if (!cf.paired || (c->opts.genotypes_per_warp == 0 && batch_pairable(b, cf))) cands.push_back(cf);
    const size_t gbytes = sizeof(float) * (size_t)b.total * (6 + ADGB_MAX_TORS);
    float *tg = nullptr, *te = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&tg, gbytes);
    if (e == cudaSuccess) e = cudaMalloc(&te, sizeof(float) * (size_t)b.total);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = INFINITY;
    EvalCfg best{};
    for (const EvalCfg &cfg : cands) {
        if (e != cudaSuccess) break;
        const int budget = batch_budget(b, cfg);
        const int grid = items_grid(cfg, budget, c->device);
        if (grid < 1) continue;
        float ms_min = INFINITY;
        for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
            e = cudaMemcpyAsync(tg, genes_dev, gbytes, cudaMemcpyDeviceToDevice, c->stream);
            if (e == cudaSuccess) e = upload_items(b, batch_items(b, cfg, tg, te, iters, 0.8f, 1e-2f), c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
            if (e == cudaSuccess)
                e = launch_eval_items(b.d_items, b.n_items, b.d_ligs, b.d_recs, b.d_counter, cfg, budget,
                                      grid, c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_min = std::min(ms_min, ms);
        }
        if (e == cudaSuccess && ms_min < best_ms) {
            best_ms = ms_min;
            best = cfg;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(tg);
    cudaFree(te);
    if (e != cudaSuccess) return cuda_fail(c, e, "batch_autotune");
    if (!(best_ms < INFINITY)) return fail(c, ADGB_EINVAL, "batch_autotune: no launch shape fits");
    b.cfg = best;
    b.tuned = true;
    if (b.exec) {
        cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
    }
    c->tune_table[tune_key(b)] = best;
    if (chosen) {
        chosen->threads_per_pose = best.tpp;
        chosen->poses_per_block = best.ppb;
        chosen->reduce_variant = best.variant;
        chosen->pair_rounds = c->opts.pair_rounds;
        chosen->genotypes_per_warp = best.paired ? 0 : 1;
    }
    return ADGB_OK;
}
