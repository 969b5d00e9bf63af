// Continuous-batching docking server (dock_submit / dock_poll / dock_wait /
// dock_result / dock_cancel).
//
// One host thread drives the device through its own stream in ticks.  A tick
// advances every active job by one step of its Lamarckian GA: new jobs get
// their initial population, the others one GA generation (per-job launches);
// then ONE persistent multi-ligand local-search launch runs the individuals
// of all active jobs together (work items of the jobs' ligands against their
// receptors); then each job's run bests and evaluation counts are updated.
// A job whose runs are all done is rescored in FP64, its results copied to
// host memory and its device memory released; queued jobs are admitted in
// arrival order as soon as the device-memory budget allows.  Populations,
// ligands, counters and RNG state (counter-based, nothing to store) stay on
// the device between ticks.
//
// A job's arithmetic does not depend on the other jobs in the launch: the
// kernels are per individual, the shared-memory layout of a ligand depends
// on the ligand alone, and the GA stream is keyed by the job's seed.  A job
// therefore returns the same bits alone and in any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "adgb_internal.cuh"

using namespace adgb;

namespace {

enum { JOB_QUEUED = 1, JOB_RUNNING = 2, JOB_DONE = 0 };
// ligand-size classes of the local-search launches: two genotypes a warp
// (pair_eligible ligands), then 32, 64 and 128 threads a genotype
constexpr int NCLS = 4;

struct Job {
    long long id = 0;
    int status = JOB_QUEUED;   // JOB_* or ADGB_ECANCELLED / ADGB_EDEVICE (under the server lock)
    std::atomic<bool> cancel{false};
    RecDev rec{};
    LigandBlob blob;
    LigDev lig{};
    DockCfg d{};
    int G = 0, cur = 0, gen = -1;   // gen -1: initial population not yet scored (server thread)
    int gen_pub = 0;                // generations done, published under the server lock
    size_t bytes = 0;
    unsigned char *mem = nullptr;
    DockScratch w{};
    float *d_best_genes = nullptr;
    double *d_best_e = nullptr;
    long long *h_evals = nullptr;   // pinned, per run; followed by the runs' stop flags (int)
    std::vector<float> best_genes;
    std::vector<double> best_e;
    std::vector<long long> evals;
    double t_submit = 0, t_start = -1, t_finish = -1;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// device bytes of a job: ligand blob, populations and counters, results
size_t job_layout(Job &j, unsigned char *base) {
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = al256(off + b); return o; };
    const int n = j.d.n_runs * j.d.pop, runs = j.d.n_runs, G = j.G;
    const size_t ob = take(j.blob.bytes.size());
    const size_t og0 = take(4 * (size_t)n * G), og1 = take(4 * (size_t)n * G), oe = take(4 * (size_t)n),
                 oi = take(4 * (size_t)n), obe = take(4 * (size_t)runs), ov = take(8 * (size_t)runs),
                 od = take(4 * (size_t)runs), obg = take(4 * (size_t)runs * G), ore = take(8 * (size_t)runs);
    if (base) {
        j.lig = bind_ligand(j.blob, base + ob);
        j.w.genes[0] = (float *)(base + og0);
        j.w.genes[1] = (float *)(base + og1);
        j.w.energy = (float *)(base + oe);
        j.w.iters = (int *)(base + oi);
        j.w.best_e = (float *)(base + obe);
        j.w.evals = (long long *)(base + ov);
        j.w.done = (int *)(base + od);
        j.d_best_genes = (float *)(base + obg);
        j.d_best_e = (double *)(base + ore);
    }
    return off;
}

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct adgb_server {
    adgb_ctx *ctx = nullptr;
    int device = 0;
    adgb_serve_options opts{};
    EvalCfg cfg{32, 4, 0, 1, 0};
    bool forced_shape = false;   // threads/poses a block set by the caller: one class (and
                                 // the two-genotypes-a-warp class for eligible ligands)
    bool paired = true;          // two genotypes a warp where the ligand qualifies
    size_t budget = 0, used = 0;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> queue;
    std::vector<Job *> active;
    std::map<long long, std::unique_ptr<Job>> jobs;
    bool stop = false;
    long long next_id = 1;
    cudaStream_t stream = nullptr;
    // the size classes' local-search launches run concurrently, one stream
    // each, between two events of the main stream (tables ready / all done)
    cudaStream_t cls_stream[NCLS] = {};
    cudaEvent_t ev_tables = nullptr, ev_cls[NCLS] = {};
    std::chrono::steady_clock::time_point t0;
    std::string err;
    // per-tick tables (pinned staging, device copies)
    WorkItem *h_items = nullptr, *d_items = nullptr;
    LigDev *h_ligs = nullptr, *d_ligs = nullptr;
    RecDev *h_recs = nullptr, *d_recs = nullptr;
    int cap_items = 0, cap_jobs = 0;
    int *d_counter = nullptr;        // 2 ints per size class (work counter, finished blocks)
    long long ticks = 0, items_run = 0;
    double busy_s = 0;
};

namespace {

cudaError_t grow_tables(adgb_server *s, int items, int njobs) {
    cudaError_t e = cudaSuccess;
    if (items > s->cap_items) {
        const int cap = std::max(items, 2 * s->cap_items);
        if (s->h_items) cudaFreeHost(s->h_items);
        if (s->d_items) cudaFree(s->d_items);
        s->h_items = nullptr;
        s->d_items = nullptr;
        e = cudaHostAlloc((void **)&s->h_items, sizeof(WorkItem) * cap, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_items, sizeof(WorkItem) * cap);
        if (e != cudaSuccess) return e;
        s->cap_items = cap;
    }
    if (njobs > s->cap_jobs) {
        const int cap = std::max(njobs, 2 * s->cap_jobs);
        if (s->h_ligs) cudaFreeHost(s->h_ligs);
        if (s->h_recs) cudaFreeHost(s->h_recs);
        if (s->d_ligs) cudaFree(s->d_ligs);
        if (s->d_recs) cudaFree(s->d_recs);
        s->h_ligs = nullptr;
        s->h_recs = nullptr;
        s->d_ligs = nullptr;
        s->d_recs = nullptr;
        e = cudaHostAlloc((void **)&s->h_ligs, sizeof(LigDev) * cap, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_recs, sizeof(RecDev) * cap, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_ligs, sizeof(LigDev) * cap);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_recs, sizeof(RecDev) * cap);
        if (e != cudaSuccess) return e;
        s->cap_jobs = cap;
    }
    return e;
}

void release_job_device(adgb_server *s, Job *j) {
    if (j->mem) cudaFreeAsync(j->mem, s->stream);
    if (j->h_evals) cudaFreeHost(j->h_evals);
    j->mem = nullptr;
    j->h_evals = nullptr;
}

// One tick over the active jobs (device work on the server's stream).
cudaError_t tick(adgb_server *s, std::vector<Job *> &act) {
    cudaError_t e = cudaSuccess;
    // admission work and GA generations
    for (Job *j : act) {
        if (j->gen < 0) {
            if (!j->mem) {
                e = cudaMallocAsync((void **)&j->mem, j->bytes, s->stream);
                if (e != cudaSuccess) return e;
                job_layout(*j, j->mem);
                e = cudaMemcpyAsync(j->mem, j->blob.bytes.data(), j->blob.bytes.size(),
                                    cudaMemcpyHostToDevice, s->stream);
                if (e == cudaSuccess)
                    e = cudaHostAlloc((void **)&j->h_evals, 12 * (size_t)j->d.n_runs, cudaHostAllocDefault);
                if (e == cudaSuccess) e = launch_job_start(j->rec, j->lig.n_tors, j->d, j->w, s->stream);
                if (e != cudaSuccess) return e;
            }
        } else {
            e = launch_job_ga(j->d, j->G, j->gen + 1, j->w, j->cur, s->stream);
            if (e != cudaSuccess) return e;
        }
    }
    // multi-ligand local-search launches over every active individual: one
    // per size class (threads a genotype as for a single-ligand call),
    // each a persistent launch over that class's work items (a job's class
    // depends on its ligand alone)
    std::vector<int> cls(act.size());
    EvalCfg ccfg[NCLS];
    for (int c = 0; c < NCLS; c++) {
        ccfg[c] = s->cfg;
        ccfg[c].paired = 0;
        if (!s->forced_shape && c > 0) {
            ccfg[c].tpp = 32 << (c - 1);
            ccfg[c].ppb = 128 / ccfg[c].tpp;
        }
    }
    ccfg[0].tpp = 32;   // two genotypes a warp, the single-ligand calls' shape
    ccfg[0].ppb = s->forced_shape ? s->cfg.ppb : 4;
    ccfg[0].paired = 1;
    int n_items = 0;
    for (size_t u = 0; u < act.size(); u++) {
        const LigDev &l = act[u]->lig;
        const int t = s->forced_shape ? s->cfg.tpp : threads_for_atoms(l.n_atoms);
        const bool pair = s->paired && pair_eligible(l.n_atoms, l.n_tors, l.n_pairs, l.n_rounds,
                                                     l.r_lanes, t);
        cls[u] = pair ? 0 : (s->forced_shape ? 1 : (t == 32 ? 1 : (t == 64 ? 2 : 3)));
        n_items += (act[u]->d.n_runs * act[u]->d.pop + ccfg[cls[u]].ppb - 1) / ccfg[cls[u]].ppb;
    }
    e = grow_tables(s, n_items, (int)act.size());
    if (e != cudaSuccess) return e;
    for (size_t u = 0; u < act.size(); u++) {
        s->h_ligs[u] = act[u]->lig;
        s->h_recs[u] = act[u]->rec;
    }
    int k = 0, first[NCLS], count[NCLS], budget[NCLS];
    for (int c = 0; c < NCLS; c++) {
        first[c] = k;
        budget[c] = 1024;
        const EvalCfg &cf = ccfg[c];
        for (size_t u = 0; u < act.size(); u++) {
            if (cls[u] != c) continue;
            Job *j = act[u];
            const int src = j->gen < 0 ? 0 : (j->cur ^ 1);   // population the LS works on
            budget[c] = std::max(budget[c], items_layout_bytes(cf, j->lig.n_atoms, j->lig.n_tors,
                                                               j->lig.n_pairs));
            const int n = j->d.n_runs * j->d.pop;
            const int cost = j->lig.n_pairs + 8 * j->lig.n_atoms + 64;
            for (int p = 0; p < n; p += cf.ppb) {
                WorkItem &w = s->h_items[k++];
                w.lig = (int)u;
                w.rec = (int)u;
                w.count = std::min(cf.ppb, n - p);
                w.gstride = j->G;
                w.genes = j->w.genes[src] + (size_t)p * j->G;
                w.energy = j->w.energy + p;
                w.iters = j->w.iters + p;
                w.iters_all = 0;
                w.cost = cost;
                w.rho = j->d.rho;
                w.eps = j->d.eps;
            }
        }
        count[c] = k - first[c];
        std::stable_sort(s->h_items + first[c], s->h_items + k, [](const WorkItem &x, const WorkItem &y) {
            return x.cost > y.cost;
        });
    }
    e = cudaMemcpyAsync(s->d_items, s->h_items, sizeof(WorkItem) * n_items, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_ligs, s->h_ligs, sizeof(LigDev) * act.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_recs, s->h_recs, sizeof(RecDev) * act.size(), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return e;
    // one persistent launch per size class, concurrently: a class with few
    // items no longer leaves the GPU idle while it drains
    e = cudaEventRecord(s->ev_tables, s->stream);
    if (e != cudaSuccess) return e;
    for (int c = 0; c < NCLS; c++) {
        if (!count[c]) continue;
        const int grid = items_grid(ccfg[c], budget[c], s->device);
        if (grid < 1) return cudaErrorInvalidConfiguration;
        e = cudaStreamWaitEvent(s->cls_stream[c], s->ev_tables, 0);
        if (e == cudaSuccess)
            e = launch_eval_items(s->d_items + first[c], count[c], s->d_ligs, s->d_recs,
                                  s->d_counter + 2 * c, ccfg[c], budget[c], grid, s->cls_stream[c]);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev_cls[c], s->cls_stream[c]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev_cls[c], 0);
        if (e != cudaSuccess) return e;
    }
    s->items_run += n_items;
    // accounting per job
    for (Job *j : act) {
        const int src = j->gen < 0 ? 0 : (j->cur ^ 1);
        e = launch_job_best(j->d, j->G, j->gen < 0 ? 0 : j->gen + 1, j->w, src, j->d_best_genes,
                            s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(j->h_evals, j->w.evals, 8 * j->d.n_runs, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(j->h_evals + j->d.n_runs, j->w.done, 4 * j->d.n_runs,
                                cudaMemcpyDeviceToHost, s->stream);
        if (e != cudaSuccess) return e;
    }
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return e;
    for (Job *j : act) {
        if (j->gen >= 0) j->cur ^= 1;
        j->gen += 1;
    }
    return cudaSuccess;
}

// Every run has stopped: generation limit, evaluation budget or early stopping.
bool job_finished(const Job *j) {
    if (j->gen >= j->d.max_gens) return true;
    const int *stopped = reinterpret_cast<const int *>(j->h_evals + j->d.n_runs);
    for (int r = 0; r < j->d.n_runs; r++)
        if (j->h_evals[r] < j->d.max_evals && !stopped[r]) return false;
    return true;
}

cudaError_t finish_job(adgb_server *s, Job *j) {
    cudaError_t e = launch_rescore_fp64(j->rec, j->lig, j->d.n_runs, j->d_best_genes, j->d_best_e, s->stream);
    j->best_genes.resize((size_t)j->d.n_runs * j->G);
    j->best_e.resize(j->d.n_runs);
    j->evals.resize(j->d.n_runs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(j->best_genes.data(), j->d_best_genes, 4 * j->best_genes.size(),
                            cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(j->best_e.data(), j->d_best_e, 8 * j->best_e.size(), cudaMemcpyDeviceToHost,
                            s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(j->evals.data(), j->w.evals, 8 * j->evals.size(), cudaMemcpyDeviceToHost,
                            s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e;
}

void server_loop(adgb_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // admission in arrival order while the memory budget allows
        while (!s->queue.empty()) {
            Job *j = s->queue.front();
            if (j->cancel) {
                s->queue.pop_front();
                j->status = ADGB_ECANCELLED;
                j->t_finish = now_s(s->t0);
                s->cv_done.notify_all();
                continue;
            }
            if (s->opts.max_active_jobs > 0 && (int)s->active.size() >= s->opts.max_active_jobs) break;
            if (s->used + j->bytes > s->budget) break;
            s->queue.pop_front();
            s->used += j->bytes;
            j->status = JOB_RUNNING;
            j->t_start = now_s(s->t0);
            s->active.push_back(j);
        }
        if (s->active.empty()) {
            if (s->stop && s->queue.empty()) break;
            s->cv_work.wait(lk);
            continue;
        }
        std::vector<Job *> act = s->active;
        lk.unlock();
        const double t_tick = now_s(s->t0);
        cudaError_t e = tick(s, act);
        std::vector<Job *> finished;
        if (e == cudaSuccess) {
            for (Job *j : act)
                if (j->cancel || job_finished(j)) finished.push_back(j);
            for (Job *j : finished)
                if (!j->cancel && e == cudaSuccess) e = finish_job(s, j);
        }
        for (Job *j : (e == cudaSuccess ? finished : act)) release_job_device(s, j);
        cudaStreamSynchronize(s->stream);
        lk.lock();
        s->busy_s += now_s(s->t0) - t_tick;
        s->ticks++;
        for (Job *j : act) j->gen_pub = j->gen < 0 ? 0 : j->gen;
        if (e != cudaSuccess) {
            s->err = std::string("serving tick: ") + cudaGetErrorString(e);
            finished = act;
        }
        for (Job *j : finished) {
            j->status = e != cudaSuccess ? (int)ADGB_EDEVICE
                                         : (j->cancel ? (int)ADGB_ECANCELLED : (int)JOB_DONE);
            j->t_finish = now_s(s->t0);
            s->used -= j->bytes;
            s->active.erase(std::find(s->active.begin(), s->active.end(), j));
        }
        if (!finished.empty()) s->cv_done.notify_all();
        if (s->stop) {
            for (Job *j : s->active) j->cancel = true;
            for (Job *j : s->queue) j->cancel = true;
        }
    }
}

void fill_info(const adgb_server *s, const Job *j, adgb_job_info *info) {
    if (!info) return;
    info->status = j->status;
    info->n_runs = j->d.n_runs;
    info->n_genes = j->G;
    info->generations = j->gen_pub;
    long long ev = 0;
    if (j->status == JOB_DONE)   // results are complete before the status is published
        for (long long v : j->evals) ev += v;
    info->evals = ev;
    info->submit_s = j->t_submit;
    info->start_s = j->t_start;
    info->finish_s = j->t_finish;
    (void)s;
}

}  // namespace

extern "C" {

static void release_streams(adgb_server *s) {
    for (int c = 0; c < NCLS; c++) {
        if (s->cls_stream[c]) cudaStreamDestroy(s->cls_stream[c]);
        if (s->ev_cls[c]) cudaEventDestroy(s->ev_cls[c]);
        s->cls_stream[c] = nullptr;
        s->ev_cls[c] = nullptr;
    }
    if (s->ev_tables) cudaEventDestroy(s->ev_tables);
    if (s->d_counter) cudaFree(s->d_counter);
    if (s->stream) cudaStreamDestroy(s->stream);
    s->ev_tables = nullptr;
    s->d_counter = nullptr;
    s->stream = nullptr;
}

int serve_start(adgb_ctx *ctx, const adgb_serve_options *opts, adgb_server **out) {
    if (!ctx || !out) return ADGB_EINVAL;
    *out = nullptr;
    adgb_server *s = new (std::nothrow) adgb_server();
    if (!s) return ADGB_ENOMEM;
    s->ctx = ctx;
    s->device = ctx_device(ctx);
    if (opts) s->opts = *opts;
    const int tpp = s->opts.threads_per_pose > 0 ? s->opts.threads_per_pose : 32;
    int ppb = s->opts.poses_per_block > 0 ? s->opts.poses_per_block : 128 / tpp;
    if ((tpp != 32 && tpp != 64 && tpp != 128) || ppb < 1 || tpp * ppb > 128 ||
        s->opts.max_active_jobs < 0 || s->opts.mem_budget_bytes < 0) {
        delete s;
        return ADGB_EINVAL;
    }
    const int variant = s->opts.reduce_variant >= 0 ? s->opts.reduce_variant : ctx_default_variant(ctx);
    if (variant >= ADGB_REDUCE_N) {
        delete s;
        return ADGB_EINVAL;
    }
    s->cfg = EvalCfg{tpp, ppb, variant, 1, 0};
    s->forced_shape = s->opts.threads_per_pose > 0 || s->opts.poses_per_block > 0;
    s->paired = ctx_genotypes_per_warp(ctx) == 0;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    for (int c = 0; c < NCLS && e == cudaSuccess; c++) {
        e = cudaStreamCreateWithFlags(&s->cls_stream[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_cls[c], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_tables, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_counter, 2 * NCLS * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(s->d_counter, 0, 2 * NCLS * sizeof(int));
    if (e != cudaSuccess) {
        release_streams(s);
        if (prev >= 0) cudaSetDevice(prev);
        delete s;
        return ADGB_EDEVICE;
    }
    if (prev >= 0) cudaSetDevice(prev);
    s->budget = s->opts.mem_budget_bytes > 0 ? (size_t)s->opts.mem_budget_bytes : free_b / 4;
    s->t0 = std::chrono::steady_clock::now();
    s->th = std::thread(server_loop, s);
    *out = s;
    return ADGB_OK;
}

int serve_stop(adgb_server *s) {
    if (!s) return ADGB_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Job *j : s->queue) j->cancel = true;
        for (Job *j : s->active) j->cancel = true;
    }
    s->cv_work.notify_all();
    s->th.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
    if (s->h_items) cudaFreeHost(s->h_items);
    if (s->h_ligs) cudaFreeHost(s->h_ligs);
    if (s->h_recs) cudaFreeHost(s->h_recs);
    cudaFree(s->d_items);
    cudaFree(s->d_ligs);
    cudaFree(s->d_recs);
    release_streams(s);
    if (prev >= 0) cudaSetDevice(prev);
    s->cv_done.notify_all();
    delete s;
    return ADGB_OK;
}

const char *serve_last_error(adgb_server *s) { return s ? s->err.c_str() : "null server"; }

int dock_submit(adgb_server *s, int receptor_id, const adgb_ligand_desc *lig,
                const adgb_dock_params *p, long long *job_id) {
    if (!s || !job_id) return ADGB_EINVAL;
    std::unique_ptr<Job> j(new (std::nothrow) Job());
    if (!j) return ADGB_ENOMEM;
    std::string err;
    int variant = 0;
    int rc = dock_cfg_from_params(p, s->cfg.variant, j->d, variant, &err);
    if (rc == ADGB_OK && j->d.ls_method != 0) {
        rc = ADGB_EINVAL;
        err = "dock_submit: the serving loop runs the ADADELTA local search only";
    }
    if (rc == ADGB_OK) rc = make_ligand_blob(&err, lig, ctx_pair_rounds(s->ctx), j->blob);
    int n_type_maps = 0;
    if (rc == ADGB_OK && ctx_receptor(s->ctx, receptor_id, &j->rec, &n_type_maps) != ADGB_OK) {
        rc = ADGB_ENOTFOUND;
        err = "unknown receptor id";
    }
    if (rc == ADGB_OK && j->blob.max_type >= n_type_maps) {
        rc = ADGB_EINVAL;
        err = "ligand type without a receptor map";
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (rc != ADGB_OK) {
        s->err = "dock_submit: " + err;
        return rc;
    }
    j->G = 6 + j->blob.rel.n_tors;
    j->bytes = job_layout(*j, nullptr);
    if (j->bytes > s->budget) {
        s->err = "dock_submit: the job needs more device memory than the server's budget";
        return ADGB_EREJECTED;
    }
    if (s->stop) {
        s->err = "dock_submit: server is stopping";
        return ADGB_EREJECTED;
    }
    j->id = s->next_id++;
    j->t_submit = now_s(s->t0);
    Job *raw = j.get();
    s->jobs[raw->id] = std::move(j);
    s->queue.push_back(raw);
    *job_id = raw->id;
    s->cv_work.notify_all();
    return ADGB_OK;
}

int dock_poll(adgb_server *s, long long job_id, adgb_job_info *info) {
    if (!s) return ADGB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return ADGB_ENOTFOUND;
    fill_info(s, it->second.get(), info);
    return ADGB_OK;
}

int dock_wait(adgb_server *s, long long job_id, int timeout_ms, adgb_job_info *info) {
    if (!s) return ADGB_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return ADGB_ENOTFOUND;
    Job *j = it->second.get();
    auto pending = [&] { return j->status == JOB_QUEUED || j->status == JOB_RUNNING; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, [&] { return !pending(); });
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !pending(); })) {
        fill_info(s, j, info);
        return ADGB_ETIMEOUT;
    }
    fill_info(s, j, info);
    return ADGB_OK;
}

int dock_result(adgb_server *s, long long job_id, float *best_genes, double *best_energy,
                long long *evals) {
    if (!s) return ADGB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return ADGB_ENOTFOUND;
    Job *j = it->second.get();
    if (j->status == JOB_QUEUED || j->status == JOB_RUNNING) return ADGB_ETIMEOUT;
    if (j->status != JOB_DONE) return j->status;
    if (best_genes) std::copy(j->best_genes.begin(), j->best_genes.end(), best_genes);
    if (best_energy) std::copy(j->best_e.begin(), j->best_e.end(), best_energy);
    if (evals) std::copy(j->evals.begin(), j->evals.end(), evals);
    return ADGB_OK;
}

int dock_cancel(adgb_server *s, long long job_id) {
    if (!s) return ADGB_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return ADGB_ENOTFOUND;
        it->second->cancel = true;
    }
    s->cv_work.notify_all();
    return ADGB_OK;
}

int dock_forget(adgb_server *s, long long job_id) {
    if (!s) return ADGB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return ADGB_ENOTFOUND;
    const int st = it->second->status;
    if (st == JOB_QUEUED || st == JOB_RUNNING) return ADGB_EINVAL;
    s->jobs.erase(it);
    return ADGB_OK;
}

int serve_stats(adgb_server *s, adgb_serve_stats *out) {
    if (!s || !out) return ADGB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->queued = (int)s->queue.size();
    out->active = (int)s->active.size();
    out->ticks = s->ticks;
    out->items_run = s->items_run;
    out->device_bytes_in_use = (long long)s->used;
    out->device_bytes_budget = (long long)s->budget;
    out->busy_s = s->busy_s;
    out->uptime_s = now_s(s->t0);
    return ADGB_OK;
}

}  // extern "C"
