// Continuous-batching docking server (dock_submit / dock_poll / dock_wait /
// dock_result / dock_cancel).
//
// Every admitted job is an independent chain of launches on a stream of its
// own: its initial population and then one Lamarckian-GA generation after
// another (GA, the generation's local searches, run bests and evaluation
// accounting) - the same kernels, launch shape and order as one dock() call
// of the job, so a served job returns exactly the bits dock() returns.  The
// GPU interleaves the blocks of all active jobs' kernels; no job waits for
// another's generation.
//
// One host thread feeds the streams: it keeps two generations of each job in
// flight (the next one is queued before the previous one's counters have
// been read), reads a generation's evaluation counts and stop flags from
// pinned memory once its event has completed (cudaEventQuery, never a
// stream or device synchronisation), and when a job is done - its generation
// limit, or every run at its evaluation budget or stopped early - queues the
// FP64 rescoring and the copies of the results, publishes them once those
// land, and frees the job's stream-ordered device memory.  A generation
// queued after a job's runs had all stopped changes nothing (stopped runs
// keep their population and do no evaluations).
//
// Admission is first come, first served while the job fits the device's
// live free memory (cudaMemGetInfo plus what the stream-ordered pool holds
// unused, less a reserve), the caller's budget if it set one, and the
// active-job cap (by default: two jobs, more while their local searches
// together need less than two GPUs' worth of resident warps).  Populations, ligands and counters stay on the device
// between generations; random numbers are counter-based (nothing to store).
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
constexpr int IN_FLIGHT = 2;   // generations of a job queued ahead of the host

// A pinned host buffer from the server's pool (host memory that the device
// copies into asynchronously; reused, freed when the server stops).
struct Pinned {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Job {
    long long id = 0;
    int status = JOB_QUEUED;   // JOB_* or ADGB_ECANCELLED / ADGB_EDEVICE (under the server lock)
    std::atomic<bool> cancel{false};
    RecDev rec{};
    LigandBlob blob;
    LigDev lig{};
    DockCfg d{};
    EvalCfg cfg{};
    int G = 0;
    size_t bytes = 0;
    double fill = 0;   // resident warps its local-search launch needs, in GPU-fulls
    // server thread only
    unsigned char *mem = nullptr;
    DockScratch w{};
    float *d_best_genes = nullptr;
    double *d_best_e = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev[IN_FLIGHT] = {}, ev_fin = nullptr;
    Pinned cnt;        // [IN_FLIGHT][runs] evaluation counts, [IN_FLIGHT][runs] stop flags, blob
    Pinned res;        // results: [runs][G] genes, [runs] FP64 energies, [runs] counts,
                       // tensor-core give-up counts [2] at the start and [2] at the end
    int launched = 0;  // generations queued (0 = the initial population)
    int processed = 0; // generations whose counters have been read
    int cur = 0;       // population buffer of the last queued generation
    int gen_done = 0;  // generation at which the job is complete
    bool stop_launch = false, finishing = false, failed = false;
    bool tc_failed = false;   // a tensor-core wait gave up while the job ran (results not valid)
    // published under the server lock
    int gen_pub = 0;
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
    int variant = 0, tpp_opt = 0, ppb_opt = 0, gpw = 0;
    size_t budget = 0;           // the caller's budget (0: live free memory only)
    size_t used = 0;             // device bytes of the admitted jobs
    size_t reserve = 0;          // device memory admission leaves free
    size_t total_mem = 0;
    size_t last_avail = 0;       // the live estimate at the last admission check
    double warps_gpu = 0;        // resident warps of the whole GPU (SMs x 16, the kernels' usual)
    double fill_active = 0;      // sum of the active jobs' fill
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> queue;
    std::vector<Job *> active;
    std::map<long long, std::unique_ptr<Job>> jobs;
    bool stop = false;
    long long next_id = 1;
    std::chrono::steady_clock::time_point t0;
    std::string err;
    std::vector<Pinned> pinned_free;   // server thread only
    std::vector<void *> pinned_all;
    long long ticks = 0, items_run = 0;
    double busy_s = 0;
};

namespace {

Pinned pinned_take(adgb_server *s, size_t bytes) {
    size_t best = (size_t)-1;
    for (size_t i = 0; i < s->pinned_free.size(); i++)
        if (s->pinned_free[i].bytes >= bytes &&
            (best == (size_t)-1 || s->pinned_free[i].bytes < s->pinned_free[best].bytes))
            best = i;
    if (best != (size_t)-1) {
        Pinned p = s->pinned_free[best];
        s->pinned_free.erase(s->pinned_free.begin() + best);
        return p;
    }
    Pinned p;
    if (cudaHostAlloc(&p.p, bytes, cudaHostAllocDefault) == cudaSuccess) {
        p.bytes = bytes;
        s->pinned_all.push_back(p.p);
    } else {
        p.p = nullptr;
    }
    return p;
}

void pinned_give(adgb_server *s, Pinned &p) {
    if (p.p) s->pinned_free.push_back(p);
    p = Pinned{};
}

// Device memory a new job may take now: the free memory, plus what the
// stream-ordered pool holds without using it, less the reserve.
size_t live_available(adgb_server *s) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
    cudaMemPool_t pool;
    unsigned long long reserved = 0, in_use = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &in_use) == cudaSuccess &&
        reserved > in_use)
        free_b += (size_t)(reserved - in_use);
    return free_b > s->reserve ? free_b - s->reserve : 0;
}

// Everything the job holds on the device and in the pools (server thread).
void release_job(adgb_server *s, Job *j) {
    if (j->mem) cudaFreeAsync(j->mem, j->stream);
    j->mem = nullptr;
    for (cudaEvent_t &e : j->ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (j->ev_fin) cudaEventDestroy(j->ev_fin);
    j->ev_fin = nullptr;
    if (j->stream) cudaStreamDestroy(j->stream);   // resources go once its work is done
    j->stream = nullptr;
    if (!j->failed) {   // a failed job's copies may still be in flight: its buffers stay out
        pinned_give(s, j->cnt);
        pinned_give(s, j->res);
    }
}

// The job's tensor-core give-up snapshots (pinned): [0..1] when its first
// launch starts, [2..3] after its last.  The counts are device-wide, so a
// give-up in another job's kernels while this job ran fails this one too.
unsigned int *tc_counts(const Job *j) {
    return (unsigned int *)((char *)j->res.p + al256(4 * (size_t)j->d.n_runs * j->G) +
                            16 * (size_t)j->d.n_runs);
}

// Device state of a newly admitted job: stream, events, memory, pinned
// buffers, ligand blob, initial population.
cudaError_t setup_job(adgb_server *s, Job *j) {
    cudaError_t e = cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking);
    for (int k = 0; k < IN_FLIGHT && e == cudaSuccess; k++)
        e = cudaEventCreateWithFlags(&j->ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->ev_fin, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&j->mem, j->bytes, j->stream);
    if (e != cudaSuccess) return e;
    job_layout(*j, j->mem);
    const int runs = j->d.n_runs;
    j->cnt = pinned_take(s, IN_FLIGHT * (size_t)runs * 12 + j->blob.bytes.size());
    j->res = pinned_take(s, al256(4 * (size_t)runs * j->G) + 16 * (size_t)runs + 16);
    if (!j->cnt.p || !j->res.p) return cudaErrorMemoryAllocation;
    // the ligand blob through pinned memory (an asynchronous copy)
    unsigned char *stage = (unsigned char *)j->cnt.p + IN_FLIGHT * (size_t)runs * 12;
    std::copy(j->blob.bytes.begin(), j->blob.bytes.end(), stage);
    e = cudaMemcpyAsync(j->mem, stage, j->blob.bytes.size(), cudaMemcpyHostToDevice, j->stream);
    if (e == cudaSuccess) e = tc_gave_up_async(tc_counts(j), j->stream);
    if (e == cudaSuccess) e = launch_job_start(j->rec, j->lig.n_tors, j->d, j->w, j->stream);
    return e;
}

long long *cnt_evals(const Job *j, int g) {
    return (long long *)j->cnt.p + (size_t)(g % IN_FLIGHT) * j->d.n_runs;
}
int *cnt_done(const Job *j, int g) {
    return (int *)((long long *)j->cnt.p + (size_t)IN_FLIGHT * j->d.n_runs) +
           (size_t)(g % IN_FLIGHT) * j->d.n_runs;
}

// Queues generation g of a job (g = 0: the initial population's scoring), as
// launch_dock orders it, then the copies of its counters and its event.
cudaError_t queue_generation(adgb_server *s, Job *j, int g) {
    cudaError_t e = cudaSuccess;
    if (g > 0) {
        e = launch_job_ga(j->d, j->G, g, j->w, j->cur, j->stream);
        j->cur ^= 1;
    }
    if (e == cudaSuccess)
        e = launch_dock_ls(j->rec, j->lig, j->cfg, j->d, j->w.genes[j->cur], g, j->w, j->stream);
    if (e == cudaSuccess) e = launch_job_best(j->d, j->G, g, j->w, j->cur, j->d_best_genes, j->stream);
    const int runs = j->d.n_runs;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cnt_evals(j, g), j->w.evals, 8 * (size_t)runs, cudaMemcpyDeviceToHost, j->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cnt_done(j, g), j->w.done, 4 * (size_t)runs, cudaMemcpyDeviceToHost, j->stream);
    if (e == cudaSuccess) e = cudaEventRecord(j->ev[g % IN_FLIGHT], j->stream);
    if (e == cudaSuccess) {
        s->ticks++;
        s->items_run += (long long)j->d.n_runs * j->d.pop;
    }
    return e;
}

// Every run has stopped after generation g: generation limit, evaluation
// budget or early stopping.
bool finished_after(const Job *j, int g) {
    if (g >= j->d.max_gens) return true;
    const long long *h_ev = cnt_evals(j, g);
    const int *h_done = cnt_done(j, g);
    for (int r = 0; r < j->d.n_runs; r++)
        if (h_ev[r] < j->d.max_evals && !h_done[r]) return false;
    return true;
}

void job_error(adgb_server *s, Job *j, cudaError_t e) {
    j->failed = true;
    j->stop_launch = true;
    s->err = std::string("serving: ") + cudaGetErrorString(e);
}

// Advances one active job as far as the device allows without waiting.
// Returns true if anything changed; sets *complete when the job is over
// (results in its vectors, or cancelled / failed) and nothing of it is in
// flight any more.
bool service(adgb_server *s, Job *j, bool *complete) {
    bool progress = false;
    cudaError_t e = cudaSuccess;
    *complete = false;
    if (!j->stream && !j->failed) {
        progress = true;
        if ((e = setup_job(s, j)) != cudaSuccess) job_error(s, j, e);
    }
    // generations whose counters have landed
    while (j->stream && j->processed < j->launched) {
        const cudaError_t q = cudaEventQuery(j->ev[j->processed % IN_FLIGHT]);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) {
            job_error(s, j, q);
            break;
        }
        const int g = j->processed++;
        progress = true;
        if (!j->stop_launch) {
            j->gen_pub = g;
            if (finished_after(j, g)) {
                j->stop_launch = true;
                j->gen_done = g;
            }
        }
    }
    if (j->cancel) j->stop_launch = true;
    // keep IN_FLIGHT generations queued
    while (!j->stop_launch && j->launched - j->processed < IN_FLIGHT && j->launched <= j->d.max_gens) {
        if ((e = queue_generation(s, j, j->launched)) != cudaSuccess) {
            job_error(s, j, e);
            break;
        }
        j->launched++;
        progress = true;
    }
    if (!j->stop_launch || (j->processed < j->launched && !j->failed)) return progress;
    // nothing of the job's generations is in flight any more
    if (j->cancel || j->failed) {
        *complete = true;
        return true;
    }
    const int runs = j->d.n_runs;
    float *h_g = (float *)j->res.p;
    double *h_e = (double *)((char *)j->res.p + al256(4 * (size_t)runs * j->G));
    long long *h_v = (long long *)(h_e + runs);
    if (!j->finishing) {
        e = launch_rescore_fp64(j->rec, j->lig, runs, j->d_best_genes, j->d_best_e, j->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_g, j->d_best_genes, 4 * (size_t)runs * j->G, cudaMemcpyDeviceToHost, j->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_e, j->d_best_e, 8 * (size_t)runs, cudaMemcpyDeviceToHost, j->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_v, j->w.evals, 8 * (size_t)runs, cudaMemcpyDeviceToHost, j->stream);
        if (e == cudaSuccess) e = tc_gave_up_async(tc_counts(j) + 2, j->stream);
        if (e == cudaSuccess) e = cudaEventRecord(j->ev_fin, j->stream);
        if (e != cudaSuccess) {
            job_error(s, j, e);
            *complete = true;
            return true;
        }
        j->finishing = true;
        return true;
    }
    const cudaError_t q = cudaEventQuery(j->ev_fin);
    if (q == cudaErrorNotReady) return progress;
    if (q != cudaSuccess) {
        job_error(s, j, q);
    } else if (const unsigned int *tc = tc_counts(j); tc[0] + tc[1] != tc[2] + tc[3]) {
        j->tc_failed = true;
        s->err = "serving: a tensor-core completion wait gave up while the job ran";
    } else {
        j->best_genes.assign(h_g, h_g + (size_t)runs * j->G);
        j->best_e.assign(h_e, h_e + runs);
        j->evals.assign(h_v, h_v + runs);
    }
    *complete = true;
    return true;
}

void server_loop(adgb_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    double t_busy0 = -1;
    for (;;) {
        // admission in arrival order while memory and the active-job cap allow
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
            // default: two jobs (each fills the other's gaps between its own
            // launches), more while together they fill less than two GPUs'
            // worth of resident warps (measured: more concurrent large jobs
            // only compete for L2 and SMs)
            if (s->opts.max_active_jobs == 0 && s->active.size() >= 2 &&
                s->fill_active + j->fill > 2.0)
                break;
            if (s->budget > 0 && s->used + j->bytes > s->budget) break;
            s->last_avail = live_available(s);
            if (j->bytes > s->last_avail) break;
            s->queue.pop_front();
            s->used += j->bytes;
            s->fill_active += j->fill;
            j->status = JOB_RUNNING;
            j->t_start = now_s(s->t0);
            s->active.push_back(j);
        }
        if (s->active.empty()) {
            if (t_busy0 >= 0) {
                s->busy_s += now_s(s->t0) - t_busy0;
                t_busy0 = -1;
            }
            if (s->stop && s->queue.empty()) break;
            s->cv_work.wait(lk);
            continue;
        }
        if (t_busy0 < 0) t_busy0 = now_s(s->t0);
        std::vector<Job *> act = s->active;
        lk.unlock();
        bool progress = false;
        std::vector<Job *> complete;
        for (Job *j : act) {
            bool done = false;
            progress |= service(s, j, &done);
            if (done) {
                release_job(s, j);
                complete.push_back(j);
            }
        }
        lk.lock();
        for (Job *j : complete) {
            j->status = (j->failed || j->tc_failed)
                            ? (int)ADGB_EDEVICE
                            : (j->cancel ? (int)ADGB_ECANCELLED : (int)JOB_DONE);
            if (j->status == JOB_DONE) j->gen_pub = j->gen_done;
            j->t_finish = now_s(s->t0);
            s->used -= j->bytes;
            s->fill_active -= j->fill;
            s->active.erase(std::find(s->active.begin(), s->active.end(), j));
        }
        if (!complete.empty()) s->cv_done.notify_all();
        if (s->stop) {
            for (Job *j : s->active) j->cancel = true;
            for (Job *j : s->queue) j->cancel = true;
        }
        // nothing to do until a generation lands or a job arrives
        if (!progress && complete.empty()) s->cv_work.wait_for(lk, std::chrono::microseconds(100));
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

int serve_start(adgb_ctx *ctx, const adgb_serve_options *opts, adgb_server **out) {
    if (!ctx || !out) return ADGB_EINVAL;
    *out = nullptr;
    adgb_server *s = new (std::nothrow) adgb_server();
    if (!s) return ADGB_ENOMEM;
    s->ctx = ctx;
    s->device = ctx_device(ctx);
    if (opts) s->opts = *opts;
    const int tpp = s->opts.threads_per_pose, ppb = s->opts.poses_per_block;
    if ((tpp != 0 && tpp != 32 && tpp != 64 && tpp != 128) || ppb < 0 || ppb > 8 ||
        (tpp > 0 && ppb > 0 && tpp * ppb > 128) || s->opts.max_active_jobs < 0 ||
        s->opts.mem_budget_bytes < 0) {
        delete s;
        return ADGB_EINVAL;
    }
    s->variant = s->opts.reduce_variant >= 0 ? s->opts.reduce_variant : ctx_default_variant(ctx);
    if (s->variant >= ADGB_REDUCE_N) {
        delete s;
        return ADGB_EINVAL;
    }
    // the context's launch rule unless the server's options set one
    ctx_launch_opts(ctx, &s->tpp_opt, &s->ppb_opt);
    if (tpp > 0) s->tpp_opt = tpp;
    if (ppb > 0) s->ppb_opt = ppb;
    s->gpw = ctx_genotypes_per_warp(ctx);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    size_t free_b = 0, total_b = 0;
    const cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        delete s;
        return ADGB_EDEVICE;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    s->warps_gpu = 16.0 * (sms > 0 ? sms : 1);
    s->total_mem = total_b;
    s->reserve = std::max<size_t>(total_b / 64, (size_t)256 << 20);
    s->budget = (size_t)s->opts.mem_budget_bytes;
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
    cudaDeviceSynchronize();   // the jobs' stream-ordered frees and copies are done
    for (void *p : s->pinned_all) cudaFreeHost(p);
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
    int rc = dock_cfg_from_params(p, s->variant, j->d, variant, &err);
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
    j->cfg = launch_cfg(j->blob.rel, s->tpp_opt, s->ppb_opt, variant, s->gpw);
    j->bytes = job_layout(*j, nullptr);
    {
        const double genotypes = (double)j->d.n_runs * j->d.pop;
        const double warps = j->cfg.paired ? genotypes / 2 : genotypes * (j->cfg.tpp / 32);
        j->fill = warps / s->warps_gpu;
    }
    const size_t limit = s->budget > 0 ? s->budget
                                       : (s->total_mem > s->reserve ? s->total_mem - s->reserve : 0);
    if (j->bytes > limit) {
        s->err = "dock_submit: the job needs more device memory than the server can ever give it";
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
    out->device_bytes_budget = (long long)(s->budget > 0 ? s->budget : s->used + s->last_avail);
    out->busy_s = s->busy_s;
    out->uptime_s = now_s(s->t0);
    return ADGB_OK;
}

}  // extern "C"
