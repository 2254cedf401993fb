// queue.cu -- many CSC solves of uneven size in one persistent launch.
//
// A persistent grid (two CTAs per SM) drains a device-side queue of LGCD jobs
// (one job = one image, solved by Alg. 3 over a grid of tiles with the
// global-memory worker).  The jobs' tiles are numbered consecutively
// ("slots"); a CTA takes the next slot with one atomic, runs the worker of
// that tile, and takes another when the job ends.  A job starts only when all
// of its tiles are held (the worker's termination protocol needs every tile of
// the image at once): a CTA that holds a tile of a job not yet fully taken
// waits.  Slots are taken in order and a job never has more tiles than the
// grid has CTAs, so the job at the front of the queue always fills up: CTAs of
// the jobs ahead of it finish, because those jobs depend on nothing else.
//
// The host appends jobs while the kernel runs: it writes the job entry and the
// job's control words (header, per-tile flag counters) with copies on a side
// stream, then the new job count; the kernel reads the count with acquire
// loads.  The last CTA to leave a job writes the job's statistics and a
// completion word to pinned host memory (system-scope release), which the
// host polls without CUDA calls.  A close word ends the kernel once the queue
// is empty.  Every wait is bounded by the kernel's deadline.
#include <algorithm>
#include <atomic>
#include <vector>

#include "lgcd_global.cuh"

namespace csc {

struct QueueCtl {       // device control words (host-written njobs / close)
    int njobs;
    int pad0[31];
    int close;
    int pad1[31];
    int slot;           // next slot to take
    int pad2[31];
    int drain;          // 1: every job was published before the launch; a CTA
    int pad3[31];       //    whose slot lies past the last job's tiles exits
};

struct QueueJob {       // device job table entry
    LgcdArgs<float> a;
    int prefix;         // first slot of the job
    int W;              // tiles
    int claimed;        // tiles taken so far (device counter, zeroed by the host)
    int done;           // tiles finished
};

struct QueueHostSlot {  // pinned host memory, one per job
    int complete;       // 0 running, 1 done (written last)
    int status;
    long long updates, iterations, rejected, subtol, messages, max_iters;
    unsigned long long t_ns;  // device time from the first tile's start to the end
    unsigned long long t_start;
};

// CTAs of 256 threads, two or three per SM.  Each SM sub-partition holds
// 16,384 registers and receives two warps of every CTA:
//   two CTAs at <= 72 registers a thread hold 9,216 of them and leave room for
//   the tensor-core beta-init (two warps of <= 104 registers);
//   three CTAs at <= 64 registers hold 12,288 and leave room only for the FP32
//   correlations and the refresh kernels (one warp of <= 112 registers);
// and nearly all of every SM's shared memory stays free for those kernels.
constexpr int kQueueThreads = 256;
constexpr int kQueueCtasPerSmDefault = 2;

// A job-table entry copied to shared memory through L2 (all threads of the
// CTA, one word each).  The host writes entries while the kernel runs, and
// neighbouring entries share cache lines: a plain load could return an L1 line
// cached before the host's copy landed.
template <typename T>
__device__ __forceinline__ void stage_l2(T *dst, const T *src) {
    static_assert(sizeof(T) % 4 == 0 && sizeof(T) / 4 <= kQueueThreads, "one word per thread");
    if (threadIdx.x < sizeof(T) / 4)
        reinterpret_cast<unsigned *>(dst)[threadIdx.x] = __ldcg(reinterpret_cast<const unsigned *>(src) + threadIdx.x);
}

__device__ __forceinline__ void st_release_sys(int *p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// REGS: the register cap of the grid's density; RB: the worker's row block.
// Under 64 registers RB = 4 spills about 100 bytes a thread and RB = 2 none,
// yet RB = 4 served the 512-request trace at 165 solves/s against 134: the
// loads in flight per unit matter more than the spill traffic.
template <int REGS, int RB>
__global__ void __maxnreg__(REGS) lgcd_queue_kernel(QueueCtl *qc, QueueJob *jobs, int max_jobs,
                                                                      QueueHostSlot *host,
                                                                      unsigned long long run_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_state, s_job, s_tile;
    __shared__ LgcdArgs<float> s_args;
    const unsigned long long t_end = globaltimer_ns() + run_ns;
    for (;;) {
        if (threadIdx.x == 0) {
            const int s = atomicAdd(&qc->slot, 1);
            int state = 0, j = -1;
            for (;;) {
                const int nj = min(ld_acquire(&qc->njobs), max_jobs);
                if (nj > 0) {
                    const QueueJob &last = jobs[nj - 1];
                    if (s < ld_relaxed(&last.prefix) + ld_relaxed(&last.W)) {
                        // binary search for the job holding slot s
                        int lo = 0, hi = nj - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) / 2;
                            if (ld_relaxed(&jobs[mid].prefix) <= s) lo = mid;
                            else hi = mid - 1;
                        }
                        j = lo;
                        break;
                    }
                }
                if (ld_acquire(&qc->close)) {
                    state = 1;
                    break;
                }
                if (ld_relaxed(&qc->drain)) {  // no job will follow: nothing left for slot s
                    state = 1;
                    break;
                }
                if (globaltimer_ns() > t_end) {
                    state = 2;
                    break;
                }
                __nanosleep(1000);
            }
            if (state == 0) {
                // wait until every tile of the job is held
                const int W = ld_relaxed(&jobs[j].W);
                const int got = atomicAdd(&jobs[j].claimed, 1) + 1;
                if (got == 1) host[j].t_start = globaltimer_ns();
                while (ld_acquire(&jobs[j].claimed) < W) {
                    if (globaltimer_ns() > t_end) {
                        state = 2;
                        break;
                    }
                    __nanosleep(200);
                }
                s_job = j;
                s_tile = s - ld_relaxed(&jobs[j].prefix);
            }
            s_state = state;
        }
        __syncthreads();
        if (s_state) break;
        const int j = s_job;
        stage_l2(&s_args, &jobs[j].a);
        __syncthreads();
        global_tile_worker<float, kQueueThreads, RB>(s_args, s_tile, smem_raw);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(&jobs[j].done, 1) == ld_relaxed(&jobs[j].W) - 1) {
                // last tile of the job: statistics, then the completion word
                WsHeader *h = s_args.hdr;
                QueueHostSlot *hs = host + j;
                hs->status = ld_relaxed(&h->stop);
                hs->updates = (long long)atomicAdd((unsigned long long *)&h->stat[ST_UPDATES], 0ull);
                hs->iterations = (long long)atomicAdd((unsigned long long *)&h->stat[ST_ITERS], 0ull);
                hs->rejected = (long long)atomicAdd((unsigned long long *)&h->stat[ST_REJECTED], 0ull);
                hs->subtol = (long long)atomicAdd((unsigned long long *)&h->stat[ST_SUBTOL], 0ull);
                hs->messages = (long long)atomicAdd((unsigned long long *)&h->stat[ST_MESSAGES], 0ull);
                hs->max_iters = (long long)atomicAdd(&h->wmax[0], 0ull);
                hs->t_ns = globaltimer_ns() - hs->t_start;
                __threadfence_system();
                st_release_sys(&hs->complete, 1);
            }
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------- host side
struct Queue {
    Geom atoms;                  // P, K, L0, L1 (d = 2 view), T / Z unused
    const float *D = nullptr, *dtd = nullptr;
    double *nrm = nullptr, *dmax = nullptr;
    unsigned char *dev = nullptr;
    QueueCtl *qc = nullptr;
    QueueJob *jobs = nullptr;
    unsigned char *ctl_pool = nullptr;  // per control slot: header + flag counters
    size_t ctl_stride = 0;
    QueueHostSlot *host = nullptr;
    int max_jobs = 0, ctl_slots = 0, grid = 0, njobs = 0, next_slot = 0, ctas_per_sm = 2;
    std::vector<int> job_ctl;    // control slot of each job (-1 once released)
    std::vector<int> free_ctl;
    csc_solve_opts opts;
    cudaStream_t kstream = nullptr, sstream = nullptr;
    // deferred start: the kernel's launch arguments, kept until csc_queue_start
    bool launched = false, drain = false;
    const void *kern = nullptr;
    unsigned long long run_ns = 0;
};

static size_t q_align(size_t x) { return (x + 255) & ~(size_t)255; }

struct QueueLayout {
    size_t ctl, jobs, nrm, dmax, pool, stride, total, host;
};

static QueueLayout queue_layout(const Geom &g, int max_jobs, int ctl_slots, int grid) {
    QueueLayout L{};
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t at = off;
        off = q_align(off + b);
        return at;
    };
    L.ctl = take(sizeof(QueueCtl));
    L.jobs = take((size_t)max_jobs * sizeof(QueueJob));
    L.nrm = take((size_t)g.K * sizeof(double));
    L.dmax = take((size_t)g.K * sizeof(double));
    L.stride = q_align(sizeof(WsHeader) + (size_t)grid * kDirs * 32 * sizeof(int));
    L.pool = take((size_t)ctl_slots * L.stride);
    L.total = off;
    L.host = (size_t)max_jobs * sizeof(QueueHostSlot);
    return L;
}

static std::atomic<int> g_live_queues{0};
int live_queues() { return g_live_queues.load(); }

static int queue_grid(int ctas_per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 152;
    }
    return ctas_per_sm * sms;
}

// 0 selects the default; anything but 2 or 3 is invalid
static int queue_density(int ctas_per_sm) {
    if (ctas_per_sm == 0) return kQueueCtasPerSmDefault;
    return ctas_per_sm == 2 || ctas_per_sm == 3 ? ctas_per_sm : -1;
}

static const void *queue_kernel(int ctas_per_sm) {
    return ctas_per_sm == 3 ? (const void *)lgcd_queue_kernel<64, 4> : (const void *)lgcd_queue_kernel<72, 4>;
}

static int atoms_geom(const csc_shape *atoms, Geom *g) {
    if (!atoms || atoms->d != 2) return CSC_ERR_INVALID;
    csc_shape s = *atoms;
    s.T[0] = atoms->L[0];
    s.T[1] = atoms->L[1];
    return make_geom(&s, g);
}

}  // namespace csc

using namespace csc;

struct csc_queue : Queue {};

extern "C" {

int csc_queue_workspace_size(const csc_shape *atoms, int max_jobs, int ctl_slots, int ctas_per_sm,
                             size_t *device_bytes, size_t *host_bytes) {
    Geom g;
    int rc = atoms_geom(atoms, &g);
    if (rc) return rc;
    const int dens = queue_density(ctas_per_sm);
    if (max_jobs < 1 || ctl_slots < 1 || dens < 0 || !device_bytes || !host_bytes) return CSC_ERR_INVALID;
    const QueueLayout L = queue_layout(g, max_jobs, ctl_slots, queue_grid(dens));
    *device_bytes = L.total;
    *host_bytes = L.host;
    return CSC_OK;
}

static int queue_launch(csc_queue *q) {
    const size_t smem = 2 * (size_t)q->atoms.K * sizeof(float);
    QueueCtl *qc = q->qc;
    QueueJob *jobs = q->jobs;
    QueueHostSlot *host = q->host;
    int max_jobs = q->max_jobs;
    unsigned long long run_ns = q->run_ns;
    void *args[] = {&qc, &jobs, &max_jobs, &host, &run_ns};
    const cudaError_t e = cudaLaunchKernel(q->kern, dim3(q->grid), dim3(kQueueThreads), args, smem, q->kstream);
    if (e != cudaSuccess) return set_cuda_error(e);
    q->launched = true;
    g_live_queues.fetch_add(1);
    return CSC_OK;
}

static int queue_create(const csc_shape *atoms, const float *D, const float *dtd, const csc_solve_opts *opts,
                        int max_jobs, int ctl_slots, int ctas_per_sm, void *device_ws, size_t device_bytes,
                        void *host_ws, size_t host_bytes, double run_seconds, csc_stream_t kernel_stream,
                        csc_stream_t side_stream, bool launch, csc_queue **out) {
    Geom g;
    int rc = atoms_geom(atoms, &g);
    if (rc) return rc;
    const int dens = queue_density(ctas_per_sm);
    if (!D || !dtd || !device_ws || !host_ws || !out || max_jobs < 1 || ctl_slots < 1 || dens < 0 ||
        !(run_seconds > 0.0))
        return CSC_ERR_INVALID;
    const int grid = queue_grid(dens);
    const void *kern = queue_kernel(dens);
    const QueueLayout L = queue_layout(g, max_jobs, ctl_slots, grid);
    if (device_bytes < L.total || host_bytes < L.host) return CSC_ERR_WORKSPACE;
    // Both streams must be non-blocking: work on the legacy default stream
    // waits for every blocking stream, so a blocking kernel stream would hold
    // it until the persistent kernel ends.
    for (csc_stream_t sp : {kernel_stream, side_stream}) {
        unsigned int fl = 0;
        if (!sp || cudaStreamGetFlags((cudaStream_t)sp, &fl) != cudaSuccess) {
            cudaGetLastError();
            return CSC_ERR_INVALID;
        }
        if (!(fl & cudaStreamNonBlocking)) return CSC_ERR_INVALID;
    }
    if (kernel_stream == side_stream) return CSC_ERR_INVALID;
    // An SM's shared-memory carveout is fixed while a CTA is resident.  The
    // persistent CTAs use almost none, so they ask for the largest carveout:
    // otherwise the beta-init and refresh kernels, which need tens of KB,
    // could not start on any SM until the queue closes.
    {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    // the kernels that run beside the persistent one are loaded, and this
    // thread's pinned scratch allocated, before it starts
    if ((rc = preload_corr_kernels()) || (rc = preload_residual_kernels()) || (rc = preload_umma_kernels()))
        return rc;
    pinned_scratch();
    csc_queue *q = new csc_queue();
    q->atoms = g;
    q->D = D;
    q->dtd = dtd;
    q->dev = static_cast<unsigned char *>(device_ws);
    q->qc = reinterpret_cast<QueueCtl *>(q->dev + L.ctl);
    q->jobs = reinterpret_cast<QueueJob *>(q->dev + L.jobs);
    q->nrm = reinterpret_cast<double *>(q->dev + L.nrm);
    q->dmax = reinterpret_cast<double *>(q->dev + L.dmax);
    q->ctl_pool = q->dev + L.pool;
    q->ctl_stride = L.stride;
    q->host = static_cast<QueueHostSlot *>(host_ws);
    q->max_jobs = max_jobs;
    q->ctl_slots = ctl_slots;
    q->grid = grid;
    q->ctas_per_sm = dens;
    for (int i = ctl_slots - 1; i >= 0; i--) q->free_ctl.push_back(i);
    csc_default_opts(&q->opts);
    if (opts) q->opts = *opts;
    q->kstream = (cudaStream_t)kernel_stream;
    q->sstream = (cudaStream_t)side_stream;
    memset(host_ws, 0, L.host);
    cudaStream_t ss = q->sstream;
    int err = CSC_OK;
    auto fail = [&](cudaError_t e) {
        err = set_cuda_error(e);
        delete q;
        return err;
    };
    cudaError_t e;
    if ((e = cudaMemsetAsync(q->qc, 0, sizeof(QueueCtl), ss)) != cudaSuccess) return fail(e);
    if ((rc = launch_atom_norms<float>(g, D, q->nrm, q->dmax, ss))) {
        delete q;
        return rc;
    }
    if ((e = cudaStreamSynchronize(ss)) != cudaSuccess) return fail(e);
    q->kern = kern;
    q->run_ns = (unsigned long long)(run_seconds * 1e9);
    if (launch && (rc = queue_launch(q))) {
        delete q;
        return rc;
    }
    *out = q;
    return CSC_OK;
}

int csc_queue_create(const csc_shape *atoms, const float *D, const float *dtd, const csc_solve_opts *opts,
                     int max_jobs, int ctl_slots, int ctas_per_sm, void *device_ws, size_t device_bytes,
                     void *host_ws, size_t host_bytes, double run_seconds, csc_stream_t kernel_stream,
                     csc_stream_t side_stream, csc_queue **out) {
    return queue_create(atoms, D, dtd, opts, max_jobs, ctl_slots, ctas_per_sm, device_ws, device_bytes, host_ws,
                        host_bytes, run_seconds, kernel_stream, side_stream, true, out);
}

int csc_queue_create_deferred(const csc_shape *atoms, const float *D, const float *dtd,
                              const csc_solve_opts *opts, int max_jobs, int ctl_slots, int ctas_per_sm,
                              void *device_ws, size_t device_bytes, void *host_ws, size_t host_bytes,
                              double run_seconds, csc_stream_t kernel_stream, csc_stream_t side_stream,
                              csc_queue **out) {
    return queue_create(atoms, D, dtd, opts, max_jobs, ctl_slots, ctas_per_sm, device_ws, device_bytes, host_ws,
                        host_bytes, run_seconds, kernel_stream, side_stream, false, out);
}

int csc_queue_start(csc_queue *q, int drain) {
    if (!q || q->launched || (drain != 0 && drain != 1)) return CSC_ERR_INVALID;
    if (drain) {
        // the drain word is set by a device-side memset (no host source) before the launch
        cudaError_t e = cudaMemsetAsync(&q->qc->drain, 1, 1, q->sstream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(q->sstream);
        if (e != cudaSuccess) return set_cuda_error(e);
        q->drain = true;
    }
    // the kernel stream follows everything the side stream published
    return queue_launch(q);
}

int csc_queue_submit(csc_queue *q, int T0, int T1, float *beta, float *Z, float lambda, float tol, int warm_start,
                     const csc_solve_opts *opts, int *job_out) {
    if (!q || !beta || !Z || !job_out || !(lambda >= 0.f) || !(tol > 0.f)) return CSC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(beta) | reinterpret_cast<uintptr_t>(Z)) & 15) return CSC_ERR_INVALID;
    if (q->drain) return CSC_ERR_INVALID;  // a draining kernel takes no job published after its start
    const csc_solve_opts o = opts ? *opts : q->opts;
    if (!(o.stop_margin >= 0.0 && o.stop_margin <= 1.0) || o.mode < 0 || o.mode > 2) return CSC_ERR_INVALID;
    if (q->njobs >= q->max_jobs || q->free_ctl.empty()) return CSC_ERR_WORKSPACE;
    csc_shape s;
    s.d = 2;
    s.P = q->atoms.P;
    s.K = q->atoms.K;
    s.T[0] = T0;
    s.T[1] = T1;
    s.L[0] = q->atoms.L0;
    s.L[1] = q->atoms.L1;
    Geom g;
    int rc = make_geom(&s, &g);
    if (rc) return rc;
    Plan pl;
    // one job takes at most 7/8 of the grid unless opts.max_workers says
    // otherwise, so that small jobs queued behind a large one start beside it
    rc = make_plan_global(g, o, q->grid - q->grid / 8, 4, &pl);
    if (rc) return rc;
    const int W = pl.G0 * pl.G1;
    if (W > q->grid) return CSC_ERR_UNIMPLEMENTED;
    const int cs = q->free_ctl.back();  // taken below once the job is published
    unsigned char *ctl = q->ctl_pool + (size_t)cs * q->ctl_stride;
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ctl);
    int *flags = reinterpret_cast<int *>(ctl + sizeof(WsHeader));
    QueueJob job{};
    LgcdArgs<float> &a = job.a;
    a.beta = beta;
    a.Z = Z;
    a.dtd = q->dtd;
    a.nrm = q->nrm;
    a.dmax = q->dmax;
    a.hdr = hdr;
    a.slots = nullptr;
    a.ctl = flags;
    a.K = g.K;
    a.Z0 = g.Z0;
    a.Z1 = g.Z1;
    a.L0 = g.L0;
    a.L1 = g.L1;
    a.W0 = g.W0;
    a.W1 = g.W1;
    a.G0 = pl.G0;
    a.G1 = pl.G1;
    a.t0 = pl.t0;
    a.t1 = pl.t1;
    a.sub0 = pl.sub0;
    a.sub1 = pl.sub1;
    a.mode = o.mode == CSC_MODE_NOLOCK ? CSC_MODE_NOLOCK : CSC_MODE_ASYNC;
    a.guard_on = o.divergence_guard;
    a.cap = kMailboxCap;
    a.Mmax = 0;
    a.z_zero = warm_start ? 0 : 1;
    a.lambda = lambda;
    a.eps = (float)(o.stop_margin > 0.0 ? o.stop_margin : 0.99) * tol;  // as in the single solve
    a.max_updates = 0;
    const double tmo = o.timeout_s > 0 ? o.timeout_s : 30.0;
    a.timeout_ns = (unsigned long long)(tmo * 1e9);
    job.prefix = q->next_slot;
    job.W = W;
    job.claimed = 0;
    job.done = 0;
    // header: pending = workers, everything else zero; flag counters zero
    WsHeader h0;
    memset(&h0, 0, sizeof(h0));
    h0.pending = W;
    cudaStream_t ss = q->sstream;
    const int j = q->njobs, nj = j + 1;
    // the three records are copied from the pinned scratch (regions that do
    // not overlap), falling back to this stack frame; the copies are waited
    // for before returning either way
    static_assert(sizeof(WsHeader) + sizeof(QueueJob) + 2 * 256 <= kPinnedScratch, "scratch layout");
    unsigned char *ps = static_cast<unsigned char *>(pinned_scratch());
    const void *src_h = &h0, *src_j = &job, *src_n = &nj;
    if (ps) {
        const size_t oj = q_align(sizeof(WsHeader)), on = oj + q_align(sizeof(QueueJob));
        memcpy(ps, &h0, sizeof(h0));
        memcpy(ps + oj, &job, sizeof(job));
        memcpy(ps + on, &nj, sizeof(int));
        src_h = ps;
        src_j = ps + oj;
        src_n = ps + on;
    }
    if (!warm_start) CSC_CUDA(cudaMemsetAsync(Z, 0, (size_t)g.nz() * sizeof(float), ss));
    CSC_CUDA(cudaMemcpyAsync(hdr, src_h, sizeof(h0), cudaMemcpyHostToDevice, ss));
    CSC_CUDA(cudaMemsetAsync(flags, 0, (size_t)W * kDirs * 32 * sizeof(int), ss));
    q->host[j].complete = 0;
    CSC_CUDA(cudaMemcpyAsync(q->jobs + j, src_j, sizeof(job), cudaMemcpyHostToDevice, ss));
    CSC_CUDA(cudaMemcpyAsync(&q->qc->njobs, src_n, sizeof(int), cudaMemcpyHostToDevice, ss));
    CSC_CUDA(cudaStreamSynchronize(ss));
    q->free_ctl.pop_back();
    q->njobs = nj;
    q->next_slot += W;
    q->job_ctl.push_back(cs);
    *job_out = j;
    return CSC_OK;
}

int csc_queue_poll(csc_queue *q, int job, csc_solve_stats *stats) {
    if (!q || job < 0 || job >= q->njobs) return -CSC_ERR_INVALID;
    volatile QueueHostSlot *hs = q->host + job;
    if (!hs->complete) return 0;
    if (q->job_ctl[job] >= 0) {
        q->free_ctl.push_back(q->job_ctl[job]);
        q->job_ctl[job] = -1;
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->status = hs->status;
        stats->updates = hs->updates;
        stats->iterations = hs->iterations;
        stats->rejected_softlock = hs->rejected;
        stats->skipped_subtol = hs->subtol;
        stats->messages = hs->messages;
        stats->max_worker_iterations = hs->max_iters;
        stats->kernel_ms = (double)hs->t_ns * 1e-6;
        stats->placement = 2;
    }
    return 1;
}

int csc_queue_inspect(csc_queue *q, int job, long long *out) {
    if (!q || !out || job < 0 || job >= q->njobs) return CSC_ERR_INVALID;
    QueueCtl c;
    QueueJob jb;
    int rc;
    if ((rc = read_back(&c, q->qc, q->sstream))) return rc;
    if ((rc = read_back(&jb, q->jobs + job, q->sstream))) return rc;
    out[0] = jb.prefix;
    out[1] = jb.W;
    out[2] = jb.claimed;
    out[3] = jb.done;
    out[4] = c.njobs;
    out[5] = c.slot;
    out[6] = q->grid;
    out[7] = ((volatile QueueHostSlot *)(q->host + job))->complete;
    return CSC_OK;
}

int csc_queue_close(csc_queue *q) {
    if (!q) return CSC_ERR_INVALID;
    int rc = CSC_OK;
    cudaError_t e = cudaSuccess;
    if (q->launched) {
        // a draining kernel ends by itself once its jobs are done
        if (q->drain) e = cudaStreamSynchronize(q->kstream);
        // the close word is 0 since creation: setting its low byte makes it 1
        // (a device-side write, no host source)
        if (e == cudaSuccess) e = cudaMemsetAsync(&q->qc->close, 1, 1, q->sstream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(q->sstream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(q->kstream);
        g_live_queues.fetch_sub(1);
    } else {
        e = cudaStreamSynchronize(q->sstream);  // submits of a queue never started
    }
    if (e != cudaSuccess) rc = set_cuda_error(e);
    delete q;
    return rc;
}

int csc_refresh_beta(const csc_shape *shape, const float *X, const float *D, const float *Z, float lambda,
                     float *beta, double *max_dz_out, double *objective_out, void *ws, size_t ws_bytes,
                     csc_stream_t stream) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!X || !D || !Z || !beta || !ws) return CSC_ERR_INVALID;
    WsLayout L = plan_workspace(g, 0, 4);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
    unsigned char *wsb = static_cast<unsigned char *>(ws);
    cudaStream_t st = (cudaStream_t)stream;
    rc = launch_atom_norms<float>(g, D, reinterpret_cast<double *>(wsb + L.nrm),
                                  reinterpret_cast<double *>(wsb + L.dmax), st);
    if (rc) return rc;
    rc = launch_refresh<float>(g, L, wsb, X, D, Z, lambda, beta, st);
    if (rc) return rc;
    WsHeader hh;
    {
        const int rb_ = read_back(&hh, wsb + L.hdr, st);
        if (rb_) return rb_;
    }
    if (max_dz_out) {
        const unsigned u = (unsigned)hh.maxdz_bits;
        float f;
        memcpy(&f, &u, 4);
        *max_dz_out = f;
    }
    if (objective_out) *objective_out = 0.5 * hh.obj_f + (double)lambda * hh.obj_g;
    return CSC_OK;
}

}  // extern "C"
