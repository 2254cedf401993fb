// lgcd.cu -- locally greedy coordinate descent over a grid of worker tiles
// (Alg. 1 run inside each worker of Alg. 3): the PHASED kernel, the kernel
// for tiles kept in global memory, and the host side (tile plan, launch,
// beta refresh and the fresh-beta convergence check between launches).  The
// asynchronous shared-memory kernel (ASYNC / NOLOCK) is in lgcd_async.cu.
//
// PHASED: every tile keeps beta and Z in shared memory; tiles run in
// checkerboard colour phases separated by bounded grid barriers, each tile
// updating one sub-domain per phase of its colour and posting (k0, s0, dZ) to
// the neighbours its window reaches.  The run is deterministic and equals the
// sequential tiled schedule (the FP64 build reproduces it exactly).
//
// GLOBAL TILES: beta and Z stay in global memory for atoms too large for
// shared memory; window updates are red.global.add and a neighbour learns of
// an update through its flag counter.
//
// Termination of the asynchronous kernels (Alg. 3 "global convergence"): the
// word `pending` counts active workers plus messages in flight; pending == 0
// is stable and means that no coordinate anywhere can move by eps.  Every
// wait is bounded by a deadline from %globaltimer and by the shared stop word.
#include "lgcd_global.cuh"

namespace csc {

// ================================================================ PHASED
// Bounded grid barrier (generation counter).  Returns false when the stop
// word is set or the deadline passes.
__device__ __forceinline__ bool grid_barrier(WsHeader *h, unsigned nblocks,
                                             unsigned long long deadline) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned gen = ld_acquire_u(&h->bar_gen);
        __threadfence();
        unsigned arrived = atomicAdd(&h->bar_count, 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(&h->bar_count, 0u);
            __threadfence();
            st_release_u(&h->bar_gen, gen + 1u);
        } else {
            while (ld_acquire_u(&h->bar_gen) == gen) {
                if (ld_relaxed(&h->stop)) { ok = 0; break; }
                if (globaltimer_ns() > deadline) {
                    atomicCAS(&h->stop, 0, CSC_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (ld_relaxed(&h->stop)) ok = 0;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename real, int NT>
__global__ void __launch_bounds__(NT, 1) lgcd_phased_kernel(LgcdArgs<real> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Tile<real, NT> t;
    tile_setup<real, NT>(a, t, smem_raw);
    __shared__ int s_nmsg;

    Comm cm;
    long long n_upd = 0, n_it = 0, n_sub = 0, n_msg = 0;
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    const unsigned nblocks = gridDim.x;
    if (threadIdx.x == 0) {
        cm.ndir = 0;
        for (int d = 0; d < kDirs; d++) {
            int dr, dc;
            dir_offset(d, dr, dc);
            int r = t.ta + dr, c = t.tb + dc;
            cm.out_head[d] = cm.out_tail[d] = cm.in_tail[d] = 0;
            if (r >= 0 && r < a.G0 && c >= 0 && c < a.G1) cm.dirs[cm.ndir++] = d;
        }
    }
    const int my_color = 2 * (t.ta & 1) + (t.tb & 1);
    int m = 0, quiet_rounds = 0, round = 0;
    bool ok = true;
    while (ok) {
        for (int c = 0; c < 4 && ok; c++) {
            if ((c >> 1) > 0 && a.G0 == 1) continue;  // colour absent
            if ((c & 1) > 0 && a.G1 == 1) continue;
            ok = grid_barrier(a.hdr, nblocks, deadline);
            if (!ok) break;
            // drain every message of the previous phase
            if (threadIdx.x == 0) {
                int heads[kDirs];
                for (int i = 0; i < cm.ndir; i++)
                    heads[cm.dirs[i]] = ld_acquire(a.ctl + ((size_t)t.w * kDirs + cm.dirs[i]) * 32);
                s_nmsg = stage_messages<real, NT>(a, t, cm, heads);
            }
            __syncthreads();
            if (s_nmsg > 0) {
                apply_messages<real, NT>(a, t, s_nmsg);
                __syncthreads();
            }
            if (c != my_color) continue;
            Cand<real> best = scan_subdomain<real, NT>(a, t, m);
            n_it++;
            m = (m + 1 == t.M) ? 0 : m + 1;
            if (!(best.a >= a.eps)) {
                n_sub++;
                continue;
            }
            const unsigned pos = best.key / (unsigned)t.K;
            const int k0 = (int)(best.key % (unsigned)t.K);
            const int li0 = (int)(pos / (unsigned)a.t1), lj0 = (int)(pos % (unsigned)a.t1);
            const int idx0 = k0 * t.TS + li0 * a.t1 + lj0;
            const real dz = best.dz;
            apply_own_update<real, NT>(a, t, k0, li0, lj0, dz);
            if (threadIdx.x == 0) {
                t.sz[idx0] = best.znew;
                size_t g = ((size_t)k0 * a.Z0 + t.or0 + li0) * a.Z1 + t.oc0 + lj0;
                st_relaxed(a.Z + g, best.znew);
                int dirs[kDirs];
                int nd = target_dirs<real, NT>(a, t, li0, lj0, dirs);
                post_messages<real, NT>(a, t, cm, dirs, nd, k0, (t.or0 + li0) * a.Z1 + t.oc0 + lj0, dz);
                n_msg += nd;
                n_upd++;
                atomicAdd(&a.hdr->round_applied[round & 1], 1);
                atomicAdd(&a.hdr->updates_total, 1ull);
            }
        }
        if (!ok) break;
        ok = grid_barrier(a.hdr, nblocks, deadline);
        if (!ok) break;
        __shared__ int s_applied;
        __shared__ unsigned long long s_total;
        if (threadIdx.x == 0) {
            s_applied = ld_acquire(&a.hdr->round_applied[round & 1]);
            s_total = atomicAdd(&a.hdr->updates_total, 0ull);
            if (blockIdx.x == 0) atomicExch(&a.hdr->round_applied[(round + 1) & 1], 0);
        }
        __syncthreads();
        quiet_rounds = s_applied ? 0 : quiet_rounds + 1;
        round++;
        if (quiet_rounds >= a.Mmax) break;
        if (a.max_updates > 0 && (long long)s_total >= a.max_updates) {
            if (threadIdx.x == 0) set_stop(a.hdr, CSC_NOT_CONVERGED);
            break;
        }
    }
    // Apply what is still queued (only after an early stop) and write back.
    if (ok && grid_barrier(a.hdr, nblocks, deadline)) {
        if (threadIdx.x == 0) {
            int heads[kDirs];
            for (int i = 0; i < cm.ndir; i++)
                heads[cm.dirs[i]] = ld_acquire(a.ctl + ((size_t)t.w * kDirs + cm.dirs[i]) * 32);
            s_nmsg = stage_messages<real, NT>(a, t, cm, heads);
        }
        __syncthreads();
        if (s_nmsg > 0) apply_messages<real, NT>(a, t, s_nmsg);
    }
    write_back<real, NT>(a, t);
    if (threadIdx.x == 0) {
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_UPDATES], (unsigned long long)n_upd);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_ITERS], (unsigned long long)n_it);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_SUBTOL], (unsigned long long)n_sub);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_MESSAGES], (unsigned long long)n_msg);
    }
}

// ============================================================ GLOBAL TILES
template <typename real>
__global__ void __launch_bounds__(kGlobThreads, 2) lgcd_global_kernel(LgcdArgs<real> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    global_tile_worker<real, kGlobThreads, 4, true>(a, blockIdx.x, smem_raw);
}

// The table in the window layout of the staged window update: block
// [k0][k] = C[k][k0] as W0 rows of wrs floats, row rw's values at
// rw * wrs + 4 + cw, zeros elsewhere, and the centre of C[k0][k0] zeroed.
__global__ void wtab_kernel(const float *dtd, float *wtab, int K, int W0, int W1, int L0, int L1, int wrs, int wbs) {
    const long long n = (long long)K * K * wbs;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / wbs), r = (int)(i - (long long)b * wbs);
        const int k0 = b / K, k = b - k0 * K;
        const int rw = r / wrs, cw = r - rw * wrs - 4;
        float v = 0.f;
        if (rw < W0 && cw >= 0 && cw < W1 && !(k == k0 && rw == L0 - 1 && cw == L1 - 1))
            v = dtd[(((size_t)k * K + k0) * W0 + rw) * W1 + cw];
        wtab[i] = v;
    }
}

// Header reset before a launch: pending = number of workers, counters 0.
__global__ void reset_header_kernel(WsHeader *h, int workers) {
    h->pending = workers;
    h->stop = 0;
    h->bar_count = 0;
    h->bar_gen = 0;
    h->round_applied[0] = 0;
    h->round_applied[1] = 0;
    h->updates_total = 0;
    for (int i = 0; i < 8; i++) h->stat[i] = 0;
    h->wmax[0] = h->wmax[1] = 0;
    for (int i = 0; i < 4; i++) h->tmax[i] = 0;
    for (int i = 0; i < 6; i++) h->tph[i] = 0;
    for (int i = 0; i < 8; i++) h->tphmax[i] = 0;
    h->maxdz_bits = 0;
    h->obj_f = 0.0;
    h->obj_g = 0.0;
    h->nnz = 0;
    h->overflow = 0;
}

// ============================================================== host side
constexpr int kLgcdThreads = 256;


// Dynamic shared memory of one tile: beta and Z, the K x K x |window| table
// and the atom norms, plus a staging buffer for records (PHASED kernel; the
// asynchronous kernel stages records in its static shared memory).
static size_t tile_smem(const Geom &g, int t0, int t1, int rs, bool phased) {
    size_t n = (2 * (size_t)g.K * t0 * t1 + (size_t)g.ntab() + 2 * (size_t)g.K) * rs;
    n = (n + 15) & ~(size_t)15;
    return phased ? n + kMsgBatch * sizeof(int4) : n;
}

template <typename real>
static const void *kernel_ptr(int mode, bool global) {
    if (global) return (const void *)lgcd_global_kernel<real>;
    if (mode == CSC_MODE_PHASED) return (const void *)lgcd_phased_kernel<real, kLgcdThreads>;
    return lgcd_async_kernel_ptr(real(0));
}
static int kernel_threads(int mode, bool global) {
    if (global) return kGlobThreads;
    return mode == CSC_MODE_PHASED ? kLgcdThreads : kAsyncThreads;
}

struct DevProps {
    int dev = -1, smem_optin = 0, sms = 0, smem_sm = 0;
};
static const DevProps &dev_props() {
    static thread_local DevProps p;
    int dev = 0;
    cudaGetDevice(&dev);
    if (p.dev != dev) {
        p.dev = dev;
        cudaDeviceGetAttribute(&p.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&p.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    }
    return p;
}
static int smem_limit() { return dev_props().smem_optin; }
static int num_sms() { return dev_props().sms; }
static int smem_per_sm() { return dev_props().smem_sm; }

// Tile plan.  Full tiles must be at least L_i wide (windows then reach only
// the adjacent tiles); automatic plans use tiles of at least 2 L_i and the
// largest number of workers that can all be resident at once.
static int make_plan(const Geom &g, const csc_solve_opts &o, int rs, size_t static_smem, int max_occ, Plan *pl) {
    const bool d1 = g.d == 1;
    pl->sub0 = d1 ? 1 : (o.sub[0] > 0 ? o.sub[0] : 2 * g.L0);
    pl->sub1 = d1 ? (o.sub[0] > 0 ? o.sub[0] : 2 * g.L1) : (o.sub[1] > 0 ? o.sub[1] : 2 * g.L1);
    // the asynchronous kernel keeps one dirty flag per sub-domain
    const long long max_sub = o.mode == CSC_MODE_PHASED ? (1ll << 40) : kAsyncMaxSub;
    auto nsub = [&](int t0, int t1) { return ceil_div(t0, pl->sub0) * ceil_div(t1, pl->sub1); };
    const int lim = smem_limit(), sms = num_sms(), per_sm = smem_per_sm();
    int ut0 = d1 ? 0 : o.tile[0], ut1 = d1 ? o.tile[0] : o.tile[1];
    if (ut0 > 0 || ut1 > 0 || d1 && o.tile[0] > 0) {
        int t0 = d1 ? 1 : (ut0 > 0 ? std::min(ut0, g.Z0) : g.Z0);
        int t1 = ut1 > 0 ? std::min(ut1, g.Z1) : g.Z1;
        if ((t0 < g.L0 && t0 < g.Z0) || (t1 < g.L1 && t1 < g.Z1)) return CSC_ERR_INVALID;
        if (nsub(t0, t1) > max_sub) return CSC_ERR_INVALID;
        pl->t0 = t0;
        pl->t1 = t1;
        pl->G0 = (int)ceil_div(g.Z0, t0);
        pl->G1 = (int)ceil_div(g.Z1, t1);
        pl->smem = tile_smem(g, t0, t1, rs, o.mode == CSC_MODE_PHASED);
        if (pl->smem + static_smem > (size_t)lim) return CSC_ERR_UNIMPLEMENTED;
        return CSC_OK;
    }
    const int minT0 = d1 ? 1 : std::min(g.Z0, 2 * g.L0), minT1 = std::min(g.Z1, 2 * g.L1);
    const int maxG0 = d1 ? 1 : std::max(1, g.Z0 / minT0), maxG1 = std::max(1, g.Z1 / minT1);
    bool found = false;
    Plan best{};
    long long best_w = 0;
    for (int occ = 1; occ <= std::min(8, max_occ); occ++) {
        long long cap_w = (long long)occ * sms;
        if (o.max_workers > 0) cap_w = std::min<long long>(cap_w, o.max_workers);
        size_t budget = std::min<size_t>((size_t)lim - static_smem, (size_t)per_sm / occ - 1024 - static_smem);
        for (int G0 = 1; G0 <= maxG0; G0++) {
            int G1 = (int)std::min<long long>(maxG1, cap_w / G0);
            if (G1 < 1) break;
            for (; G1 >= 1; G1--) {
                int t0 = (int)ceil_div(g.Z0, G0), t1 = (int)ceil_div(g.Z1, G1);
                int a0 = (int)ceil_div(g.Z0, t0), a1 = (int)ceil_div(g.Z1, t1);
                if (tile_smem(g, t0, t1, rs, o.mode == CSC_MODE_PHASED) <= budget && nsub(t0, t1) <= max_sub) {
                    long long w = (long long)a0 * a1;
                    // prefer more workers, then squarer tiles
                    bool take = !found || w > best_w ||
                                (w == best_w && std::abs(t0 - t1) < std::abs(best.t0 - best.t1));
                    if (d1) take = !found || w > best_w;
                    if (take) {
                        found = true;
                        best_w = w;
                        best.G0 = a0;
                        best.G1 = a1;
                        best.t0 = t0;
                        best.t1 = t1;
                        best.smem = tile_smem(g, t0, t1, rs, o.mode == CSC_MODE_PHASED);
                    }
                    break;
                }
            }
        }
    }
    if (!found) return CSC_ERR_UNIMPLEMENTED;
    best.sub0 = pl->sub0;
    best.sub1 = pl->sub1;
    *pl = best;
    return CSC_OK;
}

// Plan for the global-memory variant: tiles of at least 2 L_i (or the
// caller's tile, at least L_i), at most `max_w` tiles, squarish in 2-D.
int make_plan_global(const Geom &g, const csc_solve_opts &o, long long max_w, int rs, Plan *pl) {
    const bool d1 = g.d == 1;
    pl->sub0 = d1 ? 1 : (o.sub[0] > 0 ? o.sub[0] : 2 * g.L0);
    pl->sub1 = d1 ? (o.sub[0] > 0 ? o.sub[0] : 2 * g.L1) : (o.sub[1] > 0 ? o.sub[1] : 2 * g.L1);
    pl->smem = 2 * (size_t)g.K * rs;
    const int ut0 = d1 ? 0 : o.tile[0], ut1 = d1 ? o.tile[0] : o.tile[1];
    if (o.max_workers > 0) max_w = std::min<long long>(max_w, o.max_workers);
    if (ut0 > 0 || ut1 > 0) {
        const int t0 = d1 ? 1 : (ut0 > 0 ? std::min(ut0, g.Z0) : g.Z0);
        const int t1 = ut1 > 0 ? std::min(ut1, g.Z1) : g.Z1;
        if ((t0 < g.L0 && t0 < g.Z0) || (t1 < g.L1 && t1 < g.Z1)) return CSC_ERR_INVALID;
        // the soft-lock of a global-memory tile tests one strip per dimension:
        // no window V(s0) may cross both edges of a tile
        if (o.mode == CSC_MODE_ASYNC && ((t0 < 2 * g.L0 - 1 && t0 < g.Z0) || (t1 < 2 * g.L1 - 1 && t1 < g.Z1)))
            return CSC_ERR_INVALID;
        pl->t0 = t0;
        pl->t1 = t1;
    } else {
        const int minT0 = d1 ? 1 : std::min(g.Z0, 2 * g.L0), minT1 = std::min(g.Z1, 2 * g.L1);
        const int maxG0 = d1 ? 1 : std::max(1, g.Z0 / minT0), maxG1 = std::max(1, g.Z1 / minT1);
        long long best_w = 0;
        int b0 = 1, b1 = 1;
        for (int G0 = 1; G0 <= maxG0; G0++) {
            const int G1 = (int)std::min<long long>(maxG1, max_w / G0);
            if (G1 < 1) break;
            const int t0 = (int)ceil_div(g.Z0, G0), t1 = (int)ceil_div(g.Z1, G1);
            const long long wk = ceil_div(g.Z0, t0) * ceil_div(g.Z1, t1);
            const int ob0 = (int)ceil_div(g.Z0, b0), ob1 = (int)ceil_div(g.Z1, b1);
            if (wk > best_w || (wk == best_w && std::abs(t0 - t1) < std::abs(ob0 - ob1))) {
                best_w = wk;
                b0 = G0;
                b1 = G1;
            }
        }
        pl->t0 = (int)ceil_div(g.Z0, b0);
        pl->t1 = (int)ceil_div(g.Z1, b1);
    }
    pl->G0 = (int)ceil_div(g.Z0, pl->t0);
    pl->G1 = (int)ceil_div(g.Z1, pl->t1);
    return CSC_OK;
}

template <typename real>
int solve_impl(const csc_shape *shape, const real *X, const real *D, const real *dtd, real *beta,
               real *Z, real lambda, real tol, const csc_solve_opts *opts_in, void *ws,
               size_t ws_bytes, csc_solve_stats *stats, cudaStream_t st) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!X || !D || !dtd || !beta || !Z || !ws) return CSC_ERR_INVALID;
    if (!(lambda >= real(0)) || !(tol > real(0))) return CSC_ERR_INVALID;
    csc_solve_opts o;
    csc_default_opts(&o);
    if (opts_in) o = *opts_in;
    if (o.mode < 0 || o.mode > 2 || o.beta_refresh < 0) return CSC_ERR_INVALID;
    if (!(o.stop_margin >= 0.0 && o.stop_margin <= 1.0)) return CSC_ERR_INVALID;
    const int rs = (int)sizeof(real);
    if (o.placement < 0 || o.placement > 2) return CSC_ERR_INVALID;
    bool global = o.placement == 2;
    if (global && o.mode == CSC_MODE_PHASED) return CSC_ERR_UNIMPLEMENTED;
    const void *kern = kernel_ptr<real>(o.mode, global);
    size_t static_smem = 0;
    {
        static thread_local std::vector<std::pair<const void *, size_t>> attr_cache;
        bool found = false;
        for (auto &c : attr_cache)
            if (c.first == kern) {
                static_smem = c.second;
                found = true;
            }
        if (!found) {
            cudaFuncAttributes fa;
            CSC_CUDA(cudaFuncGetAttributes(&fa, kern));
            static_smem = fa.sharedSizeBytes;
            attr_cache.push_back({kern, static_smem});
        }
    }
    // resident tiles per SM allowed by registers and threads alone
    int max_occ = 8;
    if (!global) {
        static thread_local std::vector<std::pair<const void *, int>> occ_cache;
        int found_occ = -1;
        for (auto &c : occ_cache)
            if (c.first == kern) found_occ = c.second;
        if (found_occ < 0) {
            CSC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&found_occ, kern, kernel_threads(o.mode, false), 0));
            occ_cache.push_back({kern, found_occ});
        }
        max_occ = std::max(1, found_occ);
    }
    Plan pl;
    rc = global ? CSC_ERR_UNIMPLEMENTED : make_plan(g, o, rs, static_smem, max_occ, &pl);
    if (rc == CSC_ERR_UNIMPLEMENTED && o.placement == 0 && o.mode != CSC_MODE_PHASED) global = true;
    if (global) {
        kern = kernel_ptr<real>(o.mode, true);
        rc = make_plan_global(g, o, 2ll * num_sms(), rs, &pl);
    }
    if (rc) return rc;
    // the FP32 global-tile worker reads and reduces beta / Z in 16-byte groups
    if (global && rs == 4 && ((reinterpret_cast<uintptr_t>(beta) | reinterpret_cast<uintptr_t>(Z)) & 15))
        return CSC_ERR_INVALID;
    const int W = pl.G0 * pl.G1;
    WsLayout L = plan_workspace(g, W, rs);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
    // FP32 global tiles with the optional workspace region: the window update
    // stages the table through as many shared-memory slots (up to 4) as fit
    // beside a second CTA on the SM; fewer than 2 and it reads dtd instead
    int wslots = 0;
    if (global && rs == 4 && ws_bytes >= L.total_beta0) {
        cudaFuncAttributes fa;
        CSC_CUDA(cudaFuncGetAttributes(&fa, kern));
        const long long slot = ((long long)L.wbs + 8) * 4;
        const long long budget =
            (long long)smem_per_sm() / 2 - 1024 - (long long)fa.sharedSizeBytes - (long long)stage_offset(g.K);
        wslots = (int)std::min<long long>(kMaxStageSlots, std::max<long long>(0, budget / slot));
        if (wslots < 2) wslots = 0;
        if (wslots) pl.smem = stage_offset(g.K) + (size_t)wslots * (size_t)slot;
    }
    unsigned char *wsb = static_cast<unsigned char *>(ws);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(wsb + L.hdr);
    double *nrm = reinterpret_cast<double *>(wsb + L.nrm);
    double *dmax = reinterpret_cast<double *>(wsb + L.dmax);

    {
        // kernel attribute and co-residency check, cached per (kernel, device, smem)
        struct Key {
            const void *k;
            int dev;
            size_t smem;
            int occ;
        };
        static thread_local std::vector<Key> cache;
        const int dev = dev_props().dev;
        int occ = -1;
        for (const Key &c : cache)
            if (c.k == kern && c.dev == dev && c.smem == pl.smem) occ = c.occ;
        if (occ < 0) {
            CSC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
            CSC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kernel_threads(o.mode, global), pl.smem));
            cache.push_back({kern, dev, pl.smem, occ});
        } else {
            CSC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
        }
        if ((long long)occ * num_sms() < W) return CSC_ERR_UNIMPLEMENTED;
    }

    if (!o.warm_start) CSC_CUDA(cudaMemsetAsync(Z, 0, (size_t)g.nz() * rs, st));
    // FP32 global tiles from a cold start keep the initial beta: the final
    // KKT test then rebuilds beta as beta0 - C * Z over the nonzeros of Z
    // instead of correlating the residual again
    const bool use_beta0 = global && rs == 4 && !o.warm_start && ws_bytes >= L.total_beta0;
    if (use_beta0) CSC_CUDA(cudaMemcpyAsync(wsb + L.beta0, beta, (size_t)g.nz() * rs, cudaMemcpyDeviceToDevice, st));
    rc = launch_atom_norms<real>(g, D, nrm, dmax, st);
    if (rc) return rc;
    float *wtab = reinterpret_cast<float *>(wsb + L.wtab);
    if constexpr (sizeof(real) == 4) {
        if (wslots) {
            const long long n = (long long)g.K * g.K * L.wbs;
            wtab_kernel<<<(unsigned)std::min<long long>(4096, (n + 255) / 256), 256, 0, st>>>(
                dtd, wtab, g.K, g.W0, g.W1, g.L0, g.L1, L.wrs, L.wbs);
            CSC_CUDA(cudaGetLastError());
        }
    }

    LgcdArgs<real> a{};
    a.beta = beta;
    a.Z = Z;
    a.dtd = dtd;
    a.nrm = nrm;
    a.dmax = dmax;
    a.hdr = hdr;
    a.slots = reinterpret_cast<int4 *>(wsb + L.mbox_slots);
    a.ctl = reinterpret_cast<int *>(wsb + L.mbox_ctl);
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
    a.mode = o.mode;
    a.guard_on = o.divergence_guard;
    a.cap = kMailboxCap;
    a.lambda = lambda;
    // FP32 solves stop at 0.99 tol so that rounding drift of the incrementally
    // maintained beta rarely pushes a coordinate back above tol on the
    // recomputed beta; the FP64 build keeps tol exactly.
    const double margin = o.stop_margin > 0.0 ? o.stop_margin : (sizeof(real) == 4 ? 0.99 : 1.0);
    a.eps = real(margin) * tol;
    a.max_updates = o.max_updates;
    a.wtab = wslots ? wtab : nullptr;
    a.wrs = L.wrs;
    a.wbs = L.wbs;
    a.wslots = wslots;
    double tmo = o.timeout_s > 0 ? o.timeout_s : 30.0;
    a.timeout_ns = (unsigned long long)(tmo * 1e9);
    {
        int mmax = 0;
        for (int ta = 0; ta < pl.G0; ta++)
            for (int tb = 0; tb < pl.G1; tb++) {
                int h = std::min(pl.t0, g.Z0 - ta * pl.t0), w = std::min(pl.t1, g.Z1 - tb * pl.t1);
                int M = (int)(ceil_div(h, pl.sub0) * ceil_div(w, pl.sub1));
                mmax = std::max(mmax, M);
            }
        a.Mmax = mmax;
    }

    csc_solve_stats S{};
    S.workers = W;
    S.placement = global ? 2 : 1;
    S.tiles[0] = g.d == 1 ? pl.G1 : pl.G0;
    S.tiles[1] = g.d == 1 ? 1 : pl.G1;
    S.tile_size[0] = g.d == 1 ? pl.t1 : pl.t0;
    S.tile_size[1] = g.d == 1 ? 1 : pl.t1;
    static thread_local cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!e0) {
        CSC_CUDA(cudaEventCreate(&e0));
        CSC_CUDA(cudaEventCreate(&e1));
    }
    int status = CSC_OK;
    float kms_total = 0.f;
    WsHeader hh;
    for (int round = 0;; round++) {
        CSC_CUDA(cudaMemsetAsync(wsb + L.mbox_ctl, 0, (size_t)W * kDirs * 32 * sizeof(int), st));
        // later rounds resume from the Z of the previous one
        a.z_zero = (round == 0 && !o.warm_start) ? 1 : 0;
        reset_header_kernel<<<1, 1, 0, st>>>(hdr, W);
        CSC_CUDA(cudaGetLastError());
        void *args[] = {&a};
        CSC_CUDA(cudaEventRecord(e0, st));
        CSC_CUDA(cudaLaunchCooperativeKernel(kern, dim3(W), dim3(kernel_threads(o.mode, global)), args, pl.smem, st));
        CSC_CUDA(cudaEventRecord(e1, st));
        // beta from scratch, KKT and objective on the current Z, then one sync
        rc = launch_refresh<real>(g, L, wsb, X, D, Z, lambda, beta, st, use_beta0 ? dtd : nullptr);
        if (rc) return rc;
        S.refresh_rounds++;
        {
            const int rb_ = read_back(&hh, hdr, st);
            if (rb_) return rb_;
        }
        float ms = 0.f;
        CSC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        kms_total += ms;
        S.updates += hh.stat[ST_UPDATES];
        S.iterations += hh.stat[ST_ITERS];
        S.rejected_softlock += hh.stat[ST_REJECTED];
        S.skipped_subtol += hh.stat[ST_SUBTOL];
        S.messages += hh.stat[ST_MESSAGES];
        S.deferred += hh.stat[ST_DEFERRED];
        S.candidates += hh.stat[ST_CAND];
        S.max_worker_iterations = std::max<long long>(S.max_worker_iterations, (long long)hh.wmax[0]);
        S.max_worker_updates = std::max<long long>(S.max_worker_updates, (long long)hh.wmax[1]);
        S.last_active_wave = std::max(S.last_active_wave, (long long)hh.tmax[0]);
        S.t_exit_us = std::max(S.t_exit_us, hh.tmax[1] * 1e-3);
        S.t_first_pause_us = std::max(S.t_first_pause_us, hh.tmax[2] * 1e-3);
        S.wakeups += (long long)hh.tmax[3];
        for (int i = 0; i < 6; i++) S.phase_cycles[i] += (long long)hh.tph[i];
        status = hh.stop;
        double maxdz;
        if (sizeof(real) == 4) {
            unsigned u = (unsigned)hh.maxdz_bits;
            float f;
            memcpy(&f, &u, 4);
            maxdz = f;
        } else {
            memcpy(&maxdz, &hh.maxdz_bits, 8);
        }
        S.max_dz_final = maxdz;
        S.objective = 0.5 * hh.obj_f + (double)lambda * hh.obj_g;
        S.nnz = hh.nnz;
        if (status != CSC_OK) break;
        if (maxdz < (double)tol) break;
        if (round >= o.beta_refresh) {
            status = CSC_NOT_CONVERGED;
            break;
        }
        a.max_updates = o.max_updates > 0 ? std::max<long long>(1, o.max_updates - S.updates) : 0;
    }
    S.kernel_ms = kms_total;
    S.status = status;
    if (stats) *stats = S;
    return status;
}

template int solve_impl<float>(const csc_shape *, const float *, const float *, const float *,
                               float *, float *, float, float, const csc_solve_opts *, void *,
                               size_t, csc_solve_stats *, cudaStream_t);
template int solve_impl<double>(const csc_shape *, const double *, const double *, const double *,
                                double *, double *, double, double, const csc_solve_opts *, void *,
                                size_t, csc_solve_stats *, cudaStream_t);

}  // namespace csc
