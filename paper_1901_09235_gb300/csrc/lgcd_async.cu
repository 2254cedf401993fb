// lgcd_async.cu -- ASYNC / NOLOCK solve with shared-memory tiles: Alg. 3 with
// the soft-lock of Eq. soft_lock (Section 4.1), each worker running Alg. 1.
//
// One CTA owns one tile S_w of the activation domain (one worker of Alg. 3).
// beta and Z of the tile and the K x K x |window| table of Eq. beta_update
// live in shared memory.  The 256 compute threads run the locally greedy
// iteration of Alg. 1 together, one sub-domain C_m (box of side 2 L_i from
// the tile origin) per step, in cyclic order m = q mod M: scan K x C_m for
// the largest |dZ| (Eq. pb_coord, a few candidates per thread and a block
// argmax), test it against the soft-lock when its window leaves the tile,
// and apply it with the beta window update (a few entries per thread).  The
// latency of one step -- not parallelism inside the tile, whose updates are
// coupled through overlapping windows -- bounds the solve, so every step uses
// the whole CTA.  A sub-domain is rescanned only when it is dirty (beta
// changed in it since its last scan); a clean one would yield no update.
//
// Soft-lock across tiles: a candidate whose window leaves the tile is applied
// when its |dZ| is larger than that of every coordinate of V(s0) in a
// lower-indexed tile and at least that of every one in a higher-indexed tile.
// Every tile writes the beta and Z entries of its border band (within L_i - 1
// of an edge that has a neighbour) through to the global arrays as they
// change, and the test reads the neighbours' values there.  The tile is the
// only writer of its entries, so both sides of a comparison evaluate the same
// stored bits: ties always go to the same side, and a set of mutually blocked
// candidates cannot persist once nothing changes (the coordinate with the
// largest |dZ| is blocked only by an equal one in a lower-indexed tile, and
// the lowest of those passes).
//
// Neighbour tiles: an update whose window leaves the tile is posted as
// (k0, s0, dZ) to every neighbour tile the window reaches (Alg. 3 "notify").
// A communication warp owns the global control words: it sends these records
// through single-producer / single-consumer rings in global memory
// (release/acquire on head and tail words) and stages the records it
// receives in shared memory, where the compute threads apply them at the
// start of a step.
//
// Termination (Alg. 3 "global convergence"): the word `pending` counts active
// tiles plus records in flight.  A tile with no dirty sub-domain and no staged
// record asks its communication warp to pause; the warp decrements `pending`
// unless records are staged or unsent, re-activates the tile (increments)
// before it stages a record that arrived, and ends the tile when `pending`
// reaches 0, which is stable.  Every wait is bounded by the stop word and by
// a deadline from %globaltimer.
#include "lgcd_common.cuh"

namespace csc {

constexpr int kAW = kAsyncCompute / 32;  // compute warps
constexpr int kInRing = 128;             // staged incoming records
constexpr int kORing = 64;               // outgoing records
enum { RESP_WOKEN = 1, RESP_TERMINATE = 2 };

struct AsyncTileState {
    int4 in_ring[kInRing];
    int4 out_rec[kORing];
    int out_mask[kORing];
    volatile int in_head, in_tail, out_head, out_tail;
    volatile int idle_seq, resp_seq, resp_kind, stop;
    // broadcast slots of the compute leader, double-buffered by step parity
    // (a step may end without a barrier; the slot of step q is rewritten
    // only in step q + 2, after every thread passed the barrier of q + 1)
    int b_m[2], b_nmsg[2], b_stop[2];
    int b_ok;
    unsigned p_key[kAW];                       // per-warp argmax key
    unsigned long long p_best[kAW];            // its |dZ| bits
    unsigned long long p_lo[kAW], p_hi[kAW];  // per-warp soft-lock maxima
    unsigned long long ph[6], t_last, t_pause, tc;  // leader's timeline (SM cycles)
};

// Order-preserving bits of |dZ| >= 0, plus one (0 stands for "none").
__device__ __forceinline__ unsigned long long sl_bits(float d) { return (unsigned long long)__float_as_uint(d) + 1ull; }
__device__ __forceinline__ unsigned long long sl_bits(double d) {
    return (unsigned long long)__double_as_longlong(d) + 1ull;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v, int) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}
__device__ __forceinline__ float abs_real(float x) { return fabsf(x); }
__device__ __forceinline__ double abs_real(double x) { return fabs(x); }

__device__ __forceinline__ void cbar() { asm volatile("bar.sync 1, %0;" ::"r"(kAsyncCompute) : "memory"); }

// Within L_i - 1 of an edge of the tile that has a neighbour tile.
template <typename real, int NT>
__device__ __forceinline__ bool near_neighbour(const LgcdArgs<real> &a, const Tile<real, NT> &t, int li, int lj) {
    return (li < a.L0 - 1 && t.ta > 0) || (li >= t.h - (a.L0 - 1) && t.ta < a.G0 - 1) ||
           (lj < a.L1 - 1 && t.tb > 0) || (lj >= t.wd - (a.L1 - 1) && t.tb < a.G1 - 1);
}

// Exact n / d for 0 <= n < 2^22, d >= 1, from the float reciprocal inv of d
// (the truncated product is off by at most one either way).
__device__ __forceinline__ int div_small(int n, int d, float inv) {
    int q = __float2int_rz(__fmul_rn((float)n, inv));
    if (q * d > n) q--;
    else if ((q + 1) * d <= n) q++;
    return q;
}

// Warp-wide winner of (largest |dZ|, then smallest key): returns the key
// (0xffffffff when every lane is empty) and the winner's |dZ| bits + 1.
__device__ __forceinline__ unsigned warp_argmax(float a, unsigned key, unsigned long long &bits) {
    const unsigned b = a < 0.f ? 0u : __float_as_uint(a) + 1u;
    const unsigned m = __reduce_max_sync(0xffffffffu, b);
    bits = m;
    if (m == 0u) return 0xffffffffu;
    return __reduce_min_sync(0xffffffffu, b == m ? key : 0xffffffffu);
}
__device__ __forceinline__ unsigned warp_argmax(double a, unsigned key, unsigned long long &bits) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oa = __shfl_xor_sync(0xffffffffu, a, o);
        const unsigned ok = __shfl_xor_sync(0xffffffffu, key, o);
        if (oa > a || (oa == a && ok < key)) {
            a = oa;
            key = ok;
        }
    }
    bits = a < 0.0 ? 0ull : sl_bits(a);
    return a < 0.0 ? 0xffffffffu : key;
}

// Set the bits of the sub-domains that the window of an update at tile-local
// (li0, lj0) touches inside the tile (compute leader; M <= 64).
template <typename real, int NT>
__device__ __forceinline__ void mark_window(const LgcdArgs<real> &a, const Tile<real, NT> &t,
                                            unsigned long long &dmask, int li0, int lj0, float inv0, float inv1) {
    const int ra = max(0, li0 - (a.L0 - 1)), rb = min(t.h - 1, li0 + a.L0 - 1);
    const int ca = max(0, lj0 - (a.L1 - 1)), cb = min(t.wd - 1, lj0 + a.L1 - 1);
    if (ra > rb || ca > cb) return;
    const int mr1 = div_small(rb, a.sub0, inv0), mc0 = div_small(ca, a.sub1, inv1), mc1 = div_small(cb, a.sub1, inv1);
    for (int mr = div_small(ra, a.sub0, inv0); mr <= mr1; mr++)
        for (int mc = mc0; mc <= mc1; mc++) dmask |= 1ull << (mr * t.ns1 + mc);
}

// The K x window entries of an update at tile-local (li0, lj0) that lie
// inside the tile, spread over the compute threads: fn(k, r, idx, li, lj),
// r the window index and idx the shared-memory index.  When the window fits
// the thread count, each thread's window offset is fixed for the whole run.
struct WinThread {
    bool fits, on;
    int r, k0, kstep, di, dj;
};
template <typename real, int NT, typename F>
__device__ __forceinline__ void for_window(const LgcdArgs<real> &a, const Tile<real, NT> &t, const WinThread &wt,
                                           int li0, int lj0, float inv_ww, float inv_w1, F fn) {
    if (wt.fits) {
        if (!wt.on) return;
        const int li = li0 + wt.di, lj = lj0 + wt.dj;
        if (li < 0 || li >= t.h || lj < 0 || lj >= t.wd) return;
        const int base = li * a.t1 + lj;
#pragma unroll 4
        for (int k = wt.k0; k < t.K; k += wt.kstep) fn(k, wt.r, k * t.TS + base, li, lj);
    } else {
        for (int q = threadIdx.x; q < t.K * t.WW; q += kAsyncCompute) {
            const int k = div_small(q, t.WW, inv_ww), r = q - k * t.WW;
            const int di = div_small(r, a.W1, inv_w1);
            const int li = li0 + di - (a.L0 - 1), lj = lj0 + (r - di * a.W1) - (a.L1 - 1);
            if (li < 0 || li >= t.h || lj < 0 || lj >= t.wd) continue;
            fn(k, r, k * t.TS + li * a.t1 + lj, li, lj);
        }
    }
}

template <typename real>
__global__ void __launch_bounds__(kAsyncThreads, 2) lgcd_async_kernel(LgcdArgs<real> a) {
    constexpr int NT = kAsyncThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ AsyncTileState S;
    Tile<real, NT> t;
    tile_setup<real, NT>(a, t, smem_raw);
    const int ns0 = (t.h + a.sub0 - 1) / a.sub0, M = ns0 * t.ns1;
    const unsigned long long t_start = globaltimer_ns(), c_start = clock64();
    const unsigned long long deadline = t_start + a.timeout_ns;
    if (threadIdx.x == 0) {
        S.in_head = S.in_tail = S.out_head = S.out_tail = 0;
        S.idle_seq = S.resp_seq = S.resp_kind = 0;
        S.stop = 0;
    }
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t plane = (size_t)a.Z0 * a.Z1;

    if (warp == kAW) {
        // ================================================ communication warp
        if (lane != 0) return;
        int ndir = 0, dirs[kDirs], in_tail[kDirs], out_head[kDirs], out_tail[kDirs];
        for (int d = 0; d < kDirs; d++) {
            int dr, dc;
            dir_offset(d, dr, dc);
            const int r = t.ta + dr, c = t.tb + dc;
            in_tail[d] = out_head[d] = out_tail[d] = 0;
            if (r >= 0 && r < a.G0 && c >= 0 && c < a.G1) dirs[ndir++] = d;
        }
        bool idle = false;
        int spins = 0, n_wake = 0;
        long long n_sent = 0;
        for (;;) {
            bool work = false;
            // ---- inbound: stage new records while the ring has room
            int heads[kDirs], avail = 0;
            for (int i = 0; i < ndir; i++) {
                heads[dirs[i]] = ld_relaxed(a.ctl + ((size_t)t.w * kDirs + dirs[i]) * 32);
                avail += heads[dirs[i]] - in_tail[dirs[i]];
            }
            if (avail > 0) {
                if (idle) {
                    atomicAdd(&a.hdr->pending, 1);  // re-activate before consuming
                    idle = false;
                    n_wake++;
                    S.resp_kind = RESP_WOKEN;
                    __threadfence_block();
                    S.resp_seq = S.idle_seq;
                }
                fence_acq_rel_gpu();
                const int ih = S.in_head;
                const int room = kInRing - (ih - S.in_tail);
                int took = 0;
                for (int i = 0; i < ndir && took < room; i++) {
                    const int d = dirs[i];
                    const int link = t.w * kDirs + d;
                    const int n = min(heads[d] - in_tail[d], room - took);
                    for (int j = 0; j < n; j++)
                        S.in_ring[(ih + took + j) & (kInRing - 1)] =
                            __ldcg(a.slots + (size_t)link * a.cap + (in_tail[d] + j) % a.cap);
                    if (n > 0) {
                        in_tail[d] += n;
                        took += n;
                        st_release(a.ctl + (size_t)link * 32 + 16, in_tail[d]);
                    }
                }
                if (took > 0) {
                    __threadfence_block();
                    S.in_head = ih + took;
                    atomicSub(&a.hdr->pending, took);
                    work = true;
                }
            }
            // ---- outbound: send queued border updates in order
            while (S.out_tail != S.out_head) {
                const int ot = S.out_tail;
                __threadfence_block();
                const int4 rec = S.out_rec[ot & (kORing - 1)];
                const int mask = S.out_mask[ot & (kORing - 1)];
                bool room = true;
                for (int d = 0; d < kDirs && room; d++) {
                    if (!(mask >> d & 1)) continue;
                    int dr, dc;
                    dir_offset(d, dr, dc);
                    const int link = ((t.ta + dr) * a.G1 + (t.tb + dc)) * kDirs + (7 - d);
                    if (out_head[d] - out_tail[d] >= a.cap) {
                        out_tail[d] = ld_acquire(a.ctl + (size_t)link * 32 + 16);
                        room = out_head[d] - out_tail[d] < a.cap;
                    }
                }
                if (!room) break;
                atomicAdd(&a.hdr->pending, __popc(mask));
                for (int d = 0; d < kDirs; d++) {
                    if (!(mask >> d & 1)) continue;
                    int dr, dc;
                    dir_offset(d, dr, dc);
                    const int link = ((t.ta + dr) * a.G1 + (t.tb + dc)) * kDirs + (7 - d);
                    __stcg(a.slots + (size_t)link * a.cap + out_head[d] % a.cap, rec);
                    out_head[d]++;
                    st_release(a.ctl + (size_t)link * 32, out_head[d]);
                }
                n_sent += __popc(mask);
                __threadfence_block();
                S.out_tail = ot + 1;
                work = true;
            }
            // ---- pause request of the compute leader
            if (!idle && S.idle_seq != S.resp_seq) {
                if (S.in_head != S.in_tail || S.out_head != S.out_tail) {
                    S.resp_kind = RESP_WOKEN;
                    __threadfence_block();
                    S.resp_seq = S.idle_seq;
                } else {
                    atomicSub(&a.hdr->pending, 1);
                    idle = true;
                }
                work = true;
            }
            if (idle && ld_acquire(&a.hdr->pending) == 0) {
                S.resp_kind = RESP_TERMINATE;
                __threadfence_block();
                S.resp_seq = S.idle_seq;
                break;
            }
            if (++spins >= 64 || !work) {
                spins = 0;
                const int st = ld_relaxed(&a.hdr->stop);
                const bool late = globaltimer_ns() > deadline;
                if (late) set_stop(a.hdr, CSC_ERR_TIMEOUT);
                if (st || late) {
                    S.stop = 1;
                    S.resp_kind = RESP_TERMINATE;
                    __threadfence_block();
                    S.resp_seq = S.idle_seq;
                    break;
                }
            }
            if (!work) __nanosleep(idle ? 200 : 32);
        }
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_MESSAGES], (unsigned long long)n_sent);
        atomicAdd(&a.hdr->tmax[3], (unsigned long long)n_wake);
        return;
    }

    // ========================================================= compute threads
    real guard = real(0);
    if (a.guard_on) {
        double g = 1e300;
        for (int k = 0; k < a.K; k++) g = fmin(g, 50.0 / a.dmax[k]);
        guard = real(g);
    }
    const float inv_sub0 = 1.f / a.sub0, inv_sub1 = 1.f / a.sub1, inv_K = 1.f / t.K;
    const float inv_t0 = 1.f / a.t0, inv_t1 = 1.f / a.t1, inv_W1 = 1.f / a.W1, inv_WW = 1.f / t.WW;
    // fixed per-thread offsets: window entry (r, first atom) and position in a
    // full sub-domain (dr, dc, first atom)
    WinThread wt;
    wt.fits = t.WW <= kAsyncCompute;
    wt.kstep = wt.fits ? kAsyncCompute / t.WW : 1;
    wt.on = wt.fits && tid < wt.kstep * t.WW;
    wt.r = wt.fits ? tid % t.WW : 0;
    wt.k0 = wt.fits ? tid / t.WW : 0;
    wt.di = wt.r / a.W1 - (a.L0 - 1);
    wt.dj = wt.r % a.W1 - (a.L1 - 1);
    const int nbf = a.sub0 * a.sub1;
    const bool s_fits = nbf <= kAsyncCompute;
    const int s_kstep = s_fits ? kAsyncCompute / nbf : 1;
    const bool s_on = s_fits && tid < s_kstep * nbf;
    const int s_r = s_fits ? tid % nbf : 0, s_k0 = s_fits ? tid / nbf : 0;
    const int s_dr = s_r / a.sub1, s_dc = s_r % a.sub1;
    // counters and the timeline are the leader's (thread 0)
    int n_upd = 0, n_it = 0, n_rej = 0, n_sub = 0, n_def = 0, n_step = 0;
    long long n_cand = 0;  // positions scanned (times K at the end)
    if (tid == 0) {
        for (int i = 0; i < 6; i++) S.ph[i] = 0;
        S.t_last = S.t_pause = 0;
        S.tc = clock64();
    }
    auto lap = [&](int i) {
        if (tid == 0) {
            const unsigned long long c = clock64();
            S.ph[i] += c - S.tc;
            S.tc = c;
        }
    };
    // leader state: dirty sub-domains as a bit mask, cyclic cursor, inbox tail
    unsigned long long dmask = M >= 64 ? ~0ull : ((1ull << M) - 1ull);
    int cursor = 0, in_tail = 0, par = 0;
    for (;; par ^= 1) {
        // ---- top: the leader picks the next piece of work; this barrier
        // also closes the previous step's window update
        if (tid == 0) {
            int nm = S.in_head - in_tail, m = -1, bstop = S.stop;
            while (!bstop && nm == 0) {
                if (dmask) {
                    const unsigned long long x = dmask >> cursor;
                    m = x ? cursor + __ffsll((long long)x) - 1 : __ffsll((long long)dmask) - 1;
                    break;
                }
                // nothing to do: pause until a record arrives or every tile is done
                if (!S.t_pause) S.t_pause = globaltimer_ns();
                const unsigned long long tp = clock64();
                const int seq = S.idle_seq + 1;
                __threadfence_block();
                S.idle_seq = seq;
                const unsigned long long late = deadline + 2000000000ull;
                while (S.resp_seq != seq) {
                    if (globaltimer_ns() > late) {
                        set_stop(a.hdr, CSC_ERR_TIMEOUT);
                        S.stop = 1;
                        break;
                    }
                    __nanosleep(64);
                }
                S.ph[5] += clock64() - tp;
                bstop = S.stop || S.resp_kind == RESP_TERMINATE;
                nm = S.in_head - in_tail;
            }
            if (m >= 0 && nm == 0) {
                dmask &= ~(1ull << m);
                cursor = m + 1 < M ? m + 1 : 0;
            }
            S.b_m[par] = nm == 0 ? m : -1;
            S.b_nmsg[par] = nm;
            S.b_stop[par] = bstop;
        }
        cbar();
        lap(0);
        const int bstop = S.b_stop[par], nmsg = S.b_nmsg[par], m = S.b_m[par];
        if (bstop) break;
        n_step++;
        if (nmsg > 0) {
            // ---- neighbour updates (Alg. 3 "receive messages and update beta")
            const int base = in_tail;  // equal in every thread: the leader's copy
            for (int i = 0; i < nmsg; i++) {
                const int4 msg = S.in_ring[(base + i) & (kInRing - 1)];
                real dz;
                unpack_msg(msg, dz);
                const int gi = div_small(msg.y, a.Z1, 1.f / a.Z1);
                const int li0 = gi - t.or0, lj0 = msg.y - gi * a.Z1 - t.oc0;
                const int kmsg = msg.x;
                for_window<real, NT>(a, t, wt, li0, lj0, inv_WW, inv_W1, [&](int k, int r, int idx, int, int) {
                    const real c = t.sdtd[((size_t)kmsg * t.K + k) * t.WW + r];
                    atomicAdd(&t.sbeta[idx], -(c * dz));
                });
            }
            cbar();
            for (int i = 0; i < nmsg; i++) {
                const int4 msg = S.in_ring[(base + i) & (kInRing - 1)];
                const int gi = div_small(msg.y, a.Z1, 1.f / a.Z1);
                const int li0 = gi - t.or0, lj0 = msg.y - gi * a.Z1 - t.oc0;
                for_window<real, NT>(a, t, wt, li0, lj0, inv_WW, inv_W1, [&](int k, int, int idx, int li, int lj) {
                    if (near_neighbour<real, NT>(a, t, li, lj))
                        st_relaxed(a.beta + k * plane + (size_t)(t.or0 + li) * a.Z1 + t.oc0 + lj, t.sbeta[idx]);
                });
                if (tid == 0) mark_window<real, NT>(a, t, dmask, li0, lj0, inv_sub0, inv_sub1);
            }
            cbar();
            in_tail = base + nmsg;
            if (tid == 0) {
                __threadfence_block();
                S.in_tail = in_tail;
            }
            lap(1);
            continue;
        }
        if (m < 0) continue;
        // ---- candidate scan of C_m (Eq. pb_coord) with the oracle's tie-break
        const int mr = div_small(m, t.ns1, 1.f / t.ns1), mc = m - mr * t.ns1;
        const int r0 = mr * a.sub0, c0 = mc * a.sub1;
        const int bh = min(a.sub0, t.h - r0), bw = min(a.sub1, t.wd - c0), nb = bh * bw;
        real ba = real(-1);
        unsigned bkey = 0xffffffffu;
        auto consider = [&](int base, int k) {
            const int idx = base + k * t.TS;
            const real d = abs_real(coord_update(t.sbeta[idx], a.lambda, t.snrm[k], t.sinv[k]) - t.sz[idx]);
            const unsigned key = (unsigned)base * (unsigned)t.K + (unsigned)k;
            if (d > ba || (d == ba && key < bkey)) {
                ba = d;
                bkey = key;
            }
        };
        if (s_fits && bh == a.sub0 && bw == a.sub1) {
            if (s_on) {
                const int base = (r0 + s_dr) * a.t1 + c0 + s_dc;
#pragma unroll 4
                for (int k = s_k0; k < t.K; k += s_kstep) consider(base, k);
            }
        } else {
            const float inv_nb = 1.f / nb, inv_bw = 1.f / bw;
            for (int q = tid; q < t.K * nb; q += kAsyncCompute) {
                const int k = div_small(q, nb, inv_nb), r = q - k * nb;
                const int dr = div_small(r, bw, inv_bw);
                consider((r0 + dr) * a.t1 + c0 + (r - dr * bw), k);
            }
        }
        unsigned long long best_bits = 0;
        unsigned best_key = 0xffffffffu;
        {
            unsigned long long wb;
            const unsigned wkey = warp_argmax(ba, bkey, wb);
            if constexpr (sizeof(real) == 4) {
                // (bits, ~key) packed: the largest packed value is the winner
                if (lane == 0) S.p_best[warp] = wkey == 0xffffffffu ? 0ull : (wb << 32) | (0xffffffffu - wkey);
                cbar();
                unsigned long long pk = 0;
#pragma unroll
                for (int w = 0; w < kAW; w++) pk = S.p_best[w] > pk ? S.p_best[w] : pk;
                best_bits = pk >> 32;
                best_key = 0xffffffffu - (unsigned)(pk & 0xffffffffull);
            } else {
                if (lane == 0) {
                    S.p_key[warp] = wkey;
                    S.p_best[warp] = wkey == 0xffffffffu ? 0ull : wb;
                }
                cbar();
#pragma unroll
                for (int w = 0; w < kAW; w++) {
                    const unsigned long long bb = S.p_best[w];
                    const unsigned kk = S.p_key[w];
                    if (bb > best_bits || (bb == best_bits && bb != 0 && kk < best_key)) {
                        best_bits = bb;
                        best_key = kk;
                    }
                }
            }
        }
        n_it++;
        n_cand += nb;
        lap(2);
        if (best_bits == 0) {
            n_sub++;
            continue;
        }
        const int pos = div_small((int)best_key, t.K, inv_K);
        const int k0 = (int)best_key - pos * t.K;
        const int li0 = div_small(pos, a.t1, inv_t1), lj0 = pos - li0 * a.t1;
        const int idx0 = k0 * t.TS + li0 * a.t1 + lj0;
        const real znew = coord_update(t.sbeta[idx0], a.lambda, t.snrm[k0], t.sinv[k0]);
        const real dz = znew - t.sz[idx0];
        const real adz = abs_real(dz);
        if (!(adz >= a.eps)) {
            n_sub++;
            continue;
        }
        const bool border = near_neighbour<real, NT>(a, t, li0, lj0);
        int dl[kDirs], nd = 0;
        if (border) {
            // soft-lock over the part of V(s0) in other tiles (Eq. soft_lock)
            unsigned long long lo = 0, hi = 0;
            if (a.mode == CSC_MODE_ASYNC) {
                // all loads of a batch are issued before any is used
                constexpr int B = sizeof(real) == 4 ? 6 : 3;
                const int gi0 = t.or0 + li0 - (a.L0 - 1), gj0 = t.oc0 + lj0 - (a.L1 - 1);
                const int WW = t.WW, KW = t.K * WW;
                const int kinc = kAsyncCompute / WW, rinc = kAsyncCompute - kinc * WW;
                int k = wt.fits ? wt.k0 : tid / WW, r = wt.fits ? wt.r : tid % WW;
                for (int base = tid; base < KW; base += B * kAsyncCompute) {
                    real vb[B], vz[B];
                    int kk[B], side[B];
#pragma unroll
                    for (int u = 0; u < B; u++) {
                        side[u] = 0;
                        kk[u] = k;
                        vb[u] = vz[u] = real(0);
                        if (base + u * kAsyncCompute < KW) {
                            const int di = div_small(r, a.W1, inv_W1);
                            const int gi = gi0 + di, gj = gj0 + (r - di * a.W1);
                            const bool in_dom = gi >= 0 && gi < a.Z0 && gj >= 0 && gj < a.Z1;
                            const bool in_tile =
                                gi >= t.or0 && gi < t.or0 + t.h && gj >= t.oc0 && gj < t.oc0 + t.wd;
                            if (in_dom && !in_tile) {
                                const size_t g = k * plane + (size_t)gi * a.Z1 + gj;
                                vb[u] = __ldcg(a.beta + g);
                                vz[u] = __ldcg(a.Z + g);
                                const int owner = div_small(gi, a.t0, inv_t0) * a.G1 + div_small(gj, a.t1, inv_t1);
                                side[u] = owner < t.w ? 1 : 2;
                            }
                        }
                        k += kinc;
                        r += rinc;
                        if (r >= WW) {
                            r -= WW;
                            k++;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < B; u++) {
                        if (!side[u]) continue;
                        const unsigned long long bb = sl_bits(
                            abs_real(coord_update(vb[u], a.lambda, t.snrm[kk[u]], t.sinv[kk[u]]) - vz[u]));
                        if (side[u] == 1) lo = bb > lo ? bb : lo;
                        else hi = bb > hi ? bb : hi;
                    }
                }
                if constexpr (sizeof(real) == 4) {
                    // |dZ| bits + 1 fit 32 bits in FP32
                    lo = __reduce_max_sync(0xffffffffu, (unsigned)lo);
                    hi = __reduce_max_sync(0xffffffffu, (unsigned)hi);
                } else {
                    lo = warp_max_u64(lo, 0);
                    hi = warp_max_u64(hi, 0);
                }
            }
            if (lane == 0) {
                S.p_lo[warp] = lo;
                S.p_hi[warp] = hi;
            }
            if (tid == 0) {
                // room on the outgoing ring for the record (only ever grows meanwhile)
                nd = target_dirs<real, NT>(a, t, li0, lj0, dl);
                S.b_ok = nd == 0 || S.out_head - S.out_tail < kORing;
            }
            cbar();
            unsigned long long mlo = 0, mhi = 0;
#pragma unroll
            for (int w = 0; w < kAW; w++) {
                mlo = S.p_lo[w] > mlo ? S.p_lo[w] : mlo;
                mhi = S.p_hi[w] > mhi ? S.p_hi[w] : mhi;
            }
            const unsigned long long mine = sl_bits(adz);
            const bool accept = mine > mlo && mine >= mhi;
            lap(3);
            if (!accept || !S.b_ok) {
                if (tid == 0) {
                    dmask |= 1ull << m;  // try again later
                    if (!accept) n_rej++;
                    else n_def++;
                }
                continue;
            }
        }
        // ---- beta window update (Eq. beta_update), border entries published;
        // the next step's top barrier closes it
        {
            for_window<real, NT>(a, t, wt, li0, lj0, inv_WW, inv_W1, [&](int k, int r, int idx, int li, int lj) {
                if (k == k0 && li == li0 && lj == lj0) return;
                const real c = t.sdtd[((size_t)k0 * t.K + k) * t.WW + r];
                const real v = sub_prod(t.sbeta[idx], c, dz);
                t.sbeta[idx] = v;
                if (near_neighbour<real, NT>(a, t, li, lj))
                    st_relaxed(a.beta + k * plane + (size_t)(t.or0 + li) * a.Z1 + t.oc0 + lj, v);
            });
        }
        if (tid == 0) {
            t.sz[idx0] = znew;
            const int gpos = (t.or0 + li0) * a.Z1 + t.oc0 + lj0;
            if (border) st_relaxed(a.Z + k0 * plane + gpos, znew);
            mark_window<real, NT>(a, t, dmask, li0, lj0, inv_sub0, inv_sub1);
            if (nd > 0) {
                int mask = 0;
                for (int i = 0; i < nd; i++) mask |= 1 << dl[i];
                const int oh = S.out_head;
                S.out_rec[oh & (kORing - 1)] = pack_msg(k0, gpos, dz);
                S.out_mask[oh & (kORing - 1)] = mask;
                __threadfence_block();
                S.out_head = oh + 1;
            }
            n_upd++;
            S.t_last = clock64();
            if (a.max_updates > 0) {
                const unsigned long long prev = atomicAdd(&a.hdr->updates_total, 1ull);
                if ((long long)prev + 1 >= a.max_updates) set_stop(a.hdr, CSC_NOT_CONVERGED);
            }
            if (a.guard_on && abs_real(znew) > guard) set_stop(a.hdr, CSC_ERR_DIVERGED);
        }
        lap(4);
    }
    // wait (bounded) for the communication warp before the tile is written back
    if (tid == 0) {
        const unsigned long long late = deadline + 4000000000ull;
        while (S.resp_kind != RESP_TERMINATE && !S.stop && globaltimer_ns() < late) __nanosleep(64);
    }
    cbar();
    const int hw = t.h * t.wd;
    for (int q = tid; q < t.K * hw; q += kAsyncCompute) {
        const int k = q / hw, r = q % hw, li = r / t.wd, lj = r % t.wd;
        const size_t g = k * plane + (size_t)(t.or0 + li) * a.Z1 + t.oc0 + lj;
        a.beta[g] = t.sbeta[k * t.TS + li * a.t1 + lj];
        a.Z[g] = t.sz[k * t.TS + li * a.t1 + lj];
    }
    if (tid == 0) {
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_UPDATES], (unsigned long long)n_upd);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_ITERS], (unsigned long long)n_it);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_CAND], (unsigned long long)(n_cand * t.K));
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_REJECTED], (unsigned long long)n_rej);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_SUBTOL], (unsigned long long)n_sub);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_DEFERRED], (unsigned long long)n_def);
        atomicMax(&a.hdr->wmax[0], (unsigned long long)n_step);
        atomicMax(&a.hdr->wmax[1], (unsigned long long)n_upd);
        if (S.t_last) {
            // SM cycles of the last update converted with this tile's own clock rate
            const unsigned long long c_end = clock64(), g_end = globaltimer_ns();
            const double ns_per_cycle = c_end > c_start ? (double)(g_end - t_start) / (double)(c_end - c_start) : 0.0;
            atomicMax(&a.hdr->tmax[0], (unsigned long long)((double)(S.t_last - c_start) * ns_per_cycle));
        }
        atomicMax(&a.hdr->tmax[1], globaltimer_ns() - t_start);
        if (S.t_pause) atomicMax(&a.hdr->tmax[2], S.t_pause - t_start);
        for (int i = 0; i < 6; i++) {
            atomicAdd(&a.hdr->tph[i], S.ph[i]);
            atomicMax(&a.hdr->tphmax[i], S.ph[i]);
        }
    }
}

const void *lgcd_async_kernel_ptr(float) { return (const void *)lgcd_async_kernel<float>; }
const void *lgcd_async_kernel_ptr(double) { return (const void *)lgcd_async_kernel<double>; }

}  // namespace csc
