// lgcd.cu -- persistent locally greedy coordinate descent over a grid of
// worker tiles (Alg. 1 run inside each worker of Alg. 3).
//
// One CTA owns one tile S_w of the activation domain and keeps beta and Z of
// that tile in shared memory, with the K x K x |window| table of
// Eq. beta_update.  Each iteration scans one sub-domain C_m of the tile
// (boxes of side 2L_i, cyclic order m = q mod M), takes the largest
// |dZ| = |ST(beta, lambda)/||D_k||^2 - Z| and, when it is at least eps,
// applies it and the beta window update.
//
// Neighbouring tiles exchange the triplets (k0, s0, dZ) of updates whose
// window V(s0) leaves the tile (Alg. 3) through single-producer /
// single-consumer ring buffers in global memory (release/acquire on the head
// and tail words).  Instead of mirroring the neighbours' beta and Z on an
// extension E_L(S_w), every tile publishes the beta and Z entries of its own
// border band (within L_i - 1 of an edge) to the global arrays as they change
// ("write-through"); the soft-lock test of Eq. soft_lock reads the
// neighbours' current values there.  Both sides of a soft-lock comparison
// therefore evaluate the same stored bits.
//
// Modes: ASYNC (soft-lock on border candidates, Section 4.1), NOLOCK (the
// same without the test, the ablation of Section 5.1) and PHASED (tiles run
// in checkerboard colour phases separated by grid barriers, which makes the
// run deterministic and equal to a sequential schedule).
//
// Termination without a central server (Alg. 3 "global convergence"): the
// word `pending` counts active workers plus messages in flight.  A worker that
// finished a full sweep of its M sub-domains without seeing |dZ| >= eps and
// without receiving a message decrements it and waits; a message wakes it
// (it increments before consuming).  pending == 0 is stable and means that no
// coordinate anywhere can move by eps.  Every wait is bounded by a deadline
// from %globaltimer and by the shared stop word.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace csc {

template <typename real>
struct LgcdArgs {
    real *beta;
    real *Z;
    const real *dtd;
    const double *nrm;
    const double *dmax;
    WsHeader *hdr;
    int4 *slots;  // [G][kDirs][cap] records
    int *ctl;     // [G][kDirs][32]: head at +0, tail at +16
    int K, Z0, Z1, L0, L1, W0, W1;
    int G0, G1, t0, t1, sub0, sub1;
    int mode, guard_on, cap, Mmax;
    real lambda, eps;
    long long max_updates;
    unsigned long long timeout_ns;
};

template <typename real>
struct Cand {
    real a;        // |dZ|
    unsigned key;  // (row-major position in the tile) * K + k
    real znew;     // Z' = ST(beta, lambda) / ||D_k||^2
    real dz;       // Z' - Z
};

template <typename real>
__device__ __forceinline__ bool better(const Cand<real> &x, const Cand<real> &y) {
    return x.a > y.a || (x.a == y.a && x.key < y.key);
}

__device__ __forceinline__ int4 pack_msg(int k, int s, float dz) {
    return make_int4(k, s, __float_as_int(dz), 0);
}
__device__ __forceinline__ int4 pack_msg(int k, int s, double dz) {
    long long b = __double_as_longlong(dz);
    return make_int4(k, s, (int)(b & 0xffffffffll), (int)(b >> 32));
}
__device__ __forceinline__ void unpack_msg(const int4 &m, float &dz) { dz = __int_as_float(m.z); }
__device__ __forceinline__ void unpack_msg(const int4 &m, double &dz) {
    long long b = ((long long)(unsigned)m.z) | ((long long)m.w << 32);
    dz = __longlong_as_double(b);
}

__device__ __forceinline__ void fence_acq_rel_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

constexpr int kMsgBatch = 64;

// Direction index of neighbour offset (dr, dc) in {-1,0,1}^2 \ {(0,0)};
// the opposite direction is 7 - dir.
__device__ __forceinline__ int dir_index(int dr, int dc) {
    int q = (dr + 1) * 3 + (dc + 1);
    return q < 4 ? q : q - 1;
}
__device__ __forceinline__ void dir_offset(int dir, int &dr, int &dc) {
    int q = dir < 4 ? dir : dir + 1;
    dr = q / 3 - 1;
    dc = q % 3 - 1;
}

template <typename real, int NT>
struct Tile {
    // geometry of this worker
    int ta, tb, w, or0, oc0, h, wd, TS, K, WW, M, ns1;
    real *sbeta, *sz, *sdtd, *snrm, *sinv;
    int4 *smsg;
};

// Block-wide argmax of Cand with the tie-break of the oracle (larger |dZ|,
// then smaller row-major position, then smaller k).  Result broadcast.
template <typename real, int NT>
__device__ __forceinline__ Cand<real> block_argmax(Cand<real> c) {
    __shared__ Cand<real> red[NT / 32];
    __shared__ Cand<real> res;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Cand<real> y;
        y.a = __shfl_xor_sync(0xffffffffu, c.a, o);
        y.key = __shfl_xor_sync(0xffffffffu, c.key, o);
        y.znew = __shfl_xor_sync(0xffffffffu, c.znew, o);
        y.dz = __shfl_xor_sync(0xffffffffu, c.dz, o);
        if (better(y, c)) c = y;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        Cand<real> x = threadIdx.x < NT / 32 ? red[threadIdx.x] : Cand<real>{real(-1), 0xffffffffu, real(0), real(0)};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            Cand<real> y;
            y.a = __shfl_xor_sync(0xffffffffu, x.a, o);
            y.key = __shfl_xor_sync(0xffffffffu, x.key, o);
            y.znew = __shfl_xor_sync(0xffffffffu, x.znew, o);
            y.dz = __shfl_xor_sync(0xffffffffu, x.dz, o);
            if (better(y, x)) x = y;
        }
        if (threadIdx.x == 0) res = x;
    }
    __syncthreads();
    return res;
}

template <typename real, int NT>
__device__ __forceinline__ real block_max2(real v, real u, real *out_u) {
    __shared__ real r1[NT / 32], r2[NT / 32];
    __shared__ real o1, o2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        u = max(u, __shfl_xor_sync(0xffffffffu, u, o));
    }
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = v;
        r2[threadIdx.x >> 5] = u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        real a = r1[0], b = r2[0];
        for (int i = 1; i < NT / 32; i++) {
            a = max(a, r1[i]);
            b = max(b, r2[i]);
        }
        o1 = a;
        o2 = b;
    }
    __syncthreads();
    *out_u = o2;
    return o1;
}

// ------------------------------------------------------------ tile setup
template <typename real, int NT>
__device__ void tile_setup(const LgcdArgs<real> &a, Tile<real, NT> &t, unsigned char *smem) {
    t.w = blockIdx.x;
    t.ta = t.w / a.G1;
    t.tb = t.w % a.G1;
    t.or0 = t.ta * a.t0;
    t.oc0 = t.tb * a.t1;
    t.h = min(a.t0, a.Z0 - t.or0);
    t.wd = min(a.t1, a.Z1 - t.oc0);
    t.TS = a.t0 * a.t1;
    t.K = a.K;
    t.WW = a.W0 * a.W1;
    int ns0 = (t.h + a.sub0 - 1) / a.sub0;
    t.ns1 = (t.wd + a.sub1 - 1) / a.sub1;
    t.M = ns0 * t.ns1;
    t.sbeta = reinterpret_cast<real *>(smem);
    t.sz = t.sbeta + (size_t)t.K * t.TS;
    t.sdtd = t.sz + (size_t)t.K * t.TS;
    t.snrm = t.sdtd + (size_t)t.K * t.K * t.WW;
    t.sinv = t.snrm + t.K;
    size_t off = (size_t)(t.sinv + t.K - reinterpret_cast<real *>(smem)) * sizeof(real);
    off = (off + 15) & ~(size_t)15;
    t.smsg = reinterpret_cast<int4 *>(smem + off);

    const int K = t.K, hw = t.h * t.wd;
    for (int q = threadIdx.x; q < K * hw; q += NT) {
        int k = q / hw, r = q % hw, li = r / t.wd, lj = r % t.wd;
        size_t g = ((size_t)k * a.Z0 + t.or0 + li) * a.Z1 + t.oc0 + lj;
        t.sbeta[k * t.TS + li * a.t1 + lj] = a.beta[g];
        t.sz[k * t.TS + li * a.t1 + lj] = a.Z[g];
    }
    // sdtd[k0][k][w] = C_{k,k0}[w]: the row read by an update of atom k0.
    for (int q = threadIdx.x; q < K * K * t.WW; q += NT) {
        int k0 = q / (K * t.WW), r = q % (K * t.WW), k = r / t.WW, ww = r % t.WW;
        t.sdtd[q] = a.dtd[((size_t)k * K + k0) * t.WW + ww];
    }
    for (int k = threadIdx.x; k < K; k += NT) {
        t.snrm[k] = real(a.nrm[k]);
        t.sinv[k] = real(1.0 / a.nrm[k]);
    }
    __syncthreads();
}

__device__ __forceinline__ bool in_band(int li, int lj, int h, int wd, int L0, int L1) {
    return li < L0 - 1 || li >= h - (L0 - 1) || lj < L1 - 1 || lj >= wd - (L1 - 1);
}

// Scan of sub-domain m: the candidate of Eq. gcd_candidate.
template <typename real, int NT>
__device__ __forceinline__ Cand<real> scan_subdomain(const LgcdArgs<real> &a, const Tile<real, NT> &t,
                                                     int m) {
    const int mr = m / t.ns1, mc = m % t.ns1;
    const int r0 = mr * a.sub0, c0 = mc * a.sub1;
    const int bh = min(a.sub0, t.h - r0), bw = min(a.sub1, t.wd - c0);
    const int nb = bh * bw, n = t.K * nb;
    Cand<real> c{real(-1), 0xffffffffu, real(0), real(0)};
    for (int q = threadIdx.x; q < n; q += NT) {
        int k = q / nb, r = q % nb;
        int li = r0 + r / bw, lj = c0 + r % bw;
        int idx = k * t.TS + li * a.t1 + lj;
        real zn = coord_update(t.sbeta[idx], a.lambda, t.snrm[k], t.sinv[k]);
        real dz = zn - t.sz[idx];
        Cand<real> x{dz < real(0) ? -dz : dz, (unsigned)((li * a.t1 + lj) * t.K + k), zn, dz};
        if (better(x, c)) c = x;
    }
    return block_argmax<real, NT>(c);
}

// Soft-lock test (Eq. soft_lock): the largest |dZ| over K x (V(s0) outside
// the tile), read from the neighbours' published band, split by whether the
// owning tile has a lower or a higher index.
template <typename real, int NT>
__device__ __forceinline__ void softlock_maxima(const LgcdArgs<real> &a, const Tile<real, NT> &t,
                                                int li0, int lj0, real *m_lo, real *m_hi) {
    real lo = real(-1), hi = real(-1);
    const int gi0 = t.or0 + li0, gj0 = t.oc0 + lj0;
    for (int q = threadIdx.x; q < t.K * t.WW; q += NT) {
        int k = q / t.WW, r = q % t.WW;
        int gi = gi0 + r / a.W1 - (a.L0 - 1), gj = gj0 + r % a.W1 - (a.L1 - 1);
        if (gi < 0 || gi >= a.Z0 || gj < 0 || gj >= a.Z1) continue;
        if (gi >= t.or0 && gi < t.or0 + t.h && gj >= t.oc0 && gj < t.oc0 + t.wd) continue;
        size_t g = ((size_t)k * a.Z0 + gi) * a.Z1 + gj;
        real b = ld_relaxed(a.beta + g), z = ld_relaxed(a.Z + g);
        real d = coord_update(b, a.lambda, t.snrm[k], t.sinv[k]) - z;
        d = d < real(0) ? -d : d;
        int owner = (gi / a.t0) * a.G1 + gj / a.t1;
        if (owner < t.w) lo = max(lo, d);
        else hi = max(hi, d);
    }
    *m_lo = block_max2<real, NT>(lo, hi, m_hi);
}

// beta_k[s] -= C[k][k0][s - s0] dz over V(s0) inside the tile, except
// (k0, s0) itself (Eq. beta_update); border entries are published.
template <typename real, int NT>
__device__ __forceinline__ void apply_own_update(const LgcdArgs<real> &a, const Tile<real, NT> &t,
                                                 int k0, int li0, int lj0, real dz) {
    const real *row = t.sdtd + (size_t)k0 * t.K * t.WW;
    for (int q = threadIdx.x; q < t.K * t.WW; q += NT) {
        int k = q / t.WW, r = q % t.WW;
        int di = r / a.W1 - (a.L0 - 1), dj = r % a.W1 - (a.L1 - 1);
        int li = li0 + di, lj = lj0 + dj;
        if (li < 0 || li >= t.h || lj < 0 || lj >= t.wd) continue;
        if (k == k0 && di == 0 && dj == 0) continue;
        int idx = k * t.TS + li * a.t1 + lj;
        real v = sub_prod(t.sbeta[idx], row[q], dz);
        t.sbeta[idx] = v;
        if (in_band(li, lj, t.h, t.wd, a.L0, a.L1))
            st_relaxed(a.beta + ((size_t)k * a.Z0 + t.or0 + li) * a.Z1 + t.oc0 + lj, v);
    }
}

// Apply staged neighbour messages to the tile's beta.  Windows of different
// messages may overlap, so the updates are shared-memory atomics; each
// touched entry lies in the border band and is published afterwards.
template <typename real, int NT>
__device__ __forceinline__ void apply_messages(const LgcdArgs<real> &a, const Tile<real, NT> &t,
                                               int nmsg) {
    const int per = t.K * t.WW;
    for (int q = threadIdx.x; q < nmsg * per; q += NT) {
        int mi = q / per, e = q % per;
        int4 m = t.smsg[mi];
        real dz;
        unpack_msg(m, dz);
        int gi = m.y / a.Z1, gj = m.y % a.Z1;
        int k = e / t.WW, r = e % t.WW;
        int li = gi - t.or0 + r / a.W1 - (a.L0 - 1), lj = gj - t.oc0 + r % a.W1 - (a.L1 - 1);
        if (li < 0 || li >= t.h || lj < 0 || lj >= t.wd) continue;
        real c = t.sdtd[((size_t)m.x * t.K + k) * t.WW + r];
        atomicAdd(&t.sbeta[k * t.TS + li * a.t1 + lj], -(c * dz));
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nmsg * per; q += NT) {
        int mi = q / per, e = q % per;
        int4 m = t.smsg[mi];
        int gi = m.y / a.Z1, gj = m.y % a.Z1;
        int k = e / t.WW, r = e % t.WW;
        int li = gi - t.or0 + r / a.W1 - (a.L0 - 1), lj = gj - t.oc0 + r % a.W1 - (a.L1 - 1);
        if (li < 0 || li >= t.h || lj < 0 || lj >= t.wd) continue;
        int idx = k * t.TS + li * a.t1 + lj;
        st_relaxed(a.beta + ((size_t)k * a.Z0 + t.or0 + li) * a.Z1 + t.oc0 + lj, t.sbeta[idx]);
    }
}

// Control state of thread 0 (the only thread that touches mailboxes).
struct Comm {
    int out_head[kDirs];
    int out_tail[kDirs];  // cached tails of the neighbours' inboxes
    int in_tail[kDirs];
    int prefetch[kDirs];  // relaxed-loaded heads of own inboxes
    int ndir;
    int dirs[kDirs];
};

// Neighbour directions whose tile V(s0) reaches.
template <typename real, int NT>
__device__ __forceinline__ int target_dirs(const LgcdArgs<real> &a, const Tile<real, NT> &t, int li0,
                                           int lj0, int *dirs) {
    int n = 0;
    for (int dr = -1; dr <= 1; dr++) {
        if (dr == -1 && !(t.ta > 0 && li0 < a.L0 - 1)) continue;
        if (dr == 1 && !(t.ta < a.G0 - 1 && li0 + a.L0 - 1 >= t.h)) continue;
        for (int dc = -1; dc <= 1; dc++) {
            if (dr == 0 && dc == 0) continue;
            if (dc == -1 && !(t.tb > 0 && lj0 < a.L1 - 1)) continue;
            if (dc == 1 && !(t.tb < a.G1 - 1 && lj0 + a.L1 - 1 >= t.wd)) continue;
            dirs[n++] = dir_index(dr, dc);
        }
    }
    return n;
}

// Thread 0: room for one record on every target link?
template <typename real, int NT>
__device__ __forceinline__ bool links_have_room(const LgcdArgs<real> &a, const Tile<real, NT> &t,
                                                Comm &cm, const int *dirs, int n) {
    for (int i = 0; i < n; i++) {
        int d = dirs[i], dr, dc;
        dir_offset(d, dr, dc);
        int recv = (t.ta + dr) * a.G1 + (t.tb + dc);
        int link = recv * kDirs + (7 - d);
        if (cm.out_head[d] - cm.out_tail[d] >= a.cap) {
            cm.out_tail[d] = ld_acquire(a.ctl + (size_t)link * 32 + 16);
            if (cm.out_head[d] - cm.out_tail[d] >= a.cap) return false;
        }
    }
    return true;
}

template <typename real, int NT>
__device__ __forceinline__ void post_messages(const LgcdArgs<real> &a, const Tile<real, NT> &t, Comm &cm,
                                              const int *dirs, int n, int k0, int s_lin, real dz) {
    if (n == 0) return;
    atomicAdd(&a.hdr->pending, n);
    int4 rec = pack_msg(k0, s_lin, dz);
    for (int i = 0; i < n; i++) {
        int d = dirs[i], dr, dc;
        dir_offset(d, dr, dc);
        int recv = (t.ta + dr) * a.G1 + (t.tb + dc);
        int link = recv * kDirs + (7 - d);
        int slot = cm.out_head[d] % a.cap;
        __stcg(a.slots + (size_t)link * a.cap + slot, rec);
        cm.out_head[d]++;
        st_release(a.ctl + (size_t)link * 32, cm.out_head[d]);
    }
}

// Thread 0: copy available records of the own inboxes into shared memory
// (heads taken from `heads`), release the consumed slots.  Returns the count.
template <typename real, int NT>
__device__ __forceinline__ int stage_messages(const LgcdArgs<real> &a, const Tile<real, NT> &t, Comm &cm,
                                              const int *heads) {
    int cnt = 0;
    bool any = false;
    for (int i = 0; i < cm.ndir; i++) any |= heads[cm.dirs[i]] != cm.in_tail[cm.dirs[i]];
    if (!any) return 0;
    fence_acq_rel_gpu();
    for (int i = 0; i < cm.ndir && cnt < kMsgBatch; i++) {
        int d = cm.dirs[i];
        int link = t.w * kDirs + d;
        int avail = heads[d] - cm.in_tail[d];
        int take = min(avail, kMsgBatch - cnt);
        for (int j = 0; j < take; j++)
            t.smsg[cnt++] = __ldcg(a.slots + (size_t)link * a.cap + (cm.in_tail[d] + j) % a.cap);
        if (take > 0) {
            cm.in_tail[d] += take;
            st_release(a.ctl + (size_t)link * 32 + 16, cm.in_tail[d]);
        }
    }
    return cnt;
}

__device__ __forceinline__ void set_stop(WsHeader *h, int code) { atomicCAS(&h->stop, 0, code); }

template <typename real, int NT>
__device__ void write_back(const LgcdArgs<real> &a, const Tile<real, NT> &t) {
    __syncthreads();
    const int hw = t.h * t.wd;
    for (int q = threadIdx.x; q < t.K * hw; q += NT) {
        int k = q / hw, r = q % hw, li = r / t.wd, lj = r % t.wd;
        size_t g = ((size_t)k * a.Z0 + t.or0 + li) * a.Z1 + t.oc0 + lj;
        a.beta[g] = t.sbeta[k * t.TS + li * a.t1 + lj];
        a.Z[g] = t.sz[k * t.TS + li * a.t1 + lj];
    }
}

// ============================================================ ASYNC / NOLOCK
template <typename real, int NT>
__global__ void __launch_bounds__(NT, 1) lgcd_async_kernel(LgcdArgs<real> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Tile<real, NT> t;
    tile_setup<real, NT>(a, t, smem_raw);

    __shared__ int s_nmsg, s_state, s_accept;
    __shared__ real s_mlo, s_mhi;

    Comm cm;
    long long n_upd = 0, n_it = 0, n_rej = 0, n_sub = 0, n_msg = 0, n_def = 0;
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    real guard = real(0);
    if (a.guard_on) {
        double g = 1e300;
        for (int k = 0; k < a.K; k++) g = fmin(g, 50.0 / a.dmax[k]);
        guard = real(g);
    }
    if (threadIdx.x == 0) {
        cm.ndir = 0;
        for (int d = 0; d < kDirs; d++) {
            int dr, dc;
            dir_offset(d, dr, dc);
            int r = t.ta + dr, c = t.tb + dc;
            cm.out_head[d] = cm.out_tail[d] = cm.in_tail[d] = 0;
            cm.prefetch[d] = 0;
            if (r >= 0 && r < a.G0 && c >= 0 && c < a.G1) cm.dirs[cm.ndir++] = d;
        }
        for (int i = 0; i < cm.ndir; i++)
            cm.prefetch[cm.dirs[i]] = ld_relaxed(a.ctl + ((size_t)t.w * kDirs + cm.dirs[i]) * 32);
    }
    int stop_seen = 0;
    int m = 0, quiet = 0;
    for (;;) {
        // ---- receive (Alg. 3: "receive messages and update beta")
        if (threadIdx.x == 0) {
            int n = stage_messages<real, NT>(a, t, cm, cm.prefetch);
            if (n > 0) atomicSub(&a.hdr->pending, n);
            s_nmsg = n;
            s_state = stop_seen ? 2 : (globaltimer_ns() > deadline ? 3 : 0);
        }
        __syncthreads();
        if (s_state != 0) {
            if (threadIdx.x == 0 && s_state == 3) set_stop(a.hdr, CSC_ERR_TIMEOUT);
            break;
        }
        const int nmsg = s_nmsg;
        if (nmsg > 0) {
            apply_messages<real, NT>(a, t, nmsg);
            __syncthreads();
        }
        // ---- local greedy candidate on C_m
        Cand<real> best = scan_subdomain<real, NT>(a, t, m);
        n_it++;
        bool active = best.a >= a.eps;
        if (active) {
            const unsigned pos = best.key / (unsigned)t.K;
            const int k0 = (int)(best.key % (unsigned)t.K);
            const int li0 = (int)(pos / (unsigned)a.t1), lj0 = (int)(pos % (unsigned)a.t1);
            bool border = in_band(li0, lj0, t.h, t.wd, a.L0, a.L1);
            bool accept = true;
            if (border && a.mode == CSC_MODE_ASYNC) {
                real mlo, mhi;
                softlock_maxima<real, NT>(a, t, li0, lj0, &mlo, &mhi);
                accept = best.a > mlo && best.a >= mhi;
            }
            int dirs[kDirs];
            int nd = 0;
            if (threadIdx.x == 0) {
                if (accept && border) {
                    nd = target_dirs<real, NT>(a, t, li0, lj0, dirs);
                    if (!links_have_room<real, NT>(a, t, cm, dirs, nd)) {
                        accept = false;
                        n_def++;
                    }
                }
                s_accept = accept;
            }
            __syncthreads();
            accept = s_accept;
            if (accept) {
                const int idx0 = k0 * t.TS + li0 * a.t1 + lj0;
                const real dz = best.dz;
                apply_own_update<real, NT>(a, t, k0, li0, lj0, dz);
                if (threadIdx.x == 0) {
                    t.sz[idx0] = best.znew;
                    if (border) {
                        size_t g = ((size_t)k0 * a.Z0 + t.or0 + li0) * a.Z1 + t.oc0 + lj0;
                        st_relaxed(a.Z + g, best.znew);
                    }
                    int s_lin = (t.or0 + li0) * a.Z1 + t.oc0 + lj0;
                    post_messages<real, NT>(a, t, cm, dirs, nd, k0, s_lin, dz);
                    n_msg += nd;
                    n_upd++;
                    if (a.max_updates > 0) {
                        unsigned long long prev = atomicAdd(&a.hdr->updates_total, 1ull);
                        if ((long long)prev + 1 >= a.max_updates) set_stop(a.hdr, CSC_NOT_CONVERGED);
                    }
                    real az = best.znew < real(0) ? -best.znew : best.znew;
                    if (a.guard_on && az > guard) set_stop(a.hdr, CSC_ERR_DIVERGED);
                }
            } else if (threadIdx.x == 0 && border) {
                n_rej++;
            }
        } else {
            n_sub++;
        }
        quiet = (active || nmsg > 0) ? 0 : quiet + 1;
        m = (m + 1 == t.M) ? 0 : m + 1;
        // ---- prefetch control words for the next iteration (relaxed: no stall)
        if (threadIdx.x == 0) {
            for (int i = 0; i < cm.ndir; i++)
                cm.prefetch[cm.dirs[i]] = ld_relaxed(a.ctl + ((size_t)t.w * kDirs + cm.dirs[i]) * 32);
            stop_seen = ld_relaxed(&a.hdr->stop);
        }
        // ---- idle: a full sweep with nothing to do (Alg. 3 pause)
        if (quiet >= t.M) {
            if (threadIdx.x == 0) {
                atomicSub(&a.hdr->pending, 1);
                int state = 0;
                for (;;) {
                    bool wake = false;
                    for (int i = 0; i < cm.ndir; i++) {
                        int d = cm.dirs[i];
                        int hd = ld_relaxed(a.ctl + ((size_t)t.w * kDirs + d) * 32);
                        cm.prefetch[d] = hd;
                        wake |= hd != cm.in_tail[d];
                    }
                    if (wake) {
                        atomicAdd(&a.hdr->pending, 1);
                        state = 0;
                        break;
                    }
                    if (ld_acquire(&a.hdr->pending) == 0) { state = 1; break; }
                    if (ld_relaxed(&a.hdr->stop)) { state = 1; break; }
                    if (globaltimer_ns() > deadline) {
                        set_stop(a.hdr, CSC_ERR_TIMEOUT);
                        state = 1;
                        break;
                    }
                    __nanosleep(256);
                }
                s_state = state;
            }
            __syncthreads();
            if (s_state == 1) break;
            quiet = 0;
        } else {
            __syncthreads();
        }
    }
    write_back<real, NT>(a, t);
    if (threadIdx.x == 0) {
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_UPDATES], (unsigned long long)n_upd);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_ITERS], (unsigned long long)n_it);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_REJECTED], (unsigned long long)n_rej);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_SUBTOL], (unsigned long long)n_sub);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_MESSAGES], (unsigned long long)n_msg);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_DEFERRED], (unsigned long long)n_def);
    }
}

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
    h->maxdz_bits = 0;
    h->obj_f = 0.0;
    h->obj_g = 0.0;
    h->nnz = 0;
    h->overflow = 0;
}

// ============================================================== host side
constexpr int kLgcdThreads = 256;

struct Plan {
    int G0, G1, t0, t1, sub0, sub1;
    size_t smem;
};

static size_t tile_smem(const Geom &g, int t0, int t1, int rs) {
    size_t n = (2 * (size_t)g.K * t0 * t1 + (size_t)g.ntab() + 2 * (size_t)g.K) * rs;
    n = (n + 15) & ~(size_t)15;
    return n + kMsgBatch * sizeof(int4);
}

template <typename real>
static const void *kernel_ptr(int mode) {
    if (mode == CSC_MODE_PHASED) return (const void *)lgcd_phased_kernel<real, kLgcdThreads>;
    return (const void *)lgcd_async_kernel<real, kLgcdThreads>;
}

static int smem_limit() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}
static int num_sms() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
}
static int smem_per_sm() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    return v;
}

// Tile plan.  Full tiles must be at least L_i wide (windows then reach only
// the adjacent tiles); automatic plans use tiles of at least 2 L_i and the
// largest number of workers that can all be resident at once.
static int make_plan(const Geom &g, const csc_solve_opts &o, int rs, Plan *pl) {
    const bool d1 = g.d == 1;
    pl->sub0 = d1 ? 1 : (o.sub[0] > 0 ? o.sub[0] : 2 * g.L0);
    pl->sub1 = d1 ? (o.sub[0] > 0 ? o.sub[0] : 2 * g.L1) : (o.sub[1] > 0 ? o.sub[1] : 2 * g.L1);
    const int lim = smem_limit(), sms = num_sms(), per_sm = smem_per_sm();
    int ut0 = d1 ? 0 : o.tile[0], ut1 = d1 ? o.tile[0] : o.tile[1];
    if (ut0 > 0 || ut1 > 0 || d1 && o.tile[0] > 0) {
        int t0 = d1 ? 1 : (ut0 > 0 ? std::min(ut0, g.Z0) : g.Z0);
        int t1 = ut1 > 0 ? std::min(ut1, g.Z1) : g.Z1;
        if ((t0 < g.L0 && t0 < g.Z0) || (t1 < g.L1 && t1 < g.Z1)) return CSC_ERR_INVALID;
        pl->t0 = t0;
        pl->t1 = t1;
        pl->G0 = (int)ceil_div(g.Z0, t0);
        pl->G1 = (int)ceil_div(g.Z1, t1);
        pl->smem = tile_smem(g, t0, t1, rs);
        if ((int)pl->smem > lim) return CSC_ERR_UNIMPLEMENTED;
        return CSC_OK;
    }
    const int minT0 = d1 ? 1 : std::min(g.Z0, 2 * g.L0), minT1 = std::min(g.Z1, 2 * g.L1);
    const int maxG0 = d1 ? 1 : std::max(1, g.Z0 / minT0), maxG1 = std::max(1, g.Z1 / minT1);
    bool found = false;
    Plan best{};
    long long best_w = 0;
    for (int occ = 1; occ <= 8; occ++) {
        long long cap_w = (long long)occ * sms;
        if (o.max_workers > 0) cap_w = std::min<long long>(cap_w, o.max_workers);
        size_t budget = std::min<size_t>((size_t)lim, (size_t)per_sm / occ - 1024);
        for (int G0 = 1; G0 <= maxG0; G0++) {
            int G1 = (int)std::min<long long>(maxG1, cap_w / G0);
            if (G1 < 1) break;
            for (; G1 >= 1; G1--) {
                int t0 = (int)ceil_div(g.Z0, G0), t1 = (int)ceil_div(g.Z1, G1);
                int a0 = (int)ceil_div(g.Z0, t0), a1 = (int)ceil_div(g.Z1, t1);
                if (tile_smem(g, t0, t1, rs) <= budget) {
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
                        best.smem = tile_smem(g, t0, t1, rs);
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
    const int rs = (int)sizeof(real);
    Plan pl;
    rc = make_plan(g, o, rs, &pl);
    if (rc) return rc;
    const int W = pl.G0 * pl.G1;
    WsLayout L = plan_workspace(g, W, rs);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
    unsigned char *wsb = static_cast<unsigned char *>(ws);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(wsb + L.hdr);
    double *nrm = reinterpret_cast<double *>(wsb + L.nrm);
    double *dmax = reinterpret_cast<double *>(wsb + L.dmax);

    const void *kern = kernel_ptr<real>(o.mode);
    CSC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
    int occ = 0;
    CSC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kLgcdThreads, pl.smem));
    if ((long long)occ * num_sms() < W) return CSC_ERR_UNIMPLEMENTED;

    if (!o.warm_start) CSC_CUDA(cudaMemsetAsync(Z, 0, (size_t)g.nz() * rs, st));
    rc = launch_atom_norms<real>(g, D, nrm, dmax, st);
    if (rc) return rc;

    LgcdArgs<real> a;
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
    a.eps = tol;
    a.max_updates = o.max_updates;
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
    S.tiles[0] = g.d == 1 ? pl.G1 : pl.G0;
    S.tiles[1] = g.d == 1 ? 1 : pl.G1;
    S.tile_size[0] = g.d == 1 ? pl.t1 : pl.t0;
    S.tile_size[1] = g.d == 1 ? 1 : pl.t1;
    cudaEvent_t e0, e1;
    CSC_CUDA(cudaEventCreate(&e0));
    CSC_CUDA(cudaEventCreate(&e1));
    int status = CSC_OK;
    float kms_total = 0.f;
    WsHeader hh;
    for (int round = 0;; round++) {
        CSC_CUDA(cudaMemsetAsync(wsb + L.mbox_ctl, 0, (size_t)W * kDirs * 32 * sizeof(int), st));
        reset_header_kernel<<<1, 1, 0, st>>>(hdr, W);
        CSC_CUDA(cudaGetLastError());
        void *args[] = {&a};
        CSC_CUDA(cudaEventRecord(e0, st));
        CSC_CUDA(cudaLaunchCooperativeKernel(kern, dim3(W), dim3(kLgcdThreads), args, pl.smem, st));
        CSC_CUDA(cudaEventRecord(e1, st));
        // stop word -> status, then the solve counters
        CSC_CUDA(cudaMemcpyAsync(&hh, hdr, sizeof(WsHeader), cudaMemcpyDeviceToHost, st));
        CSC_CUDA(cudaStreamSynchronize(st));
        float ms = 0.f;
        CSC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        kms_total += ms;
        S.updates += hh.stat[ST_UPDATES];
        S.iterations += hh.stat[ST_ITERS];
        S.rejected_softlock += hh.stat[ST_REJECTED];
        S.skipped_subtol += hh.stat[ST_SUBTOL];
        S.messages += hh.stat[ST_MESSAGES];
        status = hh.stop;
        // beta from scratch, KKT and objective on the current Z
        rc = launch_refresh<real>(g, L, wsb, X, D, Z, lambda, beta, st);
        if (rc) return rc;
        S.refresh_rounds++;
        CSC_CUDA(cudaMemcpyAsync(&hh, hdr, sizeof(WsHeader), cudaMemcpyDeviceToHost, st));
        CSC_CUDA(cudaStreamSynchronize(st));
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
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
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
