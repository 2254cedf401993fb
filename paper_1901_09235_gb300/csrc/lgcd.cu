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
template <typename real, int NT, int TN = NT>
__device__ void tile_setup(const LgcdArgs<real> &a, Tile<real, TN> &t, unsigned char *smem) {
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
// Warp-specialised worker: NTC compute threads run the LGCD iterations and
// synchronise among themselves on named barrier 1; one extra warp (the
// communication warp) owns every global control word -- the neighbour
// inboxes and outboxes, the `pending` termination counter, the stop word and
// the deadline -- so the compute warps never wait on global-memory latency
// except for the soft-lock reads of a neighbour's published band.
//
// Shared-memory protocol between the two roles:
//   in_ring  : records staged by the communication warp (in_head) and
//              consumed by the compute warps (in_tail);
//   out_ring : accepted border updates pushed by the compute leader
//              (out_head) and sent by the communication warp (out_tail);
//   idle_seq / resp_seq / resp_kind : the compute leader asks to pause after
//              a quiet sweep; the communication warp answers WOKEN (a message
//              arrived or was pending) or TERMINATE (pending == 0, stop word,
//              or deadline);
//   stop     : set by the communication warp when the run must end.
constexpr int kCompute = 256;
constexpr int kAsyncThreads = kCompute + 32;
constexpr int kWarps = kCompute / 32;
constexpr int kWout = 8;  // border records one warp may emit per wave
constexpr int kInRing = 128;
constexpr int kOutRing = 32;
enum { RESP_WOKEN = 1, RESP_TERMINATE = 2 };

struct AsyncShared {
    int4 in_ring[kInRing];
    int4 out_rec[kOutRing];
    int out_mask[kOutRing];
    volatile int in_head, in_tail, out_head, out_tail;
    volatile int idle_seq, resp_seq, resp_kind, stop;
    // compute-side broadcast slots
    int nmsg, bstop, room, idle_res;
    volatile long long n_msg_sent;
};

__device__ __forceinline__ void cbar() { asm volatile("bar.sync 1, %0;" ::"r"(kCompute) : "memory"); }

template <typename real>
__device__ __forceinline__ Cand<real> cand_shfl_max(Cand<real> c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Cand<real> y;
        y.a = __shfl_xor_sync(0xffffffffu, c.a, o);
        y.key = __shfl_xor_sync(0xffffffffu, c.key, o);
        y.znew = __shfl_xor_sync(0xffffffffu, c.znew, o);
        y.dz = __shfl_xor_sync(0xffffffffu, c.dz, o);
        if (better(y, c)) c = y;
    }
    return c;
}

// Candidate scan of sub-domain m by the compute threads; every compute
// thread returns the block-wide winner (one named barrier).
template <typename real>
__device__ __forceinline__ Cand<real> scan_v2(const LgcdArgs<real> &a, const Tile<real, kCompute> &t,
                                              int m, Cand<real> *part) {
    const int mr = m / t.ns1, mc = m % t.ns1;
    const int r0 = mr * a.sub0, c0 = mc * a.sub1;
    const int bh = min(a.sub0, t.h - r0), bw = min(a.sub1, t.wd - c0);
    const int nb = bh * bw;
    Cand<real> c{real(-1), 0xffffffffu, real(0), real(0)};
    const int tid = threadIdx.x;
    if (nb <= kCompute) {
        const int kstep = kCompute / nb;
        if (tid < kstep * nb) {
            const int r = tid % nb;
            const int li = r0 + r / bw, lj = c0 + r % bw;
            const unsigned pos = (unsigned)(li * a.t1 + lj) * (unsigned)t.K;
            int idx = (tid / nb) * t.TS + li * a.t1 + lj;
            for (int k = tid / nb; k < t.K; k += kstep, idx += kstep * t.TS) {
                real zn = coord_update(t.sbeta[idx], a.lambda, t.snrm[k], t.sinv[k]);
                real dz = zn - t.sz[idx];
                Cand<real> x{dz < real(0) ? -dz : dz, pos + (unsigned)k, zn, dz};
                if (better(x, c)) c = x;
            }
        }
    } else {
        for (int q = tid; q < t.K * nb; q += kCompute) {
            int k = q / nb, r = q % nb;
            int li = r0 + r / bw, lj = c0 + r % bw;
            int idx = k * t.TS + li * a.t1 + lj;
            real zn = coord_update(t.sbeta[idx], a.lambda, t.snrm[k], t.sinv[k]);
            real dz = zn - t.sz[idx];
            Cand<real> x{dz < real(0) ? -dz : dz, (unsigned)((li * a.t1 + lj) * t.K + k), zn, dz};
            if (better(x, c)) c = x;
        }
    }
    c = cand_shfl_max(c);
    if ((tid & 31) == 0) part[tid >> 5] = c;
    cbar();
    Cand<real> b = part[0];
#pragma unroll
    for (int w = 1; w < kCompute / 32; w++)
        if (better(part[w], b)) b = part[w];
    return b;
}

// Loop over the K x window entries of an update at tile-local (li0, lj0)
// that fall inside the tile; fn(k, r, idx) with r the window index.
template <typename real, typename F>
__device__ __forceinline__ void for_window(const LgcdArgs<real> &a, const Tile<real, kCompute> &t,
                                           int li0, int lj0, F fn) {
    const int tid = threadIdx.x, WW = t.WW;
    if (WW <= kCompute) {
        const int kstep = kCompute / WW;
        if (tid >= kstep * WW) return;
        const int r = tid % WW;
        const int li = li0 + r / a.W1 - (a.L0 - 1), lj = lj0 + r % a.W1 - (a.L1 - 1);
        if (li < 0 || li >= t.h || lj < 0 || lj >= t.wd) return;
        int idx = (tid / WW) * t.TS + li * a.t1 + lj;
        for (int k = tid / WW; k < t.K; k += kstep, idx += kstep * t.TS) fn(k, r, idx, li, lj);
    } else {
        for (int q = tid; q < t.K * WW; q += kCompute) {
            int k = q / WW, r = q % WW;
            int li = li0 + r / a.W1 - (a.L0 - 1), lj = lj0 + r % a.W1 - (a.L1 - 1);
            if (li < 0 || li >= t.h || lj < 0 || lj >= t.wd) continue;
            fn(k, r, k * t.TS + li * a.t1 + lj, li, lj);
        }
    }
}

// Warp-wide winner of (largest |dZ|, then smallest key); returns the key
// (0xffffffff when every lane is empty).  FP32 uses the redux unit on the
// order-preserving bits of |dZ|.
__device__ __forceinline__ unsigned warp_argmax_key(float a, unsigned key) {
    const unsigned bits = a < 0.f ? 0u : __float_as_uint(a) + 1u;  // empty lanes sort lowest
    const unsigned m = __reduce_max_sync(0xffffffffu, bits);
    if (m == 0u) return 0xffffffffu;
    return __reduce_min_sync(0xffffffffu, bits == m ? key : 0xffffffffu);
}
__device__ __forceinline__ unsigned warp_argmax_key(double a, unsigned key) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oa = __shfl_xor_sync(0xffffffffu, a, o);
        const unsigned ok = __shfl_xor_sync(0xffffffffu, key, o);
        if (oa > a || (oa == a && ok < key)) {
            a = oa;
            key = ok;
        }
    }
    return a < 0.0 ? 0xffffffffu : key;
}

// One warp applies an accepted update: beta window (Eq. beta_update), Z, the
// write-through of border entries and, for a border update, the record for
// the neighbours (needs a free out-ring slot, else the update is deferred).
template <typename real, int kWarps, int kWout>
__device__ __forceinline__ void apply_update_warp(const LgcdArgs<real> &a, const Tile<real, kCompute> &t, int k0,
                                                  int li0, int lj0, real znew, real dz, bool border, int lane,
                                                  int warp, int par, int &room_left, int (*wout_n)[kWarps],
                                                  int4 (*wout_rec)[kWarps][kWout],
                                                  int (*wout_mask)[kWarps][kWout], long long &n_upd,
                                                  long long &n_def, real guard) {
    int dl[kDirs];
    int nd = 0;
    if (border) {
        int ok = 0;
        if (lane == 0) {
            nd = target_dirs<real, kCompute>(a, t, li0, lj0, dl);
            if (nd == 0) ok = 1;
            else if (wout_n[par][warp] < kWout) {
                ok = atomicSub(&room_left, 1) > 0;
                if (!ok) atomicAdd(&room_left, 1);
            }
            if (!ok) n_def++;
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) return;
    }
    const real *__restrict__ row = t.sdtd + (size_t)k0 * t.K * t.WW;
    real *__restrict__ sb = t.sbeta;
    for (int r = lane; r < t.WW; r += 32) {
        const int li = li0 + r / a.W1 - (a.L0 - 1), lj = lj0 + r % a.W1 - (a.L1 - 1);
        if (li < 0 || li >= t.h || lj < 0 || lj >= t.wd) continue;
        const bool band = in_band(li, lj, t.h, t.wd, a.L0, a.L1);
        const int kskip = (li == li0 && lj == lj0) ? k0 : -1;
        const int base = li * a.t1 + lj;
        real *gb = a.beta + ((size_t)t.or0 + li) * a.Z1 + t.oc0 + lj;
        const size_t gstride = (size_t)a.Z0 * a.Z1;
#pragma unroll 4
        for (int k = 0; k < t.K; k++) {
            if (k == kskip) continue;
            const int idx = base + k * t.TS;
            const real v = sub_prod(sb[idx], row[k * t.WW + r], dz);
            sb[idx] = v;
            if (band) st_relaxed(gb + k * gstride, v);
        }
    }
    if (lane == 0) {
        t.sz[k0 * t.TS + li0 * a.t1 + lj0] = znew;
        n_upd++;
        if (border) {
            st_relaxed(a.Z + ((size_t)k0 * a.Z0 + t.or0 + li0) * a.Z1 + t.oc0 + lj0, znew);
            if (nd > 0) {
                int mask = 0;
                for (int i = 0; i < nd; i++) mask |= 1 << dl[i];
                const int o = wout_n[par][warp]++;
                wout_rec[par][warp][o] = pack_msg(k0, (t.or0 + li0) * a.Z1 + t.oc0 + lj0, dz);
                wout_mask[par][warp][o] = mask;
            }
        }
        if (a.max_updates > 0) {
            unsigned long long prev = atomicAdd(&a.hdr->updates_total, 1ull);
            if ((long long)prev + 1 >= a.max_updates) set_stop(a.hdr, CSC_NOT_CONVERGED);
        }
        const real az = znew < real(0) ? -znew : znew;
        if (a.guard_on && az > guard) set_stop(a.hdr, CSC_ERR_DIVERGED);
    }
    __syncwarp();
}

template <typename real>
__global__ void __launch_bounds__(kAsyncThreads, 2) lgcd_async_kernel(LgcdArgs<real> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ AsyncShared S;
    __shared__ Cand<real> part[kCompute / 32];
    __shared__ real lpart[kCompute / 32][2];
    Tile<real, kCompute> t;
    tile_setup<real, kAsyncThreads, kCompute>(a, t, smem_raw);
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    if (threadIdx.x == 0) {
        S.in_head = S.in_tail = S.out_head = S.out_tail = 0;
        S.idle_seq = S.resp_seq = S.resp_kind = 0;
        S.stop = 0;
        S.n_msg_sent = 0;
    }
    __syncthreads();

    if (threadIdx.x >= kCompute) {
        // ------------------------------------------------ communication warp
        if (threadIdx.x != kCompute) return;
        int ndir = 0, dirs[kDirs], in_tail[kDirs], out_head[kDirs], out_tail[kDirs];
        for (int d = 0; d < kDirs; d++) {
            int dr, dc;
            dir_offset(d, dr, dc);
            int r = t.ta + dr, c = t.tb + dc;
            in_tail[d] = out_head[d] = out_tail[d] = 0;
            if (r >= 0 && r < a.G0 && c >= 0 && c < a.G1) dirs[ndir++] = d;
        }
        bool idle = false;
        int spins = 0;
        for (;;) {
            bool work = false;
            // inbound: stage new records while the ring has room
            int heads[kDirs];
            for (int i = 0; i < ndir; i++)
                heads[dirs[i]] = ld_relaxed(a.ctl + ((size_t)t.w * kDirs + dirs[i]) * 32);
            int avail = 0;
            for (int i = 0; i < ndir; i++) avail += heads[dirs[i]] - in_tail[dirs[i]];
            if (avail > 0) {
                if (idle) {
                    atomicAdd(&a.hdr->pending, 1);  // reactivate before consuming
                    idle = false;
                    S.resp_kind = RESP_WOKEN;
                    __threadfence_block();
                    S.resp_seq = S.idle_seq;
                }
                fence_acq_rel_gpu();
                int ih = S.in_head;
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
            // outbound: send queued border updates in order
            while (S.out_tail != S.out_head) {
                const int ot = S.out_tail;
                const int4 rec = S.out_rec[ot & (kOutRing - 1)];
                const int mask = S.out_mask[ot & (kOutRing - 1)];
                bool room_all = true;
                for (int d = 0; d < kDirs && room_all; d++) {
                    if (!(mask >> d & 1)) continue;
                    int dr, dc;
                    dir_offset(d, dr, dc);
                    const int link = ((t.ta + dr) * a.G1 + (t.tb + dc)) * kDirs + (7 - d);
                    if (out_head[d] - out_tail[d] >= a.cap) {
                        out_tail[d] = ld_acquire(a.ctl + (size_t)link * 32 + 16);
                        room_all = out_head[d] - out_tail[d] < a.cap;
                    }
                }
                if (!room_all) break;
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
                S.n_msg_sent = S.n_msg_sent + __popc(mask);
                __threadfence_block();
                S.out_tail = ot + 1;
                work = true;
            }
            // pause request after a quiet sweep
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
        return;
    }

    // ------------------------------------------------------- compute warps
    // Colour waves: sub-domain (mr, mc) of the tile has colour
    // 2 (mr mod 2) + (mc mod 2).  Two sub-domains of one colour are at least
    // one full sub-domain (2 L_i) apart, so an update in one changes beta only
    // outside the other and their cost changes add up (the cross term of
    // Prop. A.2 is zero).  Each wave processes every sub-domain of one colour,
    // one warp per sub-domain; a sweep visits every colour once.
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ int wact[2][kWarps], wout_n[2][kWarps], room_left;
    __shared__ int4 wout_rec[2][kWarps][kWout];
    __shared__ int wout_mask[2][kWarps][kWout];
    constexpr int kPend = 2;  // border candidates one warp may park per wave
    __shared__ int pend_n[kWarps];
    __shared__ int pend_pos[kWarps][kPend][3];  // k0, li0, lj0
    __shared__ real pend_z[kWarps][kPend][2];   // Z', dZ
    __shared__ unsigned pend_lo[kWarps * kPend], pend_hi[kWarps * kPend];
    long long n_upd = 0, n_it = 0, n_rej = 0, n_sub = 0, n_def = 0, n_wave = 0;
    __shared__ unsigned long long t_first_idle;
    long long last_active_wave = 0;
    __shared__ int n_wake;
    const unsigned long long t_start = globaltimer_ns();
    if (tid == 0) {
        t_first_idle = 0;
        n_wake = 0;
    }
    real guard = real(0);
    if (a.guard_on) {
        double g = 1e300;
        for (int k = 0; k < a.K; k++) g = fmin(g, 50.0 / a.dmax[k]);
        guard = real(g);
    }
    const int ns0 = (t.h + a.sub0 - 1) / a.sub0, ns1 = t.ns1;
    int ccount[4], ncol = 0, colors[4];
    for (int c = 0; c < 4; c++) {
        const int rc = c >> 1, cc = c & 1;
        const int nr = rc < ns0 ? (ns0 - rc + 1) / 2 : 0, nc = cc < ns1 ? (ns1 - cc + 1) / 2 : 0;
        ccount[c] = nr * nc;
        if (ccount[c] > 0) colors[ncol++] = c;
    }
    int ci = 0, quiet = 0;
    unsigned long long ph[6] = {0, 0, 0, 0, 0, 0}, tc = clock64(), tn;
    for (;;) {
        if (tid == 0) {
            S.nmsg = S.in_head - S.in_tail;
            S.bstop = S.stop;
            room_left = kOutRing - (S.out_head - S.out_tail);
        }
        cbar();
        tn = clock64();
        ph[0] += tn - tc;
        tc = tn;
        if (S.bstop) break;
        const int par = (int)(n_wave & 1);
        if (lane == 0) {
            wact[par][warp] = 0;
            wout_n[par][warp] = 0;
            pend_n[warp] = 0;
        }
        const int nmsg = S.nmsg;
        if (nmsg > 0) {
            // neighbour updates (Alg. 3 "receive messages and update beta")
            const int base = S.in_tail;
            for (int i = 0; i < nmsg; i++) {
                const int4 msg = S.in_ring[(base + i) & (kInRing - 1)];
                real dz;
                unpack_msg(msg, dz);
                const int gi = msg.y / a.Z1, gj = msg.y % a.Z1;
                const real *row = t.sdtd + (size_t)msg.x * t.K * t.WW;
                for_window(a, t, gi - t.or0, gj - t.oc0, [&](int k, int r, int idx, int li, int lj) {
                    atomicAdd(&t.sbeta[idx], -(row[k * t.WW + r] * dz));
                });
            }
            cbar();
            for (int i = 0; i < nmsg; i++) {
                const int4 msg = S.in_ring[(base + i) & (kInRing - 1)];
                const int gi = msg.y / a.Z1, gj = msg.y % a.Z1;
                for_window(a, t, gi - t.or0, gj - t.oc0, [&](int k, int r, int idx, int li, int lj) {
                    st_relaxed(a.beta + ((size_t)k * a.Z0 + t.or0 + li) * a.Z1 + t.oc0 + lj, t.sbeta[idx]);
                });
            }
            cbar();
            if (tid == 0) S.in_tail = base + nmsg;
        }
        tn = clock64();
        ph[1] += tn - tc;
        tc = tn;
        // ---- one wave: the sub-domains of colour c, one warp each
        const int c = colors[ci];
        const int rc = c >> 1, cc = c & 1, ncc = (ns1 - cc + 1) / 2;
        for (int j = warp; j < ccount[c]; j += kWarps) {
            const int mr = rc + 2 * (j / ncc), mc = cc + 2 * (j % ncc);
            const int r0 = mr * a.sub0, c0 = mc * a.sub1;
            const int bh = min(a.sub0, t.h - r0), bw = min(a.sub1, t.wd - c0), nb = bh * bw;
            // candidate scan (Eq. gcd_candidate) with the oracle's tie-break
            real ba = real(-1);
            unsigned bkey = 0xffffffffu;
            const real *__restrict__ sbr = t.sbeta;
            const real *__restrict__ szr = t.sz;
            for (int r = lane; r < nb; r += 32) {
                const int li = r0 + r / bw, lj = c0 + r % bw;
                const unsigned pos = (unsigned)(li * a.t1 + lj) * (unsigned)t.K;
                const int base = li * a.t1 + lj;
#pragma unroll 4
                for (int k = 0; k < t.K; k++) {
                    const int idx = base + k * t.TS;
                    const real zn = coord_update(sbr[idx], a.lambda, t.snrm[k], t.sinv[k]);
                    real d = zn - szr[idx];
                    d = d < real(0) ? -d : d;
                    const unsigned key = pos + (unsigned)k;
                    if (d > ba || (d == ba && key < bkey)) {
                        ba = d;
                        bkey = key;
                    }
                }
            }
            const unsigned wkey = warp_argmax_key(ba, bkey);
            n_it += (lane == 0);
            if (wkey == 0xffffffffu) continue;
            const unsigned pos = wkey / (unsigned)t.K;
            const int k0 = (int)(wkey % (unsigned)t.K);
            const int li0 = (int)(pos / (unsigned)a.t1), lj0 = (int)(pos % (unsigned)a.t1);
            const int idx0 = k0 * t.TS + li0 * a.t1 + lj0;
            const real znew = coord_update(t.sbeta[idx0], a.lambda, t.snrm[k0], t.sinv[k0]);
            const real dz = znew - t.sz[idx0];
            const real adz = dz < real(0) ? -dz : dz;
            if (!(adz >= a.eps)) {
                n_sub += (lane == 0);
                continue;
            }
            if (lane == 0) wact[par][warp] = 1;
            const bool border = in_band(li0, lj0, t.h, t.wd, a.L0, a.L1);
            if (border && a.mode == CSC_MODE_ASYNC) {
                // park it: the soft-lock test runs for all parked candidates at once
                if (lane == 0) {
                    const int o = pend_n[warp];
                    if (o < kPend) {
                        pend_pos[warp][o][0] = k0;
                        pend_pos[warp][o][1] = li0;
                        pend_pos[warp][o][2] = lj0;
                        pend_z[warp][o][0] = znew;
                        pend_z[warp][o][1] = dz;
                        pend_lo[warp * kPend + o] = 0u;
                        pend_hi[warp * kPend + o] = 0u;
                        pend_n[warp] = o + 1;
                    } else {
                        n_def++;
                    }
                }
                __syncwarp();
                continue;
            }
            apply_update_warp(a, t, k0, li0, lj0, znew, dz, border, lane, warp, par, room_left, wout_n,
                              wout_rec, wout_mask, n_upd, n_def, guard);
        }
        cbar();
        tn = clock64();
        ph[2] += tn - tc;
        tc = tn;
        // ---- soft-lock test of the parked border candidates (Eq. soft_lock),
        // all compute threads together: one batch of loads per thread
        int ncand = 0;
        for (int w = 0; w < kWarps; w++) ncand += pend_n[w];
        if (ncand > 0) {
            // candidate c's K x window entries are split over the compute
            // threads; each warp reduces its maxima before one shared atomic
            const int per = t.K * t.WW;
            constexpr int B = 8;
            for (int c = 0; c < ncand; c++) {
                int slot = -1, rem = c;
                for (int w = 0; w < kWarps; w++) {
                    if (rem < pend_n[w]) {
                        slot = w * kPend + rem;
                        break;
                    }
                    rem -= pend_n[w];
                }
                const int *pp = pend_pos[slot / kPend][slot % kPend];
                const int gi0 = t.or0 + pp[1] - (a.L0 - 1), gj0 = t.oc0 + pp[2] - (a.L1 - 1);
                unsigned lo = 0u, hi = 0u;
                for (int base = tid; base < per; base += B * kCompute) {
                    real vb[B], vz[B];
                    int kk[B], side[B];
#pragma unroll
                    for (int u = 0; u < B; u++) {
                        const int q = base + u * kCompute;
                        side[u] = 0;
                        kk[u] = 0;
                        vb[u] = real(0);
                        vz[u] = real(0);
                        if (q < per) {
                            const int k = q / t.WW, r = q % t.WW;
                            const int gi = gi0 + r / a.W1, gj = gj0 + r % a.W1;
                            const bool in_dom = gi >= 0 && gi < a.Z0 && gj >= 0 && gj < a.Z1;
                            const bool in_tile = gi >= t.or0 && gi < t.or0 + t.h && gj >= t.oc0 && gj < t.oc0 + t.wd;
                            if (in_dom && !in_tile) {
                                const size_t g = ((size_t)k * a.Z0 + gi) * a.Z1 + gj;
                                vb[u] = ld_relaxed(a.beta + g);
                                vz[u] = ld_relaxed(a.Z + g);
                                kk[u] = k;
                                side[u] = ((gi / a.t0) * a.G1 + gj / a.t1) < t.w ? 1 : 2;
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < B; u++) {
                        if (side[u] == 0) continue;
                        real d = coord_update(vb[u], a.lambda, t.snrm[kk[u]], t.sinv[kk[u]]) - vz[u];
                        d = d < real(0) ? -d : d;
                        const unsigned bits = (unsigned)nonneg_bits((float)d) + 1u;
                        if (side[u] == 1) lo = max(lo, bits);
                        else hi = max(hi, bits);
                    }
                }
                lo = __reduce_max_sync(0xffffffffu, lo);
                hi = __reduce_max_sync(0xffffffffu, hi);
                if (lane == 0) {
                    if (lo) atomicMax(&pend_lo[slot], lo);
                    if (hi) atomicMax(&pend_hi[slot], hi);
                }
            }
            cbar();
            for (int o = 0; o < pend_n[warp]; o++) {
                const int slot = warp * kPend + o;
                const int k0 = pend_pos[warp][o][0], li0 = pend_pos[warp][o][1], lj0 = pend_pos[warp][o][2];
                const real znew = pend_z[warp][o][0], dz = pend_z[warp][o][1];
                const real adz = dz < real(0) ? -dz : dz;
                // compare in the same float encoding the maxima were taken in
                const unsigned mine = (unsigned)nonneg_bits((float)adz) + 1u;
                const bool accept = mine > pend_lo[slot] && mine >= pend_hi[slot];
                if (!accept) {
                    n_rej += (lane == 0);
                    continue;
                }
                apply_update_warp(a, t, k0, li0, lj0, znew, dz, true, lane, warp, par, room_left, wout_n,
                                  wout_rec, wout_mask, n_upd, n_def, guard);
            }
        }
        cbar();
        tn = clock64();
        ph[3] += tn - tc;
        tc = tn;
        // ---- end of wave: hand border updates to the communication warp
        bool any = nmsg > 0;
        for (int w = 0; w < kWarps; w++) any |= wact[par][w] != 0;
        if (tid == 0) {
            const int oh0 = S.out_head;
            int oh = oh0;
            for (int w = 0; w < kWarps; w++)
                for (int i = 0; i < wout_n[par][w]; i++, oh++) {
                    S.out_rec[oh & (kOutRing - 1)] = wout_rec[par][w][i];
                    S.out_mask[oh & (kOutRing - 1)] = wout_mask[par][w][i];
                }
            if (oh != oh0) {
                __threadfence_block();
                S.out_head = oh;
            }
        }
        n_wave++;
        ci = ci + 1 == ncol ? 0 : ci + 1;
        quiet = any ? 0 : quiet + 1;
        if (any) last_active_wave = n_wave;
        if (quiet >= ncol) {
            // a full sweep without work: pause (Alg. 3)
            if (tid == 0) {
                if (t_first_idle == 0) t_first_idle = globaltimer_ns();
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
                S.idle_res = (S.resp_kind == RESP_TERMINATE) || S.stop;
                n_wake += !S.idle_res;
            }
            cbar();
            if (S.idle_res) break;
            quiet = 0;
            tn = clock64();
            ph[5] += tn - tc;
            tc = tn;
        }
        tn = clock64();
        ph[4] += tn - tc;
        tc = tn;
    }
    // wait for the communication warp to finish before the tile is written
    if (tid == 0) {
        const unsigned long long late = deadline + 4000000000ull;
        while (S.resp_kind != RESP_TERMINATE && !S.stop && globaltimer_ns() < late) __nanosleep(64);
    }
    cbar();
    const int hw = t.h * t.wd;
    for (int q = tid; q < t.K * hw; q += kCompute) {
        const int k = q / hw, r = q % hw, li = r / t.wd, lj = r % t.wd;
        const size_t g = ((size_t)k * a.Z0 + t.or0 + li) * a.Z1 + t.oc0 + lj;
        a.beta[g] = t.sbeta[k * t.TS + li * a.t1 + lj];
        a.Z[g] = t.sz[k * t.TS + li * a.t1 + lj];
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_upd += __shfl_xor_sync(0xffffffffu, n_upd, o);
        n_it += __shfl_xor_sync(0xffffffffu, n_it, o);
        n_rej += __shfl_xor_sync(0xffffffffu, n_rej, o);
        n_sub += __shfl_xor_sync(0xffffffffu, n_sub, o);
        n_def += __shfl_xor_sync(0xffffffffu, n_def, o);
    }
    if (lane == 0) {
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_UPDATES], (unsigned long long)n_upd);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_ITERS], (unsigned long long)n_it);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_REJECTED], (unsigned long long)n_rej);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_SUBTOL], (unsigned long long)n_sub);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_DEFERRED], (unsigned long long)n_def);
    }
    if (tid == 0) {
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_MESSAGES], (unsigned long long)S.n_msg_sent);
        atomicMax(&a.hdr->wmax[0], (unsigned long long)n_wave);
        atomicMax(&a.hdr->tmax[0], (unsigned long long)last_active_wave);
        atomicMax(&a.hdr->tmax[1], globaltimer_ns() - t_start);
        if (t_first_idle) atomicMax(&a.hdr->tmax[2], t_first_idle - t_start);
        atomicAdd(&a.hdr->tmax[3], (unsigned long long)n_wake);
        for (int i = 0; i < 6; i++) atomicAdd(&a.hdr->tph[i], ph[i]);
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

// ============================================================ GLOBAL TILES
// Variant for tiles whose beta / Z / table do not fit in shared memory (large
// atoms, e.g. 25 atoms of 32 x 32).  beta and Z stay in global memory (HBM,
// L2) and the table is read from L2.  Every beta window update is a
// red.global.add, so updates from neighbouring tiles that land in the same
// entries add up instead of overwriting each other, and an update whose
// window V(s0) crosses into a neighbour is applied there directly.  The
// neighbour learns that its beta changed through its flag counter (one word
// per tile): a worker bumps the counter of every tile V(s0) reaches.  The
// counters carry the same termination accounting as the mailboxes of the
// shared-memory variant: `pending` counts active workers plus flag bumps not
// yet observed by their tile.  One sub-domain per iteration, scanned and
// updated by the whole CTA.
constexpr int kGlobThreads = 512;

template <typename real>
__global__ void __launch_bounds__(kGlobThreads, 2) lgcd_global_kernel(LgcdArgs<real> a) {
    constexpr int NT = kGlobThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *snrm = reinterpret_cast<real *>(smem_raw), *sinv = snrm + a.K;
    const int w = blockIdx.x, ta = w / a.G1, tb = w % a.G1;
    const int or0 = ta * a.t0, oc0 = tb * a.t1;
    const int h = min(a.t0, a.Z0 - or0), wd = min(a.t1, a.Z1 - oc0);
    const int ns0 = (h + a.sub0 - 1) / a.sub0, ns1 = (wd + a.sub1 - 1) / a.sub1, M = ns0 * ns1;
    const int K = a.K, WW = a.W0 * a.W1;
    const size_t plane = (size_t)a.Z0 * a.Z1;
    for (int k = threadIdx.x; k < K; k += NT) {
        snrm[k] = real(a.nrm[k]);
        sinv[k] = real(1.0 / a.nrm[k]);
    }
    int *flag = a.ctl + (size_t)w * kDirs * 32;  // this tile's counter
    __shared__ int s_ctl[4];                     // new flag bumps, state, accept
    __shared__ Cand<real> s_best;
    long long n_upd = 0, n_it = 0, n_rej = 0, n_sub = 0, n_msg = 0;
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    real guard = real(0);
    if (a.guard_on) {
        double g = 1e300;
        for (int k = 0; k < K; k++) g = fmin(g, 50.0 / a.dmax[k]);
        guard = real(g);
    }
    int seen = 0, m = 0, quiet = 0;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            int got = 0, state = 0;
            const int f = ld_relaxed(flag);
            if (f != seen) {
                got = f - seen;
                seen = f;
                atomicSub(&a.hdr->pending, got);  // observed: no longer in flight
            }
            if (ld_relaxed(&a.hdr->stop)) state = 1;
            else if (globaltimer_ns() > deadline) {
                set_stop(a.hdr, CSC_ERR_TIMEOUT);
                state = 1;
            }
            s_ctl[0] = got;
            s_ctl[1] = state;
        }
        __syncthreads();
        if (s_ctl[1]) break;
        const int got = s_ctl[0];
        // ---- scan sub-domain m (Eq. gcd_candidate)
        const int mr = m / ns1, mc = m % ns1;
        const int r0 = mr * a.sub0, c0 = mc * a.sub1;
        const int bh = min(a.sub0, h - r0), bw = min(a.sub1, wd - c0), nb = bh * bw;
        Cand<real> c{real(-1), 0xffffffffu, real(0), real(0)};
        for (int q = threadIdx.x; q < K * nb; q += NT) {
            const int k = q / nb, r = q % nb, li = r0 + r / bw, lj = c0 + r % bw;
            const size_t g = k * plane + (size_t)(or0 + li) * a.Z1 + oc0 + lj;
            const real zn = coord_update(__ldcg(a.beta + g), a.lambda, snrm[k], sinv[k]);
            const real dz = zn - a.Z[g];
            Cand<real> x{dz < real(0) ? -dz : dz, (unsigned)((li * a.t1 + lj) * K + k), zn, dz};
            if (better(x, c)) c = x;
        }
        const Cand<real> best = block_argmax<real, NT>(c);
        n_it++;
        const bool active = best.a >= a.eps;
        if (active) {
            const unsigned pos = best.key / (unsigned)K;
            const int k0 = (int)(best.key % (unsigned)K);
            const int li0 = (int)(pos / (unsigned)a.t1), lj0 = (int)(pos % (unsigned)a.t1);
            const int gi0 = or0 + li0, gj0 = oc0 + lj0;
            const bool border = in_band(li0, lj0, h, wd, a.L0, a.L1);
            bool accept = true;
            if (border && a.mode == CSC_MODE_ASYNC) {
                // soft-lock over the part of V(s0) outside the tile: at most one
                // strip of rows outside the tile rows (full width of V) and one
                // strip of columns outside the tile columns (tile rows only)
                const int v0 = max(0, gi0 - (a.L0 - 1)), v1 = min(a.Z0, gi0 + a.L0);
                const int u0 = max(0, gj0 - (a.L1 - 1)), u1 = min(a.Z1, gj0 + a.L1);
                const int ra0 = v0 < or0 ? v0 : max(v0, or0 + h), ra1 = v0 < or0 ? min(v1, or0) : v1;
                const int rb0 = max(v0, or0), rb1 = min(v1, or0 + h);
                const int cb0 = u0 < oc0 ? u0 : max(u0, oc0 + wd), cb1 = u0 < oc0 ? min(u1, oc0) : u1;
                const int n1 = max(0, ra1 - ra0) * (u1 - u0), n2 = max(0, rb1 - rb0) * max(0, cb1 - cb0);
                real lo = real(-1), hi = real(-1);
                for (int q = threadIdx.x; q < K * (n1 + n2); q += NT) {
                    const int k = q / (n1 + n2), e = q % (n1 + n2);
                    int gi, gj;
                    if (e < n1) {
                        gi = ra0 + e / (u1 - u0);
                        gj = u0 + e % (u1 - u0);
                    } else {
                        gi = rb0 + (e - n1) / (cb1 - cb0);
                        gj = cb0 + (e - n1) % (cb1 - cb0);
                    }
                    const size_t g = k * plane + (size_t)gi * a.Z1 + gj;
                    real d = coord_update(ld_relaxed(a.beta + g), a.lambda, snrm[k], sinv[k]) - ld_relaxed(a.Z + g);
                    d = d < real(0) ? -d : d;
                    if ((gi / a.t0) * a.G1 + gj / a.t1 < w) lo = max(lo, d);
                    else hi = max(hi, d);
                }
                real mhi;
                const real mlo = block_max2<real, NT>(lo, hi, &mhi);
                accept = best.a > mlo && best.a >= mhi;
                if (!accept) n_rej += threadIdx.x == 0;
            }
            if (accept) {
                // beta_k[s] -= C[k][k0][s - s0] dz on V(s0) within the domain
                const real dz = best.dz;
                for (int q = threadIdx.x; q < K * WW; q += NT) {
                    const int k = q / WW, r = q % WW;
                    const int gi = gi0 + r / a.W1 - (a.L0 - 1), gj = gj0 + r % a.W1 - (a.L1 - 1);
                    if (gi < 0 || gi >= a.Z0 || gj < 0 || gj >= a.Z1) continue;
                    if (k == k0 && gi == gi0 && gj == gj0) continue;
                    const real cval = __ldg(a.dtd + ((size_t)k * K + k0) * WW + r);
                    atomicAdd(a.beta + k * plane + (size_t)gi * a.Z1 + gj, -(cval * dz));
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    a.Z[k0 * plane + (size_t)gi0 * a.Z1 + gj0] = best.znew;
                    n_upd++;
                    int dl[kDirs];
                    Tile<real, NT> tt;
                    tt.ta = ta;
                    tt.tb = tb;
                    tt.h = h;
                    tt.wd = wd;
                    const int nd = border ? target_dirs<real, NT>(a, tt, li0, lj0, dl) : 0;
                    if (nd > 0) {
                        __threadfence();  // the window's reductions before the flags
                        atomicAdd(&a.hdr->pending, nd);
                        for (int i = 0; i < nd; i++) {
                            int dr, dc;
                            dir_offset(dl[i], dr, dc);
                            atomicAdd(a.ctl + (size_t)((ta + dr) * a.G1 + (tb + dc)) * kDirs * 32, 1);
                        }
                        n_msg += nd;
                    }
                    if (a.max_updates > 0) {
                        unsigned long long prev = atomicAdd(&a.hdr->updates_total, 1ull);
                        if ((long long)prev + 1 >= a.max_updates) set_stop(a.hdr, CSC_NOT_CONVERGED);
                    }
                    const real az = best.znew < real(0) ? -best.znew : best.znew;
                    if (a.guard_on && az > guard) set_stop(a.hdr, CSC_ERR_DIVERGED);
                }
            }
        } else {
            n_sub++;
        }
        quiet = (active || got > 0) ? 0 : quiet + 1;
        m = (m + 1 == M) ? 0 : m + 1;
        __syncthreads();
        if (quiet >= M) {
            // pause until a neighbour bumps the flag or every worker is done
            if (threadIdx.x == 0) {
                atomicSub(&a.hdr->pending, 1);
                int state = 0;
                for (;;) {
                    if (ld_relaxed(flag) != seen) {
                        atomicAdd(&a.hdr->pending, 1);
                        break;
                    }
                    if (ld_acquire(&a.hdr->pending) == 0 || ld_relaxed(&a.hdr->stop)) {
                        state = 1;
                        break;
                    }
                    if (globaltimer_ns() > deadline) {
                        set_stop(a.hdr, CSC_ERR_TIMEOUT);
                        state = 1;
                        break;
                    }
                    __nanosleep(256);
                }
                s_ctl[2] = state;
            }
            __syncthreads();
            if (s_ctl[2]) break;
            quiet = 0;
        }
    }
    if (threadIdx.x == 0) {
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_UPDATES], (unsigned long long)n_upd);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_ITERS], (unsigned long long)n_it);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_REJECTED], (unsigned long long)n_rej);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_SUBTOL], (unsigned long long)n_sub);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_MESSAGES], (unsigned long long)n_msg);
        atomicMax(&a.hdr->wmax[0], (unsigned long long)n_it);
        atomicMax(&a.hdr->wmax[1], (unsigned long long)n_upd);
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
static const void *kernel_ptr(int mode, bool global) {
    if (global) return (const void *)lgcd_global_kernel<real>;
    if (mode == CSC_MODE_PHASED) return (const void *)lgcd_phased_kernel<real, kLgcdThreads>;
    return (const void *)lgcd_async_kernel<real>;
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
static int make_plan(const Geom &g, const csc_solve_opts &o, int rs, size_t static_smem, Plan *pl) {
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
        if (pl->smem + static_smem > (size_t)lim) return CSC_ERR_UNIMPLEMENTED;
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
        size_t budget = std::min<size_t>((size_t)lim - static_smem, (size_t)per_sm / occ - 1024 - static_smem);
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

// Plan for the global-memory variant: tiles of at least 2 L_i (or the
// caller's tile, at least L_i), at most `max_w` tiles, squarish in 2-D.
static int make_plan_global(const Geom &g, const csc_solve_opts &o, long long max_w, int rs, Plan *pl) {
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
    Plan pl;
    rc = global ? CSC_ERR_UNIMPLEMENTED : make_plan(g, o, rs, static_smem, &pl);
    if (rc == CSC_ERR_UNIMPLEMENTED && o.placement == 0 && o.mode != CSC_MODE_PHASED) global = true;
    if (global) {
        kern = kernel_ptr<real>(o.mode, true);
        rc = make_plan_global(g, o, 2ll * num_sms(), rs, &pl);
    }
    if (rc) return rc;
    const int W = pl.G0 * pl.G1;
    WsLayout L = plan_workspace(g, W, rs);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
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
    // FP32 solves stop at 0.99 tol so that rounding drift of the incrementally
    // maintained beta rarely pushes a coordinate back above tol on the
    // recomputed beta; the FP64 build keeps tol exactly.
    a.eps = sizeof(real) == 4 ? real(0.99) * tol : tol;
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
        reset_header_kernel<<<1, 1, 0, st>>>(hdr, W);
        CSC_CUDA(cudaGetLastError());
        void *args[] = {&a};
        CSC_CUDA(cudaEventRecord(e0, st));
        CSC_CUDA(cudaLaunchCooperativeKernel(kern, dim3(W), dim3(kernel_threads(o.mode, global)), args, pl.smem, st));
        CSC_CUDA(cudaEventRecord(e1, st));
        // beta from scratch, KKT and objective on the current Z, then one sync
        rc = launch_refresh<real>(g, L, wsb, X, D, Z, lambda, beta, st);
        if (rc) return rc;
        S.refresh_rounds++;
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
        S.deferred += hh.stat[ST_DEFERRED];
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
