// lgcd_common.cuh -- shared pieces of the LGCD solvers (Alg. 1 inside each
// worker of Alg. 3): launch arguments, tile geometry and shared-memory tile
// setup, candidate reductions, neighbour directions and the mailbox records
// exchanged between tiles.
#pragma once
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
    int z_zero;  // Z is all zero when the launch starts (cold start)
    real lambda, eps;
    long long max_updates;
    unsigned long long timeout_ns;
    // FP32 global tiles of the single-solve kernel: the table in its window
    // layout (null: the window update reads dtd), its row and block strides
    // in floats and the number of shared-memory slots that stage it
    const float *wtab;
    int wrs, wbs, wslots;
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

// Tile plan of a solve: a G0 x G1 grid of tiles of t0 x t1 positions,
// sub-domains of sub0 x sub1, and the dynamic shared memory of one tile.
struct Plan {
    int G0, G1, t0, t1, sub0, sub1;
    size_t smem;
};
// Plan for tiles kept in global memory: tiles of at least 2 L_i (or the
// caller's tile, at least L_i), at most max_w tiles, squarish in 2-D.
int make_plan_global(const Geom &g, const csc_solve_opts &o, long long max_w, int rs, Plan *pl);

// Shared-memory tiles, ASYNC and NOLOCK modes (lgcd_async.cu): 8 compute
// warps and one communication warp.
constexpr int kAsyncCompute = 256;
constexpr int kAsyncThreads = kAsyncCompute + 32;
constexpr int kAsyncMaxSub = 64;  // sub-domains per tile
// Host: the kernel entry of lgcd_async.cu for float / double elements.
const void *lgcd_async_kernel_ptr(float);
const void *lgcd_async_kernel_ptr(double);

}  // namespace csc
