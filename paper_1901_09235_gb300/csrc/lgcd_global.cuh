// lgcd_global.cuh -- LGCD worker for tiles kept in global memory (Alg. 1 in
// each worker of Alg. 3), shared by the single-solve kernel and the batched
// queue kernel.
#pragma once
#include <cstdint>
#include <type_traits>

#include "lgcd_common.cuh"

namespace csc {

// ============================================================ GLOBAL TILES
// Variant for tiles whose beta / Z / table do not fit in shared memory (large
// atoms, e.g. 25 atoms of 32 x 32).  beta and Z stay in global memory (HBM,
// L2); the table is read from L2, or (single-solve FP32 kernel) staged
// through shared memory by bulk copies, one block C[k][k0] at a time.  Every beta window update is a
// red.global.add, so updates from neighbouring tiles that land in the same
// entries add up instead of overwriting each other, and an update whose
// window V(s0) crosses into a neighbour is applied there directly.  The
// neighbour learns that its beta changed through its notification counters
// (one per neighbour direction): a worker bumps, in every tile V(s0) reaches,
// the counter of the direction it lies in.  The counters carry the same termination accounting as the mailboxes of the
// shared-memory variant: `pending` counts active workers plus counter bumps
// not yet observed by their tile.  One sub-domain per iteration, scanned and
// updated by the whole CTA.
// Threads per worker CTA of the single-solve kernel (two CTAs per SM).
// Measured on the 4096^2 image (25 atoms of 32 x 32): 456 x 256, 608 x 256
// and 304 x 512 threads solve in the same time, the shorter per-tile chains
// of more tiles offset by slower iterations; with 304 tiles, 448 threads (72
// registers each) take 41.1 ms, 384 (80) 42.1 ms, 512 (64, a few spills in
// the soft-lock path) 42.9 ms and 320 44.3 ms.
constexpr int kGlobThreads = 448;
// Tasks whose loads a thread issues together in the FP32 scan and window
// update: two each fit the registers of two CTAs per SM without spilling;
// three (384 threads) and three to six (512, with spills) were slower on the
// 4096^2 image.
constexpr int kScanBatch = 2, kWindowBatch = 2;
// Boxes of K x rows x cols are walked in units of (atom, block of RB rows,
// 32-column chunk): a warp takes units NW apart, issues the loads of all rows
// of its unit, then evaluates them.  Two divisions per unit, none per
// element.  RB is at most the largest block a kernel holds in registers
// without spilling (the single-solve kernel takes 4: 6 and 8 spill nothing
// but were 2 % slower on the 4096^2 image, 5 was 7 % slower).

template <typename real, int NT, int RB, bool STAGED = false>
__device__ void global_tile_worker(const LgcdArgs<real> &a, int w, unsigned char *smem_raw);

// Warp argmax with the oracle's tie-break (larger |dZ|, then smaller key);
// every lane gets the winner, with its Z' and dZ.
template <typename real>
__device__ __forceinline__ Cand<real> warp_argmax(const Cand<real> &c) {
    real am = c.a;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) am = max(am, __shfl_xor_sync(0xffffffffu, am, o));
    unsigned km = c.a == am ? c.key : 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) km = min(km, __shfl_xor_sync(0xffffffffu, km, o));
    const unsigned who = __ballot_sync(0xffffffffu, c.a == am && c.key == km);
    const int src = who ? __ffs(who) - 1 : 0;
    Cand<real> r;
    r.a = am;
    r.key = km;
    r.znew = __shfl_sync(0xffffffffu, c.znew, src);
    r.dz = __shfl_sync(0xffffffffu, c.dz, src);
    return r;
}

// One 16-byte reduction: four consecutive floats added at L2 as one request
// (p 16-byte aligned).  Lanes with nothing to add pass 0.  No memory clobber:
// the only other accesses near it are read-only table loads, which may move
// across it.
__device__ __forceinline__ void red_add_v4(float *p, float x, float y, float z, float w) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x), "f"(y), "f"(z), "f"(w));
}

// Vector form of the scan and of the window update, for FP32 arrays whose
// beta and Z start on 16-byte boundaries.  A row segment of the array is
// covered by the aligned groups of four floats that meet it: with s the
// segment's first flat index mod 4, group j starts at flat index
// (first - s + 4 j), and lanes outside the segment are masked.  Tasks
// (atom, row, group) are dealt to the threads in order, so a warp covers whole
// rows with consecutive 16-byte accesses; (atom, row, group) of a thread's next
// task follow from its current one by a fixed step (no division per task).
struct TaskStep {
    int k, r, j;      // current task
    int dk, dr, dj;   // step of NT tasks
    int R, NG;        // rows per atom, groups per row
    __device__ __forceinline__ void init(int t, int nt, int R_, int NG_) {
        R = R_;
        NG = NG_;
        const int per_k = R * NG;
        k = t / per_k;
        const int rem = t - k * per_k;
        r = rem / NG;
        j = rem - r * NG;
        dk = nt / per_k;
        const int srem = nt - dk * per_k;
        dr = srem / NG;
        dj = srem - dr * NG;
    }
    __device__ __forceinline__ void next() {
        j += dj;
        r += dr;
        k += dk;
        if (j >= NG) {
            j -= NG;
            r++;
        }
        if (r >= R) {
            r -= R;
            k++;
        }
    }
};

// Candidates of sub-domain rows [r0, r0 + bh) x columns [c0, c0 + bw) of the
// tile at (or0, oc0): the loads of B tasks are issued before any is
// evaluated; the evaluation replays the tasks' indices from a saved step.
// With `zskip` the sub-domain holds no nonzero of Z and Z is not read.
template <int NT, int B>
__device__ __forceinline__ Cand<float> scan_v4(const LgcdArgs<float> &a, const float *snrm, const float *sinv,
                                               int or0, int oc0, int r0, int c0, int bh, int bw, bool zskip) {
    const int K = a.K;
    const long long plane = (long long)a.Z0 * a.Z1, nall = (long long)K * plane;
    // low two bits of a flat index, from 32-bit arithmetic (they depend only
    // on the low bits of each term)
    const unsigned plane_lo = (unsigned)plane, base_lo = (unsigned)(or0 + r0) * (unsigned)a.Z1 + oc0 + c0;
    const int NG = (bw + 6) >> 2;  // groups of 4 that can meet bw columns
    const int total = K * bh * NG;
    // the thread's best |dZ| so far, with Z', dZ and its position (task
    // index x 4 + element): a thread keeps the first of equal |dZ| in its
    // own (atom-major) order, and the key ((row-major tile position) x K + k)
    // that the warp and block reductions compare is built once, at the end
    float ba = -1.f, bzn = 0.f, bdz = 0.f;
    int bt = -1;
    TaskStep ts;
    ts.init(threadIdx.x, NT, bh, NG);
    for (int t = threadIdx.x; t < total; t += B * NT) {
        const int k_s = ts.k, r_s = ts.r, j_s = ts.j;
        float4 bv[B], zv[B];
#pragma unroll
        for (int u = 0; u < B; u++) {
            if (t + u * NT < total) {
                const int sft = (int)((ts.k * plane_lo + base_lo + (unsigned)ts.r * (unsigned)a.Z1) & 3u);
                const int off = 4 * ts.j - sft;  // sub-domain column of the group's first lane
                if (off < bw) {
                    const long long gf = (long long)ts.k * plane + (long long)(or0 + r0 + ts.r) * a.Z1 + oc0 + c0 + off;
                    if (gf + 3 < nall) {
                        bv[u] = __ldcg(reinterpret_cast<const float4 *>(a.beta + gf));
                        zv[u] = zskip ? make_float4(0.f, 0.f, 0.f, 0.f)
                                      : __ldcg(reinterpret_cast<const float4 *>(a.Z + gf));
                    } else {  // the array's last group: element by element
                        float b4[4], z4[4];
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const bool in = off + e >= 0 && off + e < bw;
                            b4[e] = in ? __ldcg(a.beta + gf + e) : 0.f;
                            z4[e] = (in && !zskip) ? __ldcg(a.Z + gf + e) : 0.f;
                        }
                        bv[u] = make_float4(b4[0], b4[1], b4[2], b4[3]);
                        zv[u] = make_float4(z4[0], z4[1], z4[2], z4[3]);
                    }
                }
            }
            ts.next();
        }
        TaskStep rs = ts;
        rs.k = k_s;
        rs.r = r_s;
        rs.j = j_s;
#pragma unroll
        for (int u = 0; u < B; u++) {
            const int k = rs.k;
            const int sft = (int)((k * plane_lo + base_lo + (unsigned)rs.r * (unsigned)a.Z1) & 3u);
            const int lj0 = c0 + 4 * rs.j - sft;  // tile column of the group's first lane
            rs.next();
            if (t + u * NT >= total || lj0 >= c0 + bw) continue;
            const float nk = snrm[k], ik = sinv[k];
            const float b4[4] = {bv[u].x, bv[u].y, bv[u].z, bv[u].w};
            const float z4[4] = {zv[u].x, zv[u].y, zv[u].z, zv[u].w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int lj = lj0 + e;
                if (lj >= c0 && lj < c0 + bw) {
                    const float zn = coord_update(b4[e], a.lambda, nk, ik);
                    const float dz = zn - z4[e];
                    const float ad = fabsf(dz);
                    const int t4 = (t + u * NT) * 4 + e;
                    if (ad > ba) {
                        ba = ad;
                        bt = t4;
                        bzn = zn;
                        bdz = dz;
                    }
                }
            }
        }
    }
    unsigned key = 0xffffffffu;
    if (bt >= 0) {
        const int per_k = bh * NG, t = bt >> 2, k = t / per_k, rem = t - k * per_k, r = rem / NG, j = rem - r * NG;
        const int sft = (int)((k * plane_lo + base_lo + (unsigned)r * (unsigned)a.Z1) & 3u);
        key = (unsigned)(((r0 + r) * a.t1 + c0 + 4 * j - sft + (bt & 3)) * K + k);
    }
    return Cand<float>{ba, key, bzn, bdz};
}

// beta_k[s] -= C[k][k0][s - s0] dz over V(s0) within the domain, except
// (k0, s0) itself (Eq. beta_update), as 16-byte reductions.  The table loads
// of B tasks are issued before their reductions.
template <int NT, int B>
__device__ __forceinline__ void window_v4(const LgcdArgs<float> &a, int k0, int gi0, int gj0, float dz) {
    const int K = a.K, W0 = a.W0, W1 = a.W1;
    const long long plane = (long long)a.Z0 * a.Z1, nall = (long long)K * plane;
    const int NG = (W1 + 6) >> 2, total = K * W0 * NG;
    const int gjs = gj0 - (a.L1 - 1);  // domain column of window column 0
    const bool col_edge = gjs < 0 || gj0 + a.L1 - 1 >= a.Z1;
    TaskStep ts;
    ts.init(threadIdx.x, NT, W0, NG);
    for (int t = threadIdx.x; t < total; t += B * NT) {
        float v[B][4];
        long long gf[B];
        unsigned ok[B];
#pragma unroll
        for (int u = 0; u < B; u++) {
            const int k = ts.k, rw = ts.r, j = ts.j;
            ts.next();
            ok[u] = 0;
            gf[u] = 0;
            const int gi = gi0 + rw - (a.L0 - 1);
            if (t + u * NT >= total || gi < 0 || gi >= a.Z0) continue;
            const long long row = (long long)k * plane + (long long)gi * a.Z1 + gjs;  // window column 0
            const int cw0 = 4 * j - (int)(row & 3);  // window column of the group's first lane
            if (cw0 >= W1) continue;
            const float *crow = a.dtd + ((size_t)(k * K + k0) * W0 + rw) * W1;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int cw = cw0 + e, gj = gjs + cw;
                const bool in = cw >= 0 && cw < W1 && (!col_edge || (gj >= 0 && gj < a.Z1)) &&
                                !(k == k0 && rw == a.L0 - 1 && cw == a.L1 - 1);
                v[u][e] = in ? __ldg(crow + cw) : 0.f;
                ok[u] |= (in ? 1u : 0u) << e;
            }
            gf[u] = row + cw0;
        }
#pragma unroll
        for (int u = 0; u < B; u++) {
            if (!ok[u]) continue;
            float d[4];
#pragma unroll
            for (int e = 0; e < 4; e++) d[e] = (ok[u] >> e & 1u) ? -(v[u][e] * dz) : 0.f;
            if (gf[u] >= 0 && gf[u] + 3 < nall) {
                red_add_v4(a.beta + gf[u], d[0], d[1], d[2], d[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; e++)
                    if (ok[u] >> e & 1u) atomicAdd(a.beta + gf[u] + e, d[e]);
            }
        }
    }
}

// ------------------------------------------------------------ soft-lock
// The part of V(s0) outside the tile as strip A = rows outside the tile rows
// (full width of V, nA rows from ra0, wA columns from u0) and strip B = tile
// rows, columns outside the tile columns (nB rows from rb0, wB columns from
// cb0).
struct SoftlockStrips {
    int ra0, nA, u0, wA, rb0, nB, cb0, wB;
};
template <typename real>
struct Pair {
    real x, y;
};

// This warp's maxima of |dZ| over the coordinates of both strips held by
// lower-ranked (x) and higher-ranked (y) tiles, in units of (atom, block of RB
// rows, 32-column chunk); a warp stops once any warp of the CTA found a
// blocker of the candidate's |dZ| ba (Eq. soft_lock: it loses to a
// lower-ranked tile on a tie, to a higher-ranked one only when strictly
// smaller).  Out of line, so that its registers do not weigh on the rest of
// the worker (inlined, its spills cost up to 40 % of the phase).
template <typename real, int NT, int RB>
__device__ __noinline__ Pair<real> softlock_maxima(const real *beta, const real *Zg, const real *snrm,
                                                   const real *sinv, real lambda, int K, int Z1, size_t plane, int G1,
                                                   int w, int ta, int tb, int or0, int oc0, int h, int wd,
                                                   SoftlockStrips sl, real ba, volatile int *s_block) {
    constexpr int NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    real lo = real(-1), hi = real(-1);
    const int nchA = (sl.wA + 31) >> 5, nchB = (sl.wB + 31) >> 5;
    const int unA = ((sl.nA + RB - 1) / RB) * nchA;
    const int per_k = unA + ((sl.nB + RB - 1) / RB) * nchB;
    for (int u = warp; u < K * per_k; u += NW) {
        if (*s_block) break;  // another warp already rejects the candidate
        const int k = u / per_k, rem = u - k * per_k;
        const bool inA = rem < unA;
        const int nchS = inA ? nchA : nchB, remS = inA ? rem : rem - unA;
        const int rb = remS / nchS, ch = remS - rb * nchS;
        const int cc = ch * 32 + lane;
        const int gi = (inA ? sl.ra0 : sl.rb0) + rb * RB, gj = (inA ? sl.u0 : sl.cb0) + cc;
        const int nrow = cc < (inA ? sl.wA : sl.wB) ? min(RB, (inA ? sl.nA : sl.nB) - rb * RB) : 0;
        const real *bk = beta + (size_t)k * plane, *zk = Zg + (size_t)k * plane;
        const int o0 = gi * Z1 + gj;
        real bv[RB], zv[RB];
#pragma unroll
        for (int q = 0; q < RB; q++) {
            if (q < nrow) {
                bv[q] = ld_relaxed(bk + (o0 + q * Z1));
                zv[q] = ld_relaxed(zk + (o0 + q * Z1));
            }
        }
        // rank of the tile holding (gi + q, gj): neighbours of a tile are at
        // most one tile away in each direction
        const int tj = gj < oc0 ? tb - 1 : (gj >= oc0 + wd ? tb + 1 : tb);
        const real nk = snrm[k], ik = sinv[k];
#pragma unroll
        for (int q = 0; q < RB; q++) {
            if (q < nrow) {
                real d = coord_update(bv[q], lambda, nk, ik) - zv[q];
                d = d < real(0) ? -d : d;
                const int gq = gi + q;
                const int ti = gq < or0 ? ta - 1 : (gq >= or0 + h ? ta + 1 : ta);
                if (ti * G1 + tj < w) lo = max(lo, d);
                else hi = max(hi, d);
            }
        }
        if (__any_sync(0xffffffffu, lo >= ba || hi > ba) && lane == 0) *s_block = 1;
    }
    return Pair<real>{lo, hi};
}

// ------------------------------------------------ staged window update
// The single-solve FP32 kernel stages the K blocks C[k][k0] (k = 0..K-1) of
// an update in shared memory: a ring of a.wslots slots, each filled by one
// bulk copy (cp.async.bulk) whose completion lands on the slot's mbarrier,
// so that the table reads of an update overlap one another and the
// reductions instead of costing one L2 round trip per group of four.  The
// workspace copy of the table is laid out for it: block (k0, k) holds W0 rows
// of wrs floats, row rw's W1 values starting at rw * wrs + 4 with zeros
// around them, and the centre of C[k0][k0] is 0 (an update leaves beta at
// (k0, s0) itself alone).  Because wrs = Z1 (mod 4), the four values of every
// 16-byte group of beta in one block start at the same offset mod 4 of the
// slot: two aligned 16-byte loads and a fixed selection per block.
constexpr int kMaxStageSlots = 4;

// Byte offset of the first slot in the worker's dynamic shared memory (after
// the 2 K atom norms and inverses, 128-byte aligned).
__host__ __device__ constexpr size_t stage_offset(int K) { return ((size_t)2 * K * 8 + 127) & ~(size_t)127; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void stage_issue(uint32_t dst, const float *src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Waits for the phase of the given parity of a slot's mbarrier; false after
// 100 ms (a bulk copy of a few kB lands in microseconds).
__device__ __forceinline__ bool stage_wait(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (globaltimer_ns() - t0 > 100000000ull) return false;
    }
}

// beta_k[s] -= C[k][k0][s - s0] dz over the window rows of atom k, the
// block C[k][k0] read from a slot; CP = the slot offset mod 4 of every group.
template <int NT, int CP>
__device__ __forceinline__ void window_block(const LgcdArgs<float> &a, const float *blk, int k, int gi0, int gjs,
                                             bool col_edge, float dz) {
    const long long plane = (long long)a.Z0 * a.Z1, nall = (long long)a.K * plane;
    const int W1 = a.W1, RS = a.wrs, NG = (W1 + 6) >> 2;
    for (int t = threadIdx.x; t < a.W0 * NG; t += NT) {
        const int rw = t / NG, j = t - rw * NG;
        const int gi = gi0 + rw - (a.L0 - 1);
        if (gi < 0 || gi >= a.Z0) continue;
        const long long row = (long long)k * plane + (long long)gi * a.Z1 + gjs;  // window column 0
        const int cw0 = 4 * j - (int)(row & 3);  // window column of the group's first lane
        if (cw0 >= W1) continue;
        const int idx = rw * RS + 4 + cw0;
        float c[4];
        if ((idx & 3) == CP) {
            const float *p = blk + (idx - CP);  // 16-byte aligned
            const float4 lo = *reinterpret_cast<const float4 *>(p);
            if constexpr (CP == 0) {
                c[0] = lo.x;
                c[1] = lo.y;
                c[2] = lo.z;
                c[3] = lo.w;
            } else {
                const float4 hi = *reinterpret_cast<const float4 *>(p + 4);
                const float v[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
                for (int e = 0; e < 4; e++) c[e] = v[CP + e];
            }
        } else {  // not reached (wrs = Z1 mod 4); element by element
#pragma unroll
            for (int e = 0; e < 4; e++) c[e] = blk[idx + e];
        }
        if (col_edge) {
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int gj = gjs + cw0 + e;
                if (gj < 0 || gj >= a.Z1) c[e] = 0.f;
            }
        }
        const long long gf = row + cw0;
        if (gf >= 0 && gf + 3 < nall) {
            red_add_v4(a.beta + gf, -(c[0] * dz), -(c[1] * dz), -(c[2] * dz), -(c[3] * dz));
        } else {
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (gf + e >= 0 && gf + e < nall && c[e] != 0.f) atomicAdd(a.beta + gf + e, -(c[e] * dz));
        }
    }
}

// The window update of an accepted candidate (k0, (gi0, gj0)) through the
// staged table.  q counts the blocks this CTA has consumed (the same value
// in every thread).  Returns false when a copy did not land in time; the
// copies still in flight are then waited for once more and the caller stops
// the solve.
template <int NT>
__device__ bool window_staged(const LgcdArgs<float> &a, float *ring, uint64_t *bars, unsigned &q, int k0, int gi0,
                              int gj0, float dz) {
    const int K = a.K, S = a.wslots, slotf = a.wbs + 8;
    const long long plane = (long long)a.Z0 * a.Z1;
    const int gjs = gj0 - (a.L1 - 1);
    const bool col_edge = gjs < 0 || gj0 + a.L1 - 1 >= a.Z1;
    const float *src0 = a.wtab + (size_t)k0 * K * a.wbs;
    const uint32_t bytes = (uint32_t)a.wbs * 4u;
    const int first = min(S, K);
    if (threadIdx.x == 0)
        for (int i = 0; i < first; i++) {
            const int sl = (int)((q + i) % (unsigned)S);
            stage_issue(smem_u32(ring + (size_t)sl * slotf), src0 + (size_t)i * a.wbs, bytes, smem_u32(&bars[sl]));
        }
    int issued = first;
    bool ok = true;
    int k = 0;
    for (; k < K; k++) {
        const unsigned n = q + k;
        const int sl = (int)(n % (unsigned)S);
        const bool mine = stage_wait(smem_u32(&bars[sl]), (n / (unsigned)S) & 1u);
        if (mine) {
            const long long row0 = (long long)k * plane + (long long)(gi0 - (a.L0 - 1)) * a.Z1 + gjs;
            const int cp = (4 - (int)(row0 & 3)) & 3;
            const float *blk = ring + (size_t)sl * slotf;
            switch (cp) {
                case 0: window_block<NT, 0>(a, blk, k, gi0, gjs, col_edge, dz); break;
                case 1: window_block<NT, 1>(a, blk, k, gi0, gjs, col_edge, dz); break;
                case 2: window_block<NT, 2>(a, blk, k, gi0, gjs, col_edge, dz); break;
                default: window_block<NT, 3>(a, blk, k, gi0, gjs, col_edge, dz); break;
            }
        }
        // every thread is done with the slot (and agrees on the outcome)
        ok = __syncthreads_and(mine) != 0;
        if (!ok) break;
        if (threadIdx.x == 0 && k + S < K) {
            stage_issue(smem_u32(ring + (size_t)sl * slotf), src0 + (size_t)(k + S) * a.wbs, bytes,
                        smem_u32(&bars[sl]));
        }
        if (k + S < K) issued++;
    }
    if (!ok && threadIdx.x == 0) {
        // blocks k .. issued - 1 may still be in flight: one more bounded wait each
        for (int i = k; i < issued; i++) {
            const unsigned n = q + i;
            stage_wait(smem_u32(&bars[n % (unsigned)S]), (n / (unsigned)S) & 1u);
        }
    }
    q += K;
    return ok;
}

// The worker of tile w (all NT threads of the CTA); smem_raw holds at least
// 2 K elements, then (single-solve FP32 kernel with a staged table) the
// window slots from byte stage_offset(K).  Returns when the solve of `a`
// ends.
//
// One sub-domain per iteration.  Barriers per iteration: one after the scan
// (per-warp argmax partials, double-buffered by iteration parity, with the
// notification counters and the stop word read by warp 0 while it scanned),
// one after the soft-lock maxima (border candidates only) and one after the
// window update (accepted candidates only; the staged update adds one per
// table block).
template <typename real, int NT, int RB, bool STAGED>
__device__ void global_tile_worker(const LgcdArgs<real> &a, int w, unsigned char *smem_raw) {
    constexpr int kRowBlock = RB;
    // the staged window update (FP32 kernels built with it, a table in the
    // window layout given)
    const bool staged = STAGED && std::is_same<real, float>::value && a.wtab != nullptr;
    __shared__ __align__(8) uint64_t s_tbar[kMaxStageSlots];
    float *ring = reinterpret_cast<float *>(smem_raw + stage_offset(a.K));
    unsigned q_stage = 0;
    constexpr int NW = NT / 32;
    real *snrm = reinterpret_cast<real *>(smem_raw), *sinv = snrm + a.K;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ta = w / a.G1, tb = w % a.G1;
    const int or0 = ta * a.t0, oc0 = tb * a.t1;
    const int h = min(a.t0, a.Z0 - or0), wd = min(a.t1, a.Z1 - oc0);
    const int ns0 = (h + a.sub0 - 1) / a.sub0, ns1 = (wd + a.sub1 - 1) / a.sub1, M = ns0 * ns1;
    const int K = a.K;
    const size_t plane = (size_t)a.Z0 * a.Z1;
    for (int k = threadIdx.x; k < K; k += NT) {
        snrm[k] = real(a.nrm[k]);
        sinv[k] = real(1.0 / a.nrm[k]);
    }
    // this tile's notification counters, one per neighbour direction (each on
    // its own 128-byte line): a neighbour in direction d bumps counter d
    int *flag = a.ctl + (size_t)w * kDirs * 32;
    __shared__ Cand<real> s_red[2][NW];          // per-warp argmax, by iteration parity
    __shared__ int s_ctl[2][2];                  // bumps seen, stop state
    __shared__ real s_lo[NW], s_hi[NW];          // soft-lock maxima per warp
    __shared__ int s_pause;
    __shared__ volatile int s_block;  // a warp found a soft-lock blocker
    // state only thread 0 uses, kept out of every thread's registers
    __shared__ unsigned long long s_deadline;
    __shared__ real s_guard;
    __shared__ int s_seen[kDirs], s_cnt[5];  // bumps seen per direction; updates, iterations,
                                             // rejected, below tol, messages
    // sub-domains that the windows of the neighbour in direction d can reach
    // (rows / columns within L_i - 1 of the shared edge or corner)
    __shared__ unsigned long long s_dirmask[kDirs], s_wake;
    __shared__ unsigned long long s_gm[2];  // sub-domains next to the directions of new bumps
    // nonzeros of Z per sub-domain (tiles of at most 64): counted from a cold
    // start, never below the true count; a sub-domain at zero is scanned
    // without reading Z
    __shared__ int s_nz[64];
    // SM cycles of thread 0 per phase: scan, wait for the scan barrier,
    // soft-lock, window update, update barrier and flags, pause
    __shared__ unsigned long long s_ph[6], s_t;
    __shared__ unsigned long long s_cand;  // candidates scanned (K x |C_m| per iteration)
    if (threadIdx.x == 0) {
        s_deadline = globaltimer_ns() + a.timeout_ns;
        real guard = real(0);
        if (a.guard_on) {
            double g = 1e300;
            for (int k = 0; k < K; k++) g = fmin(g, 50.0 / a.dmax[k]);
            guard = real(g);
        }
        s_guard = guard;
        for (int d = 0; d < kDirs; d++) s_seen[d] = 0;
        for (int i = 0; i < 5; i++) s_cnt[i] = 0;
        for (int i = 0; i < 6; i++) s_ph[i] = 0;
        s_cand = 0;
        s_t = clock64();
        if (staged) {
            for (int i = 0; i < a.wslots; i++)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_tbar[i])) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    // Dirty sub-domains (tiles of at most 64): a bit is cleared when a scan
    // finds nothing above tol and set again when beta in the sub-domain may
    // have changed -- an accepted update whose window V(s0) reaches it, or a
    // neighbour's notification for those facing that neighbour.  The worker
    // pauses once no sub-domain is dirty.  Larger tiles scan cyclically and
    // pause after M quiet iterations.
    const bool use_mask = M <= 64;
    for (int q = threadIdx.x; q < 64; q += NT) s_nz[q] = a.z_zero ? 0 : (1 << 24);
    unsigned long long dmask = 0;
    if (threadIdx.x < kDirs) s_dirmask[threadIdx.x] = 0;  // tiles of more than 64 sub-domains: unused
    if (use_mask) {
        dmask = M == 64 ? ~0ull : ((1ull << M) - 1ull);
        if (threadIdx.x < kDirs) {
            int dr, dc;
            dir_offset(threadIdx.x, dr, dc);
            // rows [ra, rb) x columns [ca, cb) of the tile that the windows of
            // that neighbour reach
            const int ra = dr > 0 ? h - (a.L0 - 1) : 0, rb = dr < 0 ? a.L0 - 1 : h;
            const int ca = dc > 0 ? wd - (a.L1 - 1) : 0, cb = dc < 0 ? a.L1 - 1 : wd;
            unsigned long long mk = 0;
            for (int q = 0; q < M; q++) {
                const int qr = q / ns1, qc = q - qr * ns1;
                const int rr0 = qr * a.sub0, rr1 = min(h, rr0 + a.sub0), cc0 = qc * a.sub1, cc1 = min(wd, cc0 + a.sub1);
                if (rr0 < rb && rr1 > ra && cc0 < cb && cc1 > ca) mk |= 1ull << q;
            }
            s_dirmask[threadIdx.x] = mk;
        }
    }
    int m = 0, quiet = 0, par = 0;
    __syncthreads();
    for (;;) {
        // lane d of warp 0 reads this tile's counter of direction d, thread 0
        // the stop word; the loads overlap their share of the scan
        int f_now = 0, stop_now = 0;
        if (threadIdx.x < kDirs) f_now = ld_relaxed(flag + threadIdx.x * 32);
        if (threadIdx.x == 0) stop_now = ld_relaxed(&a.hdr->stop);
        // ---- scan sub-domain m (Eq. gcd_candidate)
        const int mr = m / ns1, mc = m - mr * ns1;
        const int r0 = mr * a.sub0, c0 = mc * a.sub1;
        const int bh = min(a.sub0, h - r0), bw = min(a.sub1, wd - c0);
        Cand<real> c{real(-1), 0xffffffffu, real(0), real(0)};
        if constexpr (std::is_same<real, float>::value) {
            // FP32: the vector scan (beta and Z start on 16-byte boundaries,
            // checked by the host)
            c = scan_v4<NT, kScanBatch>(a, snrm, sinv, or0, oc0, r0, c0, bh, bw, use_mask && s_nz[m] == 0);
        } else {
            const int nrb = (bh + kRowBlock - 1) / kRowBlock, nch = (bw + 31) >> 5, per_k = nrb * nch;
            for (int u = warp; u < K * per_k; u += NW) {
                const int k = u / per_k, rem = u - k * per_k, rb = rem / nch, ch = rem - rb * nch;
                const int cc = ch * 32 + lane, lj = c0 + cc, li = r0 + rb * kRowBlock;
                const int nrow = cc < bw ? min(kRowBlock, bh - rb * kRowBlock) : 0;
                // positions are below 2^31: 32-bit offsets within atom k's plane
                const real *bk = a.beta + (size_t)k * plane, *zk = a.Z + (size_t)k * plane;
                const int o0 = (or0 + li) * a.Z1 + oc0 + lj;
                real bv[kRowBlock], zv[kRowBlock];
#pragma unroll
                for (int q = 0; q < kRowBlock; q++) {
                    if (q < nrow) {
                        bv[q] = __ldcg(bk + (o0 + q * a.Z1));
                        // Z through L2: in the persistent queue an L1 line may
                        // still hold this address from an earlier job
                        zv[q] = __ldcg(zk + (o0 + q * a.Z1));
                    }
                }
                const real nk = snrm[k], ik = sinv[k];
#pragma unroll
                for (int q = 0; q < kRowBlock; q++) {
                    if (q < nrow) {
                        const real zn = coord_update(bv[q], a.lambda, nk, ik);
                        const real dz = zn - zv[q];
                        Cand<real> x{dz < real(0) ? -dz : dz, (unsigned)(((li + q) * a.t1 + lj) * K + k), zn, dz};
                        if (better(x, c)) c = x;
                    }
                }
            }
        }
        c = warp_argmax(c);
        if (warp == 0) {
            // bumps per direction since the last look: their count and the
            // directions they came from
            int got = 0;
            if (lane < kDirs) {
                got = f_now - s_seen[lane];
                s_seen[lane] = f_now;
            }
            const int gmask = (int)(__ballot_sync(0xffffffffu, got != 0) & ((1u << kDirs) - 1u));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) got += __shfl_xor_sync(0xffffffffu, got, o);
            if (lane == 0) {
                const unsigned long long t = clock64();
                s_ph[0] += t - s_t;
                s_t = t;
                int state = 0;
                unsigned long long gm = 0;
                if (got) {
                    atomicSub(&a.hdr->pending, got);  // observed: no longer in flight
                    for (int d = 0; d < kDirs; d++)
                        if (gmask >> d & 1) gm |= s_dirmask[d];
                }
                s_gm[par] = gm;
                if (stop_now) state = 1;
                else if (globaltimer_ns() > s_deadline) {
                    set_stop(a.hdr, CSC_ERR_TIMEOUT);
                    state = 1;
                }
                s_ctl[par][0] = got;
                s_ctl[par][1] = state;
            }
        }
        if (lane == 0) s_red[par][warp] = c;
        if (threadIdx.x == 0) s_block = 0;  // read after the barrier below
        __syncthreads();
        if (s_ctl[par][1]) break;
        const int got = s_ctl[par][0];
        Cand<real> best = s_red[par][0];
#pragma unroll 4
        for (int i = 1; i < NW; i++) {
            const Cand<real> y = s_red[par][i];
            if (better(y, best)) best = y;
        }
        par ^= 1;
        if (threadIdx.x == 0) {
            s_cnt[1]++;
            s_cand += (unsigned long long)K * bh * bw;
            const unsigned long long t = clock64();
            s_ph[1] += t - s_t;
            s_t = t;
        }
        const bool active = best.a >= a.eps;
        bool accepted = false;
        int li0 = 0, lj0 = 0;
        if (active) {
            const unsigned pos = best.key / (unsigned)K;
            const int k0 = (int)(best.key - pos * (unsigned)K);
            li0 = (int)(pos / (unsigned)a.t1);
            lj0 = (int)(pos - (unsigned)li0 * (unsigned)a.t1);
            const int gi0 = or0 + li0, gj0 = oc0 + lj0;
            const bool border = in_band(li0, lj0, h, wd, a.L0, a.L1);
            bool accept = true;
            if (border && a.mode == CSC_MODE_ASYNC) {
                // soft-lock over the part of V(s0) outside the tile: strip A =
                // rows outside the tile rows (full width of V), strip B = tile
                // rows, columns outside the tile columns
                const int v0 = max(0, gi0 - (a.L0 - 1)), v1 = min(a.Z0, gi0 + a.L0);
                const int u0 = max(0, gj0 - (a.L1 - 1)), u1 = min(a.Z1, gj0 + a.L1);
                const int ra0 = v0 < or0 ? v0 : max(v0, or0 + h), ra1 = v0 < or0 ? min(v1, or0) : v1;
                const int rb0 = max(v0, or0), rb1 = min(v1, or0 + h);
                const int cb0 = u0 < oc0 ? u0 : max(u0, oc0 + wd), cb1 = u0 < oc0 ? min(u1, oc0) : u1;
                const int nA = max(0, ra1 - ra0), nB = (cb1 > cb0) ? max(0, rb1 - rb0) : 0;
                const int wA = u1 - u0, wB = max(0, cb1 - cb0);
                const SoftlockStrips sl{ra0, nA, u0, wA, rb0, nB, cb0, wB};
                const Pair<real> lh = softlock_maxima<real, NT, kRowBlock>(
                    a.beta, a.Z, snrm, sinv, a.lambda, K, a.Z1, plane, a.G1, w, ta, tb, or0, oc0, h, wd, sl, best.a,
                    &s_block);
                real lo = lh.x, hi = lh.y;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    lo = max(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
                }
                if (lane == 0) {
                    s_lo[warp] = lo;
                    s_hi[warp] = hi;
                }
                __syncthreads();
                real mlo = s_lo[0], mhi = s_hi[0];
#pragma unroll 4
                for (int i = 1; i < NW; i++) {
                    mlo = max(mlo, s_lo[i]);
                    mhi = max(mhi, s_hi[i]);
                }
                accept = best.a > mlo && best.a >= mhi;
                if (threadIdx.x == 0) {
                    if (!accept) s_cnt[2]++;
                    const unsigned long long t = clock64();
                    s_ph[2] += t - s_t;
                    s_t = t;
                }
            }
            if (accept) {
                accepted = true;
                // Z first: the barrier after the window update publishes both
                // to the next scan
                if (threadIdx.x == 0) {
                    a.Z[k0 * plane + (size_t)gi0 * a.Z1 + gj0] = best.znew;
                    if (use_mask) {
                        // Z was zero exactly when Z' - dZ is (dZ = Z' - 0 is exact);
                        // the converse can fail only towards a larger count
                        const bool was0 = best.znew - best.dz == real(0), now0 = best.znew == real(0);
                        if (was0 && !now0) s_nz[m]++;
                        else if (!was0 && now0) s_nz[m]--;
                    }
                }
                // beta_k[s] -= C[k][k0][s - s0] dz on V(s0) within the domain
                const real dz = best.dz;
                if constexpr (std::is_same<real, float>::value) {
                    if (staged) {
                        if (!window_staged<NT>(a, ring, s_tbar, q_stage, k0, gi0, gj0, dz) && threadIdx.x == 0)
                            set_stop(a.hdr, CSC_ERR_TIMEOUT);
                    } else {
                        window_v4<NT, kWindowBatch>(a, k0, gi0, gj0, dz);
                    }
                } else {
                    // the table loads of a unit first, then its reductions
                    const int W0 = a.W0, W1 = a.W1;
                    const int nrb = (W0 + kRowBlock - 1) / kRowBlock, nch = (W1 + 31) >> 5, per_k = nrb * nch;
                    for (int u = warp; u < K * per_k; u += NW) {
                        const int k = u / per_k, rem = u - k * per_k, rb = rem / nch, ch = rem - rb * nch;
                        const int cw = ch * 32 + lane, rw0 = rb * kRowBlock;
                        const int gj = gj0 + cw - (a.L1 - 1), gi = gi0 + rw0 - (a.L0 - 1);
                        // rows of this unit inside the domain: [q_lo, q_hi)
                        const bool colok = cw < W1 && gj >= 0 && gj < a.Z1;
                        const int q_lo = max(0, -gi), q_hi = colok ? min(min(kRowBlock, W0 - rw0), a.Z0 - gi) : 0;
                        const real *crow = a.dtd + (((size_t)k * K + k0) * W0 + rw0) * W1 + cw;
                        real cv[kRowBlock];
#pragma unroll
                        for (int q = 0; q < kRowBlock; q++)
                            if (q >= q_lo && q < q_hi) cv[q] = __ldg(crow + q * W1);
                        real *bk = a.beta + (size_t)k * plane;
                        const int o0 = gi * a.Z1 + gj;
#pragma unroll
                        for (int q = 0; q < kRowBlock; q++)
                            if (q >= q_lo && q < q_hi && !(k == k0 && gi + q == gi0 && gj == gj0))
                                atomicAdd(bk + (o0 + q * a.Z1), -(cv[q] * dz));
                    }
                }
                if (threadIdx.x == 0) {
                    const unsigned long long t = clock64();
                    s_ph[3] += t - s_t;
                    s_t = t;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    s_cnt[0]++;
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
                            // the receiver sees this tile in the opposite direction
                            atomicAdd(a.ctl + (size_t)((ta + dr) * a.G1 + (tb + dc)) * kDirs * 32 +
                                          (size_t)(kDirs - 1 - dl[i]) * 32,
                                      1);
                        }
                        s_cnt[4] += nd;
                    }
                    if (a.max_updates > 0) {
                        unsigned long long prev = atomicAdd(&a.hdr->updates_total, 1ull);
                        if ((long long)prev + 1 >= a.max_updates) set_stop(a.hdr, CSC_NOT_CONVERGED);
                    }
                    const real az = best.znew < real(0) ? -best.znew : best.znew;
                    if (a.guard_on && az > s_guard) set_stop(a.hdr, CSC_ERR_DIVERGED);
                    const unsigned long long t = clock64();
                    s_ph[4] += t - s_t;
                    s_t = t;
                }
            }
        } else if (threadIdx.x == 0) {
            s_cnt[3]++;
        }
        bool pause;
        if (use_mask) {
            if (!active) dmask &= ~(1ull << m);
            if (accepted) {
                // sub-domains that V(s0) reaches (rows / columns within L - 1)
                const int qr0 = max(0, li0 - (a.L0 - 1)) / a.sub0, qr1 = min(h - 1, li0 + a.L0 - 1) / a.sub0;
                const int qc0 = max(0, lj0 - (a.L1 - 1)) / a.sub1, qc1 = min(wd - 1, lj0 + a.L1 - 1) / a.sub1;
                for (int qr = qr0; qr <= qr1; qr++)
                    for (int qc = qc0; qc <= qc1; qc++) dmask |= 1ull << (qr * ns1 + qc);
            }
            // sub-domains next to the neighbours that notified (this
            // iteration's parity, flipped since)
            dmask |= s_gm[par ^ 1];
            pause = dmask == 0;
        } else {
            quiet = (active || got > 0) ? 0 : quiet + 1;
            pause = quiet >= M;
        }
        if (pause) {
            // pause until a neighbour bumps a counter or every worker is done
            if (threadIdx.x == 0) {
                atomicSub(&a.hdr->pending, 1);
                int state = 0;
                for (;;) {
                    bool woken = false;
                    for (int d = 0; d < kDirs; d++) woken |= ld_relaxed(flag + d * 32) != s_seen[d];
                    if (woken) {
                        atomicAdd(&a.hdr->pending, 1);
                        break;
                    }
                    if (ld_acquire(&a.hdr->pending) == 0 || ld_relaxed(&a.hdr->stop)) {
                        state = 1;
                        break;
                    }
                    if (globaltimer_ns() > s_deadline) {
                        set_stop(a.hdr, CSC_ERR_TIMEOUT);
                        state = 1;
                        break;
                    }
                    __nanosleep(256);
                }
                if (!state) {
                    // the directions that woke this tile (at least one)
                    unsigned long long wk = 0;
                    for (int d = 0; d < kDirs; d++)
                        if (ld_relaxed(flag + d * 32) != s_seen[d]) wk |= s_dirmask[d];
                    s_wake = wk;
                }
                s_pause = state;
                const unsigned long long t = clock64();
                s_ph[5] += t - s_t;
                s_t = t;
            }
            __syncthreads();
            if (s_pause) break;
            quiet = 0;
            // woken by a notification: beta next to that neighbour has changed
            // (the next iteration reads the counters and accounts for the bumps)
            if (use_mask) dmask |= s_wake;
            if (use_mask && dmask == 0) dmask = M == 64 ? ~0ull : ((1ull << M) - 1ull);
        }
        if (use_mask) {
            // the next dirty sub-domain after m, cyclically
            const unsigned long long above = m + 1 < 64 ? (dmask >> (m + 1)) << (m + 1) : 0ull;
            m = above ? __ffsll((long long)above) - 1 : __ffsll((long long)dmask) - 1;
        } else {
            m = (m + 1 == M) ? 0 : m + 1;
        }
    }
    if (threadIdx.x == 0) {
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_UPDATES], (unsigned long long)s_cnt[0]);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_ITERS], (unsigned long long)s_cnt[1]);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_REJECTED], (unsigned long long)s_cnt[2]);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_SUBTOL], (unsigned long long)s_cnt[3]);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_MESSAGES], (unsigned long long)s_cnt[4]);
        atomicAdd((unsigned long long *)&a.hdr->stat[ST_CAND], s_cand);
        atomicMax(&a.hdr->wmax[0], (unsigned long long)s_cnt[1]);
        atomicMax(&a.hdr->wmax[1], (unsigned long long)s_cnt[0]);
        for (int i = 0; i < 6; i++) {
            atomicAdd(&a.hdr->tph[i], s_ph[i]);
            atomicMax(&a.hdr->tphmax[i], s_ph[i]);
        }
    }
}

}  // namespace csc
