// residual.cu -- the residual X - Z*D, the objective of Eq. csc in FP64,
// beta recomputed from its definition (Section 3) and the final
// max |dZ| check of Alg. 1 on that fresh beta.
//
// Z is sparse at the optimum, so the reconstruction is a scatter from the
// compacted nonzeros of Z with FP64 atomics: every nonzero (k, s, z) adds
// -z D_k to the residual on s + Theta.  If the nonzeros do not fit the list
// the residual is rebuilt densely instead.
#include <cstdint>

#include "lgcd_global.cuh"

namespace csc {

// Nonzeros of Z into (k, s, z) lists; order is unspecified (one atomic per
// warp).  Counts past the capacity only set the overflow flag.  The same
// pass accumulates ||Z||_1 in FP64.
// The same for FP32 Z on a 16-byte boundary: each thread reads four entries
// with one 16-byte load; a warp reserves its nonzeros with one atomic and
// places them by a prefix sum of the per-thread counts.
template <int NT>
__global__ void __launch_bounds__(NT) compact_v4_kernel(const float *Z, long long zpos, int K, int *nk, int *ns,
                                                       float *nzv, long long cap, WsHeader *h) {
    const long long n = (long long)K * zpos, n4 = n / 4, groups = (n + 3) / 4;
    const int lane = threadIdx.x & 31;
    double l1 = 0.0;
    const float4 *Z4 = reinterpret_cast<const float4 *>(Z);
    // the loop bound is the same for every thread of the block (warp-wide
    // shuffles below); threads past the end hold no entries
    for (long long base = (long long)blockIdx.x * NT; base < groups; base += (long long)gridDim.x * NT) {
        const long long g = base + threadIdx.x, i0 = 4 * g;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (g < n4) {
            const float4 w = __ldcs(Z4 + g);
            v[0] = w.x;
            v[1] = w.y;
            v[2] = w.z;
            v[3] = w.w;
        } else if (g < groups) {  // the last n mod 4 entries
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (i0 + e < n) v[e] = Z[i0 + e];
        }
        unsigned m4 = 0;
#pragma unroll
        for (int e = 0; e < 4; e++) m4 |= (v[e] != 0.f ? 1u : 0u) << e;
        const int c = __popc(m4);
        int x = c;  // inclusive prefix of the counts over the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int total = __shfl_sync(0xffffffffu, x, 31);
        if (total == 0) continue;
        unsigned long long wbase = 0;
        if (lane == 0) wbase = atomicAdd((unsigned long long *)&h->nnz, (unsigned long long)total);
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        long long idx = (long long)wbase + x - c;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            if (m4 >> e & 1u) {
                l1 += fabs((double)v[e]);
                const long long i = i0 + e;
                if (idx < cap) {
                    nk[idx] = (int)(i / zpos);
                    ns[idx] = (int)(i % zpos);
                    nzv[idx] = v[e];
                } else {
                    h->overflow = 1;
                }
                idx++;
            }
        }
    }
    block_sum_atomic<NT>(l1, &h->obj_g);
}

template <typename real, int NT>
__global__ void __launch_bounds__(NT) compact_any_kernel(const real *Z, long long zpos, int K,
                                                         int *nk, int *ns, real *nzv, long long cap,
                                                         WsHeader *h) {
    const long long n = (long long)K * zpos;
    const int lane = threadIdx.x & 31;
    double l1 = 0.0;
    for (long long base = (long long)blockIdx.x * NT; base < n; base += (long long)gridDim.x * NT) {
        long long i = base + threadIdx.x;
        real v = i < n ? Z[i] : real(0);
        bool nzb = v != real(0);
        unsigned ball = __ballot_sync(0xffffffffu, nzb);
        if (ball == 0) continue;
        if (nzb) l1 += fabs((double)v);
        unsigned long long wbase = 0;
        if (lane == 0) wbase = atomicAdd((unsigned long long *)&h->nnz, (unsigned long long)__popc(ball));
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (nzb) {
            long long idx = (long long)wbase + __popc(ball & ((1u << lane) - 1u));
            if (idx < cap) {
                nk[idx] = (int)(i / zpos);
                ns[idx] = (int)(i % zpos);
                nzv[idx] = v;
            } else {
                h->overflow = 1;
            }
        }
    }
    block_sum_atomic<NT>(l1, &h->obj_g);
}

template <typename real>
__global__ void residual_init_kernel(const real *X, double *R, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        R[i] = (double)X[i];
}

// R_p[s + tau] -= z D_kp[tau] for every listed nonzero (FP64 atomics).
template <typename real, int NT>
__global__ void __launch_bounds__(NT) scatter_kernel(const int *nk, const int *ns, const real *nzv,
                                                     const WsHeader *h, long long cap, const real *D,
                                                     double *R, int P, int L0, int L1, int T0, int T1,
                                                     int Z1) {
    if (h->overflow) return;
    const long long cnt = h->nnz < cap ? h->nnz : cap;
    const int LL = L0 * L1, per = P * LL;
    for (long long e = blockIdx.x; e < cnt; e += gridDim.x) {
        const int k = nk[e], s = ns[e];
        const double z = (double)nzv[e];
        const int i = s / Z1, j = s % Z1;
        for (int q = threadIdx.x; q < per; q += NT) {
            int p = q / LL, r = q % LL, ta = r / L1, tb = r % L1;
            double v = z * (double)D[(size_t)k * per + q];
            atomicAdd(&R[((size_t)p * T0 + i + ta) * T1 + j + tb], -v);
        }
    }
}

// Dense fallback when the nonzero list overflowed:
// R_p[t] = X_p[t] - sum_k sum_tau Z_k[t - tau] D_kp[tau].
template <typename real>
__global__ void recon_dense_kernel(const real *X, const real *Z, const real *D, const WsHeader *h,
                                   double *R, int P, int K, int T0, int T1, int L0, int L1, int Z0,
                                   int Z1) {
    if (!h->overflow) return;
    const long long n = (long long)P * T0 * T1;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        int p = (int)(q / ((long long)T0 * T1));
        int rem = (int)(q % ((long long)T0 * T1));
        int t0 = rem / T1, t1 = rem % T1;
        double acc = 0.0;
        for (int k = 0; k < K; k++)
            for (int a = 0; a < L0; a++) {
                int s0 = t0 - a;
                if (s0 < 0 || s0 >= Z0) continue;
                for (int b = 0; b < L1; b++) {
                    int s1 = t1 - b;
                    if (s1 < 0 || s1 >= Z1) continue;
                    acc += (double)Z[((size_t)k * Z0 + s0) * Z1 + s1] *
                           (double)D[(((size_t)k * P + p) * L0 + a) * L1 + b];
                }
            }
        R[q] = (double)X[q] - acc;
    }
}

// sum of squared residuals (FP64) and the residual in the solve precision.
template <typename real, int NT>
__global__ void __launch_bounds__(NT) residual_finish_kernel(const double *R, real *Rr, long long n,
                                                             double *out) {
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
        const double r = R[i];
        s += r * r;
        if (Rr) Rr[i] = (real)r;
    }
    block_sum_atomic<NT>(s, out);
}

__global__ void refresh_reset_kernel(WsHeader *h) {
    h->nnz = 0;
    h->overflow = 0;
    h->obj_f = 0.0;
    h->obj_g = 0.0;
    h->maxdz_bits = 0ull;
}

static int grid_for(long long n, int nt) {
    long long b = ceil_div(n, nt);
    return (int)(b < 152 * 8 ? (b < 1 ? 1 : b) : 152 * 8);
}

// ------------------------------------------- beta rebuilt from the initial beta
// beta = beta0 - sum over the nonzeros (k', s', z') of C[k][k'][s - s'] z',
// (k, s) != (k', s'): the definition of beta (Section 3), DtX - DtD Z with
// the diagonal term removed, evaluated from the initial beta0 = D~ * X kept
// by the solve.  Every kernel returns at once when the nonzero list
// overflowed; the correlation of the residual then runs instead.
template <int NT>
__global__ void __launch_bounds__(NT) copy_beta0_kernel(const float *src, float *dst, long long n,
                                                         const WsHeader *h) {
    if (h->overflow) return;
    const long long n4 = n >> 2;  // both arrays start on 16-byte boundaries
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n4; i += (long long)gridDim.x * NT)
        d4[i] = __ldcs(s4 + i);
    for (long long i = 4 * n4 + (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT)
        dst[i] = src[i];
}

template <int NT>
__global__ void __launch_bounds__(NT) nz_window_kernel(LgcdArgs<float> a, const int *nk, const int *ns,
                                                        const float *nzv, const WsHeader *h, long long cap) {
    if (h->overflow) return;
    const long long cnt = h->nnz < cap ? h->nnz : cap;
    for (long long e = blockIdx.x; e < cnt; e += gridDim.x) {
        const int s = ns[e], i = s / a.Z1;
        window_v4<NT, 2>(a, nk[e], i, s - i * a.Z1, nzv[e]);
    }
}

// max |ST(beta, lambda) / ||D_k||^2 - Z| over every coordinate (blockIdx.y = k):
// the aligned groups of four inside atom k's plane by 16-byte loads, the few
// elements before the first and after the last group one by one
__device__ __forceinline__ unsigned long long dz_bits(float b, float z, float lambda, float nr, float inv) {
    float dz = coord_update(b, lambda, nr, inv) - z;
    return nonneg_bits(dz < 0.f ? -dz : dz);
}

template <int NT>
__global__ void __launch_bounds__(NT) maxdz_kernel(const float *beta, const float *Z, const double *nrm,
                                                    float lambda, long long plane, const WsHeader *h,
                                                    unsigned long long *bits) {
    if (h->overflow) return;
    const int k = blockIdx.y;
    const double nk = nrm[k];
    const float nr = (float)nk, inv = (float)(1.0 / nk);
    const long long beg = (long long)k * plane, end = beg + plane;
    const long long g0 = (beg + 3) >> 2, g1 = end >> 2;  // whole groups [g0, g1)
    const float4 *b4 = reinterpret_cast<const float4 *>(beta), *z4 = reinterpret_cast<const float4 *>(Z);
    unsigned long long m = 0;
    for (long long g = g0 + (long long)blockIdx.x * NT + threadIdx.x; g < g1; g += (long long)gridDim.x * NT) {
        const float4 b = __ldcs(b4 + g), z = __ldcs(z4 + g);
        unsigned long long v = dz_bits(b.x, z.x, lambda, nr, inv);
        unsigned long long u = dz_bits(b.y, z.y, lambda, nr, inv);
        v = u > v ? u : v;
        u = dz_bits(b.z, z.z, lambda, nr, inv);
        v = u > v ? u : v;
        u = dz_bits(b.w, z.w, lambda, nr, inv);
        v = u > v ? u : v;
        m = v > m ? v : m;
    }
    if (blockIdx.x == 0 && threadIdx.x < 8) {
        // up to three elements before the first whole group and three after the last
        const long long i = threadIdx.x < 4 ? beg + threadIdx.x : 4 * (g1 > g0 ? g1 : g0) + (threadIdx.x - 4);
        const bool head = threadIdx.x < 4 && i < 4 * g0 && i < end;
        const bool tail = threadIdx.x >= 4 && i >= 4 * g0 && i < end;
        if (head || tail) {
            const unsigned long long v = dz_bits(beta[i], Z[i], lambda, nr, inv);
            m = v > m ? v : m;
        }
    }
    block_max_atomic<NT>(m, bits);
}

// ---------------------------------- the rebuilt beta as a gather (K <= 32)
// The same beta = beta0 - sum C[k][k'][s - s'] z' over the nonzeros, without
// reductions: the nonzeros are sorted into bins of gbh x gbw positions (a
// count, a prefix sum, a fill), then one thread per output position sums the
// terms of the nonzeros whose window holds it -- the CTA of an output tile
// stages the nonzeros of the bins within L_i - 1 of the tile in shared
// memory -- for every atom at once, writes beta and takes max |dZ| on it.
// The table is read transposed, C_t[k'][delta][k] (K padded to a multiple of
// four), so that the K coefficients of one term are contiguous (measured:
// 5.7 ms against 8.2 ms reading C as stored on the 4096^2 image).
struct GatherArgs {
    const float *beta0, *Z, *ct;  // ct: C_t
    float *beta;
    const int *off;    // [nbins + 1] bin offsets into the list
    const int4 *list;  // (k, row, column, z bits) by bin
    const double *nrm;
    const WsHeader *h;
    unsigned long long *bits;
    float lambda;
    int K, Kp, Z0, Z1, L0, L1, W0, W1, bh, bw, nb0, nb1;
};

constexpr int kGatherStage = 1024;  // staged nonzeros per pass (16 KB)

__global__ void ctab_kernel(const float *dtd, float *ct, int K, int Kp, int W) {
    const long long n = (long long)K * W * Kp;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(q % Kp);
        const long long r = q / Kp;  // k2 * W + delta
        const int k2 = (int)(r / W), d = (int)(r % W);
        ct[q] = k < K ? dtd[((size_t)k * K + k2) * W + d] : 0.f;
    }
}

__global__ void bin_count_kernel(const int *ns, const WsHeader *h, long long cap, int *cnt, int Z1, int bh, int bw,
                                 int nb1) {
    if (h->overflow) return;
    const long long n = h->nnz < cap ? h->nnz : cap;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int s = ns[e], i = s / Z1, j = s - i * Z1;
        atomicAdd(&cnt[(i / bh) * nb1 + j / bw], 1);
    }
}

// exclusive prefix sum of cnt[0..n) into off[0..n] (off[n] = total) and a
// copy into cur (the fill cursors); one CTA
template <int NT>
__global__ void __launch_bounds__(NT) bin_scan_kernel(const int *cnt, int *off, int *cur, int n, const WsHeader *h) {
    if (h->overflow) return;
    __shared__ int part[NT];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += NT) {
        const int i = base + threadIdx.x;
        const int v = i < n ? cnt[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < NT; d <<= 1) {  // inclusive scan (Hillis-Steele)
            const int t = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        const int ex = carry + part[threadIdx.x] - v;
        if (i < n) {
            off[i] = ex;
            cur[i] = ex;
        }
        __syncthreads();
        if (threadIdx.x == NT - 1) carry += part[NT - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

__global__ void bin_fill_kernel(const int *nk, const int *ns, const float *nzv, const WsHeader *h, long long cap,
                                int *cur, int4 *list, int Z1, int bh, int bw, int nb1) {
    if (h->overflow) return;
    const long long n = h->nnz < cap ? h->nnz : cap;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int s = ns[e], i = s / Z1, j = s - i * Z1;
        const int at = atomicAdd(&cur[(i / bh) * nb1 + j / bw], 1);
        list[at] = make_int4(nk[e], i, j, __float_as_int(nzv[e]));
    }
}

template <int NT, int KMAX>
__global__ void __launch_bounds__(NT) gather_beta_kernel(GatherArgs a) {
    if (a.h->overflow) return;
    __shared__ int4 snz[kGatherStage];
    const int r0 = blockIdx.y * a.bh, c0 = blockIdx.x * a.bw;
    const int tr = threadIdx.x / a.bw;
    const int i = r0 + tr, j = c0 + (threadIdx.x - tr * a.bw);
    const bool live = tr < a.bh && i < a.Z0 && j < a.Z1;
    const long long plane = (long long)a.Z0 * a.Z1;
    const long long at = (long long)i * a.Z1 + j;
    // ||D_k||^2 and its inverse in FP32, rounded as the LGCD worker rounds
    // them, once per CTA (an FP64 division per position and atom would make
    // the FP64 pipe the kernel's bound)
    __shared__ float s_nk[KMAX], s_ik[KMAX];
    if (threadIdx.x < a.K && threadIdx.x < KMAX) {
        const double nk = a.nrm[threadIdx.x];
        s_nk[threadIdx.x] = (float)nk;
        s_ik[threadIdx.x] = (float)(1.0 / nk);
    }
    float acc[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; k++) acc[k] = (live && k < a.K) ? __ldcs(a.beta0 + k * plane + at) : 0.f;
    // the nonzeros of Z at this position, seen among the staged ones (up to two)
    int zk0 = -1, zk1 = -1;
    float zv0 = 0.f, zv1 = 0.f;
    bool zmany = false;
    // bins within L_i - 1 of the tile; the bins of one bin row are contiguous
    // in the list.  Up to 32 bin rows at a time: their ranges are read in one
    // go, then every staged nonzero in one pass.
    __shared__ int s_beg[32], s_pre[33];
    const int hr0 = max(0, r0 - (a.L0 - 1)), hr1 = min(a.Z0 - 1, r0 + a.bh - 1 + a.L0 - 1);
    const int hc0 = max(0, c0 - (a.L1 - 1)), hc1 = min(a.Z1 - 1, c0 + a.bw - 1 + a.L1 - 1);
    const int bc0 = hc0 / a.bw, bc1 = hc1 / a.bw;
    for (int brg = hr0 / a.bh; brg <= hr1 / a.bh; brg += 32) {
        const int nbr = min(32, hr1 / a.bh - brg + 1);
        __syncthreads();
        if (threadIdx.x < nbr) {
            const int br = brg + threadIdx.x;
            const int beg = __ldcg(a.off + br * a.nb1 + bc0), end = __ldcg(a.off + br * a.nb1 + bc1 + 1);
            s_beg[threadIdx.x] = beg;
            s_pre[threadIdx.x + 1] = end - beg;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_pre[0] = 0;
            for (int r = 1; r <= nbr; r++) s_pre[r] += s_pre[r - 1];
        }
        __syncthreads();
        const int total = s_pre[nbr];
        for (int base = 0; base < total; base += kGatherStage) {
            const int n = min(kGatherStage, total - base);
            if (base > 0) __syncthreads();
            for (int q = threadIdx.x; q < n; q += NT) {
                int r = 0;
                while (s_pre[r + 1] <= base + q) r++;
                snz[q] = __ldcg(a.list + s_beg[r] + (base + q - s_pre[r]));
            }
            __syncthreads();
            if (!live) continue;
            for (int q = 0; q < n; q++) {
                const int4 e = snz[q];
                const int di = i - e.y, dj = j - e.z;
                if (di <= -a.L0 || di >= a.L0 || dj <= -a.L1 || dj >= a.L1) continue;
                const float z = __int_as_float(e.w);
                // C_t[k'][delta][0..K): the K coefficients of the term, contiguous
                const float4 *row = reinterpret_cast<const float4 *>(
                    a.ct + ((size_t)(e.x * a.W0 + di + a.L0 - 1) * a.W1 + dj + a.L1 - 1) * a.Kp);
                // the term of (k, s) itself is left out; its z is Z at this position
                const int self = (di == 0 && dj == 0) ? e.x : -1;
                if (self >= 0) {
                    if (zk0 < 0) zk0 = self, zv0 = z;
                    else if (zk1 < 0) zk1 = self, zv1 = z;
                    else zmany = true;
                }
#pragma unroll
                for (int g = 0; g < KMAX / 4; g++) {
                    if (4 * g >= a.K) break;
                    const float4 c = __ldg(row + g);
                    const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                    for (int u = 0; u < 4; u++)
                        if (4 * g + u != self) acc[4 * g + u] -= cv[u] * z;
                }
            }
        }
    }
    unsigned long long m = 0;
    __syncthreads();  // s_nk, s_ik
    if (live) {
#pragma unroll
        for (int k = 0; k < KMAX; k++) {
            if (k >= a.K) break;
            a.beta[k * plane + at] = acc[k];
            // Z here: from the staged nonzeros (a position with more than two
            // nonzero atoms reads Z itself)
            const float zk = zmany ? __ldcs(a.Z + k * plane + at) : (k == zk0 ? zv0 : (k == zk1 ? zv1 : 0.f));
            float dz = coord_update(acc[k], a.lambda, s_nk[k], s_ik[k]) - zk;
            dz = dz < 0.f ? -dz : dz;
            const unsigned long long b = nonneg_bits(dz);
            m = b > m ? b : m;
        }
    }
    block_max_atomic<NT>(m, a.bits);
}

template <typename real>
int launch_refresh(const Geom &g, const WsLayout &L, unsigned char *ws, const real *X,
                   const real *D, const real *Z, real lambda, real *beta, cudaStream_t st,
                   const real *dtd) {
    WsHeader *h = reinterpret_cast<WsHeader *>(ws + L.hdr);
    int *nk = reinterpret_cast<int *>(ws + L.nnz_k);
    int *ns = reinterpret_cast<int *>(ws + L.nnz_s);
    real *nzv = reinterpret_cast<real *>(ws + L.nnz_z);
    double *R = reinterpret_cast<double *>(ws + L.r64);
    real *Rr = reinterpret_cast<real *>(ws + L.rr);
    const double *nrm = reinterpret_cast<const double *>(ws + L.nrm);
    const long long nx = g.nx(), nz = g.nz();

    refresh_reset_kernel<<<1, 1, 0, st>>>(h);
    bool v4 = false;
    if constexpr (sizeof(real) == 4) v4 = (reinterpret_cast<uintptr_t>(Z) & 15) == 0;
    if (v4) {
        if constexpr (sizeof(real) == 4)
            compact_v4_kernel<256><<<grid_for((nz + 3) / 4, 256), 256, 0, st>>>(Z, g.nzpos(), g.K, nk, ns, nzv,
                                                                                 L.nnz_cap, h);
    } else {
        compact_any_kernel<real, 256><<<grid_for(nz, 256), 256, 0, st>>>(Z, g.nzpos(), g.K, nk, ns, nzv,
                                                                          L.nnz_cap, h);
    }
    residual_init_kernel<real><<<grid_for(nx, 256), 256, 0, st>>>(X, R, nx);
    scatter_kernel<real, 128><<<152 * 8, 128, 0, st>>>(nk, ns, nzv, h, L.nnz_cap, D, R, g.P, g.L0,
                                                       g.L1, g.T0, g.T1, g.Z1);
    recon_dense_kernel<real><<<grid_for(nx, 256), 256, 0, st>>>(X, Z, D, h, R, g.P, g.K, g.T0, g.T1,
                                                                g.L0, g.L1, g.Z0, g.Z1);
    const bool from_beta0 = beta && dtd;
    // the FP32 residual feeds the correlation, which the beta0 form needs only
    // after an overflow (the residual is then the dense one either way)
    residual_finish_kernel<real, 256><<<grid_for(nx, 256), 256, 0, st>>>(R, beta ? Rr : nullptr, nx,
                                                                         &h->obj_f);
    CSC_CUDA(cudaGetLastError());
    if (!beta) return CSC_OK;
    if constexpr (sizeof(real) == 4) {
        if (from_beta0) {
            const float *b0 = reinterpret_cast<const float *>(ws + L.beta0);
            const long long plane = g.nzpos();
            if (g.K <= 32) {
                const int nbins = L.gnb0 * L.gnb1;
                int *cnt = reinterpret_cast<int *>(ws + L.gbin), *cur = cnt + nbins + 1;
                int4 *list = reinterpret_cast<int4 *>(ws + L.glist);
                float *ct = reinterpret_cast<float *>(ws + L.gtab);
                const int W = g.W0 * g.W1;
                ctab_kernel<<<grid_for((long long)g.K * W * L.gkp, 256), 256, 0, st>>>(dtd, ct, g.K, L.gkp, W);
                CSC_CUDA(cudaMemsetAsync(cnt, 0, (size_t)nbins * sizeof(int), st));
                bin_count_kernel<<<grid_for(L.nnz_cap, 256), 256, 0, st>>>(ns, h, L.nnz_cap, cnt, g.Z1, L.gbh,
                                                                           L.gbw, L.gnb1);
                bin_scan_kernel<1024><<<1, 1024, 0, st>>>(cnt, cnt, cur, nbins, h);
                bin_fill_kernel<<<grid_for(L.nnz_cap, 256), 256, 0, st>>>(nk, ns, nzv, h, L.nnz_cap, cur, list, g.Z1,
                                                                          L.gbh, L.gbw, L.gnb1);
                GatherArgs ga{b0, Z, ct, beta, cnt, list, nrm, h, &h->maxdz_bits, lambda, g.K, L.gkp, g.Z0, g.Z1,
                              g.L0, g.L1, g.W0, g.W1, L.gbh, L.gbw, L.gnb0, L.gnb1};
                const int nt = L.gbh * L.gbw;  // 512 threads, one per position of the tile
                gather_beta_kernel<512, 32><<<dim3((unsigned)L.gnb1, (unsigned)L.gnb0), nt, 0, st>>>(ga);
            } else {
                copy_beta0_kernel<256><<<grid_for(nz / 4 + 1, 256), 256, 0, st>>>(b0, beta, nz, h);
                LgcdArgs<float> a{};
                a.beta = beta;
                a.Z = const_cast<float *>(Z);
                a.dtd = dtd;
                a.K = g.K;
                a.Z0 = g.Z0;
                a.Z1 = g.Z1;
                a.L0 = g.L0;
                a.L1 = g.L1;
                a.W0 = g.W0;
                a.W1 = g.W1;
                nz_window_kernel<256><<<152 * 8, 256, 0, st>>>(a, nk, ns, nzv, h, L.nnz_cap);
                dim3 grid((unsigned)std::min<long long>(ceil_div(plane, 4 * 256), std::max(1, 152 * 8 / g.K)),
                          (unsigned)g.K);
                maxdz_kernel<256><<<grid, 256, 0, st>>>(beta, Z, nrm, lambda, plane, h, &h->maxdz_bits);
            }
            CSC_CUDA(cudaGetLastError());
            // overflow: the correlation of the (dense) residual instead
            return launch_corr_refresh<real>(g, Rr, D, Z, nrm, lambda, beta, &h->maxdz_bits, st, &h->overflow);
        }
    }
    return launch_corr_refresh<real>(g, Rr, D, Z, nrm, lambda, beta, &h->maxdz_bits, st);
}

int preload_residual_kernels() {
    const void *fns[] = {
        (const void *)refresh_reset_kernel,
        (const void *)compact_any_kernel<float, 256>,
        (const void *)compact_v4_kernel<256>,
        (const void *)residual_init_kernel<float>,
        (const void *)scatter_kernel<float, 128>,
        (const void *)recon_dense_kernel<float>,
        (const void *)residual_finish_kernel<float, 256>,
        (const void *)copy_beta0_kernel<256>,
        (const void *)ctab_kernel,
        (const void *)bin_count_kernel,
        (const void *)bin_scan_kernel<1024>,
        (const void *)bin_fill_kernel,
        (const void *)gather_beta_kernel<512, 32>,
        (const void *)nz_window_kernel<256>,
        (const void *)maxdz_kernel<256>,
    };
    return preload_functions(fns, (int)(sizeof(fns) / sizeof(fns[0])));
}

template int launch_refresh<float>(const Geom &, const WsLayout &, unsigned char *, const float *,
                                   const float *, const float *, float, float *, cudaStream_t, const float *);
template int launch_refresh<double>(const Geom &, const WsLayout &, unsigned char *, const double *,
                                    const double *, const double *, double, double *, cudaStream_t,
                                    const double *);

}  // namespace csc
