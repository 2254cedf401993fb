// dict.cu -- dictionary update of Section 4.2 / Alg. 2.
//
// Statistics from the sparse Z:
//   psi_kp[tau]      = sum_s Z_k[s] X_p[s + tau]          (tau in Theta)
//   phi_{k,k2}[d]    = sum_s Z_k[s] Z_k2[s + d]           (Eq. phi, d in Phi)
// The nonzeros are compacted deterministically in (position, atom) order.
// psi is accumulated per CTA in shared memory over a chunk of nonzeros and
// flushed with FP64 atomics; phi enumerates, for each nonzero, the other
// nonzeros inside its window by binary search in the position-sorted list,
// so its cost is the number of interacting pairs, not K |Phi| per nonzero.
//
// Dictionary step: projected gradient descent with Armijo backtracking on
// one thread-block cluster (up to 16 CTAs).  Each CTA owns a slice of the
// entries of D; cluster barriers separate the phases and partial sums are
// combined through distributed shared memory.  The Armijo condition
//   F(D+) <= F(D) + <grad, D+ - D> + ||D+ - D||^2 / (2 eta)
// is evaluated in the algebraically equal form
//   <D+ - D, phi * (D+ - D)> eta <= ||D+ - D||^2,
// which holds exactly for the quadratic F of Eq. dict_update and avoids the
// cancellation of subtracting two nearly equal objective values in FP32.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "dict.cuh"

namespace cg = cooperative_groups;

namespace csc {

// ------------------------------------------------ deterministic compaction
// Pass 1: nonzeros per block of positions.
template <int NT>
__global__ void __launch_bounds__(NT) nz_count_kernel(const float *Z, long long zpos, int K,
                                                      int *blk_cnt) {
    long long s = (long long)blockIdx.x * NT + threadIdx.x;
    int c = 0;
    if (s < zpos)
        for (int k = 0; k < K; k++) c += Z[(size_t)k * zpos + s] != 0.f;
    __shared__ int red[NT / 32];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < NT / 32; w++) t += red[w];
        blk_cnt[blockIdx.x] = t;
    }
}

// Pass 2: exclusive scan of the block counts (one CTA).
template <int NT>
__global__ void __launch_bounds__(NT) nz_scan_kernel(const int *blk_cnt, int *blk_off, int nblk,
                                                     WsHeader *h) {
    __shared__ int warp_tot[NT / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblk; base += NT) {
        int i = base + threadIdx.x;
        int v = i < nblk ? blk_cnt[i] : 0;
        int x = v;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        int woff = 0;
        for (int w = 0; w < wid; w++) woff += warp_tot[w];
        if (i < nblk) blk_off[i] = carry + woff + x - v;
        __syncthreads();
        if (threadIdx.x == NT - 1) carry += woff + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) h->scan_total = carry;
}

// Pass 3: write (k, s, z) in (position, atom) order.
template <int NT>
__global__ void __launch_bounds__(NT) nz_write_kernel(const float *Z, long long zpos, int K,
                                                      const int *blk_off, const WsHeader *h,
                                                      long long cap, int *nk, int *ns, float *nzv) {
    if (h->scan_total > cap) return;
    long long s = (long long)blockIdx.x * NT + threadIdx.x;
    int c = 0;
    if (s < zpos)
        for (int k = 0; k < K; k++) c += Z[(size_t)k * zpos + s] != 0.f;
    __shared__ int warp_tot[NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = c;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    int off = blk_off[blockIdx.x];
    for (int w = 0; w < wid; w++) off += warp_tot[w];
    off += x - c;
    if (s < zpos)
        for (int k = 0; k < K; k++) {
            float v = Z[(size_t)k * zpos + s];
            if (v != 0.f) {
                nk[off] = k;
                ns[off] = (int)s;
                nzv[off] = v;
                off++;
            }
        }
}

// psi: a CTA takes a chunk of nonzeros (staged in shared memory as atom,
// row, column, value); thread e owns entry (p, tau) of every atom in shared
// memory, so no two threads touch the same word, and keeps eight X loads in
// flight per pass over the chunk.
constexpr int kPsiChunk = 64;

template <int NT>
__global__ void __launch_bounds__(NT) psi_kernel(const int *nk, const int *ns, const float *nzv,
                                                 const WsHeader *h, int cap, const float *X, double *psi64,
                                                 int P, int K, int T0, int T1, int L0, int L1, int Z1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *acc = reinterpret_cast<float *>(smem_raw);
    __shared__ int c_k[kPsiChunk], c_off[kPsiChunk];
    __shared__ float c_z[kPsiChunk];
    const int LL = L0 * L1, per = P * LL;
    const int cnt = h->scan_total;  // a count above cap: the list was not written
    const int lo = blockIdx.x * kPsiChunk, n = min(cnt, lo + kPsiChunk) - lo;
    if (n <= 0 || cnt > cap) return;
    for (int q = threadIdx.x; q < K * per; q += NT) acc[q] = 0.f;
    for (int q = threadIdx.x; q < n; q += NT) {
        const int s = ns[lo + q], i = s / Z1;
        c_k[q] = nk[lo + q];
        c_off[q] = i * T1 + (s - i * Z1);  // X offset of the window's corner
        c_z[q] = nzv[lo + q];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < per; e += NT) {
        const int p = e / LL, r = e - p * LL, d0 = r / L1, d1 = r - d0 * L1;
        const float *xp = X + (size_t)p * T0 * T1 + (size_t)d0 * T1 + d1;
        for (int n0 = 0; n0 < n; n0 += 8) {
            float xv[8];
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (n0 + u < n) xv[u] = __ldg(xp + c_off[n0 + u]);
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (n0 + u < n) acc[c_k[n0 + u] * per + e] += c_z[n0 + u] * xv[u];
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < K * per; q += NT)
        if (acc[q] != 0.f) atomicAdd(&psi64[q], (double)acc[q]);
}

// phi by pair enumeration over the position-sorted nonzeros.
__device__ __forceinline__ int lower_bound_pos(const int *ns, int n, int key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (ns[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void phi_pairs_kernel(const int *nk, const int *ns, const float *nzv, const WsHeader *h, int cap,
                                 double *phi64, int K, int L0, int L1, int Z0, int Z1) {
    const int cnt = h->scan_total;
    if (cnt > cap) return;  // the list was not written
    const int W0 = 2 * L0 - 1, W1 = 2 * L1 - 1;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < cnt; n += gridDim.x * blockDim.x) {
        const int k = nk[n], s = ns[n];
        const double z = (double)nzv[n];
        const int i = s / Z1, j = s % Z1;
        for (int d0 = -L0 + 1; d0 < L0; d0++) {
            const int i2 = i + d0;
            if (i2 < 0 || i2 >= Z0) continue;
            const int jlo = max(0, j - L1 + 1), jhi = min(Z1 - 1, j + L1 - 1);
            int m = lower_bound_pos(ns, cnt, i2 * Z1 + jlo);
            const int end_key = i2 * Z1 + jhi;
            for (; m < cnt && ns[m] <= end_key; m++) {
                const int d1 = ns[m] % Z1 - j;
                atomicAdd(&phi64[(((size_t)k * K + nk[m]) * W0 + d0 + L0 - 1) * W1 + d1 + L1 - 1],
                          z * (double)nzv[m]);
            }
        }
    }
}

__global__ void to_float_kernel(const double *src, float *dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// count_on_host: read the nonzero count back (one synchronisation) to size the
// phi / psi grids and report an overflow at once; otherwise the grids cover
// the list capacity, the kernels read the count from the workspace header, and
// the caller checks it against the capacity after a later synchronisation.
static int stats_launch(const Geom &g, const float *Z, const float *X, float *phi, float *psi,
                        unsigned char *ws, const WsLayout &L, cudaStream_t st, bool count_on_host) {
    WsHeader *h = reinterpret_cast<WsHeader *>(ws + L.hdr);
    int *nk = reinterpret_cast<int *>(ws + L.nnz_k);
    int *ns = reinterpret_cast<int *>(ws + L.nnz_s);
    float *nzv = reinterpret_cast<float *>(ws + L.nnz_z);
    int *blk_cnt = reinterpret_cast<int *>(ws + L.blk);
    int *blk_off = blk_cnt + L.blk_cap;
    double *phi64 = reinterpret_cast<double *>(ws + L.phi64);
    double *psi64 = reinterpret_cast<double *>(ws + L.psi64);
    const long long zpos = g.nzpos();
    const int nblk = (int)ceil_div(zpos, 256);
    if (nblk > L.blk_cap) return CSC_ERR_WORKSPACE;
    const int cap = (int)L.nnz_cap;

    nz_count_kernel<256><<<nblk, 256, 0, st>>>(Z, zpos, g.K, blk_cnt);
    nz_scan_kernel<1024><<<1, 1024, 0, st>>>(blk_cnt, blk_off, nblk, h);
    long long total = cap;  // grid coverage
    if (count_on_host) {
        int t = 0;
        const int rb_ = read_back(&t, &h->scan_total, st);
        if (rb_) return rb_;
        if (t > cap) return CSC_ERR_WORKSPACE;
        total = t;
    }
    nz_write_kernel<256><<<nblk, 256, 0, st>>>(Z, zpos, g.K, blk_off, h, cap, nk, ns, nzv);
    CSC_CUDA(cudaMemsetAsync(phi64, 0, (size_t)g.ntab() * sizeof(double), st));
    CSC_CUDA(cudaMemsetAsync(psi64, 0, (size_t)g.nd() * sizeof(double), st));
    if (total > 0) {
        const int chunk = kPsiChunk;
        size_t smem = (size_t)g.nd() * sizeof(float);
        if (smem > 227 * 1024) return CSC_ERR_UNIMPLEMENTED;
        if (smem > 48 * 1024)
            CSC_CUDA(cudaFuncSetAttribute(psi_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        psi_kernel<256><<<(int)ceil_div(total, chunk), 256, smem, st>>>(
            nk, ns, nzv, h, cap, X, psi64, g.P, g.K, g.T0, g.T1, g.L0, g.L1, g.Z1);
        phi_pairs_kernel<<<(int)ceil_div(total, 128), 128, 0, st>>>(nk, ns, nzv, h, cap, phi64, g.K, g.L0,
                                                                    g.L1, g.Z0, g.Z1);
    }
    to_float_kernel<<<(int)std::min<long long>(ceil_div(g.ntab(), 256), 4096), 256, 0, st>>>(
        phi64, phi, g.ntab());
    to_float_kernel<<<(int)std::min<long long>(ceil_div(g.nd(), 256), 4096), 256, 0, st>>>(
        psi64, psi, g.nd());
    CSC_CUDA(cudaGetLastError());
    return CSC_OK;
}

int dict_stats_impl(const Geom &g, const float *Z, const float *X, float *phi, float *psi,
                    unsigned char *ws, const WsLayout &L, cudaStream_t st) {
    return stats_launch(g, Z, X, phi, psi, ws, L, st, true);
}

int sparse_code_impl(const Geom &g, const float *Z, int *k_out, int *s_out, float *val_out, long long cap,
                     long long *nnz_out, unsigned char *ws, const WsLayout &L, cudaStream_t st) {
    WsHeader *h = reinterpret_cast<WsHeader *>(ws + L.hdr);
    int *blk_cnt = reinterpret_cast<int *>(ws + L.blk);
    int *blk_off = blk_cnt + L.blk_cap;
    const long long zpos = g.nzpos();
    const int nblk = (int)ceil_div(zpos, 256);
    if (nblk > L.blk_cap) return CSC_ERR_WORKSPACE;
    nz_count_kernel<256><<<nblk, 256, 0, st>>>(Z, zpos, g.K, blk_cnt);
    nz_scan_kernel<1024><<<1, 1024, 0, st>>>(blk_cnt, blk_off, nblk, h);
    CSC_CUDA(cudaGetLastError());
    int t = 0;
    const int rb_ = read_back(&t, &h->scan_total, st);
    if (rb_) return rb_;
    *nnz_out = t;
    if (t > cap) return CSC_ERR_WORKSPACE;
    if (t > 0) {
        nz_write_kernel<256><<<nblk, 256, 0, st>>>(Z, zpos, g.K, blk_off, h, cap, k_out, s_out, val_out);
        CSC_CUDA(cudaGetLastError());
    }
    return CSC_OK;
}

int dict_stats_deferred(const Geom &g, const float *Z, const float *X, float *phi, float *psi,
                        unsigned char *ws, const WsLayout &L, cudaStream_t st) {
    return stats_launch(g, Z, X, phi, psi, ws, L, st, false);
}

// ====================================================== PGD + Armijo step
// The data-fit term F(D) = 1/2||X||^2 - <psi, D> + 1/2 <D, phi * D> is
// quadratic, so a projected step from D with step eta,
//   D+_k = s_k (D_k - eta G_k),  s_k = 1 / max(1, ||D_k - eta G_k||),
// moves every atom inside span{D_k, G_k}: D+ - D = sum_k (alpha_k D_k +
// beta_k G_k) restricted to atom k, alpha_k = s_k - 1, beta_k = -s_k eta.
// With the per-atom scalars a_k = ||D_k||^2, b_k = <D_k, G_k>, c_k = ||G_k||^2
// and the K x K matrices M_XY[k][k2] = <X_k, phi * Y_k2> (X, Y in {D, G};
// M_GD[k][k2] = M_DG[k2][k] because the operator is self-adjoint):
//   ||D+ - D||^2            = sum_k alpha_k^2 a_k + 2 alpha_k beta_k b_k + beta_k^2 c_k
//   <D+ - D, phi*(D+ - D)>  = sum_{k,k2} alpha_k alpha_k2 M_DD + alpha_k beta_k2 M_DG
//                             + beta_k alpha_k2 M_DG[k2][k] + beta_k beta_k2 M_GG.
// Every Armijo trial (condition <D+ - D, phi * (D+ - D)> eta <= ||D+ - D||^2,
// the exact form of F(D+) <= F(D) + <G, D+ - D> + ||D+ - D||^2 / (2 eta)
// for this quadratic F) is therefore O(K^2) scalar work.  One iteration
// needs a single convolution: with QX_k2 = phi * (X restricted to atom k2)
// kept per source atom, the accepted step gives G+ = G + sum_k2 (alpha_k2
// QD_k2 + beta_k2 QG_k2) and QD+_k2 = s_k2 (QD_k2 - eta QG_k2) linearly,
// and only QG+ is convolved again.
//
// Layout: one thread-block cluster, CTA r owns atoms [r ka, (r+1) ka).  Its
// D and G slices live in shared memory, its per-source convolutions QD/QG in
// shared memory when they fit (else global scratch).  Every CTA also holds
// the full G and every atom's scalars / Gram rows: their owners write them
// into each CTA's shared memory (distributed shared memory stores) before a
// cluster barrier, so after the barrier they are read locally (two cluster
// barriers per iteration).
struct PgdArgs {
    const float *phi, *psi;
    float *D;      // in/out
    float *qd, *qg;  // per-CTA scratch: [cluster rank][K sources][ka * per]
    double *out;   // [objective, iterations, eta, Armijo trials, phase cycles x 6]
    double x_sqnorm, tol;
    const double *x_sqnorm_dev;  // when set, ||X||^2 is read here instead of x_sqnorm
    const int *gate;             // when set and *gate > gate_cap, D is left unchanged
    int gate_cap;
    int K, P, L0, L1, max_iter, ka, stage_phi, q_in_smem;
};

constexpr int kPgdThreads = 512;
constexpr int kPgdWarps = kPgdThreads / 32;
constexpr int kPgdMaxK = 32;
constexpr int kPgdTrialWarps = 4;  // Armijo trials evaluated at once
constexpr int kPgdMaxCluster = 16;  // CTAs of the cluster, at most
constexpr float kPgdMinTol = 4.0f / 16777216.0f;  // 4 x 2^-24

// Block-wide sum returned to every thread (warp 0 combines the warp sums).
__device__ __forceinline__ double block_reduce_sum(double v, double *scratch) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = warp_sum(threadIdx.x < kPgdWarps ? scratch[threadIdx.x] : 0.0);
        if (threadIdx.x == 0) scratch[kPgdWarps] = s;
    }
    __syncthreads();
    return scratch[kPgdWarps];
}

// One group of NP channels of conv_per_source: lane positions o0 and o1
// (valid when v0 / v1), phi row ph of the (k, k2) pair, source rows sv.
// NP is a template argument so that no FMA of an absent channel is issued.
template <int NP>
__device__ __forceinline__ void conv_channels(const float *__restrict__ ph, const float *__restrict__ sv, int LL,
                                              int L0, int L1, int W1, int base0, int base1, bool v0, bool v1,
                                              float *__restrict__ dst, int o0, int o1) {
    float acc0[NP], acc1[NP];
#pragma unroll
    for (int j = 0; j < NP; j++) acc0[j] = acc1[j] = 0.f;
    for (int a2 = 0; a2 < L0; a2++) {
        const float *__restrict__ srow = sv + a2 * L1;
        const int off = a2 * W1;
        int b2 = 0;
        if ((LL & 3) == 0 && (L1 & 3) == 0) {
            // four taps at a time: the source values of every channel as one
            // 16-byte load each, the eight phi values, then the products; two
            // groups in flight (up to five channels, within the register cap) so
            // that the loads of one overlap the other's FMAs
#pragma unroll(NP <= 5 ? 2 : 1)
            for (; b2 < L1; b2 += 4) {
                float f0[4], f1[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    f0[u] = v0 ? ph[base0 - off - b2 - u] : 0.f;
                    f1[u] = v1 ? ph[base1 - off - b2 - u] : 0.f;
                }
#pragma unroll
                for (int j = 0; j < NP; j++) {
                    const float4 g = *reinterpret_cast<const float4 *>(srow + (size_t)j * LL + b2);
                    acc0[j] = fmaf(f0[0], g.x, acc0[j]);
                    acc1[j] = fmaf(f1[0], g.x, acc1[j]);
                    acc0[j] = fmaf(f0[1], g.y, acc0[j]);
                    acc1[j] = fmaf(f1[1], g.y, acc1[j]);
                    acc0[j] = fmaf(f0[2], g.z, acc0[j]);
                    acc1[j] = fmaf(f1[2], g.z, acc1[j]);
                    acc0[j] = fmaf(f0[3], g.w, acc0[j]);
                    acc1[j] = fmaf(f1[3], g.w, acc1[j]);
                }
            }
        }
#pragma unroll 4
        for (; b2 < L1; b2++) {
            const float f0 = v0 ? ph[base0 - off - b2] : 0.f;
            const float f1 = v1 ? ph[base1 - off - b2] : 0.f;
#pragma unroll
            for (int j = 0; j < NP; j++) {
                const float g = srow[(size_t)j * LL + b2];
                acc0[j] = fmaf(f0, g, acc0[j]);
                acc1[j] = fmaf(f1, g, acc1[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NP; j++) {
        if (v0) dst[(size_t)j * LL + o0] = acc0[j];
        if (v1) dst[(size_t)j * LL + o1] = acc1[j];
    }
}

// out[k2][e] = sum_tau2 phi_{k,k2}[tau - tau2] src[k2][p][tau2] for the own
// output entries e = (kl, p, tau) of this CTA and every source atom k2
// (per-source stride own_cap).  One warp per (k2, kl, chunk of 64 positions
// of the L0 x L1 plane); each lane keeps two positions (o, o + 32) for up to
// eight channels, so one phi value serves every channel and one source value
// (a broadcast) serves two positions.
__device__ __forceinline__ void conv_per_source(const PgdArgs &a, const float *sphi, int k_lo, int nk,
                                                const float *src, float *out, int own_cap) {
    const int LL = a.L0 * a.L1, per = a.P * LL;
    const int W1 = 2 * a.L1 - 1, WW = (2 * a.L0 - 1) * W1;
    const int chunks = (LL + 63) / 64;
    const int items = a.K * nk * chunks;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int it = warp; it < items; it += kPgdWarps) {
        const int k2 = it / (nk * chunks), rem = it - k2 * (nk * chunks);
        const int kl = rem / chunks, ch = rem - kl * chunks;
        const float *__restrict__ ph =
            (a.stage_phi ? sphi + (size_t)kl * a.K * WW : a.phi + (size_t)(k_lo + kl) * a.K * WW) + (size_t)k2 * WW;
        const float *__restrict__ sv = src + (size_t)k2 * per;
        const int o0 = ch * 64 + lane, o1 = o0 + 32;
        const bool v0 = o0 < LL, v1 = o1 < LL;
        // phi index of position (ta, tb) and tap (a2, b2): base(ta, tb) - (a2 W1 + b2)
        const int base0 = v0 ? (o0 / a.L1 + a.L0 - 1) * W1 + o0 % a.L1 + a.L1 - 1 : 0;
        const int base1 = v1 ? (o1 / a.L1 + a.L0 - 1) * W1 + o1 % a.L1 + a.L1 - 1 : 0;
        float *__restrict__ dst = out + (size_t)k2 * own_cap + (size_t)kl * per;
        for (int pc = 0; pc < a.P; pc += 8) {
            const float *s = sv + (size_t)pc * LL;
            float *d = dst + (size_t)pc * LL;
#define PGD_CONV(NP) conv_channels<NP>(ph, s, LL, a.L0, a.L1, W1, base0, base1, v0, v1, d, o0, o1)
            switch (min(8, a.P - pc)) {
                case 1: PGD_CONV(1); break;
                case 2: PGD_CONV(2); break;
                case 3: PGD_CONV(3); break;
                case 4: PGD_CONV(4); break;
                case 5: PGD_CONV(5); break;
                case 6: PGD_CONV(6); break;
                case 7: PGD_CONV(7); break;
                default: PGD_CONV(8); break;
            }
#undef PGD_CONV
        }
    }
}

__global__ void __launch_bounds__(kPgdThreads, 1) pgd_kernel(PgdArgs a) {
    // statistics that were not computed (their nonzero list overflowed): every
    // CTA of the cluster returns before any barrier, D is left as it is
    if (a.gate && *a.gate > a.gate_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.out[0] = 0.0;
            a.out[1] = 0.0;
        }
        return;
    }
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = a.K, LL = a.L0 * a.L1, per = a.P * LL, n = K * per;
    const int WW = (2 * a.L0 - 1) * (2 * a.L1 - 1);
    const int rank = (int)cl.block_rank(), ncl = (int)cl.num_blocks();
    const int k_lo = min(K, rank * a.ka), k_hi = min(K, k_lo + a.ka);
    const int nk = k_hi - k_lo, nown = nk * per, e0 = k_lo * per;
    const int own_cap = a.ka * per;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // dynamic shared memory; every CTA holds the full G (the static arrays
    // below hold every atom's scalars and Gram rows, written by their owners
    // before a cluster barrier)
    float *gall = reinterpret_cast<float *>(smem_raw);
    float *sD = gall + n, *sG = sD + own_cap;
    float *sphi = sG + own_cap;
    float *qsm = sphi + (a.stage_phi ? (size_t)a.ka * K * WW : 0);
    float *qd = a.q_in_smem ? qsm : a.qd + (size_t)rank * K * own_cap;
    float *qg = a.q_in_smem ? qsm + (size_t)K * own_cap : a.qg + (size_t)rank * K * own_cap;

    __shared__ double scratch[kPgdWarps + 1];
    __shared__ float s_alpha[kPgdMaxK], s_beta[kPgdMaxK], s_scale[kPgdMaxK];
    __shared__ float fsa[kPgdMaxK], fsa1[kPgdMaxK], fsb[kPgdMaxK], fsc[kPgdMaxK];
    __shared__ float fMDD[kPgdMaxK * kPgdMaxK], fMDG[kPgdMaxK * kPgdMaxK], fMGG[kPgdMaxK * kPgdMaxK];
    __shared__ double s_ctl[4];  // eta, dsq, dnorm, stop
    __shared__ int s_pass[2][kPgdTrialWarps];  // Armijo test per trial, by round parity
    __shared__ float s_ta[kPgdTrialWarps][kPgdMaxK], s_tb[kPgdTrialWarps][kPgdMaxK];  // per-trial alpha, beta
    __shared__ double s_lip;

    // stage own slices and phi rows; the full D is the first convolution input
    for (int e = threadIdx.x; e < nown; e += kPgdThreads) sD[e] = a.D[e0 + e];
    for (int e = threadIdx.x; e < n; e += kPgdThreads) gall[e] = a.D[e];
    if (a.stage_phi)
        for (size_t e = threadIdx.x; e < (size_t)nk * K * WW; e += kPgdThreads)
            sphi[e] = a.phi[(size_t)k_lo * K * WW + e];
    __syncthreads();
    // Lipschitz bound of the gradient: max_k sum_k2 sum_d |phi_{k,k2}[d]|
    double lip_loc = 0.0;
    for (int kl = 0; kl < nk; kl++) {
        double t = 0.0;
        for (size_t q = threadIdx.x; q < (size_t)K * WW; q += kPgdThreads)
            t += fabs((double)a.phi[(size_t)(k_lo + kl) * K * WW + q]);
        lip_loc = fmax(lip_loc, block_reduce_sum(t, scratch));
    }
    if (threadIdx.x == 0) s_lip = lip_loc;
    // QD = phi * D per source; G = sum_k2 QD_k2 - psi, written to every CTA's full G
    conv_per_source(a, sphi, k_lo, nk, gall, qd, own_cap);
    __syncthreads();
    cl.sync();  // every CTA has finished reading D from its full copy
    for (int e = threadIdx.x; e < nown; e += kPgdThreads) {
        float g = -a.psi[e0 + e];
        for (int k2 = 0; k2 < K; k2++) g += qd[(size_t)k2 * own_cap + e];
        sG[e] = g;
        for (int r = 0; r < ncl; r++) cl.map_shared_rank(gall, (unsigned)r)[e0 + e] = g;
    }
    cl.sync();
    double lip = 0.0;
    for (int r = 0; r < ncl; r++) lip = fmax(lip, *cl.map_shared_rank(&s_lip, (unsigned)r));

    // SM cycles per phase, kept by thread 0 in shared memory (no registers)
    __shared__ unsigned long long s_ph[6], s_tc;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 6; i++) s_ph[i] = 0;
        s_tc = clock64();
    }
#define PGD_TICK(i)                              \
    if (threadIdx.x == 0) {                      \
        const unsigned long long tn_ = clock64(); \
        s_ph[i] += tn_ - s_tc;                   \
        s_tc = tn_;                              \
    }
    // QG = phi * G per source, then the own atoms' scalars and Gram rows,
    // written to every CTA; after the barrier they are read locally
    auto refresh_stats = [&]() {
        conv_per_source(a, sphi, k_lo, nk, gall, qg, own_cap);
        __syncthreads();
        PGD_TICK(4)
        // warp w handles (own atom kl, item i) pairs: items 0..2 = the FP64
        // scalars ||D_k||^2, <D_k, G_k>, ||G_k||^2; items 3..K+2 = the Gram
        // entries of source k2 = i - 3.  Lanes 0 .. ncl-1 store the FP32 values
        // straight into one CTA each; the cluster barrier publishes them, and
        // no CTA reads them before its next Armijo step
        for (int q = warp; q < nk * (K + 3); q += kPgdWarps) {
            const int kl = q / (K + 3), i = q - kl * (K + 3);
            const int k = k_lo + kl;
            const float *d = sD + (size_t)kl * per, *g = sG + (size_t)kl * per;
            if (i < 3) {
                const float *x = i == 2 ? g : d, *y = i == 0 ? d : g;
                double acc = 0.0;
                for (int e = lane; e < per; e += 32) acc = fma((double)x[e], (double)y[e], acc);
                acc = warp_sum(acc);
                for (int r = lane; r < ncl; r += 32) {
                    if (i == 0) {
                        cl.map_shared_rank(fsa, (unsigned)r)[k] = (float)acc;
                        cl.map_shared_rank(fsa1, (unsigned)r)[k] = (float)(acc - 1.0);  // before rounding
                    } else {
                        cl.map_shared_rank(i == 1 ? fsb : fsc, (unsigned)r)[k] = (float)acc;
                    }
                }
            } else {
                const int k2 = i - 3;
                const float *qdr = qd + (size_t)k2 * own_cap + (size_t)kl * per;
                const float *qgr = qg + (size_t)k2 * own_cap + (size_t)kl * per;
                float dd = 0.f, dg = 0.f, gg = 0.f;
                for (int e = lane; e < per; e += 32) {
                    dd = fmaf(d[e], qdr[e], dd);
                    dg = fmaf(d[e], qgr[e], dg);
                    gg = fmaf(g[e], qgr[e], gg);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    dd += __shfl_xor_sync(0xffffffffu, dd, o);
                    dg += __shfl_xor_sync(0xffffffffu, dg, o);
                    gg += __shfl_xor_sync(0xffffffffu, gg, o);
                }
                for (int r = lane; r < ncl; r += 32) {
                    cl.map_shared_rank(fMDD, (unsigned)r)[k * K + k2] = dd;
                    cl.map_shared_rank(fMDG, (unsigned)r)[k * K + k2] = dg;
                    cl.map_shared_rank(fMGG, (unsigned)r)[k * K + k2] = gg;
                }
            }
        }
        cl.sync();
    };
    refresh_stats();

    double eta = lip > 0.0 ? 1.0 / lip : 0.0;
    int it = 0, n_trials = 0;
    if (lip > 0.0) {
        for (it = 0; it < a.max_iter; it++) {
            // Armijo backtracking by warp 0 on the per-atom scalars, in FP32:
            // with delta_k = ||D_k - eta G_k||^2 - 1 = (||D_k||^2 - 1)
            // - 2 eta <D_k, G_k> + eta^2 ||G_k||^2 (the first term taken from the
            // FP64 sum) and s_k = 1 / sqrt(1 + delta_k), the scale deviation
            // s_k - 1 = -delta_k s_k^2 / (1 + s_k) has no cancellation
            // Lane k holds atom k (K <= 32).  The backtracking trials
            // eta_t = eta_0 2^-t run kPgdTrialWarps at a time, trial t on warp
            // t mod kPgdTrialWarps, each with its own alpha / beta scratch; the
            // first trial that passes is taken, with the same arithmetic as if
            // they ran one after another.
            if (warp < kPgdTrialWarps) {
                const bool own = lane < K;
                const float ak = own ? fsa[lane] : 0.f, a1k = own ? fsa1[lane] : 0.f;
                const float bk = own ? fsb[lane] : 0.f, ck = own ? fsc[lane] : 0.f;
                const float e0 = it > 0 ? 2.0f * (float)eta : (float)eta;
                for (int t0 = 0;; t0 += kPgdTrialWarps) {
                    const int t = t0 + warp;
                    const float e_try = ldexpf(e0, -t);  // exact halvings
                    const float delta = a1k + e_try * (e_try * ck - 2.0f * bk);
                    float sk = 1.f, al = 0.f;
                    if (own && delta > 0.f) {
                        float r = rsqrtf(1.f + delta);
                        r = r * (1.5f - 0.5f * (1.f + delta) * r * r);  // one Newton step
                        sk = r;
                        al = -delta * r * r / (1.f + r);
                    }
                    const float be = own ? -sk * e_try : 0.f;
                    float ds = al * (al * ak + 2.f * be * bk) + be * be * ck;
                    float da = al * al * ak + fabsf(2.f * al * be * bk) + be * be * ck;  // |terms|
                    // <D+ - D, phi * (D+ - D)> from the Gram entries
                    float *ta = s_ta[warp], *tb = s_tb[warp];
                    if (own) {
                        ta[lane] = al;
                        tb[lane] = be;
                    }
                    __syncwarp();
                    float qf = 0.f;
                    for (int q = lane; q < K * K; q += 32) {
                        const int k = q / K, k2 = q - k * K;
                        const float alk = ta[k], bek = tb[k], al2 = ta[k2], be2 = tb[k2];
                        qf += alk * (al2 * fMDD[q] + be2 * fMDG[q]) + bek * (al2 * fMDG[k2 * K + k] + be2 * fMGG[q]);
                    }
                    for (int o = 16; o > 0; o >>= 1) {
                        qf += __shfl_xor_sync(0xffffffffu, qf, o);
                        ds += __shfl_xor_sync(0xffffffffu, ds, o);
                        da += __shfl_xor_sync(0xffffffffu, da, o);
                    }
                    const int par = (t0 / kPgdTrialWarps) & 1;
                    if (lane == 0) s_pass[par][warp] = (qf * e_try <= ds || t >= 59) ? 1 : 0;
                    asm volatile("bar.sync 2, %0;" ::"r"(kPgdTrialWarps * 32) : "memory");
                    int win = -1;
#pragma unroll
                    for (int w = kPgdTrialWarps - 1; w >= 0; w--)
                        if (s_pass[par][w]) win = w;
                    if (win < 0) continue;  // every trial of this round failed
                    if (threadIdx.x == 0) n_trials += t0 + win + 1;
                    if (warp == win) {
                        if (own) {
                            s_scale[lane] = sk;
                            s_alpha[lane] = al;
                            s_beta[lane] = be;
                        }
                        float dnorm = ak;
                        for (int o = 16; o > 0; o >>= 1) dnorm += __shfl_xor_sync(0xffffffffu, dnorm, o);
                        if (lane == 0) {
                            s_ctl[0] = e_try;
                            s_ctl[1] = ds;
                            s_ctl[2] = dnorm;
                            // stop when ||D+ - D|| < tol ||D|| (a relative change below
                            // the FP32 resolution of D is noise), or when the computed
                            // ||D+ - D||^2 lies within its own rounding bound, 2 gamma_{K+3}
                            // times the sum of its terms' magnitudes: near a solution with
                            // active norm constraints alpha_k D_k and beta_k G_k cancel, and
                            // below that level the FP32 scalars no longer resolve the change
                            // (the test that follows it would then take steps blindly)
                            const float tol = fmaxf((float)a.tol, kPgdMinTol);
                            const float floor_ds = 2.f * (float)(K + 3) * 5.96e-8f * da;
                            s_ctl[3] = (sqrtf(fmaxf(ds, 0.f)) < tol * sqrtf(dnorm) || ds <= floor_ds) ? 1.0 : 0.0;
                        }
                    }
                    break;
                }
            }
            __syncthreads();
            PGD_TICK(0)
            eta = s_ctl[0];
            const float feta = (float)eta;
            const bool stop = s_ctl[3] != 0.0;
            // accept: D+ = D + alpha D + beta G; G+ = G + sum_k2 (alpha QD + beta QG),
            // written to every CTA's full G; QD+ linear
            for (int e = threadIdx.x; e < nown; e += kPgdThreads) {
                const int k = k_lo + e / per;
                const float d = sD[e], g = sG[e];
                sD[e] = fmaf(s_beta[k], g, (1.0f + s_alpha[k]) * d);
                float gn = g;
                for (int k2 = 0; k2 < K; k2++) {
                    const size_t o = (size_t)k2 * own_cap + e;
                    const float qdv = qd[o], qgv = qg[o];
                    gn = fmaf(s_alpha[k2], qdv, fmaf(s_beta[k2], qgv, gn));
                    qd[o] = s_scale[k2] * fmaf(-feta, qgv, qdv);
                }
                sG[e] = gn;
                if (!stop)
                    for (int r = 0; r < ncl; r++) cl.map_shared_rank(gall, (unsigned)r)[e0 + e] = gn;
            }
            PGD_TICK(1)
            if (stop) {
                it++;
                break;
            }
            cl.sync();  // every CTA's full G is complete
            PGD_TICK(2)
            refresh_stats();
            PGD_TICK(5)
        }
    }
    __syncthreads();
    // F(D) = 1/2||X||^2 - 1/2 <psi, D> + 1/2 <D, G>; write D back
    double pdv = 0.0, dgv = 0.0;
    for (int e = threadIdx.x; e < nown; e += kPgdThreads) {
        pdv += (double)a.psi[e0 + e] * sD[e];
        dgv += (double)sD[e] * sG[e];
        a.D[e0 + e] = sD[e];
    }
    pdv = block_reduce_sum(pdv, scratch);
    dgv = block_reduce_sum(dgv, scratch);
    __shared__ double fin[2];
    if (threadIdx.x == 0) {
        fin[0] = pdv;
        fin[1] = dgv;
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
        double tp = 0.0, tg = 0.0;
        for (int r = 0; r < ncl; r++) {
            tp += cl.map_shared_rank(fin, (unsigned)r)[0];
            tg += cl.map_shared_rank(fin, (unsigned)r)[1];
        }
        a.out[0] = 0.5 * (a.x_sqnorm_dev ? *a.x_sqnorm_dev : a.x_sqnorm) - 0.5 * tp + 0.5 * tg;
        a.out[1] = (double)it;
        a.out[2] = eta;
        a.out[3] = (double)n_trials;
        for (int i = 0; i < 6; i++) a.out[4 + i] = (double)s_ph[i];
    }
    cl.sync();  // keep every rank's shared memory alive until all reads are done
}
#undef PGD_TICK

static size_t pgd_smem(const Geom &g, int ka, bool stage, bool qsm) {
    const long long per = (long long)g.P * g.L0 * g.L1, n = g.nd();
    const int K = g.K;
    size_t f = ((size_t)n + 2 * (size_t)ka * per + (stage ? (size_t)ka * K * g.nw() : 0) +
                (qsm ? 2 * (size_t)K * ka * per : 0)) *
               sizeof(float);
    return f;
}

int dict_update_impl(const Geom &g, const float *phi, const float *psi, double x_sqnorm, float *D,
                     int max_iter, double tol, double *obj_out, int *it_out, unsigned char *ws,
                     const WsLayout &L, cudaStream_t st, const double *x_sqnorm_dev, const int *gate,
                     int gate_cap) {
    if (g.K > kPgdMaxK) return CSC_ERR_UNIMPLEMENTED;
    WsHeader *h = reinterpret_cast<WsHeader *>(ws + L.hdr);
    PgdArgs a;
    a.phi = phi;
    a.psi = psi;
    a.D = D;
    a.qd = reinterpret_cast<float *>(ws + L.pgd);
    a.qg = a.qd + (size_t)g.K * g.nd() + 16 * (size_t)g.natom() * g.K;
    a.out = h->pgd_out;
    a.x_sqnorm = x_sqnorm;
    a.x_sqnorm_dev = x_sqnorm_dev;
    a.gate = gate;
    a.gate_cap = gate_cap;
    a.tol = tol;
    a.K = g.K;
    a.P = g.P;
    a.L0 = g.L0;
    a.L1 = g.L1;
    a.max_iter = max_iter;
    const size_t lim = 200 * 1024;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kPgdThreads);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // fewest atoms per CTA (largest cluster, at most 16) that fits and can be
    // scheduled; the choice is cached per (device, K, P, L0, L1)
    struct Choice {
        int dev, K, P, L0, L1, ka, stage, qsm;
        size_t smem;
    };
    static thread_local std::vector<Choice> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    int hit = -1;
    for (size_t i = 0; i < cache.size(); i++) {
        const Choice &c = cache[i];
        if (c.dev == dev && c.K == g.K && c.P == g.P && c.L0 == g.L0 && c.L1 == g.L1) hit = (int)i;
    }
    if (hit < 0) {
        CSC_CUDA(cudaFuncSetAttribute(pgd_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        bool ok = false;
        Choice ch{dev, g.K, g.P, g.L0, g.L1, 0, 0, 0, 0};
        for (int ka = (int)ceil_div(g.K, kPgdMaxCluster); ka <= g.K && !ok; ka++) {
            const int cs = (int)ceil_div(g.K, ka);
            if (pgd_smem(g, ka, false, false) > lim) break;
            ch.ka = ka;
            ch.qsm = pgd_smem(g, ka, false, true) <= lim;
            ch.stage = pgd_smem(g, ka, true, ch.qsm) <= lim;
            ch.smem = pgd_smem(g, ka, ch.stage, ch.qsm);
            CSC_CUDA(cudaFuncSetAttribute(pgd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)ch.smem));
            cfg.gridDim = dim3(cs);
            cfg.dynamicSmemBytes = ch.smem;
            attr[0].val.clusterDim.x = cs;
            int nclusters = 0;
            cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, pgd_kernel, &cfg);
            if (e == cudaSuccess && nclusters >= 1) ok = true;
            else cudaGetLastError();
        }
        if (!ok) return CSC_ERR_UNIMPLEMENTED;
        cache.push_back(ch);
        hit = (int)cache.size() - 1;
    }
    const Choice ch = cache[hit];
    a.ka = ch.ka;
    a.stage_phi = ch.stage;
    a.q_in_smem = ch.qsm;
    const int cs = (int)ceil_div(g.K, ch.ka);
    CSC_CUDA(cudaFuncSetAttribute(pgd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ch.smem));
    cfg.gridDim = dim3(cs);
    cfg.dynamicSmemBytes = ch.smem;
    attr[0].val.clusterDim.x = cs;
    CSC_CUDA(cudaLaunchKernelEx(&cfg, pgd_kernel, a));
    if (obj_out || it_out) {
        double out[3];
        {
            const int rb_ = read_back(&out, h->pgd_out, st);  // all three values
            if (rb_) return rb_;
        }
        if (obj_out) *obj_out = out[0];
        if (it_out) *it_out = (int)out[1];
    }
    return CSC_OK;
}

}  // namespace csc
