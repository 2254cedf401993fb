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

// psi: a CTA takes a chunk of nonzeros; thread e owns entry (p, tau) of
// every atom in shared memory, so no two threads touch the same word.
template <int NT>
__global__ void __launch_bounds__(NT) psi_kernel(const int *nk, const int *ns, const float *nzv,
                                                 const WsHeader *h, const float *X, double *psi64,
                                                 int P, int K, int T0, int T1, int L0, int L1, int Z1,
                                                 int chunk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *acc = reinterpret_cast<float *>(smem_raw);
    const int LL = L0 * L1, per = P * LL;
    const int cnt = h->scan_total;
    const int lo = blockIdx.x * chunk, hi = min(cnt, lo + chunk);
    if (lo >= hi) return;
    for (int q = threadIdx.x; q < K * per; q += NT) acc[q] = 0.f;
    __syncthreads();
    for (int n = lo; n < hi; n++) {
        const int k = nk[n], s = ns[n];
        const float z = nzv[n];
        const int i = s / Z1, j = s % Z1;
        for (int e = threadIdx.x; e < per; e += NT) {
            int p = e / LL, r = e % LL;
            acc[k * per + e] += z * X[((size_t)p * T0 + i + r / L1) * T1 + j + r % L1];
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

__global__ void phi_pairs_kernel(const int *nk, const int *ns, const float *nzv, const WsHeader *h,
                                 double *phi64, int K, int L0, int L1, int Z0, int Z1) {
    const int cnt = h->scan_total;
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

int dict_stats_impl(const Geom &g, const float *Z, const float *X, float *phi, float *psi,
                    unsigned char *ws, const WsLayout &L, cudaStream_t st) {
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

    nz_count_kernel<256><<<nblk, 256, 0, st>>>(Z, zpos, g.K, blk_cnt);
    nz_scan_kernel<1024><<<1, 1024, 0, st>>>(blk_cnt, blk_off, nblk, h);
    int total = 0;
    CSC_CUDA(cudaMemcpyAsync(&total, &h->scan_total, sizeof(int), cudaMemcpyDeviceToHost, st));
    CSC_CUDA(cudaStreamSynchronize(st));
    if (total > L.nnz_cap) return CSC_ERR_WORKSPACE;
    nz_write_kernel<256><<<nblk, 256, 0, st>>>(Z, zpos, g.K, blk_off, h, L.nnz_cap, nk, ns, nzv);
    CSC_CUDA(cudaMemsetAsync(phi64, 0, (size_t)g.ntab() * sizeof(double), st));
    CSC_CUDA(cudaMemsetAsync(psi64, 0, (size_t)g.nd() * sizeof(double), st));
    if (total > 0) {
        const int chunk = 64;
        size_t smem = (size_t)g.nd() * sizeof(float);
        if (smem > 227 * 1024) return CSC_ERR_UNIMPLEMENTED;
        if (smem > 48 * 1024)
            CSC_CUDA(cudaFuncSetAttribute(psi_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        psi_kernel<256><<<(int)ceil_div(total, chunk), 256, smem, st>>>(
            nk, ns, nzv, h, X, psi64, g.P, g.K, g.T0, g.T1, g.L0, g.L1, g.Z1, chunk);
        phi_pairs_kernel<<<(int)ceil_div(total, 128), 128, 0, st>>>(nk, ns, nzv, h, phi64, g.K, g.L0,
                                                                    g.L1, g.Z0, g.Z1);
    }
    to_float_kernel<<<(int)std::min<long long>(ceil_div(g.ntab(), 256), 4096), 256, 0, st>>>(
        phi64, phi, g.ntab());
    to_float_kernel<<<(int)std::min<long long>(ceil_div(g.nd(), 256), 4096), 256, 0, st>>>(
        psi64, psi, g.nd());
    CSC_CUDA(cudaGetLastError());
    return CSC_OK;
}

// ====================================================== PGD + Armijo step
// Cluster layout: CTA r owns whole atoms [r ka, (r+1) ka), so the
// projection norms are local.  Its slices of D, the gradient G, the trial
// point and phi * (trial - D) live in shared memory; the trial difference is
// published (double-buffered) for the other CTAs, which gather the full
// difference through distributed shared memory before the convolution.
// Scalars are combined by publishing per-CTA partials and reading them from
// every rank after one cluster barrier (double-buffered as well), so one
// Armijo trial costs two cluster barriers.
struct PgdArgs {
    const float *phi, *psi;
    float *D;      // in/out
    double *out;   // [objective, iterations, eta]
    double x_sqnorm, tol;
    int K, P, L0, L1, max_iter, ka, stage_phi;
};

constexpr int kPgdThreads = 1024;
constexpr int kPgdWarps = kPgdThreads / 32;

struct PgdSmem {
    float *del;       // full trial difference, K * per (gathered)
    float *pubdel[2]; // own trial difference, ka * per, double-buffered
    float *d, *g, *dn, *q;
    float *phi;       // own rows of phi (optional)
};

// Block-wide sum returned to every thread (warp 0 combines the warp sums).
__device__ __forceinline__ double block_reduce_sum(double v, double *scratch) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = warp_sum(scratch[threadIdx.x]);
        if (threadIdx.x == 0) scratch[kPgdWarps] = s;
    }
    __syncthreads();
    return scratch[kPgdWarps];
}

// q[e] = sum_k2 sum_tau2 phi_{k,k2}[tau - tau2] src[k2][p][tau2] for the own
// entries e = (k, p, ta, tb).  A task is (own row (k, p, ta), four
// consecutive tb, one source atom k2): it slides a four-wide window of the
// phi row along tau2 so every step is one broadcast load of src, one load
// of phi and four FMAs; the K partial sums of an output are combined with
// shared-memory atomics.
__device__ __forceinline__ void phi_conv_own(const PgdArgs &a, const PgdSmem &S, int k_lo, int nown,
                                             const float *src, float *q) {
    const int LL = a.L0 * a.L1, per = a.P * LL;
    const int W0 = 2 * a.L0 - 1, W1 = 2 * a.L1 - 1, WW = W0 * W1;
    for (int e = threadIdx.x; e < nown; e += kPgdThreads) q[e] = 0.f;
    __syncthreads();
    const int nb = (a.L1 + 3) / 4;                 // tb blocks per row
    const int rows = nown / a.L1;                  // own rows (k, p, ta)
    const int ntask = rows * nb * a.K;
    for (int task = threadIdx.x; task < ntask; task += kPgdThreads) {
        const int k2 = task % a.K;
        const int rb = task / a.K;
        const int row = rb / nb, tb0 = (rb % nb) * 4;
        const int kl = row / (a.P * a.L0), rem = row % (a.P * a.L0), p = rem / a.L0, ta = rem % a.L0;
        const float *ph = (a.stage_phi ? S.phi + (size_t)kl * a.K * WW
                                       : a.phi + (size_t)(k_lo + kl) * a.K * WW) + (size_t)k2 * WW;
        const float *sv = src + (size_t)k2 * per + p * LL;
        float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
        for (int a2 = 0; a2 < a.L0; a2++) {
            // phi index along the row: tb - b2 + L1 - 1, for tb = tb0 .. tb0 + 3
            const float *prow = ph + (ta - a2 + a.L0 - 1) * W1 + tb0 + a.L1 - 1;
            const float *srow = sv + a2 * a.L1;
            // f_q holds phi at row index tb0 + q - b2 + L1 - 1; outputs past the
            // row end (ragged last block) start at zero and are discarded
            float f0 = prow[0];
            float f1 = tb0 + 1 < a.L1 ? prow[1] : 0.f;
            float f2 = tb0 + 2 < a.L1 ? prow[2] : 0.f;
            float f3 = tb0 + 3 < a.L1 ? prow[3] : 0.f;
            for (int b2 = 0; b2 < a.L1; b2++) {
                const float x = srow[b2];
                acc0 = fmaf(f0, x, acc0);
                acc1 = fmaf(f1, x, acc1);
                acc2 = fmaf(f2, x, acc2);
                acc3 = fmaf(f3, x, acc3);
                f3 = f2;
                f2 = f1;
                f1 = f0;
                f0 = (b2 + 1 < a.L1) ? prow[-(b2 + 1)] : 0.f;
            }
        }
        float *qo = q + (size_t)row * a.L1 + tb0;
        atomicAdd(qo, acc0);
        if (tb0 + 1 < a.L1) atomicAdd(qo + 1, acc1);
        if (tb0 + 2 < a.L1) atomicAdd(qo + 2, acc2);
        if (tb0 + 3 < a.L1) atomicAdd(qo + 3, acc3);
    }
}

__global__ void __launch_bounds__(kPgdThreads, 1) pgd_kernel(PgdArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int LL = a.L0 * a.L1, per = a.P * LL, n = a.K * per;
    const int W0 = 2 * a.L0 - 1, W1 = 2 * a.L1 - 1, WW = W0 * W1;
    const int rank = (int)cl.block_rank(), ncl = (int)cl.num_blocks();
    const int k_lo = min(a.K, rank * a.ka), k_hi = min(a.K, k_lo + a.ka);
    const int nk = k_hi - k_lo, nown = nk * per, e0 = k_lo * per;
    const int own_cap = a.ka * per;

    PgdSmem S;
    float *f = reinterpret_cast<float *>(smem_raw);
    S.del = f;
    f += n;
    S.pubdel[0] = f;
    f += own_cap;
    S.pubdel[1] = f;
    f += own_cap;
    S.d = f;
    f += own_cap;
    S.g = f;
    f += own_cap;
    S.dn = f;
    f += own_cap;
    S.q = f;
    f += own_cap;
    S.phi = f;

    __shared__ double pub[2][8];
    __shared__ double scratch[kPgdWarps + 1];
    __shared__ double anrm[16];
    __shared__ double bcast[4];
    int pb = 0;
    // publish up to 4 block totals, one cluster barrier, read the cluster sums
    auto cluster_sum4 = [&](double v0, double v1, double v2, double v3, double *out4, bool as_max0) {
        if (threadIdx.x == 0) {
            pub[pb][0] = v0;
            pub[pb][1] = v1;
            pub[pb][2] = v2;
            pub[pb][3] = v3;
        }
        cl.sync();
        if (threadIdx.x < 32) {
            double t[4] = {0, 0, 0, 0};
            if ((int)threadIdx.x < ncl) {
                const double *rp = cl.map_shared_rank(&pub[pb][0], (unsigned)threadIdx.x);
                for (int i = 0; i < 4; i++) t[i] = rp[i];
            }
            for (int o = 16; o > 0; o >>= 1) {
                double x = __shfl_xor_sync(0xffffffffu, t[0], o);
                t[0] = as_max0 ? fmax(t[0], x) : t[0] + x;
                for (int i = 1; i < 4; i++) t[i] += __shfl_xor_sync(0xffffffffu, t[i], o);
            }
            if (threadIdx.x == 0)
                for (int i = 0; i < 4; i++) bcast[i] = t[i];
        }
        __syncthreads();
        for (int i = 0; i < 4; i++) out4[i] = bcast[i];
        pb ^= 1;
    };

    // stage own slices, own rows of phi, the full D (for the first gradient)
    for (int e = threadIdx.x; e < nown; e += kPgdThreads) S.d[e] = a.D[e0 + e];
    for (int e = threadIdx.x; e < n; e += kPgdThreads) S.del[e] = a.D[e];
    if (a.stage_phi)
        for (size_t e = threadIdx.x; e < (size_t)nk * a.K * WW; e += kPgdThreads)
            S.phi[e] = a.phi[(size_t)k_lo * a.K * WW + e];
    __syncthreads();

    // Lipschitz bound max_k sum_k2 sum_d |phi_{k,k2}[d]| over own rows, then cluster max
    double lip_loc = 0.0;
    for (int kl = 0; kl < nk; kl++) {
        double s = 0.0;
        for (size_t q = threadIdx.x; q < (size_t)a.K * WW; q += kPgdThreads)
            s += fabs((double)a.phi[(size_t)(k_lo + kl) * a.K * WW + q]);
        lip_loc = fmax(lip_loc, block_reduce_sum(s, scratch));
    }
    // G = phi * D - psi on the own slice
    phi_conv_own(a, S, k_lo, nown, S.del, S.q);
    __syncthreads();
    for (int e = threadIdx.x; e < nown; e += kPgdThreads) S.g[e] = S.q[e] - a.psi[e0 + e];
    double tot[4];
    cluster_sum4(lip_loc, 0, 0, 0, tot, true);
    const double lip = tot[0];

    double eta = lip > 0.0 ? 1.0 / lip : 0.0;
    int it = 0, tb = 0;
    if (lip > 0.0) {
        for (it = 0; it < a.max_iter; it++) {
            if (it > 0) eta *= 2.0;
            double dsq = 0.0, dnorm = 0.0;
            for (int bt = 0; bt < 60; bt++) {
                // trial point, projected atom by atom (norms are local)
                __syncthreads();
                for (int e = threadIdx.x; e < nown; e += kPgdThreads) S.dn[e] = S.d[e] - (float)eta * S.g[e];
                __syncthreads();
                for (int kl = 0; kl < nk; kl++) {
                    double s = 0.0;
                    for (int e = threadIdx.x; e < per; e += kPgdThreads) {
                        double v = S.dn[kl * per + e];
                        s += v * v;
                    }
                    s = block_reduce_sum(s, scratch);
                    if (threadIdx.x == 0) anrm[kl] = sqrt(s);
                }
                __syncthreads();
                double dd = 0.0, d0 = 0.0;
                float *pd = S.pubdel[tb];
                for (int e = threadIdx.x; e < nown; e += kPgdThreads) {
                    double nr = anrm[e / per];
                    float v = S.dn[e];
                    if (nr > 1.0) v = (float)((double)v / nr);
                    S.dn[e] = v;
                    float dl = v - S.d[e];
                    pd[e] = dl;
                    dd += (double)dl * dl;
                    d0 += (double)S.d[e] * S.d[e];
                }
                dd = block_reduce_sum(dd, scratch);
                d0 = block_reduce_sum(d0, scratch);
                cluster_sum4(dd, d0, 0, 0, tot, false);  // also publishes pubdel[tb]
                dsq = tot[0];
                dnorm = tot[1];
                // gather the full difference from every rank
                for (int r = 0; r < ncl; r++) {
                    const int rlo = min(a.K, r * a.ka) * per, rhi = min(a.K, r * a.ka + a.ka) * per;
                    const float *rp = cl.map_shared_rank(S.pubdel[tb], r);
                    for (int e = threadIdx.x; e < rhi - rlo; e += kPgdThreads) S.del[rlo + e] = rp[e];
                }
                __syncthreads();
                phi_conv_own(a, S, k_lo, nown, S.del, S.q);
                __syncthreads();
                double qd = 0.0;
                for (int e = threadIdx.x; e < nown; e += kPgdThreads) qd += (double)pd[e] * S.q[e];
                qd = block_reduce_sum(qd, scratch);
                cluster_sum4(qd, 0, 0, 0, tot, false);
                tb ^= 1;
                if (tot[0] * eta <= dsq) break;
                eta *= 0.5;
            }
            // accept: D = D+, G = G + phi * (D+ - D)
            for (int e = threadIdx.x; e < nown; e += kPgdThreads) {
                S.d[e] = S.dn[e];
                S.g[e] += S.q[e];
            }
            if (sqrt(dsq) < a.tol * sqrt(dnorm)) {
                it++;
                break;
            }
        }
    }
    __syncthreads();
    // F(D) = 1/2||X||^2 - 1/2 <psi, D> + 1/2 <D, G>; write D back
    double pdv = 0.0, dg = 0.0;
    for (int e = threadIdx.x; e < nown; e += kPgdThreads) {
        pdv += (double)a.psi[e0 + e] * S.d[e];
        dg += (double)S.d[e] * S.g[e];
        a.D[e0 + e] = S.d[e];
    }
    pdv = block_reduce_sum(pdv, scratch);
    dg = block_reduce_sum(dg, scratch);
    cluster_sum4(pdv, dg, 0, 0, tot, false);
    if (rank == 0 && threadIdx.x == 0) {
        a.out[0] = 0.5 * a.x_sqnorm - 0.5 * tot[0] + 0.5 * tot[1];
        a.out[1] = (double)it;
        a.out[2] = eta;
    }
    cl.sync();  // keep every rank's shared memory alive until all reads are done
}

int dict_update_impl(const Geom &g, const float *phi, const float *psi, double x_sqnorm, float *D,
                     int max_iter, double tol, double *obj_out, int *it_out, unsigned char *ws,
                     const WsLayout &L, cudaStream_t st) {
    WsHeader *h = reinterpret_cast<WsHeader *>(ws + L.hdr);
    const long long per = (long long)g.P * g.L0 * g.L1, n = g.nd();
    PgdArgs a;
    a.phi = phi;
    a.psi = psi;
    a.D = D;
    a.out = h->pgd_out;
    a.x_sqnorm = x_sqnorm;
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
        int dev, K, P, L0, L1, ka, stage;
        size_t smem;
    };
    static thread_local std::vector<Choice> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const Choice *hit = nullptr;
    for (const Choice &c : cache)
        if (c.dev == dev && c.K == g.K && c.P == g.P && c.L0 == g.L0 && c.L1 == g.L1) hit = &c;
    if (!hit) {
        CSC_CUDA(cudaFuncSetAttribute(pgd_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        bool ok = false;
        Choice ch{dev, g.K, g.P, g.L0, g.L1, 0, 0, 0};
        for (int ka = (int)ceil_div(g.K, 16); ka <= 16 && !ok; ka++) {
            const int cs = (int)ceil_div(g.K, ka);
            size_t base = ((size_t)n + 6 * (size_t)ka * per) * sizeof(float);
            size_t phi_bytes = (size_t)ka * g.K * g.nw() * sizeof(float);
            if (base > lim) break;
            ch.ka = ka;
            ch.stage = base + phi_bytes <= lim;
            ch.smem = base + (ch.stage ? phi_bytes : 0);
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
        hit = &cache.back();
    }
    a.ka = hit->ka;
    a.stage_phi = hit->stage;
    const int cs = (int)ceil_div(g.K, hit->ka);
    CSC_CUDA(cudaFuncSetAttribute(pgd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hit->smem));
    cfg.gridDim = dim3(cs);
    cfg.dynamicSmemBytes = hit->smem;
    attr[0].val.clusterDim.x = cs;
    CSC_CUDA(cudaLaunchKernelEx(&cfg, pgd_kernel, a));
    if (obj_out || it_out) {
        double out[3];
        CSC_CUDA(cudaMemcpyAsync(out, h->pgd_out, sizeof(out), cudaMemcpyDeviceToHost, st));
        CSC_CUDA(cudaStreamSynchronize(st));
        if (obj_out) *obj_out = out[0];
        if (it_out) *it_out = (int)out[1];
    }
    return CSC_OK;
}

}  // namespace csc
