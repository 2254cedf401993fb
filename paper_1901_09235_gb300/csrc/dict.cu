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
struct PgdArgs {
    const float *phi, *psi;
    float *D;      // in/out
    float *G;      // gradient phi * D - psi
    float *Dn;     // trial point
    float *Del;    // D+ - D (read by every CTA)
    float *Q;      // phi * (D+ - D)
    double *out;   // [objective, iterations, eta]
    double x_sqnorm, tol;
    int K, P, L0, L1, max_iter;
};

constexpr int kPgdThreads = 1024;
constexpr int kPgdMaxK = 64;

// Sum over the cluster of per-CTA partial vectors of length n (n <= 64).
__device__ __forceinline__ void cluster_sum(cg::cluster_group &cl, double *part, double *tot, int n) {
    cl.sync();
    if (threadIdx.x < n) {
        double s = 0.0;
        for (unsigned r = 0; r < cl.num_blocks(); r++) s += cl.map_shared_rank(part, r)[threadIdx.x];
        tot[threadIdx.x] = s;
    }
    cl.sync();
}

// Block-wide sums of up to 4 values into part[0..3] (thread 0 writes).
__device__ __forceinline__ void block_sums4(double v0, double v1, double v2, double v3, double *part) {
    __shared__ double red[4][kPgdThreads / 32];
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    v3 = warp_sum(v3);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = v0;
        red[1][threadIdx.x >> 5] = v1;
        red[2][threadIdx.x >> 5] = v2;
        red[3][threadIdx.x >> 5] = v3;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kPgdThreads / 32; w++) s += red[threadIdx.x][w];
        part[threadIdx.x] = s;
    }
    __syncthreads();
}

// out[e] = sum_k2 sum_tau2 phi_{k,k2}[tau - tau2] src[k2][p][tau2] over this
// CTA's slice of entries e = (k, p, tau); src is staged in shared memory.
__device__ __forceinline__ void phi_conv_slice(const PgdArgs &a, const float *ssrc, float *out, int lo,
                                               int hi) {
    const int LL = a.L0 * a.L1, per = a.P * LL;
    const int W0 = 2 * a.L0 - 1, W1 = 2 * a.L1 - 1;
    for (int e = lo + threadIdx.x; e < hi; e += kPgdThreads) {
        const int k = e / per, r = e % per, p = r / LL, t = r % LL, ta = t / a.L1, tb = t % a.L1;
        float acc = 0.f;
        for (int k2 = 0; k2 < a.K; k2++) {
            const float *ph = a.phi + (size_t)(k * a.K + k2) * W0 * W1;
            const float *sv = ssrc + (size_t)k2 * per + p * LL;
            for (int a2 = 0; a2 < a.L0; a2++) {
                const float *prow = ph + (ta - a2 + a.L0 - 1) * W1 + tb + a.L1 - 1;
                const float *srow = sv + a2 * a.L1;
                for (int b2 = 0; b2 < a.L1; b2++) acc = fmaf(__ldg(prow - b2), srow[b2], acc);
            }
        }
        out[e] = acc;
    }
}

__global__ void __launch_bounds__(kPgdThreads, 1) pgd_kernel(PgdArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int LL = a.L0 * a.L1, per = a.P * LL, n = a.K * per;
    float *ssrc = reinterpret_cast<float *>(smem_raw);  // full D or Delta
    __shared__ double part[kPgdMaxK + 8], tot[kPgdMaxK + 8];
    __shared__ double sc[4];
    const int rank = (int)cl.block_rank(), ncl = (int)cl.num_blocks();
    const int chunk = (n + ncl - 1) / ncl;
    const int lo = min(n, rank * chunk), hi = min(n, lo + chunk);
    const int W0 = 2 * a.L0 - 1, W1 = 2 * a.L1 - 1;

    // Lipschitz bound: max_k sum_k2 sum_d |phi_{k,k2}[d]| (rows split over CTAs).
    {
        const long long row = (long long)a.K * W0 * W1;
        for (int k = 0; k < a.K; k++) {
            double s = 0.0;
            long long rlo = row * rank / ncl, rhi = row * (rank + 1) / ncl;
            for (long long q = rlo + threadIdx.x; q < rhi; q += kPgdThreads)
                s += fabs((double)a.phi[(size_t)k * row + q]);
            block_sums4(s, 0, 0, 0, sc);
            if (threadIdx.x == 0) part[k] = sc[0];
        }
        cluster_sum(cl, part, tot, a.K);
    }
    double lip = 0.0;
    for (int k = 0; k < a.K; k++) lip = fmax(lip, tot[k]);

    // G = phi * D - psi
    for (int e = threadIdx.x; e < n; e += kPgdThreads) ssrc[e] = a.D[e];
    __syncthreads();
    phi_conv_slice(a, ssrc, a.G, lo, hi);
    for (int e = lo + threadIdx.x; e < hi; e += kPgdThreads) a.G[e] -= a.psi[e];

    double eta = lip > 0.0 ? 1.0 / lip : 0.0;
    int it = 0;
    if (lip > 0.0) {
        for (it = 0; it < a.max_iter; it++) {
            if (it > 0) eta *= 2.0;
            double dsq = 0.0, dnorm = 0.0;
            for (int bt = 0; bt < 60; bt++) {
                // trial point and per-atom squared norms
                for (int k = threadIdx.x; k < a.K; k += kPgdThreads) part[k] = 0.0;
                __syncthreads();
                for (int e = lo + threadIdx.x; e < hi; e += kPgdThreads) {
                    float v = a.D[e] - (float)eta * a.G[e];
                    a.Dn[e] = v;
                    atomicAdd(&part[e / per], (double)v * (double)v);
                }
                cluster_sum(cl, part, tot, a.K);
                double dd = 0.0, d0 = 0.0;
                for (int e = lo + threadIdx.x; e < hi; e += kPgdThreads) {
                    double nr = sqrt(tot[e / per]);
                    float v = a.Dn[e];
                    if (nr > 1.0) v = (float)((double)v / nr);
                    a.Dn[e] = v;
                    float dl = v - a.D[e];
                    a.Del[e] = dl;
                    dd += (double)dl * dl;
                    d0 += (double)a.D[e] * a.D[e];
                }
                cl.sync();  // Delta complete in global memory
                for (int e = threadIdx.x; e < n; e += kPgdThreads) ssrc[e] = __ldcg(a.Del + e);
                __syncthreads();
                phi_conv_slice(a, ssrc, a.Q, lo, hi);
                double qd = 0.0;
                for (int e = lo + threadIdx.x; e < hi; e += kPgdThreads) qd += (double)ssrc[e] * a.Q[e];
                block_sums4(dd, d0, qd, 0.0, sc);
                if (threadIdx.x < 3) part[threadIdx.x] = sc[threadIdx.x];
                cluster_sum(cl, part, tot, 3);
                dsq = tot[0];
                dnorm = tot[1];
                const double quad = tot[2];
                if (quad * eta <= dsq) break;
                eta *= 0.5;
            }
            // accept: D = D+, G = G + phi * (D+ - D)
            for (int e = lo + threadIdx.x; e < hi; e += kPgdThreads) {
                a.D[e] = a.Dn[e];
                a.G[e] += a.Q[e];
            }
            if (sqrt(dsq) < a.tol * sqrt(dnorm)) {
                it++;
                break;
            }
        }
    }
    // F(D) = 1/2||X||^2 - 1/2 <psi, D> + 1/2 <D, G>
    double pd = 0.0, dg = 0.0;
    for (int e = lo + threadIdx.x; e < hi; e += kPgdThreads) {
        pd += (double)a.psi[e] * a.D[e];
        dg += (double)a.D[e] * a.G[e];
    }
    block_sums4(pd, dg, 0.0, 0.0, sc);
    if (threadIdx.x < 2) part[threadIdx.x] = sc[threadIdx.x];
    cluster_sum(cl, part, tot, 2);
    if (rank == 0 && threadIdx.x == 0) {
        a.out[0] = 0.5 * a.x_sqnorm - 0.5 * tot[0] + 0.5 * tot[1];
        a.out[1] = (double)it;
        a.out[2] = eta;
    }
}

int dict_update_impl(const Geom &g, const float *phi, const float *psi, double x_sqnorm, float *D,
                     int max_iter, double tol, double *obj_out, int *it_out, unsigned char *ws,
                     const WsLayout &L, cudaStream_t st) {
    if (g.K > kPgdMaxK) return CSC_ERR_UNIMPLEMENTED;
    WsHeader *h = reinterpret_cast<WsHeader *>(ws + L.hdr);
    float *buf = reinterpret_cast<float *>(ws + L.pgd);
    const long long n = g.nd();
    PgdArgs a;
    a.phi = phi;
    a.psi = psi;
    a.D = D;
    a.G = buf;
    a.Dn = buf + n;
    a.Del = buf + 2 * n;
    a.Q = buf + 3 * n;
    a.out = h->pgd_out;
    a.x_sqnorm = x_sqnorm;
    a.tol = tol;
    a.K = g.K;
    a.P = g.P;
    a.L0 = g.L0;
    a.L1 = g.L1;
    a.max_iter = max_iter;
    size_t smem = (size_t)n * sizeof(float);
    if (smem > 200 * 1024) return CSC_ERR_UNIMPLEMENTED;
    CSC_CUDA(cudaFuncSetAttribute(pgd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CSC_CUDA(cudaFuncSetAttribute(pgd_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    const double work = (double)n * g.K * g.L0 * g.L1;
    int cs = work < 2e5 ? 2 : (work < 2e6 ? 8 : 16);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kPgdThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the largest cluster (<= cs) that the device can schedule
    for (;; cs /= 2) {
        cfg.gridDim = dim3(cs);
        attr[0].val.clusterDim.x = cs;
        int nclusters = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, pgd_kernel, &cfg);
        if (e == cudaSuccess && nclusters >= 1) break;
        cudaGetLastError();
        if (cs == 1) return CSC_ERR_UNIMPLEMENTED;
    }
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
