// residual.cu -- the residual X - Z*D, the objective of Eq. csc in FP64,
// beta recomputed from its definition (Section 3) and the final
// max |dZ| check of Alg. 1 on that fresh beta.
//
// Z is sparse at the optimum, so the reconstruction is a scatter from the
// compacted nonzeros of Z with FP64 atomics: every nonzero (k, s, z) adds
// -z D_k to the residual on s + Theta.  If the nonzeros do not fit the list
// the residual is rebuilt densely instead.
#include "lgcd_global.cuh"

namespace csc {

// Nonzeros of Z into (k, s, z) lists; order is unspecified (one atomic per
// warp).  Counts past the capacity only set the overflow flag.  The same
// pass accumulates ||Z||_1 in FP64.
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
    compact_any_kernel<real, 256><<<grid_for(nz, 256), 256, 0, st>>>(Z, g.nzpos(), g.K, nk, ns, nzv,
                                                                      L.nnz_cap, h);
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
            const long long plane = g.nzpos();
            dim3 grid((unsigned)std::min<long long>(ceil_div(plane, 4 * 256), std::max(1, 152 * 8 / g.K)), (unsigned)g.K);
            maxdz_kernel<256><<<grid, 256, 0, st>>>(beta, Z, nrm, lambda, plane, h, &h->maxdz_bits);
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
        (const void *)residual_init_kernel<float>,
        (const void *)scatter_kernel<float, 128>,
        (const void *)recon_dense_kernel<float>,
        (const void *)residual_finish_kernel<float, 256>,
        (const void *)copy_beta0_kernel<256>,
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
