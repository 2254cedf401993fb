// corr.cu -- dense correlations of the CSC path on CUDA cores:
//   beta_k[s] = sum_p sum_tau D_kp[tau] S_p[s + tau]   (Alg. 1 initialisation
//               with S = X; the from-scratch recomputation of beta with
//               S = X - Z*D plus ||D_k||^2 Z_k, Section 3),
//   C[k][k2][delta] = sum_p sum_tau D_kp[tau] D_k2p[tau + delta]
//               (the table of Eq. beta_update),
//   ||D_k||^2 in FP64 and max |D_k| (Section 5.1 divergence bound).
#include <algorithm>

#include "common.cuh"

namespace csc {

template <typename real>
struct CorrArgs {
    const real *S;      // P x T0 x T1
    const real *Wt;     // K x P x L0 x L1
    real *out;          // K x Z0 x Z1
    const real *Zc;     // refresh: current Z (K x Z0 x Z1)
    const double *nrm;  // refresh: ||D_k||^2
    real lambda;
    unsigned long long *bits;  // init: max |beta|; refresh: max |dZ|
    int P, K, T0, T1, L0, L1, Z0, Z1;
    const int *gate;  // refresh: when set, the kernel runs only if *gate != 0
};

enum { EPI_INIT = 0, EPI_REFRESH = 1 };

// One CTA computes a TR x TC block of positions for KC atoms (blockIdx.z
// selects the atom chunk).  The signal patch of one channel and the matching
// atom slice are staged in shared memory; thread (r, cg) owns positions
// (r, cg + q * TPR), q < NQ, so a warp reads consecutive words of the patch
// while the atom weight is a broadcast.
template <typename real, int NT, int TR, int NQ, int KC, int EPI>
__global__ void __launch_bounds__(NT) corr_kernel(CorrArgs<real> a) {
    if (EPI == EPI_REFRESH && a.gate && *a.gate == 0) return;
    constexpr int TPR = NT / TR;
    constexpr int TC = TPR * NQ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *sS = reinterpret_cast<real *>(smem_raw);
    const int PR = TR + a.L0 - 1, PC = TC + a.L1 - 1;
    real *sW = sS + (size_t)PR * PC;
    const int LL = a.L0 * a.L1;

    const int i0 = blockIdx.y * TR, j0 = blockIdx.x * TC, k0 = blockIdx.z * KC;
    const int r = threadIdx.x / TPR, cg = threadIdx.x % TPR;

    real acc[KC][NQ];
#pragma unroll
    for (int kk = 0; kk < KC; kk++)
#pragma unroll
        for (int q = 0; q < NQ; q++) acc[kk][q] = real(0);

    for (int p = 0; p < a.P; p++) {
        __syncthreads();
        const real *Sp = a.S + (size_t)p * a.T0 * a.T1;
        for (int e = threadIdx.x; e < PR * PC; e += NT) {
            int rr = e / PC, cc = e % PC;
            int gi = i0 + rr, gj = j0 + cc;
            sS[e] = (gi < a.T0 && gj < a.T1) ? Sp[(size_t)gi * a.T1 + gj] : real(0);
        }
        for (int e = threadIdx.x; e < KC * LL; e += NT) {
            int kk = e / LL, t = e % LL;
            int k = k0 + kk;
            sW[e] = k < a.K ? a.Wt[((size_t)k * a.P + p) * LL + t] : real(0);
        }
        __syncthreads();
        for (int ta = 0; ta < a.L0; ta++) {
            const real *row = sS + (size_t)(r + ta) * PC + cg;
            const real *wrow = sW + ta * a.L1;
            for (int tb = 0; tb < a.L1; tb++) {
                real x[NQ];
#pragma unroll
                for (int q = 0; q < NQ; q++) x[q] = row[q * TPR + tb];
#pragma unroll
                for (int kk = 0; kk < KC; kk++) {
                    real wv = wrow[kk * LL + tb];
#pragma unroll
                    for (int q = 0; q < NQ; q++) acc[kk][q] = fma(wv, x[q], acc[kk][q]);
                }
            }
        }
    }

    unsigned long long m = 0;
    const int i = i0 + r;
#pragma unroll
    for (int kk = 0; kk < KC; kk++) {
        int k = k0 + kk;
        if (k >= a.K || i >= a.Z0) continue;
        double nk = 0.0;
        real nr = real(0), inv = real(0);
        if (EPI == EPI_REFRESH) {
            nk = a.nrm[k];
            nr = real(nk);
            inv = real(1.0 / nk);
        }
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            int j = j0 + cg + q * TPR;
            if (j >= a.Z1) continue;
            size_t at = ((size_t)k * a.Z0 + i) * a.Z1 + j;
            real v = acc[kk][q];
            if (EPI == EPI_INIT) {
                a.out[at] = v;
                unsigned long long b = nonneg_bits(v < real(0) ? -v : v);
                m = b > m ? b : m;
            } else {
                real z = a.Zc[at];
                v = v + nr * z;
                a.out[at] = v;
                real dz = coord_update(v, a.lambda, nr, inv) - z;
                dz = dz < real(0) ? -dz : dz;
                unsigned long long b = nonneg_bits(dz);
                m = b > m ? b : m;
            }
        }
    }
    block_max_atomic<NT>(m, a.bits);
}

// FP32 correlations by rows: a CTA covers TR output rows x TC columns for KC
// atoms; thread (r, c) owns the NQ consecutive positions (i0 + r, j0 + c NQ
// + q).  Taps go in blocks of NQ along a tap row: the 2 NQ signal values of
// row i0 + r + tau0 held in registers serve the NQ x NQ products of every
// atom, so each shared-memory word feeds NQ KC FMAs.  Weights are staged
// tap-major (the KC atoms of a tap contiguous, padded to KCP = a multiple of
// four, read as 16-byte broadcasts), tap columns padded with zero weights to a
// multiple of NQ.  Every output accumulates
// channel by channel, tap row by tap row and tap by tap, as corr_kernel does.
template <int NT, int TR, int NQ, int KC, int EPI>
__global__ void __launch_bounds__(NT) corr_rows_kernel(CorrArgs<float> a) {
    if (EPI == EPI_REFRESH && a.gate && *a.gate == 0) return;
    constexpr int TPR = NT / TR, TC = TPR * NQ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L0 = a.L0, L1 = a.L1, Lp = (L1 + NQ - 1) / NQ * NQ;
    constexpr int KCP = (KC + 3) / 4 * 4;
    const int PR = TR + L0 - 1, PC = (TC + Lp + NQ + 3) / 4 * 4;  // patch rows, padded row length
    float *sS = reinterpret_cast<float *>(smem_raw);  // PR x PC signal patch
    float *sW = sS + (size_t)PR * PC;                  // L0 x Lp x KCP weights
    const int i0 = blockIdx.y * TR, j0 = blockIdx.x * TC, k0 = blockIdx.z * KC;
    const int r = threadIdx.x / TPR, s0 = (threadIdx.x % TPR) * NQ;
    float acc[KC][NQ];
#pragma unroll
    for (int kk = 0; kk < KC; kk++)
#pragma unroll
        for (int q = 0; q < NQ; q++) acc[kk][q] = 0.f;
    for (int p = 0; p < a.P; p++) {
        __syncthreads();
        const float *Sp = a.S + (size_t)p * a.T0 * a.T1;
        for (int e = threadIdx.x; e < PR * PC; e += NT) {
            const int rr = e / PC, cc = e - rr * PC, gi = i0 + rr, gj = j0 + cc;
            sS[e] = (gi < a.T0 && gj < a.T1) ? Sp[(size_t)gi * a.T1 + gj] : 0.f;
        }
        for (int e = threadIdx.x; e < L0 * Lp * KCP; e += NT) {
            const int tt = e / KCP, kk = e - tt * KCP, ta = tt / Lp, tb = tt - ta * Lp, k = k0 + kk;
            sW[e] = (kk < KC && tb < L1 && k < a.K) ? a.Wt[(((size_t)k * a.P + p) * L0 + ta) * L1 + tb] : 0.f;
        }
        __syncthreads();
        for (int ta = 0; ta < L0; ta++) {
            const float *row = sS + (size_t)(r + ta) * PC + s0;
            const float *wta = sW + (size_t)ta * Lp * KCP;
            for (int tb = 0; tb < Lp; tb += NQ) {
                float x[2 * NQ];
#pragma unroll
                for (int i = 0; i < 2 * NQ; i += 4) {
                    const float4 v = *reinterpret_cast<const float4 *>(row + tb + i);
                    x[i] = v.x;
                    x[i + 1] = v.y;
                    x[i + 2] = v.z;
                    x[i + 3] = v.w;
                }
#pragma unroll
                for (int u = 0; u < NQ; u++) {
                    const float4 *wt = reinterpret_cast<const float4 *>(wta + (tb + u) * KCP);
                    float w[KCP];
#pragma unroll
                    for (int g = 0; g < KCP / 4; g++) {
                        const float4 v = wt[g];
                        w[4 * g] = v.x;
                        w[4 * g + 1] = v.y;
                        w[4 * g + 2] = v.z;
                        w[4 * g + 3] = v.w;
                    }
#pragma unroll
                    for (int kk = 0; kk < KC; kk++) {
#pragma unroll
                        for (int q = 0; q < NQ; q++) acc[kk][q] = fmaf(w[kk], x[q + u], acc[kk][q]);
                    }
                }
            }
        }
    }
    unsigned long long m = 0;
    const int i = i0 + r;
#pragma unroll
    for (int kk = 0; kk < KC; kk++) {
        const int k = k0 + kk;
        if (k >= a.K || i >= a.Z0) continue;
        float nr = 0.f, inv = 0.f;
        if (EPI == EPI_REFRESH) {
            const double nk = a.nrm[k];
            nr = (float)nk;
            inv = (float)(1.0 / nk);
        }
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const int j = j0 + s0 + q;
            if (j >= a.Z1) continue;
            const size_t at = ((size_t)k * a.Z0 + i) * a.Z1 + j;
            float v = acc[kk][q];
            if (EPI == EPI_INIT) {
                a.out[at] = v;
                const unsigned long long b = nonneg_bits(v < 0.f ? -v : v);
                m = b > m ? b : m;
            } else {
                const float z = a.Zc[at];
                v = v + nr * z;
                a.out[at] = v;
                float dz = coord_update(v, a.lambda, nr, inv) - z;
                dz = dz < 0.f ? -dz : dz;
                const unsigned long long b = nonneg_bits(dz);
                m = b > m ? b : m;
            }
        }
    }
    block_max_atomic<NT>(m, a.bits);
}

template <int NT, int TR, int NQ, int KC, int EPI>
static int run_corr_rows(const Geom &g, CorrArgs<float> a, cudaStream_t st) {
    constexpr int TC = (NT / TR) * NQ;
    auto kern = corr_rows_kernel<NT, TR, NQ, KC, EPI>;
    const int Lp = (g.L1 + NQ - 1) / NQ * NQ;
    const int PR = TR + g.L0 - 1, PC = (TC + Lp + NQ + 3) / 4 * 4;
    const size_t smem = ((size_t)PR * PC + (size_t)g.L0 * Lp * ((KC + 3) / 4 * 4)) * sizeof(float);
    if (smem > 227 * 1024) return CSC_ERR_UNIMPLEMENTED;
    if (smem > 48 * 1024)
        CSC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)ceil_div(g.Z1, TC), (unsigned)ceil_div(g.Z0, TR), (unsigned)ceil_div(g.K, KC));
    kern<<<grid, NT, smem, st>>>(a);
    CSC_CUDA(cudaGetLastError());
    return CSC_OK;
}

template <int EPI>
static int corr_rows_dispatch(const Geom &g, CorrArgs<float> a, cudaStream_t st) {
    if (g.Z0 == 1) {
        // 1-D: 128 threads x 4 positions, measured fastest on the 1-D workload
        // (P = 5, T = 200,000, K = 10, L = 64) among 64 / 128 / 256 x 4 / 8
        if (g.K <= 4) return run_corr_rows<128, 1, 4, 4, EPI>(g, a, st);
        if (g.K <= 8) return run_corr_rows<128, 1, 4, 8, EPI>(g, a, st);
        if (g.K <= 10) return run_corr_rows<128, 1, 4, 10, EPI>(g, a, st);
        return run_corr_rows<128, 1, 4, 16, EPI>(g, a, st);
    }
    // 2-D: the atom chunk that pads K least -- 5 atoms x 8 positions a
    // thread on 24 rows x 128 columns per CTA of 384 threads (72 registers),
    // else 8, 13 or 16 atoms x 4 positions on 8 rows x 128 columns per CTA of
    // 256.  On the 4096^2 image with 25 atoms of 32 x 32: 14.5 ms for five
    // chunks of 5 against 15.8 ms for two of 13 (256 x 8 rows), 15.0 ms for
    // 5 atoms on 256 x 16 rows, 14.6 on 384 x 12 or 48 rows, 16.2-16.9 on 320,
    // 448 or 512 threads, 19.6-19.8 for 128 threads x 4 rows.  Beside a running
    // queue kernel only one warp of 128 registers fits per SM sub-partition:
    // 128 threads x 4 rows then.
    const long long w5 = ceil_div(g.K, 5) * 5, w13 = ceil_div(g.K, 13) * 13, w16 = ceil_div(g.K, 16) * 16;
    if (live_queues() > 0) {
        if (g.K <= 8) return run_corr_rows<128, 4, 4, 8, EPI>(g, a, st);
        if (w13 < w16) return run_corr_rows<128, 4, 4, 13, EPI>(g, a, st);
        return run_corr_rows<128, 4, 4, 16, EPI>(g, a, st);
    }
    // chunks of 5 cost about 12/13 as much per atom as the others
    const long long wmin = std::min<long long>(g.K <= 8 ? 8 : w13, w16);
    if (12 * w5 <= 13 * wmin) return run_corr_rows<384, 24, 8, 5, EPI>(g, a, st);
    if (g.K <= 8) return run_corr_rows<256, 8, 4, 8, EPI>(g, a, st);
    if (w13 < w16) return run_corr_rows<256, 8, 4, 13, EPI>(g, a, st);
    return run_corr_rows<256, 8, 4, 16, EPI>(g, a, st);
}

template <typename real, int NT, int TR, int NQ, int KC, int EPI>
static int run_corr(const Geom &g, CorrArgs<real> a, cudaStream_t st) {
    constexpr int TC = (NT / TR) * NQ;
    auto kern = corr_kernel<real, NT, TR, NQ, KC, EPI>;
    size_t smem = ((size_t)(TR + g.L0 - 1) * (TC + g.L1 - 1) + (size_t)KC * g.L0 * g.L1) * sizeof(real);
    if (smem > 48 * 1024) {
        if (smem > 227 * 1024) return CSC_ERR_UNIMPLEMENTED;
        CSC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    dim3 grid((unsigned)ceil_div(g.Z1, TC), (unsigned)ceil_div(g.Z0, TR), (unsigned)ceil_div(g.K, KC));
    kern<<<grid, NT, smem, st>>>(a);
    CSC_CUDA(cudaGetLastError());
    return CSC_OK;
}

template <typename real, int EPI>
static int corr_dispatch(const Geom &g, CorrArgs<real> a, cudaStream_t st) {
    if constexpr (sizeof(real) == 4) {
        const int rc = corr_rows_dispatch<EPI>(g, a, st);
        if (rc != CSC_ERR_UNIMPLEMENTED) return rc;  // too large for shared memory: the generic kernel
    }
    if (g.Z0 == 1) return run_corr<real, 256, 1, 4, 8, EPI>(g, a, st);
    return run_corr<real, 256, 8, 4, 8, EPI>(g, a, st);
}

template <typename real>
int launch_corr_init(const Geom &g, const real *X, const real *D, real *beta,
                     unsigned long long *lmax_bits, cudaStream_t st) {
    CorrArgs<real> a{X, D, beta, nullptr, nullptr, real(0), lmax_bits,
                     g.P, g.K, g.T0, g.T1, g.L0, g.L1, g.Z0, g.Z1, nullptr};
    return corr_dispatch<real, EPI_INIT>(g, a, st);
}

template <typename real>
int launch_corr_refresh(const Geom &g, const real *R, const real *D, const real *Z,
                        const double *nrm, real lambda, real *beta,
                        unsigned long long *maxdz_bits, cudaStream_t st, const int *gate) {
    CorrArgs<real> a{R, D, beta, Z, nrm, lambda, maxdz_bits,
                     g.P, g.K, g.T0, g.T1, g.L0, g.L1, g.Z0, g.Z1, gate};
    return corr_dispatch<real, EPI_REFRESH>(g, a, st);
}

// ------------------------------------------------------------- DtD table
// One CTA per atom pair (k, k2): both atoms are staged in shared memory and
// each thread produces table entries delta = (d0, d1).
template <typename real, int NT>
__global__ void __launch_bounds__(NT) dtd_kernel(const real *D, real *tab, int P, int K, int L0,
                                                 int L1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *Da = reinterpret_cast<real *>(smem_raw);
    const int n = P * L0 * L1;
    real *Db = Da + n;
    const int k = blockIdx.y, k2 = blockIdx.x;
    for (int e = threadIdx.x; e < n; e += NT) {
        Da[e] = D[(size_t)k * n + e];
        Db[e] = D[(size_t)k2 * n + e];
    }
    __syncthreads();
    const int W0 = 2 * L0 - 1, W1 = 2 * L1 - 1;
    for (int w = threadIdx.x; w < W0 * W1; w += NT) {
        const int d0 = w / W1 - (L0 - 1), d1 = w % W1 - (L1 - 1);
        const int a_lo = d0 < 0 ? -d0 : 0, a_hi = d0 > 0 ? L0 - d0 : L0;
        const int b_lo = d1 < 0 ? -d1 : 0, b_hi = d1 > 0 ? L1 - d1 : L1;
        real acc = real(0);
        for (int p = 0; p < P; p++)
            for (int ta = a_lo; ta < a_hi; ta++) {
                const real *ra = Da + ((size_t)p * L0 + ta) * L1;
                const real *rb = Db + ((size_t)p * L0 + ta + d0) * L1 + d1;
                for (int tb = b_lo; tb < b_hi; tb++) acc = fma(ra[tb], rb[tb], acc);
            }
        tab[((size_t)k * K + k2) * W0 * W1 + w] = acc;
    }
}

template <typename real>
int launch_dtd(const Geom &g, const real *D, real *dtd, cudaStream_t st) {
    size_t smem = 2 * (size_t)g.natom() * sizeof(real);
    auto kern = dtd_kernel<real, 256>;
    if (smem > 48 * 1024) {
        if (smem > 227 * 1024) return CSC_ERR_UNIMPLEMENTED;
        CSC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    kern<<<dim3(g.K, g.K), 256, smem, st>>>(D, dtd, g.P, g.K, g.L0, g.L1);
    CSC_CUDA(cudaGetLastError());
    return CSC_OK;
}

// ||D_k||^2 accumulated in FP64 and max_{p,tau} |D_kp[tau]|, one CTA per atom.
template <typename real, int NT>
__global__ void __launch_bounds__(NT) atom_norm_kernel(const real *D, int n, double *nrm,
                                                       double *dmax) {
    const int k = blockIdx.x;
    double s = 0.0, m = 0.0;
    for (int e = threadIdx.x; e < n; e += NT) {
        double v = (double)D[(size_t)k * n + e];
        s += v * v;
        m = fmax(m, fabs(v));
    }
    __shared__ double rs[NT / 32], rm[NT / 32];
    s = warp_sum(s);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) {
        rs[threadIdx.x >> 5] = s;
        rm[threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tm = 0.0;
        for (int w = 0; w < NT / 32; w++) {
            ts += rs[w];
            tm = fmax(tm, rm[w]);
        }
        nrm[k] = ts;
        dmax[k] = tm;
    }
}

template <typename real>
int launch_atom_norms(const Geom &g, const real *D, double *nrm, double *dmax, cudaStream_t st) {
    atom_norm_kernel<real, 256><<<g.K, 256, 0, st>>>(D, (int)g.natom(), nrm, dmax);
    CSC_CUDA(cudaGetLastError());
    return CSC_OK;
}

int preload_functions(const void *const *fns, int n) {
    for (int i = 0; i < n; i++) {
        cudaFuncAttributes fa;
        const cudaError_t e = cudaFuncGetAttributes(&fa, fns[i]);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return CSC_OK;
}

int preload_corr_kernels() {
    const void *fns[] = {
        (const void *)corr_kernel<float, 256, 8, 4, 8, EPI_INIT>,
        (const void *)corr_kernel<float, 256, 1, 4, 8, EPI_INIT>,
        (const void *)corr_kernel<float, 256, 8, 4, 8, EPI_REFRESH>,
        (const void *)corr_kernel<float, 256, 1, 4, 8, EPI_REFRESH>,
        (const void *)corr_rows_kernel<128, 1, 4, 4, EPI_INIT>,
        (const void *)corr_rows_kernel<128, 1, 4, 8, EPI_INIT>,
        (const void *)corr_rows_kernel<128, 1, 4, 10, EPI_INIT>,
        (const void *)corr_rows_kernel<128, 1, 4, 16, EPI_INIT>,
        (const void *)corr_rows_kernel<128, 4, 4, 8, EPI_INIT>,
        (const void *)corr_rows_kernel<128, 4, 4, 13, EPI_INIT>,
        (const void *)corr_rows_kernel<128, 4, 4, 16, EPI_INIT>,
        (const void *)corr_rows_kernel<256, 8, 4, 8, EPI_INIT>,
        (const void *)corr_rows_kernel<256, 8, 4, 13, EPI_INIT>,
        (const void *)corr_rows_kernel<256, 8, 4, 16, EPI_INIT>,
        (const void *)corr_rows_kernel<384, 24, 8, 5, EPI_INIT>,
        (const void *)corr_rows_kernel<128, 1, 4, 4, EPI_REFRESH>,
        (const void *)corr_rows_kernel<128, 1, 4, 8, EPI_REFRESH>,
        (const void *)corr_rows_kernel<128, 1, 4, 10, EPI_REFRESH>,
        (const void *)corr_rows_kernel<128, 1, 4, 16, EPI_REFRESH>,
        (const void *)corr_rows_kernel<128, 4, 4, 8, EPI_REFRESH>,
        (const void *)corr_rows_kernel<128, 4, 4, 13, EPI_REFRESH>,
        (const void *)corr_rows_kernel<128, 4, 4, 16, EPI_REFRESH>,
        (const void *)corr_rows_kernel<256, 8, 4, 8, EPI_REFRESH>,
        (const void *)corr_rows_kernel<256, 8, 4, 13, EPI_REFRESH>,
        (const void *)corr_rows_kernel<256, 8, 4, 16, EPI_REFRESH>,
        (const void *)corr_rows_kernel<384, 24, 8, 5, EPI_REFRESH>,
        (const void *)dtd_kernel<float, 256>,
        (const void *)atom_norm_kernel<float, 256>,
    };
    return preload_functions(fns, (int)(sizeof(fns) / sizeof(fns[0])));
}

#define CSC_INST(real)                                                                         \
    template int launch_corr_init<real>(const Geom &, const real *, const real *, real *,     \
                                        unsigned long long *, cudaStream_t);                  \
    template int launch_corr_refresh<real>(const Geom &, const real *, const real *,          \
                                           const real *, const double *, real, real *,        \
                                           unsigned long long *, cudaStream_t, const int *);  \
    template int launch_dtd<real>(const Geom &, const real *, real *, cudaStream_t);          \
    template int launch_atom_norms<real>(const Geom &, const real *, double *, double *,      \
                                         cudaStream_t);
CSC_INST(float)
CSC_INST(double)
#undef CSC_INST

}  // namespace csc
