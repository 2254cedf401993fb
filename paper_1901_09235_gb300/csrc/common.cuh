// common.cuh -- internal helpers of the sm_103a CSC library: geometry,
// workspace layout, status plumbing and small device primitives (scoped
// loads/stores, the global timer, warp/block reductions).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/dicodile_gb.h"

namespace csc {

// ----------------------------------------------------------------- geometry
// Every computation works on a 2-D view: a 1-D signal is one row
// (T0 = L0 = 1).  Z0 x Z1 is the valid activation domain, W0 x W1 the window
// prod [-L_i + 1, L_i[ of Eq. beta_update.
struct Geom {
    int d, P, K;
    int T0, T1, L0, L1;
    int Z0, Z1, W0, W1;
    long long nx() const { return (long long)P * T0 * T1; }
    long long nz() const { return (long long)K * Z0 * Z1; }
    long long nzpos() const { return (long long)Z0 * Z1; }
    long long natom() const { return (long long)P * L0 * L1; }
    long long nd() const { return (long long)K * natom(); }
    long long nw() const { return (long long)W0 * W1; }
    long long ntab() const { return (long long)K * K * nw(); }
};

// Validates a public shape and builds the 2-D view.  Returns CSC_OK or
// CSC_ERR_INVALID.
int make_geom(const csc_shape *s, Geom *g);

// ------------------------------------------------------------- workspace
// Device-side control block at the start of every workspace.  Contended
// words sit on their own 128-byte lines.
struct alignas(128) WsHeader {
    int pending;            // active workers + messages in flight (termination)
    int pad0[31];
    int stop;               // 0 = running, else a csc_status that stops every worker
    int pad1[31];
    unsigned int bar_count; // grid barrier arrivals
    int pad2[31];
    unsigned int bar_gen;   // grid barrier generation
    int pad3[31];
    int round_applied[2];   // phased mode: updates applied in the current round
    int pad4[30];
    unsigned long long updates_total;  // global update count (max_updates check)
    int pad5[30];
    long long stat[8];      // updates, iterations, rejected, subtol, messages, deferred, candidates
    unsigned long long wmax[2];        // largest per-worker iteration / update counts
    unsigned long long tmax[4];        // worker timeline (ns after its start): last update, exit, first pause; wake-ups
    unsigned long long tph[6];         // SM cycles per wave phase, summed over workers
    unsigned long long lmax_bits;      // max |beta| (as bits of a non-negative float/double)
    unsigned long long maxdz_bits;     // max |dZ| on a fresh beta
    long long nnz;          // compacted nonzeros of Z (may exceed the capacity)
    int overflow;           // nnz exceeded the list capacity
    int status;             // final status of the last solve launch
    double obj_f;           // sum of squared residuals
    double obj_g;           // sum |Z|
    double pgd_out[12];     // dictionary step: objective, iterations, last step, spare, phase cycles [4..9]
    int scan_total;         // deterministic compaction: total count
    int pad6a;
    double xsq;             // ||X||^2 when a call computes it on the device
    int pad6[12];
    unsigned long long tphmax[8];      // largest per-worker SM cycles per phase
};

enum StatIdx { ST_UPDATES = 0, ST_ITERS, ST_REJECTED, ST_SUBTOL, ST_MESSAGES, ST_DEFERRED, ST_CAND };

constexpr int kMailboxCap = 512;    // records per directed neighbour link
constexpr int kDirs = 8;            // neighbour directions in a 2-D tile grid

struct WsLayout {
    size_t hdr, nrm, dmax, nnz_k, nnz_s, nnz_z, blk, r64, rr, phi64, psi64, pgd, mbox_slots,
        mbox_ctl, total, beta0, total_beta0;  // beta0: optional region up to total_beta0
    // inside the optional region, after beta0: the rebuilt-beta gather's bin
    // offsets and cursors, its binned nonzero list and the transposed table
    size_t gbin, glist, gtab;
    int gbh, gbw, gnb0, gnb1, gkp;  // bin rows / columns, bins per dimension, padded K
    // and the table in the window layout of the staged window update: K x K
    // blocks [k0][k] of wbs floats, W0 rows of wrs floats each
    size_t wtab;
    int wrs, wbs;
    long long nnz_cap;
    int max_workers;
    int blk_cap;
};

// Byte layout of the workspace for a geometry (element size of the solve's
// real type `rs`, 4 or 8).  Every region is 256-byte aligned.
WsLayout plan_workspace(const Geom &g, int max_workers, int rs);

// ------------------------------------------------------- status plumbing
int set_cuda_error(cudaError_t e);
#define CSC_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return set_cuda_error(e_); \
    } while (0)

// -------------------------------------------------------- device helpers
__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_acquire_u(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_u(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ float ld_relaxed(const float *p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ double ld_relaxed(const double *p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(float *p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(double *p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Order-preserving bits of a non-negative value (for atomicMax).
__device__ __forceinline__ unsigned long long nonneg_bits(float v) {
    return (unsigned long long)__float_as_uint(v);
}
__device__ __forceinline__ unsigned long long nonneg_bits(double v) {
    return (unsigned long long)__double_as_longlong(v);
}

// Soft-thresholding ST(u, lambda) = sign(u) max(|u| - lambda, 0) (Section 2).
template <typename real>
__device__ __forceinline__ real soft_threshold(real u, real lam) {
    return u > lam ? u - lam : (u < -lam ? u + lam : real(0));
}

// b - c * t with the rounding of the written expression.  In FP64 the
// product and the difference are rounded separately (no contraction) so the
// verification build reproduces a plain sequential evaluation; in FP32 the
// fused form is used.
__device__ __forceinline__ double sub_prod(double b, double c, double t) {
    return __dsub_rn(b, __dmul_rn(c, t));
}
__device__ __forceinline__ float sub_prod(float b, float c, float t) { return fmaf(-c, t, b); }

// Z' = ST(beta, lambda) / ||D_k||^2 (Eq. pb_coord).  FP64 divides (the
// rounding of the definition); FP32 multiplies by the stored reciprocal.
// The product is rounded on its own (never contracted into a following
// subtraction), so |Z' - Z| has the same bits wherever it is evaluated: the
// owner of a coordinate and a neighbour running the soft-lock test must
// agree exactly, or a tie between two border candidates is rejected on both
// sides and neither worker ever updates again.
__device__ __forceinline__ double coord_update(double beta, double lam, double nrm, double inv) {
    (void)inv;
    return __ddiv_rn(soft_threshold(beta, lam), nrm);
}
__device__ __forceinline__ float coord_update(float beta, float lam, float nrm, float inv) {
    (void)nrm;
    return __fmul_rn(soft_threshold(beta, lam), inv);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Block-wide sum into *out via one FP64 atomic per block.
template <int NT>
__device__ __forceinline__ void block_sum_atomic(double v, double *out) {
    __shared__ double red[NT / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0 && s != 0.0) atomicAdd(out, s);
    }
}

template <int NT>
__device__ __forceinline__ void block_max_atomic(unsigned long long v, unsigned long long *out) {
    __shared__ unsigned long long red[NT / 32];
    v = warp_max_u64(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long s = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0ull;
        s = warp_max_u64(s);
        if (threadIdx.x == 0 && s != 0ull) atomicMax(out, s);
    }
}

inline long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

// ------------------------------------------------ launchers (per .cu file)
template <typename real>
int launch_corr_init(const Geom &g, const real *X, const real *D, real *beta,
                     unsigned long long *lmax_bits, cudaStream_t st);
template <typename real>
int launch_corr_refresh(const Geom &g, const real *R, const real *D, const real *Z,
                        const double *nrm, real lambda, real *beta,
                        unsigned long long *maxdz_bits, cudaStream_t st, const int *gate = nullptr);
template <typename real>
int launch_dtd(const Geom &g, const real *D, real *dtd, cudaStream_t st);

// Small host <-> device transfers (scalars read back, control records) go
// through one pinned host buffer per host thread, allocated on first use and
// kept for the thread's lifetime (never freed: freeing pinned memory can wait
// for the whole device).  A copy to or from pageable memory costs hundreds of
// microseconds on this platform, a pinned one a few.
constexpr size_t kPinnedScratch = 8192;
void *pinned_scratch();  // kPinnedScratch bytes, or nullptr when it cannot be allocated

// dst <- *src_dev (device), then the stream is synchronised
template <typename T>
int read_back(T *dst, const void *src_dev, cudaStream_t st) {
    static_assert(sizeof(T) <= kPinnedScratch, "small transfers only");
    void *s = pinned_scratch();
    if (s) {
        CSC_CUDA(cudaMemcpyAsync(s, src_dev, sizeof(T), cudaMemcpyDeviceToHost, st));
        CSC_CUDA(cudaStreamSynchronize(st));
        memcpy(dst, s, sizeof(T));
    } else {
        CSC_CUDA(cudaMemcpyAsync(dst, src_dev, sizeof(T), cudaMemcpyDeviceToHost, st));
        CSC_CUDA(cudaStreamSynchronize(st));
    }
    return CSC_OK;
}

// Load the FP32 kernels of beta-init / refresh / objective (and the tensor-core
// beta-init) into the context now.  With lazy module loading a kernel is
// loaded on its first launch, and that load may wait for the kernels already
// running: a first launch beside a persistent kernel would then stall until
// the persistent kernel ends.
int preload_corr_kernels();
// Queues whose persistent kernel is running (created and not yet closed).
// Kernels launched beside one must fit the registers it leaves free on each
// SM sub-partition; the 2-D FP32 correlations then take their smaller shape.
int live_queues();
int preload_residual_kernels();
int preload_umma_kernels();
int preload_functions(const void *const *fns, int n);
template <typename real>
int launch_atom_norms(const Geom &g, const real *D, double *nrm, double *dmax, cudaStream_t st);

// Residual / objective / KKT on the current Z (writes beta recomputed from
// scratch when `beta` is non-null).  Leaves obj_f, obj_g, maxdz_bits, nnz in
// the header.  With `dtd` given (FP32 only), beta is rebuilt from the initial
// beta kept in the workspace's beta0 region: beta0 minus C * Z over the
// nonzero list (the correlation of the residual when the list overflowed).
template <typename real>
int launch_refresh(const Geom &g, const WsLayout &L, unsigned char *ws, const real *X,
                   const real *D, const real *Z, real lambda, real *beta, cudaStream_t st,
                   const real *dtd = nullptr);

template <typename real>
int solve_impl(const csc_shape *shape, const real *X, const real *D, const real *dtd, real *beta,
               real *Z, real lambda, real tol, const csc_solve_opts *opts, void *ws,
               size_t ws_bytes, csc_solve_stats *stats, cudaStream_t st);

int dict_stats_impl(const Geom &g, const float *Z, const float *X, float *phi, float *psi,
                    unsigned char *ws, const WsLayout &L, cudaStream_t st);
// x_sqnorm_dev (optional): ||X||^2 in device memory, read by the kernel in
// place of x_sqnorm.  gate (optional): when *gate > gate_cap at run time the
// step leaves D unchanged (statistics that were not computed).
int dict_update_impl(const Geom &g, const float *phi, const float *psi, double x_sqnorm, float *D,
                     int max_iter, double tol, double *obj_out, int *it_out, unsigned char *ws,
                     const WsLayout &L, cudaStream_t st, const double *x_sqnorm_dev = nullptr,
                     const int *gate = nullptr, int gate_cap = 0);

}  // namespace csc
