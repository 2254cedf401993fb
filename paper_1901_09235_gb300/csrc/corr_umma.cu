// corr_umma.cu -- beta = D~ * X (Alg. 1 initialisation) as an implicit GEMM
// on the 5th-generation tensor cores, with split-bf16 products (bf16 x 3).
//
//   beta_k[s0][s1] = sum_p sum_tau0 sum_tau1 D_kp[tau0][tau1] X_p[s0 + tau0][s1 + tau1]
//
// GEMM view of one tile (one row s0 of the activation domain, 128
// consecutive s1): rows m = s1 - s1_0 (M = 128), columns n = atom k (N = K
// rounded up to 16), reduction over r = (p, tau0, tau1) with tau1 padded to
// a multiple of 16 (zero taps).  For a fixed (p, tau0) the A operand
// A[m][tau1] = X_p[s0 + tau0][s1_0 + m + tau1] is a Hankel matrix, so the
// 8 x 8 core matrix (row group g, tap group h) depends only on g + h: only the
// 16 + L1/8 distinct core matrices of each (p, tau0) are stored, and the
// operand descriptor addresses core g + h by giving both strides (LBO, SBO)
// the spacing of the stored core matrices.
//
// Precision: x = x_hi + x_lo with x_hi = bf16(x), x_lo = bf16(x - x_hi); the
// products x_hi d_hi + x_hi d_lo + x_lo d_hi accumulate in FP32 in tensor
// memory.  The dropped and rounded parts are below (2^-18 + 2^-17) |x||d|
// per product.
//
// Each CTA (128 threads = the 128 TMEM lanes of the accumulator) keeps the
// split dictionary in shared memory and loops over tiles; the A operand is
// built in chunks of (p, tau0) pairs into two buffers, so building one chunk
// overlaps the MMAs of the other.  One thread issues tcgen05.mma and commits
// each chunk to the buffer's mbarrier; every wait is bounded and sets an
// error word when it gives up.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"

namespace csc {

struct UmmaCorrArgs {
    const float *X, *D;
    float *beta;
    unsigned *lmax_bits;  // max |beta| as float bits (atomicMax)
    int *err;             // non-zero when a wait gave up
    int P, K, T0, T1, L0, L1, Z0, Z1;
    int Np, L1p, R, NC, CH, NS, npairs, nchunk, tiles_row, ntiles, tmem_cols;
    unsigned long long spin_limit;
};

// Eight warps, so that at most two sit on one SM sub-partition (each of the
// four has a quarter of the register file): the kernel then still fits beside
// a persistent kernel that holds half of every sub-partition's registers.
constexpr int kUmmaBuilders = 224;                 // warps 0-6: operand builders
constexpr int kUmmaThreads = kUmmaBuilders + 32;   // warp 7: MMA issuer
constexpr int kUmmaIssuer = kUmmaBuilders / 32;
constexpr int kUmmaEpi = 128;                      // warps 0-3: epilogue (one per TMEM lane quarter)
constexpr int kUmmaMaxStages = 4;
// Core matrices of the A operand are 144 bytes apart (128 + 16): the 32 lanes
// that each write a 16-byte row of their own core then hit every bank group
// (a 128-byte spacing would put all of them on the same four banks).
constexpr int kCoreStride = 144;

__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // start >> 4 [0,14), LBO >> 4 [16,30), SBO >> 4 [32,46), version 1 [46,48),
    // no swizzle (layout type 0)
    return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// Bounded wait for the phase of the given parity of an mbarrier; gives up
// (false) after `limit` polls or when another role has set the abort word.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, unsigned long long limit,
                                          volatile int *abort) {
    for (unsigned long long it = 0; it < limit; it++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255) == 255 && *abort) return false;
    }
    *abort = 1;
    return false;
}

// Split x into bf16 x_hi + x_lo and return both as packed pairs.
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
    const __nv_bfloat16 al = __float2bfloat16_rn(a - __bfloat162float(ah));
    const __nv_bfloat16 bl = __float2bfloat16_rn(b - __bfloat162float(bh));
    hi = (uint32_t)__bfloat16_as_ushort(ah) | ((uint32_t)__bfloat16_as_ushort(bh) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(al) | ((uint32_t)__bfloat16_as_ushort(bl) << 16);
}

__global__ void __launch_bounds__(kUmmaThreads, 1) corr_umma_kernel(UmmaCorrArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[kUmmaMaxStages], empty[kUmmaMaxStages], accfull[2], accempty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_word;
    volatile int *abort = &abort_word;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // dynamic shared memory: B = [D_hi; D_lo] (2 Np x R), then NS stages of (A_hi, A_lo)
    const size_t bbytes = (size_t)a.Np * a.R * 2;
    const size_t abytes = (size_t)a.CH * a.NC * kCoreStride;
    unsigned char *sB = smem_raw;
    unsigned char *sA = smem_raw + 2 * bbytes;
    const uint32_t sbo_b = (uint32_t)(a.R / 8) * 128u;
    const size_t plane = (size_t)a.Z0 * a.Z1;

    // split dictionary, rows n < Np the hi parts and rows Np + n the lo parts:
    // element (row, r) at (row / 8) SBO_B + (r / 8) 128 + (row % 8) 16 + (r % 8) 2
    for (int e = tid; e < a.Np * (a.R / 2); e += kUmmaThreads) {
        const int n = e / (a.R / 2), r = 2 * (e % (a.R / 2));
        float v[2];
        for (int u = 0; u < 2; u++) {
            const int rr = r + u, q = rr / a.L1p, t1 = rr % a.L1p;  // q = p * L0 + tau0
            const int p = q / a.L0, t0 = q % a.L0;
            v[u] = (n < a.K && t1 < a.L1) ? a.D[(((size_t)n * a.P + p) * a.L0 + t0) * a.L1 + t1] : 0.f;
        }
        uint32_t hi, lo;
        split_bf16x2(v[0], v[1], hi, lo);
        const size_t off = (size_t)(n / 8) * sbo_b + (size_t)(r / 8) * 128 + (n % 8) * 16 + (r % 8) * 2;
        *reinterpret_cast<uint32_t *>(sB + off) = hi;
        *reinterpret_cast<uint32_t *>(sB + bbytes + off) = lo;  // row Np + n (Np multiple of 8)
    }
    if (tid == 0) {
        abort_word = 0;
        for (int i = 0; i < a.NS; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(&full[i])),
                         "r"(kUmmaBuilders)
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&empty[i]))
                         : "memory");
        }
        for (int i = 0; i < 2; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&accfull[i]))
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(&accempty[i])),
                         "r"(kUmmaEpi)
                         : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kUmmaIssuer) {
        const uint32_t slot = (uint32_t)__cvta_generic_to_shared(&tmem_slot);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const int my_tiles = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int acc_cols = a.tmem_cols / 2;  // two accumulators side by side

    if (warp == kUmmaIssuer) {
        // ================================================ MMA issuer (one thread)
        if (lane == 0) {
            // A_hi x [D_hi; D_lo] (N = 2 Np) and A_lo x D_hi (N = Np), FP32 accumulators
            const uint32_t idesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(2 * a.Np >> 3) << 17) | (8u << 24);
            const uint32_t idesc1 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a.Np >> 3) << 17) | (8u << 24);
            const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(sB);
            const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(sA);
            // descriptors advance by (byte offset) / 16 in the start-address field
            const uint64_t bdesc0 = umma_smem_desc(b0, 128, sbo_b);
            int seq = 0;
            for (int i = 0; i < my_tiles && !*abort; i++) {
                const int acc = i & 1;
                // the epilogue of the tile that last used this accumulator is done
                if (i >= 2 && !mbar_wait((uint32_t)__cvta_generic_to_shared(&accempty[acc]), ((i >> 1) - 1) & 1,
                                         a.spin_limit, abort))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dt = tmem + (uint32_t)(acc * acc_cols);
                for (int c = 0; c < a.nchunk; c++, seq++) {
                    const int st = seq % a.NS, use = seq / a.NS;
                    if (!mbar_wait((uint32_t)__cvta_generic_to_shared(&full[st]), use & 1, a.spin_limit, abort))
                        break;
                    const uint32_t ah0 = a0 + (uint32_t)(st * 2 * abytes);
                    const uint64_t ahd0 = umma_smem_desc(ah0, kCoreStride, kCoreStride);
                    const uint64_t ald0 = ahd0 + (uint64_t)(abytes >> 4);
                    const int q0 = c * a.CH, nq = min(a.CH, a.npairs - q0);
                    const int nt = a.L1p / 16;
                    for (int ql = 0; ql < nq; ql++) {
                        const uint64_t aq = (uint64_t)(ql * a.NC * (kCoreStride / 16));
                        const uint64_t bq = (uint64_t)((q0 + ql) * a.L1p);           // ((q L1p / 8) 128) / 16
                        for (int t = 0; t < nt; t++) {
                            const uint64_t ad = aq + (uint64_t)(2 * t * (kCoreStride / 16)), bd = bq + (uint64_t)(16 * t);
                            umma_bf16(dt, ahd0 + ad, bdesc0 + bd, idesc2, (c == 0 && ql == 0 && t == 0) ? 0u : 1u);
                            umma_bf16(dt, ald0 + ad, bdesc0 + bd, idesc1, 1u);
                        }
                    }
                    umma_commit((uint32_t)__cvta_generic_to_shared(&empty[st]));  // stage free when done
                }
                umma_commit((uint32_t)__cvta_generic_to_shared(&accfull[acc]));  // tile done
            }
        }
        __syncwarp();
    } else {
        // ===================================== operand builders and epilogue
        float lmax = 0.f;
        int seq = 0;
        auto epilogue = [&](int i) -> bool {
            if (warp >= kUmmaEpi / 32) return true;
            const int tile = (int)blockIdx.x + i * (int)gridDim.x;
            const int s0 = tile / a.tiles_row, s1_0 = (tile % a.tiles_row) * 128, acc = i & 1;
            if (!mbar_wait((uint32_t)__cvta_generic_to_shared(&accfull[acc]), (i >> 1) & 1, a.spin_limit, abort))
                return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int quarter = warp;
            const int m = 32 * quarter + lane, s1 = s1_0 + m;
            for (int n0 = 0; n0 < a.Np; n0 += 16) {
                uint32_t v[16], w[16];
                const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(acc * acc_cols + n0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                    "%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr)
                    : "memory");
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                    "%15}, [%16];"
                    : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
                      "=r"(w[7]), "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]),
                      "=r"(w[14]), "=r"(w[15])
                    : "r"(taddr + (uint32_t)a.Np)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (s1 < a.Z1) {
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const int k = n0 + j;
                        if (k < a.K) {
                            const float b = __uint_as_float(v[j]) + __uint_as_float(w[j]);
                            a.beta[(size_t)k * plane + (size_t)s0 * a.Z1 + s1] = b;
                            lmax = fmaxf(lmax, fabsf(b));
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive((uint32_t)__cvta_generic_to_shared(&accempty[acc]));
            return true;
        };
        // the core matrix this thread builds in a chunk (at most one: CH NC <= 224)
        // comes from X_p[s0 + tau0][col0 .. col0 + 15], col0 = s1_0 + 8 cc; rows
        // rr = 0..7 hold elements rr .. rr + 7.  The values of the next chunk's
        // core are loaded before waiting for its stage.
        auto load_core = [&](int tile, int c, float *v) -> bool {
            const int q0 = c * a.CH, nq = min(a.CH, a.npairs - q0);
            if (tid >= nq * a.NC) return false;
            const int s0 = tile / a.tiles_row, s1_0 = (tile % a.tiles_row) * 128;
            const int ql = tid / a.NC, cc = tid % a.NC;
            const int q = q0 + ql, p = q / a.L0, t0 = q % a.L0;
            const float *xr = a.X + ((size_t)p * a.T0 + (s0 + t0)) * a.T1;
            const int col0 = s1_0 + 8 * cc;
            if (col0 + 16 <= a.T1 && ((a.T1 & 3) == 0)) {
                const float4 *x4 = reinterpret_cast<const float4 *>(xr + col0);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const float4 f = __ldg(x4 + u);
                    v[4 * u] = f.x;
                    v[4 * u + 1] = f.y;
                    v[4 * u + 2] = f.z;
                    v[4 * u + 3] = f.w;
                }
            } else {
#pragma unroll
                for (int u = 0; u < 16; u++) v[u] = (col0 + u < a.T1) ? __ldg(xr + col0 + u) : 0.f;
            }
            return true;
        };
        bool ok = true;
        float vn[16];
        bool have = my_tiles > 0 ? load_core((int)blockIdx.x, 0, vn) : false;
        for (int i = 0; i < my_tiles && ok; i++) {
            const int tile = (int)blockIdx.x + i * (int)gridDim.x;
            for (int c = 0; c < a.nchunk; c++, seq++) {
                const int st = seq % a.NS, use = seq / a.NS;
                float v[16];
                const bool mine = have;
#pragma unroll
                for (int u = 0; u < 16; u++) v[u] = vn[u];
                // next chunk (or the next tile's first chunk)
                if (c + 1 < a.nchunk) have = load_core(tile, c + 1, vn);
                else if (i + 1 < my_tiles) have = load_core(tile + (int)gridDim.x, 0, vn);
                else have = false;
                if (use > 0 &&
                    !mbar_wait((uint32_t)__cvta_generic_to_shared(&empty[st]), (use - 1) & 1, a.spin_limit, abort)) {
                    ok = false;
                    break;
                }
                if (mine) {
                    unsigned char *ch = sA + (size_t)st * 2 * abytes + (size_t)tid * kCoreStride, *cl = ch + abytes;
                    // pairs (2m, 2m + 1) of the hi and lo parts, then (2m + 1, 2m + 2)
                    uint32_t eh[8], el[8], oh[7], ol[7];
#pragma unroll
                    for (int m = 0; m < 8; m++) split_bf16x2(v[2 * m], v[2 * m + 1], eh[m], el[m]);
#pragma unroll
                    for (int m = 0; m < 7; m++) {
                        oh[m] = __byte_perm(eh[m], eh[m + 1], 0x5432);
                        ol[m] = __byte_perm(el[m], el[m + 1], 0x5432);
                    }
#pragma unroll
                    for (int r2 = 0; r2 < 4; r2++) {
                        // row 2 r2 from the even pairs, row 2 r2 + 1 from the odd ones
                        *reinterpret_cast<uint4 *>(ch + (2 * r2) * 16) = make_uint4(eh[r2], eh[r2 + 1], eh[r2 + 2], eh[r2 + 3]);
                        *reinterpret_cast<uint4 *>(cl + (2 * r2) * 16) = make_uint4(el[r2], el[r2 + 1], el[r2 + 2], el[r2 + 3]);
                        *reinterpret_cast<uint4 *>(ch + (2 * r2 + 1) * 16) = make_uint4(oh[r2], oh[r2 + 1], oh[r2 + 2], oh[r2 + 3]);
                        *reinterpret_cast<uint4 *>(cl + (2 * r2 + 1) * 16) = make_uint4(ol[r2], ol[r2 + 1], ol[r2 + 2], ol[r2 + 3]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive((uint32_t)__cvta_generic_to_shared(&full[st]));
            }
            // the previous tile's results while this tile's MMAs run
            if (ok && i > 0) ok = epilogue(i - 1);
        }
        if (ok && my_tiles > 0) ok = epilogue(my_tiles - 1);
        const unsigned lb = __reduce_max_sync(0xffffffffu, __float_as_uint(lmax));
        if (lane == 0 && a.lmax_bits) atomicMax(a.lmax_bits, lb);
    }
    __syncthreads();
    if (tid == 0 && *abort) atomicExch(a.err, 1);
    // after an abort, wait (bounded) for commits still in flight before TMEM is freed
    if (tid == 0 && *abort) {
        for (int i = 0; i < 2; i++) {
            const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&accfull[i]);
            for (int it = 0; it < 1 << 16; it++) {
                uint32_t d0, d1;
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(d0) : "r"(mb), "r"(0) : "memory");
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(d1) : "r"(mb), "r"(1) : "memory");
                if (d0 || d1) break;
                __nanosleep(1000);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kUmmaIssuer)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                     : "memory");
}

// The dynamic shared-memory limit of the kernel, raised once to the device's
// opt-in maximum (the launch still asks only for what its plan needs).  Set
// before a persistent kernel starts, so that no attribute call is made while
// it runs.
static int umma_set_smem_limit() {
    static int done_dev = -1;
    int dev = 0, optin = 0;
    CSC_CUDA(cudaGetDevice(&dev));
    if (done_dev == dev) return CSC_OK;
    CSC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    CSC_CUDA(cudaFuncGetAttributes(&fa, (const void *)corr_umma_kernel));
    CSC_CUDA(cudaFuncSetAttribute(corr_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - (int)fa.sharedSizeBytes));
    CSC_CUDA(cudaFuncSetAttribute(corr_umma_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared));
    done_dev = dev;
    return CSC_OK;
}

int preload_umma_kernels() {
    const void *fns[] = {(const void *)corr_umma_kernel};
    const int rc = preload_functions(fns, 1);
    return rc ? rc : umma_set_smem_limit();
}

}  // namespace csc

using namespace csc;

// Host side: plan and launch.  Returns CSC_ERR_UNIMPLEMENTED when the split
// dictionary and two A chunks do not fit in shared memory.
static int umma_plan(const Geom &g, UmmaCorrArgs &a, size_t *smem) {
    a.P = g.P;
    a.K = g.K;
    a.T0 = g.T0;  // 1-D problems are rows of a 2-D one (T0 = L0 = 1)
    a.T1 = g.T1;
    a.L0 = g.L0;
    a.L1 = g.L1;
    a.Z0 = g.Z0;
    a.Z1 = g.Z1;
    a.Np = (int)ceil_div(g.K, 16) * 16;
    a.L1p = (int)ceil_div(a.L1, 16) * 16;
    a.npairs = a.P * a.L0;
    a.R = a.npairs * a.L1p;
    a.NC = 16 + a.L1p / 8;
    a.tiles_row = (int)ceil_div(a.Z1, 128);
    a.ntiles = a.Z0 * a.tiles_row;
    int cols = 32;
    while (cols < 4 * a.Np) cols *= 2;  // two accumulators of 2 Np columns (hi and lo parts)
    a.tmem_cols = cols;
    if (2 * a.Np > 256 || cols > 512) return CSC_ERR_UNIMPLEMENTED;
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t bbytes = (size_t)a.Np * a.R * 2;
    const size_t static_reserve = 1024;
    // the most pairs per chunk (up to 8), then the most stages (2..4), that fit
    for (int ch = std::min(a.npairs, std::min(8, kUmmaBuilders / a.NC)); ch >= 1; ch--) {
        for (int ns = kUmmaMaxStages; ns >= 2; ns--) {
            const size_t need = 2 * bbytes + 2 * (size_t)ns * ch * a.NC * kCoreStride;
            if (need + static_reserve <= (size_t)optin) {
                a.CH = ch;
                a.NS = ns;
                a.nchunk = (int)ceil_div(a.npairs, ch);
                *smem = need;
                return CSC_OK;
            }
        }
    }
    return CSC_ERR_UNIMPLEMENTED;
}

extern "C" int csc_init_beta_bf16x3(const csc_shape *shape, const float *X, const float *D, float *beta,
                                    float *dtd, double *lambda_max_out, void *ws, size_t ws_bytes,
                                    csc_stream_t stream) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!X || !D || !beta || !dtd || !ws) return CSC_ERR_INVALID;
    WsLayout L = plan_workspace(g, 0, 4);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
    UmmaCorrArgs a{};
    size_t smem = 0;
    rc = umma_plan(g, a, &smem);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *wsb = static_cast<unsigned char *>(ws);
    WsHeader *h = reinterpret_cast<WsHeader *>(wsb + L.hdr);
    a.X = X;
    a.D = D;
    a.beta = beta;
    a.lmax_bits = reinterpret_cast<unsigned *>(&h->lmax_bits);
    a.err = &h->overflow;
    a.spin_limit = 1ull << 24;
    CSC_CUDA(cudaMemsetAsync(&h->lmax_bits, 0, sizeof(h->lmax_bits), st));
    CSC_CUDA(cudaMemsetAsync(&h->overflow, 0, sizeof(int), st));
    if ((rc = umma_set_smem_limit())) return rc;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(a.ntiles, sms));
    corr_umma_kernel<<<grid, kUmmaThreads, smem, st>>>(a);
    CSC_CUDA(cudaGetLastError());
    // the D^T D table and the atom norms: the FP32 path
    rc = launch_dtd<float>(g, D, dtd, st);
    if (rc) return rc;
    if (lambda_max_out) {
        unsigned bits = 0;
        int err = 0;
        if ((rc = read_back(&bits, &h->lmax_bits, st))) return rc;
        if ((rc = read_back(&err, &h->overflow, st))) return rc;
        if (err) return CSC_ERR_TIMEOUT;
        float f;
        memcpy(&f, &bits, 4);
        *lambda_max_out = f;
    }
    return CSC_OK;
}
