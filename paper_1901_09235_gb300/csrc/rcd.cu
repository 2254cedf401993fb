// rcd.cu -- coordinate descent in a given order on one worker: the
// randomized baseline (RCD) of the coordinate-selection comparison (Section
// 5.1, Fig. compare_cd) when the caller draws the order uniformly at random.
//
// For each flat index c = k |Omega| + s of the sequence, in order,
// Z_k[s] <- ST(beta_k[s], lambda) / ||D_k||^2 (Eq. pb_coord), followed by the
// beta update of Eq. beta_update when the value changes.  One CTA walks the
// sequence: the NT coordinates that follow the last applied update are
// evaluated at once, the first of them whose value changes is applied (Z, then
// the beta window, each entry by one thread), and evaluation resumes after it.
// Coordinates evaluated past an applied update are evaluated again, so the
// result is that of one coordinate at a time, in order.  Indices outside
// K x Omega stop the walk and are reported; the walk has a deadline.
#include "common.cuh"

namespace csc {

constexpr int kRcdThreads = 512;

struct RcdArgs {
    float *beta, *Z;
    const float *dtd;
    const double *nrm;
    const unsigned *coords;
    long long n;
    WsHeader *hdr;
    int K, Z0, Z1, L0, L1, W0, W1;
    float lambda;
    unsigned long long timeout_ns;
};

__global__ void __launch_bounds__(kRcdThreads, 1) rcd_kernel(RcdArgs a) {
    constexpr int NW = kRcdThreads / 32;
    extern __shared__ float sn[];  // ||D_k||^2 and its inverse, K each
    __shared__ int s_first[NW], s_stop;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = a.K, WW = a.W0 * a.W1;
    const unsigned plane = (unsigned)a.Z0 * (unsigned)a.Z1;  // positions < 2^31
    const unsigned long long total = (unsigned long long)K * plane;
    for (int k = threadIdx.x; k < K; k += kRcdThreads) {
        sn[k] = (float)a.nrm[k];
        sn[K + k] = (float)(1.0 / a.nrm[k]);
    }
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    long long i = 0, changed = 0;
    int status = 0;
    __syncthreads();
    while (i < a.n) {
        const long long j = i + threadIdx.x;
        bool ch = false;
        if (j < a.n) {
            const unsigned c = a.coords[j];
            if (c < total) {
                const int k = (int)(c / plane);
                const float zn = coord_update(__ldcg(a.beta + c), a.lambda, sn[k], sn[K + k]);
                ch = zn != __ldcg(a.Z + c);
            } else {
                ch = true;  // the walk stops at the first bad index
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ch);
        if (lane == 0) s_first[warp] = bal ? 32 * warp + __ffs(bal) - 1 : kRcdThreads;
        if (threadIdx.x == 0) s_stop = globaltimer_ns() > deadline;
        __syncthreads();
        int first = kRcdThreads;
#pragma unroll
        for (int w = 0; w < NW; w++) first = min(first, s_first[w]);
        const int stop = s_stop;
        __syncthreads();  // s_first and s_stop are written again next round
        if (stop) {
            status = CSC_ERR_TIMEOUT;
            break;
        }
        if (first == kRcdThreads) {  // none of these changes
            i += kRcdThreads;
            continue;
        }
        const long long jf = i + first;
        const unsigned c = a.coords[jf];
        if (c >= total) {
            status = CSC_ERR_INVALID;
            break;
        }
        // every thread evaluates the same coordinate again (same values)
        const int k0 = (int)(c / plane);
        const unsigned s = c - (unsigned)k0 * plane;
        const int i0 = (int)(s / (unsigned)a.Z1), j0 = (int)(s - (unsigned)i0 * (unsigned)a.Z1);
        const float zn = coord_update(__ldcg(a.beta + c), a.lambda, sn[k0], sn[K + k0]);
        const float dz = zn - __ldcg(a.Z + c);
        __syncthreads();  // every read of Z[c] before the write below
        if (threadIdx.x == 0) a.Z[c] = zn;
        // beta_k[s'] -= C[k][k0][s' - s] dz on V(s) within the domain
        for (int q = threadIdx.x; q < K * WW; q += kRcdThreads) {
            const int k = q / WW, r = q - k * WW;
            const int d0 = r / a.W1, d1 = r - d0 * a.W1;
            const int ii = i0 + d0 - (a.L0 - 1), jj = j0 + d1 - (a.L1 - 1);
            if (ii < 0 || ii >= a.Z0 || jj < 0 || jj >= a.Z1) continue;
            if (k == k0 && ii == i0 && jj == j0) continue;
            float *b = a.beta + (size_t)k * plane + (size_t)ii * a.Z1 + jj;
            *b = *b - __ldg(a.dtd + ((size_t)k * K + k0) * WW + r) * dz;
        }
        __syncthreads();
        changed++;
        i = jf + 1;
    }
    if (threadIdx.x == 0) {
        a.hdr->stat[ST_UPDATES] = (unsigned long long)changed;
        a.hdr->stat[ST_ITERS] = (unsigned long long)min(i, a.n);
        a.hdr->stop = status;
    }
}

}  // namespace csc

using namespace csc;

extern "C" int csc_rcd_solve(const csc_shape *shape, const float *D, const float *dtd, float *beta, float *Z,
                             float lambda, const unsigned *coords, long long n, long long *updates_out,
                             void *ws, size_t ws_bytes, csc_stream_t stream) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!D || !dtd || !beta || !Z || !ws || (n > 0 && !coords) || n < 0 || !(lambda >= 0.f))
        return CSC_ERR_INVALID;
    WsLayout L = plan_workspace(g, 0, 4);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *wsb = static_cast<unsigned char *>(ws);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(wsb + L.hdr);
    double *nrm = reinterpret_cast<double *>(wsb + L.nrm), *dmax = reinterpret_cast<double *>(wsb + L.dmax);
    CSC_CUDA(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st));
    if ((rc = launch_atom_norms<float>(g, D, nrm, dmax, st))) return rc;
    RcdArgs a;
    a.beta = beta;
    a.Z = Z;
    a.dtd = dtd;
    a.nrm = nrm;
    a.coords = coords;
    a.n = n;
    a.hdr = hdr;
    a.K = g.K;
    a.Z0 = g.Z0;
    a.Z1 = g.Z1;
    a.L0 = g.L0;
    a.L1 = g.L1;
    a.W0 = g.W0;
    a.W1 = g.W1;
    a.lambda = lambda;
    a.timeout_ns = 60ull * 1000000000ull;
    rcd_kernel<<<1, kRcdThreads, 2 * (size_t)g.K * sizeof(float), st>>>(a);
    CSC_CUDA(cudaGetLastError());
    WsHeader hh;
    {
        const int rb_ = read_back(&hh, hdr, st);
        if (rb_) return rb_;
    }
    if (updates_out) *updates_out = (long long)hh.stat[ST_UPDATES];
    return hh.stop;
}
