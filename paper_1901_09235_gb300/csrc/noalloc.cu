// noalloc.cu -- the dictionary-update statistics (phi, psi) for callers that
// cannot hand the library a workspace.
//
// Some callers have no way to allocate device memory when they need these
// statistics: for example a plugin running inside a host application that owns
// every device allocation through its own pool, or a service that reserves all
// of its device memory at start-up and forbids any later allocation.  For them
// this entry point uses a fixed scratch area that lives in the library itself
// (a file-scope __device__ array of CSC_NOALLOC_SCRATCH_BYTES on every GPU that
// loads the library, held until the process exits) instead of a caller
// workspace.  It calls no allocator: no cudaMalloc / cudaFree and no library
// routine that allocates.
//
// The array's device address is looked up once per device with
// cudaGetSymbolAddress, on the first call made while that device is current;
// in host code the array's name is only a stand-in and must never be passed to
// a kernel.  All calls share the one array and it keeps whatever the previous
// call left there, so everything that must start at zero is cleared by each
// call; two calls whose work overlaps on the GPU (for example on two streams)
// race on it.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace csc {

constexpr size_t kNoAllocScratchBytes = CSC_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mutex;
static void *g_noalloc_addr[kMaxDevices];

// Device address of the scratch array on the current device (looked up once).
static int noalloc_scratch(unsigned char **out) {
    int dev = 0;
    CSC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return CSC_ERR_UNIMPLEMENTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        CSC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_noalloc_addr[dev]);
    return CSC_OK;
}

// Layout of the statistics' scratch inside the fixed array: the control
// header, the nonzero list, the compaction block counts and the FP64
// accumulators of phi and psi (the same sizes the workspace form uses).
static WsLayout noalloc_layout(const Geom &g) {
    WsLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return at;
    };
    L.nnz_cap = std::min<long long>(g.nz(), std::max<long long>(1ll << 16, g.nz() / 16));
    L.blk_cap = (int)ceil_div(g.nzpos(), 256) + 1;
    L.hdr = take(sizeof(WsHeader));
    L.nnz_k = take((size_t)L.nnz_cap * sizeof(int));
    L.nnz_s = take((size_t)L.nnz_cap * sizeof(int));
    L.nnz_z = take((size_t)L.nnz_cap * sizeof(float));
    L.blk = take(2 * (size_t)L.blk_cap * sizeof(int));
    L.phi64 = take((size_t)g.ntab() * sizeof(double));
    L.psi64 = take((size_t)g.nd() * sizeof(double));
    L.total = off;
    return L;
}

}  // namespace csc

using namespace csc;

extern "C" int cdl_dict_stats_noalloc(const csc_shape *shape, const float *Z, const float *X, float *phi,
                                      float *psi, csc_stream_t stream) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!Z || !X || !phi || !psi) return CSC_ERR_INVALID;
    const WsLayout L = noalloc_layout(g);
    if (L.total > kNoAllocScratchBytes) return CSC_ERR_WORKSPACE;
    unsigned char *ws = nullptr;
    rc = noalloc_scratch(&ws);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // the previous call's header is still there: clear it
    CSC_CUDA(cudaMemsetAsync(ws + L.hdr, 0, sizeof(WsHeader), st));
    return dict_stats_impl(g, Z, X, phi, psi, ws, L, st);
}
