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
// The array's device address is looked up with cudaGetSymbolAddress on the
// first call made while a device is current, and again whenever that
// device's context has changed since (a cudaDeviceReset, or a primary context
// released and created anew, gives the array a new address); in host code
// the array's name is only a stand-in and must never be passed to a kernel.
// All calls share the one array and it keeps whatever the previous call left
// there, so everything that must start at zero is cleared by each call; two
// calls whose work overlaps on the GPU (for example on two streams) race on
// it.
#include <cuda.h>  // context handle types only; the driver is reached through the runtime

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace csc {

constexpr size_t kNoAllocScratchBytes = CSC_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mutex;
struct NoAllocAddr {
    unsigned long long ctx_id;  // the context the address belongs to (0: none yet)
    void *addr;
};
static NoAllocAddr g_noalloc_addr[kMaxDevices];

// Unique id of the calling thread's current context (0 when there is none),
// through the driver entry points the runtime hands out (no driver library
// is linked).
static int current_context_id(unsigned long long *id) {
    typedef CUresult (*GetCurrentFn)(CUcontext *);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        CSC_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1));
        CSC_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return CSC_ERR_UNIMPLEMENTED;
        get_current = reinterpret_cast<GetCurrentFn>(f1);
        get_id = reinterpret_cast<GetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    *id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS) return CSC_ERR_CUDA;
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return CSC_ERR_CUDA;
    return CSC_OK;
}

// Device address of the scratch array in the current device's current
// context (looked up once per context).
static int noalloc_scratch(unsigned char **out) {
    int dev = 0;
    CSC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return CSC_ERR_UNIMPLEMENTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    unsigned long long id = 0;
    int rc = current_context_id(&id);
    if (rc) return rc;
    NoAllocAddr &e = g_noalloc_addr[dev];
    if (id == 0 || e.ctx_id != id || !e.addr) {
        void *p = nullptr;
        CSC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));  // makes the runtime's context current
        if ((rc = current_context_id(&id))) return rc;
        e.ctx_id = id;
        e.addr = p;
    }
    *out = static_cast<unsigned char *>(e.addr);
    return CSC_OK;
}

// Layout of the statistics' scratch inside the fixed array: the control
// header, the compaction block counts and the FP64 accumulators of phi and
// psi, then the nonzero list (k, s, z), as long as the rest of the array
// allows (at most one entry per coordinate).  Returns the layout; nnz_cap is
// 0 when not even one entry fits.
static WsLayout noalloc_layout(const Geom &g) {
    WsLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return at;
    };
    L.blk_cap = (int)ceil_div(g.nzpos(), 256) + 1;
    L.hdr = take(sizeof(WsHeader));
    L.blk = take(2 * (size_t)L.blk_cap * sizeof(int));
    L.phi64 = take((size_t)g.ntab() * sizeof(double));
    L.psi64 = take((size_t)g.nd() * sizeof(double));
    // three lists of 4-byte entries, each starting on a 256-byte boundary
    const size_t left = off + 3 * 256 < kNoAllocScratchBytes ? kNoAllocScratchBytes - off - 3 * 256 : 0;
    L.nnz_cap = std::min<long long>(g.nz(), (long long)(left / 12));
    L.nnz_k = take((size_t)L.nnz_cap * sizeof(int));
    L.nnz_s = take((size_t)L.nnz_cap * sizeof(int));
    L.nnz_z = take((size_t)L.nnz_cap * sizeof(float));
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
    if (L.nnz_cap < 1 || L.total > kNoAllocScratchBytes) return CSC_ERR_WORKSPACE;
    unsigned char *ws = nullptr;
    rc = noalloc_scratch(&ws);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // the previous call's header is still there: clear it
    CSC_CUDA(cudaMemsetAsync(ws + L.hdr, 0, sizeof(WsHeader), st));
    return dict_stats_impl(g, Z, X, phi, psi, ws, L, st);
}
