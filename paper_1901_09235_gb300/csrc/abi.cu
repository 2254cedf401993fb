// abi.cu -- the extern "C" entry points declared in include/dicodile_gb.h:
// argument validation, workspace layout and dispatch to the kernels.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "dict.cuh"

namespace csc {

static thread_local int g_last_cuda = 0;

int set_cuda_error(cudaError_t e) {
    g_last_cuda = (int)e;
    return CSC_ERR_CUDA;
}

void *pinned_scratch() {
    static thread_local void *buf = nullptr;
    static thread_local bool failed = false;
    if (!buf && !failed) {
        if (cudaHostAlloc(&buf, kPinnedScratch, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            buf = nullptr;
            failed = true;
        }
    }
    return buf;
}

int make_geom(const csc_shape *s, Geom *g) {
    if (!s || !g) return CSC_ERR_INVALID;
    if (s->d != 1 && s->d != 2) return CSC_ERR_INVALID;
    if (s->P < 1 || s->K < 1) return CSC_ERR_INVALID;
    g->d = s->d;
    g->P = s->P;
    g->K = s->K;
    if (s->d == 1) {
        if (s->T[1] != 1 || s->L[1] != 1) return CSC_ERR_INVALID;
        g->T0 = 1;
        g->L0 = 1;
        g->T1 = s->T[0];
        g->L1 = s->L[0];
    } else {
        g->T0 = s->T[0];
        g->T1 = s->T[1];
        g->L0 = s->L[0];
        g->L1 = s->L[1];
    }
    if (g->L0 < 1 || g->L1 < 1 || g->L0 > g->T0 || g->L1 > g->T1) return CSC_ERR_INVALID;
    g->Z0 = g->T0 - g->L0 + 1;
    g->Z1 = g->T1 - g->L1 + 1;
    g->W0 = 2 * g->L0 - 1;
    g->W1 = 2 * g->L1 - 1;
    // positions are addressed with 32-bit indices
    if ((long long)g->Z0 * g->Z1 >= (1ll << 31) || (long long)g->P * g->T0 * g->T1 >= (1ll << 31))
        return CSC_ERR_INVALID;
    if (g->K > 4096) return CSC_ERR_INVALID;
    return CSC_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout plan_workspace(const Geom &g, int max_workers, int rs) {
    WsLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align256(off + bytes);
        return at;
    };
    L.max_workers = max_workers;
    L.nnz_cap = std::min<long long>(g.nz(), std::max<long long>(1ll << 16, g.nz() / 16));
    L.blk_cap = (int)ceil_div(g.nzpos(), 256) + 1;
    L.hdr = take(sizeof(WsHeader));
    L.nrm = take((size_t)g.K * sizeof(double));
    L.dmax = take((size_t)g.K * sizeof(double));
    L.nnz_k = take((size_t)L.nnz_cap * sizeof(int));
    L.nnz_s = take((size_t)L.nnz_cap * sizeof(int));
    L.nnz_z = take((size_t)L.nnz_cap * rs);
    L.blk = take(2 * (size_t)L.blk_cap * sizeof(int));
    L.r64 = take((size_t)g.nx() * sizeof(double));
    L.rr = take((size_t)g.nx() * rs);
    L.phi64 = take((size_t)g.ntab() * sizeof(double));
    L.psi64 = take((size_t)g.nd() * sizeof(double));
    // per-source convolutions of the dictionary step: [cluster rank][K][atoms per CTA x atom]
    L.pgd = take(2 * ((size_t)g.K * g.nd() + 16 * (size_t)g.natom() * g.K) * sizeof(float));
    L.mbox_slots = take((size_t)max_workers * kDirs * kMailboxCap * sizeof(int4));
    L.mbox_ctl = take((size_t)max_workers * kDirs * 32 * sizeof(int));
    L.total = off;
    // optional, after the required regions: the initial beta of an FP32
    // solve, from which the global-tile solve rebuilds beta for its final
    // KKT test (a workspace that ends at `total` takes the correlation)
    L.beta0 = off;
    if (rs == 4) {
        size_t o2 = align256(off + (size_t)g.nz() * rs);
        // gather of the rebuilt beta: bins of gbh x gbw positions (one output
        // tile of its kernel each), their offsets and fill cursors, the binned
        // list (16 bytes per nonzero) and C transposed to [k2][delta][k]
        L.gbh = g.d == 1 ? 1 : 8;
        L.gbw = g.d == 1 ? 512 : 64;
        L.gnb0 = (int)ceil_div(g.Z0, L.gbh);
        L.gnb1 = (int)ceil_div(g.Z1, L.gbw);
        L.gkp = (g.K + 3) / 4 * 4;
        const size_t nbins = (size_t)L.gnb0 * L.gnb1;
        L.gbin = o2;
        o2 = align256(o2 + 2 * (nbins + 1) * sizeof(int));
        L.glist = o2;
        o2 = align256(o2 + (size_t)L.nnz_cap * 16);
        L.gtab = o2;
        o2 = align256(o2 + (size_t)g.K * g.W0 * g.W1 * L.gkp * sizeof(float));
        // rows of W1 values with 4 zeros before and at least 4 after, the row
        // stride equal to Z1 mod 4; blocks a multiple of 16 bytes
        L.wrs = g.W1 + 8 + ((g.Z1 - (g.W1 + 8)) & 3);
        L.wbs = (g.W0 * L.wrs + 3) / 4 * 4;
        L.wtab = o2;
        o2 = align256(o2 + (size_t)g.K * g.K * L.wbs * sizeof(float));
        L.total_beta0 = o2;
    } else {
        L.total_beta0 = off;
    }
    return L;
}

// Upper bound on the number of tiles any plan can use for this geometry:
// every tile is at least min(Z_i, L_i) wide.
static int worker_bound(const Geom &g, const csc_solve_opts *o) {
    long long a = ceil_div(g.Z0, std::min(g.Z0, g.L0));
    long long b = ceil_div(g.Z1, std::min(g.Z1, g.L1));
    long long w = a * b;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 152;
    }
    w = std::min<long long>(w, 8ll * sms);
    if (o && o->max_workers > 0) w = std::min<long long>(w, o->max_workers);
    return (int)std::max<long long>(w, 1);
}

template <typename real>
static int init_beta_impl(const csc_shape *shape, const real *X, const real *D, real *beta,
                          real *dtd, double *lmax, void *ws, size_t ws_bytes, cudaStream_t st) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!X || !D || !beta || !dtd || !ws) return CSC_ERR_INVALID;
    WsLayout L = plan_workspace(g, 0, sizeof(real));
    if (ws_bytes < L.hdr + sizeof(WsHeader)) return CSC_ERR_WORKSPACE;
    WsHeader *h = reinterpret_cast<WsHeader *>(static_cast<unsigned char *>(ws) + L.hdr);
    CSC_CUDA(cudaMemsetAsync(&h->lmax_bits, 0, sizeof(unsigned long long), st));
    rc = launch_corr_init<real>(g, X, D, beta, &h->lmax_bits, st);
    if (rc) return rc;
    rc = launch_dtd<real>(g, D, dtd, st);
    if (rc) return rc;
    if (lmax) {
        unsigned long long bits = 0;
        if ((rc = read_back(&bits, &h->lmax_bits, st))) return rc;
        if (sizeof(real) == 4) {
            unsigned u = (unsigned)bits;
            float f;
            memcpy(&f, &u, 4);
            *lmax = f;
        } else {
            memcpy(lmax, &bits, 8);
        }
    }
    return CSC_OK;
}

}  // namespace csc

using namespace csc;

extern "C" {

void csc_default_opts(csc_solve_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->mode = CSC_MODE_ASYNC;
    o->beta_refresh = 2;
    o->timeout_s = 30.0;
}

int csc_workspace_size(const csc_shape *shape, const csc_solve_opts *opts, size_t *bytes) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!bytes) return CSC_ERR_INVALID;
    int w = worker_bound(g, opts);
    size_t a = plan_workspace(g, w, 4).total_beta0, b = plan_workspace(g, w, 8).total;
    *bytes = std::max(a, b);
    return CSC_OK;
}

int csc_init_beta(const csc_shape *shape, const float *X, const float *D, float *beta, float *dtd,
                  double *lambda_max_out, void *ws, size_t ws_bytes, csc_stream_t stream) {
    return init_beta_impl<float>(shape, X, D, beta, dtd, lambda_max_out, ws, ws_bytes,
                                 (cudaStream_t)stream);
}

int csc_init_beta_f64(const csc_shape *shape, const double *X, const double *D, double *beta,
                      double *dtd, double *lambda_max_out, void *ws, size_t ws_bytes,
                      csc_stream_t stream) {
    return init_beta_impl<double>(shape, X, D, beta, dtd, lambda_max_out, ws, ws_bytes,
                                  (cudaStream_t)stream);
}

int csc_lgcd_solve(const csc_shape *shape, const float *X, const float *D, const float *dtd,
                   float *beta, float *Z, float lambda, float tol, const csc_solve_opts *opts,
                   void *ws, size_t ws_bytes, csc_solve_stats *stats, csc_stream_t stream) {
    return solve_impl<float>(shape, X, D, dtd, beta, Z, lambda, tol, opts, ws, ws_bytes, stats,
                             (cudaStream_t)stream);
}

int csc_lgcd_solve_f64(const csc_shape *shape, const double *X, const double *D, const double *dtd,
                       double *beta, double *Z, double lambda, double tol,
                       const csc_solve_opts *opts, void *ws, size_t ws_bytes,
                       csc_solve_stats *stats, csc_stream_t stream) {
    return solve_impl<double>(shape, X, D, dtd, beta, Z, lambda, tol, opts, ws, ws_bytes, stats,
                              (cudaStream_t)stream);
}

int csc_objective(const csc_shape *shape, const float *X, const float *D, const float *Z,
                  double lambda, double *objective_out, void *ws, size_t ws_bytes,
                  csc_stream_t stream) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!X || !D || !Z || !ws || !objective_out) return CSC_ERR_INVALID;
    WsLayout L = plan_workspace(g, 0, 4);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
    unsigned char *wsb = static_cast<unsigned char *>(ws);
    cudaStream_t st = (cudaStream_t)stream;
    rc = launch_refresh<float>(g, L, wsb, X, D, Z, 0.f, nullptr, st);
    if (rc) return rc;
    WsHeader hh;
    {
        const int rb_ = read_back(&hh, wsb + L.hdr, st);
        if (rb_) return rb_;
    }
    *objective_out = 0.5 * hh.obj_f + lambda * hh.obj_g;
    return CSC_OK;
}

int cdl_dict_stats(const csc_shape *shape, const float *Z, const float *X, float *phi, float *psi,
                   void *ws, size_t ws_bytes, csc_stream_t stream) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!Z || !X || !phi || !psi || !ws) return CSC_ERR_INVALID;
    WsLayout L = plan_workspace(g, 0, 4);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
    return dict_stats_impl(g, Z, X, phi, psi, static_cast<unsigned char *>(ws), L,
                           (cudaStream_t)stream);
}

int cdl_dict_update(const csc_shape *shape, const float *phi, const float *psi, double x_sqnorm,
                    float *D, int max_iter, double tol, double *objective_out, int *iterations_out,
                    void *ws, size_t ws_bytes, csc_stream_t stream) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!phi || !psi || !D || !ws || max_iter < 0 || !(tol >= 0.0)) return CSC_ERR_INVALID;
    WsLayout L = plan_workspace(g, 0, 4);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
    return dict_update_impl(g, phi, psi, x_sqnorm, D, max_iter, tol, objective_out, iterations_out,
                            static_cast<unsigned char *>(ws), L, (cudaStream_t)stream);
}

int csc_sparse_code(const csc_shape *shape, const float *Z, int *k_out, int *s_out, float *val_out,
                    long long cap, long long *nnz_out, void *ws, size_t ws_bytes, csc_stream_t stream) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!Z || !nnz_out || !ws || cap < 0 || (cap > 0 && (!k_out || !s_out || !val_out))) return CSC_ERR_INVALID;
    WsLayout L = plan_workspace(g, 0, 4);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
    return sparse_code_impl(g, Z, k_out, s_out, val_out, cap, nnz_out, static_cast<unsigned char *>(ws), L,
                            (cudaStream_t)stream);
}

const char *csc_status_string(int s) {
    switch (s) {
        case CSC_OK: return "ok";
        case CSC_ERR_INVALID: return "invalid argument";
        case CSC_ERR_CUDA: return "CUDA error";
        case CSC_NOT_CONVERGED: return "not converged (max_updates or refresh rounds exhausted)";
        case CSC_ERR_TIMEOUT: return "device wait timed out";
        case CSC_ERR_DIVERGED: return "diverged (||Z||_inf above min_k 50/||D_k||_inf)";
        case CSC_ERR_UNIMPLEMENTED: return "unsupported shape/options";
        case CSC_ERR_WORKSPACE: return "workspace too small";
        default: return "unknown status";
    }
}

int csc_last_cuda_error(void) { return g_last_cuda; }

}  // extern "C"
