// cdl.cu -- the outer convolutional dictionary learning loop (Alg. 2):
// repeat { Z <- CSC(X, D) by LGCD with soft-locks; phi, psi <- statistics of
// Z; D <- PGD with Armijo on (phi, psi) } until the cost varies by less than
// nu (relative) or max_outer iterations are done.  Host-side driver over the
// kernels of the other files; every step runs on the GPU.  cdl_step is one
// pass of the loop body as a single call.
#include <cmath>
#include <cstddef>
#include <cstring>

#include "common.cuh"
#include "dict.cuh"

namespace csc {

// ||X||^2 in FP64 into *out (one atomic per block).
template <int NT>
__global__ void __launch_bounds__(NT) sumsq_kernel(const float *x, long long n, double *out) {
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
        const double v = x[i];
        s += v * v;
    }
    block_sum_atomic<NT>(s, out);
}

}  // namespace csc

using namespace csc;

extern "C" int cdl_fit(const csc_shape *shape, const float *X, float *D, float *Z, float *beta, float *dtd,
                       float *phi, float *psi, double reg, double tol, int max_outer, double nu,
                       int pgd_max_iter, double pgd_tol, const csc_solve_opts *opts, void *ws,
                       size_t ws_bytes, double *trace, int *n_outer, csc_stream_t stream) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!X || !D || !Z || !beta || !dtd || !phi || !psi || !ws) return CSC_ERR_INVALID;
    if (!(reg > 0.0) || !(tol > 0.0) || max_outer < 1 || !(nu >= 0.0) || pgd_max_iter < 0)
        return CSC_ERR_INVALID;
    WsLayout L = plan_workspace(g, 0, 4);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *wsb = static_cast<unsigned char *>(ws);
    WsHeader *h = reinterpret_cast<WsHeader *>(wsb + L.hdr);

    // ||X||^2 once (the constant term of the dictionary objective)
    CSC_CUDA(cudaMemsetAsync(&h->obj_f, 0, sizeof(double), st));
    sumsq_kernel<256><<<1216, 256, 0, st>>>(X, g.nx(), &h->obj_f);
    CSC_CUDA(cudaGetLastError());
    double xsq = 0.0;
    {
        const int rb_ = read_back(&xsq, &h->obj_f, st);
        if (rb_) return rb_;
    }

    csc_solve_opts o;
    csc_default_opts(&o);
    if (opts) o = *opts;
    if (o.beta_init < 0 || o.beta_init > 1) return CSC_ERR_INVALID;
    o.warm_start = 0;  // Z = 0 at every CSC step (Alg. 1 / Alg. 3 initialisation)
    double lambda = 0.0, prev = 0.0;
    int q = 0, status = CSC_OK;
    for (q = 0; q < max_outer; q++) {
        double lmax = 0.0;
        // the first beta is exact (it fixes lambda); later ones may run on the tensor cores
        if (q > 0 && o.beta_init == 1)
            rc = csc_init_beta_bf16x3(shape, X, D, beta, dtd, nullptr, ws, ws_bytes, stream);
        else
            rc = csc_init_beta(shape, X, D, beta, dtd, q == 0 ? &lmax : nullptr, ws, ws_bytes, stream);
        if (rc) return rc;
        if (q == 0) lambda = (double)(float)(reg * lmax);  // fixed from D0, as the solver receives it
        csc_solve_stats S;
        rc = csc_lgcd_solve(shape, X, D, dtd, beta, Z, (float)lambda, (float)tol, &o, ws, ws_bytes, &S,
                            stream);
        if (rc != CSC_OK && rc != CSC_NOT_CONVERGED) return rc;
        if (rc == CSC_NOT_CONVERGED) status = CSC_NOT_CONVERGED;
        rc = cdl_dict_stats(shape, Z, X, phi, psi, ws, ws_bytes, stream);
        if (rc) return rc;
        double fd = 0.0;
        int it = 0;
        rc = cdl_dict_update(shape, phi, psi, xsq, D, pgd_max_iter, pgd_tol, &fd, &it, ws, ws_bytes, stream);
        if (rc) return rc;
        // The cost after the dictionary step from the residual with FP64
        // sums, like the cost the solve reports: the PGD value fd comes from
        // phi * D in FP32, whose relative error (about 1e-5 at K = 25 atoms of
        // 32 x 32) would blur the relative-change test against nu.
        double after = 0.0;
        rc = csc_objective(shape, X, D, Z, lambda, &after, ws, ws_bytes, stream);
        if (rc) return rc;
        if (trace) {
            trace[2 * q] = S.objective;
            trace[2 * q + 1] = after;
        }
        if (q > 0 && std::fabs(prev - after) < nu * std::fabs(after)) {
            q++;
            break;
        }
        prev = after;
    }
    if (n_outer) *n_outer = q;
    return status;
}

extern "C" int cdl_step(const csc_shape *shape, const float *X, float *D, float *Z, float *beta, float *dtd,
                        float *phi, float *psi, double reg, double lambda, double tol, double x_sqnorm,
                        int pgd_max_iter, double pgd_tol, const csc_solve_opts *opts, void *ws, size_t ws_bytes,
                        csc_solve_stats *stats, double *lambda_out, double *dict_cost_out, int *dict_iters_out,
                        csc_stream_t stream) {
    Geom g;
    int rc = make_geom(shape, &g);
    if (rc) return rc;
    if (!X || !D || !Z || !beta || !dtd || !phi || !psi || !ws) return CSC_ERR_INVALID;
    if (!(lambda > 0.0) && !(reg > 0.0)) return CSC_ERR_INVALID;
    if (!(tol > 0.0) || std::isnan(x_sqnorm) || pgd_max_iter < 0 || !(pgd_tol >= 0.0) || std::isnan(lambda))
        return CSC_ERR_INVALID;
    csc_solve_opts o;
    csc_default_opts(&o);
    if (opts) o = *opts;
    if (o.beta_init < 0 || o.beta_init > 1) return CSC_ERR_INVALID;
    WsLayout L = plan_workspace(g, 0, 4);
    if (ws_bytes < L.total) return CSC_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *wsb = static_cast<unsigned char *>(ws);
    WsHeader *h = reinterpret_cast<WsHeader *>(wsb + L.hdr);

    // ||X||^2 on the device when the caller does not give it; the dictionary
    // step reads it there (no synchronisation)
    const double *xsq_dev = nullptr;
    if (x_sqnorm < 0.0) {
        CSC_CUDA(cudaMemsetAsync(&h->xsq, 0, sizeof(double), st));
        sumsq_kernel<256><<<1216, 256, 0, st>>>(X, g.nx(), &h->xsq);
        CSC_CUDA(cudaGetLastError());
        xsq_dev = &h->xsq;
    }
    // beta and the D^T D table.  A given lambda (> 0) is used as it is, so that
    // the calls of an outer loop solve one fixed problem (Alg. 2); otherwise
    // lambda = reg * lambda_max of this D, from the FP32 beta-init.  With a
    // given lambda, opts->beta_init = 1 runs the beta-init on the tensor cores.
    float lam;
    if (lambda > 0.0) {
        lam = (float)lambda;
        rc = o.beta_init == 1 ? csc_init_beta_bf16x3(shape, X, D, beta, dtd, nullptr, ws, ws_bytes, stream)
                              : csc_init_beta(shape, X, D, beta, dtd, nullptr, ws, ws_bytes, stream);
        if (rc) return rc;
    } else {
        double lmax = 0.0;
        if ((rc = csc_init_beta(shape, X, D, beta, dtd, &lmax, ws, ws_bytes, stream))) return rc;
        lam = (float)(reg * lmax);
    }
    if (lambda_out) *lambda_out = lam;
    // Z by LGCD with soft-locks (Alg. 3)
    const int solve_rc = csc_lgcd_solve(shape, X, D, dtd, beta, Z, lam, (float)tol, &o, ws, ws_bytes, stats,
                                        stream);
    if (solve_rc != CSC_OK && solve_rc != CSC_NOT_CONVERGED) return solve_rc;
    // phi, psi and the dictionary step, queued without a synchronisation in
    // between; a nonzero list that overflowed leaves D unchanged
    if ((rc = dict_stats_deferred(g, Z, X, phi, psi, wsb, L, st))) return rc;
    if ((rc = dict_update_impl(g, phi, psi, x_sqnorm, D, pgd_max_iter, pgd_tol, nullptr, nullptr, wsb, L, st,
                               xsq_dev, &h->scan_total, (int)L.nnz_cap)))
        return rc;
    // one read-back: the dictionary step's results and the nonzero count
    struct Tail {
        double pgd[12];
        int scan_total;
    };
    static_assert(offsetof(WsHeader, scan_total) == offsetof(WsHeader, pgd_out) + sizeof(double) * 12,
                  "pgd_out and scan_total are adjacent");
    Tail t;
    if ((rc = read_back(&t, &h->pgd_out[0], st))) return rc;
    if (t.scan_total > L.nnz_cap) return CSC_ERR_WORKSPACE;
    if (dict_cost_out) *dict_cost_out = t.pgd[0];
    if (dict_iters_out) *dict_iters_out = (int)t.pgd[1];
    return solve_rc;
}
