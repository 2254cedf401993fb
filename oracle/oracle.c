/*
 * oracle.c -- plain, sequential, FP64 restatement of the convolutional sparse
 * coding (CSC) and dictionary-update computations of DiCoDiLe
 * (Moreau & Gramfort, "Distributed Convolutional Dictionary Learning").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct checker
 * against which the CUDA path is compared.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library, and nothing in the
 * library may call it.
 *
 * Every array is dense and row-major.  A 1-D signal is stored as a single row:
 * T0 = L0 = 1.  With Tz_i = T_i - L_i + 1 (the "valid" activation domain):
 *   X    : P  x T0  x T1                    (observation)
 *   D    : K  x P   x L0 x L1               (dictionary, atom k channel p)
 *   Z    : K  x Tz0 x Tz1                   (activations)
 *   beta : K  x Tz0 x Tz1                   (auxiliary variable of Section 3)
 *   C    : K  x K   x (2L0-1) x (2L1-1)     (atom cross-correlation table)
 *          C[k][k2][d0+L0-1][d1+L1-1] = sum_p sum_tau D[k][p][tau] D[k2][p][tau+d]
 *   phi  : same layout as C                 (Eq. phi, restricted to Phi)
 *   psi  : K  x P   x L0 x L1               (psi = Z~ * X restricted to Theta)
 *
 * Readings of passages that the paper leaves ambiguous are taken as follows
 * and are the same ones the CUDA path implements:
 *   - the activation domain is the valid one, so that X = Z * D fits Omega;
 *   - the reversal makes beta-init a cross-correlation (Section 3, Alg. 1
 *     initialisation): beta_k[s] = sum_p sum_tau D_kp[tau] X_p[s + tau];
 *   - the beta update after Z_k0[s0] += dz is beta_k[s] -= C[k][k0][s-s0] dz
 *     for (k,s) != (k0,s0) (Eq. beta_update);
 *   - sub-domains are boxes of side sub_i visited in row-major order,
 *     m = q mod M (Section 3);
 *   - argmax ties go to the smaller row-major position, then to the smaller k;
 *   - a candidate with |dZ| < eps is not applied; the solve stops after M
 *     consecutive iterations that applied nothing (Alg. 1 stopping rule);
 *   - the dictionary gradient is phi * D - psi (the paper prints its
 *     negative, Section 4.2).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX3(a, b, c, B, C) (((size_t)(a) * (B) + (b)) * (C) + (c))
#define IDX4(a, b, c, d, B, C, Dd) ((((size_t)(a) * (B) + (b)) * (C) + (c)) * (Dd) + (d))

/* Soft-thresholding ST(u, lambda) = sign(u) max(|u| - lambda, 0) (Section 2). */
static double soft_threshold(double u, double lam)
{
    if (u > lam) return u - lam;
    if (u < -lam) return u + lam;
    return 0.0;
}

/* beta_k[s] = (D~_k * X)[s] = sum_p sum_tau D_kp[tau] X_p[s + tau]
 * (Alg. 1 initialisation; Section 2, lambda_max = ||X * D~||_inf). */
void orc_beta_init(int P, int K, int T0, int T1, int L0, int L1,
                   const double *X, const double *D, double *beta)
{
    int Z0 = T0 - L0 + 1, Z1 = T1 - L1 + 1;
    for (int k = 0; k < K; k++)
        for (int i = 0; i < Z0; i++)
            for (int j = 0; j < Z1; j++) {
                double acc = 0.0;
                for (int p = 0; p < P; p++)
                    for (int a = 0; a < L0; a++)
                        for (int b = 0; b < L1; b++)
                            acc += D[IDX4(k, p, a, b, P, L0, L1)] *
                                   X[IDX3(p, i + a, j + b, T0, T1)];
                beta[IDX3(k, i, j, Z0, Z1)] = acc;
            }
}

/* C[k][k2][d] = sum_p sum_tau D_kp[tau] D_k2p[tau + d], d in Phi
 * (the (D_k0 * D~_k) table of Eq. beta_update, support prod [-L_i+1, L_i[). */
void orc_dtd(int P, int K, int L0, int L1, const double *D, double *C)
{
    int W0 = 2 * L0 - 1, W1 = 2 * L1 - 1;
    for (int k = 0; k < K; k++)
        for (int k2 = 0; k2 < K; k2++)
            for (int d0 = -L0 + 1; d0 < L0; d0++)
                for (int d1 = -L1 + 1; d1 < L1; d1++) {
                    double acc = 0.0;
                    for (int p = 0; p < P; p++)
                        for (int a = 0; a < L0; a++)
                            for (int b = 0; b < L1; b++) {
                                int a2 = a + d0, b2 = b + d1;
                                if (a2 < 0 || a2 >= L0 || b2 < 0 || b2 >= L1) continue;
                                acc += D[IDX4(k, p, a, b, P, L0, L1)] *
                                       D[IDX4(k2, p, a2, b2, P, L0, L1)];
                            }
                    C[IDX4(k, k2, d0 + L0 - 1, d1 + L1 - 1, K, W0, W1)] = acc;
                }
}

/* ||D_k||_2^2 over all channels and positions (Eq. pb_coord denominator). */
void orc_atom_sqnorms(int P, int K, int L0, int L1, const double *D, double *nrm)
{
    size_t n = (size_t)P * L0 * L1;
    for (int k = 0; k < K; k++) {
        double acc = 0.0;
        for (size_t q = 0; q < n; q++) acc += D[k * n + q] * D[k * n + q];
        nrm[k] = acc;
    }
}

/* lambda_max = ||X * D~||_inf (Section 2): the largest |beta_init|. */
double orc_lambda_max(int P, int K, int T0, int T1, int L0, int L1,
                      const double *X, const double *D)
{
    int Z0 = T0 - L0 + 1, Z1 = T1 - L1 + 1;
    size_t n = (size_t)K * Z0 * Z1;
    double *beta = malloc(n * sizeof(double));
    orc_beta_init(P, K, T0, T1, L0, L1, X, D, beta);
    double m = 0.0;
    for (size_t q = 0; q < n; q++) if (fabs(beta[q]) > m) m = fabs(beta[q]);
    free(beta);
    return m;
}

/* (Z * D)_p[t] = sum_k sum_tau Z_k[t - tau] D_kp[tau] (Eq. model, Section 2). */
void orc_reconstruct(int P, int K, int T0, int T1, int L0, int L1,
                     const double *Z, const double *D, double *out)
{
    int Z0 = T0 - L0 + 1, Z1 = T1 - L1 + 1;
    for (int p = 0; p < P; p++)
        for (int t0 = 0; t0 < T0; t0++)
            for (int t1 = 0; t1 < T1; t1++) {
                double acc = 0.0;
                for (int k = 0; k < K; k++)
                    for (int a = 0; a < L0; a++)
                        for (int b = 0; b < L1; b++) {
                            int s0 = t0 - a, s1 = t1 - b;
                            if (s0 < 0 || s0 >= Z0 || s1 < 0 || s1 >= Z1) continue;
                            acc += Z[IDX3(k, s0, s1, Z0, Z1)] *
                                   D[IDX4(k, p, a, b, P, L0, L1)];
                        }
                out[IDX3(p, t0, t1, T0, T1)] = acc;
            }
}

/* F(Z, D) + G(Z) = 1/2 ||X - Z * D||_2^2 + lambda ||Z||_1 (Eq. cdl / Eq. csc). */
double orc_objective(int P, int K, int T0, int T1, int L0, int L1,
                     const double *X, const double *D, const double *Z, double lambda)
{
    int Z0 = T0 - L0 + 1, Z1 = T1 - L1 + 1;
    size_t nx = (size_t)P * T0 * T1, nz = (size_t)K * Z0 * Z1;
    double *rec = malloc(nx * sizeof(double));
    orc_reconstruct(P, K, T0, T1, L0, L1, Z, D, rec);
    double f = 0.0, g = 0.0;
    for (size_t q = 0; q < nx; q++) {
        double r = X[q] - rec[q];
        f += r * r;
    }
    for (size_t q = 0; q < nz; q++) g += fabs(Z[q]);
    free(rec);
    return 0.5 * f + lambda * g;
}

/* beta from its definition (Section 3):
 * beta_k[s] = ((X - Z*D + Z_k[s] e_s * D_k) * D~_k)[s]
 *           = sum_p sum_tau D_kp[tau] (X - Z*D)_p[s+tau] + ||D_k||^2 Z_k[s]. */
void orc_beta_from_Z(int P, int K, int T0, int T1, int L0, int L1,
                     const double *X, const double *D, const double *Z, double *beta)
{
    int Z0 = T0 - L0 + 1, Z1 = T1 - L1 + 1;
    size_t nx = (size_t)P * T0 * T1;
    double *res = malloc(nx * sizeof(double));
    double *nrm = malloc((size_t)K * sizeof(double));
    orc_reconstruct(P, K, T0, T1, L0, L1, Z, D, res);
    for (size_t q = 0; q < nx; q++) res[q] = X[q] - res[q];
    orc_beta_init(P, K, T0, T1, L0, L1, res, D, beta);
    orc_atom_sqnorms(P, K, L0, L1, D, nrm);
    for (int k = 0; k < K; k++)
        for (int i = 0; i < Z0; i++)
            for (int j = 0; j < Z1; j++)
                beta[IDX3(k, i, j, Z0, Z1)] += nrm[k] * Z[IDX3(k, i, j, Z0, Z1)];
    free(res);
    free(nrm);
}

/* max_{k,s} |ST(beta_k[s], lambda) / ||D_k||^2 - Z_k[s]|: the quantity that
 * Alg. 1 drives below eps. */
double orc_max_dz(int K, int Z0, int Z1, const double *beta, const double *Z,
                  const double *nrm, double lambda)
{
    double m = 0.0;
    for (int k = 0; k < K; k++)
        for (size_t q = 0; q < (size_t)Z0 * Z1; q++) {
            size_t at = (size_t)k * Z0 * Z1 + q;
            double dz = fabs(soft_threshold(beta[at], lambda) / nrm[k] - Z[at]);
            if (dz > m) m = dz;
        }
    return m;
}

/* ---------------------------------------------------------------------------
 * LGCD (Alg. 1) and its tiled, checkerboard-phased schedule.
 * ------------------------------------------------------------------------ */

typedef struct {
    int P, K, Z0, Z1, L0, L1;
    double lambda, eps;
    double *beta, *Z, *C, *nrm;
} lgcd_state;

typedef struct {
    long long cap, n;
    int *k0;
    long long *s0;
    double *z_old, *z_new, *beta_at;
} lgcd_trace;

/* One LGCD iteration on the sub-domain box [r0,r1) x [c0,c1): evaluate
 * Z' = ST(beta, lambda)/||D_k||^2 on K x C_m (Eq. pb_coord), pick the largest
 * |dZ| (ties: smaller row-major position, then smaller k), and if
 * |dZ| >= eps apply it and the beta update of Eq. beta_update.
 * Returns 1 when an update was applied. */
static int lgcd_step(lgcd_state *S, int r0, int r1, int c0, int c1, lgcd_trace *tr)
{
    int K = S->K, Z0 = S->Z0, Z1 = S->Z1, L0 = S->L0, L1 = S->L1;
    int W0 = 2 * L0 - 1, W1 = 2 * L1 - 1;
    double best = -1.0, best_new = 0.0;
    int bk = -1, bi = -1, bj = -1;
    for (int i = r0; i < r1; i++)
        for (int j = c0; j < c1; j++)
            for (int k = 0; k < K; k++) {
                size_t at = IDX3(k, i, j, Z0, Z1);
                double znew = soft_threshold(S->beta[at], S->lambda) / S->nrm[k];
                double a = fabs(znew - S->Z[at]);
                if (a > best) { best = a; best_new = znew; bk = k; bi = i; bj = j; }
            }
    if (bk < 0 || best < S->eps) return 0;

    size_t at0 = IDX3(bk, bi, bj, Z0, Z1);
    double dz = best_new - S->Z[at0];
    if (tr && tr->n < tr->cap) {
        tr->k0[tr->n] = bk;
        tr->s0[tr->n] = (long long)bi * Z1 + bj;
        tr->z_old[tr->n] = S->Z[at0];
        tr->z_new[tr->n] = best_new;
        tr->beta_at[tr->n] = S->beta[at0];
    }
    if (tr) tr->n++;
    S->Z[at0] = best_new;
    /* beta_k[s] -= C[k][k0][s - s0] dz for s in V(s0), (k,s) != (k0,s0). */
    for (int k = 0; k < K; k++)
        for (int d0 = -L0 + 1; d0 < L0; d0++)
            for (int d1 = -L1 + 1; d1 < L1; d1++) {
                int i = bi + d0, j = bj + d1;
                if (i < 0 || i >= Z0 || j < 0 || j >= Z1) continue;
                if (k == bk && d0 == 0 && d1 == 0) continue;
                double c = S->C[IDX4(k, bk, d0 + L0 - 1, d1 + L1 - 1, K, W0, W1)];
                double t = c * dz;
                S->beta[IDX3(k, i, j, Z0, Z1)] = S->beta[IDX3(k, i, j, Z0, Z1)] - t;
            }
    return 1;
}

static int ceil_div(int a, int b) { return (a + b - 1) / b; }

/* Tiled LGCD with the checkerboard-phased schedule.
 *
 * The activation domain is split into tiles of tile0 x tile1 (the worker
 * sub-domains S_w of Alg. 3, the last row/column of tiles ragged).  Each tile
 * has its own partition into sub-domains of sub0 x sub1 anchored at the tile
 * origin and its own cyclic counter m_w (Alg. 3).  A round runs the four
 * colours c = 2 (a mod 2) + (b mod 2) of tile (a,b) in order; within a colour
 * every tile of that colour makes one LGCD iteration, in row-major tile
 * order.  Tiles of one colour are at least one full tile apart, so when every
 * full tile is at least L_i wide their updates do not interact and the order
 * inside a colour does not matter.  The solve stops after max_w M_w
 * consecutive rounds in which no tile applied an update; at that point every
 * sub-domain of every tile has been scanned against the final beta.
 *
 * With a single tile covering the domain this is exactly Alg. 1.
 * Returns 0 when converged, 1 when max_updates was reached. */
int orc_lgcd_tiled(int P, int K, int T0, int T1, int L0, int L1,
                   const double *X, const double *D, double lambda, double eps,
                   int tile0, int tile1, int sub0, int sub1, long long max_updates,
                   double *Z, double *beta_out, long long *n_updates, long long *n_iters,
                   long long trace_cap, int *tr_k0, long long *tr_s0, double *tr_zold,
                   double *tr_znew, double *tr_beta)
{
    int Z0 = T0 - L0 + 1, Z1 = T1 - L1 + 1;
    int W0 = 2 * L0 - 1, W1 = 2 * L1 - 1;
    size_t nz = (size_t)K * Z0 * Z1;
    lgcd_state S;
    S.P = P; S.K = K; S.Z0 = Z0; S.Z1 = Z1; S.L0 = L0; S.L1 = L1;
    S.lambda = lambda; S.eps = eps;
    S.beta = malloc(nz * sizeof(double));
    S.Z = Z;
    S.C = malloc((size_t)K * K * W0 * W1 * sizeof(double));
    S.nrm = malloc((size_t)K * sizeof(double));
    memset(Z, 0, nz * sizeof(double));                        /* Z = 0 (Alg. 1) */
    orc_beta_init(P, K, T0, T1, L0, L1, X, D, S.beta);        /* beta = D~ * X   */
    orc_dtd(P, K, L0, L1, D, S.C);
    orc_atom_sqnorms(P, K, L0, L1, D, S.nrm);

    lgcd_trace tr, *trp = NULL;
    if (trace_cap > 0) {
        tr.cap = trace_cap; tr.n = 0; tr.k0 = tr_k0; tr.s0 = tr_s0;
        tr.z_old = tr_zold; tr.z_new = tr_znew; tr.beta_at = tr_beta;
        trp = &tr;
    }

    if (tile0 <= 0 || tile0 > Z0) tile0 = Z0;
    if (tile1 <= 0 || tile1 > Z1) tile1 = Z1;
    if (sub0 <= 0) sub0 = 2 * L0;
    if (sub1 <= 0) sub1 = 2 * L1;
    int G0 = ceil_div(Z0, tile0), G1 = ceil_div(Z1, tile1), G = G0 * G1;
    int *M = malloc((size_t)G * sizeof(int)), *m = calloc((size_t)G, sizeof(int));
    int Mmax = 0;
    for (int w = 0; w < G; w++) {
        int a = w / G1, b = w % G1;
        int h = (a + 1) * tile0 <= Z0 ? tile0 : Z0 - a * tile0;
        int wd = (b + 1) * tile1 <= Z1 ? tile1 : Z1 - b * tile1;
        M[w] = ceil_div(h, sub0) * ceil_div(wd, sub1);
        if (M[w] > Mmax) Mmax = M[w];
    }

    long long upd = 0, it = 0;
    int quiet_rounds = 0, status = 0;
    while (quiet_rounds < Mmax) {
        int applied_round = 0;
        for (int c = 0; c < 4 && !status; c++)
            for (int w = 0; w < G; w++) {
                int a = w / G1, b = w % G1;
                if (2 * (a % 2) + (b % 2) != c) continue;
                int tr0 = a * tile0, tc0 = b * tile1;
                int tr1 = tr0 + tile0 < Z0 ? tr0 + tile0 : Z0;
                int tc1 = tc0 + tile1 < Z1 ? tc0 + tile1 : Z1;
                int ns1 = ceil_div(tc1 - tc0, sub1);
                int mr = m[w] / ns1, mc = m[w] % ns1;
                int r0 = tr0 + mr * sub0, c0 = tc0 + mc * sub1;
                int r1 = r0 + sub0 < tr1 ? r0 + sub0 : tr1;
                int c1 = c0 + sub1 < tc1 ? c0 + sub1 : tc1;
                int ap = lgcd_step(&S, r0, r1, c0, c1, trp);
                it++;
                m[w] = (m[w] + 1) % M[w];
                if (ap) {
                    applied_round = 1;
                    if (++upd >= max_updates && max_updates > 0) { status = 1; break; }
                }
            }
        if (status) break;
        quiet_rounds = applied_round ? 0 : quiet_rounds + 1;
    }
    if (beta_out) memcpy(beta_out, S.beta, nz * sizeof(double));
    if (n_updates) *n_updates = upd;
    if (n_iters) *n_iters = it;
    free(S.beta); free(S.C); free(S.nrm); free(M); free(m);
    return status;
}

/* Sequential LGCD on the whole domain (Alg. 1): the tiled schedule with one
 * tile.  sub = (1,1) gives cyclic CD and sub = (Z0, Z1) gives greedy CD
 * (Section 3). */
int orc_lgcd(int P, int K, int T0, int T1, int L0, int L1,
             const double *X, const double *D, double lambda, double eps,
             int sub0, int sub1, long long max_updates, double *Z, double *beta_out,
             long long *n_updates, long long *n_iters,
             long long trace_cap, int *tr_k0, long long *tr_s0, double *tr_zold,
             double *tr_znew, double *tr_beta)
{
    return orc_lgcd_tiled(P, K, T0, T1, L0, L1, X, D, lambda, eps, 0, 0, sub0, sub1,
                          max_updates, Z, beta_out, n_updates, n_iters, trace_cap,
                          tr_k0, tr_s0, tr_zold, tr_znew, tr_beta);
}

/* Coordinate descent in a given order: the randomized baseline (RCD) of the
 * selection comparison (Section 5.1, Fig. compare_cd) when the order is drawn
 * uniformly at random.  For each flat index c = k |Omega| + s of coords[0..n)
 * in turn, Z_k[s] <- Z'_k[s] = ST(beta_k[s], lambda) / ||D_k||^2 (Eq.
 * pb_coord), followed by the beta update of Eq. beta_update when the value
 * changes.  The order is an input so that the caller chooses its
 * distribution.  beta and Z are the state on entry and on exit (Z = 0 with
 * beta = D~ * X is the cold start of Alg. 1).  Returns the number of
 * coordinates whose value changed, or -1 for an index outside K x Omega. */
long long orc_rcd(int P, int K, int T0, int T1, int L0, int L1, const double *D, double lambda,
                  const unsigned *coords, long long n, double *Z, double *beta)
{
    int Z0 = T0 - L0 + 1, Z1 = T1 - L1 + 1;
    int W0 = 2 * L0 - 1, W1 = 2 * L1 - 1;
    size_t plane = (size_t)Z0 * Z1;
    double *C = malloc((size_t)K * K * W0 * W1 * sizeof(double));
    double *nrm = malloc((size_t)K * sizeof(double));
    orc_dtd(P, K, L0, L1, D, C);
    orc_atom_sqnorms(P, K, L0, L1, D, nrm);
    long long changed = 0;
    for (long long q = 0; q < n; q++) {
        size_t c = coords[q];
        if (c >= (size_t)K * plane) { changed = -1; break; }
        int k0 = (int)(c / plane), s = (int)(c % plane), i0 = s / Z1, j0 = s % Z1;
        double znew = soft_threshold(beta[c], lambda) / nrm[k0];
        double dz = znew - Z[c];
        if (dz == 0.0) continue;
        Z[c] = znew;
        changed++;
        for (int k = 0; k < K; k++)
            for (int d0 = -L0 + 1; d0 < L0; d0++)
                for (int d1 = -L1 + 1; d1 < L1; d1++) {
                    int i = i0 + d0, j = j0 + d1;
                    if (i < 0 || i >= Z0 || j < 0 || j >= Z1) continue;
                    if (k == k0 && d0 == 0 && d1 == 0) continue;
                    beta[IDX3(k, i, j, Z0, Z1)] -= C[IDX4(k, k0, d0 + L0 - 1, d1 + L1 - 1, K, W0, W1)] * dz;
                }
    }
    free(C);
    free(nrm);
    return changed;
}

/* ---------------------------------------------------------------------------
 * Dictionary update (Section 4.2).
 * ------------------------------------------------------------------------ */

/* phi_{k,k2}[d] = sum_s Z_k[s] Z_k2[s + d] for d in Phi (Eq. phi) and
 * psi_kp[tau] = sum_s Z_k[s] X_p[s + tau] for tau in Theta.  Terms with
 * Z_k[s] = 0 are zero and are skipped. */
void orc_phi_psi(int P, int K, int T0, int T1, int L0, int L1,
                 const double *Z, const double *X, double *phi, double *psi)
{
    int Z0 = T0 - L0 + 1, Z1 = T1 - L1 + 1;
    int W0 = 2 * L0 - 1, W1 = 2 * L1 - 1;
    memset(phi, 0, (size_t)K * K * W0 * W1 * sizeof(double));
    memset(psi, 0, (size_t)K * P * L0 * L1 * sizeof(double));
    for (int k = 0; k < K; k++)
        for (int i = 0; i < Z0; i++)
            for (int j = 0; j < Z1; j++) {
                double z = Z[IDX3(k, i, j, Z0, Z1)];
                if (z == 0.0) continue;
                for (int k2 = 0; k2 < K; k2++)
                    for (int d0 = -L0 + 1; d0 < L0; d0++)
                        for (int d1 = -L1 + 1; d1 < L1; d1++) {
                            int i2 = i + d0, j2 = j + d1;
                            if (i2 < 0 || i2 >= Z0 || j2 < 0 || j2 >= Z1) continue;
                            phi[IDX4(k, k2, d0 + L0 - 1, d1 + L1 - 1, K, W0, W1)] +=
                                z * Z[IDX3(k2, i2, j2, Z0, Z1)];
                        }
                for (int p = 0; p < P; p++)
                    for (int a = 0; a < L0; a++)
                        for (int b = 0; b < L1; b++)
                            psi[IDX4(k, p, a, b, P, L0, L1)] +=
                                z * X[IDX3(p, i + a, j + b, T0, T1)];
            }
}

/* (phi * D)_kp[tau] = sum_k2 sum_tau2 phi_{k,k2}[tau - tau2] D_k2p[tau2]. */
static void phi_conv(int P, int K, int L0, int L1, const double *phi,
                     const double *D, double *out)
{
    int W0 = 2 * L0 - 1, W1 = 2 * L1 - 1;
    for (int k = 0; k < K; k++)
        for (int p = 0; p < P; p++)
            for (int a = 0; a < L0; a++)
                for (int b = 0; b < L1; b++) {
                    double acc = 0.0;
                    for (int k2 = 0; k2 < K; k2++)
                        for (int a2 = 0; a2 < L0; a2++)
                            for (int b2 = 0; b2 < L1; b2++)
                                acc += phi[IDX4(k, k2, a - a2 + L0 - 1, b - b2 + L1 - 1,
                                                K, W0, W1)] *
                                       D[IDX4(k2, p, a2, b2, P, L0, L1)];
                    out[IDX4(k, p, a, b, P, L0, L1)] = acc;
                }
}

/* grad_D F = phi * D - psi (Section 4.2, sign as derived from Eq. dict_update). */
void orc_dict_grad(int P, int K, int L0, int L1, const double *phi, const double *psi,
                   const double *D, double *grad)
{
    size_t n = (size_t)K * P * L0 * L1;
    phi_conv(P, K, L0, L1, phi, D, grad);
    for (size_t q = 0; q < n; q++) grad[q] -= psi[q];
}

/* F(D) = 1/2 ||X||^2 - <psi, D> + 1/2 <D, phi * D>: the data-fit term of
 * Eq. dict_update written with the sufficient statistics phi and psi. */
double orc_dict_objective(int P, int K, int L0, int L1, const double *phi,
                          const double *psi, double x_sqnorm, const double *D)
{
    size_t n = (size_t)K * P * L0 * L1;
    double *q = malloc(n * sizeof(double));
    phi_conv(P, K, L0, L1, phi, D, q);
    double lin = 0.0, quad = 0.0;
    for (size_t i = 0; i < n; i++) {
        lin += psi[i] * D[i];
        quad += D[i] * q[i];
    }
    free(q);
    return 0.5 * x_sqnorm - lin + 0.5 * quad;
}

/* Projection onto {||D_k||_2 <= 1} (Eq. cdl constraint): D_k /= max(1, ||D_k||). */
static void project_atoms(int P, int K, int L0, int L1, double *D)
{
    size_t n = (size_t)P * L0 * L1;
    for (int k = 0; k < K; k++) {
        double s = 0.0;
        for (size_t q = 0; q < n; q++) s += D[k * n + q] * D[k * n + q];
        double nr = sqrt(s);
        if (nr > 1.0)
            for (size_t q = 0; q < n; q++) D[k * n + q] /= nr;
    }
}

/* Projected gradient descent on D with Armijo backtracking (Alg. 2, Section
 * 4.2).  Step: eta_0 = 1 / max_k sum_k2 sum_d |phi_{k,k2}[d]| (a bound on the
 * Lipschitz constant of the gradient); every later iteration starts from twice
 * the last accepted step and halves it until
 *   F(D+) <= F(D) + <grad, D+ - D> + ||D+ - D||^2 / (2 eta).
 * Stops after max_iter iterations or when ||D+ - D|| < tol ||D||.
 * Returns the number of iterations made; *f_out receives F(D) at the end. */
int orc_pgd_armijo(int P, int K, int L0, int L1, const double *phi, const double *psi,
                   double x_sqnorm, double *D, int max_iter, double tol, double *f_out)
{
    int W0 = 2 * L0 - 1, W1 = 2 * L1 - 1;
    size_t n = (size_t)K * P * L0 * L1;
    double lip = 0.0;
    for (int k = 0; k < K; k++) {
        double row = 0.0;
        for (size_t q = 0; q < (size_t)K * W0 * W1; q++) row += fabs(phi[(size_t)k * K * W0 * W1 + q]);
        if (row > lip) lip = row;
    }
    double f = orc_dict_objective(P, K, L0, L1, phi, psi, x_sqnorm, D);
    if (lip <= 0.0) { if (f_out) *f_out = f; return 0; }
    double *g = malloc(n * sizeof(double)), *Dn = malloc(n * sizeof(double));
    double eta = 1.0 / lip;
    int it;
    for (it = 0; it < max_iter; it++) {
        orc_dict_grad(P, K, L0, L1, phi, psi, D, g);
        if (it > 0) eta *= 2.0;
        double fn = f, dsq = 0.0, lin = 0.0;
        for (int bt = 0; bt < 60; bt++) {
            for (size_t q = 0; q < n; q++) Dn[q] = D[q] - eta * g[q];
            project_atoms(P, K, L0, L1, Dn);
            fn = orc_dict_objective(P, K, L0, L1, phi, psi, x_sqnorm, Dn);
            dsq = 0.0; lin = 0.0;
            for (size_t q = 0; q < n; q++) {
                double dd = Dn[q] - D[q];
                dsq += dd * dd;
                lin += g[q] * dd;
            }
            if (fn <= f + lin + dsq / (2.0 * eta)) break;
            eta *= 0.5;
        }
        double dn = 0.0;
        for (size_t q = 0; q < n; q++) dn += D[q] * D[q];
        memcpy(D, Dn, n * sizeof(double));
        f = fn;
        if (sqrt(dsq) < tol * sqrt(dn)) { it++; break; }
    }
    free(g); free(Dn);
    if (f_out) *f_out = f;
    return it;
}

/* ---------------------------------------------------------------------------
 * Single outputs, for checks on problems too large for the full routines.
 * ------------------------------------------------------------------------ */

/* beta_k[s] = sum_p sum_tau D_kp[tau] X_p[s + tau] at n listed (k, s), s a
 * row-major index of the activation domain (Alg. 1 initialisation). */
void orc_beta_at(int P, int K, int T0, int T1, int L0, int L1, const double *X, const double *D,
                 long long n, const int *ks, const long long *ss, double *out)
{
    int Z1 = T1 - L1 + 1;
    for (long long q = 0; q < n; q++) {
        int k = ks[q], i = (int)(ss[q] / Z1), j = (int)(ss[q] % Z1);
        double acc = 0.0;
        for (int p = 0; p < P; p++)
            for (int a = 0; a < L0; a++)
                for (int b = 0; b < L1; b++)
                    acc += D[IDX4(k, p, a, b, P, L0, L1)] * X[IDX3(p, i + a, j + b, T0, T1)];
        out[q] = acc;
    }
    (void)K;
}

/* beta from its definition (Section 3) at n listed (k, s):
 * sum_p sum_tau D_kp[tau] (X - Z*D)_p[s+tau] + ||D_k||^2 Z_k[s], with the
 * residual evaluated only where it is needed. */
void orc_beta_from_Z_at(int P, int K, int T0, int T1, int L0, int L1, const double *X,
                        const double *D, const double *Z, long long n, const int *ks,
                        const long long *ss, double *out)
{
    int Z0 = T0 - L0 + 1, Z1 = T1 - L1 + 1;
    for (long long q = 0; q < n; q++) {
        int k = ks[q], i = (int)(ss[q] / Z1), j = (int)(ss[q] % Z1);
        double acc = 0.0, nrm = 0.0;
        for (int p = 0; p < P; p++)
            for (int a = 0; a < L0; a++)
                for (int b = 0; b < L1; b++) {
                    int t0 = i + a, t1 = j + b;
                    double rec = 0.0; /* (Z*D)_p[t] */
                    for (int k2 = 0; k2 < K; k2++)
                        for (int a2 = 0; a2 < L0; a2++)
                            for (int b2 = 0; b2 < L1; b2++) {
                                int s0 = t0 - a2, s1 = t1 - b2;
                                if (s0 < 0 || s0 >= Z0 || s1 < 0 || s1 >= Z1) continue;
                                double z = Z[IDX3(k2, s0, s1, Z0, Z1)];
                                if (z != 0.0) rec += z * D[IDX4(k2, p, a2, b2, P, L0, L1)];
                            }
                    double d = D[IDX4(k, p, a, b, P, L0, L1)];
                    acc += d * (X[IDX3(p, t0, t1, T0, T1)] - rec);
                    nrm += d * d;
                }
        out[q] = acc + nrm * Z[IDX3(k, i, j, Z0, Z1)];
    }
}

/* 1/2 ||X - Z * D||^2 + lambda ||Z||_1 (Eq. csc) with the reconstruction
 * accumulated from the nonzeros of Z (zero terms skipped). */
double orc_objective_sparse(int P, int K, int T0, int T1, int L0, int L1, const double *X,
                            const double *D, const double *Z, double lambda)
{
    int Z0 = T0 - L0 + 1, Z1 = T1 - L1 + 1;
    size_t nx = (size_t)P * T0 * T1;
    double *res = malloc(nx * sizeof(double));
    memcpy(res, X, nx * sizeof(double));
    double g = 0.0;
    for (int k = 0; k < K; k++)
        for (int i = 0; i < Z0; i++)
            for (int j = 0; j < Z1; j++) {
                double z = Z[IDX3(k, i, j, Z0, Z1)];
                if (z == 0.0) continue;
                g += fabs(z);
                for (int p = 0; p < P; p++)
                    for (int a = 0; a < L0; a++)
                        for (int b = 0; b < L1; b++)
                            res[IDX3(p, i + a, j + b, T0, T1)] -= z * D[IDX4(k, p, a, b, P, L0, L1)];
            }
    double f = 0.0;
    for (size_t q = 0; q < nx; q++) f += res[q] * res[q];
    free(res);
    return 0.5 * f + lambda * g;
}

/* The same objective from a list of nonzeros (atom k, row i, column j,
 * value z) instead of a dense Z, for activation maps too large to hold on
 * the host in FP64. */
double orc_objective_nz(int P, int K, int T0, int T1, int L0, int L1, const double *X,
                        const double *D, long long nnz, const long long *kk, const long long *ii,
                        const long long *jj, const double *zz, double lambda)
{
    size_t nx = (size_t)P * T0 * T1;
    double *res = malloc(nx * sizeof(double));
    memcpy(res, X, nx * sizeof(double));
    double g = 0.0;
    for (long long n = 0; n < nnz; n++) {
        int k = (int)kk[n], i = (int)ii[n], j = (int)jj[n];
        double z = zz[n];
        if (k < 0 || k >= K) continue;
        g += fabs(z);
        for (int p = 0; p < P; p++)
            for (int a = 0; a < L0; a++)
                for (int b = 0; b < L1; b++)
                    res[IDX3(p, i + a, j + b, T0, T1)] -= z * D[IDX4(k, p, a, b, P, L0, L1)];
    }
    double f = 0.0;
    for (size_t q = 0; q < nx; q++) f += res[q] * res[q];
    free(res);
    return 0.5 * f + lambda * g;
}

/* phi and psi (Eq. phi; psi = Z~ * X on Theta) from a list of nonzeros
 * (atom k, row i, column j, value z) instead of a dense Z, for activation maps
 * too large to hold on the host in FP64.  The list must not repeat a
 * coordinate.  psi takes each nonzero's term directly; for phi the nonzeros
 * are grouped by row (a counting sort), and every nonzero a is paired with
 * every nonzero b whose row and column lie within L_i - 1 of its own, adding
 * z_a z_b to phi_{k_a,k_b}[s_b - s_a]: exactly the nonzero terms of
 * sum_s Z_k[s] Z_k2[s + d] for d in Phi.  Returns 0, or -1 for an index
 * outside the activation domain. */
int orc_phi_psi_nz(int P, int K, int T0, int T1, int L0, int L1, const double *X,
                   long long nnz, const long long *kk, const long long *ii,
                   const long long *jj, const double *zz, double *phi, double *psi)
{
    int Z0 = T0 - L0 + 1, Z1 = T1 - L1 + 1;
    int W0 = 2 * L0 - 1, W1 = 2 * L1 - 1;
    memset(phi, 0, (size_t)K * K * W0 * W1 * sizeof(double));
    memset(psi, 0, (size_t)K * P * L0 * L1 * sizeof(double));
    for (long long n = 0; n < nnz; n++)
        if (kk[n] < 0 || kk[n] >= K || ii[n] < 0 || ii[n] >= Z0 || jj[n] < 0 || jj[n] >= Z1)
            return -1;
    /* psi_kp[tau] += z X_p[s + tau] */
    for (long long n = 0; n < nnz; n++) {
        int k = (int)kk[n], i = (int)ii[n], j = (int)jj[n];
        for (int p = 0; p < P; p++)
            for (int a = 0; a < L0; a++)
                for (int b = 0; b < L1; b++)
                    psi[IDX4(k, p, a, b, P, L0, L1)] += zz[n] * X[IDX3(p, i + a, j + b, T0, T1)];
    }
    /* nonzeros by row: start[r] .. start[r + 1] in `order` */
    long long *start = calloc((size_t)Z0 + 1, sizeof(long long));
    long long *fill = calloc((size_t)Z0, sizeof(long long));
    long long *order = malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(long long));
    for (long long n = 0; n < nnz; n++) start[ii[n] + 1]++;
    for (int r = 0; r < Z0; r++) start[r + 1] += start[r];
    for (long long n = 0; n < nnz; n++) order[start[ii[n]] + fill[ii[n]]++] = n;
    for (long long a = 0; a < nnz; a++) {
        int ka = (int)kk[a], ia = (int)ii[a], ja = (int)jj[a];
        int r0 = ia - (L0 - 1) < 0 ? 0 : ia - (L0 - 1);
        int r1 = ia + (L0 - 1) >= Z0 ? Z0 - 1 : ia + (L0 - 1);
        for (int r = r0; r <= r1; r++)
            for (long long q = start[r]; q < start[r + 1]; q++) {
                long long b = order[q];
                int d0 = r - ia, d1 = (int)jj[b] - ja;
                if (d1 <= -L1 || d1 >= L1) continue;
                phi[IDX4(ka, kk[b], d0 + L0 - 1, d1 + L1 - 1, K, W0, W1)] += zz[a] * zz[b];
            }
    }
    free(start);
    free(fill);
    free(order);
    return 0;
}
