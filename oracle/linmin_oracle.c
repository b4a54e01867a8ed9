/*
 * FP64 CPU oracle for LinMin's per-pixel fully constrained unmixing.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never calls it
 * and shares no code, header or table with it.
 *
 * What it computes (Schmidt, Legendre & Le Mouelic, "LinMin"):
 *
 *   Sec. 2.1, eq. LinearMixing / UnconstrainedProblem: least squares fit of
 *     one observed spectrum y (L bands) by the library S (P spectra).
 *   Sec. 2.2, eqs. NonNegativity and SumToOne: abundances x >= 0, sum x = 1
 *     (FCLS).
 *   Sec. 2.3, eq. RenormalizedProblem: the criterion is whitened by the noise
 *     covariance, C^-1 = L L^T, X' = X L, S' = S L.  For a diagonal C with
 *     per-band standard deviation sigma_l this is W = diag(1/sigma_l).
 *   Sec. 2.2 (IPLS, primal-dual interior point): the paper cites the solver
 *     without stating it.  The reading used here is the textbook Mehrotra
 *     predictor-corrector primal-dual method for the convex QP
 *
 *        minimise f(x) = 1/2 |W (y - S^T x)|^2   s.t.  x >= 0,  1^T x = 1
 *
 *     i.e. 1/2 x^T G x - c^T x + 1/2 s with G = S W^2 S^T, c = S W^2 y,
 *     s = y^T W^2 y.  The paper's F has no factor 1/2; the minimiser is the
 *     same.  Each Newton system is the bordered KKT system
 *
 *        [ G + X^-1 Lambda   1 ] [dx ]   [ -r_d - X^-1 r_c ]
 *        [ 1^T               0 ] [dnu] = [ -r_p            ]
 *
 *     with r_d = G x - c - lambda + nu 1, r_p = 1^T x - 1, r_c = x o lambda
 *     - sigma mu 1, solved as a whole by Gaussian elimination with partial
 *     pivoting (G alone may be singular: the minimiser is unique when
 *     rank [S^T; 1^T] = P, Sec. 5, not when G is regular).
 *   Sec. 2.3, last paragraph: "the error on the mixing coefficient is
 *     provided by the Hessian".  Reading: the standard deviation of the
 *     estimator under the Gaussian noise model, i.e. the square root of the
 *     diagonal of the top-left block of [[G_SS, 1],[1^T, 0]]^-1 on the
 *     support S of the solution, and 0 off the support.
 *   RMS (Sec. 3.1, Sec. 4 detection conditions): sqrt(mean_l (y - S^T x)^2),
 *     unwhitened.
 *   Constraint sets of the runs of Sec. 4 (Sec. 2.2): "slo" (x >= 0,
 *     1^T x <= 1, the inequality with its own slack and multiplier) and
 *     "pos" (x >= 0 alone), each an interior-point method of the same kind
 *     written from its own KKT conditions (oracle_slo, oracle_pos); their
 *     uncertainty is taken on the support, bordered by the sum constraint
 *     only where it is active.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------ prep */

/* Whitened Gram matrix G (P x P, row-major) and B = W^2 S (P x L) of the
 * library S (P x L row-major: row j is spectrum j).  Sec. 2.3. */
int oracle_prep(int L, int P, const float *S, const float *sigma, double *G,
                double *B)
{
    if (L <= 0 || P <= 0) return 1;
    for (int l = 0; l < L; l++)
        if (!(sigma[l] > 0.0f)) return 2;
    for (int i = 0; i < P; i++) {
        for (int j = 0; j <= i; j++) {
            long double acc = 0.0L;
            for (int l = 0; l < L; l++) {
                long double w = 1.0L / (long double)sigma[l];
                acc += ((long double)S[(size_t)i * L + l] * w) *
                       ((long double)S[(size_t)j * L + l] * w);
            }
            G[(size_t)i * P + j] = (double)acc;
            G[(size_t)j * P + i] = (double)acc;
        }
        for (int l = 0; l < L; l++) {
            long double w = 1.0L / (long double)sigma[l];
            B[(size_t)i * L + l] = (double)((long double)S[(size_t)i * L + l] * w * w);
        }
    }
    return 0;
}

/* c = B y (P values) and s = y^T W^2 y for one pixel y. */
void oracle_project(int L, int P, const double *B, const float *sigma,
                    const float *y, double *c, double *s)
{
    for (int j = 0; j < P; j++) {
        long double acc = 0.0L;
        for (int l = 0; l < L; l++) acc += (long double)B[(size_t)j * L + l] * y[l];
        c[j] = (double)acc;
    }
    long double ss = 0.0L;
    for (int l = 0; l < L; l++) {
        long double w = (long double)y[l] / (long double)sigma[l];
        ss += w * w;
    }
    *s = (double)ss;
}

/* ----------------------------------------------------- dense linear algebra */

/* LU with partial pivoting of the n x n row-major matrix M, in place.
 * Returns 0, or 1 when a pivot is exactly zero. */
static int lu_factor(int n, double *M, int *piv)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(M[(size_t)k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double v = fabs(M[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (best == 0.0) return 1;
        if (p != k)
            for (int j = 0; j < n; j++) {
                double t = M[(size_t)k * n + j];
                M[(size_t)k * n + j] = M[(size_t)p * n + j];
                M[(size_t)p * n + j] = t;
            }
        for (int i = k + 1; i < n; i++) {
            double m = M[(size_t)i * n + k] / M[(size_t)k * n + k];
            M[(size_t)i * n + k] = m;
            for (int j = k + 1; j < n; j++) M[(size_t)i * n + j] -= m * M[(size_t)k * n + j];
        }
    }
    return 0;
}

static void lu_solve(int n, const double *M, const int *piv, double *b)
{
    for (int k = 0; k < n; k++) {
        int p = piv[k];
        if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < i; j++) b[i] -= M[(size_t)i * n + j] * b[j];
    for (int i = n - 1; i >= 0; i--) {
        for (int j = i + 1; j < n; j++) b[i] -= M[(size_t)i * n + j] * b[j];
        b[i] /= M[(size_t)i * n + i];
    }
}

/* ------------------------------------------------------------- IPLS (FP64) */

/* Largest step in (0, 1] keeping v + a dv >= 0 (fraction-to-boundary). */
static double max_step(int P, const double *v, const double *dv)
{
    double a = 1.0;
    for (int i = 0; i < P; i++)
        if (dv[i] < 0.0) {
            double t = -v[i] / dv[i];
            if (t < a) a = t;
        }
    return a;
}

/* Status codes of oracle_fcls. */
#define OR_OK 0
#define OR_MAXITER 1
#define OR_SINGULAR 2

/*
 * Mehrotra predictor-corrector IPM for min 1/2 x'Gx - c'x + s/2,
 * x >= 0, 1'x = 1.  G is P x P row-major.  Writes x, lambda, nu, the
 * iteration count and the final mu = x'lambda/P.  Returns a status code.
 *
 * Start: x = 1/P, lambda = max(|c|_inf / P, 1e-3) 1, nu = 0.
 * Stop:  |r_d|_inf <= 1e-12 (1 + |c|_inf), |r_p| <= 1e-14,
 *        mu <= 1e-13 (1 + |f|), or max_iter iterations.
 * Step:  Mehrotra's corrected direction, or a centred Newton direction
 *        (r_c = x o lambda - mu/2) when the corrected step would not reduce
 *        mu by 1% of its length; one length alpha = min(1, 0.995 * max
 *        feasible) for x, lambda and nu together.  In a QP the dual residual r_d = G x - c - lambda +
 *        nu 1 couples x and (lambda, nu): after a step it is r_d (1 -
 *        alpha_d) + (alpha_p - alpha_d) G dx, so separate primal and dual
 *        lengths (the linear-programming rule) can leave it stuck.
 */
int oracle_fcls(int P, const double *G, const double *c, double s, int max_iter,
                double *x, double *lam, double *nu_out, int *iters_out,
                double *mu_out)
{
    const int n = P + 1;
    double *K = malloc(sizeof(double) * n * n);
    int *piv = malloc(sizeof(int) * n);
    double *rd = malloc(sizeof(double) * P), *gx = malloc(sizeof(double) * P);
    double *rhs = malloc(sizeof(double) * n), *dxa = malloc(sizeof(double) * P);
    double *dla = malloc(sizeof(double) * P), *dx = malloc(sizeof(double) * P);
    double *dl = malloc(sizeof(double) * P), *rc = malloc(sizeof(double) * P);
    double *tmp = malloc(sizeof(double) * P);
    int status = OR_MAXITER, it = 0;

    double cinf = 0.0;
    for (int i = 0; i < P; i++) cinf = fmax(cinf, fabs(c[i]));
    double lam0 = fmax(cinf / P, 1e-3);
    double nu = 0.0;
    for (int i = 0; i < P; i++) { x[i] = 1.0 / P; lam[i] = lam0; }
    double mu = 0.0;

    for (it = 0; it <= max_iter; it++) {
        /* residuals */
        double rp = -1.0, rdinf = 0.0, xgx = 0.0, cx = 0.0;
        mu = 0.0;
        for (int i = 0; i < P; i++) {
            double acc = 0.0;
            for (int j = 0; j < P; j++) acc += G[(size_t)i * P + j] * x[j];
            gx[i] = acc;
            rd[i] = acc - c[i] - lam[i] + nu;
            rdinf = fmax(rdinf, fabs(rd[i]));
            rp += x[i];
            mu += x[i] * lam[i];
            xgx += x[i] * acc;
            cx += c[i] * x[i];
        }
        mu /= P;
        double f = 0.5 * xgx - cx + 0.5 * s;
        if (rdinf <= 1e-12 * (1.0 + cinf) && fabs(rp) <= 1e-14 &&
            mu <= 1e-13 * (1.0 + fabs(f))) {
            status = OR_OK;
            break;
        }
        if (it == max_iter) break;

        /* bordered KKT matrix, factored once for both solves */
        for (int i = 0; i < P; i++) {
            for (int j = 0; j < P; j++) K[(size_t)i * n + j] = G[(size_t)i * P + j];
            K[(size_t)i * n + i] += lam[i] / x[i];
            K[(size_t)i * n + P] = 1.0;
            K[(size_t)P * n + i] = 1.0;
        }
        K[(size_t)P * n + P] = 0.0;
        if (lu_factor(n, K, piv)) { status = OR_SINGULAR; break; }

        /* predictor (affine scaling): r_c = x o lambda */
        for (int i = 0; i < P; i++) rhs[i] = -rd[i] - lam[i];
        rhs[P] = -rp;
        lu_solve(n, K, piv, rhs);
        for (int i = 0; i < P; i++) {
            dxa[i] = rhs[i];
            dla[i] = -lam[i] - lam[i] / x[i] * dxa[i];
        }
        double ap = max_step(P, x, dxa), ad = max_step(P, lam, dla);
        double mua = 0.0;
        for (int i = 0; i < P; i++) mua += (x[i] + ap * dxa[i]) * (lam[i] + ad * dla[i]);
        mua /= P;
        double sig = pow(mua / mu, 3.0);

        /* corrector: r_c = x o lambda + dx_aff o dlam_aff - sigma mu; if
         * its step does not reduce mu by at least 1% of the step length,
         * a centred Newton step (r_c = x o lambda - mu/2) instead, which
         * breaks the cycles the corrector can fall into */
        double dnu = 0.0, a = 0.0;
        for (int pass = 0; pass < 2; pass++) {
            for (int i = 0; i < P; i++) {
                rc[i] = pass == 0 ? x[i] * lam[i] + dxa[i] * dla[i] - sig * mu
                                  : x[i] * lam[i] - 0.5 * mu;
                rhs[i] = -rd[i] - rc[i] / x[i];
            }
            rhs[P] = -rp;
            lu_solve(n, K, piv, rhs);
            dnu = rhs[P];
            for (int i = 0; i < P; i++) {
                dx[i] = rhs[i];
                dl[i] = (-rc[i] - lam[i] * dx[i]) / x[i];
            }
            a = fmin(1.0, 0.995 * fmin(max_step(P, x, dx), max_step(P, lam, dl)));
            double mun = 0.0;
            for (int i = 0; i < P; i++) mun += (x[i] + a * dx[i]) * (lam[i] + a * dl[i]);
            if (mun / P <= (1.0 - 0.01 * a) * mu) break;
        }
        for (int i = 0; i < P; i++) {
            x[i] += a * dx[i];
            lam[i] += a * dl[i];
        }
        nu += a * dnu;
        (void)tmp;
    }
    /* x <- max(x, 0) / sum */
    double sum = 0.0;
    for (int i = 0; i < P; i++) { if (x[i] < 0.0) x[i] = 0.0; sum += x[i]; }
    for (int i = 0; i < P; i++) x[i] /= sum;

    *nu_out = nu;
    *iters_out = it;
    *mu_out = mu;
    free(K); free(piv); free(rd); free(gx); free(rhs); free(dxa);
    free(dla); free(dx); free(dl); free(rc); free(tmp);
    return status;
}

/* ------------------------------------- constraint sets pos and slo (Sec. 2.2)
 *
 * The paper unmixes real images under three constraint sets (Sec. 2.2 and
 * the runs of Sec. 4): "sto" (x >= 0, 1^T x = 1, oracle_fcls above), "slo"
 * (x >= 0, 1^T x <= 1) and "pos" (x >= 0 alone).  Each is written here from
 * its own definition, as a primal-dual interior-point method of the same
 * kind (Mehrotra predictor-corrector, one step length of 0.995 of the
 * largest feasible one for primal and dual together, LU with partial
 * pivoting).
 */

/*
 * pos: minimise 1/2 x'Gx - c'x + s/2 subject to x >= 0, with no bound on the
 * sum.  KKT: G x - c - lambda = 0, x o lambda = 0, x, lambda >= 0.  Newton:
 *    (G + X^-1 Lambda) dx = -r_d - X^-1 r_c,   dlambda = -X^-1 (r_c + Lambda dx)
 * with r_d = G x - c - lambda, r_c = x o lambda - sigma mu 1, mu = x'lambda/P.
 * Start x = 1/P, lambda = max(|c|_inf / P, 1e-3) 1.  Stop: |r_d|_inf <=
 * 1e-12 (1 + |c|_inf) and mu <= 1e-13 (1 + |f|).  The minimiser is unique
 * when G is regular (rank S = P).
 */
int oracle_pos(int P, const double *G, const double *c, double s, int max_iter,
               double *x, double *lam, int *iters_out, double *mu_out)
{
    double *K = malloc(sizeof(double) * P * P);
    int *piv = malloc(sizeof(int) * P);
    double *rd = malloc(sizeof(double) * P), *rhs = malloc(sizeof(double) * P);
    double *dxa = malloc(sizeof(double) * P), *dla = malloc(sizeof(double) * P);
    double *dx = malloc(sizeof(double) * P), *dl = malloc(sizeof(double) * P);
    double *rc = malloc(sizeof(double) * P);
    int status = OR_MAXITER, it = 0;
    double cinf = 0.0;
    for (int i = 0; i < P; i++) cinf = fmax(cinf, fabs(c[i]));
    const double lam0 = fmax(cinf / P, 1e-3);
    for (int i = 0; i < P; i++) { x[i] = 1.0 / P; lam[i] = lam0; }
    double mu = 0.0;
    for (it = 0; it <= max_iter; it++) {
        double rdinf = 0.0, xgx = 0.0, cx = 0.0;
        mu = 0.0;
        for (int i = 0; i < P; i++) {
            double acc = 0.0;
            for (int j = 0; j < P; j++) acc += G[(size_t)i * P + j] * x[j];
            rd[i] = acc - c[i] - lam[i];
            rdinf = fmax(rdinf, fabs(rd[i]));
            mu += x[i] * lam[i];
            xgx += x[i] * acc;
            cx += c[i] * x[i];
        }
        mu /= P;
        const double f = 0.5 * xgx - cx + 0.5 * s;
        if (rdinf <= 1e-12 * (1.0 + cinf) && mu <= 1e-13 * (1.0 + fabs(f))) {
            status = OR_OK;
            break;
        }
        if (it == max_iter) break;
        for (int i = 0; i < P; i++) {
            for (int j = 0; j < P; j++) K[(size_t)i * P + j] = G[(size_t)i * P + j];
            K[(size_t)i * P + i] += lam[i] / x[i];
        }
        if (lu_factor(P, K, piv)) { status = OR_SINGULAR; break; }
        /* predictor: r_c = x o lambda */
        for (int i = 0; i < P; i++) rhs[i] = -rd[i] - lam[i];
        lu_solve(P, K, piv, rhs);
        for (int i = 0; i < P; i++) {
            dxa[i] = rhs[i];
            dla[i] = -lam[i] - lam[i] / x[i] * dxa[i];
        }
        double ap = max_step(P, x, dxa), ad = max_step(P, lam, dla);
        double mua = 0.0;
        for (int i = 0; i < P; i++) mua += (x[i] + ap * dxa[i]) * (lam[i] + ad * dla[i]);
        mua /= P;
        const double sig = pow(mua / mu, 3.0);
        /* corrector: r_c = x o lambda + dx_aff o dlam_aff - sigma mu 1, or
         * the centred Newton step when it does not reduce mu (as in
         * oracle_fcls) */
        double a = 0.0;
        for (int pass = 0; pass < 2; pass++) {
            for (int i = 0; i < P; i++) {
                rc[i] = pass == 0 ? x[i] * lam[i] + dxa[i] * dla[i] - sig * mu
                                  : x[i] * lam[i] - 0.5 * mu;
                rhs[i] = -rd[i] - rc[i] / x[i];
            }
            lu_solve(P, K, piv, rhs);
            for (int i = 0; i < P; i++) {
                dx[i] = rhs[i];
                dl[i] = (-rc[i] - lam[i] * dx[i]) / x[i];
            }
            a = fmin(1.0, 0.995 * fmin(max_step(P, x, dx), max_step(P, lam, dl)));
            double mun = 0.0;
            for (int i = 0; i < P; i++) mun += (x[i] + a * dx[i]) * (lam[i] + a * dl[i]);
            if (mun / P <= (1.0 - 0.01 * a) * mu) break;
        }
        for (int i = 0; i < P; i++) {
            x[i] += a * dx[i];
            lam[i] += a * dl[i];
        }
    }
    for (int i = 0; i < P; i++) if (x[i] < 0.0) x[i] = 0.0;
    *iters_out = it;
    *mu_out = mu;
    free(K); free(piv); free(rd); free(rhs); free(dxa); free(dla); free(dx); free(dl);
    free(rc);
    return status;
}

/*
 * slo: minimise 1/2 x'Gx - c'x + s/2 subject to x >= 0 and 1'x <= 1.  The
 * inequality gets its own slack w = 1 - 1'x >= 0 and multiplier omega >= 0.
 * KKT: G x - c - lambda + omega 1 = 0, 1'x + w = 1, x o lambda = 0,
 * w omega = 0.  Eliminating dlambda and dw from the Newton equations
 * leaves the bordered system
 *    [ G + X^-1 Lambda   1          ] [dx    ]   [ -r_d - X^-1 r_c      ]
 *    [ 1^T              -w / omega  ] [domega] = [ -r_p + r_cw / omega  ]
 * with r_d = G x - c - lambda + omega 1, r_p = 1'x + w - 1, r_c = x o lambda
 * - sigma mu 1, r_cw = w omega - sigma mu, mu = (x'lambda + w omega)/(P+1);
 * then dlambda = -X^-1 (r_c + Lambda dx), dw = -(r_cw + w domega) / omega.
 * Start x = 1/(P+1) (so w = 1/(P+1)), lambda = omega = max(|c|_inf / P, 1e-3).
 * Stop: |r_d|_inf <= 1e-12 (1 + |c|_inf), |r_p| <= 1e-14 and
 * mu <= 1e-13 (1 + |f|).  The minimiser is unique when rank S = P.
 */
int oracle_slo(int P, const double *G, const double *c, double s, int max_iter,
               double *x, double *lam, double *w_out, double *omega_out, int *iters_out,
               double *mu_out)
{
    const int n = P + 1;
    double *K = malloc(sizeof(double) * n * n);
    int *piv = malloc(sizeof(int) * n);
    double *rd = malloc(sizeof(double) * P), *rhs = malloc(sizeof(double) * n);
    double *dxa = malloc(sizeof(double) * P), *dla = malloc(sizeof(double) * P);
    double *dx = malloc(sizeof(double) * P), *dl = malloc(sizeof(double) * P);
    double *rc = malloc(sizeof(double) * P);
    int status = OR_MAXITER, it = 0;
    double cinf = 0.0;
    for (int i = 0; i < P; i++) cinf = fmax(cinf, fabs(c[i]));
    const double lam0 = fmax(cinf / P, 1e-3);
    for (int i = 0; i < P; i++) { x[i] = 1.0 / (P + 1); lam[i] = lam0; }
    double w = 1.0 / (P + 1), om = lam0, mu = 0.0;
    for (it = 0; it <= max_iter; it++) {
        double rdinf = 0.0, rp = w - 1.0, xgx = 0.0, cx = 0.0;
        mu = w * om;
        for (int i = 0; i < P; i++) {
            double acc = 0.0;
            for (int j = 0; j < P; j++) acc += G[(size_t)i * P + j] * x[j];
            rd[i] = acc - c[i] - lam[i] + om;
            rdinf = fmax(rdinf, fabs(rd[i]));
            rp += x[i];
            mu += x[i] * lam[i];
            xgx += x[i] * acc;
            cx += c[i] * x[i];
        }
        mu /= P + 1;
        const double f = 0.5 * xgx - cx + 0.5 * s;
        if (rdinf <= 1e-12 * (1.0 + cinf) && fabs(rp) <= 1e-14 &&
            mu <= 1e-13 * (1.0 + fabs(f))) {
            status = OR_OK;
            break;
        }
        if (it == max_iter) break;
        for (int i = 0; i < P; i++) {
            for (int j = 0; j < P; j++) K[(size_t)i * n + j] = G[(size_t)i * P + j];
            K[(size_t)i * n + i] += lam[i] / x[i];
            K[(size_t)i * n + P] = 1.0;
            K[(size_t)P * n + i] = 1.0;
        }
        K[(size_t)P * n + P] = -w / om;
        if (lu_factor(n, K, piv)) { status = OR_SINGULAR; break; }
        /* predictor: r_c = x o lambda, r_cw = w omega */
        for (int i = 0; i < P; i++) rhs[i] = -rd[i] - lam[i];
        rhs[P] = -rp + w;
        lu_solve(n, K, piv, rhs);
        for (int i = 0; i < P; i++) {
            dxa[i] = rhs[i];
            dla[i] = -lam[i] - lam[i] / x[i] * dxa[i];
        }
        const double doa = rhs[P];
        const double dwa = -w - w * doa / om;
        double ap = fmin(max_step(P, x, dxa), max_step(1, &w, &dwa));
        double ad = fmin(max_step(P, lam, dla), max_step(1, &om, &doa));
        double mua = (w + ap * dwa) * (om + ad * doa);
        for (int i = 0; i < P; i++) mua += (x[i] + ap * dxa[i]) * (lam[i] + ad * dla[i]);
        mua /= P + 1;
        const double sig = pow(mua / mu, 3.0);
        /* corrector, or the centred Newton step when it does not reduce
         * mu (as in oracle_fcls) */
        double dom = 0.0, dw = 0.0, a = 0.0;
        for (int pass = 0; pass < 2; pass++) {
            for (int i = 0; i < P; i++) {
                rc[i] = pass == 0 ? x[i] * lam[i] + dxa[i] * dla[i] - sig * mu
                                  : x[i] * lam[i] - 0.5 * mu;
                rhs[i] = -rd[i] - rc[i] / x[i];
            }
            const double rcw = pass == 0 ? w * om + dwa * doa - sig * mu : w * om - 0.5 * mu;
            rhs[P] = -rp + rcw / om;
            lu_solve(n, K, piv, rhs);
            for (int i = 0; i < P; i++) {
                dx[i] = rhs[i];
                dl[i] = (-rc[i] - lam[i] * dx[i]) / x[i];
            }
            dom = rhs[P];
            dw = -(rcw + w * dom) / om;
            a = fmin(1.0, 0.995 * fmin(fmin(max_step(P, x, dx), max_step(1, &w, &dw)),
                                       fmin(max_step(P, lam, dl), max_step(1, &om, &dom))));
            double mun = (w + a * dw) * (om + a * dom);
            for (int i = 0; i < P; i++) mun += (x[i] + a * dx[i]) * (lam[i] + a * dl[i]);
            if (mun / (P + 1) <= (1.0 - 0.01 * a) * mu) break;
        }
        for (int i = 0; i < P; i++) {
            x[i] += a * dx[i];
            lam[i] += a * dl[i];
        }
        w += a * dw;
        om += a * dom;
    }
    for (int i = 0; i < P; i++) if (x[i] < 0.0) x[i] = 0.0;
    *w_out = w;
    *omega_out = om;
    *iters_out = it;
    *mu_out = mu;
    free(K); free(piv); free(rd); free(rhs); free(dxa); free(dla); free(dx); free(dl);
    free(rc);
    return status;
}

/* --------------------------------------------------------- uncertainty */

/* Support of the final iterate: i is active when its barrier term
 * lambda_i / x_i is below its curvature G_ii. */
int oracle_support(int P, const double *G, const double *x, const double *lam,
                   int *in_S)
{
    int k = 0;
    for (int i = 0; i < P; i++) {
        in_S[i] = lam[i] < x[i] * G[(size_t)i * P + i];
        k += in_S[i];
    }
    return k;
}

/* sigma_x of an active set: sqrt of the diagonal of the inverse of the
 * Hessian restricted to the support S, bordered by the sum constraint when
 * it is active (bordered != 0: top-left block of [[G_SS, 1],[1^T, 0]]^-1;
 * else (G_SS)^-1), and 0 off the support.  Returns 0, or 1 when that system
 * is singular (sx is then set to NaN on S). */
int oracle_sigma_x_set(int P, const double *G, const int *in_S, int bordered, double *sx)
{
    int k = 0;
    int *idx = malloc(sizeof(int) * P);
    for (int i = 0; i < P; i++) if (in_S[i]) idx[k++] = i;
    for (int i = 0; i < P; i++) sx[i] = 0.0;
    const int n = k + (bordered ? 1 : 0);
    int bad = 0;
    double *K = malloc(sizeof(double) * (n * n + 1));
    int *piv = malloc(sizeof(int) * (n + 1));
    double *e = malloc(sizeof(double) * (n + 1));
    for (int a = 0; a < k; a++) {
        for (int b = 0; b < k; b++) K[(size_t)a * n + b] = G[(size_t)idx[a] * P + idx[b]];
        if (bordered) {
            K[(size_t)a * n + k] = 1.0;
            K[(size_t)k * n + a] = 1.0;
        }
    }
    if (bordered) K[(size_t)k * n + k] = 0.0;
    if (k == 0 || lu_factor(n, K, piv)) {
        bad = 1;
        for (int a = 0; a < k; a++) sx[idx[a]] = NAN;
    } else {
        for (int a = 0; a < k; a++) {
            for (int b = 0; b < n; b++) e[b] = (a == b) ? 1.0 : 0.0;
            lu_solve(n, K, piv, e);
            /* e[a] = [K^-1]_aa; it is >= 0 up to rounding */
            sx[idx[a]] = sqrt(fmax(e[a], 0.0));
        }
    }
    free(idx); free(K); free(piv); free(e);
    return bad;
}

/* sigma_x under the sum-to-one constraint (always bordered). */
int oracle_sigma_x(int P, const double *G, const int *in_S, double *sx)
{
    return oracle_sigma_x_set(P, G, in_S, 1, sx);
}

/* Unwhitened RMS of the fit: sqrt(mean_l (y_l - sum_j x_j S_jl)^2). */
double oracle_rms(int L, int P, const float *S, const double *x, const float *y)
{
    long double acc = 0.0L;
    for (int l = 0; l < L; l++) {
        long double m = 0.0L;
        for (int j = 0; j < P; j++) m += (long double)x[j] * S[(size_t)j * L + l];
        long double r = (long double)y[l] - m;
        acc += r * r;
    }
    return (double)sqrtl(acc / L);
}

/* ------------------------------------------------------------ whole cube */

typedef struct {
    int L, P, max_iter;
    const float *S, *sigma, *X;
    const double *G, *B;
    long long lo, hi;
    double *x, *sx, *rms, *lam, *nu, *mu;
    int *iters, *status, *ksup;
    int constraint;               /* 0 sto, 1 slo, 2 pos */
    double *slack, *omega;        /* slo: w and omega per pixel (optional) */
} job_t;

static void *unmix_range(void *arg)
{
    job_t *j = (job_t *)arg;
    int P = j->P, L = j->L;
    double *c = malloc(sizeof(double) * P);
    double *lam = malloc(sizeof(double) * P);
    int *in_S = malloc(sizeof(int) * P);
    for (long long n = j->lo; n < j->hi; n++) {
        const float *y = j->X + (size_t)n * L;
        double s, nu, mu;
        int it;
        double *x = j->x + (size_t)n * P;
        oracle_project(L, P, j->B, j->sigma, y, c, &s);
        int st, k, bordered = 1;
        double w = 0.0, om = 0.0;
        if (j->constraint == 2) {
            st = oracle_pos(P, j->G, c, s, j->max_iter, x, lam, &it, &mu);
            nu = 0.0;
            bordered = 0;
        } else if (j->constraint == 1) {
            st = oracle_slo(P, j->G, c, s, j->max_iter, x, lam, &w, &om, &it, &mu);
            nu = om;
            /* the sum constraint is active when its multiplier exceeds its
             * slack (unit curvature for the slack, as lambda_i < x_i G_ii
             * for the coordinates) */
            bordered = om > w;
        } else {
            st = oracle_fcls(P, j->G, c, s, j->max_iter, x, lam, &nu, &it, &mu);
        }
        k = oracle_support(P, j->G, x, lam, in_S);
        if (oracle_sigma_x_set(P, j->G, in_S, bordered, j->sx + (size_t)n * P)) st |= 4;
        if (j->slack) j->slack[n] = w;
        if (j->omega) j->omega[n] = om;
        j->rms[n] = oracle_rms(L, P, j->S, x, y);
        j->iters[n] = (st & 3) == OR_OK ? it : -it - 1;
        if (j->status) j->status[n] = st;
        if (j->ksup) j->ksup[n] = k;
        if (j->lam) memcpy(j->lam + (size_t)n * P, lam, sizeof(double) * P);
        if (j->nu) j->nu[n] = nu;
        if (j->mu) j->mu[n] = mu;
    }
    free(c); free(lam); free(in_S);
    return NULL;
}

int oracle_nproc(void)
{
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/*
 * Unmix N pixels of the pixel-major cube X (N x L) against the library S
 * (P x L).  Outputs (caller-allocated): x and sx (N x P), rms (N), iters (N,
 * negative = did not converge); optional (may be NULL): lam (N x P), nu, mu,
 * status, ksup (N).  nthreads <= 0 uses every online core.  Returns 0, or a
 * non-zero code for invalid arguments.
 */
int oracle_unmix_set(int L, int P, const float *S, const float *sigma, long long N,
                     const float *X, int constraint, int max_iter, int nthreads, double *x,
                     double *sx, double *rms, int *iters, double *lam, double *nu,
                     double *mu, int *status, int *ksup, double *slack, double *omega)
{
    if (constraint < 0 || constraint > 2) return 1;
    if (N < 0 || L <= 0 || P <= 0) return 1;
    if (N == 0) return 0;
    double *G = malloc(sizeof(double) * P * P);
    double *B = malloc(sizeof(double) * (size_t)P * L);
    int rc = oracle_prep(L, P, S, sigma, G, B);
    if (rc) { free(G); free(B); return rc; }
    if (nthreads <= 0) nthreads = oracle_nproc();
    if ((long long)nthreads > N) nthreads = (int)N;
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    job_t *jobs = malloc(sizeof(job_t) * nthreads);
    for (int t = 0; t < nthreads; t++) {
        job_t j = {L, P, max_iter, S, sigma, X, G, B,
                   N * t / nthreads, N * (t + 1) / nthreads,
                   x, sx, rms, lam, nu, mu, iters, status, ksup,
                   constraint, slack, omega};
        jobs[t] = j;
        pthread_create(&th[t], NULL, unmix_range, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th); free(jobs); free(G); free(B);
    return 0;
}

/* Sum-to-one unmixing of a whole cube (the sto constraint set). */
int oracle_unmix(int L, int P, const float *S, const float *sigma, long long N,
                 const float *X, int max_iter, int nthreads, double *x,
                 double *sx, double *rms, int *iters, double *lam, double *nu,
                 double *mu, int *status, int *ksup)
{
    return oracle_unmix_set(L, P, S, sigma, N, X, 0, max_iter, nthreads, x, sx, rms, iters,
                            lam, nu, mu, status, ksup, NULL, NULL);
}
