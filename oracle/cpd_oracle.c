/*
 * FP64 CPU oracle for the EM loop of Fast Coherent Point Drift
 * (Feng, Feng & Zhu, "Fast Coherent Point Drift", arXiv 2006.06281).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the library itself never does.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * Notation follows the paper: X (M x D) model points, Y (N x D) scene
 * points, T = X + Phi W the transformed model points (Eq. 9-11), Phi the
 * Gaussian Gram matrix of X, sigma2 the GMM variance, w the outlier weight,
 * lambda the regularisation weight, beta the kernel width.  Points are stored
 * row-major (point-major, D contiguous).  Everything is double precision,
 * straightforward loops, each step in the order the paper states it.  OpenMP
 * only splits independent outer loops (each output keeps one fixed summation
 * order), so results do not depend on the thread count.
 *
 * The eigendecomposition of Phi (Eq. 16) is not here: the Python side calls
 * LAPACK (numpy.linalg.eigh) and passes U (M x K, row-major) and the
 * eigenvalues (descending, clamped at 0) in.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_get_num_threads(void) { return 1; }
static int omp_get_thread_num(void) { return 0; }
#endif

#define ORACLE_OK 0
#define ORACLE_ENUMERIC 5

/* Eq. 11: Phi_ij = exp(-|x_i - x_j|^2 / (2 beta^2)), M x M row-major. */
void fcpd_oracle_gram(const double *X, int64_t M, int32_t D, double beta, double *Phi)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        for (int64_t j = 0; j < M; ++j) {
            double d2 = 0.0;
            for (int32_t d = 0; d < D; ++d) {
                double diff = X[i * D + d] - X[j * D + d];
                d2 += diff * diff;
            }
            Phi[i * M + j] = exp(-d2 / (2.0 * beta * beta));
        }
    }
}

/* Initial variance "from the data" (the paper does not state it; reading):
 * sigma2_0 = sum_m sum_n |y_n - x_m|^2 / (D M N), straight from the
 * definition, O(MN).  W_0 = 0, so T_0 = X. */
double fcpd_oracle_sigma2_init(const double *X, int64_t M, const double *Y, int64_t N, int32_t D)
{
    double total = 0.0;
#pragma omp parallel for schedule(static) reduction(+:total)
    for (int64_t m = 0; m < M; ++m) {
        double row = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            for (int32_t d = 0; d < D; ++d) {
                double diff = Y[n * D + d] - X[m * D + d];
                row += diff * diff;
            }
        }
        total += row;
    }
    return total / ((double)D * (double)M * (double)N);
}

/* Outlier constant of Eq. 4: c = (2 pi sigma2)^(D/2) * w/(1-w) * M/N. */
double fcpd_oracle_outlier_c(double sigma2, double w, int64_t M, int64_t N, int32_t D)
{
    return pow(2.0 * M_PI * sigma2, 0.5 * (double)D) * (w / (1.0 - w)) * ((double)M / (double)N);
}

static double gauss_e(const double *T, int64_t m, const double *Y, int64_t n, int32_t D, double sigma2)
{
    double d2 = 0.0;
    for (int32_t d = 0; d < D; ++d) {
        double diff = Y[n * D + d] - T[m * D + d];
        d2 += diff * diff;
    }
    return exp(-d2 / (2.0 * sigma2));
}

/*
 * E-step.  Eq. 4: p_mn = e_mn / (sum_k e_kn + c), e_mn = exp(-|y_n - t_m|^2 / (2 sigma2)).
 * Eq. 5 (the corresponding constraint): each row of P is rescaled to sum to 1,
 * p^_mn = p_mn / sum_n p_mn, and Ytil_m = sum_n p^_mn y_n (the estimate
 * defined after Eq. 13).
 *
 * Outputs (any may be NULL except where noted):
 *   den[N]   sum_k e_kn + c                      (column denominators of Eq. 4)
 *   P1[M]    sum_n p_mn                          (row mass before Eq. 5)
 *   PY[M*D]  sum_n p_mn y_n
 *   S[M]     sum_n p_mn |y_n|^2
 *   Ytil[M*D] PY_m / P1_m                        (required)
 *   loglik   Eq. 3 log-likelihood at (T, sigma2): sum_n ln den_n
 *            + N ln((1-w)/M) - (N D / 2) ln(2 pi sigma2)
 * Returns ORACLE_ENUMERIC if some row mass P1_m is 0 or not finite (the row
 * cannot be normalised), else ORACLE_OK.
 */
int fcpd_oracle_estep(const double *T, int64_t M, const double *Y, int64_t N, int32_t D,
                      double sigma2, double w, double *den, double *P1, double *PY,
                      double *S, double *Ytil, double *loglik)
{
    const double c = fcpd_oracle_outlier_c(sigma2, w, M, N, D);
    double *dn = den;
    /* the column denominators are needed by every row: den must be given;
     * at most 16 coordinates per point */
    if (!dn || !Ytil || D < 1 || D > 16) return -1;

#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double s = 0.0;
        for (int64_t k = 0; k < M; ++k)
            s += gauss_e(T, k, Y, n, D, sigma2);
        dn[n] = s + c;
    }

    int bad = 0;
#pragma omp parallel for schedule(static) reduction(|:bad)
    for (int64_t m = 0; m < M; ++m) {
        double p1 = 0.0, s2 = 0.0;
        double py[16];
        for (int32_t d = 0; d < D; ++d) py[d] = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            double p = gauss_e(T, m, Y, n, D, sigma2) / dn[n];
            double yy = 0.0;
            p1 += p;
            for (int32_t d = 0; d < D; ++d) {
                py[d] += p * Y[n * D + d];
                yy += Y[n * D + d] * Y[n * D + d];
            }
            s2 += p * yy;
        }
        if (P1) P1[m] = p1;
        if (S) S[m] = s2;
        for (int32_t d = 0; d < D; ++d) {
            if (PY) PY[m * D + d] = py[d];
            Ytil[m * D + d] = py[d] / p1;
        }
        if (!(p1 > 0.0) || !isfinite(p1)) bad = 1;
    }

    if (loglik) {
        double ll = 0.0;
        for (int64_t n = 0; n < N; ++n) ll += log(dn[n]);
        ll += (double)N * log((1.0 - w) / (double)M) - 0.5 * (double)N * (double)D * log(2.0 * M_PI * sigma2);
        *loglik = ll;
    }
    return bad ? ORACLE_ENUMERIC : ORACLE_OK;
}

/*
 * M-step, Eq. 17 (K = M) or Eq. 20 (K < M, top-K eigenpairs):
 *   W = U (Lambda + lambda sigma2 I)^-1 U^T (Ytil - X)
 * and the transformed points T = X + Phi W (Eq. 9-11) with Phi taken through
 * its eigendecomposition (Eq. 16): Phi U = U Lambda, hence
 *   T = X + U diag(l_i / (l_i + lambda sigma2)) U^T (Ytil - X).
 * U is M x K row-major (U[m*K + i] = i-th eigenvector, m-th entry), lam[K].
 * A (K x D, required) receives U^T (Ytil - X); W (M x D, optional) the
 * coefficients of Eq. 17 / Eq. 20.
 */
void fcpd_oracle_mstep(const double *U, const double *lam, int64_t M, int64_t K,
                       const double *X, const double *Ytil, int32_t D,
                       double lambda, double sigma2, double *T, double *W, double *A)
{
    /* the diagonal update: only (Lambda + lambda sigma2 I)^-1 changes per
     * iteration (the paper's point after Eq. 17) */
    double *dinv = NULL, *sdiag = NULL;
    dinv = (double *)malloc((size_t)K * sizeof(double));
    sdiag = (double *)malloc((size_t)K * sizeof(double));
    for (int64_t i = 0; i < K; ++i) {
        dinv[i] = 1.0 / (lam[i] + lambda * sigma2);
        sdiag[i] = lam[i] * dinv[i];
    }
    /* A = U^T (Ytil - X): for each (i, d) a sum over m in ascending order.
     * Threads split the columns i; each walks the rows m in order. */
#pragma omp parallel
    {
        int nt = omp_get_num_threads(), t = omp_get_thread_num();
        int64_t i0 = K * t / nt, i1 = K * (t + 1) / nt;
        for (int64_t i = i0; i < i1; ++i)
            for (int32_t d = 0; d < D; ++d) A[i * D + d] = 0.0;
        for (int64_t m = 0; m < M; ++m) {
            for (int64_t i = i0; i < i1; ++i) {
                double u = U[m * K + i];
                for (int32_t d = 0; d < D; ++d)
                    A[i * D + d] += u * (Ytil[m * D + d] - X[m * D + d]);
            }
        }
    }
    /* T = X + U diag(l_i / (l_i + lambda sigma2)) A ; W = U diag(1/(l_i + lambda sigma2)) A */
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < M; ++m) {
        for (int32_t d = 0; d < D; ++d) {
            double t = 0.0, wv = 0.0;
            for (int64_t i = 0; i < K; ++i) {
                t += U[m * K + i] * sdiag[i] * A[i * D + d];
                wv += U[m * K + i] * dinv[i] * A[i * D + d];
            }
            T[m * D + d] = X[m * D + d] + t;
            if (W) W[m * D + d] = wv;
        }
    }
    free(dinv);
    free(sdiag);
}

/*
 * Eq. 18, read over the row-normalised posterior P^ (rows sum to 1 after
 * Eq. 5, so the total mass is M, matching the 1/(DM) factor):
 *   sigma2 = [ sum_m S_m / P1_m - 2 sum_m Ytil_m . T_m + sum_m |T_m|^2 ] / (D M)
 * where sum_m S_m / P1_m = tr(Y^T d(P^T 1) Y) over P^, and T is the NEW
 * transformed point set from the M-step.
 */
double fcpd_oracle_sigma2(const double *S, const double *P1, const double *Ytil,
                          const double *T, int64_t M, int32_t D)
{
    double t1 = 0.0, t2 = 0.0, t3 = 0.0;
    for (int64_t m = 0; m < M; ++m) {
        t1 += S[m] / P1[m];
        for (int32_t d = 0; d < D; ++d) {
            t2 += Ytil[m * D + d] * T[m * D + d];
            t3 += T[m * D + d] * T[m * D + d];
        }
    }
    return (t1 - 2.0 * t2 + t3) / ((double)D * (double)M);
}

/*
 * The EM loop: fixed iteration count (the paper runs 50 or 100 iterations).
 * Per iteration: E-step with the current (T, sigma2); M-step with the same
 * sigma2; then sigma2 from Eq. 18 with the new T.
 * Scratch: den[N], P1[M], PY[M*D], S[M], Ytil[M*D], A[K*D] supplied by the caller.
 * sigma2_hist (n_iter, optional) receives sigma2 after each iteration;
 * loglik_hist (n_iter, optional) receives Eq. 3 at each E-step.
 * T (M x D) is the output; on entry it must hold the starting points (X for W_0 = 0).
 * Returns ORACLE_ENUMERIC (and stops) on a row that cannot be normalised or a
 * variance that is not positive and finite.
 */
int fcpd_oracle_register(const double *X, int64_t M, const double *Y, int64_t N, int32_t D,
                         const double *U, const double *lam, int64_t K,
                         double w, double lambda, double sigma2_0, int32_t n_iter,
                         double *T, double *W, double *sigma2_out, int32_t *iters_done,
                         double *sigma2_hist, double *loglik_hist,
                         double *den, double *P1, double *PY, double *S, double *Ytil, double *A)
{
    double sigma2 = sigma2_0;
    *iters_done = 0;
    for (int32_t it = 0; it < n_iter; ++it) {
        double ll = 0.0;
        int st = fcpd_oracle_estep(T, M, Y, N, D, sigma2, w, den, P1, PY, S, Ytil, &ll);
        if (st != ORACLE_OK) { *sigma2_out = sigma2; return st; }
        if (loglik_hist) loglik_hist[it] = ll;
        fcpd_oracle_mstep(U, lam, M, K, X, Ytil, D, lambda, sigma2, T, W, A);
        sigma2 = fcpd_oracle_sigma2(S, P1, Ytil, T, M, D);
        if (sigma2_hist) sigma2_hist[it] = sigma2;
        *iters_done = it + 1;
        if (!(sigma2 > 0.0) || !isfinite(sigma2)) { *sigma2_out = sigma2; return ORACLE_ENUMERIC; }
    }
    *sigma2_out = sigma2;
    return ORACLE_OK;
}

/* Eq. 22: RMSE of the transformed model points against ground truth. */
double fcpd_oracle_rmse(const double *T, const double *Yhat, int64_t M, int32_t D)
{
    double s = 0.0;
    for (int64_t m = 0; m < M; ++m)
        for (int32_t d = 0; d < D; ++d) {
            double diff = T[m * D + d] - Yhat[m * D + d];
            s += diff * diff;
        }
    return sqrt(s / (double)M);
}
