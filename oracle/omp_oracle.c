/*
 * FP64 CPU oracle for batched Orthogonal Matching Pursuit.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this
 * file; it exists so that tests, the smoke check and the CPU baseline of the
 * benchmark have an independent, obviously correct statement of what the
 * GPU path computes.  It shares no code, header or constant with the CUDA
 * library.
 *
 * What it computes (paper: Sec. II-B, Algorithm 1 "Orthogonal matching
 * pursuit"; the restricted fine step of Algorithm 2 "Zero tree OMP" is the
 * same loop over a gathered sub-dictionary):
 *
 *   r <- y, Omega <- {}
 *   for n = 1..K:
 *     stop if ||r||^2 <= eps_r * ||y||^2
 *     proxy:       score_i = |<a_i, r>| / ||a_i||  for every column i
 *                  (angle reading of the proxy; ||a_i|| dropped when
 *                  normalize == 0); columns already in Omega and columns with
 *                  ||a_i|| <= 1e-12 * max_j ||a_j|| are not eligible
 *     k = argmax over eligible i, ties to the lowest i
 *     support merge: Omega <- Omega u {k}
 *     projection:  alpha = argmin_b ||y - A_Omega b||_2, solved FROM SCRATCH
 *                  by Householder QR of A_Omega (no incremental update)
 *                  if |R_kk| <= eps_d * ||a_k||, a_k depends on the atoms
 *                  already chosen: drop k and stop
 *     residue:     r = y - A_Omega alpha
 *
 * Columns of A are stored atom-major: column i is A[i*M .. i*M+M-1].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Householder QR of the M x k matrix whose columns are cols[0..k-1], then
 * least squares: alpha = R^{-1} (Q^T y)[0..k-1].  Returns |R[k-1][k-1]|.
 * work needs M*k + M + k doubles. */
static double ls_householder(int M, int k, const double *const *cols, const double *y,
                             double *alpha, double *work)
{
    double *Qr = work;            /* M x k, column-major, overwritten by reflectors */
    double *qty = work + (size_t)M * k;
    double *diag = qty + M;       /* R[j][j] */
    for (int j = 0; j < k; ++j)
        memcpy(Qr + (size_t)j * M, cols[j], sizeof(double) * (size_t)M);
    memcpy(qty, y, sizeof(double) * (size_t)M);

    for (int j = 0; j < k; ++j) {
        double *x = Qr + (size_t)j * M;
        double nrm = 0.0;
        for (int i = j; i < M; ++i) nrm += x[i] * x[i];
        nrm = sqrt(nrm);
        if (nrm == 0.0) { diag[j] = 0.0; continue; }
        double s = (x[j] >= 0.0) ? 1.0 : -1.0;
        diag[j] = -s * nrm;
        /* v = x[j:] + s*nrm*e1, stored in place; H = I - 2 v v^T / (v^T v) */
        x[j] += s * nrm;
        double vtv = 0.0;
        for (int i = j; i < M; ++i) vtv += x[i] * x[i];
        /* apply H to remaining columns */
        for (int c = j + 1; c < k; ++c) {
            double *z = Qr + (size_t)c * M;
            double d = 0.0;
            for (int i = j; i < M; ++i) d += x[i] * z[i];
            double f = 2.0 * d / vtv;
            for (int i = j; i < M; ++i) z[i] -= f * x[i];
        }
        /* apply H to y */
        double d = 0.0;
        for (int i = j; i < M; ++i) d += x[i] * qty[i];
        double f = 2.0 * d / vtv;
        for (int i = j; i < M; ++i) qty[i] -= f * x[i];
    }
    /* back substitution R alpha = qty[0..k-1]; R's strict upper part sits in
     * Qr above the diagonal (rows < column index), untouched by reflectors
     * of later columns. */
    for (int j = k - 1; j >= 0; --j) {
        double acc = qty[j];
        for (int c = j + 1; c < k; ++c) acc -= Qr[(size_t)c * M + j] * alpha[c];
        alpha[j] = (diag[j] != 0.0) ? acc / diag[j] : 0.0;
    }
    return fabs(diag[k - 1]);
}

/* One OMP problem.  Returns k_eff.  omega/alpha hold k_eff entries in
 * selection order.  *rsq gets ||r||^2 at exit; *flops gets the proxy
 * multiply-adds times two (2*M per column per iteration). */
int oracle_omp_one(int M, int T, const double *A, const double *y, int K,
                   double eps_r, double eps_d, int normalize,
                   int *omega, double *alpha, double *rsq, long long *flops)
{
    double *norms = (double *)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)M);
    double *work = (double *)malloc(sizeof(double) * ((size_t)M * (K + 1) + M + K + 1));
    double *a_tmp = (double *)malloc(sizeof(double) * (size_t)(K + 1));
    const double **cols = (const double **)malloc(sizeof(double *) * (size_t)(K + 1));
    char *chosen = (char *)calloc((size_t)(T > 0 ? T : 1), 1);
    long long fl = 0;

    double maxn = 0.0;
    for (int i = 0; i < T; ++i) {
        double s = 0.0;
        for (int m = 0; m < M; ++m) s += A[(size_t)i * M + m] * A[(size_t)i * M + m];
        norms[i] = sqrt(s);
        if (norms[i] > maxn) maxn = norms[i];
    }
    double ysq = 0.0;
    for (int m = 0; m < M; ++m) { r[m] = y[m]; ysq += y[m] * y[m]; }
    double cur_rsq = ysq;

    int k = 0;
    for (int n = 0; n < K; ++n) {
        if (cur_rsq <= eps_r * ysq) break;
        /* proxy */
        int best = -1;
        double best_s = -1.0;
        for (int i = 0; i < T; ++i) {
            const double *a = A + (size_t)i * M;
            double c = 0.0;
            for (int m = 0; m < M; ++m) c += a[m] * r[m];
            fl += 2LL * M;
            if (chosen[i] || norms[i] <= 1e-12 * maxn) continue;
            double s = normalize ? fabs(c) / norms[i] : fabs(c);
            if (s > best_s) { best_s = s; best = i; }   /* strict: lowest index wins ties */
        }
        if (best < 0) break;
        /* support merge + projection from scratch */
        omega[k] = best;
        cols[k] = A + (size_t)best * M;
        double rkk = ls_householder(M, k + 1, cols, y, a_tmp, work);
        if (rkk <= eps_d * norms[best]) {               /* dependent atom: drop it, stop */
            omega[k] = -1;
            break;
        }
        chosen[best] = 1;
        ++k;
        for (int j = 0; j < k; ++j) alpha[j] = a_tmp[j];
        /* residue */
        cur_rsq = 0.0;
        for (int m = 0; m < M; ++m) {
            double v = y[m];
            for (int j = 0; j < k; ++j) v -= cols[j][m] * alpha[j];
            r[m] = v;
            cur_rsq += v * v;
        }
    }
    *rsq = cur_rsq;
    if (flops) *flops = fl;
    free(norms); free(r); free(work); free(a_tmp); free(cols); free(chosen);
    return k;
}

/* Batch over independent problems.  Problem b uses the M x T_cols[b] matrix at
 * A_ptrs[b] (atom-major), measurement Y[b*M ..], budget K[b] <= Kmax.  Outputs
 * are B x Kmax (unused tail: omega = -1, alpha = 0).  Returns 0. */
int oracle_omp_batch(int B, int M, const double *const *A_ptrs, const int *T_cols,
                     const double *Y, const int *K, int Kmax, double eps_r, double eps_d,
                     int normalize, int nthreads, int *omega, double *alpha, int *k_eff,
                     double *rsq, long long *flops)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int b = 0; b < B; ++b) {
        int *om = omega + (size_t)b * Kmax;
        double *al = alpha + (size_t)b * Kmax;
        for (int j = 0; j < Kmax; ++j) { om[j] = -1; al[j] = 0.0; }
        int Kb = K[b] < Kmax ? K[b] : Kmax;
        long long f = 0;
        double rr = 0.0;
        k_eff[b] = oracle_omp_one(M, T_cols[b], A_ptrs[b], Y + (size_t)b * M, Kb, eps_r, eps_d,
                                  normalize, om, al, &rr, &f);
        if (rsq) rsq[b] = rr;
        if (flops) flops[b] = f;
    }
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
