/*
 * tdeig_oracle.c -- plain FP64 CPU oracle for the divide-and-conquer
 * tridiagonal eigensolver (Li, Liao, Liu, Jiang, "New fast divide-and-conquer
 * algorithms for the symmetric tridiagonal eigenvalue problem").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Every routine works in IEEE double precision, loops in the order the
 * mathematics is written, and does no blocking or fusion.  The outer loops
 * over independent roots / rows carry an OpenMP pragma, mirroring the paper's
 * parallelisation of the secular equations over roots (Sec. 4.3); without
 * OpenMP they run sequentially and give identical results.
 *
 * Readings of passages the paper leaves silent are stated at each routine.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EPS 1.1102230246251565e-16 /* unit roundoff 2^-53 */

/* ------------------------------------------------------------------------ */
/* Leaf solver: symmetric tridiagonal QR with Wilkinson shift.              */
/* Sec. 2.3, Algorithm 1 ("use QR algorithm" below the leaf size).          */
/* Implicit single-shift QR step by bulge chasing (Golub & Van Loan,        */
/* Matrix Computations, Sec. 8.3).  a[n] diagonal, b[n-1] off-diagonal      */
/* (destroyed).  On return lam[n] ascending and Q (n x n, column-major,     */
/* leading dimension n) holds the eigenvectors.  Returns 0, or -1 if the    */
/* iteration cap (30 n sweeps) is hit.                                      */
/* ------------------------------------------------------------------------ */
int orc_leaf_qr(int n, const double* a_in, const double* b_in, double* lam, double* Q)
{
    double a[64], b[64];
    if (n <= 0) return 0;
    if (n > 64) return -2;
    for (int i = 0; i < n; i++) a[i] = a_in[i];
    for (int i = 0; i < n - 1; i++) b[i] = b_in[i];
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) Q[i + (size_t)j * n] = (i == j) ? 1.0 : 0.0;

    int sweeps = 0;
    int h = n - 1;
    while (h > 0) {
        /* negligible off-diagonals are set to zero */
        for (int i = 0; i < h; i++)
            if (fabs(b[i]) <= ORC_EPS * (fabs(a[i]) + fabs(a[i + 1]))) b[i] = 0.0;
        while (h > 0 && b[h - 1] == 0.0) h--;
        if (h == 0) break;
        int l = h - 1;
        while (l > 0 && b[l - 1] != 0.0) l--;
        if (++sweeps > 30 * n) return -1;

        /* Wilkinson shift from the trailing 2x2 of the active block [l, h] */
        double dd = 0.5 * (a[h - 1] - a[h]);
        double bh = b[h - 1];
        double sg = (dd >= 0.0) ? 1.0 : -1.0;
        double mu = a[h] - bh * bh / (dd + sg * hypot(dd, bh));

        double x = a[l] - mu, z = b[l];
        for (int k = l; k < h; k++) {
            /* rotation G on (k, k+1) with G^T [x; z] = [r; 0] */
            double r = hypot(x, z);
            double c = 1.0, s = 0.0;
            if (r != 0.0) { c = x / r; s = -z / r; }
            if (k > l) b[k - 1] = r;
            double p = a[k], q = b[k], w = a[k + 1];
            a[k]     = c * c * p - 2.0 * c * s * q + s * s * w;
            a[k + 1] = s * s * p + 2.0 * c * s * q + c * c * w;
            b[k]     = c * s * (p - w) + (c * c - s * s) * q;
            if (k + 1 < h) {
                double e = b[k + 1];
                z = -s * e;
                b[k + 1] = c * e;
                x = b[k];
            }
            /* accumulate Q <- Q G */
            for (int i = 0; i < n; i++) {
                double qk = Q[i + (size_t)k * n], qk1 = Q[i + (size_t)(k + 1) * n];
                Q[i + (size_t)k * n]       = c * qk - s * qk1;
                Q[i + (size_t)(k + 1) * n] = s * qk + c * qk1;
            }
        }
    }
    /* selection sort of the eigenpairs, ascending */
    for (int i = 0; i < n; i++) lam[i] = a[i];
    for (int i = 0; i < n - 1; i++) {
        int m = i;
        for (int j = i + 1; j < n; j++) if (lam[j] < lam[m]) m = j;
        if (m != i) {
            double t = lam[i]; lam[i] = lam[m]; lam[m] = t;
            for (int r = 0; r < n; r++) {
                double u = Q[r + (size_t)i * n];
                Q[r + (size_t)i * n] = Q[r + (size_t)m * n];
                Q[r + (size_t)m * n] = u;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Deflation (Sec. 4.3 names the LAPACK deflation step; the paper gives no  */
/* criteria).  Reading, after Gu & Eisenstat (SIMAX 1995):                   */
/*   d[n] ascending, z[n] of unit norm, rho > 0 (M = diag(d) + rho z z^T).  */
/*   tau = 8 eps max(max|d|, rho max|z|).                                    */
/*   Sweep i ascending; j = the last survivor so far.                        */
/*   (a) rho |z_i| <= tau: i deflates with eigenvalue d_i.                   */
/*   (b) otherwise, with t = d_i - d_j, r = sqrt(z_i^2 + z_j^2), c = z_i/r,  */
/*       s = z_j / r: if |t c s| <= tau the rotation [q_j q_i] G,            */
/*       G = [[c, s], [-s, c]], zeroes z_j; then z_i = r, d_j and d_i take    */
/*       the diagonal of G^T diag(d_j, d_i) G, and j deflates.              */
/* Every operation is rounded once, as written (the file is compiled        */
/* without floating-point contraction): for nearly equal poles t is a few   */
/* ulp, so the decisions depend on the exact rounding of the rotated poles. */
/* W (n x n, column-major, leading dim ldw) holds the columns that go with  */
/* d; rotated columns are updated in place.  keep[i] = 1 for survivors.     */
/* rot (optional, NULL to skip): the rotations in sweep order, rot_j[t],    */
/* rot_i[t], rot_c[t], rot_s[t] (up to n of them), *nrot their count.       */
/* Returns the number of survivors K.                                       */
/* ------------------------------------------------------------------------ */
int orc_deflate(int n, double* d, double* z, double rho, double* W, int nrow, int ldw, int* keep,
                int* rot_j, int* rot_i, double* rot_c, double* rot_s, int* nrot)
{
    double dmax = 0.0, zmax = 0.0;
    for (int i = 0; i < n; i++) {
        if (fabs(d[i]) > dmax) dmax = fabs(d[i]);
        if (fabs(z[i]) > zmax) zmax = fabs(z[i]);
    }
    double tau = 8.0 * ORC_EPS * fmax(dmax, rho * zmax);
    int j = -1, K = 0, nr = 0;
    for (int i = 0; i < n; i++) {
        keep[i] = 0;
        if (rho * fabs(z[i]) <= tau) { z[i] = 0.0; continue; }
        if (j < 0) { keep[i] = 1; j = i; continue; }
        double t = d[i] - d[j];
        /* both weights belong to survivors, rho |z| > tau >= 8 eps rho max|z|:
           their squares neither underflow nor overflow */
        double r = sqrt(z[i] * z[i] + z[j] * z[j]);
        double c = z[i] / r, s = z[j] / r;
        if (fabs(t * c * s) <= tau) {
            double dj = d[j], di = d[i];
            d[j] = c * c * dj + s * s * di;
            d[i] = s * s * dj + c * c * di;
            z[i] = r;
            z[j] = 0.0;
            for (int row = 0; row < nrow; row++) {
                double qj = W[row + (size_t)j * ldw], qi = W[row + (size_t)i * ldw];
                W[row + (size_t)j * ldw] = c * qj - s * qi;
                W[row + (size_t)i * ldw] = s * qj + c * qi;
            }
            keep[j] = 0;
            if (rot_j) {
                rot_j[nr] = j;
                rot_i[nr] = i;
                rot_c[nr] = c;
                rot_s[nr] = s;
            }
            nr++;
        }
        keep[i] = 1;
        j = i;
    }
    for (int i = 0; i < n; i++) K += keep[i];
    if (nrot) *nrot = nr;
    return K;
}

/* ------------------------------------------------------------------------ */
/* Secular equation (Theorem 1; Remark 1 for gamma/mu).                     */
/* f(lam) = 1 + rho sum_j z_j^2 / (d_j - lam), d strictly ascending, K >= 2. */
/* Root i lies in (d_i, d_{i+1}) for i < K-1 and in (d_{K-1},               */
/* d_{K-1} + rho |z|^2] for the last one.                                    */
/* Reading (the paper defers to LAPACK's dlaed4): the origin is the nearer   */
/* pole, chosen by the sign of f at the interval midpoint; the unknown is    */
/* tau = lam - d_origin; each step fits psi (poles j <= i) by A + B/(d_i-x) */
/* and phi (poles j > i) by C + D/(d_{i+1}-x), matching value and slope at   */
/* the current point (Bunch, Nielsen & Sorensen 1978), and takes the root of */
/* the model inside the bracket; a step leaving the bracket is replaced by   */
/* bisection.  Stop when |f| <= 8 eps (1 + |psi| + |phi| + |tau| f') or the  */
/* bracket is exhausted.  Returns iterations used, -1 on the 200-step cap.   */
/* Outputs lam = d_origin + tau, gamma = lam - d_i, mu = d_{i+1} - lam.      */
/* ------------------------------------------------------------------------ */
static void orc_secular_terms(int K, const double* delta, const double* w, int i, double tau,
                              double* psi, double* dpsi, double* phi, double* dphi)
{
    double s1 = 0, s2 = 0, s3 = 0, s4 = 0;
    for (int j = 0; j <= i; j++) {
        double q = 1.0 / (delta[j] - tau);
        s1 += w[j] * q; s2 += w[j] * q * q;
    }
    for (int j = i + 1; j < K; j++) {
        double q = 1.0 / (delta[j] - tau);
        s3 += w[j] * q; s4 += w[j] * q * q;
    }
    *psi = s1; *dpsi = s2; *phi = s3; *dphi = s4;
}

int orc_secular_root(int K, const double* d, const double* z, double rho, int i,
                     double* lam, double* gamma, double* mu, double* work)
{
    /* work: 2K doubles (delta, w) */
    double* delta = work;
    double* w = work + K;
    for (int j = 0; j < K; j++) w[j] = rho * z[j] * z[j];
    if (K == 1) {
        *lam = d[0] + w[0]; *gamma = w[0]; *mu = 0.0;
        return 0;
    }
    int last = (i == K - 1);
    int org;
    double lo, hi;
    if (!last) {
        double gap = d[i + 1] - d[i];
        double half = 0.5 * gap;
        /* f at the midpoint, relative to d_i */
        double f = 1.0;
        for (int j = 0; j < K; j++) f += w[j] / ((d[j] - d[i]) - half);
        if (f >= 0.0) { org = i; lo = 0.0; hi = half; }
        else          { org = i + 1; lo = -half; hi = 0.0; }
    } else {
        double zz = 0.0;
        for (int j = 0; j < K; j++) zz += w[j];
        org = i; lo = 0.0; hi = zz;
    }
    for (int j = 0; j < K; j++) delta[j] = d[j] - d[org];

    double tau = 0.5 * (lo + hi);
    int it;
    for (it = 1; it <= 200; it++) {
        double psi, dpsi, phi, dphi;
        orc_secular_terms(K, delta, w, i, tau, &psi, &dpsi, &phi, &dphi);
        double f = 1.0 + psi + phi;
        double err = 8.0 * ORC_EPS * (1.0 + fabs(psi) + fabs(phi) + fabs(tau) * (dpsi + dphi));
        if (fabs(f) <= err) break;
        if (f > 0.0) hi = tau; else lo = tau;
        if (hi - lo <= 4.0 * ORC_EPS * fmax(fabs(lo), fabs(hi))) break;

        double a1 = delta[i] - tau;             /* < 0 */
        double step;
        int ok = 1;
        if (!last) {
            double a2 = delta[i + 1] - tau;     /* > 0 */
            double E = f - dpsi * a1 - dphi * a2;
            double beta = E * (a1 + a2) + dpsi * a1 * a1 + dphi * a2 * a2;
            double c0 = a1 * a2 * f;
            double disc = beta * beta - 4.0 * E * c0;
            if (disc < 0.0) disc = 0.0;
            double den = beta + (beta >= 0.0 ? sqrt(disc) : -sqrt(disc));
            if (den == 0.0) ok = 0; else step = 2.0 * c0 / den;
        } else {
            double E = f - dpsi * a1;
            if (E == 0.0) ok = 0; else step = a1 * f / E;
        }
        double nt = ok ? tau + step : 0.5 * (lo + hi);
        if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
        if (nt == tau) break;
        tau = nt;
    }
    *lam = d[org] + tau;
    if (last) {
        *gamma = tau; *mu = 0.0;
    } else if (org == i) {
        *gamma = tau; *mu = (d[i + 1] - d[i]) - tau;
    } else {
        *mu = -tau; *gamma = (d[i + 1] - d[i]) + tau;
    }
    return it > 200 ? -1 : it;
}

/* All K roots; work must hold 2K doubles per thread (nthreads rows). */
int orc_secular_all(int K, const double* d, const double* z, double rho,
                    double* lam, double* gamma, double* mu, int* iters, double* work, int nthreads)
{
    int bad = 0;
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 16) reduction(+:bad)
    for (int i = 0; i < K; i++) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int r = orc_secular_root(K, d, z, rho, i, &lam[i], &gamma[i], &mu[i], work + (size_t)tid * 2 * K);
        iters[i] = r;
        if (r < 0) bad++;
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* d_k - lam_j by Remark 1 (eq. d-lambda):                                   */
/*   (d_k - d_j) - gamma_j   if k <= j                                       */
/*   (d_k - d_{j+1}) + mu_j  if k >  j                                       */
/* ------------------------------------------------------------------------ */
static double orc_dminus(const double* d, const double* gamma, const double* mu, int k, int j)
{
    if (k <= j) return (d[k] - d[j]) - gamma[j];
    return (d[k] - d[j + 1]) + mu[j];
}

/* ------------------------------------------------------------------------ */
/* Loewner recomputation of the rank-one vector (eq. ev_z).  Reading: the   */
/* paper's formula is for rho = 1; for M = D + rho u u^T the squared entry   */
/* is divided by rho:                                                        */
/*   uhat_i^2 = (lam_i - d_i)/rho * prod_{j<i} (lam_j - d_i)/(d_j - d_i)     */
/*                                * prod_{j>i} (lam_j - d_i)/(d_j - d_i)     */
/* every lam_j - d_i formed by Remark 1; factors taken j < i first, then     */
/* j > i, as printed.  sign(uhat_i) = sign(z_i).                             */
/* ------------------------------------------------------------------------ */
void orc_lowner(int K, const double* d, const double* gamma, const double* mu, double rho,
                const double* z, double* uhat)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < K; i++) {
        double p = gamma[i] / rho;
        for (int j = 0; j < i; j++)
            p *= (-orc_dminus(d, gamma, mu, i, j)) / (d[j] - d[i]);
        for (int j = i + 1; j < K; j++)
            p *= (-orc_dminus(d, gamma, mu, i, j)) / (d[j] - d[i]);
        uhat[i] = copysign(sqrt(p), z[i]);
    }
}

/* ------------------------------------------------------------------------ */
/* Cauchy-like eigenvector matrix (Theorem 1, eq. Ev-Q):                     */
/*   v_j = 1 / sqrt(sum_k uhat_k^2 / (d_k - lam_j)^2)                        */
/*   Qhat[k, j] = uhat_k v_j / (d_k - lam_j)                                 */
/* Qhat is K x K column-major with leading dimension K.  v may be NULL.      */
/* ------------------------------------------------------------------------ */
void orc_cauchy(int K, const double* d, const double* gamma, const double* mu,
                const double* uhat, double* v, double* Qhat)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < K; j++) {
        double s = 0.0;
        for (int k = 0; k < K; k++) {
            double t = uhat[k] / orc_dminus(d, gamma, mu, k, j);
            s += t * t;
        }
        double vj = 1.0 / sqrt(s);
        if (v) v[j] = vj;
        for (int k = 0; k < K; k++)
            Qhat[k + (size_t)j * K] = uhat[k] * vj / orc_dminus(d, gamma, mu, k, j);
    }
}

/* Entries of the Cauchy-like matrix at given global rows / columns:         */
/*   out[a + b*nr] = uhat[rows[a]] v[cols[b]] / (d_rows[a] - lam_cols[b]).   */
/* Used to fill HSS generators D_i and B_i from the four vectors (Sec. 4.1). */
void orc_cauchy_entries(int nr, const int* rows, int nc, const int* cols, const double* d,
                        const double* gamma, const double* mu, const double* uhat,
                        const double* v, double* out)
{
    for (int b = 0; b < nc; b++)
        for (int a = 0; a < nr; a++) {
            int k = rows[a], j = cols[b];
            out[a + (size_t)b * nr] = uhat[k] * v[j] / orc_dminus(d, gamma, mu, k, j);
        }
}

/* The differences d_rows[a] - lam_cols[b] themselves (Remark 1), used as the */
/* denominators of the generator form in the Schur-complement compression.   */
void orc_dminus_entries(int nr, const int* rows, int nc, const int* cols, const double* d,
                        const double* gamma, const double* mu, double* out)
{
    for (int b = 0; b < nc; b++)
        for (int a = 0; a < nr; a++)
            out[a + (size_t)b * nr] = orc_dminus(d, gamma, mu, rows[a], cols[b]);
}
