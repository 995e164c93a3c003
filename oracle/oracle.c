/*
 * FP64 CPU oracle kernels for the contour-integral eigensolver (test infrastructure only).
 *
 * Only the test suite, the smoke check and the bench's CPU-baseline leg load this library.
 * The GPU path never links, calls or includes it, and it includes nothing from the GPU path.
 *
 * Three textbook building blocks, written plainly (no blocking, no reordering):
 *   1. complex banded Gaussian elimination with partial pivoting, for the shifted systems
 *      (z_j B - A) X_j = B V at a quadrature node (Eq. quadrature_appendix, Algorithm 1);
 *   2. real banded LDL^T without pivoting of (A - sigma B), counting negative pivots
 *      (Sylvester's law of inertia: the count equals the number of eigenvalues below sigma,
 *      the eigenvalue-counting technique of the paper's Section 3.3);
 *   3. cyclic Jacobi for a dense real symmetric matrix, used for the small projected problems
 *      (Algorithm 1, "solve the reduced GEP") and for the Gram matrix of the basis.
 *
 * Storage conventions
 *   Band (complex, general): row-major, row i holds columns i-kl .. i+ku+kl, so
 *     a(i,j) = ab[i*W + (j - i + kl)],  W = 2*kl + ku + 1.
 *   The extra kl super-diagonals hold the fill created by row interchanges.
 *   Band (real, symmetric lower): row i holds columns i-bw .. i, a(i,j) = ab[i*(bw+1) + (j-i+bw)].
 *   Dense: row-major p x p.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (strict IEEE double, round to nearest).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef double _Complex zdouble;

/* Factor the n x n band matrix in place: P A = L U.  ipiv[k] = row swapped with row k at step k.
 * Returns 0, or k+1 if the pivot of column k is exactly zero (matrix singular). */
int oracle_zband_lu_factor(int64_t n, int64_t kl, int64_t ku, zdouble *ab, int64_t *ipiv)
{
    const int64_t W = 2 * kl + ku + 1;
#define A(i, j) ab[(i) * W + ((j) - (i) + kl)]
    for (int64_t k = 0; k < n; ++k) {
        int64_t last = k + kl < n - 1 ? k + kl : n - 1;
        /* pivot: largest |a(i,k)| over i = k..last */
        int64_t p = k;
        double best = cabs(A(k, k));
        for (int64_t i = k + 1; i <= last; ++i) {
            double v = cabs(A(i, k));
            if (v > best) { best = v; p = i; }
        }
        ipiv[k] = p;
        if (best == 0.0) return (int)(k + 1);
        int64_t jend = k + ku + kl < n - 1 ? k + ku + kl : n - 1;
        if (p != k) {
            for (int64_t j = k; j <= jend; ++j) {
                zdouble t = A(k, j); A(k, j) = A(p, j); A(p, j) = t;
            }
        }
        zdouble piv = A(k, k);
        for (int64_t i = k + 1; i <= last; ++i) {
            zdouble l = A(i, k) / piv;
            A(i, k) = l;
            if (l == 0.0) continue;
            for (int64_t j = k + 1; j <= jend; ++j)
                A(i, j) -= l * A(k, j);
        }
    }
#undef A
    return 0;
}

/* Solve A X = B with the factors from oracle_zband_lu_factor.  B is n x nrhs row-major and is
 * overwritten by X. */
void oracle_zband_lu_solve(int64_t n, int64_t kl, int64_t ku, const zdouble *ab, const int64_t *ipiv,
                           int64_t nrhs, zdouble *B)
{
    const int64_t W = 2 * kl + ku + 1;
#define A(i, j) ab[(i) * W + ((j) - (i) + kl)]
    /* forward: apply the interchanges and the unit-lower multipliers in elimination order */
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = ipiv[k];
        if (p != k) {
            for (int64_t r = 0; r < nrhs; ++r) {
                zdouble t = B[k * nrhs + r]; B[k * nrhs + r] = B[p * nrhs + r]; B[p * nrhs + r] = t;
            }
        }
        int64_t last = k + kl < n - 1 ? k + kl : n - 1;
        for (int64_t i = k + 1; i <= last; ++i) {
            zdouble l = A(i, k);
            if (l == 0.0) continue;
            for (int64_t r = 0; r < nrhs; ++r) B[i * nrhs + r] -= l * B[k * nrhs + r];
        }
    }
    /* backward: upper triangle has bandwidth ku + kl */
    for (int64_t k = n - 1; k >= 0; --k) {
        int64_t jend = k + ku + kl < n - 1 ? k + ku + kl : n - 1;
        for (int64_t j = k + 1; j <= jend; ++j) {
            zdouble u = A(k, j);
            if (u == 0.0) continue;
            for (int64_t r = 0; r < nrhs; ++r) B[k * nrhs + r] -= u * B[j * nrhs + r];
        }
        zdouble d = A(k, k);
        for (int64_t r = 0; r < nrhs; ++r) B[k * nrhs + r] /= d;
    }
#undef A
}

/* LDL^T of a real symmetric band matrix (lower band, bandwidth bw) without pivoting, in place.
 * Returns the number of negative pivots d_k.  An exactly zero pivot is replaced by
 * tiny * max|a(k,:)| (recorded in *nzero) so the count is that of a nearby shift. */
int64_t oracle_dband_ldlt_negcount(int64_t n, int64_t bw, double *ab, int64_t *nzero)
{
    const int64_t W = bw + 1;
#define S(i, j) ab[(i) * W + ((j) - (i) + bw)]
    int64_t neg = 0;
    if (nzero) *nzero = 0;
    for (int64_t k = 0; k < n; ++k) {
        double d = S(k, k);
        if (d == 0.0) {
            d = 1e-300;
            if (nzero) ++*nzero;
        }
        if (d < 0.0) ++neg;
        int64_t last = k + bw < n - 1 ? k + bw : n - 1;
        /* rows i > k: a(i,j) -= a(i,k) a(j,k) / d for k < j <= i; then l(i,k) = a(i,k)/d */
        for (int64_t i = k + 1; i <= last; ++i) {
            double aik = S(i, k);
            if (aik == 0.0) continue;
            double f = aik / d;
            for (int64_t j = k + 1; j <= i; ++j) S(i, j) -= f * S(j, k);
        }
        for (int64_t i = k + 1; i <= last; ++i) S(i, k) /= d;
        S(k, k) = d;
    }
#undef S
    return neg;
}

/* Cyclic Jacobi (row-by-row sweeps) for a dense symmetric p x p matrix a (row-major, destroyed).
 * On return w[i] = eigenvalue i (unsorted) and column i of v (row-major p x p) its unit
 * eigenvector.  Stops when the off-diagonal Frobenius norm is <= tol * ||a||_F or after
 * maxsweep sweeps; returns the number of sweeps used (maxsweep+1 if not converged). */
int oracle_jacobi_eig(int64_t p, double *a, double *w, double *v, double tol, int maxsweep)
{
#define M_(i, j) a[(i) * p + (j)]
#define V_(i, j) v[(i) * p + (j)]
    double fro = 0.0;
    for (int64_t i = 0; i < p * p; ++i) fro += a[i] * a[i];
    fro = sqrt(fro);
    for (int64_t i = 0; i < p; ++i)
        for (int64_t j = 0; j < p; ++j) V_(i, j) = (i == j) ? 1.0 : 0.0;
    int sweep;
    for (sweep = 1; sweep <= maxsweep + 1; ++sweep) {
        double off = 0.0;
        for (int64_t i = 0; i < p; ++i)
            for (int64_t j = 0; j < p; ++j)
                if (i != j) off += M_(i, j) * M_(i, j);
        if (sqrt(off) <= tol * fro || fro == 0.0) break;
        if (sweep == maxsweep + 1) break;
        for (int64_t q = 0; q < p - 1; ++q) {
            for (int64_t r = q + 1; r < p; ++r) {
                double apq = M_(q, r);
                if (apq == 0.0) continue;
                /* rotation angle that zeroes a(q,r) (Golub & Van Loan, symmetric Schur 2x2) */
                double tau = (M_(r, r) - M_(q, q)) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                /* A <- J^T A J with J = rotation in the (q, r) plane */
                for (int64_t k = 0; k < p; ++k) {
                    double akq = M_(k, q), akr = M_(k, r);
                    M_(k, q) = c * akq - s * akr;
                    M_(k, r) = s * akq + c * akr;
                }
                for (int64_t k = 0; k < p; ++k) {
                    double aqk = M_(q, k), ark = M_(r, k);
                    M_(q, k) = c * aqk - s * ark;
                    M_(r, k) = s * aqk + c * ark;
                }
                for (int64_t k = 0; k < p; ++k) {
                    double vkq = V_(k, q), vkr = V_(k, r);
                    V_(k, q) = c * vkq - s * vkr;
                    V_(k, r) = s * vkq + c * vkr;
                }
            }
        }
    }
    for (int64_t i = 0; i < p; ++i) w[i] = M_(i, i);
#undef M_
#undef V_
    return sweep;
}
