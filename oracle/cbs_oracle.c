/*
 * cbs_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for cyclic
 * compact banded solves (test infrastructure only).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The GPU library never
 * links, includes or calls anything from here, and nothing here is derived
 * from the GPU code: the oracle computes the plain definition of the result,
 *
 *     x = A^{-1} d,   d = S f,
 *
 * where S is the periodic central-difference right-hand side of the compact
 * scheme (paper Eq. 1) and A the cyclic banded left-hand side.  The paper's
 * method (partitioning, generalized PCR, the reduced interface system) is a
 * direct solver (abstract; Sec. 3), so its exact result is this definition
 * and the oracle uses textbook direct solvers instead of the paper's
 * algorithm:
 *
 *   - cyclic tridiagonal: Thomas elimination on the acyclic part plus the
 *     Sherman-Morrison correction for the two corner entries (the classic
 *     "cyclic" construction with gamma = -b_0);
 *   - any cyclic banded matrix of half-bandwidth r: banded LU without
 *     pivoting of the acyclic part plus a rank-2r Woodbury correction for the
 *     corner blocks, using the capacitance form (I + K P^T B^{-1} P) so the
 *     corner block K never needs to be inverted;
 *   - a dense Gaussian elimination with partial pivoting for tiny systems.
 *
 * Conventions.  A batch of `lines` independent systems of length n is stored
 * line-contiguous: element j of line l is at [l*n + j].  Banded matrices are
 * stored by diagonals: band[k*n + i] = A[i, (i + k - r) mod n] for
 * k = 0..2r (k = r is the main diagonal).  A batch of band sets either has
 * one set shared by all lines (band_line_stride = 0) or one per line
 * (band_line_stride = (2r+1)*n).
 *
 * Parity pins live in the tests (closed-form modified wavenumbers, dense
 * brute force, FFT circulant solves, Taylor-matched scheme coefficients,
 * finite differences); nothing here is checked against the GPU path.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static long wrap(long i, long n) {
    long m = i % n;
    return m < 0 ? m + n : m;
}

/* Threads the batched routines use (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Periodic central-difference right-hand side of the compact first-derivative
 * scheme (paper Eq. 1, Lele's form extended to K terms):
 *
 *     d_i = sum_{k=1..K} coef[k-1] * (f_{i+k} - f_{i-k}) / (2 k h),
 *
 * indices taken modulo n.  With K = 2, coef = (a, b) this is exactly the
 * right-hand side of Eq. 1; (a, b) = (4/3, -1/3) is the 4th-order explicit
 * central difference.
 */
void orc_central_rhs(const double *f, double *d, long lines, long n,
                     const double *coef, int K, double h) {
    long l;
#pragma omp parallel for schedule(static)
    for (l = 0; l < lines; l++) {
        const double *fl = f + l * n;
        double *dl = d + l * n;
        for (long i = 0; i < n; i++) {
            double s = 0.0;
            for (int k = 1; k <= K; k++) {
                s += coef[k - 1] * (fl[wrap(i + k, n)] - fl[wrap(i - k, n)]) / (2.0 * k * h);
            }
            dl[i] = s;
        }
    }
}

/*
 * Transpose of orc_central_rhs, written as the scatter of each row of S into
 * the columns it touches: out = S^T g.  Used for the gradient with respect to
 * the field f (grad_f = S^T lambda).
 */
void orc_central_rhs_transpose(const double *g, double *out, long lines, long n,
                               const double *coef, int K, double h) {
    long l;
#pragma omp parallel for schedule(static)
    for (l = 0; l < lines; l++) {
        const double *gl = g + l * n;
        double *ol = out + l * n;
        for (long j = 0; j < n; j++) ol[j] = 0.0;
        for (long i = 0; i < n; i++) {
            for (int k = 1; k <= K; k++) {
                double w = coef[k - 1] / (2.0 * k * h);
                ol[wrap(i + k, n)] += w * gl[i]; /* S[i, i+k] = +w */
                ol[wrap(i - k, n)] -= w * gl[i]; /* S[i, i-k] = -w */
            }
        }
    }
}

/*
 * Right-hand sides of the staggered schemes (App. A.2): the sixth-order
 * staggered first derivative (kind 0) and the compact midpoint interpolation
 * of Eq. 2 (kind 1), both between a grid and the grid shifted by half a
 * spacing.  Input element j holds the field at x_{j+1/2} when shift = 0
 * (staggered -> nodes) and at x_j when shift = 1 (nodes -> staggered, output
 * element i at x_{i+1/2}).  Term k couples the two input points at distance
 * (k - 1/2) h on either side of the output point, i.e. elements
 * i + k - 1 + shift and i - k + shift:
 *
 *   kind 0:  d_i = sum_k coef[k-1] (f_up - f_dn) / ((2k - 1) h)
 *   kind 1:  d_i = sum_k coef[k-1] (f_up + f_dn) / 2
 */
void orc_staggered_rhs(const double *f, double *d, long lines, long n,
                       const double *coef, int K, double h, int shift, int kind) {
    long l;
#pragma omp parallel for schedule(static)
    for (l = 0; l < lines; l++) {
        const double *fl = f + l * n;
        double *dl = d + l * n;
        for (long i = 0; i < n; i++) {
            double s = 0.0;
            for (int k = 1; k <= K; k++) {
                double up = fl[wrap(i + k - 1 + shift, n)];
                double dn = fl[wrap(i - k + shift, n)];
                if (kind == 0) s += coef[k - 1] * (up - dn) / ((2.0 * k - 1.0) * h);
                else s += coef[k - 1] * (up + dn) / 2.0;
            }
            dl[i] = s;
        }
    }
}

/* Transpose of orc_staggered_rhs as the scatter of each row into its columns. */
void orc_staggered_rhs_transpose(const double *g, double *out, long lines, long n,
                                 const double *coef, int K, double h, int shift, int kind) {
    long l;
#pragma omp parallel for schedule(static)
    for (l = 0; l < lines; l++) {
        const double *gl = g + l * n;
        double *ol = out + l * n;
        for (long j = 0; j < n; j++) ol[j] = 0.0;
        for (long i = 0; i < n; i++) {
            for (int k = 1; k <= K; k++) {
                double w = (kind == 0) ? coef[k - 1] / ((2.0 * k - 1.0) * h) : coef[k - 1] / 2.0;
                ol[wrap(i + k - 1 + shift, n)] += w * gl[i];
                if (kind == 0) ol[wrap(i - k + shift, n)] -= w * gl[i];
                else ol[wrap(i - k + shift, n)] += w * gl[i];
            }
        }
    }
}

/*
 * Acyclic tridiagonal solve by Thomas elimination (no pivoting):
 *   a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i],  a[0] and c[n-1] ignored.
 * Returns 0, or -1 on a zero pivot.  tmp holds n doubles.
 */
static int thomas(const double *a, const double *b, const double *c,
                  const double *d, double *x, long n, double *tmp) {
    double piv = b[0];
    if (piv == 0.0) return -1;
    x[0] = d[0] / piv;
    for (long i = 1; i < n; i++) {
        tmp[i] = c[i - 1] / piv;
        piv = b[i] - a[i] * tmp[i];
        if (piv == 0.0) return -1;
        x[i] = (d[i] - a[i] * x[i - 1]) / piv;
    }
    for (long i = n - 2; i >= 0; i--) x[i] -= tmp[i + 1] * x[i + 1];
    return 0;
}

/*
 * Cyclic tridiagonal solve, one line, bands per row:
 *   lo[i] x[i-1] + di[i] x[i] + up[i] x[i+1] = d[i]   (indices mod n).
 * Thomas plus Sherman-Morrison: with gamma = -di[0], solve
 *   B y = d and B z = u, u = (gamma, 0, ..., 0, up[n-1]),
 * where B is A with its corners removed and with di[0] -> di[0] - gamma,
 * di[n-1] -> di[n-1] - up[n-1] lo[0] / gamma; then
 *   x = y - z (y0 + lo0 y_{n-1}/gamma) / (1 + z0 + lo0 z_{n-1}/gamma).
 * work holds 4n doubles.  n >= 3.  Returns 0 or -1 (zero pivot).
 */
int orc_cyclic_tri_line(const double *lo, const double *di, const double *up,
                        const double *d, double *x, long n, double *work) {
    double *bb = work, *z = work + n, *u = work + 2 * n, *tmp = work + 3 * n;
    double alpha = up[n - 1]; /* A[n-1, 0] */
    double beta = lo[0];      /* A[0, n-1] */
    double gamma = -di[0];
    if (gamma == 0.0) return -1;
    for (long i = 0; i < n; i++) bb[i] = di[i];
    bb[0] = di[0] - gamma;
    bb[n - 1] = di[n - 1] - alpha * beta / gamma;
    if (thomas(lo, bb, up, d, x, n, tmp)) return -1;
    for (long i = 0; i < n; i++) u[i] = 0.0;
    u[0] = gamma;
    u[n - 1] = alpha;
    if (thomas(lo, bb, up, u, z, n, tmp)) return -1;
    double fact = (x[0] + beta * x[n - 1] / gamma) / (1.0 + z[0] + beta * z[n - 1] / gamma);
    for (long i = 0; i < n; i++) x[i] -= fact * z[i];
    return 0;
}

/* Batched cyclic tridiagonal solve; band layout as in the file header (r = 1). */
int orc_cyclic_tri(const double *bands, long band_line_stride, const double *d,
                   double *x, long lines, long n) {
    int bad = 0;
    long l;
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * 4 * n);
#pragma omp for schedule(static)
        for (l = 0; l < lines; l++) {
            const double *bl = bands + l * band_line_stride;
            if (orc_cyclic_tri_line(bl, bl + n, bl + 2 * n, d + l * n, x + l * n, n, work)) {
#pragma omp atomic write
                bad = 1;
            }
        }
        free(work);
    }
    return bad ? -1 : 0;
}

/*
 * Dense Gaussian elimination with partial pivoting, A is m x m row-major,
 * overwritten; b (length m) is overwritten by the solution.  Returns 0 or -1.
 */
int orc_dense_solve(double *A, double *b, long m) {
    for (long k = 0; k < m; k++) {
        long p = k;
        for (long i = k + 1; i < m; i++)
            if (fabs(A[i * m + k]) > fabs(A[p * m + k])) p = i;
        if (A[p * m + k] == 0.0) return -1;
        if (p != k) {
            for (long j = 0; j < m; j++) {
                double t = A[k * m + j]; A[k * m + j] = A[p * m + j]; A[p * m + j] = t;
            }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (long i = k + 1; i < m; i++) {
            double l = A[i * m + k] / A[k * m + k];
            if (l == 0.0) continue;
            for (long j = k; j < m; j++) A[i * m + j] -= l * A[k * m + j];
            b[i] -= l * b[k];
        }
    }
    for (long k = m - 1; k >= 0; k--) {
        double s = b[k];
        for (long j = k + 1; j < m; j++) s -= A[k * m + j] * b[j];
        b[k] = s / A[k * m + k];
    }
    return 0;
}

/*
 * Banded LU of the acyclic part B of a banded matrix (half-bandwidth r),
 * without pivoting, in place on a (2r+1) x n diagonal-major copy:
 *   L[i, i-q] stored at F[(r-q)*n + i]   (q = 1..r, multipliers)
 *   U[i, i+q] stored at F[(r+q)*n + i]   (q = 0..r)
 * Entries that would wrap around (cyclic corners) are excluded from B.
 */
static int band_lu(double *F, long n, int r) {
#define FB(k, i) F[(long)(k) * n + (i)]
    /* Clear the wrapped corner entries: B is the acyclic part of A. */
    for (long i = 0; i < n; i++)
        for (int k = 0; k <= 2 * r; k++) {
            long j = i + k - r;
            if (j < 0 || j >= n) FB(k, i) = 0.0;
        }
    for (long kcol = 0; kcol < n; kcol++) {
        double piv = FB(r, kcol);
        if (piv == 0.0) return -1;
        for (int q = 1; q <= r && kcol + q < n; q++) {
            long i = kcol + q;
            /* A[i, kcol] lives on diagonal index k = kcol - i + r = r - q */
            double l = FB(r - q, i) / piv;
            FB(r - q, i) = l;
            /* row i -= l * row kcol over columns kcol+1 .. kcol+r */
            for (int t = 1; t <= r; t++) {
                long j = kcol + t;
                if (j >= n) break;
                long kk = j - i + r; /* diagonal index of A[i, j] */
                if (kk > 2 * r) break;
                FB(kk, i) -= l * FB(r + t, kcol);
            }
        }
    }
    return 0;
#undef FB
}

/* Solve B y = rhs with the factors of band_lu (forward then backward). */
static void band_lu_solve(const double *F, long n, int r, const double *rhs, double *y) {
#define FB(k, i) F[(long)(k) * n + (i)]
    for (long i = 0; i < n; i++) {
        double s = rhs[i];
        for (int q = 1; q <= r && i - q >= 0; q++) s -= FB(r - q, i) * y[i - q];
        y[i] = s;
    }
    for (long i = n - 1; i >= 0; i--) {
        double s = y[i];
        for (int q = 1; q <= r && i + q < n; q++) s -= FB(r + q, i) * y[i + q];
        y[i] = s / FB(r, i);
    }
#undef FB
}

/*
 * Cyclic banded solve, one line, half-bandwidth r, bands as in the header.
 * A = B + P K P^T, where P = [e_0 .. e_{r-1}, e_{n-r} .. e_{n-1}] and the
 * 2r x 2r block K holds the wrapped corner entries.  With y = B^{-1} d and
 * Z = B^{-1} P (n x 2r), Woodbury in capacitance form gives
 *   x = y - Z (I + K P^T Z)^{-1} K P^T y.
 * work holds (2r+1)n + 2r n + n + 8r^2 doubles.  Requires n >= 2r + 1... and
 * n >= 4r so the corner rows do not overlap.
 */
int orc_cyclic_banded_line(const double *band, const double *d, double *x,
                           long n, int r, double *work) {
    int w = 2 * r + 1, m = 2 * r;
    double *F = work;
    double *Z = F + (long)w * n;       /* column c at Z[c*n + i] */
    double *col = Z + (long)m * n;     /* length n */
    double *K = col + n;               /* m x m */
    double *C = K + m * m;             /* m x m capacitance */
    double rhs[64];
    long idx[32];
    if (m > 32 || n < 4 * r) return -1;
    memcpy(F, band, sizeof(double) * w * n);
    for (int c = 0; c < r; c++) { idx[c] = c; idx[r + c] = n - r + c; }
    /* K[a][b] = wrapped entry A[idx[a], idx[b]] (zero when not a corner). */
    for (int a = 0; a < m; a++)
        for (int b = 0; b < m; b++) {
            long i = idx[a], j = idx[b];
            double v = 0.0;
            for (int k = 0; k < w; k++) {
                long jj = i + k - r;
                if ((jj < 0 || jj >= n) && wrap(jj, n) == j) v += band[(long)k * n + i];
            }
            K[a * m + b] = v;
        }
    if (band_lu(F, n, r)) return -1;
    band_lu_solve(F, n, r, d, x);                   /* x <- y = B^{-1} d */
    for (int c = 0; c < m; c++) {                   /* Z = B^{-1} P */
        for (long i = 0; i < n; i++) col[i] = 0.0;
        col[idx[c]] = 1.0;
        band_lu_solve(F, n, r, col, Z + (long)c * n);
    }
    /* C = I + K P^T Z ; rhs = K P^T y */
    for (int a = 0; a < m; a++) {
        double s = 0.0;
        for (int b = 0; b < m; b++) s += K[a * m + b] * x[idx[b]];
        rhs[a] = s;
        for (int c = 0; c < m; c++) {
            double t = (a == c) ? 1.0 : 0.0;
            for (int b = 0; b < m; b++) t += K[a * m + b] * Z[(long)c * n + idx[b]];
            C[a * m + c] = t;
        }
    }
    if (orc_dense_solve(C, rhs, m)) return -1;
    for (long i = 0; i < n; i++) {
        double s = 0.0;
        for (int c = 0; c < m; c++) s += Z[(long)c * n + i] * rhs[c];
        x[i] -= s;
    }
    return 0;
}

/* Batched cyclic banded solve (half-bandwidth r); layout as in the header. */
int orc_cyclic_banded(const double *bands, long band_line_stride, const double *d,
                      double *x, long lines, long n, int r) {
    int bad = 0;
    long l;
    long wsize = (long)(2 * r + 1) * n + (long)(2 * r) * n + n + 8L * r * r + 16;
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * wsize);
#pragma omp for schedule(dynamic, 1)
        for (l = 0; l < lines; l++) {
            if (orc_cyclic_banded_line(bands + l * band_line_stride, d + l * n, x + l * n, n, r, work)) {
#pragma omp atomic write
                bad = 1;
            }
        }
        free(work);
    }
    return bad ? -1 : 0;
}

/*
 * Acyclic (non-periodic) banded solve x = B^{-1} d, B the banded matrix
 * without the wrapped corner entries (Sec. 3, acyclic case): banded LU
 * without pivoting (B diagonally dominant), forward and backward solve.
 * Layout as orc_cyclic_banded; entries of `bands` that would wrap are ignored.
 */
int orc_acyclic_banded(const double *bands, long band_line_stride, const double *d,
                       double *x, long lines, long n, int r) {
    int bad = 0;
    long l;
    const long w = 2 * r + 1;
#pragma omp parallel
    {
        double *F = (double *)malloc(sizeof(double) * w * n);
#pragma omp for schedule(dynamic, 1)
        for (l = 0; l < lines; l++) {
            memcpy(F, bands + l * band_line_stride, sizeof(double) * w * n);
            if (band_lu(F, n, r)) {
#pragma omp atomic write
                bad = 1;
            } else {
                band_lu_solve(F, n, r, d + l * n, x + l * n);
            }
        }
        free(F);
    }
    return bad ? -1 : 0;
}

/*
 * out = A x for cyclic banded A (half-bandwidth r), used for residuals
 * ||A x - d|| and for building right-hand sides from known solutions.
 */
void orc_banded_matvec(const double *bands, long band_line_stride, const double *x,
                       double *out, long lines, long n, int r) {
    long l;
#pragma omp parallel for schedule(static)
    for (l = 0; l < lines; l++) {
        const double *b = bands + l * band_line_stride;
        const double *xl = x + l * n;
        double *ol = out + l * n;
        for (long i = 0; i < n; i++) {
            double s = 0.0;
            for (int k = 0; k <= 2 * r; k++) s += b[(long)k * n + i] * xl[wrap(i + k - r, n)];
            ol[i] = s;
        }
    }
}
