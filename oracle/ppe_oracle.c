/*
 * FP64 CPU oracle for the pressure Poisson equation (PPE) on a non-uniform
 * cell-centred Cartesian grid.  TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the benchmark's CPU-baseline leg call it; the product path
 * never does.  It shares no code with the CUDA path.
 *
 * What it computes (Sec. 2.1, Eq. 6; Sec. 2.2, Eq. 10):
 *   The PPE  Dt*D*G*dp = D*u* - bc2  is written  M dp = S  (Eq. 10) with M the
 *   discrete Laplacian.  On a cell-centred grid with widths dx[i], dy[j] the
 *   gradient across the face between cells i and i+1 is
 *   (p[i+1]-p[i]) / ((dx[i]+dx[i+1])/2) and the divergence divides the net
 *   face flux by the cell width.  Homogeneous Neumann walls carry no flux.
 *   Multiplying row (i,j) by -V[i,j] = -dx[i]*dy[j] gives the symmetric
 *   positive semidefinite matrix
 *     A = -V M,   b = -V S,
 *   whose off-diagonals are  -dy[j]*2/(dx[i]+dx[i+1])  (x faces) and
 *   -dx[i]*2/(dy[j]+dy[j+1])  (y faces), with the diagonal equal to minus the
 *   sum of the off-diagonals of its row.
 *
 *   The null space of A is the constant vector.  A solution exists iff
 *   sum(b) = 0; b is projected onto that subspace and every residual too.
 *   The answer is the unique solution with zero volume-weighted mean.
 *
 * The assembled matrix is plain CSR, rows in [ny][nx] row-major order.
 *
 * Built plain (gcc -O2) it runs on one thread; that build is the one the
 * tests use.  Built with -fopenmp (the benchmark's all-core CPU timing only)
 * the vector loops below run on every host core; the reductions then add in
 * a different order, which changes results only at rounding level.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_INCOMPATIBLE = 4, OR_ERR_NOT_CONVERGED = 5 };

/* number of stored entries of the assembled operator */
long or_nnz(int nx, int ny)
{
    long n = (long)nx * ny;
    return n + 2L * (long)(nx - 1) * ny + 2L * (long)nx * (ny - 1);
}

/* CSR assembly of A = -V*M.  rowptr has nx*ny+1 entries; col/val or_nnz(). */
int or_assemble(int nx, int ny, const double *dx, const double *dy,
                long *rowptr, int *col, double *val)
{
    if (nx < 1 || ny < 1) return OR_ERR_ARG;
    long k = 0;
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long row = (long)j * nx + i;
            rowptr[row] = k;
            double aS = 0.0, aW = 0.0, aE = 0.0, aN = 0.0;
            if (j > 0)      aS = -dx[i] * 2.0 / (dy[j - 1] + dy[j]);
            if (i > 0)      aW = -dy[j] * 2.0 / (dx[i - 1] + dx[i]);
            if (i < nx - 1) aE = -dy[j] * 2.0 / (dx[i] + dx[i + 1]);
            if (j < ny - 1) aN = -dx[i] * 2.0 / (dy[j] + dy[j + 1]);
            double diag = -(aS + aW + aE + aN);
            if (j > 0)      { col[k] = (int)(row - nx); val[k++] = aS; }
            if (i > 0)      { col[k] = (int)(row - 1);  val[k++] = aW; }
            col[k] = (int)row; val[k++] = diag;
            if (i < nx - 1) { col[k] = (int)(row + 1);  val[k++] = aE; }
            if (j < ny - 1) { col[k] = (int)(row + nx); val[k++] = aN; }
        }
    }
    rowptr[(long)nx * ny] = k;
    return OR_OK;
}

/* y = A x */
void or_spmv(long n, const long *rowptr, const int *col, const double *val,
             const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (long r = 0; r < n; ++r) {
        double s = 0.0;
        for (long k = rowptr[r]; k < rowptr[r + 1]; ++k) s += val[k] * x[col[k]];
        y[r] = s;
    }
}

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* v <- v - mean(v): projection onto range(A) = {sum v = 0} */
static void project(long n, double *v)
{
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (long i = 0; i < n; ++i) s += v[i];
    s /= (double)n;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) v[i] -= s;
}

/*
 * Jacobi-preconditioned CG on A x = b with b in range(A), from the given x.
 * The residual is projected onto range(A) after every update.  Stops when the
 * recursive residual norm is <= tol_abs or after maxit iterations.
 * Returns the number of iterations taken.
 */
long or_jpcg(long n, const long *rowptr, const int *col, const double *val,
             const double *b, double *x, double tol_abs, long maxit)
{
    double *r = malloc(n * sizeof(double)), *z = malloc(n * sizeof(double));
    double *p = malloc(n * sizeof(double)), *q = malloc(n * sizeof(double));
    double *dinv = malloc(n * sizeof(double));
    for (long i = 0; i < n; ++i) {
        double d = 0.0;
        for (long k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (col[k] == i) d = val[k];
        dinv[i] = d > 0.0 ? 1.0 / d : 0.0;
    }
    or_spmv(n, rowptr, col, val, x, q);
    for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
    project(n, r);
    for (long i = 0; i < n; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
    double rz = dot(n, r, z);
    long it = 0;
    while (it < maxit && sqrt(dot(n, r, r)) > tol_abs) {
        or_spmv(n, rowptr, col, val, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) break;
        double alpha = rz / pq;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        project(n, r);
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        ++it;
    }
    free(r); free(z); free(p); free(q); free(dinv);
    return it;
}

/* b = -V S, with V[j][i] = dx[i]*dy[j] */
void or_scaled_rhs(int nx, int ny, const double *dx, const double *dy,
                   const double *S, double *b)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            b[(long)j * nx + i] = -dx[i] * dy[j] * S[(long)j * nx + i];
}

/*
 * Full solve of M x = S on the grid: returns the solution with zero
 * volume-weighted mean whose true relative residual ||P(b - A x)|| / ||P b||
 * is <= tol_rel (P: projection onto range(A)).
 *   x        in: initial guess, out: solution
 *   out[0]   true relative residual reached
 *   out[1]   total CG iterations
 *   out[2]   |sum b| / sum |b| before projection (compatibility defect)
 * Returns OR_ERR_INCOMPATIBLE if that defect exceeds 1e-6.
 */
int or_solve(int nx, int ny, const double *dx, const double *dy,
             const double *S, double *x, double tol_rel, long maxit,
             double *out)
{
    long n = (long)nx * ny;
    long nnz = or_nnz(nx, ny);
    long *rowptr = malloc((n + 1) * sizeof(long));
    int *col = malloc(nnz * sizeof(int));
    double *val = malloc(nnz * sizeof(double));
    double *b = malloc(n * sizeof(double)), *r = malloc(n * sizeof(double));
    or_assemble(nx, ny, dx, dy, rowptr, col, val);
    or_scaled_rhs(nx, ny, dx, dy, S, b);
    double sb = 0.0, sab = 0.0;
    for (long i = 0; i < n; ++i) { sb += b[i]; sab += fabs(b[i]); }
    out[2] = sab > 0.0 ? fabs(sb) / sab : 0.0;
    int status = OR_OK;
    if (out[2] > 1e-6) status = OR_ERR_INCOMPATIBLE;
    project(n, b);
    double bnorm = sqrt(dot(n, b, b));
    long iters = 0;
    double relres = 0.0;
    if (status == OR_OK && bnorm > 0.0) {
        for (int restart = 0; restart < 20; ++restart) {
            or_spmv(n, rowptr, col, val, x, r);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < n; ++i) r[i] = b[i] - r[i];
            project(n, r);
            relres = sqrt(dot(n, r, r)) / bnorm;
            if (relres <= tol_rel || iters >= maxit) break;
            iters += or_jpcg(n, rowptr, col, val, b, x, 0.5 * tol_rel * bnorm, maxit - iters);
        }
        if (relres > tol_rel) status = OR_ERR_NOT_CONVERGED;
    }
    if (bnorm == 0.0) for (long i = 0; i < n; ++i) x[i] = 0.0;
    /* zero volume-weighted mean */
    double sv = 0.0, svx = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double v = dx[i] * dy[j];
            sv += v;
            svx += v * x[(long)j * nx + i];
        }
    for (long i = 0; i < n; ++i) x[i] -= svx / sv;
    out[0] = relres;
    out[1] = (double)iters;
    free(rowptr); free(col); free(val); free(b); free(r);
    return status;
}
