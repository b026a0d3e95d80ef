/*
 * Oracle for the red-black Gauss-Seidel (RBGS) solve of the 2D Poisson equation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct CPU
 * statement of what the GPU path computes.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may build, load or call it; the library under
 * paper_2607_01735_gb300/ never does, and this file shares no code with it.
 *
 * Build: gcc -O2 -ffp-contract=off (IEEE binary64 / binary32, round to nearest even,
 * no fused multiply-add, so every operation below is one correctly rounded op).
 *
 * Problem (Section 2 of the paper): Poisson's equation with Dirichlet data on the unit
 * square, discretised on a uniform grid with h = 1/(N+1).  We use the -Lap u = f sign
 * (the paper writes Lap u = f, i.e. the same problem with f -> -f), so the 5-point
 * update of Eq. (1) reads
 *
 *     u_ij <- (h^2 f_ij + u_{i-1,j} + u_{i+1,j} + u_{i,j-1} + u_{i,j+1}) * 0.25
 *
 * summed left to right in exactly that order.  Multiplying by 0.25 equals dividing by
 * 4 in IEEE arithmetic (both are the correctly rounded value of the same real number).
 *
 * Colouring (Section 2): a point is red when i + j is even, black otherwise, with the
 * boundary ring at index 0 and N+1 and the interior 1-based.  One sweep updates every
 * red point, then every black point (Algorithm 1 / Algorithm 2: red then black per
 * iteration).  A sweep count of n means n red+black pairs.
 *
 * Storage here is the natural row-major (ni+2) x (nj+2) grid u[i][j] with the ring
 * included, and an ni x nj array f.  i is the row (x, slow) and j the column (y, fast).
 * Rectangular grids and a parity offset exist only so that tests can cut a window out
 * of a large grid: a point (i, j) of the window is red when (i + j + parity) is even.
 */
#include <math.h>
#include <stddef.h>

#define U(i, j) u[(size_t)(i) * (size_t)(nj + 2) + (size_t)(j)]
#define F(i, j) f[(size_t)((i) - 1) * (size_t)nj + (size_t)((j) - 1)]

/* One colour of Eq. (1): every interior point whose colour is `colour` (0 red, 1 black). */
static void half_sweep_f64(int ni, int nj, double h2, const double *f, double *u,
                           int parity, int colour)
{
    for (int i = 1; i <= ni; ++i) {
        for (int j = 1; j <= nj; ++j) {
            if (((i + j + parity) & 1) != colour)
                continue;
            double s = h2 * F(i, j);
            s = s + U(i - 1, j);
            s = s + U(i + 1, j);
            s = s + U(i, j - 1);
            s = s + U(i, j + 1);
            U(i, j) = s * 0.25;
        }
    }
}

/* nsweeps red+black sweeps in float64 (Section 2, Eq. (1); Algorithm 1's sweep order). */
void ref_sweeps_f64(int ni, int nj, double h2, const double *f, double *u, long nsweeps,
                    int parity)
{
    for (long it = 0; it < nsweeps; ++it) {
        half_sweep_f64(ni, nj, h2, f, u, parity, 0);
        half_sweep_f64(ni, nj, h2, f, u, parity, 1);
    }
}

/* Single half-sweep, exported for tests of the colour phases. */
void ref_half_sweep_f64(int ni, int nj, double h2, const double *f, double *u, int parity,
                        int colour)
{
    half_sweep_f64(ni, nj, h2, f, u, parity, colour);
}

/* The same iteration carried out in binary32 (the mixed-precision inner solver). */
void ref_sweeps_f32(int ni, int nj, float h2, const float *f, float *u, long nsweeps,
                    int parity)
{
    for (long it = 0; it < nsweeps; ++it) {
        for (int colour = 0; colour < 2; ++colour) {
            for (int i = 1; i <= ni; ++i) {
                for (int j = 1; j <= nj; ++j) {
                    if (((i + j + parity) & 1) != colour)
                        continue;
                    float s = h2 * F(i, j);
                    s = s + U(i - 1, j);
                    s = s + U(i + 1, j);
                    s = s + U(i, j - 1);
                    s = s + U(i, j + 1);
                    U(i, j) = s * 0.25f;
                }
            }
        }
    }
}

/*
 * Scaled residual of the discrete system A u = b, A = (4 I - neighbours) / h^2 on the
 * interior, b = f plus the ring values / h^2 (Eq. (1) moved to one side):
 *
 *   rt_ij  = (((h^2 f_ij + u_{i-1,j}) + u_{i+1,j}) + u_{i,j-1}) + u_{i,j+1} - 4 u_ij
 *          = h^2 (b - A u)_ij
 *   hb_ij  = h^2 f_ij + the neighbours of (i, j) that lie on the ring, in the same order
 *          = h^2 b_ij
 *
 * sums of squares accumulate in plain i-major order.  Writes sum rt^2 and sum hb^2 and
 * returns rho = sqrt(sum rt^2) / sqrt(sum hb^2), or sqrt(sum rt^2) when b = 0.
 */
double ref_residual_f64(int ni, int nj, double h2, const double *f, const double *u,
                        double *sum_r2, double *sum_b2)
{
    double r2 = 0.0, b2 = 0.0;
    for (int i = 1; i <= ni; ++i) {
        for (int j = 1; j <= nj; ++j) {
            double hf = h2 * F(i, j);
            double s = hf;
            s = s + U(i - 1, j);
            s = s + U(i + 1, j);
            s = s + U(i, j - 1);
            s = s + U(i, j + 1);
            double r = s - 4.0 * U(i, j);
            r2 = r2 + r * r;
            double b = hf;
            if (i == 1)  b = b + U(i - 1, j);
            if (i == ni) b = b + U(i + 1, j);
            if (j == 1)  b = b + U(i, j - 1);
            if (j == nj) b = b + U(i, j + 1);
            b2 = b2 + b * b;
        }
    }
    if (sum_r2) *sum_r2 = r2;
    if (sum_b2) *sum_b2 = b2;
    return b2 > 0.0 ? sqrt(r2) / sqrt(b2) : sqrt(r2);
}

/* Pointwise scaled residual rt (ni x nj), for tests of the residual's structure. */
void ref_residual_field_f64(int ni, int nj, double h2, const double *f, const double *u,
                            double *r)
{
    for (int i = 1; i <= ni; ++i) {
        for (int j = 1; j <= nj; ++j) {
            double s = h2 * F(i, j);
            s = s + U(i - 1, j);
            s = s + U(i + 1, j);
            s = s + U(i, j - 1);
            s = s + U(i, j + 1);
            r[(size_t)(i - 1) * (size_t)nj + (size_t)(j - 1)] = s - 4.0 * U(i, j);
        }
    }
}

/*
 * Solve to a relative residual: check rho every `check_every` sweeps (and before the
 * first sweep), stop at rho <= tol or after max_sweeps.  Returns the sweeps done and
 * writes the last rho.  The paper fixes the iteration count instead (Section 4); the
 * stopping rule is the library's convergence control, stated here in its plain form.
 */
long ref_solve_f64(int ni, int nj, double h2, const double *f, double *u, double tol,
                   int check_every, long max_sweeps, double *rho_out)
{
    long done = 0;
    double rho = ref_residual_f64(ni, nj, h2, f, u, NULL, NULL);
    while (!(rho <= tol) && done < max_sweeps && isfinite(rho)) {
        long k = check_every;
        if (k > max_sweeps - done) k = max_sweeps - done;
        ref_sweeps_f64(ni, nj, h2, f, u, k, 0);
        done += k;
        rho = ref_residual_f64(ni, nj, h2, f, u, NULL, NULL);
    }
    if (rho_out) *rho_out = rho;
    return done;
}

/*
 * Mixed-precision iterative refinement (not in the paper: the growth direction in which
 * the sweeps run in binary32 and only the residual and the correction stay in binary64).
 * One outer step, in this order:
 *   1. rt = h^2 (b - A u) pointwise in binary64 (as ref_residual_field_f64), rho, and
 *      mx = max |rt|;
 *   2. e with mx = m 2^e, 0.5 <= m < 1 (frexp); r32 = (float)(rt * 2^-e);
 *   3. d = `inner` binary32 sweeps of the same red-black iteration on
 *      (4 I - Adj) d = r32, from d = 0 with a zero ring (h^2 f replaced by r32, i.e.
 *      ref_sweeps_f32 with h2 = 1);
 *   4. u = u + (double)d * 2^e at interior points.
 * Stops when rho <= tol (checked before the first step and after each) or after
 * max_sweeps inner sweeps; the last step is shortened to fit.  Returns the inner sweeps
 * done; writes rho and the number of outer steps.
 */
#include <stdlib.h>

long ref_refine_solve(int ni, int nj, double h2, const double *f, double *u, double tol,
                      long inner, long max_sweeps, double *rho_out, long *outer_out)
{
    size_t m = (size_t)ni * (size_t)nj, g = (size_t)(ni + 2) * (size_t)(nj + 2);
    double *rt = (double *)malloc(m * sizeof(double));
    float *r32 = (float *)malloc(m * sizeof(float));
    float *d = (float *)malloc(g * sizeof(float));
    long done = 0, outer = 0;
    double rho = ref_residual_f64(ni, nj, h2, f, u, NULL, NULL);
    ref_residual_field_f64(ni, nj, h2, f, u, rt);
    while (!(rho <= tol) && done < max_sweeps && isfinite(rho)) {
        double mx = 0.0;
        for (size_t q = 0; q < m; ++q)
            if (fabs(rt[q]) > mx) mx = fabs(rt[q]);
        int e = 0;
        frexp(mx, &e);
        double down = ldexp(1.0, -e), up = ldexp(1.0, e);
        for (size_t q = 0; q < m; ++q) r32[q] = (float)(rt[q] * down);
        for (size_t q = 0; q < g; ++q) d[q] = 0.0f;
        long k = inner;
        if (k > max_sweeps - done) k = max_sweeps - done;
        ref_sweeps_f32(ni, nj, 1.0f, r32, d, k, 0);
        for (int i = 1; i <= ni; ++i)
            for (int j = 1; j <= nj; ++j) {
                size_t q = (size_t)i * (size_t)(nj + 2) + (size_t)j;
                u[q] = u[q] + (double)d[q] * up;
            }
        done += k;
        outer += 1;
        rho = ref_residual_f64(ni, nj, h2, f, u, NULL, NULL);
        ref_residual_field_f64(ni, nj, h2, f, u, rt);
    }
    free(rt);
    free(r32);
    free(d);
    if (rho_out) *rho_out = rho;
    if (outer_out) *outer_out = outer;
    return done;
}

/*
 * The fused update (not in the paper: the library's fused mode, rbgs_opts.fma = 1),
 * stated plainly.  Sweeps run in blocks of at most 1024; before each block of m sweeps
 *
 *   B = max |u| over the whole grid, ring included;  Q = max |h2 f_ij| over the interior;
 *   S = (4 B) + ((2 m + 1) Q), each operation rounded to binary64;
 *   e = 61 - k with S = x 2^k, 0.5 <= x < 1 (frexp), at most 1020; e = 0 when S = 0.
 *
 * Within the block every update of Eq. (1), in the same red-then-black order, is
 *
 *   u_ij = RN( (T(h2 f_ij) + T(u_{i-1,j}) + T(u_{i+1,j}) + T(u_{i,j-1}) + T(u_{i,j+1})) 2^-(e+2) )
 *
 * with T(t) = trunc(t 2^e) an integer: the five terms on a fixed-point grid of step 2^-e,
 * summed exactly, divided by 4 and rounded once to binary64 (C's conversion of a 64-bit
 * integer to double rounds to nearest; scaling by a power of two is then exact because
 * e <= 1020 keeps every nonzero result normal).  If B, Q or S is not finite, every point
 * the block updates becomes NaN.  `bq`, when not NULL, supplies B and Q for the first
 * block (a window cut out of a larger grid takes the whole grid's values).
 */
static long long fixed_term(double t, int e)
{
    return (long long)ldexp(t, e);  /* exact scaling, then truncation toward zero */
}

static int block_scale(int ni, int nj, double h2, const double *f, const double *u, long m,
                       const double *bq, int *e_out)
{
    double B = 0.0, Q = 0.0;
    int nan_seen = 0;
    if (bq) {
        B = bq[0];
        Q = bq[1];
    } else {
        for (int i = 0; i <= ni + 1; ++i)
            for (int j = 0; j <= nj + 1; ++j) {
                double a = fabs(U(i, j));
                if (isnan(a)) nan_seen = 1;
                else if (a > B) B = a;
            }
        for (int i = 1; i <= ni; ++i)
            for (int j = 1; j <= nj; ++j) {
                double a = fabs(h2 * F(i, j));
                if (isnan(a)) nan_seen = 1;
                else if (a > Q) Q = a;
            }
    }
    if (nan_seen)
        return 0;
    double t1 = 4.0 * B;
    double t2 = (double)(2 * m + 1) * Q;
    double S = t1 + t2;
    if (!isfinite(S))
        return 0;
    int k = 0, e = 0;
    if (S > 0.0) {
        frexp(S, &k);
        e = 61 - k;
        if (e > 1020) e = 1020;
    }
    *e_out = e;
    return 1;
}

void ref_sweeps_fused(int ni, int nj, double h2, const double *f, double *u, long nsweeps,
                      int parity, const double *bq)
{
    long done = 0;
    while (done < nsweeps) {
        long m = nsweeps - done < 1024 ? nsweeps - done : 1024;
        int e = 0;
        int ok = block_scale(ni, nj, h2, f, u, m, done == 0 ? bq : NULL, &e);
        for (long it = 0; it < m; ++it) {
            for (int colour = 0; colour < 2; ++colour) {
                for (int i = 1; i <= ni; ++i) {
                    for (int j = 1; j <= nj; ++j) {
                        if (((i + j + parity) & 1) != colour)
                            continue;
                        if (!ok) {
                            U(i, j) = NAN;
                            continue;
                        }
                        long long s = fixed_term(h2 * F(i, j), e);
                        s += fixed_term(U(i - 1, j), e);
                        s += fixed_term(U(i + 1, j), e);
                        s += fixed_term(U(i, j - 1), e);
                        s += fixed_term(U(i, j + 1), e);
                        U(i, j) = ldexp((double)s, -(e + 2));
                    }
                }
            }
        }
        done += m;
    }
}

/*
 * The three-dimensional variant (the paper's outlook, Section 5, names 3D problems as
 * future work for the red-black scheme): -Lap u = f on the unit cube, u = g on its
 * boundary, h = 1/(N+1), and the 7-point analogue of Eq. (1),
 *
 *     u_ijk <- (h^2 f_ijk + u_{i-1,j,k} + u_{i+1,j,k} + u_{i,j-1,k} + u_{i,j+1,k}
 *                         + u_{i,j,k-1} + u_{i,j,k+1}) / 6,
 *
 * summed left to right in that order and divided by 6 (one correctly rounded division).
 * A point is red when i + j + k is even; a sweep updates every red point, then every
 * black one.  Storage: the natural (N+2)^3 grid u[i][j][k] (k fastest) with the boundary
 * shell, and an N^3 array f.
 */
#define U3(i, j, k) u[((size_t)(i) * (size_t)(n + 2) + (size_t)(j)) * (size_t)(n + 2) + (size_t)(k)]
#define F3(i, j, k) f[((size_t)((i) - 1) * (size_t)n + (size_t)((j) - 1)) * (size_t)n + (size_t)((k) - 1)]

void ref_sweeps3d_f64(int n, double h2, const double *f, double *u, long nsweeps)
{
    for (long it = 0; it < nsweeps; ++it) {
        for (int colour = 0; colour < 2; ++colour) {
            for (int i = 1; i <= n; ++i) {
                for (int j = 1; j <= n; ++j) {
                    for (int k = 1; k <= n; ++k) {
                        if (((i + j + k) & 1) != colour)
                            continue;
                        double s = h2 * F3(i, j, k);
                        s = s + U3(i - 1, j, k);
                        s = s + U3(i + 1, j, k);
                        s = s + U3(i, j - 1, k);
                        s = s + U3(i, j + 1, k);
                        s = s + U3(i, j, k - 1);
                        s = s + U3(i, j, k + 1);
                        U3(i, j, k) = s / 6.0;
                    }
                }
            }
        }
    }
}

/*
 * Scaled residual of the 3D system: rt = (h^2 f + the six neighbours, in the update's
 * order) - 6 u at every interior point, hb = h^2 f plus the neighbours on the boundary
 * shell (in the same order); rho = sqrt(sum rt^2) / sqrt(sum hb^2) (sqrt(sum rt^2) when
 * b = 0), sums in plain i-major order.
 */
double ref_residual3d_f64(int n, double h2, const double *f, const double *u, double *sum_r2,
                          double *sum_b2)
{
    double r2 = 0.0, b2 = 0.0;
    for (int i = 1; i <= n; ++i) {
        for (int j = 1; j <= n; ++j) {
            for (int k = 1; k <= n; ++k) {
                double hf = h2 * F3(i, j, k);
                double s = hf;
                s = s + U3(i - 1, j, k);
                s = s + U3(i + 1, j, k);
                s = s + U3(i, j - 1, k);
                s = s + U3(i, j + 1, k);
                s = s + U3(i, j, k - 1);
                s = s + U3(i, j, k + 1);
                double r = s - 6.0 * U3(i, j, k);
                r2 = r2 + r * r;
                double b = hf;
                if (i == 1) b = b + U3(i - 1, j, k);
                if (i == n) b = b + U3(i + 1, j, k);
                if (j == 1) b = b + U3(i, j - 1, k);
                if (j == n) b = b + U3(i, j + 1, k);
                if (k == 1) b = b + U3(i, j, k - 1);
                if (k == n) b = b + U3(i, j, k + 1);
                b2 = b2 + b * b;
            }
        }
    }
    if (sum_r2) *sum_r2 = r2;
    if (sum_b2) *sum_b2 = b2;
    return b2 > 0.0 ? sqrt(r2) / sqrt(b2) : sqrt(r2);
}
