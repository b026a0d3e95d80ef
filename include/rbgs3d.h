/*
 * rbgs3d.h -- C ABI of the 3D red-black Gauss-Seidel variant in librbgs.so.
 *
 * The paper's outlook (Section 5) names the extension of the red-black scheme to 3D
 * problems as future work; this is that variant for the 7-point Laplacian:
 *   -Lap u = f on the unit cube, u = g on its boundary, h = 1/(N+1), and the 3D analogue
 *   of Eq. (1),
 *       u_ijk <- (h^2 f_ijk + u_{i-1,j,k} + u_{i+1,j,k} + u_{i,j-1,k} + u_{i,j+1,k}
 *                            + u_{i,j,k-1} + u_{i,j,k+1}) / 6,
 *   applied to every red point (i + j + k even), then to every black point.
 * Arithmetic: the six adds in that order, each correctly rounded, then one correctly
 * rounded division by 6: the same bits as a plain sequential C loop.
 *
 * Grids, row-major with k fastest: f is N^3 interior values (f_ijk at ((i-1) N + (j-1)) N
 * + (k-1)); u is (N+2)^3 including the boundary shell (u_ijk at ((i (N+2) + j) (N+2) + k).
 * Pointers may address host or device memory; the caller keeps ownership of what it
 * passes, the context owns its device buffers (about 4 (N+2)^3 doubles).  Statuses,
 * streams and threads as in rbgs.h.
 */
#ifndef RBGS3D_H
#define RBGS3D_H

#include "rbgs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbgs3d_ctx *rbgs3d_t;

/*
 * Section 5's 3D variant (Eq. (1) with six neighbours).  Creates a solver for one N^3
 * problem (1 <= N <= 2048): f (N^3 values), u_init ((N+2)^3 values with the boundary
 * shell and the initial guess), h2 = h*h as the caller wants it rounded, stream a
 * cudaStream_t (NULL: legacy default).  RBGS_EINVAL for bad arguments, RBGS_ENOMEM when
 * the device buffers do not fit.
 */
rbgs_status rbgs3d_create(int n, double h2, const double *f, const double *u_init, void *cuda_stream,
                          rbgs3d_t *out);

/* nsweeps red+black sweeps of the 7-point update (Section 5's 3D variant of Eq. (1)). Async. */
rbgs_status rbgs3d_sweep(rbgs3d_t ctx, long nsweeps);

/*
 * Not in the paper (it fixes the iteration count, Section 4): relative residual
 * rho = ||b - A u||_2 / ||b||_2 of the 3D system, A = (6 I - neighbours)/h^2, the shell
 * folded into b.  Synchronises the stream; RBGS_ENONFINITE when rho is NaN or Inf.
 */
rbgs_status rbgs3d_residual(rbgs3d_t ctx, double *rel);

/* Copies the iterate, shell included, into u_out ((N+2)^3 values).  Not in the paper:
 * library mechanics. */
rbgs_status rbgs3d_get_solution(rbgs3d_t ctx, double *u_out);

/* Frees the context (NULL is ignored).  Not in the paper: library mechanics. */
void rbgs3d_destroy(rbgs3d_t ctx);

#ifdef __cplusplus
}
#endif

#endif /* RBGS3D_H */
