/* gpmg3d: the 3-D MAC extension of the ghost-point multigrid on the box
 * domain [0, 1]^3 (walls only, no immersed body).
 *
 * The paper (Sect. 3, "Discretization in space") states that the method
 * extends directly to three dimensions: a staggered grid with u, v, w on the
 * faces and p at the cell centres, the box relaxation of Sect. 4.1.1 on
 * 7 x 7 systems (a cell's pressure and its six faces), and the transfers of
 * Sect. 4.2-4.3 acting per axis.  This library solves the Crank-Nicolson
 * system of Eqs. (NSCN1), (spaceprob) in 3-D:
 *   (1 + 6 a) u - a (six neighbours) + q (p_E - p_W) = b on interior faces
 *   (a = alpha / h^2, q = 1 / h; v and w alike), the continuity rows
 *   q div u - xi = b, the mean row h^3 sum p = b (Eq. spaceprobaug),
 *   velocity on its own wall: x = b; a velocity half a cell outside a wall
 *   next to an interior node: 3/8 x_G + 3/4 x_1 - 1/8 x_2 = b (Eq. BCu with
 *   theta_normal = 1/2); every other outside node is inactive (x = b).
 * V(nu1, nu2) cycles: seven-colour box relaxation ((i + 2 j + 3 k) mod 7),
 * the (xi, mean) update, lambda Jacobi sweeps w += dtau r over the wall and
 * box-ghost rows (Eq. ghostrelax); class-aware restriction, trilinear
 * prolongation renormalised over active coarse nodes, the coarsest level
 * solved exactly by a dense inverse built on the device.
 *
 * Layout of a level with N cells per side: four frames (u, v, w, p) of
 * F = (N + 2)^3 slots, node (i, j, k) of every grid at
 * ((k + 1)(N + 2) + (j + 1))(N + 2) + (i + 1), i, j, k in [-1, N], then 32
 * scalars, scalar 0 = xi (unknown) / the mean row (equation).  Vectors are
 * FP64 device arrays of gp3_vec_len(N) entries; slots outside a grid's
 * range are inactive.
 *
 * Ownership: the caller allocates every device buffer, including the
 * workspace (gp3_workspace_size); the library allocates no device memory
 * and never frees caller memory.  Every call is ordered on the context's
 * stream; calls that return a norm or a status read back synchronise it.
 * Errors: the return code (gp_status of gpmg.h) and gp3_last_error().
 */
#pragma once

#include <stddef.h>
#include <cuda_runtime.h>

#include "gpmg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gp3_ctx gp3_ctx;

/* entries of a level vector: 4 (N + 2)^3 + 32 */
long long gp3_vec_len(int N);

/* bytes of device workspace for N cells per side and `levels` levels
 * (N, N/2, ..., N/2^(levels-1); N <= 1024, divisible by 2^(levels-1),
 * coarsest >= 2, at most 1024 unknowns on the coarsest level) and precision
 * (0 FP64, 1 mixed: adds the FP32 vectors).  GP_INVALID otherwise. */
gp_status gp3_workspace_size(int N, int levels, int precision, size_t *bytes);

/* Create a context: alpha = dt / (2 Re); nu1, nu2 pre/post relaxations;
 * lambda ghost sweeps of step dtau per relaxation; precision 0: gp3_solve
 * runs FP64 cycles; 1: each iteration rounds the FP64 residual to FP32, runs
 * `inner` (1..16) FP32 cycles from zero on it and adds the correction to x in
 * FP64 (the cycle pieces gp3_smooth ... gp3_cycle are FP64 in both).  ws:
 * caller-owned device workspace of at least gp3_workspace_size bytes,
 * 256-byte aligned.  Builds the node types of every level and the
 * coarsest-level inverse (synchronous). */
gp_status gp3_create(gp3_ctx **out, int N, int levels, double alpha, int nu1, int nu2, int lambda, double dtau,
                     int precision, int inner, void *ws, size_t ws_bytes, cudaStream_t stream);
gp_status gp3_destroy(gp3_ctx *ctx);
const char *gp3_last_error(gp3_ctx *ctx);

/* node types of a level (4 F bytes, frame order u, v, w, p): 0 inactive,
 * 1 interior, 3 wall, 4 box ghost */
gp_status gp3_types(gp3_ctx *ctx, int level, unsigned char *types);

/* r = b - M x on a level; ||r||_inf into *norm_host when it is not NULL */
gp_status gp3_residual(gp3_ctx *ctx, int level, const double *x, const double *b, double *r, double *norm_host);

/* nu relaxations (Algorithm relax) in place on x */
gp_status gp3_smooth(gp3_ctx *ctx, int level, double *x, const double *b, int nu);

/* restriction of a residual of `level` into the right-hand side of level + 1 */
gp_status gp3_restrict(gp3_ctx *ctx, int level, const double *r, double *bH);

/* x += P eH on every active node of `level` (eH on level + 1) */
gp_status gp3_prolong(gp3_ctx *ctx, int level, const double *eH, double *x);

/* one V(nu1, nu2) cycle on the finest level, in place */
gp_status gp3_cycle(gp3_ctx *ctx, double *x, const double *b);

/* iterations from x until the FP64 ||b - M x||_inf <= tol or max_cycles
 * cycles (FP32 cycles in the mixed mode); *cycles, *iterations and *res (each
 * may be NULL) report them, hist_host (may be NULL) receives the FP64
 * residual before each iteration and after the last (at most max_cycles + 1
 * entries).  GP_NOT_CONVERGED at the cap, GP_DIVERGED on NaN or growth by 1e6. */
gp_status gp3_solve(gp3_ctx *ctx, double *x, const double *b, double tol, int max_cycles, int *cycles,
                    int *iterations, double *res, double *hist_host);

/* Ghost points of the sphere |x - c| < R (Sect. 3.3 in 3-D) on the grids of a
 * level with N cells per side (the object is phi = R - |x - c| > 0).  Every
 * velocity node of the box interior with phi >= 0 and a fluid neighbour
 * (phi < 0) among its six is a ghost.  Algorithm 1 on the trilinear
 * interpolant of phi on the grid's own nodes gives its boundary point B; its
 * row of Eq. (BCu) interpolates at B from the 27 nodes G - (k, l, m) s h
 * (k, l, m in {0, 1, 2}, s = the signs of the normal at G) with the weights
 * L_k(theta_x) L_l(theta_y) L_m(theta_z), theta = s (x_G - x_B) / h.  The
 * paper has no 3-D formulas; these are its 2-D rows with a third axis.
 * Device outputs of capacity cap (order unspecified): node[n] and st[27 n]
 * as indices into the level vector (frame g * (N + 2)^3 + slot), B[3 n],
 * theta[3 n], w[27 n] (stencil node (k, l, m) at 9 m + 3 l + k).
 * count_dev: two device ints of scratch; *count_host receives the number of
 * ghosts.  Synchronises the stream.  GP_GEOMETRY when the ghosts exceed cap,
 * a march does not leave the object or a stencil leaves the frame. */
gp_status gp3_sphere_ghosts(int N, double cx, double cy, double cz, double R, int cap, int *count_dev, int *node,
                            double *B, double *theta, int *st, double *w, int *count_host, cudaStream_t stream);

/* kernel timer: CUDA events around every box-relaxation launch of `level`
 * until gp3_timer_stop, which returns the launches and their total ms */
gp_status gp3_timer_start(gp3_ctx *ctx, int level);
gp_status gp3_timer_stop(gp3_ctx *ctx, long long *launches, double *ms);

#ifdef __cplusplus
}
#endif
