/*
 * gpmg.h -- C ABI of libgpmg: the monolithic ghost-point multigrid solve of
 * one Crank-Nicolson step of the incompressible Navier-Stokes equations on a
 * staggered (MAC) grid around an object given by a level set
 * (Coco, arXiv 1911.00994).
 *
 * The linear problem (Sect. 2, Eq. spaceprobaug): find (u, v, p, xi) with
 *     u - alpha lap u + grad p = f~   in the fluid,
 *     div u - xi = g                  in the fluid,
 *     sum of p over internal cells = 0 (Eq. midpoint),
 *     u = u_b on the boundary (ghost rows, Eq. BCu),
 * alpha = dt / (2 Re), p the pressure scaled by dt.  Discretised as
 * Algorithm LS (Sect. 3) and solved by geometric multigrid (Sect. 4).
 *
 * Conventions
 *  - All array arguments are DEVICE pointers (CUDA global memory) unless the
 *    name ends in _host.  The caller owns every buffer; the library never
 *    allocates or frees device memory: it carves its internal arrays out of
 *    one caller-provided workspace (gp_workspace_size / gp_create).
 *  - Vector layout of a level with N cells per side (FP64, or FP32 where
 *    stated): three frames of (N+2) rows x P columns, P = gp_pitch(N) (N+2
 *    rounded up to a multiple of 32), then 32 scalars.  Node (i, j) of any
 *    grid lives at frame offset (j+1)*P + (i+1):
 *      u frame (offset 0):        i in [0, N],  j in [-1, N]  at (x0+i h, y0+(j+1/2) h)
 *      v frame (offset F):        i in [-1, N], j in [0, N]   at (x0+(i+1/2) h, y0+j h)
 *      p frame (offset 2F):       i, j in [0, N)              at cell centres
 *      scalar 0 (offset 3F):      xi in an unknown vector, the mean row in a
 *                                 right-hand side or residual.
 *    F = (N+2)*P.  Frame slots outside a grid's range must hold 0.
 *  - Level set: phi on the half-cell lattice, (2N+1) x (2N+1) FP64 values,
 *    phi[b*(2N+1) + a] at (x0 + a h/2, y0 + b h/2).  Paper convention
 *    (Sect. 3.1): phi > 0 inside the object, phi < 0 in the fluid; pass
 *    phi_fluid_positive = 1 for the opposite sign.
 *  - Every call is ordered on the context's stream.  Calls that return host
 *    values (norms, counts, statuses) synchronise that stream.
 *  - Errors: the return code; gp_last_error gives a message.  No call aborts,
 *    traps or waits without bound.  On GP_NOT_CONVERGED / GP_DIVERGED the
 *    iterate holds the last completed cycle.
 */
#ifndef GPMG_H
#define GPMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gp_status {
    GP_OK = 0,
    GP_INVALID = 1,        /* bad argument, size or call order */
    GP_GEOMETRY = 2,       /* level set unusable (no normal, projection failed, body too close to the walls) */
    GP_SINGULAR = 3,       /* zero pivot in the coarsest-level inversion */
    GP_NOT_CONVERGED = 4,  /* cycle cap reached before the tolerance */
    GP_DIVERGED = 5,       /* NaN/Inf or residual above 1e6 x the initial one */
    GP_CUDA = 6            /* a CUDA runtime call failed */
} gp_status;

typedef enum gp_precision { GP_FP64 = 0, GP_MIXED = 1 } gp_precision;

typedef struct gp_params {
    int N;              /* cells per side on the finest grid */
    double x0, y0, L;   /* domain [x0, x0+L] x [y0, y0+L] */
    int levels;         /* grids N, N/2, ..., N/2^(levels-1); the last is solved exactly */
    double alpha;       /* dt / (2 Re) */
    int nu1, nu2;       /* pre / post relaxations (Algorithm relax) */
    int gamma;          /* 1: V-cycle, 2: W-cycle */
    int lambda;         /* ghost sweeps per relaxation (Algorithm relax) */
    double dtau;        /* fictitious time step of Eq. (ghostrelax) */
    double snap;        /* a node within snap*h of the boundary counts as external */
    int precision;      /* gp_precision */
    int max_cycles;     /* cap for mg_solve: cycles of the FP32 corrections (GP_MIXED without krylov),
                           iterations otherwise */
    int cn_buffers;     /* nonzero: carve the four finest-level vectors cn_step needs */
    int graphs;         /* nonzero: mg_solve replays each cycle as a captured CUDA graph
                           (needs a stream other than the legacy default stream) */
    int band;           /* moving bodies (Sect. 3.4): external nodes of the finest grid within
                           `band` index steps of the fluid are ghosts too (extrapolation rows),
                           so that the previous step has values where the fluid advances */
    int krylov;         /* 0: plain cycles; 1: BiCGSTAB preconditioned on the right by one
                           cycle (two cycles per iteration), same stopping test */
    int tile_min;       /* levels with at least this many cells per side sweep their full
                           boxes in one pass of shared-memory tiles (same iterate as the five
                           colour passes); 0: 128 for the FP32 cycles of the mixed mode and
                           never for FP64; negative: never */
    int adjoint;        /* nonzero: carve the arrays of the adjoint solve (mg_solve_t and the
                           gp_*_t calls; one FP64 vector per level and the ghost column lists) */
    int inner;          /* GP_MIXED without krylov: most FP32 cycles per FP64 residual correction
                           (1..GP_MAX_INNER; 0: GP_MAX_INNER).  After the first correction mg_solve takes as
                           many as the last corrections' reduction rate predicts are still needed
                           to reach tol, so the cycle count stays that of one cycle per
                           correction while the FP64 residuals are fewer */
    int wave_min;       /* tiled levels with at least this many cells per side stream their full
                           boxes down strips of rows (same iterate as the tiles); 0: 4096;
                           negative: never */
    int fuse_restrict;  /* positive: the cycle restricts each level's residual in the pass that
                           computes it (the fine residual never goes to memory; the right-hand sides
                           equal the separate passes' but for the rounding of the mean row's sum);
                           0: a residual pass, then a restriction pass (faster on GB300) */
} gp_params;

#define GP_MAX_INNER 8

typedef struct gp_report {
    int cycles;          /* multigrid cycles done */
    int iterations;      /* outer iterations (= cycles for plain cycles; BiCGSTAB: 2 cycles each) */
    double res0;         /* ||b - M x||_inf before the first cycle */
    double res;          /* after the last cycle */
    double rho;          /* geometric mean residual reduction per cycle */
    double xi;           /* final xi */
    double *hist_host;   /* optional host array of max_cycles + 1 norms (one per iteration), or NULL */
} gp_report;

/* Rigid-body velocity of the object: u_b(B) = (U - omega (B_y - cy),
 * V + omega (B_x - cx)) at a boundary point B. */
typedef struct gp_body {
    double U, V, omega, cx, cy;
} gp_body;

/* Tangential velocities of the four box walls (the wall-normal velocities
 * are 0): u on y = y0, u on y = y0 + L, v on x = x0, v on x = x0 + L. */
typedef struct gp_walls {
    double u_bottom, u_top, v_left, v_right;
} gp_walls;

typedef struct gp_cn_report {
    int picard;          /* Picard iterations (Eq. NSitconv); 0 when extrapolated */
    int cycles;          /* multigrid cycles over all solves of the step */
    double res;          /* final ||b - M x||_inf of the last solve */
    double mom_res;      /* Eq. (iterativeNS) residual of the last Picard iterate */
} gp_cn_report;

typedef struct gp_ctx gp_ctx;

/* Defaults: levels down to a 16 x 16 grid, V(2,1), lambda 5, dtau 0.9,
 * snap 0.3, FP64, 100 cycles, alpha = L/N/2, cn_buffers 1, graphs 1. */
gp_status gp_params_default(gp_params *prm, int N, double x0, double y0, double L);

/* Row pitch P and doubles per vector of a level with N cells per side. */
int gp_pitch(int N);
int64_t gp_vector_length(int N);

/* Bytes of device workspace that gp_create needs for these parameters. */
gp_status gp_workspace_size(const gp_params *prm, size_t *bytes);

/* Create a context using `workspace` (device, >= gp_workspace_size bytes,
 * 256-byte aligned, owned by the caller and kept alive until gp_destroy)
 * and `stream` (a cudaStream_t, NULL for the default stream). */
gp_status gp_create(gp_ctx **out, const gp_params *prm, void *workspace, size_t bytes, void *stream);
gp_status gp_destroy(gp_ctx *ctx);
const char *gp_last_error(const gp_ctx *ctx);

/* Change alpha = dt / (2 Re); the coarsest-level inverse is rebuilt on the
 * next call that needs it. */
gp_status gp_set_alpha(gp_ctx *ctx, double alpha);

/* Algorithm LS + Algorithm 1 on every level (Sect. 3.1-3.3): node types,
 * ghost rows (Eq. BCu and extrapolation rows), cut-cell lists and the
 * coarsest-level inverse.  phi: half lattice as described above. */
gp_status geometry_build(gp_ctx *ctx, const double *phi, int phi_fluid_positive);

/* Shapes of the test bodies (Sect. 5, Eq. domains) moving rigidly: at time t
 * the body centre is c(t) = (xc + R cos(2 pi t / T + phase), yc + R sin(...))
 * (R = orbit_r; a fixed body when R = 0) and the body is turned by omega t
 * about c(t).  In body coordinates q:
 *   GP_CIRCLE:  phi = a - |q|
 *   GP_ELLIPSE: phi = 1 - sqrt(q_x^2 / a^2 + q_y^2 / b^2)
 *   GP_FLOWER:  phi = a + b sin(k atan2(q_y, q_x)) - |q|
 * (paper sign: positive inside the body). */
typedef enum gp_shape_kind { GP_CIRCLE = 0, GP_ELLIPSE = 1, GP_FLOWER = 2 } gp_shape_kind;

typedef struct gp_shape {
    int kind;
    double a, b;
    int k;
    double xc, yc;
    double orbit_r, orbit_period, orbit_phase;
    double omega;
} gp_shape;

/* geometry_build for a shape at time t: the level set is evaluated on the
 * half-cell lattice on the device (Sect. 3.1), then as geometry_build.  The
 * rigid-body velocity at t (dc/dt and omega about c(t)) is returned in
 * body_out when it is not NULL. */
gp_status geometry_build_shape(gp_ctx *ctx, const gp_shape *shape, double t, gp_body *body_out);

/* The level-set lattice the geometry was built from, (2N+1)^2 FP64 values in
 * the paper sign, copied to phi_out (device). */
gp_status gp_level_set(gp_ctx *ctx, double *phi_out);

/* Level-set transport for deforming bodies (Sect. 3.1).  phi: the (2N+1)^2
 * half-cell lattice of the context's finest grid (the layout geometry_build
 * reads, spacing dx = h/2), FP64, in place.  work: caller-owned device
 * scratch, 2 (2N+1)^2 doubles for the reinitialisation, (2N+1)^2 for the
 * advection.  Beyond the lattice border phi is taken equal to its border
 * value.  Both return GP_INVALID for bad arguments and are asynchronous on the
 * context stream (no synchronisation).
 *
 * gp_levelset_reinit: `iters` forward-Euler steps in the fictitious time mu
 *   of Eq. (sdf), d phi / d mu = S (1 - |grad phi|), from the current phi
 *   (phi0), S = phi0 / sqrt(phi0^2 + dx^2) and |grad phi| by Godunov's upwind
 *   rule; dtau <= dx (GP_INVALID above), dx / 2 is the usual choice.  The
 *   zero level set stays put to a fraction of dx and phi becomes the signed
 *   distance within about iters * dtau of it.
 * gp_levelset_advect: `steps` first-order upwind steps of
 *   phi_t + w . grad phi = 0 with the velocity (wx, wy) given on the same
 *   lattice; stable for dt (|wx| + |wy|) <= dx (the caller's bound). */
gp_status gp_levelset_reinit(gp_ctx *ctx, double *phi, double *work, int iters, double dtau);
gp_status gp_levelset_advect(gp_ctx *ctx, double *phi, double *work, const double *wx, const double *wy, double dt,
                             int steps);

/* Level information: cells per side, vector length, mesh size. */
gp_status gp_level_info(const gp_ctx *ctx, int level, int *N, int64_t *len, double *h);

/* Node types of a level copied to three device byte arrays of F bytes each
 * (0 inactive, 1 internal, 2 ghost, 3 wall, 4 box ghost). */
gp_status gp_types(gp_ctx *ctx, int level, uint8_t *tu, uint8_t *tv, uint8_t *tp);

/* Number of object ghost rows of a level, and of all ghost-class rows
 * (object ghosts + walls + box ghosts). */
gp_status gp_ghost_count(gp_ctx *ctx, int level, int *n_object, int *n_rows);

/* Object ghost rows of a level, in (grid, j, i) order, copied to device
 * arrays of n_object entries: node = vector index of the ghost, kind
 * (0 Eq. BCu, 1 extrapolation, 2 copy), nst, st[9*n] vector indices of the
 * stencil (row-major per ghost), w[9*n], B[2*n] boundary points, th[2*n]. */
gp_status gp_ghost_rows(gp_ctx *ctx, int level, int *node, uint8_t *kind, uint8_t *nst, int *st, double *w,
                        double *B, double *th);

/* r = b - M x on a level, Eq. (LS); returns ||r||_inf in *norm_host (may be
 * NULL).  x, b, r: FP64 vectors of that level. */
gp_status gp_residual(gp_ctx *ctx, int level, const double *x, const double *b, double *r, double *norm_host);

/* The same residual and norm as gp_residual, for callers that cannot
 * allocate device memory: a plug-in running inside a host application that
 * owns all device memory and hands out none, or a caller whose workspace was
 * sized once for other work and may not grow.  The paper has no counterpart;
 * this is a property of the library only.  It calls no allocator and uses
 * none of the workspace's reduction area: its scratch is a fixed array of
 * about 128 KB inside the library, which every GPU that loads the library
 * keeps until the process exits.  Levels with more than 8192 cells per side
 * return GP_INVALID.  All calls share that array (it keeps the last call's
 * contents; each call clears what must start at zero), so two calls whose
 * kernels overlap on one GPU race.  The first call on a device looks up the
 * array's device address; make that first call before any stream capture.
 * norm_host may be NULL: then only r is returned and the call does not
 * synchronise; otherwise it synchronises the stream to read the norm. */
gp_status gp_residual_static(gp_ctx *ctx, int level, const double *x, const double *b, double *r, double *norm_host);

/* Pieces of the relaxation (Sect. 4.1), in place on x: */
gp_status gp_box_sweep(gp_ctx *ctx, int level, double *x, const double *b);     /* all box colours */
gp_status gp_scalar_update(gp_ctx *ctx, int level, double *x, const double *b); /* xi and mean pressure */
gp_status gp_ghost_sweep(gp_ctx *ctx, int level, double *x, const double *b);   /* one Eq. (ghostrelax) sweep */
gp_status gp_smooth(gp_ctx *ctx, int level, double *x, const double *b, int nu); /* Algorithm relax */

/* Restriction (Sect. 4.2, Eqs. restop, restop5) of a residual of `level`
 * into the right-hand side of level+1. */
gp_status gp_restrict(gp_ctx *ctx, int level, const double *r_fine, double *b_coarse);

/* Prolongation (Sect. 4.3): x_fine += bilinear interpolation of e_coarse. */
gp_status gp_prolong(gp_ctx *ctx, int level, const double *e_coarse, double *x_fine);

/* Exact solve on the coarsest level: x = M^-1 b (Sect. 4.3). */
gp_status gp_coarse_solve(gp_ctx *ctx, const double *b, double *x);

/* One cycle (V or W per params) on the finest level, in place. */
gp_status gp_cycle(gp_ctx *ctx, double *x, const double *b);

/* Iterations from the iterate x until ||b - M x||_inf <= tol (absolute) or
 * max_cycles iterations.  Plain cycles (krylov = 0): each iteration is one
 * cycle; precision GP_MIXED computes the FP64 residual, runs one FP32 cycle
 * on it from zero and adds the FP32 correction to x in FP64.  krylov = 1:
 * BiCGSTAB with one cycle from zero as right preconditioner (FP64 cycle, or
 * FP32 cycle on the FP64 vector in GP_MIXED).  rep may be NULL. */
gp_status mg_solve(gp_ctx *ctx, double *x, const double *b, double tol, gp_report *rep);

/* One Crank-Nicolson step (Sect. 2) on the finest level, in place.
 *  x:      state (u, v with ghost values, p scaled by dt, xi) at t^n, FP64
 *          vector of the finest level; on return the state at t^(n+1) (and
 *          the multigrid warm start is the old state).
 *  N1, N2: convective terms u.grad u of steps n-1 and n-2 (same layout);
 *          rotated on return (N2 <- N1, N1 <- N^n).  Unused for n < 2.
 *  step:   n.  n < 2: mid-point Picard iteration (Eq. NSitconv) until
 *          Eq. (iterativeNS) holds with eps, at most kmax solves; n >= 2:
 *          extrapolation N^n + N^(n-1)/2 - N^(n-2)/2 (Eq. extrUdU).
 *  f:      forcing at t^(n+1/2) on the u, v frames (NULL for none).
 *  bc:     boundary values on the ghost, wall and box-ghost rows of the
 *          finest vector layout (Eq. BCu rows: velocity at B, see
 *          gp_ghost_rows); NULL: rigid-body velocity `body` on the object
 *          and `walls` on the box.
 *  dt, Re: alpha = dt / (2 Re) is set on the context (the coarsest inverse
 *          is rebuilt when alpha changes).
 *  Each linear solve runs mg_solve to `tol`.  The right-hand side is
 *  u^n + alpha lap u^n + dt f - dt N^(n+1/2) on internal momentum rows
 *  (Eqs. NSCN1, spaceprob), g on continuity rows (0 unless set by
 *  gp_set_continuity_source), 0 on extrapolation and mean rows.
 *  Needs cn_buffers.  rep may be NULL. */
gp_status cn_step(gp_ctx *ctx, double *x, double *N1, double *N2, int step, const double *f, const double *bc,
                  double dt, double Re, const gp_body *body, const gp_walls *walls, double tol, double eps, int kmax,
                  gp_cn_report *rep);

/* Continuity source for manufactured solutions (Sect. 5.1: the continuity
 * equation generalised to div u - xi = g with g the divergence of the exact
 * velocity).  g: a finest-level FP64 device vector whose p frame holds g at
 * the cell centres (other slots are not read), owned by the caller and read
 * by every later cn_step and gp_cn_rhs, which write it into the continuity
 * rows of internal cells; NULL restores g = 0.  The adjoint is unaffected (g
 * is a constant of the step). */
gp_status gp_set_continuity_source(gp_ctx *ctx, const double *g);

/* Pieces of cn_step for tests: the convective term of x on internal u, v
 * nodes (0 elsewhere on the u, v frames), and the right-hand side for a
 * given N^(n+1/2). */
gp_status gp_convective(gp_ctx *ctx, const double *x, double *out);
gp_status gp_cn_rhs(gp_ctx *ctx, const double *xn, const double *Nh, const double *f, double dt, const double *bc,
                    const gp_body *body, const gp_walls *walls, double *b);

/* ---- Adjoint of the linear solve: M^T lam = c.
 *
 * For a scalar function J of the solution x of M x = b, dJ/db = lam with
 * M^T lam = dJ/dx; through the right-hand side of cn_step this gives the
 * gradient with respect to the forcing (dt times the momentum entries of
 * lam).  The solver is the transpose of the multigrid cycle: a cycle from
 * zero is a linear map B of b whose stages (box solves, ghost Jacobi steps,
 * the (xi, mean) update, the coarse-grid correction P B_H R) each add
 * Q (b - M x); B^T is the cycle for M^T with the stages in reverse order and
 * each Q transposed (transposed box matrices, cut colours in reverse then full
 * colours 4..0, ghost sweeps before the (xi, mean) step, post- before
 * pre-relaxations, P^T as restriction, R^T as interpolation, the coarsest
 * solve with the transposed inverse).  Rows of M^T at inactive nodes (only
 * ghost rows reference those nodes) are solved exactly after each cycle.
 * FP64 only.  All vectors are device pointers in the layout of the level
 * (gp_vector_length); lam and c use the row slots of M (the xi slot holds
 * the mean row's unknown).  The context must be created with
 * gp_params.adjoint = 1 (else GP_INVALID); the first call after a geometry
 * copies the ghost rows to the host once to list the columns they reference.
 *
 * gp_residual_t: r = c - M^T lam on level `level`, ||r||_inf into *norm_host
 *                when not NULL (synchronises).
 * gp_box_sweep_t, gp_scalar_update_t, gp_ghost_sweep_t, gp_smooth_t: the
 *                transposed relaxation stages, in place on lam.
 * gp_restrict_t: lam_fine += R^T y_coarse (R the restriction level -> level+1).
 * gp_prolong_t:  c_coarse = P^T r_fine (P the interpolation level+1 -> level).
 * gp_cycle_t:    one transposed cycle on the finest level, in place on lam.
 * mg_solve_t:    transposed cycles from lam until ||c - M^T lam||_inf <= tol
 *                (at most max_cycles); the report as for mg_solve. */
gp_status gp_residual_t(gp_ctx *ctx, int level, const double *lam, const double *c, double *r, double *norm_host);
gp_status gp_box_sweep_t(gp_ctx *ctx, int level, double *lam, const double *c);
gp_status gp_scalar_update_t(gp_ctx *ctx, int level, double *lam, const double *c);
gp_status gp_ghost_sweep_t(gp_ctx *ctx, int level, double *lam, const double *c);
gp_status gp_smooth_t(gp_ctx *ctx, int level, double *lam, const double *c, int nu);
gp_status gp_restrict_t(gp_ctx *ctx, int level, const double *y_coarse, double *lam_fine);
gp_status gp_prolong_t(gp_ctx *ctx, int level, const double *r_fine, double *c_coarse);
gp_status gp_cycle_t(gp_ctx *ctx, double *lam, const double *c);
gp_status mg_solve_t(gp_ctx *ctx, double *lam, const double *c, double tol, gp_report *rep);

/* Backward pass of one Crank-Nicolson step (the adjoint of cn_step with
 * bc = NULL, a fixed number kmax of Picard iterations for steps 0 and 1,
 * i.e. eps = 0).  The geometry of step+1 must be built (as for the forward
 * step).  Step m maps x^m to x^(m+1) = M^-1 b, b = A x^m + dt E f - dt E Nh
 * + amp g (A x = x + alpha lap x and E on the internal momentum rows, g the
 * rigid-body velocity `body` at unit amplitude on the Eq. (BCu) rows, Nh the
 * convective term of Eq. extrUdU or of the Picard iteration, Eq. NSitconv).
 * Given xbar_next = dL/dx^(m+1) it adds to xbar_m the derivative through this
 * step, to fbar dL/df (dt E lam summed over the step's solves), to *abar
 * (host) dL/damp, and to nbar0/nbar1/nbar2 the adjoints of the stored
 * convective terms of steps m, m-1, m-2; nbar0 is complete at this step and
 * is turned into xbar_m through the transposed convective Jacobian (the
 * caller then shifts nbar1 -> nbar0, nbar2 -> nbar1 and zeroes nbar2).  Each
 * lam solves M^T lam = xbar by mg_solve_t to `tol`; Picard iterates are
 * recomputed by mg_solve.  All vectors are finest-level device vectors;
 * x_m, f (NULL: no forcing) and xbar_next are read only.  Needs
 * gp_params.adjoint and cn_buffers; walls are the (unscaled) box velocities. */
gp_status cn_step_adjoint(gp_ctx *ctx, int step, const double *x_m, const double *f, double dt, double Re,
                          const gp_body *body, double amp, const gp_walls *walls, double tol, int kmax,
                          const double *xbar_next, double *xbar_m, double *nbar0, double *nbar1, double *nbar2,
                          double *fbar, double *abar);

/* Instrumentation (no counterpart in the paper; used by the benchmark).
 * gp_launch_count: kernels this context has launched so far.
 * gp_timer_start: record CUDA events on the context stream around every
 * launch of one kernel family on one level (kernel: 0 residual, 1 full-box
 * colour sweep, 2 cut-box colour sweep, 3 ghost sweep, 4 xi/mean partial
 * sums, 5 restriction, 6 prolongation, 7 coarsest GEMV); gp_timer_stop
 * synchronises and returns the number of timed launches and their summed
 * device time in milliseconds. */
int64_t gp_launch_count(const gp_ctx *ctx);

/* Arithmetic ceilings of the current device for the FP64 kernels' roofline:
 * FP64 and FP32 fused multiply-add throughput in TFLOP/s (an FMA counts as two
 * flops), measured with CUDA events over 5 launches of a full-occupancy grid
 * whose threads run 8 independent FMA chains of 4096 steps.  sink: a device
 * buffer of at least 8 * 8 * (multiprocessor count) bytes that the kernels may
 * write (they do not for these inputs); stream: a cudaStream_t or NULL.
 * Synchronises the stream. */
gp_status gp_fma_peak(void *sink, void *stream, double *fp64_tflops, double *fp32_tflops);
gp_status gp_timer_start(gp_ctx *ctx, int kernel, int level);
gp_status gp_timer_stop(gp_ctx *ctx, int64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* GPMG_H */
