/*
 * gpmg_oracle.c -- plain, slow, FP64 CPU oracle for the ghost-point multigrid
 * solve of one Crank-Nicolson step (Coco, arXiv 1911.00994).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * Built serially by default.  The benchmark's multi-core CPU baseline builds
 * it a second time with OpenMP: the only parallel loops are the boxes of one
 * colour (independent by construction) and row-wise loops whose rows write
 * disjoint outputs (residual, restriction, interpolation), so the iterate is
 * bitwise the same for any thread count; every sum stays serial.
 *
 * Everything is written the direct way: every equation of the linear system
 * is produced by one function (get_row) that lists its coefficients, and the
 * residual, the assembled matrix, the box relaxation and the ghost relaxation
 * all read those rows.  Nothing is fused, blocked or reordered.
 *
 * Paper sections followed:
 *   Sect. 2, Eq. (spaceprobaug)  augmented problem (u, v, p, xi)
 *   Sect. 3.2                    MAC central differences, internal points
 *   Eq. (midpoint)               zero-mean pressure row
 *   Sect. 3.3, Algorithm 1       boundary point B from a ghost point G
 *   Eq. (BCu)                    biquadratic upwind ghost row
 *   Remark 1                     which external points are ghosts
 *   Algorithm LS                 row per grid point
 *   Sect. 4.1                    box relaxation and ghost relaxation,
 *                                Eq. (ghostrelax), Algorithm relax
 *   Sect. 4.2, Eqs. (restop), (restop5)  boundary-aware restriction
 *   Sect. 4.3                    bilinear interpolation, cycle, exact coarsest solve
 *   Eq. (convfact)               residual infinity norm
 *
 * Readings where the paper is silent (numbered as in the design notes):
 *   theta sign: theta = s (x_G - x_B)/h, so the Lagrange node k sits at theta = k.
 *   p ghosts: p_G - 2 p_1 + p_2 = 0; u/v ghosts with theta > 1 on an axis
 *     (B beyond the first stencil point; such ghosts only enter other ghost
 *     stencils): x_G - 3 x_1 + 3 x_2 - x_3 = 0; both along the dominant
 *     normal axis a (tie -> x), s = SIGN(n_a), nodes x_k = x_{G - k s e_a},
 *     used where phi decreases strictly along the nodes, else a copy of the
 *     axis neighbour of smallest phi.
 *   outer walls: wall-normal velocity on the wall is a Dirichlet row; the
 *     tangential velocity half a cell outside the wall has the Eq. (BCu) row
 *     with theta_normal = 1/2, theta_tangential = 0: 3/8 x_G + 3/4 x_1 - 1/8 x_2.
 *   ghosts: the external points coupled to the internal equations, closed
 *     under the ghost stencils (the alternative marking of Remark 1), the
 *     closure limited to points within two index steps of an internal point
 *     of the same grid; a ghost stencil point beyond that is inactive (value 0,
 *     the fictitious row of Algorithm LS).
 *   a pressure cell with no internal face is not internal (its continuity row
 *     would not contain any box unknown).
 *   xi / mean pair: after each box sweep xi <- mean(div u - b_c) over internal
 *     cells, then a constant shift of all internal and ghost p makes the mean
 *     row exact.  The mean row is stored as h^2 * sum(p).
 *   box contents: p_ij and the internal or object-ghost borders of the cell
 *     (their own rows); wall and box-ghost borders frozen.
 *   box colouring: cells without ghost borders by (i + 3 j) mod 5, then cells
 *     with ghost borders by (i mod 5, j mod 5); boxes of one colour are
 *     independent.
 *   internal faces that belong to no internal box: point Jacobi after the box
 *     sweep.
 *   ghost relaxation: Jacobi over all ghost-class rows, lambda sweeps; mode 0
 *     w += dtau r (as printed), mode 1 w += dtau r / c_G.
 *   restriction classes: internal, and ghost-class = ghost, wall, box ghost;
 *     mean-row residual injected.
 *   prolongation: bilinear over the active coarse nodes around the fine
 *     node, weights renormalised; p next to the box walls: linear
 *     extrapolation from the two nearest coarse cells.
 *   snap: a node within snap * h of the boundary (phi / |grad phi|) is
 *     external (default 0.3).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXLEV 16
#define OR_MAXMARCH 64

enum { T_INACTIVE = 0, T_INTERNAL = 1, T_GHOST = 2, T_WALL = 3, T_BOXGHOST = 4, T_EXT = 5 };
enum { G_U = 0, G_V = 1, G_P = 2 };
enum { OR_OK = 0, OR_INVALID = 1, OR_GEOMETRY = 2, OR_SINGULAR = 3, OR_NOT_CONVERGED = 4, OR_DIVERGED = 5 };

/* offsets of node (0,0) of each grid, in half cells: u (0,1), v (1,0), p (1,1) */
static const int OX2[3] = {0, 1, 1};
static const int OY2[3] = {1, 0, 1};

typedef struct {
    int grid, i, j;
    double xB, yB;     /* boundary point (u, v ghosts) */
    double nx, ny;     /* unit normal at G from the bilinear interpolant */
    int sx, sy;        /* upwind signs SIGN(n) */
    double thx, thy;   /* Lagrange coordinates of B */
    int axis;          /* extrapolation rows: 0 = x, 1 = y */
    int kind;          /* 0: Eq. (BCu) row; 1: extrapolation row; 2: copy row */
    int nst;
    int si[9], sj[9];
    double w[9];       /* w[0] multiplies the ghost value itself */
} ghost_t;

typedef struct {
    int N;
    double h;
    int nU, nV, nP, n;
    int8_t *tU, *tV, *tP;
    int *gid;          /* unknown index -> ghost index, or -1 */
    int8_t *prim;      /* 1: ghost referenced directly by an internal or box-ghost row */
    ghost_t *gh;
    int ngh;
    int n_int;         /* internal pressure cells */
    /* coarsest level: dense LU factors */
    double *lu;
    int *piv;
    /* cycle work vectors */
    double *x, *b, *r;
    /* adjoint: the columns of M (compressed by column) and, on the coarsest
     * level, the LU factors of M^T */
    int *cptr, *crow;
    double *cval;
    double *lut;
    int *pivt;
    /* colour of every cut cell (cell j N + i; -1 for other cells) */
    int *cutcol;
    int ncutcol;
} level_t;

typedef struct {
    int N, L;
    double x0, y0, len, alpha;
    int nu1, nu2, gamma, lam, ghost_mode, order_mode;
    double dtau;
    double snap;       /* nodes with phi / |grad phi| >= -snap h are external */
    int band;          /* extra ghost layers around the fluid (moving bodies) */
    const double *csrc; /* continuity source g (flat vector, p block), or NULL */
    unsigned rng;
    double *phi;       /* half lattice (2N+1)^2, paper sign */
    level_t lv[OR_MAXLEV];
    int geom_ok;
    int adj_ok;        /* columns and transposed factors built for adj_alpha */
    double adj_alpha;
    char err[256];
} ctx_t;

typedef struct {
    int n;
    int col[12];
    double a[12];
} row_t;

/* ---------------------------------------------------------------- indexing */

static int inU(const level_t *l, int i, int j) { return i >= 0 && i <= l->N && j >= -1 && j <= l->N; }
static int inV(const level_t *l, int i, int j) { return i >= -1 && i <= l->N && j >= 0 && j <= l->N; }
static int inP(const level_t *l, int i, int j) { return i >= 0 && i < l->N && j >= 0 && j < l->N; }
static int inG(const level_t *l, int g, int i, int j)
{
    return g == G_U ? inU(l, i, j) : g == G_V ? inV(l, i, j) : inP(l, i, j);
}
static int iU(const level_t *l, int i, int j) { return (j + 1) * (l->N + 1) + i; }
static int iV(const level_t *l, int i, int j) { return l->nU + j * (l->N + 2) + (i + 1); }
static int iP(const level_t *l, int i, int j) { return l->nU + l->nV + j * l->N + i; }
static int iG(const level_t *l, int g, int i, int j)
{
    return g == G_U ? iU(l, i, j) : g == G_V ? iV(l, i, j) : iP(l, i, j);
}
static int iXI(const level_t *l) { return l->n - 1; }

static int8_t *tref(level_t *l, int g, int i, int j)
{
    if (g == G_U) return &l->tU[(j + 1) * (l->N + 1) + i];
    if (g == G_V) return &l->tV[j * (l->N + 2) + (i + 1)];
    return &l->tP[j * l->N + i];
}
static int ttype(level_t *l, int g, int i, int j)
{
    if (!inG(l, g, i, j)) return T_INACTIVE;
    return *tref(l, g, i, j);
}

static void seterr(ctx_t *c, const char *m)
{
    if (!c->err[0]) snprintf(c->err, sizeof c->err, "%s", m);
}

/* ----------------------------------------------------------- level set */

/* phi at node (i, j) of grid g on level lev, read from the half lattice */
static int phi_node(ctx_t *c, int lev, int g, int i, int j, double *out)
{
    int m = 1 << lev;
    int a = m * (2 * i + OX2[g]);
    int b = m * (2 * j + OY2[g]);
    int M = 2 * c->N;
    if (a < 0 || a > M || b < 0 || b > M) return 0;
    *out = c->phi[(size_t)b * (M + 1) + a];
    return 1;
}

static double node_x(ctx_t *c, int lev, int g, int i) { return c->x0 + (double)(2 * i + OX2[g]) * (0.5 * c->lv[lev].h); }
static double node_y(ctx_t *c, int lev, int g, int j) { return c->y0 + (double)(2 * j + OY2[g]) * (0.5 * c->lv[lev].h); }

/* Bilinear interpolant of phi on the 2x2 cell of grid g that contains (x, y)
 * (cell chosen by floor in each axis), its value and gradient (Sect. 3.3). */
static int bilin(ctx_t *c, int lev, int g, double x, double y, double *val, double *gx, double *gy)
{
    double h = c->lv[lev].h;
    double sx = (x - c->x0) / h - 0.5 * (double)OX2[g];
    double sy = (y - c->y0) / h - 0.5 * (double)OY2[g];
    double fi = floor(sx), fj = floor(sy);
    if (!(fi > -1e9 && fi < 1e9 && fj > -1e9 && fj < 1e9)) return 0;
    int i0 = (int)fi, j0 = (int)fj;
    double fx = sx - fi, fy = sy - fj;
    double p00, p10, p01, p11;
    if (!phi_node(c, lev, g, i0, j0, &p00) || !phi_node(c, lev, g, i0 + 1, j0, &p10) ||
        !phi_node(c, lev, g, i0, j0 + 1, &p01) || !phi_node(c, lev, g, i0 + 1, j0 + 1, &p11))
        return 0;
    double ex = 1.0 - fx, ey = 1.0 - fy;
    *val = ex * ey * p00 + fx * ey * p10 + ex * fy * p01 + fx * fy * p11;
    *gx = (ey * (p10 - p00) + fy * (p11 - p01)) / h;
    *gy = (ex * (p01 - p00) + fx * (p11 - p10)) / h;
    return 1;
}

static int unit_normal(ctx_t *c, int lev, int g, double x, double y, double *nx, double *ny)
{
    double v, gx, gy;
    if (!bilin(c, lev, g, x, y, &v, &gx, &gy)) return 0;
    double nrm = sqrt(gx * gx + gy * gy);
    if (!(nrm > 0.0)) return 0;
    *nx = gx / nrm;
    *ny = gy / nrm;
    return 1;
}

/* Algorithm 1: march from G against the normal by h/2 until phi <= 0, then
 * ceil(log2(|HK| / (0.01 h))) bisection steps; B is the last midpoint.
 * A ghost inside the fluid (phi(G) < 0, a snapped node) marches along the
 * normal instead, until phi >= 0; the bisection is the same. */
static int ghost_to_boundary(ctx_t *c, int lev, int g, int i, int j, double *xB, double *yB)
{
    double h = c->lv[lev].h;
    double xG = node_x(c, lev, g, i), yG = node_y(c, lev, g, j);
    double phH;
    if (!phi_node(c, lev, g, i, j, &phH)) return 0;
    double sg = phH > 0.0 ? 1.0 : -1.0;
    double xH = xG, yH = yG, xK = xG, yK = yG;
    int steps = 0;
    while (sg * phH > 0.0) {
        double nx, ny, gx, gy;
        xK = xH;
        yK = yH;
        if (!unit_normal(c, lev, g, xH, yH, &nx, &ny)) return 0;
        xH = xH - sg * (0.5 * h * nx);
        yH = yH - sg * (0.5 * h * ny);
        if (!bilin(c, lev, g, xH, yH, &phH, &gx, &gy)) return 0;
        if (++steps > OR_MAXMARCH) return 0;
    }
    if (steps == 0) { /* phi(G) = 0: the ghost lies on the boundary */
        *xB = xG;
        *yB = yG;
        return 1;
    }
    double dx = xH - xK, dy = yH - yK;
    double dist = sqrt(dx * dx + dy * dy);
    int nb = (int)ceil(log2(dist / (0.01 * h)));
    double xm = xH, ym = yH;
    for (int it = 0; it < nb; it++) {
        double phB, gx, gy;
        xm = 0.5 * (xH + xK);
        ym = 0.5 * (yH + yK);
        if (!bilin(c, lev, g, xm, ym, &phB, &gx, &gy)) return 0;
        if (phB * phH < 0.0) {
            xK = xm;
            yK = ym;
        } else {
            xH = xm;
            yH = ym;
            phH = phB;
        }
    }
    *xB = xm;
    *yB = ym;
    return 1;
}

/* Lagrange weights on nodes theta = 0, 1, 2 (Eq. BCu) */
static void lagrange3(double t, double T[3])
{
    T[0] = (1.0 - t) * (2.0 - t) / 2.0;
    T[1] = t * (2.0 - t);
    T[2] = t * (t - 1.0) / 2.0;
}

/* Row of an external node acting as a ghost.
 *  u, v ghosts referenced directly by an internal or box-ghost row whose
 *  boundary point B lies within one cell of G along both axes
 *  (theta_x, theta_y <= 1): Eq. (BCu) on the upwind nine-point stencil.
 *  Other u, v ghosts (only other ghost stencils use them): quadratic
 *  extrapolation along the dominant normal axis a, s = SIGN(n_a):
 *      x_G - 3 x_{G - s e_a} + 3 x_{G - 2 s e_a} - x_{G - 3 s e_a} = 0.
 *  p ghosts: linear extrapolation along the same axis:
 *      p_G - 2 p_{G - s e_a} + p_{G - 2 s e_a} = 0.
 *  An extrapolation row is used only where phi strictly decreases along its
 *  nodes; elsewhere (a body thinner than the stencil) the ghost copies the
 *  axis neighbour of smallest phi, x_G - x_nb = 0.  Every extrapolation or
 *  copy row thus refers to nodes of smaller phi only. */
static int ghost_setup(ctx_t *c, int lev, int g, int i, int j, ghost_t *G)
{
    double h = c->lv[lev].h;
    double xG = node_x(c, lev, g, i), yG = node_y(c, lev, g, j);
    double nx, ny;
    if (!unit_normal(c, lev, g, xG, yG, &nx, &ny)) return 0;
    memset(G, 0, sizeof *G);
    G->grid = g;
    G->i = i;
    G->j = j;
    G->nx = nx;
    G->ny = ny;
    G->sx = nx >= 0.0 ? 1 : -1;
    G->sy = ny >= 0.0 ? 1 : -1;
    G->axis = fabs(nx) >= fabs(ny) ? 0 : 1;
    G->kind = 1;
    if (g != G_P) {
        double xB, yB;
        if (!ghost_to_boundary(c, lev, g, i, j, &xB, &yB)) return 0;
        G->xB = xB;
        G->yB = yB;
        G->thx = (double)G->sx * (xG - xB) / h;
        G->thy = (double)G->sy * (yG - yB) / h;
        if (c->lv[lev].prim[iG(&c->lv[lev], g, i, j)] && G->thx <= 1.0 && G->thy <= 1.0) G->kind = 0;
    }
    if (G->kind == 0) {
        double Tx[3], Ty[3];
        lagrange3(G->thx, Tx);
        lagrange3(G->thy, Ty);
        G->nst = 9;
        for (int ky = 0; ky < 3; ky++)
            for (int kx = 0; kx < 3; kx++) {
                G->si[ky * 3 + kx] = i - kx * G->sx;
                G->sj[ky * 3 + kx] = j - ky * G->sy;
                G->w[ky * 3 + kx] = Tx[kx] * Ty[ky];
            }
        return 1;
    }
    /* extrapolation along the dominant normal axis toward the fluid, used
     * only where phi strictly decreases along the stencil (so that no chain
     * of extrapolation rows can loop back on itself) */
    static const double e3[3] = {1.0, -2.0, 1.0};
    static const double e4[4] = {1.0, -3.0, 3.0, -1.0};
    int s = G->axis == 0 ? G->sx : G->sy;
    int n = g == G_P ? 3 : 4;
    double ph[4];
    int mono = 1;
    for (int k = 0; k < n && mono; k++) {
        int ii = i - (G->axis == 0 ? k * s : 0), jj = j - (G->axis == 1 ? k * s : 0);
        if (!phi_node(c, lev, g, ii, jj, &ph[k])) mono = 0;
        else if (k > 0 && !(ph[k] < ph[k - 1])) mono = 0;
    }
    if (mono) {
        G->nst = n;
        for (int k = 0; k < n; k++) {
            G->si[k] = i - (G->axis == 0 ? k * s : 0);
            G->sj[k] = j - (G->axis == 1 ? k * s : 0);
            G->w[k] = g == G_P ? e3[k] : e4[k];
        }
        return 1;
    }
    /* otherwise copy the value of the axis neighbour with the smallest phi
     * below phi(G) (order of preference: -x, +x, -y, +y on ties) */
    static const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
    double pG, best = 0.0;
    int kb = -1;
    if (!phi_node(c, lev, g, i, j, &pG)) return 0;
    for (int k = 0; k < 4; k++) {
        double q;
        if (!phi_node(c, lev, g, i + di[k], j + dj[k], &q)) continue;
        if (q < pG && (kb < 0 || q < best)) { best = q; kb = k; }
    }
    if (kb < 0) return 0;
    G->kind = 2;
    G->nst = 2;
    G->si[0] = i; G->sj[0] = j; G->w[0] = 1.0;
    G->si[1] = i + di[kb]; G->sj[1] = j + dj[kb]; G->w[1] = -1.0;
    return 1;
}

/* ------------------------------------------------------------ geometry */

static void free_level(level_t *l)
{
    free(l->tU); free(l->tV); free(l->tP); free(l->gid); free(l->prim); free(l->gh);
    free(l->lu); free(l->piv); free(l->x); free(l->b); free(l->r);
    free(l->cptr); free(l->crow); free(l->cval); free(l->lut); free(l->pivt); free(l->cutcol);
    memset(l, 0, sizeof *l);
}

/* Mark node (g,i,j) as needed by an internal or box-ghost row: an external
 * node becomes a ghost. */
static int mark_needed(ctx_t *c, level_t *l, int g, int i, int j, int *changed)
{
    if (!inG(l, g, i, j)) { seterr(c, "stencil leaves the grid"); return 0; }
    int8_t *t = tref(l, g, i, j);
    if (*t == T_EXT) { *t = T_GHOST; *changed = 1; }
    else if (*t == T_INACTIVE) { seterr(c, "stencil reaches an inactive corner node"); return 0; }
    if (*t == T_GHOST) l->prim[iG(l, g, i, j)] = 1;
    return 1;
}

/* Is (g,i,j) within two index steps (Chebyshev) of an internal node of the
 * same grid?  Only such nodes may join the ghost set through the stencil of
 * another ghost; farther stencil nodes stay inactive (value 0). */
static int near_internal(level_t *l, int g, int i, int j, int rad)
{
    for (int dj = -rad; dj <= rad; dj++)
        for (int di = -rad; di <= rad; di++)
            if (ttype(l, g, i + di, j + dj) == T_INTERNAL) return 1;
    return 0;
}

/* Mark a node referenced by a ghost stencil. */
static int mark_stencil(ctx_t *c, level_t *l, int g, int i, int j, int *changed)
{
    if (!inG(l, g, i, j)) { seterr(c, "stencil leaves the grid"); return 0; }
    int8_t *t = tref(l, g, i, j);
    int rad = (c->band > 2 && l == &c->lv[0]) ? c->band : 2;
    if (*t == T_EXT && near_internal(l, g, i, j, rad)) { *t = T_GHOST; *changed = 1; }
    return 1;
}

/* Algorithm LS marks a node internal when phi < 0.  A node closer than
 * snap * h to the boundary (first-order distance phi / |grad phi| of the
 * bilinear interpolant of its own grid) is treated as external, so that no
 * Eq. (BCu) row has its boundary point next to an internal node (vanishing
 * ghost coefficient) and no internal cell sits on the boundary. */
static int node_internal(ctx_t *c, int lev, int g, int i, int j, double ph)
{
    if (!(ph < 0.0)) return 0;
    if (c->snap <= 0.0) return 1;
    double v, gx, gy;
    if (!bilin(c, lev, g, node_x(c, lev, g, i), node_y(c, lev, g, j), &v, &gx, &gy)) return 1;
    double gn = sqrt(gx * gx + gy * gy);
    return ph < -c->snap * c->lv[lev].h * gn;
}

static int classify_level(ctx_t *c, int lev)
{
    level_t *l = &c->lv[lev];
    int N = l->N;
    double ph;
    memset(l->prim, 0, (size_t)l->n);
    /* Algorithm LS: internal if phi < 0; walls and box ghosts by position */
    for (int j = -1; j <= N; j++)
        for (int i = 0; i <= N; i++) {
            int8_t *t = tref(l, G_U, i, j);
            if (j == -1 || j == N) *t = (i >= 1 && i <= N - 1) ? T_BOXGHOST : T_INACTIVE;
            else if (i == 0 || i == N) *t = T_WALL;
            else {
                if (!phi_node(c, lev, G_U, i, j, &ph)) { seterr(c, "phi missing"); return 0; }
                *t = node_internal(c, lev, G_U, i, j, ph) ? T_INTERNAL : T_EXT;
            }
        }
    for (int j = 0; j <= N; j++)
        for (int i = -1; i <= N; i++) {
            int8_t *t = tref(l, G_V, i, j);
            if (i == -1 || i == N) *t = (j >= 1 && j <= N - 1) ? T_BOXGHOST : T_INACTIVE;
            else if (j == 0 || j == N) *t = T_WALL;
            else {
                if (!phi_node(c, lev, G_V, i, j, &ph)) { seterr(c, "phi missing"); return 0; }
                *t = node_internal(c, lev, G_V, i, j, ph) ? T_INTERNAL : T_EXT;
            }
        }
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++) {
            if (!phi_node(c, lev, G_P, i, j, &ph)) { seterr(c, "phi missing"); return 0; }
            *tref(l, G_P, i, j) = node_internal(c, lev, G_P, i, j, ph) ? T_INTERNAL : T_EXT;
        }
    /* a pressure cell whose four faces are all non-internal has no box */
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++) {
            int8_t *t = tref(l, G_P, i, j);
            if (*t != T_INTERNAL) continue;
            if (ttype(l, G_U, i, j) != T_INTERNAL && ttype(l, G_U, i + 1, j) != T_INTERNAL &&
                ttype(l, G_V, i, j) != T_INTERNAL && ttype(l, G_V, i, j + 1) != T_INTERNAL)
                *t = T_EXT;
        }
    /* external nodes referenced by internal rows and box-ghost rows */
    int ch = 0;
    for (int j = 0; j < N; j++)
        for (int i = 1; i < N; i++)
            if (ttype(l, G_U, i, j) == T_INTERNAL) {
                if (!mark_needed(c, l, G_U, i + 1, j, &ch) || !mark_needed(c, l, G_U, i - 1, j, &ch) ||
                    !mark_needed(c, l, G_U, i, j + 1, &ch) || !mark_needed(c, l, G_U, i, j - 1, &ch) ||
                    !mark_needed(c, l, G_P, i, j, &ch) || !mark_needed(c, l, G_P, i - 1, j, &ch))
                    return 0;
            }
    for (int j = 1; j < N; j++)
        for (int i = 0; i < N; i++)
            if (ttype(l, G_V, i, j) == T_INTERNAL) {
                if (!mark_needed(c, l, G_V, i + 1, j, &ch) || !mark_needed(c, l, G_V, i - 1, j, &ch) ||
                    !mark_needed(c, l, G_V, i, j + 1, &ch) || !mark_needed(c, l, G_V, i, j - 1, &ch) ||
                    !mark_needed(c, l, G_P, i, j, &ch) || !mark_needed(c, l, G_P, i, j - 1, &ch))
                    return 0;
            }
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++)
            if (ttype(l, G_P, i, j) == T_INTERNAL) {
                if (!mark_needed(c, l, G_U, i, j, &ch) || !mark_needed(c, l, G_U, i + 1, j, &ch) ||
                    !mark_needed(c, l, G_V, i, j, &ch) || !mark_needed(c, l, G_V, i, j + 1, &ch))
                    return 0;
            }
    for (int i = 1; i < N; i++) {
        if (!mark_needed(c, l, G_U, i, 0, &ch) || !mark_needed(c, l, G_U, i, 1, &ch) ||
            !mark_needed(c, l, G_U, i, N - 1, &ch) || !mark_needed(c, l, G_U, i, N - 2, &ch))
            return 0;
    }
    for (int j = 1; j < N; j++) {
        if (!mark_needed(c, l, G_V, 0, j, &ch) || !mark_needed(c, l, G_V, 1, j, &ch) ||
            !mark_needed(c, l, G_V, N - 1, j, &ch) || !mark_needed(c, l, G_V, N - 2, j, &ch))
            return 0;
    }
    /* moving bodies (Sect. 3.4): on the finest grid every external node
     * within `band` index steps of an internal node of its grid is a ghost
     * too, so that values from the previous step exist where the fluid
     * advances; the closure radius grows to `band` there */
    if (c->band > 0 && lev == 0)
        for (int g = 0; g < 3; g++) {
            int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? N - 1 : N;
            int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? N - 1 : N;
            for (int j = jlo; j <= jhi; j++)
                for (int i = ilo; i <= ihi; i++) {
                    int8_t *t = tref(l, g, i, j);
                    if (*t != T_EXT) continue;
                    int near = 0;
                    for (int dj = -c->band; dj <= c->band && !near; dj++)
                        for (int di = -c->band; di <= c->band && !near; di++)
                            if (ttype(l, g, i + di, j + dj) == T_INTERNAL) near = 1;
                    if (near) *t = T_GHOST;
                }
        }
    /* close the ghost set under the ghost stencils (Remark 1, coupled ghosts) */
    for (int pass = 0;; pass++) {
        if (pass > 64) { seterr(c, "ghost marking does not close"); return 0; }
        ch = 0;
        for (int g = 0; g < 3; g++) {
            int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? N - 1 : N;
            int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? N - 1 : N;
            for (int j = jlo; j <= jhi; j++)
                for (int i = ilo; i <= ihi; i++) {
                    if (ttype(l, g, i, j) != T_GHOST) continue;
                    ghost_t G;
                    if (!ghost_setup(c, lev, g, i, j, &G)) { seterr(c, "boundary projection failed"); return 0; }
                    for (int k = 1; k < G.nst; k++)
                        if (!mark_stencil(c, l, g, G.si[k], G.sj[k], &ch)) return 0;
                }
        }
        if (!ch) break;
    }
    /* everything else external is inactive; collect ghosts in (grid, j, i) order */
    int ng = 0;
    for (int g = 0; g < 3; g++) {
        int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? N - 1 : N;
        int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? N - 1 : N;
        for (int j = jlo; j <= jhi; j++)
            for (int i = ilo; i <= ihi; i++) {
                int8_t *t = tref(l, g, i, j);
                if (*t == T_EXT) *t = T_INACTIVE;
                if (*t == T_GHOST) ng++;
            }
    }
    l->gh = (ghost_t *)calloc(ng > 0 ? ng : 1, sizeof(ghost_t));
    l->ngh = 0;
    for (int k = 0; k < l->n; k++) l->gid[k] = -1;
    for (int g = 0; g < 3; g++) {
        int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? N - 1 : N;
        int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? N - 1 : N;
        for (int j = jlo; j <= jhi; j++)
            for (int i = ilo; i <= ihi; i++) {
                if (ttype(l, g, i, j) != T_GHOST) continue;
                ghost_t *G = &l->gh[l->ngh];
                if (!ghost_setup(c, lev, g, i, j, G)) {
                    seterr(c, "boundary projection failed");
                    return 0;
                }
                l->gid[iG(l, g, i, j)] = l->ngh;
                l->ngh++;
            }
    }
    l->n_int = 0;
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++)
            if (ttype(l, G_P, i, j) == T_INTERNAL) l->n_int++;
    if (l->n_int == 0) { seterr(c, "no internal pressure cell"); return 0; }
    return 1;
}

/* ------------------------------------------------------------------ rows */

static void radd(row_t *R, int col, double a)
{
    R->col[R->n] = col;
    R->a[R->n] = a;
    R->n++;
}

/* Coefficients of the equation written at node (g, i, j) (Algorithm LS). */
static int get_row(ctx_t *c, int lev, int g, int i, int j, row_t *R)
{
    level_t *l = &c->lv[lev];
    int N = l->N;
    double h = l->h;
    double q = 1.0 / h, a = c->alpha / (h * h), d = 1.0 + 4.0 * a;
    int t = ttype(l, g, i, j);
    R->n = 0;
    switch (t) {
    case T_INTERNAL:
        if (g == G_U) { /* u - alpha lap u + dp/dx */
            radd(R, iU(l, i, j), d);
            radd(R, iU(l, i + 1, j), -a);
            radd(R, iU(l, i - 1, j), -a);
            radd(R, iU(l, i, j + 1), -a);
            radd(R, iU(l, i, j - 1), -a);
            radd(R, iP(l, i, j), q);
            radd(R, iP(l, i - 1, j), -q);
        } else if (g == G_V) {
            radd(R, iV(l, i, j), d);
            radd(R, iV(l, i + 1, j), -a);
            radd(R, iV(l, i - 1, j), -a);
            radd(R, iV(l, i, j + 1), -a);
            radd(R, iV(l, i, j - 1), -a);
            radd(R, iP(l, i, j), q);
            radd(R, iP(l, i, j - 1), -q);
        } else { /* div u - xi */
            radd(R, iU(l, i + 1, j), q);
            radd(R, iU(l, i, j), -q);
            radd(R, iV(l, i, j + 1), q);
            radd(R, iV(l, i, j), -q);
            radd(R, iXI(l), -1.0);
        }
        break;
    case T_GHOST: {
        ghost_t *G = &l->gh[l->gid[iG(l, g, i, j)]];
        for (int k = 0; k < G->nst; k++) radd(R, iG(l, g, G->si[k], G->sj[k]), G->w[k]);
        break;
    }
    case T_WALL:
        radd(R, iG(l, g, i, j), 1.0);
        break;
    case T_BOXGHOST:
        if (g == G_U) {
            int s = j == -1 ? 1 : -1;
            radd(R, iU(l, i, j), 3.0 / 8.0);
            radd(R, iU(l, i, j + s), 3.0 / 4.0);
            radd(R, iU(l, i, j + 2 * s), -1.0 / 8.0);
        } else {
            int s = i == -1 ? 1 : -1;
            radd(R, iV(l, i, j), 3.0 / 8.0);
            radd(R, iV(l, i + s, j), 3.0 / 4.0);
            radd(R, iV(l, i + 2 * s, j), -1.0 / 8.0);
        }
        break;
    default: /* inactive: x = b (b = 0) */
        radd(R, iG(l, g, i, j), 1.0);
        break;
    }
    (void)N;
    return t;
}

static double row_residual(const row_t *R, const double *x, double b)
{
    double s = b;
    for (int k = 0; k < R->n; k++) s -= R->a[k] * x[R->col[k]];
    return s;
}

/* ----------------------------------------------------------------- public */

/* threads of the OpenMP build (1 in the serial build); returns the count in use */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void *or_create(int N, double x0, double y0, double len, int levels, double alpha)
{
    if (N < 4 || levels < 1 || levels > OR_MAXLEV) return NULL;
    if (N % (1 << (levels - 1)) != 0) return NULL;
    ctx_t *c = (ctx_t *)calloc(1, sizeof(ctx_t));
    c->N = N;
    c->L = levels;
    c->x0 = x0;
    c->y0 = y0;
    c->len = len;
    c->alpha = alpha;
    c->nu1 = 2; c->nu2 = 1; c->gamma = 1; c->lam = 5;
    c->dtau = 0.9; c->ghost_mode = 0; c->order_mode = 0; c->rng = 12345u; c->snap = 0.3;
    for (int k = 0; k < levels; k++) {
        level_t *l = &c->lv[k];
        l->N = N >> k;
        l->h = len / (double)l->N;
        l->nU = (l->N + 1) * (l->N + 2);
        l->nV = (l->N + 2) * (l->N + 1);
        l->nP = l->N * l->N;
        l->n = l->nU + l->nV + l->nP + 1;
        l->tU = (int8_t *)calloc(l->nU, 1);
        l->tV = (int8_t *)calloc(l->nV, 1);
        l->tP = (int8_t *)calloc(l->nP, 1);
        l->gid = (int *)malloc(sizeof(int) * l->n);
        l->prim = (int8_t *)calloc(l->n, 1);
        l->x = (double *)calloc(l->n, sizeof(double));
        l->b = (double *)calloc(l->n, sizeof(double));
        l->r = (double *)calloc(l->n, sizeof(double));
    }
    size_t M = 2 * (size_t)N + 1;
    c->phi = (double *)calloc(M * M, sizeof(double));
    return c;
}

void or_destroy(void *vc)
{
    ctx_t *c = (ctx_t *)vc;
    if (!c) return;
    for (int k = 0; k < c->L; k++) free_level(&c->lv[k]);
    free(c->phi);
    free(c);
}

void or_set_params(void *vc, int nu1, int nu2, int gamma, int lam, double dtau, int ghost_mode, int order_mode, unsigned seed)
{
    ctx_t *c = (ctx_t *)vc;
    c->nu1 = nu1; c->nu2 = nu2; c->gamma = gamma; c->lam = lam;
    c->dtau = dtau; c->ghost_mode = ghost_mode; c->order_mode = order_mode; c->rng = seed ? seed : 1u;
}

void or_set_alpha(void *vc, double alpha) { ((ctx_t *)vc)->alpha = alpha; }

void or_set_snap(void *vc, double snap) { ((ctx_t *)vc)->snap = snap; }
void or_set_band(void *vc, int band) { ((ctx_t *)vc)->band = band; }

const char *or_last_error(void *vc) { return ((ctx_t *)vc)->err; }

int or_n(void *vc, int lev) { return ((ctx_t *)vc)->lv[lev].n; }
int or_n_int(void *vc, int lev) { return ((ctx_t *)vc)->lv[lev].n_int; }
int or_num_ghosts(void *vc, int lev) { return ((ctx_t *)vc)->lv[lev].ngh; }

static int factor_coarsest(ctx_t *c);

/* phi: (2N+1)^2 half lattice, row b (y) major, paper sign (phi > 0 in the object) */
static int cut_colouring(ctx_t *c, int lev);

int or_geometry(void *vc, const double *phi)
{
    ctx_t *c = (ctx_t *)vc;
    c->err[0] = 0;
    c->geom_ok = 0;
    c->adj_ok = 0;
    size_t M = 2 * (size_t)c->N + 1;
    memcpy(c->phi, phi, M * M * sizeof(double));
    for (int k = 0; k < c->L; k++) {
        level_t *l = &c->lv[k];
        free(l->gh); l->gh = NULL; l->ngh = 0;
        if (!classify_level(c, k)) return OR_GEOMETRY;
    }
    for (int k = 0; k < c->L; k++)
        if (!cut_colouring(c, k)) return OR_GEOMETRY;
    int st = factor_coarsest(c);
    if (st != OR_OK) return st;
    c->geom_ok = 1;
    return OR_OK;
}

/* types of every unknown of level lev in the flat layout (mean slot = -1) */
int or_types(void *vc, int lev, int8_t *out)
{
    level_t *l = &((ctx_t *)vc)->lv[lev];
    memcpy(out, l->tU, l->nU);
    memcpy(out + l->nU, l->tV, l->nV);
    memcpy(out + l->nU + l->nV, l->tP, l->nP);
    out[l->n - 1] = -1;
    return l->n;
}

/* ghost records: ints [grid, i, j, sx, sy, axis + 2 kind, nst] and doubles
 * [xB, yB, nx, ny, thx, thy, w0..w8]; stencil nodes [si0, sj0, ...] */
int or_ghosts(void *vc, int lev, int *iout, double *dout, int *sout, int cap)
{
    level_t *l = &((ctx_t *)vc)->lv[lev];
    int n = l->ngh < cap ? l->ngh : cap;
    for (int k = 0; k < n; k++) {
        ghost_t *G = &l->gh[k];
        int *ip = iout + 7 * k;
        ip[0] = G->grid; ip[1] = G->i; ip[2] = G->j; ip[3] = G->sx; ip[4] = G->sy; ip[5] = G->axis + 2 * G->kind; ip[6] = G->nst;
        double *dp = dout + 15 * k;
        dp[0] = G->xB; dp[1] = G->yB; dp[2] = G->nx; dp[3] = G->ny; dp[4] = G->thx; dp[5] = G->thy;
        for (int m = 0; m < 9; m++) dp[6 + m] = m < G->nst ? G->w[m] : 0.0;
        int *sp = sout + 18 * k;
        for (int m = 0; m < 9; m++) {
            sp[2 * m] = m < G->nst ? G->si[m] : 0;
            sp[2 * m + 1] = m < G->nst ? G->sj[m] : 0;
        }
    }
    return l->ngh;
}

/* Algorithm 1 on its own, for tests: B of node (g, i, j) of level lev */
int or_boundary_point(void *vc, int lev, int g, int i, int j, double *xy)
{
    ctx_t *c = (ctx_t *)vc;
    return ghost_to_boundary(c, lev, g, i, j, &xy[0], &xy[1]) ? OR_OK : OR_GEOMETRY;
}

/* full residual r = b - M x on level lev; returns ||r||_inf */
double or_residual(void *vc, int lev, const double *x, const double *b, double *r)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[lev];
    int N = l->N;
    double mx = 0.0;
    for (int g = 0; g < 3; g++) {
        int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? N - 1 : N;
        int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? N - 1 : N;
#pragma omp parallel for schedule(static)
        for (int j = jlo; j <= jhi; j++)
            for (int i = ilo; i <= ihi; i++) {
                row_t R;
                int k = iG(l, g, i, j);
                get_row(c, lev, g, i, j, &R);
                r[k] = row_residual(&R, x, b[k]);
            }
    }
    for (int k = 0; k < l->n - 1; k++) {
        double v = r[k];
        if (fabs(v) > mx || v != v) mx = v != v ? NAN : fabs(v);
    }
    /* mean row, Eq. (midpoint) scaled by h^2 */
    double s = 0.0;
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++)
            if (ttype(l, G_P, i, j) == T_INTERNAL) s += x[iP(l, i, j)];
    double v = b[iXI(l)] - l->h * l->h * s;
    r[iXI(l)] = v;
    if (fabs(v) > mx) mx = fabs(v);
    return mx;
}

/* assembled M_h in COO form (Eq. LS); returns nnz or -needed if cap too small */
int or_assemble(void *vc, int lev, int *ri, int *ci, double *val, int cap)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[lev];
    int N = l->N, nnz = 0;
    row_t R;
    for (int g = 0; g < 3; g++) {
        int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? N - 1 : N;
        int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? N - 1 : N;
        for (int j = jlo; j <= jhi; j++)
            for (int i = ilo; i <= ihi; i++) {
                int k = iG(l, g, i, j);
                get_row(c, lev, g, i, j, &R);
                for (int m = 0; m < R.n; m++) {
                    if (nnz < cap) { ri[nnz] = k; ci[nnz] = R.col[m]; val[nnz] = R.a[m]; }
                    nnz++;
                }
            }
    }
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++)
            if (ttype(l, G_P, i, j) == T_INTERNAL) {
                if (nnz < cap) { ri[nnz] = iXI(l); ci[nnz] = iP(l, i, j); val[nnz] = l->h * l->h; }
                nnz++;
            }
    return nnz <= cap ? nnz : -nnz;
}

/* ------------------------------------------------------- dense LU (pivoted) */

static int lu_factor(int n, double *A, int *piv)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double v = fabs(A[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (!(best > 0.0)) return 0;
        if (p != k)
            for (int jj = 0; jj < n; jj++) {
                double t = A[(size_t)k * n + jj];
                A[(size_t)k * n + jj] = A[(size_t)p * n + jj];
                A[(size_t)p * n + jj] = t;
            }
        double dkk = A[(size_t)k * n + k];
        for (int i = k + 1; i < n; i++) {
            double m = A[(size_t)i * n + k] / dkk;
            A[(size_t)i * n + k] = m;
            if (m != 0.0)
                for (int jj = k + 1; jj < n; jj++) A[(size_t)i * n + jj] -= m * A[(size_t)k * n + jj];
        }
    }
    return 1;
}

static void lu_solve(int n, const double *A, const int *piv, double *b)
{
    for (int k = 0; k < n; k++) {
        if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    }
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int jj = 0; jj < i; jj++) s -= A[(size_t)i * n + jj] * b[jj];
        b[i] = s;
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = b[i];
        for (int jj = i + 1; jj < n; jj++) s -= A[(size_t)i * n + jj] * b[jj];
        b[i] = s / A[(size_t)i * n + i];
    }
}

/* dense solve of A x = b in place (A overwritten), for tests */
int or_dense_solve(int n, double *A, double *b)
{
    int *piv = (int *)malloc(sizeof(int) * n);
    int ok = lu_factor(n, A, piv);
    if (ok) lu_solve(n, A, piv, b);
    free(piv);
    return ok ? OR_OK : OR_SINGULAR;
}

static int dense_matrix(ctx_t *c, int lev, double *A)
{
    level_t *l = &c->lv[lev];
    int n = l->n;
    int cap = 12 * n + l->nP + 16;
    int *ri = (int *)malloc(sizeof(int) * cap), *ci = (int *)malloc(sizeof(int) * cap);
    double *v = (double *)malloc(sizeof(double) * cap);
    int nnz = or_assemble(c, lev, ri, ci, v, cap);
    memset(A, 0, sizeof(double) * (size_t)n * n);
    for (int k = 0; k < nnz; k++) A[(size_t)ri[k] * n + ci[k]] += v[k];
    free(ri); free(ci); free(v);
    return nnz > 0;
}

static int factor_coarsest(ctx_t *c)
{
    level_t *l = &c->lv[c->L - 1];
    int n = l->n;
    free(l->lu); free(l->piv);
    l->lu = (double *)malloc(sizeof(double) * (size_t)n * n);
    l->piv = (int *)malloc(sizeof(int) * n);
    dense_matrix(c, c->L - 1, l->lu);
    if (!lu_factor(n, l->lu, l->piv)) { seterr(c, "coarsest matrix is singular"); return OR_SINGULAR; }
    return OR_OK;
}

/* dense matrix of level lev (row-major n x n), for tests */
int or_dense_matrix(void *vc, int lev, double *A) { return dense_matrix((ctx_t *)vc, lev, A) ? OR_OK : OR_INVALID; }

/* exact solve on the coarsest level: x = M^-1 b */
int or_coarse_solve(void *vc, const double *b, double *x)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[c->L - 1];
    memcpy(x, b, sizeof(double) * l->n);
    lu_solve(l->n, l->lu, l->piv, x);
    return OR_OK;
}

/* ------------------------------------------------------------- smoothers */

static unsigned rng_next(ctx_t *c)
{
    c->rng = c->rng * 1664525u + 1013904223u;
    return c->rng >> 8;
}

/* Box relaxation of the cell (i, j) (Sect. 4.1.1): the unknowns are p_ij and
 * the variables on the cell borders; the rows of those unknowns are solved
 * together with everything else frozen.  A border variable takes part when it
 * is internal (momentum row) or a ghost of the object (its ghost row); wall
 * and box-ghost borders stay frozen. */
static void box_relax(ctx_t *c, int lev, double *x, const double *b, int i, int j)
{
    level_t *l = &c->lv[lev];
    int gg[5], ii[5], jj[5], unk[5], nu = 0;
    const int fg[4] = {G_U, G_U, G_V, G_V};
    const int fi[4] = {i, i + 1, i, i};
    const int fj[4] = {j, j, j, j + 1};
    for (int f = 0; f < 4; f++) {
        int t = ttype(l, fg[f], fi[f], fj[f]);
        if (t == T_INTERNAL || t == T_GHOST) {
            gg[nu] = fg[f]; ii[nu] = fi[f]; jj[nu] = fj[f];
            unk[nu] = iG(l, fg[f], fi[f], fj[f]);
            nu++;
        }
    }
    gg[nu] = G_P; ii[nu] = i; jj[nu] = j; unk[nu] = iP(l, i, j); nu++;
    double A[25], rhs[5];
    int piv[5];
    for (int r = 0; r < nu; r++) {
        row_t R;
        get_row(c, lev, gg[r], ii[r], jj[r], &R);
        rhs[r] = row_residual(&R, x, b[unk[r]]);
        for (int cc = 0; cc < nu; cc++) {
            double sum = 0.0;
            for (int k = 0; k < R.n; k++)
                if (R.col[k] == unk[cc]) sum += R.a[k];
            A[r * nu + cc] = sum;
        }
    }
    if (!lu_factor(nu, A, piv)) return;
    lu_solve(nu, A, piv, rhs);
    for (int r = 0; r < nu; r++) x[unk[r]] += rhs[r];
}

static int cut_cell(level_t *l, int i, int j)
{
    return ttype(l, G_U, i, j) == T_GHOST || ttype(l, G_U, i + 1, j) == T_GHOST ||
           ttype(l, G_V, i, j) == T_GHOST || ttype(l, G_V, i, j + 1) == T_GHOST;
}

/* The unknowns of the box of cell (i, j): its faces that are internal or
 * ghosts of the object, then p (as box_relax). */
static int box_unknowns(level_t *l, int i, int j, int *gg, int *ii, int *jj, int *unk)
{
    const int fg[4] = {G_U, G_U, G_V, G_V};
    const int fi[4] = {i, i + 1, i, i};
    const int fj[4] = {j, j, j, j + 1};
    int nu = 0;
    for (int f = 0; f < 4; f++) {
        int t = ttype(l, fg[f], fi[f], fj[f]);
        if (t == T_INTERNAL || t == T_GHOST) {
            gg[nu] = fg[f]; ii[nu] = fi[f]; jj[nu] = fj[f];
            unk[nu] = iG(l, fg[f], fi[f], fj[f]);
            nu++;
        }
    }
    gg[nu] = G_P; ii[nu] = i; jj[nu] = j; unk[nu] = iP(l, i, j);
    return nu + 1;
}

#define OR_MAXCUTCOL 64

/* Colours of the cut cells: two cut boxes conflict when a row of one
 * references an unknown of the other (their updates then depend on the order);
 * cells are coloured in lexicographic order (j, then i), each with the
 * smallest colour that no conflicting cell coloured before it has.  Boxes of
 * one colour are then independent. */
static int cut_colouring(ctx_t *c, int lev)
{
    level_t *l = &c->lv[lev];
    int N = l->N, n = l->n;
    free(l->cutcol);
    l->cutcol = (int *)malloc(sizeof(int) * (size_t)N * N);
    for (int k = 0; k < N * N; k++) l->cutcol[k] = -1;
    int *cells = (int *)malloc(sizeof(int) * (size_t)N * N), nc = 0;
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++)
            if (ttype(l, G_P, i, j) == T_INTERNAL && cut_cell(l, i, j)) cells[nc++] = j * N + i;
    /* owners of every unknown (a face belongs to at most two boxes) */
    int *own = (int *)malloc(sizeof(int) * 2 * (size_t)n);
    for (int k = 0; k < 2 * n; k++) own[k] = -1;
    int gg[5], ii[5], jj[5], unk[5];
    for (int a = 0; a < nc; a++) {
        int nu = box_unknowns(l, cells[a] % N, cells[a] / N, gg, ii, jj, unk);
        for (int q = 0; q < nu; q++) {
            int *o = own + 2 * (size_t)unk[q];
            if (o[0] < 0) o[0] = a;
            else o[1] = a;
        }
    }
    /* conflict lists: for every referenced column, its owners */
    int cap = 64, *nb = (int *)malloc(sizeof(int) * (size_t)nc * cap), *nnb = (int *)calloc(nc, sizeof(int));
    int ok = 1;
    for (int a = 0; a < nc && ok; a++) {
        int nu = box_unknowns(l, cells[a] % N, cells[a] / N, gg, ii, jj, unk);
        for (int q = 0; q < nu && ok; q++) {
            row_t R;
            get_row(c, lev, gg[q], ii[q], jj[q], &R);
            for (int e = 0; e < R.n && ok; e++) {
                if (R.col[e] >= n - 1) continue; /* xi: no box owns it */
                for (int w = 0; w < 2; w++) {
                    int bcell = own[2 * (size_t)R.col[e] + w];
                    if (bcell < 0 || bcell == a) continue;
                    /* add the edge both ways (once) */
                    int pairs[2][2] = {{a, bcell}, {bcell, a}};
                    for (int z = 0; z < 2; z++) {
                        int x0 = pairs[z][0], y0 = pairs[z][1], dup = 0;
                        for (int t = 0; t < nnb[x0]; t++)
                            if (nb[(size_t)x0 * cap + t] == y0) { dup = 1; break; }
                        if (dup) continue;
                        if (nnb[x0] >= cap) { ok = 0; break; }
                        nb[(size_t)x0 * cap + nnb[x0]++] = y0;
                    }
                }
            }
        }
    }
    int ncol = 0;
    int *col = (int *)malloc(sizeof(int) * (nc > 0 ? nc : 1));
    for (int a = 0; a < nc && ok; a++) {
        unsigned long long used = 0ull;
        for (int t = 0; t < nnb[a]; t++) {
            int bcell = nb[(size_t)a * cap + t];
            if (bcell < a) used |= 1ull << col[bcell];
        }
        int cc = 0;
        while (cc < OR_MAXCUTCOL && (used >> cc & 1ull)) cc++;
        if (cc >= OR_MAXCUTCOL) { ok = 0; break; }
        col[a] = cc;
        if (cc + 1 > ncol) ncol = cc + 1;
        l->cutcol[cells[a]] = cc;
    }
    l->ncutcol = ncol;
    free(cells); free(own); free(nb); free(nnb); free(col);
    if (!ok) seterr(c, "cut-cell colouring exceeded its limits");
    return ok;
}

static void shuffle(ctx_t *c, int *v, int n)
{
    for (int k = n - 1; k > 0; k--) {
        int m = (int)(rng_next(c) % (unsigned)(k + 1));
        int t = v[k]; v[k] = v[m]; v[m] = t;
    }
}

/* One box sweep over the internal cells: cells with no ghost border in five
 * colours (i + 3 j) mod 5, then cells with a ghost border (their boxes reach
 * further through the ghost rows) in the colours of cut_colouring; boxes of
 * one colour never touch each other's unknowns.  Then a point-Jacobi update
 * of internal faces that belong to no internal cell. */
void or_box_sweep(void *vc, int lev, double *x, const double *b)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[lev];
    int N = l->N;
    int *cells = (int *)malloc(sizeof(int) * (size_t)N * N);
    if (c->order_mode == 2) { /* lexicographic Gauss-Seidel (ablation) */
        for (int j = 0; j < N; j++)
            for (int i = 0; i < N; i++)
                if (ttype(l, G_P, i, j) == T_INTERNAL) box_relax(c, lev, x, b, i, j);
    } else {
        for (int col = 0; col < 5; col++) {
            int nc = 0;
            for (int j = 0; j < N; j++)
                for (int i = 0; i < N; i++)
                    if ((i + 3 * j) % 5 == col && ttype(l, G_P, i, j) == T_INTERNAL && !cut_cell(l, i, j))
                        cells[nc++] = j * N + i;
            if (c->order_mode == 1) shuffle(c, cells, nc); /* random order inside a colour */
            /* boxes of one colour are independent: any order, or several
             * threads, give the same iterate */
#pragma omp parallel for schedule(static)
            for (int k = 0; k < nc; k++) box_relax(c, lev, x, b, cells[k] % N, cells[k] / N);
        }
        for (int col = 0; col < l->ncutcol; col++) {
            int nc = 0;
            for (int j = 0; j < N; j++)
                for (int i = 0; i < N; i++)
                    if (l->cutcol[j * N + i] == col) cells[nc++] = j * N + i;
            if (c->order_mode == 1) shuffle(c, cells, nc);
#pragma omp parallel for schedule(static)
            for (int k = 0; k < nc; k++) box_relax(c, lev, x, b, cells[k] % N, cells[k] / N);
        }
    }
    free(cells);
    /* internal faces with no internal cell on either side */
    int cnt = 0;
    int *idx = (int *)malloc(sizeof(int) * (l->nU + l->nV));
    double *upd = (double *)malloc(sizeof(double) * (l->nU + l->nV));
    row_t R;
    for (int j = 0; j < N; j++)
        for (int i = 1; i < N; i++)
            if (ttype(l, G_U, i, j) == T_INTERNAL && ttype(l, G_P, i - 1, j) != T_INTERNAL &&
                ttype(l, G_P, i, j) != T_INTERNAL) {
                get_row(c, lev, G_U, i, j, &R);
                idx[cnt] = iU(l, i, j);
                upd[cnt++] = row_residual(&R, x, b[iU(l, i, j)]) / R.a[0];
            }
    for (int j = 1; j < N; j++)
        for (int i = 0; i < N; i++)
            if (ttype(l, G_V, i, j) == T_INTERNAL && ttype(l, G_P, i, j - 1) != T_INTERNAL &&
                ttype(l, G_P, i, j) != T_INTERNAL) {
                get_row(c, lev, G_V, i, j, &R);
                idx[cnt] = iV(l, i, j);
                upd[cnt++] = row_residual(&R, x, b[iV(l, i, j)]) / R.a[0];
            }
    for (int k = 0; k < cnt; k++) x[idx[k]] += upd[k];
    free(idx);
    free(upd);
}

/* relaxation of the (xi, mean) pair: xi from the continuity rows, then a
 * uniform pressure shift that satisfies the mean row exactly */
void or_scalar_update(void *vc, int lev, double *x, const double *b)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[lev];
    int N = l->N;
    double h = l->h, s = 0.0, m = 0.0;
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++)
            if (ttype(l, G_P, i, j) == T_INTERNAL) {
                double div = (x[iU(l, i + 1, j)] - x[iU(l, i, j)] + x[iV(l, i, j + 1)] - x[iV(l, i, j)]) / h;
                s += div - b[iP(l, i, j)];
                m += x[iP(l, i, j)];
            }
    x[iXI(l)] = s / (double)l->n_int;
    double shift = (b[iXI(l)] - h * h * m) / (h * h * (double)l->n_int);
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++) {
            int t = ttype(l, G_P, i, j);
            if (t == T_INTERNAL || t == T_GHOST) x[iP(l, i, j)] += shift;
        }
}

static int ghost_class(int t) { return t == T_GHOST || t == T_WALL || t == T_BOXGHOST; }

/* One Jacobi sweep of Eq. (ghostrelax) over every ghost, wall and box-ghost row */
void or_ghost_sweep(void *vc, int lev, double *x, const double *b)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[lev];
    int N = l->N;
    int *idx = (int *)malloc(sizeof(int) * l->n);
    double *upd = (double *)malloc(sizeof(double) * l->n);
    int cnt = 0;
    row_t R;
    for (int g = 0; g < 3; g++) {
        int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? N - 1 : N;
        int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? N - 1 : N;
        for (int j = jlo; j <= jhi; j++)
            for (int i = ilo; i <= ihi; i++) {
                if (!ghost_class(ttype(l, g, i, j))) continue;
                int k = iG(l, g, i, j);
                get_row(c, lev, g, i, j, &R);
                double res = row_residual(&R, x, b[k]);
                double cg = R.a[0]; /* the first entry is the node itself */
                idx[cnt] = k;
                upd[cnt++] = c->ghost_mode == 1 ? c->dtau * res / cg : c->dtau * res;
            }
    }
    for (int k = 0; k < cnt; k++) x[idx[k]] += upd[k];
    free(idx);
    free(upd);
}

/* Algorithm relax: nu x {box sweep; (xi, mean) update; lambda ghost sweeps} */
void or_smooth(void *vc, int lev, double *x, const double *b, int nu)
{
    ctx_t *c = (ctx_t *)vc;
    for (int s = 0; s < nu; s++) {
        or_box_sweep(c, lev, x, b);
        or_scalar_update(c, lev, x, b);
        for (int k = 0; k < c->lam; k++) or_ghost_sweep(c, lev, x, b);
    }
}

/* ------------------------------------------------------------- transfers */

static int same_class(int tc, int tf)
{
    if (tc == T_INTERNAL) return tf == T_INTERNAL;
    return ghost_class(tf);
}

/* restriction of the fine residual r (level lev) to the rhs bH of lev+1,
 * Eq. (restop) where every stencil point is of the coarse point's class,
 * otherwise the plain mean over the points of that class, Eq. (restop5). */
void or_restrict(void *vc, int lev, const double *r, double *bH)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *f = &c->lv[lev], *C = &c->lv[lev + 1];
    int Nc = C->N;
    for (int g = 0; g < 3; g++) {
        int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? Nc - 1 : Nc;
        int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? Nc - 1 : Nc;
#pragma omp parallel for schedule(static)
        for (int J = jlo; J <= jhi; J++)
            for (int I = ilo; I <= ihi; I++) {
                int tc = ttype(C, g, I, J);
                int kc = iG(C, g, I, J);
                if (tc == T_INACTIVE) { bH[kc] = 0.0; continue; }
                int fi[6], fj[6], ns = 0;
                double wt[6];
                if (g == G_U) {
                    for (int dj = 0; dj <= 1; dj++)
                        for (int di = -1; di <= 1; di++) {
                            fi[ns] = 2 * I + di; fj[ns] = 2 * J + dj; wt[ns] = (di == 0 ? 2.0 : 1.0) / 8.0; ns++;
                        }
                } else if (g == G_V) {
                    for (int dj = -1; dj <= 1; dj++)
                        for (int di = 0; di <= 1; di++) {
                            fi[ns] = 2 * I + di; fj[ns] = 2 * J + dj; wt[ns] = (dj == 0 ? 2.0 : 1.0) / 8.0; ns++;
                        }
                } else {
                    for (int dj = 0; dj <= 1; dj++)
                        for (int di = 0; di <= 1; di++) {
                            fi[ns] = 2 * I + di; fj[ns] = 2 * J + dj; wt[ns] = 0.25; ns++;
                        }
                }
                int all = 1, cnt = 0;
                double sw = 0.0, su = 0.0;
                for (int k = 0; k < ns; k++) {
                    int tf = ttype(f, g, fi[k], fj[k]);
                    if (same_class(tc, tf)) {
                        double v = r[iG(f, g, fi[k], fj[k])];
                        sw += wt[k] * v;
                        su += v;
                        cnt++;
                    } else all = 0;
                }
                bH[kc] = all ? sw : (cnt > 0 ? su / (double)cnt : 0.0);
            }
    }
    bH[iXI(C)] = r[iXI(f)];
}

/* 1-D interpolation taps for fine index k on a coarse line with valid
 * indices [lo, hi].  aligned != 0: fine nodes sit on coarse nodes or halfway
 * between two; otherwise (staggered direction) fine node k sits a quarter of
 * a coarse cell from its nearest coarse node Kc and three quarters from the
 * next one Ko.  Where Ko does not exist, linear extrapolation from Kc and the
 * node on its other side. */
static int taps(int k, int aligned, int lo, int hi, int *K, double *w)
{
    int even = (k % 2 == 0);
    if (aligned) {
        if (even) { K[0] = k / 2; w[0] = 1.0; return 1; }
        K[0] = (k - 1) / 2; w[0] = 0.5;
        K[1] = K[0] + 1; w[1] = 0.5;
        return 2;
    }
    int Kc = even ? k / 2 : (k - 1) / 2;
    int Ko = even ? Kc - 1 : Kc + 1;
    if (Ko < lo || Ko > hi) {
        K[0] = Kc; w[0] = 1.25;
        K[1] = 2 * Kc - Ko; w[1] = -0.25;
        return 2;
    }
    K[0] = Kc; w[0] = 0.75;
    K[1] = Ko; w[1] = 0.25;
    return 2;
}

/* bilinear interpolation of the coarse correction eH (level lev+1) added to
 * every active node of the fine iterate x (level lev), Sect. 4.3.  Inactive
 * coarse nodes carry no value: the weights of the active ones are
 * renormalised to sum to one. */
void or_prolong(void *vc, int lev, const double *eH, double *x)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *f = &c->lv[lev], *C = &c->lv[lev + 1];
    int N = f->N, Nc = C->N;
    for (int g = 0; g < 3; g++) {
        int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? N - 1 : N;
        int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? N - 1 : N;
        int Ilo = g == G_V ? -1 : 0, Ihi = g == G_P ? Nc - 1 : Nc;
        int Jlo = g == G_U ? -1 : 0, Jhi = g == G_P ? Nc - 1 : Nc;
#pragma omp parallel for schedule(static)
        for (int j = jlo; j <= jhi; j++)
            for (int i = ilo; i <= ihi; i++) {
                if (ttype(f, g, i, j) == T_INACTIVE) continue;
                int KI[2], KJ[2];
                double wi[2], wj[2];
                int ni = taps(i, g == G_U, Ilo, Ihi, KI, wi);
                int nj = taps(j, g == G_V, Jlo, Jhi, KJ, wj);
                double s = 0.0, ws = 0.0;
                for (int a = 0; a < nj; a++)
                    for (int bb = 0; bb < ni; bb++) {
                        if (ttype(C, g, KI[bb], KJ[a]) == T_INACTIVE) continue;
                        double w = wj[a] * wi[bb];
                        s += w * eH[iG(C, g, KI[bb], KJ[a])];
                        ws += w;
                    }
                if (ws > 0.0) x[iG(f, g, i, j)] += s / ws;
            }
    }
    x[iXI(f)] += eH[iXI(C)];
}

/* -------------------------------------------------------------- the cycle */

static void zero_inactive(ctx_t *c, int lev, double *x)
{
    level_t *l = &c->lv[lev];
    for (int k = 0; k < l->nU; k++) if (l->tU[k] == T_INACTIVE) x[k] = 0.0;
    for (int k = 0; k < l->nV; k++) if (l->tV[k] == T_INACTIVE) x[l->nU + k] = 0.0;
    for (int k = 0; k < l->nP; k++) if (l->tP[k] == T_INACTIVE) x[l->nU + l->nV + k] = 0.0;
}

static void cycle_rec(ctx_t *c, int lev, double *x, const double *b)
{
    if (lev == c->L - 1) {
        or_coarse_solve(c, b, x);
        return;
    }
    level_t *l = &c->lv[lev], *C = &c->lv[lev + 1];
    or_smooth(c, lev, x, b, c->nu1);
    or_residual(c, lev, x, b, l->r);
    or_restrict(c, lev, l->r, C->b);
    memset(C->x, 0, sizeof(double) * C->n);
    for (int k = 0; k < c->gamma; k++) cycle_rec(c, lev + 1, C->x, C->b);
    or_prolong(c, lev, C->x, x);
    or_smooth(c, lev, x, b, c->nu2);
}

/* one V (gamma = 1) or W (gamma = 2) cycle on level lev */
int or_cycle(void *vc, int lev, double *x, const double *b)
{
    ctx_t *c = (ctx_t *)vc;
    if (!c->geom_ok) return OR_INVALID;
    cycle_rec(c, lev, x, b);
    return OR_OK;
}

/* cycles from x until ||b - M x||_inf <= tol; hist[0..ncyc] residual norms */
int or_solve(void *vc, double *x, const double *b, double tol, int max_cycles, double *hist, int *ncyc)
{
    ctx_t *c = (ctx_t *)vc;
    if (!c->geom_ok) return OR_INVALID;
    level_t *l = &c->lv[0];
    zero_inactive(c, 0, x);
    double r0 = or_residual(c, 0, x, b, l->r);
    hist[0] = r0;
    *ncyc = 0;
    if (r0 <= tol) return OR_OK;
    for (int k = 1; k <= max_cycles; k++) {
        cycle_rec(c, 0, x, b);
        double rn = or_residual(c, 0, x, b, l->r);
        hist[k] = rn;
        *ncyc = k;
        if (!(rn == rn) || rn > 1e6 * r0) return OR_DIVERGED;
        if (rn <= tol) return OR_OK;
    }
    return OR_NOT_CONVERGED;
}

/* ------------------------------------------------------ Crank-Nicolson step */

/* Convective term N = u . grad u at every internal u and v node of level 0
 * (Sect. 2; central differences, the cross velocity averaged over the four
 * nearest nodes of the other grid).  out is a flat vector, zero elsewhere. */
void or_convective(void *vc, const double *x, double *out)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[0];
    int N = l->N;
    double h = l->h;
    memset(out, 0, sizeof(double) * l->n);
    for (int j = 0; j < N; j++)
        for (int i = 1; i < N; i++) {
            if (ttype(l, G_U, i, j) != T_INTERNAL) continue;
            double u = x[iU(l, i, j)];
            double vb = 0.25 * (x[iV(l, i - 1, j)] + x[iV(l, i, j)] + x[iV(l, i - 1, j + 1)] + x[iV(l, i, j + 1)]);
            double dudx = (x[iU(l, i + 1, j)] - x[iU(l, i - 1, j)]) / (2.0 * h);
            double dudy = (x[iU(l, i, j + 1)] - x[iU(l, i, j - 1)]) / (2.0 * h);
            out[iU(l, i, j)] = u * dudx + vb * dudy;
        }
    for (int j = 1; j < N; j++)
        for (int i = 0; i < N; i++) {
            if (ttype(l, G_V, i, j) != T_INTERNAL) continue;
            double v = x[iV(l, i, j)];
            double ub = 0.25 * (x[iU(l, i, j - 1)] + x[iU(l, i + 1, j - 1)] + x[iU(l, i, j)] + x[iU(l, i + 1, j)]);
            double dvdx = (x[iV(l, i + 1, j)] - x[iV(l, i - 1, j)]) / (2.0 * h);
            double dvdy = (x[iV(l, i, j + 1)] - x[iV(l, i, j - 1)]) / (2.0 * h);
            out[iV(l, i, j)] = ub * dvdx + v * dvdy;
        }
}

/* Continuity source of a manufactured solution (Sect. 5.1): the continuity
 * equation reads div u - xi = g with g the divergence of the exact velocity.
 * g is a flat vector (p block read; NULL for g = 0) kept by reference. */
void or_set_continuity_source(void *vc, const double *g) { ((ctx_t *)vc)->csrc = g; }

/* Right-hand side of the CN system (Eq. NSCN1 with the convective term moved
 * to the right, Eq. spaceprob): at internal u, v nodes
 *     b = u^n + alpha lap u^n + dt f - dt Nh,
 * continuity rows g (0 unless a source is set), ghost rows (Eq. BCu) the
 * rigid-body velocity at B,
 * wall and box-ghost rows the wall velocities, extrapolation rows and the
 * mean row 0.  Boundary values: from the flat vector bc at the ghost-class
 * rows when bc is given; otherwise body = {U, V, omega, cx, cy}:
 * u_b(B) = (U - omega (B_y - cy), V + omega (B_x - cx)) and walls = {u on
 * y = y0, u on y = y0 + L, v on x = x0, v on x = x0 + L} (tangential
 * velocities; normal velocities 0).
 * f: flat vector with the forcing at internal u, v nodes (NULL for none). */
void or_cn_rhs(void *vc, const double *xn, const double *Nh, const double *f, double dt, const double *bc,
               const double *body, const double *walls, double *b)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[0];
    int N = l->N;
    double h = l->h, a = c->alpha / (h * h);
    memset(b, 0, sizeof(double) * l->n);
    for (int j = 0; j < N; j++)
        for (int i = 1; i < N; i++) {
            if (ttype(l, G_U, i, j) != T_INTERNAL) continue;
            int k = iU(l, i, j);
            double lap = xn[iU(l, i + 1, j)] + xn[iU(l, i - 1, j)] + xn[iU(l, i, j + 1)] + xn[iU(l, i, j - 1)] - 4.0 * xn[k];
            b[k] = xn[k] + a * lap + dt * (f ? f[k] : 0.0) - dt * Nh[k];
        }
    for (int j = 1; j < N; j++)
        for (int i = 0; i < N; i++) {
            if (ttype(l, G_V, i, j) != T_INTERNAL) continue;
            int k = iV(l, i, j);
            double lap = xn[iV(l, i + 1, j)] + xn[iV(l, i - 1, j)] + xn[iV(l, i, j + 1)] + xn[iV(l, i, j - 1)] - 4.0 * xn[k];
            b[k] = xn[k] + a * lap + dt * (f ? f[k] : 0.0) - dt * Nh[k];
        }
    if (c->csrc)
        for (int j = 0; j < N; j++)
            for (int i = 0; i < N; i++)
                if (ttype(l, G_P, i, j) == T_INTERNAL) b[iP(l, i, j)] = c->csrc[iP(l, i, j)];
    for (int k = 0; k < l->ngh; k++) {
        ghost_t *G = &l->gh[k];
        if (G->kind != 0) continue;
        int kk = iG(l, G->grid, G->i, G->j);
        double ub = body[0] - body[2] * (G->yB - body[4]);
        double vb = body[1] + body[2] * (G->xB - body[3]);
        b[kk] = bc ? bc[kk] : (G->grid == G_U ? ub : vb);
    }
    for (int i = 1; i < N; i++) {
        b[iU(l, i, -1)] = bc ? bc[iU(l, i, -1)] : walls[0];
        b[iU(l, i, N)] = bc ? bc[iU(l, i, N)] : walls[1];
    }
    for (int j = 1; j < N; j++) {
        b[iV(l, -1, j)] = bc ? bc[iV(l, -1, j)] : walls[2];
        b[iV(l, N, j)] = bc ? bc[iV(l, N, j)] : walls[3];
    }
    if (bc) { /* wall-normal velocities on the walls */
        for (int j = 0; j < N; j++) {
            b[iU(l, 0, j)] = bc[iU(l, 0, j)];
            b[iU(l, N, j)] = bc[iU(l, N, j)];
        }
        for (int i = 0; i < N; i++) {
            b[iV(l, i, 0)] = bc[iV(l, i, 0)];
            b[iV(l, i, N)] = bc[iV(l, i, N)];
        }
    }
}

/* max |b - M x| over internal momentum rows (Eq. iterativeNS) and max |b| there */
void or_momentum_residual(void *vc, const double *x, const double *b, double *res, double *bmax)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[0];
    int N = l->N;
    row_t R;
    double m = 0.0, mb = 0.0;
    for (int g = 0; g < 2; g++) {
        int ilo = g == G_V ? -1 : 0, jlo = g == G_U ? -1 : 0;
        for (int j = jlo; j <= N; j++)
            for (int i = ilo; i <= N; i++) {
                if (ttype(l, g, i, j) != T_INTERNAL) continue;
                int k = iG(l, g, i, j);
                get_row(c, 0, g, i, j, &R);
                double v = fabs(row_residual(&R, x, b[k]));
                if (v > m) m = v;
                if (fabs(b[k]) > mb) mb = fabs(b[k]);
            }
    }
    *res = m;
    *bmax = mb;
}

/* One CN step (Sect. 2) from the state x (u^n, v^n, p, xi on level 0) with the
 * convective history N1 = N^{n-1}, N2 = N^{n-2} (flat vectors).  step is n.
 * n < 2: mid-point Picard iteration (Eq. NSitconv) until Eq. (iterativeNS)
 * holds with eps (at most kmax iterations); n >= 2: extrapolation
 * (Eq. extrUdU).  Each linear solve runs the multigrid to tol from the
 * previous iterate.  On return x holds the new state, N1/N2 are rotated.
 * info = {picard iterations, total cycles, last residual}. */
int or_cn_step(void *vc, double *x, double *N1, double *N2, int step, const double *f, const double *bc, double dt,
               const double *body, const double *walls, double tol, double eps, int kmax, double *info)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[0];
    int n = l->n, st = OR_OK, cycles = 0, it = 0;
    double *Nn = (double *)malloc(sizeof(double) * n), *Nh = (double *)malloc(sizeof(double) * n);
    double *Nk = (double *)malloc(sizeof(double) * n), *b = (double *)malloc(sizeof(double) * n);
    double *xn = (double *)malloc(sizeof(double) * n), *hist = (double *)malloc(sizeof(double) * 1024);
    memcpy(xn, x, sizeof(double) * n);
    or_convective(c, xn, Nn);
    double res = 0.0;
    if (step >= 2) {
        for (int k = 0; k < n; k++) Nh[k] = Nn[k] + 0.5 * N1[k] - 0.5 * N2[k];
        or_cn_rhs(c, xn, Nh, f, dt, bc, body, walls, b);
        int nc = 0;
        st = or_solve(c, x, b, tol, 1000, hist, &nc);
        cycles += nc;
        res = hist[nc];
    } else {
        /* ||f~|| of Eq. (iterativeNS): f~ = u^n + alpha lap u^n + dt f */
        double fmax, dummy;
        memset(Nk, 0, sizeof(double) * n);
        or_cn_rhs(c, xn, Nk, f, dt, bc, body, walls, b);
        or_momentum_residual(c, xn, b, &dummy, &fmax);
        memcpy(Nh, Nn, sizeof(double) * n); /* u^{n+1,0} = u^n */
        for (it = 1; it <= kmax; it++) {
            or_cn_rhs(c, xn, Nh, f, dt, bc, body, walls, b);
            int nc = 0;
            st = or_solve(c, x, b, tol, 1000, hist, &nc);
            cycles += nc;
            res = hist[nc];
            if (st != OR_OK) break;
            or_convective(c, x, Nk);
            for (int k = 0; k < n; k++) Nh[k] = 0.5 * (Nn[k] + Nk[k]);
            or_cn_rhs(c, xn, Nh, f, dt, bc, body, walls, b);
            double rm, bm;
            or_momentum_residual(c, x, b, &rm, &bm);
            double lim = eps * (fmax > 1.0 ? fmax : 1.0);
            if (rm < lim) break;
        }
        if (it > kmax) it = kmax;
    }
    memcpy(N2, N1, sizeof(double) * n);
    memcpy(N1, Nn, sizeof(double) * n);
    info[0] = it;
    info[1] = cycles;
    info[2] = res;
    free(Nn); free(Nh); free(Nk); free(b); free(xn); free(hist);
    return st;
}

/* ------------------------------------------------- Krylov acceleration */

static double dotv(const double *a, const double *b, int n)
{
    double s = 0.0;
    for (int k = 0; k < n; k++) s += a[k] * b[k];
    return s;
}

/* y = M x on the finest level (the residual of x against b = 0, negated) */
static void apply_M(ctx_t *c, const double *x, double *y, double *zero)
{
    level_t *l = &c->lv[0];
    or_residual(c, 0, x, zero, y);
    for (int k = 0; k < l->n; k++) y[k] = -y[k];
}

/* BiCGSTAB on M x = b, preconditioned on the right by one multigrid cycle
 * from zero (the same cycle as or_solve).  Stops when ||b - M x||_inf <= tol
 * (the true residual, computed every iteration); hist[k] is that norm after
 * iteration k. */
int or_solve_krylov(void *vc, double *x, const double *b, double tol, int maxit, double *hist, int *nit)
{
    ctx_t *c = (ctx_t *)vc;
    if (!c->geom_ok) return OR_INVALID;
    level_t *l = &c->lv[0];
    int n = l->n;
    double *r = calloc(n, sizeof(double)), *rh = calloc(n, sizeof(double)), *p = calloc(n, sizeof(double));
    double *v = calloc(n, sizeof(double)), *s = calloc(n, sizeof(double)), *t = calloc(n, sizeof(double));
    double *y = calloc(n, sizeof(double)), *z = calloc(n, sizeof(double)), *zero = calloc(n, sizeof(double));
    zero_inactive(c, 0, x);
    double r0 = or_residual(c, 0, x, b, r);
    memcpy(rh, r, sizeof(double) * n);
    hist[0] = r0;
    *nit = 0;
    int st = OR_NOT_CONVERGED;
    if (r0 <= tol) st = OR_OK;
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    for (int it = 1; st == OR_NOT_CONVERGED && it <= maxit; it++) {
        double rn = dotv(rh, r, n);
        double beta = (rn / rho) * (alpha / omega);
        rho = rn;
        for (int k = 0; k < n; k++) p[k] = r[k] + beta * (p[k] - omega * v[k]);
        memset(y, 0, sizeof(double) * n);
        cycle_rec(c, 0, y, p);
        apply_M(c, y, v, zero);
        alpha = rho / dotv(rh, v, n);
        for (int k = 0; k < n; k++) s[k] = r[k] - alpha * v[k];
        memset(z, 0, sizeof(double) * n);
        cycle_rec(c, 0, z, s);
        apply_M(c, z, t, zero);
        omega = dotv(t, s, n) / dotv(t, t, n);
        for (int k = 0; k < n; k++) {
            x[k] += alpha * y[k] + omega * z[k];
            r[k] = s[k] - omega * t[k];
        }
        // residual replacement: the recurrence continues from the true
        // residual b - M x, so that rounding accumulated in the recurrence
        // cannot hold the true residual above the tolerance
        double rt = or_residual(c, 0, x, b, r);
        hist[it] = rt;
        *nit = it;
        if (!(rt == rt) || rt > 1e6 * r0) st = OR_DIVERGED;
        else if (rt <= tol) st = OR_OK;
    }
    free(r); free(rh); free(p); free(v); free(s); free(t); free(y); free(z); free(zero);
    return st;
}


/* ------------------------------------------------------------- adjoint
 *
 * The adjoint of one linear solve is the transposed system M^T lam = c.  Its
 * multigrid cycle is the transpose of the cycle above.  One relaxation stage
 * of the cycle changes x by Q (b - M x) for a fixed matrix Q (a box solve, the
 * lonely-face Jacobi step, the (xi, mean) update, a ghost Jacobi sweep, the
 * coarse-grid correction P B_H R), so a cycle from x = 0 is a linear map B
 * of b.  Writing I - B M as the product of the stages' (I - Q M) and
 * transposing gives B^T = the cycle for M^T whose stages run in reverse
 * order, each with Q^T: boxes with the transposed box matrix, colours in
 * reverse order, post-relaxations before pre-relaxations, P^T as restriction
 * and R^T as interpolation, and the coarsest solve with M^T.  The tests check
 * <B b, c> = <b, C c> for this cycle C.  Inactive rows of M (x = b, Alg. LS)
 * are referenced by ghost stencils, so the adjoint unknown at an inactive
 * node is c minus those ghost contributions; no stage of the cycle touches
 * it, and it appears in no other equation of M^T, so the solve sets it
 * exactly after each cycle. */

/* columns of M on level lev (from the assembled rows and the mean row) */
static void build_columns(ctx_t *c, int lev)
{
    level_t *l = &c->lv[lev];
    int n = l->n, cap = 12 * n + l->nP + 16;
    int *ri = (int *)malloc(sizeof(int) * cap), *ci = (int *)malloc(sizeof(int) * cap);
    double *v = (double *)malloc(sizeof(double) * cap);
    int nnz = or_assemble(c, lev, ri, ci, v, cap);
    free(l->cptr); free(l->crow); free(l->cval);
    l->cptr = (int *)calloc(n + 1, sizeof(int));
    l->crow = (int *)malloc(sizeof(int) * (nnz > 0 ? nnz : 1));
    l->cval = (double *)malloc(sizeof(double) * (nnz > 0 ? nnz : 1));
    for (int k = 0; k < nnz; k++) l->cptr[ci[k] + 1]++;
    for (int k = 0; k < n; k++) l->cptr[k + 1] += l->cptr[k];
    int *fill = (int *)malloc(sizeof(int) * n);
    memcpy(fill, l->cptr, sizeof(int) * n);
    for (int k = 0; k < nnz; k++) {
        int at = fill[ci[k]]++;
        l->crow[at] = ri[k];
        l->cval[at] = v[k];
    }
    free(fill); free(ri); free(ci); free(v);
}

static int adjoint_prepare(ctx_t *c)
{
    if (!c->geom_ok) return OR_INVALID;
    if (c->adj_ok && c->adj_alpha == c->alpha) return OR_OK;
    for (int k = 0; k < c->L; k++) build_columns(c, k);
    level_t *l = &c->lv[c->L - 1];
    int n = l->n;
    double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
    dense_matrix(c, c->L - 1, A);
    free(l->lut); free(l->pivt);
    l->lut = (double *)malloc(sizeof(double) * (size_t)n * n);
    l->pivt = (int *)malloc(sizeof(int) * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) l->lut[(size_t)i * n + j] = A[(size_t)j * n + i];
    free(A);
    if (!lu_factor(n, l->lut, l->pivt)) { seterr(c, "transposed coarsest matrix is singular"); return OR_SINGULAR; }
    c->adj_alpha = c->alpha;
    c->adj_ok = 1;
    return OR_OK;
}

/* (c - M^T lam) at unknown k */
static double col_residual(const level_t *l, int k, const double *lam, const double *cc)
{
    double s = cc[k];
    for (int e = l->cptr[k]; e < l->cptr[k + 1]; e++) s -= l->cval[e] * lam[l->crow[e]];
    return s;
}

/* r = c - M^T lam on level lev; returns ||r||_inf */
double or_residual_t(void *vc, int lev, const double *lam, const double *cc, double *r)
{
    ctx_t *c = (ctx_t *)vc;
    if (adjoint_prepare(c) != OR_OK) return NAN;
    level_t *l = &c->lv[lev];
    double mx = 0.0;
    for (int k = 0; k < l->n; k++) {
        double v = col_residual(l, k, lam, cc);
        r[k] = v;
        if (fabs(v) > mx || v != v) mx = v != v ? NAN : fabs(v);
    }
    return mx;
}

/* the box of cell (i, j) relaxed on M^T: same unknowns as box_relax, the
 * transposed box matrix, residuals of the transposed rows */
static void box_relax_t(ctx_t *c, int lev, double *lam, const double *cc, int i, int j)
{
    level_t *l = &c->lv[lev];
    int gg[5], ii[5], jj[5], unk[5], nu = 0;
    const int fg[4] = {G_U, G_U, G_V, G_V};
    const int fi[4] = {i, i + 1, i, i};
    const int fj[4] = {j, j, j, j + 1};
    for (int f = 0; f < 4; f++) {
        int t = ttype(l, fg[f], fi[f], fj[f]);
        if (t == T_INTERNAL || t == T_GHOST) {
            gg[nu] = fg[f]; ii[nu] = fi[f]; jj[nu] = fj[f];
            unk[nu] = iG(l, fg[f], fi[f], fj[f]);
            nu++;
        }
    }
    gg[nu] = G_P; ii[nu] = i; jj[nu] = j; unk[nu] = iP(l, i, j); nu++;
    double A[25], At[25], rhs[5];
    int piv[5];
    for (int r = 0; r < nu; r++) {
        row_t R;
        get_row(c, lev, gg[r], ii[r], jj[r], &R);
        for (int q = 0; q < nu; q++) {
            double sum = 0.0;
            for (int k = 0; k < R.n; k++)
                if (R.col[k] == unk[q]) sum += R.a[k];
            A[r * nu + q] = sum;
        }
    }
    for (int r = 0; r < nu; r++) {
        rhs[r] = col_residual(l, unk[r], lam, cc);
        for (int q = 0; q < nu; q++) At[r * nu + q] = A[q * nu + r];
    }
    if (!lu_factor(nu, At, piv)) return;
    lu_solve(nu, At, piv, rhs);
    for (int r = 0; r < nu; r++) lam[unk[r]] += rhs[r];
}

/* the transposed box sweep: the lonely faces, then the cut cells in their
 * colours in reverse, then the other cells in colours 4..0 (colour-by-colour
 * ordering) */
void or_box_sweep_t(void *vc, int lev, double *lam, const double *cc)
{
    ctx_t *c = (ctx_t *)vc;
    if (adjoint_prepare(c) != OR_OK) return;
    level_t *l = &c->lv[lev];
    int N = l->N;
    /* lonely internal faces: point Jacobi with the diagonal d */
    int cnt = 0;
    int *idx = (int *)malloc(sizeof(int) * (l->nU + l->nV));
    double *upd = (double *)malloc(sizeof(double) * (l->nU + l->nV));
    row_t R;
    for (int j = 0; j < N; j++)
        for (int i = 1; i < N; i++)
            if (ttype(l, G_U, i, j) == T_INTERNAL && ttype(l, G_P, i - 1, j) != T_INTERNAL &&
                ttype(l, G_P, i, j) != T_INTERNAL) {
                get_row(c, lev, G_U, i, j, &R);
                idx[cnt] = iU(l, i, j);
                upd[cnt++] = col_residual(l, iU(l, i, j), lam, cc) / R.a[0];
            }
    for (int j = 1; j < N; j++)
        for (int i = 0; i < N; i++)
            if (ttype(l, G_V, i, j) == T_INTERNAL && ttype(l, G_P, i, j - 1) != T_INTERNAL &&
                ttype(l, G_P, i, j) != T_INTERNAL) {
                get_row(c, lev, G_V, i, j, &R);
                idx[cnt] = iV(l, i, j);
                upd[cnt++] = col_residual(l, iV(l, i, j), lam, cc) / R.a[0];
            }
    for (int k = 0; k < cnt; k++) lam[idx[k]] += upd[k];
    free(idx);
    free(upd);
    for (int col = l->ncutcol - 1; col >= 0; col--)
        for (int j = 0; j < N; j++)
            for (int i = 0; i < N; i++)
                if (l->cutcol[j * N + i] == col) box_relax_t(c, lev, lam, cc, i, j);
    for (int col = 4; col >= 0; col--)
        for (int j = 0; j < N; j++)
            for (int i = 0; i < N; i++)
                if ((i + 3 * j) % 5 == col && ttype(l, G_P, i, j) == T_INTERNAL && !cut_cell(l, i, j))
                    box_relax_t(c, lev, lam, cc, i, j);
}

/* transpose of the (xi, mean) update: the update adds -1/n_int times the
 * mean of the continuity residuals to xi and 1/(h^2 n_int) times the mean-row
 * residual to every internal and ghost p, so its transpose adds -1/n_int times
 * the xi residual of M^T to the unknown of every internal continuity row and
 * 1/(h^2 n_int) times the sum of the p residuals of M^T to the mean-row
 * unknown (both residuals taken before either change) */
void or_scalar_update_t(void *vc, int lev, double *lam, const double *cc)
{
    ctx_t *c = (ctx_t *)vc;
    if (adjoint_prepare(c) != OR_OK) return;
    level_t *l = &c->lv[lev];
    int N = l->N;
    double h = l->h;
    double rxi = col_residual(l, iXI(l), lam, cc);
    double sp = 0.0;
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++) {
            int t = ttype(l, G_P, i, j);
            if (t == T_INTERNAL || t == T_GHOST) sp += col_residual(l, iP(l, i, j), lam, cc);
        }
    double n = (double)l->n_int;
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++)
            if (ttype(l, G_P, i, j) == T_INTERNAL) lam[iP(l, i, j)] += -rxi / n;
    lam[iXI(l)] += sp / (h * h * n);
}

/* transpose of one ghost Jacobi sweep: the same diagonal step on the rows of
 * M^T at every ghost, wall and box-ghost node */
void or_ghost_sweep_t(void *vc, int lev, double *lam, const double *cc)
{
    ctx_t *c = (ctx_t *)vc;
    if (adjoint_prepare(c) != OR_OK) return;
    level_t *l = &c->lv[lev];
    int N = l->N;
    int *idx = (int *)malloc(sizeof(int) * l->n);
    double *upd = (double *)malloc(sizeof(double) * l->n);
    int cnt = 0;
    row_t R;
    for (int g = 0; g < 3; g++) {
        int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? N - 1 : N;
        int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? N - 1 : N;
        for (int j = jlo; j <= jhi; j++)
            for (int i = ilo; i <= ihi; i++) {
                if (!ghost_class(ttype(l, g, i, j))) continue;
                int k = iG(l, g, i, j);
                get_row(c, lev, g, i, j, &R);
                double res = col_residual(l, k, lam, cc);
                idx[cnt] = k;
                upd[cnt++] = c->ghost_mode == 1 ? c->dtau * res / R.a[0] : c->dtau * res;
            }
    }
    for (int k = 0; k < cnt; k++) lam[idx[k]] += upd[k];
    free(idx);
    free(upd);
}

/* transposed relaxation: nu x {lambda transposed ghost sweeps; transposed
 * (xi, mean) update; transposed box sweep} */
void or_smooth_t(void *vc, int lev, double *lam, const double *cc, int nu)
{
    ctx_t *c = (ctx_t *)vc;
    for (int s = 0; s < nu; s++) {
        for (int k = 0; k < c->lam; k++) or_ghost_sweep_t(c, lev, lam, cc);
        or_scalar_update_t(c, lev, lam, cc);
        or_box_sweep_t(c, lev, lam, cc);
    }
}

/* R^T: lam (level lev) += R^T yH (yH on level lev+1), R the restriction of
 * or_restrict */
void or_restrict_t(void *vc, int lev, const double *yH, double *lam)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *f = &c->lv[lev], *C = &c->lv[lev + 1];
    int Nc = C->N;
    for (int g = 0; g < 3; g++) {
        int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? Nc - 1 : Nc;
        int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? Nc - 1 : Nc;
#pragma omp parallel for schedule(static)
        for (int J = jlo; J <= jhi; J++)
            for (int I = ilo; I <= ihi; I++) {
                int tc = ttype(C, g, I, J);
                if (tc == T_INACTIVE) continue;
                double y = yH[iG(C, g, I, J)];
                int fi[6], fj[6], ns = 0;
                double wt[6];
                if (g == G_U) {
                    for (int dj = 0; dj <= 1; dj++)
                        for (int di = -1; di <= 1; di++) {
                            fi[ns] = 2 * I + di; fj[ns] = 2 * J + dj; wt[ns] = (di == 0 ? 2.0 : 1.0) / 8.0; ns++;
                        }
                } else if (g == G_V) {
                    for (int dj = -1; dj <= 1; dj++)
                        for (int di = 0; di <= 1; di++) {
                            fi[ns] = 2 * I + di; fj[ns] = 2 * J + dj; wt[ns] = (dj == 0 ? 2.0 : 1.0) / 8.0; ns++;
                        }
                } else {
                    for (int dj = 0; dj <= 1; dj++)
                        for (int di = 0; di <= 1; di++) {
                            fi[ns] = 2 * I + di; fj[ns] = 2 * J + dj; wt[ns] = 0.25; ns++;
                        }
                }
                int all = 1, cnt = 0;
                for (int k = 0; k < ns; k++) {
                    if (same_class(tc, ttype(f, g, fi[k], fj[k]))) cnt++;
                    else all = 0;
                }
                for (int k = 0; k < ns; k++) {
                    if (!same_class(tc, ttype(f, g, fi[k], fj[k]))) continue;
                    lam[iG(f, g, fi[k], fj[k])] += all ? wt[k] * y : y / (double)cnt;
                }
            }
    }
    lam[iXI(f)] += yH[iXI(C)];
}

/* P^T: cH (level lev+1) = P^T r (r on level lev), P the interpolation of
 * or_prolong */
void or_prolong_t(void *vc, int lev, const double *r, double *cH)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *f = &c->lv[lev], *C = &c->lv[lev + 1];
    int N = f->N, Nc = C->N;
    memset(cH, 0, sizeof(double) * C->n);
    for (int g = 0; g < 3; g++) {
        int ilo = g == G_V ? -1 : 0, ihi = g == G_P ? N - 1 : N;
        int jlo = g == G_U ? -1 : 0, jhi = g == G_P ? N - 1 : N;
        int Ilo = g == G_V ? -1 : 0, Ihi = g == G_P ? Nc - 1 : Nc;
        int Jlo = g == G_U ? -1 : 0, Jhi = g == G_P ? Nc - 1 : Nc;
#pragma omp parallel for schedule(static)
        for (int j = jlo; j <= jhi; j++)
            for (int i = ilo; i <= ihi; i++) {
                if (ttype(f, g, i, j) == T_INACTIVE) continue;
                int KI[2], KJ[2];
                double wi[2], wj[2];
                int ni = taps(i, g == G_U, Ilo, Ihi, KI, wi);
                int nj = taps(j, g == G_V, Jlo, Jhi, KJ, wj);
                double ws = 0.0;
                for (int a = 0; a < nj; a++)
                    for (int bb = 0; bb < ni; bb++)
                        if (ttype(C, g, KI[bb], KJ[a]) != T_INACTIVE) ws += wj[a] * wi[bb];
                if (!(ws > 0.0)) continue;
                double y = r[iG(f, g, i, j)];
                for (int a = 0; a < nj; a++)
                    for (int bb = 0; bb < ni; bb++)
                        if (ttype(C, g, KI[bb], KJ[a]) != T_INACTIVE)
                            cH[iG(C, g, KI[bb], KJ[a])] += wj[a] * wi[bb] / ws * y;
            }
    }
    cH[iXI(C)] += r[iXI(f)];
}

static void cycle_t_rec(ctx_t *c, int lev, double *lam, const double *cc)
{
    level_t *l = &c->lv[lev];
    if (lev == c->L - 1) {
        memcpy(lam, cc, sizeof(double) * l->n);
        lu_solve(l->n, l->lut, l->pivt, lam);
        return;
    }
    level_t *C = &c->lv[lev + 1];
    or_smooth_t(c, lev, lam, cc, c->nu2);
    or_residual_t(c, lev, lam, cc, l->r);
    or_prolong_t(c, lev, l->r, C->b);
    memset(C->x, 0, sizeof(double) * C->n);
    for (int k = 0; k < c->gamma; k++) cycle_t_rec(c, lev + 1, C->x, C->b);
    or_restrict_t(c, lev, C->x, lam);
    or_smooth_t(c, lev, lam, cc, c->nu1);
}

/* one transposed cycle on level lev (the transpose of or_cycle from zero) */
int or_cycle_t(void *vc, int lev, double *lam, const double *cc)
{
    ctx_t *c = (ctx_t *)vc;
    int st = adjoint_prepare(c);
    if (st != OR_OK) return st;
    cycle_t_rec(c, lev, lam, cc);
    return OR_OK;
}

/* the rows of M^T at inactive nodes: lam_k = c_k - (ghost-row terms) */
static void fix_inactive_t(ctx_t *c, double *lam, const double *cc)
{
    level_t *l = &c->lv[0];
    for (int k = 0; k < l->n - 1; k++) {
        int t = k < l->nU ? l->tU[k] : k < l->nU + l->nV ? l->tV[k - l->nU] : l->tP[k - l->nU - l->nV];
        if (t == T_INACTIVE) lam[k] += col_residual(l, k, lam, cc);
    }
}

/* transposed cycles from lam until ||c - M^T lam||_inf <= tol */
int or_solve_t(void *vc, double *lam, const double *cc, double tol, int max_cycles, double *hist, int *ncyc)
{
    ctx_t *c = (ctx_t *)vc;
    int st = adjoint_prepare(c);
    if (st != OR_OK) return st;
    level_t *l = &c->lv[0];
    fix_inactive_t(c, lam, cc);
    double r0 = or_residual_t(c, 0, lam, cc, l->r);
    hist[0] = r0;
    *ncyc = 0;
    if (r0 <= tol) return OR_OK;
    for (int k = 1; k <= max_cycles; k++) {
        cycle_t_rec(c, 0, lam, cc);
        fix_inactive_t(c, lam, cc);
        double rn = or_residual_t(c, 0, lam, cc, l->r);
        hist[k] = rn;
        *ncyc = k;
        if (!(rn == rn) || rn > 1e6 * r0) return OR_DIVERGED;
        if (rn <= tol) return OR_OK;
    }
    return OR_NOT_CONVERGED;
}

/* ------------------------------------------- adjoint of the CN step
 *
 * One CN step m (geometry of step m+1 built) maps x^m to x^(m+1) = M^-1 b with
 * b = A x^m + dt E f - dt E Nh + a g on the rows of Eq. (spaceprob): A x =
 * x + alpha lap x and E the internal momentum rows, g the rigid-body velocity
 * on the Eq. (BCu) rows (a its amplitude), Nh the convective term of
 * Eq. (extrUdU) (m >= 2: N(x^m) + N^(m-1)/2 - N^(m-2)/2 with the stored terms
 * of the two previous steps) or of the mid-point Picard iteration
 * (Eq. NSitconv) with a fixed number K of iterations (m = 0, 1: iterate k
 * uses (N(x^m) + N(x^(k)))/2, x^(0) = x^m).  The backward pass applies the
 * transposes in reverse: lam = M^-T xbar, fbar += dt E lam, abar += g.lam,
 * xbar^m += A^T lam, and the convective term's adjoint goes to the stored
 * term it came from; the adjoint of a stored term N(x^j) is turned into
 * xbar^j by the transposed Jacobian when step j is processed (with that
 * step's geometry), after all later steps have added to it. */

static int internal_mom(const level_t *l, int k)
{
    if (k < l->nU) return l->tU[k] == T_INTERNAL;
    if (k < l->nU + l->nV) return l->tV[k - l->nU] == T_INTERNAL;
    return 0;
}

/* out += J_N(x)^T y: transpose of the linearised convective term at x (rows:
 * internal u, v nodes; entries of y elsewhere are ignored) */
void or_convective_jt(void *vc, const double *x, const double *y, double *out)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[0];
    int N = l->N;
    double h2 = 2.0 * l->h;
    for (int j = 0; j < N; j++)
        for (int i = 1; i < N; i++) {
            if (ttype(l, G_U, i, j) != T_INTERNAL) continue;
            double w = y[iU(l, i, j)];
            double u = x[iU(l, i, j)];
            double vb = 0.25 * (x[iV(l, i - 1, j)] + x[iV(l, i, j)] + x[iV(l, i - 1, j + 1)] + x[iV(l, i, j + 1)]);
            double dudx = (x[iU(l, i + 1, j)] - x[iU(l, i - 1, j)]) / h2;
            double dudy = (x[iU(l, i, j + 1)] - x[iU(l, i, j - 1)]) / h2;
            out[iU(l, i, j)] += w * dudx;
            out[iU(l, i + 1, j)] += w * u / h2;
            out[iU(l, i - 1, j)] -= w * u / h2;
            out[iU(l, i, j + 1)] += w * vb / h2;
            out[iU(l, i, j - 1)] -= w * vb / h2;
            double cv = 0.25 * w * dudy;
            out[iV(l, i - 1, j)] += cv;
            out[iV(l, i, j)] += cv;
            out[iV(l, i - 1, j + 1)] += cv;
            out[iV(l, i, j + 1)] += cv;
        }
    for (int j = 1; j < N; j++)
        for (int i = 0; i < N; i++) {
            if (ttype(l, G_V, i, j) != T_INTERNAL) continue;
            double w = y[iV(l, i, j)];
            double v = x[iV(l, i, j)];
            double ub = 0.25 * (x[iU(l, i, j - 1)] + x[iU(l, i + 1, j - 1)] + x[iU(l, i, j)] + x[iU(l, i + 1, j)]);
            double dvdx = (x[iV(l, i + 1, j)] - x[iV(l, i - 1, j)]) / h2;
            double dvdy = (x[iV(l, i, j + 1)] - x[iV(l, i, j - 1)]) / h2;
            out[iV(l, i, j)] += w * dvdy;
            out[iV(l, i + 1, j)] += w * ub / h2;
            out[iV(l, i - 1, j)] -= w * ub / h2;
            out[iV(l, i, j + 1)] += w * v / h2;
            out[iV(l, i, j - 1)] -= w * v / h2;
            double cu = 0.25 * w * dvdx;
            out[iU(l, i, j - 1)] += cu;
            out[iU(l, i + 1, j - 1)] += cu;
            out[iU(l, i, j)] += cu;
            out[iU(l, i + 1, j)] += cu;
        }
}

/* out += A^T y, A x = x + alpha lap x on the internal u, v rows */
void or_explicit_t(void *vc, const double *y, double *out)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[0];
    int N = l->N;
    double a = c->alpha / (l->h * l->h);
    for (int j = 0; j < N; j++)
        for (int i = 1; i < N; i++) {
            if (ttype(l, G_U, i, j) != T_INTERNAL) continue;
            double w = y[iU(l, i, j)];
            out[iU(l, i, j)] += (1.0 - 4.0 * a) * w;
            out[iU(l, i + 1, j)] += a * w;
            out[iU(l, i - 1, j)] += a * w;
            out[iU(l, i, j + 1)] += a * w;
            out[iU(l, i, j - 1)] += a * w;
        }
    for (int j = 1; j < N; j++)
        for (int i = 0; i < N; i++) {
            if (ttype(l, G_V, i, j) != T_INTERNAL) continue;
            double w = y[iV(l, i, j)];
            out[iV(l, i, j)] += (1.0 - 4.0 * a) * w;
            out[iV(l, i + 1, j)] += a * w;
            out[iV(l, i - 1, j)] += a * w;
            out[iV(l, i, j + 1)] += a * w;
            out[iV(l, i, j - 1)] += a * w;
        }
}

#define OR_MAXPICARD 16

/* Backward pass of CN step `step` (geometry of step+1 built, alpha set).
 * xm: the state x^m; f: forcing (or NULL); body: the rigid-body motion at
 * unit amplitude {U, V, omega, cx, cy}, amp its amplitude; walls: the box
 * velocities (not scaled); kmax: the fixed Picard count of steps 0, 1.
 * xbar_next = dL/dx^(m+1) (in); xbar_m += dL/dx^m through this step (the
 * caller adds other paths); nb0, nb1, nb2: adjoints of the stored convective
 * terms of steps m, m-1, m-2 (accumulated; nb0 is turned into xbar_m here);
 * fbar += dL/df, *abar += dL/da. */
int or_cn_step_adjoint(void *vc, int step, const double *xm, const double *f, double dt, const double *body,
                       double amp, const double *walls, double tol, int kmax, const double *xbar_next, double *xbar_m,
                       double *nb0, double *nb1, double *nb2, double *fbar, double *abar)
{
    ctx_t *c = (ctx_t *)vc;
    if (!c->geom_ok || kmax < 1 || kmax > OR_MAXPICARD) return OR_INVALID;
    level_t *l = &c->lv[0];
    int n = l->n, st = OR_OK, nc = 0;
    double *g = (double *)calloc(n, sizeof(double)), *zero = (double *)calloc(n, sizeof(double));
    double *lam = (double *)calloc(n, sizeof(double)), *el = (double *)calloc(n, sizeof(double));
    double *xb = (double *)malloc(sizeof(double) * n), *hist = (double *)malloc(sizeof(double) * 1001);
    double nowalls[4] = {0, 0, 0, 0};
    double bamp[5] = {amp * body[0], amp * body[1], amp * body[2], body[3], body[4]};
    or_cn_rhs(c, zero, zero, NULL, dt, NULL, body, nowalls, g);
    /* only the Eq. (BCu) rows carry the body velocity */
    for (int k = 0; k < n; k++)
        if (internal_mom(l, k)) g[k] = 0.0;
    memcpy(xb, xbar_next, sizeof(double) * n);
    double **X = NULL;
    int K = step >= 2 ? 1 : kmax;
    if (step < 2) {
        /* the Picard iterates x^(1..K-1) of the forward step, recomputed */
        X = (double **)calloc(K + 1, sizeof(double *));
        double *Nn = (double *)malloc(sizeof(double) * n), *Nh = (double *)malloc(sizeof(double) * n);
        double *b = (double *)malloc(sizeof(double) * n);
        or_convective(c, xm, Nn);
        memcpy(Nh, Nn, sizeof(double) * n);
        X[0] = (double *)malloc(sizeof(double) * n);
        memcpy(X[0], xm, sizeof(double) * n);
        for (int k = 1; k < K && st == OR_OK; k++) {
            X[k] = (double *)malloc(sizeof(double) * n);
            memcpy(X[k], X[k - 1], sizeof(double) * n);
            or_cn_rhs(c, xm, Nh, f, dt, NULL, bamp, walls, b);
            st = or_solve(c, X[k], b, tol, 1000, hist, &nc);
            or_convective(c, X[k], Nh);
            for (int q = 0; q < n; q++) Nh[q] = 0.5 * (Nn[q] + Nh[q]);
        }
        free(Nn); free(Nh); free(b);
    }
    for (int k = K - 1; k >= 0 && st == OR_OK; k--) {
        memset(lam, 0, sizeof(double) * n);
        st = or_solve_t(c, lam, xb, tol, 1000, hist, &nc);
        if (st != OR_OK) break;
        for (int q = 0; q < n; q++) el[q] = internal_mom(l, q) ? lam[q] : 0.0;
        double ga = 0.0;
        for (int q = 0; q < n; q++) {
            fbar[q] += dt * el[q];
            ga += g[q] * lam[q];
        }
        *abar += ga;
        or_explicit_t(c, lam, xbar_m);
        if (step >= 2) {
            for (int q = 0; q < n; q++) {
                nb0[q] -= dt * el[q];
                nb1[q] -= 0.5 * dt * el[q];
                nb2[q] += 0.5 * dt * el[q];
            }
        } else if (k >= 1) {
            for (int q = 0; q < n; q++) {
                nb0[q] -= 0.5 * dt * el[q];
                el[q] *= -0.5 * dt;
            }
            memset(xb, 0, sizeof(double) * n);
            or_convective_jt(c, X[k], el, xb);
        } else {
            for (int q = 0; q < n; q++) nb0[q] -= dt * el[q];
        }
    }
    if (st == OR_OK) or_convective_jt(c, xm, nb0, xbar_m);
    if (X) {
        for (int k = 0; k <= K; k++) free(X[k]);
        free(X);
    }
    free(g); free(zero); free(lam); free(el); free(xb); free(hist);
    return st;
}

/* colours of the cut cells of level lev (cell j N + i, -1 for other cells);
 * returns the number of colours */
int or_cut_colours(void *vc, int lev, int *out)
{
    ctx_t *c = (ctx_t *)vc;
    level_t *l = &c->lv[lev];
    if (!c->geom_ok || !l->cutcol) return -1;
    memcpy(out, l->cutcol, sizeof(int) * (size_t)l->N * l->N);
    return l->ncutcol;
}
