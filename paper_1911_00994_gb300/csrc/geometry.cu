// Level-set geometry on every multigrid level (Sect. 3.1-3.3):
// node classification (Algorithm LS), ghost marking (Remark 1), boundary
// points (Algorithm 1), ghost rows (Eq. BCu and extrapolation rows), the
// cut-cell and lonely-face lists used by the relaxation.
//
// This file is compiled with -fmad=false: the floating-point decisions taken
// here (march steps, floor cells, bisection signs, snapping, row choice) use
// separately rounded products and sums in a fixed order, so that every node
// gets the same classification as in a plain IEEE evaluation of the same
// formulas.
#include <cmath>
#include <cstdio>

#include "gpmg_internal.cuh"

namespace gpmg {

__constant__ int c_OX2[3] = {0, 1, 1};
__constant__ int c_OY2[3] = {1, 0, 1};

struct Geo {
    const double *phi;  // paper-sign half lattice of the finest grid
    int Nf;             // finest cells per side
    int lev;
    int N;              // cells per side on this level
    int P;
    long long F;
    double x0, y0, h, snap;
    int band;           // extra ghost layers (finest level only)
    uint8_t *t[3];      // node types per grid (frame layout)
    uint8_t *prim;      // [3F]
    uint8_t *done;      // [3F]
    unsigned *err;
    int *flag;
};

__device__ inline bool phi_node(const Geo &G, int g, int i, int j, double *out)
{
    int m = 1 << G.lev;
    int a = m * (2 * i + c_OX2[g]);
    int b = m * (2 * j + c_OY2[g]);
    int M = 2 * G.Nf;
    if (a < 0 || a > M || b < 0 || b > M) return false;
    *out = G.phi[(size_t)b * (M + 1) + a];
    return true;
}

__device__ inline double node_x(const Geo &G, int g, int i) { return G.x0 + (double)(2 * i + c_OX2[g]) * (0.5 * G.h); }
__device__ inline double node_y(const Geo &G, int g, int j) { return G.y0 + (double)(2 * j + c_OY2[g]) * (0.5 * G.h); }

__device__ inline uint8_t ttype(const Geo &G, int g, int i, int j)
{
    if (!in_grid(g, G.N, i, j)) return T_INACTIVE;
    return G.t[g][(j + 1) * G.P + (i + 1)];
}

// bilinear interpolant of phi on the 2x2 cell of grid g containing (x, y),
// cell chosen by floor in each axis
__device__ bool bilin(const Geo &G, int g, double x, double y, double *val, double *gx, double *gy)
{
    double h = G.h;
    double sx = (x - G.x0) / h - 0.5 * (double)c_OX2[g];
    double sy = (y - G.y0) / h - 0.5 * (double)c_OY2[g];
    double fi = floor(sx), fj = floor(sy);
    if (!(fi > -1e9 && fi < 1e9 && fj > -1e9 && fj < 1e9)) return false;
    int i0 = (int)fi, j0 = (int)fj;
    double fx = sx - fi, fy = sy - fj;
    double p00, p10, p01, p11;
    if (!phi_node(G, g, i0, j0, &p00) || !phi_node(G, g, i0 + 1, j0, &p10) || !phi_node(G, g, i0, j0 + 1, &p01) ||
        !phi_node(G, g, i0 + 1, j0 + 1, &p11))
        return false;
    double ex = 1.0 - fx, ey = 1.0 - fy;
    *val = ex * ey * p00 + fx * ey * p10 + ex * fy * p01 + fx * fy * p11;
    *gx = (ey * (p10 - p00) + fy * (p11 - p01)) / h;
    *gy = (ex * (p01 - p00) + fx * (p11 - p10)) / h;
    return true;
}

__device__ bool unit_normal(const Geo &G, int g, double x, double y, double *nx, double *ny)
{
    double v, gx, gy;
    if (!bilin(G, g, x, y, &v, &gx, &gy)) return false;
    double nrm = sqrt(gx * gx + gy * gy);
    if (!(nrm > 0.0)) return false;
    *nx = gx / nrm;
    *ny = gy / nrm;
    return true;
}

// Algorithm 1 (march by h/2 against the normal, then bisection); a node
// inside the fluid marches along the normal
__device__ bool ghost_to_boundary(const Geo &G, int g, int i, int j, double *xB, double *yB)
{
    double h = G.h;
    double xG = node_x(G, g, i), yG = node_y(G, g, j);
    double phH;
    if (!phi_node(G, g, i, j, &phH)) return false;
    double sg = phH > 0.0 ? 1.0 : -1.0;
    double xH = xG, yH = yG, xK = xG, yK = yG;
    int steps = 0;
    while (sg * phH > 0.0) {
        double nx, ny, gx, gy;
        xK = xH;
        yK = yH;
        if (!unit_normal(G, g, xH, yH, &nx, &ny)) return false;
        xH = xH - sg * (0.5 * h * nx);
        yH = yH - sg * (0.5 * h * ny);
        if (!bilin(G, g, xH, yH, &phH, &gx, &gy)) return false;
        if (++steps > MAX_MARCH) return false;
    }
    if (steps == 0) {
        *xB = xG;
        *yB = yG;
        return true;
    }
    double dx = xH - xK, dy = yH - yK;
    double dist = sqrt(dx * dx + dy * dy);
    int nb = (int)ceil(log2(dist / (0.01 * h)));
    double xm = xH, ym = yH;
    for (int it = 0; it < nb; it++) {
        double phB, gx, gy;
        xm = 0.5 * (xH + xK);
        ym = 0.5 * (yH + yK);
        if (!bilin(G, g, xm, ym, &phB, &gx, &gy)) return false;
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
    return true;
}

__device__ inline void lagrange3(double t, double T[3])
{
    T[0] = (1.0 - t) * (2.0 - t) / 2.0;
    T[1] = t * (2.0 - t);
    T[2] = t * (t - 1.0) / 2.0;
}

struct GhostRow {
    int kind, nst;
    int si[9], sj[9];
    double w[9];
    double xB, yB, thx, thy;
};

// Row of an external node acting as a ghost: Eq. (BCu) for u, v ghosts that
// an internal or box-ghost row references and whose B is within one cell on
// both axes; otherwise extrapolation along the dominant normal axis toward
// the fluid (quadratic for u, v; linear for p) where phi decreases strictly
// along its nodes, else a copy of the axis neighbour of smallest phi.
__device__ bool ghost_setup(const Geo &G, int g, int i, int j, GhostRow *R)
{
    double h = G.h;
    double xG = node_x(G, g, i), yG = node_y(G, g, j);
    double nx, ny;
    if (!unit_normal(G, g, xG, yG, &nx, &ny)) return false;
    int sx = nx >= 0.0 ? 1 : -1;
    int sy = ny >= 0.0 ? 1 : -1;
    int axis = fabs(nx) >= fabs(ny) ? 0 : 1;
    R->kind = K_EXTRAP;
    R->xB = 0.0; R->yB = 0.0; R->thx = 0.0; R->thy = 0.0;
    if (g != G_P) {
        double xB, yB;
        if (!ghost_to_boundary(G, g, i, j, &xB, &yB)) return false;
        R->xB = xB;
        R->yB = yB;
        R->thx = (double)sx * (xG - xB) / h;
        R->thy = (double)sy * (yG - yB) / h;
        if (G.prim[(long long)g * G.F + (j + 1) * G.P + (i + 1)] && R->thx <= 1.0 && R->thy <= 1.0) R->kind = K_BCU;
    }
    if (R->kind == K_BCU) {
        double Tx[3], Ty[3];
        lagrange3(R->thx, Tx);
        lagrange3(R->thy, Ty);
        R->nst = 9;
        for (int ky = 0; ky < 3; ky++)
            for (int kx = 0; kx < 3; kx++) {
                R->si[ky * 3 + kx] = i - kx * sx;
                R->sj[ky * 3 + kx] = j - ky * sy;
                R->w[ky * 3 + kx] = Tx[kx] * Ty[ky];
            }
        return true;
    }
    const double e3[3] = {1.0, -2.0, 1.0};
    const double e4[4] = {1.0, -3.0, 3.0, -1.0};
    int s = axis == 0 ? sx : sy;
    int n = g == G_P ? 3 : 4;
    double ph[4];
    bool mono = true;
    for (int k = 0; k < n && mono; k++) {
        int ii = i - (axis == 0 ? k * s : 0), jj = j - (axis == 1 ? k * s : 0);
        if (!phi_node(G, g, ii, jj, &ph[k])) mono = false;
        else if (k > 0 && !(ph[k] < ph[k - 1])) mono = false;
    }
    if (mono) {
        R->nst = n;
        for (int k = 0; k < n; k++) {
            R->si[k] = i - (axis == 0 ? k * s : 0);
            R->sj[k] = j - (axis == 1 ? k * s : 0);
            R->w[k] = g == G_P ? e3[k] : e4[k];
        }
        return true;
    }
    const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
    double pG, best = 0.0;
    int kb = -1;
    if (!phi_node(G, g, i, j, &pG)) return false;
    for (int k = 0; k < 4; k++) {
        double q;
        if (!phi_node(G, g, i + di[k], j + dj[k], &q)) continue;
        if (q < pG && (kb < 0 || q < best)) {
            best = q;
            kb = k;
        }
    }
    if (kb < 0) return false;
    R->kind = K_COPY;
    R->nst = 2;
    R->si[0] = i; R->sj[0] = j; R->w[0] = 1.0;
    R->si[1] = i + di[kb]; R->sj[1] = j + dj[kb]; R->w[1] = -1.0;
    return true;
}

// Algorithm LS: internal when phi < 0, and farther than snap*h from the
// boundary (first-order distance phi / |grad phi| of the bilinear interpolant)
__device__ bool node_internal(const Geo &G, int g, int i, int j, double ph)
{
    if (!(ph < 0.0)) return false;
    if (G.snap <= 0.0) return true;
    double v, gx, gy;
    if (!bilin(G, g, node_x(G, g, i), node_y(G, g, j), &v, &gx, &gy)) return true;
    double gn = sqrt(gx * gx + gy * gy);
    return ph < -G.snap * G.h * gn;
}

// ------------------------------------------------------------------ kernels

// level set of a rigidly moving test body on the half-cell lattice (paper
// sign), see gp_shape in gpmg.h
__global__ void k_shape_phi(double *phi, int Nf, double x0, double y0, double L, gp_shape sh, double cx, double cy,
                            double ang)
{
    long long n = (long long)(2 * Nf + 1) * (2 * Nf + 1);
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int a = (int)(k % (2 * Nf + 1)), bq = (int)(k / (2 * Nf + 1));
    double hh = 0.5 * (L / Nf);
    double x = x0 + a * hh, y = y0 + bq * hh;
    double dx = x - cx, dy = y - cy;
    double c = cos(ang), s = sin(ang);
    double qx = c * dx + s * dy, qy = -s * dx + c * dy;  // rotate by -ang
    double r = sqrt(qx * qx + qy * qy);
    double v;
    if (sh.kind == GP_CIRCLE) v = sh.a - r;
    else if (sh.kind == GP_ELLIPSE) v = 1.0 - sqrt(qx * qx / (sh.a * sh.a) + qy * qy / (sh.b * sh.b));
    else v = sh.a + sh.b * sin(sh.k * atan2(qy, qx)) - r;
    phi[k] = v;
}

__global__ void k_phi_sign(const double *in, double *out, long long n, double s)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) out[k] = s * in[k];
}

__global__ void k_classify(Geo G)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= G.P) return;
    int i = col - 1, j = row - 1, N = G.N;
    long long s = (long long)row * G.P + col;
    double ph;
    uint8_t t;
    // u
    if (!in_grid(G_U, N, i, j)) t = T_INACTIVE;
    else if (j == -1 || j == N) t = (i >= 1 && i <= N - 1) ? T_BOXGHOST : T_INACTIVE;
    else if (i == 0 || i == N) t = T_WALL;
    else if (!phi_node(G, G_U, i, j, &ph)) { atomicOr(G.err, E_STENCIL_OUT); t = T_INACTIVE; }
    else t = node_internal(G, G_U, i, j, ph) ? T_INTERNAL : T_EXT;
    G.t[G_U][s] = t;
    // v
    if (!in_grid(G_V, N, i, j)) t = T_INACTIVE;
    else if (i == -1 || i == N) t = (j >= 1 && j <= N - 1) ? T_BOXGHOST : T_INACTIVE;
    else if (j == 0 || j == N) t = T_WALL;
    else if (!phi_node(G, G_V, i, j, &ph)) { atomicOr(G.err, E_STENCIL_OUT); t = T_INACTIVE; }
    else t = node_internal(G, G_V, i, j, ph) ? T_INTERNAL : T_EXT;
    G.t[G_V][s] = t;
    // p
    if (!in_grid(G_P, N, i, j)) t = T_INACTIVE;
    else if (!phi_node(G, G_P, i, j, &ph)) { atomicOr(G.err, E_STENCIL_OUT); t = T_INACTIVE; }
    else t = node_internal(G, G_P, i, j, ph) ? T_INTERNAL : T_EXT;
    G.t[G_P][s] = t;
    G.prim[s] = 0; G.prim[G.F + s] = 0; G.prim[2 * G.F + s] = 0;
    G.done[s] = 0; G.done[G.F + s] = 0; G.done[2 * G.F + s] = 0;
}

// a pressure cell whose four faces are all non-internal has no box
__global__ void k_pcell_reclass(Geo G)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    int i = col - 1, j = row - 1;
    if (!in_grid(G_P, G.N, i, j)) return;
    long long s = (long long)row * G.P + col;
    if (G.t[G_P][s] != T_INTERNAL) return;
    if (ttype(G, G_U, i, j) != T_INTERNAL && ttype(G, G_U, i + 1, j) != T_INTERNAL &&
        ttype(G, G_V, i, j) != T_INTERNAL && ttype(G, G_V, i, j + 1) != T_INTERNAL)
        G.t[G_P][s] = T_EXT;
}

__device__ inline void mark_needed(const Geo &G, int g, int i, int j)
{
    if (!in_grid(g, G.N, i, j)) {
        atomicOr(G.err, E_STENCIL_OUT);
        return;
    }
    long long s = (long long)(j + 1) * G.P + (i + 1);
    uint8_t t = G.t[g][s];
    if (t == T_EXT || t == T_GHOST) {
        G.t[g][s] = T_GHOST;
        G.prim[g * G.F + s] = 1;
    } else if (t == T_INACTIVE) {
        atomicOr(G.err, E_INACTIVE_REF);
    }
}

// external nodes referenced by internal and box-ghost rows become ghosts
__global__ void k_mark_primary(Geo G)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= G.P) return;
    int i = col - 1, j = row - 1, N = G.N;
    if (ttype(G, G_U, i, j) == T_INTERNAL) {
        mark_needed(G, G_U, i + 1, j); mark_needed(G, G_U, i - 1, j);
        mark_needed(G, G_U, i, j + 1); mark_needed(G, G_U, i, j - 1);
        mark_needed(G, G_P, i, j); mark_needed(G, G_P, i - 1, j);
    }
    if (ttype(G, G_V, i, j) == T_INTERNAL) {
        mark_needed(G, G_V, i + 1, j); mark_needed(G, G_V, i - 1, j);
        mark_needed(G, G_V, i, j + 1); mark_needed(G, G_V, i, j - 1);
        mark_needed(G, G_P, i, j); mark_needed(G, G_P, i, j - 1);
    }
    if (ttype(G, G_P, i, j) == T_INTERNAL) {
        mark_needed(G, G_U, i, j); mark_needed(G, G_U, i + 1, j);
        mark_needed(G, G_V, i, j); mark_needed(G, G_V, i, j + 1);
    }
    if (j == -1 && i >= 1 && i <= N - 1) {  // u box-ghost rows reference two nodes inward
        mark_needed(G, G_U, i, 0); mark_needed(G, G_U, i, 1);
        mark_needed(G, G_U, i, N - 1); mark_needed(G, G_U, i, N - 2);
    }
    if (i == -1 && j >= 1 && j <= N - 1) {
        mark_needed(G, G_V, 0, j); mark_needed(G, G_V, 1, j);
        mark_needed(G, G_V, N - 1, j); mark_needed(G, G_V, N - 2, j);
    }
}

__device__ inline bool near_internal(const Geo &G, int g, int i, int j, int rad)
{
    for (int dj = -rad; dj <= rad; dj++)
        for (int di = -rad; di <= rad; di++)
            if (ttype(G, g, i + di, j + dj) == T_INTERNAL) return true;
    return false;
}

// moving bodies (Sect. 3.4): external nodes of the finest grid within `band`
// index steps of an internal node of their grid are ghosts too
__global__ void k_mark_band(Geo G)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= G.P) return;
    int i = col - 1, j = row - 1;
    long long s = (long long)row * G.P + col;
    for (int g = 0; g < 3; g++)
        if (G.t[g][s] == T_EXT && near_internal(G, g, i, j, G.band)) G.t[g][s] = T_GHOST;
}

// one closure pass: the stencil of every ghost not processed yet marks its
// external nodes within two steps of an internal node as ghosts
__global__ void k_closure(Geo G)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= G.P) return;
    int i = col - 1, j = row - 1;
    long long s = (long long)row * G.P + col;
    for (int g = 0; g < 3; g++) {
        if (G.t[g][s] != T_GHOST || G.done[g * G.F + s]) continue;
        G.done[g * G.F + s] = 1;
        GhostRow R;
        if (!ghost_setup(G, g, i, j, &R)) {
            atomicOr(G.err, E_PROJECTION);
            continue;
        }
        for (int k = 1; k < R.nst; k++) {
            int ii = R.si[k], jj = R.sj[k];
            if (!in_grid(g, G.N, ii, jj)) {
                atomicOr(G.err, E_STENCIL_OUT);
                continue;
            }
            long long s2 = (long long)(jj + 1) * G.P + (ii + 1);
            if (G.t[g][s2] == T_EXT && near_internal(G, g, ii, jj, G.band > 2 ? G.band : 2)) {
                G.t[g][s2] = T_GHOST;
                atomicExch(G.flag, 1);
            }
        }
    }
}

__global__ void k_finalize_types(Geo G, int *nint)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= G.P) return;
    long long s = (long long)row * G.P + col;
    for (int g = 0; g < 3; g++)
        if (G.t[g][s] == T_EXT) G.t[g][s] = T_INACTIVE;
    if (G.t[G_P][s] == T_INTERNAL) atomicAdd(nint, 1);
}

// ghost counts per (grid, row): one thread per row
__global__ void k_row_counts(Geo G, int *cnt)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int R = G.N + 2;
    if (r >= 3 * R) return;
    int g = r / R, row = r % R;
    const uint8_t *t = G.t[g] + (long long)row * G.P;
    int c = 0;
    for (int col = 0; col < G.P; col++) c += (t[col] == T_GHOST);
    cnt[r] = c;
}

// exclusive scan of n ints by one thread (n <= 3 * (N + 2)); cnt[n] = total
__global__ void k_scan_serial(int *cnt, int n)
{
    if (threadIdx.x || blockIdx.x) return;
    int acc = 0;
    for (int k = 0; k < n; k++) {
        int c = cnt[k];
        cnt[k] = acc;
        acc += c;
    }
    cnt[n] = acc;
}

__global__ void k_scatter_ghosts(Geo G, const int *off, GhostList gh)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int R = G.N + 2;
    if (r >= 3 * R) return;
    int g = r / R, row = r % R;
    const uint8_t *t = G.t[g] + (long long)row * G.P;
    int k = off[r];
    for (int col = 0; col < G.P; col++)
        if (t[col] == T_GHOST) {
            if (k < gh.cap) gh.node[k] = (int)(g * G.F + (long long)row * G.P + col);
            k++;
        }
}

__global__ void k_ghost_rows(Geo G, GhostList gh, int nobj)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nobj || k >= gh.cap) return;
    int v = gh.node[k];
    int g = (int)(v / G.F);
    int s = (int)(v - g * G.F);
    int i = s % G.P - 1, j = s / G.P - 1;
    GhostRow R;
    if (!ghost_setup(G, g, i, j, &R)) {
        atomicOr(G.err, E_PROJECTION);
        R.kind = K_COPY; R.nst = 1; R.si[0] = i; R.sj[0] = j; R.w[0] = 1.0;
    }
    gh.kind[k] = (uint8_t)R.kind;
    gh.nst[k] = (uint8_t)R.nst;
    for (int m = 0; m < GH_ST; m++) {
        int idx = v;
        double w = 0.0;
        if (m < R.nst) {
            if (in_grid(g, G.N, R.si[m], R.sj[m])) idx = (int)(g * G.F + (long long)(R.sj[m] + 1) * G.P + (R.si[m] + 1));
            else atomicOr(G.err, E_STENCIL_OUT);
            w = R.w[m];
        }
        gh.st[(long long)m * gh.cap + k] = idx;
        gh.w[(long long)m * gh.cap + k] = w;
        gh.wf[(long long)m * gh.cap + k] = (float)w;
    }
    gh.B[k] = R.xB;
    gh.B[gh.cap + k] = R.yB;
    gh.th[k] = R.thx;
    gh.th[gh.cap + k] = R.thy;
}

// walls and box ghosts after the object ghosts: for each grid 2N wall rows
// then 2(N-1) box-ghost rows
__global__ void k_wall_rows(Geo G, GhostList gh, int nobj)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int N = G.N;
    int per = 2 * N + 2 * (N - 1);
    if (k >= 2 * per) return;
    int g = k / per, q = k % per;
    int pos = nobj + k;
    if (pos >= gh.cap) {
        atomicOr(G.err, E_GHOST_CAP);
        return;
    }
    int i, j, kind, nst = 1;
    int si[3], sj[3];
    double w[3] = {1.0, 0.0, 0.0};
    if (q < 2 * N) {  // wall: wall-normal velocity on the wall, Dirichlet
        kind = K_WALL;
        if (g == G_U) { i = (q < N) ? 0 : N; j = q % N; }
        else { j = (q < N) ? 0 : N; i = q % N; }
        si[0] = i; sj[0] = j;
    } else {  // box ghost: 3/8 x_G + 3/4 x_1 - 1/8 x_2 = value on the wall
        int q2 = q - 2 * N;
        kind = K_BOXGHOST;
        nst = 3;
        w[0] = 3.0 / 8.0; w[1] = 3.0 / 4.0; w[2] = -1.0 / 8.0;
        int t = q2 % (N - 1) + 1;
        bool lo = q2 < N - 1;
        if (g == G_U) {
            i = t; j = lo ? -1 : N;
            int s = lo ? 1 : -1;
            for (int m = 0; m < 3; m++) { si[m] = i; sj[m] = j + m * s; }
        } else {
            j = t; i = lo ? -1 : N;
            int s = lo ? 1 : -1;
            for (int m = 0; m < 3; m++) { si[m] = i + m * s; sj[m] = j; }
        }
    }
    gh.node[pos] = (int)(g * G.F + (long long)(j + 1) * G.P + (i + 1));
    gh.kind[pos] = (uint8_t)kind;
    gh.nst[pos] = (uint8_t)nst;
    for (int m = 0; m < GH_ST; m++) {
        int idx = gh.node[pos];
        double ww = 0.0;
        if (m < nst) {
            idx = (int)(g * G.F + (long long)(sj[m] + 1) * G.P + (si[m] + 1));
            ww = w[m];
        }
        gh.st[(long long)m * gh.cap + pos] = idx;
        gh.w[(long long)m * gh.cap + pos] = ww;
        gh.wf[(long long)m * gh.cap + pos] = (float)ww;
    }
    gh.B[pos] = 0.0; gh.B[gh.cap + pos] = 0.0;
    gh.th[pos] = 0.0; gh.th[gh.cap + pos] = 0.0;
}

__device__ inline int find_ghost(const GhostList &gh, int nobj, int v)
{
    int lo = 0, hi = nobj - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int x = gh.node[mid];
        if (x == v) return mid;
        if (x < v) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

__device__ inline bool cut_cell(const Geo &G, int i, int j)
{
    return ttype(G, G_U, i, j) == T_GHOST || ttype(G, G_U, i + 1, j) == T_GHOST || ttype(G, G_V, i, j) == T_GHOST ||
           ttype(G, G_V, i, j + 1) == T_GHOST;
}

// pass 0: count cut cells per colour; pass 1: scatter (order inside a colour
// is irrelevant: boxes of one colour are independent)
__global__ void k_cut_cells(Geo G, CutList cut, GhostList gh, int nobj, int pass, int *cursor)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    int i = col - 1, j = row - 1;
    if (!in_grid(G_P, G.N, i, j)) return;
    if (ttype(G, G_P, i, j) != T_INTERNAL || !cut_cell(G, i, j)) return;
    int c = (j % 5) * 5 + (i % 5);
    if (pass == 0) {
        atomicAdd(&cursor[c], 1);
        return;
    }
    int pos = atomicAdd(&cursor[c], 1);
    if (pos >= cut.cap) {
        atomicOr(G.err, E_CUT_CAP);
        return;
    }
    cut.cell[pos] = row * G.P + col;
    const int fg[4] = {G_U, G_U, G_V, G_V};
    const int fi[4] = {i, i + 1, i, i};
    const int fj[4] = {j, j, j, j + 1};
    for (int f = 0; f < 4; f++) {
        int q = -1;
        if (ttype(G, fg[f], fi[f], fj[f]) == T_GHOST)
            q = find_ghost(gh, nobj, (int)(fg[f] * G.F + (long long)(fj[f] + 1) * G.P + (fi[f] + 1)));
        cut.gface[(long long)f * cut.cap + pos] = q;
    }
}

__global__ void k_cut_offsets(int *cursor, int *off)
{
    if (threadIdx.x || blockIdx.x) return;
    int acc = 0;
    for (int c = 0; c < 25; c++) {
        off[c] = acc;
        int n = cursor[c];
        cursor[c] = acc;
        acc += n;
    }
    off[25] = acc;
}

// internal faces with no internal cell on either side
__global__ void k_lonely(Geo G, int *list, int *n, int cap)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= G.P) return;
    int i = col - 1, j = row - 1;
    long long s = (long long)row * G.P + col;
    if (ttype(G, G_U, i, j) == T_INTERNAL && ttype(G, G_P, i - 1, j) != T_INTERNAL && ttype(G, G_P, i, j) != T_INTERNAL) {
        int k = atomicAdd(n, 1);
        if (k < cap) list[k] = (int)s;
    }
    if (ttype(G, G_V, i, j) == T_INTERNAL && ttype(G, G_P, i, j - 1) != T_INTERNAL && ttype(G, G_P, i, j) != T_INTERNAL) {
        int k = atomicAdd(n, 1);
        if (k < cap) list[k] = (int)(G.F + s);
    }
}

// ------------------------------------------------------------- host driver

static Geo make_geo(Ctx *c, int lev)
{
    Level &l = c->lv[lev];
    Geo G;
    G.phi = c->phi;
    G.Nf = c->prm.N;
    G.lev = lev;
    G.N = l.N;
    G.P = l.P;
    G.F = l.F;
    G.x0 = c->prm.x0;
    G.y0 = c->prm.y0;
    G.h = c->prm.L / (double)l.N;
    G.snap = c->prm.snap;
    G.band = lev == 0 ? c->prm.band : 0;
    G.t[0] = l.tU; G.t[1] = l.tV; G.t[2] = l.tP;
    G.prim = l.prim;
    G.done = l.done;
    G.err = c->err;
    G.flag = c->flag;
    return G;
}

static int cuda_fail(Ctx *c, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return 0;
    snprintf(c->msg, sizeof c->msg, "%s: %s", where, cudaGetErrorString(e));
    return 1;
}

// returns a gp_status
void shape_phi(Ctx *c, const gp_shape &sh, double cx, double cy, double ang)
{
    int Nf = c->prm.N;
    long long nphi = (long long)(2 * Nf + 1) * (2 * Nf + 1);
    k_shape_phi<<<(unsigned)((nphi + 255) / 256), 256, 0, c->stream>>>(c->phi, Nf, c->prm.x0, c->prm.y0, c->prm.L, sh, cx,
                                                                       cy, ang);
}

// phi_in == nullptr: the context's lattice is already filled (paper sign)
int build_geometry_levels(Ctx *c, const double *phi_in, int phi_fluid_positive)
{
    cudaStream_t st = c->stream;
    int Nf = c->prm.N;
    long long nphi = (long long)(2 * Nf + 1) * (2 * Nf + 1);
    if (phi_in)
        k_phi_sign<<<(unsigned)((nphi + 255) / 256), 256, 0, st>>>(phi_in, c->phi, nphi, phi_fluid_positive ? -1.0 : 1.0);
    if (cuda_fail(c, cudaMemsetAsync(c->err, 0, sizeof(unsigned), st), "memset")) return GP_CUDA;
    int *hflag = (int *)c->hostbuf;
    for (int lev = 0; lev < c->L; lev++) {
        Level &l = c->lv[lev];
        Geo G = make_geo(c, lev);
        dim3 blk(128), grd((l.P + 127) / 128, l.N + 2);
        k_classify<<<grd, blk, 0, st>>>(G);
        k_pcell_reclass<<<grd, blk, 0, st>>>(G);
        k_mark_primary<<<grd, blk, 0, st>>>(G);
        if (G.band > 0) k_mark_band<<<grd, blk, 0, st>>>(G);
        int pass = 0;
        for (;; pass++) {
            if (pass > 64) {
                snprintf(c->msg, sizeof c->msg, "ghost marking does not close on level %d", lev);
                return GP_GEOMETRY;
            }
            cudaMemsetAsync(c->flag, 0, sizeof(int), st);
            k_closure<<<grd, blk, 0, st>>>(G);
            cudaMemcpyAsync(hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (cuda_fail(c, cudaStreamSynchronize(st), "closure")) return GP_CUDA;
            if (!*hflag) break;
        }
        cudaMemsetAsync(l.nint, 0, sizeof(int), st);
        k_finalize_types<<<grd, blk, 0, st>>>(G, l.nint);
        // compaction of object ghosts in (grid, row, col) order
        int nrows = 3 * (l.N + 2);
        int *cnt = (int *)c->part;  // scratch: nrows + 1 ints
        k_row_counts<<<(nrows + 127) / 128, 128, 0, st>>>(G, cnt);
        k_scan_serial<<<1, 1, 0, st>>>(cnt, nrows);
        k_scatter_ghosts<<<(nrows + 127) / 128, 128, 0, st>>>(G, cnt, l.gh);
        int nobj = 0;
        cudaMemcpyAsync(hflag, cnt + nrows, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (cuda_fail(c, cudaStreamSynchronize(st), "ghost count")) return GP_CUDA;
        nobj = *hflag;
        int nwall = 2 * (2 * l.N + 2 * (l.N - 1));
        if (nobj + nwall > l.gh.cap) {
            snprintf(c->msg, sizeof c->msg, "level %d: %d ghost rows exceed the capacity %d", lev, nobj + nwall, l.gh.cap);
            return GP_GEOMETRY;
        }
        if (nobj > 0) k_ghost_rows<<<(nobj + 127) / 128, 128, 0, st>>>(G, l.gh, nobj);
        k_wall_rows<<<(nwall + 127) / 128, 128, 0, st>>>(G, l.gh, nobj);
        l.h_nghost = nobj;
        l.h_nrows = nobj + nwall;
        int hc[2] = {nobj, nobj + nwall};
        cudaMemcpyAsync(l.gh.count, hc, 2 * sizeof(int), cudaMemcpyHostToDevice, st);
        // cut cells by colour
        int *cursor = cnt;  // 25 ints of scratch
        cudaMemsetAsync(cursor, 0, 25 * sizeof(int), st);
        dim3 grp((l.P + 127) / 128, l.N + 2);
        k_cut_cells<<<grp, blk, 0, st>>>(G, l.cut, l.gh, nobj, 0, cursor);
        k_cut_offsets<<<1, 1, 0, st>>>(cursor, l.cut.off);
        k_cut_cells<<<grp, blk, 0, st>>>(G, l.cut, l.gh, nobj, 1, cursor);
        cudaMemsetAsync(l.nlonely, 0, sizeof(int), st);
        k_lonely<<<grd, blk, 0, st>>>(G, l.lonely, l.nlonely, l.lonely_cap);
        cudaMemcpyAsync(l.h_cutoff, l.cut.off, 26 * sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&l.h_nlonely, l.nlonely, sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&l.h_nint, l.nint, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (cuda_fail(c, cudaStreamSynchronize(st), "geometry")) return GP_CUDA;
        l.h_ncut = l.h_cutoff[25];
        l.cut.ncol = 25;  // recoloured once the rows of the cut boxes are prepared
        if (l.h_ncut > l.cut.cap) {
            snprintf(c->msg, sizeof c->msg, "level %d: %d cut cells exceed the capacity %d", lev, l.h_ncut, l.cut.cap);
            return GP_GEOMETRY;
        }
        if (l.h_nlonely > l.lonely_cap) {
            snprintf(c->msg, sizeof c->msg, "level %d: too many lonely faces", lev);
            return GP_GEOMETRY;
        }
        if (l.h_nint == 0) {
            snprintf(c->msg, sizeof c->msg, "level %d: no internal pressure cell", lev);
            return GP_GEOMETRY;
        }
    }
    unsigned herr = 0;
    cudaMemcpyAsync(&herr, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (cuda_fail(c, cudaStreamSynchronize(st), "geometry status")) return GP_CUDA;
    if (herr) {
        snprintf(c->msg, sizeof c->msg, "geometry error bits 0x%x (1 stencil leaves the grid, 2 inactive reference, "
                 "4 boundary projection failed, 8 ghost capacity, 16 cut capacity)", herr);
        return GP_GEOMETRY;
    }
    return GP_OK;
}

}  // namespace gpmg
