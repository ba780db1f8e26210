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

// half-cell offsets (x, y) of node (0, 0) of the u, v and p grids
__constant__ int c_half[3][2] = {{0, 1}, {1, 0}, {1, 1}};

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

// One grid of one level, read through the finest half-cell lattice: its node
// (i, j) is lattice point (step (2 i + hx), step (2 j + hy)), step = 2^lev,
// so the coarse grids see phi by injection.
struct GridView {
    const double *phi;
    int side, step, hx, hy;
    double x0, y0, h;
    __device__ GridView(const Geo &G, int g)
        : phi(G.phi), side(2 * G.Nf + 1), step(1 << G.lev), hx(c_half[g][0]), hy(c_half[g][1]), x0(G.x0),
          y0(G.y0), h(G.h)
    {
    }
    __device__ bool at(int i, int j, double &v) const
    {
        const int a = step * (2 * i + hx), b = step * (2 * j + hy);
        if (a < 0 || b < 0 || a >= side || b >= side) return false;
        v = phi[(size_t)b * side + a];
        return true;
    }
    __device__ double xc(int i) const { return x0 + (double)(2 * i + hx) * (0.5 * h); }
    __device__ double yc(int j) const { return y0 + (double)(2 * j + hy) * (0.5 * h); }
};

// phi's bilinear interpolant on the grid cell holding a point (Sect. 3.3):
// value and gradient.  The cell is the one whose lower-left node is the floor
// of the point's grid coordinates (reading R7).
struct Patch {
    double v, gx, gy;
};

__device__ bool patch_at(const GridView &V, double x, double y, Patch &P)
{
    const double cx = (x - V.x0) / V.h - 0.5 * (double)V.hx;
    const double cy = (y - V.y0) / V.h - 0.5 * (double)V.hy;
    const double bx = floor(cx), by = floor(cy);
    if (!(bx > -1e9 && bx < 1e9 && by > -1e9 && by < 1e9)) return false;
    const int i = (int)bx, j = (int)by;
    double c00, c10, c01, c11;  // corners: (i, j), (i + 1, j), (i, j + 1), (i + 1, j + 1)
    if (!V.at(i, j, c00) || !V.at(i + 1, j, c10) || !V.at(i, j + 1, c01) || !V.at(i + 1, j + 1, c11)) return false;
    const double tx = cx - bx, ty = cy - by, sx = 1.0 - tx, sy = 1.0 - ty;
    P.v = sx * sy * c00 + tx * sy * c10 + sx * ty * c01 + tx * ty * c11;
    P.gx = (sy * (c10 - c00) + ty * (c11 - c01)) / V.h;
    P.gy = (sx * (c01 - c00) + tx * (c11 - c10)) / V.h;
    return true;
}

// direction of grad phi (toward the object) at a point
__device__ bool normal_at(const GridView &V, double x, double y, double &nx, double &ny)
{
    Patch P;
    if (!patch_at(V, x, y, P)) return false;
    const double len = sqrt(P.gx * P.gx + P.gy * P.gy);
    if (!(len > 0.0)) return false;
    nx = P.gx / len;
    ny = P.gy / len;
    return true;
}

// Algorithm 1 for the node (i, j): walk in steps of h/2 along -grad phi (a
// node inside the fluid, snapped to a ghost, walks along +grad phi) until phi
// changes sign, then halve the last step ceil(log2(step length / 0.01 h))
// times; the boundary point is the last midpoint (reading R7).  The walk's two
// ends live in registers: `far` on the node's side of the boundary, `near` the
// point before it.
__device__ bool find_boundary(const GridView &V, int i, int j, double &bx, double &by)
{
    double f;
    if (!V.at(i, j, f)) return false;
    const double side = f > 0.0 ? 1.0 : -1.0;
    const double px = V.xc(i), py = V.yc(j);
    double fx = px, fy = py, nx0 = px, ny0 = py;
    int walked = 0;
    while (side * f > 0.0) {
        double dx, dy;
        nx0 = fx;
        ny0 = fy;
        if (!normal_at(V, fx, fy, dx, dy)) return false;
        fx = fx - side * (0.5 * V.h * dx);
        fy = fy - side * (0.5 * V.h * dy);
        Patch P;
        if (!patch_at(V, fx, fy, P)) return false;
        f = P.v;
        if (++walked > MAX_MARCH) return false;
    }
    if (walked == 0) {  // phi = 0 at the node: it lies on the boundary
        bx = px;
        by = py;
        return true;
    }
    const double ex = fx - nx0, ey = fy - ny0;
    const int halvings = (int)ceil(log2(sqrt(ex * ex + ey * ey) / (0.01 * V.h)));
    double mx = fx, my = fy;
    for (int k = 0; k < halvings; k++) {
        mx = 0.5 * (fx + nx0);
        my = 0.5 * (fy + ny0);
        Patch P;
        if (!patch_at(V, mx, my, P)) return false;
        if (P.v * f < 0.0) {  // the sign change lies between the midpoint and fx
            nx0 = mx;
            ny0 = my;
        } else {
            fx = mx;
            fy = my;
            f = P.v;
        }
    }
    bx = mx;
    by = my;
    return true;
}

struct GhostRow {
    int kind, nst;
    int si[9], sj[9];
    double w[9];
    double xB, yB, thx, thy;
};

// three-point Lagrange basis on the nodes 0, 1, 2 evaluated at t (Eq. BCu)
__device__ inline double lagrange_basis(int k, double t)
{
    return k == 0 ? (1.0 - t) * (2.0 - t) / 2.0 : k == 1 ? t * (2.0 - t) : t * (t - 1.0) / 2.0;
}

// signed binomial weight (-1)^k C(n-1, k): the n-point extrapolation row
// x_0 - C(n-1,1) x_1 + ... = 0 that is exact for polynomials of degree n - 2
__device__ inline double extrap_weight(int n, int k)
{
    double c = 1.0;
    for (int q = 0; q < k; q++) c = c * (double)(n - 1 - q) / (double)(q + 1);
    return (k & 1) ? -c : c;
}

// The row of a ghost node (readings R2, R5):
//  * Eq. (BCu) on the upwind nine-point stencil for a u or v ghost that an
//    internal or box-ghost row references directly and whose boundary point B
//    is at most one cell away on both axes (theta_x, theta_y <= 1), theta =
//    SIGN(n) (x_G - x_B) / h so that stencil node k sits at theta = k;
//  * otherwise extrapolation toward the fluid along the axis where |n| is
//    largest (x on ties), four points for u, v and three for p, used only
//    when phi decreases strictly along the row's nodes;
//  * otherwise a copy of the axis neighbour with the smallest phi below
//    phi(G), the neighbours tried as -x, +x, -y, +y (first one wins a tie).
__device__ bool ghost_setup(const Geo &G, int g, int i, int j, GhostRow *R)
{
    const GridView V(G, g);
    const double gxn = V.xc(i), gyn = V.yc(j);
    double nx, ny;
    if (!normal_at(V, gxn, gyn, nx, ny)) return false;
    const int ux = nx >= 0.0 ? 1 : -1, uy = ny >= 0.0 ? 1 : -1;  // SIGN(n), SIGN(0) = 1
    R->kind = K_EXTRAP;
    R->xB = R->yB = R->thx = R->thy = 0.0;
    if (g != G_P) {
        if (!find_boundary(V, i, j, R->xB, R->yB)) return false;
        R->thx = (double)ux * (gxn - R->xB) / V.h;
        R->thy = (double)uy * (gyn - R->yB) / V.h;
        const bool direct = G.prim[(long long)g * G.F + (j + 1) * G.P + (i + 1)] != 0;
        if (direct && R->thx <= 1.0 && R->thy <= 1.0) R->kind = K_BCU;
    }
    if (R->kind == K_BCU) {
        R->nst = 9;
        for (int q = 0; q < 9; q++) {
            const int kx = q % 3, ky = q / 3;
            R->si[q] = i - kx * ux;
            R->sj[q] = j - ky * uy;
            R->w[q] = lagrange_basis(kx, R->thx) * lagrange_basis(ky, R->thy);
        }
        return true;
    }
    // extrapolation: nodes G, G - e, G - 2e (, G - 3e), e one step toward the fluid
    const bool along_x = fabs(nx) >= fabs(ny);
    const int ex = along_x ? ux : 0, ey = along_x ? 0 : uy;
    const int npts = g == G_P ? 3 : 4;
    bool falling = true;
    double prev = 0.0;
    for (int k = 0; k < npts && falling; k++) {
        double f;
        if (!V.at(i - k * ex, j - k * ey, f) || (k > 0 && !(f < prev))) falling = false;
        prev = f;
    }
    if (falling) {
        R->nst = npts;
        for (int k = 0; k < npts; k++) {
            R->si[k] = i - k * ex;
            R->sj[k] = j - k * ey;
            R->w[k] = extrap_weight(npts, k);
        }
        return true;
    }
    // copy row
    double fG;
    if (!V.at(i, j, fG)) return false;
    int bi = 0, bj = 0;
    double fbest = 0.0;
    bool found = false;
    for (int q = 0; q < 4; q++) {
        const int di = q < 2 ? 2 * q - 1 : 0, dj = q < 2 ? 0 : 2 * q - 5;  // -x, +x, -y, +y
        double f;
        if (!V.at(i + di, j + dj, f) || !(f < fG)) continue;
        if (!found || f < fbest) {
            found = true;
            fbest = f;
            bi = di;
            bj = dj;
        }
    }
    if (!found) return false;
    R->kind = K_COPY;
    R->nst = 2;
    R->si[0] = i;
    R->sj[0] = j;
    R->w[0] = 1.0;
    R->si[1] = i + bi;
    R->sj[1] = j + bj;
    R->w[1] = -1.0;
    return true;
}

// Algorithm LS's internal test with the snap of reading R4: phi < 0 and the
// first-order distance -phi / |grad phi~| above snap h
__device__ bool node_internal(const Geo &G, int g, int i, int j, double ph)
{
    if (!(ph < 0.0)) return false;
    if (G.snap <= 0.0) return true;
    const GridView V(G, g);
    Patch P;
    if (!patch_at(V, V.xc(i), V.yc(j), P)) return true;
    const double gn = sqrt(P.gx * P.gx + P.gy * P.gy);
    return ph < -G.snap * G.h * gn;
}

// node value of phi on grid g of this level (false outside the lattice)
__device__ inline bool phi_node(const Geo &G, int g, int i, int j, double *out) { return GridView(G, g).at(i, j, *out); }

__device__ inline uint8_t ttype(const Geo &G, int g, int i, int j)
{
    if (!in_grid(g, G.N, i, j)) return T_INACTIVE;
    return G.t[g][(j + 1) * G.P + (i + 1)];
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
