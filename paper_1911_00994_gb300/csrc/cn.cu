// One Crank-Nicolson step (Sect. 2): convective term, right-hand side of the
// linear system (Eqs. NSCN1, spaceprob), mid-point Picard iteration for the
// first two steps (Eqs. NSitconv, iterativeNS) and extrapolation of the
// convective term afterwards (Eq. extrUdU).  FP64 on the finest level.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "gpmg_internal.cuh"

namespace gpmg {

// N = u . grad u at internal u and v nodes, zero on every other slot of the
// vector (the p frame and the scalars included).
// mode 0: out = N(x); mode 1: out = (Nn + N(x)) / 2
__global__ void k_convective(int P, long long F, double h, const uint8_t *tU, const uint8_t *tV, const double *x,
                             const double *Nn, double *out, int mode)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= P) return;
    long long s = (long long)row * P + col;
    const double *u = x, *v = x + F;
    double nu = 0.0, nv = 0.0;
    if (tU[s] == T_INTERNAL) {
        // v at (i-1, j), (i, j), (i-1, j+1), (i, j+1) relative to u(i, j)
        double vb = 0.25 * (v[s - 1] + v[s] + v[s + P - 1] + v[s + P]);
        nu = u[s] * ((u[s + 1] - u[s - 1]) / (2.0 * h)) + vb * ((u[s + P] - u[s - P]) / (2.0 * h));
    }
    if (tV[s] == T_INTERNAL) {
        // u at (i, j-1), (i+1, j-1), (i, j), (i+1, j) relative to v(i, j)
        double ub = 0.25 * (u[s - P] + u[s - P + 1] + u[s] + u[s + 1]);
        nv = ub * ((v[s + 1] - v[s - 1]) / (2.0 * h)) + v[s] * ((v[s + P] - v[s - P]) / (2.0 * h));
    }
    if (mode == 1) {
        nu = 0.5 * (Nn[s] + nu);
        nv = 0.5 * (Nn[F + s] + nv);
    }
    out[s] = nu;
    out[F + s] = nv;
    out[2 * F + s] = 0.0;
    if (row == 0 && col < NSCAL) out[3 * F + col] = 0.0;
}

// Nh = Nn + N1/2 - N2/2 on the u, v frames
__global__ void k_extrapolate(long long n, const double *Nn, const double *N1, const double *N2, double *Nh)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) Nh[k] = Nn[k] + 0.5 * N1[k] - 0.5 * N2[k];
}

// internal momentum rows b = u^n + alpha lap u^n + dt f - dt Nh; every other
// slot of the vector 0 (ghost-class rows are filled by k_cn_rhs_bc)
__global__ void k_cn_rhs(int P, long long F, double a, double dt, const uint8_t *tU, const uint8_t *tV,
                         const uint8_t *tP, const double *xn, const double *Nh, const double *f, const double *g,
                         double *b)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= P) return;
    long long s = (long long)row * P + col;
    for (int g = 0; g < 2; g++) {
        long long k = g * F + s;
        double val = 0.0;
        if ((g == 0 ? tU[s] : tV[s]) == T_INTERNAL) {
            double lap = xn[k + 1] + xn[k - 1] + xn[k + P] + xn[k - P] - 4.0 * xn[k];
            val = xn[k] + a * lap + dt * (f ? f[k] : 0.0) - dt * Nh[k];
        }
        b[k] = val;
    }
    // continuity rows: div u - xi = g (g = 0 unless a source is set)
    b[2 * F + s] = (g && tP[s] == T_INTERNAL) ? g[2 * F + s] : 0.0;
    if (row == 0 && col == 0)
        for (int q = 0; q < NSCAL; q++) b[3 * F + q] = 0.0;
}

// ghost-class rows: Eq. (BCu) rows take the boundary velocity at B (from the
// vector bc when given, else the rigid-body motion), wall and box-ghost rows
// the wall velocity (bc, else the walls), extrapolation and copy rows 0
__global__ void k_cn_rhs_bc(GhostList gh, int nrows, int nobj, long long F, int N, int P, const double *bc, gp_body body,
                            gp_walls walls, double *b)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrows) return;
    int node = gh.node[k];
    int kind = gh.kind[k];
    double val = 0.0;
    if (bc) {
        if (kind == K_BCU || kind == K_WALL || kind == K_BOXGHOST) val = bc[node];
    } else if (kind == K_BCU) {
        double xB = gh.B[k], yB = gh.B[gh.cap + k];
        val = node < F ? body.U - body.omega * (yB - body.cy) : body.V + body.omega * (xB - body.cx);
    } else if (kind == K_BOXGHOST) {
        int g = node < F ? 0 : 1;
        long long s = node - g * F;
        int row = (int)(s / P), col = (int)(s % P);
        if (g == 0) val = row == 0 ? walls.u_bottom : walls.u_top;
        else val = col == 0 ? walls.v_left : walls.v_right;
    }
    b[node] = val;
    (void)nobj;
    (void)N;
}

// max |b - M x| and max |b| over internal momentum rows (Eq. iterativeNS)
__global__ void k_mom_residual_max(int P, long long F, double q, double a, double d, const uint8_t *tU, const uint8_t *tV,
                                   const double *x, const double *b, unsigned long long *bits)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    double rm = 0.0, bm = 0.0;
    if (col < P) {
        long long s = (long long)row * P + col;
        const double *u = x, *v = x + F, *p = x + 2 * F;
        if (tU[s] == T_INTERNAL) {
            double r = b[s] - (d * u[s] - a * (u[s + 1] + u[s - 1] + u[s + P] + u[s - P]) + q * (p[s] - p[s - 1]));
            rm = fabs(r);
            bm = fabs(b[s]);
        }
        if (tV[s] == T_INTERNAL) {
            double r = b[F + s] - (d * v[s] - a * (v[s + 1] + v[s - 1] + v[s + P] + v[s - P]) + q * (p[s] - p[s - P]));
            rm = fmax(rm, fabs(r));
            bm = fmax(bm, fabs(b[F + s]));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        rm = fmax(rm, __shfl_down_sync(0xffffffffu, rm, o));
        bm = fmax(bm, __shfl_down_sync(0xffffffffu, bm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (rm > 0.0 || rm != rm) atomicMax(&bits[0], (unsigned long long)__double_as_longlong(rm != rm ? (double)INFINITY : rm));
        if (bm > 0.0) atomicMax(&bits[1], (unsigned long long)__double_as_longlong(bm));
    }
}

__global__ void k_copy(const double *a, double *b, long long n)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) b[k] = a[k];
}

// ------------------------------------------------- adjoint of the CN step

// out += J_N(x)^T y on the u, v frames: the transpose of the linearised
// convective term at x, as a gather over the rows that reference each node
// (u rows at s, s +- 1, s +- P and the v rows whose averaged u holds u(s);
// likewise for v).  y is read on internal u, v rows only.
__global__ void k_convective_jt(int P, long long F, int R, double h, const uint8_t *tU, const uint8_t *tV,
                                const double *x, const double *y, double *out)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= P) return;
    const long long s = (long long)row * P + col, NS = (long long)R * P;
    const double *u = x, *v = x + F, *yu = y, *yv = y + F;
    const double h2 = 2.0 * h;
    auto iu = [&](long long r) { return r >= 0 && r < NS && tU[r] == T_INTERNAL; };
    auto iv = [&](long long r) { return r >= 0 && r < NS && tV[r] == T_INTERNAL; };
    auto vbar = [&](long long r) { return 0.25 * (v[r - 1] + v[r] + v[r + P - 1] + v[r + P]); };
    auto ubar = [&](long long r) { return 0.25 * (u[r - P] + u[r - P + 1] + u[r] + u[r + 1]); };
    double su = 0.0, sv = 0.0;
    if (iu(s)) su += yu[s] * ((u[s + 1] - u[s - 1]) / h2);
    if (iu(s - 1)) su += yu[s - 1] * u[s - 1] / h2;
    if (iu(s + 1)) su -= yu[s + 1] * u[s + 1] / h2;
    if (iu(s - P)) su += yu[s - P] * vbar(s - P) / h2;
    if (iu(s + P)) su -= yu[s + P] * vbar(s + P) / h2;
    const long long rv[4] = {s + P, s + P - 1, s, s - 1};
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (iv(rv[q])) su += 0.25 * yv[rv[q]] * ((v[rv[q] + 1] - v[rv[q] - 1]) / h2);
    if (iv(s)) sv += yv[s] * ((v[s + P] - v[s - P]) / h2);
    if (iv(s - 1)) sv += yv[s - 1] * ubar(s - 1) / h2;
    if (iv(s + 1)) sv -= yv[s + 1] * ubar(s + 1) / h2;
    if (iv(s - P)) sv += yv[s - P] * v[s - P] / h2;
    if (iv(s + P)) sv -= yv[s + P] * v[s + P] / h2;
    const long long ru[4] = {s + 1, s, s - P + 1, s - P};
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (iu(ru[q])) sv += 0.25 * yu[ru[q]] * ((u[ru[q] + P] - u[ru[q] - P]) / h2);
    out[s] += su;
    out[F + s] += sv;
}

// out += A^T y, A x = x + alpha lap x on the internal u, v rows
__global__ void k_explicit_t(int P, long long F, int R, double a, const uint8_t *tU, const uint8_t *tV,
                             const double *y, double *out)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= P) return;
    const long long s = (long long)row * P + col, NS = (long long)R * P;
#pragma unroll
    for (int g = 0; g < 2; g++) {
        const uint8_t *t = g == 0 ? tU : tV;
        const double *yy = y + g * F;
        double acc = 0.0;
        if (t[s] == T_INTERNAL) acc += (1.0 - 4.0 * a) * yy[s];
        const long long nb[4] = {s + 1, s - 1, s + P, s - P};
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (nb[q] >= 0 && nb[q] < NS && t[nb[q]] == T_INTERNAL) acc += a * yy[nb[q]];
        out[g * F + s] += acc;
    }
}

// el = lam on internal u, v rows (0 elsewhere on the u, v frames)
__global__ void k_mask_mom(int P, long long F, const uint8_t *tU, const uint8_t *tV, const double *lam, double *el)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= P) return;
    const long long s = (long long)row * P + col;
    el[s] = tU[s] == T_INTERNAL ? lam[s] : 0.0;
    el[F + s] = tV[s] == T_INTERNAL ? lam[F + s] : 0.0;
}

// acc_q += c_q el on the u, v frames for up to four (acc, c) pairs
__global__ void k_axpy4(long long n, const double *el, double *a0, double c0, double *a1, double c1, double *a2,
                        double c2, double *a3, double c3)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double e = el[k];
    if (a0) a0[k] += c0 * e;
    if (a1) a1[k] += c1 * e;
    if (a2) a2[k] += c2 * e;
    if (a3) a3[k] += c3 * e;
}

// out[0] = sum over ghost-class rows of g * lam (one block, fixed order)
__global__ void k_dot_rows(const int *node, int n, const double *g, const double *lam, double *out)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += g[node[k]] * lam[node[k]];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// ------------------------------------------------------------- host side

static dim3 fgrid(const Level &l) { return dim3((l.P + 255) / 256, l.N + 2); }

void cn_convective(Ctx *c, const double *x, const double *Nn, double *out, int mode)
{
    const Level &l = c->lv[0];
    k_convective<<<fgrid(l), 256, 0, c->stream>>>(l.P, l.F, l.h, l.tU, l.tV, x, Nn, out, mode);
    c->launches++;
}

void cn_rhs(Ctx *c, const double *xn, const double *Nh, const double *f, double dt, const double *bc, const gp_body &body,
            const gp_walls &walls, double *b)
{
    const Level &l = c->lv[0];
    double a = c->prm.alpha / (l.h * l.h);
    k_cn_rhs<<<fgrid(l), 256, 0, c->stream>>>(l.P, l.F, a, dt, l.tU, l.tV, l.tP, xn, Nh, f, c->csrc, b);
    if (l.h_nrows > 0)
        k_cn_rhs_bc<<<(l.h_nrows + 255) / 256, 256, 0, c->stream>>>(l.gh, l.h_nrows, l.h_nghost, l.F, l.N, l.P, bc, body,
                                                                      walls, b);
    c->launches += 1 + (l.h_nrows > 0);
}

// returns max |b - M x| and max |b| over internal momentum rows (syncs)
int cn_momentum_residual(Ctx *c, const double *x, const double *b, double *res, double *bmax)
{
    const Level &l = c->lv[0];
    double q = 1.0 / l.h, a = c->prm.alpha / (l.h * l.h), d = 1.0 + 4.0 * a;
    unsigned long long *bits = c->maxbits + 2;
    cudaMemsetAsync(bits, 0, 2 * sizeof(unsigned long long), c->stream);
    k_mom_residual_max<<<fgrid(l), 256, 0, c->stream>>>(l.P, l.F, q, a, d, l.tU, l.tV, x, b, bits);
    c->launches++;
    unsigned long long hb[2] = {0, 0};
    cudaMemcpyAsync(hb, bits, sizeof hb, cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return GP_CUDA;
    double r, m;
    memcpy(&r, &hb[0], 8);
    memcpy(&m, &hb[1], 8);
    *res = r;
    *bmax = m;
    return GP_OK;
}

void cn_extrapolate(Ctx *c, const double *Nn, const double *N1, const double *N2, double *Nh)
{
    long long n = 2 * c->lv[0].F;
    k_extrapolate<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, Nn, N1, N2, Nh);
    c->launches++;
}

void cn_copy(Ctx *c, const double *a, double *b, long long n)
{
    k_copy<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(a, b, n);
    c->launches++;
}

void cn_convective_jt(Ctx *c, const double *x, const double *y, double *out)
{
    const Level &l = c->lv[0];
    k_convective_jt<<<fgrid(l), 256, 0, c->stream>>>(l.P, l.F, l.N + 2, l.h, l.tU, l.tV, x, y, out);
    c->launches++;
}

void cn_explicit_t(Ctx *c, const double *y, double *out)
{
    const Level &l = c->lv[0];
    k_explicit_t<<<fgrid(l), 256, 0, c->stream>>>(l.P, l.F, l.N + 2, c->prm.alpha / (l.h * l.h), l.tU, l.tV, y, out);
    c->launches++;
}

void cn_mask_mom(Ctx *c, const double *lam, double *el)
{
    const Level &l = c->lv[0];
    k_mask_mom<<<fgrid(l), 256, 0, c->stream>>>(l.P, l.F, l.tU, l.tV, lam, el);
    c->launches++;
}

void cn_axpy4(Ctx *c, const double *el, double *a0, double c0, double *a1, double c1, double *a2, double c2,
              double *a3, double c3)
{
    long long n = 2 * c->lv[0].F;
    k_axpy4<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, el, a0, c0, a1, c1, a2, c2, a3, c3);
    c->launches++;
}

// sum over the ghost-class rows of the finest level of g * lam (into out, device)
void cn_dot_rows(Ctx *c, const double *g, const double *lam, double *out)
{
    const Level &l = c->lv[0];
    k_dot_rows<<<1, 256, 0, c->stream>>>(l.gh.node, l.h_nrows, g, lam, out);
    c->launches++;
}

}  // namespace gpmg
