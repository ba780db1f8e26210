// Krylov acceleration of the multigrid solve: BiCGSTAB on M x = b,
// preconditioned on the right by one multigrid cycle from zero (FP64 cycle,
// or FP32 cycle on an FP64 vector in the mixed mode), and on the adjoint
// system M^T lam = c with the transposed cycle.  Every iteration ends with
// the true residual, which also replaces the recurrence's residual.  The stopping test is
// the true residual ||b - M x||_inf after every iteration, as for the plain
// cycles.  All scalars stay on the device; one iteration is a fixed sequence
// of launches that mg_solve replays as a CUDA graph.
#include <cmath>
#include <cstdio>

#include "gpmg_internal.cuh"

namespace gpmg {

template <typename T> void residual(Ctx *c, int lev, const T *x, const T *b, T *r);
void residual_t(Ctx *c, int lev, const double *lam, const double *cc, double *r);
void cycle_t_rec(Ctx *c, int lev, double *lam, const double *cc);
void fix_inactive_t(Ctx *c, double *lam, const double *cc);
template <typename T> void cycle_rec(Ctx *c, int lev, T *x, const T *b);
template <typename T> void zero_vec(Ctx *c, T *x, long long n);
void to_float(Ctx *c, const double *a, float *b, long long n);
void float_to_double(Ctx *c, const float *e, double *y, long long n);

enum { KS_RHO = 0, KS_ALPHA = 1, KS_OMEGA = 2, KS_BETA = 3 };

constexpr int DOT_BLOCKS = 1024;

// partial sums of a.b (and of c.d when c is given), fixed grid
__global__ void k_dot_partial(const double *a, const double *b, const double *c, const double *d, long long n,
                              double *part)
{
    double s1 = 0.0, s2 = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        s1 += a[k] * b[k];
        if (c) s2 += c[k] * d[k];
    }
    __shared__ double x1[256], x2[256];
    x1[threadIdx.x] = s1;
    x2[threadIdx.x] = s2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            x1[threadIdx.x] += x1[threadIdx.x + o];
            x2[threadIdx.x] += x2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = x1[0];
        part[2 * blockIdx.x + 1] = x2[0];
    }
}

__device__ double block_sum(const double *part, int nb, int which)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) s += part[2 * k + which];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// rho_new = rh.r; beta = (rho_new / rho) (alpha / omega); rho = rho_new
__global__ void k_bicg_beta(const double *part, int nb, double *ks)
{
    double rn = block_sum(part, nb, 0);
    if (threadIdx.x == 0) {
        ks[KS_BETA] = (rn / ks[KS_RHO]) * (ks[KS_ALPHA] / ks[KS_OMEGA]);
        ks[KS_RHO] = rn;
    }
}

// alpha = rho / (rh.v) with vn = -v
__global__ void k_bicg_alpha(const double *part, int nb, double *ks)
{
    double d = block_sum(part, nb, 0);
    if (threadIdx.x == 0) ks[KS_ALPHA] = -ks[KS_RHO] / d;
}

// omega = (t.s) / (t.t) with tn = -t
__global__ void k_bicg_omega(const double *part, int nb, double *ks)
{
    double ts = block_sum(part, nb, 0);
    double tt = block_sum(part, nb, 1);
    if (threadIdx.x == 0) ks[KS_OMEGA] = -ts / tt;
}

__global__ void k_bicg_init(double *ks)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ks[KS_RHO] = 1.0;
        ks[KS_ALPHA] = 1.0;
        ks[KS_OMEGA] = 1.0;
        ks[KS_BETA] = 0.0;
    }
}

// p = r + beta (p - omega v) = r + beta (p + omega vn)
__global__ void k_bicg_p(double *p, const double *r, const double *vn, const double *ks, long long n)
{
    const double beta = ks[KS_BETA], omega = ks[KS_OMEGA];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        p[k] = r[k] + beta * (p[k] + omega * vn[k]);
}

// s = r - alpha v = r + alpha vn
__global__ void k_bicg_s(double *s, const double *r, const double *vn, const double *ks, long long n)
{
    const double alpha = ks[KS_ALPHA];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        s[k] = r[k] + alpha * vn[k];
}

// x += alpha y + omega z; r = s - omega t = s + omega tn
__global__ void k_bicg_xr(double *x, double *r, const double *y, const double *z, const double *s, const double *tn,
                          const double *ks, long long n)
{
    const double alpha = ks[KS_ALPHA], omega = ks[KS_OMEGA];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        x[k] += alpha * y[k] + omega * z[k];
        r[k] = s[k] + omega * tn[k];
    }
}

__global__ void k_to_double(const float *a, double *b, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        b[k] = (double)a[k];
}

__global__ void k_copy_vec(const double *a, double *b, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        b[k] = a[k];
}

// ------------------------------------------------------------- host side

static int vblocks(long long n)
{
    long long b = (n + 255) / 256;
    return (int)(b < 4096 ? b : 4096);
}

static void dot(Ctx *c, const double *a, const double *b, const double *cc, const double *d, long long n)
{
    int nb = (int)((n + 255) / 256 < DOT_BLOCKS ? (n + 255) / 256 : DOT_BLOCKS);
    k_dot_partial<<<nb, 256, 0, c->stream>>>(a, b, cc, d, n, c->kpart);
    c->kpart_n = nb;
    c->launches++;
}

// y = one cycle from zero applied to the vector v (FP64, or FP32 in the mixed mode)
static void precondition(Ctx *c, const double *v, double *y)
{
    Level &l0 = c->lv[0];
    long long n = l0.VL;
    if (c->prm.precision == GP_MIXED) {
        to_float(c, v, l0.bf, n);
        zero_vec<float>(c, l0.xf, n);
        cycle_rec<float>(c, 0, l0.xf, l0.bf);
        float_to_double(c, l0.xf, y, n);
    } else {
        zero_vec<double>(c, y, n);
        cycle_rec<double>(c, 0, y, v);
    }
}

// r = b - M x, rh = r, p = vn = 0, scalars 1 (x already zero on inactive nodes)
void krylov_init(Ctx *c, double *x, const double *b)
{
    Level &l0 = c->lv[0];
    long long n = l0.VL;
    residual<double>(c, 0, x, b, c->kv[0]);
    k_copy_vec<<<vblocks(n), 256, 0, c->stream>>>(c->kv[0], c->kv[1], n);
    zero_vec<double>(c, c->kv[2], n);
    zero_vec<double>(c, c->kv[3], n);
    k_bicg_init<<<1, 32, 0, c->stream>>>(c->ks);
    c->launches += 2;
}

// The same iteration on the adjoint system M^T lam = c: the operator is the
// transposed residual, the preconditioner one transposed cycle from zero
// followed by the exact solve of the inactive rows (as every iteration of
// the plain adjoint solve ends); the true residual's norm lands in
// c->red[4].  `adj` selects this form.
static void apply_op(Ctx *c, bool adj, const double *y, const double *zero, double *out)
{
    if (adj) residual_t(c, 0, y, zero, out);  // out = -M^T y
    else residual<double>(c, 0, y, zero, out);  // out = -M y
}

static void precondition_any(Ctx *c, bool adj, const double *v, double *y)
{
    if (!adj) {
        precondition(c, v, y);
        return;
    }
    zero_vec<double>(c, y, c->lv[0].VL);
    cycle_t_rec(c, 0, y, v);
    fix_inactive_t(c, y, v);
}

// r = c - M^T lam, rh = r, p = vn = 0, scalars 1
void krylov_init_t(Ctx *c, double *lam, const double *cc)
{
    Level &l0 = c->lv[0];
    long long n = l0.VL;
    fix_inactive_t(c, lam, cc);
    residual_t(c, 0, lam, cc, c->kv[0]);
    k_copy_vec<<<vblocks(n), 256, 0, c->stream>>>(c->kv[0], c->kv[1], n);
    zero_vec<double>(c, c->kv[2], n);
    zero_vec<double>(c, c->kv[3], n);
    k_bicg_init<<<1, 32, 0, c->stream>>>(c->ks);
    c->launches += 2;
}

static void bicg_iteration(Ctx *c, bool adj, double *x, const double *b);

// one BiCGSTAB iteration and the true residual of x (norm in c->red[0])
void krylov_iteration(Ctx *c, double *x, const double *b) { bicg_iteration(c, false, x, b); }

// one BiCGSTAB iteration on M^T lam = c (norm in c->red[4])
void krylov_iteration_t(Ctx *c, double *lam, const double *cc) { bicg_iteration(c, true, lam, cc); }

static void bicg_iteration(Ctx *c, bool adj, double *x, const double *b)
{
    Level &l0 = c->lv[0];
    long long n = l0.VL;
    double *r = c->kv[0], *rh = c->kv[1], *p = c->kv[2], *vn = c->kv[3], *s = c->kv[4], *tn = c->kv[5];
    double *y = c->kv[6], *z = c->kv[7], *zero = c->kv[8];
    int vb = vblocks(n);
    dot(c, rh, r, nullptr, nullptr, n);
    k_bicg_beta<<<1, 256, 0, c->stream>>>(c->kpart, c->kpart_n, c->ks);
    k_bicg_p<<<vb, 256, 0, c->stream>>>(p, r, vn, c->ks, n);
    precondition_any(c, adj, p, y);
    apply_op(c, adj, y, zero, vn);  // vn = -M y (or -M^T y)
    dot(c, rh, vn, nullptr, nullptr, n);
    k_bicg_alpha<<<1, 256, 0, c->stream>>>(c->kpart, c->kpart_n, c->ks);
    k_bicg_s<<<vb, 256, 0, c->stream>>>(s, r, vn, c->ks, n);
    precondition_any(c, adj, s, z);
    apply_op(c, adj, z, zero, tn);  // tn = -M z (or -M^T z)
    dot(c, tn, s, tn, tn, n);
    k_bicg_omega<<<1, 256, 0, c->stream>>>(c->kpart, c->kpart_n, c->ks);
    k_bicg_xr<<<vb, 256, 0, c->stream>>>(x, r, y, z, s, tn, c->ks, n);
    // residual replacement: the recurrence continues from the true residual
    // b - M x (whose norm is the stopping test), so that rounding accumulated
    // in the recurrence cannot hold the true residual above the tolerance
    if (adj) residual_t(c, 0, x, b, r);
    else residual<double>(c, 0, x, b, r);
    c->launches += 6;
}

}  // namespace gpmg
