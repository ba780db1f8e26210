// gp_residual_static: the residual r = b - M x and ||r||_inf of one level,
// like gp_residual, but with its reduction scratch in a fixed device array of
// this library instead of the context workspace.
//
// Who needs it: callers that cannot allocate device memory, such as a plug-in
// running inside a host application that owns all device memory and hands
// out none, or a caller whose workspace was sized once for other work and
// may not grow.  This entry point calls no allocator and takes nothing from
// the workspace's reduction area.
//
// Scratch: one (sum, max) pair per frame row plus a few result slots, in
// g_static_scratch below.  Every GPU that loads the library holds this array
// (about 128 KB) until the process exits.  Levels with more than 8192 cells
// per side are rejected.  All calls share the array and it keeps the last
// call's contents; the slot that must start at zero is cleared at the start
// of each call.  Two calls whose kernels overlap on one GPU (for example on two
// streams) race on the array.  The first call on a device looks up the
// array's device address (cudaGetSymbolAddress, which may load the module);
// make that first call before any stream capture.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "gpmg_internal.cuh"

namespace gpmg {

constexpr int STATIC_MAX_ROWS = 8194;           // frame rows of N = 8192
constexpr int STATIC_SLOTS = 2 * STATIC_MAX_ROWS + 32;

// [0, 2R): per-row (sum of internal p, max |r|); [2R]: max bits of ghost
// rows; [2R + 1]: the norm
static __device__ __align__(256) double g_static_scratch[STATIC_SLOTS];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double *g_dev_ptr[MAX_DEVICES] = {nullptr};

// device address of the scratch array for the current device, looked up once
// per device with that device current
int scratch_ptr(double **out, char *msg, size_t nmsg)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        snprintf(msg, nmsg, "gp_residual_static: no current device (%s)", cudaGetErrorString(e));
        return GP_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            snprintf(msg, nmsg, "gp_residual_static: cudaGetSymbolAddress failed (%s)", cudaGetErrorString(e));
            return GP_CUDA;
        }
        g_dev_ptr[dev] = p;
    }
    *out = g_dev_ptr[dev];
    return GP_OK;
}

__device__ inline double nmax(double a, double b) { return (a != a || b != b) ? (double)NAN : fmax(a, b); }

__global__ void k_static_clear(double *s, int rows)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) s[2 * rows] = 0.0;
}

// one block per frame row: internal and inactive rows, per-row partials
__global__ void k_static_rows(int P, long long F, double q, double a, double d, const uint8_t *tU, const uint8_t *tV,
                              const uint8_t *tP, const double *x, const double *b, double *r, double *s)
{
    int row = blockIdx.x;
    double psum = 0.0, rmax = 0.0;
    const double *u = x, *v = x + F, *p = x + 2 * F;
    double xi = x[3 * F];
    for (int col = threadIdx.x; col < P; col += blockDim.x) {
        long long k = (long long)row * P + col;
        uint8_t tu = tU[k], tv = tV[k], tp = tP[k];
        if (tu == T_INTERNAL) {
            double rr = b[k] - (d * u[k] - a * (u[k + 1] + u[k - 1] + u[k + P] + u[k - P]) + q * (p[k] - p[k - 1]));
            r[k] = rr;
            rmax = nmax(rmax, fabs(rr));
        } else if (tu == T_INACTIVE) r[k] = 0.0;
        if (tv == T_INTERNAL) {
            double rr = b[F + k] - (d * v[k] - a * (v[k + 1] + v[k - 1] + v[k + P] + v[k - P]) + q * (p[k] - p[k - P]));
            r[F + k] = rr;
            rmax = nmax(rmax, fabs(rr));
        } else if (tv == T_INACTIVE) r[F + k] = 0.0;
        if (tp == T_INTERNAL) {
            double rr = b[2 * F + k] - (q * (u[k + 1] - u[k] + v[k + P] - v[k]) - xi);
            r[2 * F + k] = rr;
            rmax = nmax(rmax, fabs(rr));
            psum += p[k];
        } else if (tp == T_INACTIVE) r[2 * F + k] = 0.0;
    }
    __shared__ double ss[256], sm[256];
    ss[threadIdx.x] = psum;
    sm[threadIdx.x] = rmax;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] = nmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        s[2 * row] = ss[0];
        s[2 * row + 1] = sm[0];
    }
}

// ghost, wall and box-ghost rows; max into the bits slot
__global__ void k_static_ghosts(GhostList gh, int nrows, const double *x, const double *b, double *r, double *s, int rows)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    if (k < nrows) {
        int nst = gh.nst[k];
        int node = gh.node[k];
        double acc = b[node];
        for (int q = 0; q < nst; q++) acc -= gh.w[(long long)q * gh.cap + k] * x[gh.st[(long long)q * gh.cap + k]];
        r[node] = acc;
        m = fabs(acc);
    }
    for (int o = 16; o > 0; o >>= 1) m = nmax(m, __shfl_down_sync(0xffffffffu, m, o));
    unsigned long long *bits = (unsigned long long *)(s + 2 * rows);
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(bits, (unsigned long long)__double_as_longlong(m));
    if ((threadIdx.x & 31) == 0 && m != m) atomicMax(bits, 0x7ff8000000000000ull);
}

// mean row and the norm; one block
__global__ void k_static_final(double *s, int rows, const double *b, double *r, long long imean, double h2)
{
    __shared__ double ss[256], sm[256];
    double a = 0.0, m = 0.0;
    for (int k = threadIdx.x; k < rows; k += blockDim.x) {
        a += s[2 * k];
        m = nmax(m, s[2 * k + 1]);
    }
    ss[threadIdx.x] = a;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] = nmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double rm = b[imean] - h2 * ss[0];
        r[imean] = rm;
        double g = __longlong_as_double((long long)*(unsigned long long *)(s + 2 * rows));
        s[2 * rows + 1] = nmax(nmax(sm[0], g), fabs(rm));
    }
}

}  // namespace

int residual_static(Ctx *c, int lev, const double *x, const double *b, double *r, double *norm_host)
{
    const Level &l = c->lv[lev];
    int rows = l.N + 2;
    if (rows > STATIC_MAX_ROWS) {
        snprintf(c->msg, sizeof c->msg,
                 "gp_residual_static: level with %d cells per side exceeds the static scratch limit of 8192", l.N);
        return GP_INVALID;
    }
    double *s = nullptr;
    int st = scratch_ptr(&s, c->msg, sizeof c->msg);
    if (st != GP_OK) return st;
    cudaStream_t stream = c->stream;
    double h = c->prm.L / (double)l.N;
    double q = 1.0 / h, a = c->prm.alpha / (h * h), d = 1.0 + 4.0 * (c->prm.alpha / (h * h));
    k_static_clear<<<1, 32, 0, stream>>>(s, rows);
    k_static_rows<<<rows, 256, 0, stream>>>(l.P, l.F, q, a, d, l.tU, l.tV, l.tP, x, b, r, s);
    if (l.h_nrows > 0) k_static_ghosts<<<(l.h_nrows + 255) / 256, 256, 0, stream>>>(l.gh, l.h_nrows, x, b, r, s, rows);
    k_static_final<<<1, 256, 0, stream>>>(s, rows, b, r, 3 * l.F, h * h);
    c->launches += 3 + (l.h_nrows > 0);
    if (norm_host) {
        cudaError_t e = cudaMemcpyAsync(norm_host, s + 2 * rows + 1, sizeof(double), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            snprintf(c->msg, sizeof c->msg, "gp_residual_static: %s", cudaGetErrorString(e));
            return GP_CUDA;
        }
    }
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        snprintf(c->msg, sizeof c->msg, "gp_residual_static: %s", cudaGetErrorString(e));
        return GP_CUDA;
    }
    return GP_OK;
}

}  // namespace gpmg
