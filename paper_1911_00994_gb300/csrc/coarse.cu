// Exact solve on the coarsest grid (Sect. 4.3): the coarsest system is
// assembled densely (flat unknown order: u block, v block, p block, xi) and
// inverted once per geometry by Gauss-Jordan elimination with partial
// pivoting; each cycle then applies the inverse with one GEMV.
#include <cmath>
#include <cstdio>

#include "gpmg_internal.cuh"

namespace gpmg {

// dense rows of internal and inactive nodes (ghost-class rows and the mean
// row are written by the two kernels below); right half = identity
__global__ void k_dense_rows(double *aug, int n, const int *cmap, const int *inv, int N, int P, long long F,
                             const uint8_t *tU, const uint8_t *tV, const uint8_t *tP, double q, double a, double d)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    double *row = aug + (long long)f * 2 * n;
    for (int c = 0; c < 2 * n; c++) row[c] = 0.0;
    row[n + f] = 1.0;
    if (f == n - 1) return;  // mean row
    long long v = cmap[f];
    int g = (int)(v / F);
    long long s = v - g * F;
    const uint8_t *tt = g == G_U ? tU : g == G_V ? tV : tP;
    uint8_t t = tt[s];
    if (t == T_INACTIVE) {
        row[f] = 1.0;
        return;
    }
    if (t != T_INTERNAL) return;
    if (g == G_U || g == G_V) {
        row[inv[v]] += d;
        row[inv[v + 1]] -= a;
        row[inv[v - 1]] -= a;
        row[inv[v + P]] -= a;
        row[inv[v - P]] -= a;
        long long pm = g == G_U ? s - 1 : s - P;
        row[inv[2 * F + s]] += q;
        row[inv[2 * F + pm]] -= q;
    } else {
        row[inv[s + 1]] += q;
        row[inv[s]] -= q;
        row[inv[F + s + P]] += q;
        row[inv[F + s]] -= q;
        row[n - 1] -= 1.0;
    }
}

__global__ void k_dense_ghost_rows(double *aug, int n, const int *inv, GhostList gh, int nrows)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrows) return;
    double *row = aug + (long long)inv[gh.node[k]] * 2 * n;
    int nst = gh.nst[k];
    for (int m = 0; m < nst; m++) row[inv[gh.st[(long long)m * gh.cap + k]]] += gh.w[(long long)m * gh.cap + k];
}

__global__ void k_dense_mean_row(double *aug, int n, const int *cmap, long long F, const uint8_t *tP, double h2)
{
    if (threadIdx.x || blockIdx.x) return;
    double *row = aug + (long long)(n - 1) * 2 * n;
    for (int f = 0; f < n - 1; f++) {
        long long v = cmap[f];
        if (v >= 2 * F && v < 3 * F && tP[v - 2 * F] == T_INTERNAL) row[f] += h2;
    }
}

// pivot search in column k (first largest |a_rk|, r >= k), row swap and
// scaling of the pivot row; one block
__global__ void k_gj_pivot(double *aug, int n, int k, unsigned *err)
{
    __shared__ double bv[1024];
    __shared__ int br[1024];
    double best = -1.0;
    int brow = k;
    for (int r = k + threadIdx.x; r < n; r += blockDim.x) {
        double v = fabs(aug[(long long)r * 2 * n + k]);
        if (v > best) { best = v; brow = r; }
    }
    bv[threadIdx.x] = best;
    br[threadIdx.x] = brow;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            double v2 = bv[threadIdx.x + o];
            int r2 = br[threadIdx.x + o];
            if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && r2 < br[threadIdx.x])) {
                bv[threadIdx.x] = v2;
                br[threadIdx.x] = r2;
            }
        }
        __syncthreads();
    }
    int piv = br[0];
    double pval = aug[(long long)piv * 2 * n + k];
    if (!(bv[0] > 0.0)) {
        if (threadIdx.x == 0) atomicOr(err, E_SINGULAR);
        return;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) {
        double a = aug[(long long)piv * 2 * n + c];
        double b = aug[(long long)k * 2 * n + c];
        aug[(long long)piv * 2 * n + c] = b;
        aug[(long long)k * 2 * n + c] = a / pval;
    }
}

__global__ void k_gj_factors(const double *aug, int n, int k, double *fac)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) fac[r] = r == k ? 0.0 : aug[(long long)r * 2 * n + k];
}

__global__ void k_gj_eliminate(double *aug, int n, int k, const double *fac)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (c >= 2 * n || r == k) return;
    double f = fac[r];
    if (f != 0.0) aug[(long long)r * 2 * n + c] -= f * aug[(long long)k * 2 * n + c];
}

__global__ void k_gj_extract(const double *aug, int n, double *Minv, float *Minvf)
{
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    long long r = e / n, c = e % n;
    double v = aug[r * 2 * n + n + c];
    Minv[e] = v;
    Minvf[e] = (float)v;
}

template <typename T> __global__ void k_gather(const T *b, const int *cmap, T *cv, int n)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < n) cv[f] = b[cmap[f]];
}

template <typename T> __global__ void k_scatter(const T *cv, const int *cmap, T *x, int n)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < n) x[cmap[f]] = cv[f];
}

// y = M x, one warp per row
template <typename T> __global__ void k_gemv(const T *M, const T *x, T *y, int n)
{
    int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    const T *m = M + (long long)row * n;
    T s = 0;
    for (int c = lane; c < n; c += 32) s += m[c] * x[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
}

template <typename T> __global__ void k_zero_n(T *x, long long n)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) x[k] = 0;
}

// flat order of the coarsest level (same as the CPU reference order)
void coarse_maps_host(int N, int P, long long F, int *cmap, int *inv, long long vl)
{
    for (long long v = 0; v < vl; v++) inv[v] = -1;
    int f = 0;
    for (int j = -1; j <= N; j++)
        for (int i = 0; i <= N; i++) { cmap[f] = (int)((long long)(j + 1) * P + (i + 1)); f++; }
    for (int j = 0; j <= N; j++)
        for (int i = -1; i <= N; i++) { cmap[f] = (int)(F + (long long)(j + 1) * P + (i + 1)); f++; }
    for (int j = 0; j < N; j++)
        for (int i = 0; i < N; i++) { cmap[f] = (int)(2 * F + (long long)(j + 1) * P + (i + 1)); f++; }
    cmap[f] = (int)(3 * F);
    f++;
    for (int k = 0; k < f; k++) inv[cmap[k]] = k;
}

int build_coarse_inverse(Ctx *c)
{
    cudaStream_t st = c->stream;
    Level &l = c->lv[c->L - 1];
    int n = c->nc;
    double h = c->prm.L / (double)l.N;
    double q = 1.0 / h, a = c->prm.alpha / (h * h), d = 1.0 + 4.0 * (c->prm.alpha / (h * h));
    int *inv = c->cmap + n;
    k_dense_rows<<<(n + 127) / 128, 128, 0, st>>>(c->aug, n, c->cmap, inv, l.N, l.P, l.F, l.tU, l.tV, l.tP, q, a, d);
    if (l.h_nrows > 0) k_dense_ghost_rows<<<(l.h_nrows + 127) / 128, 128, 0, st>>>(c->aug, n, inv, l.gh, l.h_nrows);
    k_dense_mean_row<<<1, 1, 0, st>>>(c->aug, n, c->cmap, l.F, l.tP, h * h);
    cudaMemsetAsync(c->err, 0, sizeof(unsigned), st);
    dim3 ge((2 * n + 255) / 256, n);
    for (int k = 0; k < n; k++) {
        k_gj_pivot<<<1, 1024, 0, st>>>(c->aug, n, k, c->err);
        k_gj_factors<<<(n + 255) / 256, 256, 0, st>>>(c->aug, n, k, c->cvec);
        k_gj_eliminate<<<ge, 256, 0, st>>>(c->aug, n, k, c->cvec);
    }
    long long nn = (long long)n * n;
    k_gj_extract<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(c->aug, n, c->Minv, c->Minvf);
    unsigned herr = 0;
    cudaMemcpyAsync(&herr, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        snprintf(c->msg, sizeof c->msg, "coarse inverse: %s", cudaGetErrorString(e));
        return GP_CUDA;
    }
    if (herr & E_SINGULAR) {
        snprintf(c->msg, sizeof c->msg, "coarsest-level matrix is singular");
        return GP_SINGULAR;
    }
    c->coarse_ok = 1;
    c->alpha_factored = c->prm.alpha;
    return GP_OK;
}

template <typename T> const T *minv_ptr(const Ctx *c);
template <> const double *minv_ptr<double>(const Ctx *c) { return c->Minv; }
template <> const float *minv_ptr<float>(const Ctx *c) { return c->Minvf; }
template <typename T> T *cvec_ptr(const Ctx *c);
template <> double *cvec_ptr<double>(const Ctx *c) { return c->cvec; }
template <> float *cvec_ptr<float>(const Ctx *c) { return c->cvecf; }

template <typename T> void coarse_solve(Ctx *c, const T *b, T *x)
{
    cudaStream_t st = c->stream;
    const Level &l = c->lv[c->L - 1];
    int n = c->nc;
    T *cv = cvec_ptr<T>(c);
    k_zero_n<T><<<(unsigned)((l.VL + 255) / 256), 256, 0, st>>>(x, l.VL);
    k_gather<T><<<(n + 255) / 256, 256, 0, st>>>(b, c->cmap, cv, n);
    tmr_begin(c, KT_COARSE, c->L - 1);
    k_gemv<T><<<(n + 7) / 8, 256, 0, st>>>(minv_ptr<T>(c), cv, cv + n, n);
    tmr_end(c, KT_COARSE, c->L - 1);
    k_scatter<T><<<(n + 255) / 256, 256, 0, st>>>(cv + n, c->cmap, x, n);
    c->launches += 4;
}

template void coarse_solve<double>(Ctx *, const double *, double *);
template void coarse_solve<float>(Ctx *, const float *, float *);

}  // namespace gpmg
