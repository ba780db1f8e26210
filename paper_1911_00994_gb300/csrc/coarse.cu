// Exact solve on the coarsest grid (Sect. 4.3): the coarsest system is
// assembled densely (flat unknown order: u block, v block, p block, xi) and
// inverted once per geometry by Gauss-Jordan elimination with partial
// pivoting (one launch per column); each cycle then applies the inverse with
// one GEMV.
#include <cmath>
#include <cstdio>

#include "gpmg_internal.cuh"

namespace gpmg {

// dense rows of internal and inactive nodes (ghost-class rows and the mean
// row are written by the two kernels below); right half zero (the
// elimination fills it)
__global__ void k_dense_rows(double *aug, int n, const int *cmap, const int *inv, int N, int P, long long F,
                             const uint8_t *tU, const uint8_t *tV, const uint8_t *tP, double q, double a, double d)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    double *row = aug + (long long)f * 2 * n;
    for (int c = 0; c < 2 * n; c++) row[c] = 0.0;
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

// Gauss-Jordan elimination with partial pivoting, one launch per column and
// no row exchanges or scaling: step k eliminates column k from every row
// but the pivot row p_k (the unused row with the largest |a_ik|), which
// keeps its place and scale.  The right half is kept in pivot order: its
// slot t holds column p_t of the transformed identity, which is the unit
// column e_(p_t) until step t, so step k touches the n - k - 1 remaining
// left columns and the k + 1 filled slots (n columns in all).  Afterwards
// row p_k holds a_(p_k,k) in the left half, and row k of the inverse is
// a_(p_k,k)^-1 times row p_k of the right half, slot t giving column p_t.
// The pivot of column k + 1 is chosen during step k from the updated column:
// keys[k + 1] is the atomic maximum of (top 32 bits of |a_i,k+1|, ~i) over
// the rows not yet used, so the first of equally large candidates wins.

__device__ __forceinline__ unsigned long long pivot_key(double v, int i)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(v));
    return ((bits >> 32) << 32) | (unsigned long long)(0xffffffffu - (unsigned)i);
}

__device__ __forceinline__ int pivot_row(unsigned long long key) { return (int)(0xffffffffu - (unsigned)key); }

// pivot of column 0
__global__ void k_gj_first(const double *aug, int n, unsigned long long *keys)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const unsigned long long key = pivot_key(aug[(long long)i * 2 * n], i);
        if (key >> 32) atomicMax(keys, key);
    }
}

// step k over a 128-column x 8-row tile per block (a warp covers 4 x 32
// columns of one row, 32 consecutive ones per pass); column c < n - k - 1 is
// left column k + 1 + c, the others are right-half slots c - (n - k - 1)
__global__ void __launch_bounds__(256) k_gj_step(double *aug, int n, int k, unsigned long long *keys, uint8_t *used,
                                                 unsigned *err)
{
    const long long W = 2LL * n;
    const int i = blockIdx.y * 8 + threadIdx.y;
    const unsigned long long key = keys[k];
    if (!(key >> 32)) {  // no nonzero candidate in column k
        if (threadIdx.x == 0 && threadIdx.y == 0 && blockIdx.x == 0 && blockIdx.y == 0) atomicOr(err, E_SINGULAR);
        return;
    }
    const int p = pivot_row(key);
    __shared__ double s_rp;
    __shared__ unsigned long long s_best[8];
    if (threadIdx.x == 0 && threadIdx.y == 0) s_rp = 1.0 / aug[(long long)p * W + k];
    __syncthreads();
    unsigned long long cand = 0;
    const int nleft = n - k - 1;
    if (i < n) {
        const double m = i != p ? aug[(long long)i * W + k] * s_rp : 0.0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int c = blockIdx.x * 128 + q * 32 + threadIdx.x;
            if (c >= n) continue;
            const long long j = c < nleft ? k + 1 + c : n + (c - nleft);  // element column
            if (c < nleft || c - nleft < k) {
                if (i != p) {
                    double v = aug[(long long)i * W + j];
                    if (m != 0.0) v -= m * aug[(long long)p * W + j];
                    aug[(long long)i * W + j] = v;
                    if (c == 0 && !used[i]) cand = pivot_key(v, i);
                }
            } else {
                // slot k: the unit column e_p after this step's elimination
                aug[(long long)i * W + j] = i == p ? 1.0 : -m;
            }
            if (i == p && c == n - 1) used[p] = 1;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long c2 = __shfl_xor_sync(0xffffffffu, cand, o);
        cand = c2 > cand ? c2 : cand;
    }
    if (threadIdx.x == 0) s_best[threadIdx.y] = cand;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        unsigned long long best = 0;
        for (int y = 0; y < 8; y++) best = s_best[y] > best ? s_best[y] : best;
        if (best >> 32) atomicMax(keys + k + 1, best);
    }
}

// row r of the inverse from the pivot row of column r: slot t gives column p_t
__global__ void k_gj_extract(const double *aug, int n, const unsigned long long *keys, double *Minv, float *Minvf)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    const long long r = e / n, t = e % n;
    const unsigned long long kr = keys[r], kt = keys[t];
    // a singular matrix (flagged by the steps) leaves later keys empty
    if (!(kr >> 32) || !(kt >> 32)) {
        Minv[e] = 0.0;
        Minvf[e] = 0.0f;
        return;
    }
    const int p = pivot_row(kr), col = pivot_row(kt);
    const double v = aug[(long long)p * 2 * n + n + t] / aug[(long long)p * 2 * n + r];
    Minv[r * n + col] = v;
    Minvf[r * n + col] = (float)v;
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

// the elimination of the assembled [M | I]: its arguments are fixed for the
// context, so it is captured once as a CUDA graph and replayed for every
// geometry
static void gj_launches(Ctx *c)
{
    cudaStream_t st = c->stream;
    const int n = c->nc;
    cudaMemsetAsync(c->err, 0, sizeof(unsigned), st);
    cudaMemsetAsync(c->gjkeys, 0, sizeof(unsigned long long) * n, st);
    cudaMemsetAsync(c->gjused, 0, n, st);
    k_gj_first<<<(n + 255) / 256, 256, 0, st>>>(c->aug, n, c->gjkeys);
    const dim3 ge((n + 127) / 128, (n + 7) / 8), be(32, 8);
    for (int k = 0; k < n; k++) k_gj_step<<<ge, be, 0, st>>>(c->aug, n, k, c->gjkeys, c->gjused, c->err);
    const long long nn = (long long)n * n;
    k_gj_extract<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(c->aug, n, c->gjkeys, c->Minv, c->Minvf);
}

// replay the captured elimination; false when graphs are unavailable here
static bool gj_graph(Ctx *c)
{
    if (!c->prm.graphs || c->graphs_off || c->stream == nullptr) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;
    }
    if (!c->gj_exec) {
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        gj_launches(c);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gj_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->gj_exec = nullptr;
            return false;
        }
    }
    if (cudaGraphLaunch(c->gj_exec, c->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(c->gj_exec);
        c->gj_exec = nullptr;
        return false;
    }
    return true;
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
    if (!gj_graph(c)) gj_launches(c);
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
