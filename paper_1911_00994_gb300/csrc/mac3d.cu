// The 3-D MAC extension on the box domain (include/gpmg3d.h): node types,
// the rows of the Crank-Nicolson system in 3-D, seven-colour 7 x 7 box
// relaxation, the (xi, mean) update, Jacobi sweeps over the wall and
// box-ghost rows, class-aware restriction, trilinear prolongation, a dense
// inverse of the coarsest level built on the device, and V-cycles.
//
// Every level keeps all four grids in one index space of (N + 2)^3 slots,
// slot ((k + 1) S + (j + 1)) S + (i + 1) with S = N + 2, so that the
// neighbours of any node are at +-1, +-S, +-S^2 on every grid.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/gpmg3d.h"

namespace gp3 {

constexpr int NSCAL = 32;
constexpr int NCOL = 7;            // box colours (i + 2 j + 3 k) mod 7
constexpr int MAX_LEVELS = 12;
constexpr int COARSE_MAX = 1024;   // unknowns of the coarsest level's dense inverse
enum : unsigned char { T_INACTIVE = 0, T_INTERNAL = 1, T_WALL = 3, T_BOXGHOST = 4 };

struct Lev {
    int N, S;
    long long F, VL;
    double a, q, d, h3;  // alpha / h^2, 1 / h, 1 + 6 a, h^3
    double ida, id, idet;  // 1 / (d + a), 1 / d, 1 / (d^2 - a^2): the box solves divide only once
    unsigned char *t;    // 4 F node types
    double *x, *b, *r;   // FP64 level vectors (x, b of the coarse levels; r of every level)
    float *xf, *bf, *rf; // FP32 level vectors of the mixed mode's inner cycles (x, b, r of every level)
    long long *gl;       // the wall and box-ghost rows (vector entries), listed once at creation
    int ng;              // how many
};

// wall and box-ghost rows of a level with N cells per side: per grid 2 N^2
// on its own walls and 4 N (N - 1) half a cell outside the others
__host__ __device__ inline long long ghost_cap(int N) { return 18LL * N * N; }

__host__ __device__ inline long long vlen(int N)
{
    const long long S = N + 2;
    return 4 * S * S * S + NSCAL;
}

// ------------------------------------------------------------ node types

// coordinate of slot s along array axis ax (0: i, 1: j, 2: k), in [-1, N]
// (32-bit: a frame has fewer than 2^31 slots for N <= 1024)
__device__ inline int coord(long long s, int S, int ax)
{
    const unsigned u = (unsigned)s, US = (unsigned)S;
    if (ax == 0) return (int)(u % US) - 1;
    if (ax == 1) return (int)((u / US) % US) - 1;
    return (int)(u / (US * US)) - 1;
}

// the frame (0 u, 1 v, 2 w, 3 p) of vector entry e < 4 F
__device__ inline int frame_of(long long e, long long F)
{
    return e < F ? 0 : e < 2 * F ? 1 : e < 3 * F ? 2 : 3;
}

__global__ void k3_types(int N, long long F, unsigned char *t)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= 4 * F) return;
    const int g = frame_of(e, F);
    const long long s = e - g * F;
    const int S = N + 2;
    int c[3] = {coord(s, S, 0), coord(s, S, 1), coord(s, S, 2)};
    auto inside = [&](int v) { return v >= 0 && v <= N - 1; };
    unsigned char ty = T_INACTIVE;
    if (g == 3) {
        if (inside(c[0]) && inside(c[1]) && inside(c[2])) ty = T_INTERNAL;
    } else {
        // own axis g: faces 0..N; the two transverse axes: cells
        const int own = c[g], t1 = c[(g + 1) % 3], t2 = c[(g + 2) % 3];
        const bool face_ok = own >= 0 && own <= N, interior = own >= 1 && own <= N - 1;
        const bool in1 = inside(t1), in2 = inside(t2);
        const bool out1 = t1 == -1 || t1 == N, out2 = t2 == -1 || t2 == N;
        if (face_ok && in1 && in2) ty = interior ? T_INTERNAL : T_WALL;
        else if (interior && ((out1 && in2) || (out2 && in1))) ty = T_BOXGHOST;
    }
    t[e] = ty;
}

// ------------------------------------------------------------ the rows

// (M x) of the velocity or continuity row at slot s of grid g (not the mean
// row); X(e) returns entry e of the vector (a level vector, or a unit
// vector when the dense matrix is assembled)
template <typename T, typename Acc>
__device__ inline T apply_row(const Lev &L, const unsigned char *t, int g, long long s, const Acc &X)
{
    const long long F = L.F, S = L.S, S2 = S * S;
    const T q = (T)L.q, d = (T)L.d, a = (T)L.a;
    // the slot stride along axis ax (selected, not indexed: no local array)
    auto off = [&](int ax) -> long long { return ax == 0 ? 1 : ax == 1 ? S : S2; };
    const unsigned char ty = t[g * F + s];
    const long long e = g * F + s;
    if (g == 3) {
        if (ty != T_INTERNAL) return X(e);
        // continuity: q (u_E - u_W + v_N - v_S + w_T - w_B) - xi
        return q * ((X(s + 1) - X(s)) + (X(F + s + S) - X(F + s)) + (X(2 * F + s + S2) - X(2 * F + s))) - X(4 * F);
    }
    if (ty == T_INTERNAL) {
        const T lap = X(e + 1) + X(e - 1) + X(e + S) + X(e - S) + X(e + S2) + X(e - S2);
        // p of the cell on the + side (same slot) minus the cell on the - side
        return d * X(e) - a * lap + q * (X(3 * F + s) - X(3 * F + s - off(g)));
    }
    if (ty == T_BOXGHOST) {
        // the transverse axis that leaves [0, N): step inwards from the ghost
        const int N = L.N;
        long long in = 0;
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            if (ax == g) continue;
            const int c = coord(s, L.S, ax);
            if (c == -1) in = off(ax);
            else if (c == N) in = -off(ax);
        }
        return (T)0.375 * X(e) + (T)0.75 * X(e + in) - (T)0.125 * X(e + 2 * in);
    }
    return X(e);  // wall (Dirichlet) and inactive rows
}

template <typename T> struct VecAcc {
    const T *v;
    __device__ T operator()(long long e) const { return v[e]; }
};
struct UnitAcc {
    long long c;
    __device__ double operator()(long long e) const { return e == c ? 1.0 : 0.0; }
};

// |v| as the bits of v with the sign cleared, and back
template <typename T> struct AbsBits3;
template <> struct AbsBits3<float> {
    typedef unsigned int U;
    __device__ static U of(float v) { return __float_as_uint(v) & 0x7fffffffu; }
    __device__ static double value(U u) { return (double)__uint_as_float(u); }
};
template <> struct AbsBits3<double> {
    typedef unsigned long long U;
    __device__ static U of(double v) { return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull; }
    __device__ static double value(U u) { return __longlong_as_double((long long)u); }
};

// a sum and a NaN-keeping maximum over a block of 256 threads; thread 0
// writes part[2 b], part[2 b + 1]
__device__ inline void block_sum_max(double s, double m, double *part)
{
    __shared__ double ss[256], sm[256];
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            const double a = sm[threadIdx.x], b = sm[threadIdx.x + o];
            sm[threadIdx.x] = (a != a || b != b) ? (double)NAN : fmax(a, b);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = ss[0];
        part[2 * blockIdx.x + 1] = sm[0];
    }
}

// r = b - M x over the four frames; per block [0] sum of the interior p,
// [1] max |r| (grid-stride)
// (T: the arithmetic; R: the output, FP32 when the FP64 residual becomes the
// right-hand side of the inner FP32 cycles)
template <typename T, typename R>
__global__ void __launch_bounds__(256) k3_residual(Lev L, const T *x, const T *b, R *r, double *part)
{
    const VecAcc<T> X{x};
    // per thread: the sum of p in T and max |r| as the integer maximum of
    // sign-cleared bits (the numeric order for non-negative floats, NaN
    // above infinity), so an FP32 residual does no FP64 work per entry
    T sp = 0;
    typename AbsBits3<T>::U mb = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 4 * L.F;
         e += (long long)gridDim.x * blockDim.x) {
        const int g = frame_of(e, L.F);
        const long long s = e - g * L.F;
        const T v = b[e] - apply_row<T>(L, L.t, g, s, X);
        r[e] = (R)v;
        mb = max(mb, AbsBits3<T>::of(v));
        if (g == 3 && L.t[e] == T_INTERNAL) sp += x[e];
    }
    block_sum_max((double)sp, AbsBits3<T>::value(mb), part);
}

// the mean row and the norm: r[4F] = b[4F] - h^3 sum p
template <typename T, typename R>
__global__ void k3_residual_final(Lev L, const double *part, int nb, const T *b, R *r, double *out)
{
    __shared__ double ss[256], sm[256];
    double s = 0.0, m = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        s += part[2 * k];
        const double v = part[2 * k + 1];
        m = (v != v || m != m) ? (double)NAN : fmax(m, v);
    }
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            const double a = sm[threadIdx.x], c = sm[threadIdx.x + o];
            sm[threadIdx.x] = (a != a || c != c) ? (double)NAN : fmax(a, c);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double rm = (double)b[4 * L.F] - L.h3 * ss[0];
        r[4 * L.F] = (R)rm;
        const double a = sm[0];
        out[0] = (a != a || rm != rm) ? (double)NAN : fmax(a, fabs(rm));
    }
}

// ------------------------------------------------------------ relaxation

// One colour of box relaxation (Sect. 4.1.1 in 3-D): the box of cell
// (i, j, k) holds p and its interior faces W, E (u), S, N (v), B, T (w);
// everything else is frozen.  Eliminating the faces leaves one equation for
// the pressure correction: per direction, both faces couple through -a and
// give q (r_hi - r_lo + 2 q dp) / (d + a) to the continuity row, a single
// face -q (r_lo - q dp) / d or q (r_hi + q dp) / d (with the level's
// reciprocals: one division per box).  One thread per cell of the colour,
// cells numbered along i within each (j, k) row.
template <typename T>
__global__ void __launch_bounds__(256) k3_box(Lev L, T *x, const T *b, int colour)
{
    const int N = L.N;
    const unsigned per_row = (N + NCOL - 1) / NCOL;
    const unsigned n = per_row * N * N;  // below 2^31 for N <= 1024
    const unsigned id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int m = (int)(id % per_row);
    const unsigned jk = id / per_row;
    const int j = (int)(jk % (unsigned)N), k = (int)(jk / (unsigned)N);
    // first i with (i + 2 j + 3 k) mod 7 = colour
    const int i = (int)((unsigned)(colour + 7 * 4 * (N + 1) - 2 * j - 3 * k) % 7u) + NCOL * m;
    if (i >= N) return;
    const long long S = L.S, S2 = S * S, F = L.F;
    const long long s = ((long long)(k + 1) * S + (j + 1)) * S + (i + 1);
    const VecAcc<T> X{x};
    // faces: lo and hi of each direction
    const long long fe[6] = {s, s + 1, F + s, F + s + S, 2 * F + s, 2 * F + s + S2};
    bool on[6];
    T r[6];
#pragma unroll
    for (int f = 0; f < 6; f++) {
        on[f] = L.t[fe[f]] == T_INTERNAL;
        r[f] = on[f] ? b[fe[f]] - apply_row<T>(L, L.t, f / 2, fe[f] - (f / 2) * F, X) : (T)0;
    }
    const T rC = b[3 * F + s] - apply_row<T>(L, L.t, 3, s, X);
    const T a = (T)L.a, d = (T)L.d, q = (T)L.q, ida = (T)L.ida, rd = (T)L.id, idet = (T)L.idet;
    T c0 = 0, c1 = 0;
#pragma unroll
    for (int dir = 0; dir < 3; dir++) {
        const bool lo = on[2 * dir], hi = on[2 * dir + 1];
        if (lo && hi) {
            c0 += q * (r[2 * dir + 1] - r[2 * dir]) * ida;
            c1 += (T)2 * q * q * ida;
        } else if (lo) {
            c0 -= q * r[2 * dir] * rd;
            c1 += q * q * rd;
        } else if (hi) {
            c0 += q * r[2 * dir + 1] * rd;
            c1 += q * q * rd;
        }
    }
    if (c1 == (T)0) return;
    const T dp = (rC - c0) / c1;
#pragma unroll
    for (int dir = 0; dir < 3; dir++) {
        const bool lo = on[2 * dir], hi = on[2 * dir + 1];
        const T fl = r[2 * dir] - q * dp, fh = r[2 * dir + 1] + q * dp;
        if (lo && hi) {
            x[fe[2 * dir]] += (d * fl + a * fh) * idet;
            x[fe[2 * dir + 1]] += (a * fl + d * fh) * idet;
        } else if (lo) {
            x[fe[2 * dir]] += fl * rd;
        } else if (hi) {
            x[fe[2 * dir + 1]] += fh * rd;
        }
    }
    x[3 * F + s] += dp;
}

// (xi, mean) step: per block [0] sum of (div u - b_c), [1] sum of p over the cells
template <typename T>
__global__ void __launch_bounds__(256) k3_scalar_partial(Lev L, const T *x, const T *b, double *part)
{
    const long long F = L.F, S = L.S, S2 = S * S;
    const T q = (T)L.q;
    T sd = 0, sp = 0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < F; s += (long long)gridDim.x * blockDim.x) {
        if (L.t[3 * F + s] != T_INTERNAL) continue;
        const T div = q * ((x[s + 1] - x[s]) + (x[F + s + S] - x[F + s]) + (x[2 * F + s + S2] - x[2 * F + s]));
        sd += div - b[3 * F + s];
        sp += x[3 * F + s];
    }
    __shared__ double ss[256], sm[256];
    ss[threadIdx.x] = (double)sd;
    sm[threadIdx.x] = (double)sp;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] += sm[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = ss[0];
        part[2 * blockIdx.x + 1] = sm[0];
    }
}

// xi <- mean(div u - b_c); shift[0] <- (b_mean - h^3 sum p) / (h^3 n_cells)
template <typename T>
__global__ void k3_scalar_final(Lev L, const double *part, int nb, T *x, const T *b, double *shift)
{
    __shared__ double ss[256], sm[256];
    double s = 0.0, m = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        s += part[2 * k];
        m += part[2 * k + 1];
    }
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] += sm[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = (double)L.N * L.N * L.N;
        x[4 * L.F] = (T)(ss[0] / n);
        shift[0] = ((double)b[4 * L.F] - L.h3 * sm[0]) / (L.h3 * n);
    }
}

template <typename T> __global__ void k3_pshift(Lev L, T *x, const double *shift)
{
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= L.F || L.t[3 * L.F + s] != T_INTERNAL) return;
    x[3 * L.F + s] += (T)shift[0];
}

// the wall and box-ghost rows of a level into L.gl (order unspecified; the
// sweeps below are Jacobi, so it does not matter); one atomic per warp
__global__ void k3_ghost_list(Lev L, int *count)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool is = e < 3 * L.F && (L.t[e] == T_WALL || L.t[e] == T_BOXGHOST);
    const unsigned m = __ballot_sync(0xffffffffu, is);
    if (m == 0u) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(m, base, leader);
    const int k = base + __popc(m & ((1u << lane) - 1u));
    if (is && k < ghost_cap(L.N)) L.gl[k] = e;
}

// Eq. (ghostrelax): lambda Jacobi sweeps x += dtau r over the listed wall and
// box-ghost rows.  On the box domain no listed row reads another: a wall row
// reads only itself, a box-ghost row itself and the two interior nodes
// inwards of it, which the sweeps leave alone.  So lambda sweeps over the
// whole list are lambda updates of each row in turn, one thread per row and
// one launch, with the same operations as sweep-by-sweep passes.
template <typename T> __global__ void k3_ghost_sweeps(Lev L, T *x, const T *b, T dtau, int lambda)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.ng) return;
    const long long e = L.gl[k];
    const int g = frame_of(e, L.F);
    const T be = b[e];
    for (int it = 0; it < lambda; it++) x[e] += dtau * (be - apply_row<T>(L, L.t, g, e - g * L.F, VecAcc<T>{x}));
}

// ------------------------------------------------------------ transfers

// restriction class: 1 interior, 2 wall or box ghost, 0 inactive
__device__ inline int rclass(unsigned char t) { return t == T_INTERNAL ? 1 : (t == T_WALL || t == T_BOXGHOST) ? 2 : 0; }

// Restriction (Eqs. restop, restop5 per axis): coarse node of grid g; along
// its own axis the fine faces 2O - 1, 2O, 2O + 1 weigh 1/4, 1/2, 1/4, along
// a cell-centred axis the fine cells 2T, 2T + 1 weigh 1/2 each.  The
// weighted sum when every fine node lies in the frame and is of the coarse
// node's class, else the plain mean of those that are, 0 if none.
template <typename T>
__global__ void __launch_bounds__(256) k3_restrict(Lev f, Lev c, const T *r, T *bH)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= 4 * c.F) {
        if (e == 4 * c.F) bH[4 * c.F] = r[4 * f.F];  // the mean row: injected
        return;
    }
    const int g = frame_of(e, c.F);
    const long long s = e - g * c.F;
    const int cc = rclass(c.t[e]);
    if (cc == 0) {
        bH[e] = (T)0;
        return;
    }
    const int C[3] = {coord(s, c.S, 0), coord(s, c.S, 1), coord(s, c.S, 2)};
    const long long Sf = f.S;
    T sw = 0, su = 0;
    int cnt = 0;
    bool all = true;
    const int n2 = (g == 0) ? 3 : 2, n1 = (g == 1) ? 3 : 2, n0 = (g == 2) ? 3 : 2;  // offsets along k, j, i
    for (int ok = 0; ok < n0; ok++)
        for (int oj = 0; oj < n1; oj++)
            for (int oi = 0; oi < n2; oi++) {
                const int o[3] = {oi, oj, ok};
                int fc[3];
                T w = 1;
                bool in = true;
                for (int ax = 0; ax < 3; ax++) {
                    const bool own = g < 3 && ax == g;
                    const int off = own ? o[ax] - 1 : o[ax];
                    fc[ax] = 2 * C[ax] + off;
                    w *= own ? (off == 0 ? (T)0.5 : (T)0.25) : (T)0.5;
                    in = in && fc[ax] >= -1 && fc[ax] <= f.N;
                }
                if (in) {
                    const long long fs = ((long long)(fc[2] + 1) * Sf + (fc[1] + 1)) * Sf + (fc[0] + 1);
                    if (rclass(f.t[g * f.F + fs]) == cc) {
                        const T v = r[g * f.F + fs];
                        sw += w * v;
                        su += v;
                        cnt++;
                        continue;
                    }
                }
                all = false;
            }
    bH[e] = all ? sw : (cnt > 0 ? su / (T)cnt : (T)0);
}

// interpolation taps of fine index fi along one axis: a face axis (aligned,
// even: the coarse face, odd: the two around it) or a cell-centred axis
// (the two coarse cells around fi / 2 - 1/4, extrapolated past [lo, hi]).
// The weights are multiples of 1/4 below 2 in magnitude, so they and their
// products are exact in either precision.
template <typename T> __device__ inline int taps3(int fi, bool aligned, int lo, int hi, int *K, T *w)
{
    if (aligned) {
        if ((fi & 1) == 0) {
            K[0] = fi / 2;
            w[0] = (T)1;
            return 1;
        }
        K[0] = (fi - 1) / 2;
        K[1] = (fi + 1) / 2;
        w[0] = w[1] = (T)0.5;
        return 2;
    }
    int k0 = (fi - 1) >> 1;  // floor(fi / 2 - 1/4)
    k0 = k0 < lo ? lo : (k0 > hi - 1 ? hi - 1 : k0);
    K[0] = k0;
    K[1] = k0 + 1;
    w[1] = (T)(2 * fi - 1 - 4 * k0) * (T)0.25;  // fi / 2 - 1/4 - k0
    w[0] = (T)1 - w[1];
    return 2;
}

// Prolongation (Sect. 4.3): x += P eH on every active fine node, trilinear
// over the active coarse nodes with the weights renormalised; xi += xi_H
template <typename T>
__global__ void __launch_bounds__(256) k3_prolong(Lev f, Lev c, const T *eH, T *x)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= 4 * f.F) {
        if (e == 4 * f.F) x[4 * f.F] += eH[4 * c.F];
        return;
    }
    if (f.t[e] == T_INACTIVE) return;
    const int g = frame_of(e, f.F);
    const long long s = e - g * f.F;
    int K[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    T W[3][2];
    int n[3];
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        const bool own = g < 3 && ax == g;
        const int lo = g == 3 ? 0 : (own ? 0 : -1), hi = g == 3 ? c.N - 1 : c.N;
        n[ax] = taps3<T>(coord(s, f.S, ax), own, lo, hi, K[ax], W[ax]);
    }
    // per axis and tap: the coarse slot offset, or -1 outside the frame
    // (entries of the coarse vector stay below 2^31: 4 (N/2 + 2)^3 for N <= 1024)
    const int Sc = c.S;
    int off[3][2];
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        const int stride = ax == 0 ? 1 : ax == 1 ? Sc : Sc * Sc;
#pragma unroll
        for (int a = 0; a < 2; a++)
            off[ax][a] = (a < n[ax] && K[ax][a] >= -1 && K[ax][a] <= c.N) ? (K[ax][a] + 1) * stride : -1;
    }
    const int gbase = g * (int)c.F;
    T acc = 0, ws = 0;
#pragma unroll
    for (int a2 = 0; a2 < 2; a2++)
#pragma unroll
        for (int a1 = 0; a1 < 2; a1++)
#pragma unroll
            for (int a0 = 0; a0 < 2; a0++) {
                // a one-tap axis has off = -1 for its second tap; the sum runs in tap order
                if (off[0][a0] < 0 || off[1][a1] < 0 || off[2][a2] < 0) continue;
                const int cs = gbase + off[2][a2] + off[1][a1] + off[0][a0];
                if (c.t[cs] == T_INACTIVE) continue;
                const T w = W[0][a0] * W[1][a1] * W[2][a2];
                acc += w * eH[cs];
                ws += w;
            }
    if (ws > (T)0) x[e] += (ws == (T)1 ? acc : acc / ws);
}

// ------------------------------------------------------------ coarsest level

// dense matrix of the coarsest level: M[row][col] = (M e_col)_row for the
// 4 F + 1 unknowns (the last is xi, whose row is the mean row h^3 sum p)
__global__ void k3_assemble(Lev L, double *M, int n)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)n * n) return;
    const int row = (int)(id / n), col = (int)(id % n);
    double v;
    if (row == n - 1) {
        v = (col >= 3 * L.F && col < 4 * L.F && L.t[col] == T_INTERNAL) ? L.h3 : 0.0;
    } else {
        const int g = (int)(row / L.F);
        v = apply_row<double>(L, L.t, g, row - g * L.F, UnitAcc{col});
    }
    M[id] = v;
}

// Gauss-Jordan with partial pivoting on [M | I] (n x 2n, row-major), one
// column per step: the pivot of column k among rows k.., the swap, the
// scaling of row k, then the elimination of column k from every other row
__global__ void k3_gj_pivot(double *A, int n, int k, int *piv)
{
    __shared__ double bv[256];
    __shared__ int bi[256];
    double best = -1.0;
    int bidx = k;
    for (int r = k + threadIdx.x; r < n; r += blockDim.x) {
        const double v = fabs(A[(long long)r * 2 * n + k]);
        if (v > best) {
            best = v;
            bidx = r;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bidx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double a = bv[threadIdx.x + o];
            const int ia = bi[threadIdx.x + o];
            if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ia < bi[threadIdx.x])) {
                bv[threadIdx.x] = a;
                bi[threadIdx.x] = ia;
            }
        }
        __syncthreads();
    }
    const int p = bi[0];
    if (threadIdx.x == 0 && bv[0] == 0.0) piv[0] = 1;  // singular
    // swap rows p and k, then scale row k by 1 / pivot
    for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) {
        const double t = A[(long long)p * 2 * n + c];
        A[(long long)p * 2 * n + c] = A[(long long)k * 2 * n + c];
        A[(long long)k * 2 * n + c] = t;
    }
    __syncthreads();
    const double pv = A[(long long)k * 2 * n + k];
    __syncthreads();
    if (pv != 0.0)
        for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) A[(long long)k * 2 * n + c] /= pv;
}

__global__ void k3_gj_eliminate(double *A, int n, int k, double *colk)
{
    // colk: column k of every row before the elimination (saved first)
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)n * 2 * n) return;
    const int r = (int)(id / (2 * n)), c = (int)(id % (2 * n));
    if (r == k) return;
    const double f = colk[r];
    if (f != 0.0) A[id] -= f * A[(long long)k * 2 * n + c];
}

__global__ void k3_gj_savecol(const double *A, int n, int k, double *colk)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) colk[r] = A[(long long)r * 2 * n + k];
}

__global__ void k3_gj_init(const double *M, double *A, int n)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)n * 2 * n) return;
    const int r = (int)(id / (2 * n)), c = (int)(id % (2 * n));
    A[id] = c < n ? M[(long long)r * n + c] : (c - n == r ? 1.0 : 0.0);
}

// x[0, n) = Minv b, one warp per row (the right half of the eliminated [M | I])
template <typename T> __global__ void k3_gemv(const double *A, int n, const T *b, T *x)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s += A[(long long)warp * 2 * n + n + c] * (double)b[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[warp] = (T)s;
}

template <typename T> __global__ void k3_zero(T *x, long long n)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < n) x[e] = (T)0;
}

// x += e over the four frames and xi: the FP32 correction of the mixed mode
__global__ void k3_add_float(double *x, const float *e, long long n)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) x[k] += (double)e[k];
}

// ------------------------------------------------------------ host side

struct Ctx {
    int N, L, nu1, nu2, lambda;
    int precision, inner;  // 0 FP64 cycles; 1 up to `inner` FP32 cycles per FP64 residual correction
    double alpha, dtau;
    cudaStream_t st;
    Lev lv[MAX_LEVELS];
    double *part, *red, *colk, *A, *M;
    int *flag;
    int nc;        // unknowns of the coarsest level
    int npart;
    char msg[256];
    // box-relaxation timer
    int tmr_level;
    std::vector<cudaEvent_t> ev;
    long long tmr_n;
    double tmr_ms;
};

static inline unsigned nblk(long long n) { return (unsigned)((n + 255) / 256); }

static bool valid(int N, int levels)
{
    // N <= 1024 keeps every frame below 2^31 slots (32-bit slot arithmetic)
    if (N < 2 || levels < 1 || levels > MAX_LEVELS || N > 1024) return false;
    if (N % (1 << (levels - 1))) return false;
    const int Nc = N >> (levels - 1);
    if (Nc < 2) return false;
    const long long Sc = Nc + 2;
    return 4 * Sc * Sc * Sc + 1 <= COARSE_MAX;
}

// carve the workspace (every array 256-byte aligned); with base == nullptr
// only count.  mixed: the FP32 vectors of the inner cycles too
static size_t carve(Ctx *c, char *base, int N, int levels, bool mixed)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        off = (off + 255) & ~(size_t)255;
        char *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    int npart = 2 * 1024;
    for (int l = 0; l < levels; l++) {
        const int Nl = N >> l;
        const long long S = Nl + 2, F = S * S * S, VL = vlen(Nl);
        unsigned char *t = (unsigned char *)take((size_t)4 * F);
        double *x = l > 0 ? (double *)take(sizeof(double) * VL) : nullptr;
        double *b = l > 0 ? (double *)take(sizeof(double) * VL) : nullptr;
        double *r = (double *)take(sizeof(double) * VL);
        float *xf = mixed ? (float *)take(sizeof(float) * VL) : nullptr;
        float *bf = mixed ? (float *)take(sizeof(float) * VL) : nullptr;
        float *rf = mixed ? (float *)take(sizeof(float) * VL) : nullptr;
        long long *gl = (long long *)take(sizeof(long long) * ghost_cap(Nl));
        if (c) {
            Lev &L = c->lv[l];
            L.N = Nl;
            L.S = (int)S;
            L.F = F;
            L.VL = VL;
            const double h = 1.0 / Nl;
            L.a = c->alpha / (h * h);
            L.q = 1.0 / h;
            L.d = 1.0 + 6.0 * L.a;
            L.h3 = h * h * h;
            L.ida = 1.0 / (L.d + L.a);
            L.id = 1.0 / L.d;
            L.idet = 1.0 / (L.d * L.d - L.a * L.a);
            L.t = t;
            L.x = x;
            L.b = b;
            L.r = r;
            L.xf = xf;
            L.bf = bf;
            L.rf = rf;
            L.gl = gl;
            L.ng = 0;
        }
    }
    const int Nc = N >> (levels - 1);
    const long long Sc = Nc + 2;
    const int nc = (int)(4 * Sc * Sc * Sc + 1);
    double *part = (double *)take(sizeof(double) * npart);
    double *red = (double *)take(sizeof(double) * 8);
    double *colk = (double *)take(sizeof(double) * nc);
    double *A = (double *)take(sizeof(double) * (size_t)nc * 2 * nc);
    double *M = (double *)take(sizeof(double) * (size_t)nc * nc);
    int *flag = (int *)take(sizeof(int) * 4);
    if (c) {
        c->part = part;
        c->red = red;
        c->colk = colk;
        c->A = A;
        c->M = M;
        c->flag = flag;
        c->nc = nc;
        c->npart = npart / 2;
    }
    return off + 256;
}

static gp_status fail(Ctx *c, gp_status st, const char *what)
{
    if (c) snprintf(c->msg, sizeof c->msg, "%s", what);
    return st;
}

static gp_status cuda_check(Ctx *c, const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return GP_OK;
    if (c) snprintf(c->msg, sizeof c->msg, "%s: %s", where, cudaGetErrorString(e));
    return GP_CUDA;
}

// blocks of 256 threads for a grid-stride reduction kernel over n entries:
// one wave of resident blocks (a partial second wave would leave SMs idle),
// at most the 1024 partial results the workspace holds
template <typename K> static int red_grid(K kernel, long long n, int &cache)
{
    if (cache <= 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        cache = sms * per_sm < 1024 ? sms * per_sm : 1024;
    }
    const long long b = (n + 255) / 256;
    return (int)(b < cache ? (b < 1 ? 1 : b) : cache);
}

// the level vectors and the ghost-sweep scratch of precision T
template <typename T> struct Vecs;
template <> struct Vecs<double> {
    static double *x(const Lev &L) { return L.x; }
    static double *b(const Lev &L) { return L.b; }
    static double *r(const Lev &L) { return L.r; }
};
template <> struct Vecs<float> {
    static float *x(const Lev &L) { return L.xf; }
    static float *b(const Lev &L) { return L.bf; }
    static float *r(const Lev &L) { return L.rf; }
};

template <typename T, typename R> static void residual(Ctx *c, int l, const T *x, const T *b, R *r)
{
    const Lev &L = c->lv[l];
    static int resident = 0;
    const int nb = red_grid(k3_residual<T, R>, 4 * L.F, resident);
    k3_residual<T, R><<<nb, 256, 0, c->st>>>(L, x, b, r, c->part);
    k3_residual_final<T, R><<<1, 256, 0, c->st>>>(L, c->part, nb, b, r, c->red);
}

template <typename T> static void smooth(Ctx *c, int l, T *x, const T *b, int nu)
{
    const Lev &L = c->lv[l];
    const int per_row = (L.N + NCOL - 1) / NCOL;
    const long long nbox = (long long)per_row * L.N * L.N;
    for (int it = 0; it < nu; it++) {
        for (int col = 0; col < NCOL; col++) {
            const bool timed = c->tmr_level == l && !c->ev.empty();
            if (timed) cudaEventRecord(c->ev[2 * (c->tmr_n % 256)], c->st);
            k3_box<T><<<nblk(nbox), 256, 0, c->st>>>(L, x, b, col);
            if (timed) {
                cudaEventRecord(c->ev[2 * (c->tmr_n % 256) + 1], c->st);
                cudaEventSynchronize(c->ev[2 * (c->tmr_n % 256) + 1]);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, c->ev[2 * (c->tmr_n % 256)], c->ev[2 * (c->tmr_n % 256) + 1]);
                c->tmr_ms += ms;
                c->tmr_n++;
            }
        }
        static int resident = 0;
        const int nb = red_grid(k3_scalar_partial<T>, L.F, resident);
        k3_scalar_partial<T><<<nb, 256, 0, c->st>>>(L, x, b, c->part);
        k3_scalar_final<T><<<1, 256, 0, c->st>>>(L, c->part, nb, x, b, c->red + 1);
        k3_pshift<T><<<nblk(L.F), 256, 0, c->st>>>(L, x, c->red + 1);
        if (c->lambda > 0) k3_ghost_sweeps<T><<<nblk(L.ng), 256, 0, c->st>>>(L, x, b, (T)c->dtau, c->lambda);
    }
}

template <typename T> static void coarse_solve(Ctx *c, const T *b, T *x)
{
    const int n = c->nc;
    k3_gemv<T><<<(unsigned)((n * 32 + 255) / 256), 256, 0, c->st>>>(c->A, n, b, x);
}

template <typename T> static void cycle(Ctx *c, int l, T *x, const T *b)
{
    if (l == c->L - 1) {
        coarse_solve<T>(c, b, x);
        return;
    }
    const Lev &L = c->lv[l], &C = c->lv[l + 1];
    T *r = Vecs<T>::r(L), *xc = Vecs<T>::x(C), *bc = Vecs<T>::b(C);
    smooth<T>(c, l, x, b, c->nu1);
    residual<T, T>(c, l, x, b, r);
    k3_restrict<T><<<nblk(4 * C.F + 1), 256, 0, c->st>>>(L, C, r, bc);
    k3_zero<T><<<nblk(C.VL), 256, 0, c->st>>>(xc, C.VL);
    cycle<T>(c, l + 1, xc, bc);
    k3_prolong<T><<<nblk(4 * L.F + 1), 256, 0, c->st>>>(L, C, xc, x);
    smooth<T>(c, l, x, b, c->nu2);
}

static gp_status build_coarse(Ctx *c)
{
    const Lev &L = c->lv[c->L - 1];
    const int n = c->nc;
    cudaMemsetAsync(c->flag, 0, sizeof(int), c->st);
    k3_assemble<<<nblk((long long)n * n), 256, 0, c->st>>>(L, c->M, n);
    k3_gj_init<<<nblk((long long)n * 2 * n), 256, 0, c->st>>>(c->M, c->A, n);
    for (int k = 0; k < n; k++) {
        k3_gj_pivot<<<1, 256, 0, c->st>>>(c->A, n, k, c->flag);
        k3_gj_savecol<<<nblk(n), 256, 0, c->st>>>(c->A, n, k, c->colk);
        k3_gj_eliminate<<<nblk((long long)n * 2 * n), 256, 0, c->st>>>(c->A, n, k, c->colk);
    }
    int sing = 0;
    cudaMemcpyAsync(&sing, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "coarse inverse");
    if (sing) return fail(c, GP_SINGULAR, "coarsest-level matrix is singular");
    return cuda_check(c, "coarse inverse");
}

}  // namespace gp3

using namespace gp3;

struct gp3_ctx {
    Ctx c;
};

extern "C" {

long long gp3_vec_len(int N) { return N >= 1 ? vlen(N) : 0; }

gp_status gp3_workspace_size(int N, int levels, int precision, size_t *bytes)
{
    if (!bytes || !valid(N, levels) || precision < 0 || precision > 1) return GP_INVALID;
    *bytes = carve(nullptr, nullptr, N, levels, precision == 1);
    return GP_OK;
}

gp_status gp3_create(gp3_ctx **out, int N, int levels, double alpha, int nu1, int nu2, int lambda, double dtau,
                     int precision, int inner, void *ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!out || !ws || !valid(N, levels) || !(alpha >= 0.0) || nu1 < 0 || nu2 < 0 || nu1 + nu2 < 1 || lambda < 0 ||
        !(dtau > 0.0) || ((uintptr_t)ws % 256) || precision < 0 || precision > 1 || inner < 1 || inner > 16)
        return GP_INVALID;
    if (ws_bytes < carve(nullptr, nullptr, N, levels, precision == 1)) return GP_INVALID;
    nvtxRangePushA("gp3_create");
    gp3_ctx *h = new gp3_ctx();
    Ctx *c = &h->c;
    c->N = N;
    c->L = levels;
    c->alpha = alpha;
    c->nu1 = nu1;
    c->nu2 = nu2;
    c->lambda = lambda;
    c->dtau = dtau;
    c->precision = precision;
    c->inner = inner;
    c->st = stream;
    c->tmr_level = -1;
    c->tmr_n = 0;
    c->tmr_ms = 0.0;
    c->msg[0] = 0;
    carve(c, (char *)ws, N, levels, precision == 1);
    for (int l = 0; l < levels; l++) {
        Lev &L = c->lv[l];
        k3_types<<<nblk(4 * L.F), 256, 0, stream>>>(L.N, L.F, L.t);
        // the wall and box-ghost rows, counted in flag[1]
        int ng = 0;
        cudaMemsetAsync(c->flag + 1, 0, sizeof(int), stream);
        k3_ghost_list<<<nblk(3 * L.F), 256, 0, stream>>>(L, c->flag + 1);
        cudaMemcpyAsync(&ng, c->flag + 1, sizeof(int), cudaMemcpyDeviceToHost, stream);
        if (cudaStreamSynchronize(stream) != cudaSuccess || ng > ghost_cap(L.N)) {
            cudaGetLastError();
            nvtxRangePop();
            gp3_destroy(h);
            return GP_CUDA;
        }
        L.ng = ng;
    }
    gp_status st = build_coarse(c);
    nvtxRangePop();
    if (st != GP_OK) {
        gp3_destroy(h);
        return st;
    }
    *out = h;
    return GP_OK;
}

gp_status gp3_destroy(gp3_ctx *h)
{
    if (!h) return GP_INVALID;
    for (cudaEvent_t e : h->c.ev) cudaEventDestroy(e);
    delete h;
    return GP_OK;
}

const char *gp3_last_error(gp3_ctx *h) { return h ? h->c.msg : "null context"; }

gp_status gp3_types(gp3_ctx *h, int level, unsigned char *types)
{
    if (!h || !types || level < 0 || level >= h->c.L) return GP_INVALID;
    Ctx *c = &h->c;
    cudaMemcpyAsync(types, c->lv[level].t, (size_t)4 * c->lv[level].F, cudaMemcpyDeviceToDevice, c->st);
    return cuda_check(c, "gp3_types");
}

gp_status gp3_residual(gp3_ctx *h, int level, const double *x, const double *b, double *r, double *norm_host)
{
    if (!h || !x || !b || !r || level < 0 || level >= h->c.L) return GP_INVALID;
    Ctx *c = &h->c;
    residual<double, double>(c, level, x, b, r);
    if (norm_host) {
        cudaMemcpyAsync(norm_host, c->red, sizeof(double), cudaMemcpyDeviceToHost, c->st);
        if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "gp3_residual");
    }
    return cuda_check(c, "gp3_residual");
}

gp_status gp3_smooth(gp3_ctx *h, int level, double *x, const double *b, int nu)
{
    if (!h || !x || !b || level < 0 || level >= h->c.L || nu < 0) return GP_INVALID;
    smooth<double>(&h->c, level, x, b, nu);
    return cuda_check(&h->c, "gp3_smooth");
}

gp_status gp3_restrict(gp3_ctx *h, int level, const double *r, double *bH)
{
    if (!h || !r || !bH || level < 0 || level >= h->c.L - 1) return GP_INVALID;
    Ctx *c = &h->c;
    k3_restrict<double><<<nblk(4 * c->lv[level + 1].F + 1), 256, 0, c->st>>>(c->lv[level], c->lv[level + 1], r, bH);
    return cuda_check(c, "gp3_restrict");
}

gp_status gp3_prolong(gp3_ctx *h, int level, const double *eH, double *x)
{
    if (!h || !eH || !x || level < 0 || level >= h->c.L - 1) return GP_INVALID;
    Ctx *c = &h->c;
    k3_prolong<double><<<nblk(4 * c->lv[level].F + 1), 256, 0, c->st>>>(c->lv[level], c->lv[level + 1], eH, x);
    return cuda_check(c, "gp3_prolong");
}

gp_status gp3_cycle(gp3_ctx *h, double *x, const double *b)
{
    if (!h || !x || !b) return GP_INVALID;
    nvtxRangePushA("gp3_cycle");
    cycle<double>(&h->c, 0, x, b);
    nvtxRangePop();
    return cuda_check(&h->c, "gp3_cycle");
}

gp_status gp3_solve(gp3_ctx *h, double *x, const double *b, double tol, int max_cycles, int *cycles,
                    int *iterations, double *res, double *hist_host)
{
    if (!h || !x || !b || !(tol > 0.0) || max_cycles < 0) return GP_INVALID;
    Ctx *c = &h->c;
    nvtxRangePushA("gp3_solve");
    const Lev &L = c->lv[0];
    const bool mixed = c->precision == 1;
    double r0 = 0.0, rn = 0.0;
    int k = 0, ncyc = 0;
    gp_status st = GP_OK;
    for (;; k++) {
        // the FP64 residual (mixed: written rounded to FP32 as the inner cycles' right-hand side)
        if (mixed)
            residual<double, float>(c, 0, x, b, L.bf);
        else
            residual<double, double>(c, 0, x, b, L.r);
        cudaMemcpyAsync(&rn, c->red, sizeof(double), cudaMemcpyDeviceToHost, c->st);
        if (cudaStreamSynchronize(c->st) != cudaSuccess) {
            st = cuda_check(c, "gp3_solve");
            break;
        }
        if (k == 0) r0 = rn;
        if (hist_host) hist_host[k] = rn;
        if (rn != rn || rn > 1e6 * r0) {
            st = fail(c, GP_DIVERGED, "gp3_solve: diverged");
            break;
        }
        if (rn <= tol) break;
        if (ncyc >= max_cycles) {
            st = fail(c, GP_NOT_CONVERGED, "gp3_solve: not converged");
            break;
        }
        if (mixed) {
            // up to `inner` FP32 cycles from zero on the correction, added to x in FP64
            const int n = c->inner < max_cycles - ncyc ? c->inner : max_cycles - ncyc;
            k3_zero<float><<<nblk(L.VL), 256, 0, c->st>>>(L.xf, L.VL);
            for (int q = 0; q < n; q++) cycle<float>(c, 0, L.xf, L.bf);
            k3_add_float<<<nblk(4 * L.F + 1), 256, 0, c->st>>>(x, L.xf, 4 * L.F + 1);
            ncyc += n;
        } else {
            cycle<double>(c, 0, x, b);
            ncyc++;
        }
    }
    if (cycles) *cycles = ncyc;
    if (iterations) *iterations = k;
    if (res) *res = rn;
    nvtxRangePop();
    return st;
}

gp_status gp3_timer_start(gp3_ctx *h, int level)
{
    if (!h || level < 0 || level >= h->c.L) return GP_INVALID;
    Ctx *c = &h->c;
    if (c->ev.empty()) {
        c->ev.resize(512);
        for (auto &e : c->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return cuda_check(c, "gp3_timer_start");
    }
    c->tmr_level = level;
    c->tmr_n = 0;
    c->tmr_ms = 0.0;
    return GP_OK;
}

gp_status gp3_timer_stop(gp3_ctx *h, long long *launches, double *ms)
{
    if (!h) return GP_INVALID;
    Ctx *c = &h->c;
    c->tmr_level = -1;
    if (launches) *launches = c->tmr_n;
    if (ms) *ms = c->tmr_ms;
    return GP_OK;
}

}  // extern "C"
