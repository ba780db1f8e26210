// Operator, relaxation and transfer kernels of one multigrid level
// (Sect. 3.2 rows, Sect. 4.1 relaxation, Sect. 4.2 restriction, Sect. 4.3
// interpolation), in FP64 and FP32.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <unordered_map>
#include <utility>
#include <vector>

#include "gpmg_internal.cuh"

namespace gpmg {

// levels solved by the one-block smoother, ghost lists swept by one block,
// and levels whose full boxes are swept by shared-memory tiles
constexpr int SMALL_N = 64;  // levels whose whole relaxation runs in one block
constexpr size_t SMALL_STAGE_BYTES = 200 * 1024;  // x and b of such a level staged in shared memory up to this size
constexpr int TILE_MIN_N = 128;  // default smallest FP32 level swept by TMA tiles (gp_params.tile_min overrides)
constexpr int WAVE_MIN_N = 4096;  // default smallest tiled level swept down strips of rows (gp_params.wave_min)
constexpr int GHOST_BLOCK_ROWS = 1024;  // at most this many ghost-class rows: the lambda sweeps in one block
constexpr int CUT_SPLIT = 64;  // cut boxes per colour above which the cut sweep leaves a single block
constexpr int CUT_COLOUR_LAUNCHES = 6;  // at most this many colours: one launch per colour, else one cluster

// constants of the box solves of one level (Sect. 4.1.1), reciprocals
// precomputed so that a box needs no division
template <typename T> struct BoxK {
    T a, d, q;          // alpha/h^2, 1 + 4 alpha/h^2, 1/h
    T qida, qid;        // q/(d + a), q/d
    T id, idet;         // 1/d, 1/(d^2 - a^2)
    T ic1[9];           // 1/c1 for (faces in x) * 3 + (faces in y), c1 the pressure pivot of the Schur complement
};

template <typename T> struct LevelArgs {
    int N, P;
    long long F;
    T q, a, d;          // 1/h, alpha/h^2, 1 + 4 alpha/h^2
    T h2;               // h^2
    const uint8_t *tU, *tV, *tP;
    const uint8_t *bc;  // box codes
    BoxK<T> K;
};

template <typename T> __device__ inline const T *gw(const GhostList &gh);
template <> __device__ inline const double *gw<double>(const GhostList &gh) { return gh.w; }
template <> __device__ inline const float *gw<float>(const GhostList &gh) { return gh.wf; }
template <typename T> __device__ inline T *gupd(const GhostList &gh);
template <> __device__ inline double *gupd<double>(const GhostList &gh) { return gh.upd; }
template <> __device__ inline float *gupd<float>(const GhostList &gh) { return gh.updf; }

// b - sum_q w_q x[st_q] of ghost-class row k (Eq. ghostrelax, Sect. 3.4):
// every index and then every value of the row is loaded before the
// arithmetic, which keeps the serial order q = 0, 1, ... (a plain loop over
// the stencil would wait on each gather in turn).  With `acc`, the stencil
// value of a node that is itself a ghost-class row is x + acc[that row].
template <typename T, bool ACC>
__device__ __forceinline__ T ghost_row_residual(const GhostList &gh, int k, const T *x, const T *b, const T *acc)
{
    const T *w = gw<T>(gh);
    const int nst = gh.nst[k];
    int idx[GH_ST], lnk[GH_ST];
    T wv[GH_ST], xv[GH_ST];
#pragma unroll
    for (int q = 0; q < GH_ST; q++) {
        const long long e = (long long)q * gh.cap + k;
        idx[q] = q < nst ? gh.st[e] : 0;
        lnk[q] = (ACC && q < nst) ? gh.strow[e] : -1;
        wv[q] = q < nst ? w[e] : (T)0;
    }
#pragma unroll
    for (int q = 0; q < GH_ST; q++) {
        xv[q] = q < nst ? x[idx[q]] : (T)0;
        if (ACC && lnk[q] >= 0) xv[q] += acc[lnk[q]];
    }
    T s = b[gh.node[k]];
#pragma unroll
    for (int q = 0; q < GH_ST; q++)
        if (q < nst) s -= wv[q] * xv[q];
    return s;
}

__device__ inline double nanmax(double a, double b) { return (a != a || b != b) ? (double)NAN : fmax(a, b); }

// ---------------------------------------------------------------- residual

// |v| as bits (sign cleared): for non-negative floats the integer order is
// the numeric order and a NaN sorts above infinity, so an integer max is an
// exact max norm that keeps NaN, without floating-point (or FP64) work
template <typename T> struct AbsBits;
template <> struct AbsBits<float> {
    typedef unsigned int U;
    __device__ static U of(float v) { return __float_as_uint(v) & 0x7fffffffu; }
    __device__ static double value(U u) { return (double)__uint_as_float(u); }
};
template <> struct AbsBits<double> {
    typedef unsigned long long U;
    __device__ static U of(double v) { return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull; }
    __device__ static double value(U u) { return __longlong_as_double((long long)u); }
};

// 16-byte vector loads and stores of four consecutive slots (the slot is a
// multiple of 4 and every frame starts 128-byte aligned)
__device__ __forceinline__ void ld4(const float *p, float *o)
{
    float4 t = *(const float4 *)p;
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double *o)
{
    double2 a = *(const double2 *)p, c = *(const double2 *)(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = c.x; o[3] = c.y;
}
__device__ __forceinline__ void st4(float *p, const float *o) { *(float4 *)p = make_float4(o[0], o[1], o[2], o[3]); }
__device__ __forceinline__ void st4(double *p, const double *o)
{
    *(double2 *)p = make_double2(o[0], o[1]);
    *(double2 *)(p + 2) = make_double2(o[2], o[3]);
}
__device__ __forceinline__ void ldt4(const uint8_t *p, uint8_t *o)
{
    uchar4 t = *(const uchar4 *)p;
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}

// The residual of the internal rows (Eq. LS, Sect. 3.2) on four consecutive
// slots per thread: one vector load per frame and neighbour row, all loads of
// a quad issued before the arithmetic.  r may be of a narrower type than the
// arithmetic (the FP64 residual written as the FP32 right-hand side of the
// next inner cycle).  Per block: [0] sum of p over internal cells, [1] max |r|.  Slots that are not internal get 0 (the
// ghost-class rows are written afterwards by k_ghost_residual); rows 0 and
// N + 1 of the frames hold no internal row.
template <typename T, typename R>
__global__ void __launch_bounds__(256) k_residual4(LevelArgs<T> A, const T *x, const T *b, R *r, double *part)
{
    T psum = 0;
    typename AbsBits<T>::U rbits = 0;
    const int P = A.P;
    const long long F = A.F, nq = (long long)(A.N + 2) * P / 4;
    const T *u = x, *v = x + F, *p = x + 2 * F;
    const T xi = x[3 * F];
    for (long long qd = blockIdx.x * (long long)blockDim.x + threadIdx.x; qd < nq; qd += (long long)gridDim.x * blockDim.x) {
        // F < 2^31 (checked when the context is created), so slots fit an int
        const int s0 = (int)(4 * qd);
        const int row = s0 / P;
        R ru[4] = {0, 0, 0, 0}, rv[4] = {0, 0, 0, 0}, rp[4] = {0, 0, 0, 0};
        uint8_t tu[4], tv[4], tp[4];
        ldt4(A.tU + s0, tu);
        ldt4(A.tV + s0, tv);
        ldt4(A.tP + s0, tp);
        // every load is issued before the types are tested: the neighbour
        // rows and columns are clamped into the frame on its first and last
        // rows, where no internal row is
        const int up = row < A.N + 1 ? P : 0, dn = row > 0 ? P : 0, lf = s0 > 0 ? 1 : 0;
        T uh[6], uU[4], uD[4], vh[6], vU[4], vD[4], ph[5], pD[4], bu[4], bv[4], bp[4];
        ld4(u + s0, uh + 1);
        uh[0] = u[s0 - lf];
        uh[5] = u[s0 + 4];
        ld4(u + s0 + up, uU);
        ld4(u + s0 - dn, uD);
        ld4(v + s0, vh + 1);
        vh[0] = v[s0 - lf];
        vh[5] = v[s0 + 4];
        ld4(v + s0 + up, vU);
        ld4(v + s0 - dn, vD);
        ld4(p + s0, ph + 1);
        ph[0] = p[s0 - lf];
        ld4(p + s0 - dn, pD);
        ld4(b + s0, bu);
        ld4(b + F + s0, bv);
        ld4(b + 2 * F + s0, bp);
        if (row > 0 && row < A.N + 1) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                if (tu[q] == T_INTERNAL) {
                    T Au = A.d * uh[q + 1] - A.a * (uh[q + 2] + uh[q] + uU[q] + uD[q]) + A.q * (ph[q + 1] - ph[q]);
                    T rr = bu[q] - Au;
                    ru[q] = (R)rr;
                    rbits = max(rbits, AbsBits<T>::of(rr));
                }
                if (tv[q] == T_INTERNAL) {
                    T Av = A.d * vh[q + 1] - A.a * (vh[q + 2] + vh[q] + vU[q] + vD[q]) + A.q * (ph[q + 1] - pD[q]);
                    T rr = bv[q] - Av;
                    rv[q] = (R)rr;
                    rbits = max(rbits, AbsBits<T>::of(rr));
                }
                if (tp[q] == T_INTERNAL) {
                    T Ac = A.q * (uh[q + 2] - uh[q + 1] + vU[q] - vh[q + 1]) - xi;
                    T rr = bp[q] - Ac;
                    rp[q] = (R)rr;
                    rbits = max(rbits, AbsBits<T>::of(rr));
                    psum += ph[q + 1];
                }
            }
        }
        st4(r + s0, ru);
        st4(r + F + s0, rv);
        st4(r + 2 * F + s0, rp);
    }
    __shared__ double ss[256], sm[256];
    ss[threadIdx.x] = (double)psum;
    sm[threadIdx.x] = AbsBits<T>::value(rbits);
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] = nanmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = ss[0];
        part[2 * blockIdx.x + 1] = sm[0];
    }
}

template <typename T, typename R>
__global__ void k_ghost_residual(GhostList gh, int nrows, const T *x, const T *b, R *r, unsigned long long *maxbits)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    if (k < nrows) {
        const T s = ghost_row_residual<T, false>(gh, k, x, b, nullptr);
        r[gh.node[k]] = (R)s;
        m = fabs((double)s);
    }
    // warp max then one atomic per warp (max of non-negative doubles by bits)
    for (int o = 16; o > 0; o >>= 1) m = nanmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(m));
    if ((threadIdx.x & 31) == 0 && m != m) atomicMax(maxbits, 0x7ff8000000000000ull);
}

// mean row (h^2 * sum of internal p) and the norm; one block
template <typename T, typename R>
__global__ void k_residual_final(const double *part, int nb, const T *b, R *r, long long imean, double h2,
                                 unsigned long long *maxbits, double *out, const T *x, const int *nint,
                                 R *also = nullptr)
{
    __shared__ double ss[256], sm[256];
    double s = 0.0, m = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        s += part[2 * k];
        m = nanmax(m, part[2 * k + 1]);
    }
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] = nanmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // an FP32 iterate carries its pressure shift unapplied (PSHIFT_SLOT)
        const double sig = sizeof(T) == 4 ? (double)x[imean + PSHIFT_SLOT] * (double)*nint : 0.0;
        double rm = (double)b[imean] - h2 * (ss[0] + sig);
        r[imean] = (R)rm;
        if (also) *also = (R)rm;  // the mean row of a restricted right-hand side
        double g = __longlong_as_double((long long)*maxbits);
        double nrm = nanmax(nanmax(sm[0], g), fabs(rm));
        out[0] = nrm;
        *maxbits = 0ull;
    }
}

// ------------------------------------------------------------ box smoother

// One frame's slots around a box, addressed by (rows up, columns right) of
// the box's cell: a frame of uniform row pitch (global memory or a tile), or
// four separately addressed rows -1 .. 2 (a ring of rows in shared memory).
template <typename T> struct PitchRows {
    T *c;
    int pitch;
    __device__ __forceinline__ T &at(int dr, int dc) const { return c[dr * pitch + dc]; }
};
template <typename T> struct RingRows {
    T *r[4];
    __device__ __forceinline__ T &at(int dr, int dc) const { return r[dr + 1][dc]; }
};

// Box relaxation of one cell without ghost borders (Sect. 4.1.1): Schur
// complement of the pressure unknown.  U, V, Pv: the u, v and p frames around
// the cell; bW, bE, bS, bN, bC: the right-hand side of the box's five rows.
// W, E, S, Nn: the faces that are internal (the others stay frozen); ALL: all
// four are.
template <typename T, bool ALL = false, typename View>
__device__ __forceinline__ void box_solve_v(const View &U, const View &V, const View &Pv, const T bW, const T bE,
                                            const T bS, const T bN, const T bC, const T xi, bool W, bool E, bool S,
                                            bool Nn, const BoxK<T> &K)
{
    const T a = K.a, d = K.d, q = K.q;
    if (ALL) W = E = S = Nn = true;
    T rW = 0, rE = 0, rS = 0, rN = 0;
    if (W)
        rW = bW - (d * U.at(0, 0) - a * (U.at(0, 1) + U.at(0, -1) + U.at(1, 0) + U.at(-1, 0)) +
                   q * (Pv.at(0, 0) - Pv.at(0, -1)));
    if (E)
        rE = bE - (d * U.at(0, 1) - a * (U.at(0, 2) + U.at(0, 0) + U.at(1, 1) + U.at(-1, 1)) +
                   q * (Pv.at(0, 1) - Pv.at(0, 0)));
    if (S)
        rS = bS - (d * V.at(0, 0) - a * (V.at(0, 1) + V.at(0, -1) + V.at(1, 0) + V.at(-1, 0)) +
                   q * (Pv.at(0, 0) - Pv.at(-1, 0)));
    if (Nn)
        rN = bN - (d * V.at(1, 0) - a * (V.at(1, 1) + V.at(1, -1) + V.at(2, 0) + V.at(0, 0)) +
                   q * (Pv.at(1, 0) - Pv.at(0, 0)));
    T rC = bC - (q * (U.at(0, 1) - U.at(0, 0) + V.at(1, 0) - V.at(0, 0)) - xi);
    // eliminating the velocities leaves c1 dp = rC - c0 for the pressure;
    // each direction contributes to c0, and c1 depends only on which faces
    // take part
    T c0 = 0;
    int nx = 0, ny = 0;
    if (W && E) {
        c0 += K.qida * (rE - rW);
        nx = 2;
    } else if (W) {
        c0 -= K.qid * rW;
        nx = 1;
    } else if (E) {
        c0 += K.qid * rE;
        nx = 1;
    }
    if (S && Nn) {
        c0 += K.qida * (rN - rS);
        ny = 2;
    } else if (S) {
        c0 -= K.qid * rS;
        ny = 1;
    } else if (Nn) {
        c0 += K.qid * rN;
        ny = 1;
    }
    if (nx + ny == 0) return;
    // select the pivot reciprocal with constant indices (a dynamic index
    // would copy the table to local memory)
    const int kc = nx * 3 + ny;
    T ic = K.ic1[1];
#pragma unroll
    for (int k = 2; k < 9; k++)
        if (kc == k) ic = K.ic1[k];
    T dp = (rC - c0) * ic;
    // velocity corrections with dp known
    T fW = rW - q * dp, fE = rE + q * dp, fS = rS - q * dp, fN = rN + q * dp;
    if (W && E) {
        U.at(0, 0) += (d * fW + a * fE) * K.idet;
        U.at(0, 1) += (a * fW + d * fE) * K.idet;
    } else if (W) U.at(0, 0) += fW * K.id;
    else if (E) U.at(0, 1) += fE * K.id;
    if (S && Nn) {
        V.at(0, 0) += (d * fS + a * fN) * K.idet;
        V.at(1, 0) += (a * fS + d * fN) * K.idet;
    } else if (S) V.at(0, 0) += fS * K.id;
    else if (Nn) V.at(1, 0) += fN * K.id;
    Pv.at(0, 0) += dp;
}

// the same on frames of row pitch `pitch`, u, v, p at the cell's slot
template <typename T, bool ALL = false>
__device__ __forceinline__ void box_solve(T *u, T *v, T *p, const int pitch, const T bW, const T bE, const T bS,
                                          const T bN, const T bC, const T xi, bool W, bool E, bool S, bool Nn,
                                          const BoxK<T> &K)
{
    box_solve_v<T, ALL>(PitchRows<T>{u, pitch}, PitchRows<T>{v, pitch}, PitchRows<T>{p, pitch}, bW, bE, bS, bN, bC,
                        xi, W, E, S, Nn, K);
}

// the same with the right-hand side read at bu, bv, bp (bN at bv[bpitch])
template <typename T, bool ALL = false>
__device__ __forceinline__ void box_core(T *u, T *v, T *p, const int pitch, const T *bu, const T *bv, const T *bp,
                                         const long long bpitch, const T xi, bool W, bool E, bool S, bool Nn,
                                         const BoxK<T> &K)
{
    box_solve<T, ALL>(u, v, p, pitch, bu[0], bu[1], bv[0], bv[bpitch], bp[0], xi, W, E, S, Nn, K);
}

// the full box of cell (i, j), if it is one (box code BOX_FULL)
template <typename T>
__device__ __forceinline__ void box_full_one(const LevelArgs<T> &A, T *x, const T *b, int i, int j)
{
    const long long s = (long long)(j + 1) * A.P + (i + 1);
    const unsigned code = A.bc[s];
    if (!(code & BOX_FULL)) return;
    if (code == BOX_ALL)
        box_core<T, true>(x + s, x + A.F + s, x + 2 * A.F + s, A.P, b + s, b + A.F + s, b + 2 * A.F + s, A.P,
                          x[3 * A.F], true, true, true, true, A.K);
    else
        box_core<T>(x + s, x + A.F + s, x + 2 * A.F + s, A.P, b + s, b + A.F + s, b + 2 * A.F + s, A.P, x[3 * A.F],
                    code & BOX_W, code & BOX_E, code & BOX_S, code & BOX_N, A.K);
}

// All five colours of the full boxes in one pass over the level.  Each
// block owns TH x TW frame slots (all three frames).  One TMA copy brings the
// u, v, p frames of a (TH + 20) x LW window around them into shared memory
// (10 slots above and below, 16 left, at least 10 right) and another the
// box codes of the same window.  Colour c relaxes the boxes within
// 2 (4 - c) + 1 cells below and 2 (4 - c) cells above the owned cells: a box
// reads only values written by boxes at most two cells away, so the owned
// slots see the same sequence of updates as the global colour-by-colour
// sweep (the extra cell below gives the owned west and south faces the update
// of the box on their far side).  The boxes of one colour are numbered row by
// row (M per row, every fifth cell) and dealt to the threads in that order.
// The block then writes every owned slot, changed or not, to the other
// vector y, so y is a complete copy of the swept x and no block reads what
// another writes.
template <typename T> struct TileGeom;
template <> struct TileGeom<float> {
    static constexpr int TW = 64, LW = 96, TH = 32, THREADS = 640;
};
template <> struct TileGeom<double> {
    static constexpr int TW = 32, LW = 64, TH = 32, THREADS = 384;
};
constexpr int TT_RLO = 10;           // rows loaded above (and below) the owned ones
constexpr int TT_CLO = 16;           // columns loaded left of the owned ones (TMA x offsets: multiples of 16 bytes)
constexpr unsigned long long TT_WAIT_NS = 2000000000ull;  // bound on the wait for the tile copies
template <typename T> __host__ __device__ constexpr int tt_lh() { return TileGeom<T>::TH + 2 * TT_RLO; }
// every TMA x coordinate (c0 - TT_CLO with c0 a multiple of TW) and the window
// width must be whole 16-byte units of the one-byte box-code map, which makes
// them whole units of the value frames too
static_assert(TT_CLO % 16 == 0, "the box-code map's x coordinate must be a multiple of 16 bytes");
static_assert(TileGeom<float>::TW % 16 == 0 && TileGeom<double>::TW % 16 == 0, "tile widths: multiples of 16");
static_assert(TileGeom<float>::LW % 16 == 0 && TileGeom<double>::LW % 16 == 0, "window widths: multiples of 16");
// the colour windows stay inside the loaded window: colour 0 reaches 9 cells
// below / 8 above the owned ones and a box reads one row (column) below and two
// above (right of) its cell
static_assert(TT_RLO >= 10 && TT_CLO >= 10, "halo too small for the five-colour window");
static_assert(TileGeom<float>::LW - TT_CLO - TileGeom<float>::TW >= 10 &&
              TileGeom<double>::LW - TT_CLO - TileGeom<double>::TW >= 10, "right halo too small");

template <typename T> __host__ __device__ constexpr size_t tt_smem()
{
    return (size_t)tt_lh<T>() * TileGeom<T>::LW * (3 * sizeof(T) + 1) + 16;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// wait for phase 0 of the barrier for at most `ns` nanoseconds
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned long long ns)
{
    unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, 0))
        if (global_ns() - t0 > ns) return false;
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];"
        :
        : "r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        :
        : "r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
};
template <> struct Vec16<double> {
    using type = double2;
};

template <typename T>
__global__ void __launch_bounds__(TileGeom<T>::THREADS) k_box_tma(const __grid_constant__ CUtensorMap mx,
                                                           const __grid_constant__ CUtensorMap mc, LevelArgs<T> A,
                                                           const T *x, const T *b, T *y, unsigned *err)
{
    constexpr int TW = TileGeom<T>::TW, LW = TileGeom<T>::LW, TH = TileGeom<T>::TH, LH = tt_lh<T>(), FR = LH * LW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *su = (T *)smem_raw;
    T *sv = su + FR;
    T *sp = sv + FR;
    uint8_t *sc = (uint8_t *)(sp + FR);
    uint64_t *bar = (uint64_t *)(sc + FR);
    const int c0 = blockIdx.x * TW, r0 = blockIdx.y * TH;
    const int col0 = c0 - TT_CLO, row0 = r0 - TT_RLO;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned bytes = (unsigned)(FR * (3 * sizeof(T) + 1));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                     : "memory");
        tma_load_3d(su, &mx, col0, row0, 0, bar);
        tma_load_2d(sc, &mc, col0, row0, bar);
    }
    bool ok = __syncthreads_and(mbar_wait_bounded(bar, TT_WAIT_NS));
    if (!ok) {
        // copies still in flight get a second bounded wait before the block
        // leaves; the NaN in the scalar block makes the solve report failure
        mbar_wait_bounded(bar, TT_WAIT_NS / 2);
        if (threadIdx.x == 0) {
            atomicOr(err + 2, 1u);
            y[3 * A.F] = (T)NAN;
        }
        return;
    }
    const T xi = x[3 * A.F];
    for (int colour = 0; colour < 5; colour++) {
        const int hi = 2 * (4 - colour), lo = hi + 1;
        const int ilo = max(c0 - 1 - lo, 0), ihi = min(c0 - 1 + TW + hi, A.N);
        const int jlo = max(r0 - 1 - lo, 0), jhi = min(r0 - 1 + TH + hi, A.N);
        if (ilo >= ihi || jlo >= jhi) continue;
        // M boxes per row; k / M as (k * ceil(2^16 / M)) >> 16, exact for
        // k < 2^16 / M (here k < 81 * 17 and M <= 17)
        const int M = (ihi - ilo + 4) / 5, nslot = (jhi - jlo) * M;
        const unsigned inv = (65536u + (unsigned)M - 1u) / (unsigned)M;
        for (int k = threadIdx.x; k < nslot; k += TileGeom<T>::THREADS) {
            const int jj = (int)(((unsigned)k * inv) >> 16), m = k - jj * M;
            const int j = jlo + jj;
            // first cell of colour (i + 3 j) mod 5 = colour at or after ilo
            const int i = ilo + (int)((unsigned)(colour + (5 << 28) - 3 * j - ilo) % 5u) + 5 * m;
            if (i >= ihi) continue;
            const int ls = (j + 1 - row0) * LW + (i + 1 - col0);
            const unsigned code = sc[ls];
            if (!(code & BOX_FULL)) continue;
            const long long gs = (long long)(j + 1) * A.P + (i + 1);
            if (code == BOX_ALL)
                box_core<T, true>(su + ls, sv + ls, sp + ls, LW, b + gs, b + A.F + gs, b + 2 * A.F + gs, A.P, xi,
                                  true, true, true, true, A.K);
            else
                box_core<T>(su + ls, sv + ls, sp + ls, LW, b + gs, b + A.F + gs, b + 2 * A.F + gs, A.P, xi,
                            code & BOX_W, code & BOX_E, code & BOX_S, code & BOX_N, A.K);
        }
        __syncthreads();
    }
    // owned slots of the three frames, 16 bytes at a time (P and TW are
    // multiples of 32 elements, so every row segment is whole vectors)
    using V = typename Vec16<T>::type;
    constexpr int VW = 16 / sizeof(T);
    // (compile-time strides: TH rows of TW / VW vectors per frame, the edge
    // tiles' missing rows and columns skipped)
    const int rows = min(TH, A.N + 2 - r0), vpr = min(TW, A.P - c0) / VW;
    constexpr int VPR = TW / VW, PER_FRAME = TH * VPR;
    for (int k = threadIdx.x; k < 3 * PER_FRAME; k += blockDim.x) {
        const int f = k / PER_FRAME, rem = k - f * PER_FRAME;
        const int rr = rem / VPR, vv = rem - rr * VPR;
        if (rr >= rows || vv >= vpr) continue;
        const V *src = (const V *)(su + f * FR + (rr + TT_RLO) * LW + TT_CLO) + vv;
        V *dst = (V *)(y + f * A.F + (long long)(r0 + rr) * A.P + c0) + vv;
        *dst = *src;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < NSCAL) y[3 * A.F + threadIdx.x] = x[3 * A.F + threadIdx.x];
}

// All five colours of the full boxes in one pass, streaming down strips of
// rows.  Block (sx, sy) owns TW slot columns [c0, c0 + TW) of the frame rows
// [r0, r0 + SH) (all three frames).  Its colour-c window is the same as the
// tile sweep's: cells within 2 (4 - c) + 1 columns (rows) before and 2 (4 - c)
// after the owned ones.  The block walks up its rows in phases: in phase d
// colour c relaxes the R cell rows [A0 + R d - (R + 2) c, ... + R) of its
// window (A0 = r0 - 10), all five colours in the same phase, with one block
// barrier between phases.  A box of cell row j reads frame rows j .. j + 3
// and writes frame rows j + 1 and j + 2, so colours R + 2 rows apart touch
// disjoint rows within a phase; across phases every box sees exactly the
// updates of the colour-by-colour sweep: colour c - 1 has finished every row
// up to two above it, colour c + 1 has not reached any row within two below.
// The windows only widen the owned slots horizontally, so a strip recomputes
// 9 of every TW + 9 boxes (the 32-row tiles recompute 48%).
//
// A phase holds twenty row tasks (five colours x R = 4 rows) for ten warps:
// warp w takes tasks w and w + 10, task t being row t mod 4 of colour t / 4,
// one lane per box of the row.
//
// The frames stream through a ring of ten chunks of R rows in shared memory:
// chunk n (frame rows [C0 + n R, C0 + n R + R), C0 = A0 - 4 (R + 2)) lives
// in ring rows [(n mod 10) R, ...).  Phase d reads chunks d .. d + 7; chunk
// d + 8 is copied by TMA during phase d into the slot of chunk d - 2, whose
// owned rows the block wrote out (16 bytes a lane) during phase d - 1, chunk
// n being final once phase n is over.  The right-hand side is read from
// global memory, pulled into L2 two chunks ahead by a bulk tensor prefetch.
// As in the tile sweep the result goes to the level's other vector y, a
// complete copy of the swept x.
template <typename T> struct WaveGeom;
template <> struct WaveGeom<float> {
    static constexpr int TW = 128, LW = 160;
};
template <> struct WaveGeom<double> {
    static constexpr int TW = 64, LW = 96;
};
constexpr int WV_R = 4;               // cell rows of a colour per phase, frame rows per chunk
constexpr int WV_LAG = WV_R + 2;      // rows between consecutive colours within a phase
constexpr int WV_NCHK = 10;           // ring chunks
constexpr int WV_RB = WV_NCHK * WV_R; // ring rows
constexpr int WV_NW = 10;             // warps: two of the 5 R row tasks each
constexpr int WV_THREADS = 32 * WV_NW;
constexpr int WV_A = 10;              // colour 0's window starts 10 rows below the owned ones
// phase d reads frame rows [C0 + R d, C0 + R d + 4 LAG + R + 3) = chunks d .. d + 7,
// chunk d is final after it, and the ring holds chunks d - 1 (written out) .. d + 8 (in flight)
static_assert(WV_R == 4 && WV_LAG == 6 && (4 * WV_LAG + WV_R + 3 - 1) / WV_R == 7 && WV_NCHK == 10,
              "the chunk schedule is worked out for R = 4");
static_assert(5 * WV_R == 2 * WV_NW, "two row tasks per warp");
// R rows up move the colour pattern (i + 3 j) mod 5 by three columns: -3 R = 3 (mod 5)
static_assert((3 * WV_R) % 5 == 2, "the per-phase pattern advance assumes -3 R = 3 (mod 5)");
// every box of a colour row fits the 32 lanes of its warp
static_assert((WaveGeom<float>::TW + 16 + 1 + 4) / 5 <= 32 && (WaveGeom<double>::TW + 16 + 1 + 4) / 5 <= 32,
              "a colour row holds more boxes than a warp has lanes");
// TMA: x coordinates c0 - TT_CLO and widths in whole 16-byte units of the box-code map
static_assert(WaveGeom<float>::TW % 16 == 0 && WaveGeom<double>::TW % 16 == 0, "strip widths: multiples of 16");
static_assert(WaveGeom<float>::LW % 16 == 0 && WaveGeom<double>::LW % 16 == 0, "window widths: multiples of 16");
static_assert(WaveGeom<float>::LW - TT_CLO - WaveGeom<float>::TW >= 10 &&
              WaveGeom<double>::LW - TT_CLO - WaveGeom<double>::TW >= 10, "right halo too small");
// the write-out: one 16-byte vector per lane covers a strip row of a frame
static_assert(WaveGeom<float>::TW * sizeof(float) <= 32 * 16 && WaveGeom<double>::TW * sizeof(double) <= 32 * 16,
              "a strip row must be at most 32 vectors of 16 bytes");
// TMA destinations: every chunk slot and frame of the ring starts on 128 bytes
static_assert((WV_R * WaveGeom<float>::LW) % 128 == 0 && (WV_R * WaveGeom<double>::LW) % 128 == 0,
              "chunk slots must stay 128-byte aligned");

template <typename T> __host__ __device__ constexpr size_t wv_smem()
{
    return (size_t)WV_RB * WaveGeom<T>::LW * (3 * sizeof(T) + 1) + WV_NCHK * sizeof(uint64_t);
}

// the four ring rows -1 .. 2 around a box, as element offsets into a frame
template <typename T> struct RingRows4 {
    T *c;
    int o0, o1, o2, o3;
    __device__ __forceinline__ T &at(int dr, int dc) const
    {
        return c[(dr < 0 ? o0 : dr == 0 ? o1 : dr == 1 ? o2 : o3) + dc];
    }
};

// wait for the phase of the given parity of the barrier, at most `ns` nanoseconds
__device__ __forceinline__ bool mbar_wait_parity_bounded(uint64_t *bar, unsigned parity, unsigned long long ns)
{
    unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > ns) return false;
    return true;
}

__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *map, int x, int y, int z)
{
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];"
                 :
                 : "l"(map), "r"(x), "r"(y), "r"(z)
                 : "memory");
}

// the right-hand side of the box rows of cell (i, j): bW, bE, bS, bN, bC
// (32-bit slot offsets: 3 F + P stays below 2^31 on the levels swept here)
template <typename T> __device__ __forceinline__ void wave_rhs(const T *b, int F, int P, int i, int j, T *q)
{
    const int gs = (j + 1) * P + (i + 1);
    q[0] = b[gs];
    q[1] = b[gs + 1];
    q[2] = b[F + gs];
    q[3] = b[F + gs + P];
    q[4] = b[2 * F + gs];
}

template <typename T>
__global__ void __launch_bounds__(WV_THREADS, 2) k_box_wave(const __grid_constant__ CUtensorMap mx,
                                                            const __grid_constant__ CUtensorMap mc,
                                                            const __grid_constant__ CUtensorMap mb, LevelArgs<T> A,
                                                            const T *x, const T *b, T *y, int SH, unsigned *err)
{
    constexpr int TW = WaveGeom<T>::TW, LW = WaveGeom<T>::LW, R = WV_R, RB = WV_RB, FR = RB * LW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *su = (T *)smem_raw;
    T *sv = su + FR;
    T *sp = sv + FR;
    uint8_t *sc = (uint8_t *)(sp + FR);
    uint64_t *bar = (uint64_t *)(sc + FR);
    const int N = A.N;
    const int c0 = blockIdx.x * TW, r0 = blockIdx.y * SH;
    const int col0 = c0 - TT_CLO, A0 = r0 - WV_A;
    const int rend = min(r0 + SH, N + 2);
    // phases: until colour 4, the last, has passed the end of its window
    // (every other colour's window ends earlier in phase terms)
    int ND = 0;
#pragma unroll
    for (int c = 0; c < 5; c++) {
        const int jhi = min(r0 - 1 + SH + 2 * (4 - c), N);
        ND = max(ND, (jhi - (A0 - WV_LAG * c) + R - 1) / R);
    }
    // the highest chunk a box reads: colour 0's last row plus two
    const int LAST = (min(r0 - 1 + SH + 8, N) + 2 - A0) / R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < WV_NCHK; q++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + q)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int rows_total = N + 2;
    auto load_chunk = [&](int n) {
        const int q = n % WV_NCHK, X = A0 + n * R;
        const unsigned bytes = (unsigned)(R * LW * (3 * sizeof(T) + 1));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar + q)), "r"(bytes)
                     : "memory");
        for (int f = 0; f < 3; f++) tma_load_3d(su + f * FR + q * R * LW, &mx, col0, X, f, bar + q);
        tma_load_2d(sc + q * R * LW, &mc, col0, X, bar + q);
        // a hint for the right-hand side three chunks on, kept inside the tensor
        const int Xb = X + 3 * R;
        if (Xb < rows_total) tma_prefetch_3d(&mb, max(col0, 0), max(Xb, 0), 0);
    };
    // chunk n sits in slot n mod 10, the (n / 10)-th copy into that slot
    auto wait_chunk = [&](int n, unsigned long long ns) {
        return mbar_wait_parity_bounded(bar + n % WV_NCHK, (unsigned)(n / WV_NCHK) & 1u, ns);
    };
    if (threadIdx.x == 0) {
        load_chunk(0);
        if (LAST >= 1) load_chunk(1);
    }
    const T xi = x[3 * A.F];
    const int F = (int)A.F, P = A.P;
    // task k of this warp: row rr of colour cc; at phase d its cell row is
    // j = A0 + R d - LAG cc + rr, at ring row lm = (j - A0) mod RB (rows
    // below A0 are never read), and lane `lane` relaxes column
    // i = iu + ph + 5 lane, the first cell of the colour pattern
    // (i + 3 j) mod 5 = cc at or after iu plus every fifth.  bq[k]: the
    // right-hand side of that box, bn[k] the next phase's; each is loaded two
    // phases ahead of its use.
    int jt[2], lm[2], ph[2], iu[2], jlo[2], jhi[2], ilo[2], ihi[2];
    bool act[2], actn[2];  // the lane's box of this phase, of the next, lies in the window
    T bq[2][5], bn[2][5];
    auto in_window = [&](int k, int j, int i) {
        return j >= jlo[k] && j < jhi[k] && i >= ilo[k] && i < ihi[k];
    };
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int t = warp + WV_NW * k, rr = t & 3, cc = t >> 2;
        const int lo = 2 * (4 - cc) + 1, hi = lo - 1;
        iu[k] = c0 - 1 - lo;
        jlo[k] = max(r0 - 1 - lo, 0);
        jhi[k] = min(r0 - 1 + SH + hi, N);
        ilo[k] = max(iu[k], 0);
        ihi[k] = min(c0 - 1 + TW + hi, N);
        jt[k] = A0 - WV_LAG * cc + rr;
        lm[k] = (2 * RB - WV_LAG * cc + rr) % RB;
        ph[k] = (int)((unsigned)(cc + (5 << 28) - 3 * jt[k] - iu[k]) % 5u);
#pragma unroll
        for (int q = 0; q < 5; q++) bq[k][q] = bn[k][q] = (T)0;
        const int i = iu[k] + ph[k] + 5 * lane;
        act[k] = in_window(k, jt[k], i);
        if (act[k]) wave_rhs(b, F, P, i, jt[k], bq[k]);
        const int p1 = ph[k] + 3 < 5 ? ph[k] + 3 : ph[k] - 2, i1 = iu[k] + p1 + 5 * lane;
        actn[k] = in_window(k, jt[k] + R, i1);
        if (actn[k]) wave_rhs(b, F, P, i1, jt[k] + R, bn[k]);
    }
    using V = typename Vec16<T>::type;
    constexpr int VW = 16 / sizeof(T);
    // owned rows of chunk n: twelve (frame, row) pairs over the ten warps,
    // one 16-byte vector per lane
    auto write_chunk = [&](int n) {
        const int col = c0 + lane * VW;
        if (lane * VW >= TW || col >= A.P) return;
        for (int p = warp; p < 3 * R; p += WV_NW) {
            const int f = p / R, rr = p - f * R, X = A0 + n * R + rr;
            if (X >= r0 && X < rend) {
                const int o = ((n % WV_NCHK) * R + rr) * LW + TT_CLO + lane * VW;
                *(V *)(y + f * A.F + (long long)X * A.P + col) = *(const V *)(su + f * FR + o);
            }
        }
    };
    for (int d = 0; d < ND; d++) {
        // phase d reads chunks d - 6 .. d + 1 (those in 0 .. LAST); d + 1 is
        // the only one not yet confirmed (at d = 0: both of the prologue)
        // (warp 0 waits on the barriers, the block barrier passes the copies
        // on to the other warps)
        bool ok = true;
        if (warp == 0) {
            if (d == 0) ok = wait_chunk(0, TT_WAIT_NS);
            if (d + 1 <= LAST) ok = wait_chunk(d + 1, TT_WAIT_NS) && ok;
        }
        if (!__syncthreads_and(ok)) {
            // copies still in flight get a second bounded wait before the
            // block leaves; the NaN in the scalar block makes the solve fail
            if (warp == 0) {
                if (d == 0) wait_chunk(0, TT_WAIT_NS / 2);
                if (d + 1 <= LAST) wait_chunk(d + 1, TT_WAIT_NS / 2);
            }
            if (threadIdx.x == 0) {
                atomicOr(err + 2, 1u);
                y[3 * A.F] = (T)NAN;
            }
            return;
        }
        // chunk d + 2 into the slot of chunk d - 8 (written out before the
        // barrier above); the generic-proxy reads are ordered before the copy
        if (threadIdx.x == 0 && d + 2 <= LAST) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            load_chunk(d + 2);
        }
#pragma unroll
        for (int k = 0; k < 2; k++) {
            if (act[k]) {
                const int lc = iu[k] + ph[k] + 5 * lane + 1 - col0;
                const int l1 = lm[k] + 1 < RB ? lm[k] + 1 : lm[k] + 1 - RB;
                const int l2 = lm[k] + 2 < RB ? lm[k] + 2 : lm[k] + 2 - RB;
                const int l3 = lm[k] + 3 < RB ? lm[k] + 3 : lm[k] + 3 - RB;
                const int o0 = lm[k] * LW + lc, o1 = l1 * LW + lc, o2 = l2 * LW + lc, o3 = l3 * LW + lc;
                const unsigned code = sc[o1];
                if (code & BOX_FULL) {
                    const RingRows4<T> U{su, o0, o1, o2, o3}, Vv{sv, o0, o1, o2, o3}, Pv{sp, o0, o1, o2, o3};
                    const T *q = bq[k];
                    if (code == BOX_ALL)
                        box_solve_v<T, true>(U, Vv, Pv, q[0], q[1], q[2], q[3], q[4], xi, true, true, true, true, A.K);
                    else
                        box_solve_v<T>(U, Vv, Pv, q[0], q[1], q[2], q[3], q[4], xi, code & BOX_W, code & BOX_E,
                                       code & BOX_S, code & BOX_N, A.K);
                }
            }
            // this task's box of the next phase: R rows up, the pattern three
            // columns on; its right-hand side is already loaded, the one of
            // the phase after is fetched now
            jt[k] += R;
            lm[k] = lm[k] + R < RB ? lm[k] + R : lm[k] + R - RB;
            ph[k] = ph[k] + 3 < 5 ? ph[k] + 3 : ph[k] - 2;
#pragma unroll
            for (int q = 0; q < 5; q++) bq[k][q] = bn[k][q];
            act[k] = actn[k];
            const int p2 = ph[k] + 3 < 5 ? ph[k] + 3 : ph[k] - 2, i2 = iu[k] + p2 + 5 * lane;
            actn[k] = in_window(k, jt[k] + R, i2);
            if (actn[k]) wave_rhs(b, F, P, i2, jt[k] + R, bn[k]);
        }
        // chunk d - 7 became final with phase d - 1 and is not read any more
        if (d >= 7) write_chunk(d - 7);
    }
    __syncthreads();
    for (int n = max(ND - 7, 0); n <= LAST; n++) write_chunk(n);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < NSCAL) y[3 * A.F + threadIdx.x] = x[3 * A.F + threadIdx.x];
}

// Box code of every cell (one byte per slot): BOX_FULL for an internal cell
// with no ghost face (a full box of Sect. 4.1.1), with BOX_W, BOX_E, BOX_S,
// BOX_N for its internal faces; 0 for every other slot.  Once per geometry.
__global__ void k_box_codes(int N, int P, long long F, const uint8_t *tU, const uint8_t *tV, const uint8_t *tP,
                            uint8_t *code)
{
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= F) return;
    const int row = (int)(s / P), col = (int)(s - (long long)row * P);
    uint8_t c = 0;
    if (row >= 1 && row <= N && col >= 1 && col <= N && tP[s] == T_INTERNAL) {
        const uint8_t tW = tU[s], tE = tU[s + 1], tS = tV[s], tN = tV[s + P];
        if (tW != T_GHOST && tE != T_GHOST && tS != T_GHOST && tN != T_GHOST)
            c = BOX_FULL | (tW == T_INTERNAL ? BOX_W : 0) | (tE == T_INTERNAL ? BOX_E : 0) |
                (tS == T_INTERNAL ? BOX_S : 0) | (tN == T_INTERNAL ? BOX_N : 0);
    }
    code[s] = c;
}

template <typename T>
__global__ void k_box_full(LevelArgs<T> A, T *x, const T *b, int colour)
{
    int j = blockIdx.y;
    int i0 = ((colour - 3 * j) % 5 + 5) % 5;
    int i = i0 + 5 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= A.N) return;
    box_full_one<T>(A, x, b, i, j);
}

// Prepare the rows of every cut box for the current alpha: the full row of
// each box unknown as (index, coefficient) pairs (frozen neighbours
// included, so that the residual needs only gathers) and the inverse of the
// box matrix by the same pivoted LU (FP64; an FP32 copy for FP32 sweeps).
__global__ void k_cut_prepare(LevelArgs<double> A, CutList cut, GhostList gh, int n)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long s = cut.cell[k];
    const long long F = A.F, P = A.P;
    long long unk[5] = {s, s + 1, F + s, F + s + P, 2 * F + s};
    uint8_t ft[4] = {A.tU[s], A.tU[s + 1], A.tV[s], A.tV[s + P]};
    bool act[5];
    for (int f = 0; f < 4; f++) act[f] = ft[f] == T_INTERNAL || ft[f] == T_GHOST;
    act[4] = true;
    double M[5][5];
    for (int r = 0; r < 5; r++)
        for (int c = 0; c < 5; c++) M[r][c] = 0.0;
    auto put = [&](int f, int m, long long idx, double coef) {
        cut.sidx[(long long)(f * CUT_ST + m) * cut.cap + k] = (int)idx;
        cut.scoef[(long long)(f * CUT_ST + m) * cut.cap + k] = coef;
        cut.scoeff[(long long)(f * CUT_ST + m) * cut.cap + k] = (float)coef;
        for (int c = 0; c < 5; c++)
            if (act[c] && unk[c] == idx) M[f][c] += coef;
    };
    for (int f = 0; f < 5; f++)
        for (int m = 0; m < CUT_ST; m++) {
            cut.sidx[(long long)(f * CUT_ST + m) * cut.cap + k] = (int)unk[4];
            cut.scoef[(long long)(f * CUT_ST + m) * cut.cap + k] = 0.0;
            cut.scoeff[(long long)(f * CUT_ST + m) * cut.cap + k] = 0.f;
        }
    for (int f = 0; f < 4; f++) {
        cut.row[(long long)f * cut.cap + k] = act[f] ? (int)unk[f] : -1;
        if (!act[f]) {
            M[f][f] = 1.0;
            continue;
        }
        if (ft[f] == T_INTERNAL) {
            long long o = unk[f];
            bool isu = f < 2;
            long long loc = isu ? o : o - F;
            long long base = isu ? 0 : F;
            long long pm = isu ? loc - 1 : loc - P;
            put(f, 0, o, A.d);
            put(f, 1, base + loc + 1, -A.a);
            put(f, 2, base + loc - 1, -A.a);
            put(f, 3, base + loc + P, -A.a);
            put(f, 4, base + loc - P, -A.a);
            put(f, 5, 2 * F + loc, A.q);
            put(f, 6, 2 * F + pm, -A.q);
        } else {
            int g = cut.gface[(long long)f * cut.cap + k];
            int nst = gh.nst[g];
            for (int m = 0; m < nst; m++) put(f, m, gh.st[(long long)m * gh.cap + g], gh.w[(long long)m * gh.cap + g]);
        }
    }
    cut.row[4ll * cut.cap + k] = (int)unk[4];
    put(4, 0, s + 1, A.q);
    put(4, 1, s, -A.q);
    put(4, 2, F + s + P, A.q);
    put(4, 3, F + s, -A.q);
    put(4, 4, 3 * F, -1.0);
    // inverse by pivoted LU on [M | I]
    double I[5][5];
    for (int r = 0; r < 5; r++)
        for (int c = 0; c < 5; c++) I[r][c] = r == c ? 1.0 : 0.0;
    bool ok = true;
    for (int c = 0; c < 5; c++) {
        int pr = c;
        double best = fabs(M[c][c]);
        for (int r = c + 1; r < 5; r++)
            if (fabs(M[r][c]) > best) {
                best = fabs(M[r][c]);
                pr = r;
            }
        if (!(best > 0.0)) { ok = false; break; }
        for (int m = 0; m < 5; m++) {
            double t = M[c][m]; M[c][m] = M[pr][m]; M[pr][m] = t;
            t = I[c][m]; I[c][m] = I[pr][m]; I[pr][m] = t;
        }
        for (int r = c + 1; r < 5; r++) {
            double fct = M[r][c] / M[c][c];
            for (int m = 0; m < 5; m++) {
                M[r][m] -= fct * M[c][m];
                I[r][m] -= fct * I[c][m];
            }
        }
    }
    for (int col = 0; col < 5; col++)
        for (int r = 4; r >= 0; r--) {
            double acc = ok ? I[r][col] : 0.0;
            for (int m = r + 1; m < 5; m++) acc -= M[r][m] * I[m][col];
            I[r][col] = ok ? acc / M[r][r] : 0.0;
        }
    for (int r = 0; r < 5; r++)
        for (int c = 0; c < 5; c++) {
            cut.minv[(long long)(r * 5 + c) * cut.cap + k] = I[r][c];
            cut.minvf[(long long)(r * 5 + c) * cut.cap + k] = (float)I[r][c];
        }
}

template <typename T> __device__ inline const T *cut_coef(const CutList &c);
template <> __device__ inline const double *cut_coef<double>(const CutList &c) { return c.scoef; }
template <> __device__ inline const float *cut_coef<float>(const CutList &c) { return c.scoeff; }
template <typename T> __device__ inline const T *cut_minv(const CutList &c);
template <> __device__ inline const double *cut_minv<double>(const CutList &c) { return c.minv; }
template <> __device__ inline const float *cut_minv<float>(const CutList &c) { return c.minvf; }

// one prepared cut box: gather the five row residuals, apply the inverse
template <typename T> __device__ __forceinline__ void box_cut_pre(T *x, const T *b, const CutList &cut, int k)
{
    const T *coef = cut_coef<T>(cut);
    const T *mi = cut_minv<T>(cut);
    T r[5];
    int row[5];
#pragma unroll
    for (int f = 0; f < 5; f++) {
        row[f] = cut.row[(long long)f * cut.cap + k];
        T acc = 0;
#pragma unroll
        for (int m = 0; m < CUT_ST; m++) {
            long long e = (long long)(f * CUT_ST + m) * cut.cap + k;
            acc += coef[e] * x[cut.sidx[e]];
        }
        r[f] = row[f] >= 0 ? b[row[f]] - acc : (T)0;
    }
#pragma unroll
    for (int f = 0; f < 5; f++) {
        if (row[f] < 0) continue;
        T d = 0;
#pragma unroll
        for (int c = 0; c < 5; c++) d += mi[(long long)(f * 5 + c) * cut.cap + k] * r[c];
        x[row[f]] += d;
    }
}

// one prepared cut box relaxed by a whole warp: lane e (and e + 32) loads
// entry e of the 5 x CUT_ST row entries and gathers its x, so the gathers of
// a box are in flight together; lanes 0..4 then accumulate one row each in
// the order box_cut_pre uses (same rounding) and apply the inverse.  k must
// be the same on every lane of the warp.
template <typename T> __device__ __forceinline__ void box_cut_warp(T *x, const T *b, const CutList &cut, int k, int lane)
{
    constexpr int NE = 5 * CUT_ST;
    const T *coef = cut_coef<T>(cut);
    const T *mi = cut_minv<T>(cut);
    T c0 = 0, x0 = 0, c1 = 0, x1 = 0;
    {
        const long long e = (long long)lane * cut.cap + k;
        c0 = coef[e];
        x0 = x[cut.sidx[e]];
    }
    if (lane < NE - 32) {
        const long long e = (long long)(lane + 32) * cut.cap + k;
        c1 = coef[e];
        x1 = x[cut.sidx[e]];
    }
    const int f = lane < 5 ? lane : 0;
    const int row = cut.row[(long long)f * cut.cap + k];
    const T bf = row >= 0 ? b[row] : (T)0;
    T acc = 0;
#pragma unroll
    for (int m = 0; m < CUT_ST; m++) {
        const int e = f * CUT_ST + m;
        const T ca = __shfl_sync(0xffffffffu, c0, e & 31), xa = __shfl_sync(0xffffffffu, x0, e & 31);
        const T cb = __shfl_sync(0xffffffffu, c1, e & 31), xb = __shfl_sync(0xffffffffu, x1, e & 31);
        acc += (e < 32 ? ca : cb) * (e < 32 ? xa : xb);
    }
    const T r = row >= 0 ? bf - acc : (T)0;
    T d = 0;
#pragma unroll
    for (int cc = 0; cc < 5; cc++) {
        const T rc = __shfl_sync(0xffffffffu, r, cc);
        d += mi[(long long)(f * 5 + cc) * cut.cap + k] * rc;
    }
    if (lane < 5 && row >= 0) x[row] += d;
}

// all colours of the cut boxes in one block of 32
// warps: the barrier between colours orders them; boxes of one colour are
// independent
template <typename T>
__global__ void __launch_bounds__(1024) k_box_cut(LevelArgs<T> A, T *x, const T *b, CutList cut, GhostList gh)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int colour = 0; colour < cut.ncol; colour++) {
        int beg = cut.off[colour], end = cut.off[colour + 1];
        for (int k = beg + warp; k < end; k += nw) box_cut_warp<T>(x, b, cut, k, lane);
        __syncthreads();
    }
}

// ------------------------------------------------------- cluster kernels
// The CTAs of a thread-block cluster are scheduled together and share a
// hardware barrier, so phases that must follow one another (the colours of
// the cut boxes) run in one launch over several SMs instead of one launch per
// phase.  Ghost sweeps and whole small-level relaxations were measured slower
// on a cluster (its SMs limit the memory parallelism of their gathers).
constexpr int CL_CTAS = 8;        // CTAs per cluster (the portable maximum)
constexpr int CL_THREADS = 1024;  // threads per CTA

__device__ __forceinline__ unsigned cl_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cl_size()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// every thread of the cluster: writes before it are seen by reads after it
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// all colours of the cut boxes, a warp per box over the whole cluster
template <typename T> __global__ void __launch_bounds__(CL_THREADS) k_box_cut_cluster(T *x, const T *b, CutList cut)
{
    const int lane = threadIdx.x & 31;
    const int wpc = blockDim.x >> 5;
    const int gw = (int)cl_rank() * wpc + (threadIdx.x >> 5), nw = (int)cl_size() * wpc;
    for (int colour = 0; colour < cut.ncol; colour++) {
        const int beg = cut.off[colour], end = cut.off[colour + 1];
        for (int k = beg + gw; k < end; k += nw) box_cut_warp<T>(x, b, cut, k, lane);
        cl_sync();
    }
}

// the cut boxes [beg, end) of one colour, a warp per box over the whole GPU
template <typename T> __global__ void __launch_bounds__(256) k_box_cut_colour(T *x, const T *b, CutList cut, int beg, int end)
{
    const int k = beg + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (k < end) box_cut_warp<T>(x, b, cut, k, threadIdx.x & 31);
}

// internal faces with no internal cell: point Jacobi (compute, then apply)
template <typename T>
__global__ void k_lonely_update(LevelArgs<T> A, const T *x, const T *b, const int *list, int n, T *upd)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    long long o = list[k];
    bool isu = o < A.F;
    long long loc = isu ? o : o - A.F;
    const T *xx = isu ? x : x + A.F;
    const T *pp = x + 2 * A.F;
    long long pm = isu ? loc - 1 : loc - A.P;
    T Ax = A.d * xx[loc] - A.a * (xx[loc + 1] + xx[loc - 1] + xx[loc + A.P] + xx[loc - A.P]) + A.q * (pp[loc] - pp[pm]);
    upd[k] = (b[o] - Ax) / A.d;
}

template <typename T> __global__ void k_apply_list(T *x, const int *list, const T *upd, int n)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) x[list[k]] += upd[k];
}

// ------------------------------------------------------- xi / mean pressure

// per-thread sums in the arithmetic type (FP32 for FP32 sweeps: no FP64
// work per cell), block sums in FP64
template <typename T>
__global__ void k_scalar_partial(LevelArgs<T> A, const T *x, const T *b, double *part)
{
    T s = 0, m = 0;
    const long long nq = (long long)(A.N + 2) * A.P / 4;
    const T *u = x, *v = x + A.F, *p = x + 2 * A.F;
    // four consecutive cells per thread, vector loads (internal cells lie in
    // frame rows 1..N, so the loads one row up stay in the frame)
    for (long long qd = blockIdx.x * (long long)blockDim.x + threadIdx.x; qd < nq; qd += (long long)gridDim.x * blockDim.x) {
        const long long s0 = 4 * qd;
        uint8_t tp[4];
        ldt4(A.tP + s0, tp);
        if (tp[0] != T_INTERNAL && tp[1] != T_INTERNAL && tp[2] != T_INTERNAL && tp[3] != T_INTERNAL) continue;
        T uh[5], v4[4], vU[4], bc[4], p4[4];
        ld4(u + s0, uh);
        uh[4] = u[s0 + 4];
        ld4(v + s0, v4);
        ld4(v + s0 + A.P, vU);
        ld4(b + 2 * A.F + s0, bc);
        ld4(p + s0, p4);
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (tp[q] == T_INTERNAL) {
                T div = (uh[q + 1] - uh[q] + vU[q] - v4[q]) * A.q;
                s += div - bc[q];
                m += p4[q];
            }
    }
    __shared__ double ss[256], sm[256];
    ss[threadIdx.x] = (double)s;
    sm[threadIdx.x] = (double)m;
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

// xi <- mean(div u - b_c); shift <- (b_mean - h^2 sum p) / (h^2 n_int)
template <typename T>
__global__ void k_scalar_final(const double *part, int nb, T *x, const T *b, long long imean, double h2, const int *nint,
                               double *shift, int defer)
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
        double n = (double)*nint;
        x[imean] = (T)(ss[0] / n);
        const double sh = ((double)b[imean] - h2 * sm[0]) / (h2 * n);
        shift[0] = sh;
        // deferred: the shift that makes the stored pressures satisfy the
        // mean row, kept beside xi instead of being added to every p
        if (defer) x[imean + PSHIFT_SLOT] = (T)sh;
    }
}

// p += shift on internal and ghost cells, four consecutive slots per thread
template <typename T> __global__ void k_pshift(LevelArgs<T> A, T *x, const double *shift)
{
    int c0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    int row = blockIdx.y;
    if (c0 >= A.P) return;
    long long s0 = (long long)row * A.P + c0;
    uint8_t t[4];
    ldt4(A.tP + s0, t);
    if (t[0] < T_INTERNAL && t[1] < T_INTERNAL && t[2] < T_INTERNAL && t[3] < T_INTERNAL) return;
    T p4[4];
    ld4(x + 2 * A.F + s0, p4);
    const T sh = (T)shift[0];
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (t[q] == T_INTERNAL || t[q] == T_GHOST) p4[q] += sh;
    st4(x + 2 * A.F + s0, p4);
}

// --------------------------------------------------------- ghost relaxation

// Eq. (ghostrelax), Jacobi over every ghost-class row: w += dtau (g - B w)
template <typename T>
__global__ void k_ghost_update(GhostList gh, int nrows, const T *x, const T *b, T dtau)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrows) return;
    gupd<T>(gh)[k] = dtau * ghost_row_residual<T, false>(gh, k, x, b, nullptr);
}

template <typename T> __global__ void k_ghost_apply(GhostList gh, int nrows, T *x)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nrows) x[gh.node[k]] += gupd<T>(gh)[k];
}

// lambda Jacobi sweeps of Eq. (ghostrelax) with x fixed: after sweep s the
// ghost-class values are x + d_s (d_0 = 0), and sweep s + 1 computes
// d_(s+1) = d_s + dtau (b - B (x + d_s)) reading d_s of the referenced ghost
// rows through strow; the last d is added to x by k_ghost_acc_apply.  The
// iterates are those of the compute/apply pairs (up to rounding), in lambda + 1
// launches instead of 2 lambda.
template <typename T> __device__ inline T *gacc(const GhostList &gh);
template <> __device__ inline double *gacc<double>(const GhostList &gh) { return gh.acc; }
template <> __device__ inline float *gacc<float>(const GhostList &gh) { return gh.accf; }

template <typename T>
__global__ void k_ghost_acc_sweep(GhostList gh, int nrows, const T *x, const T *b, T dtau, int sweep)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrows) return;
    const T *din = gacc<T>(gh) + (long long)(sweep & 1) * gh.cap;
    T *dout = gacc<T>(gh) + (long long)((sweep + 1) & 1) * gh.cap;
    const T s = sweep > 0 ? ghost_row_residual<T, true>(gh, k, x, b, din) : ghost_row_residual<T, false>(gh, k, x, b, nullptr);
    dout[k] = (sweep > 0 ? din[k] : (T)0) + dtau * s;
}

template <typename T> __global__ void k_ghost_acc_apply(GhostList gh, int nrows, T *x, int sweeps)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nrows) x[gh.node[k]] += gacc<T>(gh)[(long long)(sweeps & 1) * gh.cap + k];
}

// The lambda sweeps of k_ghost_acc_sweep in one launch (Eq. ghostrelax with x
// fixed).  Block q owns rows [q GC_OWN, (q + 1) GC_OWN) and relaxes them with
// their closure (every row within lambda - 1 stencil links) in shared memory:
// after sweep s a row at link distance h is exact for s <= lambda - h, so the
// owned rows end with exactly the iterate of the one-sweep-per-launch form, and
// a link that leaves the closure (distance lambda) counts as zero.  Each row
// repeats that form's expressions in the same order (no correction added in
// the first sweep).  The owned rows' corrections go
// where k_ghost_acc_apply reads them after lambda sweeps; no block writes x.
template <typename T>
__global__ void __launch_bounds__(GC_THREADS) k_ghost_fused(GhostList gh, int nrows, const T *x, const T *b, T dtau,
                                                             int lambda)
{
    constexpr int RPT = GC_CAP / GC_THREADS;
    __shared__ T dsh[2][GC_CAP];
    const int n = gh.cl_n[blockIdx.x];
    const int lo = blockIdx.x * GC_OWN, hi = min(lo + GC_OWN, nrows);
    const int *grow = gh.cl_row + (long long)blockIdx.x * GC_CAP;
    const int16_t *glnk = gh.cl_lnk + (long long)blockIdx.x * GH_ST * GC_CAP;
    const T *w = gw<T>(gh);
    int kr[RPT], nst[RPT], lnk[RPT][GH_ST];
    T wv[RPT][GH_ST], xv[RPT][GH_ST], bv[RPT];
#pragma unroll
    for (int r = 0; r < RPT; r++) {
        const int c = threadIdx.x + r * GC_THREADS;
        const bool valid = c < n;
        const int k = valid ? grow[c] : 0;
        kr[r] = valid ? k : -1;
        nst[r] = valid ? gh.nst[k] : 0;
        int idx[GH_ST];
#pragma unroll
        for (int q = 0; q < GH_ST; q++) {
            const long long e = (long long)q * gh.cap + k;
            idx[q] = q < nst[r] ? gh.st[e] : 0;
            lnk[r][q] = q < nst[r] ? (int)glnk[q * GC_CAP + c] : -1;
            wv[r][q] = q < nst[r] ? w[e] : (T)0;
        }
#pragma unroll
        for (int q = 0; q < GH_ST; q++) xv[r][q] = q < nst[r] ? x[idx[q]] : (T)0;
        bv[r] = valid ? b[gh.node[k]] : (T)0;
        if (valid) dsh[0][c] = (T)0;
    }
    __syncthreads();
    int cur = 0;
    for (int s = 0; s < lambda; s++) {
#pragma unroll
        for (int r = 0; r < RPT; r++) {
            if (kr[r] < 0) continue;
            const int c = threadIdx.x + r * GC_THREADS;
            T xs[GH_ST];
#pragma unroll
            for (int q = 0; q < GH_ST; q++) {
                xs[q] = xv[r][q];
                if (s > 0 && lnk[r][q] >= 0) xs[q] += dsh[cur][lnk[r][q]];
            }
            T res = bv[r];
#pragma unroll
            for (int q = 0; q < GH_ST; q++)
                if (q < nst[r]) res -= wv[r][q] * xs[q];
            dsh[cur ^ 1][c] = dsh[cur][c] + dtau * res;
        }
        __syncthreads();
        cur ^= 1;
    }
    T *dout = gacc<T>(gh) + (long long)(lambda & 1) * gh.cap;
#pragma unroll
    for (int r = 0; r < RPT; r++)
        if (kr[r] >= lo && kr[r] < hi) dout[kr[r]] = dsh[cur][threadIdx.x + r * GC_THREADS];
}

// ---------------------------------------------------------------- transfers

// Eq. (restop) where the whole stencil is of the coarse node's class,
// otherwise the plain mean of the fine residuals of that class (Eq. restop5)
template <typename T>
__global__ void k_restrict(int Nf, int Pf, long long Ff, const uint8_t *tUf, const uint8_t *tVf, const uint8_t *tPf,
                           int Nc, int Pc, long long Fc, const uint8_t *tUc, const uint8_t *tVc, const uint8_t *tPc,
                           const T *r, T *bH, T *xz)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= Pc) return;
    int I = col - 1, J = row - 1;
    long long sc = (long long)row * Pc + col;
    const uint8_t *tf[3] = {tUf, tVf, tPf};
    const uint8_t tcg[3] = {tUc[sc], tVc[sc], tPc[sc]};
    // every type and residual of the three stencils is loaded before the
    // arithmetic (fine indices clamped into the frame; only nodes of the
    // grid take part)
    uint8_t tff[3][6];
    T rv[3][6];
    bool in[3][6];
#pragma unroll
    for (int g = 0; g < 3; g++)
#pragma unroll
        for (int k = 0; k < 6; k++) {
            int di, dj;
            if (g == G_U) { di = k % 3 - 1; dj = k / 3; }
            else if (g == G_V) { di = k % 2; dj = k / 2 - 1; }
            else { di = k % 2; dj = k / 2; }
            const int fi = 2 * I + di, fj = 2 * J + dj;
            in[g][k] = (g != G_P || k < 4) && in_grid(g, Nf, fi, fj);
            const int ci = min(max(fi, -1), Nf), cj = min(max(fj, -1), Nf);
            const long long sl = (long long)(cj + 1) * Pf + (ci + 1);
            tff[g][k] = tf[g][sl];
            rv[g][k] = r[g * Ff + sl];
        }
#pragma unroll
    for (int g = 0; g < 3; g++) {
        const uint8_t t = tcg[g];
        T out = 0;
        if (t != T_INACTIVE) {
            bool all = true;
            int cnt = 0;
            T sw = 0, su = 0;
#pragma unroll
            for (int k = 0; k < 6; k++) {
                if (g == G_P && k >= 4) break;
                const T wt = g == G_U ? (T)(k % 3 == 1 ? 0.25 : 0.125) : g == G_V ? (T)(k / 2 == 1 ? 0.25 : 0.125) : (T)0.25;
                if (in[g][k] && same_class(t, tff[g][k])) {
                    sw += wt * rv[g][k];
                    su += rv[g][k];
                    cnt++;
                } else all = false;
            }
            out = all ? sw : (cnt > 0 ? su / (T)cnt : (T)0);
        }
        bH[g * Fc + sc] = out;
        if (xz) xz[g * Fc + sc] = (T)0;  // the coarse iterate starts from zero
    }
    if (row == 0 && col == 0) {
        bH[3 * Fc] = r[3 * Ff];
        if (xz)
            for (int q = 0; q < NSCAL; q++) xz[3 * Fc + q] = (T)0;
    }
}

// The residual of a level restricted in one pass (the cycle's residual and
// Eq. restop / restop5 fused): block tiles of RR_TX x RR_TY coarse slots,
// grid-stride.  For each tile the block first computes, into shared memory,
// the fine residuals of the fine slots its restriction stencils reach: the
// internal rows from x and b (the expressions of k_residual4, so the same
// bits), the ghost-class rows read from r (k_ghost_residual wrote them just
// before), 0 elsewhere.  Then each thread restricts one coarse slot exactly
// as k_restrict does and zeroes the coarse iterate.  The fine residual never
// goes to memory.  Per block: [0] the sum of p over the internal fine cells
// of its tiles (each fine cell lies in the stencil of one coarse cell), for
// the mean row that k_residual_final then writes into bH; [1] 0 (no norm).
constexpr int RR_TX = 32, RR_TY = 8;
// fine slots of a tile's stencils: columns [2 C0 - 4, 2 C0 + 64) (whole
// 16-byte quads), rows [2 R0 - 2, 2 R0 + 15)
constexpr int RR_FW = 2 * RR_TX + 4, RR_FH = 2 * RR_TY + 1, RR_QW = RR_FW / 4;
static_assert(RR_TX * RR_TY == 256, "one coarse slot per thread");
static_assert(RR_TX % 2 == 0 && RR_FW % 4 == 0, "quads of the region start on 16-byte slots");

template <typename T> __host__ __device__ constexpr size_t rr_smem()
{
    return (size_t)3 * RR_FW * RR_FH * (sizeof(T) + 1);
}

template <typename T>
__global__ void __launch_bounds__(256) k_residual_restrict(LevelArgs<T> A, int Nc, int Pc, long long Fc,
                                                           const uint8_t *tUc, const uint8_t *tVc,
                                                           const uint8_t *tPc, const T *x, const T *b, const T *r,
                                                           T *bH, T *xz, double *part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *rs = (T *)smem_raw;                                      // [3][RR_FH][RR_FW]
    uint8_t *ts = (uint8_t *)(rs + 3 * RR_FW * RR_FH);         // [3][RR_FH][RR_FW]
    constexpr int FS = RR_FW * RR_FH;
    const int Nf = A.N, P = A.P;
    const long long Ff = A.F;
    const T *u = x, *v = x + Ff, *p = x + 2 * Ff;
    const T xi = x[3 * Ff];
    const int ntx = (Pc + RR_TX - 1) / RR_TX, nty = (Nc + 2 + RR_TY - 1) / RR_TY;
    double psum = 0.0;
    for (int tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
        const int C0 = (tile % ntx) * RR_TX, R0 = (tile / ntx) * RR_TY;
        const int fc0 = 2 * C0 - 4, fr0 = 2 * R0 - 2;  // slot of the region's first column and row
        for (int e4 = threadIdx.x; e4 < RR_QW * RR_FH; e4 += blockDim.x) {
            const int fr = e4 / RR_QW, qc = e4 - fr * RR_QW;
            const int row = fr0 + fr, c4 = fc0 + 4 * qc, e = fr * RR_FW + 4 * qc;
            T ru[4] = {0, 0, 0, 0}, rv[4] = {0, 0, 0, 0}, rp[4] = {0, 0, 0, 0};
            uint8_t tu[4] = {T_INACTIVE, T_INACTIVE, T_INACTIVE, T_INACTIVE}, tv[4], tp[4];
#pragma unroll
            for (int q = 0; q < 4; q++) tv[q] = tp[q] = T_INACTIVE;
            // the pitch is a multiple of 32, so a quad is wholly in or out of the frame
            if (row >= 0 && row < Nf + 2 && c4 >= 0 && c4 < P) {
                const int s0 = row * P + c4;  // F < 2^31 (checked when the context is created)
                ldt4(A.tU + s0, tu);
                ldt4(A.tV + s0, tv);
                ldt4(A.tP + s0, tp);
                // as in k_residual4: every load issued before the types are
                // tested, neighbour rows and columns clamped into the frame
                // on its first and last rows, where no internal row is
                const int up = row < Nf + 1 ? P : 0, dn = row > 0 ? P : 0, lf = s0 > 0 ? 1 : 0;
                T uh[6], uU[4], uD[4], vh[6], vU[4], vD[4], ph[5], pD[4], bu[4], bv[4], bp[4];
                ld4(u + s0, uh + 1);
                uh[0] = u[s0 - lf];
                uh[5] = u[s0 + 4];
                ld4(u + s0 + up, uU);
                ld4(u + s0 - dn, uD);
                ld4(v + s0, vh + 1);
                vh[0] = v[s0 - lf];
                vh[5] = v[s0 + 4];
                ld4(v + s0 + up, vU);
                ld4(v + s0 - dn, vD);
                ld4(p + s0, ph + 1);
                ph[0] = p[s0 - lf];
                ld4(p + s0 - dn, pD);
                ld4(b + s0, bu);
                ld4(b + Ff + s0, bv);
                ld4(b + 2 * Ff + s0, bp);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    // internal rows: the expressions of k_residual4; ghost-class
                    // rows (few): k_ghost_residual's values in r
                    if (tu[q] == T_INTERNAL) {
                        T Au = A.d * uh[q + 1] - A.a * (uh[q + 2] + uh[q] + uU[q] + uD[q]) + A.q * (ph[q + 1] - ph[q]);
                        ru[q] = bu[q] - Au;
                    } else if (same_class(T_GHOST, tu[q])) {
                        ru[q] = r[s0 + q];
                    }
                    if (tv[q] == T_INTERNAL) {
                        T Av = A.d * vh[q + 1] - A.a * (vh[q + 2] + vh[q] + vU[q] + vD[q]) + A.q * (ph[q + 1] - pD[q]);
                        rv[q] = bv[q] - Av;
                    } else if (same_class(T_GHOST, tv[q])) {
                        rv[q] = r[Ff + s0 + q];
                    }
                    if (tp[q] == T_INTERNAL) {
                        T Ac = A.q * (uh[q + 2] - uh[q + 1] + vU[q] - vh[q + 1]) - xi;
                        rp[q] = bp[q] - Ac;
                        // the tile's own fine cells: columns [2 C0 - 1, 2 C0 + 63), rows from 2 R0 - 1
                        const int fc = 4 * qc + q;
                        if (fr >= 1 && fc >= 3 && fc < RR_FW - 1) psum += (double)ph[q + 1];
                    } else if (same_class(T_GHOST, tp[q])) {
                        rp[q] = r[2 * Ff + s0 + q];
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                rs[e + q] = ru[q];
                rs[FS + e + q] = rv[q];
                rs[2 * FS + e + q] = rp[q];
                ts[e + q] = tu[q];
                ts[FS + e + q] = tv[q];
                ts[2 * FS + e + q] = tp[q];
            }
        }
        __syncthreads();
        const int col = C0 + (threadIdx.x % RR_TX), row = R0 + threadIdx.x / RR_TX;
        if (col < Pc && row < Nc + 2) {
            const int I = col - 1, J = row - 1;
            const long long sc = (long long)row * Pc + col;
            const uint8_t tcg[3] = {tUc[sc], tVc[sc], tPc[sc]};
#pragma unroll
            for (int g = 0; g < 3; g++) {
                const uint8_t t = tcg[g];
                T out = 0;
                if (t != T_INACTIVE) {
                    bool all = true;
                    int cnt = 0;
                    T sw = 0, su = 0;
#pragma unroll
                    for (int k = 0; k < 6; k++) {
                        if (g == G_P && k >= 4) break;
                        int di, dj;
                        if (g == G_U) { di = k % 3 - 1; dj = k / 3; }
                        else if (g == G_V) { di = k % 2; dj = k / 2 - 1; }
                        else { di = k % 2; dj = k / 2; }
                        const int fi = 2 * I + di, fj = 2 * J + dj;
                        // the fine slot, clamped into the frame, lies in the tile's region
                        const int ci = min(max(fi, -1), Nf), cj = min(max(fj, -1), Nf);
                        const int e = (cj + 1 - fr0) * RR_FW + (ci + 1 - fc0);
                        const T wt = g == G_U ? (T)(k % 3 == 1 ? 0.25 : 0.125)
                                   : g == G_V ? (T)(k / 2 == 1 ? 0.25 : 0.125) : (T)0.25;
                        if (in_grid(g, Nf, fi, fj) && same_class(t, ts[g * FS + e])) {
                            const T rv = rs[g * FS + e];
                            sw += wt * rv;
                            su += rv;
                            cnt++;
                        } else all = false;
                    }
                    out = all ? sw : (cnt > 0 ? su / (T)cnt : (T)0);
                }
                bH[g * Fc + sc] = out;
                if (xz) xz[g * Fc + sc] = (T)0;  // the coarse iterate starts from zero
            }
        }
        __syncthreads();
    }
    if (xz && blockIdx.x == 0)
        for (int q = threadIdx.x; q < NSCAL; q += blockDim.x) xz[3 * Fc + q] = (T)0;
    __shared__ double ss[256];
    ss[threadIdx.x] = psum;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) ss[threadIdx.x] += ss[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = ss[0];
        part[2 * blockIdx.x + 1] = 0.0;
    }
}

// Prolongation code of every fine node (one byte per slot and grid, once per
// geometry): PRO_ON when the node is in its grid and active (it receives
// x + P e), PRO_ALL when besides every coarse node of its interpolation
// stencil is active, so that the weights sum to 1 and no type needs looking
// up during the cycle.

__global__ void k_prolong_codes(int Nf, int Pf, long long Ff, const uint8_t *tUf, const uint8_t *tVf,
                                const uint8_t *tPf, int Nc, int Pc, const uint8_t *tUc, const uint8_t *tVc,
                                const uint8_t *tPc, uint8_t *code)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x, row = blockIdx.y, g = blockIdx.z;
    if (col >= Pf) return;
    const long long s = (long long)row * Pf + col;
    const uint8_t *tf = g == G_U ? tUf : g == G_V ? tVf : tPf;
    const uint8_t *tc = g == G_U ? tUc : g == G_V ? tVc : tPc;
    const int i = col - 1, j = row - 1;
    uint8_t c = 0;
    if (in_grid(g, Nf, i, j) && tf[s] != T_INACTIVE) {
        c = PRO_ON;
        const int Ilo = g == G_V ? -1 : 0, Ihi = g == G_P ? Nc - 1 : Nc;
        const int Jlo = g == G_U ? -1 : 0, Jhi = g == G_P ? Nc - 1 : Nc;
        int KI[2], KJ[2];
        double wi[2], wj[2];
        const int ni = taps<double>(i, g == G_U, Ilo, Ihi, KI, wi);
        const int nj = taps<double>(j, g == G_V, Jlo, Jhi, KJ, wj);
        bool all = true;
        for (int a = 0; a < nj; a++)
            for (int bb = 0; bb < ni; bb++) all = all && tget(tc, g, Nc, Pc, KI[bb], KJ[a]) != T_INACTIVE;
        if (all) c |= PRO_ALL;
    }
    code[g * Ff + s] = c;
}

// Interpolation of the coarse correction (Sect. 4.3): bilinear over the active
// coarse nodes around each fine node, weights renormalised (inactive coarse
// nodes carry no value); y = x + P eH on every slot (y may be x).  Four
// consecutive fine slots per thread: vector loads and stores of x, y and the
// fine prolongation codes, the row taps shared by the four slots.  Nodes
// whose stencil is wholly active (PRO_ALL) skip the coarse type lookups.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong4(int Nf, int Pf, long long Ff, const uint8_t *pcode, int Nc, int Pc,
                                                  long long Fc, const uint8_t *tUc, const uint8_t *tVc,
                                                  const uint8_t *tPc, const T *eH, const T *x, T *y)
{
    const int c0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int row = blockIdx.y;
    if (c0 >= Pf) return;
    const int j = row - 1;
    const long long s0 = (long long)row * Pf + c0;
    if (row == 0 && c0 < NSCAL)
        for (int q = 0; q < 4; q++) y[3 * Ff + c0 + q] = c0 + q == 0 ? x[3 * Ff] + eH[3 * Fc] : x[3 * Ff + c0 + q];
    const uint8_t *tc[3] = {tUc, tVc, tPc};
    // an FP32 coarse iterate carries its pressure shift unapplied: every
    // pressure correction (weights summing to one) gets it once
    const T sigH = sizeof(T) == 4 ? eH[3 * Fc + PSHIFT_SLOT] : (T)0;
#pragma unroll
    for (int g = 0; g < 3; g++) {
        const T sg = g == G_P ? sigH : (T)0;
        uint8_t pc[4];
        T xv[4], out[4];
        ldt4(pcode + g * Ff + s0, pc);
        ld4(x + g * Ff + s0, xv);
        const int Ilo = g == G_V ? -1 : 0, Ihi = g == G_P ? Nc - 1 : Nc;
        const int Jlo = g == G_U ? -1 : 0, Jhi = g == G_P ? Nc - 1 : Nc;
        int KJ[2];
        T wj[2];
        const int nj = taps<T>(j, g == G_V, Jlo, Jhi, KJ, wj);
        const T *e = eH + g * Fc;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int i = c0 + q - 1;
            out[q] = xv[q];
            if (!(pc[q] & PRO_ON)) continue;
            int KI[2];
            T wi[2];
            const int ni = taps<T>(i, g == G_U, Ilo, Ihi, KI, wi);
            T sacc = 0, ws = 0;
            if (pc[q] & PRO_ALL) {
                for (int a = 0; a < nj; a++)
                    for (int bb = 0; bb < ni; bb++)
                        sacc += (wj[a] * wi[bb]) * e[(long long)(KJ[a] + 1) * Pc + (KI[bb] + 1)];
                out[q] = xv[q] + (sacc + sg);
                continue;
            }
            for (int a = 0; a < nj; a++)
                for (int bb = 0; bb < ni; bb++) {
                    if (tget(tc[g], g, Nc, Pc, KI[bb], KJ[a]) == T_INACTIVE) continue;
                    T w = wj[a] * wi[bb];
                    sacc += w * e[(long long)(KJ[a] + 1) * Pc + (KI[bb] + 1)];
                    ws += w;
                }
            if (ws > (T)0) out[q] = xv[q] + ((ws == (T)1 ? sacc : sacc / ws) + sg);
        }
        st4(y + g * Ff + s0, out);
    }
}

template <typename T> __global__ void k_copy_t(const T *a, T *b, long long n)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) b[k] = a[k];
}

// x[0, n) = 0: 16-byte stores where x is 16-byte aligned, then the tail
template <typename T> __global__ void k_zero(T *x, long long n)
{
    using V = typename Vec16<T>::type;
    constexpr int VW = 16 / sizeof(T);
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nv = ((uintptr_t)x % 16 == 0) ? n / VW : 0;
    if (k < nv) ((V *)x)[k] = V{};
    for (long long q = nv * VW + k; q < n; q += (long long)gridDim.x * blockDim.x) x[q] = 0;
}

// x = 0 on inactive nodes of a level
template <typename T> __global__ void k_zero_inactive(LevelArgs<T> A, T *x)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= A.P) return;
    long long s = (long long)row * A.P + col;
    if (A.tU[s] == T_INACTIVE) x[s] = 0;
    if (A.tV[s] == T_INACTIVE) x[A.F + s] = 0;
    if (A.tP[s] == T_INACTIVE) x[2 * A.F + s] = 0;
}

__global__ void k_to_float(const double *a, float *b, long long n)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) b[k] = (float)a[k];
}

// y (+)= e for an FP32 iterate e of the finest level, its pending pressure
// shift applied to the internal and ghost pressures (and not copied itself)
__global__ void k_float_to_double(long long F, const uint8_t *tP, const float *e, double *y, long long n, int add)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    double v = (double)e[k];
    if (k >= 2 * F && k < 3 * F) {
        const uint8_t t = tP[k - 2 * F];
        if (t == T_INTERNAL || t == T_GHOST) v = (double)(e[k] + e[3 * F + PSHIFT_SLOT]);
    } else if (k == 3 * F + PSHIFT_SLOT) {
        v = 0.0;
    }
    y[k] = add ? y[k] + v : v;
}

// the same on four consecutive slots per thread (n a multiple of 4; F is a
// multiple of 32, so a quad lies in one frame or in the scalar block)
__global__ void k_float_to_double4(long long F, const uint8_t *tP, const float *e, double *y, long long n, int add)
{
    const long long q = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
    if (q >= n) return;
    float ev[4];
    double v[4];
    ld4(e + q, ev);
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = (double)ev[k];
    if (q >= 2 * F && q < 3 * F) {
        uint8_t t[4];
        ldt4(tP + (q - 2 * F), t);
        const float sig = e[3 * F + PSHIFT_SLOT];
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (t[k] == T_INTERNAL || t[k] == T_GHOST) v[k] = (double)(ev[k] + sig);
    } else if (q <= 3 * F + PSHIFT_SLOT && 3 * F + PSHIFT_SLOT < q + 4) {
        v[3 * F + PSHIFT_SLOT - q] = 0.0;
    }
    if (add) {
        double yv[4];
        ld4(y + q, yv);
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] += yv[k];
    }
    st4(y + q, v);
}

// ---------------------------------------------- one-block kernels, small levels

// lambda Eq. (ghostrelax) Jacobi sweeps in one block (levels with few rows)
template <typename T>
__device__ __forceinline__ void ghost_sweeps_block(GhostList &gh, int nrows, T *x, const T *b, T dtau, int lambda)
{
    T *upd = gupd<T>(gh);
    for (int it = 0; it < lambda; it++) {
        for (int k = threadIdx.x; k < nrows; k += blockDim.x) upd[k] = dtau * ghost_row_residual<T, false>(gh, k, x, b, nullptr);
        __syncthreads();
        for (int k = threadIdx.x; k < nrows; k += blockDim.x) x[gh.node[k]] += upd[k];
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_ghost_block(GhostList gh, int nrows, T *x, const T *b, T dtau, int lambda)
{
    ghost_sweeps_block<T>(gh, nrows, x, b, dtau, lambda);
}

// nu relaxations (Algorithm relax) of a small level in one block: full boxes
// by 5 colours, cut boxes by their colours, lonely faces, xi and the mean
// pressure, lambda ghost sweeps; the same steps in the same order as the
// multi-kernel path, with block barriers in place of kernel boundaries
template <typename T>
__global__ void __launch_bounds__(512) k_smooth_small(LevelArgs<T> A, T *xg, const T *bg, CutList cut, GhostList gh,
                                                         int nrows, const int *lonely, int nlonely, const int *nint,
                                                         double h2, T dtau, int lambda, int nu, long long vl, int staged)
{
    // with `staged`, x and b (vl slots each) are copied into shared memory,
    // relaxed there, and x is copied back: every access of the many short
    // steps is a shared-memory one instead of an L2 round trip
    extern __shared__ __align__(16) unsigned char small_smem[];
    T *x = xg;
    const T *b = bg;
    if (staged) {
        T *xs = (T *)small_smem, *bs = xs + vl;
        for (long long k = threadIdx.x; k < vl; k += blockDim.x) {
            xs[k] = xg[k];
            bs[k] = bg[k];
        }
        __syncthreads();
        x = xs;
        b = bs;
    }
    __shared__ double ss[1024], sm[1024];
    __shared__ double shift;
    const int N = A.N;
    const int per_row = (N + 4) / 5;
    T *upd = gupd<T>(gh);
    for (int sweep = 0; sweep < nu; sweep++) {
        for (int colour = 0; colour < 5; colour++) {
            for (int idx = threadIdx.x; idx < N * per_row; idx += blockDim.x) {
                int j = idx / per_row, t = idx - j * per_row;
                int i = ((colour - 3 * j) % 5 + 5) % 5 + 5 * t;
                if (i < N) box_full_one<T>(A, x, b, i, j);
            }
            __syncthreads();
        }
        for (int colour = 0; colour < cut.ncol; colour++) {
            int beg = cut.off[colour], end = cut.off[colour + 1];
            for (int k = beg + threadIdx.x; k < end; k += blockDim.x) box_cut_pre<T>(x, b, cut, k);
            __syncthreads();
        }
        if (nlonely > 0) {
            for (int k = threadIdx.x; k < nlonely; k += blockDim.x) {
                long long o = lonely[k];
                bool isu = o < A.F;
                long long loc = isu ? o : o - A.F;
                const T *xx = isu ? x : x + A.F;
                const T *pp = x + 2 * A.F;
                long long pm = isu ? loc - 1 : loc - A.P;
                T Ax = A.d * xx[loc] - A.a * (xx[loc + 1] + xx[loc - 1] + xx[loc + A.P] + xx[loc - A.P]) +
                       A.q * (pp[loc] - pp[pm]);
                upd[k] = (b[o] - Ax) / A.d;
            }
            __syncthreads();
            for (int k = threadIdx.x; k < nlonely; k += blockDim.x) x[lonely[k]] += upd[k];
            __syncthreads();
        }
        // xi and the mean pressure
        double sa = 0.0, ma = 0.0;
        const long long nslot = (long long)(N + 2) * A.P;
        for (long long sl = threadIdx.x; sl < nslot; sl += blockDim.x)
            if (A.tP[sl] == T_INTERNAL) {
                T div = (x[sl + 1] - x[sl] + x[A.F + sl + A.P] - x[A.F + sl]) * A.q;
                sa += (double)(div - b[2 * A.F + sl]);
                ma += (double)x[2 * A.F + sl];
            }
        ss[threadIdx.x] = sa;
        sm[threadIdx.x] = ma;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                ss[threadIdx.x] += ss[threadIdx.x + o];
                sm[threadIdx.x] += sm[threadIdx.x + o];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double n = (double)*nint;
            x[3 * A.F] = (T)(ss[0] / n);
            shift = ((double)b[3 * A.F] - h2 * sm[0]) / (h2 * n);
        }
        __syncthreads();
        T sh = (T)shift;
        for (long long sl = threadIdx.x; sl < nslot; sl += blockDim.x) {
            uint8_t t = A.tP[sl];
            if (t == T_INTERNAL || t == T_GHOST) x[2 * A.F + sl] += sh;
        }
        __syncthreads();
        ghost_sweeps_block<T>(gh, nrows, x, b, dtau, lambda);
    }
    if (staged) {
        __syncthreads();
        for (long long k = threadIdx.x; k < vl; k += blockDim.x) xg[k] = x[k];
    }
}

// ------------------------------------------------------------- event timer

void tmr_flush(Ctx *c)
{
    if (c->tmr_n == 0) return;
    cudaEventSynchronize(c->tmr_ev[2 * c->tmr_n - 1]);
    for (int k = 0; k < c->tmr_n; k++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->tmr_ev[2 * k], c->tmr_ev[2 * k + 1]) == cudaSuccess) c->tmr_ms += ms;
    }
    c->tmr_launches += c->tmr_n;
    c->tmr_n = 0;
}

void tmr_begin(Ctx *c, int kernel, int lev)
{
    if (c->tmr_kernel != kernel || c->tmr_level != lev) return;
    if (c->tmr_n == 512) tmr_flush(c);
    cudaEventRecord(c->tmr_ev[2 * c->tmr_n], c->stream);
}

void tmr_end(Ctx *c, int kernel, int lev)
{
    if (c->tmr_kernel != kernel || c->tmr_level != lev) return;
    cudaEventRecord(c->tmr_ev[2 * c->tmr_n + 1], c->stream);
    c->tmr_n++;
}

// ----------------------------------------------------------- host wrappers

template <typename T> LevelArgs<T> level_args(const Ctx *c, int lev)
{
    const Level &l = c->lv[lev];
    LevelArgs<T> A;
    A.N = l.N;
    A.P = l.P;
    A.F = l.F;
    double h = c->prm.L / (double)l.N;
    A.q = (T)(1.0 / h);
    A.a = (T)(c->prm.alpha / (h * h));
    A.d = (T)(1.0 + 4.0 * (c->prm.alpha / (h * h)));
    A.h2 = (T)(h * h);
    A.tU = l.tU;
    A.tV = l.tV;
    A.tP = l.tP;
    A.bc = l.bcode;
    const double q = 1.0 / h, a = c->prm.alpha / (h * h), d = 1.0 + 4.0 * a;
    A.K.a = (T)a;
    A.K.d = (T)d;
    A.K.q = (T)q;
    A.K.qida = (T)(q / (d + a));
    A.K.qid = (T)(q / d);
    A.K.id = (T)(1.0 / d);
    A.K.idet = (T)(1.0 / (d * d - a * a));
    const double cx[3] = {0.0, q * q / d, 2.0 * q * q / (d + a)};
    for (int nx = 0; nx < 3; nx++)
        for (int ny = 0; ny < 3; ny++) A.K.ic1[nx * 3 + ny] = nx + ny == 0 ? (T)0 : (T)(1.0 / (cx[nx] + cx[ny]));
    return A;
}

static inline dim3 frame_grid(const Level &l) { return dim3((l.P + 255) / 256, l.N + 2); }

// the other vector of the tiled sweep: the level's residual vector, which is
// dead during relaxation (it is recomputed before restriction)
template <typename T> T *tile_scratch(Ctx *c, int lev);
template <> double *tile_scratch<double>(Ctx *c, int lev) { return c->lv[lev].r; }
template <> float *tile_scratch<float>(Ctx *c, int lev) { return c->lv[lev].rf; }

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime
static EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// tensor map over `nf` frames of a level (x: column, y: frame row, z:
// frame when nf = 3), box = the tile window of k_box_tma
static bool encode_frames(CUtensorMap *m, const void *base, CUtensorMapDataType dt, int esize, const Level &l,
                          long long frame_stride_bytes, int nf, int LW, int LH, int box_nf = 0)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)l.P, (cuuint64_t)(l.N + 2), (cuuint64_t)nf};
    cuuint64_t strides[2] = {(cuuint64_t)l.P * esize, (cuuint64_t)frame_stride_bytes};
    cuuint32_t box[3] = {(cuuint32_t)LW, (cuuint32_t)LH, (cuuint32_t)(box_nf > 0 ? box_nf : nf)};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, dt, nf > 1 ? 3 : 2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// does this level sweep its full boxes with k_box_tma (T's other vector must exist)
template <typename T> static bool tiled(Ctx *c, int lev)
{
    const Level &l = c->lv[lev];
    // default: FP32 levels from TILE_MIN_N; FP64 boxes are bound by the FP64
    // units, where the halo boxes a tile recomputes cost more than the four
    // extra passes over memory they save
    int tmin = c->prm.tile_min != 0 ? c->prm.tile_min : sizeof(T) == 4 ? TILE_MIN_N : -1;
    return tmin >= 0 && l.N >= tmin && tile_scratch<T>(c, lev) && encode_fn();
}

// does this tiled level stream its full boxes down strips of rows (k_box_wave)
template <typename T> static bool wave(Ctx *c, int lev)
{
    int wmin = c->prm.wave_min != 0 ? c->prm.wave_min : WAVE_MIN_N;
    const Level &l = c->lv[lev];
    // the sweep addresses the right-hand side with 32-bit slot offsets
    return wmin >= 0 && l.N >= wmin && 3 * l.F + l.P < (1ll << 31) && tiled<T>(c, lev);
}

void prepare_cuts(Ctx *c)
{
    for (int lev = 0; lev < c->L; lev++) {
        const Level &l = c->lv[lev];
        if (l.h_ncut <= 0) continue;
        k_cut_prepare<<<(l.h_ncut + 127) / 128, 128, 0, c->stream>>>(level_args<double>(c, lev), l.cut, l.gh, l.h_ncut);
    }
}

// one cluster of CL_CTAS CTAs of `threads` threads on the stream
template <typename... KArgs, typename... Args>
static cudaError_t launch_cluster(cudaStream_t st, int threads, void (*kernel)(KArgs...), Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL_CTAS, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL_CTAS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Colours of the cut boxes: two boxes conflict when a row of one references
// an unknown of the other (the unknowns of a box are its internal and ghost
// faces and p; its rows are the prepared rows of k_cut_prepare).  Boxes in
// slot order, i.e. lexicographic (j, i), take the smallest colour that no
// conflicting box before them has; the list is then sorted by colour (slot
// order inside a colour).  Needs prepared rows; the caller prepares again for
// the new order.  Host work once per geometry (the rows are copied back).
int recolour_cuts(Ctx *c)
{
    cudaStream_t st = c->stream;
    for (int lev = 0; lev < c->L; lev++) {
        Level &l = c->lv[lev];
        const int n = l.h_ncut, cap = l.cut.cap;
        if (n <= 0) {
            l.cut.ncol = 0;
            l.h_cutoff[0] = 0;
            continue;
        }
        std::vector<int> cell(n), row((size_t)5 * n), sidx((size_t)5 * CUT_ST * n), gface((size_t)4 * n);
        cudaMemcpyAsync(cell.data(), l.cut.cell, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
        for (int f = 0; f < 5; f++)
            cudaMemcpyAsync(row.data() + (size_t)f * n, l.cut.row + (size_t)f * cap, sizeof(int) * n,
                            cudaMemcpyDeviceToHost, st);
        for (int e = 0; e < 5 * CUT_ST; e++)
            cudaMemcpyAsync(sidx.data() + (size_t)e * n, l.cut.sidx + (size_t)e * cap, sizeof(int) * n,
                            cudaMemcpyDeviceToHost, st);
        for (int f = 0; f < 4; f++)
            cudaMemcpyAsync(gface.data() + (size_t)f * n, l.cut.gface + (size_t)f * cap, sizeof(int) * n,
                            cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            snprintf(c->msg, sizeof c->msg, "cut colouring: %s", cudaGetErrorString(cudaGetLastError()));
            return GP_CUDA;
        }
        // boxes in slot order; owners of every unknown (at most two boxes)
        std::vector<int> ord(n);
        for (int k = 0; k < n; k++) ord[k] = k;
        std::sort(ord.begin(), ord.end(), [&](int a, int b) { return cell[a] < cell[b]; });
        std::vector<int> rank(n);
        for (int r = 0; r < n; r++) rank[ord[r]] = r;
        std::unordered_map<int, std::pair<int, int>> own;
        own.reserve((size_t)5 * n);
        for (int k = 0; k < n; k++)
            for (int f = 0; f < 5; f++) {
                int u = row[(size_t)f * n + k];
                if (u < 0) continue;
                auto it = own.find(u);
                if (it == own.end()) own.emplace(u, std::make_pair(rank[k], -1));
                else it->second.second = rank[k];
            }
        std::vector<std::vector<int>> nb(n);
        for (int k = 0; k < n; k++) {
            const int a = rank[k];
            for (int e = 0; e < 5 * CUT_ST; e++) {
                auto it = own.find(sidx[(size_t)e * n + k]);
                if (it == own.end()) continue;
                const int bs[2] = {it->second.first, it->second.second};
                for (int z = 0; z < 2; z++)
                    if (bs[z] >= 0 && bs[z] != a) {
                        nb[a].push_back(bs[z]);
                        nb[bs[z]].push_back(a);
                    }
            }
        }
        std::vector<int> col(n, -1);
        int ncol = 0;
        for (int a = 0; a < n; a++) {
            unsigned long long used = 0ull;
            for (int b : nb[a])
                if (b < a) used |= 1ull << col[b];
            int cc = 0;
            while (cc < MAX_CUTCOL && ((used >> cc) & 1ull)) cc++;
            if (cc >= MAX_CUTCOL) {
                snprintf(c->msg, sizeof c->msg, "level %d: cut boxes need more than %d colours", lev, MAX_CUTCOL);
                return GP_GEOMETRY;
            }
            col[a] = cc;
            ncol = std::max(ncol, cc + 1);
        }
        // the list sorted by (colour, slot)
        std::vector<int> perm(n);
        for (int r = 0; r < n; r++) perm[r] = r;
        std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return col[a] < col[b]; });
        std::vector<int> cell2(n), gface2((size_t)4 * n);
        for (int q = 0; q < n; q++) {
            const int k = ord[perm[q]];
            cell2[q] = cell[k];
            for (int f = 0; f < 4; f++) gface2[(size_t)f * n + q] = gface[(size_t)f * n + k];
        }
        for (int cc = 0; cc <= ncol; cc++) l.h_cutoff[cc] = 0;
        for (int r = 0; r < n; r++) l.h_cutoff[col[r] + 1]++;
        for (int cc = 0; cc < ncol; cc++) l.h_cutoff[cc + 1] += l.h_cutoff[cc];
        l.cut.ncol = ncol;
        cudaMemcpyAsync(l.cut.cell, cell2.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
        for (int f = 0; f < 4; f++)
            cudaMemcpyAsync(l.cut.gface + (size_t)f * cap, gface2.data() + (size_t)f * n, sizeof(int) * n,
                            cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(l.cut.off, l.h_cutoff, sizeof(int) * (ncol + 1), cudaMemcpyHostToDevice, st);
        // the host vectors must outlive the copies
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            snprintf(c->msg, sizeof c->msg, "cut colouring: %s", cudaGetErrorString(cudaGetLastError()));
            return GP_CUDA;
        }
    }
    return GP_OK;
}

// box codes of every level and prolongation codes of every level but the
// coarsest (k_box_codes, k_prolong_codes); once per geometry
void box_codes(Ctx *c)
{
    for (int lev = 0; lev < c->L; lev++) {
        const Level &l = c->lv[lev];
        k_box_codes<<<(unsigned)((l.F + 255) / 256), 256, 0, c->stream>>>(l.N, l.P, l.F, l.tU, l.tV, l.tP, l.bcode);
        if (lev + 1 < c->L) {
            const Level &C = c->lv[lev + 1];
            k_prolong_codes<<<dim3((l.P + 127) / 128, l.N + 2, 3), 128, 0, c->stream>>>(
                l.N, l.P, l.F, l.tU, l.tV, l.tP, C.N, C.P, C.tU, C.tV, C.tP, l.pcode);
        }
    }
}

// For every stencil entry of every ghost-class row, the index of the row
// whose unknown it is (or -1): the fused ghost sweeps read the accumulated
// correction of that row.  Once per geometry, on the device: the rows are
// scattered into a node -> row map over the level's vector (held in the
// level's residual vector, free at this point), then read back per entry.
__global__ void k_row_of_node(const int *node, int n, int *map)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) map[node[k]] = k;
}

__global__ void k_stencil_rows(GhostList gh, int n, const int *map)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int nst = gh.nst[k];
    for (int q = 0; q < GH_ST; q++) {
        const long long e = (long long)q * gh.cap + k;
        gh.strow[e] = q < nst ? map[gh.st[e]] : -1;
    }
}

// The closure of each block of GC_OWN ghost-class rows for k_ghost_fused:
// the rows within lambda - 1 stencil links (breadth first over a bitmap of
// the level's rows in shared memory), listed in ascending order, and for
// each stencil entry of each listed row the list position of the entry's row
// (or -1 when that row is outside the closure or no row).  cl_n = -1 when the
// closure has more than GC_CAP rows.  Once per geometry.
__global__ void __launch_bounds__(GC_THREADS) k_ghost_closure(GhostList gh, int n, int lambda)
{
    extern __shared__ unsigned cl_smem[];
    const int words = (n + 31) >> 5;
    unsigned *cur = cl_smem, *nxt = cl_smem + words;
    int *rows = (int *)(nxt + words);  // GC_CAP
    int *scan = rows + GC_CAP;         // GC_THREADS + 1
    const int lo = blockIdx.x * GC_OWN, hi = min(lo + GC_OWN, n);
    for (int wd = threadIdx.x; wd < words; wd += blockDim.x) {
        unsigned m = 0;
        for (int bit = 0; bit < 32; bit++) {
            const int r = (wd << 5) + bit;
            if (r >= lo && r < hi) m |= 1u << bit;
        }
        cur[wd] = m;
        nxt[wd] = m;
    }
    __syncthreads();
    for (int hop = 1; hop < lambda; hop++) {
        for (int wd = threadIdx.x; wd < words; wd += blockDim.x) {
            unsigned m = cur[wd];
            while (m) {
                const int r = (wd << 5) + __ffs(m) - 1;
                m &= m - 1;
                const int ns = gh.nst[r];
                for (int q = 0; q < ns && q < GH_ST; q++) {
                    const int l = gh.strow[(long long)q * gh.cap + r];
                    if (l >= 0 && l < n) atomicOr(&nxt[l >> 5], 1u << (l & 31));
                }
            }
        }
        __syncthreads();
        for (int wd = threadIdx.x; wd < words; wd += blockDim.x) cur[wd] = nxt[wd];
        __syncthreads();
    }
    // ascending list: each thread lists a contiguous run of words at the
    // offset of an exclusive scan of the runs' counts
    const int per = (words + blockDim.x - 1) / blockDim.x;
    const int w0 = min((int)threadIdx.x * per, words), w1 = min(w0 + per, words);
    int cnt = 0;
    for (int wd = w0; wd < w1; wd++) cnt += __popc(cur[wd]);
    scan[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < (int)blockDim.x; t++) {
            const int v = scan[t];
            scan[t] = acc;
            acc += v;
        }
        scan[blockDim.x] = acc;
    }
    __syncthreads();
    const int total = scan[blockDim.x];
    if (total > GC_CAP) {
        if (threadIdx.x == 0) gh.cl_n[blockIdx.x] = -1;
        return;
    }
    int pos = scan[threadIdx.x];
    for (int wd = w0; wd < w1; wd++) {
        unsigned m = cur[wd];
        while (m) {
            rows[pos++] = (wd << 5) + __ffs(m) - 1;
            m &= m - 1;
        }
    }
    __syncthreads();
    int *grow = gh.cl_row + (long long)blockIdx.x * GC_CAP;
    int16_t *glnk = gh.cl_lnk + (long long)blockIdx.x * GH_ST * GC_CAP;
    for (int ci = threadIdx.x; ci < total; ci += blockDim.x) {
        const int r = rows[ci];
        grow[ci] = r;
        const int ns = gh.nst[r];
        for (int q = 0; q < GH_ST; q++) {
            int loc = -1;
            const int l = q < ns ? gh.strow[(long long)q * gh.cap + r] : -1;
            if (l >= 0 && l < n && ((cur[l >> 5] >> (l & 31)) & 1u)) {
                int a = 0, z = total - 1;
                while (a < z) {
                    const int mid = (a + z) >> 1;
                    if (rows[mid] < l) a = mid + 1;
                    else z = mid;
                }
                loc = a;
            }
            glnk[q * GC_CAP + ci] = (int16_t)loc;
        }
    }
    if (threadIdx.x == 0) gh.cl_n[blockIdx.x] = total;
}

static size_t closure_smem(int n) { return 2 * sizeof(unsigned) * (size_t)((n + 31) / 32) + sizeof(int) * (GC_CAP + GC_THREADS + 1); }
constexpr size_t CLOSURE_SMEM_MAX = 200 * 1024;

int ghost_row_links(Ctx *c)
{
    cudaStream_t st = c->stream;
    for (int lev = 0; lev < c->L; lev++) {
        Level &l = c->lv[lev];
        const int n = l.h_nrows;
        if (n <= 0) continue;
        int *map = (int *)l.r;  // VL ints fit in the VL doubles of r
        cudaMemsetAsync(map, 0xff, sizeof(int) * (size_t)l.VL, st);
        k_row_of_node<<<(n + 255) / 256, 256, 0, st>>>(l.gh.node, n, map);
        k_stencil_rows<<<(n + 255) / 256, 256, 0, st>>>(l.gh, n, map);
    }
    // closures for the fused sweeps of the levels above the one-block size
    // (lambda > 1; one sweep needs no closure)
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_ghost_closure, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CLOSURE_SMEM_MAX);
        attr = true;
    }
    std::vector<std::vector<int>> hn(c->L);
    for (int lev = 0; lev < c->L; lev++) {
        Level &l = c->lv[lev];
        l.h_fused = 0;
        const int n = l.h_nrows;
        if (n <= GHOST_BLOCK_ROWS || c->prm.lambda <= 1 || closure_smem(n) > CLOSURE_SMEM_MAX) continue;
        const int nblk = (n + GC_OWN - 1) / GC_OWN;
        k_ghost_closure<<<nblk, GC_THREADS, closure_smem(n), st>>>(l.gh, n, c->prm.lambda);
        hn[lev].resize(nblk);
        cudaMemcpyAsync(hn[lev].data(), l.gh.cl_n, sizeof(int) * nblk, cudaMemcpyDeviceToHost, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        snprintf(c->msg, sizeof c->msg, "ghost links: %s", cudaGetErrorString(e));
        return GP_CUDA;
    }
    for (int lev = 0; lev < c->L; lev++) {
        if (hn[lev].empty()) continue;
        bool ok = true;
        for (int v : hn[lev]) ok = ok && v >= 0;
        c->lv[lev].h_fused = ok ? 1 : 0;
    }
    return GP_OK;
}

void tiles_init()
{
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(k_box_tma<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tt_smem<double>());
    cudaFuncSetAttribute(k_box_tma<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tt_smem<float>());
    cudaFuncSetAttribute(k_box_wave<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wv_smem<double>());
    cudaFuncSetAttribute(k_box_wave<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wv_smem<float>());
    cudaFuncSetAttribute(k_smooth_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMALL_STAGE_BYTES);
    cudaFuncSetAttribute(k_smooth_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMALL_STAGE_BYTES);
    done = true;
}

template <typename T> static void copy_vec(Ctx *c, const T *a, T *b, long long n)
{
    k_copy_t<T><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(a, b, n);
    c->launches++;
}

// blocks of 256 threads of `kernel` that are resident on the device at once
template <typename K> static int resident_blocks(K kernel)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return sms * per_sm;
}

// blocks of a grid-stride reduction kernel: one block per 256 threads' worth
// of slots, at most one wave of resident blocks (every block then loops the
// same number of times and no partial second wave trails)
template <typename K> static int red_blocks(const Level &l, K kernel, int &cache)
{
    if (cache <= 0) cache = resident_blocks(kernel);
    const long long n = (l.F + 255) / 256;
    return (int)(n < cache ? n : cache);
}

template <typename T, typename R> void residual_into(Ctx *c, int lev, const T *x, const T *b, R *r)
{
    const Level &l = c->lv[lev];
    cudaStream_t st = c->stream;
    static int resident = 0;
    int nb = red_blocks(l, k_residual4<T, R>, resident);
    tmr_begin(c, KT_RESIDUAL, lev);
    k_residual4<T, R><<<nb, 256, 0, st>>>(level_args<T>(c, lev), x, b, r, c->part);
    tmr_end(c, KT_RESIDUAL, lev);
    if (l.h_nrows > 0)
        k_ghost_residual<T, R><<<(l.h_nrows + 255) / 256, 256, 0, st>>>(l.gh, l.h_nrows, x, b, r, c->maxbits);
    double h = c->prm.L / (double)l.N;
    k_residual_final<T, R><<<1, 256, 0, st>>>(c->part, nb, b, r, 3 * l.F, h * h, c->maxbits, c->red, x, l.nint);
    c->launches += 2 + (l.h_nrows > 0);
}

template <typename T> void residual(Ctx *c, int lev, const T *x, const T *b, T *r) { residual_into<T, T>(c, lev, x, b, r); }

// the FP64 residual of the finest level written as the FP32 right-hand side
// of the next inner cycle (the scalars past the mean row are left as they are)
void residual_to_float(Ctx *c, const double *x, const double *b, float *r) { residual_into<double, float>(c, 0, x, b, r); }

// full boxes from `in` into `out`: with out != in the level is tiled and out
// becomes a complete copy of the swept vector; with out == in the five colour
// passes run in place.  Then the cut boxes and lonely faces, in place on out.
template <typename T> static void box_pass(Ctx *c, int lev, const T *in, T *out, const T *b)
{
    const Level &l = c->lv[lev];
    cudaStream_t st = c->stream;
    LevelArgs<T> A = level_args<T>(c, lev);
    bool done = false;
    if (out != in && wave<T>(c, lev)) {
        constexpr int TW = WaveGeom<T>::TW, LW = WaveGeom<T>::LW;
        const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
        const long long fs = l.F * (long long)sizeof(T);
        CUtensorMap mx, mc, mb;
        if (encode_frames(&mx, in, dt, (int)sizeof(T), l, fs, 3, LW, WV_R, 1) &&
            encode_frames(&mc, l.bcode, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, l, l.F, 1, LW, WV_R) &&
            encode_frames(&mb, b, dt, (int)sizeof(T), l, fs, 3, LW, WV_R, 3)) {
            // strips of TW columns, each cut into segments of SH rows so that
            // the grid is about one wave of resident blocks
            static int resident = 0;
            if (resident <= 0) {
                int dev = 0, sms = 0, per_sm = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_box_wave<T>, WV_THREADS, wv_smem<T>()) !=
                        cudaSuccess ||
                    per_sm < 1) {
                    cudaGetLastError();
                    per_sm = 1;
                }
                resident = sms * per_sm;
            }
            const int gx = (l.P + TW - 1) / TW, rows = l.N + 2;
            int nseg = resident / gx;
            nseg = nseg < 1 ? 1 : nseg > (rows + WV_R - 1) / WV_R ? (rows + WV_R - 1) / WV_R : nseg;
            int SH = (rows + nseg - 1) / nseg;
            SH = (SH + WV_R - 1) / WV_R * WV_R;
            nseg = (rows + SH - 1) / SH;
            tmr_begin(c, KT_BOX_FULL, lev);
            k_box_wave<T><<<dim3(gx, nseg), WV_THREADS, wv_smem<T>(), st>>>(mx, mc, mb, A, in, b, out, SH, c->err);
            tmr_end(c, KT_BOX_FULL, lev);
            c->launches++;
            done = true;
        }
    }
    if (out != in && !done) {
        constexpr int TW = TileGeom<T>::TW, LW = TileGeom<T>::LW, TH = TileGeom<T>::TH;
        const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
        CUtensorMap mx, mc;
        if (encode_frames(&mx, in, dt, (int)sizeof(T), l, l.F * (long long)sizeof(T), 3, LW, tt_lh<T>()) &&
            encode_frames(&mc, l.bcode, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, l, l.F, 1, LW, tt_lh<T>())) {
            dim3 gt((l.P + TW - 1) / TW, (l.N + 2 + TH - 1) / TH);
            tmr_begin(c, KT_BOX_FULL, lev);
            k_box_tma<T><<<gt, TileGeom<T>::THREADS, tt_smem<T>(), st>>>(mx, mc, A, in, b, out, c->err);
            tmr_end(c, KT_BOX_FULL, lev);
            c->launches++;
            done = true;
        } else {
            copy_vec<T>(c, in, out, l.VL);
        }
    }
    if (!done) {
        int per_row = (l.N + 4) / 5;
        dim3 g((per_row + 127) / 128, l.N);
        for (int colour = 0; colour < 5; colour++) {
            tmr_begin(c, KT_BOX_FULL, lev);
            k_box_full<T><<<g, 128, 0, st>>>(A, out, b, colour);
            tmr_end(c, KT_BOX_FULL, lev);
            c->launches++;
        }
    }
    T *x = out;
    int most = 0;  // largest colour of cut boxes
    for (int colour = 0; colour < l.cut.ncol; colour++) most = max(most, l.h_cutoff[colour + 1] - l.h_cutoff[colour]);
    if (most > CUT_SPLIT && l.cut.ncol <= CUT_COLOUR_LAUNCHES) {
        // few colours with many boxes each: one launch per colour across the GPU
        tmr_begin(c, KT_BOX_CUT, lev);
        for (int colour = 0; colour < l.cut.ncol; colour++) {
            const int beg = l.h_cutoff[colour], end = l.h_cutoff[colour + 1];
            if (end <= beg) continue;
            k_box_cut_colour<T><<<(end - beg + 7) / 8, 256, 0, st>>>(x, b, l.cut, beg, end);
            c->launches++;
        }
        tmr_end(c, KT_BOX_CUT, lev);
    } else if (most > CUT_SPLIT) {
        tmr_begin(c, KT_BOX_CUT, lev);
        launch_cluster(st, CL_THREADS, k_box_cut_cluster<T>, x, b, l.cut);
        tmr_end(c, KT_BOX_CUT, lev);
        c->launches++;
    } else if (l.h_ncut > 0) {
        tmr_begin(c, KT_BOX_CUT, lev);
        k_box_cut<T><<<1, 1024, 0, st>>>(A, x, b, l.cut, l.gh);
        tmr_end(c, KT_BOX_CUT, lev);
        c->launches++;
    }
    if (l.h_nlonely > 0) {
        T *upd = (T *)c->part;
        k_lonely_update<T><<<(l.h_nlonely + 127) / 128, 128, 0, st>>>(A, x, b, l.lonely, l.h_nlonely, upd);
        k_apply_list<T><<<(l.h_nlonely + 127) / 128, 128, 0, st>>>(x, l.lonely, upd, l.h_nlonely);
        c->launches += 2;
    }
}

// one box sweep in place on x (a tiled level sweeps into its other vector and
// copies back)
template <typename T> void box_sweep(Ctx *c, int lev, T *x, const T *b)
{
    if (tiled<T>(c, lev)) {
        T *t = tile_scratch<T>(c, lev);
        box_pass<T>(c, lev, x, t, b);
        copy_vec<T>(c, t, x, c->lv[lev].VL);
    } else {
        box_pass<T>(c, lev, x, x, b);
    }
}

template <typename T> void scalar_update(Ctx *c, int lev, T *x, const T *b)
{
    const Level &l = c->lv[lev];
    cudaStream_t st = c->stream;
    LevelArgs<T> A = level_args<T>(c, lev);
    static int resident = 0;
    int nb = red_blocks(l, k_scalar_partial<T>, resident);
    tmr_begin(c, KT_SCALAR, lev);
    k_scalar_partial<T><<<nb, 256, 0, st>>>(A, x, b, c->part);
    tmr_end(c, KT_SCALAR, lev);
    double h = c->prm.L / (double)l.N;
    // FP32 iterates (the inner cycles of the mixed mode) keep the pressure
    // shift pending: every row but the mean row is blind to a constant added
    // to the internal and ghost pressures, so the shift is applied only where
    // the iterate leaves its level (the mean-row residual, the prolongation,
    // the FP64 update); FP64 iterates get it at once
    const bool defer = sizeof(T) == 4;
    k_scalar_final<T><<<1, 256, 0, st>>>(c->part, nb, x, b, 3 * l.F, h * h, l.nint, c->red + 1, defer);
    if (!defer) k_pshift<T><<<dim3((l.P / 4 + 255) / 256, l.N + 2), 256, 0, st>>>(A, x, c->red + 1);
    c->launches += defer ? 2 : 3;
}

template <typename T> void ghost_sweep(Ctx *c, int lev, T *x, const T *b)
{
    const Level &l = c->lv[lev];
    if (l.h_nrows <= 0) return;
    cudaStream_t st = c->stream;
    int nb = (l.h_nrows + 255) / 256;
    tmr_begin(c, KT_GHOST, lev);
    k_ghost_update<T><<<nb, 256, 0, st>>>(l.gh, l.h_nrows, x, b, (T)c->prm.dtau);
    tmr_end(c, KT_GHOST, lev);
    k_ghost_apply<T><<<nb, 256, 0, st>>>(l.gh, l.h_nrows, x);
    c->launches += 2;
}

// nu relaxations (Algorithm relax) of the iterate held in `in` (x or the
// level's other vector); the result ends in x.  Tiled levels alternate
// between the two vectors, so an even count from x, or an odd count from the
// other vector, needs no copy.
// levels whose whole relaxation runs in one block, in place (a cluster of
// CTAs was measured slower here than one block or than one launch per phase
// over the whole GPU: its barriers cost more and its few SMs limit the memory
// parallelism); tiled levels keep their ping-pong sweeps
template <typename T> static bool one_kernel_level(Ctx *c, int lev)
{
    const Level &l = c->lv[lev];
    return l.N <= SMALL_N && l.h_nlonely <= l.gh.cap && !tiled<T>(c, lev);
}

template <typename T> void smooth_from(Ctx *c, int lev, T *x, T *in, const T *b, int nu)
{
    const Level &l = c->lv[lev];
    const bool tl = tiled<T>(c, lev);
    const bool one = one_kernel_level<T>(c, lev);
    if (in != x && (nu <= 0 || !tl || one)) {
        copy_vec<T>(c, in, x, l.VL);
        in = x;
    }
    if (nu <= 0) return;
    if (one) {
        double h = c->prm.L / (double)l.N;
        tmr_begin(c, KT_BOX_FULL, lev);
        const size_t stage = 2 * sizeof(T) * (size_t)l.VL;
        const int staged = stage <= SMALL_STAGE_BYTES;
        k_smooth_small<T><<<1, 512, staged ? stage : 0, c->stream>>>(
            level_args<T>(c, lev), x, b, l.cut, l.gh, l.h_nrows, l.lonely, l.h_nlonely, l.nint, h * h,
            (T)c->prm.dtau, c->prm.lambda, nu, l.VL, staged);
        tmr_end(c, KT_BOX_FULL, lev);
        c->launches++;
        return;
    }
    T *t = tl ? tile_scratch<T>(c, lev) : x;
    T *cur = in;
    for (int s = 0; s < nu; s++) {
        T *out = tl ? (cur == x ? t : x) : cur;
        box_pass<T>(c, lev, cur, out, b);
        cur = out;
        scalar_update<T>(c, lev, cur, b);
        if (l.h_nrows > 0 && l.h_nrows <= GHOST_BLOCK_ROWS && c->prm.lambda > 0) {
            tmr_begin(c, KT_GHOST, lev);
            k_ghost_block<T><<<1, 1024, 0, c->stream>>>(l.gh, l.h_nrows, cur, b, (T)c->prm.dtau, c->prm.lambda);
            tmr_end(c, KT_GHOST, lev);
            c->launches++;
        } else if (l.h_nrows > 0 && c->prm.lambda > 0) {
            const int nb = (l.h_nrows + 255) / 256;
            tmr_begin(c, KT_GHOST, lev);
            if (l.h_fused) {
                k_ghost_fused<T><<<(l.h_nrows + GC_OWN - 1) / GC_OWN, GC_THREADS, 0, c->stream>>>(
                    l.gh, l.h_nrows, cur, b, (T)c->prm.dtau, c->prm.lambda);
                c->launches += 1;
            } else {
                for (int k = 0; k < c->prm.lambda; k++)
                    k_ghost_acc_sweep<T><<<nb, 256, 0, c->stream>>>(l.gh, l.h_nrows, cur, b, (T)c->prm.dtau, k);
                c->launches += c->prm.lambda;
            }
            k_ghost_acc_apply<T><<<nb, 256, 0, c->stream>>>(l.gh, l.h_nrows, cur, c->prm.lambda);
            tmr_end(c, KT_GHOST, lev);
            c->launches += 1;
        }
    }
    if (cur != x) copy_vec<T>(c, cur, x, l.VL);
}

template <typename T> void smooth(Ctx *c, int lev, T *x, const T *b, int nu) { smooth_from<T>(c, lev, x, x, b, nu); }

// where the cycle should put x + P e before `nu` post-relaxations so that the
// tiled sweeps end in x without a copy
template <typename T> T *post_buffer(Ctx *c, int lev, T *x, int nu)
{
    if (nu % 2 == 0 || !tiled<T>(c, lev) || one_kernel_level<T>(c, lev)) return x;
    return tile_scratch<T>(c, lev);
}

// restriction into bH; with xz non-null the same launch also zeroes the
// coarse iterate xz (every slot of its frames and scalars)
template <typename T> void restrict_level(Ctx *c, int lev, const T *r, T *bH, T *xz)
{
    const Level &f = c->lv[lev], &C = c->lv[lev + 1];
    dim3 g((C.P + 255) / 256, C.N + 2);
    tmr_begin(c, KT_RESTRICT, lev);
    k_restrict<T><<<g, 256, 0, c->stream>>>(f.N, f.P, f.F, f.tU, f.tV, f.tP, C.N, C.P, C.F, C.tU, C.tV, C.tP, r, bH,
                                             xz);
    tmr_end(c, KT_RESTRICT, lev);
    c->launches++;
}

// the residual of `lev` restricted into bH, the coarse iterate xz zeroed, in
// one pass over the fine frames (k_residual_restrict); r receives only the
// ghost-class rows, the mean row goes straight into bH
template <typename T> void residual_restrict(Ctx *c, int lev, const T *x, const T *b, T *r, T *bH, T *xz)
{
    const Level &f = c->lv[lev], &C = c->lv[lev + 1];
    cudaStream_t st = c->stream;
    static int resident = 0;
    if (resident <= 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_residual_restrict<T>, 256, rr_smem<T>()) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        resident = sms * per_sm;
    }
    const long long ntiles = (long long)((C.P + RR_TX - 1) / RR_TX) * ((C.N + 2 + RR_TY - 1) / RR_TY);
    const int nb = (int)(ntiles < resident ? ntiles : resident);
    if (f.h_nrows > 0)
        k_ghost_residual<T, T><<<(f.h_nrows + 255) / 256, 256, 0, st>>>(f.gh, f.h_nrows, x, b, r, c->maxbits);
    tmr_begin(c, KT_RESTRICT, lev);
    k_residual_restrict<T><<<nb, 256, rr_smem<T>(), st>>>(level_args<T>(c, lev), C.N, C.P, C.F, C.tU, C.tV, C.tP, x,
                                                          b, r, bH, xz, c->part);
    tmr_end(c, KT_RESTRICT, lev);
    const double h = c->prm.L / (double)f.N;
    k_residual_final<T, T><<<1, 256, 0, st>>>(c->part, nb, b, r, 3 * f.F, h * h, c->maxbits, c->red, x, f.nint,
                                              bH + 3 * C.F);
    c->launches += 2 + (f.h_nrows > 0);
}

template <typename T> void prolong_to(Ctx *c, int lev, const T *eH, const T *x, T *y)
{
    const Level &f = c->lv[lev], &C = c->lv[lev + 1];
    dim3 g((f.P / 4 + 255) / 256, f.N + 2);
    tmr_begin(c, KT_PROLONG, lev);
    k_prolong4<T><<<g, 256, 0, c->stream>>>(f.N, f.P, f.F, f.pcode, C.N, C.P, C.F, C.tU, C.tV, C.tP, eH, x, y);
    tmr_end(c, KT_PROLONG, lev);
    c->launches++;
}

template <typename T> void prolong_level(Ctx *c, int lev, const T *eH, T *x) { prolong_to<T>(c, lev, eH, x, x); }

template <typename T> void zero_vec(Ctx *c, T *x, long long n)
{
    const long long nv = (n + 16 / (long long)sizeof(T) - 1) / (16 / (long long)sizeof(T));
    k_zero<T><<<(unsigned)((nv + 255) / 256), 256, 0, c->stream>>>(x, n);
    c->launches++;
}

template <typename T> void zero_inactive(Ctx *c, int lev, T *x)
{
    k_zero_inactive<T><<<frame_grid(c->lv[lev]), 256, 0, c->stream>>>(level_args<T>(c, lev), x);
    c->launches++;
}

void to_float(Ctx *c, const double *a, float *b, long long n)
{
    k_to_float<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(a, b, n);
    c->launches++;
}

static void f2d(Ctx *c, const float *e, double *y, long long n, int add)
{
    const Level &l = c->lv[0];
    if (n % 4 == 0 && (uintptr_t)e % 16 == 0 && (uintptr_t)y % 16 == 0)
        k_float_to_double4<<<(unsigned)((n / 4 + 255) / 256), 256, 0, c->stream>>>(l.F, l.tP, e, y, n, add);
    else
        k_float_to_double<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(l.F, l.tP, e, y, n, add);
    c->launches++;
}

void add_float(Ctx *c, double *x, const float *e, long long n) { f2d(c, e, x, n, 1); }

void float_to_double(Ctx *c, const float *e, double *y, long long n) { f2d(c, e, y, n, 0); }

#define INST(T)                                                                 \
    template void residual<T>(Ctx *, int, const T *, const T *, T *);           \
    template void box_sweep<T>(Ctx *, int, T *, const T *);                     \
    template void scalar_update<T>(Ctx *, int, T *, const T *);                 \
    template void ghost_sweep<T>(Ctx *, int, T *, const T *);                   \
    template void smooth<T>(Ctx *, int, T *, const T *, int);                   \
    template void smooth_from<T>(Ctx *, int, T *, T *, const T *, int);         \
    template T *post_buffer<T>(Ctx *, int, T *, int);                           \
    template void prolong_to<T>(Ctx *, int, const T *, const T *, T *);         \
    template void restrict_level<T>(Ctx *, int, const T *, T *, T *);           \
    template void residual_restrict<T>(Ctx *, int, const T *, const T *, T *, T *, T *); \
    template void prolong_level<T>(Ctx *, int, const T *, T *);                 \
    template void zero_vec<T>(Ctx *, T *, long long);                           \
    template void zero_inactive<T>(Ctx *, int, T *);
INST(double)
INST(float)

}  // namespace gpmg
