// Internal definitions shared by the CUDA translation units of libgpmg.
//
// Device layout of one multigrid level with N cells per side:
//   frame of R = N + 2 rows and P >= N + 2 columns (P a multiple of 32);
//   slot (row, col) = row * P + col, row = j + 1, col = i + 1 for every grid;
//   u(i, j): i in [0, N],  j in [-1, N]   (rows j = -1 and j = N: box ghosts)
//   v(i, j): i in [-1, N], j in [0, N]    (columns i = -1 and i = N: box ghosts)
//   p(i, j): i, j in [0, N)
//   vector = [u frame | v frame | p frame | 32 scalars], scalar 0 = xi
//   (unknown) / mean row (equation).  Slots outside a grid's range are
//   inactive and hold 0.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gpmg.h"

namespace gpmg {

enum NodeType : uint8_t { T_INACTIVE = 0, T_INTERNAL = 1, T_GHOST = 2, T_WALL = 3, T_BOXGHOST = 4, T_EXT = 5 };
enum Grid { G_U = 0, G_V = 1, G_P = 2 };
// row kinds of the ghost list
enum RowKind : uint8_t { K_BCU = 0, K_EXTRAP = 1, K_COPY = 2, K_WALL = 3, K_BOXGHOST = 4 };

constexpr int MAX_LEVELS = 16;
constexpr int MAX_MARCH = 64;
constexpr int NSCAL = 32;
// scalar slot of an FP32 iterate holding its pending pressure shift (the
// internal and ghost pressures are the stored ones plus this value)
constexpr int PSHIFT_SLOT = 1;
constexpr int MAX_CUTCOL = 64;  // colours of the cut boxes
constexpr int ADJ_KMAX = 8;  // Picard iterations cn_step_adjoint can differentiate
// box codes (one byte per cell): a full box (internal cell, no ghost face)
// and which of its four faces are internal
constexpr unsigned BOX_FULL = 1, BOX_W = 2, BOX_E = 4, BOX_S = 8, BOX_N = 16, BOX_ALL = 31;
// prolongation codes (one byte per node and grid): the node is active and in
// its grid; every coarse node of its interpolation stencil is active too
constexpr uint8_t PRO_ON = 1, PRO_ALL = 2;
constexpr int GRAPH_T = 4 + GP_MAX_INNER - 1;  // captured kind: one transposed cycle and its residual
constexpr int GRAPH_KT = GRAPH_T + 1;          // captured kind: one BiCGSTAB iteration of the adjoint solve
constexpr int NGRAPH = GRAPH_KT + 1;           // captured iteration kinds
constexpr int GH_ST = 9;  // stencil slots per ghost row
// fused ghost sweeps: each block owns GC_OWN consecutive ghost-class rows and
// relaxes them together with every row they reach through at most lambda - 1
// stencil links (their closure, at most GC_CAP rows)
constexpr int GC_OWN = 128, GC_CAP = 512, GC_THREADS = 256;

// error bits written by kernels into the context's device status word
enum ErrBits : unsigned {
    E_STENCIL_OUT = 1u, E_INACTIVE_REF = 2u, E_PROJECTION = 4u, E_GHOST_CAP = 8u, E_CUT_CAP = 16u,
    E_NO_NORMAL = 32u, E_NO_INTERNAL = 64u, E_CLOSURE = 128u, E_SINGULAR = 256u
};

__host__ __device__ inline int frame_pitch(int N) { return ((N + 2 + 31) / 32) * 32; }
__host__ __device__ inline long long frame_size(int N) { return (long long)(N + 2) * frame_pitch(N); }
__host__ __device__ inline long long vec_len(int N) { return 3 * frame_size(N) + NSCAL; }

// Ghost-class rows of one level (object ghosts first, in (grid, j, i) order,
// then walls and box ghosts), structure of arrays of capacity `cap`.
struct GhostList {
    int *count;        // device: [0] object ghosts, [1] all rows
    int *node;         // global vector index of the row's own unknown
    uint8_t *kind;
    uint8_t *nst;
    int *st;           // [GH_ST][cap] vector indices of the stencil nodes
    double *w;         // [GH_ST][cap]
    float *wf;         // [GH_ST][cap]
    double *B;         // [2][cap] boundary point (Eq. BCu rows)
    double *th;        // [2][cap] theta
    double *upd;       // [cap] Jacobi update scratch
    float *updf;
    double *acc;       // [2][cap] accumulated corrections of the fused sweeps (ping-pong)
    float *accf;
    int *strow;        // [GH_ST][cap] ghost-row index of each stencil node, or -1
    int *cl_row;       // [cap / GC_OWN + 1][GC_CAP] rows of each block's closure, ascending
    int16_t *cl_lnk;   // [cap / GC_OWN + 1][GH_ST][GC_CAP] closure position of each stencil node's row, or -1
    int *cl_n;         // [cap / GC_OWN + 1] closure size of each block (-1: above GC_CAP)
    int cap;
};

// cut cells (internal cells with a ghost border) sorted by colour (recolour_cuts)
constexpr int CUT_ST = 9;  // stencil entries per box row
struct CutList {
    int *count;        // device [1]
    int *off;          // device [MAX_CUTCOL + 1] colour offsets
    int *cell;         // slot of the cell (row * P + col)
    int *gface;        // [4][cap] ghost-list index of face W, E, S, N (or -1)
    // box rows prepared for the current alpha (k_cut_prepare): for row
    // f = W, E, S, N, continuity: the vector index of its unknown and rhs
    // (-1 when the row takes no part), CUT_ST (index, coefficient) pairs of
    // the full row, and the inverse of the 5 x 5 box matrix
    int *row;          // [5][cap]
    int *sidx;         // [5 * CUT_ST][cap]
    double *scoef;     // [5 * CUT_ST][cap]
    float *scoeff;
    double *minv;      // [25][cap]
    float *minvf;
    int cap;
    int ncol;          // colours (the list is sorted by colour)
};

struct Level {
    int N;
    int P;
    long long F;       // frame size
    long long VL;      // vector length
    double h;
    uint8_t *tU, *tV, *tP;
    uint8_t *bcode;    // [F] box code of each cell (BOX_FULL and its internal faces, or 0)
    uint8_t *pcode;    // [3 F] prolongation code of each node (from the next coarser level; not on the coarsest)
    uint8_t *prim;     // [3 * F] ghost referenced by an internal row
    uint8_t *done;     // [3 * F] ghost row computed (closure passes)
    double *x, *b, *r; // vectors owned by the context (coarse levels; r on all)
    float *xf, *bf, *rf;
    GhostList gh;
    CutList cut;
    int *lonely;       // list of lonely internal faces (vector indices)
    int *nlonely;      // device [1]
    int lonely_cap;
    int *nint;         // device [1] internal pressure cells
    int h_nint;        // host copy
    int h_nghost;      // host copies after geometry_build
    int h_nrows;
    int h_ncut;
    int h_cutoff[MAX_CUTCOL + 1];
    int h_nlonely;
    int h_fused;       // the lambda ghost sweeps run as one launch over the row closures
    // adjoint (carved when gp_params.adjoint is set): the columns of M
    // referenced by ghost-class rows, sorted, each with its (row node,
    // weight) entries; the ghost-row part of M^T lam at those columns (0 at
    // every other slot); the column-list index of each cut-box unknown
    int *tl_node, *tl_ptr, *tl_src;
    double *tl_w;
    int tl_cap, h_tl_n;
    double *gtd;
    int *cut_tl;
};

struct Ctx {
    gp_params prm;
    cudaStream_t stream;
    char *ws;
    size_t ws_bytes;
    int L;
    Level lv[MAX_LEVELS];
    double *phi;        // paper-sign half lattice (2N+1)^2
    double *cn_xn, *cn_Nn, *cn_Nh, *cn_b;  // cn_step scratch (finest level)
    const double *csrc;  // continuity source g (caller's finest-level vector, p frame), or null
    // coarsest level dense inverse
    int nc;             // unknowns of the coarsest level (flat order)
    double *Minv;       // nc x nc
    float *Minvf;
    double *aug;        // nc x 2nc work for Gauss-Jordan
    unsigned long long *gjkeys;  // nc pivot keys (|a| and row) of the Gauss-Jordan steps
    uint8_t *gjused;    // nc flags: row already a pivot row
    cudaGraphExec_t gj_exec;  // the captured Gauss-Jordan elimination (null until first used)
    int *cmap;          // flat index -> vector index on the coarsest level
    double *cvec;       // 2 * nc gather/scatter buffer
    float *cvecf;
    int *piv;           // device pivot index
    // reductions
    double *part;       // block partials
    int npart;
    double *red;        // small result area (device)
    unsigned long long *maxbits;
    unsigned *err;      // device error words: [0] geometry / coarse factorisation, [2] a tile copy wait ran out
    int *flag;          // device change flag
    double hostbuf[8];   // host staging for small device-to-host reads
    // instrumentation: kernels launched, and an optional event timer around
    // the launches of one kernel family on one level
    long long launches;
    int tmr_kernel, tmr_level, tmr_n, tmr_ready;
    cudaEvent_t tmr_ev[2 * 512];
    double tmr_ms;
    long long tmr_launches;
    // captured mg_solve iterations: [0] FP64 cycle + residual, [1] FP32 cycle
    // inside FP64 residual correction, [2] / [3] BiCGSTAB iteration with an
    // FP64 / FP32 cycle, [4 + k - 2] k FP32 cycles inside one FP64 residual
    // correction, [GRAPH_T] / [GRAPH_KT] an iteration of the plain / BiCGSTAB
    // adjoint solve; keyed by the iterate and rhs pointers
    cudaGraphExec_t gexec[NGRAPH];
    const void *gx[NGRAPH], *gb[NGRAPH];
    int gvalid[NGRAPH];
    long long glaunches[NGRAPH];
    int inner_now;       // FP32 cycles of the next residual correction
    int graphs_off;
    // BiCGSTAB vectors (finest level): r, rh, p, -v, s, -t, y, z, 0, true residual
    double *kv[10];
    double *ks;          // device scalars rho, alpha, omega, beta
    double *kpart;       // dot-product partials
    int kpart_n;
    int geom_ok;
    int coarse_ok;
    double alpha_factored;
    int adj_ok;            // adjoint column lists built for this geometry
    double *adjv[12];      // finest-level vectors of cn_step_adjoint (lam, E lam, g, xbar, Picard iterates)
    char msg[256];
};

// kernel families for the event timer (gp_timer_start)
enum TimedKernel { KT_RESIDUAL = 0, KT_BOX_FULL = 1, KT_BOX_CUT = 2, KT_GHOST = 3, KT_SCALAR = 4, KT_RESTRICT = 5,
                   KT_PROLONG = 6, KT_COARSE = 7 };

void tmr_begin(Ctx *c, int kernel, int lev);
void tmr_end(Ctx *c, int kernel, int lev);

// ------------------------------------------------------------ indexing
__host__ __device__ inline int slot_u(int P, int i, int j) { return (j + 1) * P + (i + 1); }

__device__ inline bool in_grid(int g, int N, int i, int j)
{
    if (g == G_U) return i >= 0 && i <= N && j >= -1 && j <= N;
    if (g == G_V) return i >= -1 && i <= N && j >= 0 && j <= N;
    return i >= 0 && i < N && j >= 0 && j < N;
}

// ------------------------------------------ grid transfers (Sects. 4.2, 4.3)
__device__ inline bool same_class(uint8_t tc, uint8_t tf)
{
    if (tc == T_INTERNAL) return tf == T_INTERNAL;
    return tf == T_GHOST || tf == T_WALL || tf == T_BOXGHOST;
}

__device__ inline uint8_t tget(const uint8_t *t, int g, int N, int P, int i, int j)
{
    if (!in_grid(g, N, i, j)) return T_INACTIVE;
    return t[(long long)(j + 1) * P + (i + 1)];
}

// Bilinear interpolation (Sect. 4.3) factors into one-axis taps.  Along an
// axis where the grid's nodes lie on the nodes or cell midpoints of its
// coarse grid ("aligned"), fine index k sits at coarse coordinate c = k / 2;
// along a staggered axis at c = k / 2 - 1 / 4.  With q = 4 c (an integer), the
// taps are the coarse nodes floor(c) and floor(c) + 1 with linear weights,
// the nearer node first (the lower one when c is midway; a single tap when c
// is a coarse node).  A far node outside [lo, hi] is replaced by linear
// extrapolation from the near node and the one beyond it, 5/4 and -1/4.
template <typename T> __device__ inline int taps(int k, bool aligned, int lo, int hi, int *K, T *w)
{
    const int q = aligned ? 2 * k : 2 * k - 1;
    const int fl = q >= 0 ? q / 4 : -((3 - q) / 4);  // floor(q / 4)
    const int r = q - 4 * fl;                         // 4 (c - floor(c)), 0..3
    if (r == 0) {
        K[0] = fl;
        w[0] = (T)1;
        return 1;
    }
    const int near = r == 3 ? fl + 1 : fl, far = r == 3 ? fl : fl + 1;
    if (far < lo || far > hi) {
        K[0] = near;
        w[0] = (T)1.25;
        K[1] = 2 * near - far;
        w[1] = (T)-0.25;
        return 2;
    }
    K[0] = near;
    w[0] = (T)(r == 2 ? 0.5 : 0.75);
    K[1] = far;
    w[1] = (T)(r == 2 ? 0.5 : 0.25);
    return 2;
}

}  // namespace gpmg
