// Adjoint of the multigrid solve: the transposed system M^T lam = c (the
// gradient of a function of the solution of Eq. (LS) with respect to its
// right-hand side) and the transposed cycle, FP64.
//
// A cycle from x = 0 is a linear map B of b made of stages that each add
// Q (b - M x); its transpose is the cycle for M^T with the stages in reverse
// order and each Q transposed: ghost Jacobi sweeps before the (xi, mean)
// step, the lonely faces, the cut boxes in reverse colour order, the full boxes in
// colours 4..0, post- before pre-relaxations, P^T as restriction, R^T as
// interpolation, and the coarsest solve with the transposed inverse.  Rows of
// M^T at inactive nodes involve only ghost-row terms and are solved exactly
// after each cycle.
//
// (M^T lam)_k is the sum over the rows of M that reference node k: the
// internal momentum, continuity and mean rows (fixed patterns, gathered with
// type checks) and the ghost-class rows (their stencils reach arbitrary
// nodes near the body; the referenced columns are listed once per geometry
// with their (row, weight) entries).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gpmg_internal.cuh"

namespace gpmg {

struct TArgs {
    int N, P;
    long long F;
    double q, a, d, h2;
    double qida, qid, id, idet;
    double ic1[9];
    const uint8_t *tU, *tV, *tP;
};

static TArgs targs(const Ctx *c, int lev)
{
    const Level &l = c->lv[lev];
    TArgs A;
    A.N = l.N;
    A.P = l.P;
    A.F = l.F;
    double h = c->prm.L / (double)l.N;
    A.q = 1.0 / h;
    A.a = c->prm.alpha / (h * h);
    A.d = 1.0 + 4.0 * A.a;
    A.h2 = h * h;
    A.qida = A.q / (A.d + A.a);
    A.qid = A.q / A.d;
    A.id = 1.0 / A.d;
    A.idet = 1.0 / (A.d * A.d - A.a * A.a);
    const double cx[3] = {0.0, A.q * A.q / A.d, 2.0 * A.q * A.q / (A.d + A.a)};
    for (int nx = 0; nx < 3; nx++)
        for (int ny = 0; ny < 3; ny++) A.ic1[nx * 3 + ny] = nx + ny == 0 ? 0.0 : 1.0 / (cx[nx] + cx[ny]);
    A.tU = l.tU;
    A.tV = l.tV;
    A.tP = l.tP;
    return A;
}

// the part of (M^T lam) at slot s of grid g that comes from internal rows,
// the mean row and the node's own inactive row
__device__ inline double colt_struct(const TArgs &A, const double *lam, int g, long long s)
{
    const int P = A.P;
    const long long row = s / P;
    const int col = (int)(s - row * P);
    const bool hw = col > 0, he = col < P - 1, hs = row > 0, hn = row < A.N + 1;
    const double *lu = lam, *lv = lam + A.F, *lp = lam + 2 * A.F;
    double sum = 0.0;
    if (g == G_U) {
        const uint8_t *t = A.tU;
        if (t[s] == T_INTERNAL) sum += A.d * lu[s];
        else if (t[s] == T_INACTIVE) sum += lu[s];
        if (he && t[s + 1] == T_INTERNAL) sum -= A.a * lu[s + 1];
        if (hw && t[s - 1] == T_INTERNAL) sum -= A.a * lu[s - 1];
        if (hn && t[s + P] == T_INTERNAL) sum -= A.a * lu[s + P];
        if (hs && t[s - P] == T_INTERNAL) sum -= A.a * lu[s - P];
        if (A.tP[s] == T_INTERNAL) sum -= A.q * lp[s];             // continuity row of cell (i, j)
        if (hw && A.tP[s - 1] == T_INTERNAL) sum += A.q * lp[s - 1];  // of cell (i - 1, j)
    } else if (g == G_V) {
        const uint8_t *t = A.tV;
        if (t[s] == T_INTERNAL) sum += A.d * lv[s];
        else if (t[s] == T_INACTIVE) sum += lv[s];
        if (he && t[s + 1] == T_INTERNAL) sum -= A.a * lv[s + 1];
        if (hw && t[s - 1] == T_INTERNAL) sum -= A.a * lv[s - 1];
        if (hn && t[s + P] == T_INTERNAL) sum -= A.a * lv[s + P];
        if (hs && t[s - P] == T_INTERNAL) sum -= A.a * lv[s - P];
        if (A.tP[s] == T_INTERNAL) sum -= A.q * lp[s];
        if (hs && A.tP[s - P] == T_INTERNAL) sum += A.q * lp[s - P];
    } else {
        if (A.tU[s] == T_INTERNAL) sum += A.q * lu[s];               // u(i, j) row: + q p(i, j)
        if (he && A.tU[s + 1] == T_INTERNAL) sum -= A.q * lu[s + 1];  // u(i + 1, j) row: - q p(i, j)
        if (A.tV[s] == T_INTERNAL) sum += A.q * lv[s];
        if (hn && A.tV[s + P] == T_INTERNAL) sum -= A.q * lv[s + P];
        if (A.tP[s] == T_INTERNAL) sum += A.h2 * lam[3 * A.F];       // mean row
        else if (A.tP[s] == T_INACTIVE) sum += lp[s];
    }
    return sum;
}

__device__ inline double ghost_part(const Level &l, int t, const double *lam)
{
    if (t < 0) return 0.0;
    double s = 0.0;
    for (int e = l.tl_ptr[t]; e < l.tl_ptr[t + 1]; e++) s += l.tl_w[e] * lam[l.tl_src[e]];
    return s;
}

// gtd at every listed column: the ghost-row part of (M^T lam)
__global__ void k_gtd(Level l, const double *lam)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < l.h_tl_n) l.gtd[l.tl_node[t]] = ghost_part(l, t, lam);
}

// r = c - M^T lam on internal, ghost and inactive slots of the grids (0 on
// padding); per block: [0] sum of lam over internal continuity rows, [1] max |r|
__global__ void k_residual_t(TArgs A, const double *lam, const double *cc, const double *gtd, double *r,
                             double *part)
{
    double lsum = 0.0, rmax = 0.0;
    const long long nslot = (long long)(A.N + 2) * A.P;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nslot; s += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(s / A.P), col = (int)(s - (long long)row * A.P);
        for (int g = 0; g < 3; g++) {
            const long long k = g * A.F + s;
            if (!in_grid(g, A.N, col - 1, row - 1)) {
                r[k] = 0.0;
                continue;
            }
            double v = cc[k] - colt_struct(A, lam, g, s) - gtd[k];
            r[k] = v;
            rmax = (rmax != rmax || v != v) ? (double)NAN : fmax(rmax, fabs(v));
        }
        if (A.tP[s] == T_INTERNAL) lsum += lam[2 * A.F + s];
    }
    __shared__ double ss[256], sm[256];
    ss[threadIdx.x] = lsum;
    sm[threadIdx.x] = rmax;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            double a = sm[threadIdx.x], b = sm[threadIdx.x + o];
            sm[threadIdx.x] = (a != a || b != b) ? (double)NAN : fmax(a, b);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = ss[0];
        part[2 * blockIdx.x + 1] = sm[0];
    }
}

// the xi slot (xi column of M: -1 at every internal continuity row), the
// padding scalars and the norm (out[0])
__global__ void k_residual_t_final(const double *part, int nb, const double *cc, double *r, long long ixi, double *out)
{
    __shared__ double ss[256], sm[256];
    double s = 0.0, m = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        s += part[2 * k];
        double v = part[2 * k + 1];
        m = (m != m || v != v) ? (double)NAN : fmax(m, v);
    }
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            double a = sm[threadIdx.x], b = sm[threadIdx.x + o];
            sm[threadIdx.x] = (a != a || b != b) ? (double)NAN : fmax(a, b);
        }
        __syncthreads();
    }
    if (threadIdx.x < NSCAL) r[ixi + threadIdx.x] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double rx = cc[ixi] + ss[0];
        r[ixi] = rx;
        double v = sm[0];
        out[0] = (v != v || rx != rx) ? (double)NAN : fmax(v, fabs(rx));
    }
}

// transposed ghost Jacobi: upd = dtau (c - M^T lam) at every ghost-class node
__global__ void k_ghost_update_t(TArgs A, GhostList gh, int n, const double *lam, const double *cc, const double *gtd,
                                 double dtau)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long node = gh.node[k];
    const int g = (int)(node / A.F);
    const long long s = node - g * A.F;
    gh.upd[k] = dtau * (cc[node] - colt_struct(A, lam, g, s) - gtd[node]);
}

__global__ void k_apply_upd(const int *node, const double *upd, int n, double *lam)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) lam[node[k]] += upd[k];
}

// transposed (xi, mean) step, partial sums: [0] lam over internal continuity
// rows, [1] (c - M^T lam) over internal and ghost p
__global__ void k_scalar_t_partial(TArgs A, const double *lam, const double *cc, const double *gtd, double *part)
{
    double a1 = 0.0, a2 = 0.0;
    const long long nslot = (long long)(A.N + 2) * A.P;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nslot; s += (long long)gridDim.x * blockDim.x) {
        const uint8_t t = A.tP[s];
        if (t == T_INTERNAL) a1 += lam[2 * A.F + s];
        if (t == T_INTERNAL || t == T_GHOST) {
            const long long k = 2 * A.F + s;
            a2 += cc[k] - colt_struct(A, lam, G_P, s) - gtd[k];
        }
    }
    __shared__ double s1[256], s2[256];
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1[0];
        part[2 * blockIdx.x + 1] = s2[0];
    }
}

// red[0] = -(xi residual of M^T) / n_int, red[1] = (sum of p residuals) / (h^2 n_int)
__global__ void k_scalar_t_final(const double *part, int nb, const double *cc, long long ixi, double h2, const int *nint,
                                 double *red)
{
    __shared__ double s1[256], s2[256];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double n = (double)nint[0];
        double rxi = cc[ixi] + s1[0];
        red[0] = -rxi / n;
        red[1] = s2[0] / (h2 * n);
    }
}

__global__ void k_scalar_t_apply(TArgs A, const double *red, double *lam)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= A.P) return;
    long long s = (long long)row * A.P + col;
    if (A.tP[s] == T_INTERNAL) lam[2 * A.F + s] += red[0];
    if (row == 0 && col == 0) lam[3 * A.F] += red[1];
}

// inactive rows of M^T: lam_k = c_k - (ghost-row part)
__global__ void k_fix_inactive_t(TArgs A, const double *cc, const double *gtd, double *lam)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= A.P) return;
    long long s = (long long)row * A.P + col;
    const uint8_t *t[3] = {A.tU, A.tV, A.tP};
#pragma unroll
    for (int g = 0; g < 3; g++) {
        if (!in_grid(g, A.N, col - 1, row - 1) || t[g][s] != T_INACTIVE) continue;
        const long long k = g * A.F + s;
        lam[k] = cc[k] - gtd[k];
    }
}

// ------------------------------------------------------- transposed boxes

// solve A d = r for a full box (the Schur-complement solve of the forward
// sweep); false when no face takes part
__device__ inline bool box_solve(const TArgs &A, bool W, bool E, bool S, bool Nn, double rW, double rE, double rS,
                                 double rN, double rC, double &dW, double &dE, double &dS, double &dN, double &dp)
{
    double c0 = 0.0;
    int nx = 0, ny = 0;
    if (W && E) {
        c0 += A.qida * (rE - rW);
        nx = 2;
    } else if (W) {
        c0 -= A.qid * rW;
        nx = 1;
    } else if (E) {
        c0 += A.qid * rE;
        nx = 1;
    }
    if (S && Nn) {
        c0 += A.qida * (rN - rS);
        ny = 2;
    } else if (S) {
        c0 -= A.qid * rS;
        ny = 1;
    } else if (Nn) {
        c0 += A.qid * rN;
        ny = 1;
    }
    if (nx + ny == 0) return false;
    const int kc = nx * 3 + ny;
    double ic = A.ic1[1];
#pragma unroll
    for (int k = 2; k < 9; k++)
        if (kc == k) ic = A.ic1[k];
    dp = (rC - c0) * ic;
    const double q = A.q, a = A.a, d = A.d;
    double fW = rW - q * dp, fE = rE + q * dp, fS = rS - q * dp, fN = rN + q * dp;
    dW = dE = dS = dN = 0.0;
    if (W && E) {
        dW = (d * fW + a * fE) * A.idet;
        dE = (a * fW + d * fE) * A.idet;
    } else if (W) dW = fW * A.id;
    else if (E) dE = fE * A.id;
    if (S && Nn) {
        dS = (d * fS + a * fN) * A.idet;
        dN = (a * fS + d * fN) * A.idet;
    } else if (S) dS = fS * A.id;
    else if (Nn) dN = fN * A.id;
    return true;
}

// one colour of the full boxes on M^T.  The box matrix A couples the faces
// to p antisymmetrically (+q in the momentum rows, -q in the continuity
// row), so A^T = S A S with S = diag(1, 1, 1, 1, -1): the transposed box is
// the forward solve with the p residual and the p correction negated.
__global__ void k_box_full_t(TArgs A, double *lam, const double *cc, const double *gtd, int colour)
{
    int j = blockIdx.y;
    int i0 = ((colour - 3 * j) % 5 + 5) % 5;
    int i = i0 + 5 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= A.N) return;
    const long long s = (long long)(j + 1) * A.P + (i + 1), F = A.F;
    if (A.tP[s] != T_INTERNAL) return;
    const uint8_t tW = A.tU[s], tE = A.tU[s + 1], tS = A.tV[s], tN = A.tV[s + A.P];
    if (tW == T_GHOST || tE == T_GHOST || tS == T_GHOST || tN == T_GHOST) return;
    const bool W = tW == T_INTERNAL, E = tE == T_INTERNAL, S = tS == T_INTERNAL, Nn = tN == T_INTERNAL;
    double rW = W ? cc[s] - colt_struct(A, lam, G_U, s) - gtd[s] : 0.0;
    double rE = E ? cc[s + 1] - colt_struct(A, lam, G_U, s + 1) - gtd[s + 1] : 0.0;
    double rS = S ? cc[F + s] - colt_struct(A, lam, G_V, s) - gtd[F + s] : 0.0;
    double rN = Nn ? cc[F + s + A.P] - colt_struct(A, lam, G_V, s + A.P) - gtd[F + s + A.P] : 0.0;
    double rC = cc[2 * F + s] - colt_struct(A, lam, G_P, s) - gtd[2 * F + s];
    double dW, dE, dS, dN, dp;
    if (!box_solve(A, W, E, S, Nn, rW, rE, rS, rN, -rC, dW, dE, dS, dN, dp)) return;
    if (W) lam[s] += dW;
    if (E) lam[s + 1] += dE;
    if (S) lam[F + s] += dS;
    if (Nn) lam[F + s + A.P] += dN;
    lam[2 * F + s] -= dp;
}

// one colour of the cut boxes on M^T: residuals of the transposed rows at the
// box unknowns (ghost-row parts summed on the fly: ghost unknowns of this
// colour change), the transposed stored inverse.  Eight lanes per box: lane
// f < 5 computes row f's residual, then its correction from the five
// residuals of the group (warp shuffles), in the serial order.
__global__ void k_box_cut_t(TArgs A, Level l, double *lam, const double *cc, int beg, int end)
{
    const int lane = threadIdx.x & 31, f = lane & 7;
    const int k = beg + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 3);
    const bool valid = k < end && f < 5;
    const CutList &cut = l.cut;
    int row = -1;
    double r = 0.0;
    if (valid) {
        row = cut.row[(long long)f * cut.cap + k];
        if (row >= 0) {
            const int g = (int)(row / A.F);
            const long long s = row - g * A.F;
            r = cc[row] - colt_struct(A, lam, g, s) - ghost_part(l, l.cut_tl[(long long)f * cut.cap + k], lam);
        }
    }
    double d = 0.0;
#pragma unroll
    for (int c = 0; c < 5; c++) {
        const double rc = __shfl_sync(0xffffffffu, r, (lane & ~7) + c);
        if (valid) d += cut.minv[(long long)(c * 5 + f) * cut.cap + k] * rc;
    }
    if (valid && row >= 0) lam[row] += d;
}

// lonely internal faces on M^T: point Jacobi with the diagonal d
__global__ void k_lonely_t(TArgs A, const int *list, int n, const double *lam, const double *cc, const double *gtd,
                           double *upd)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long o = list[k];
    const int g = (int)(o / A.F);
    const long long s = o - g * A.F;
    upd[k] = (cc[o] - colt_struct(A, lam, g, s) - gtd[o]) / A.d;
}

// --------------------------------------------------- transposed transfers

// cH = P^T r: every active coarse node gathers the fine nodes whose
// interpolation taps reach it (fine offsets -2..3 from 2I, 2J cover the
// aligned, staggered and extrapolated taps), with the fine node's
// renormalised weight
__global__ void k_prolong_t(int Nf, int Pf, long long Ff, const uint8_t *pcode, int Nc, int Pc, long long Fc,
                            const uint8_t *tUc, const uint8_t *tVc, const uint8_t *tPc, const double *r, double *cH)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= Pc) return;
    const int I = col - 1, J = row - 1;
    const long long sc = (long long)row * Pc + col;
    const uint8_t *tc[3] = {tUc, tVc, tPc};
    if (row == 0 && col < NSCAL) cH[3 * Fc + col] = col == 0 ? r[3 * Ff] : 0.0;
#pragma unroll
    for (int g = 0; g < 3; g++) {
        if (!in_grid(g, Nc, I, J) || tc[g][sc] == T_INACTIVE) {
            cH[g * Fc + sc] = 0.0;
            continue;
        }
        const int Ilo = g == G_V ? -1 : 0, Ihi = g == G_P ? Nc - 1 : Nc;
        const int Jlo = g == G_U ? -1 : 0, Jhi = g == G_P ? Nc - 1 : Nc;
        double acc = 0.0;
        for (int dj = -2; dj <= 3; dj++)
            for (int di = -2; di <= 3; di++) {
                const int i = 2 * I + di, j = 2 * J + dj;
                // the fine node's prolongation code (0 outside its grid)
                const uint8_t pc = in_grid(g, Nf, i, j) ? pcode[g * Ff + (long long)(j + 1) * Pf + (i + 1)] : 0;
                if (!(pc & PRO_ON)) continue;
                int KI[2], KJ[2];
                double wi[2], wj[2];
                int ni = taps<double>(i, g == G_U, Ilo, Ihi, KI, wi);
                int nj = taps<double>(j, g == G_V, Jlo, Jhi, KJ, wj);
                double ws = 0.0, w = 0.0;
                for (int a = 0; a < nj; a++)
                    for (int bb = 0; bb < ni; bb++) {
                        // a wholly active stencil needs no type lookups (its weights sum to 1)
                        if (!(pc & PRO_ALL) && tget(tc[g], g, Nc, Pc, KI[bb], KJ[a]) == T_INACTIVE) continue;
                        ws += wj[a] * wi[bb];
                        if (KI[bb] == I && KJ[a] == J) w += wj[a] * wi[bb];
                    }
                if (ws > 0.0 && w != 0.0) acc += w / ws * r[g * Ff + (long long)(j + 1) * Pf + (i + 1)];
            }
        cH[g * Fc + sc] = acc;
    }
}

// lam += R^T yH: every fine node gathers the coarse nodes whose restriction
// stencil holds it (Eq. restop weights where the whole stencil is of the
// coarse node's class, else 1 / (members of that class), Eq. restop5)
__global__ void k_restrict_t(int Nf, int Pf, long long Ff, const uint8_t *tUf, const uint8_t *tVf, const uint8_t *tPf,
                             int Nc, int Pc, long long Fc, const uint8_t *tUc, const uint8_t *tVc, const uint8_t *tPc,
                             const double *yH, double *lam)
{
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    int row = blockIdx.y;
    if (col >= Pf) return;
    const int i = col - 1, j = row - 1;
    const long long sf = (long long)row * Pf + col;
    const uint8_t *tf[3] = {tUf, tVf, tPf};
    const uint8_t *tc[3] = {tUc, tVc, tPc};
    if (row == 0 && col == 0) lam[3 * Ff] += yH[3 * Fc];
#pragma unroll
    for (int g = 0; g < 3; g++) {
        if (!in_grid(g, Nf, i, j)) continue;
        const uint8_t tff = tf[g][sf];
        double acc = 0.0;
        for (int J = (j >> 1) - 1; J <= (j >> 1) + 1; J++)
            for (int I = (i >> 1) - 1; I <= (i >> 1) + 1; I++) {
                const uint8_t t = tget(tc[g], g, Nc, Pc, I, J);
                if (t == T_INACTIVE || !same_class(t, tff)) continue;
                int fi[6], fj[6], ns = 0;
                double wt[6];
                if (g == G_U) {
                    for (int dj = 0; dj <= 1; dj++)
                        for (int di = -1; di <= 1; di++) { fi[ns] = 2 * I + di; fj[ns] = 2 * J + dj; wt[ns] = di == 0 ? 0.25 : 0.125; ns++; }
                } else if (g == G_V) {
                    for (int dj = -1; dj <= 1; dj++)
                        for (int di = 0; di <= 1; di++) { fi[ns] = 2 * I + di; fj[ns] = 2 * J + dj; wt[ns] = dj == 0 ? 0.25 : 0.125; ns++; }
                } else {
                    for (int dj = 0; dj <= 1; dj++)
                        for (int di = 0; di <= 1; di++) { fi[ns] = 2 * I + di; fj[ns] = 2 * J + dj; wt[ns] = 0.25; ns++; }
                }
                bool all = true, mine = false;
                int cnt = 0;
                double wme = 0.0;
                for (int k = 0; k < ns; k++) {
                    if (same_class(t, tget(tf[g], g, Nf, Pf, fi[k], fj[k]))) cnt++;
                    else all = false;
                    if (fi[k] == i && fj[k] == j) {
                        mine = true;
                        wme = wt[k];
                    }
                }
                if (!mine) continue;
                const double y = yH[g * Fc + (long long)(J + 1) * Pc + (I + 1)];
                acc += all ? wme * y : y / (double)cnt;
            }
        lam[g * Ff + sf] += acc;
    }
}

// y = M^T x for a dense row-major n x n matrix: a block per 32 columns, its
// 32 thread rows take every 32nd matrix row (coalesced along the columns)
// and the 32 partial sums of a column are added in a fixed tree order
__global__ void __launch_bounds__(1024) k_gemv_t(const double *M, const double *x, double *y, int n)
{
    __shared__ double part[32][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    double s = 0.0;
    if (c < n)
        for (int r = threadIdx.y; r < n; r += 32) s += M[(long long)r * n + c] * x[r];
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) {
        if (threadIdx.y < o) part[threadIdx.y][threadIdx.x] += part[threadIdx.y + o][threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.y == 0 && c < n) y[c] = part[0][threadIdx.x];
}

__global__ void k_gather_d(const double *b, const int *cmap, double *cv, int n)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < n) cv[f] = b[cmap[f]];
}

__global__ void k_scatter_d(const double *cv, const int *cmap, double *x, int n)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < n) x[cmap[f]] = cv[f];
}

__global__ void k_zero_d(double *x, long long n)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) x[k] = 0.0;
}

// ------------------------------------------------------------- host side

static inline int nblocks_red(const Level &l)
{
    long long n = (l.F + 255) / 256;
    return (int)(n < 1024 ? n : 1024);
}

static inline dim3 fgrid(const Level &l) { return dim3((l.P + 255) / 256, l.N + 2); }

// the column lists of every level (once per geometry): the ghost-class rows
// are copied to the host, their (column, row node, weight) entries sorted by
// column, and the lists copied back with the list index of each cut-box
// unknown
int adjoint_prepare(Ctx *c)
{
    if (c->adj_ok) return GP_OK;
    if (!c->prm.adjoint) {
        snprintf(c->msg, sizeof c->msg, "adjoint arrays not carved: create the context with gp_params.adjoint = 1");
        return GP_INVALID;
    }
    cudaStream_t st = c->stream;
    struct Entry {
        int col, src;
        double w;
    };
    for (int lev = 0; lev < c->L; lev++) {
        Level &l = c->lv[lev];
        const int n = l.h_nrows, cap = l.gh.cap;
        std::vector<int> node(n > 0 ? n : 1), stv((size_t)GH_ST * (n > 0 ? n : 1));
        std::vector<uint8_t> nst(n > 0 ? n : 1);
        std::vector<double> w((size_t)GH_ST * (n > 0 ? n : 1));
        if (n > 0) {
            cudaMemcpyAsync(node.data(), l.gh.node, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(nst.data(), l.gh.nst, n, cudaMemcpyDeviceToHost, st);
            for (int q = 0; q < GH_ST; q++) {
                cudaMemcpyAsync(stv.data() + (size_t)q * n, l.gh.st + (size_t)q * cap, sizeof(int) * n,
                                cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(w.data() + (size_t)q * n, l.gh.w + (size_t)q * cap, sizeof(double) * n,
                                cudaMemcpyDeviceToHost, st);
            }
        }
        std::vector<int> crow(5 * (size_t)(l.h_ncut > 0 ? l.h_ncut : 1));
        for (int f = 0; f < 5 && l.h_ncut > 0; f++)
            cudaMemcpyAsync(crow.data() + (size_t)f * l.h_ncut, l.cut.row + (size_t)f * l.cut.cap,
                            sizeof(int) * l.h_ncut, cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            snprintf(c->msg, sizeof c->msg, "adjoint_prepare: %s", cudaGetErrorString(cudaGetLastError()));
            return GP_CUDA;
        }
        std::vector<Entry> e;
        e.reserve((size_t)n * 6);
        for (int k = 0; k < n; k++)
            for (int q = 0; q < nst[k]; q++) e.push_back({stv[(size_t)q * n + k], node[k], w[(size_t)q * n + k]});
        std::stable_sort(e.begin(), e.end(), [](const Entry &a, const Entry &b) {
            return a.col != b.col ? a.col < b.col : a.src < b.src;
        });
        if ((long long)e.size() > l.tl_cap) {
            snprintf(c->msg, sizeof c->msg, "adjoint_prepare: %zu ghost-row entries exceed the capacity %d", e.size(),
                     l.tl_cap);
            return GP_INVALID;
        }
        std::vector<int> tnode, tptr(1, 0), tsrc(e.size());
        std::vector<double> tw(e.size());
        for (size_t k = 0; k < e.size(); k++) {
            if (k == 0 || e[k].col != e[k - 1].col) {
                if (k > 0) tptr.push_back((int)k);
                tnode.push_back(e[k].col);
            }
            tsrc[k] = e[k].src;
            tw[k] = e[k].w;
        }
        if (!e.empty()) tptr.push_back((int)e.size());
        l.h_tl_n = (int)tnode.size();
        std::vector<int> ctl(5 * (size_t)(l.h_ncut > 0 ? l.h_ncut : 1), -1);
        for (int f = 0; f < 5; f++)
            for (int k = 0; k < l.h_ncut; k++) {
                int r = crow[(size_t)f * l.h_ncut + k];
                if (r < 0) continue;
                auto it = std::lower_bound(tnode.begin(), tnode.end(), r);
                if (it != tnode.end() && *it == r) ctl[(size_t)f * l.h_ncut + k] = (int)(it - tnode.begin());
            }
        if (l.h_tl_n > 0) {
            cudaMemcpyAsync(l.tl_node, tnode.data(), sizeof(int) * tnode.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(l.tl_ptr, tptr.data(), sizeof(int) * tptr.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(l.tl_src, tsrc.data(), sizeof(int) * tsrc.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(l.tl_w, tw.data(), sizeof(double) * tw.size(), cudaMemcpyHostToDevice, st);
        }
        for (int f = 0; f < 5 && l.h_ncut > 0; f++)
            cudaMemcpyAsync(l.cut_tl + (size_t)f * l.cut.cap, ctl.data() + (size_t)f * l.h_ncut, sizeof(int) * l.h_ncut,
                            cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(l.gtd, 0, sizeof(double) * l.VL, st);
        // the host vectors must outlive the copies
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            snprintf(c->msg, sizeof c->msg, "adjoint_prepare: %s", cudaGetErrorString(cudaGetLastError()));
            return GP_CUDA;
        }
    }
    c->adj_ok = 1;
    return GP_OK;
}

static void gtd_update(Ctx *c, int lev, const double *lam)
{
    const Level &l = c->lv[lev];
    if (l.h_tl_n <= 0) return;
    k_gtd<<<(l.h_tl_n + 255) / 256, 256, 0, c->stream>>>(l, lam);
    c->launches++;
}

// r = c - M^T lam; the norm goes to c->red[4]
void residual_t(Ctx *c, int lev, const double *lam, const double *cc, double *r)
{
    const Level &l = c->lv[lev];
    gtd_update(c, lev, lam);
    int nb = nblocks_red(l);
    k_residual_t<<<nb, 256, 0, c->stream>>>(targs(c, lev), lam, cc, l.gtd, r, c->part);
    k_residual_t_final<<<1, 256, 0, c->stream>>>(c->part, nb, cc, r, 3 * l.F, c->red + 4);
    c->launches += 2;
}

void ghost_sweep_t(Ctx *c, int lev, double *lam, const double *cc)
{
    const Level &l = c->lv[lev];
    if (l.h_nrows <= 0) return;
    gtd_update(c, lev, lam);
    int nb = (l.h_nrows + 255) / 256;
    k_ghost_update_t<<<nb, 256, 0, c->stream>>>(targs(c, lev), l.gh, l.h_nrows, lam, cc, l.gtd, c->prm.dtau);
    k_apply_upd<<<nb, 256, 0, c->stream>>>(l.gh.node, l.gh.upd, l.h_nrows, lam);
    c->launches += 2;
}

void scalar_update_t(Ctx *c, int lev, double *lam, const double *cc)
{
    const Level &l = c->lv[lev];
    gtd_update(c, lev, lam);
    int nb = nblocks_red(l);
    TArgs A = targs(c, lev);
    k_scalar_t_partial<<<nb, 256, 0, c->stream>>>(A, lam, cc, l.gtd, c->part);
    k_scalar_t_final<<<1, 256, 0, c->stream>>>(c->part, nb, cc, 3 * l.F, A.h2, l.nint, c->red + 5);
    k_scalar_t_apply<<<fgrid(l), 256, 0, c->stream>>>(A, c->red + 5, lam);
    c->launches += 3;
}

void box_sweep_t(Ctx *c, int lev, double *lam, const double *cc)
{
    const Level &l = c->lv[lev];
    cudaStream_t st = c->stream;
    TArgs A = targs(c, lev);
    gtd_update(c, lev, lam);
    if (l.h_nlonely > 0) {
        int nb = (l.h_nlonely + 127) / 128;
        k_lonely_t<<<nb, 128, 0, st>>>(A, l.lonely, l.h_nlonely, lam, cc, l.gtd, c->part);
        k_apply_upd<<<nb, 128, 0, st>>>(l.lonely, c->part, l.h_nlonely, lam);
        c->launches += 2;
    }
    for (int colour = l.cut.ncol - 1; colour >= 0; colour--) {
        int beg = l.h_cutoff[colour], end = l.h_cutoff[colour + 1];
        if (end <= beg) continue;
        k_box_cut_t<<<(end - beg + 15) / 16, 128, 0, st>>>(A, l, lam, cc, beg, end);
        c->launches++;
    }
    gtd_update(c, lev, lam);
    int per_row = (l.N + 4) / 5;
    dim3 g((per_row + 127) / 128, l.N);
    for (int colour = 4; colour >= 0; colour--) {
        k_box_full_t<<<g, 128, 0, st>>>(A, lam, cc, l.gtd, colour);
        c->launches++;
    }
}

void smooth_t(Ctx *c, int lev, double *lam, const double *cc, int nu)
{
    for (int s = 0; s < nu; s++) {
        for (int k = 0; k < c->prm.lambda; k++) ghost_sweep_t(c, lev, lam, cc);
        scalar_update_t(c, lev, lam, cc);
        box_sweep_t(c, lev, lam, cc);
    }
}

// cH = P^T r (r on level lev, cH on lev + 1)
void prolong_t(Ctx *c, int lev, const double *r, double *cH)
{
    const Level &f = c->lv[lev], &C = c->lv[lev + 1];
    k_prolong_t<<<dim3((C.P + 255) / 256, C.N + 2), 256, 0, c->stream>>>(f.N, f.P, f.F, f.pcode, C.N, C.P, C.F, C.tU,
                                                                          C.tV, C.tP, r, cH);
    c->launches++;
}

// lam += R^T yH (lam on level lev, yH on lev + 1)
void restrict_t(Ctx *c, int lev, const double *yH, double *lam)
{
    const Level &f = c->lv[lev], &C = c->lv[lev + 1];
    k_restrict_t<<<fgrid(f), 256, 0, c->stream>>>(f.N, f.P, f.F, f.tU, f.tV, f.tP, C.N, C.P, C.F, C.tU, C.tV, C.tP, yH,
                                                  lam);
    c->launches++;
}

// lam = M_c^-T c on the coarsest level (transpose of the stored inverse)
void coarse_solve_t(Ctx *c, const double *cc, double *lam)
{
    const Level &l = c->lv[c->L - 1];
    cudaStream_t st = c->stream;
    int n = c->nc;
    k_zero_d<<<(unsigned)((l.VL + 255) / 256), 256, 0, st>>>(lam, l.VL);
    k_gather_d<<<(n + 255) / 256, 256, 0, st>>>(cc, c->cmap, c->cvec, n);
    k_gemv_t<<<(n + 31) / 32, dim3(32, 32), 0, st>>>(c->Minv, c->cvec, c->cvec + n, n);
    k_scatter_d<<<(n + 255) / 256, 256, 0, st>>>(c->cvec + n, c->cmap, lam, n);
    c->launches += 4;
}

void cycle_t_rec(Ctx *c, int lev, double *lam, const double *cc)
{
    if (lev == c->L - 1) {
        coarse_solve_t(c, cc, lam);
        return;
    }
    Level &l = c->lv[lev], &C = c->lv[lev + 1];
    smooth_t(c, lev, lam, cc, c->prm.nu2);
    residual_t(c, lev, lam, cc, l.r);
    prolong_t(c, lev, l.r, C.b);
    k_zero_d<<<(unsigned)((C.VL + 255) / 256), 256, 0, c->stream>>>(C.x, C.VL);
    c->launches++;
    for (int k = 0; k < c->prm.gamma; k++) cycle_t_rec(c, lev + 1, C.x, C.b);
    restrict_t(c, lev, C.x, lam);
    smooth_t(c, lev, lam, cc, c->prm.nu1);
}

// the rows of M^T at inactive nodes of the finest level, solved exactly
void fix_inactive_t(Ctx *c, double *lam, const double *cc)
{
    const Level &l = c->lv[0];
    gtd_update(c, 0, lam);
    k_fix_inactive_t<<<fgrid(l), 256, 0, c->stream>>>(targs(c, 0), cc, l.gtd, lam);
    c->launches++;
}

static int read_norm(Ctx *c, double *out)
{
    if (cudaMemcpyAsync(out, c->red + 4, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        snprintf(c->msg, sizeof c->msg, "adjoint solve: %s", cudaGetErrorString(cudaGetLastError()));
        return GP_CUDA;
    }
    return GP_OK;
}

// transposed cycles from lam until ||c - M^T lam||_inf <= tol
// one iteration of the adjoint solve: a transposed cycle, the inactive rows
// fixed, the transposed residual and its norm (replayed as a CUDA graph)
void transposed_iteration(Ctx *c, double *lam, const double *cc)
{
    cycle_t_rec(c, 0, lam, cc);
    fix_inactive_t(c, lam, cc);
    residual_t(c, 0, lam, cc, c->lv[0].r);
}

bool run_graph(Ctx *c, int which, double *x, const double *b);
void krylov_init_t(Ctx *c, double *lam, const double *cc);
void krylov_iteration_t(Ctx *c, double *lam, const double *cc);

// the adjoint solve: plain transposed cycles, or (gp_params.krylov)
// BiCGSTAB preconditioned by one transposed cycle; the same stopping test
// on the transposed residual
int solve_t(Ctx *c, double *lam, const double *cc, double tol, gp_report *rep)
{
    Level &l0 = c->lv[0];
    const bool kry = c->prm.krylov != 0;
    double r0 = 0.0, rn = 0.0;
    if (kry) {
        krylov_init_t(c, lam, cc);
    } else {
        fix_inactive_t(c, lam, cc);
        residual_t(c, 0, lam, cc, l0.r);
    }
    int st = read_norm(c, &r0);
    if (st != GP_OK) return st;
    if (rep) {
        rep->res0 = r0;
        rep->cycles = rep->iterations = 0;
        if (rep->hist_host) rep->hist_host[0] = r0;
    }
    rn = r0;
    int k = 0, status = GP_NOT_CONVERGED;
    if (r0 <= tol) status = GP_OK;
    for (k = 1; status == GP_NOT_CONVERGED && k <= c->prm.max_cycles; k++) {
        if (kry) {
            if (!run_graph(c, GRAPH_KT, lam, cc)) krylov_iteration_t(c, lam, cc);
        } else if (!run_graph(c, GRAPH_T, lam, cc)) {
            transposed_iteration(c, lam, cc);
        }
        st = read_norm(c, &rn);
        if (st != GP_OK) return st;
        if (rep) {
            rep->iterations = k;
            rep->cycles = kry ? 2 * k : k;
            if (rep->hist_host) rep->hist_host[k] = rn;
        }
        if (!(rn == rn) || rn > 1e6 * r0) status = GP_DIVERGED;
        else if (rn <= tol) status = GP_OK;
    }
    if (rep) {
        rep->res = rn;
        rep->rho = rep->cycles > 0 && r0 > 0.0 ? pow(rn / r0, 1.0 / rep->cycles) : 0.0;
        double xi = 0.0;
        cudaMemcpyAsync(&xi, lam + 3 * l0.F, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        rep->xi = xi;
    }
    if (status == GP_DIVERGED) snprintf(c->msg, sizeof c->msg, "adjoint solve diverged (residual %g from %g)", rn, r0);
    else if (status == GP_NOT_CONVERGED)
        snprintf(c->msg, sizeof c->msg, "adjoint solve: residual %g after %d cycles", rn, c->prm.max_cycles);
    return status;
}

}  // namespace gpmg
