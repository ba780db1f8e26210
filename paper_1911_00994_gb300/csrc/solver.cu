// Context, workspace layout, cycle driver and the C ABI (include/gpmg.h).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "gpmg_internal.cuh"
#include <nvtx3/nvToolsExt.h>

namespace gpmg {

int build_geometry_levels(Ctx *c, const double *phi_in, int phi_fluid_positive);
void shape_phi(Ctx *c, const gp_shape &sh, double cx, double cy, double ang);
int build_coarse_inverse(Ctx *c);
void coarse_maps_host(int N, int P, long long F, int *cmap, int *inv, long long vl);
template <typename T> void residual(Ctx *c, int lev, const T *x, const T *b, T *r);
template <typename T> void box_sweep(Ctx *c, int lev, T *x, const T *b);
template <typename T> void scalar_update(Ctx *c, int lev, T *x, const T *b);
template <typename T> void ghost_sweep(Ctx *c, int lev, T *x, const T *b);
template <typename T> void smooth(Ctx *c, int lev, T *x, const T *b, int nu);
template <typename T> void restrict_level(Ctx *c, int lev, const T *r, T *bH, T *xz);
template <typename T> void residual_restrict(Ctx *c, int lev, const T *x, const T *b, T *r, T *bH, T *xz);
template <typename T> void prolong_level(Ctx *c, int lev, const T *eH, T *x);
template <typename T> void prolong_to(Ctx *c, int lev, const T *eH, const T *x, T *y);
template <typename T> void smooth_from(Ctx *c, int lev, T *x, T *in, const T *b, int nu);
template <typename T> T *post_buffer(Ctx *c, int lev, T *x, int nu);
template <typename T> void zero_vec(Ctx *c, T *x, long long n);
template <typename T> void zero_inactive(Ctx *c, int lev, T *x);
template <typename T> void coarse_solve(Ctx *c, const T *b, T *x);
void to_float(Ctx *c, const double *a, float *b, long long n);
void residual_to_float(Ctx *c, const double *x, const double *b, float *r);
void tmr_flush(Ctx *c);
void tiles_init();
void prepare_cuts(Ctx *c);
int recolour_cuts(Ctx *c);
int ghost_row_links(Ctx *c);
void box_codes(Ctx *c);
void transposed_iteration(Ctx *c, double *lam, const double *cc);
void krylov_init(Ctx *c, double *x, const double *b);
void krylov_iteration(Ctx *c, double *x, const double *b);
void krylov_iteration_t(Ctx *c, double *lam, const double *cc);
int residual_static(Ctx *c, int lev, const double *x, const double *b, double *r, double *norm_host);
int levelset_reinit(Ctx *c, double *phi, double *work, int iters, double dtau);
int levelset_advect(Ctx *c, double *phi, double *work, const double *wx, const double *wy, double dt, int steps);
void cn_convective(Ctx *c, const double *x, const double *Nn, double *out, int mode);
void cn_rhs(Ctx *c, const double *xn, const double *Nh, const double *f, double dt, const double *bc, const gp_body &body,
            const gp_walls &walls, double *b);
int cn_momentum_residual(Ctx *c, const double *x, const double *b, double *res, double *bmax);
void cn_extrapolate(Ctx *c, const double *Nn, const double *N1, const double *N2, double *Nh);
void cn_copy(Ctx *c, const double *a, double *b, long long n);
void add_float(Ctx *c, double *x, const float *e, long long n);
int adjoint_prepare(Ctx *c);
void residual_t(Ctx *c, int lev, const double *lam, const double *cc, double *r);
void box_sweep_t(Ctx *c, int lev, double *lam, const double *cc);
void scalar_update_t(Ctx *c, int lev, double *lam, const double *cc);
void ghost_sweep_t(Ctx *c, int lev, double *lam, const double *cc);
void smooth_t(Ctx *c, int lev, double *lam, const double *cc, int nu);
void prolong_t(Ctx *c, int lev, const double *r, double *cH);
void restrict_t(Ctx *c, int lev, const double *yH, double *lam);
void cycle_t_rec(Ctx *c, int lev, double *lam, const double *cc);
void fix_inactive_t(Ctx *c, double *lam, const double *cc);
int solve_t(Ctx *c, double *lam, const double *cc, double tol, gp_report *rep);
void cn_convective_jt(Ctx *c, const double *x, const double *y, double *out);
void cn_explicit_t(Ctx *c, const double *y, double *out);
void cn_mask_mom(Ctx *c, const double *lam, double *el);
void cn_axpy4(Ctx *c, const double *el, double *a0, double c0, double *a1, double c1, double *a2, double c2,
              double *a3, double c3);
void cn_dot_rows(Ctx *c, const double *g, const double *lam, double *out);

// ------------------------------------------------------------- workspace

struct Carver {
    char *base;
    size_t off;
    template <typename T> T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

static int ghost_cap(int N) { return 48 * (N + 2) + 8 * N + 1024; }
static int cut_cap(int N) { return 16 * (N + 2) + 256; }
static int lonely_cap(int N) { return 4 * (N + 2) + 64; }

static int validate(const gp_params *p, char *msg, size_t nmsg)
{
    if (!p || p->N < 4 || p->levels < 1 || p->levels > MAX_LEVELS) {
        snprintf(msg, nmsg, "invalid N or levels");
        return 0;
    }
    if (p->N % (1 << (p->levels - 1)) != 0 || (p->N >> (p->levels - 1)) < 4) {
        snprintf(msg, nmsg, "N must be divisible by 2^(levels-1) with a coarsest grid of at least 4 cells");
        return 0;
    }
    if ((p->N >> (p->levels - 1)) > 64) {
        snprintf(msg, nmsg, "coarsest grid larger than 64 cells per side (dense inverse too large)");
        return 0;
    }
    if (!(p->L > 0.0) || !(p->alpha >= 0.0) || p->nu1 < 0 || p->nu2 < 0 || p->gamma < 1 || p->gamma > 2 ||
        p->lambda < 0 || p->max_cycles < 1 || (p->precision != GP_FP64 && p->precision != GP_MIXED) ||
        p->inner < 0 || p->inner > GP_MAX_INNER) {
        snprintf(msg, nmsg, "invalid solver parameters");
        return 0;
    }
    if ((long long)(2 * p->N + 1) * (2 * p->N + 1) > (1ll << 40) || vec_len(p->N) * 3 > (1ll << 31)) {
        snprintf(msg, nmsg, "grid too large for 32-bit vector indices");
        return 0;
    }
    return 1;
}

// assigns every device array of the context (c may have base == null to size)
static size_t carve(Ctx *c, char *base)
{
    Carver cv{base, 0};
    const gp_params &p = c->prm;
    int L = p.levels;
    long long maxpart = 0;
    for (int k = 0; k < L; k++) {
        Level &l = c->lv[k];
        l.N = p.N >> k;
        l.P = frame_pitch(l.N);
        l.F = frame_size(l.N);
        l.VL = vec_len(l.N);
        l.h = p.L / (double)l.N;
        l.tU = cv.take<uint8_t>(l.F);
        l.tV = cv.take<uint8_t>(l.F);
        l.tP = cv.take<uint8_t>(l.F);
        l.bcode = cv.take<uint8_t>(l.F);
        l.pcode = k + 1 < L ? cv.take<uint8_t>(3 * l.F) : nullptr;
        l.prim = cv.take<uint8_t>(3 * l.F);
        l.done = cv.take<uint8_t>(3 * l.F);
        l.r = cv.take<double>(l.VL);
        if (k > 0) {
            l.x = cv.take<double>(l.VL);
            l.b = cv.take<double>(l.VL);
        } else {
            l.x = l.b = nullptr;
        }
        if (p.precision == GP_MIXED) {
            l.xf = cv.take<float>(l.VL);
            l.bf = cv.take<float>(l.VL);
            l.rf = cv.take<float>(l.VL);
        } else {
            l.xf = l.bf = l.rf = nullptr;
        }
        int gc = ghost_cap(l.N);
        GhostList &g = l.gh;
        g.cap = gc;
        g.count = cv.take<int>(2);
        g.node = cv.take<int>(gc);
        g.kind = cv.take<uint8_t>(gc);
        g.nst = cv.take<uint8_t>(gc);
        g.st = cv.take<int>((size_t)GH_ST * gc);
        g.w = cv.take<double>((size_t)GH_ST * gc);
        g.wf = cv.take<float>((size_t)GH_ST * gc);
        g.B = cv.take<double>(2 * (size_t)gc);
        g.th = cv.take<double>(2 * (size_t)gc);
        g.upd = cv.take<double>(gc);
        g.updf = cv.take<float>(gc);
        g.acc = cv.take<double>(2 * (size_t)gc);
        g.accf = cv.take<float>(2 * (size_t)gc);
        g.strow = cv.take<int>((size_t)GH_ST * gc);
        const size_t ncl = (size_t)gc / GC_OWN + 1;
        g.cl_row = cv.take<int>(ncl * GC_CAP);
        g.cl_lnk = cv.take<int16_t>(ncl * GH_ST * GC_CAP);
        g.cl_n = cv.take<int>(ncl);
        int cc = cut_cap(l.N);
        l.cut.cap = cc;
        l.cut.count = cv.take<int>(1);
        l.cut.off = cv.take<int>(MAX_CUTCOL + 1);
        l.cut.cell = cv.take<int>(cc);
        l.cut.gface = cv.take<int>(4 * (size_t)cc);
        l.cut.row = cv.take<int>(5 * (size_t)cc);
        l.cut.sidx = cv.take<int>(5 * CUT_ST * (size_t)cc);
        l.cut.scoef = cv.take<double>(5 * CUT_ST * (size_t)cc);
        l.cut.scoeff = cv.take<float>(5 * CUT_ST * (size_t)cc);
        l.cut.minv = cv.take<double>(25 * (size_t)cc);
        l.cut.minvf = cv.take<float>(25 * (size_t)cc);
        l.lonely_cap = lonely_cap(l.N);
        l.lonely = cv.take<int>(l.lonely_cap);
        l.nlonely = cv.take<int>(1);
        l.nint = cv.take<int>(1);
        if (p.adjoint) {
            l.tl_cap = GH_ST * gc;
            l.tl_node = cv.take<int>(l.tl_cap);
            l.tl_ptr = cv.take<int>(l.tl_cap + 1);
            l.tl_src = cv.take<int>(l.tl_cap);
            l.tl_w = cv.take<double>(l.tl_cap);
            l.gtd = cv.take<double>(l.VL);
            l.cut_tl = cv.take<int>(5 * (size_t)cc);
        } else {
            l.tl_cap = 0;
            l.tl_node = l.tl_ptr = l.tl_src = l.cut_tl = nullptr;
            l.tl_w = l.gtd = nullptr;
        }
        l.h_tl_n = 0;
        long long nb = (long long)((l.P + 255) / 256) * (l.N + 2);
        long long need = 2 * nb + 3 * (l.N + 2) + 64 + 2 * l.lonely_cap;
        if (need > maxpart) maxpart = need;
    }
    c->phi = cv.take<double>((size_t)(2 * p.N + 1) * (2 * p.N + 1));
    if (p.cn_buffers) {
        c->cn_xn = cv.take<double>(c->lv[0].VL);
        c->cn_Nn = cv.take<double>(c->lv[0].VL);
        c->cn_Nh = cv.take<double>(c->lv[0].VL);
        c->cn_b = cv.take<double>(c->lv[0].VL);
    } else {
        c->cn_xn = c->cn_Nn = c->cn_Nh = c->cn_b = nullptr;
    }
    c->npart = (int)maxpart;
    c->part = cv.take<double>(maxpart);
    c->red = cv.take<double>(32);
    c->maxbits = cv.take<unsigned long long>(4);
    c->err = cv.take<unsigned>(4);
    c->flag = cv.take<int>(4);
    for (int k = 0; k < 10; k++) c->kv[k] = p.krylov ? cv.take<double>(c->lv[0].VL) : nullptr;
    for (int k = 0; k < 12; k++)
        c->adjv[k] = (p.adjoint && p.cn_buffers && k < 4 + ADJ_KMAX - 1) ? cv.take<double>(c->lv[0].VL) : nullptr;
    c->ks = cv.take<double>(8);
    c->kpart = cv.take<double>(2 * 1024);
    const Level &lc = c->lv[L - 1];
    int nc = 2 * (lc.N + 1) * (lc.N + 2) + lc.N * lc.N + 1;
    c->nc = nc;
    c->Minv = cv.take<double>((size_t)nc * nc);
    c->Minvf = cv.take<float>((size_t)nc * nc);
    c->aug = cv.take<double>((size_t)nc * 2 * nc);
    c->gjkeys = cv.take<unsigned long long>((size_t)nc);
    c->gjused = cv.take<uint8_t>((size_t)nc);
    c->cmap = cv.take<int>((size_t)nc + lc.VL);
    c->cvec = cv.take<double>(2 * (size_t)nc + 8);
    c->cvecf = cv.take<float>(2 * (size_t)nc + 8);
    return cv.off + 256;
}

// ------------------------------------------------------------------ cycle

template <typename T> struct Vecs {
    static T *x(Ctx *c, int l);
    static T *b(Ctx *c, int l);
    static T *r(Ctx *c, int l);
};
template <> double *Vecs<double>::x(Ctx *c, int l) { return c->lv[l].x; }
template <> double *Vecs<double>::b(Ctx *c, int l) { return c->lv[l].b; }
template <> double *Vecs<double>::r(Ctx *c, int l) { return c->lv[l].r; }
template <> float *Vecs<float>::x(Ctx *c, int l) { return c->lv[l].xf; }
template <> float *Vecs<float>::b(Ctx *c, int l) { return c->lv[l].bf; }
template <> float *Vecs<float>::r(Ctx *c, int l) { return c->lv[l].rf; }

template <typename T> void cycle_rec(Ctx *c, int lev, T *x, const T *b)
{
    if (lev == c->L - 1) {
        coarse_solve<T>(c, b, x);
        return;
    }
    smooth<T>(c, lev, x, b, c->prm.nu1);
    T *r = Vecs<T>::r(c, lev);
    T *xH = Vecs<T>::x(c, lev + 1), *bH = Vecs<T>::b(c, lev + 1);
    if (c->prm.fuse_restrict > 0) {
        residual_restrict<T>(c, lev, x, b, r, bH, xH);  // also zeroes xH
    } else {
        residual<T>(c, lev, x, b, r);
        restrict_level<T>(c, lev, r, bH, xH);  // also zeroes xH
    }
    for (int k = 0; k < c->prm.gamma; k++) cycle_rec<T>(c, lev + 1, xH, bH);
    T *y = post_buffer<T>(c, lev, x, c->prm.nu2);
    prolong_to<T>(c, lev, xH, x, y);
    smooth_from<T>(c, lev, x, y, b, c->prm.nu2);
}

// one mg_solve iteration: the cycle and the finest FP64 residual (which = 0),
// or FP32 cycle on the FP64 residual and the FP64 update (which = 1)
static void solve_iteration(Ctx *c, int which, double *x, const double *b)
{
    Level &l0 = c->lv[0];
    if (which == GRAPH_T) {
        transposed_iteration(c, x, b);
        return;
    }
    if (which == GRAPH_KT) {
        krylov_iteration_t(c, x, b);
        return;
    }
    if (which >= 2) {
        krylov_iteration(c, x, b);
        return;
    }
    if (which == 1) {
        // bf holds the FP64 residual of x rounded to FP32 (written by the
        // previous residual); c->inner_now FP32 cycles on the correction
        zero_vec<float>(c, l0.xf, l0.VL);
        for (int k = 0; k < c->inner_now; k++) cycle_rec<float>(c, 0, l0.xf, l0.bf);
        add_float(c, x, l0.xf, l0.VL);
        residual_to_float(c, x, b, l0.bf);
    } else {
        cycle_rec<double>(c, 0, x, b);
        residual<double>(c, 0, x, b, l0.r);
    }
}

void graphs_reset(Ctx *c)
{
    for (int w = 0; w < NGRAPH; w++)
        if (c->gvalid[w]) {
            cudaGraphExecDestroy(c->gexec[w]);
            c->gvalid[w] = 0;
        }
}

// replay (capturing first if needed) one iteration as a CUDA graph; false
// when graphs are unavailable here (then the caller launches directly)
bool run_graph(Ctx *c, int which0, double *x, const double *b)
{
    // slot: the iteration kind, and for the FP32 corrections their cycle count
    const int which = (which0 == 1 && c->inner_now > 1) ? 4 + c->inner_now - 2 : which0;
    if (!c->prm.graphs || c->graphs_off || c->stream == nullptr || c->tmr_kernel >= 0) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;  // the caller is capturing: launch directly into its capture
    }
    if (!c->gvalid[which] || c->gx[which] != x || c->gb[which] != b) {
        if (c->gvalid[which]) {
            cudaGraphExecDestroy(c->gexec[which]);
            c->gvalid[which] = 0;
        }
        long long l0 = c->launches;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c->graphs_off = 1;
            return false;
        }
        solve_iteration(c, which0, x, b);
        long long per = c->launches - l0;  // kernels of one iteration
        c->launches = l0;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec[which], g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->graphs_off = 1;
            return false;
        }
        c->glaunches[which] = per;
        c->gx[which] = x;
        c->gb[which] = b;
        c->gvalid[which] = 1;
    }
    if (cudaGraphLaunch(c->gexec[which], c->stream) != cudaSuccess) {
        cudaGetLastError();
        graphs_reset(c);
        c->graphs_off = 1;
        return false;
    }
    c->launches += c->glaunches[which];
    return true;
}

}  // namespace gpmg

using namespace gpmg;

struct gp_ctx {
    Ctx c;
};

// an NVTX range around each entry point (and each solver iteration), for
// profilers' timelines; no effect without a profiler attached
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

static gp_status fail(gp_ctx *ctx, gp_status s, const char *m)
{
    if (ctx) snprintf(ctx->c.msg, sizeof ctx->c.msg, "%s", m);
    return s;
}

static gp_status check_cuda(gp_ctx *ctx, const char *where)
{
    cudaError_t e = cudaPeekAtLastError();
    if (e == cudaSuccess) return GP_OK;
    cudaGetLastError();
    snprintf(ctx->c.msg, sizeof ctx->c.msg, "%s: %s", where, cudaGetErrorString(e));
    return GP_CUDA;
}

static gp_status ensure_coarse(gp_ctx *ctx)
{
    Ctx *c = &ctx->c;
    if (!c->geom_ok) return fail(ctx, GP_INVALID, "geometry_build has not succeeded");
    if (c->coarse_ok && c->alpha_factored == c->prm.alpha) return GP_OK;
    graphs_reset(c);  // the captured launches carry alpha in their arguments
    prepare_cuts(c);  // cut-box rows and inverses depend on alpha
    return (gp_status)build_coarse_inverse(c);
}

static bool level_ok(gp_ctx *ctx, int level) { return ctx && level >= 0 && level < ctx->c.L; }

// why a solve diverged, when the bounded wait of a tile copy ran out
static const char *wait_note(Ctx *c)
{
    unsigned e[4] = {0, 0, 0, 0};
    cudaMemcpyAsync(e, c->err, sizeof e, cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return "";
    return e[2] ? " (a tile copy wait ran out)" : "";
}

extern "C" {

gp_status gp_params_default(gp_params *prm, int N, double x0, double y0, double L)
{
    if (!prm || N < 4 || !(L > 0.0)) return GP_INVALID;
    memset(prm, 0, sizeof *prm);
    prm->N = N;
    prm->x0 = x0;
    prm->y0 = y0;
    prm->L = L;
    int lev = 1;
    while ((N >> lev) >= 16 && (N >> (lev - 1)) > 16 && (N % (1 << lev)) == 0) lev++;
    prm->levels = lev;
    prm->alpha = L / N / 2.0;
    prm->nu1 = 2;
    prm->nu2 = 1;
    prm->gamma = 1;
    prm->lambda = 5;
    prm->dtau = 0.9;
    prm->snap = 0.3;
    prm->precision = GP_FP64;
    prm->max_cycles = 100;
    prm->cn_buffers = 1;
    prm->graphs = 1;
    return GP_OK;
}

int gp_pitch(int N) { return frame_pitch(N); }
int64_t gp_vector_length(int N) { return vec_len(N); }

gp_status gp_workspace_size(const gp_params *prm, size_t *bytes)
{
    char msg[256];
    if (!bytes || !validate(prm, msg, sizeof msg)) return GP_INVALID;
    Ctx *c = new (std::nothrow) Ctx();
    if (!c) return GP_INVALID;
    c->prm = *prm;
    c->L = prm->levels;
    *bytes = carve(c, nullptr);
    delete c;
    return GP_OK;
}

gp_status gp_create(gp_ctx **out, const gp_params *prm, void *workspace, size_t bytes, void *stream)
{
    if (!out) return GP_INVALID;
    *out = nullptr;
    gp_ctx *ctx = new (std::nothrow) gp_ctx();
    if (!ctx) return GP_INVALID;
    Ctx *c = &ctx->c;
    if (!validate(prm, c->msg, sizeof c->msg)) {
        delete ctx;
        return GP_INVALID;
    }
    c->prm = *prm;
    c->L = prm->levels;
    size_t need = carve(c, nullptr);
    if (!workspace || bytes < need || ((uintptr_t)workspace & 255)) {
        delete ctx;
        return GP_INVALID;
    }
    c->ws = (char *)workspace;
    c->ws_bytes = bytes;
    c->tmr_kernel = -1;
    tiles_init();
    c->stream = (cudaStream_t)stream;
    carve(c, c->ws);
    // coarsest-level index maps (host -> device)
    const Level &lc = c->lv[c->L - 1];
    std::vector<int> maps((size_t)c->nc + lc.VL);
    coarse_maps_host(lc.N, lc.P, lc.F, maps.data(), maps.data() + c->nc, lc.VL);
    cudaError_t e = cudaMemcpyAsync(c->cmap, maps.data(), maps.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->maxbits, 0, 4 * sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, 4 * sizeof(unsigned), c->stream);
    for (int k = 0; k < c->L && e == cudaSuccess; k++) {
        Level &l = c->lv[k];
        e = cudaMemsetAsync(l.r, 0, l.VL * sizeof(double), c->stream);
        if (e == cudaSuccess && l.x) e = cudaMemsetAsync(l.x, 0, l.VL * sizeof(double), c->stream);
        if (e == cudaSuccess && l.b) e = cudaMemsetAsync(l.b, 0, l.VL * sizeof(double), c->stream);
        if (e == cudaSuccess && l.xf) {
            cudaMemsetAsync(l.xf, 0, l.VL * sizeof(float), c->stream);
            cudaMemsetAsync(l.bf, 0, l.VL * sizeof(float), c->stream);
            e = cudaMemsetAsync(l.rf, 0, l.VL * sizeof(float), c->stream);
        }
    }
    for (int k = 0; k < 10 && e == cudaSuccess; k++)
        if (c->kv[k]) e = cudaMemsetAsync(c->kv[k], 0, c->lv[0].VL * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        delete ctx;
        return GP_CUDA;
    }
    *out = ctx;
    return GP_OK;
}

gp_status gp_destroy(gp_ctx *ctx)
{
    if (!ctx) return GP_INVALID;
    cudaStreamSynchronize(ctx->c.stream);
    if (ctx->c.tmr_ready)
        for (int k = 0; k < 2 * 512; k++) cudaEventDestroy(ctx->c.tmr_ev[k]);
    graphs_reset(&ctx->c);
    if (ctx->c.gj_exec) cudaGraphExecDestroy(ctx->c.gj_exec);
    delete ctx;
    return GP_OK;
}

int64_t gp_launch_count(const gp_ctx *ctx) { return ctx ? ctx->c.launches : -1; }

gp_status gp_timer_start(gp_ctx *ctx, int kernel, int level)
{
    if (!ctx || kernel < 0 || kernel > KT_COARSE || level < 0 || level >= ctx->c.L) return GP_INVALID;
    Ctx *c = &ctx->c;
    if (!c->tmr_ready) {
        for (int k = 0; k < 2 * 512; k++)
            if (cudaEventCreate(&c->tmr_ev[k]) != cudaSuccess) return check_cuda(ctx, "gp_timer_start");
        c->tmr_ready = 1;
    }
    tmr_flush(c);
    c->tmr_kernel = kernel;
    c->tmr_level = level;
    c->tmr_ms = 0.0;
    c->tmr_launches = 0;
    return GP_OK;
}

gp_status gp_timer_stop(gp_ctx *ctx, int64_t *launches, double *total_ms)
{
    if (!ctx) return GP_INVALID;
    Ctx *c = &ctx->c;
    tmr_flush(c);
    if (launches) *launches = c->tmr_launches;
    if (total_ms) *total_ms = c->tmr_ms;
    c->tmr_kernel = -1;
    return check_cuda(ctx, "gp_timer_stop");
}

const char *gp_last_error(const gp_ctx *ctx) { return ctx ? ctx->c.msg : "null context"; }

gp_status gp_set_alpha(gp_ctx *ctx, double alpha)
{
    if (!ctx || !(alpha >= 0.0)) return GP_INVALID;
    ctx->c.prm.alpha = alpha;
    return GP_OK;
}

static gp_status geometry_finish(gp_ctx *ctx, const double *phi, int phi_fluid_positive);

gp_status geometry_build(gp_ctx *ctx, const double *phi, int phi_fluid_positive)
{
    Range nvtx_range("geometry_build");
    if (!ctx || !phi) return GP_INVALID;
    return geometry_finish(ctx, phi, phi_fluid_positive);
}

gp_status geometry_build_shape(gp_ctx *ctx, const gp_shape *shape, double t, gp_body *body_out)
{
    Range nvtx_range("geometry_build_shape");
    if (!ctx || !shape || shape->kind < GP_CIRCLE || shape->kind > GP_FLOWER) return GP_INVALID;
    if (shape->orbit_r != 0.0 && !(shape->orbit_period > 0.0)) return GP_INVALID;
    const double two_pi = 6.283185307179586;
    double w = shape->orbit_r != 0.0 ? two_pi / shape->orbit_period : 0.0;
    double ph = w * t + shape->orbit_phase;
    double cx = shape->xc + shape->orbit_r * cos(ph), cy = shape->yc + shape->orbit_r * sin(ph);
    shape_phi(&ctx->c, *shape, cx, cy, shape->omega * t);
    if (body_out) {
        body_out->U = -shape->orbit_r * w * sin(ph);
        body_out->V = shape->orbit_r * w * cos(ph);
        body_out->omega = shape->omega;
        body_out->cx = cx;
        body_out->cy = cy;
    }
    return geometry_finish(ctx, nullptr, 0);
}

static gp_status geometry_finish(gp_ctx *ctx, const double *phi, int phi_fluid_positive)
{
    Ctx *c = &ctx->c;
    c->geom_ok = 0;
    c->coarse_ok = 0;
    c->adj_ok = 0;
    c->msg[0] = 0;
    graphs_reset(c);
    int s = build_geometry_levels(c, phi, phi_fluid_positive);
    if (s != GP_OK) return (gp_status)s;
    gp_status cs = check_cuda(ctx, "geometry_build");
    if (cs != GP_OK) return cs;
    c->geom_ok = 1;
    box_codes(c);
    prepare_cuts(c);
    s = recolour_cuts(c);
    if (s == GP_OK) s = ghost_row_links(c);
    if (s != GP_OK) {
        c->geom_ok = 0;
        return (gp_status)s;
    }
    prepare_cuts(c);
    s = build_coarse_inverse(c);
    if (s != GP_OK) {
        c->geom_ok = 0;
        return (gp_status)s;
    }
    return check_cuda(ctx, "coarse inverse");
}

gp_status gp_level_set(gp_ctx *ctx, double *phi_out)
{
    if (!ctx || !phi_out) return GP_INVALID;
    Ctx *c = &ctx->c;
    size_t n = (size_t)(2 * c->prm.N + 1) * (2 * c->prm.N + 1);
    cudaMemcpyAsync(phi_out, c->phi, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    return check_cuda(ctx, "gp_level_set");
}

gp_status gp_level_info(const gp_ctx *ctx, int level, int *N, int64_t *len, double *h)
{
    if (!ctx || level < 0 || level >= ctx->c.L) return GP_INVALID;
    const Level &l = ctx->c.lv[level];
    if (N) *N = l.N;
    if (len) *len = l.VL;
    if (h) *h = l.h;
    return GP_OK;
}

gp_status gp_types(gp_ctx *ctx, int level, uint8_t *tu, uint8_t *tv, uint8_t *tp)
{
    if (!level_ok(ctx, level) || !ctx->c.geom_ok) return GP_INVALID;
    Ctx *c = &ctx->c;
    const Level &l = c->lv[level];
    cudaMemcpyAsync(tu, l.tU, l.F, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tv, l.tV, l.F, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tp, l.tP, l.F, cudaMemcpyDeviceToDevice, c->stream);
    return check_cuda(ctx, "gp_types");
}

gp_status gp_ghost_count(gp_ctx *ctx, int level, int *n_object, int *n_rows)
{
    if (!level_ok(ctx, level) || !ctx->c.geom_ok) return GP_INVALID;
    if (n_object) *n_object = ctx->c.lv[level].h_nghost;
    if (n_rows) *n_rows = ctx->c.lv[level].h_nrows;
    return GP_OK;
}

gp_status gp_ghost_rows(gp_ctx *ctx, int level, int *node, uint8_t *kind, uint8_t *nst, int *st, double *w, double *B,
                        double *th)
{
    if (!level_ok(ctx, level) || !ctx->c.geom_ok) return GP_INVALID;
    Ctx *c = &ctx->c;
    const Level &l = c->lv[level];
    int n = l.h_nghost;
    if (n == 0) return GP_OK;
    cudaStream_t s = c->stream;
    if (node) cudaMemcpyAsync(node, l.gh.node, n * sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (kind) cudaMemcpyAsync(kind, l.gh.kind, n, cudaMemcpyDeviceToDevice, s);
    if (nst) cudaMemcpyAsync(nst, l.gh.nst, n, cudaMemcpyDeviceToDevice, s);
    // stencils and weights: [m][cap] -> row-major [k][m]
    for (int m = 0; m < GH_ST; m++) {
        if (st) cudaMemcpy2DAsync(st + m, GH_ST * sizeof(int), l.gh.st + (size_t)m * l.gh.cap, sizeof(int), sizeof(int), n,
                                  cudaMemcpyDeviceToDevice, s);
        if (w) cudaMemcpy2DAsync(w + m, GH_ST * sizeof(double), l.gh.w + (size_t)m * l.gh.cap, sizeof(double),
                                 sizeof(double), n, cudaMemcpyDeviceToDevice, s);
    }
    for (int m = 0; m < 2; m++) {
        if (B) cudaMemcpy2DAsync(B + m, 2 * sizeof(double), l.gh.B + (size_t)m * l.gh.cap, sizeof(double), sizeof(double), n,
                                 cudaMemcpyDeviceToDevice, s);
        if (th) cudaMemcpy2DAsync(th + m, 2 * sizeof(double), l.gh.th + (size_t)m * l.gh.cap, sizeof(double),
                                  sizeof(double), n, cudaMemcpyDeviceToDevice, s);
    }
    return check_cuda(ctx, "gp_ghost_rows");
}

gp_status gp_residual(gp_ctx *ctx, int level, const double *x, const double *b, double *r, double *norm_host)
{
    if (!level_ok(ctx, level) || !ctx->c.geom_ok || !x || !b || !r) return GP_INVALID;
    Ctx *c = &ctx->c;
    residual<double>(c, level, x, b, r);
    if (norm_host) {
        cudaMemcpyAsync(norm_host, c->red, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(ctx, "gp_residual");
    }
    return check_cuda(ctx, "gp_residual");
}

gp_status gp_levelset_reinit(gp_ctx *ctx, double *phi, double *work, int iters, double dtau)
{
    if (!ctx || !phi || !work || iters < 0 || !(dtau > 0.0)) return GP_INVALID;
    return (gp_status)levelset_reinit(&ctx->c, phi, work, iters, dtau);
}

gp_status gp_levelset_advect(gp_ctx *ctx, double *phi, double *work, const double *wx, const double *wy, double dt,
                             int steps)
{
    if (!ctx || !phi || !work || !wx || !wy || steps < 0 || !(dt > 0.0)) return GP_INVALID;
    return (gp_status)levelset_advect(&ctx->c, phi, work, wx, wy, dt, steps);
}

gp_status gp_residual_static(gp_ctx *ctx, int level, const double *x, const double *b, double *r, double *norm_host)
{
    if (!level_ok(ctx, level) || !ctx->c.geom_ok || !x || !b || !r) return GP_INVALID;
    return (gp_status)residual_static(&ctx->c, level, x, b, r, norm_host);
}

gp_status gp_box_sweep(gp_ctx *ctx, int level, double *x, const double *b)
{
    if (!level_ok(ctx, level) || !ctx->c.geom_ok || !x || !b) return GP_INVALID;
    gp_status es = ensure_coarse(ctx);
    if (es != GP_OK) return es;
    box_sweep<double>(&ctx->c, level, x, b);
    return check_cuda(ctx, "gp_box_sweep");
}

gp_status gp_scalar_update(gp_ctx *ctx, int level, double *x, const double *b)
{
    if (!level_ok(ctx, level) || !ctx->c.geom_ok || !x || !b) return GP_INVALID;
    scalar_update<double>(&ctx->c, level, x, b);
    return check_cuda(ctx, "gp_scalar_update");
}

gp_status gp_ghost_sweep(gp_ctx *ctx, int level, double *x, const double *b)
{
    if (!level_ok(ctx, level) || !ctx->c.geom_ok || !x || !b) return GP_INVALID;
    ghost_sweep<double>(&ctx->c, level, x, b);
    return check_cuda(ctx, "gp_ghost_sweep");
}

gp_status gp_smooth(gp_ctx *ctx, int level, double *x, const double *b, int nu)
{
    if (!level_ok(ctx, level) || !ctx->c.geom_ok || !x || !b || nu < 0) return GP_INVALID;
    gp_status es = ensure_coarse(ctx);
    if (es != GP_OK) return es;
    smooth<double>(&ctx->c, level, x, b, nu);
    return check_cuda(ctx, "gp_smooth");
}

gp_status gp_restrict(gp_ctx *ctx, int level, const double *r_fine, double *b_coarse)
{
    if (!ctx || level < 0 || level + 1 >= ctx->c.L || !ctx->c.geom_ok || !r_fine || !b_coarse) return GP_INVALID;
    restrict_level<double>(&ctx->c, level, r_fine, b_coarse, nullptr);
    return check_cuda(ctx, "gp_restrict");
}

gp_status gp_prolong(gp_ctx *ctx, int level, const double *e_coarse, double *x_fine)
{
    if (!ctx || level < 0 || level + 1 >= ctx->c.L || !ctx->c.geom_ok || !e_coarse || !x_fine) return GP_INVALID;
    prolong_level<double>(&ctx->c, level, e_coarse, x_fine);
    return check_cuda(ctx, "gp_prolong");
}

gp_status gp_coarse_solve(gp_ctx *ctx, const double *b, double *x)
{
    if (!ctx || !b || !x) return GP_INVALID;
    gp_status s = ensure_coarse(ctx);
    if (s != GP_OK) return s;
    coarse_solve<double>(&ctx->c, b, x);
    return check_cuda(ctx, "gp_coarse_solve");
}

gp_status gp_cycle(gp_ctx *ctx, double *x, const double *b)
{
    if (!ctx || !x || !b) return GP_INVALID;
    gp_status s = ensure_coarse(ctx);
    if (s != GP_OK) return s;
    cycle_rec<double>(&ctx->c, 0, x, b);
    return check_cuda(ctx, "gp_cycle");
}

gp_status mg_solve(gp_ctx *ctx, double *x, const double *b, double tol, gp_report *rep)
{
    Range nvtx_range("mg_solve");
    if (!ctx || !x || !b || !(tol >= 0.0)) return GP_INVALID;
    gp_status s = ensure_coarse(ctx);
    if (s != GP_OK) return s;
    Ctx *c = &ctx->c;
    Level &l0 = c->lv[0];
    bool mixed = c->prm.precision == GP_MIXED;
    bool kry = c->prm.krylov != 0;
    zero_inactive<double>(c, 0, x);
    if (kry) krylov_init(c, x, b);
    if (mixed && !kry) residual_to_float(c, x, b, l0.bf);
    else residual<double>(c, 0, x, b, l0.r);
    double nrm = 0.0;
    cudaMemcpyAsync(&nrm, c->red, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(ctx, "mg_solve");
    double r0 = nrm;
    if (rep) {
        rep->res0 = r0;
        rep->cycles = 0;
        rep->iterations = 0;
        if (rep->hist_host) rep->hist_host[0] = r0;
    }
    gp_status st = GP_NOT_CONVERGED;
    int k = 0, cycles = 0;
    // FP32 corrections: the first takes one cycle; each later one as many
    // as the reduction per cycle of the previous correction (taken 10%
    // faster, so that a correction rarely overshoots tol) predicts are still
    // needed, at most `inner`
    const bool multi = mixed && !kry;
    const int inner_max = c->prm.inner > 0 ? c->prm.inner : GP_MAX_INNER;
    double prev = r0;
    c->inner_now = 1;
    if (!(r0 == r0)) st = GP_DIVERGED;
    else if (r0 <= tol) st = GP_OK;
    else
        // max_cycles caps the cycles of the FP32 corrections and the
        // iterations otherwise (a BiCGSTAB iteration applies two cycles)
        for (k = 1; multi ? cycles < c->prm.max_cycles : k <= c->prm.max_cycles; k++) {
            int which = (kry ? 2 : 0) + (mixed ? 1 : 0);
            if (multi) c->inner_now = std::min(c->inner_now, c->prm.max_cycles - cycles);
            Range iter_range("mg_solve iteration");
            if (!run_graph(c, which, x, b)) solve_iteration(c, which, x, b);
            const int done = kry ? 2 : multi ? c->inner_now : 1;
            cycles += done;
            cudaMemcpyAsync(&nrm, c->red, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
            if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(ctx, "mg_solve");
            if (rep && rep->hist_host) rep->hist_host[k] = nrm;
            if (!(nrm == nrm) || nrm > 1e6 * r0) {
                st = GP_DIVERGED;
                break;
            }
            if (nrm <= tol) {
                st = GP_OK;
                break;
            }
            if (multi) {
                const double rate = 0.9 * pow(nrm / prev, 1.0 / done);
                int want = 1;
                if (!(tol > 0.0)) want = inner_max;
                else if (rate > 0.0 && rate < 1.0) want = (int)std::min(ceil(log(tol / nrm) / log(rate)), (double)inner_max);
                c->inner_now = std::max(1, std::min(inner_max, want));
                prev = nrm;
            }
        }
    if (st == GP_NOT_CONVERGED) k--;  // the loop ran out: k is one past the last iteration
    c->inner_now = 1;
    if (rep) {
        rep->iterations = k;
        rep->cycles = cycles;
        rep->res = nrm;
        rep->rho = (cycles > 0 && r0 > 0 && nrm > 0) ? pow(nrm / r0, 1.0 / cycles) : 0.0;
        double xi = 0.0;
        cudaMemcpyAsync(&xi, x + 3 * l0.F, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        rep->xi = xi;
    }
    if (st == GP_NOT_CONVERGED) snprintf(c->msg, sizeof c->msg, "not converged: %.3e after %d cycles", nrm, k);
    if (st == GP_DIVERGED) snprintf(c->msg, sizeof c->msg, "diverged: %.3e (initial %.3e)%s", nrm, r0, wait_note(c));
    gp_status cs = check_cuda(ctx, "mg_solve");
    return cs != GP_OK ? cs : st;
}

gp_status gp_convective(gp_ctx *ctx, const double *x, double *out)
{
    if (!ctx || !ctx->c.geom_ok || !x || !out) return GP_INVALID;
    cn_convective(&ctx->c, x, nullptr, out, 0);
    return check_cuda(ctx, "gp_convective");
}

gp_status gp_set_continuity_source(gp_ctx *ctx, const double *g)
{
    if (!ctx) return GP_INVALID;
    ctx->c.csrc = g;
    return GP_OK;
}

gp_status gp_cn_rhs(gp_ctx *ctx, const double *xn, const double *Nh, const double *f, double dt, const double *bc,
                    const gp_body *body, const gp_walls *walls, double *b)
{
    if (!ctx || !ctx->c.geom_ok || !xn || !Nh || !b) return GP_INVALID;
    gp_body bd = body ? *body : gp_body{0, 0, 0, 0, 0};
    gp_walls wl = walls ? *walls : gp_walls{0, 0, 0, 0};
    cn_rhs(&ctx->c, xn, Nh, f, dt, bc, bd, wl, b);
    return check_cuda(ctx, "gp_cn_rhs");
}

gp_status cn_step(gp_ctx *ctx, double *x, double *N1, double *N2, int step, const double *f, const double *bc,
                  double dt, double Re, const gp_body *body, const gp_walls *walls, double tol, double eps, int kmax,
                  gp_cn_report *rep)
{
    Range nvtx_range("cn_step");
    if (!ctx || !x || !N1 || !N2 || step < 0 || !(dt > 0.0) || !(Re > 0.0) || !(tol >= 0.0) || kmax < 1)
        return GP_INVALID;
    Ctx *c = &ctx->c;
    if (!c->cn_xn) return fail(ctx, GP_INVALID, "cn_step needs cn_buffers in gp_params");
    if (!c->geom_ok) return fail(ctx, GP_INVALID, "geometry_build has not succeeded");
    c->prm.alpha = dt / (2.0 * Re);
    gp_body bd = body ? *body : gp_body{0, 0, 0, 0, 0};
    gp_walls wl = walls ? *walls : gp_walls{0, 0, 0, 0};
    const Level &l0 = c->lv[0];
    long long VL = l0.VL;
    cn_copy(c, x, c->cn_xn, VL);
    cn_convective(c, c->cn_xn, nullptr, c->cn_Nn, 0);
    gp_report r;
    memset(&r, 0, sizeof r);
    int cycles = 0, picard = 0;
    double mom = 0.0;
    gp_status st = GP_OK;
    if (step >= 2) {
        cn_extrapolate(c, c->cn_Nn, N1, N2, c->cn_Nh);
        cn_rhs(c, c->cn_xn, c->cn_Nh, f, dt, bc, bd, wl, c->cn_b);
        st = mg_solve(ctx, x, c->cn_b, tol, &r);
        cycles = r.cycles;
    } else {
        // ||f~|| with f~ = u^n + alpha lap u^n + dt f (Eq. iterativeNS)
        double dummy = 0.0, fmax = 0.0;
        cudaMemsetAsync(c->cn_Nh, 0, VL * sizeof(double), c->stream);
        cn_rhs(c, c->cn_xn, c->cn_Nh, f, dt, bc, bd, wl, c->cn_b);
        if (cn_momentum_residual(c, c->cn_xn, c->cn_b, &dummy, &fmax) != GP_OK) return check_cuda(ctx, "cn_step");
        cn_copy(c, c->cn_Nn, c->cn_Nh, VL);  // u^(n+1,0) = u^n
        for (picard = 1; picard <= kmax; picard++) {
            cn_rhs(c, c->cn_xn, c->cn_Nh, f, dt, bc, bd, wl, c->cn_b);
            st = mg_solve(ctx, x, c->cn_b, tol, &r);
            cycles += r.cycles;
            if (st != GP_OK) break;
            cn_convective(c, x, c->cn_Nn, c->cn_Nh, 1);
            cn_rhs(c, c->cn_xn, c->cn_Nh, f, dt, bc, bd, wl, c->cn_b);
            double bm = 0.0;
            if (cn_momentum_residual(c, x, c->cn_b, &mom, &bm) != GP_OK) return check_cuda(ctx, "cn_step");
            if (mom < eps * (fmax > 1.0 ? fmax : 1.0)) break;
        }
        if (picard > kmax) picard = kmax;
    }
    cn_copy(c, N1, N2, VL);
    cn_copy(c, c->cn_Nn, N1, VL);
    if (rep) {
        rep->picard = step >= 2 ? 0 : picard;
        rep->cycles = cycles;
        rep->res = r.res;
        rep->mom_res = mom;
    }
    gp_status cs = check_cuda(ctx, "cn_step");
    return cs != GP_OK ? cs : st;
}

// ------------------------------------------------------------- adjoint

// common checks of the adjoint calls: geometry, coarse inverse and cut boxes
// for the current alpha, column lists
static gp_status adjoint_ready(gp_ctx *ctx, int level, bool need_coarse_level)
{
    if (!ctx || !ctx->c.geom_ok || level < 0 || level >= ctx->c.L || (need_coarse_level && level + 1 >= ctx->c.L))
        return GP_INVALID;
    gp_status es = ensure_coarse(ctx);
    if (es != GP_OK) return es;
    int st = adjoint_prepare(&ctx->c);
    return (gp_status)st;
}

gp_status gp_residual_t(gp_ctx *ctx, int level, const double *lam, const double *c, double *r, double *norm_host)
{
    if (!lam || !c || !r) return GP_INVALID;
    gp_status st = adjoint_ready(ctx, level, false);
    if (st != GP_OK) return st;
    Ctx *cx = &ctx->c;
    residual_t(cx, level, lam, c, r);
    if (norm_host) {
        cudaMemcpyAsync(norm_host, cx->red + 4, sizeof(double), cudaMemcpyDeviceToHost, cx->stream);
        if (cudaStreamSynchronize(cx->stream) != cudaSuccess) return check_cuda(ctx, "gp_residual_t");
    }
    return check_cuda(ctx, "gp_residual_t");
}

gp_status gp_box_sweep_t(gp_ctx *ctx, int level, double *lam, const double *c)
{
    if (!lam || !c) return GP_INVALID;
    gp_status st = adjoint_ready(ctx, level, false);
    if (st != GP_OK) return st;
    box_sweep_t(&ctx->c, level, lam, c);
    return check_cuda(ctx, "gp_box_sweep_t");
}

gp_status gp_scalar_update_t(gp_ctx *ctx, int level, double *lam, const double *c)
{
    if (!lam || !c) return GP_INVALID;
    gp_status st = adjoint_ready(ctx, level, false);
    if (st != GP_OK) return st;
    scalar_update_t(&ctx->c, level, lam, c);
    return check_cuda(ctx, "gp_scalar_update_t");
}

gp_status gp_ghost_sweep_t(gp_ctx *ctx, int level, double *lam, const double *c)
{
    if (!lam || !c) return GP_INVALID;
    gp_status st = adjoint_ready(ctx, level, false);
    if (st != GP_OK) return st;
    ghost_sweep_t(&ctx->c, level, lam, c);
    return check_cuda(ctx, "gp_ghost_sweep_t");
}

gp_status gp_smooth_t(gp_ctx *ctx, int level, double *lam, const double *c, int nu)
{
    if (!lam || !c || nu < 0) return GP_INVALID;
    gp_status st = adjoint_ready(ctx, level, false);
    if (st != GP_OK) return st;
    smooth_t(&ctx->c, level, lam, c, nu);
    return check_cuda(ctx, "gp_smooth_t");
}

gp_status gp_restrict_t(gp_ctx *ctx, int level, const double *y_coarse, double *lam_fine)
{
    if (!y_coarse || !lam_fine) return GP_INVALID;
    gp_status st = adjoint_ready(ctx, level, true);
    if (st != GP_OK) return st;
    restrict_t(&ctx->c, level, y_coarse, lam_fine);
    return check_cuda(ctx, "gp_restrict_t");
}

gp_status gp_prolong_t(gp_ctx *ctx, int level, const double *r_fine, double *c_coarse)
{
    if (!r_fine || !c_coarse) return GP_INVALID;
    gp_status st = adjoint_ready(ctx, level, true);
    if (st != GP_OK) return st;
    prolong_t(&ctx->c, level, r_fine, c_coarse);
    return check_cuda(ctx, "gp_prolong_t");
}

gp_status gp_cycle_t(gp_ctx *ctx, double *lam, const double *c)
{
    if (!lam || !c) return GP_INVALID;
    gp_status st = adjoint_ready(ctx, 0, false);
    if (st != GP_OK) return st;
    cycle_t_rec(&ctx->c, 0, lam, c);
    return check_cuda(ctx, "gp_cycle_t");
}

gp_status mg_solve_t(gp_ctx *ctx, double *lam, const double *c, double tol, gp_report *rep)
{
    Range nvtx_range("mg_solve_t");
    if (!lam || !c || !(tol >= 0.0)) return GP_INVALID;
    gp_status st = adjoint_ready(ctx, 0, false);
    if (st != GP_OK) return st;
    int s = solve_t(&ctx->c, lam, c, tol, rep);
    gp_status cs = check_cuda(ctx, "mg_solve_t");
    return cs != GP_OK ? cs : (gp_status)s;
}

gp_status cn_step_adjoint(gp_ctx *ctx, int step, const double *x_m, const double *f, double dt, double Re,
                          const gp_body *body, double amp, const gp_walls *walls, double tol, int kmax,
                          const double *xbar_next, double *xbar_m, double *nbar0, double *nbar1, double *nbar2,
                          double *fbar, double *abar)
{
    Range nvtx_range("cn_step_adjoint");
    if (!ctx || !x_m || !xbar_next || !xbar_m || !nbar0 || !nbar1 || !nbar2 || !fbar || !abar || step < 0 ||
        !(dt > 0.0) || !(Re > 0.0) || !(tol >= 0.0))
        return GP_INVALID;
    Ctx *c = &ctx->c;
    if (!c->adjv[0]) return fail(ctx, GP_INVALID, "cn_step_adjoint needs gp_params.adjoint and cn_buffers");
    if (step < 2 && (kmax < 1 || kmax > ADJ_KMAX)) return fail(ctx, GP_INVALID, "kmax must be 1..8 for Picard steps");
    if (!c->geom_ok) return fail(ctx, GP_INVALID, "geometry_build has not succeeded");
    c->prm.alpha = dt / (2.0 * Re);
    gp_status st = adjoint_ready(ctx, 0, false);
    if (st != GP_OK) return st;
    const Level &l0 = c->lv[0];
    const long long VL = l0.VL;
    gp_body unit = body ? *body : gp_body{0, 0, 0, 0, 0};
    gp_body bamp = {amp * unit.U, amp * unit.V, amp * unit.omega, unit.cx, unit.cy};
    gp_walls wl = walls ? *walls : gp_walls{0, 0, 0, 0};
    const gp_walls nowalls = {0, 0, 0, 0};
    double *lam = c->adjv[0], *el = c->adjv[1], *g = c->adjv[2], *xb = c->adjv[3];
    // g: the rigid-body velocity at unit amplitude on the Eq. (BCu) rows
    cudaMemsetAsync(el, 0, VL * sizeof(double), c->stream);
    cn_rhs(c, el, el, nullptr, dt, nullptr, unit, nowalls, g);
    cn_copy(c, xbar_next, xb, VL);
    const int K = step >= 2 ? 1 : kmax;
    const double *X[ADJ_KMAX];
    X[0] = x_m;
    if (step < 2) {
        // the Picard iterates x^(1..K-1) of the forward step, recomputed
        cn_convective(c, x_m, nullptr, c->cn_Nn, 0);
        cn_copy(c, c->cn_Nn, c->cn_Nh, VL);
        for (int k = 1; k < K; k++) {
            double *xk = c->adjv[3 + k];
            cn_copy(c, X[k - 1], xk, VL);
            cn_rhs(c, x_m, c->cn_Nh, f, dt, nullptr, bamp, wl, c->cn_b);
            st = mg_solve(ctx, xk, c->cn_b, tol, nullptr);
            if (st != GP_OK) return st;
            cn_convective(c, xk, c->cn_Nn, c->cn_Nh, 1);
            X[k] = xk;
        }
    }
    double ga = 0.0, acc = 0.0;
    for (int k = K - 1; k >= 0; k--) {
        cudaMemsetAsync(lam, 0, VL * sizeof(double), c->stream);
        int s = solve_t(c, lam, xb, tol, nullptr);
        if (s != GP_OK) return (gp_status)s;
        cn_mask_mom(c, lam, el);
        cn_dot_rows(c, g, lam, c->red + 7);
        cudaMemcpyAsync(&ga, c->red + 7, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(ctx, "cn_step_adjoint");
        acc += ga;
        cn_explicit_t(c, lam, xbar_m);
        if (step >= 2) {
            cn_axpy4(c, el, fbar, dt, nbar0, -dt, nbar1, -0.5 * dt, nbar2, 0.5 * dt);
        } else if (k >= 1) {
            cn_axpy4(c, el, fbar, dt, nbar0, -0.5 * dt, nullptr, 0.0, nullptr, 0.0);
            // the iterate's share: xbar^(k) = J_N(x^(k))^T (-dt/2 E lam)
            cudaMemsetAsync(xb, 0, VL * sizeof(double), c->stream);
            cudaMemsetAsync(c->cn_Nh, 0, VL * sizeof(double), c->stream);
            cn_axpy4(c, el, c->cn_Nh, -0.5 * dt, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0);
            cn_convective_jt(c, X[k], c->cn_Nh, xb);
        } else {
            cn_axpy4(c, el, fbar, dt, nbar0, -dt, nullptr, 0.0, nullptr, 0.0);
        }
    }
    cn_convective_jt(c, x_m, nbar0, xbar_m);
    *abar += acc;
    return check_cuda(ctx, "cn_step_adjoint");
}

}  // extern "C"
