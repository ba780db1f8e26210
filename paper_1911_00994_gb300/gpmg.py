"""Thin Python binding of libgpmg (include/gpmg.h): argument marshalling only.

Every step of the solve runs in the CUDA library; this module loads it with
ctypes, passes torch device pointers and sizes, and converts between the
device vector layout and the flat layout (index maps, for tests and I/O).
It raises if the compiled library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpmg.so")

GP_OK, GP_INVALID, GP_GEOMETRY, GP_SINGULAR, GP_NOT_CONVERGED, GP_DIVERGED, GP_CUDA = range(7)
GP_FP64, GP_MIXED = 0, 1
STATUS = {0: "GP_OK", 1: "GP_INVALID", 2: "GP_GEOMETRY", 3: "GP_SINGULAR", 4: "GP_NOT_CONVERGED",
          5: "GP_DIVERGED", 6: "GP_CUDA"}


class gp_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("L", ctypes.c_double),
                ("levels", ctypes.c_int), ("alpha", ctypes.c_double), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("gamma", ctypes.c_int), ("lam", ctypes.c_int), ("dtau", ctypes.c_double), ("snap", ctypes.c_double),
                ("precision", ctypes.c_int), ("max_cycles", ctypes.c_int), ("cn_buffers", ctypes.c_int),
                ("graphs", ctypes.c_int), ("band", ctypes.c_int), ("krylov", ctypes.c_int),
                ("tile_min", ctypes.c_int), ("adjoint", ctypes.c_int), ("inner", ctypes.c_int),
                ("wave_min", ctypes.c_int), ("fuse_restrict", ctypes.c_int)]


class gp_report(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("iterations", ctypes.c_int), ("res0", ctypes.c_double),
                ("res", ctypes.c_double),
                ("rho", ctypes.c_double), ("xi", ctypes.c_double), ("hist_host", ctypes.POINTER(ctypes.c_double))]


class gp_body(ctypes.Structure):
    _fields_ = [("U", ctypes.c_double), ("V", ctypes.c_double), ("omega", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double)]


class gp_walls(ctypes.Structure):
    _fields_ = [("u_bottom", ctypes.c_double), ("u_top", ctypes.c_double), ("v_left", ctypes.c_double),
                ("v_right", ctypes.c_double)]


class gp_shape(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_double), ("b", ctypes.c_double), ("k", ctypes.c_int),
                ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("orbit_r", ctypes.c_double),
                ("orbit_period", ctypes.c_double), ("orbit_phase", ctypes.c_double), ("omega", ctypes.c_double)]


GP_CIRCLE, GP_ELLIPSE, GP_FLOWER = 0, 1, 2


class gp_cn_report(ctypes.Structure):
    _fields_ = [("picard", ctypes.c_int), ("cycles", ctypes.c_int), ("res", ctypes.c_double),
                ("mom_res", ctypes.c_double)]


class GpmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None

# (name, restype, argtypes) of every exported entry point of include/gpmg.h
_VP, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_P = ctypes.POINTER
SIGNATURES = [
    ("gp_params_default", _I, [_P(gp_params), _I, _D, _D, _D]),
    ("gp_pitch", _I, [_I]),
    ("gp_vector_length", ctypes.c_int64, [_I]),
    ("gp_workspace_size", _I, [_P(gp_params), _P(ctypes.c_size_t)]),
    ("gp_create", _I, [_P(_VP), _P(gp_params), _VP, ctypes.c_size_t, _VP]),
    ("gp_destroy", _I, [_VP]),
    ("gp_last_error", ctypes.c_char_p, [_VP]),
    ("gp_set_alpha", _I, [_VP, _D]),
    ("geometry_build", _I, [_VP, _VP, _I]),
    ("geometry_build_shape", _I, [_VP, _P(gp_shape), _D, _P(gp_body)]),
    ("gp_level_set", _I, [_VP, _VP]),
    ("gp_level_info", _I, [_VP, _I, _P(_I), _P(ctypes.c_int64), _P(_D)]),
    ("gp_types", _I, [_VP, _I, _VP, _VP, _VP]),
    ("gp_ghost_count", _I, [_VP, _I, _P(_I), _P(_I)]),
    ("gp_ghost_rows", _I, [_VP, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("gp_residual", _I, [_VP, _I, _VP, _VP, _VP, _P(_D)]),
    ("gp_residual_static", _I, [_VP, _I, _VP, _VP, _VP, _P(_D)]),
    ("gp_box_sweep", _I, [_VP, _I, _VP, _VP]),
    ("gp_scalar_update", _I, [_VP, _I, _VP, _VP]),
    ("gp_ghost_sweep", _I, [_VP, _I, _VP, _VP]),
    ("gp_smooth", _I, [_VP, _I, _VP, _VP, _I]),
    ("gp_restrict", _I, [_VP, _I, _VP, _VP]),
    ("gp_prolong", _I, [_VP, _I, _VP, _VP]),
    ("gp_coarse_solve", _I, [_VP, _VP, _VP]),
    ("gp_cycle", _I, [_VP, _VP, _VP]),
    ("mg_solve", _I, [_VP, _VP, _VP, _D, _P(gp_report)]),
    ("cn_step", _I, [_VP, _VP, _VP, _VP, _I, _VP, _VP, _D, _D, _P(gp_body), _P(gp_walls), _D, _D, _I,
                     _P(gp_cn_report)]),
    ("gp_convective", _I, [_VP, _VP, _VP]),
    ("gp_set_continuity_source", _I, [_VP, _VP]),
    ("gp_cn_rhs", _I, [_VP, _VP, _VP, _VP, _D, _VP, _P(gp_body), _P(gp_walls), _VP]),
    ("gp_residual_t", _I, [_VP, _I, _VP, _VP, _VP, _P(_D)]),
    ("gp_box_sweep_t", _I, [_VP, _I, _VP, _VP]),
    ("gp_scalar_update_t", _I, [_VP, _I, _VP, _VP]),
    ("gp_ghost_sweep_t", _I, [_VP, _I, _VP, _VP]),
    ("gp_smooth_t", _I, [_VP, _I, _VP, _VP, _I]),
    ("gp_restrict_t", _I, [_VP, _I, _VP, _VP]),
    ("gp_prolong_t", _I, [_VP, _I, _VP, _VP]),
    ("gp_cycle_t", _I, [_VP, _VP, _VP]),
    ("mg_solve_t", _I, [_VP, _VP, _VP, _D, _P(gp_report)]),
    ("cn_step_adjoint", _I, [_VP, _I, _VP, _VP, _D, _D, _P(gp_body), _D, _P(gp_walls), _D, _I, _VP, _VP, _VP, _VP,
                             _VP, _VP, _P(_D)]),
    ("gp_launch_count", ctypes.c_int64, [_VP]),
    ("gp_fma_peak", _I, [_VP, _VP, _P(_D), _P(_D)]),
    ("gp_levelset_reinit", _I, [_VP, _VP, _VP, _I, _D]),
    ("gp_levelset_advect", _I, [_VP, _VP, _VP, _VP, _VP, _D, _I]),
    ("gp_timer_start", _I, [_VP, _I, _I]),
    ("gp_timer_stop", _I, [_VP, _P(ctypes.c_int64), _P(_D)]),
]
KERNELS = {"residual": 0, "box_full": 1, "box_cut": 2, "ghost": 3, "scalar": 4, "restrict": 5, "prolong": 6,
           "coarse": 7}


def lib():
    """Load libgpmg.so (built by build.py).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libgpmg.so is not built (run paper_1911_00994_gb300/build.py): %s" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def pitch(N: int) -> int:
    return ((N + 2 + 31) // 32) * 32


def frame(N: int) -> int:
    return (N + 2) * pitch(N)


def vec_len(N: int) -> int:
    return 3 * frame(N) + 32


def flat_to_vec(N: int) -> np.ndarray:
    """Vector index (device layout) of every entry of the flat layout."""
    P, F = pitch(N), frame(N)
    ju, iu = np.meshgrid(np.arange(-1, N + 1), np.arange(0, N + 1), indexing="ij")
    jv, iv = np.meshgrid(np.arange(0, N + 1), np.arange(-1, N + 1), indexing="ij")
    jp, ip = np.meshgrid(np.arange(0, N), np.arange(0, N), indexing="ij")
    u = (ju + 1) * P + (iu + 1)
    v = F + (jv + 1) * P + (iv + 1)
    p = 2 * F + (jp + 1) * P + (ip + 1)
    return np.concatenate([u.ravel(), v.ravel(), p.ravel(), [3 * F]]).astype(np.int64)


def fma_peak(device="cuda", stream=None):
    """gp_fma_peak: (FP64, FP32) FMA throughput of the device in TFLOP/s."""
    import torch
    dev = torch.device(device)
    sink = torch.zeros(8 * 1024, dtype=torch.float64, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    s = lib().gp_fma_peak(ctypes.c_void_p(sink.data_ptr()), ctypes.c_void_p(st.cuda_stream), ctypes.byref(a),
                          ctypes.byref(b))
    if s != GP_OK:
        raise GpmgError(s, "gp_fma_peak")
    return a.value, b.value


class Solver:
    """One solver context: parameters, caller-owned workspace (a torch byte
    tensor on the device) and the device stream."""

    def __init__(self, N, x0, y0, L, levels=None, alpha=None, nu1=2, nu2=1, gamma=1, lam=5, dtau=0.9,
                 snap=0.3, precision=GP_FP64, max_cycles=100, device="cuda", stream=None, cn_buffers=True,
                 graphs=True, band=0, krylov=False, tile_min=0, adjoint=False, inner=0, wave_min=0,
                 fuse_restrict=0):
        import torch
        self.torch = torch
        self.L = lib()
        p = gp_params()
        st = self.L.gp_params_default(ctypes.byref(p), N, x0, y0, L)
        if st:
            raise GpmgError(st, "gp_params_default")
        if levels is not None:
            p.levels = levels
        if alpha is not None:
            p.alpha = alpha
        p.nu1, p.nu2, p.gamma, p.lam, p.dtau, p.snap = nu1, nu2, gamma, lam, dtau, snap
        p.precision, p.max_cycles = precision, max_cycles
        p.cn_buffers = 1 if cn_buffers else 0
        p.graphs = 1 if graphs else 0
        p.band = int(band)
        p.krylov = 1 if krylov else 0
        p.tile_min = int(tile_min)
        p.adjoint = 1 if adjoint else 0
        p.inner = int(inner)
        p.wave_min = int(wave_min)
        p.fuse_restrict = int(fuse_restrict)
        self.prm = p
        nb = ctypes.c_size_t(0)
        st = self.L.gp_workspace_size(ctypes.byref(p), ctypes.byref(nb))
        if st:
            raise GpmgError(st, "gp_workspace_size")
        self.device = torch.device(device)
        self.ws = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        off = (-base) % 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = ctypes.c_void_p(0)
        st = self.L.gp_create(ctypes.byref(ctx), ctypes.byref(p), ctypes.c_void_p(base + off),
                              ctypes.c_size_t(nb.value), ctypes.c_void_p(self.stream.cuda_stream))
        if st:
            raise GpmgError(st, "gp_create")
        self.ctx = ctx
        self.N, self.levels = N, p.levels
        self.x0, self.y0, self.len = x0, y0, L
        self._maps = {}

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                self.L.gp_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    def _check(self, st, where):
        if st != GP_OK:
            raise GpmgError(st, "%s: %s" % (where, self.L.gp_last_error(self.ctx).decode()))

    # ---------------------------------------------------------------- layout
    def Nl(self, lev):
        return self.N >> lev

    def vec_len(self, lev=0):
        return vec_len(self.Nl(lev))

    def new_vec(self, lev=0, dtype=None):
        dtype = dtype or self.torch.float64
        return self.torch.zeros(self.vec_len(lev), dtype=dtype, device=self.device)

    def maps(self, lev):
        if lev not in self._maps:
            self._maps[lev] = self.torch.from_numpy(flat_to_vec(self.Nl(lev))).to(self.device)
        return self._maps[lev]

    def to_device(self, flat, lev=0):
        v = self.new_vec(lev)
        v[self.maps(lev)] = self.torch.as_tensor(np.asarray(flat), dtype=self.torch.float64, device=self.device)
        return v

    def to_flat(self, vec, lev=0):
        return vec[self.maps(lev)].double().cpu().numpy()

    # -------------------------------------------------------------- geometry
    def set_alpha(self, alpha):
        self._check(self.L.gp_set_alpha(self.ctx, alpha), "gp_set_alpha")

    def geometry(self, phi, phi_fluid_positive=0):
        t = self.torch.as_tensor(phi, dtype=self.torch.float64, device=self.device).contiguous()
        self._phi = t
        return self.L.geometry_build(self.ctx, _ptr(t), int(phi_fluid_positive))

    def geometry_shape(self, kind, a, b=0.0, k=0, xc=0.0, yc=0.0, orbit_r=0.0, orbit_period=1.0, orbit_phase=0.0,
                       omega=0.0, t=0.0):
        """geometry_build_shape: level set of a moving test body at time t,
        evaluated on the device; returns (status, body velocity tuple)."""
        sh = gp_shape(kind, a, b, k, xc, yc, orbit_r, orbit_period, orbit_phase, omega)
        bd = gp_body()
        st = self.L.geometry_build_shape(self.ctx, ctypes.byref(sh), t, ctypes.byref(bd))
        return st, (bd.U, bd.V, bd.omega, bd.cx, bd.cy)

    def level_set(self):
        """gp_level_set: the context's level-set lattice (paper sign)."""
        n = 2 * self.N + 1
        out = self.torch.empty(n * n, dtype=self.torch.float64, device=self.device)
        self._check(self.L.gp_level_set(self.ctx, _ptr(out)), "gp_level_set")
        return out.view(n, n)

    def error(self):
        return self.L.gp_last_error(self.ctx).decode()

    def types_flat(self, lev=0):
        F = frame(self.Nl(lev))
        t = self.torch.zeros(3 * F, dtype=self.torch.uint8, device=self.device)
        self._check(self.L.gp_types(self.ctx, lev, _ptr(t), _ptr(t[F:]), _ptr(t[2 * F:])), "gp_types")
        m = self.maps(lev)
        out = t[m[:-1]].cpu().numpy().astype(np.int8)
        return np.concatenate([out, np.array([-1], np.int8)])

    def ghost_rows(self, lev=0):
        no, nr = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self.L.gp_ghost_count(self.ctx, lev, ctypes.byref(no), ctypes.byref(nr)), "gp_ghost_count")
        n = no.value
        T = self.torch
        dev = self.device
        node = T.zeros(max(n, 1), dtype=T.int32, device=dev)
        kind = T.zeros(max(n, 1), dtype=T.uint8, device=dev)
        nst = T.zeros(max(n, 1), dtype=T.uint8, device=dev)
        st = T.zeros(max(n, 1) * 9, dtype=T.int32, device=dev)
        w = T.zeros(max(n, 1) * 9, dtype=T.float64, device=dev)
        B = T.zeros(max(n, 1) * 2, dtype=T.float64, device=dev)
        th = T.zeros(max(n, 1) * 2, dtype=T.float64, device=dev)
        self._check(self.L.gp_ghost_rows(self.ctx, lev, _ptr(node), _ptr(kind), _ptr(nst), _ptr(st), _ptr(w),
                                         _ptr(B), _ptr(th)), "gp_ghost_rows")
        T.cuda.synchronize(dev)
        return dict(node=node[:n].cpu().numpy(), kind=kind[:n].cpu().numpy(), nst=nst[:n].cpu().numpy(),
                    st=st[:9 * n].cpu().numpy().reshape(n, 9), w=w[:9 * n].cpu().numpy().reshape(n, 9),
                    B=B[:2 * n].cpu().numpy().reshape(n, 2), theta=th[:2 * n].cpu().numpy().reshape(n, 2),
                    n_rows=nr.value)

    # ------------------------------------------------------------ operators
    def residual(self, x, b, lev=0):
        r = self.new_vec(lev)
        nrm = ctypes.c_double(0.0)
        self._check(self.L.gp_residual(self.ctx, lev, _ptr(x), _ptr(b), _ptr(r), ctypes.byref(nrm)), "gp_residual")
        return r, nrm.value

    def residual_static(self, x, b, lev=0, r=None, want_norm=True):
        """gp_residual_static: same result as residual(), scratch in a fixed
        library array instead of the workspace (no allocation).  r: an
        existing output vector of the level (a new zeroed one when None);
        want_norm=False passes a NULL norm pointer (no synchronisation) and
        returns None for the norm."""
        if r is None:
            r = self.new_vec(lev)
        nrm = ctypes.c_double(0.0)
        self._check(self.L.gp_residual_static(self.ctx, lev, _ptr(x), _ptr(b), _ptr(r),
                                              ctypes.byref(nrm) if want_norm else None),
                    "gp_residual_static")
        return r, (nrm.value if want_norm else None)

    def box_sweep(self, x, b, lev=0):
        self._check(self.L.gp_box_sweep(self.ctx, lev, _ptr(x), _ptr(b)), "gp_box_sweep")

    def scalar_update(self, x, b, lev=0):
        self._check(self.L.gp_scalar_update(self.ctx, lev, _ptr(x), _ptr(b)), "gp_scalar_update")

    def ghost_sweep(self, x, b, lev=0):
        self._check(self.L.gp_ghost_sweep(self.ctx, lev, _ptr(x), _ptr(b)), "gp_ghost_sweep")

    def smooth(self, x, b, nu=1, lev=0):
        self._check(self.L.gp_smooth(self.ctx, lev, _ptr(x), _ptr(b), nu), "gp_smooth")

    def restrict(self, r, lev=0):
        out = self.new_vec(lev + 1)
        self._check(self.L.gp_restrict(self.ctx, lev, _ptr(r), _ptr(out)), "gp_restrict")
        return out

    def prolong(self, eH, x, lev=0):
        self._check(self.L.gp_prolong(self.ctx, lev, _ptr(eH), _ptr(x)), "gp_prolong")

    def coarse_solve(self, b):
        x = self.new_vec(self.levels - 1)
        self._check(self.L.gp_coarse_solve(self.ctx, _ptr(b), _ptr(x)), "gp_coarse_solve")
        return x

    def cycle(self, x, b):
        self._check(self.L.gp_cycle(self.ctx, _ptr(x), _ptr(b)), "gp_cycle")

    # ---------------------------------------- adjoint (M^T lam = c)
    def residual_t(self, lam, c, lev=0):
        r = self.new_vec(lev)
        nrm = ctypes.c_double(0.0)
        self._check(self.L.gp_residual_t(self.ctx, lev, _ptr(lam), _ptr(c), _ptr(r), ctypes.byref(nrm)),
                    "gp_residual_t")
        return r, nrm.value

    def box_sweep_t(self, lam, c, lev=0):
        self._check(self.L.gp_box_sweep_t(self.ctx, lev, _ptr(lam), _ptr(c)), "gp_box_sweep_t")

    def scalar_update_t(self, lam, c, lev=0):
        self._check(self.L.gp_scalar_update_t(self.ctx, lev, _ptr(lam), _ptr(c)), "gp_scalar_update_t")

    def ghost_sweep_t(self, lam, c, lev=0):
        self._check(self.L.gp_ghost_sweep_t(self.ctx, lev, _ptr(lam), _ptr(c)), "gp_ghost_sweep_t")

    def smooth_t(self, lam, c, nu=1, lev=0):
        self._check(self.L.gp_smooth_t(self.ctx, lev, _ptr(lam), _ptr(c), nu), "gp_smooth_t")

    def restrict_t(self, yH, lam, lev=0):
        """lam += R^T yH (in place on lam, level lev)."""
        self._check(self.L.gp_restrict_t(self.ctx, lev, _ptr(yH), _ptr(lam)), "gp_restrict_t")

    def prolong_t(self, r, lev=0):
        """P^T r on level lev + 1."""
        out = self.new_vec(lev + 1)
        self._check(self.L.gp_prolong_t(self.ctx, lev, _ptr(r), _ptr(out)), "gp_prolong_t")
        return out

    def cycle_t(self, lam, c):
        self._check(self.L.gp_cycle_t(self.ctx, _ptr(lam), _ptr(c)), "gp_cycle_t")

    def solve_t(self, lam, c, tol, hist=True):
        rep = gp_report()
        h = None
        if hist:
            h = (ctypes.c_double * (self.prm.max_cycles + 1))()
            rep.hist_host = ctypes.cast(h, ctypes.POINTER(ctypes.c_double))
        st = self.L.mg_solve_t(self.ctx, _ptr(lam), _ptr(c), tol, ctypes.byref(rep))
        hist_arr = np.array(h[:rep.iterations + 1]) if hist else None
        return st, rep, hist_arr

    def cn_step_adjoint(self, step, xm, dt, Re, xbar_next, xbar_m, nb, fbar, f=None, body=(0, 0, 0, 0, 0), amp=1.0,
                        walls=(0, 0, 0, 0), tol=1e-11, kmax=4):
        """Backward pass of one CN step (see cn_step_adjoint in gpmg.h);
        xbar_m, nb[0..2] and fbar are updated in place; returns dL/damp of
        this step."""
        bd, wl = gp_body(*body), gp_walls(*walls)
        ab = ctypes.c_double(0.0)
        self._check(self.L.cn_step_adjoint(self.ctx, step, _ptr(xm), self._opt(f), dt, Re, ctypes.byref(bd), amp,
                                           ctypes.byref(wl), tol, kmax, _ptr(xbar_next), _ptr(xbar_m), _ptr(nb[0]),
                                           _ptr(nb[1]), _ptr(nb[2]), _ptr(fbar), ctypes.byref(ab)), "cn_step_adjoint")
        return ab.value

    # ------------------------------------------------ Crank-Nicolson step
    @staticmethod
    def _opt(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else None

    def levelset_reinit(self, phi, iters, dtau):
        """gp_levelset_reinit in place on a (2N+1)^2 FP64 device lattice."""
        n = (2 * self.N + 1) ** 2
        work = self.torch.empty(2 * n, dtype=self.torch.float64, device=self.device)
        work.record_stream(self.stream)
        self._check(self.L.gp_levelset_reinit(self.ctx, _ptr(phi), _ptr(work), int(iters), float(dtau)),
                    "gp_levelset_reinit")
        return phi

    def levelset_advect(self, phi, wx, wy, dt, steps):
        """gp_levelset_advect in place; wx, wy on the same lattice."""
        n = (2 * self.N + 1) ** 2
        work = self.torch.empty(n, dtype=self.torch.float64, device=self.device)
        work.record_stream(self.stream)
        self._check(self.L.gp_levelset_advect(self.ctx, _ptr(phi), _ptr(work), _ptr(wx), _ptr(wy), float(dt),
                                              int(steps)), "gp_levelset_advect")
        return phi

    def set_continuity_source(self, g):
        """gp_set_continuity_source: g (a finest-level vector whose p frame
        holds the source) is kept referenced while set; None clears it."""
        self._csrc = g
        self._check(self.L.gp_set_continuity_source(self.ctx, self._opt(g)), "gp_set_continuity_source")

    def convective(self, x):
        out = self.new_vec()
        self._check(self.L.gp_convective(self.ctx, _ptr(x), _ptr(out)), "gp_convective")
        return out

    def cn_rhs(self, xn, Nh, dt, f=None, bc=None, body=(0, 0, 0, 0, 0), walls=(0, 0, 0, 0)):
        b = self.new_vec()
        bd, wl = gp_body(*body), gp_walls(*walls)
        self._check(self.L.gp_cn_rhs(self.ctx, _ptr(xn), _ptr(Nh), self._opt(f), dt, self._opt(bc),
                                     ctypes.byref(bd), ctypes.byref(wl), _ptr(b)), "gp_cn_rhs")
        return b

    def cn_step(self, x, N1, N2, step, dt, Re, f=None, bc=None, body=(0, 0, 0, 0, 0), walls=(0, 0, 0, 0),
                tol=1e-10, eps=1e-6, kmax=10):
        """One Crank-Nicolson step in place on x (and the history N1, N2)."""
        bd, wl = gp_body(*body), gp_walls(*walls)
        rep = gp_cn_report()
        st = self.L.cn_step(self.ctx, _ptr(x), _ptr(N1), _ptr(N2), step, self._opt(f), self._opt(bc), dt, Re,
                            ctypes.byref(bd), ctypes.byref(wl), tol, eps, kmax, ctypes.byref(rep))
        return st, rep

    def launch_count(self):
        return int(self.L.gp_launch_count(self.ctx))

    def timer_start(self, kernel, level=0):
        self._check(self.L.gp_timer_start(self.ctx, KERNELS[kernel], level), "gp_timer_start")

    def timer_stop(self):
        n, ms = ctypes.c_int64(0), ctypes.c_double(0.0)
        self._check(self.L.gp_timer_stop(self.ctx, ctypes.byref(n), ctypes.byref(ms)), "gp_timer_stop")
        return int(n.value), float(ms.value)

    def solve(self, x, b, tol, hist=True):
        rep = gp_report()
        h = None
        if hist:
            h = (ctypes.c_double * (self.prm.max_cycles + 1))()
            rep.hist_host = ctypes.cast(h, ctypes.POINTER(ctypes.c_double))
        st = self.L.mg_solve(self.ctx, _ptr(x), _ptr(b), tol, ctypes.byref(rep))
        hist_arr = np.array(h[:rep.iterations + 1]) if hist else None
        return st, rep, hist_arr
