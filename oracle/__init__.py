"""FP64 CPU oracle for the ghost-point multigrid solve (arXiv 1911.00994).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product path (the CUDA library and its binding) never imports it.

The arithmetic lives in ``gpmg_oracle.c`` (plain C, no FMA contraction); this
module only builds it with gcc and marshals numpy arrays through ctypes.

Flat vector layout of one level with N cells per side (all FP64):
  u block: (N+2) rows j = -1..N, (N+1) columns i = 0..N     index (j+1)(N+1) + i
  v block: (N+1) rows j = 0..N,  (N+2) columns i = -1..N    index nU + j(N+2) + i+1
  p block: N rows, N columns                                index nU + nV + jN + i
  last entry: xi (unknown) / mean row (equation)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpmg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

INACTIVE, INTERNAL, GHOST, WALL, BOXGHOST = 0, 1, 2, 3, 4
OK, INVALID, GEOMETRY, SINGULAR, NOT_CONVERGED, DIVERGED = range(6)


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, -ffp-contract=off);
    omp=True: the OpenMP build liboracle_omp.so (same source, same iterates;
    used only for the multi-core CPU baseline)."""
    out = _LIB_OMP if omp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"] +
                              (["-fopenmp"] if omp else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def lib(omp: bool = False):
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if omp else _lib) is None:
            L = ctypes.CDLL(build(omp=omp))
            vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            P = ctypes.POINTER
            L.or_create.restype = vp
            L.or_create.argtypes = [i, d, d, d, i, d]
            L.or_destroy.argtypes = [vp]
            L.or_set_params.argtypes = [vp, i, i, i, i, d, i, i, ctypes.c_uint]
            L.or_set_alpha.argtypes = [vp, d]
            L.or_set_snap.argtypes = [vp, d]
            L.or_set_band.argtypes = [vp, i]
            L.or_last_error.restype = ctypes.c_char_p
            L.or_last_error.argtypes = [vp]
            for f in (L.or_n, L.or_n_int, L.or_num_ghosts):
                f.argtypes = [vp, i]
                f.restype = i
            L.or_geometry.argtypes = [vp, P(d)]
            L.or_types.argtypes = [vp, i, P(ctypes.c_int8)]
            L.or_ghosts.argtypes = [vp, i, P(i), P(d), P(i), i]
            L.or_boundary_point.argtypes = [vp, i, i, i, i, P(d)]
            L.or_residual.restype = d
            L.or_residual.argtypes = [vp, i, P(d), P(d), P(d)]
            L.or_assemble.argtypes = [vp, i, P(i), P(i), P(d), i]
            L.or_dense_solve.argtypes = [i, P(d), P(d)]
            L.or_dense_matrix.argtypes = [vp, i, P(d)]
            L.or_coarse_solve.argtypes = [vp, P(d), P(d)]
            for f in (L.or_box_sweep, L.or_scalar_update, L.or_ghost_sweep):
                f.argtypes = [vp, i, P(d), P(d)]
            L.or_smooth.argtypes = [vp, i, P(d), P(d), i]
            L.or_restrict.argtypes = [vp, i, P(d), P(d)]
            L.or_prolong.argtypes = [vp, i, P(d), P(d)]
            L.or_cycle.argtypes = [vp, i, P(d), P(d)]
            L.or_solve.argtypes = [vp, P(d), P(d), d, i, P(d), P(i)]
            L.or_residual_t.restype = d
            L.or_residual_t.argtypes = [vp, i, P(d), P(d), P(d)]
            for f in (L.or_box_sweep_t, L.or_scalar_update_t, L.or_ghost_sweep_t):
                f.argtypes = [vp, i, P(d), P(d)]
            L.or_smooth_t.argtypes = [vp, i, P(d), P(d), i]
            L.or_restrict_t.argtypes = [vp, i, P(d), P(d)]
            L.or_prolong_t.argtypes = [vp, i, P(d), P(d)]
            L.or_cycle_t.argtypes = [vp, i, P(d), P(d)]
            L.or_solve_t.argtypes = [vp, P(d), P(d), d, i, P(d), P(i)]
            L.or_cut_colours.argtypes = [vp, i, P(i)]
            L.or_cut_colours.restype = i
            L.or_convective_jt.argtypes = [vp, P(d), P(d), P(d)]
            L.or_explicit_t.argtypes = [vp, P(d), P(d)]
            L.or_cn_step_adjoint.argtypes = [vp, i, P(d), vp, d, P(d), d, P(d), d, i, P(d), P(d), P(d), P(d),
                                             P(d), P(d), P(d)]
            L.or_convective.argtypes = [vp, P(d), P(d)]
            L.or_set_continuity_source.argtypes = [vp, vp]
            L.or_solve_krylov.argtypes = [vp, P(d), P(d), d, i, P(d), P(i)]
            L.or_cn_rhs.argtypes = [vp, P(d), P(d), vp, d, vp, P(d), P(d), P(d)]
            L.or_momentum_residual.argtypes = [vp, P(d), P(d), P(d), P(d)]
            L.or_cn_step.argtypes = [vp, P(d), P(d), P(d), i, vp, vp, d, P(d), P(d), d, d, i, P(d)]
            L.or_set_threads.argtypes = [i]
            L.or_set_threads.restype = i
            if omp:
                _lib_omp = L
            else:
                _lib = L
    return _lib_omp if omp else _lib


def _p(a, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def sizes(N: int):
    nU = (N + 1) * (N + 2)
    nV = (N + 2) * (N + 1)
    nP = N * N
    return nU, nV, nP, nU + nV + nP + 1


def split(vec: np.ndarray, N: int):
    """Flat oracle vector -> (u[(N+2),(N+1)], v[(N+1),(N+2)], p[N,N], xi)."""
    nU, nV, nP, n = sizes(N)
    u = vec[:nU].reshape(N + 2, N + 1)
    v = vec[nU:nU + nV].reshape(N + 1, N + 2)
    p = vec[nU + nV:nU + nV + nP].reshape(N, N)
    return u, v, p, vec[n - 1]


def join(u, v, p, xi, N: int) -> np.ndarray:
    nU, nV, nP, n = sizes(N)
    out = np.zeros(n)
    out[:nU] = np.asarray(u).reshape(-1)
    out[nU:nU + nV] = np.asarray(v).reshape(-1)
    out[nU + nV:nU + nV + nP] = np.asarray(p).reshape(-1)
    out[n - 1] = xi
    return out


class Oracle:
    """One discretisation: N cells per side on [x0, x0+L] x [y0, y0+L], `levels`
    grids (N, N/2, ...), alpha = dt / (2 Re)."""

    def __init__(self, N, x0, y0, L, levels, alpha, nu1=2, nu2=1, gamma=1, lam=5, dtau=0.9,
                 ghost_mode=0, order_mode=0, seed=12345, snap=0.3, band=0, threads=1):
        self.L = lib(omp=threads > 1)
        self.threads = self.L.or_set_threads(threads) if threads > 1 else 1
        self.N, self.x0, self.y0, self.len, self.levels, self.alpha = N, x0, y0, L, levels, alpha
        self.h = L / N
        self.c = self.L.or_create(N, x0, y0, L, levels, alpha)
        if not self.c:
            raise ValueError("oracle: invalid sizes")
        self.set_params(nu1, nu2, gamma, lam, dtau, ghost_mode, order_mode, seed)
        self.snap = snap
        self.L.or_set_snap(self.c, snap)
        self.band = band
        self.L.or_set_band(self.c, band)

    def set_params(self, nu1=2, nu2=1, gamma=1, lam=5, dtau=0.9, ghost_mode=0, order_mode=0, seed=12345):
        self.params = dict(nu1=nu1, nu2=nu2, gamma=gamma, lam=lam, dtau=dtau, ghost_mode=ghost_mode,
                           order_mode=order_mode, seed=seed)
        self.L.or_set_params(self.c, nu1, nu2, gamma, lam, dtau, ghost_mode, order_mode, seed)

    def __del__(self):
        try:
            if self.c:
                self.L.or_destroy(self.c)
                self.c = None
        except Exception:
            pass

    def error(self):
        return self.L.or_last_error(self.c).decode()

    def n(self, lev=0):
        return self.L.or_n(self.c, lev)

    def Nl(self, lev):
        return self.N >> lev

    def geometry(self, phi_paper: np.ndarray) -> int:
        """phi on the (2N+1)^2 half lattice, paper sign (phi > 0 inside the object)."""
        phi = np.ascontiguousarray(phi_paper, dtype=np.float64)
        assert phi.shape == (2 * self.N + 1, 2 * self.N + 1)
        self._phi = phi
        return self.L.or_geometry(self.c, _p(phi))

    def types(self, lev=0) -> np.ndarray:
        out = np.zeros(self.n(lev), dtype=np.int8)
        self.L.or_types(self.c, lev, _p(out, ctypes.c_int8))
        return out

    def n_int(self, lev=0):
        return self.L.or_n_int(self.c, lev)

    def ghosts(self, lev=0):
        ng = self.L.or_num_ghosts(self.c, lev)
        iv = np.zeros((max(ng, 1), 7), dtype=np.int32)
        dv = np.zeros((max(ng, 1), 15))
        sv = np.zeros((max(ng, 1), 18), dtype=np.int32)
        self.L.or_ghosts(self.c, lev, _p(iv, ctypes.c_int), _p(dv), _p(sv, ctypes.c_int), ng)
        return dict(grid=iv[:ng, 0], i=iv[:ng, 1], j=iv[:ng, 2], sx=iv[:ng, 3], sy=iv[:ng, 4],
                    axis=iv[:ng, 5] % 2, kind=iv[:ng, 5] // 2, nst=iv[:ng, 6], B=dv[:ng, 0:2], n=dv[:ng, 2:4], theta=dv[:ng, 4:6],
                    w=dv[:ng, 6:15], st=sv[:ng].reshape(ng, 9, 2))

    def boundary_point(self, lev, grid, i, j):
        out = np.zeros(2)
        st = self.L.or_boundary_point(self.c, lev, grid, i, j, _p(out))
        return st, out

    def residual(self, x, b, lev=0):
        r = np.zeros(self.n(lev))
        x = np.ascontiguousarray(x, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        nrm = self.L.or_residual(self.c, lev, _p(x), _p(b), _p(r))
        return r, nrm

    def assemble(self, lev=0):
        n = self.n(lev)
        cap = 12 * n + n
        ri = np.zeros(cap, dtype=np.int32)
        ci = np.zeros(cap, dtype=np.int32)
        v = np.zeros(cap)
        nnz = self.L.or_assemble(self.c, lev, _p(ri, ctypes.c_int), _p(ci, ctypes.c_int), _p(v), cap)
        assert nnz >= 0
        return ri[:nnz], ci[:nnz], v[:nnz]

    def dense_matrix(self, lev=0):
        n = self.n(lev)
        A = np.zeros((n, n))
        self.L.or_dense_matrix(self.c, lev, _p(A))
        return A

    def dense_solve(self, b, lev=0):
        A = self.dense_matrix(lev)
        x = np.array(b, dtype=np.float64)
        st = self.L.or_dense_solve(A.shape[0], _p(A), _p(x))
        return st, x

    def coarse_solve(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        self.L.or_coarse_solve(self.c, _p(b), _p(x))
        return x

    def _inplace(self, fn, lev, x, b, *extra):
        x2 = np.array(x, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        fn(self.c, lev, _p(x2), _p(b), *extra)
        return x2

    def box_sweep(self, x, b, lev=0):
        return self._inplace(self.L.or_box_sweep, lev, x, b)

    def scalar_update(self, x, b, lev=0):
        return self._inplace(self.L.or_scalar_update, lev, x, b)

    def ghost_sweep(self, x, b, lev=0):
        return self._inplace(self.L.or_ghost_sweep, lev, x, b)

    def smooth(self, x, b, nu=1, lev=0):
        return self._inplace(self.L.or_smooth, lev, x, b, nu)

    def restrict(self, r, lev=0):
        out = np.zeros(self.n(lev + 1))
        r = np.ascontiguousarray(r, dtype=np.float64)
        self.L.or_restrict(self.c, lev, _p(r), _p(out))
        return out

    def prolong(self, eH, x, lev=0):
        x2 = np.array(x, dtype=np.float64)
        eH = np.ascontiguousarray(eH, dtype=np.float64)
        self.L.or_prolong(self.c, lev, _p(eH), _p(x2))
        return x2

    def cycle(self, x, b, lev=0):
        x2 = np.array(x, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        st = self.L.or_cycle(self.c, lev, _p(x2), _p(b))
        return st, x2

    # ---- adjoint (transposed system M^T lam = c, transposed cycle)

    def residual_t(self, lam, cc, lev=0):
        """r = c - M^T lam and ||r||_inf."""
        r = np.zeros(self.n(lev))
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        cc = np.ascontiguousarray(cc, dtype=np.float64)
        nrm = self.L.or_residual_t(self.c, lev, _p(lam), _p(cc), _p(r))
        return r, nrm

    def box_sweep_t(self, lam, cc, lev=0):
        return self._inplace(self.L.or_box_sweep_t, lev, lam, cc)

    def scalar_update_t(self, lam, cc, lev=0):
        return self._inplace(self.L.or_scalar_update_t, lev, lam, cc)

    def ghost_sweep_t(self, lam, cc, lev=0):
        return self._inplace(self.L.or_ghost_sweep_t, lev, lam, cc)

    def smooth_t(self, lam, cc, nu=1, lev=0):
        return self._inplace(self.L.or_smooth_t, lev, lam, cc, nu)

    def restrict_t(self, yH, lam, lev=0):
        """lam + R^T yH (R the restriction from level lev to lev + 1)."""
        out = np.array(lam, dtype=np.float64)
        yH = np.ascontiguousarray(yH, dtype=np.float64)
        self.L.or_restrict_t(self.c, lev, _p(yH), _p(out))
        return out

    def prolong_t(self, r, lev=0):
        """P^T r (P the interpolation from level lev + 1 to lev)."""
        out = np.zeros(self.n(lev + 1))
        r = np.ascontiguousarray(r, dtype=np.float64)
        self.L.or_prolong_t(self.c, lev, _p(r), _p(out))
        return out

    def cycle_t(self, lam, cc, lev=0):
        lam2 = np.array(lam, dtype=np.float64)
        cc = np.ascontiguousarray(cc, dtype=np.float64)
        st = self.L.or_cycle_t(self.c, lev, _p(lam2), _p(cc))
        return st, lam2

    def solve_t(self, lam, cc, tol, max_cycles=50):
        lam2 = np.array(lam, dtype=np.float64)
        cc = np.ascontiguousarray(cc, dtype=np.float64)
        hist = np.zeros(max_cycles + 1)
        nc = ctypes.c_int(0)
        st = self.L.or_solve_t(self.c, _p(lam2), _p(cc), tol, max_cycles, _p(hist), ctypes.byref(nc))
        return st, lam2, hist[:nc.value + 1]

    def cut_colours(self, lev=0):
        """(number of colours, colour of every cell j N + i or -1) of the cut
        cells of level lev."""
        Nl = self.N >> lev
        out = np.zeros(Nl * Nl, dtype=np.int32)
        nc = self.L.or_cut_colours(self.c, lev, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return nc, out

    def convective_jt(self, x, y):
        """J_N(x)^T y (transpose of the linearised convective term at x)."""
        out = np.zeros(self.n())
        self.L.or_convective_jt(self.c, _p(np.ascontiguousarray(x, dtype=np.float64)),
                                _p(np.ascontiguousarray(y, dtype=np.float64)), _p(out))
        return out

    def explicit_t(self, y):
        """A^T y with A x = x + alpha lap x on the internal u, v rows."""
        out = np.zeros(self.n())
        self.L.or_explicit_t(self.c, _p(np.ascontiguousarray(y, dtype=np.float64)), _p(out))
        return out

    def cn_step_adjoint(self, step, xm, dt, xbar_next, nb, fbar, abar, f=None, body=(0, 0, 0, 0, 0), amp=1.0,
                        walls=(0, 0, 0, 0), tol=1e-12, kmax=4):
        """Backward pass of one CN step (see gpmg_oracle.c).  nb = [nb0, nb1,
        nb2] and fbar are updated in place; returns (status, xbar_m, abar)."""
        xbar_m = np.zeros(self.n())
        ab = np.array([abar], dtype=np.float64)
        f = self._opt(f)
        st = self.L.or_cn_step_adjoint(self.c, step, _p(np.ascontiguousarray(xm, dtype=np.float64)),
                                       None if f is None else f.ctypes.data,
                                       dt, _p(np.array(body, dtype=np.float64)), amp,
                                       _p(np.array(walls, dtype=np.float64)), tol, kmax,
                                       _p(np.ascontiguousarray(xbar_next, dtype=np.float64)), _p(xbar_m),
                                       _p(nb[0]), _p(nb[1]), _p(nb[2]), _p(fbar), _p(ab))
        return st, xbar_m, float(ab[0])

    def solve(self, x, b, tol, max_cycles=50):
        x2 = np.array(x, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        hist = np.zeros(max_cycles + 1)
        nc = ctypes.c_int(0)
        st = self.L.or_solve(self.c, _p(x2), _p(b), tol, max_cycles, _p(hist), ctypes.byref(nc))
        return st, x2, hist[:nc.value + 1]

    def solve_krylov(self, x, b, tol, maxit=100):
        """BiCGSTAB preconditioned by one cycle; hist = true residual norms."""
        x2 = np.array(x, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        hist = np.zeros(maxit + 1)
        nc = ctypes.c_int(0)
        st = self.L.or_solve_krylov(self.c, _p(x2), _p(b), tol, maxit, _p(hist), ctypes.byref(nc))
        return st, x2, hist[:nc.value + 1]

    # ------------------------------------------------- Crank-Nicolson step
    def set_continuity_source(self, g):
        """g: flat vector whose p block holds the continuity source (kept
        referenced while set); None clears it."""
        self._csrc = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
        self.L.or_set_continuity_source(self.c, None if self._csrc is None else self._csrc.ctypes.data)

    def convective(self, x):
        out = np.zeros(self.n())
        x = np.ascontiguousarray(x, dtype=np.float64)
        self.L.or_convective(self.c, _p(x), _p(out))
        return out

    @staticmethod
    def _opt(a):
        return None if a is None else np.ascontiguousarray(a, dtype=np.float64)

    def cn_rhs(self, xn, Nh, dt, f=None, bc=None, body=(0, 0, 0, 0, 0), walls=(0, 0, 0, 0)):
        b = np.zeros(self.n())
        xn = np.ascontiguousarray(xn, dtype=np.float64)
        Nh = np.ascontiguousarray(Nh, dtype=np.float64)
        f, bc = self._opt(f), self._opt(bc)
        bd = np.array(body, dtype=np.float64)
        wl = np.array(walls, dtype=np.float64)
        self.L.or_cn_rhs(self.c, _p(xn), _p(Nh), None if f is None else f.ctypes.data, dt,
                         None if bc is None else bc.ctypes.data, _p(bd), _p(wl), _p(b))
        return b

    def cn_step(self, x, N1, N2, step, dt, f=None, bc=None, body=(0, 0, 0, 0, 0), walls=(0, 0, 0, 0), tol=1e-10,
                eps=1e-6, kmax=10):
        x2 = np.array(x, dtype=np.float64)
        N1 = np.array(N1, dtype=np.float64)
        N2 = np.array(N2, dtype=np.float64)
        f, bc = self._opt(f), self._opt(bc)
        bd = np.array(body, dtype=np.float64)
        wl = np.array(walls, dtype=np.float64)
        info = np.zeros(3)
        st = self.L.or_cn_step(self.c, _p(x2), _p(N1), _p(N2), step, None if f is None else f.ctypes.data,
                               None if bc is None else bc.ctypes.data, dt, _p(bd), _p(wl), tol, eps, kmax, _p(info))
        return st, x2, N1, N2, info

