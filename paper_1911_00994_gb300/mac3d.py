"""ctypes binding of the 3-D MAC extension (include/gpmg3d.h): marshalling
only, every step runs in libgpmg.so's kernels (raises if it is missing).

Vectors of a level with N cells per side are FP64 device tensors of
gp3_vec_len(N) entries: four frames (u, v, w, p) of (N + 2)^3 slots, slot
((k + 1)(N + 2) + (j + 1))(N + 2) + (i + 1), then 32 scalars (0: xi).  The
first 4 (N + 2)^3 + 1 entries are the vector of the plain layout the tests
use, so to_device / to_flat only pad and cut.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .gpmg import GpmgError, _ptr, lib as _lib2d

_sig_done = False

SIGNATURES = [
    ("gp3_vec_len", ctypes.c_longlong, [ctypes.c_int]),
    ("gp3_workspace_size", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_size_t)]),
    ("gp3_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("gp3_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("gp3_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("gp3_types", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("gp3_residual", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_double)]),
    ("gp3_smooth", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("gp3_restrict", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("gp3_prolong", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("gp3_cycle", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("gp3_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("gp3_sphere_ghosts", ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    ("gp3_timer_start", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("gp3_timer_stop", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_double)]),
]


def lib():
    global _sig_done
    L = _lib2d()
    if not _sig_done:
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _sig_done = True
    return L


def plain_len(N: int) -> int:
    return 4 * (N + 2) ** 3 + 1


class Solver3D:
    """One 3-D context on the box domain: caller-owned workspace (a torch
    byte tensor on the device) and the device stream."""

    def __init__(self, N, levels, alpha, nu1=2, nu2=1, lam=5, dtau=0.9, precision=0, inner=4, device="cuda",
                 stream=None):
        import torch
        self.torch = torch
        self.L = lib()
        self.N, self.levels = N, levels
        self.device = torch.device(device)
        nb = ctypes.c_size_t(0)
        st = self.L.gp3_workspace_size(N, levels, precision, ctypes.byref(nb))
        if st:
            raise GpmgError(st, "gp3_workspace_size")
        self.ws = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self._ws_ptr = ctypes.c_void_p((base + 255) // 256 * 256)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = ctypes.c_void_p()
        st = self.L.gp3_create(ctypes.byref(ctx), N, levels, alpha, nu1, nu2, lam, dtau, precision, inner, self._ws_ptr,
                               nb.value, ctypes.c_void_p(self.stream.cuda_stream))
        if st:
            raise GpmgError(st, "gp3_create")
        self.ctx = ctx

    def __del__(self):
        if getattr(self, "ctx", None):
            self.L.gp3_destroy(self.ctx)
            self.ctx = None

    def _check(self, st, what):
        if st:
            raise GpmgError(st, "%s: %s" % (what, self.error()))

    def error(self):
        return self.L.gp3_last_error(self.ctx).decode()

    def Nl(self, lev):
        return self.N >> lev

    def vec_len(self, lev=0):
        return int(self.L.gp3_vec_len(self.Nl(lev)))

    def new_vec(self, lev=0):
        return self.torch.zeros(self.vec_len(lev), dtype=self.torch.float64, device=self.device)

    def to_device(self, flat, lev=0):
        v = self.new_vec(lev)
        n = plain_len(self.Nl(lev))
        v[:n] = self.torch.from_numpy(np.ascontiguousarray(flat[:n], dtype=np.float64)).to(self.device)
        return v

    def to_flat(self, v, lev=0):
        self.torch.cuda.synchronize(self.device)
        return v[:plain_len(self.Nl(lev))].cpu().numpy()

    def types(self, lev=0):
        F = (self.Nl(lev) + 2) ** 3
        t = self.torch.zeros(4 * F, dtype=self.torch.uint8, device=self.device)
        self._check(self.L.gp3_types(self.ctx, lev, _ptr(t)), "gp3_types")
        self.torch.cuda.synchronize(self.device)
        return t.cpu().numpy()

    def residual(self, x, b, lev=0):
        r = self.new_vec(lev)
        nrm = ctypes.c_double(0.0)
        self._check(self.L.gp3_residual(self.ctx, lev, _ptr(x), _ptr(b), _ptr(r), ctypes.byref(nrm)), "gp3_residual")
        return r, nrm.value

    def smooth(self, x, b, nu=1, lev=0):
        self._check(self.L.gp3_smooth(self.ctx, lev, _ptr(x), _ptr(b), nu), "gp3_smooth")

    def restrict(self, r, lev=0):
        out = self.new_vec(lev + 1)
        self._check(self.L.gp3_restrict(self.ctx, lev, _ptr(r), _ptr(out)), "gp3_restrict")
        return out

    def prolong(self, eH, x, lev=0):
        self._check(self.L.gp3_prolong(self.ctx, lev, _ptr(eH), _ptr(x)), "gp3_prolong")

    def cycle(self, x, b):
        self._check(self.L.gp3_cycle(self.ctx, _ptr(x), _ptr(b)), "gp3_cycle")

    def solve(self, x, b, tol, max_cycles=100):
        """Returns (status, cycles, final residual, FP64 residual history:
        one entry before each iteration and one after the last)."""
        cyc, it, res = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
        h = (ctypes.c_double * (max_cycles + 1))()
        st = self.L.gp3_solve(self.ctx, _ptr(x), _ptr(b), tol, max_cycles, ctypes.byref(cyc), ctypes.byref(it),
                              ctypes.byref(res), h)
        return st, cyc.value, res.value, np.array(h[:it.value + 1])

    def timer_start(self, lev=0):
        self._check(self.L.gp3_timer_start(self.ctx, lev), "gp3_timer_start")

    def timer_stop(self):
        n, ms = ctypes.c_longlong(0), ctypes.c_double(0.0)
        self._check(self.L.gp3_timer_stop(self.ctx, ctypes.byref(n), ctypes.byref(ms)), "gp3_timer_stop")
        return int(n.value), float(ms.value)


def sphere_ghosts(N, c, R, cap=200000, device="cuda"):
    """gp3_sphere_ghosts: the 3-D ghost rows of a sphere on a grid of N cells
    per side, as numpy arrays sorted by node index (node, B, theta, st, w)."""
    import torch
    L = lib()
    dev = torch.device(device)
    cnt = torch.zeros(2, dtype=torch.int32, device=dev)
    node = torch.zeros(max(cap, 1), dtype=torch.int32, device=dev)
    B = torch.zeros(3 * max(cap, 1), dtype=torch.float64, device=dev)
    th = torch.zeros(3 * max(cap, 1), dtype=torch.float64, device=dev)
    st = torch.zeros(27 * max(cap, 1), dtype=torch.int32, device=dev)
    w = torch.zeros(27 * max(cap, 1), dtype=torch.float64, device=dev)
    n = ctypes.c_int(0)
    stream = torch.cuda.current_stream(dev)
    rc = L.gp3_sphere_ghosts(N, c[0], c[1], c[2], R, cap, _ptr(cnt), _ptr(node), _ptr(B), _ptr(th), _ptr(st),
                             _ptr(w), ctypes.byref(n), ctypes.c_void_p(stream.cuda_stream))
    if rc:
        raise GpmgError(rc, "gp3_sphere_ghosts")
    k = n.value
    nd = node[:k].cpu().numpy()
    o = np.argsort(nd)
    return dict(node=nd[o], B=B[:3 * k].cpu().numpy().reshape(k, 3)[o],
                theta=th[:3 * k].cpu().numpy().reshape(k, 3)[o], st=st[:27 * k].cpu().numpy().reshape(k, 27)[o],
                w=w[:27 * k].cpu().numpy().reshape(k, 27)[o])
