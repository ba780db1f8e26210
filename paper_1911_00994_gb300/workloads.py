"""Seeded synthetic inputs: level sets, manufactured solutions, right-hand sides.

This module holds no arithmetic of the method.  It only samples closed-form
functions (level sets of the test bodies, exact solutions and the forcing
they imply) at points it is given, so that the CUDA path and the oracle can be
fed identical inputs.

Level-set sign: every function here returns the paper's convention
(Sect. 3.1): phi > 0 inside the object, phi < 0 in the fluid.

Vectors built here use the flat layout (u block (N+2) x (N+1) with rows
j = -1..N; v block (N+1) x (N+2) with columns i = -1..N; p block N x N;
one trailing scalar).  The binding converts to the device layout.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable

import numpy as np

INACTIVE, INTERNAL, GHOST, WALL, BOXGHOST = 0, 1, 2, 3, 4


# ----------------------------------------------------------------- level sets

def half_lattice(N: int, x0: float, y0: float, L: float):
    """Coordinates of the (2N+1)^2 half-cell lattice, X[b, a] = x0 + a h/2."""
    h = L / N
    a = x0 + np.arange(2 * N + 1) * (0.5 * h)
    b = y0 + np.arange(2 * N + 1) * (0.5 * h)
    X, Y = np.meshgrid(a, b)
    return X, Y


def circle(R: float, xc: float = 0.0, yc: float = 0.0):
    """Disc of radius R: phi = R - r."""
    return lambda X, Y: R - np.hypot(X - xc, Y - yc)


def ellipse(a: float, b: float, xc: float = 0.0, yc: float = 0.0):
    """Axis-aligned ellipse: phi = 1 - sqrt((x-xc)^2/a^2 + (y-yc)^2/b^2)."""
    return lambda X, Y: 1.0 - np.sqrt((X - xc) ** 2 / a ** 2 + (Y - yc) ** 2 / b ** 2)


def flower(A: float, B: float, k: int, xc: float = 0.0, yc: float = 0.0):
    """Flower r < A + B sin(k theta): phi = A + B sin(k theta) - r."""
    def f(X, Y):
        dx, dy = X - xc, Y - yc
        return A + B * np.sin(k * np.arctan2(dy, dx)) - np.hypot(dx, dy)
    return f


def phi_half_lattice(shape: Callable, N: int, x0: float, y0: float, L: float) -> np.ndarray:
    X, Y = half_lattice(N, x0, y0, L)
    return np.ascontiguousarray(shape(X, Y), dtype=np.float64)


# ------------------------------------------------------- manufactured fields

@dataclass
class Exact:
    """Exact (u, v, p) with the derivatives needed for a manufactured rhs."""
    u: Callable
    v: Callable
    p: Callable
    lap_u: Callable
    lap_v: Callable
    px: Callable
    py: Callable
    div: Callable


def taylor_green():
    """u = (sin x cos y, -cos x sin y), p = sin x sin y (divergence free)."""
    s, c = np.sin, np.cos
    return Exact(
        u=lambda x, y: s(x) * c(y),
        v=lambda x, y: -c(x) * s(y),
        p=lambda x, y: s(x) * s(y),
        lap_u=lambda x, y: -2.0 * s(x) * c(y),
        lap_v=lambda x, y: 2.0 * c(x) * s(y),
        px=lambda x, y: c(x) * s(y),
        py=lambda x, y: s(x) * c(y),
        div=lambda x, y: 0.0 * x,
    )


def biquadratic(seed: int = 0):
    """Random u, v in span{x^a y^b : a, b <= 2} and linear p.  Every row of the
    discretisation is exact for these, so the discrete solution is the sampled
    field itself (p up to a constant)."""
    rng = np.random.default_rng(seed)
    cu = rng.standard_normal((3, 3))
    cv = rng.standard_normal((3, 3))
    cp = rng.standard_normal(3)

    def ev(cf, x, y, dx=0, dy=0):
        out = 0.0 * x
        for a in range(3):
            for b in range(3):
                if a < dx or b < dy:
                    continue
                fa = math.factorial(a) // math.factorial(a - dx)
                fb = math.factorial(b) // math.factorial(b - dy)
                out = out + cf[a, b] * fa * fb * x ** (a - dx) * y ** (b - dy)
        return out

    return Exact(
        u=lambda x, y: ev(cu, x, y),
        v=lambda x, y: ev(cv, x, y),
        p=lambda x, y: cp[0] + cp[1] * x + cp[2] * y,
        lap_u=lambda x, y: ev(cu, x, y, 2, 0) + ev(cu, x, y, 0, 2),
        lap_v=lambda x, y: ev(cv, x, y, 2, 0) + ev(cv, x, y, 0, 2),
        px=lambda x, y: cp[1] + 0.0 * x,
        py=lambda x, y: cp[2] + 0.0 * x,
        div=lambda x, y: ev(cu, x, y, 1, 0) + ev(cv, x, y, 0, 1),
    )


# ------------------------------------------- the paper's accuracy study (Sect. 5)

def paper_shape(name: str, omega: float = 0.0, t: float = 0.0):
    """The bodies of Eq. (domains) at time t, turned about the origin by
    omega t: phi(x, t) = phi0(R(-omega t) x).  Paper sign (> 0 inside).
    circle: R^2 - r^2, R = 1/sqrt(15); ellipse: 1 - ((c x - s y)^2 / A^2 +
    (s x + c y)^2 / B^2), A = 1/sqrt(14), B = 1/sqrt(2), angle pi/6; flower:
    r < 0.5 + 0.15 sin(5 theta) (the printed formula, r - A - B Im((x + i
    y)^5) / r^5, is positive outside the flower; its negative is used)."""
    ca, sa = math.cos(omega * t), math.sin(omega * t)

    def rot(X, Y):
        return ca * X + sa * Y, -sa * X + ca * Y

    if name == "none":
        return lambda X, Y: -1.0 + 0.0 * X
    if name == "circle":
        R2 = 1.0 / 15.0
        return lambda X, Y: R2 - (X * X + Y * Y)
    if name == "ellipse":
        A2, B2 = 1.0 / 14.0, 0.5
        c, s = math.cos(math.pi / 6), math.sin(math.pi / 6)

        def f(X, Y):
            x, y = rot(X, Y)
            return 1.0 - ((c * x - s * y) ** 2 / A2 + (s * x + c * y) ** 2 / B2)
        return f
    if name == "flower":
        def f(X, Y):
            x, y = rot(X, Y)
            r = np.hypot(x, y)
            im5 = y ** 5 + 5 * x ** 4 * y - 10 * x ** 2 * y ** 3
            rs = np.where(r > 0, r, 1.0)
            return 0.5 + 0.15 * np.where(r > 0, im5 / rs ** 5, 0.0) - r
        return f
    raise ValueError(name)


class PaperExact:
    """The exact solution of Eq. (sol:exa) and the data it implies:
        u = cos(5x) cos(6y log(t+2)),  v = sin(4t) sin(3x^2 + 4y^2 + 2),
        p = cos(6xt) sin(2yt) log(3t+1) + sin(5t),
    the forcing f = u_t + u.grad u + grad p - lap u / Re of the momentum
    equation and the continuity source g = div u."""

    def __init__(self, Re: float = 100.0):
        self.Re = Re

    @staticmethod
    def u(x, y, t):
        return np.cos(5 * x) * np.cos(6 * y * math.log(t + 2))

    @staticmethod
    def v(x, y, t):
        return math.sin(4 * t) * np.sin(3 * x * x + 4 * y * y + 2)

    @staticmethod
    def p(x, y, t):
        return np.cos(6 * x * t) * np.sin(2 * y * t) * math.log(3 * t + 1) + math.sin(5 * t)

    @staticmethod
    def _du(x, y, t):
        Lg = math.log(t + 2)
        c5, s5 = np.cos(5 * x), np.sin(5 * x)
        cy, sy = np.cos(6 * y * Lg), np.sin(6 * y * Lg)
        u_t = -c5 * sy * 6 * y / (t + 2)
        u_x = -5 * s5 * cy
        u_y = -6 * Lg * c5 * sy
        lap = -(25 + 36 * Lg * Lg) * c5 * cy
        return u_t, u_x, u_y, lap

    @staticmethod
    def _dv(x, y, t):
        S = 3 * x * x + 4 * y * y + 2
        s4, c4 = math.sin(4 * t), math.cos(4 * t)
        cS, sS = np.cos(S), np.sin(S)
        v_t = 4 * c4 * sS
        v_x = s4 * cS * 6 * x
        v_y = s4 * cS * 8 * y
        lap = s4 * (14 * cS - (36 * x * x + 64 * y * y) * sS)
        return v_t, v_x, v_y, lap

    @staticmethod
    def _dp(x, y, t):
        lg = math.log(3 * t + 1)
        p_x = -6 * t * np.sin(6 * x * t) * np.sin(2 * y * t) * lg
        p_y = 2 * t * np.cos(6 * x * t) * np.cos(2 * y * t) * lg
        return p_x, p_y

    def f_u(self, x, y, t):
        u_t, u_x, u_y, lap = self._du(x, y, t)
        p_x, _ = self._dp(x, y, t)
        return u_t + self.u(x, y, t) * u_x + self.v(x, y, t) * u_y + p_x - lap / self.Re

    def f_v(self, x, y, t):
        v_t, v_x, v_y, lap = self._dv(x, y, t)
        _, p_y = self._dp(x, y, t)
        return v_t + self.u(x, y, t) * v_x + self.v(x, y, t) * v_y + p_y - lap / self.Re

    def div(self, x, y, t):
        return self._du(x, y, t)[1] + self._dv(x, y, t)[2]


# ----------------------------------------------------------- node positions

def flat_sizes(N: int):
    nU = (N + 1) * (N + 2)
    nV = (N + 2) * (N + 1)
    nP = N * N
    return nU, nV, nP, nU + nV + nP + 1


def flat_coords(N: int, x0: float, y0: float, L: float):
    """(grid, i, j, x, y) of every unknown of the flat layout (mean slot last)."""
    h = L / N
    ju, iu = np.meshgrid(np.arange(-1, N + 1), np.arange(0, N + 1), indexing="ij")
    jv, iv = np.meshgrid(np.arange(0, N + 1), np.arange(-1, N + 1), indexing="ij")
    jp, ip = np.meshgrid(np.arange(0, N), np.arange(0, N), indexing="ij")
    g = np.concatenate([np.zeros(iu.size, int), np.ones(iv.size, int), 2 * np.ones(ip.size, int), [-1]])
    i = np.concatenate([iu.ravel(), iv.ravel(), ip.ravel(), [0]])
    j = np.concatenate([ju.ravel(), jv.ravel(), jp.ravel(), [0]])
    ox = np.array([0.0, 0.5, 0.5, 0.0])[g]
    oy = np.array([0.5, 0.0, 0.5, 0.0])[g]
    x = x0 + (i + ox) * h
    y = y0 + (j + oy) * h
    return g, i, j, x, y


def manufactured_rhs(ex: Exact, N: int, x0: float, y0: float, L: float, alpha: float,
                     types: np.ndarray, ghost_grid, ghost_i, ghost_j, ghost_B, ghost_kind=None) -> np.ndarray:
    """rhs of Eq. (spaceprobaug) in the flat layout for the exact field `ex`:
    internal momentum rows u - alpha lap u + grad p, continuity rows div u,
    boundary-condition ghost rows the exact velocity at the boundary point B
    (extrapolation ghost rows 0), wall rows the exact
    velocity on the wall, pressure-ghost and mean rows 0."""
    g, i, j, x, y = flat_coords(N, x0, y0, L)
    nU, nV, nP, n = flat_sizes(N)
    b = np.zeros(n)
    t = types.astype(int)
    m = (t == INTERNAL) & (g == 0)
    b[m] = ex.u(x[m], y[m]) - alpha * ex.lap_u(x[m], y[m]) + ex.px(x[m], y[m])
    m = (t == INTERNAL) & (g == 1)
    b[m] = ex.v(x[m], y[m]) - alpha * ex.lap_v(x[m], y[m]) + ex.py(x[m], y[m])
    m = (t == INTERNAL) & (g == 2)
    b[m] = ex.div(x[m], y[m])
    # walls: the node itself lies on the wall
    m = (t == WALL) & (g == 0)
    b[m] = ex.u(x[m], y[m])
    m = (t == WALL) & (g == 1)
    b[m] = ex.v(x[m], y[m])
    # box ghosts: the condition holds on the wall half a cell inside
    m = (t == BOXGHOST) & (g == 0)
    yw = np.where(j[m] < 0, y0, y0 + L)
    b[m] = ex.u(x[m], yw)
    m = (t == BOXGHOST) & (g == 1)
    xw = np.where(i[m] < 0, x0, x0 + L)
    b[m] = ex.v(xw, y[m])
    # object ghosts with a boundary-condition row: exact velocity at B
    # (extrapolation rows, kind 1, keep rhs 0)
    if ghost_kind is None:
        ghost_kind = [0] * len(ghost_grid)
    for gg, ii, jj, B, kd in zip(ghost_grid, ghost_i, ghost_j, ghost_B, ghost_kind):
        if gg == 2 or kd != 0:
            continue
        k = flat_index(N, gg, ii, jj)
        b[k] = (ex.u if gg == 0 else ex.v)(B[0], B[1])
    return b


def flat_index(N: int, g: int, i: int, j: int) -> int:
    nU, nV, nP, n = flat_sizes(N)
    if g == 0:
        return (j + 1) * (N + 1) + i
    if g == 1:
        return nU + j * (N + 2) + (i + 1)
    return nU + nV + j * N + i


def exact_flat(ex: Exact, N: int, x0: float, y0: float, L: float, types: np.ndarray) -> np.ndarray:
    """Sampled exact field on every active node (0 on inactive nodes); the
    pressure is shifted to zero mean over the internal cells."""
    g, i, j, x, y = flat_coords(N, x0, y0, L)
    out = np.zeros(g.size)
    t = types.astype(int)
    act = (t != INACTIVE) & (g >= 0)
    for gg, f in ((0, ex.u), (1, ex.v), (2, ex.p)):
        m = act & (g == gg)
        out[m] = f(x[m], y[m])
    mp = (g == 2) & (t == INTERNAL)
    mean = out[mp].mean()
    out[(g == 2) & act] -= mean
    out[-1] = 0.0
    return out


def random_flat(N: int, types: np.ndarray, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded N(0, scale^2) values on active nodes, 0 elsewhere."""
    rng = np.random.default_rng(seed)
    out = rng.standard_normal(types.size) * scale
    out[types.astype(int) == INACTIVE] = 0.0
    out[-1] = rng.standard_normal() * scale
    return out


def div_free_flat(N: int, x0: float, y0: float, L: float, types: np.ndarray, seed: int, amp: float = 0.1,
                  modes: int = 6) -> np.ndarray:
    """A seeded velocity field that is discretely divergence-free on the MAC
    grid (the initial state of the 8192^2 seven-petal-flower solve): u and v
    are the centred differences of a
    smooth random stream function psi (sum of `modes` plane waves with
    wave numbers pi * (1..4)) across each face, u = (psi(x, y + h/2) -
    psi(x, y - h/2)) / h and v = -(psi(x + h/2, y) - psi(x - h/2, y)) / h, so
    the divergence of every cell telescopes to zero.  Scaled so that
    max |u|, |v| = amp; pressure, xi and inactive nodes are 0."""
    rng = np.random.default_rng(seed)
    kx = np.pi * rng.integers(1, 5, modes) * rng.choice([-1, 1], modes)
    ky = np.pi * rng.integers(1, 5, modes) * rng.choice([-1, 1], modes)
    c = rng.standard_normal(modes)
    ph = rng.uniform(0.0, 2 * np.pi, modes)

    def psi(x, y):
        s = np.zeros_like(x)
        for m in range(modes):
            s += c[m] * np.sin(kx[m] * x + ky[m] * y + ph[m])
        return s

    h = L / N
    g, i, j, x, y = flat_coords(N, x0, y0, L)
    out = np.zeros(g.size)
    mu, mv = g == 0, g == 1
    out[mu] = (psi(x[mu], y[mu] + h / 2) - psi(x[mu], y[mu] - h / 2)) / h
    out[mv] = -(psi(x[mv] + h / 2, y[mv]) - psi(x[mv] - h / 2, y[mv])) / h
    out[types.astype(int) == INACTIVE] = 0.0
    out[-1] = 0.0
    peak = np.abs(out[mu | mv]).max()
    return out * (amp / peak if peak > 0 else 0.0)


def div_free_device(N: int, x0: float, L: float, P: int, seed: int, amp: float = 0.1, modes: int = 6, device=None):
    """div_free_flat's field (same seeded stream function) built directly in
    the device vector layout with torch: three frames of (N + 2) rows x P
    (node (i, j) at (j + 1) P + i + 1), then 32 scalars; pressure, xi and the
    frame padding 0.  Unlike div_free_flat it does not zero inactive nodes
    (the solver does) and scales by the maximum over every node.  For the
    full-size cases, where the flat host arrays would be large."""
    import torch
    rng = np.random.default_rng(seed)
    kx = np.pi * rng.integers(1, 5, modes) * rng.choice([-1, 1], modes)
    ky = np.pi * rng.integers(1, 5, modes) * rng.choice([-1, 1], modes)
    c = rng.standard_normal(modes)
    ph = rng.uniform(0.0, 2 * np.pi, modes)
    h = L / N
    F = (N + 2) * P
    out = torch.zeros(3 * F + 32, dtype=torch.float64, device=device)
    rows = torch.arange(N + 2, dtype=torch.float64, device=device).view(-1, 1)
    cols = torch.arange(P, dtype=torch.float64, device=device).view(1, -1)

    def psi(x, y):
        s = torch.zeros(torch.broadcast_shapes(x.shape, y.shape), dtype=torch.float64, device=device)
        for m in range(modes):
            s += float(c[m]) * torch.sin(float(kx[m]) * x + float(ky[m]) * y + float(ph[m]))
        return s

    xu, yu = x0 + (cols - 1) * h, x0 + (rows - 0.5) * h      # u(i, j) at (i h, (j + 1/2) h)
    u = (psi(xu, yu + h / 2) - psi(xu, yu - h / 2)) / h
    u[:, 0] = 0.0
    u[:, N + 2:] = 0.0                                        # i in [0, N]
    xv, yv = x0 + (cols - 0.5) * h, x0 + (rows - 1) * h      # v(i, j) at ((i + 1/2) h, j h)
    v = -(psi(xv + h / 2, yv) - psi(xv - h / 2, yv)) / h
    v[0, :] = 0.0                                             # j in [0, N]
    v[:, N + 2:] = 0.0                                        # i in [-1, N]
    peak = max(float(u.abs().max()), float(v.abs().max()))
    scale = amp / peak if peak > 0 else 0.0
    out[:F] = (u * scale).reshape(-1)
    out[F:2 * F] = (v * scale).reshape(-1)
    return out
