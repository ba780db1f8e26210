"""Oracle of the 3-D ghost points of a sphere: plain Python, FP64.

Test infrastructure only (imported by tests/).  In three dimensions the
ghost-point boundary condition keeps its form (Sect. 3.3 and the 3-D
remark of Sect. 3): for a velocity ghost G, Algorithm 1 finds the boundary
point B by marching from G along the normal of the interpolated level set
and bisecting, and Eq. (BCu) interpolates the velocity at B from the 27
nodes G - (k, l, m) s h, k, l, m in {0, 1, 2}, with the product of three
one-dimensional quadratic Lagrange bases (Eq. BCu's 3 x 3 stencil becomes
3 x 3 x 3).  Readings, as in 2-D:

* the object is {phi > 0}, phi = R - |x - c|; a velocity node of the box
  interior is INTERNAL when phi < 0 at it, a GHOST when phi >= 0 and one of
  its six neighbours is INTERNAL (the ghosts an interior momentum row reads);
* phi~ is the trilinear interpolant of phi on the grid's own nodes in the
  cell found by floor (R7), n = grad phi~ / |grad phi~|;
* Algorithm 1: H <- H - h/2 n(H) while phi~(H) > 0 (at most 64 steps), then
  ceil(log2(|H_prev - H| / 0.01 h)) bisections (a strict < 0 test), B the
  last midpoint; phi(G) = 0 gives B = G (R7, C13, C14);
* s_a = SIGN(n_a(G)) (SIGN(0) = 1), theta_a = s_a (x_G - x_B)_a / h (R2),
  stencil node (k, l, m) at G - (k s_x, l s_y, m s_z) h with weight
  L_k(theta_x) L_l(theta_y) L_m(theta_z), L_0(t) = (t-1)(t-2)/2,
  L_1(t) = -t(t-2), L_2(t) = t(t-1)/2.

The arithmetic is written in a fixed order of separately rounded operations
so that the march's decisions can be compared node for node.
"""
from __future__ import annotations

import math

import numpy as np

MAX_MARCH = 64


def node_xyz(g, i, j, k, h):
    """Position of node (i, j, k) of grid g (0 u, 1 v, 2 w) on [0, 1]^3."""
    ox = 0.0 if g == 0 else 0.5
    oy = 0.0 if g == 1 else 0.5
    oz = 0.0 if g == 2 else 0.5
    return (i + ox) * h, (j + oy) * h, (k + oz) * h


def phi(c, R, x, y, z):
    dx, dy, dz = x - c[0], y - c[1], z - c[2]
    return R - math.sqrt(dx * dx + dy * dy + dz * dz)


def lagrange(t):
    return ((t - 1.0) * (t - 2.0) * 0.5, -t * (t - 2.0), t * (t - 1.0) * 0.5)


class Ghosts3D:
    def __init__(self, N, c, R):
        self.N, self.c, self.R = N, c, R
        self.h = 1.0 / N

    def phi_node(self, g, i, j, k):
        return phi(self.c, self.R, *node_xyz(g, i, j, k, self.h))

    def interior(self, g, i, j, k):
        # the box-interior positions of grid g (its own axis 1..N-1, the others 0..N-1)
        N = self.N
        own = (i, j, k)[g]
        t = [(i, j, k)[a] for a in range(3) if a != g]
        return 1 <= own <= N - 1 and all(0 <= v <= N - 1 for v in t)

    def fluid(self, g, i, j, k):
        return self.interior(g, i, j, k) and self.phi_node(g, i, j, k) < 0.0

    def ghost_nodes(self, g):
        """Ghost nodes of grid g in (k, j, i) order."""
        N = self.N
        out = []
        for k in range(-1, N + 1):
            for j in range(-1, N + 1):
                for i in range(-1, N + 1):
                    if not self.interior(g, i, j, k) or self.phi_node(g, i, j, k) < 0.0:
                        continue
                    if any(self.fluid(g, i + di, j + dj, k + dk)
                           for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))):
                        out.append((i, j, k))
        return out

    def interp(self, g, x, y, z):
        """phi~ and grad phi~ at (x, y, z): trilinear on grid g's own nodes."""
        h = self.h
        ox = 0.0 if g == 0 else 0.5
        oy = 0.0 if g == 1 else 0.5
        oz = 0.0 if g == 2 else 0.5
        X, Y, Z = x / h - ox, y / h - oy, z / h - oz
        i0, j0, k0 = math.floor(X), math.floor(Y), math.floor(Z)
        tx, ty, tz = X - i0, Y - j0, Z - k0
        f = [[[self.phi_node(g, i0 + a, j0 + b, k0 + cc) for a in (0, 1)] for b in (0, 1)] for cc in (0, 1)]
        # f[cz][cy][cx]
        sx, sy, sz = 1.0 - tx, 1.0 - ty, 1.0 - tz
        v00 = sx * f[0][0][0] + tx * f[0][0][1]
        v10 = sx * f[0][1][0] + tx * f[0][1][1]
        v01 = sx * f[1][0][0] + tx * f[1][0][1]
        v11 = sx * f[1][1][0] + tx * f[1][1][1]
        val = sz * (sy * v00 + ty * v10) + tz * (sy * v01 + ty * v11)
        gx = (sz * (sy * (f[0][0][1] - f[0][0][0]) + ty * (f[0][1][1] - f[0][1][0])) +
              tz * (sy * (f[1][0][1] - f[1][0][0]) + ty * (f[1][1][1] - f[1][1][0]))) / h
        gy = (sz * (sx * (f[0][1][0] - f[0][0][0]) + tx * (f[0][1][1] - f[0][0][1])) +
              tz * (sx * (f[1][1][0] - f[1][0][0]) + tx * (f[1][1][1] - f[1][0][1]))) / h
        gz = (sy * (sx * (f[1][0][0] - f[0][0][0]) + tx * (f[1][0][1] - f[0][0][1])) +
              ty * (sx * (f[1][1][0] - f[0][1][0]) + tx * (f[1][1][1] - f[0][1][1]))) / h
        return val, (gx, gy, gz)

    def unit_normal(self, g, x, y, z):
        _, (gx, gy, gz) = self.interp(g, x, y, z)
        nn = math.sqrt(gx * gx + gy * gy + gz * gz)
        return gx / nn, gy / nn, gz / nn

    def project(self, g, i, j, k):
        """Algorithm 1 from ghost (i, j, k): (B, n at G, steps)."""
        h = self.h
        G = node_xyz(g, i, j, k, h)
        nG = self.unit_normal(g, *G)
        if self.phi_node(g, i, j, k) == 0.0:
            return G, nG, 0
        H = G
        Hp = G
        steps = 0
        while self.interp(g, *H)[0] > 0.0:
            if steps == MAX_MARCH:
                raise RuntimeError("march did not leave the object")
            n = self.unit_normal(g, *H)
            Hp = H
            H = (H[0] - 0.5 * h * n[0], H[1] - 0.5 * h * n[1], H[2] - 0.5 * h * n[2])
            steps += 1
        dx, dy, dz = Hp[0] - H[0], Hp[1] - H[1], Hp[2] - H[2]
        dist = math.sqrt(dx * dx + dy * dy + dz * dz)
        nb = math.ceil(math.log2(dist / (0.01 * h)))
        K = H
        Mid = H
        for _ in range(nb):
            Mid = (0.5 * (Hp[0] + K[0]), 0.5 * (Hp[1] + K[1]), 0.5 * (Hp[2] + K[2]))
            if self.interp(g, *Mid)[0] < 0.0:
                K = Mid
            else:
                Hp = Mid
        return Mid, nG, steps

    def rows(self, g):
        """Per ghost of grid g: (i, j, k), B, theta, the 27 stencil nodes and weights."""
        h = self.h
        out = []
        for (i, j, k) in self.ghost_nodes(g):
            B, nG, _ = self.project(g, i, j, k)
            G = node_xyz(g, i, j, k, h)
            s = [1 if v >= 0.0 else -1 for v in nG]
            th = [s[a] * (G[a] - B[a]) / h for a in range(3)]
            L = [lagrange(t) for t in th]
            st, w = [], []
            for m in range(3):
                for l in range(3):
                    for kk in range(3):
                        st.append((i - kk * s[0], j - l * s[1], k - m * s[2]))
                        w.append(L[0][kk] * L[1][l] * L[2][m])
            out.append(dict(node=(i, j, k), B=B, theta=th, s=s, st=st, w=np.array(w)))
        return out
