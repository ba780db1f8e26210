"""Oracle of the 3-D MAC extension on the box domain: plain, slow, FP64 numpy.

Test infrastructure only (imported by tests/).
The paper states that the method extends directly to three dimensions
(Sect. 3, "Discretization in space"): the staggered grid gains a w velocity,
the box of a cell holds its pressure and six faces (a 7 x 7 system, Sect.
4.1.1), and the transfers act per axis.  This module builds that system on
the cube [0, 1]^3 with walls only (no immersed body), in the same readings
as the 2-D oracle:

* unknowns u(i, j, k) at (i h, (j+1/2) h, (k+1/2) h), i in [0, N],
  j, k in [-1, N]; v and w likewise with their own axis staggered; p at cell
  centres, i, j, k in [0, N); the scalar xi of Eq. (spaceprobaug);
* node types: a velocity node on its own wall is a WALL row (Dirichlet);
  a node half a cell outside a wall next to an interior node (exactly one
  transverse index outside [0, N)) is a BOXGHOST row
  3/8 x_G + 3/4 x_1 - 1/8 x_2 = b (Eq. BCu with theta_normal = 1/2,
  theta_tangential = 0, as on the 2-D box walls); other outside nodes are
  INACTIVE (value 0, row x = b);
* momentum rows (1 + 6 a) u - a (six neighbours) + q (p_E - p_W) = b with
  a = alpha / h^2, q = 1 / h (Eqs. NSCN1, spaceprob); continuity
  q (div of the cell's faces) - xi = b; the mean row h^3 sum p = b;
* relaxation (Algorithm relax): box Gauss-Seidel over the cells in seven
  colours (i + 2 j + 3 k) mod 7, each box solving its pressure and interior
  faces with everything else frozen; then xi <- mean(div u - b_c) and a
  uniform pressure shift that makes the mean row exact; then lambda Jacobi
  sweeps w += dtau r over the WALL and BOXGHOST rows (Eq. ghostrelax);
* restriction (Eqs. restop, restop5 per axis): a coarse node of class K
  (interior or wall/box-ghost) takes the weighted residual of its fine
  stencil if every fine node is of class K, else their plain mean, 0 if
  none; the mean row is injected;
* prolongation (Sect. 4.3): trilinear over the active coarse nodes, weights
  renormalised, cell-centred axes extrapolated linearly at the walls;
* coarsest level solved exactly (dense LU of the assembled matrix).

Indexing: every grid lives in a (N+2)^3 array indexed [k+1, j+1, i+1];
flattened in C order (slot ((k+1)(N+2) + (j+1))(N+2) + (i+1)) the four
frames u, v, w, p followed by xi form the vector.
"""
from __future__ import annotations

import numpy as np

INACTIVE, INTERNAL, WALL, BOXGHOST = 0, 1, 3, 4
G_U, G_V, G_W, G_P = 0, 1, 2, 3
NCOL = 7


def colour(i, j, k):
    """Seven colours: no two boxes of one colour share or read each other's unknowns."""
    return (i + 2 * j + 3 * k) % NCOL


class Mac3D:
    def __init__(self, N, alpha, levels, lam=5, dtau=0.9, nu1=2, nu2=1):
        self.N, self.alpha, self.levels = N, alpha, levels
        self.lam, self.dtau, self.nu1, self.nu2 = lam, dtau, nu1, nu2
        self.types = [self._types(N >> l) for l in range(levels)]
        self._coarse = None

    # ------------------------------------------------------------ layout
    @staticmethod
    def _types(N):
        S = N + 2
        t = np.zeros((4, S, S, S), np.int8)
        r = np.arange(-1, N + 1)
        K, J, I = np.meshgrid(r, r, r, indexing="ij")
        inside = lambda a: (a >= 0) & (a <= N - 1)
        for g in range(3):
            # own axis coordinate: faces 0..N; transverse: cells -1..N
            own, t1, t2 = [(I, J, K), (J, K, I), (K, I, J)][g]
            face_ok = (own >= 0) & (own <= N)
            interior = (own >= 1) & (own <= N - 1)
            tin1, tin2 = inside(t1), inside(t2)
            tg = np.full(I.shape, INACTIVE, np.int8)
            tg[face_ok & tin1 & tin2 & interior] = INTERNAL
            tg[face_ok & tin1 & tin2 & ~interior] = WALL
            out1 = (t1 == -1) | (t1 == N)
            out2 = (t2 == -1) | (t2 == N)
            tg[interior & ((out1 & tin2) | (out2 & tin1))] = BOXGHOST
            t[g] = tg
        t[G_P][1:N + 1, 1:N + 1, 1:N + 1] = INTERNAL
        return t

    def n(self, lev=0):
        S = (self.N >> lev) + 2
        return 4 * S ** 3 + 1

    def split(self, x, lev=0):
        S = (self.N >> lev) + 2
        F = S ** 3
        return [x[g * F:(g + 1) * F].reshape(S, S, S) for g in range(4)], x[4 * F:4 * F + 1]

    # ------------------------------------------------------------ the rows
    def residual(self, x, b, lev=0):
        """r = b - M x, every row of Eq. (LS) in 3-D; returns (r, ||r||_inf)."""
        N = self.N >> lev
        h = 1.0 / N
        a, q = self.alpha / h ** 2, 1.0 / h
        d = 1.0 + 6.0 * a
        (u, v, w, p), xi = self.split(x, lev)
        (bu, bv, bw, bp), bm = self.split(b, lev)
        t = self.types[lev]
        r = np.zeros_like(x)
        (ru, rv, rw, rp), rm = self.split(r, lev)
        vel = [u, v, w]
        bs = [bu, bv, bw]
        rs = [ru, rv, rw]
        S = N + 2
        for g in range(3):
            x3, b3, r3, tg = vel[g], bs[g], rs[g], t[g]
            Mx = np.zeros_like(x3)
            sl = np.s_[1:S - 1, 1:S - 1, 1:S - 1]
            # momentum rows on the interior slots (neighbours exist in the array)
            lap = np.zeros_like(x3)
            lap[sl] = (x3[2:, 1:-1, 1:-1] + x3[:-2, 1:-1, 1:-1] + x3[1:-1, 2:, 1:-1] + x3[1:-1, :-2, 1:-1] +
                       x3[1:-1, 1:-1, 2:] + x3[1:-1, 1:-1, :-2])
            grad = np.zeros_like(x3)
            # pressure difference across the face: p(cell on the + side) - p(cell on the - side);
            # the + side cell of face (i) along the own axis has the same index, the - side is index - 1
            ax = 2 - g  # array axis of the own direction ([k, j, i] order)
            pm = np.roll(p, 1, axis=ax)
            grad = p - pm
            Mx = d * x3 - a * lap + q * grad
            rr = np.zeros_like(x3)
            m = tg == INTERNAL
            rr[m] = b3[m] - Mx[m]
            m = (tg == WALL) | (tg == INACTIVE)
            rr[m] = b3[m] - x3[m]
            # box-ghost rows: 3/8 x_G + 3/4 x_1 - 1/8 x_2 along the outward transverse axis
            for tax in range(3):
                if tax == ax:
                    continue
                for side in (0, S - 1):
                    idx = [slice(None)] * 3
                    idx[tax] = side
                    i1 = list(idx)
                    i2 = list(idx)
                    i1[tax] = 1 if side == 0 else S - 2
                    i2[tax] = 2 if side == 0 else S - 3
                    tsl = tg[tuple(idx)]
                    mg = tsl == BOXGHOST
                    val = 0.375 * x3[tuple(idx)] + 0.75 * x3[tuple(i1)] - 0.125 * x3[tuple(i2)]
                    blk = rr[tuple(idx)]
                    blk[mg] = b3[tuple(idx)][mg] - val[mg]
                    rr[tuple(idx)] = blk
            r3[...] = rr
        # continuity rows (pressure slots outside the cells: x = b)
        rp[...] = bp - p
        rp[1:-1, 1:-1, 1:-1] = bp[1:-1, 1:-1, 1:-1] - (self.div(x, lev) - xi[0])
        rm[0] = bm[0] - h ** 3 * p[1:-1, 1:-1, 1:-1].sum()
        return r, float(np.abs(r).max())

    def div(self, x, lev=0):
        """q (u_E - u_W + v_N - v_S + w_T - w_B) of every cell, [k, j, i]."""
        N = self.N >> lev
        (u, v, w, p), xi = self.split(x, lev)
        return ((u[1:-1, 1:-1, 2:] - u[1:-1, 1:-1, 1:-1]) + (v[1:-1, 2:, 1:-1] - v[1:-1, 1:-1, 1:-1]) +
                (w[2:, 1:-1, 1:-1] - w[1:-1, 1:-1, 1:-1])) * N

    # ------------------------------------------------------------ relaxation
    def box_sweep(self, x, b, lev=0):
        """Seven colours of box relaxation (Sect. 4.1.1): each box solves its
        pressure and interior faces exactly, everything else frozen; the
        boxes of one colour are updated together from the same iterate."""
        x = x.copy()
        N = self.N >> lev
        h = 1.0 / N
        a, q = self.alpha / h ** 2, 1.0 / h
        d = 1.0 + 6.0 * a
        S = N + 2
        F = S ** 3
        t = self.types[lev]
        kk, jj, ii = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
        col = colour(ii, jj, kk)
        slot = lambda i, j, k: ((k + 1) * S + (j + 1)) * S + (i + 1)
        for c in range(NCOL):
            r, _ = self.residual(x, b, lev)
            I, J, K = ii[col == c], jj[col == c], kk[col == c]
            # box unknowns: faces W, E (u), S, N (v), B, T (w), then p
            fslots = [G_U * F + slot(I, J, K), G_U * F + slot(I + 1, J, K), G_V * F + slot(I, J, K),
                      G_V * F + slot(I, J + 1, K), G_W * F + slot(I, J, K), G_W * F + slot(I, J, K + 1)]
            tflat = t.reshape(-1)
            present = np.stack([tflat[fs] == INTERNAL for fs in fslots], axis=1)
            pslot = G_P * F + slot(I, J, K)
            sign = [1.0, -1.0, 1.0, -1.0, 1.0, -1.0]  # coefficient of p in the momentum row (+q for a face below)
            pat = present.dot(1 << np.arange(6))
            for pt in np.unique(pat):
                sel = pat == pt
                faces = [f for f in range(6) if (pt >> f) & 1]
                n = len(faces) + 1
                A = np.zeros((n, n))
                for r_, f in enumerate(faces):
                    A[r_, r_] = d
                    partner = f ^ 1
                    if partner in faces:
                        A[r_, faces.index(partner)] = -a
                    A[r_, n - 1] = sign[f] * q
                    A[n - 1, r_] = -sign[f] * q  # continuity: + q for the upper face, - q for the lower
                rows = [fslots[f][sel] for f in faces] + [pslot[sel]]
                R = np.stack([r[rw] for rw in rows])
                D = np.linalg.solve(A, R)
                for m, rw in enumerate(rows):
                    x[rw] += D[m]
        return x

    def scalar_update(self, x, b, lev=0):
        """xi <- mean(div u - b_c); then a uniform pressure shift makes the mean row exact."""
        x = x.copy()
        N = self.N >> lev
        h = 1.0 / N
        (u, v, w, p), xi = self.split(x, lev)
        (bu, bv, bw, bp), bm = self.split(b, lev)
        xi[0] = (self.div(x, lev) - bp[1:-1, 1:-1, 1:-1]).mean()
        p[1:-1, 1:-1, 1:-1] += (bm[0] - h ** 3 * p[1:-1, 1:-1, 1:-1].sum()) / (h ** 3 * N ** 3)
        return x

    def ghost_sweep(self, x, b, lev=0):
        """One Jacobi sweep w += dtau r over the wall and box-ghost rows (Eq. ghostrelax)."""
        x = x.copy()
        r, _ = self.residual(x, b, lev)
        S = (self.N >> lev) + 2
        tf = self.types[lev][:3].reshape(-1)
        m = np.zeros(x.size, bool)
        m[:3 * S ** 3] = (tf == WALL) | (tf == BOXGHOST)
        x[m] += self.dtau * r[m]
        return x

    def smooth(self, x, b, nu=1, lev=0):
        """Algorithm relax: nu times (box sweep, (xi, mean) update, lambda ghost sweeps)."""
        for _ in range(nu):
            x = self.box_sweep(x, b, lev)
            x = self.scalar_update(x, b, lev)
            for _ in range(self.lam):
                x = self.ghost_sweep(x, b, lev)
        return x

    # ------------------------------------------------------------ transfers
    @staticmethod
    def _cls(t):
        """restriction class: 1 interior, 2 wall or box ghost, 0 inactive"""
        return np.where(t == INTERNAL, 1, np.where((t == WALL) | (t == BOXGHOST), 2, 0))

    def restrict(self, r, lev=0):
        """Residual of level lev to the right-hand side of level lev + 1."""
        Nf = self.N >> lev
        Nc = Nf >> 1
        Sf, Sc = Nf + 2, Nc + 2
        (rf_u, rf_v, rf_w, rf_p), rf_m = self.split(r, lev)
        rfs = [rf_u, rf_v, rf_w, rf_p]
        out = np.zeros(self.n(lev + 1))
        (ou, ov, ow, op), om = self.split(out, lev + 1)
        outs = [ou, ov, ow, op]
        tf, tc = self.types[lev], self.types[lev + 1]
        rc = np.arange(Sc)  # coarse array index; coordinate = index - 1
        for g in range(4):
            cf, cc = self._cls(tf[g]), self._cls(tc[g])
            # per array axis [k, j, i]: fine offsets and weights of the stencil
            axes = []
            for ax in range(3):
                own = g < 3 and ax == 2 - g
                if own:
                    axes.append([(-1, 0.25), (0, 0.5), (1, 0.25)])  # faces 2O - 1, 2O, 2O + 1
                else:
                    axes.append([(0, 0.5), (1, 0.5)])  # cells 2T, 2T + 1
            acc_w = np.zeros((Sc, Sc, Sc))
            acc_s = np.zeros((Sc, Sc, Sc))
            cnt = np.zeros((Sc, Sc, Sc))
            allk = np.ones((Sc, Sc, Sc), bool)
            K, J, I = np.meshgrid(rc - 1, rc - 1, rc - 1, indexing="ij")
            C = [K, J, I]
            for ok, wk in axes[0]:
                for oj, wj in axes[1]:
                    for oi, wi in axes[2]:
                        fk, fj, fi = 2 * C[0] + ok, 2 * C[1] + oj, 2 * C[2] + oi
                        inn = (fk >= -1) & (fk <= Nf) & (fj >= -1) & (fj <= Nf) & (fi >= -1) & (fi <= Nf)
                        ak, aj, ai = np.clip(fk + 1, 0, Sf - 1), np.clip(fj + 1, 0, Sf - 1), np.clip(fi + 1, 0, Sf - 1)
                        cls_f = np.where(inn, cf[ak, aj, ai], -1)
                        val = rfs[g][ak, aj, ai]
                        same = inn & (cls_f == cc)
                        acc_w += np.where(same, wk * wj * wi * val, 0.0)
                        acc_s += np.where(same, val, 0.0)
                        cnt += same
                        allk &= same
            res = np.where(allk, acc_w, np.where(cnt > 0, acc_s / np.maximum(cnt, 1), 0.0))
            outs[g][...] = np.where(cc > 0, res, 0.0)
        om[0] = rf_m[0]
        return out

    @staticmethod
    def _taps(f, aligned, lo, hi):
        """Coarse nodes and weights interpolating fine index f along one axis:
        a face axis (aligned) or a cell-centred one, extrapolating past [lo, hi]."""
        if aligned:
            return [(f // 2, 1.0)] if f % 2 == 0 else [((f - 1) // 2, 0.5), ((f + 1) // 2, 0.5)]
        c = f / 2.0 - 0.25
        k0 = int(np.floor(c))
        k0 = min(max(k0, lo), hi - 1)
        w1 = c - k0
        return [(k0, 1.0 - w1), (k0 + 1, w1)]

    def prolong(self, eH, x, lev=0):
        """x + P eH on every active node of level lev (trilinear, renormalised)."""
        Nf = self.N >> lev
        Nc = Nf >> 1
        Sc = Nc + 2
        x = x.copy()
        (xu, xv, xw, xp), xxi = self.split(x, lev)
        xs = [xu, xv, xw, xp]
        (eu, ev, ew, ep), exi = self.split(eH, lev + 1)
        es = [eu, ev, ew, ep]
        tf, tc = self.types[lev], self.types[lev + 1]
        for g in range(4):
            actc = tc[g] != INACTIVE
            rng_f = [np.arange(-1, Nf + 1)] * 3
            taps = []
            for ax in range(3):
                own = g < 3 and ax == 2 - g
                if g == G_P:
                    lo, hi = 0, Nc - 1
                elif own:
                    lo, hi = 0, Nc
                else:
                    lo, hi = -1, Nc
                taps.append([self._taps(f, own, lo, hi) for f in range(-1, Nf + 1)])
            act = tf[g] != INACTIVE
            for ak in range(Nf + 2):
                for aj in range(Nf + 2):
                    for ai in range(Nf + 2):
                        if not act[ak, aj, ai]:
                            continue
                        s = ws = 0.0
                        for ck, wk in taps[0][ak]:
                            for cj, wj in taps[1][aj]:
                                for ci, wi in taps[2][ai]:
                                    if not (-1 <= ck <= Nc and -1 <= cj <= Nc and -1 <= ci <= Nc):
                                        continue
                                    if not actc[ck + 1, cj + 1, ci + 1]:
                                        continue
                                    w = wk * wj * wi
                                    s += w * es[g][ck + 1, cj + 1, ci + 1]
                                    ws += w
                        if ws > 0:
                            xs[g][ak, aj, ai] += s if ws == 1.0 else s / ws
        xxi[0] += exi[0]
        return x

    # ------------------------------------------------------------ coarsest, cycle, solve
    def assemble(self, lev):
        """Dense M of level lev, column c = M e_c (from the residual with b = 0)."""
        n = self.n(lev)
        M = np.zeros((n, n))
        z = np.zeros(n)
        for c in range(n):
            e = np.zeros(n)
            e[c] = 1.0
            M[:, c] = -self.residual(e, z, lev)[0]
        return M

    def coarse_solve(self, b):
        if self._coarse is None:
            self._coarse = self.assemble(self.levels - 1)
        return np.linalg.solve(self._coarse, b)

    def cycle(self, x, b, lev=0):
        """One V(nu1, nu2) cycle on level lev."""
        if lev == self.levels - 1:
            return self.coarse_solve(b)
        x = self.smooth(x, b, self.nu1, lev)
        r, _ = self.residual(x, b, lev)
        eH = self.cycle(np.zeros(self.n(lev + 1)), self.restrict(r, lev), lev + 1)
        x = self.prolong(eH, x, lev)
        return self.smooth(x, b, self.nu2, lev)

    def solve(self, x, b, tol, max_cycles=60):
        """Cycles until ||b - M x||_inf <= tol; returns (x, residual history)."""
        hist = [self.residual(x, b)[1]]
        for _ in range(max_cycles):
            if hist[-1] <= tol:
                break
            x = self.cycle(x, b)
            hist.append(self.residual(x, b)[1])
        return x, hist
