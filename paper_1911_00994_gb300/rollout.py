"""A rollout of Crank-Nicolson steps around a rigidly moving body and its
adjoint with checkpoints: the gradient of L = sum_k w_k (x^n_k)^2 (x^n the
state after the last step, w a weight vector on the finest vector layout)
with respect to the forcing f (the same field at every step) and the
amplitude of the body velocity.

Orchestration only: the geometry of every step (`geometry_build_shape`),
every forward step (`cn_step`, fixed Picard count for steps 0 and 1) and
every backward pass (`cn_step_adjoint`) run in the CUDA library.  The
forward pass keeps (x, N^(n-1), N^(n-2)) every `every` steps; the backward
pass recomputes each segment from its checkpoint, keeping the segment's
states, and runs the adjoint steps of the segment in reverse.
"""
from __future__ import annotations


class Rollout:
    def __init__(self, solver, shape, dt, Re, steps, kmax=4, tol=1e-11, every=10, walls=(0.0, 0.0, 0.0, 0.0)):
        """shape: keyword arguments of Solver.geometry_shape without t (kind,
        a, b, k, xc, yc, orbit_r, orbit_period, orbit_phase, omega); step m
        uses the geometry at t = (m + 1) dt."""
        self.s = solver
        self.shape = dict(shape)
        self.dt, self.Re, self.steps = dt, Re, steps
        self.kmax, self.tol, self.every = kmax, tol, max(1, every)
        self.walls = walls

    def _geometry(self, m):
        st, body = self.s.geometry_shape(t=(m + 1) * self.dt, **self.shape)
        if st:
            raise RuntimeError("geometry_build_shape failed: %s" % self.s.error())
        return body

    def _step(self, m, x, N1, N2, f, amp):
        body = self._geometry(m)
        bd = (amp * body[0], amp * body[1], amp * body[2], body[3], body[4])
        st, rep = self.s.cn_step(x, N1, N2, m, self.dt, self.Re, f=f, body=bd, walls=self.walls, tol=self.tol,
                                 eps=0.0, kmax=self.kmax)
        if st:
            raise RuntimeError("cn_step %d failed: %s" % (m, self.s.error()))

    def forward(self, f, amp, x0=None, checkpoints=None):
        """Run all steps from x0 (default: fluid at rest); returns the final
        state.  With a dict `checkpoints`, stores (x, N1, N2) at every
        multiple of `every`."""
        s = self.s
        x = s.new_vec() if x0 is None else x0.clone()
        N1, N2 = s.new_vec(), s.new_vec()
        for m in range(self.steps):
            if checkpoints is not None and m % self.every == 0:
                checkpoints[m] = (x.clone(), N1.clone(), N2.clone())
            self._step(m, x, N1, N2, f, amp)
        return x

    def vjp(self, f, amp, checkpoints, xbar):
        """Backward pass from the checkpoints of a forward run: given xbar =
        dL/dx_final, returns (dL/df, dL/damp, dL/dx0).  Each segment is
        recomputed from its checkpoint, then its adjoint steps run in
        reverse."""
        s = self.s
        xbar = xbar.clone()
        nb = [s.new_vec(), s.new_vec(), s.new_vec()]
        fbar = s.new_vec()
        abar = 0.0
        for a in reversed(sorted(checkpoints)):
            b = min(a + self.every, self.steps)
            xs = {}
            xc, n1, n2 = (t.clone() for t in checkpoints[a])
            for m in range(a, b):
                xs[m] = xc.clone()
                if m + 1 < b:
                    self._step(m, xc, n1, n2, f, amp)
            for m in reversed(range(a, b)):
                body = self._geometry(m)
                xbar_m = s.new_vec()
                abar += s.cn_step_adjoint(m, xs[m], self.dt, self.Re, xbar, xbar_m, nb, fbar, f=f, body=body,
                                          amp=amp, walls=self.walls, tol=self.tol, kmax=self.kmax)
                xbar = xbar_m
                nb = [nb[1], nb[2], s.new_vec()]
        return fbar, abar, xbar

    def loss_and_gradient(self, f, amp, w, x0=None):
        """(L, dL/df, dL/damp) for L = sum w x_final^2."""
        ck = {}
        x = self.forward(f, amp, x0, ck)
        loss = float((w * x * x).sum())
        fbar, abar, _ = self.vjp(f, amp, ck, 2.0 * w * x)
        return loss, fbar, abar
