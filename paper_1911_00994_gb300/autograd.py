"""torch.autograd.Function wrappers of one Crank-Nicolson step and of a
checkpointed rollout.

Forward passes call `cn_step` of the CUDA library; backward passes call
`cn_step_adjoint`, which solves the transposed ghost-point system
M^T lam = xbar with the transposed multigrid cycle (Sect. 4 read backwards:
transposed box solves, ghost sweeps and transfers) and applies the
transposed right-hand-side and convective Jacobians of Sect. 2 (Eqs. NSCN1,
extrUdU, NSitconv).  Nothing here computes: these classes marshal tensors
between torch's autograd and the C ABI.

Differentiated map of one step m (the geometry of step m + 1 fixed):

    (x^m, N^(m-1), N^(m-2), f, amp)  ->  (x^(m+1), N^m)

x are finest-level FP64 vectors in the library's layout, f the forcing on
the u, v frames, amp the amplitude of the rigid-body velocity on the object
(the box-wall velocities are not scaled), N^m = u.grad u of x^m the history
later steps extrapolate with.  Steps 0 and 1 run a fixed number `kmax` of
Picard iterations (no adaptive exit, so the map is smooth); later steps the
extrapolation N^m + N^(m-1)/2 - N^(m-2)/2.  Each solve runs to `tol`; the
gradients are those of the exact discrete map, up to that tolerance.
"""
from __future__ import annotations

import torch

from .gpmg import GpmgError


def _zeros_like_vec(solver, t):
    return t.contiguous() if t is not None else solver.new_vec()


class CNStep(torch.autograd.Function):
    """x_next, N_m = CNStep.apply(x, N1, N2, f, amp, solver, step, dt, Re,
    body, walls, tol, kmax, geometry)

    solver: a `gpmg.Solver` created with adjoint=True; body: the unscaled
    rigid-body velocity (U, V, omega, cx, cy) at t^(m+1); geometry: a
    callable that builds the geometry of step m + 1 on the solver (called
    before the forward step and again before the backward step, since other
    steps rebuild it in between), or None for a fixed geometry already
    built.  f may be None (no forcing; no gradient)."""

    @staticmethod
    def forward(ctx, x, N1, N2, f, amp, solver, step, dt, Re, body, walls, tol, kmax, geometry):
        if geometry is not None:
            geometry()
        a = float(amp)
        xn = x.detach().clone()
        n1 = N1.detach().clone()
        n2 = N2.detach().clone()
        fd = f.detach().contiguous() if f is not None else None
        bd = (a * body[0], a * body[1], a * body[2], body[3], body[4])
        st, rep = solver.cn_step(xn, n1, n2, step, dt, Re, f=fd, body=bd, walls=walls, tol=tol, eps=0.0,
                                 kmax=kmax)
        if st:
            raise GpmgError(st, "cn_step: %s" % solver.error())
        ctx.solver, ctx.step, ctx.dt, ctx.Re = solver, step, dt, Re
        ctx.body, ctx.walls, ctx.tol, ctx.kmax, ctx.geometry, ctx.amp = body, walls, tol, kmax, geometry, a
        ctx.has_f = f is not None
        ctx.save_for_backward(x.detach().clone(), fd)
        # after the step n1 holds N^m (the history rotates N2 <- N1 <- N^m)
        return xn, n1

    @staticmethod
    def backward(ctx, gx, gN):
        s = ctx.solver
        x_m, fd = ctx.saved_tensors
        if ctx.geometry is not None:
            ctx.geometry()
        xbar_next = _zeros_like_vec(s, gx)
        nb = [gN.contiguous().clone() if gN is not None else s.new_vec(), s.new_vec(), s.new_vec()]
        xbar_m, fbar = s.new_vec(), s.new_vec()
        abar = s.cn_step_adjoint(ctx.step, x_m, ctx.dt, ctx.Re, xbar_next, xbar_m, nb, fbar, f=fd, body=ctx.body,
                                 amp=ctx.amp, walls=ctx.walls, tol=ctx.tol, kmax=ctx.kmax)
        g_amp = torch.tensor(abar, dtype=torch.float64)
        return (xbar_m, nb[1], nb[2], fbar if ctx.has_f else None, g_amp,
                None, None, None, None, None, None, None, None, None)


class RolloutFn(torch.autograd.Function):
    """x_final = RolloutFn.apply(f, amp, x0, rollout)

    rollout: a `rollout.Rollout` (its solver created with adjoint=True).
    The forward pass stores (x, N^(m-1), N^(m-2)) every `rollout.every`
    steps; the backward pass recomputes each segment from its checkpoint and
    runs the segment's adjoint steps in reverse.  x0 may be None (fluid at
    rest)."""

    @staticmethod
    def forward(ctx, f, amp, x0, rollout):
        ck = {}
        fd = f.detach().contiguous()
        x = rollout.forward(fd, float(amp), None if x0 is None else x0.detach(), ck)
        ctx.rollout, ctx.ck, ctx.f, ctx.amp = rollout, ck, fd, float(amp)
        ctx.has_x0 = x0 is not None
        return x

    @staticmethod
    def backward(ctx, gx):
        ro = ctx.rollout
        fbar, abar, x0bar = ro.vjp(ctx.f, ctx.amp, ctx.ck, _zeros_like_vec(ro.s, gx))
        return fbar, torch.tensor(abar, dtype=torch.float64), (x0bar if ctx.has_x0 else None), None


def cn_step(x, N1, N2, f, amp, solver, step, dt, Re, body, walls=(0.0, 0.0, 0.0, 0.0), tol=1e-11, kmax=4,
            geometry=None):
    """Differentiable Crank-Nicolson step; returns (x^(m+1), N^m)."""
    if not torch.is_tensor(amp):
        amp = torch.tensor(float(amp), dtype=torch.float64)
    return CNStep.apply(x, N1, N2, f, amp, solver, step, dt, Re, tuple(body), tuple(walls), tol, kmax, geometry)


def rollout(f, amp, rollout_obj, x0=None):
    """Differentiable checkpointed rollout; returns the final state."""
    if not torch.is_tensor(amp):
        amp = torch.tensor(float(amp), dtype=torch.float64)
    return RolloutFn.apply(f, amp, x0, rollout_obj)
