#!/usr/bin/env python
"""Benchmark of the ghost-point multigrid solve of one Crank-Nicolson step.

Workload (lid-driven cavity around a steady flower): [0,1]^2 with N x N
cells (default 4096), flower r < 0.2 + 0.05 sin(5 theta) centred at
(0.5, 0.5), Re = 1000, dt = h (alpha = dt / (2 Re)), no-slip on the flower
and the walls, lid u = 1 at y = 1.  One step = the linear system of the first
Crank-Nicolson step from rest solved from a zero start to ||r||_inf <= 1e-10
by V(2,1) cycles.  The headline runs FP32 cycles inside FP64 residual
correction; the plain FP64 solve of the same system is timed in the same run.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
same system instead (one V-cycle per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-10 residual per CN step & MG cycles/s at 4096²; HBM GB/s % peak"
TOL = 1e-10


def workload(N):
    return {"workload": "lid-driven cavity %dx%d on [0,1]^2, steady flower r=0.2+0.05sin(5t) at (0.5,0.5), "
                        "Re=1000, dt=h; first CN step from rest, V(2,1) to ||r||_inf<=1e-10 from zero" % (N, N),
            "N": N, "Re": 1000.0, "dt": "h", "tol": TOL}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_sha1():
    """sha1 of the source of the roofline kernel (the box constants, the box
    solve and the streaming sweep in ops.cu): DRAM traffic measured by ncu
    stays valid while this text is unchanged."""
    src = open(os.path.join(ROOT, "paper_1911_00994_gb300", "csrc", "ops.cu")).read()
    parts = []
    a = src.index("template <typename T> struct BoxK")
    parts.append(src[a:src.index("template <typename T> struct LevelArgs", a)])
    a = src.index("template <typename T, bool ALL = false, typename View>")
    parts.append(src[a:src.index("// the same on frames of row pitch", a)])
    a = src.index("template <typename T> struct WaveGeom;")
    b = src.index("k_box_wave(", a)
    parts.append(src[a:src.index("\n}\n", b)])
    return hashlib.sha1("".join(parts).encode()).hexdigest()


def ncu_traffic(kernel, N):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source and on an N x N finest level."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        e = d.get(kernel)
        if e and e.get("kernel_source_sha1") == kernel_source_sha1() and e.get("N") == N:
            return e
    except Exception:
        pass
    return None


WAVE_MIN = 0  # gp_params.wave_min of every case (0: the library's default)


def build_case(N, precision, device, stream, levels=None, krylov=False, inner=0, gamma=1, alpha=None):
    import torch
    from paper_1911_00994_gb300 import gpmg
    from paper_1911_00994_gb300 import workloads as W
    h = 1.0 / N
    alpha = h / (2.0 * 1000.0) if alpha is None else alpha
    s = gpmg.Solver(N, 0.0, 0.0, 1.0, levels=levels, alpha=alpha, precision=precision, device=device,
                    max_cycles=200, stream=stream, krylov=krylov, inner=inner, gamma=gamma, wave_min=WAVE_MIN)
    phi = torch.from_numpy(W.phi_half_lattice(W.flower(0.2, 0.05, 5, 0.5, 0.5), N, 0.0, 0.0, 1.0)).to(device)
    st = s.geometry(phi, 0)
    if st:
        raise RuntimeError("geometry_build: " + s.error())
    b = s.new_vec()
    P = gpmg.pitch(N)
    # lid: box-ghost rows of u above the top wall carry u = 1
    b[(N + 1) * P + 2:(N + 1) * P + N + 1] = 1.0
    return s, b


def adjoint_rollout(dev, stream, steps=50, every=10, N=512, krylov=True):
    """Adjoint rollout of the orbiting circle (r = 0.25, orbit radius 0.2,
    period 1) at Re = 100 on [-1, 1]^2, a rollout of `steps` CN steps from
    rest, and the gradient of the kinetic energy on a 64 x 64 probe window
    (u and v nodes with array indices i in [352, 416), j in [224, 288)) with
    respect to the forcing (4 seeded Gaussian bumps, sigma = 0.1) and the
    body-velocity amplitude, checkpoints every `every` steps.  dt = 0.3 h:
    the paper bounds the step by h / max |u| and at dt = h the first steps'
    Picard iteration diverges.  The forward and adjoint solves use BiCGSTAB
    preconditioned by one (transposed) cycle unless `krylov` is false."""
    import numpy as np
    import torch
    from paper_1911_00994_gb300 import gpmg
    from paper_1911_00994_gb300 import workloads as W
    from paper_1911_00994_gb300.rollout import Rollout
    x0, L, Re = -1.0, 2.0, 100.0
    dt = 0.3 * L / N
    s = gpmg.Solver(N, x0, x0, L, alpha=dt / (2 * Re), band=3, adjoint=True, max_cycles=400, device=dev,
                    stream=stream, krylov=krylov)
    shape = dict(kind=gpmg.GP_CIRCLE, a=0.25, orbit_r=0.2, orbit_period=1.0)
    st, body = s.geometry_shape(t=0.0, **shape)
    if st:
        raise RuntimeError("geometry failed: %s" % s.error())
    t = s.types_flat()
    g, i, j, X, Y = W.flat_coords(N, x0, x0, L)
    rng = np.random.default_rng(1234)
    f = np.zeros(len(t))
    for _ in range(4):
        while True:
            c = rng.uniform(-0.9, 0.9, 2)
            if np.hypot(c[0], c[1]) > 0.55:  # outside the orbit's reach
                break
        amp = rng.standard_normal(2)
        bump = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2) / (2 * 0.1 ** 2))
        f += np.where(g == 0, amp[0] * bump, 0.0) + np.where(g == 1, amp[1] * bump, 0.0)
    f = np.where(((g == 0) | (g == 1)) & (t == 1), f, 0.0)
    w = (((g == 0) | (g == 1)) & (i >= 352) & (i < 416) & (j >= 224) & (j < 288)).astype(float)
    fd, wd = s.to_device(f), s.to_device(w)
    ro = Rollout(s, shape, dt, Re, steps, kmax=4, tol=1e-10, every=every)
    torch.cuda.synchronize(dev)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    ro.forward(fd, 1.0)
    e[1].record(stream)
    e[2].record(stream)
    loss, fbar, abar = ro.loss_and_gradient(fd, 1.0, wd)
    e[3].record(stream)
    torch.cuda.synchronize(dev)
    fw, gr = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    return {"N": N, "steps": steps, "checkpoint_every": every, "dt": "0.3h", "Re": Re,
            "solver": "BiCGSTAB, one (transposed) V(2,1) cycle per preconditioner" if krylov else "V(2,1) cycles",
            "forward_ms": fw,
            "loss_and_gradient_ms": gr, "gradient_over_forward": gr / fw, "loss": loss,
            "dL_damp": abar, "dL_df_norm": float(fbar.norm())}


def moving_ellipse(dev, stream, steps=20, warm=4, N=1024):
    """The moving ellipse with semi-axes 0.4 and 0.2 on
    [-1, 1]^2, translating on a circle of radius 0.3 with period 1, Re = 100,
    from rest; the ghost-point geometry is rebuilt every step.  dt = 0.3 h
    (the paper's time-step bound; see the rollout above).  BiCGSTAB
    preconditioned by one cycle (plain cycles diverge on this body's coarse
    levels), FP64 and mixed precision.  Per step: the geometry rebuild and
    the CN step (Picard for steps 0 and 1), timed on the host around
    synchronised calls, over `steps` steps after `warm`."""
    import torch
    from paper_1911_00994_gb300 import gpmg
    Re = 100.0
    dt = 0.3 * 2.0 / N
    shape = dict(kind=gpmg.GP_ELLIPSE, a=0.4, b=0.2, orbit_r=0.3, orbit_period=1.0)
    out = {"N": N, "steps": steps, "dt": "0.3h", "Re": Re, "solver": "BiCGSTAB, one V(2,1) cycle per preconditioner"}
    for name, prec in (("fp64", gpmg.GP_FP64), ("mixed", gpmg.GP_MIXED)):
        s = gpmg.Solver(N, -1.0, -1.0, 2.0, alpha=dt / (2 * Re), band=3, precision=prec, max_cycles=400,
                        device=dev, stream=stream, krylov=True)
        x, N1, N2 = s.new_vec(), s.new_vec(), s.new_vec()
        tg = ts = 0.0
        cyc = 0
        for m in range(warm + steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            st, body = s.geometry_shape(t=(m + 1) * dt, **shape)
            if st:
                raise RuntimeError("geometry failed: %s" % s.error())
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            st, rep = s.cn_step(x, N1, N2, m, dt, Re, body=body, tol=1e-10, eps=1e-6, kmax=4)
            if st:
                raise RuntimeError("cn_step %d failed: %s" % (m, s.error()))
            torch.cuda.synchronize(dev)
            t2 = time.perf_counter()
            if m >= warm:
                tg += t1 - t0
                ts += t2 - t1
                cyc += rep.cycles
        out[name] = {"geometry_ms": tg / steps * 1e3, "cn_step_ms": ts / steps * 1e3, "cycles_per_step": cyc / steps}
        del s
        torch.cuda.empty_cache()
    return out


def fp64_roofline(N, nres, res_ms, nbox, box_ms, dev, stream):
    """Achieved FP64 flop rates of the finest level's residual and full-box
    sweep against the device's FP64 FMA throughput (gp_fma_peak).  Flops
    counted from the formulas: a momentum row 9 (five-point Laplacian,
    pressure difference, b - A x), a continuity row 6, the mean-row sum 1:
    25 per cell for the residual; a full box about 70 (five rows 42, the
    Schur elimination and back substitution 28), one box per cell per sweep
    (five colour launches)."""
    from paper_1911_00994_gb300 import gpmg
    p64, p32 = gpmg.fma_peak(dev, stream)
    cells = float(N) * N
    out = {"peak_fp64_tflops": p64, "peak_fp32_tflops": p32,
           "peak_source": "measured by gp_fma_peak (FMA chains, an FMA = 2 flops)"}
    if nres:
        t = res_ms / nres
        ach = 25.0 * cells / (t / 1e3) / 1e12
        out["residual_fp64"] = {"kernel": "k_residual4<double, double> (finest level)", "avg_launch_ms": t,
                                "launches": nres, "achieved_tflops": ach, "frac": ach / p64,
                                "flops_per_cell": 25}
    if nbox:
        t = box_ms * 5.0 / nbox   # five colour launches per sweep
        ach = 70.0 * cells / (t / 1e3) / 1e12
        out["box_sweep_fp64"] = {"kernel": "k_box_full<double> (finest level, five colour launches)",
                                 "avg_sweep_ms": t, "launches": nbox, "achieved_tflops": ach, "frac": ach / p64,
                                 "flops_per_box": 70}
    return out


def cavity_cn_steps(dev, stream, N=4096, warm=10, steps=5):
    """Crank-Nicolson steps of the lid-driven cavity with the five-petal
    flower (the headline system's problem) at N^2, Re = 1000, dt = h, from
    rest: `warm` untimed steps (steps 0 and 1 by the mid-point Picard
    iteration, later ones extrapolated), then `steps` timed steps, each
    `cn_step` warm-started from the previous state with the extrapolated
    convective term, solved to ||r||_inf <= 1e-10.  FP64 and mixed.  The
    right-hand side work of a step (convective term and Eq. NSCN1's
    right-hand side, the same kernels cn_step launches) is timed apart on
    the same stream; the rest of the step is the solve."""
    import torch
    from paper_1911_00994_gb300 import gpmg
    Re, h = 1000.0, 1.0 / N
    dt = h
    out = {"N": N, "Re": Re, "dt": "h", "warm_steps": warm, "timed_steps": steps, "tol": TOL,
           "solver": "V(2,1) cycles"}
    for name, prec in (("mixed", gpmg.GP_MIXED), ("fp64", gpmg.GP_FP64)):
        s, _ = build_case(N, prec, dev, stream)
        walls = (0.0, 1.0, 0.0, 0.0)
        x, N1, N2 = s.new_vec(), s.new_vec(), s.new_vec()
        for m in range(warm):
            st, rep = s.cn_step(x, N1, N2, m, dt, Re, walls=walls, tol=TOL, eps=1e-6, kmax=10)
            if st:
                raise RuntimeError("cavity cn_step %d: %s" % (m, s.error()))
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cyc = 0
        for m in range(warm, warm + steps):
            st, rep = s.cn_step(x, N1, N2, m, dt, Re, walls=walls, tol=TOL, eps=1e-6, kmax=10)
            if st:
                raise RuntimeError("cavity cn_step %d: %s" % (m, s.error()))
            cyc += rep.cycles
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        # the right-hand side work of one extrapolated step, on its own
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(steps):
            Nn = s.convective(x)
            b = s.cn_rhs(x, Nn, dt, walls=walls)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        rhs_ms = f0.elapsed_time(f1) / steps
        out[name] = {"cn_step_ms": ms, "rhs_ms": rhs_ms, "solve_ms": ms - rhs_ms, "cycles_per_step": cyc / steps,
                     "cycles_per_s": cyc / steps / (ms / 1e3)}
        del s, x, N1, N2
        torch.cuda.empty_cache()
    return out


def accuracy_study(Ns=(60, 120), T=0.5):
    """The six tests of Sect. 5.1 (Eq. sol:exa, Re = 100, the bodies of
    Eq. domains steady and turned at omega = 2 pi / 5) on a short horizon:
    L^1 (mean) and L^inf errors of u, v and div u at t = T and the observed
    orders.  The paper reports t = 10; there the central convective term
    (reading C18) goes unstable where the exact solution flows out through
    the body at cell Peclet numbers above 2, so the numbers here are not the
    paper's, which are given beside them as context.  BiCGSTAB solves (plain
    cycles diverge on the thin ellipse's coarse levels), tol 1e-9."""
    from paper_1911_00994_gb300.accuracy import AccuracyRun
    m = math
    with open(os.path.join(ROOT, "tests", "golden", "accuracy_tables.json")) as fh:
        paper = json.load(fh)
    out = {"T": T, "Re": 100.0, "dt": "h / (4 sqrt 2)", "N": list(Ns), "paper_t": 10.0, "tests": {}}
    for shape in ("circle", "ellipse", "flower"):
        for moving in (False, True):
            name = ("moving_" if moving else "steady_") + shape
            res = {}
            for N in Ns:
                t0 = time.perf_counter()
                r = AccuracyRun(N, shape, omega=2 * m.pi / 5 if moving else 0.0, T=T, tol=1e-9, krylov=True)
                r.run()
                e = r.errors()
                res[str(N)] = {"u": e["u"], "v": e["v"], "div": e["div"], "steps": r.steps,
                               "seconds": time.perf_counter() - t0}
            a, b = str(Ns[0]), str(Ns[-1])
            orders = {q: [m.log(res[a][q][k] / res[b][q][k]) / m.log(Ns[-1] / Ns[0]) for k in range(2)]
                      for q in ("u", "v", "div")}
            out["tests"][name] = {"errors": res, "orders": orders, "paper_t10_N60": paper[name]["errors"]["60"]}
    return out


def mac3d_box(dev, stream, N=256, steps=3):
    """The 3-D MAC extension on the box [0, 1]^3 (walls only): FP64 V(2,1)
    cycles to ||r||_inf <= 1e-10 from zero, the right-hand side seeded
    normals on the interior momentum and continuity rows; the 7-colour box
    relaxation of the finest level timed per launch."""
    import numpy as np
    import torch
    from paper_1911_00994_gb300 import mac3d
    levels = 1
    while (N >> levels) >= 4 and 4 * ((N >> levels) + 2) ** 3 + 1 > 1024:
        levels += 1
    levels += 1
    h = 1.0 / N
    alpha = h / (2.0 * 1000.0)  # Re = 1000, dt = h
    s = mac3d.Solver3D(N, levels, alpha, device=dev, stream=stream)
    S = N + 2
    F = S ** 3
    t = s.types(0)
    rng = np.random.default_rng(0)
    b = np.zeros(mac3d.plain_len(N))
    act = t == 1
    b[:4 * F][act] = rng.standard_normal(int(act.sum()))
    bg = s.to_device(b)
    x = s.new_vec()
    st, cyc, res, hist = s.solve(x, bg, 1e-10, 200)
    if st:
        return {"N": N, "status": "failed: " + s.error()}
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cycles = 0
    for _ in range(steps):
        x.zero_()
        st, cyc, res, hist = s.solve(x, bg, 1e-10, 200)
        cycles += cyc
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    s.timer_start(0)
    x.zero_()
    s.solve(x, bg, 1e-10, 200)
    nbox, box_ms = s.timer_stop()
    # the same system with FP32 cycles (up to four) inside FP64 residual correction
    del s
    torch.cuda.empty_cache()
    sm = mac3d.Solver3D(N, levels, alpha, precision=1, inner=4, device=dev, stream=stream)
    xm = sm.new_vec()
    stm, cm, rm, hm = sm.solve(xm, bg, 1e-10, 200)
    e0.record(stream)
    mcyc = 0
    for k in range(steps):
        xm.zero_()
        if k == 0:
            torch.cuda.nvtx.range_push("mac3d_mixed")  # the launch list's range (host marker only)
        stm, cm, rm, hm = sm.solve(xm, bg, 1e-10, 200)
        if k == 0:
            torch.cuda.nvtx.range_pop()
        mcyc += cm
    e1.record(stream)
    torch.cuda.synchronize(dev)
    mixed = {"time_to_tol_ms": e0.elapsed_time(e1) / steps, "cycles_per_step": mcyc / steps,
             "corrections_per_step": len(hm) - 1, "status": "ok" if stm == 0 else "failed: " + sm.error()}
    sm.timer_start(0)
    xm.zero_()
    sm.solve(xm, bg, 1e-10, 200)
    nboxf, boxf_ms = sm.timer_stop()
    mixed["box_sweep_fp32_ms"] = 7.0 * boxf_ms / max(1, nboxf)
    mixed["box_sweep_fp32_gbs"] = N ** 3 * (12 * 4 + 4.0) / (mixed["box_sweep_fp32_ms"] / 1e3) / 1e9
    del sm
    hbm, src = peaks()
    sweep_ms = 7.0 * box_ms / max(1, nbox)
    # algorithmic bytes of one seven-colour sweep: per cell read x and b (4
    # words each) and the four type bytes, write x (4 words), FP64
    sweep_bytes = N ** 3 * (12 * 8 + 4.0)
    rho = float((hist[-1] / hist[max(0, len(hist) - 5)]) ** (1.0 / min(4, len(hist) - 1))) if len(hist) > 1 else None
    # FP64 flops of a box, counted from the formulas (an FMA = 2): six momentum
    # rows of 11 (seven-point Laplacian, pressure difference, b - A x), the
    # continuity row 9, the elimination and back substitution about 60
    from paper_1911_00994_gb300 import gpmg
    p64, _ = gpmg.fma_peak(dev, stream)
    ach = 135.0 * N ** 3 / (sweep_ms / 1e3) / 1e12
    return {"N": N, "unknowns": int((t != 0).sum()) + 1, "levels": levels, "Re": 1000.0, "dt": "h",
            "precision": "fp64", "cycle": "V(2,1)", "mixed": mixed, "time_to_tol_ms": ms, "cycles_per_step": cycles / steps,
            "cycles_per_s": cycles / steps / (ms / 1e3), "rho_last4": rho,
            "box_sweep": {"kernel": "k3_box (seven colour launches)", "ms_per_sweep": sweep_ms,
                          "achieved_gbs": sweep_bytes / (sweep_ms / 1e3) / 1e9,
                          "frac_of_hbm": sweep_bytes / (sweep_ms / 1e3) / 1e9 / hbm,
                          "algorithmic_bytes_per_sweep": sweep_bytes, "flops_per_box": 135,
                          "achieved_fp64_tflops": ach, "frac_of_fp64_peak": ach / p64,
                          "fp64_peak_tflops": p64}}


def largest_solve(dev, stream, N=8192, steps=2):
    """The largest single solve: the seven-petal flower
    r = 0.5 + 0.1 sin(7 theta) on [-1, 1]^2 at 8192^2 (201 M unknowns),
    Re = 500, dt = h, the CN system of a seeded divergence-free velocity of
    amplitude 0.1 (explicit convective term), solved to ||r||_inf <= 1e-10
    from that velocity.  BiCGSTAB preconditioned by one cycle (plain cycles
    diverge on this body's coarse levels): the mixed path next to the FP64
    path, one untimed solve each, then `steps` timed."""
    import torch
    from paper_1911_00994_gb300 import gpmg
    from paper_1911_00994_gb300 import workloads as W
    x0, L, Re = -1.0, 2.0, 500.0
    dt = L / N
    nU, nV, nP, n = W.flat_sizes(N)
    out = {"N": N, "unknowns": n, "Re": Re, "dt": "h",
           "solver": "BiCGSTAB, one V(2,1) cycle per preconditioner", "steps": steps}
    b = xn = None
    for name, prec in (("mixed", gpmg.GP_MIXED), ("fp64", gpmg.GP_FP64)):
        s = gpmg.Solver(N, x0, x0, L, alpha=dt / (2 * Re), precision=prec, krylov=True, max_cycles=200,
                        device=dev, stream=stream)
        st, body = s.geometry_shape(kind=gpmg.GP_FLOWER, a=0.5, b=0.1, k=7)
        if st:
            raise RuntimeError("geometry failed: %s" % s.error())
        if b is None:
            xn = W.div_free_device(N, x0, L, gpmg.pitch(N), seed=5, amp=0.1, device=dev)
            b = s.cn_rhs(xn, s.convective(xn), dt)
        x = xn.clone()
        s.solve(x, b, TOL, hist=False)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cyc = 0
        for _ in range(steps):
            x.copy_(xn)
            st, rep, _ = s.solve(x, b, TOL, hist=False)
            if st:
                raise RuntimeError("8192^2 flower solve failed: %s" % s.error())
            cyc += rep.cycles
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"time_to_tol_ms": ms, "cycles_per_step": cyc / steps, "cycles_per_s": cyc / steps / (ms / 1e3)}
        del s, x
        torch.cuda.empty_cache()
    return out


def cycle_ablation(dev, stream, tol, barrier, cases=((256, 8.0), (1024, 0.512), (4096, 2.048))):
    """V(2,1) against W(2,1) cycles (the W-cycle is the one the paper adopts,
    Sect. 4, and its convergence factor is reported for W-cycles, Sect. 5), both
    mixed precision, on the cavity-with-flower system at N^2 with
    alpha / h^2 as given (1024^2 and 4096^2: Re = 1000, dt = h): cycles, the
    geometric-mean residual reduction per cycle and the time to the tolerance
    (the second of two solves), or the failure.  A W-cycle visits level l
    2^l times, so its coarse levels cost far more launches."""
    import torch
    from paper_1911_00994_gb300 import gpmg
    out = []
    for N, ah2 in cases:
        row = {"N": N, "alpha_over_h2": ah2}
        for name, gamma in (("V", 1), ("W", 2)):
            s, b = build_case(N, gpmg.GP_MIXED, dev, stream, gamma=gamma, alpha=ah2 / N ** 2)
            x = s.new_vec()
            st, rep, _ = s.solve(x, b, tol, hist=False)
            r = {"levels": s.levels}
            if st == 0:
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                x.zero_()
                e0.record(stream)
                st, rep, _ = s.solve(x, b, tol, hist=False)
                e1.record(stream)
                barrier()
                r["time_to_tol_ms"] = e0.elapsed_time(e1)
            else:
                # every replica solves the same system, so all of them take this branch
                barrier()
                barrier()
            r.update({"status": "ok" if st == 0 else "failed: %s" % s.error(), "cycles": rep.cycles,
                      "rho": rep.rho if math.isfinite(rep.rho) else None})
            row[name] = r
            del s
            torch.cuda.empty_cache()
        out.append(row)
    return out


def combine_over_ranks(ms, cycles, device, dist):
    """Timing of a replicated run (one independent solve per rank): the
    slowest rank's time and the cycles of all ranks, on every rank."""
    if not dist:
        return ms, float(cycles)
    import torch
    import torch.distributed as tdist
    tmax = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    tsum = torch.tensor([float(cycles)], dtype=torch.float64, device=device)
    tdist.all_reduce(tmax, op=tdist.ReduceOp.MAX)
    tdist.all_reduce(tsum, op=tdist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0])


def run_ours(args):
    import numpy as np
    import torch
    from paper_1911_00994_gb300 import gpmg

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N = args.N
    gpmg.lib()

    def barrier():
        if dist:
            import torch.distributed as tdist
            tdist.barrier()
        torch.cuda.synchronize(dev)

    # ---- mixed precision (headline); the solver runs on its own stream so that
    # each multigrid iteration is replayed as a captured CUDA graph
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    s, b = build_case(N, gpmg.GP_MIXED, dev, stream)
    x = s.new_vec()
    for _ in range(args.warmup):
        x.zero_()
        st, rep, _ = s.solve(x, b, TOL, hist=False)
        if st:
            raise RuntimeError("warm-up solve failed: %s" % s.error())
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    l0 = s.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    cycles, iters = 0, 0
    rhos = []
    for _ in range(args.steps):
        x.zero_()
        st, rep, _ = s.solve(x, b, TOL, hist=False)
        if st:
            raise RuntimeError("solve failed: %s" % s.error())
        cycles += rep.cycles
        iters += rep.iterations
        rhos.append(rep.rho)
    e1.record(stream)
    barrier()
    torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    launches = s.launch_count() - l0
    clocks = sampler.stop()
    # the dominant kernel, timed with CUDA events around each of its launches
    # over a second pass of the same steps (the event timer replaces graph
    # replay with direct launches; the kernels are the same)
    s.timer_start("box_full", 0)
    for _ in range(args.steps):
        x.zero_()
        s.solve(x, b, TOL, hist=False)
    nbox, box_ms = s.timer_stop()
    ms_all, cycles_all = combine_over_ranks(ms, cycles, dev, dist)
    value = cycles_all / (ms_all / 1e3)

    # ---- end to end through the public API with host buffers: every step
    # copies its input (the right-hand side b) from pinned host memory, solves
    # from a zero iterate (zeroed on the device, as a caller solving from zero
    # would) and reads its solution back.  Serial: copy, solve, copy on one
    # stream.  Pipelined (the `e2e` figure): the copies run on a second stream
    # through double-buffered device staging vectors, so that step k + 1's
    # input arrives and step k's solution leaves while the GPU solves step k;
    # the solver's own b is filled from the staging vector on the device.
    b_host = b.cpu().pin_memory()
    out_host = [torch.empty(s.vec_len(), dtype=torch.float64).pin_memory() for _ in range(2)]
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    scycles = 0
    for _ in range(args.steps):
        b.copy_(b_host, non_blocking=True)
        x.zero_()
        st, rep, _ = s.solve(x, b, TOL, hist=False)
        scycles += rep.cycles
        out_host[0].copy_(x, non_blocking=True)
    f1.record(stream)
    barrier()
    serial_ms = f0.elapsed_time(f1)

    cs = torch.cuda.Stream(dev)
    sb = [torch.empty_like(b) for _ in range(2)]
    so = [torch.empty_like(x) for _ in range(2)]
    ev_in, ev_used, ev_out, ev_sent = ([torch.cuda.Event() for _ in range(2)] for _ in range(4))

    def send(k):
        i = k % 2
        with torch.cuda.stream(cs):
            if k >= 2:
                cs.wait_event(ev_used[i])
            sb[i].copy_(b_host, non_blocking=True)
            ev_in[i].record(cs)

    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_e2e0 = time.perf_counter()
    f0.record(stream)
    cs.wait_event(f0)
    send(0)
    ecycles = 0
    for k in range(args.steps):
        i = k % 2
        if k + 1 < args.steps:
            send(k + 1)
        stream.wait_event(ev_in[i])
        b.copy_(sb[i], non_blocking=True)
        x.zero_()
        ev_used[i].record(stream)
        st, rep, _ = s.solve(x, b, TOL, hist=False)
        if st:
            raise RuntimeError("e2e solve failed: %s" % s.error())
        ecycles += rep.cycles
        if k >= 2:
            stream.wait_event(ev_sent[i])
        so[i].copy_(x, non_blocking=True)
        ev_out[i].record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_out[i])
            out_host[i].copy_(so[i], non_blocking=True)
            ev_sent[i].record(cs)
    stream.wait_stream(cs)
    f1.record(stream)
    barrier()
    e2e_ms = f0.elapsed_time(f1)
    e2e = {"value": ecycles / (e2e_ms / 1e3), "unit": "V-cycles/s",
           "h2d_bytes_per_step": 8 * s.vec_len(), "d2h_bytes_per_step": 8 * s.vec_len(),
           "ms_per_step": e2e_ms / args.steps, "host_wall_s": time.perf_counter() - t_e2e0,
           "copies": "pinned host buffers, second stream, double-buffered device staging (overlapped with the solve)",
           "serial": {"value": scycles / (serial_ms / 1e3), "ms_per_step": serial_ms / args.steps,
                      "copies": "same stream, before and after each solve"}}
    del sb, so

    levels = s.levels
    del s
    torch.cuda.empty_cache()
    # ---- BiCGSTAB preconditioned by one mixed-precision cycle, same system
    sk, bk = build_case(N, gpmg.GP_MIXED, dev, stream, krylov=True)
    xk = sk.new_vec()
    for _ in range(max(1, args.warmup // 2)):
        xk.zero_()
        sk.solve(xk, bk, TOL, hist=False)
    barrier()
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    kc, kit = 0, 0
    nk = max(1, min(args.steps, 5))
    for _ in range(nk):
        xk.zero_()
        st, repk, _ = sk.solve(xk, bk, TOL, hist=False)
        if st:
            raise RuntimeError("krylov solve failed: %s" % sk.error())
        kc += repk.cycles
        kit += repk.iterations
    k1.record(stream)
    barrier()
    msk = k0.elapsed_time(k1)
    del sk
    # ---- plain FP64 solve of the same system
    torch.cuda.empty_cache()
    s64, b64 = build_case(N, gpmg.GP_FP64, dev, stream)
    x64 = s64.new_vec()
    for _ in range(max(1, args.warmup // 2)):
        x64.zero_()
        s64.solve(x64, b64, TOL, hist=False)
    barrier()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(s64.stream)
    c64 = 0
    n64 = max(1, min(args.steps, 3))
    for _ in range(n64):
        x64.zero_()
        st, rep64, _ = s64.solve(x64, b64, TOL, hist=False)
        if st:
            raise RuntimeError("fp64 solve failed: %s" % s64.error())
        c64 += rep64.cycles
    g1.record(s64.stream)
    barrier()
    ms64 = g0.elapsed_time(g1)
    # the FP64 kernels against the FP64 arithmetic ceiling: the finest level's
    # residual (25 flops per cell) and full-box colour sweeps (about 70 flops
    # per box), CUDA events around every launch of one more solve
    s64.timer_start("residual", 0)
    x64.zero_()
    s64.solve(x64, b64, TOL, hist=False)
    nres64, res64_ms = s64.timer_stop()
    s64.timer_start("box_full", 0)
    x64.zero_()
    s64.solve(x64, b64, TOL, hist=False)
    nbox64, box64_ms = s64.timer_stop()
    del s64
    torch.cuda.empty_cache()
    # ---- the mixed solve with one FP32 cycle per FP64 residual correction
    s1, b1 = build_case(N, gpmg.GP_MIXED, dev, stream, inner=1)
    x1 = s1.new_vec()
    for _ in range(max(1, args.warmup // 2)):
        x1.zero_()
        s1.solve(x1, b1, TOL, hist=False)
    barrier()
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    c1, it1 = 0, 0
    n1 = max(1, min(args.steps, 3))
    for _ in range(n1):
        x1.zero_()
        st, rep1, _ = s1.solve(x1, b1, TOL, hist=False)
        if st:
            raise RuntimeError("mixed solve (one cycle per correction) failed: %s" % s1.error())
        c1 += rep1.cycles
        it1 += rep1.iterations
    h1.record(stream)
    barrier()
    ms1 = h0.elapsed_time(h1)
    del s1
    torch.cuda.empty_cache()
    wcy = cycle_ablation(dev, stream, TOL, barrier) if not args.no_wcycle else None
    adj = adjoint_rollout(dev, stream) if not args.no_adjoint else None
    mov = moving_ellipse(dev, stream, steps=args.moving_steps, warm=args.moving_warm) if not args.no_moving else None
    big = largest_solve(dev, stream) if not args.no_large else None
    m3d = mac3d_box(dev, stream, N=args.n3d) if not args.no_3d else None
    cav = cavity_cn_steps(dev, stream, N=N) if not args.no_cavity else None
    acc = accuracy_study() if args.accuracy else None

    if rank != 0:
        if dist:
            import torch.distributed as tdist
            tdist.destroy_process_group()
        return None

    hbm, src = peaks()
    # algorithmic bytes of one launch of the FP32 streaming full-box sweep
    # (all five colours): per cell of the N x N grid, read x and b (3 words
    # each) and the box-code byte, write x (3 words)
    bytes_per_launch = N * N * (9 * 4 + 1.0)
    avg_ms = box_ms / max(1, nbox)
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    # levels from 4096^2 (or --wave-min) stream down strips of rows, smaller ones use tiles
    wmin = WAVE_MIN if WAVE_MIN != 0 else 4096
    roof_kernel = "k_box_wave<float>" if 0 <= wmin <= N else "k_box_tma<float>"
    tr = ncu_traffic(roof_kernel, N)
    line = {
        "metric": METRIC, "value": value, "unit": "V-cycles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(workload(N), precision="fp32 V-cycles in fp64 residual correction (up to 8 per correction)",
                       levels=levels,
                       l2="inputs larger than L2 (each vector %.0f MB)" % (8 * gpmg.vec_len(N) / 1e6),
                       parallelism="replicas" if world > 1 else "single GPU"),
        "time_to_tol_ms": ms_all / args.steps, "cycles_per_step": cycles / args.steps,
        "rho_mean": float(np.mean(rhos)),
        "fp64": {"time_to_tol_ms": ms64 / n64, "cycles_per_step": c64 / n64, "cycles_per_s": c64 / (ms64 / 1e3),
                 "steps": n64},
        "fp64_roofline": fp64_roofline(N, nres64, res64_ms, nbox64, box64_ms, dev, stream),
        "corrections_per_step": iters / args.steps,
        "mixed_one_cycle_per_correction": {"time_to_tol_ms": ms1 / n1, "cycles_per_step": c1 / n1,
                                           "corrections_per_step": it1 / n1, "cycles_per_s": c1 / (ms1 / 1e3),
                                           "steps": n1},
        "v_and_w_cycles_flower_cavity": wcy,
        "bicgstab_mixed": {"time_to_tol_ms": msk / nk, "iterations_per_step": kit / nk, "cycles_per_step": kc / nk,
                           "cycles_per_s": kc / (msk / 1e3), "steps": nk},
        "adjoint_rollout_orbiting_circle_512": adj,
        "moving_ellipse_1024": mov,
        "largest_solve_flower7_8192": big,
        "mac3d_box": m3d,
        "cavity_cn_steps": cav,
        "accuracy_sol_exa": acc,
        "roofline": {"kernel": roof_kernel + " (finest-level full-box sweep, five colours in one pass)",
                     "bound": "hbm",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "peak_source": src, "avg_launch_ms": avg_ms, "launches": nbox,
                     "timing": "CUDA events on the solver stream around every launch, second pass of the timed steps",
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "traffic": tr["bytes_per_launch"] if tr else None},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(N)
    print(json.dumps(line), flush=True)
    return line


def _oracle_case(N, threads=1):
    """The oracle on the benchmark's system (geometry built, lid right-hand
    side), with `threads` host threads (the OpenMP build when > 1)."""
    import numpy as np

    import oracle as O
    from paper_1911_00994_gb300 import workloads as W
    h = 1.0 / N
    lev = 1
    while (N >> lev) >= 16:
        lev += 1
    o = O.Oracle(N, 0.0, 0.0, 1.0, lev, h / 2000.0, threads=threads)
    st = o.geometry(W.phi_half_lattice(W.flower(0.2, 0.05, 5, 0.5, 0.5), N, 0.0, 0.0, 1.0))
    if st:
        return o, None
    b = np.zeros(o.n())
    g, i, j, X, Y = W.flat_coords(N, 0.0, 0.0, 1.0)
    t = o.types()
    b[(g == 0) & (j == N) & (t == W.BOXGHOST)] = 1.0
    return o, b


def cpu_baseline(N):
    """The oracle, as it stands, timed on the host: one V-cycle of the same
    system (geometry built outside the timed region), on every host core (the
    OpenMP build: boxes of one colour and row-wise loops in parallel, same
    iterate as one thread), and on one thread."""
    import numpy as np
    cores = os.cpu_count() or 1
    out = None
    for threads in ((cores, 1) if cores > 1 else (1,)):
        o, b = _oracle_case(N, threads)
        if b is None:
            return {"value": None, "error": o.error()}
        x = np.zeros_like(b)
        t0 = time.perf_counter()
        st, x = o.cycle(x, b)
        dt = time.perf_counter() - t0
        entry = {"value": 1.0 / dt, "unit": "V-cycles/s", "cores": o.threads, "kind": "oracle",
                 "sample": "one V(2,1) cycle of the %dx%d system from zero (FP64, %d thread%s; geometry excluded)"
                           % (N, N, o.threads, "s" if o.threads > 1 else ""),
                 "seconds": dt}
        if out is None:
            out = entry
        else:
            out["single_thread"] = entry
    return out


def run_reference(args):
    """--impl reference: the CPU oracle on the same system, one V-cycle per
    step, on every host core (the OpenMP build)."""
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    N = args.N
    o, b = _oracle_case(N, os.cpu_count() or 1)
    if b is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle geometry failed: " + o.error()}))
        return None
    x = np.zeros_like(b)
    for _ in range(args.warmup):
        st, x = o.cycle(x, b)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st, x = o.cycle(x, b)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "V-cycles/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload(N),
            "cpu_baseline": {"value": value, "unit": "V-cycles/s", "cores": o.threads, "kind": "oracle",
                             "sample": "one V(2,1) cycle per step of the %dx%d system (FP64, %d host threads)"
                                       % (N, N, o.threads)},
            "e2e": {"value": value, "unit": "V-cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-moving", action="store_true")
    ap.add_argument("--moving-steps", type=int, default=20, help="timed steps of the moving ellipse (the config: 200)")
    ap.add_argument("--moving-warm", type=int, default=4, help="untimed steps before them (the config: 0, from rest)")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3-D box-domain solve")
    ap.add_argument("--n3d", type=int, default=256, help="cells per side of the 3-D box-domain solve")
    ap.add_argument("--no-wcycle", action="store_true")
    ap.add_argument("--no-cavity", action="store_true")
    ap.add_argument("--accuracy", action="store_true", help="add the Sect. 5.1 accuracy study (about 3.5 min)")
    ap.add_argument("--wave-min", type=int, default=0,
                    help="smallest level swept down strips of rows (gp_params.wave_min; 0: library default)")
    args = ap.parse_args()
    global WAVE_MIN
    WAVE_MIN = args.wave_min
    if args.impl == "reference":
        args.steps = 2 if args.steps is None else args.steps
        args.warmup = 1 if args.warmup is None else args.warmup
        run_reference(args)
    else:
        args.steps = 10 if args.steps is None else args.steps
        args.warmup = 3 if args.warmup is None else args.warmup
        run_ours(args)


if __name__ == "__main__":
    main()
