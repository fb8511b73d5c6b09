"""Throughput of the micro-macro parareal hot path on GB300.

One step = one parareal iteration of the double-well workload (2^20
particles, 50 slices x 1000 Euler-Maruyama steps, FP32 state, 512 bins):
fine propagation of every slice with the matching fused into its prologue
and the restriction into its epilogue, the coarse propagator on all start
states, and the serial quantile-iterator update.  `value` is particle-steps
per second over the whole job (all ranks); ranks are independent replicas.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--legs a,b|all] [--legs-out FILE]

The last stdout line is one compact JSON object (under 1 KB): the headline,
the dominant kernel's roofline, the end-to-end figure through the C ABI with
host buffers, the CPU oracle baseline, clocks, and three scalars (binary32
over FP64 fine-kernel rate, iterations and time to W1 <= 1e-3).  Side legs
(the other workloads, standalone passes, studies) run only when named with
--legs; each prints one JSON line {"leg": name, ...} to stderr, and
--legs-out writes every figure into one JSON file.

`--impl reference` times the FP64 CPU oracle (the only reference this method
has) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "fine-propagator particle-steps/s (FP32 vs FP64 GPU) and parareal iter time at W1≤1e-3"
UNIT = "particle-steps/s"
WORKLOAD = workloads.DOUBLE_WELL
# Thread-instructions per particle-step of the binary32 fine kernel (d = 1,
# 4 particles per thread): ncu smsp__inst_executed.sum x 32 over the
# particle-steps of the launch, double-well workload at 2^16 and at 2^20
# particles x 9 slices x 1000 steps (the same count at both sizes).
INST_PER_PARTICLE_STEP = 41.58
# DRAM bytes per particle per slice of that kernel, read + write (ncu
# dram__bytes_read.sum + dram__bytes_write.sum of the 9-slice launch at 2^21
# particles, inputs larger than L2, scaled by particle-slices to the full
# launch); the algorithmic figure is
# 16 B (x and y read once and written once, binary32).
TRAFFIC_BYTES_PER_PARTICLE_SLICE = 13.75
SMS = 152
ISSUE_LANES_PER_SM_CLK = 4 * 32       # 4 sub-partitions x one 32-wide warp instruction per clock


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    from paper_1912_09240_gb300.replicas import rank_env
    return rank_env()


def _cpu_sample(seconds_target: float = 12.0, detail: bool = False):
    """Time the oracle on a bounded sample of the double-well workload on
    this machine's host cores (all of them).  With `detail`, also at one
    core, one slice of the 16-dimensional fast space at 2^16 particles, and
    the plain FP64 workload's whole parareal run."""
    from oracle import oracle as orc
    orc.build()
    w = WORKLOAD
    om = orc.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    x0, y0 = workloads.initial_ensemble(w)
    cores = orc.num_threads()

    def rate_of(n_max, target):
        # calibrate on a small sample, then size the timed sample to ~target seconds
        n_cal, s_cal = 1 << 12, 100
        t0 = time.perf_counter()
        orc.fine_propagate(om, w.seed, x0[None, :n_cal], y0[None, :, :n_cal], 1, s_cal, w.step_dt)
        rate = n_cal * s_cal / max(time.perf_counter() - t0, 1e-6)
        n = int(min(n_max, max(1 << 12, rate * target / w.steps)))
        # all particles and still short of the target: several slices
        nsl = max(1, min(w.K - 1, int(rate * target / (n * w.steps) + 0.5)))
        xs = np.ascontiguousarray(np.broadcast_to(x0[:n], (nsl, n)))
        ys = np.ascontiguousarray(np.broadcast_to(y0[:, :n], (nsl, w.fast_dim, n)))
        t0 = time.perf_counter()
        orc.fine_propagate(om, w.seed, xs, ys, 1, w.steps, w.step_dt)
        el = time.perf_counter() - t0
        return nsl * n * w.steps / el, n, el, nsl

    value, n, el, nsl = rate_of(w.N, seconds_target)
    out = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{nsl} slices x {n} particles x {w.steps} EM steps, {el:.1f} s"}
    if not detail:
        return out
    orc.set_num_threads(1)
    try:
        v1, n1, el1, _ = rate_of(w.N, seconds_target / 3)
    finally:
        orc.set_num_threads(cores)
    # one slice of the 16-dimensional fast space, 2^16 particles
    lw = workloads.LARGE_FAST
    nl = 1 << 16
    lm = orc.Model(lw.kind, lw.fast_dim, lw.lam, lw.beta, lw.eps, lw.tau_x)
    lx, ly = workloads.initial_ensemble(lw.scaled(N=nl))
    t0 = time.perf_counter()
    orc.fine_propagate(lm, lw.seed, lx[None], ly[None], 1, lw.steps, lw.step_dt)
    el_l = time.perf_counter() - t0
    # the plain FP64 workload in full (4096 particles, 8 slices, 4 iterations)
    ow = workloads.OU_SMALL
    ox, oy = workloads.initial_ensemble(ow)
    t0 = time.perf_counter()
    orc.parareal(orc.Model(ow.kind, ow.fast_dim, ow.lam, ow.beta, ow.eps, ow.tau_x), orc.Grid(ow.bins, ow.lo, ow.hi),
                 ow.seed, ox, oy, ow.K, ow.steps, ow.step_dt, iters=ow.iters)
    el_o = time.perf_counter() - t0
    out.update({"single_core": {"value": v1, "unit": UNIT, "cores": 1,
                                "sample": f"{n1} particles x 1 slice x {w.steps} steps, {el1:.1f} s"},
                "fast16": {"value": nl * lw.steps / el_l, "unit": UNIT, "cores": cores,
                           "sample": f"{nl} particles x 1 slice x {lw.steps} steps of the 16-dimensional "
                                     f"fast-space workload, {el_l:.1f} s"},
                "ou_fp64_full_parareal_s": el_o})
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = WORKLOAD
    from oracle import oracle as orc
    orc.build()
    om = orc.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    x0, y0 = workloads.initial_ensemble(w)
    n = min(1 << 15, w.N)
    for _ in range(args.warmup):
        orc.fine_propagate(om, w.seed, x0[None, :n], y0[None, :, :n], 1, 20, w.step_dt)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.fine_propagate(om, w.seed, x0[None, :n], y0[None, :, :n], 1, w.steps, w.step_dt)
        times.append(time.perf_counter() - t0)
    el = sum(times)
    value = args.steps * n * w.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "sample_particles": n, "slices_per_step": 1,
                   "steps_per_slice": w.steps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
                         "sample": f"{n} particles x 1 slice x {w.steps} EM steps per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _ev_time(fn, stream, reps: int) -> float:
    """Mean milliseconds of `fn` over `reps` calls, CUDA events on `stream`, after one warm call."""
    import torch
    fn(0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for r in range(reps):
        fn(r + 1)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _unfused_leg(L, solver, w, stream, hbm_peak):
    """Restriction and matching as standalone passes over the 49 non-initial
    slices of the double-well state (4 B and 8 B per particle), alternating
    between the two ensemble buffers so the working set (412 MB) exceeds L2;
    the coarse propagator on 50 states and the serial sweep over 50 slices."""
    n, K = w.N, w.K
    bufs = [solver.xa[1:], solver.xb[1:]]
    S = K - 1
    t_r = _ev_time(lambda r: L.pr_restrict(L.PR_F32, bufs[r % 2], n, S, solver.grid, solver.counts_s[1:],
                                           solver.start[1:], stream=stream), stream, 10)
    prior, target = solver.f_star_prev[:S], solver.rho[1:K]
    t_m = _ev_time(lambda r: L.pr_match(L.PR_F32, bufs[r % 2], bufs[(r + 1) % 2], n, S, solver.grid, prior,
                                        target, stream=stream), stream, 10)
    t_c = _ev_time(lambda r: L.pr_coarse_fp(solver.coarse, solver.start, solver.c_star, K, stream=stream),
                   stream, 20)
    t_u = _ev_time(lambda r: L.pr_parareal_update(solver.coarse, L.PR_ITER_QUANTILE, L.PR_QMODE_TWO_SIDED, K,
                                                  solver.cdf0, solver.f_star, solver.c_star, solver._rho_next,
                                                  solver._status[0], stream=stream), stream, 20)
    # Monte Carlo estimator (Eq. MCestimator): mean and second moment of x per slice
    import torch
    mom = torch.empty(S, 2, dtype=torch.float64, device=solver.x0.device)
    mws = torch.empty(L.pr_moments_workspace(n, S, 2), dtype=torch.uint8, device=solver.x0.device)
    t_e = _ev_time(lambda r: L.pr_moments(L.PR_F32, bufs[r % 2], n, None, n, S, 2, mom, mws, stream=stream),
                   stream, 10)
    rb, mb = 4.0 * n * S, 8.0 * n * S
    out = {"restrict": {"ms": t_r, "algorithmic_bytes": rb, "gbs": rb / t_r / 1e6},
           "match": {"ms": t_m, "algorithmic_bytes": mb, "gbs": mb / t_m / 1e6},
           "moments_q2": {"ms": t_e, "algorithmic_bytes": rb, "gbs": rb / t_e / 1e6,
                          "fp64_ops_per_particle": 2,
                          "fp64_ops_per_s": 2.0 * n * S / t_e / 1e-3},
           "coarse_fp_us": 1e3 * t_c, "serial_sweep_us": 1e3 * t_u,
           "note": f"{S} slices x {n} binary32 particles; coarse step on {K} states of {w.bins} bins; "
                   f"sweep over {K} slices"}
    if hbm_peak:
        out["restrict"]["frac_of_measured_hbm"] = out["restrict"]["gbs"] / hbm_peak
        out["match"]["frac_of_measured_hbm"] = out["match"]["gbs"] / hbm_peak
    return out


def _plain_leg(L, dev, stream, rank):
    """The plain FP64 workload in full (4096 particles, 8 slices x 125 steps,
    256 bins): iteration time eager and graph-replayed, iterations to
    W1 <= 1e-3 against the serial fine solution; and the same OU system at
    2^20 particles in binary32 and FP64 (time per iteration, W1 between them)."""
    import torch
    from paper_1912_09240_gb300.parareal import PararealSolver
    out = {}
    for wname, w, precs in (("ou_fp64_full", workloads.OU_SMALL, (L.PR_F64,)),
                            ("ou_n2^20", workloads.OU_SMALL.scaled(N=1 << 20, name="ou_n2^20_k8"),
                             (L.PR_F32, L.PR_F64))):
        model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
        grid = L.Grid(w.bins, w.lo, w.hi)
        x0, y0 = workloads.initial_ensemble(w)
        res, rhos = {}, {}
        for prec in precs:
            dty = torch.float32 if prec == L.PR_F32 else torch.float64
            x0t = torch.tensor(x0, dtype=dty, device=dev)
            y0t = torch.tensor(y0, dtype=dty, device=dev)
            r = {}
            for graph in (False, True):
                sv = PararealSolver(model, grid, w.N, w.K, w.steps, w.step_dt, precision=prec,
                                    rng=L.Rng(w.seed, rank), device=str(dev), graph=graph)
                sv.set_initial(x0t, y0t)
                _, _, rser = sv.serial_reference()
                sv.set_initial(x0t, y0t)
                for _ in range(3):
                    sv.iterate()
                torch.cuda.synchronize()
                reps = 20 if w.N < 100000 else 5
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    sv.iterate()
                sv.join()
                e1.record(stream)
                torch.cuda.synchronize()
                r["graph_ms" if graph else "eager_ms"] = e0.elapsed_time(e1) / reps
                if not graph:
                    sv.set_initial(x0t, y0t)
                    kstar = None
                    for k in range(1, w.K + 1):
                        sv.iterate()
                        if kstar is None and float(sv.w1_to(rser).max().item()) <= 1e-3:
                            kstar = k
                    r["iterations_to_w1_1e-3"] = kstar
                    rhos[prec] = sv.rho.clone()
                sv.close()
            ps = w.particle_steps_per_iteration
            r["particle_steps_per_s"] = ps / (min(r["eager_ms"], r["graph_ms"]) / 1e3)
            res["f32" if prec == L.PR_F32 else "f64"] = r
        if len(rhos) == 2:
            wv = torch.empty(w.K + 1, dtype=torch.float64, device=dev)
            L.pr_w1(grid, w.K + 1, rhos[L.PR_F32], rhos[L.PR_F64], wv)
            res["fp32_vs_fp64_max_w1_at_k_iterations"] = float(wv.max().item())
            res["f64_over_f32_time"] = (min(res["f64"]["eager_ms"], res["f64"]["graph_ms"]) /
                                        min(res["f32"]["eager_ms"], res["f32"]["graph_ms"]))
        res.update({"N": w.N, "K": w.K, "steps_per_slice": w.steps})
        out[wname] = res
    return out


def _matching_leg(L, dev, stream, rank, chunk, iters=10):
    """The matchings of Sections 5.1 and 5.2 on the double-well workload:
    time per pipelined iteration and max_n W1(rho_k^n, R X_serial^n) per
    iteration (same random numbers), and the standalone reweighting and
    resampling passes over 49 slices."""
    import torch
    from paper_1912_09240_gb300.parareal import PararealSolver
    w = WORKLOAD
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    grid = L.Grid(w.bins, w.lo, w.hi)
    x0, y0 = workloads.initial_ensemble(w)
    x0t = torch.tensor(x0, dtype=torch.float32, device=dev)
    y0t = torch.tensor(y0, dtype=torch.float32, device=dev)
    out = {}
    for matching in ("quantile", "resample", "resample_det", "reweight"):
        sv = PararealSolver(model, grid, w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32,
                            rng=L.Rng(w.seed, rank), device=str(dev), chunk=chunk, matching=matching)
        sv.set_initial(x0t, y0t)
        _, _, rser = sv.serial_reference()
        sv.w1_to(rser).max().item()
        sv.set_initial(x0t, y0t)
        times, w1s = [], []
        for _ in range(iters):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sv.iterate()
            sv.join()
            e1.record(stream)
            w1s.append(float(sv.w1_to(rser).max().item()))
            times.append(e0.elapsed_time(e1))
        k_star = next((k + 1 for k, v in enumerate(w1s) if v <= 1e-3), None)
        out[matching] = {"iteration_ms": statistics.median(times[1:]), "max_w1_per_iteration": w1s,
                         "iterations_to_w1_1e-3": k_star, "status": int(sv.status.item())}
        sv.close()
        del sv
    # standalone Section 5.2 passes over the 49 non-initial slices
    S, n = w.K - 1, w.N
    xs = torch.tensor(np.tile(x0.astype(np.float32), (S, 1)), device=dev)
    cdfs = torch.empty(S, w.bins + 1, dtype=torch.float64, device=dev)
    cnt = torch.empty(S, w.bins, dtype=torch.int32, device=dev)
    L.pr_restrict(L.PR_F32, xs, n, S, grid, cnt, cdfs)
    tgt = torch.empty_like(cdfs)
    L.pr_restrict(L.PR_F32, xs + 0.05, n, S, grid, cnt, tgt)
    wts = torch.empty(S, n, dtype=torch.float64, device=dev)
    t_rw = _ev_time(lambda r: L.pr_reweight(L.PR_F32, xs, False, None, n, S, grid, cdfs, tgt, wts, stream=stream),
                    stream, 10)
    ws = torch.empty(L.pr_resample_workspace(n, S), dtype=torch.uint8, device=dev)
    xo = torch.empty_like(xs)
    yo = torch.empty_like(xs).reshape(S, 1, n)
    ys = xs.reshape(S, 1, n)
    t_rs = _ev_time(lambda r: L.pr_resample(L.PR_F32, 1, xs, ys, False, wts, n, S, 1, L.PR_RESAMPLE_STRATIFIED,
                                            L.Rng(0), None, xo, yo, ws, stream=stream), stream, 10)
    out["standalone"] = {"slices": S, "particles": n, "reweight_ms": t_rw, "resample_gather_ms": t_rs,
                         "reweight_particles_per_s": S * n / (t_rw / 1e3),
                         "resample_particles_per_s": S * n / (t_rs / 1e3)}
    return out


def _advection_leg(L, dev, stream, iters=4):
    """The linear advection case of Section 6: parareal with the Fokker-Planck
    equation (potential x/eps, diffusion 1/beta, eps = beta = 1) as the fine
    propagator and a biased one as the coarse propagator, 288 bins on
    [-12, 6], 10 slices of 0.2, Gaussian start N(1, 0.5^2): max_n W1 against
    the serial fine solution per iteration, for every iterator."""
    import math
    import torch
    from paper_1912_09240_gb300.fp_parareal import FPParareal
    bins, lo, hi, K, dT = 288, -12.0, 6.0, 10, 0.2
    edges = np.array([lo + i * (hi - lo) / bins for i in range(bins + 1)])
    c = np.array([0.5 * (1 + math.erf((v - 1.0) / (0.5 * math.sqrt(2)))) for v in edges])
    cdf0 = torch.tensor((c - c[0]) / (c[-1] - c[0]), dtype=torch.float64, device=dev)
    grid = L.Grid(bins, lo, hi)
    fine = L.Model(L.PR_MODEL_ADVECTION, 1, 0.0, 1.0, 1.0)
    cases = {"underdiffusive (beta~ = 2)": (1.0, 2.0), "advection (eps~ = 0.5)": (0.5, 1.0),
             "overdiffusive (beta~ = 0.5)": (1.0, 0.5)}
    names = {L.PR_ITER_QUANTILE: "quantile", L.PR_ITER_ADD: "add", L.PR_ITER_MULT: "mult", L.PR_ITER_ROT: "rot"}
    out = {}
    for label, (eps_c, beta_c) in cases.items():
        row = {}
        for it, nm in names.items():
            fp = FPParareal(grid, fine, L.Model(L.PR_MODEL_ADVECTION, 1, 0.0, beta_c, eps_c), K, dT, iterator=it,
                            device=str(dev))
            fp.set_initial(cdf0)
            ref = fp.serial_reference()
            w1 = [float(fp.w1_to(ref).max().item())]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms = []
            for _ in range(iters):
                e0.record(stream)
                fp.iterate()
                e1.record(stream)
                w1.append(float(fp.w1_to(ref).max().item()))
                ms.append(e0.elapsed_time(e1))
            row[nm] = {"max_w1_per_iteration": w1, "iteration_ms": statistics.median(ms)}
            fp.close()
        out[label] = row
    return out


def _chem_leg(L, dev, stream, rank, chunk, iters=20):
    """The paper's chemical-reaction workload (Section 2.1.2, Table 1: 1e5
    particles, 20 slices of 2000 steps, 600 cells on [0, 600]): time per
    pipelined parareal iteration in binary32 and FP64, and max_n W1 against
    the serial fine solution with the same random numbers per iteration."""
    import torch
    from paper_1912_09240_gb300.parareal import PararealSolver
    w = workloads.CHEM
    model = L.Model(w.kind, 1, 0.0, 1.0, w.eps, w.tau_x, w.rates)
    grid = L.Grid(w.bins, w.lo, w.hi)
    x0, y0 = workloads.initial_ensemble(w)
    out = {"workload": w.name, "particle_steps_per_iteration": w.particle_steps_per_iteration}
    for prec, tag in ((L.PR_F32, "f32"), (L.PR_F64, "f64")):
        dty = torch.float32 if prec == L.PR_F32 else torch.float64
        sv = PararealSolver(model, grid, w.N, w.K, w.steps, w.step_dt, precision=prec, rng=L.Rng(w.seed, rank),
                            device=str(dev), chunk=chunk)
        x0t, y0t = torch.tensor(x0, dtype=dty, device=dev), torch.tensor(y0, dtype=dty, device=dev)
        sv.set_initial(x0t, y0t)
        _, _, rser = sv.serial_reference()
        sv.w1_to(rser).max().item()
        sv.set_initial(x0t, y0t)
        w1s = [float(sv.w1_to(rser).max().item())]
        for _ in range(iters if prec == L.PR_F32 else 2):
            sv.iterate()
            w1s.append(float(sv.w1_to(rser).max().item()))
        # time per iteration back to back (as the headline), after the above
        reps = 10 if prec == L.PR_F32 else 2
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            sv.iterate()
        sv.join()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[tag] = {"iteration_ms": ms, "particle_steps_per_s": w.particle_steps_per_iteration / (ms / 1e3),
                    "max_w1_per_iteration": w1s, "status": int(sv.status.item())}
        sv.close()
    out["f64_over_f32_iteration_time"] = out["f64"]["iteration_ms"] / out["f32"]["iteration_ms"]
    return out


def _studies_leg(L, dev, stream, rank, n=None, iters=20):
    """The convergence studies of Section 6 on the chemical system with the
    defaults of Table 1 (1e5 particles, T = 40, fine step 1e-3, 600 cells):
    varying the time-scale separation eps (20 slices), and the number of
    slices N = 20, 50, 100 at eps = 2.5e-2; every iterator with every
    matching; per iteration, the L2 error of the slow variable's histogram
    (piecewise-constant densities) and W1 against a serial fine solution with
    ten times the particles, at T and as the maximum over slices."""
    from paper_1912_09240_gb300.studies import ConvergenceStudy
    base = workloads.CHEM if n is None else workloads.CHEM.scaled(N=n)
    iterators = {"quantile": L.PR_ITER_QUANTILE, "add": L.PR_ITER_ADD, "mult": L.PR_ITER_MULT,
                 "rot": L.PR_ITER_ROT}
    matchings = ("quantile", "resample", "resample_det", "reweight")
    r4 = lambda v: [float(f"{a:.4g}") for a in v]

    def study(w):
        x0, y0 = workloads.initial_ensemble(w)
        xe, ye = workloads.initial_ensemble(w.scaled(N=9 * w.N), seed=w.seed + 1)
        model = L.Model(w.kind, 1, 0.0, 1.0, w.eps, w.tau_x, w.rates)
        st = ConvergenceStudy(model, L.Grid(w.bins, w.lo, w.hi), w.K, w.steps, w.step_dt, x0, y0,
                              np.concatenate([x0, xe]), np.concatenate([y0, ye], axis=1), seed=w.seed)
        res = {}
        for it_name, it in iterators.items():
            for m in matchings:
                r = st.run(iters, iterator=it, matching=m)
                res[f"{it_name}/{m}"] = {"l2_at_T": r4(r["l2"][:, -1].tolist()),
                                         "l2_max": r4(r["l2"].max(dim=1).values.tolist()),
                                         "w1_max": r4(r["w1"].max(dim=1).values.tolist()),
                                         "status": r["status"]}
        return res

    out = {"workload": base.name, "particles": base.N, "reference_particles": 10 * base.N, "T": base.T,
           "iterations": iters,
           "errors": "L2 of the piecewise-constant densities sqrt(sum (m_i - m_ref,i)^2 / h) at T and max over "
                     "slices; W1 max over slices; the reference's first N particles are the parareal ensemble"}
    out["time_scale_separation"] = {f"eps={eps:g}": study(base.scaled(eps=eps))
                                    for eps in (2.5e-2, 1e-2, 5e-3, 2.5e-3)}
    out["number_of_intervals"] = {f"slices={K}": study(base.scaled(K=K)) for K in (20, 50, 100)}
    return out


def _adjoint_leg(L, dev, stream, rank, n=None):
    """Pathwise gradients of the adjoint workload (2^20 particles, 20 slices x
    1000 steps, checkpoints every 256 steps): the forward alone, the gradient
    of E[X_T^2] (forward + adjoint), and the gradient of the 512-point
    quantile function (per-particle adjoint + order statistics)."""
    import torch
    from paper_1912_09240_gb300.adjoint import quantile_gradient, second_moment_gradient
    w = workloads.ADJOINT
    if n:
        w = w.scaled(N=n, name=w.name + f"_n{n}")
    x0, y0 = workloads.initial_ensemble(w)
    gx0 = torch.tensor(x0, dtype=torch.float32, device=dev)
    gy0 = torch.tensor(y0[0], dtype=torch.float32, device=dev)
    model = L.Model(w.kind, 1, w.lam, w.beta, w.eps, w.tau_x)
    rng = L.Rng(w.seed, rank)
    x = gx0.reshape(1, -1).clone()
    y = gy0.reshape(1, 1, -1).clone()

    def forward():
        x.copy_(gx0.reshape(1, -1))
        y.copy_(gy0.reshape(1, 1, -1))
        for n in range(w.K):
            L.pr_fine_propagate(model, L.PR_F32, rng, x, y, False, x, y, w.N, n, 1, w.steps, w.step_dt)

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    t_f, _ = timed(forward)
    t_g, (val, grad) = timed(lambda: second_moment_gradient(model, rng, gx0, gy0, 0, w.K, w.steps, w.step_dt))
    t_q, _ = timed(lambda: quantile_gradient(model, rng, gx0, gy0, 0, w.K, w.steps, w.step_dt))
    # checkpoints every 12 steps (the replay block): more memory, one replay less
    t_g12, (val12, grad12) = timed(lambda: second_moment_gradient(model, rng, gx0, gy0, 0, w.K, w.steps, w.step_dt,
                                                                   ckpt_every=12))
    t_q12, _ = timed(lambda: quantile_gradient(model, rng, gx0, gy0, 0, w.K, w.steps, w.step_dt, ckpt_every=12))
    ps = w.N * w.K * w.steps
    return {"workload": w.name, "particle_steps": ps,
            "forward_ms": t_f, "second_moment_grad_ms": t_g, "quantile_grad_ms": t_q,
            "second_moment_grad_ms_ckpt12": t_g12,
            "quantile_grad_ms_ckpt12": t_q12,
            "ckpt12_workspace_bytes": L.pr_fine_adjoint_workspace(w.N, w.K, w.steps, 12),
            "ckpt12_grad_max_rel_diff": float(((grad12 - grad).abs() / grad.abs().clamp_min(1e-300)).max().item()),
            "forward_particle_steps_per_s": ps / (t_f / 1e3),
            "second_moment_grad_particle_steps_per_s": ps / (t_g / 1e3),
            "grad_over_forward": t_g / t_f,
            "second_moment": float(val.item()), "grad_lambda_beta_eps": [float(v) for v in grad.cpu()]}


def _large_leg(L, dev, stream, rank, chunk, n=None, k=None, iters=1):
    """One parareal iteration of the 16-dimensional fast-space workload
    (4e6 particles, 100 slices x 1000 steps, 1024 bins), after a warm-up
    iteration."""
    import torch
    from paper_1912_09240_gb300.parareal import PararealSolver
    w = workloads.LARGE_FAST
    if n or k:
        w = w.scaled(N=n or w.N, K=k or w.K, T=w.slice_dt * (k or w.K))
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    grid = L.Grid(w.bins, w.lo, w.hi)
    x0t = torch.tensor(workloads.initial_slow(w), dtype=torch.float32, device=dev)   # Y_0 = X_0 (1, ..., 1)
    solver = PararealSolver(model, grid, w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32,
                            rng=L.Rng(w.seed, rank), device=str(dev), chunk=chunk)
    solver.set_initial(x0t, x0t.expand(w.fast_dim, w.N).contiguous())
    solver.iterate()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(iters):
        solver.iterate()
    solver.join()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    status = int(solver.status.item())
    solver.close()
    ps = w.particle_steps_per_iteration
    return {"workload": w.name, "N": w.N, "K": w.K, "steps_per_slice": w.steps, "fast_dim": w.fast_dim,
            "bins": w.bins, "particle_steps_per_iteration": ps, "iteration_ms": ms,
            "particle_steps_per_s": ps / (ms / 1e3), "status": status}


def _fp64_leg(L, w, model, stream, fine_ms):
    """The plain FP64 fine kernel on a sample of the workload (2 slices of all
    particles), against the binary32 fine kernel's rate in the main launch."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    x0, y0 = workloads.initial_ensemble(w)
    xs = torch.tensor(np.stack([x0, x0]), dtype=torch.float64, device=dev)
    ys = torch.tensor(np.stack([y0, y0]), dtype=torch.float64, device=dev)
    L.pr_fine_propagate(model, L.PR_F64, L.Rng(w.seed), xs, ys, False, xs, ys, w.N, 1, 2, 50, w.step_dt)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    L.pr_fine_propagate(model, L.PR_F64, L.Rng(w.seed), xs, ys, False, xs, ys, w.N, 1, 2, w.steps, w.step_dt)
    f1.record(stream)
    torch.cuda.synchronize()
    fp64_rate = 2 * w.N * w.steps / (f0.elapsed_time(f1) / 1e3)
    fine_rate = (w.K - 1) * w.N * w.steps / (fine_ms / 1e3) if fine_ms else None
    return {"fp64_particle_steps_per_s": fp64_rate, "fp32_fine_particle_steps_per_s": fine_rate,
            "fp32_over_fp64": (fine_rate / fp64_rate) if fine_rate else None,
            "sample": f"FP64 fine kernel, {w.N} particles x 2 slices x {w.steps} steps"}


def _fp64_iteration_leg(L, w, model, grid, stream, rank, chunk, ms):
    """One whole parareal iteration of the workload on the plain FP64 path
    (pipelined driver), after one warm-up iteration."""
    import torch
    from paper_1912_09240_gb300.parareal import PararealSolver
    dev = torch.device("cuda", torch.cuda.current_device())
    x0, y0 = workloads.initial_ensemble(w)
    sv = PararealSolver(model, grid, w.N, w.K, w.steps, w.step_dt, precision=L.PR_F64,
                        rng=L.Rng(w.seed, rank), device=str(dev), chunk=chunk)
    sv.set_initial(torch.tensor(x0, dtype=torch.float64, device=dev),
                   torch.tensor(y0, dtype=torch.float64, device=dev))
    sv.iterate()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    sv.iterate()
    sv.join()
    f1.record(stream)
    torch.cuda.synchronize()
    out = {"fp64_iteration_ms": f0.elapsed_time(f1), "fp32_iteration_ms": ms,
           "fp64_over_fp32_iteration_time": f0.elapsed_time(f1) / ms}
    sv.close()
    return out


def _convergence_leg(L, solver, w, model, grid, stream, rank, chunk, ms, x0t, y0t, detail):
    """Iterations until max_n W1(rho_k^n, R X_serial^n) <= 1e-3 against the
    serial fine solution with the same random numbers, and the time to that
    target.  With `detail`: the same skipping converged slices, graph-replayed
    iterations, and binary32 against FP64 on a paired smaller run."""
    import torch
    from paper_1912_09240_gb300.parareal import PararealSolver
    dev = x0t.device
    _, _, rho_ser = solver.serial_reference()
    solver.w1_to(rho_ser).max().item()   # first launch of the W1 kernel (module load) outside the clock
    solver.set_initial(x0t, y0t)
    w1_hist, k_star = [], None
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for k in range(1, w.iters + 1):
        solver.iterate()
        w1k = float(solver.w1_to(rho_ser).max().item())
        w1_hist.append(w1k)
        if k_star is None and w1k <= 1e-3:
            k_star = k
            c1.record(stream)
    torch.cuda.synchronize()
    conv = {"w1_target": 1e-3, "iterations_to_target": k_star, "max_w1_per_iteration": w1_hist,
            "iteration_ms": ms, "time_to_target_ms": (c0.elapsed_time(c1) if k_star else None),
            "note": "W1 between the parareal macroscopic states and the restriction of the serial fine "
                    "solution with the same random numbers, max over slices; time includes the per-"
                    "iteration W1 reduction"}
    if not detail:
        return conv
    # the same iterations skipping the converged slices (iteration k propagates
    # slices k..K-1 only; exactness property): same states, less fine work
    if k_star:
        ss = PararealSolver(model, grid, w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32,
                            rng=L.Rng(w.seed, rank), device=str(dev), chunk=chunk, skip_converged=True)
        ss.set_initial(x0t, y0t)
        ss.iterate()                      # module loads and scratch outside the clock
        torch.cuda.synchronize()
        ss.set_initial(x0t, y0t)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(k_star):           # timed like the loop above, W1 included
            ss.iterate()
            w1_skip = float(ss.w1_to(rho_ser).max().item())
        s1.record(stream)
        torch.cuda.synchronize()
        conv["skip_converged"] = {
            "time_to_target_ms": s0.elapsed_time(s1),
            "fine_slices_propagated": sum(w.K - k for k in range(k_star)),
            "fine_slices_full": k_star * w.K,
            "max_w1_at_target": w1_skip, "same_as_full": w1_skip == w1_hist[k_star - 1]}
        ss.close()
        del ss
    # wall time per iteration as CUDA graph replays (pipelined chunks inside
    # each graph), median of 10 after two warm-up iterations
    gs = PararealSolver(model, grid, w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32,
                        rng=L.Rng(w.seed, rank), device=str(dev), chunk=chunk, graph=True)
    gs.set_initial(x0t, y0t)
    for _ in range(3):
        gs.iterate()
    torch.cuda.synchronize()
    gt = []
    for _ in range(10):
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        gs.iterate()
        g1.record(stream)
        g1.synchronize()
        gt.append(g0.elapsed_time(g1))
    gs.close()
    del gs
    conv["graph_iteration_ms_median"] = statistics.median(gt)
    conv["time_to_target_graph_ms"] = (k_star * statistics.median(gt)) if k_star else None
    # binary32 against the plain FP64 path on a paired smaller run (2^16 particles, 10 slices, 3 iterations)
    ws_ = w.scaled(N=1 << 16, K=10, T=w.slice_dt * 10, iters=3)
    x0s, y0s = workloads.initial_ensemble(ws_)
    rhos = {}
    for prec in (L.PR_F32, L.PR_F64):
        dty = torch.float32 if prec == L.PR_F32 else torch.float64
        sv = PararealSolver(model, grid, ws_.N, ws_.K, ws_.steps, ws_.step_dt, precision=prec,
                            rng=L.Rng(w.seed, rank), device=str(dev))
        sv.set_initial(torch.tensor(x0s, dtype=dty, device=dev), torch.tensor(y0s, dtype=dty, device=dev))
        for _ in range(ws_.iters):
            sv.iterate()
        rhos[prec] = sv.rho.clone()
        sv.close()
    wv = torch.empty(ws_.K + 1, dtype=torch.float64, device=dev)
    L.pr_w1(grid, ws_.K + 1, rhos[L.PR_F32], rhos[L.PR_F64], wv)
    conv["fp32_vs_fp64_max_w1"] = float(wv.max().item())
    conv["fp32_vs_fp64_case"] = "2^16 particles, 10 slices x 1000 steps, 3 iterations"
    return conv


def _batched_leg(L, dev, stream, rank, ws, dist):
    """Batched serving: 64 independent OU problems with uneven eps, lambda and
    particle counts, one persistent launch per iteration, graph-replayed,
    scheduling picked by the autotuner; then the batch's convergence from X_0."""
    import torch
    from paper_1912_09240_gb300.batch import BatchSolver
    from paper_1912_09240_gb300.replicas import max_over_ranks, shard, sum_over_ranks
    bw = workloads.batched_problems()
    probs, bx, by = [], [], []
    # independent problems: each rank serves its share, no collective
    mine = shard([float(pw.N * pw.K * pw.steps) for pw in bw.problems], rank, ws)
    for pw in (bw.problems[i] for i in mine):
        probs.append(L.Problem(L.Model(pw.kind, 1, pw.lam, pw.beta, pw.eps), L.Grid(pw.bins, pw.lo, pw.hi),
                               pw.N, pw.K, pw.steps, pw.step_dt, pw.seed))
        xx, yy = workloads.initial_ensemble(pw)
        bx.append(xx.astype(np.float32))
        by.append(yy[0].astype(np.float32))
    bs = BatchSolver(probs, device=str(dev))
    bs.set_initial(bx, by)
    t_tune0 = time.perf_counter()
    tuned_ms = bs.tune(steps_div=8)
    tune_s = time.perf_counter() - t_tune0
    bs.set_initial(bx, by)
    bs.iterate()   # zeroth -> first iteration (eager)
    bs.iterate()   # first graph replay (captures)
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nb = 3
    b0.record(stream)
    for _ in range(nb):
        bs.iterate()
    b1.record(stream)
    torch.cuda.synchronize()
    bms = max_over_ranks(b0.elapsed_time(b1) / nb, dist, dev)
    b_ps = sum_over_ranks(bs.particle_steps, dist, dev)
    ppt, work, items = bs.config()
    batched = {"workload": bw.name, "problems": len(bw.problems), "problems_per_rank": len(probs),
               "particle_steps_per_iteration": b_ps,
               "iteration_ms": bms, "particle_steps_per_s": b_ps / (bms / 1e3),
               "graph_replayed": True, "tuned": {"particles_per_thread": ppt, "item_particle_steps": work,
                                                  "items": items, "tune_s": tune_s, "trial_ms": tuned_ms},
               "status": bs.status()}
    # convergence of the batch from X_0: after each iteration, how many
    # problems have max_n W1(rho_k^n, rho_{k-1}^n) <= 1e-3 (12 iterations)
    bs.set_initial(bx, by)
    prev = bs.snapshot()
    within, worst = [], []
    for _ in range(12):
        bs.iterate()
        cur = bs.snapshot()
        inc_b = bs.increments(prev, cur)
        within.append(int((inc_b <= 1e-3).sum().item()))
        worst.append(float(inc_b.max().item()))
        prev = cur
    batched["increments"] = {"tol": 1e-3, "problems_within_tol_per_iteration": within,
                             "max_increment_per_iteration": worst,
                             "note": "increment = max over slices of W1 between consecutive iterates; "
                                     "the exactness theorem makes it 0 at iteration K + 1"}
    bs.close()
    return batched


# Side legs: off by default (the default run measures the headline, the
# dominant kernel, the end-to-end path and the CPU baseline); `--legs a,b` or
# `--legs all` adds them.  Each leg's result goes to stderr as one JSON line
# {"leg": name, ...} and, with --legs-out, into one JSON file.
LEGS = ("fp64_iteration", "convergence_detail", "batched", "unfused", "plain_ou", "matchings", "advection",
        "chem", "studies", "adjoint", "fast16", "cpu_detail")


def parse_legs(spec: str | None) -> list:
    if not spec:
        return []
    names = [s.strip() for s in spec.split(",") if s.strip()]
    if names == ["all"]:
        return list(LEGS)
    bad = [n for n in names if n not in LEGS]
    if bad:
        raise SystemExit(f"unknown leg(s) {bad}; choose from {', '.join(LEGS)} or all")
    return names


def _r(v, digits=4):
    """A float rounded to `digits` significant digits (compact JSON)."""
    if v is None:
        return None
    return float(f"{v:.{digits}g}")


def compact_line(*, metric, value, unit, n_gpus, steps, warmup, ms_per_step, workload, config, clocks, roofline,
                 cpu, e2e, launches, fp32_over_fp64=None, iters_to_w1=None, time_to_w1_ms=None) -> dict:
    """The final stdout line: the contract's keys only, rounded, well under
    1 KB (side legs are reported elsewhere).  `iters_to_w1` is the number of
    parareal iterations until max_n W1(rho_k^n, R X_serial^n) <= 1e-3 and
    `ms_to_w1` the time they take; `fp32_over_fp64` the binary32 fine
    kernel's rate over the plain FP64 kernel's; the roofline is that of the
    dominant kernel, fine_f32_d1_kernel."""
    line = {
        "metric": metric, "value": _r(value), "unit": unit, "n_gpus": n_gpus, "steps": steps, "warmup": warmup,
        "ms_per_step": _r(ms_per_step), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": dict(workload=workload, **config),
        "gpu_launches": launches,
        "clocks": {"sm_mhz": clocks.get("sm_mhz"), "sm_max_mhz": clocks.get("sm_max_mhz"),
                   "reasons": clocks.get("reasons", [])},
        "roofline": None if roofline is None else {
            "bound": roofline["bound"], "achieved": _r(roofline["achieved"]), "peak": _r(roofline["peak"]),
            "unit": roofline["unit"], "frac": _r(roofline["frac"]),
            "traffic": None if roofline.get("traffic") is None else _r(roofline["traffic"])},
        "cpu_baseline": None if cpu is None else {"value": _r(cpu["value"]), "unit": cpu["unit"],
                                                  "cores": cpu["cores"], "kind": cpu["kind"],
                                                  "sample": cpu["sample"]},
        "e2e": None if e2e is None else {"value": _r(e2e["value"]), "unit": e2e["unit"],
                                         "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                                         "d2h_bytes_per_step": e2e["d2h_bytes_per_step"]},
        "fp32_over_fp64": _r(fp32_over_fp64, 3), "iters_to_w1": iters_to_w1, "ms_to_w1": _r(time_to_w1_ms),
    }
    return line


def emit_line(line: dict) -> str:
    s = json.dumps(line, separators=(",", ":"), ensure_ascii=False)
    if len(s.encode()) >= 1024:
        raise RuntimeError(f"final bench line is {len(s.encode())} bytes (limit 1024)")
    print(s, flush=True)
    return s


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1912_09240_gb300 import _lib as L
    from paper_1912_09240_gb300 import build as b
    from paper_1912_09240_gb300.parareal import PararealSolver
    from paper_1912_09240_gb300.replicas import max_over_ranks, sum_over_ranks
    if rank == 0 or ws == 1:
        b.build()
    if dist:
        dist.barrier()
    if args.update_cluster:
        L.pr_set_update_cluster(args.update_cluster)
    legs = parse_legs(args.legs)
    w = WORKLOAD
    model = L.Model(w.kind, w.fast_dim, w.lam, w.beta, w.eps, w.tau_x)
    grid = L.Grid(w.bins, w.lo, w.hi)
    x0, y0 = workloads.initial_ensemble(w)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    # pipelined driver: fine launches in chunks of PIPE_CHUNK slices on two
    # streams, the serial sweep on a third, hidden behind the fine work
    solver = PararealSolver(model, grid, w.N, w.K, w.steps, w.step_dt, precision=L.PR_F32,
                            rng=L.Rng(w.seed, rank), device=str(dev), chunk=args.chunk)
    x0t = torch.tensor(x0, dtype=torch.float32, device=dev)
    y0t = torch.tensor(y0, dtype=torch.float32, device=dev)
    solver.set_initial(x0t, y0t)

    for _ in range(args.warmup):
        solver.iterate()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        launches0 = solver.launches
        t0.record(stream)
        for _ in range(args.steps):
            solver.iterate()
        solver.join()
        t1.record(stream)
        launches = solver.launches - launches0
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = t0.elapsed_time(t1) / args.steps
    # the dominant kernel on its own: sequential iterations (one fine launch
    # over slices 1..K-1 each), timed with events around that launch on the
    # stream it runs on
    chunk_saved, solver.chunk = solver.chunk, 0
    solver.fine_events = []
    for _ in range(2):
        solver.iterate()
    torch.cuda.synchronize()
    fine_times = solver.fine_events
    solver.fine_events = None
    solver.chunk = chunk_saved
    ms = max_over_ranks(ms, dist, dev)
    ps_per_step = w.particle_steps_per_iteration
    value = ws * ps_per_step / (ms / 1e3)
    fine_ms = statistics.mean(a.elapsed_time(b_) for a, b_ in fine_times) if fine_times else None

    # end to end through the C ABI with host buffers: every step copies X_0
    # and Y_0 from page-locked host memory (pr_copy_to_device), runs R X_0,
    # the zeroth iteration and one parareal iteration, and copies rho back
    # (pr_copy_to_host) before the host synchronises
    x0h = torch.tensor(x0, dtype=torch.float32).pin_memory()
    y0h = torch.tensor(y0, dtype=torch.float32).pin_memory()
    rho_h = torch.empty(w.K + 1, w.bins + 1, dtype=torch.float64).pin_memory()
    solver.set_initial_host(x0h, y0h)
    solver.iterate()
    solver.rho_to_host(rho_h)
    L.pr_stream_synchronize(stream)
    if dist:
        dist.barrier()
    te0 = time.perf_counter()
    for _ in range(args.steps):
        solver.set_initial_host(x0h, y0h)
        solver.iterate()
        solver.rho_to_host(rho_h)
        L.pr_stream_synchronize(stream)
    e2e_s = max_over_ranks((time.perf_counter() - te0) / args.steps, dist, dev)
    e2e = {"value": ws * ps_per_step / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(x0h.numel() * 4 + y0h.numel() * 4),
           "d2h_bytes_per_step": int(rho_h.numel() * 8)}

    fp64 = _fp64_leg(L, w, model, stream, fine_ms)
    conv = _convergence_leg(L, solver, w, model, grid, stream, rank, args.chunk, ms, x0t, y0t,
                            "convergence_detail" in legs)

    side = {}

    def leg(name, fn):
        if name in legs:
            t = time.perf_counter()
            side[name] = fn()
            if rank == 0:
                print(json.dumps({"leg": name, "s": round(time.perf_counter() - t, 1), **side[name]}),
                      file=sys.stderr, flush=True)

    if "convergence_detail" in legs and rank == 0:
        print(json.dumps({"leg": "convergence_detail", **conv}), file=sys.stderr, flush=True)
        side["convergence_detail"] = conv
    if rank == 0:
        print(json.dumps({"leg": "fp64_sample", **fp64}), file=sys.stderr, flush=True)
    leg("fp64_iteration", lambda: _fp64_iteration_leg(L, w, model, grid, stream, rank, args.chunk, ms))
    leg("batched", lambda: _batched_leg(L, dev, stream, rank, ws, dist))
    leg("unfused", lambda: _unfused_leg(L, solver, w, stream, _peaks().get("hbm_gbs")))
    leg("plain_ou", lambda: _plain_leg(L, dev, stream, rank))
    leg("matchings", lambda: _matching_leg(L, dev, stream, rank, args.chunk))
    leg("advection", lambda: _advection_leg(L, dev, stream))
    leg("chem", lambda: _chem_leg(L, dev, stream, rank, args.chunk))
    leg("studies", lambda: _studies_leg(L, dev, stream, rank, n=args.studies_n))
    leg("adjoint", lambda: _adjoint_leg(L, dev, stream, rank, n=args.adjoint_n))
    if "fast16" in legs:
        solver.close()

        def fast16():
            r = _large_leg(L, dev, stream, rank, args.chunk, n=args.large_n, k=args.large_k)
            if dist:
                r["particle_steps_per_s"] = sum_over_ranks(r["particle_steps_per_iteration"], dist, dev) / (
                    max_over_ranks(r["iteration_ms"], dist, dev) / 1e3)
            return r
        leg("fast16", fast16)

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        solver.close()
        return 0

    peaks = _peaks()
    clocks = clk.summary()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    roofline = None
    if fine_ms and INST_PER_PARTICLE_STEP:
        launch_ps = (w.K - 1) * w.N * w.steps
        achieved = INST_PER_PARTICLE_STEP * launch_ps / (fine_ms / 1e3) / 1e12
        peak = SMS * ISSUE_LANES_PER_SM_CLK * sm_max * 1e6 / 1e12
        traffic = (TRAFFIC_BYTES_PER_PARTICLE_SLICE * (w.K - 1) * w.N
                   if TRAFFIC_BYTES_PER_PARTICLE_SLICE else None)
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s",
                    "frac": achieved / peak, "traffic": traffic, "kernel": "fine_f32_d1_kernel"}
        if rank == 0:
            print(json.dumps({"leg": "roofline_detail", **roofline, "fine_ms_per_launch": fine_ms,
                              "achieved_in_step": INST_PER_PARTICLE_STEP * ps_per_step / (ms / 1e3) / 1e12,
                              "peak_basis": f"152 SMs x 4 warp-instr/clk x 32 lanes x {sm_max:.0f} MHz",
                              "algorithmic": f"{INST_PER_PARTICLE_STEP} thread-instructions per particle-step x "
                                             f"{launch_ps:.3e} particle-steps per launch"}),
                  file=sys.stderr, flush=True)
    cpu = None
    if not args.no_cpu:
        cpu = _cpu_sample(detail="cpu_detail" in legs)
        print(json.dumps({"leg": "cpu_baseline", **cpu}), file=sys.stderr, flush=True)
    if args.legs_out:
        with open(args.legs_out, "w") as f:
            json.dump({"fp64_sample": fp64, "convergence": conv, "e2e": e2e, "clocks": clocks,
                       "roofline": roofline, "fine_ms_per_launch": fine_ms, "cpu_baseline": cpu, **side}, f,
                      indent=1)
    line = compact_line(
        metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms, workload=w.name,
        config={"bins": w.bins, "parallelism": f"replicas x{ws}", "l2": "inputs>L2"},
        clocks=clocks, roofline=roofline, cpu=cpu, e2e=e2e, launches=launches,
        fp32_over_fp64=fp64.get("fp32_over_fp64"), iters_to_w1=conv.get("iterations_to_target"),
        time_to_w1_ms=conv.get("time_to_target_ms"))
    emit_line(line)
    solver.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--legs", default="", help=f"side legs to run: comma list of {', '.join(LEGS)}, or all")
    ap.add_argument("--legs-out", default=None, help="write every measured figure as one JSON file")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--update-cluster", type=int, default=None, help="CTAs of the serial-sweep cluster")
    ap.add_argument("--chunk", type=int, default=5, help="slices per pipelined chunk (0: sequential)")
    ap.add_argument("--adjoint-n", type=int, default=None, help="particles of the adjoint leg")
    ap.add_argument("--studies-n", type=int, default=None, help="particles of the studies leg (default 1e5)")
    ap.add_argument("--large-n", type=int, default=None, help="particles of the 16-dimensional leg")
    ap.add_argument("--large-k", type=int, default=None, help="slices of the 16-dimensional leg")
    ap.add_argument("--n", type=int, default=None, help="particles (smaller case for profiling)")
    ap.add_argument("--k", type=int, default=None, help="slices (smaller case for profiling)")
    args = ap.parse_args()
    global WORKLOAD
    if args.n or args.k:
        WORKLOAD = WORKLOAD.scaled(N=args.n or WORKLOAD.N, K=args.k or WORKLOAD.K,
                                   T=WORKLOAD.slice_dt * (args.k or WORKLOAD.K),
                                   name=WORKLOAD.name + f"_n{args.n or WORKLOAD.N}_k{args.k or WORKLOAD.K}")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
