#!/usr/bin/env python3
"""mixTS-PIMD step benchmark on one GB300 (or N independent replicas).

Workload (the plain method at size): 512 flexible waters in a 24.83 A
periodic box, mixTS bead counts H 32 / O 4, FP64 forces and integration,
300 K, dt 0.25 fs, PILE-L tau 100 fs. One step = neighbour search + mixTS
pair sweep + bonded terms + normal-mode propagation + thermostat +
estimators. The uniform-bead form (all atoms P = 32) runs beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mixTS-PIMD ns/day and bead-pair force evals/s vs uniform-bead FP64, 1 GB300"
WORKLOAD = dict(workload="512 flexible waters, 24.83 A box, mixTS H32/O4, FP64, 300 K, dt 0.25 fs",
                n_waters=512, box_A=24.83, P_H=32, P_O=4, dt_fs=0.25, T_K=300.0, tau_fs=100.0,
                r_cut_A=9.0, dsf_alpha=0.2)
DT = 0.25
# algorithmic FP64 flops per in-cutoff bead-pair term of the pair kernel,
# counted from its source (add/mul 1, fma 2, rsqrt/erfc/exp 1 each):
# displacement 6, r^2 5, r and 1/r^2 2, DSF energy+force 21, scaling and
# accumulation 9 -> 43; terms with a Lennard-Jones part add 20.
FLOPS_PAIR = 43
FLOPS_LJ_EXTRA = 20
# FP64 ALU peak: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 ALU peak: 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# algorithmic FP32 flops per pair term of the FP32 kernel (counted once,
# though the full-list kernel evaluates it from both atoms): hi/lo
# displacement 12, r^2 5, table 21, scaling 3, accumulation 12 -> 53;
# Lennard-Jones adds 22
FLOPS32_PAIR = 53
FLOPS32_LJ_EXTRA = 22
ION_ELECTRON = dict(workload="256 waters H8/O1 + ion(+3) + electron P=1024, 18.6 A box, dt 0.1 fs",
                    n_waters=256, box_A=18.6, P_H=8, P_O=1, P_e=1024, dt_fs=0.1)
L2_FLUSH_BYTES = 256 << 20
BATCH = dict(workload="64 independent water boxes at 0.997 g/cm3, waters drawn from {32..512}, H beads from "
                      "{4..64}, O = H/4 (min 1), seeds 0-63, FP32 forces + FP64 integration, dt 0.25 fs",
             n_systems=64, draw_seed=1000)
GRAD = dict(workload="512 waters + ion(+3) + electron P=1024, 24.83 A box, H16/O2: V_mix, dV/dq, dV/dtheta "
                     "(theta = sigma, A, b of O and H, q_O, eps_OO)",
            n_waters=512, box_A=24.83, P_H=16, P_O=2, P_e=1024)


def measured_alu_peaks(torch, stream, clocks_idx):
    """FP64 and FP32 FMA-chain throughput of this GPU (the library's probe,
    CUDA events), with the SM clocks sampled while it runs. Each is the best of
    three timed launches (~5-10 ms each)."""
    from paper_2411_11988_gb300 import alu_peak_tflops
    clk = Clocks(clocks_idx)
    clk.__enter__()
    with torch.cuda.stream(stream):
        f64 = max(alu_peak_tflops(True, 6000, stream)[0] for _ in range(3))
        f32 = max(alu_peak_tflops(False, 120000, stream)[0] for _ in range(3))
    clk.__exit__()
    return {"fp64_tflops": f64, "fp32_tflops": f32, "clocks": clk.summary(),
            "method": "mixts_alu_probe: SM-filling grid of 16 independent FMA chains per thread, best of 3"}


def ncu_pipe_pct(kernel, workload):
    """The pipe utilisation ncu recorded for `kernel` on `workload` in its
    committed profile summary (profiles/<kernel>_<workload>*.md), with the
    file it came from; None when no capture of that workload is committed."""
    import glob
    import re
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_{workload}*.md"))):
        for line in open(f):
            m = re.match(r"\|\s*sm__(?:pipe_fp64_cycles_active|pipe_fma_cycles_active|inst_executed_pipe_fma)"
                         r"[^|]*\|\s*([\d.]+)\s*%", line)
            if m:
                return {"pipe_pct": float(m.group(1)), "metric": line.split("|")[1].strip(),
                        "source": os.path.relpath(f, ROOT)}
    return None


def ncu_dram_bytes(kernel, workload):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from the
    ncu capture in its committed profile summary, with the file it came from;
    (None, None) when no capture of that workload is committed."""
    import glob
    import re
    units = {"B": 1.0, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_{workload}*.md"))):
        total, seen = 0.0, False
        for line in open(f):
            if not line.startswith("| dram__bytes_"):
                continue
            cells = line.split("|")
            vals = re.findall(r"([\d.]+)\s*(GB|MB|KB|B)\b", cells[2])
            for v, u in vals[:2]:
                total += float(v) * units[u]
            seen = seen or bool(vals)
        if seen:
            return total, os.path.relpath(f, ROOT)
    return None, None


def ns_per_day(ms_per_step, dt=DT):
    return (1000.0 / ms_per_step) * dt * 86400.0 * 1e-6


class Clocks:
    """Samples SM clocks and throttle reasons while the timed region runs."""

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile(prefix="clocks_", suffix=".csv", delete=False)
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.close()

    def summary(self):
        rows = []
        try:
            for line in open(self.f.name):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def build_system(P_H, P_O, seed):
    import synth
    return synth.water_box(WORKLOAD["n_waters"], WORKLOAD["box_A"], P_H, P_O, seed=seed)


CHUNK = 10


def timed_run(m, torch, stream, steps, warmup, flush, clocks_idx=None, chunk=CHUNK):
    """Device time of exactly `steps` steps, run as chunks of `chunk` steps
    (one mixts_step call each, the production loop: one captured-graph
    launch per chunk); L2 is flushed before every chunk, outside the timed
    events. A second pass of the same chunks with per-phase event timing on
    (plain launches) gives the per-kernel durations."""
    for _ in range(warmup):
        flush.zero_()
        m.step(1)
    flush.zero_()
    m.step(chunk)  # captures the step graph outside the timed region
    stream.synchronize()
    k0 = m.timing()[2]
    sizes = [min(chunk, steps - i) for i in range(0, steps, chunk)]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in sizes]
    clk = Clocks(clocks_idx) if clocks_idx is not None else None
    if clk:
        clk.__enter__()
    stream.synchronize()
    with torch.cuda.stream(stream):
        for (a, b), n in zip(ev, sizes):
            flush.zero_()
            a.record(stream)
            m.step(n)
            b.record(stream)
    stream.synchronize()
    if clk:
        clk.__exit__()
    ms = [a.elapsed_time(b) for a, b in ev]
    k1 = m.timing()[2]
    m.set_timing(True)
    with torch.cuda.stream(stream):
        for n in sizes:
            flush.zero_()
            m.step(n)
    ph_ms, ph_calls, _ = m.timing()
    m.set_timing(False)
    return sum(ms) / steps, ph_ms, ph_calls, k1 - k0, (clk.summary() if clk else None)


def single_call_ms(m, torch, stream, steps, flush):
    """Mean device time of one mixts_step(1) call with L2 flushed before each."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stream.synchronize()
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            m.step(1)
            b.record(stream)
    stream.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def variant(torch, stream, flush, dev, sysm, dt, precision, steps, seed, peaks=None, workload="water512"):
    from paper_2411_11988_gb300 import MixTS
    m = MixTS(sysm, T=300.0, dt=dt, tau=100.0, seed=seed, device=str(dev), stream=stream, precision=precision)
    ms, ph, calls, _, _ = timed_run(m, torch, stream, steps, 3, flush)
    e = m.estimators()
    m.close()
    pair_ms = ph["pair"] / max(1, calls["pair"])
    out = {"ns_per_day": ns_per_day(ms, dt), "ms_per_step": ms, "steps": steps, "pair_kernel_ms": pair_ms,
           "phase_ms_per_call": {k: ph[k] / max(1, calls[k]) for k in ph if calls[k]},
           "bead_pair_evals_per_step": e["n_evals"], "pseudo_evals_per_step": e["n_pseudo_evals"]}
    if precision == 1:
        flops = (e["n_evals"] - e["n_lj_evals"]) * FLOPS32_PAIR + e["n_lj_evals"] * (FLOPS32_PAIR + FLOPS32_LJ_EXTRA)
        ach = flops / (pair_ms * 1e-3) / 1e12
        pk = peaks["fp32_tflops"] if peaks else FP32_PEAK_TFLOPS
        out["roofline_pair"] = {"bound": "alu", "kernel": "k_pair32w", "timed": "k_list_seg32 + k_pair32w",
                                "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                                "frac": ach / pk, "peak_source": "measured FP32 FMA chains" if peaks else "nominal",
                                "frac_of_nominal": ach / FP32_PEAK_TFLOPS, "ncu": ncu_pipe_pct("k_pair32w", workload),
                                "note": "algorithmic flops count each term once"}
    return out


def batch_variant(torch, stream, flush, dev, steps, peaks=None):
    """The batched workload: tune the graph shapes, then time `steps` steps of
    all systems as graph launches of CHUNK steps (L2 flushed before each)."""
    import synth
    from paper_2411_11988_gb300 import MixTSBatch
    draws = synth.systems.batched_draws(BATCH["n_systems"], BATCH["draw_seed"])
    systems = [synth.water_box(w, synth.density_box_length(w), ph, po, seed=i)
               for i, (w, ph, po) in enumerate(draws)]
    b = MixTSBatch(systems, T=300.0, dt=DT, tau=100.0, precision=1, seeds=range(len(systems)), device=str(dev),
                   stream=stream)
    b.step(3)
    t0 = time.perf_counter()
    tune = b.tune(steps_per_launch=CHUNK)
    tune_s = time.perf_counter() - t0
    b.step(CHUNK)
    stream.synchronize()
    k0 = b.timing()[2]
    sizes = [min(CHUNK, steps - i) for i in range(0, steps, CHUNK)]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in sizes]
    with torch.cuda.stream(stream):
        for (a, c), n in zip(ev, sizes):
            flush.zero_()
            a.record(stream)
            b.step(n)
            c.record(stream)
    stream.synchronize()
    ms = sum(a.elapsed_time(c) for a, c in ev) / steps
    k1 = b.timing()[2]
    est = b.estimators()
    evals = sum(e["n_evals"] for e in est)
    # per-phase device times of the same step (eager launches with CUDA events:
    # one launch per phase for all members when the batch runs that way)
    b.set_timing(True)
    b.step(2)
    ph, calls, _ = b.timing()
    b.set_timing(False)
    b.close()
    pair_ms = ph["pair"] / 2.0
    flops = sum((e["n_evals"] - e["n_lj_evals"]) * FLOPS32_PAIR + e["n_lj_evals"] * (FLOPS32_PAIR + FLOPS32_LJ_EXTRA)
                for e in est)
    return {"workload": BATCH["workload"], "draws": [list(d) for d in draws],
            "gpu_launches_per_step": (k1 - k0) / steps,
            "total_beads": int(sum(x.n_beads for x in systems)),
            "ns_per_day_aggregate": len(systems) * ns_per_day(ms), "ms_per_step": ms, "steps": steps,
            "bead_pair_evals_per_step": evals, "bead_pair_evals_per_s": evals * 1000.0 / ms,
            "gpu_launches": k1 - k0, "tuning": tune, "tuning_s": tune_s,
            "phase_ms_per_step": {k: v / 2.0 for k, v in ph.items() if calls[k]},
            "roofline_pair": {"bound": "alu", "kernel": "k_list_seg32_b + k_pair32_b" if tune.get("persistent") else
                              "k_pair32 per member",
                              "achieved": flops / (pair_ms * 1e-3) / 1e12,
                              "peak": peaks["fp32_tflops"] if peaks else FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": flops / (pair_ms * 1e-3) / 1e12 / (peaks["fp32_tflops"] if peaks else FP32_PEAK_TFLOPS),
                              "note": "one eager launch per phase for all members, CUDA events"}}


def _run_observables(torch, stream, dev, sysm, dt, precision, n_eq, n_samp, every, pairs, dr=0.02, nbins=400):
    """One sampled run through the package's analysis module: (KE_cv stats,
    Rg2 stats, g(r) per pair)."""
    from paper_2411_11988_gb300 import MixTS, analysis
    m = MixTS(sysm, T=300.0, dt=dt, tau=100.0, seed=0, device=str(dev), stream=stream, precision=precision)
    res = analysis.sample(m, n_eq, n_samp, every, pairs, dr, nbins)
    m.close()
    return res["KE_cv"], res["Rg2"], res["g"]


def observables(torch, stream, dev):
    """Sampled observables of the plain method at size (mixTS H32/O4 against
    uniform 32 beads, FP64) and of the precision variant (FP32 forces against
    FP64 forces on the ion + electron system, both on the GPU; the FP64 path
    matches the FP64 oracle per step to 1e-11)."""
    import numpy as np
    import synth
    names = {0: "O", 1: "H"}
    out = {}
    # bench workload: 4,000 equilibration + 6,000 sampled steps each (10^4 in all)
    res = {}
    for key, (ph, po) in {"mixts_H32_O4": (32, 4), "uniform_32": (32, 32)}.items():
        (ke_m, ke_e), _, g = _run_observables(torch, stream, dev, build_system(ph, po, 0), DT, 0, 4000, 6000, 10,
                                              [(0, 0), (0, 1), (1, 1)])
        res[key] = (ke_m, ke_e, g)
    r = (np.arange(400) + 0.5) * 0.02
    water = {"steps": "4000 equilibration + 6000 sampled (every 10), dt 0.25 fs, FP64, RDF bins 0.02 A to 8 A"}
    for key, (ke_m, ke_e, g) in res.items():
        water[key] = {"KE_cv_kcal_mol": {names[t]: [float(ke_m[t]), float(ke_e[t])] for t in (0, 1)},
                      "rdf_first_peak": {f"{names[a]}{names[b]}": [float(r[np.argmax(gg[60:]) + 60]),
                                                                   float(np.max(gg[60:]))]
                                         for (a, b), gg in g.items()}}
    water["rdf_max_abs_diff_mixts_vs_uniform"] = {
        f"{names[a]}{names[b]}": float(np.max(np.abs(res["mixts_H32_O4"][2][(a, b)] - res["uniform_32"][2][(a, b)])))
        for (a, b) in [(0, 0), (0, 1), (1, 1)]}
    out["water512"] = water
    # precision variant: ion + electron, FP32 forces against FP64 forces
    ie = ION_ELECTRON
    sie = synth.water_box(ie["n_waters"], ie["box_A"], ie["P_H"], ie["P_O"], seed=0, ion=dict(synth.systems.ION3),
                          electron_P=ie["P_e"])
    res = {}
    for key, prec in {"fp64": 0, "fp32_forces": 1}.items():
        _, (rg_m, rg_e), g = _run_observables(torch, stream, dev, sie, ie["dt_fs"], prec, 5000, 45000, 10, [(2, 0)])
        res[key] = (rg_m[3], rg_e[3], g[(2, 0)])
    rg64, rg32 = res["fp64"], res["fp32_forces"]
    # partial quantisation (Sec. "System I"): H and O bead counts chosen independently
    from paper_2411_11988_gb300 import analysis
    combos = [(1, 1), (4, 1), (1, 4), (4, 4), (32, 1), (32, 4), (32, 32)]
    out["partial_quantisation"] = dict(
        steps="8000 equilibration + 16000 sampled (every 10) per bead-count pair, dt 0.25 fs, FP64; "
              "[mean, 8-block standard error]",
        **analysis.quantisation_sweep(lambda ph, po: build_system(ph, po, 0), combos, dt=DT, n_eq=8000, n_samp=16000,
                                      every=10, device=str(dev), stream=stream))
    out["ion_electron"] = {
        "steps": "5000 equilibration + 45000 sampled (every 10), dt 0.1 fs (5e4 steps, the workload's length)",
        "electron_Rg_A": {"fp64": [float(np.sqrt(rg64[0])), float(rg64[1] / (2 * np.sqrt(rg64[0])))],
                          "fp32_forces": [float(np.sqrt(rg32[0])), float(rg32[1] / (2 * np.sqrt(rg32[0])))]},
        "ion_O_rdf_first_peak": {k: [float(r[np.argmax(v[2][50:]) + 50]), float(np.max(v[2][50:]))]
                                 for k, v in res.items()},
        "ion_O_rdf_max_abs_diff_fp32_vs_fp64": float(np.max(np.abs(rg32[2] - rg64[2]))),
        "note": "[mean, 8-block standard error]; the FP64 run stands for the FP64 oracle, which it matches "
                "per step to 1e-11 (the oracle itself runs ~0.4 s per step here)"}
    return out


def grad_variant(torch, stream, dev, snapshots):
    """Forward + backward of the differentiable potential on snapshots of a
    short run; each gradient is checked against central differences of the
    GPU potential (h = 1e-3 relative: V carries a few 1e-13 |V| of rounding,
    which a smaller step magnifies into the difference quotient). The FP64
    oracle's gradient at this size is compared in the GPU tests."""
    import numpy as np
    import synth
    from paper_2411_11988_gb300 import MixTS, mixts_potential
    g = GRAD
    s = synth.water_box(g["n_waters"], g["box_A"], g["P_H"], g["P_O"], seed=0, ion=dict(synth.systems.ION3),
                        electron_P=g["P_e"])
    m = MixTS(s, T=300.0, dt=0.1, tau=100.0, seed=0, device=str(dev), stream=stream)
    th0 = np.array([s.pp_sigma[0], s.pp_A_eV[0], s.pp_b[0], s.pp_sigma[1], s.pp_A_eV[1], s.pp_b[1],
                    s.charge_type[0], s.lj_eps[0, 0]], dtype=np.float64)  # the system's own parameters
    times, errs, ratios = [], [], []
    for k in range(snapshots):
        m.step(5)
        with torch.cuda.stream(stream):
            q = m.q.clone().requires_grad_(True)
            th = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
            stream.synchronize()
            t0 = time.perf_counter()
            V = mixts_potential(th, q, m, 0, 1)
            V.backward()
            stream.synchronize()
            times.append((time.perf_counter() - t0) * 1000.0)
        gth = th.grad.numpy()
        worst = 0.0
        ratio = 0.0
        for j in range(8):
            h = 1e-3 * abs(th0[j])
            tp, tm = th0.copy(), th0.copy()
            tp[j] += h
            tm[j] -= h
            vp = m.potential_grad(0, 1, tp, want_dvdq=False, want_theta=False)[0]
            vm = m.potential_grad(0, 1, tm, want_dvdq=False, want_theta=False)[0]
            vp2 = m.potential_grad(0, 1, th0 + (tp - th0) / 2, want_dvdq=False, want_theta=False)[0]
            vm2 = m.potential_grad(0, 1, th0 + (tm - th0) / 2, want_dvdq=False, want_theta=False)[0]
            fd, fd2 = (vp - vm) / (2 * h), (vp2 - vm2) / h
            scale = max(abs(fd), 1e-6 * abs(V.item()))
            # bound on |gth - fd|: the rounding of V (2e-13 |V| per
            # evaluation) over 2h, plus the truncation error of the central
            # difference, which halving h shrinks by 4 (|fd - fd2| ~ 3/4 of it)
            bound = 2e-13 * abs(V.item()) / h + 4.0 / 3.0 * abs(fd - fd2)
            worst = max(worst, abs(gth[j] - fd) / scale)
            ratio = max(ratio, abs(gth[j] - fd) / bound)
        errs.append(worst)
        ratios.append(ratio)
        m.reload()
    m.close()
    return {"workload": g["workload"], "snapshots": snapshots,
            "forward_backward_ms_median": float(np.median(times)), "forward_backward_ms_max": float(np.max(times)),
            "max_rel_err_vs_central_fd": float(np.max(errs)),
            "max_err_over_fd_error_bound": float(np.max(ratios)),
            "note": "host wall time per snapshot (forward V only, backward recomputes and runs the adjoint); FD step "
                    "1e-3 relative; errors relative to max(|dV/dtheta|, 1e-6 |V|); the bound is V's rounding over "
                    "the step plus the truncation error estimated from a half step (<= 1: within the FD's own error)"}


def ewald_variant(torch, stream, flush, dev, steps, alpha=0.35, kmax=11):
    """The bench workload with the paper's electrostatics treatment: Ewald
    real space per bead pair, reciprocal sum on the centroids (coulomb = 1)."""
    from paper_2411_11988_gb300 import MixTS
    sysm = build_system(32, 4, 0)
    m = MixTS(sysm, T=300.0, dt=DT, tau=100.0, seed=0, device=str(dev), stream=stream, alpha=alpha, coulomb=1,
              ewald_kmax=kmax)
    ms, ph, calls, _, _ = timed_run(m, torch, stream, steps, 3, flush)
    m.close()
    return {"workload": WORKLOAD["workload"] + f", Ewald alpha {alpha} 1/A, |n| <= {kmax} on centroids",
            "ns_per_day": ns_per_day(ms), "ms_per_step": ms,
            "phase_ms_per_call": {k: ph[k] / max(1, calls[k]) for k in ph if calls[k]},
            "note": "pair phase = real-space sweep + reciprocal sum on centroids"}


def e2e_run(m, torch, stream, steps):
    """Host-resident state through the public API: per step upload q, p from
    pinned host memory, step, download q, p and the estimates."""
    hq = torch.empty(m.q.shape, dtype=torch.float64, pin_memory=True)
    hp = torch.empty(m.p.shape, dtype=torch.float64, pin_memory=True)
    hq.copy_(m.q)
    hp.copy_(m.p)
    stream.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(steps):
            m.q.copy_(hq, non_blocking=True)
            m.p.copy_(hp, non_blocking=True)
            m.reload()
            m.step(1)
            hq.copy_(m.q, non_blocking=True)
            hp.copy_(m.p, non_blocking=True)
            m.estimators()  # synchronises and reads the estimate record
    t1 = time.perf_counter()
    nb = m.q.numel() * 8
    return (t1 - t0) * 1000.0 / steps, 2 * nb, 2 * nb + 8 * 21


def _cpu_model():
    """CPU model string of this host (/proc/cpuinfo, else lscpu)."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def _oracle_steps(args):
    """One host process: `steps` timed oracle steps of the workload (after
    `warmup` untimed ones); returns ms per step. Runs in a spawned child."""
    steps, warmup, seed = args
    sys.path.insert(0, ROOT)
    import oracle
    s = build_system(WORKLOAD["P_H"], WORKLOAD["P_O"], seed)
    run = oracle.Runner(s, oracle.make_params(T=300.0, dt=DT, tau=100.0, lam=1.0, seed=seed))
    run.step(warmup)
    t0 = time.perf_counter()
    run.step(steps)
    return (time.perf_counter() - t0) * 1000.0 / steps


def cpu_baseline(steps, warmup=0, all_cores=True):
    """The FP64 oracle, as it stands, on this host's cores: once single-threaded
    (`steps` full steps of the workload), then as one independent oracle
    process per core (replicas, `steps` steps each, started together), whose
    aggregate throughput is the all-core figure. Processes are spawned, never
    forked, so a CUDA context in the parent is not inherited."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    ncores = os.cpu_count() or 1
    ms1 = _oracle_steps((steps, warmup, 0))
    single = {"value": ns_per_day(ms1), "unit": "ns/day", "cores": 1, "ms_per_step": ms1,
              "sample": f"{steps} full steps of the workload after {warmup} untimed, one process"}
    out = {"value": single["value"], "unit": "ns/day", "cores": 1, "kind": "oracle", "cpu_model": _cpu_model(),
           "nproc": ncores, "ms_per_step": ms1, "sample": single["sample"], "single_thread": single}
    if all_cores and ncores > 1:
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(ncores) as pool:
            per = pool.map(_oracle_steps, [(steps, warmup, i) for i in range(ncores)])
        wall = time.perf_counter() - t0
        agg = sum(ns_per_day(ms) for ms in per)
        out.update(value=agg, cores=ncores, ms_per_step=statistics.mean(per),
                   sample=f"{ncores} concurrent single-threaded oracle processes (one per core), each {steps} "
                          f"full steps of the workload after {warmup} untimed; value = summed ns/day",
                   all_cores={"value": agg, "unit": "ns/day", "cores": ncores, "wall_s": wall,
                              "ms_per_step_per_process": per})
    return out["ms_per_step"], out


def replica_reduce(step_ms, world, device=None, dt=DT):
    """Replicas only: every rank advances its own system; the job's step time
    is the slowest rank's, and the simulated time adds up over ranks.
    Returns (max step ms over ranks, aggregate ns/day)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(step_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms = float(t.item())
    return step_ms, ns_per_day(step_ms, dt) * world


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=6)
    ap.add_argument("--no-uniform", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-observables", action="store_true")
    ap.add_argument("--workload", default="water512", choices=["water512", "ion_electron"],
                    help="system of the main line (ion_electron: 256 waters + ion + 1024-bead electron, dt 0.1 fs; "
                         "for profiling that workload)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="force precision of the main line (fp32: FP32 pair forces, FP64 integration)")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3

    if args.impl == "reference":
        if rank != 0:
            return
        # bounded sample: every host core runs its own oracle replica of the
        # workload (~1-2 s per full step), warm-up steps untimed, at most 30
        # timed steps each
        k = max(1, min(args.steps, 30))
        w = min(args.warmup, 3)
        ms, cb = cpu_baseline(k, warmup=w)
        line = {"metric": METRIC, "value": cb["value"], "unit": "ns/day", "n_gpus": args.gpus,
                "steps": k, "warmup": w, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": dict(WORKLOAD, l2="n/a (host)"), "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2411_11988_gb300 import MixTS

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    if args.workload == "ion_electron":
        import synth
        ie = ION_ELECTRON
        s = synth.water_box(ie["n_waters"], ie["box_A"], ie["P_H"], ie["P_O"], seed=rank,
                            ion=dict(synth.systems.ION3), electron_P=ie["P_e"])
        dt_main, cfg_main = ie["dt_fs"], dict(ie)
    else:
        s = build_system(WORKLOAD["P_H"], WORKLOAD["P_O"], seed=rank)
        dt_main, cfg_main = DT, dict(WORKLOAD)
    prec = 1 if args.precision == "fp32" else 0
    m = MixTS(s, T=300.0, dt=dt_main, tau=100.0, seed=rank, device=str(dev), stream=stream, precision=prec)
    step_ms, ph_ms, ph_calls, kernels, clk = timed_run(m, torch, stream, args.steps, args.warmup, flush,
                                                       clocks_idx=local)
    peaks = measured_alu_peaks(torch, stream, local)
    est = m.estimators()
    single_ms = single_call_ms(m, torch, stream, max(3, args.steps // 2), flush)
    step_ms, value = replica_reduce(step_ms, world, dev, dt_main)
    evals = est["n_evals"]
    pair_ms = ph_ms["pair"] / max(1, ph_calls["pair"])
    if prec == 1:
        flops = (evals - est["n_lj_evals"]) * FLOPS32_PAIR + est["n_lj_evals"] * (FLOPS32_PAIR + FLOPS32_LJ_EXTRA)
        # the bench systems have >= 768 atoms: the window sweep, timed with
        # the list regrouping before it as the pair phase
        peak, peak_nom, kname = peaks["fp32_tflops"], FP32_PEAK_TFLOPS, "k_pair32w"
        peak_src = "measured FP32 FMA-chain throughput (mixts_alu_probe), this run"
    else:
        flops = (evals - est["n_lj_evals"]) * FLOPS_PAIR + est["n_lj_evals"] * (FLOPS_PAIR + FLOPS_LJ_EXTRA)
        peak, peak_nom, kname = peaks["fp64_tflops"], FP64_PEAK_TFLOPS, "k_pair64"
        peak_src = "measured FP64 FMA-chain throughput (mixts_alu_probe), this run"
    achieved = flops / (pair_ms * 1e-3) / 1e12
    e2e_ms, h2d, d2h = e2e_run(m, torch, stream, max(3, args.steps // 2))

    uni = None
    if not args.no_uniform:
        su = build_system(32, 32, seed=rank)
        mu = MixTS(su, T=300.0, dt=DT, tau=100.0, seed=rank, device=str(dev), stream=stream)
        ku = max(3, args.steps // 2)
        su_ms, phu, callsu, _, _ = timed_run(mu, torch, stream, ku, 3, flush)
        eu = mu.estimators()
        uni = {"ns_per_day": ns_per_day(su_ms), "ms_per_step": su_ms, "bead_pair_evals_per_step": eu["n_evals"],
               "bead_pair_evals_per_s": eu["n_evals"] * 1000.0 / su_ms, "steps": ku,
               "pair_kernel_ms": phu["pair"] / max(1, callsu["pair"])}
        mu.close()

    variants = None
    if not args.no_variants:
        import synth
        vs = max(10, args.steps)
        variants = {
            "fp32_forces_water512_H32O4": variant(torch, stream, flush, dev, build_system(32, 4, rank), DT, 1, vs,
                                                  rank, peaks),
        }
        ie = ION_ELECTRON
        for prec, key in [(1, "fp32_forces_ion_electron"), (0, "fp64_ion_electron")]:
            sie = synth.water_box(ie["n_waters"], ie["box_A"], ie["P_H"], ie["P_O"], seed=rank,
                                  ion=dict(synth.systems.ION3), electron_P=ie["P_e"])
            variants[key] = variant(torch, stream, flush, dev, sie, ie["dt_fs"], prec, vs, rank, peaks,
                                    workload="ion_electron")
            variants[key]["workload"] = ie["workload"]
        variants["batched_64_fp32"] = batch_variant(torch, stream, flush, dev, vs, peaks)
        variants["grad_ion_electron512"] = grad_variant(torch, stream, dev, 100)
        variants["fp64_ewald_centroid_water512_H32O4"] = ewald_variant(torch, stream, flush, dev, vs)
    obs = None
    if not args.no_observables:
        obs = observables(torch, stream, dev)

    cb = None
    if rank == 0 and not args.no_cpu:
        _, cb = cpu_baseline(args.cpu_steps, warmup=1)

    if rank == 0:
        per_phase = {k: ph_ms[k] / max(1, ph_calls[k]) for k in ph_ms if ph_calls[k]}
        # DRAM bytes per launch from the kernel's committed ncu summary
        # (L2-resident working set: far below the bytes the kernel touches)
        traffic, traffic_src = ncu_dram_bytes(kname, args.workload)
        line = {
            "metric": METRIC, "value": value, "unit": "ns/day", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32 forces, f64 integration", "data": "synthetic (seeded lattice water, Maxwell-Boltzmann momenta)",
            "config": dict(cfg_main, l2=f"flushed (256 MiB write, untimed) before every timed chunk of {CHUNK} "
                                        "steps; steps in a chunk run back to back as in production",
                           parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
            "bead_pair_evals_per_s": evals * 1000.0 / step_ms * world,
            "bead_pair_evals_per_step": evals,
            "ms_per_step_single_calls": single_ms,
            "uniform_fp64": uni,
            "variants": variants,
            "observables": obs,
            "mixts_speedup_vs_uniform": (uni["ms_per_step"] / step_ms) if uni else None,
            "roofline": {"bound": "alu", "kernel": kname,
                         "timed": "k_list_seg32 + k_pair32w" if prec == 1 else "k_pair64",
                         "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                         "traffic_source": traffic_src,
                         "peak_source": peak_src, "peak_nominal": peak_nom,
                         "frac_of_nominal": achieved / peak_nom, "flops_per_launch": flops, "launch_ms": pair_ms,
                         "ncu": ncu_pipe_pct(kname, args.workload)},
            "alu_peaks_measured": peaks,
            "phase_ms_per_call": per_phase,
            "cpu_baseline": cb,
            "e2e": {"value": ns_per_day(e2e_ms, dt_main) * world, "unit": "ns/day", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "note": "host-resident state: upload q,p, re-import and recompute forces, step, download"},
            "gpu_launches": kernels,
            "clocks": clk,
        }
        print(json.dumps(line))
    m.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
