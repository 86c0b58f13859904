"""Benchmark: sp-DBA spectral steps/s on one GB300 (3-D Cahn-Hilliard 256^3).

Workload (the single-GPU configuration the headline metric is quoted on):
3-D CH dc/dt = lap(c^3 - c - kappa lap c), semi-implicit spectral step,
grid 256^3 periodic, dx = 1, kappa = 1, dt = 0.01, complex64 bulk arithmetic
with FP64 activity norms, 8^3 k-space blocks (32^3 block map),
tau = 1e-6 max_{k != 0} |c_hat|, reassessed every 10 steps;
c0 = 0.1 + U[-0.05, 0.05] (seed 1234).  A "step" is one solver step of the
whole hot path (inverse FFT, nonlinearity, forward FFT, state preparation
every 10 steps, blockwise update).  The default K = 2000 timed steps are the
configuration's full run, started from c0.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                      [--workload ch3d256|ch2d128|nls512|ensemble64|ch3d384pred]
The default workload is the headline line; the others print one line each for
the remaining configurations (2-D 128^2 FP64; 512 NLS signals; the uneven
64-run ensemble, grouped vs one plan per run; 3-D 384^3 with the learned
predictor).
Under torchrun (N > 1) every rank runs an independent replica (the 256^3 run
does not shard); value = N*K / max-over-ranks time.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (256, 256, 256)
BLOCK = (8, 8, 8)
THRESHOLD = 1e-6
REASSESS = 10
DT, KAPPA = 0.01, 1.0
MEAN, AMP = 0.1, 0.05
PROF_EVERY = 37   # at least this many steps between sampled steps


def prof_every(k):
    """Sampling interval of the per-kernel events: about 20 sampled steps per run
    (at least PROF_EVERY apart), coprime with the reassessment interval so that
    every phase of a reassessment segment gets sampled."""
    import math
    e = max(PROF_EVERY, k // 20)
    while math.gcd(e, REASSESS) != 1:
        e += 1
    return e


# DRAM bytes (read + write) per launch from an ncu capture of the current
# kernels on the 256^3 field (cold L2 at the start of each launch):
# the z forward + update pass of the half-spectrum form: 250.95 MB read, 87.26 MB written;
# the paired z forward of the staged form, with block states (autotuner at step 50): 79.77 MB read, 38.01 MB written;
# the FFT passes (z inverse 144.23 + 37.44, y inverse 75.55 + 15.15, y forward 75.55 + 15.43 MB), averaged.
UPDATE_PASS_DRAM_BYTES = 250.95e6 + 87.26e6
ZFWD_PASS_DRAM_BYTES = 79.77e6 + 38.01e6
# the x pass (two real rows per transform): 75.54 MB read, 15.38 MB written;
XPASS_DRAM_BYTES = 75.54e6 + 15.38e6
# the list-driven update (autotuner's staged candidates at step 50): 173.46 MB read, 44.28 MB written;
LIST_DRAM_BYTES = 173.46e6 + 44.28e6
FFT_PASS_DRAM_BYTES = (144.23e6 + 37.44e6 + 75.55e6 + 15.15e6 + 75.55e6 + 15.43e6) / 3
METRIC = "spectral steps/s adaptive vs dense on 1 GB300 at rel-L2<=1e-4; % of HBM roofline"
WORKLOAD = "ch3d-256^3-c64-B8-tau1e-6rel-R10"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0, t1):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.lines:
            if ts < t0 or ts > t1 + 0.06:
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2609_03922_gb300 import build as B
    B.build()
    from paper_2609_03922_gb300 import spdba
    import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # a non-default stream: the plans replay their reassessment segments as CUDA graphs
    torch.cuda.set_stream(torch.cuda.Stream())
    c0 = W.ch_initial_condition(DIMS, mean=MEAN, amplitude=AMP, seed=W.BASE_SEED).astype(np.float32)
    c0_dev = torch.from_numpy(c0).to(dev)
    K, Wm = args.steps, args.warmup
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def barrier():
        if dist:
            tdist.barrier()

    def timed(plan, profile):
        # warm-up on the same plan, then restart from c0 and time exactly K steps
        plan.set_field(c0_dev)
        plan.step(Wm)
        plan.set_field(c0_dev)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if profile:
            # kernel events on one step in prof_every(K) (coprime with the reassessment interval;
            # segments without a sampled step still replay as graphs)
            plan.profile_begin(prof_every(K))
        t0 = time.time()
        e0.record(st)
        plan.step(K)
        e1.record(st)
        torch.cuda.synchronize()
        t1 = time.time()
        prof = plan.profile_end() if profile else None
        barrier()
        ms = e0.elapsed_time(e1)
        if dist:
            t = torch.tensor([ms], device=dev)
            tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, prof, (t0, t1)

    sampler = ClockSampler(local_rank) if rank == 0 else None

    def make(mode, fuse):
        return spdba.Plan(DIMS, BLOCK, threshold=THRESHOLD, reassess=REASSESS, precision=spdba.SPDBA_C64,
                          mode=mode, dt=DT, kappa=KAPPA, fuse_update=fuse)

    ada = make(spdba.SPDBA_MODE_ADAPTIVE, 1)
    # the plan's autotuner picks the update form (fused into the FFT pass or
    # staged) on a representative state of the run: a quarter of the way in,
    # where blocks have frozen (from c0 every block is active and the forms
    # that skip frozen work cannot show it); the timed run restarts from c0
    ada.set_field(c0_dev)
    ada.step(min(K // 4, 500))
    tune = ada.autotune(2 * REASSESS)
    tune["at_step"] = min(K // 4, 500)
    ada.set_field(c0_dev)
    time.sleep(0.3 if sampler else 0)
    ms_ada, prof, (t0, t1) = timed(ada, True)
    clocks = sampler.stop(t0, t1) if sampler else None
    stats = ada.get_stats()
    field_ada = torch.empty(DIMS, dtype=torch.float32, device=dev)
    ada.get_field(field_ada)

    dense = make(spdba.SPDBA_MODE_REGULAR, 1)
    dense.set_field(c0_dev)
    dense.autotune(2 * REASSESS)
    ms_dense, prof_dense, _ = timed(dense, True)
    field_dense = torch.empty(DIMS, dtype=torch.float32, device=dev)
    dense.get_field(field_dense)
    d = (field_ada.double() - field_dense.double()).norm() / field_dense.double().norm()
    rel_ada_dense = float(d.item())
    dense.close()

    # staged form (separate update kernel, as in the paper's workflow): update-stage timing
    staged = {}
    for name, mode in (("adaptive", spdba.SPDBA_MODE_ADAPTIVE), ("dense", spdba.SPDBA_MODE_REGULAR)):
        pl = make(mode, 0)
        ms, pr, _ = timed(pl, True)
        # the NL pass runs once per step: it counts the sampled steps
        nsamp = max(1, pr[0]["fft_fused_nl"]["launches"])
        upd = sum(pr[0].get(k, {"total_ms": 0.0})["total_ms"] for k in ("update_list", "update_dense", "assess"))
        staged[name] = {"steps_per_s": world * K / (ms / 1e3), "update_stage_ms": upd * K / nsamp}
        pl.close()

    # end to end through the C ABI with host buffers: upload c0, K steps, download c
    c0_pin = torch.from_numpy(c0).pin_memory()
    out_pin = torch.empty(DIMS, dtype=torch.float32).pin_memory()
    ada.set_field(c0_pin)
    ada.step(Wm)
    ada.get_field(out_pin)
    barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    ada.set_field(c0_pin)
    ada.step(K)
    ada.get_field(out_pin)          # synchronizes the plan's stream
    te1 = time.perf_counter()
    e2e_ms = (te1 - te0) * 1e3
    if dist:
        t = torch.tensor([e2e_ms], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    ada.close()

    n = int(np.prod(DIMS))
    steps_total = K * world
    value = steps_total / (ms_ada / 1e3)
    dense_value = steps_total / (ms_dense / 1e3)
    hbm, peak_kind = peaks()

    # kinds whose traffic depends on the block states: the plan records their
    # dense bytes, so no GB/s figure here (their roofline objects use the mean
    # non-frozen share)
    state_dependent = ("fft_update", "fft_z_forward")

    def kind_summary(p):
        out = {}
        tot = sum(v["total_ms"] for v in p[0].values())
        for k, v in p[0].items():
            gbs = (v["bytes"] / 1e9) / (v["total_ms"] / 1e3) if v["total_ms"] > 0 else None
            out[k] = {"launches": v["launches"], "avg_us": 1e3 * v["total_ms"] / max(1, v["launches"]),
                      "gbs": None if k in state_dependent else gbs,
                      "share": v["total_ms"] / tot if tot > 0 else None}
        return out

    kinds = kind_summary(prof)
    fp = prof[0]["fft_pass"]
    achieved = (fp["bytes"] / fp["launches"]) / (fp["total_ms"] / fp["launches"] / 1e3) / 1e9
    # the dominant kernel by time: the z forward pass with the fused update.  Its
    # algorithmic bytes per launch: g read once per output mode (8 B) and c_hat
    # read + written on the non-frozen modes (16 B times the non-frozen share).
    nonfrozen = stats["active_ratio_sum"] / max(1, stats["step"])
    n_modes = int(np.prod(DIMS))
    up = prof[0].get("fft_update")
    upd_roof = None
    # g is read from the half array: x frequencies 0 .. N2/2 of every (z, y)
    n_half = DIMS[0] * DIMS[1] * (DIMS[2] // 2 + 1)
    if up and up["launches"] > 0:
        upd_bytes = 8.0 * n_half + 16.0 * n_modes * nonfrozen
        upd_ach = upd_bytes / (up["total_ms"] / up["launches"] / 1e3) / 1e9
        upd_roof = {"bound": "hbm", "kernel": "z forward FFT pass + fused CH update (L=256, c64)",
                    "achieved": upd_ach, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s", "frac": upd_ach / hbm,
                    "traffic": UPDATE_PASS_DRAM_BYTES,
                    "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch (an early, "
                                    "mostly active step)",
                    "algorithmic_bytes_per_launch": upd_bytes}
    # staged form: the z forward pass (half array -> full transform of g) is the longest kernel
    zf = prof[0].get("fft_z_forward")
    zf_roof = None
    if zf and zf["launches"] > 0:
        # half array read once, g_hat written for the non-frozen modes only
        zf_bytes = 8.0 * n_half + 8.0 * n_modes * nonfrozen
        zf_ach = zf_bytes / (zf["total_ms"] / zf["launches"] / 1e3) / 1e9
        zf_roof = {"bound": "hbm", "kernel": "z forward FFT pass, paired half pencils (L=256, c64)",
                   "achieved": zf_ach, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s", "frac": zf_ach / hbm,
                   "traffic": ZFWD_PASS_DRAM_BYTES,
                   "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch (cold L2; part "
                                   "of the 134 MB output is still in L2 when the launch ends)",
                   "algorithmic_bytes_per_launch": zf_bytes}
    # staged form: the list-driven update (24 B per mode of a listed block, counted on the device)
    ul = prof[0].get("update_list")
    ul_roof = None
    if ul and ul["launches"] > 0 and ul["bytes"] > 0:
        ul_bytes = ul["bytes"] / ul["launches"]
        ul_ach = ul_bytes / (ul["total_ms"] / ul["launches"] / 1e3) / 1e9
        ul_roof = {"bound": "hbm", "kernel": "list-driven CH update of the non-frozen blocks (c64)",
                   "achieved": ul_ach, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s", "frac": ul_ach / hbm,
                   "traffic": LIST_DRAM_BYTES,
                   "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch (autotuner's "
                                   "staged candidates at step 50)",
                   "algorithmic_bytes_per_launch": ul_bytes}
    # the x pass: half array read and written once
    xp = prof[0].get("fft_fused_nl")
    xp_roof = None
    if xp and xp["launches"] > 0:
        xp_bytes = xp["bytes"] / xp["launches"]
        xp_ach = xp_bytes / (xp["total_ms"] / xp["launches"] / 1e3) / 1e9
        half = bool(tune["candidates"][tune["chosen"]]["half_spectrum"])
        xp_roof = {"bound": "hbm", "kernel": ("x pass: two real rows per transform, c^3 - c (L=256, c64)" if half
                                              else "x pass: inverse, c^3 - c, forward (L=256, c64)"),
                   "achieved": xp_ach, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s", "frac": xp_ach / hbm,
                   "traffic": XPASS_DRAM_BYTES if half else None,
                   "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch (cold L2)",
                   "algorithmic_bytes_per_launch": xp_bytes}
    fft_roof = {"bound": "hbm", "kernel": "FFT passes (Stockham, L=256, c64)", "achieved": achieved, "peak": hbm,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm, "traffic": FFT_PASS_DRAM_BYTES,
                "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, averaged over the "
                                "z inverse and the two y passes (cold L2 at each launch start)",
                "algorithmic_bytes_per_launch": fp["bytes"] / fp["launches"]}
    # the dominant kernel: the single kernel with the longest average launch among
    # those with a roofline object (each runs once per step)
    def avg_ms(kind):
        v = prof[0].get(kind)
        return v["total_ms"] / v["launches"] if v and v["launches"] > 0 else -1.0
    cands = [(avg_ms("fft_update"), upd_roof), (avg_ms("fft_z_forward"), zf_roof),
             (avg_ms("update_list"), ul_roof), (avg_ms("fft_fused_nl"), xp_roof)]
    cands = [c for c in cands if c[1] is not None]
    dominant = max(cands, key=lambda c: c[0])[1] if cands else fft_roof
    upd_a, upd_d = staged["adaptive"]["update_stage_ms"], staged["dense"]["update_stage_ms"]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "steps/s",
        "n_gpus": world,
        "steps": K,
        "warmup": Wm,
        "ms_per_step": ms_ada / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64 (fp32) + fp64 norms",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(DIMS), "block": list(BLOCK), "threshold_rel": THRESHOLD,
                   "reassess": REASSESS, "dt": DT, "kappa": KAPPA, "ic": "0.1+U[-0.05,0.05] seed 1234",
                   "timed": "full %d-step run from c0" % K,
                   "l2": "working set larger than L2 (c_hat 134 MB + half-spectrum workspace 75 MB per replica)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "dense_steps_per_s": dense_value,
        "adaptive_over_dense": value / dense_value,
        "staged_form": {"adaptive_steps_per_s": staged["adaptive"]["steps_per_s"],
                        "dense_steps_per_s": staged["dense"]["steps_per_s"],
                        "update_stage_steps_per_s": {"adaptive": K / (upd_a / 1e3) if upd_a > 0 else None,
                                                     "dense": K / (upd_d / 1e3) if upd_d > 0 else None},
                        "update_stage_speedup": upd_d / upd_a if upd_a > 0 else None,
                        "note": "separate list/dense update kernel; update stage = update + state preparation"},
        "autotune": tune,
        "mean_nonfrozen_ratio": stats["active_ratio_sum"] / max(1, stats["step"]),
        "rel_l2_adaptive_vs_dense": rel_ada_dense,
        "kernels": kinds,
        "kernels_dense": kind_summary(prof_dense),
        "roofline": dominant,
        "roofline_fft_passes": fft_roof,
        "roofline_z_forward": zf_roof,
        "roofline_update_list": ul_roof,
        "roofline_x_pass": xp_roof,
        "e2e": {"value": steps_total / (e2e_ms / 1e3), "unit": "steps/s",
                "h2d_bytes_per_step": 4.0 * n / K, "d2h_bytes_per_step": 4.0 * n / K,
                "note": "set_field from pinned host + %d steps + get_field to pinned host" % K},
        "gpu_launches": prof[1],
        "clocks": clocks,
    }
    return line


# ------------------------------------------------------------------ oracle timing
def oracle_sample(max_steps, budget_s):
    """The FP64 CPU oracle on the same workload: adaptive steps from c0 until
    max_steps or the time budget is used.  Returns (steps/s, steps, cores)."""
    import oracle as O
    import workloads as W
    c0 = W.ch_initial_condition(DIMS, mean=MEAN, amplitude=AMP, seed=W.BASE_SEED).astype(np.float32)
    cfg = O.CHConfig(DIMS, BLOCK, threshold=THRESHOLD, reassess=REASSESS, dt=DT, kappa=KAPPA)
    c_hat = O.fftn(c0.astype(np.float64))
    states = None
    t0 = time.perf_counter()
    done = 0
    while done < max_steps:
        c_hat, hist = O.run_ch(None, cfg, 1, start_step=done, c_hat=c_hat, states=states)
        if hist:
            states = hist[-1][1]
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return done / el, done, O.num_threads()


def run_reference(args, rank, world):
    if rank != 0:
        return None
    v, done, cores = oracle_sample(max(1, args.steps), budget_s=90.0)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": world,
            "steps": done, "warmup": 0, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(DIMS), "block": list(BLOCK)},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": "first %d adaptive steps of the 256^3 run (FP64 oracle, bounded to ~90 s)" % done},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ other configurations
def _timed_steps(plan, steps, set_input, stream=None):
    """Restart from the input and time `steps` steps with CUDA events on the plan's stream."""
    import torch
    set_input()
    torch.cuda.synchronize()
    st = stream if stream is not None else torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    plan.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _kind_summary(p):
    """Per-kernel-kind launches, average event time, GB/s and share of a profile."""
    out = {}
    tot = sum(v["total_ms"] for v in p[0].values())
    for k, v in p[0].items():
        out[k] = {"launches": v["launches"], "avg_us": 1e3 * v["total_ms"] / max(1, v["launches"]),
                  "gbs": (v["bytes"] / 1e9) / (v["total_ms"] / 1e3) if v["total_ms"] > 0 else None,
                  "share": v["total_ms"] / tot if tot > 0 else None}
    return out


def _line(metric, value, unit, steps, warmup, ms, config, extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": steps, "warmup": warmup,
         "ms_per_step": ms / max(1, steps), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
         "data": "synthetic", "config": config}
    d.update(extra)
    return d


def run_ch2d128(args):
    """2-D CH 128^2, FP64, 16^2 blocks, tau = 1e-6 max, R = 10, 200 steps (graphs on a side stream)."""
    import torch
    from paper_2609_03922_gb300 import spdba
    import workloads as W
    dims, steps = (128, 128), 200
    c0 = W.ch_initial_condition(dims, mean=0.0, seed=W.BASE_SEED)
    side = torch.cuda.Stream()
    res = {}
    with torch.cuda.stream(side):
        for mode in (1, 0):
            pl = spdba.Plan(dims, (16, 16), threshold=1e-6, reassess=10, precision=spdba.SPDBA_C128, mode=mode)
            _timed_steps(pl, steps, lambda: pl.set_field(c0), side)          # warm-up (captures the graph)
            ms = _timed_steps(pl, steps, lambda: pl.set_field(c0), side)
            res[mode] = (ms, pl.get_field(), pl.get_stats())
            pl.close()
    rel = float(np.linalg.norm(res[1][1] - res[0][1]) / np.linalg.norm(res[0][1]))
    return _line("spectral steps/s adaptive vs dense, 2-D CH 128^2 FP64", steps / (res[1][0] / 1e3), "steps/s", steps,
                 steps, res[1][0], {"workload": "ch2d-128^2-c128-B16-R10", "steps": steps},
                 {"dtype": "f64", "dense_steps_per_s": steps / (res[0][0] / 1e3),
                  "rel_l2_adaptive_vs_dense": rel,
                  "mean_nonfrozen_ratio": res[1][2]["active_ratio_sum"] / steps})


def run_nls512(args):
    """512 NLS signals, lengths 2^e (e uniform 12..18), 8 QPSK channels each, 64 blocks/signal,
    h = 0.1 km over 80 km (800 steps), one plan (groups by length), graphs on a side stream."""
    import torch
    from paper_2609_03922_gb300 import spdba
    import workloads as W
    lengths = W.nls_lengths(512)
    steps = 800
    sigs = [W.nls_signal(n, seed=W.BASE_SEED + 1 + i).astype(np.complex64) for i, n in enumerate(lengths)]
    side = torch.cuda.Stream()
    res = {}
    with torch.cuda.stream(side):
        for mode in (1, 0):
            pl = spdba.Plan(None, (-64,), threshold=1e-6, reassess=10, batch_dims=[(n,) for n in lengths],
                            model=spdba.SPDBA_MODEL_NLS, precision=spdba.SPDBA_C64, mode=mode)

            def setin():
                for r, x in enumerate(sigs):
                    pl.set_field(x, run=r)
            _timed_steps(pl, 20, setin, side)
            ms = _timed_steps(pl, steps, setin, side)
            ratio = float(np.mean([pl.get_stats(run=r)["active_ratio_sum"] / steps for r in range(0, 512, 37)]))
            f0 = pl.get_field(run=0)
            kinds = None
            if mode == 1:
                # per-kernel event timing of a short stretch (graph replay off while profiling)
                pl.profile_begin()
                pl.step(40)
                kinds = _kind_summary(pl.profile_end())
            res[mode] = (ms, ratio, f0, kinds)
            pl.close()
    total = int(sum(lengths))
    rel = float(np.linalg.norm(res[1][2] - res[0][2]) / np.linalg.norm(res[0][2]))
    return _line("NLS batch steps/s (512 signals, all advance one split step)", steps / (res[1][0] / 1e3), "steps/s",
                 steps, 20, res[1][0], {"workload": "nls-512-signals-2^12..2^18-c64-64blocks", "samples": total},
                 {"dtype": "c64", "dense_steps_per_s": steps / (res[0][0] / 1e3),
                  "samples_per_s": total * steps / (res[1][0] / 1e3),
                  "hbm_gbs_at_two_passes_per_step": 2 * 16 * total * steps / (res[1][0] / 1e3) / 1e9,
                  "mean_nonfrozen_ratio_sampled": res[1][1], "rel_l2_adaptive_vs_dense_signal0": rel,
                  "kernels": res[1][3]})


def run_ensemble64(args):
    """64 CH runs, sides uniform in {128,192,256,384,512}, means U[-0.2,0.2], c64, 16^2 blocks,
    1000 steps: one grouped plan with graph replay vs one plan per run."""
    import torch
    from paper_2609_03922_gb300 import spdba
    import workloads as W
    members = W.ensemble_members(64)
    steps = 1000
    c0s = [W.ch_initial_condition((sd, sd), mean=m, seed=seed).astype(np.float32) for sd, m, seed in members]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        pl = spdba.Plan(None, (16, 16), threshold=1e-6, reassess=10, batch_dims=[(sd, sd) for sd, _, _ in members],
                        precision=spdba.SPDBA_C64)

        def setin():
            for r, x in enumerate(c0s):
                pl.set_field(x, run=r)
        _timed_steps(pl, 20, setin, side)
        ms_g = _timed_steps(pl, steps, setin, side)
        ratio = float(np.mean([pl.get_stats(run=r)["active_ratio_sum"] / steps for r in range(64)]))
        pl.close()
        plans = [spdba.Plan((sd, sd), (16, 16), threshold=1e-6, reassess=10, precision=spdba.SPDBA_C64, use_graph=0)
                 for sd, _, _ in members]
        for p_, x in zip(plans, c0s):
            p_.set_field(x)
        for p_ in plans:
            p_.step(10)
        for p_, x in zip(plans, c0s):
            p_.set_field(x)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(side)
        for _ in range(steps // 10):
            for p_ in plans:
                p_.step(10)
        e1.record(side)
        torch.cuda.synchronize()
        ms_p = e0.elapsed_time(e1)
        for p_ in plans:
            p_.close()
    pts = sum(sd * sd for sd, _, _ in members)
    return _line("ensemble steps/s (64 uneven CH runs, all advance one step)", steps / (ms_g / 1e3), "steps/s", steps,
                 20, ms_g, {"workload": "ch2d-ensemble-64-runs-128..512-c64-B16", "points": pts},
                 {"dtype": "c64", "per_run_plans_steps_per_s": steps / (ms_p / 1e3),
                  "grouped_over_per_run": ms_p / ms_g, "mean_nonfrozen_ratio": ratio})


def run_ch3d384pred(args):
    """3-D CH 384^3 c64, 8^3 blocks (48^3 map), 5000 steps, with the learned predictor (K = 20,
    exact judge every 100), trained on traces of two seeded 256^3 runs; compared with the
    exact adaptive run (R = 10) and the dense run."""
    import torch
    from paper_2609_03922_gb300 import spdba
    from paper_2609_03922_gb300 import predictor_train as PT
    import workloads as W
    tr_steps, steps = 1000, 5000
    t0 = time.time()
    traces = [PT.collect_trace((256,) * 3, (8, 8, 8),
                               W.ch_initial_condition((256,) * 3, mean=0.1, seed=W.BASE_SEED + 500 + i).astype(np.float32),
                               tr_steps) for i in range(2)]
    pr32 = PT.TrainedPredictor((32,) * 3, max_batch=8, seed=0)
    xs, ys = [], []
    for tr in traces:
        x, y = PT.make_inputs(pr32, tr, PT.build_samples(tr, 20, 100))
        xs.append(x)
        ys.append(y)
    hist = PT.train(pr32, torch.cat(xs), torch.cat(ys), epochs=30, lr=3e-3)
    t_train = time.time() - t0
    pr48 = spdba.Predictor((48,) * 3, max_batch=1, params=pr32.params())
    dims = (384,) * 3
    c0 = W.ch_initial_condition(dims, mean=0.1, seed=W.BASE_SEED).astype(np.float32)
    out = {}
    for name, mode, pred in (("predictor", 1, pr48), ("exact", 1, None), ("dense", 0, None)):
        pl = spdba.Plan(dims, (8, 8, 8), threshold=1e-6, reassess=10, precision=spdba.SPDBA_C64, mode=mode)
        if pred is not None:
            pl.attach_predictor(pred, 20, 100, 0.5)
        ms = _timed_steps(pl, steps, lambda: pl.set_field(c0))
        st = pl.get_stats()
        out[name] = {"ms": ms, "field": pl.get_field(), "stats": st}
        pl.close()
    d = out["dense"]["field"].astype(np.float64)
    rel = {k: float(np.linalg.norm(out[k]["field"] - d) / np.linalg.norm(d)) for k in ("predictor", "exact")}
    sp, se = out["predictor"]["stats"], out["exact"]["stats"]
    return _line("spectral steps/s with the learned predictor, 3-D CH 384^3", steps / (out["predictor"]["ms"] / 1e3),
                 "steps/s", steps, 0, out["predictor"]["ms"], {"workload": "ch3d-384^3-c64-B8-K20-J100"},
                 {"dtype": "c64 + bf16 predictor", "exact_adaptive_steps_per_s": steps / (out["exact"]["ms"] / 1e3),
                  "dense_steps_per_s": steps / (out["dense"]["ms"] / 1e3),
                  "rel_l2_vs_dense": rel, "exact_scans": {"predictor": sp["assessments"] - sp["predictions"],
                                  "exact": se["assessments"] - se["predictions"]},
                  "predictions": sp["predictions"], "missed_blocks": sp["missed_blocks"],
                  "mean_nonfrozen_ratio": {"predictor": sp["active_ratio_sum"] / steps,
                                           "exact": se["active_ratio_sum"] / steps},
                  "training": {"loss_first_last": [hist[0], hist[-1]], "seconds": t_train}})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="ch3d256",
                    choices=["ch3d256", "ch2d128", "nls512", "ensemble64", "ch3d384pred"])
    args = ap.parse_args()
    if args.workload != "ch3d256":
        import torch
        from paper_2609_03922_gb300 import build as B
        B.build()
        torch.cuda.set_device(0)
        fn = {"ch2d128": run_ch2d128, "nls512": run_nls512, "ensemble64": run_ensemble64,
              "ch3d384pred": run_ch3d384pred}[args.workload]
        print(json.dumps(fn(args)), flush=True)
        return
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            v, done, cores = oracle_sample(3, budget_s=30.0)
            line["cpu_baseline"] = {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                                    "sample": "first %d adaptive steps of the same 256^3 run, FP64 oracle" % done}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
