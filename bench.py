#!/usr/bin/env python3
"""Benchmark of the exact Matérn Gaussian log-likelihood on GB300.

Metric: log-likelihood evaluations per second and Cholesky TFLOP/s at n = 90,000
(300 x 300 jittered grid on the unit square, theta0 = (sigma^2, beta, nu) =
(1, 0.03, 1.0)), mixed precision (the headline `value`) next to FP64, with the
mixed result's |dl|/|l| against the FP64 evaluation at the same theta.

One step = one full evaluation of l(theta) (Matérn generation, Cholesky,
log-determinant, solve and refinement) on inputs already resident in HBM.
Multi-GPU runs are independent replicas (weak scaling): each rank evaluates its
own field; `value` is the evaluations of all ranks over the slowest rank's time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--m 300] [--fp64-steps 1] [--prec tf32x3]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "log-lik evals/s and Cholesky TFLOP/s at n=90K: FP64 vs mixed-precision at |dl|/|l|<=1e-6"
THETA0 = (1.0, 0.03, 1.0)
NOMINAL = {"bf16": 2250.0, "tf32": 1100.0, "fp64": 1.25}  # dense TFLOP/s, for the dtype ratios


def peaks() -> dict:
    """Measured denominators (MEASURED_PEAKS.json), else the recipe's fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        src = "measured"
    else:
        d = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
        src = "fallback"
    bf = d.get("bf16_tflops_sustained", d["bf16_tflops"])
    return {"hbm_gbs": d["hbm_gbs"], "bf16": bf, "tf32": bf * NOMINAL["tf32"] / NOMINAL["bf16"],
            "fp64": d["bf16_tflops"] * NOMINAL["fp64"] / NOMINAL["bf16"], "source": src}


def probe_peaks() -> dict:
    """Short timed probes on this GPU: the library's FP64 issue-rate probes (DFMA, DMMA) and the
    measured library throughput of cuBLAS DGEMM and TF32 GEMM (torch.matmul, 8192^3), CUDA events."""
    import torch

    import paper_1908_06936_gb300 as exa

    s = torch.cuda.current_stream()
    out = {"fp64_dfma_probe": exa.exa_probe_fp64_rate(s.cuda_stream, 0),
           "fp64_dmma_probe": exa.exa_probe_fp64_rate(s.cuda_stream, 1)}

    def gemm_rate(dtype, reps, tf32):
        old = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        try:
            a = torch.randn(8192, 8192, dtype=dtype, device="cuda")
            b = torch.randn(8192, 8192, dtype=dtype, device="cuda")
            torch.matmul(a, b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            best = None
            for _ in range(reps):
                e0.record(s)
                torch.matmul(a, b)
                e1.record(s)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            return 2.0 * 8192 ** 3 / (best * 1e-3) / 1e12
        finally:
            torch.backends.cuda.matmul.allow_tf32 = old

    out["fp64_dgemm_cublas"] = gemm_rate(torch.float64, 2, False)
    out["tf32_gemm_cublas"] = gemm_rate(torch.float32, 10, True)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out["sms"] = sms
    out["how"] = ("probes: every resident CTA, 8 independent chains per thread (DFMA) or warp (DMMA m8n8k4), best of "
                  "3 launches after a warm-up; cuBLAS: best of 2 (FP64) / 10 (TF32) 8192^3 products")
    return out


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id: str | None):
        self.proc = None
        self.dev_id = dev_id

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.dev_id:
            cmd += ["-i", self.dev_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def gpu_id_for_smi() -> str | None:
    import torch

    if torch.cuda.device_count() == 1 and not os.environ.get("CUDA_VISIBLE_DEVICES"):
        return None
    try:
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[0] if vis and vis.split(",")[0].isdigit() else None


# ----------------------------------------------------------------------------- CPU oracle
CPU_CURVE_SIDES = (40, 50, 60, 70)  # oracle timed at n = 1,600 ... 4,900 (jittered m x m grids)
BATCH_REPLICATES, BATCH_SIDES_SEED = 256, 5  # the batched leg's replicates: m_i = replicate_sides(256, seed 5)


def oracle_curve(n: int, sides=CPU_CURVE_SIDES) -> dict:
    """Time the FP64 oracle's log-likelihood (theta0) on m x m jittered grids and fit
    t(n) = a n^2 + b n^3 (generation by quadrature Bessel functions is O(n^2), the unblocked
    Cholesky O(n^3)) by least squares in relative error, then extrapolate to n.  Both CPU legs
    (cpu_baseline and --impl reference) use this curve."""
    import numpy as np

    import oracle
    from paper_1908_06936_gb300 import synth

    pts = []
    for m in sides:
        locs = synth.jittered_grid(m, 0)
        z = synth.normals(m * m, 0)
        t0 = time.perf_counter()
        oracle.loglik(locs, z, THETA0)
        pts.append((m * m, time.perf_counter() - t0))
    ns = np.array([p[0] for p in pts], dtype=float)
    ts = np.array([p[1] for p in pts])
    if len(pts) >= 2:
        A = np.stack([ns ** 2 / ts, ns ** 3 / ts], axis=1)
        (a, b), *_ = np.linalg.lstsq(A, np.ones_like(ts), rcond=None)
        if a < 0 or b <= 0:  # fall back to the pure n^3 law
            a, b = 0.0, float(np.exp(np.mean(np.log(ts) - 3.0 * np.log(ns))))
    else:
        a, b = 0.0, float(ts[0] / ns[0] ** 3)
    t_n = float(a) * float(n) ** 2 + float(b) * float(n) ** 3
    return {"points": [[int(x), float(y)] for x, y in pts], "a_n2": float(a), "b_n3": float(b), "seconds_at_n": t_n,
            "work_seconds": float(ts.sum()), "threads": oracle.max_threads()}


def oracle_check(m: int, curve: dict) -> dict:
    """One oracle evaluation on an m x m grid, against the fitted law's prediction."""
    import oracle
    from paper_1908_06936_gb300 import synth

    locs = synth.jittered_grid(m, 0)
    z = synth.normals(m * m, 0)
    t0 = time.perf_counter()
    oracle.loglik(locs, z, THETA0)
    dt = time.perf_counter() - t0
    pred = curve["a_n2"] * float(m * m) ** 2 + curve["b_n3"] * float(m * m) ** 3
    return {"n": m * m, "seconds": dt, "predicted_seconds": pred, "measured_over_predicted": dt / pred}


def batched_oracle_estimate(curve: dict, nrep: int = None, seed: int = None) -> dict:
    """Oracle time for one batch of the batched leg's replicates (n_i = m_i^2, m_i from
    synth.replicate_sides), each replicate predicted by the fitted t = a n^2 + b n^3 law and summed.
    The replicates' n_i = 400 ... 6,400 lie around the fitted range (1,600 ... 4,900)."""
    from paper_1908_06936_gb300 import synth

    nrep = BATCH_REPLICATES if nrep is None else nrep
    seed = BATCH_SIDES_SEED if seed is None else seed
    ns = [int(m) ** 2 for m in synth.replicate_sides(nrep, seed=seed)]
    t = float(sum(curve["a_n2"] * n ** 2 + curve["b_n3"] * n ** 3 for n in ns))
    return {"seconds_per_batch": t, "replicate_evals_per_s": nrep / t, "unit": "replicate-evals/s",
            "cores": curve["threads"], "kind": "oracle",
            "sample": "the oracle curve of cpu_baseline (t = a n^2 + b n^3) summed over the %d replicates "
                      "(sum n_i = %d)" % (nrep, sum(ns))}


def cpu_baseline_entry(n: int, curve: dict) -> dict:
    pts = ", ".join("n=%d %.2f s" % (a, b) for a, b in curve["points"])
    return {"value": 1.0 / curve["seconds_at_n"], "unit": "evals/s", "cores": curve["threads"], "kind": "oracle",
            "sample": "oracle log-likelihood timed on jittered grids (%s; %.1f s of CPU work on %d threads), "
                      "t = a n^2 + b n^3 fitted (a = %.3e s, b = %.3e s), extrapolated to n=%d"
                      % (pts, curve["work_seconds"], curve["threads"], curve["a_n2"], curve["b_n3"], n),
            "curve": curve}


# ----------------------------------------------------------------------------- workload
def make_inputs(m: int, seed: int):
    import numpy as np
    import torch

    import paper_1908_06936_gb300 as exa
    from paper_1908_06936_gb300 import synth

    n = m * m
    locs = synth.jittered_grid(m, seed)
    eps = synth.normals(n, seed)
    dl = torch.as_tensor(locs, device="cuda")
    de = torch.as_tensor(eps, device="cuda")
    with exa.Context() as c:  # exact realisation Z = L eps from the mixed factor (data, not the timed quantity)
        dz = c.simulate(dl, de, THETA0, exa.EXA_MIXED_TF32X3)
    torch.cuda.synchronize()
    return locs, dl, dz, np.ascontiguousarray(dz.cpu().numpy())


# DRAM traffic of the dominant kernel relative to its algorithmic bytes, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum over the launch's algorithmic bytes) of the same
# kernel on a C larger than L2; the per-launch traffic of the bench is this ratio times the
# average algorithmic bytes of its timed launches.  Keyed by kernel class; the capture and its
# command are summarised in profiles/gemm_t3_pair_bench_n90000.md (all 122 launches of one
# n = 90,000 factorisation, 1-pass metrics).
TRAFFIC_RATIO = {"gemm_tf32x3_pair": 1.522}


def class_roofline(st: dict, pk: dict) -> dict:
    """Roofline of one kernel class: algorithmic flops (or bytes) of its timed launch groups over
    their event-timed duration, against the peak of the unit that bounds the class."""
    nt = st["timed_launches"]
    name = st["name"]
    if nt == 0 or st["ms"] <= 0:
        return {"kernel": name, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None}
    avg_ms = st["ms"] / nt
    extra = {}
    flop_rate = st["timed_flops"] / (st["ms"] * 1e-3) / 1e12
    if name in ("gemm_tf32x3_tc", "gemm_tf32x3_pair"):
        ach, peak = flop_rate, pk["tf32"]
        bound, unit, note = "tensor", "TFLOP/s", ("useful flops (n^3/3 accounting) vs the tf32 dense peak; three tf32 "
                                                  "MMAs per useful product (far tiles one), so the ceiling is ~1/3")
        extra["frac_of_three_product_ceiling"] = 3.0 * ach / peak
    elif name in ("gemm_ozaki_tc",):
        ach, peak = flop_rate, pk["bf16"]
        bound, unit, note = "tensor", "TFLOP/s", "useful flops vs bf16 peak (15 bf16 MMAs per useful product)"
        extra["frac_of_digit_product_ceiling"] = 15.0 * ach / peak
    elif name in ("syrk_update_fp64", "trsm_panel_fp64", "dgemm_small_fp64"):
        ach, peak = flop_rate, pk["fp64"]
        bound, unit, note = "tensor", "TFLOP/s", "FP64 DMMA"
    elif name in ("potrf_diag_fp64", "symv_residual"):
        ach, peak = flop_rate, pk["fp64"]
        bound, unit, note = "alu", "TFLOP/s", ("FP64 ALU: diagonal-block factorisation and inverse (a latency chain) "
                                               "or the symmetric product (2 FMA per 8 B read), vs the FP64 peak")
    else:
        ach = st["timed_bytes"] / (st["ms"] * 1e-3) / 1e9
        peak = pk["hbm_gbs"]
        bound, unit, note = "hbm", "GB/s", "algorithmic bytes vs measured copy bandwidth"
        if name == "matern_gen":
            note += " (the kernel is FP64-issue bound: ~14 FP64 operations per entry, FP64 pipe ~90% busy in ncu)"
    traffic = None
    if name in TRAFFIC_RATIO:
        traffic = TRAFFIC_RATIO[name] * st["timed_bytes"] / nt
        extra["algorithmic_bytes_per_launch"] = st["timed_bytes"] / nt
    out = {"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
           "traffic": traffic, "avg_launch_ms": avg_ms, "launches": nt,
           "flops_per_launch": st["timed_flops"] / nt, "peak_source": pk["source"], "note": note}
    out.update(extra)
    return out


def roofline(stats: list, pk: dict) -> dict:
    """Roofline of the dominant kernel class (largest event-timed device time)."""
    dom = max(stats, key=lambda s: s["ms"]) if stats else None
    if not dom:
        return {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None}
    return class_roofline(dom, pk)


# kernel classes of the mixed evaluation that run (wholly or partly) on the look-ahead stream, on 20 to 48
# of the GPU's SMs beside the trailing update: their fraction of the whole GPU's peak is low by construction
LOOKAHEAD_CLASSES = ("potrf_diag_fp64", "split_rows", "gemm_tf32x3_tc")


def roofline_by_kernel(stats: list, pk: dict) -> list:
    """The roofline fraction of every kernel class of the timed region, largest device time first."""
    keys = ("kernel", "bound", "achieved", "peak", "unit", "frac", "avg_launch_ms", "launches", "note")
    rows = [class_roofline(st, pk) for st in sorted(stats, key=lambda s: -s["ms"])]
    out = []
    for r in rows:
        if r["bound"] is None:
            continue
        row = {k: r.get(k) for k in keys}
        if r["kernel"] in LOOKAHEAD_CLASSES:
            row["note"] += "; look-ahead stream work, on 20-48 SMs beside the trailing update (peak is the whole GPU's)"
        out.append(row)
    return out


def batched_leg(args, ctx) -> dict:
    """Config-5 batched replicates: 256 fields, n_i = m_i^2 with m_i ~ U{20..80}, theta0 = (1, 0.1, 0.5).

    The mixed-precision batch is captured once in a CUDA graph and replayed (one graph launch per
    evaluation of all replicates); the FP64 batch is timed with CUDA events on the same inputs."""
    import numpy as np
    import torch

    import paper_1908_06936_gb300 as exa
    from paper_1908_06936_gb300 import synth

    nrep = BATCH_REPLICATES
    sides = synth.replicate_sides(nrep, seed=BATCH_SIDES_SEED)
    ns = [int(m) ** 2 for m in sides]
    dl = [torch.as_tensor(synth.jittered_grid(int(m), 1000 + r), device="cuda") for r, m in enumerate(sides)]
    dz = [torch.as_tensor(synth.normals(int(m) ** 2, 1000 + r), device="cuda") for r, m in enumerate(sides)]
    th = torch.tensor([1.0, 0.1, 0.5] * nrep, dtype=torch.float64, device="cuda")
    out = {p: torch.empty(nrep, dtype=torch.float64, device="cuda") for p in ("fp64", "mixed", "tc")}
    st = {p: torch.empty(nrep, dtype=torch.int32, device="cuda") for p in ("fp64", "mixed", "tc")}
    flops = sum(((n + 63) // 64 * 64) ** 3 / 3.0 for n in ns)
    s = torch.cuda.Stream()
    res = {}
    with torch.cuda.stream(s):
        exa.exa_ctx_set_stream(ctx.handle, s.cuda_stream)
        try:
            args_m = (ctx.handle, nrep, ns, dl, dz, th, exa.EXA_MIXED_FP32, out["mixed"], st["mixed"])
            from paper_1908_06936_gb300 import tune

            tuned = tune.autotune_batched(ctx, ns, dl, dz, th, exa.EXA_MIXED_FP32, out["mixed"], st["mixed"],
                                          cache_path=None)
            for _ in range(2):
                ctx.check(exa.exa_loglik_batched(*args_m))
            s.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                ctx.check(exa.exa_loglik_batched(*args_m))
            g.replay()
            s.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = max(1, args.batched_steps)
            e0.record(s)
            for _ in range(reps):
                g.replay()
            e1.record(s)
            s.synchronize()
            res["mixed"] = e0.elapsed_time(e1) / reps
            # tensor-core form (128-wide tiles, TF32x3 panel solves and updates): graph replay too
            args_t = (ctx.handle, nrep, ns, dl, dz, th, exa.EXA_MIXED_TF32X3, out["tc"], st["tc"])
            for _ in range(2):
                ctx.check(exa.exa_loglik_batched(*args_t))
            s.synchronize()
            gt = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gt, stream=s):
                ctx.check(exa.exa_loglik_batched(*args_t))
            gt.replay()
            s.synchronize()
            e0.record(s)
            for _ in range(reps):
                gt.replay()
            e1.record(s)
            s.synchronize()
            res["tc"] = e0.elapsed_time(e1) / reps
            exa.exa_ctx_set_batched(ctx.handle, 0, 0, 0, 0)  # FP64 leg: tile 64, all resident CTAs
            ctx.check(exa.exa_loglik_batched(ctx.handle, nrep, ns, dl, dz, th, exa.EXA_FP64, out["fp64"], st["fp64"]))
            e0.record(s)
            for _ in range(max(1, args.batched_fp64_steps)):
                ctx.check(exa.exa_loglik_batched(ctx.handle, nrep, ns, dl, dz, th, exa.EXA_FP64, out["fp64"],
                                                 st["fp64"]))
            e1.record(s)
            s.synchronize()
            res["fp64"] = e0.elapsed_time(e1) / max(1, args.batched_fp64_steps)
        finally:
            exa.exa_ctx_set_batched(ctx.handle, 0, 0, 0, 0)
            exa.exa_ctx_set_stream(ctx.handle, torch.cuda.current_stream().cuda_stream)
    lm, lt, l64 = out["mixed"].cpu().numpy(), out["tc"].cpu().numpy(), out["fp64"].cpu().numpy()
    ok = bool(all((st[p] == 0).all().item() for p in st))
    rel = np.abs(lm - l64) / np.abs(l64)
    rel_t = np.abs(lt - l64) / np.abs(l64)
    leg = {"workload": "256 replicate fields, n_i = m_i^2, m_i ~ U{20..80} (jittered grids), theta0=(1, 0.1, 0.5), "
                       "per-replicate Z",
           "sum_n": int(sum(ns)), "flops_n3_over_3": flops, "all_status_ok": ok}
    for p in ("fp64", "mixed", "tc"):
        leg[p] = {"ms_per_batch": res[p], "replicate_evals_per_s": nrep / (res[p] / 1e3),
                  "tflops": flops / (res[p] / 1e3) / 1e12}
    leg["mixed"]["graph_replays"] = max(1, args.batched_steps)
    leg["mixed"]["prec"] = "EXA_MIXED_FP32 (persistent dataflow, FP32 off-diagonal tiles)"
    leg["mixed"]["autotuned"] = {"tile_nb": tuned["tile_nb"], "ctas_per_sm": tuned["ctas_per_sm"]}
    leg["tc"]["graph_replays"] = max(1, args.batched_steps)
    leg["tc"]["prec"] = "EXA_MIXED_TF32X3 (step-synchronous, tcgen05 TF32x3 panel solves and updates, tile 128)"
    leg["fp64"]["tile_nb"] = 64
    leg["speedup_mixed_vs_fp64"] = res["fp64"] / res["mixed"]
    leg["speedup_tc_vs_fp64"] = res["fp64"] / res["tc"]
    leg["max_rel_dl_vs_fp64"] = float(rel.max())
    leg["tc_max_rel_dl_vs_fp64"] = float(rel_t.max())
    return leg


def configs_leg(args, ctx) -> dict:
    """The smaller configurations: n = 1,600 (40x40 grid, theta0 = (1, 0.1, 0.5) and 10 seeded
    perturbations; FP64 and mixed evaluations/s with the phase split, the oracle timed on the host
    and checked at theta0) and n = 22,500 (150x150 grid, theta = (1.5, 0.2, 1.5): log-likelihood +
    gradient evaluations/s in FP64)."""
    import numpy as np
    import torch

    import oracle
    import paper_1908_06936_gb300 as exa
    from paper_1908_06936_gb300 import synth

    out = {}
    th0 = (1.0, 0.1, 0.5)
    locs = synth.jittered_grid(40, 0)
    eps = synth.normals(1600, 0)
    z = oracle.simulate(locs, th0, eps)
    dl, dz = torch.as_tensor(locs, device="cuda"), torch.as_tensor(z, device="cuda")
    thetas = [th0] + [tuple(t) for t in synth.theta_perturbations(th0, 10, seed=2)]
    for name, prec in (("fp64", exa.EXA_FP64), ("mixed", exa.EXA_MIXED_TF32X3)):
        for t in thetas[:3]:
            ctx.loglik_ex(dl, dz, t, prec)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = [ctx.loglik_ex(dl, dz, t, prec) for t in thetas]
        dt = time.perf_counter() - t0
        out["n1600_" + name] = {"evals_per_s": len(thetas) / dt,
                                "ms_gen": float(np.mean([r["ms_gen"] for r in res])),
                                "ms_chol": float(np.mean([r["ms_chol"] for r in res])),
                                "ms_solve": float(np.mean([r["ms_solve"] for r in res])),
                                "loglik_theta0": res[0]["loglik"]}
    t0 = time.perf_counter()
    ref = oracle.loglik(locs, z, th0)["l"]
    out["n1600_oracle"] = {"seconds_per_eval": time.perf_counter() - t0, "threads": os.cpu_count()}
    for name in ("fp64", "mixed"):
        out["n1600_" + name]["rel_dl_vs_oracle"] = abs(out["n1600_" + name]["loglik_theta0"] - ref) / abs(ref)
    thg = (1.5, 0.2, 1.5)
    locs = synth.jittered_grid(150, 4)
    dl = torch.as_tensor(locs, device="cuda")
    dz = ctx.simulate(dl, torch.as_tensor(synth.normals(22500, 4), device="cuda"), thg, exa.EXA_FP64)
    ctx.loglik_grad(dl, dz, thg)  # warm-up (allocates the second n^2 buffer)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    l, g = ctx.loglik_grad(dl, dz, thg)
    dt = time.perf_counter() - t0
    out["n22500_gradient_fp64"] = {"evals_per_s": 1.0 / dt, "seconds": dt, "loglik": l, "grad": list(map(float, g))}
    # mixed precision: mixed factor, FP64-refined Sigma^-1 z, Sigma^-1 on the tensor cores.  At the
    # gradient configuration's smooth theta (nu = 1.5, beta = 0.2) the 35-bit products cannot hold
    # Sigma's conditioning and the library refuses (EXA_ERR_IR_NOCONV); the mixed gradient is timed
    # on the same field at theta = (1, 0.1, 0.5) against the FP64 gradient there.
    try:
        ctx.loglik_grad(dl, dz, thg, exa.EXA_MIXED_TF32X3)
        cfg4 = "accepted"
    except exa.ExaError as err:
        cfg4 = "refused: " + str(err)
    thm = (1.0, 0.1, 0.5)
    l64, g64 = ctx.loglik_grad(dl, dz, thm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    l64, g64 = ctx.loglik_grad(dl, dz, thm)
    dt64 = time.perf_counter() - t0
    ctx.loglik_grad(dl, dz, thm, exa.EXA_MIXED_TF32X3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lm, gm = ctx.loglik_grad(dl, dz, thm, exa.EXA_MIXED_TF32X3)
    dtm = time.perf_counter() - t0
    gsc = max(1.0, float(np.max(np.abs(g64))))
    out["n22500_gradient_mixed"] = {"theta": list(thm), "at_gradient_config_theta": cfg4,
                                    "evals_per_s": 1.0 / dtm, "seconds": dtm, "loglik": lm,
                                    "grad": list(map(float, gm)), "fp64_seconds": dt64,
                                    "rel_dl_vs_fp64": abs(lm - l64) / abs(l64),
                                    "grad_err_vs_fp64_over_max": (np.abs(gm - g64) / gsc).tolist(),
                                    "speedup_vs_fp64": dt64 / dtm}
    # kriging at 2,048 new locations from the same 22,500 observations (means and variances)
    new = torch.as_tensor(synth.uniform_square(2048, 5), device="cuda")
    ctx.predict(dl, dz, thg, new)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mean, var = ctx.predict(dl, dz, thg, new)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out["n22500_predict_2048"] = {"seconds": dt, "predictions_per_s": 2048 / dt,
                                  "var_min": float(var.min().item()), "var_max": float(var.max().item())}
    # Fisher information at the n = 1,600 configuration
    locs = torch.as_tensor(synth.jittered_grid(40, 0), device="cuda")
    ctx.fisher(locs, th0)
    t0 = time.perf_counter()
    F = ctx.fisher(locs, th0)
    out["n1600_fisher"] = {"seconds": time.perf_counter() - t0, "fisher": F.tolist()}
    return out


def theta_grid_leg(args, ctx) -> dict:
    """Mixed precision against the GPU's FP64 evaluation on the paper's parameter grid (Section III,
    Example 2: sigma^2 = 1, beta in {0.03, 0.1, 0.3}, nu in {0.5, 1, 2}) at n = 22,500 (150 x 150 jittered
    grid), Z = L eps at each theta from the FP64 factor.  Per theta: |dl|/|l|, the exact band, refinement
    steps, the status of the mixed call, and both device times."""
    import torch

    import paper_1908_06936_gb300 as exa
    from paper_1908_06936_gb300 import synth

    dl = torch.as_tensor(synth.jittered_grid(150, 8), device="cuda")
    de = torch.as_tensor(synth.normals(22500, 8), device="cuda")
    rows = []
    for beta in (0.03, 0.1, 0.3):
        for nu in (0.5, 1.0, 2.0):
            th = (1.0, beta, nu)
            row = {"theta": list(th)}
            try:
                dz = ctx.simulate(dl, de, th, exa.EXA_FP64)
                f = ctx.loglik_ex(dl, dz, th, exa.EXA_FP64)
            except exa.ExaError as err:
                row["fp64"] = "status %d: %s" % (err.status, err)
                rows.append(row)
                continue
            row["fp64_ms"] = f["ms_total"]
            row["loglik_fp64"] = f["loglik"]
            try:
                mx = ctx.loglik_ex(dl, dz, th, exa.EXA_MIXED_TF32X3)
                row.update({"mixed_ms": mx["ms_total"], "rel_dl": abs(mx["loglik"] - f["loglik"]) / abs(f["loglik"]),
                            "exact_band": mx["exact_band"], "n_tiles": mx["n_tiles"], "ir_iters": mx["ir_iters"],
                            "speedup": f["ms_total"] / mx["ms_total"], "mixed": "ok"})
            except exa.ExaError as err:
                row["mixed"] = "status %d: %s" % (err.status, err)
            rows.append(row)
    return {"workload": "n=22500 (150x150 jittered grid), Z = L eps per theta (FP64 factor); device times "
                        "of one evaluation each (exa_result.ms_total)", "rows": rows}


def mle_leg(args, ctx, prec_name="mixed") -> dict:
    """Maximum-likelihood fit of one field at n = 40,000 (200x200 jittered grid, theta0 = (1, 0.1, 0.5),
    Z = L eps from the mixed-precision factor): bounded Nelder-Mead in log(theta) from the lower bounds
    (the paper's start, Section III Example 2), every evaluation a log-likelihood in `prec_name`
    ("mixed" or "fp64"); the optimum is evaluated once more in FP64 for |dl|/|l| there."""
    import math

    import torch

    import paper_1908_06936_gb300 as exa
    from paper_1908_06936_gb300 import synth
    from paper_1908_06936_gb300.mle import fit_replicates_with

    th0 = (1.0, 0.1, 0.5)
    dl = torch.as_tensor(synth.jittered_grid(200, 6), device="cuda")
    dz = ctx.simulate(dl, torch.as_tensor(synth.normals(40000, 6), device="cuda"), th0, exa.EXA_MIXED_TF32X3)
    fails = [0]

    prec = exa.EXA_FP64 if prec_name == "fp64" else exa.EXA_MIXED_TF32X3

    def f(_r, t):
        try:
            return ctx.loglik(dl, dz, list(map(float, t)), prec)
        except exa.ExaError as e:
            if e.status in (2, 6):  # not SPD / refinement stalled: -inf, the search steps away
                fails[0] += 1
                return -math.inf
            raise

    f(0, th0)  # warm-up (allocates; one evaluation at theta0, not counted)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = fit_replicates_with(f, 1, ftol=1e-5, xtol=1e-4,
                              max_evals=args.mle_fp64_evals if prec_name == "fp64" else args.mle_evals)
    dt = time.perf_counter() - t0
    th = [float(v) for v in res["theta"][0]]
    lm = float(res["loglik"][0])
    l64 = ctx.loglik(dl, dz, th, exa.EXA_FP64)
    return {"workload": "n=40000 (200x200 jittered grid), Z = L eps at theta0 = (1, 0.1, 0.5); Nelder-Mead in "
                        "log(theta) from the lower bounds; %s evaluations" % prec_name,
            "evals": int(res["evals"][0]), "seconds": dt, "evals_per_s": int(res["evals"][0]) / dt,
            "not_spd_or_stalled": fails[0], "theta_hat": th, "loglik": lm, "loglik_fp64_at_theta_hat": l64,
            "rel_dl_at_theta_hat": abs(lm - l64) / abs(l64)}


def gradient_mle_leg(args, ctx) -> dict:
    """The gradient configuration's fit at n = 22,500 (150 x 150 jittered grid, Z = L eps at
    theta0 = (1.5, 0.2, 1.5), FP64 factor): L-BFGS-B with the library's FP64 adjoint gradient against
    bounded Nelder-Mead on l alone, both from the lower bounds, FP64 evaluations."""
    import torch

    import paper_1908_06936_gb300 as exa
    from paper_1908_06936_gb300 import mle, synth

    th0 = (1.5, 0.2, 1.5)
    dl = torch.as_tensor(synth.jittered_grid(150, 4), device="cuda")
    dz = ctx.simulate(dl, torch.as_tensor(synth.normals(22500, 4), device="cuda"), th0, exa.EXA_FP64)
    ctx.loglik_grad(dl, dz, th0)  # warm-up
    out = {"workload": "n=22500 (150x150 jittered grid), Z = L eps at theta0 = (1.5, 0.2, 1.5); FP64; start at "
                       "the lower bounds (0.01, 0.01, 0.1)"}
    for name, fit in (("lbfgsb_gradient", lambda: mle.fit_gradient(dl, dz, maxiter=args.grad_mle_iters, ctx=ctx)),
                      ("nelder_mead", lambda: mle.fit_derivative_free(dl, dz, maxfev=args.grad_mle_evals, ctx=ctx))):
        torch.cuda.synchronize()
        r = fit()
        out[name] = {"theta_hat": r["theta"], "loglik": r["loglik"], "evals": r["evals"], "seconds": r["seconds"],
                     "seconds_per_eval": r["time_per_eval"], "method": r["method"], "message": r.get("message")}
    return out


def batched_mle_leg(args) -> dict:
    """theta-hat distribution of the 256 config-5 replicates: every replicate fitted by its
    own bounded Nelder-Mead in log(theta), all advanced in lockstep by one CUDA-graph replay
    of the mixed-precision batch per step; the smallest replicates are re-fitted with the
    same search on the FP64 oracle (host cores) for comparison."""
    import numpy as np
    import torch

    import oracle
    import paper_1908_06936_gb300 as exa
    from paper_1908_06936_gb300 import synth
    from paper_1908_06936_gb300.mle import fit_replicates, fit_replicates_with

    nrep = 256
    sides = synth.replicate_sides(nrep, seed=5)
    locs = [synth.jittered_grid(int(m), 2000 + r) for r, m in enumerate(sides)]
    eps = [synth.normals(int(m) ** 2, 2000 + r) for r, m in enumerate(sides)]
    ns = [l.shape[0] for l in locs]
    dl = [torch.as_tensor(l, device="cuda") for l in locs]
    # exact realisations Z = L eps at theta0 (the library's FP64 factor)
    dz = []
    with exa.Context() as c:
        for l, e in zip(dl, eps):
            z = torch.empty(l.shape[0], dtype=torch.float64, device="cuda")
            c.check(exa.exa_simulate(c.handle, l, torch.as_tensor(e, device="cuda"), [1.0, 0.1, 0.5],
                                     l.shape[0], exa.EXA_FP64, z))
            dz.append(z)
    torch.cuda.synchronize()
    kw = dict(x0=None, ftol=1e-5, xtol=1e-4, max_evals=args.batched_mle_evals)
    res = fit_replicates(ns, dl, dz, exa.EXA_MIXED_FP32, **kw)
    th = res["theta"]
    small = list(np.argsort(ns)[:2])
    zs_host = [dz[r].cpu().numpy() for r in small]
    ref = fit_replicates_with(lambda i, t: oracle.loglik(locs[small[i]], zs_host[i], t)["l"], len(small), **kw)
    return {"workload": "256 replicates (config 5 sizes), Z = L eps at theta0 = (1, 0.1, 0.5); start at the lower "
                        "bounds; mixed-precision batched evaluations",
            "steps": res["steps"], "seconds": res["seconds"], "replicate_evals_per_s": res["replicate_evals_per_s"],
            "evals_mean": float(np.mean(res["evals"])), "converged_before_budget": int(np.sum(res["evals"] < kw["max_evals"])),
            "theta_hat_median": np.median(th, axis=0).tolist(), "theta_hat_mean": np.mean(th, axis=0).tolist(),
            "theta_hat_std": np.std(th, axis=0).tolist(),
            "theta_hat_q10_q90": [np.quantile(th, 0.1, axis=0).tolist(), np.quantile(th, 0.9, axis=0).tolist()],
            "oracle_check": [{"replicate": int(r), "n": int(ns[r]), "theta_gpu": th[r].tolist(),
                              "theta_oracle": ref["theta"][i].tolist(), "loglik_gpu": float(res["loglik"][r]),
                              "loglik_oracle": float(ref["loglik"][i])} for i, r in enumerate(small)]}


def aggregate_over_ranks(ms_total: float, units_per_rank: float, world: int, device=None) -> tuple[float, float]:
    """Whole-job timing of N independent replicas: the slowest rank's timed region (max over
    ranks, an all-reduce on the default process group when world > 1) and the throughput of
    all ranks' units over that time, units per second.  Returns (ms_max, value)."""
    import torch

    t = torch.tensor([float(ms_total)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as tdist

        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * units_per_rank / (ms_max / 1e3)


def record_steps(step, k: int, stream, event_cls) -> tuple[list, object]:
    """Runs step() k times with a timing event recorded on `stream` before the first step and after
    each one (k + 1 events, no synchronisation between steps).  Returns (events, last result)."""
    evs = [event_cls(enable_timing=True) for _ in range(k + 1)]
    evs[0].record(stream)
    res = None
    for i in range(k):
        res = step()
        evs[i + 1].record(stream)
    return evs, res


def step_times(evs) -> tuple[float, list[float]]:
    """(ms from the first event to the last, ms of each step) of events from record_steps, once the
    stream has been synchronised."""
    return evs[0].elapsed_time(evs[-1]), [evs[i].elapsed_time(evs[i + 1]) for i in range(len(evs) - 1)]


def run_ours(args, rank: int, world: int) -> dict | None:
    import numpy as np
    import torch

    import paper_1908_06936_gb300 as exa

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    prec = exa.PREC[args.prec]
    m = args.m
    n = m * m
    locs, dl, dz, z_host = make_inputs(m, seed=rank)
    ctx = exa.Context()
    # warm-up
    for _ in range(args.warmup):
        ctx.loglik_ex(dl, dz, THETA0, prec)
    torch.cuda.synchronize()
    exa.exa_profile_read(ctx.handle, reset=1)
    exa.exa_profile_enable(ctx.handle, 1)
    clocks = ClockSampler(gpu_id_for_smi())
    clocks.start()
    time.sleep(0.5)
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    evs, res = record_steps(lambda: ctx.loglik_ex(dl, dz, THETA0, prec), args.steps, s, torch.cuda.Event)
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    ms_total, ms_steps = step_times(evs)
    clk = clocks.stop()
    stats = exa.exa_profile_read(ctx.handle, reset=1)
    exa.exa_profile_enable(ctx.handle, 0)
    ms_max, value = aggregate_over_ranks(ms_total, args.steps, world, device="cuda")
    launches = int(sum(st["launches"] for st in stats))

    # end to end through the C ABI: pinned host inputs copied in every step, result read back
    h_locs = torch.as_tensor(locs).pin_memory()
    h_z = torch.as_tensor(z_host).pin_memory()
    d_locs2 = torch.empty_like(dl)
    d_z2 = torch.empty_like(dz)
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e2.record(s)
    for _ in range(e2e_steps):
        d_locs2.copy_(h_locs, non_blocking=True)
        d_z2.copy_(h_z, non_blocking=True)
        l_val = ctx.loglik(d_locs2, d_z2, THETA0, prec)  # the library returns l to the host
    e3.record(s)
    torch.cuda.synchronize()
    e2e_ms = e2.elapsed_time(e3) / e2e_steps
    e2e = {"value": world / (e2e_ms / 1e3), "unit": "evals/s", "h2d_bytes_per_step": int(h_locs.numel() * 8 + h_z.numel() * 8),
           "d2h_bytes_per_step": 8, "steps": e2e_steps}

    out = None
    if rank == 0:
        chol_tflops = (n ** 3 / 3.0) / (res["ms_chol"] * 1e-3) / 1e12
        fp64 = None
        if args.fp64_steps > 0:
            # warm-up: every FP64 kernel loaded and run once (a 1,600-location field); the n = 90,000
            # buffers are the mixed leg's, already held
            from paper_1908_06936_gb300 import synth as _synth

            wl = torch.as_tensor(_synth.jittered_grid(40, 9), device="cuda")
            ctx.loglik_ex(wl, torch.as_tensor(_synth.normals(1600, 9), device="cuda"), THETA0, exa.EXA_FP64)
            ms, rr = [], None
            for _ in range(args.fp64_steps):
                rr = ctx.loglik_ex(dl, dz, THETA0, exa.EXA_FP64)
                ms.append(rr["ms_total"])
            fp64 = {"evals_per_s": 1e3 / statistics.mean(ms), "ms_per_eval": statistics.mean(ms),
                    "chol_ms": rr["ms_chol"], "chol_tflops": (n ** 3 / 3.0) / (rr["ms_chol"] * 1e-3) / 1e12,
                    "chol_frac_of_fp64_peak": (n ** 3 / 3.0) / (rr["ms_chol"] * 1e-3) / 1e12 / peaks()["fp64"],
                    "loglik": rr["loglik"], "steps": args.fp64_steps,
                    "warmup": "one FP64 evaluation at n=1,600 (kernels loaded; the n=90,000 buffers are the mixed leg's)"}
        pk = peaks()
        rl = roofline(stats, pk)
        probes = probe_peaks() if args.probe_peaks else None
        if fp64 and probes:
            best64 = max(probes["fp64_dmma_probe"], probes["fp64_dgemm_cublas"], probes["fp64_dfma_probe"])
            fp64["chol_frac_of_measured_fp64_peak"] = fp64["chol_tflops"] / best64
            # clock x SMs x 4 FP64 flops per clock per SM (the part's nominal 1.25 TFLOP/s at 2,070 MHz)
            if clk.get("sm_mhz"):
                nominal = 4.0 * probes["sms"] * clk["sm_mhz"] * 1e6 / 1e12
                fp64["fp64_clock_peak"] = nominal
                fp64["chol_frac_of_clock_peak"] = fp64["chol_tflops"] / nominal
        batched = batched_leg(args, ctx) if args.batched_steps > 0 else None
        configs = configs_leg(args, ctx) if args.configs else None
        batched_mle = batched_mle_leg(args) if args.batched_mle_evals > 0 else None
        mle = mle_leg(args, ctx) if args.mle_evals > 0 else None
        mle64 = mle_leg(args, ctx, "fp64") if args.mle_fp64_evals > 0 else None
        grad_mle = gradient_mle_leg(args, ctx) if args.grad_mle_evals > 0 else None
        # CPU oracle baseline: a bounded curve of oracle timings, fitted and extrapolated
        curve = oracle_curve(n)
        theta_grid = theta_grid_leg(args, ctx) if args.theta_grid else None
        out = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+tf32x3", "data": "synthetic",
            "config": {"workload": "n=%d (%dx%d jittered grid on [0,1]^2), theta0=(1, 0.03, 1.0), %s Cholesky with exact "
                                   "band + FP64 refinement; FP64 leg at the same n" % (n, m, m, args.prec),
                       "n": n, "theta0": list(THETA0), "prec": args.prec,
                       "l2": "working set %.0f GB >> 129 MB L2 (no flush needed)" % (2 * 8 * n * n / 1e9)},
            "mixed": {"evals_per_s": value / world, "chol_tflops": chol_tflops, "ms_gen": res["ms_gen"],
                      "ms_chol": res["ms_chol"], "ms_solve": res["ms_solve"], "ir_iters": res["ir_iters"],
                      "ir_resid": res["ir_resid"], "exact_band": res["exact_band"], "n_tiles": res["n_tiles"],
                      "loglik": res["loglik"], "ms_steps": ms_steps, "ms_step_best": min(ms_steps),
                      "ms_step_median": statistics.median(ms_steps)},
            "fp64": fp64,
            "rel_dl_vs_fp64": (abs(res["loglik"] - fp64["loglik"]) / abs(fp64["loglik"])) if fp64 else None,
            "speedup_mixed_vs_fp64": (fp64["ms_per_eval"] / (ms_max / args.steps)) if fp64 else None,
            "roofline": rl,
            "roofline_by_kernel": roofline_by_kernel(stats, pk),
            "batched": batched,
            "configs": configs,
            "batched_mle": batched_mle,
            "mle_n40000": mle,
            "mle_n40000_fp64": mle64,
            "gradient_mle_n22500": grad_mle,
            "kernels": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()} for st in stats],
            "theta_grid_n22500": theta_grid,
            "peaks_measured_here": probes,
            "cpu_baseline_check": oracle_check(args.oracle_check_m, curve) if args.oracle_check_m else None,
            "cpu_baseline": cpu_baseline_entry(n, curve),
            "batched_cpu_baseline": batched_oracle_estimate(curve) if batched else None,
            "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        }
    ctx.close()
    return out


def run_reference(args) -> dict:
    """The FP64 CPU oracle on the host cores: each step times the oracle curve (n = 1,600 ... 4,900) and
    extrapolates it to the workload's n by the fitted a n^2 + b n^3 law, exactly as cpu_baseline does."""
    m = args.m
    n = m * m
    for _ in range(args.warmup):
        oracle_curve(n, sides=CPU_CURVE_SIDES[:1])
    curves = [oracle_curve(n) for _ in range(args.steps)]
    t_n = sorted(c["seconds_at_n"] for c in curves)[len(curves) // 2]  # median over steps
    curve = min(curves, key=lambda c: abs(c["seconds_at_n"] - t_n))
    cb = cpu_baseline_entry(n, curve)
    v = cb["value"]
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_n * 1e3,
            "ms_per_step_note": "projected time of one n=%d evaluation from the fitted a n^2 + b n^3 law (median over steps); "
                                "each step measured the oracle curve for %.1f s" % (n, curve["work_seconds"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "n=%d (%dx%d jittered grid), theta0=(1, 0.03, 1.0); FP64 CPU oracle timed on "
                                   "jittered grids of n = 1,600 ... 4,900 and extrapolated by the fitted a n^2 + b n^3 law"
                                   % (n, m, m), "n": n},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--m", type=int, default=300, help="grid side (n = m^2)")
    ap.add_argument("--prec", choices=["tf32x3"], default="tf32x3")
    ap.add_argument("--fp64-steps", type=int, default=1, help="FP64 evaluations at the same n (0 to skip)")
    ap.add_argument("--batched-steps", type=int, default=3,
                    help="graph replays of the 256-replicate mixed batch (0 skips the batched leg)")
    ap.add_argument("--configs", type=int, default=1, help="also time the n=1,600 and n=22,500 configurations (0 skips)")
    ap.add_argument("--mle-evals", type=int, default=0,
                    help="maximum-likelihood fit at n=40,000 with this many mixed evaluations at most (0 skips)")
    ap.add_argument("--mle-fp64-evals", type=int, default=0,
                    help="the same n=40,000 fit with FP64 evaluations, at most this many (0 skips)")
    ap.add_argument("--grad-mle-evals", type=int, default=0,
                    help="n=22,500 gradient configuration: Nelder-Mead with this many FP64 evaluations at most "
                         "against L-BFGS-B with the adjoint gradient (0 skips)")
    ap.add_argument("--grad-mle-iters", type=int, default=60, help="L-BFGS-B iterations at most")
    ap.add_argument("--batched-mle-evals", type=int, default=0,
                    help="fit theta for the 256 batched replicates with this many evaluations each (0 skips)")
    ap.add_argument("--batched-fp64-steps", type=int, default=1, help="timed FP64 runs of the same batch")
    ap.add_argument("--probe-peaks", type=int, default=1, help="time the FP64 and TF32 peak probes (0 skips)")
    ap.add_argument("--theta-grid", type=int, default=1,
                    help="mixed vs FP64 on the paper's theta grid at n=22,500 (0 skips)")
    ap.add_argument("--oracle-check-m", type=int, default=0,
                    help="also time the oracle once on an m x m grid to check the n^3 extrapolation (0 skips)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1908_06936_gb300 import build as exa_build

    if rank == 0:
        exa_build.build()
    if world > 1:
        tdist.barrier()
    out = run_ours(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as tdist

        tdist.barrier()
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
