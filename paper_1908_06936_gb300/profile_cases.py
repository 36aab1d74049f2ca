"""Single-kernel cases for profiling the library's hot kernels in isolation.

Each case runs one C-ABI call twice (a warm-up, then the call to capture) on a
problem larger than the 129 MB L2, so DRAM counters mean something, but a few GB
on the device at most, and prints the device time of the second call (CUDA
events on the context stream).  Under ncu, skip the warm-up's launches of the
kernel (``-s``) and capture one launch (``-c 1``).

  python -m paper_1908_06936_gb300.profile_cases gemm-pair --c 16384 --k 1024
  python -m paper_1908_06936_gb300.profile_cases gemm-oz --c 16384
  python -m paper_1908_06936_gb300.profile_cases potrf --n 16384
  python -m paper_1908_06936_gb300.profile_cases matern --m 128
  python -m paper_1908_06936_gb300.profile_cases timeline --m 300 --out timeline.json
  python -m paper_1908_06936_gb300.profile_cases timeline --m 150 --far-margin 12 --fp64-check

gemm-pair / gemm-oz: exa_gemm_update, C -= A B^T with C (c x c, FP64) and A, B
(c x k, FP64, standard normal); gemm-pair is the CTA-pair TF32x3 trailing-update
kernel (k = 1024 reduces two operand pairs per pass, as the fused two-panel pass
of the factorisation), gemm-oz the exact digit-slice band kernel (k <= 512).
potrf: exa_potrf of the Matern covariance of an m x m jittered grid (FP64 tiled
Cholesky: potrf_diag, trsm_panel, syrk_update).  matern: exa_covariance of an
m x m jittered grid (the generation kernel, lower triangle, one copy).  timeline: one
mixed-precision log-likelihood of an m x m jittered grid after a warm-up, with the library's
launch timeline recorded (exa_profile_timeline: start and end of every launch group on the
context and look-ahead streams), written as JSON to --out, plus per-stream busy time.
"""
from __future__ import annotations

import argparse
import json


def _timed(fn, stream):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def main(argv=None) -> dict:
    import torch

    import paper_1908_06936_gb300 as exa
    from paper_1908_06936_gb300 import synth

    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=["gemm-pair", "gemm-oz", "potrf", "matern", "timeline"])
    ap.add_argument("--out", default="timeline.json", help="timeline case: output file")
    ap.add_argument("--late", type=int, nargs=2, default=None, metavar=("ROWS", "SMS"),
                    help="timeline case: exa_ctx_set_lookahead_late(ROWS, SMS) before the evaluations")
    ap.add_argument("--fuse", type=int, default=None,
                    help="timeline case: exa_ctx_set_panel_fusion(ROWS) before the evaluations")
    ap.add_argument("--lookahead", type=int, default=None,
                    help="timeline case: exa_ctx_set_lookahead(SMS) before the evaluations")
    ap.add_argument("--far-margin", type=int, default=None,
                    help="timeline case: exa_ctx_set_far_tile_margin(BITS) before the evaluations")
    ap.add_argument("--fp64-check", action="store_true",
                    help="timeline case: also evaluate in FP64 and report |dl|/|l| of the mixed result")
    ap.add_argument("--c", type=int, default=16384, help="rows and columns of C (gemm cases)")
    ap.add_argument("--k", type=int, default=512, help="inner dimension (gemm cases)")
    ap.add_argument("--m", type=int, default=128, help="grid side, n = m^2 (potrf, matern)")
    ap.add_argument("--theta", type=float, nargs=3, default=(1.0, 0.03, 1.0))
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream()
    out = {"case": args.case}
    with exa.Context() as ctx:
        if args.case in ("gemm-pair", "gemm-oz"):
            kind = exa.EXA_GEMM_T3_PAIR if args.case == "gemm-pair" else exa.EXA_GEMM_OZ
            c, k = args.c, args.k
            g = torch.Generator(device="cuda").manual_seed(7)
            A = torch.randn((c, k), dtype=torch.float64, device="cuda", generator=g)
            B = torch.randn((c, k), dtype=torch.float64, device="cuda", generator=g)
            C = torch.zeros((c, c), dtype=torch.float64, device="cuda")
            call = lambda: ctx.check(exa.exa_gemm_update(ctx.handle, kind, c, c, k, A, B, C, c, 0))
            call()
            ms = _timed(call, s)
            out.update({"c": c, "k": k, "ms": ms, "useful_tflops": 2.0 * c * c * k / (ms * 1e-3) / 1e12,
                        "c_bytes_rw": 16.0 * c * c})
        elif args.case == "potrf":
            m = args.m
            n = m * m
            locs = torch.as_tensor(synth.jittered_grid(m, 3), device="cuda")
            S = ctx.covariance(locs, args.theta)
            work = torch.empty_like(S)

            def call():
                work.copy_(S)
                ctx.check(exa.exa_potrf(ctx.handle, work, n, n))

            call()
            ms = _timed(call, s)
            out.update({"n": n, "ms": ms, "tflops_n3_over_3": n ** 3 / 3.0 / (ms * 1e-3) / 1e12})
        elif args.case == "timeline":
            m = args.m
            n = m * m
            locs = torch.as_tensor(synth.jittered_grid(m, 0), device="cuda")
            z = torch.as_tensor(synth.normals(n, 0), device="cuda")
            if args.fp64_check:  # an exact realisation Z = L eps (FP64 factor) for the accuracy check
                z = ctx.simulate(locs, z, args.theta, exa.EXA_FP64)
            if args.late:
                ctx.check(exa.exa_ctx_set_lookahead_late(ctx.handle, args.late[0], args.late[1]))
            if args.fuse is not None:
                ctx.check(exa.exa_ctx_set_panel_fusion(ctx.handle, args.fuse))
            if args.lookahead is not None:
                ctx.check(exa.exa_ctx_set_lookahead(ctx.handle, args.lookahead))
            if args.far_margin is not None:
                ctx.check(exa.exa_ctx_set_far_tile_margin(ctx.handle, args.far_margin))
            ctx.loglik_ex(locs, z, args.theta, exa.EXA_MIXED_TF32X3)
            exa.exa_profile_enable(ctx.handle, 1)
            exa.exa_profile_timeline_enable(ctx.handle, 1)
            r = ctx.loglik_ex(locs, z, args.theta, exa.EXA_MIXED_TF32X3)
            tl = exa.exa_profile_timeline(ctx.handle)
            exa.exa_profile_enable(ctx.handle, 0)
            with open(args.out, "w") as fh:
                json.dump({"n": n, "theta": list(args.theta), "result": {k: r[k] for k in ("ms_gen", "ms_chol",
                                                                                             "ms_solve", "ms_total")},
                           "timeline": tl}, fh)
            busy = {}
            for name, st, a, b in tl:
                busy.setdefault(st, 0.0)
                busy[st] += b - a
            out.update({"n": n, "late": args.late, "fuse": args.fuse, "lookahead": args.lookahead,
                        "far_margin": args.far_margin, "loglik": r["loglik"], "records": len(tl),
                        "ms_total": r["ms_total"], "ms_chol": r["ms_chol"], "ir_iters": r["ir_iters"],
                        "busy_ms_by_stream": busy})
            if args.fp64_check:
                f = ctx.loglik_ex(locs, z, args.theta, exa.EXA_FP64)
                out["rel_dl_vs_fp64"] = abs(r["loglik"] - f["loglik"]) / abs(f["loglik"])
        else:
            m = args.m
            n = m * m
            locs = torch.as_tensor(synth.jittered_grid(m, 3), device="cuda")
            S = torch.empty((n, n), dtype=torch.float64, device="cuda")
            call = lambda: ctx.check(exa.exa_covariance(ctx.handle, locs, n, args.theta, S, n))
            call()
            ms = _timed(call, s)
            lower = n * (n + 1) / 2.0
            out.update({"n": n, "ms": ms, "entries_per_s": lower / (ms * 1e-3),
                        "write_gbs": 8.0 * lower / (ms * 1e-3) / 1e9})
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
