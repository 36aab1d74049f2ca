"""bench.py's reference arm (the FP64 CPU oracle on the host cores) keeps the JSON-line
contract: run for real (the oracle timed on small grids, extrapolated), no GPU needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["unit"] == "evals/s" and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["value"] > 0 and d["config"]["n"] == 90000 and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "jittered grids" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # each step timed the oracle on several grid sizes; the fitted a n^2 + b n^3 law gives the full workload's time
    cv = cb["curve"]
    assert len(cv["points"]) >= 2 and cv["a_n2"] >= 0 and cv["b_n3"] > 0
    n = d["config"]["n"]
    assert abs(cv["a_n2"] * n ** 2 + cv["b_n3"] * n ** 3 - cv["seconds_at_n"]) <= 1e-9 * cv["seconds_at_n"]
    assert abs(d["ms_per_step"] / 1e3 - 1.0 / d["value"]) <= 1e-9 * d["ms_per_step"] / 1e3


def test_batched_oracle_estimate_sums_the_law_over_the_batched_replicates():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1908_06936_gb300 import synth

    curve = {"a_n2": 2.0e-9, "b_n3": 3.0e-12, "threads": 16}
    est = bench.batched_oracle_estimate(curve)
    sides = synth.replicate_sides(256, seed=5)  # the batched leg's replicates (m_i ~ U{20..80})
    assert (bench.BATCH_REPLICATES, bench.BATCH_SIDES_SEED) == (256, 5)
    want = sum(2.0e-9 * float(m) ** 4 + 3.0e-12 * float(m) ** 6 for m in sides)
    assert abs(est["seconds_per_batch"] - want) <= 1e-12 * want
    assert abs(est["replicate_evals_per_s"] - 256 / want) <= 1e-12 * 256 / want
    assert est["kind"] == "oracle" and est["cores"] == 16 and "sum n_i = %d" % sum(int(m) ** 2 for m in sides) in est["sample"]
    json.dumps(est)  # goes into the bench's JSON line


def test_roofline_by_kernel_covers_every_timed_class():
    sys.path.insert(0, ROOT)
    import bench

    pk = {"hbm_gbs": 6000.0, "bf16": 1800.0, "tf32": 880.0, "fp64": 1.0, "source": "measured"}
    stats = [  # timed flops / bytes over event-timed ms, as exa_profile_read reports them
        {"name": "gemm_tf32x3_pair", "launches": 4, "timed_launches": 4, "ms": 8.0, "flops": 2.2e12,
         "bytes": 1e10, "timed_flops": 2.2e12, "timed_bytes": 1e10},
        {"name": "split_rows", "launches": 10, "timed_launches": 5, "ms": 2.0, "flops": 0.0, "bytes": 6e9,
         "timed_flops": 0.0, "timed_bytes": 3e9},
        {"name": "symv_residual", "launches": 1, "timed_launches": 1, "ms": 4.0, "flops": 2e9, "bytes": 8e9,
         "timed_flops": 2e9, "timed_bytes": 8e9},
        {"name": "other", "launches": 2, "timed_launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 1e6,
         "timed_flops": 0.0, "timed_bytes": 0.0},
    ]
    rows = bench.roofline_by_kernel(stats, pk)
    assert [r["kernel"] for r in rows] == ["gemm_tf32x3_pair", "symv_residual", "split_rows"]  # untimed dropped
    pair, symv, split = rows
    assert pair["bound"] == "tensor" and abs(pair["achieved"] - 2.2e12 / 8e-3 / 1e12) < 1e-9
    assert abs(pair["frac"] - pair["achieved"] / 880.0) < 1e-12
    assert symv["bound"] == "alu" and abs(symv["achieved"] - 0.5) < 1e-12 and symv["unit"] == "TFLOP/s"
    assert split["bound"] == "hbm" and abs(split["achieved"] - 3e9 / 2e-3 / 1e9) < 1e-9 and "look-ahead" in split["note"]
    # the headline object is the dominant class's
    assert bench.roofline(stats, pk) == bench.class_roofline(stats[0], pk)
    json.dumps(rows)
