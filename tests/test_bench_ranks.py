"""The N > 1 path of bench.py on the host: N independent replicas (one process per GPU,
no data-path collective), whole-job throughput = all ranks' evaluations over the
slowest rank's timed region.  Run as two gloo ranks on the CPU; no GPU needed."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, steps, out):
    import torch.distributed as tdist

    sys.path.insert(0, ROOT)
    import bench

    tdist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        tdist.barrier()
        out[rank] = bench.aggregate_over_ranks(times[rank], steps, world)
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("times", [(1000.0, 1500.0), (2500.0, 400.0)])
def test_two_ranks_take_the_slowest_and_count_both(times):
    world, steps = 2, 3
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), times, steps, out), nprocs=world, join=True)
        res = dict(out)
    ms_max = max(times)
    for r in range(world):
        assert res[r][0] == ms_max
        assert res[r][1] == pytest.approx(world * steps / (ms_max / 1e3), rel=1e-15)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    ms, v = bench.aggregate_over_ranks(2000.0, 3, 1)
    assert ms == 2000.0 and v == pytest.approx(1.5, rel=1e-15)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    # under torchrun the reference arm runs on rank 0 alone; the other ranks exit without work
    sys.path.insert(0, ROOT)
    import bench

    called = []
    monkeypatch.setattr(bench, "run_reference", lambda args: called.append(args) or {"impl": "reference"})
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    for rank, expect in (("1", ""), ("0", '{"impl": "reference"}\n')):
        monkeypatch.setenv("RANK", rank)
        monkeypatch.setenv("WORLD_SIZE", "2")
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.main()
        assert buf.getvalue() == expect
    assert len(called) == 1


class _Clock:
    t = 0.0


class _FakeEvent:
    """Stands in for torch.cuda.Event: record() reads a host clock that the fake steps advance."""

    def __init__(self, enable_timing=False):
        assert enable_timing
        self.t = None

    def record(self, stream):
        assert stream == "stream"
        self.t = _Clock.t

    def elapsed_time(self, other):
        return other.t - self.t


@pytest.mark.parametrize("durations", [[5.0], [3.0, 7.0, 4.0], [2.0, 2.0, 9.0, 1.0, 2.5]])
def test_timed_steps_give_each_step_and_the_whole_region(durations):
    sys.path.insert(0, ROOT)
    import bench

    _Clock.t = 100.0
    it = iter(durations)

    def step():
        d = next(it)
        _Clock.t += d
        return d

    evs, last = bench.record_steps(step, len(durations), "stream", _FakeEvent)
    assert len(evs) == len(durations) + 1 and last == durations[-1]
    total, per = bench.step_times(evs)
    assert per == durations
    assert total == pytest.approx(sum(durations))
