"""The multi-GPU path of bench.py is replicas only: every rank solves its own
copy of the workload, the job's step time is the maximum over ranks, and the
whole-job value counts every rank's units.  Checked here with two gloo ranks
on the CPU (the same reduction runs over NCCL on GPUs)."""
import importlib.util
import io
import json
import multiprocessing as mp
import os
import socket
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = load_bench()
        w, r, _ = bench.dist_setup()
        dist.barrier()
        ms_max = bench.replicas_max_ms(ms[rank], w, "cpu")
        q.put((r, w, ms_max, bench.whole_job_value(w, ms_max)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replicas_take_the_slowest_rank(world):
    ms = [12.5, 30.0, 7.0][:world]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, ms, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(o[0] for o in out) == list(range(world))
    for _, w, ms_max, value in out:
        assert w == world
        assert ms_max == max(ms)
        assert value == pytest.approx(world * 1000.0 / max(ms))


def test_single_process_needs_no_process_group():
    bench = load_bench()
    assert bench.replicas_max_ms(20.0, 1, "cpu") == 20.0
    assert bench.whole_job_value(1, 20.0) == pytest.approx(50.0)
    assert bench.whole_job_value(1, 20.0, units_per_step=4096) == pytest.approx(4096 * 50.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun the oracle arm prints its line from rank 0 alone; the
    other ranks exit 0 without work."""
    bench = load_bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a: called.append(a) or (1.0, 0.5, 0.1))
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.run_reference(type("A", (), {"steps": 2, "warmup": 1})())
    assert rc == 0 and buf.getvalue() == "" and not called
    monkeypatch.setenv("RANK", "0")
    with redirect_stdout(buf):
        rc = bench.run_reference(type("A", (), {"steps": 2, "warmup": 1})())
    line = json.loads(buf.getvalue())
    assert rc == 0 and line["impl"] == "reference" and line["n_gpus"] == 2
    # one evaluation (0.5 s) + one improvement (0.1 s) per step; a solve is
    # `systems` evaluations and `systems + outer` improvements
    systems, outer = bench.oracle_counts()
    assert len(called) == 3
    assert line["value"] == pytest.approx(1.0 / (systems * 0.5 + (systems + outer) * 0.1))
    assert line["ms_per_step"] == pytest.approx(600.0)
