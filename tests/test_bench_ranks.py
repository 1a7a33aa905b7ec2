"""The host logic of bench.py's multi-GPU runs (replicas, one process per GPU) with two gloo ranks on
the CPU: the job's time is the slowest rank's, the rate counts every rank's work, and only rank 0
runs the reference arm."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_max = bench.max_over_ranks(1.0 + rank, device="cpu")   # rank r took 1 + r seconds
    rate = bench.whole_job_rate(100.0, world, t_max)
    # the reference arm: every rank but 0 returns at once, without output
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": world})()
    buf = io.StringIO()
    if rank != 0:
        with redirect_stdout(buf):
            bench.run_reference(args)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"t_max": t_max, "rate": rate, "ref_out": buf.getvalue()}, fh)


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        res = json.load(open(tmp_path / f"r{r}.json"))
        assert res["t_max"] == 2.0                   # the slowest rank's time on every rank
        assert res["rate"] == pytest.approx(100.0)   # 2 ranks x 100 units / 2 s
        assert res["ref_out"] == ""


def test_apply_summary_and_guard():
    # per-precision summary against the FP64 apply (2-norm and infinity-norm relative errors), and
    # an auxiliary measurement that raises is recorded, not propagated
    sys.path.insert(0, ROOT)
    import bench
    ref = torch.tensor([1.0, -2.0, 4.0], dtype=torch.float64)
    out = ref + torch.tensor([0.0, 1e-6, -2e-6], dtype=torch.float64)
    s = bench.apply_summary({0: {"out": ref, "ms": 3.0, "phases": {}},
                             1: {"out": out, "ms": 1.5, "phases": {"k": (1.0, 2)}}})
    assert s["mixed"]["speedup_vs_fp64"] == pytest.approx(2.0)
    assert s["mixed"]["rel_err_inf_vs_fp64"] == pytest.approx(2e-6 / 4.0)
    assert s["mixed"]["rel_err_vs_fp64"] == pytest.approx((1e-12 + 4e-12) ** 0.5 / 21 ** 0.5)
    assert s["mixed"]["phases_ms"]["k"] == {"ms": 1.0, "calls": 2}

    def boom():
        raise RuntimeError("no device")

    assert bench.guarded(boom) == {"error": "RuntimeError: no device"}
    assert bench.guarded(lambda a: a + 1, 2) == 3
