"""Host logic of bench.py on the CPU: the multi-rank helpers (gloo, two ranks),
the reference arm's JSON line, and the kernel roofline model."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch
    import torch.distributed as dist
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    got = bench.max_over_ranks(10.0 * (rank + 1), w, torch.device("cpu"))
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((rank, got))


def test_two_rank_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 20.0, 1: 20.0}


def test_single_rank_helpers_need_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    bench.barrier(1)


class _Args:
    steps = 2
    warmup = 0


def test_reference_arm_line(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    bench.run_reference(_Args())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_reference_arm_other_ranks_print_nothing(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(_Args())
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kernel_model_counts(precision):
    import bench
    s = 4
    g = bench.kernel_model("gram", precision, s)
    assert g["flops"] == 3 * 15 * 4                      # 15 entries, 2 FMA each, 3 systems
    assert g["bytes"] == 5 * 6 * (8 if precision == "fp64" else 4)
    assert bench.kernel_model("matvec", precision, s)["fp64"] == (precision == "fp64")


def test_traffic_lookup_needs_matching_sources(tmp_path, monkeypatch):
    import bench
    f = tmp_path / "t.txt"
    f.write_text(f"traffic gram fp64 1234.5 {bench.kernel_source_hash()}\n"
                 "traffic matvec fp64 99 0000\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_traffic("gram", "fp64") == 1234.5
    assert bench.measured_traffic("matvec", "fp64") is None       # taken from other sources
    assert bench.measured_traffic("update", "fp64") is None       # not captured
