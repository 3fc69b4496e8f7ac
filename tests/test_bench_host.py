"""Host-side logic of bench.py, on CPU: the replicas' max-over-ranks timing
with two gloo ranks, the whole-job rate, and the reference arm's rank rule."""
import os
import socket
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(values[rank], dist, "cpu")
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    values = [12.5, 40.25]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 40.25, 1: 40.25}


def test_job_rate_counts_all_ranks():
    assert bench.max_over_ranks(7.0) == 7.0
    # 2 ranks x 1e6 edges x 4 steps in 2 s
    assert bench.job_rate(1_000_000, 4, 2, 2000.0) == pytest.approx(4e6)


def test_reference_arm_only_rank0_reports(monkeypatch):
    class A:
        steps, warmup, workload = 1, 0, "rmat20"
    assert bench.bench_reference(A(), rank=1, world=2) is None


def test_ncu_traffic_entries_name_a_workload_a_kernel_and_a_capture():
    """Each DRAM-traffic figure the bench reports names a timed workload, a
    kernel the bench times, the source hash it was taken of, and a committed
    capture summary that states the same read and write bytes."""
    import re
    import graphgen
    for (workload, kernel), entry in bench.NCU_TRAFFIC.items():
        assert workload in graphgen.WORKLOADS
        assert kernel in bench.KERNEL_SOURCE
        assert len(entry["source_sha256"]) == 64
        path = re.search(r"profiles/\S+\.md", entry["source"]).group(0)
        text = open(os.path.join(ROOT, path)).read()
        gb = [float(x) for x in re.findall(r"(\d+\.\d+) GB", text)]
        # some row of the summary holds the read and write figures that sum
        # to the reported bytes (to the summary's rounding)
        assert any(abs((a + b) * 1e9 - entry["bytes"]) < 0.02e9 * max(1.0, (a + b) / 10)
                   for a, b in zip(gb, gb[1:])), (workload, kernel)


def test_ncu_traffic_is_dropped_once_the_kernel_source_changes(monkeypatch):
    """Captured bytes describe one version of a kernel: with another source
    hash the bench reports no traffic."""
    kernel = "masked product, support"
    cur = bench.kernel_source_sha(kernel)
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("rmat24", kernel),
                        {"bytes": 1, "source": "x", "source_sha256": cur})
    assert bench.ncu_traffic("rmat24", kernel)["bytes"] == 1
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("rmat24", kernel),
                        {"bytes": 1, "source": "x", "source_sha256": "0" * 64})
    assert bench.ncu_traffic("rmat24", kernel) is None
    assert bench.ncu_traffic("rmat24", "peel (k_peel)") is None or \
        ("rmat24", "peel (k_peel)") in bench.NCU_TRAFFIC


def test_oracle_fixture_gives_the_whole_workload_time():
    full = bench.oracle_fixture("rmat20")
    assert full["edges"] == 15699719 and full["wall_s"] > 0
    assert bench.oracle_fixture("no_such_workload") is None
