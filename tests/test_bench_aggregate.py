"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the job's
time is the maximum over ranks and its units the sum (weak scaling of
independent problems)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate(1.0 + rank, 10.0 * (rank + 1), world, device="cpu")
    q.put((rank, t, u))
    dist.destroy_process_group()


def test_aggregate_max_time_sum_units_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t, u in res:
        assert t == pytest.approx(2.0) and u == pytest.approx(30.0)


def test_aggregate_single_rank_is_identity():
    import bench
    assert bench.aggregate(1.5, 7.0, 1) == (1.5, 7.0)


def test_kernel_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    """roofline.traffic is the DRAM count of an ncu summary only while the
    kernel sources still hash to the value recorded there: a copy whose
    source differs by one byte reports none."""
    import hashlib
    import shutil
    import bench
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_2602_06658_gb300" / "csrc"
    csrc.mkdir(parents=True)
    h = hashlib.sha1()
    for f in ("gw_softmin_tc.cu", "gw_tc.cuh", "gw_tc_ops.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_2602_06658_gb300", "csrc", f), csrc)
        h.update(open(csrc / f, "rb").read())
    (root / "profiles" / "softmin_tc_gmm8_100k_D32_f16x3.md").write_text(
        "dram_bytes_per_fused_launch: 123456789\nkernel_source_sha1: %s\n" % h.hexdigest())
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.tc_kernel_traffic()[0] == 123456789
    with open(csrc / "gw_tc.cuh", "a") as fh:
        fh.write("\n")
    t2, why2 = bench.tc_kernel_traffic()
    assert t2 is None and "changed" in why2
