"""bench.py's multi-rank host logic on CPU: two gloo ranks combine their timed
regions (max) and units (sum); the reference arm runs on rank 0 only."""

import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.combine_ranks(dist, 10.0 + rank, 100 * (rank + 1), "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, units))


def test_two_gloo_ranks_combine_max_time_and_total_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 11.0, 300), (1, 11.0, 300)]


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(None, 12.5, 7, "cpu") == (12.5, 7)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""


def test_traffic_figure_follows_the_profiled_sources(tmp_path, monkeypatch):
    """bench.py reads the NTT's DRAM bytes per limb from the committed ncu summary only while the
    transform sources hash to the value recorded there."""
    sys.path.insert(0, ROOT)
    import bench
    got = bench.ntt_traffic_per_limb("k_ntt_fwd")
    text = open(os.path.join(ROOT, "profiles", "k_ntt_fwd_traffic_genotype_N16384.md")).read()
    recorded = float(text.split("`dram_bytes_per_limb`: `")[1].split("`")[0])
    assert got in (None, recorded)   # None once the transform sources change, until re-profiled
    # a summary whose recorded hash differs gives no figure
    fake = tmp_path / "profiles"
    fake.mkdir()
    (fake / "k_ntt_fwd_traffic_genotype_N16384.md").write_text(
        "- `dram_bytes_per_limb`: `1`\n- `sources_sha256`: `00` (other sources)\n")
    csrc = tmp_path / "paper_2204_12201_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("ntt.cu", "common.cuh"):
        (csrc / f).write_bytes(open(os.path.join(ROOT, "paper_2204_12201_gb300", "csrc", f), "rb").read())
    monkeypatch.setattr(bench.os.path, "abspath", lambda p: str(tmp_path / "bench.py"))
    assert bench.ntt_traffic_per_limb("k_ntt_fwd") is None
    assert bench.ntt_traffic_per_limb("k_other") is None


def test_kernel_roofline_takes_the_slower_bound():
    """Per class the roofline time is max(modmuls / ALU peak, bytes / HBM peak); frac = that / measured."""
    sys.path.insert(0, ROOT)
    import bench
    alu, gbs = 1e12, 5000.0
    prof = {"ntt_fwd": (2.0, 3, 1.5e9, 1e9),        # ALU 1.5 ms, HBM 0.2 ms -> alu, 0.75
            "moddown": (1.0, 1, 1e8, 4e9),          # ALU 0.1 ms, HBM 0.8 ms -> hbm, 0.8
            "tensor": (0.0, 0, 0.0, 0.0)}           # not launched: absent
    r = bench.kernel_rooflines(prof, alu, gbs)
    assert set(r) == {"ntt_fwd", "moddown"}
    assert r["ntt_fwd"]["bound"] == "alu" and abs(r["ntt_fwd"]["frac"] - 0.75) < 1e-9
    assert r["moddown"]["bound"] == "hbm" and abs(r["moddown"]["frac"] - 0.8) < 1e-9
    assert abs(r["moddown"]["alu_frac"] - 0.1) < 1e-9 and abs(r["ntt_fwd"]["hbm_frac"] - 0.1) < 1e-9
