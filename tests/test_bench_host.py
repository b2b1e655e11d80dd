"""Host logic of bench.py without a GPU: the max-over-ranks reduction of the replicas' times on
two gloo ranks, the reference arm's rank handling, and the algorithmic byte model of the
roofline kernels on the benchmark's finest level."""
import os
import socket

import pytest

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.max_over_ranks(1.5 + rank, "cpu")))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 2.5, 1: 2.5}


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import argparse
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=1, warmup=0, gpus=2, impl="reference")
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("fused,kernel,expected", [(True, "g", 322_006_180), (False, "gt", 314_204_300)])
def test_roofline_bytes_of_the_finest_level(fused, kernel, expected):
    """nnzb(G) = 719,335 blocks of 10 x 10 (adaptive FSAI, t_max = 6), N = 655,360: G's values and
    columns once, plus r and the partial products (fused) or t, p, e and the FP64 iterate."""
    info = {"d": 10, "n": 65536, "nnzb_G": 719_335, "nnzb_A": 586_756, "fused_fsai": int(fused)}
    ab = bench.algorithmic_bytes(info, 4, 4, 4, 8)
    assert ab[kernel] == expected
    assert bench.ROOFLINE[fused][0] == kernel


def test_reference_arm_prints_the_contract_line(capsys, monkeypatch):
    """The reference arm (the oracle on the host cores, here on the 8x8-patch version of the
    workload) prints one JSON line with the metric, a cpu_baseline describing the sample and an
    e2e entry without host-device copies."""
    import argparse
    import json
    monkeypatch.delenv("RANK", raising=False)
    bench.run_reference(argparse.Namespace(steps=2, warmup=1, gpus=1, impl="reference", cpu_m=8))
    lines = [line for line in capsys.readouterr().out.splitlines() if line.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is False
    assert d["config"]["oracle_patches"] == "8x8" and d["steps"] == 2
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_oracle_sample_is_observed_at_its_own_size():
    """The oracle's timings come from solves of the sample problem itself (PCG to 1e-8 with the
    workload's smoother settings), with the set-up timed apart."""
    o = bench.oracle_run(2, m=8)
    assert o["m"] == 8 and o["n_levels"] == 4 and o["unknowns"] == 640
    assert len(o["solve_ms"]) == 2 and all(t > 0 for t in o["solve_ms"])
    assert 0 < o["iters"] < 50 and o["hierarchy_s"] > 0 and o["smoother_setup_s"] > 0


def test_profiled_traffic_only_for_the_captured_sources(tmp_path, monkeypatch):
    """The roofline line carries the ncu DRAM bytes of its kernel only while the kernel's sources
    hash to the value recorded with the capture; a changed source (or no summary) gives None."""
    import hashlib
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "p.md"
    prof.write_text(f"traffic_bytes_per_launch: 303114752\nkernel_source_sha256: {digest}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("p.md", ("k.cu",)) == 303114752
    assert bench.profiled_traffic(None, ("k.cu",)) is None
    src.write_text("kernel v2\n")
    assert bench.profiled_traffic("p.md", ("k.cu",)) is None
    # the committed summary matches the committed sources of the fused kernel
    monkeypatch.undo()
    _, _, profile, sources = bench.ROOFLINE[True]
    assert bench.profiled_traffic(profile, sources) is not None, f"{profile} was captured from other sources"
