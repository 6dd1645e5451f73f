"""Host logic of the benchmark on the CPU: two gloo ranks, the shared config,
the profiled records.

Every box here has one GPU, so N > 1 runs independent replicas, one per rank:
the job's time is the slowest rank's (all-reduce MAX) and its throughput is all
ranks' cell updates over that time; rank 0 alone prints.  The oracle arm runs
on rank 0 only, the other ranks exit 0 without work.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        m = bench.max_over_ranks(times[rank], ws, torch.device("cpu"))
        out[rank] = (m, bench.replica_value(1000, 10, ws, m))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    times = [12.5, 20.0]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, times, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    for r in range(ws):
        m, v = out[r]
        assert m == 20.0                                   # every rank sees the max
        assert v == pytest.approx(ws * 1000 * 10 / 0.020)  # all ranks' work over it


def test_one_rank_needs_no_process_group():
    assert bench.max_over_ranks(7.0, 1, None) == 7.0
    assert bench.replica_value(10, 3, 1, 1000.0) == pytest.approx(30.0)


def test_oracle_arm_runs_on_rank_0_only(monkeypatch):
    """Under torchrun the oracle arm's rank 1 returns 0 at once and prints nothing."""
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = bench.parse(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    assert buf.getvalue() == ""


def test_both_arms_report_the_same_config():
    """The oracle arm times the same workload as the GPU arm: one config dict."""
    args = bench.parse([])
    w = bench.workload(args)
    cfg = bench.arm_config(args, w, 1)
    assert cfg["workload"] == "sphere_512cubed_R150_ti120_f32_27pt"
    assert cfg["grid"] == [512, 512, 512] and cfg["scheme"] == "TI_<120>" and cfg["bc"] == "periodic"
    assert bench.arm_config(bench.parse(["--impl", "reference"]), w, 1) == cfg


def test_profiled_figures_only_for_the_captured_sources(monkeypatch, tmp_path):
    """The traffic and ALU-ceiling records of profiles/traffic.json are used
    only while the stencil sources hash to the captured version."""
    import json
    key = "spfm_step_kernel_f32_27pt_ti120_512"
    rec = {key: {"source_hash": bench.source_hash(), "bytes_per_launch": 1.0e9},
           "spfm_step_kernel_f32_27pt_local": {"source_hash": bench.source_hash(),
                                               "warp_inst_per_cell": 5.8}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(path))
    assert bench.profiled_traffic(key) == 1.0e9
    assert bench.profiled_record("spfm_step_kernel_f32_27pt_local", "warp_inst_per_cell") == 5.8
    assert bench.profiled_traffic("no_such_kernel") is None
    monkeypatch.setattr(bench, "source_hash", lambda names=None: "0000000000000000")
    assert bench.profiled_traffic(key) is None


def test_committed_profile_record_names_a_source_hash():
    """Every record of the committed traffic file carries the hash of the
    stencil sources it was captured on (stale records read as null)."""
    import json
    with open(bench.TRAFFIC_PATH) as f:
        d = json.load(f)
    recs = [v for v in d.values() if isinstance(v, dict) and "bytes_per_launch" in v]
    assert recs and all(len(v.get("source_hash", "")) == 16 for v in recs)
