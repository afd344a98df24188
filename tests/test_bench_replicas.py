"""The benchmark's multi-GPU path is replicas only (the hot path does not shard:
no data-path collective).  Its host logic -- the slowest replica's time sets
the whole job's, the value counts every replica's particles, only rank 0
reports, the reference arm runs on rank 0 alone -- is checked here with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r measured (r + 1) ms for the step loop and 10 (r + 1) ms end to end
        got = bench.max_over_ranks(rank + 1.0, 10.0 * (rank + 1))
        out[rank] = got
    finally:
        td.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == [2.0, 20.0]


def test_max_over_ranks_without_a_group_is_the_identity():
    assert bench.max_over_ranks(3.0, 4.5) == [3.0, 4.5]


def test_whole_job_rate_counts_every_replica_over_the_slowest_time():
    # 1e6 particles per replica, 2 replicas, 10 steps, slowest replica 20 ms
    assert bench.whole_job_rate(1_000_000, 2, 10, 20.0) == pytest.approx(1e9)
    assert bench.whole_job_rate(1_000_000, 1, 10, 20.0) == pytest.approx(5e8)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class A:
        workload, steps, warmup, threads = "weibel_512", 1, 3, 256
    assert bench.run_reference(A(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""


def test_recorded_traffic_is_used_only_at_the_captured_source(tmp_path, monkeypatch):
    """The DRAM traffic of the committed capture is reported only while the
    particle-advance sources hash as they did at capture time."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.push_source_hash()
    (prof / "traffic.txt").write_text(f"# comment\nweibel_512 123456 {h}\nthermal_2048 9 0000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "push_source_hash", lambda: h)
    assert bench.recorded_traffic("weibel_512") == 123456.0
    assert bench.recorded_traffic("thermal_2048") is None      # captured at another source
    assert bench.recorded_traffic("weibel_256") is None        # never captured


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, kind = bench.read_peaks()
    assert kind == "fallback" and peak == bench.PEAK_FALLBACK_GBS
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6779.0}')
    assert bench.read_peaks() == (6779.0, "measured")


@pytest.mark.parametrize("workload,metric", [
    ("weibel_512", "particle updates/s (push+deposit+sort)"),
    ("denoiser_fwd_2048", "denoiser forward throughput"),
])
def test_reference_arm_prints_one_contract_line(workload, metric):
    """`bench.py --impl reference` (the CPU oracle on a bounded sample) prints
    one JSON line with the keys of the contract, on the GPU arm's metric."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, bench.__file__, "--impl", "reference", "--workload", workload,
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == metric and d["value"] > 0
    assert d["higher_is_better"] is True and d["warmup"] == 3 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"] == workload
