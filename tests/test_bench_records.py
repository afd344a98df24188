"""The per-workload figures the benchmark reads from the committed ncu
summaries (profiles/issue.txt, profiles/traffic.txt) parse, and were taken at
the particle advance's current source: a change to the kernel without a new
capture fails here instead of dropping the traffic and issue figures from
the bench line without notice."""
import bench


def test_records_exist_for_the_bench_workloads_at_the_current_source():
    h = bench.push_source_hash()
    for name in ("issue.txt", "traffic.txt"):
        hashes = set()
        with open(f"{bench.ROOT}/profiles/{name}") as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                workload, value, src = line.split()[:3]
                assert float(value) > 0
                hashes.add(src)
        assert h in hashes, f"{name}: no record at the current kernel source {h}"
    assert bench.recorded_value("issue.txt", "thermal_2048") is not None
    assert bench.recorded_traffic("thermal_2048") is not None


def test_recorded_figures_are_plausible():
    # warp-instructions per 32 particles: a few hundred (the advance is a few
    # hundred instructions per particle warp); traffic per launch: at least
    # the 48 algorithmic bytes per particle moved through DRAM once, within 2x
    per32 = bench.recorded_value("issue.txt", "thermal_2048")
    assert 200 < per32 < 2000
    traffic = bench.recorded_traffic("thermal_2048")
    particles = 2048 * 2048 * 16
    assert 0.5 * 48 * particles < traffic < 2.0 * 48 * particles


def test_whole_job_rate_counts_every_replica():
    assert bench.whole_job_rate(1000, 4, 10, 2.0) == 1000 * 4 * 10 / 2e-3
