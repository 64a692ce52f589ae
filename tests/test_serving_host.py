"""Host-side serving logic (no GPU): the seeded request mix and the latency
statistics the bench reports."""
import numpy as np

from paper_2602_20516_b300 import serve


def test_workload_mix_is_seeded_and_in_range():
    a = serve.workload([0, 1, 2, 3], 2000, seed=5)
    b = serve.workload([0, 1, 2, 3], 2000, seed=5)
    assert a == b
    assert a != serve.workload([0, 1, 2, 3], 2000, seed=6)
    kinds = np.array([r["kind"] for r in a])
    mixed = np.array([r["precision"] == "mixed" for r in a])
    kappa = np.array([r["kappa"] for r in a])
    assert abs((kinds == serve.SOLVE).mean() - 0.7) < 0.04
    assert abs(mixed.mean() - 0.5) < 0.04
    assert kappa.min() >= 0.14 and kappa.max() <= 0.157
    assert {r["gauge_id"] for r in a} == {0, 1, 2, 3}
    assert len({r["source_seed"] for r in a}) == len(a)


def test_latency_stats_counts_failures_apart():
    done = [{"latency": 0.010 * (k + 1), "status": 0} for k in range(99)]
    done += [{"latency": 5.0, "status": 3}, {"latency": 7.0, "status": 4}]
    st = serve.latency_stats(done)
    assert st["n"] == 99 and st["failed"] == 2
    assert st["failed_by_status"] == {"3": 1, "4": 1}
    lat = 1e3 * 0.010 * np.arange(1, 100)
    assert abs(st["p50_ms"] - np.percentile(lat, 50)) < 1e-9
    assert abs(st["p99_ms"] - np.percentile(lat, 99)) < 1e-9
    assert serve.latency_stats([{"latency": 1.0, "status": 4}])["n"] == 0
