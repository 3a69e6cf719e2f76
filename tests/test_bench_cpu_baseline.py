"""Host logic of the all-cores CPU baseline in bench.py: one spawned process
per core, each running the oracle on its own sample of sources, summed over
the wall time."""
import os

import bench
import oracle


def test_all_cores_baseline_runs_one_process_per_sample():
    oracle.build()
    stride = 300_000  # about one source per process: seconds, not minutes
    n = min(4, os.cpu_count() or 1)
    r = bench.cpu_all_cores(stride, "crossings/s", processes=n)
    assert r["cores"] == n and r["kind"] == "oracle"
    assert r["crossings"] > 0 and r["wall_s"] > 0
    assert abs(r["value"] - r["crossings"] / r["wall_s"]) <= 1e-9 * r["value"]
    # the offsets of the processes are distinct: disjoint samples
    offsets = [(i * stride) // n for i in range(n)]
    assert len(set(offsets)) == n


def test_worker_sample_matches_a_direct_oracle_run():
    oracle.build()
    stride, offset = 300_000, 7
    grid, params = bench.make_workload()
    c_direct, _ = bench.cpu_sample(grid, params, stride, offset)
    c_worker, _ = bench._cpu_worker((stride, offset))
    assert c_worker == c_direct > 0
