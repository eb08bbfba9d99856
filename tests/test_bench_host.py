"""Host-side pieces of bench.py: the algorithmic bytes per site update that
every roofline figure divides by.  Per site update a step reads and writes
both population sets (2 x 2Q stored values) and the P, u state (2 x (1 + d)
values of the arithmetic type)."""
import pytest

import bench


@pytest.mark.parametrize("Q,D,store,field,expected", [
    (27, 3, 4, 4, 464),   # D3Q27, FP32
    (27, 3, 2, 4, 248),   # D3Q27, 16-bit storage, FP32 state
    (9, 2, 8, 8, 336),    # D2Q9, FP64
    (9, 2, 4, 4, 168),    # D2Q9, FP32
    (19, 3, 4, 4, 336),   # D3Q19, FP32
])
def test_algorithmic_bytes_per_site(Q, D, store, field, expected):
    assert bench.alg_bytes_per_site(Q, D, store, field) == expected


def test_replica_throughput_counts_every_rank():
    # 2 replicas of 1e6 sites, 100 steps in 50 ms on the slowest rank
    assert bench.replica_mlups(10 ** 6, 100, 50.0, 2) == pytest.approx(4000.0)


def test_recorded_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    """The DRAM traffic of a workload is reported only while the kernel
    sources hash to the value recorded with it, scaled by sites; otherwise
    (or with no record) it is None."""
    import json

    rec = tmp_path / "traffic.json"
    rec.write_text(json.dumps({"w": {"source_hash": "abc", "dram_bytes_per_site": 629.2}}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.recorded_traffic("w", 1000) == 629200
    assert bench.recorded_traffic("other", 1000) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.recorded_traffic("w", 1000) is None


def test_committed_traffic_record_matches_the_sources():
    """profiles/step_kernel_traffic.json was captured on the kernel sources as
    they are: the bench's traffic fields are live, not stale."""
    import json

    rec = json.load(open(bench.TRAFFIC_FILE))
    for key in ("n256-f32-split", "n256-f16-split", "bubble1-f32-batch"):
        assert rec[key]["source_hash"] == bench.kernel_source_hash(), key
