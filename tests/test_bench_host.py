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
