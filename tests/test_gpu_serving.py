"""Serving loop: continuous batching of independent solves.

A request's result must not depend on what it was served with (alone vs in
any mix, bit for bit), admission must respect the HBM budget and the member
slots, and every request must get exactly its own number of steps.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def small_trace(n=7, rate=200.0):
    return W.request_trace(n=n, rate=rate, edges=(16, 20, 24, 32), steps_range=(20, 70))


@pytest.mark.parametrize("storage", ["f16", "f32"])
def test_served_alone_equals_served_mixed(lbm, storage):
    from paper_2512_01027_gb300.serving import Server

    reqs = small_trace()
    S = Server("D3Q27", storage, chunk=8, keep_fields=True, hbm_budget=2 << 30)
    mixed = S.run(reqs)
    S.close()
    assert len(mixed.results) == len(reqs)
    assert mixed.peak_members >= 2           # the trace really overlapped
    for r, got in zip(sorted(reqs, key=lambda q: q.rid), mixed.results):
        A = Server("D3Q27", storage, chunk=5, keep_fields=True, hbm_budget=2 << 30)
        r0 = W.Request(r.rid, 0.0, r.edge, r.R, r.ratio, r.sigma, r.steps)
        alone = A.run([r0]).results[0]
        A.close()
        for x, y in zip(alone.fields, got.fields):
            assert np.array_equal(x, y)


def test_admission_respects_budget_and_slots(lbm):
    from paper_2512_01027_gb300.serving import Server

    reqs = small_trace(n=9, rate=1e6)         # all arrive at once
    probe = Server("D3Q27", "f16", chunk=8, hbm_budget=1 << 40)
    biggest = max(probe.footprint(r) for r in reqs)
    probe.close()
    S = Server("D3Q27", "f16", chunk=8, hbm_budget=2 * biggest + 1, max_members=3)
    st = S.run(reqs)
    S.close()
    assert len(st.results) == 9
    assert st.peak_bytes <= 2 * biggest + 1
    assert st.peak_members <= 3
    s = st.summary()
    assert s["p50_s"] <= s["p99_s"]
    for res in st.results:
        assert res.arrival <= res.admitted <= res.finished


def test_oversized_request_is_refused(lbm):
    from paper_2512_01027_gb300.serving import Server

    reqs = small_trace(n=1)
    S = Server("D3Q27", "f16", hbm_budget=1 << 20)
    with pytest.raises(ValueError):
        S.run(reqs)
    S.close()


def test_one_at_a_time_baseline_runs(lbm):
    from paper_2512_01027_gb300.serving import run_one_at_a_time

    reqs = small_trace(n=3, rate=1e6)
    st = run_one_at_a_time(reqs)
    assert len(st.results) == 3
    assert st.summary()["solves_per_s"] > 0


@pytest.mark.parametrize("to_end", [False, True])
def test_srpt_with_solo_requests_alone_equals_mixed(lbm, to_end):
    """policy="srpt" with solo_sites: requests of 24^3 sites and more are
    stepped alone by the split kernels, the others in the batch with
    pausing; each result equals, bit for bit, the same request served by
    itself with the same settings (the path depends on its size only)."""
    from paper_2512_01027_gb300.serving import Server

    reqs = small_trace(n=7, rate=1e6)
    kw = dict(chunk=8, keep_fields=True, hbm_budget=2 << 30, policy="srpt", fill_sites=20 ** 3,
              solo_sites=24 ** 3, solo_to_end=to_end)
    S = Server("D3Q27", "f16", **kw)
    mixed = S.run(reqs)
    S.close()
    assert len(mixed.results) == len(reqs)
    assert any(r.edge ** 3 >= 24 ** 3 for r in reqs) and any(r.edge ** 3 < 24 ** 3 for r in reqs)
    for r, got in zip(sorted(reqs, key=lambda q: q.rid), mixed.results):
        A = Server("D3Q27", "f16", **kw)
        alone = A.run([W.Request(r.rid, 0.0, r.edge, r.R, r.ratio, r.sigma, r.steps)]).results[0]
        A.close()
        for x, y in zip(alone.fields, got.fields):
            assert np.array_equal(x, y)
