"""Host logic of the serving loop (admission, continuous batching, retiring,
latency accounting) with the GPU objects replaced by fakes: no device
needed.  The fakes count steps exactly like the batch does (each member
advances by min(n, its remaining budget))."""
import pytest

import workloads as W
from paper_2512_01027_gb300 import serving


class FakeLattice:
    def __init__(self, lattice, shape, **kw):
        self.N = shape[0] * shape[1] * shape[2]
        self.steps_done = 0
        self.closed = False

    def init_fields(self, phi, P, u):
        pass

    def read_fields(self):
        return (self.steps_done,)

    def step(self, n):                 # stepped alone (srpt with solo_sites)
        self.steps_done += n
        FakeBatch.log.append(("solo", self.N))
        FakeBatch.events.append(id(self))

    def check(self):
        pass

    def close(self):
        self.closed = True


class FakeBatch:
    log = []
    events = []                        # what each chunk stepped: a solo lattice's id, or "batch"

    def __init__(self, lattice, storage):
        self.rem = {}
        self.paused = set()

    def set_tuning(self, chunk=16, use_graph=True):
        pass

    def add(self, L, steps):
        self.rem[id(L)] = [L, steps]
        FakeBatch.log.append(("add", len(self.rem)))
        FakeBatch.log.append(("add_sites", L.N))

    def remove(self, L):
        del self.rem[id(L)]
        self.paused.discard(id(L))

    def pause(self, L, paused=True):
        assert id(L) in self.rem
        (self.paused.add if paused else self.paused.discard)(id(L))
        FakeBatch.log.append(("pause", int(paused)))

    def step(self, n):
        running = [v for k, v in self.rem.items() if k not in self.paused]
        FakeBatch.log.append(("step", len(running)))
        FakeBatch.events.append("batch")
        for v in running:
            t = min(n, v[1])
            v[0].steps_done += t
            v[1] -= t
        return sum(1 for v in self.rem.values() if v[1] == 0)

    def remaining(self, L):
        return self.rem[id(L)][1]

    def info(self):
        return len(self.rem), 0

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(serving, "Lattice", FakeLattice)
    monkeypatch.setattr(serving, "Batch", FakeBatch)
    monkeypatch.setattr(serving, "_prepare", lambda r: W.Case("c", "D3Q27", (r.edge,) * 3, W.base_params(), 0, 0, 0,
                                                             (1, 1, 1), None, r.steps))
    FakeBatch.log = []
    FakeBatch.events = []


def trace(n=12):
    return W.request_trace(n=n, rate=1e9, edges=(16, 20, 24), steps_range=(7, 40))


def test_every_request_gets_exactly_its_steps(fake):
    reqs = trace()
    S = serving.Server("D3Q27", "f16", chunk=5, keep_fields=True, hbm_budget=1 << 40)
    st = S.run(reqs)
    assert [r.rid for r in st.results] == sorted(r.rid for r in reqs)
    for r, res in zip(sorted(reqs, key=lambda q: q.rid), st.results):
        assert res.fields == (r.steps,)
        assert res.arrival <= res.admitted <= res.finished


def test_admission_limits(fake):
    reqs = trace(20)
    one = serving.estimate_footprint("D3Q27", (24, 24, 24), storage="f16", inplace=1)
    S = serving.Server("D3Q27", "f16", chunk=5, hbm_budget=3 * one, max_members=2)
    st = S.run(reqs)
    assert len(st.results) == 20
    assert st.peak_members <= 2 and st.peak_bytes <= 3 * one
    S = serving.Server("D3Q27", "f16", chunk=5, hbm_budget=1 << 40, max_active_sites=2 * 24 ** 3)
    st = S.run(reqs)
    assert len(st.results) == 20
    assert max(n for e, n in FakeBatch.log if e == "add") <= 8   # never more than the site cap allows of 16^3 lattices


def test_site_cap_still_admits_one_large_request(fake):
    reqs = W.request_trace(n=3, rate=1e9, edges=(32,), steps_range=(5, 9))
    S = serving.Server("D3Q27", "f16", chunk=4, hbm_budget=1 << 40, max_active_sites=1000)
    st = S.run(reqs)
    assert len(st.results) == 3 and st.peak_members == 1


def test_sjf_admits_least_work_first(fake):
    """policy="sjf": with one member slot and every request waiting at t = 0,
    the requests run in order of their work (sites x steps); every one still
    gets exactly its steps.  A request past max_wait goes first in arrival
    order (max_wait = -1: every request is overdue, so arrival order)."""
    reqs = W.request_trace(n=10, rate=1e9, edges=(8, 12, 16), steps_range=(3, 30))
    work = {r.rid: r.edge ** 3 * r.steps for r in reqs}
    S = serving.Server("D3Q27", "f16", chunk=4, keep_fields=True, hbm_budget=1 << 40, max_members=1,
                       policy="sjf", max_wait=1e9)
    st = S.run(reqs)
    order = [r.rid for r in sorted(st.results, key=lambda q: q.admitted)]
    assert [work[i] for i in order] == sorted(work.values())
    for r in st.results:
        assert r.fields == (next(q.steps for q in reqs if q.rid == r.rid),)
    S = serving.Server("D3Q27", "f16", chunk=4, hbm_budget=1 << 40, max_members=1, policy="sjf", max_wait=-1.0)
    st = S.run(reqs)
    order = [r.rid for r in sorted(st.results, key=lambda q: q.admitted)]
    assert order == [r.rid for r in sorted(reqs, key=lambda q: q.arrival)]


def _srpt_run(fake_batch_log, reqs, **kw):
    ticks = iter(range(10 ** 9))
    S = serving.Server("D3Q27", "f16", chunk=4, keep_fields=True, hbm_budget=1 << 40, policy="srpt", **kw)
    return S.run(reqs, clock=lambda: next(ticks) * 1e-6)


def test_srpt_order_and_pausing(fake):
    """policy="srpt": every request admitted at t = 0, fill_sites below one
    lattice, so one lattice steps per chunk: they finish in order of their
    work (sites x steps), each with exactly its steps, while the others wait
    paused.  A fill of all the sites steps everyone in every chunk; with
    every request overdue (max_wait = -1) they run in arrival order."""
    reqs = W.request_trace(n=9, rate=1e9, edges=(8, 12, 16), steps_range=(3, 30))
    work = {r.rid: r.edge ** 3 * r.steps for r in reqs}
    st = _srpt_run(FakeBatch.log, reqs, fill_sites=1, max_wait=1e9)
    order = [r.rid for r in sorted(st.results, key=lambda q: q.finished)]
    assert [work[i] for i in order] == sorted(work.values())
    for r in st.results:
        assert r.fields == (next(q.steps for q in reqs if q.rid == r.rid),)
    assert {n for e, n in FakeBatch.log if e == "step"} == {1}
    FakeBatch.log = []
    st = _srpt_run(FakeBatch.log, reqs, fill_sites=1 << 40, max_wait=1e9)
    assert not any(e == "pause" and n == 1 for e, n in FakeBatch.log)   # nobody waits
    for r in st.results:
        assert r.fields == (next(q.steps for q in reqs if q.rid == r.rid),)
    st = _srpt_run(FakeBatch.log, reqs, fill_sites=1, max_wait=-1.0)
    order = [r.rid for r in sorted(st.results, key=lambda q: q.finished)]
    assert order == [r.rid for r in sorted(reqs, key=lambda q: q.arrival)]


def test_srpt_steps_large_requests_alone(fake):
    """solo_sites: a request of at least that many sites never joins the
    batch; it is stepped alone in chunk-sized slices in the same
    least-work-left order, and still gets exactly its steps."""
    reqs = W.request_trace(n=9, rate=1e9, edges=(8, 12, 16), steps_range=(3, 30))
    work = {r.rid: r.edge ** 3 * r.steps for r in reqs}
    st = _srpt_run(FakeBatch.log, reqs, fill_sites=1, max_wait=1e9, solo_sites=16 ** 3)
    for r in st.results:
        assert r.fields == (next(q.steps for q in reqs if q.rid == r.rid),)
    assert all(n < 16 ** 3 for e, n in FakeBatch.log if e == "add_sites")
    assert any(e == "solo" and n == 16 ** 3 for e, n in FakeBatch.log)
    order = [r.rid for r in sorted(st.results, key=lambda q: q.finished)]
    assert [work[i] for i in order] == sorted(work.values())
    with pytest.raises(ValueError):
        serving.Server("D3Q27", "f16", hbm_budget=1 << 40, policy="sjf", solo_sites=1)


def test_srpt_solo_to_end_runs_a_started_solo_request_through(fake):
    """solo_to_end: once a solo request has taken its first slice, nothing
    else steps until its last one; every request still gets exactly its
    steps."""
    reqs = W.request_trace(n=9, rate=1e9, edges=(8, 12, 16), steps_range=(3, 30))
    st = _srpt_run(FakeBatch.log, reqs, fill_sites=1, max_wait=1e9, solo_sites=16 ** 3, solo_to_end=True)
    for r in st.results:
        assert r.fields == (next(q.steps for q in reqs if q.rid == r.rid),)
    ev = FakeBatch.events
    solos = {e for e in ev if e != "batch"}
    assert solos
    for s in solos:
        idx = [i for i, e in enumerate(ev) if e == s]
        assert idx == list(range(idx[0], idx[-1] + 1)), "a solo request was interrupted"
