"""Serving loop: many independent multiphase LB solves on one GPU.

A request names one simulation (grid edge, droplet radius, density ratio,
surface tension, number of steps).  The server

* takes requests as they arrive (arrival times in seconds from the start),
* builds each request's initial fields on host threads while the GPU works,
* admits waiting requests while their device footprint
  (``estimate_footprint``) fits in the HBM budget, a member slot is free and
  the sites of the admitted lattices stay within ``max_active_sites`` (one
  large lattice already fills the GPU: sharing it among many large lattices
  only stretches every one of them; small lattices still run many at once),
  first come first served (``policy="fifo"``) or the least work first
  (``policy="sjf"`` and ``"srpt"``: sites x steps, which shortens the wait of
  the many small requests behind a few large ones; a request that has
  waited longer than ``max_wait`` seconds goes first whatever its size),
* advances the admitted lattices together through one ``Batch`` (two kernel
  launches per time step for the whole set, chunks replayed as CUDA graphs),
  each lattice by exactly its own number of steps.  With ``fifo`` and
  ``sjf`` every admitted lattice steps in every chunk, so they share the GPU
  evenly.  With ``srpt`` (shortest remaining processing time) a chunk steps
  only the lattices with the least work left (sites x remaining steps),
  taken in that order until their sites reach ``fill_sites`` (enough to
  fill the GPU), and pauses the others (``Batch.pause``): small requests
  then finish at the speed they would have alone, instead of at the step
  rate of the largest lattice beside them.  A lattice whose request has
  waited longer than ``max_wait`` seconds comes first, so a large request
  is not held back without end.  With ``solo_sites`` set, a request of at
  least that many sites (one that fills the GPU by itself) is stepped by the
  single-lattice split kernels instead of the batch kernel, in slices of
  ``chunk`` steps taken in the same order (with ``solo_to_end``, once its
  first slice is taken it runs to its end, so smaller arrivals no longer
  stretch the largest requests); whether a request goes solo depends on its
  size only, so its result still does not depend on the mix,
* retires a lattice the moment its steps are done: reads its fields back to
  the host, frees its memory, and admits the next request in its place
  (continuous batching).

Latency is arrival -> result on the host.  The per-site arithmetic of a
batch does not depend on the other members, so a request's result is the
same whether it is served alone or in any mix.

A request whose solve produces a non-finite phi, P or u (the method itself
diverges for some small, high-density-ratio droplets of the trace; the FP64
oracle does too) is retired when its steps are done with ``failed`` set and
no fields; the summary counts such requests apart and takes the latency
percentiles over the completed ones.
"""
from __future__ import annotations

import collections
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import LBM_ERR_NONFINITE, Batch, Lattice, LbmError, estimate_footprint


@dataclass
class Served:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    sites: int
    fields: tuple | None = None
    failed: bool = False

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    makespan: float = 0.0
    peak_members: int = 0
    peak_bytes: int = 0
    launches: int = 0

    def summary(self) -> dict:
        done = [r for r in self.results if not r.failed]
        lat = np.array([r.latency for r in done]) if done else np.zeros(1)
        sites = sum(r.sites * r.steps for r in self.results)
        return {
            "requests": len(self.results),
            "failed": len(self.results) - len(done),
            "failed_ids": [r.rid for r in self.results if r.failed],
            "solves_per_s": len(self.results) / self.makespan if self.makespan > 0 else 0.0,
            "mlups": sites / self.makespan / 1e6 if self.makespan > 0 else 0.0,
            "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)),
            "makespan_s": self.makespan,
            "peak_members": self.peak_members,
            "peak_gb": self.peak_bytes / 1e9,
            "gpu_launches": self.launches,
        }


def _prepare(req):
    c = req.case()
    return c


class Server:
    """Continuous-batching server for requests of one lattice and storage."""

    def __init__(self, lattice: str = "D3Q27", storage: str = "f16", inplace: bool = True, chunk: int = 16,
                 max_members: int = 64, hbm_budget: int | None = None, prep_threads: int = 4,
                 keep_fields: bool = False, stream=None, max_active_sites: int | None = None,
                 policy: str = "fifo", max_wait: float = 5.0, fill_sites: int = 1 << 21,
                 solo_sites: int | None = None, solo_to_end: bool = False):
        if policy not in ("fifo", "sjf", "srpt"):
            raise ValueError("policy is 'fifo', 'sjf' or 'srpt'")
        self.policy, self.max_wait = policy, float(max_wait)
        self.fill_sites = int(fill_sites)
        if solo_sites is not None and policy != "srpt":
            raise ValueError("solo_sites needs policy 'srpt'")
        self.solo_sites = solo_sites
        self.solo_to_end = bool(solo_to_end)   # a solo request, once started, runs to its end
        self._solo_running = None
        self.lattice, self.storage, self.inplace = lattice, storage, bool(inplace)
        self.chunk, self.max_members = int(chunk), int(max_members)
        self.max_active_sites = max_active_sites
        self.keep_fields = keep_fields
        if hbm_budget is None:
            import torch

            free, _total = torch.cuda.mem_get_info()
            hbm_budget = int(0.85 * free)
        self.hbm_budget = int(hbm_budget)
        self.prep_threads = prep_threads
        self.batch = Batch(lattice, storage)
        self.batch.set_tuning(chunk=self.chunk, use_graph=True)
        if stream is not None:
            self.batch.set_stream(stream)

    def footprint(self, req) -> int:
        n = req.edge
        return estimate_footprint(self.lattice, (n, n, n), storage=self.storage, inplace=int(self.inplace))

    def close(self):
        self.batch.close()

    def run(self, requests, clock=time.perf_counter) -> ServeStats:
        pend = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()          # (request, future of its initial fields)
        active = []                            # (request, Lattice, bytes, admitted)
        stats = ServeStats()
        used = 0
        sites = 0
        paused = {}                            # srpt: id(Lattice) -> paused now
        self._solo_running = None
        solo = {}                              # srpt with solo_sites: id(Lattice) -> steps left
        solo_launches = 0                      # the split form's two launches per solo step
        launches0 = self.batch.info()[1]
        with ThreadPoolExecutor(max_workers=self.prep_threads) as pool:
            t0 = clock()
            while pend or waiting or active:
                now = clock() - t0
                while pend and pend[0].arrival <= now:
                    r = pend.popleft()
                    waiting.append((r, pool.submit(_prepare, r)))
                # admission by free HBM and slots, in the policy's order
                if self.policy in ("sjf", "srpt") and len(waiting) > 1:
                    # requests waiting longer than max_wait first, in arrival
                    # order; then the least work (sites x steps) first
                    def key(rf, now=now):
                        r = rf[0]
                        if now - r.arrival > self.max_wait:
                            return (0, r.arrival, 0)
                        return (1, r.edge ** 3 * r.steps, r.arrival)

                    waiting = collections.deque(sorted(waiting, key=key))
                while waiting and len(active) < self.max_members:
                    r, fut = waiting[0]
                    need = self.footprint(r)
                    if need > self.hbm_budget:
                        raise ValueError(f"request {r.rid} needs {need} bytes, more than the HBM budget")
                    if used + need > self.hbm_budget:
                        break
                    n_sites = r.edge ** 3
                    if active and self.max_active_sites is not None and sites + n_sites > self.max_active_sites:
                        break
                    if active and not fut.done():
                        break                  # keep the GPU busy; admit it next round
                    c = fut.result()
                    waiting.popleft()
                    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
                    L = Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage=self.storage,
                                g_ext=c.params.get("g_ext", (0, 0, 0)), inplace=int(self.inplace), **prm)
                    L.init_fields(c.phi0, c.P0, c.u0)
                    if self.solo_sites is not None and n_sites >= self.solo_sites:
                        solo[id(L)] = r.steps
                    else:
                        self.batch.add(L, r.steps)
                    used += need
                    sites += n_sites
                    active.append((r, L, need, clock() - t0))
                stats.peak_members = max(stats.peak_members, len(active))
                stats.peak_bytes = max(stats.peak_bytes, used)
                if not active:
                    if waiting:
                        waiting[0][1].result()
                    elif pend:
                        time.sleep(max(0.0, min(pend[0].arrival - (clock() - t0), 0.002)))
                    continue
                lone = self._schedule(active, now, paused, solo) if self.policy == "srpt" else None
                diverged = set()
                if lone is not None:
                    k = min(self.chunk, solo[id(lone)])
                    lone.step(k)
                    solo[id(lone)] -= k
                    solo_launches += 2 * k
                    try:
                        lone.check()                   # waits for the slice
                    except LbmError as e:
                        if e.code != LBM_ERR_NONFINITE:
                            raise
                        diverged.add(id(lone))
                        solo[id(lone)] = 0
                else:
                    self.batch.step(self.chunk)
                keep = []
                for r, L, need, t_adm in active:
                    if id(L) in solo:
                        done = solo[id(L)] == 0
                    else:
                        done = self.batch.remaining(L) == 0
                    if done:
                        if id(L) in diverged:
                            out, failed = None, True
                        else:
                            out, failed = _read_result(L)
                        t_fin = clock() - t0
                        if id(L) in solo:
                            del solo[id(L)]
                        else:
                            self.batch.remove(L)
                        paused.pop(id(L), None)
                        L.close()
                        used -= need
                        sites -= L.N
                        stats.results.append(Served(r.rid, r.arrival, t_adm, t_fin, r.steps, L.N,
                                                    out if self.keep_fields else None, failed))
                    else:
                        keep.append((r, L, need, t_adm))
                active = keep
            stats.makespan = clock() - t0
        stats.launches = self.batch.info()[1] - launches0 + solo_launches
        stats.results.sort(key=lambda s: s.rid)
        return stats


    def _schedule(self, active, now, paused, solo):
        """srpt: the lattices with the least work left step in the next chunk
        (overdue requests first), until their sites reach fill_sites; the
        others pause.  Returns the solo lattice to step instead of the batch
        when one comes first in that order, else None."""

        def left(L):
            return solo[id(L)] if id(L) in solo else self.batch.remaining(L)

        def key(entry):
            r, L = entry[0], entry[1]
            if now - r.arrival > self.max_wait:
                return (0, r.arrival)
            return (1, L.N * left(L))

        if self.solo_to_end and self._solo_running is not None:
            for entry in active:
                if entry[1] is self._solo_running and solo.get(id(entry[1]), 0) > 0:
                    return entry[1]
            self._solo_running = None
        order = sorted(active, key=key)
        if order and id(order[0][1]) in solo:
            self._solo_running = order[0][1]
            return order[0][1]
        run = set()
        filled = 0
        for entry in order:
            if filled >= self.fill_sites:
                break
            if id(entry[1]) in solo:
                continue
            run.add(id(entry[1]))
            filled += entry[1].N
        for entry in active:
            L = entry[1]
            if id(L) in solo:
                continue
            want = id(L) not in run
            if paused.get(id(L), False) != want:
                self.batch.pause(L, want)
                paused[id(L)] = want
        return None


def _read_result(L: Lattice):
    """Fields of a finished lattice, or (None, True) when its solve diverged."""
    try:
        return L.read_fields(), False
    except LbmError as e:
        if e.code != LBM_ERR_NONFINITE:
            raise
        return None, True


def run_one_at_a_time(requests, storage: str = "f32", clock=time.perf_counter) -> ServeStats:
    """The same trace served without batching: one lattice at a time, in
    arrival order, each stepped with its own launches (split form)."""
    stats = ServeStats()
    t0 = clock()
    launches = 0
    for r in sorted(requests, key=lambda q: q.arrival):
        while clock() - t0 < r.arrival:
            time.sleep(min(0.002, r.arrival - (clock() - t0)))
        c = r.case()
        t_adm = clock() - t0
        prm = {k: v for k, v in c.params.items() if k != "g_ext"}
        L = Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage=storage,
                    g_ext=c.params.get("g_ext", (0, 0, 0)), **prm)
        L.init_fields(c.phi0, c.P0, c.u0)
        L.step(r.steps)
        _, failed = _read_result(L)
        launches += 2 * r.steps
        t_fin = clock() - t0
        stats.results.append(Served(r.rid, r.arrival, t_adm, t_fin, r.steps, L.N, None, failed))
        L.close()
    stats.makespan = clock() - t0
    stats.peak_members = 1
    stats.launches = launches
    return stats
