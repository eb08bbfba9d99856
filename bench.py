#!/usr/bin/env python
"""Benchmark of the coupled-LB step on GB300.

Workload (one step = one time step of the whole lattice through every row of
the hot path): 3D D3Q27 droplet impact on a liquid film, 256^3 sites, FP32,
periodic in x and y, solid planes z = 0 and z = 255, droplet R = 32 falling at
0.05 onto a film of depth 32, density ratio 1000, sigma = 1e-3, seeded 1e-4
perturbation of phi at the interface.  Inputs are synthetic (workloads/).

Metric: MLUPS (million lattice-site updates per second) of the coupled step,
the roofline fraction of the step (its algorithmic bytes over its measured
time, against the measured HBM copy bandwidth), an end-to-end MLUPS through the C ABI with host buffers, and the
FP64 oracle on the host cores as a CPU baseline.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, one independent replica per GPU (the lattices do not
exchange data: replicas only), timing = max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "coupled-lattice MLUPS & % HBM roofline; served solves/s with p50/p99 latency"
UNIT = "MLUPS"
CSRC = os.path.join(ROOT, "paper_2512_01027_gb300", "csrc")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256, help="grid edge of the workload")
    ap.add_argument("--storage", default="f32")
    ap.add_argument("--variant", type=int, default=0,
                    help="0 automatic (split form), 1 fused plane-synchronous, 2 fused pipelined, 3 split form, "
                         "4 persistent split form, 5 cluster step")
    ap.add_argument("--cluster-rows", type=int, default=0, help="CTAs per cluster of the cluster step (0 auto)")
    ap.add_argument("--staged", type=int, default=-1,
                    help="cluster step: stage the pulled rows by bulk copies (-1 auto, 0 no, 1 yes)")
    ap.add_argument("--zchunk", type=int, default=0, help="planes per CTA of the fused / cluster kernels (0 auto)")
    ap.add_argument("--inplace", action="store_true", help="one population store, AA streaming")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-requests", type=int, default=100,
                    help="requests of the serving sample: the first ones of the seeded 2000-request trace, "
                         "with its full 500..5000-step range")
    ap.add_argument("--serve-policy", default="srpt", choices=["fifo", "sjf", "srpt"],
                    help="batched server: admission in arrival order, or least work first; srpt also steps "
                         "only the lattices with the least work left in each chunk")
    ap.add_argument("--serve-max-wait", type=float, default=5.0,
                    help="sjf / srpt: seconds after which a waiting request goes first whatever its size")
    ap.add_argument("--serve-solo", type=int, default=96 ** 3,
                    help="srpt: requests of at least this many sites are stepped alone by the split kernels (0: none)")
    ap.add_argument("--serve-solo-preempt", action="store_true",
                    help="srpt: a solo request may be preempted by one with less work left (default: once "
                         "started, it runs to its end)")
    ap.add_argument("--serve-fill", type=int, default=1 << 21,
                    help="srpt: sites stepped per chunk (lattices with the least work left first)")
    ap.add_argument("--no-storage-forms", action="store_true",
                    help="skip the FP16 / BF16 storage lines of the same workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="impact", choices=["impact", "bubble1", "bubble2"],
                    help="impact: the 3D droplet impact (default); bubble1/2: the 2D rising bubble of "
                         "Sec. III.D, case 1 or 2, as a batch of --copies lattices")
    ap.add_argument("--copies", type=int, default=32, help="lattices in the batch of the bubble workload")
    ap.add_argument("--no-batch-autotune", action="store_true",
                    help="bubble workload: keep the default batch launch shape instead of lbm_batch_autotune")
    return ap.parse_args()


def kernel_source_hash() -> str:
    """Hash of what the step kernels are compiled from: the device headers,
    the instantiation units and the build flags (host-only API code is left
    out, it does not change the kernels' traffic)."""
    h = hashlib.sha256()
    files = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
             if f.endswith((".cuh", ".h")) or f.startswith("lbm_inst_")]
    files.append(os.path.join(CSRC, "..", "build.py"))
    for path in files:
        with open(path, "rb") as fh:
            h.update(os.path.basename(path).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(key: str, sites: int):
    """DRAM bytes of one step of the workload `key` from the ncu record in
    profiles/, scaled to `sites` by the sites of the capture; None unless the
    record was taken on the kernel sources as they are now."""
    try:
        with open(TRAFFIC_FILE) as f:
            ent = json.load(f).get(key, {})
        if ent.get("source_hash") != kernel_source_hash():
            return None
        return int(round(ent["dram_bytes_per_site"] * sites))
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = max(smax, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(n: int):
    R = n / 8.0
    return W.droplet_film_3d(n=n, R=R, film=R, uz=-0.05, noise=1e-4)


def alg_bytes_per_site(Q: int, D: int, store_bytes: int, field_bytes: int) -> int:
    """Read + write of both population sets and of the P, u state per site update."""
    return 2 * (2 * Q * store_bytes) + 2 * (1 + D) * field_bytes


def cpu_baseline(reps_target_s: float = 10.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the workload: the same droplet-on-film case at 64^3 (R = 8), 320 steps
    (about 10 s on 16 cores)."""
    import oracle

    c = W.droplet_film_3d(n=64, R=8.0, film=8.0, gap=8.0, uz=-0.05, noise=1e-4)
    o = oracle.Oracle("D3Q27", c.shape, oracle.make_params(**c.params), periodic=c.periodic, solid=c.solid)
    o.init(c.phi0, c.P0, c.u0)
    o.step(1)
    steps = 320
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return {"value": c.N * steps / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 C oracle, D3Q27 droplet on film 64^3 (R = 8), {steps} steps, {dt:.1f} s"}


def serving(n_requests: int, policy: str = "srpt", fill_sites: int = 1 << 21, max_wait: float = 5.0,
            solo_sites: int = 96 ** 3, solo_to_end: bool = True):
    """Served solves/s and p50/p99 latency on the serving workload: the first
    n_requests of the seeded 2000-request trace (oscillating ellipsoidal
    droplets in periodic boxes of edge {32, 48, 64, 96, 128}, density ratio
    10..1000, sigma 5e-4..2e-3, 500..5000 steps each), FP32 arithmetic with
    FP16 storage, in-place stores.
    1) closed loop: all requests at t = 0 -> capacity (solves/s);
    2) open loop: Poisson arrivals at 0.8 x capacity -> p50/p99 latency;
    3) the same open-loop trace one request at a time (FP32, split form).
    policy: the batched server's order (sjf: admission by least work first,
    with a request waiting over 5 s going first; srpt: in addition, each
    chunk steps only the lattices with the least work left, up to fill_sites
    sites, and pauses the others; requests of at least solo_sites sites are
    stepped alone by the split kernels in that same order and, with
    solo_to_end, run to their end once started)."""
    from paper_2512_01027_gb300.serving import Server, run_one_at_a_time

    full = 2000
    closed = W.request_trace(n=full, rate=1e9)[:n_requests]
    srv = Server("D3Q27", "f16", inplace=True, chunk=16, policy=policy, fill_sites=fill_sites, max_wait=max_wait,
                 solo_sites=(solo_sites or None) if policy == "srpt" else None, solo_to_end=solo_to_end)
    cl = srv.run(closed).summary()
    cap = cl["solves_per_s"]
    rate = 0.8 * cap
    opened = W.request_trace(n=full, rate=rate)[:n_requests]
    op = srv.run(opened).summary()
    srv.close()
    seq = run_one_at_a_time(opened, storage="f32").summary()
    work = sum(r.edge ** 3 * r.steps for r in closed)
    return {"workload": f"first {n_requests} of the 2000-request trace ({100.0 * n_requests / full:.0f} %), "
                        f"D3Q27 droplets, edges 32..128, 500..5000 steps, f16 storage, "
                        f"{work / 1e9:.0f} G site updates",
            "policy": policy, "fill_sites": fill_sites if policy == "srpt" else None,
            "max_wait_s": max_wait if policy != "fifo" else None,
            "solo_sites": solo_sites or None, "solo_to_end": solo_to_end,
            "fraction_of_trace": n_requests / full,
            "closed_loop": cl, "open_loop": dict(op, arrival_rate_per_s=rate), "one_at_a_time_f32": seq}


def storage_form(args, c, storage: str, f32_ms: float):
    """The same workload with populations stored in 16 bits (FP32 arithmetic),
    timed like the main line: MLUPS and the HBM roofline at its own
    algorithmic bytes per site."""
    import torch

    import paper_2512_01027_gb300 as lbm

    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage=storage,
                    g_ext=c.params["g_ext"], inplace=int(args.inplace), **prm)
    form = "split form"
    if args.variant:
        try:
            if args.cluster_rows or args.staged != -1:
                L.set_cluster(args.cluster_rows, args.staged)
            L.set_tuning(args.variant, args.zchunk)
            form = f"variant {args.variant}"
        except lbm.LbmError:
            pass                      # this storage has no such launch form: the split form
    stream = torch.cuda.current_stream()
    L.set_stream(stream)
    L.init_fields(c.phi0, c.P0, c.u0)
    L.step(args.warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    L.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    L.check()
    L.close()
    per_site = alg_bytes_per_site(27, 3, 2, 4)
    t_step = ms / args.steps / 1e3
    achieved = per_site * c.N / t_step / 1e9
    peak, peak_kind = measured_peaks()
    return {"value": round(c.N / t_step / 1e6, 2), "unit": UNIT, "ms_per_step": ms / args.steps,
            "speedup_vs_f32": round(f32_ms / (ms / args.steps), 4),
            "dtype": f"{storage}-storage/f32", "form": form,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "bytes_per_site": per_site, "peak_kind": peak_kind,
                         "traffic": recorded_traffic(f"n{args.n}-{storage}-split", c.N)
                         if form == "split form" and not args.inplace else None},
            "gpu_launches": (2 if form == "split form" else 1) * args.steps}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def reduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(sites: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job MLUPS of `world` independent replicas, each updating `sites`
    sites `steps` times, timed by the slowest rank (ms_max)."""
    return sites * steps * world / (ms_max / 1e3) / 1e6


def run_ours(args):
    import torch

    import paper_2512_01027_gb300 as lbm

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    c = workload(args.n)
    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage=args.storage,
                    g_ext=c.params["g_ext"], inplace=int(args.inplace), **prm)
    if args.cluster_rows or args.staged != -1:
        L.set_cluster(args.cluster_rows, args.staged)
    if args.variant:
        L.set_tuning(args.variant, args.zchunk)
    split = args.inplace or args.variant in (0, 3)
    form = "split" if split else f"v{args.variant}"
    kernel_name = {
        "split": "moments_kernel + collide_kernel (split form, one step = both launches)",
        "v1": "step_kernel (fused S0..S5, one launch per step)",
        "v2": "step_kernel_v2 (fused S0..S5, pipelined, one launch per step)",
        "v4": "split_persistent_kernel (both split phases in one launch per step)",
        "v5": "cluster_step_kernel (one launch per step; clusters share each plane's moments in "
              "distributed shared memory)",
    }[form]
    launches_per_step = 2 if split else 1
    stream = torch.cuda.current_stream()
    L.set_stream(stream)
    L.init_fields(c.phi0, c.P0, c.u0)
    L.step(args.warmup)
    torch.cuda.synchronize()

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    L.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    L.check()
    ms_max = reduce_max(ms, world)
    N = c.N
    value = replica_mlups(N, args.steps, ms_max, world)

    store_b = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[args.storage]
    field_b = 8 if args.storage == "f64" else 4
    per_site = alg_bytes_per_site(L.Q, L.d, store_b, field_b)
    per_launch = per_site * N
    t_launch = ms / args.steps / 1e3
    achieved = per_launch / t_launch / 1e9
    peak, peak_kind = measured_peaks()
    traffic = None
    roofline_alu = None
    try:
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        key = f"n{args.n}-{args.storage}-{form}{'-inplace' if args.inplace else ''}"
        ent = tr.get(key, {})
        if ent.get("source_hash") == kernel_source_hash():
            traffic = ent["dram_bytes_per_step"]
    except Exception:
        traffic, ent = None, {}
    try:
        if ent.get("flops_source_hash") == kernel_source_hash():
            # FP32 operations per site update (fadd + fmul + 2 ffma, both launches, ncu);
            # peak from the unit counts: SMs x 128 FP32 lanes x 2 flop x maximum SM clock
            fps = ent["fp32_flops_per_site"]
            sms = torch.cuda.get_device_properties(local).multi_processor_count
            peak_alu = sms * 128 * 2 * 2.07e9 / 1e12
            ach_alu = fps * N / t_launch / 1e12
            roofline_alu = {"bound": "alu", "achieved": round(ach_alu, 2), "peak": round(peak_alu, 1),
                            "unit": "TFLOP/s", "frac": round(ach_alu / peak_alu, 4),
                            "flops_per_site": fps,
                            "peak_kind": f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
    except Exception:
        roofline_alu = None
    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI: host fields (pinned) -> device -> K steps -> host fields
        ke = max(20, args.steps // 4)
        phi_h = torch.from_numpy(np.ascontiguousarray(c.phi0.reshape(-1))).pin_memory()
        P_h = torch.from_numpy(np.ascontiguousarray(c.P0.reshape(-1))).pin_memory()
        u_h = torch.from_numpy(np.ascontiguousarray(c.u0.reshape(3, -1))).pin_memory()
        out_phi = torch.empty(N, dtype=torch.float64).pin_memory()
        out_P = torch.empty(N, dtype=torch.float64).pin_memory()
        out_u = torch.empty(3 * N, dtype=torch.float64).pin_memory()
        import ctypes

        dptr = ctypes.POINTER(ctypes.c_double)
        cast = lambda t: ctypes.cast(t.data_ptr(), dptr)  # noqa: E731
        lib = lbm.lib()
        solves = 3
        # one untimed warm-up solve on the same host buffers: the first DMA
        # through freshly pinned host pages costs several times a later one
        # (28 vs 6 ms for the 671 MB of fields in, 16 vs 4.5 ms out, at 256^3)
        rc = lib.lbm_init_fields(L.handle, cast(phi_h), cast(P_h), cast(u_h))
        rc |= lib.lbm_step(L.handle, ke)
        rc |= lib.lbm_read_fields(L.handle, cast(out_phi), cast(out_P), cast(out_u))
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(solves):
            rc |= lib.lbm_init_fields(L.handle, cast(phi_h), cast(P_h), cast(u_h))
            rc |= lib.lbm_step(L.handle, ke)
            rc |= lib.lbm_read_fields(L.handle, cast(out_phi), cast(out_P), cast(out_u))
        t_e2e = time.perf_counter() - t0
        barrier(world)
        if rc != 0:
            raise RuntimeError(lib.lbm_last_error(L.handle))
        t_e2e = reduce_max(t_e2e, world)
        e2e = {"value": N * ke * solves * world / t_e2e / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(5 * 8 * N / ke), "d2h_bytes_per_step": int(5 * 8 * N / ke),
               "solve": f"{solves} solves back to back (after one untimed warm-up solve), each "
                        f"init_fields from pinned host fields, {ke} steps, read_fields to pinned host"}

    state_gb = L.footprint()[0] / 1e9
    forms = None
    if not args.no_storage_forms and args.storage == "f32" and world == 1:
        L.close()
        forms = {st: storage_form(args, c, st, ms / args.steps) for st in ("f16", "bf16")}
    serve = None
    if not args.no_serve:
        L.close()
        del L
        torch.cuda.empty_cache()
        serve = serving(args.serve_requests, args.serve_policy, args.serve_fill, args.serve_max_wait,
                        args.serve_solo, not args.serve_solo_preempt)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f64": "f64", "f32": "f32", "f16": "f16-storage/f32", "bf16": "bf16-storage/f32"}[args.storage],
            "data": "synthetic",
            "config": {"workload": f"D3Q27 droplet impact on a liquid film, {args.n}^3, {args.storage} storage",
                       "lattice": "D3Q27", "grid": [args.n] * 3, "storage": args.storage,
                       "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 ({state_gb:.1f} GB state per lattice)"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "peak_kind": peak_kind,
                         "kernel": kernel_name,
                         "store": "in-place AA" if args.inplace else "ping-pong",
                         "bytes_per_site": per_site},
            "roofline_alu": roofline_alu,
            "e2e": e2e,
            "gpu_launches": args.steps * launches_per_step,
            "clocks": clk,
            "cpu_baseline": cpu,
            "storage_forms": forms,
            "serving": serve,
        }
        print(json.dumps(line), flush=True)


def run_reference(args):
    """The FP64 oracle timed on the host cores as the reference arm: each step
    is one oracle step on a bounded sample of the workload (the same case at
    48^3, R = 6)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    c = W.droplet_film_3d(n=48, R=6.0, film=6.0, gap=8.0, uz=-0.05, noise=1e-4)
    o = oracle.Oracle("D3Q27", c.shape, oracle.make_params(**c.params), periodic=c.periodic, solid=c.solid)
    o.init(c.phi0, c.P0, c.u0)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = c.N * args.steps / dt / 1e6
    sample = f"FP64 C oracle, D3Q27 droplet on film 48^3 (R = 6), {args.steps} steps"
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"D3Q27 droplet impact on a liquid film, {args.n}^3, {args.storage} storage",
                       "lattice": "D3Q27", "grid": [args.n] * 3, "storage": args.storage},
            "impl": "reference",
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_bubble(args):
    """The 2D rising bubble (Sec. III.D) as a batch of identical lattices
    (one 200 x 400 lattice, 17 MB, fits in L2; `copies` of them do not),
    stepped by the batch engine, timed with CUDA events on its stream."""
    import torch

    import paper_2512_01027_gb300 as lbm

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    case = int(args.workload[-1])
    c = W.rising_bubble_2d(case)
    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    stream = torch.cuda.current_stream()
    B = lbm.Batch(c.lattice, args.storage)
    B.set_stream(stream)
    B.set_tuning(chunk=16, use_graph=True)
    lats = []
    for _ in range(args.copies):
        L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage=args.storage,
                        g_ext=c.params["g_ext"], inplace=int(args.inplace), **prm)
        L.set_stream(stream)
        L.init_fields(c.phi0, c.P0, c.u0)
        B.add(L, args.warmup + args.steps)
        lats.append(L)
    B.step(args.warmup)
    shape = None
    if not args.no_batch_autotune:
        # untimed: the trials restore every member's state and budget
        K, span, bps, ms_tuned = B.autotune(32)
        shape = {"chunk": K, "span": span, "blocks_per_sm": bps, "trial_ms_per_step": ms_tuned}
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    B.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    for L in lats:
        L.check()
    ms_max = reduce_max(ms, world)
    sites = c.N * args.copies
    value = replica_mlups(sites, args.steps, ms_max, world)
    store_b = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[args.storage]
    field_b = 8 if args.storage == "f64" else 4
    per_site = alg_bytes_per_site(9, 2, store_b, field_b)
    achieved = per_site * sites / (ms / args.steps / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    state_gb = sum(L.footprint()[0] for L in lats) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f64": "f64", "f32": "f32", "f16": "f16-storage/f32", "bf16": "bf16-storage/f32"}[args.storage],
            "data": "synthetic",
            "config": {"workload": f"2D rising bubble case {case} (Sec. III.D), 200x400 D2Q9, "
                                   f"{args.copies} lattices in one batch, {args.storage} storage",
                       "lattice": "D2Q9", "grid": list(c.shape), "copies": args.copies, "storage": args.storage,
                       "batch_shape": shape,
                       "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 ({state_gb:.2f} GB state in the batch)"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         "traffic": recorded_traffic(f"{args.workload}-{args.storage}-batch", sites)
                         if not args.inplace else None, "peak_kind": peak_kind,
                         "kernel": "batch_kernel<0> + batch_kernel<1> (split form over the batch)",
                         "store": "in-place AA" if args.inplace else "ping-pong", "bytes_per_site": per_site},
            "e2e": None, "gpu_launches": 2 * args.steps, "clocks": clk, "cpu_baseline": None,
        }), flush=True)
    B.close()
    for L in lats:
        L.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "impact":
        run_bubble(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
