"""Benchmark of the fused thermal cascaded LBM step on GB300 (lattice updates per second).

Default workload: Rayleigh-Benard convection, single 256 x 128 lattice, Ra = 1e4,
Pr = 0.71, gamma = 1.4, FP32 populations, gravity as a direct body force, FP64
Nusselt tracking.  One bench step = `--chunk` (default 1000) lattice time steps plus
one FP64 diagnostics reduction (the Nusselt sum).  A lattice update (LU) is one node
advanced one time step for both distributions f and h.

The JSON line carries: value (LU/s, inputs resident in HBM), e2e (same metric through
the C ABI with host buffers, host<->device copies inside the timed region), roofline of
the step kernel against the measured HBM copy bandwidth, a roofline probe on
lattices far larger than L2, the oracle's CPU throughput on a bounded sample, clocks
sampled during the timed region, and the number of kernel launches.

`--impl reference` times the FP64 CPU oracle on the same workload instead.
Multi-GPU (torchrun): every rank advances its own replica (weak scaling; the path has
no exchange step between independent lattices); time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_LU = {"fp32": 144, "bf16": 72, "fp16": 72}  # f + h populations read once and written once


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_source_hash():
    h = hashlib.sha256()
    # device code of the single-lattice step kernels (direct and TMA-fed)
    for rel in ("paper_1610_07114_gb300/csrc/tclbm_device.cuh", "paper_1610_07114_gb300/csrc/tclbm_tma.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(key):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(key)
        if e and e.get("source_hash") == _kernel_source_hash():
            return e.get("bytes_per_launch")
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                parts = [p.strip() for p in out.stdout.strip().split(",")]
                if len(parts) >= 8:
                    self.samples.append(parts)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


from paper_1610_07114_gb300.replicas import barrier as _barrier  # noqa: E402
from paper_1610_07114_gb300.replicas import dist_env as _dist  # noqa: E402
from paper_1610_07114_gb300.replicas import max_over_ranks as _max_over_ranks  # noqa: E402
from paper_1610_07114_gb300.replicas import sum_over_ranks as _sum_over_ranks  # noqa: E402


def _workload(args):
    from paper_1610_07114_gb300 import workloads as W

    case, fields = W.rayleigh_benard(args.nx, args.ny, Ra=args.ra, seed=1, storage=args.storage)
    return case, fields


def _oracle_rate(case, fields, budget_s, threads):
    """Oracle throughput (LU/s) on a bounded sample of the workload: as many single
    time steps as fit in about budget_s seconds of CPU work."""
    import oracle

    o = oracle.Oracle(case, fields, threads=threads)
    o.step(1)  # warm
    n = case["nx"] * case["ny"]
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    return n * steps / dt, steps, dt


def bench_reference(args):
    """The FP64 CPU oracle, as it stands, on the host cores (rank 0 only)."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    case, fields = _workload(args)
    threads = len(os.sched_getaffinity(0))
    per_step_budget = max(0.5, min(10.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        _oracle_rate(case, fields, min(per_step_budget, 1.0), threads)
    rates = []
    total_steps = 0
    for _ in range(args.steps):
        r, s, _dt = _oracle_rate(case, fields, per_step_budget, threads)
        rates.append(r)
        total_steps += s
    value = float(np.mean(rates))
    n = case["nx"] * case["ny"]
    line = {
        "impl": "reference", "metric": "lattice_updates_per_s", "value": value, "unit": "LU/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": args.chunk * n / value * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"rayleigh_benard_{args.nx}x{args.ny}_Ra{args.ra:g}", "chunk_steps": args.chunk,
                   "storage": "fp64 (oracle)"},
        "cpu_baseline": {"value": value, "unit": "LU/s", "cores": threads, "kind": "oracle",
                         "sample": f"{total_steps} single time steps of the {args.nx}x{args.ny} lattice "
                                   f"(~{per_step_budget:.1f} s per bench step), OpenMP over {threads} threads"},
        "e2e": {"value": value, "unit": "LU/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _flush_l2(buf):
    buf.add_(1.0)  # writes 256 MiB, twice the 129 MB L2


def profile_run(args):
    """Step one Rayleigh-Benard-shaped lattice only (for ncu captures of the step kernel)."""
    import torch

    torch.cuda.set_device(0)
    from paper_1610_07114_gb300 import build as B

    B.build()
    from paper_1610_07114_gb300 import tclbm
    from paper_1610_07114_gb300 import workloads as W

    case, fields = W.rayleigh_benard(args.probe_nx, args.probe_ny, Ra=1e4, seed=2, storage=args.storage)
    lat = tclbm.Lattice(case, fields)
    if args.kernel is not None:
        lat.set_kernel(args.kernel)  # before the shape: a new variant resets it
    if args.tile:
        lat.set_tile(*args.tile)
    lat.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    lat.step(args.probe_steps)
    e1.record()
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3 / args.probe_steps
    n = case["nx"] * case["ny"]
    print(json.dumps({"profile_run": f"rb_{args.probe_nx}x{args.probe_ny}_{args.storage}", "kernel": lat.describe(),
                      "us_per_step": dt * 1e6, "LU_per_s": n / dt,
                      "GBs": BYTES_PER_LU[args.storage] * n / dt / 1e9}))
    lat.close()
    return 0


def bench_batch(args, tclbm, stream):
    """Batched Rayleigh-Benard sweep (256 lattices, 64x32 .. 1024x512, FP16 deviations with
    stochastic rounding): the batched kernel against the plain path (each lattice its own
    launches), both timed with CUDA events on the same stream over the same lattices.
    With several ranks every rank runs its own sweep (weak scaling, no collective on
    the data path); times are the maximum over ranks."""
    import torch

    from paper_1610_07114_gb300 import workloads as W

    world, rank, _ = _dist()
    cases = W.batched_rb_sweep(count=args.batch_count, seed=1234 + 7919 * rank, storage=args.batch_storage)
    lats = [tclbm.Lattice(dict(c, rounding="stochastic"), f, stream=stream.cuda_stream) for c, f in cases]
    nodes = sum(c["nx"] * c["ny"] for c, _ in cases)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn):
        e0, e1 = ev(), ev()
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    k = args.batch_steps
    for l in lats:
        l.step(2)
        l.step(k)  # builds the lattice's step graph outside the timed region
    # plain, chunked: every lattice advanced k steps by its own launches (captured graphs)
    t_chunk = timed(lambda: [l.step(k) for l in lats])
    # plain, step-major: one launch per lattice per step
    k1 = max(2, k // 8)
    t_rr = timed(lambda: [l.step(1) for _ in range(k1) for l in lats]) * k / k1
    b = tclbm.Batch(lats, stream=stream.cuda_stream)
    tx, rows, pers, us = b.autotune(trial_steps=args.batch_tune_steps)
    b.step(4)
    b.step(k)  # builds the batch's step graph outside the timed region
    t_batch = timed(lambda: b.step(k))
    desc = b.describe()
    b.close()
    for l in lats:
        l.close()
    torch.cuda.synchronize()
    peak, peak_kind = _peaks()
    lu = _sum_over_ranks(float(nodes * k), world)
    t_chunk, t_rr, t_batch = (_max_over_ranks(t, world) for t in (t_chunk, t_rr, t_batch))
    plain_best = min(t_chunk, t_rr)
    achieved = BYTES_PER_LU[args.batch_storage] * lu / world / t_batch / 1e9  # one GPU's share
    return {"workload": f"rb_sweep_{args.batch_count}_{args.batch_storage}", "lattices": args.batch_count * world,
            "nodes": nodes, "steps_timed": k, "kernel": desc,
            "autotuned": {"tx": tx, "rows": rows, "persistent": pers, "us_per_step": us},
            "LU_per_s": lu / t_batch, "ms_per_step": t_batch / k * 1e3,
            "plain_chunked_LU_per_s": lu / t_chunk, "plain_launch_per_step_LU_per_s": lu / t_rr,
            "ratio_vs_plain": plain_best / t_batch,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "bytes_per_LU": BYTES_PER_LU[args.batch_storage], "peak_source": f"{peak_kind} hbm_gbs"},
            "rounding": "stochastic"}


def bench_serve(args):
    """Serving loop on Poisson-arriving requests (Couette, Taylor-Green, Rayleigh-Benard;
    FP16 deviations with stochastic rounding) against serving each request alone with
    the plain single-lattice path, both in real time on the same trace."""
    import torch

    from paper_1610_07114_gb300 import serve
    from paper_1610_07114_gb300 import workloads as W

    world, rank, _ = _dist()
    trace = W.serving_trace(duration_s=args.serve_duration, rate=args.serve_rate, seed=42 + rank,
                            steps_choices=args.serve_steps, steady_frac=args.serve_steady_frac,
                            steady_residual=args.serve_steady_residual)
    storage = args.serve_storage
    rounding = "stochastic" if storage != "fp32" else "nearest"

    def requests():
        # cases now, initial fields at admission (a long trace would not fit in host memory)
        out = []
        for i, r in enumerate(trace):
            case, _ = W.build_request(r, fields=False)
            out.append(serve.Request(rid=i, case=case, fields=lambda r=r: W.build_request(r)[1], steps=r["steps"],
                                     t_arrival=r["t_arrival"], residual=r.get("residual"),
                                     max_steps=args.serve_steady_max_steps))
        return out

    def steady(done):
        s = [r for r in done if r.residual is not None]
        return {"requests": len(s), "converged": sum(bool(r.converged) for r in s),
                "steps_max": max((r.steps_done for r in s), default=0),
                "latency_max_s": max((r.latency for r in s), default=0.0)}

    reqs = requests()  # built before either clock starts
    torch.cuda.synchronize()
    _barrier(world)
    t0 = time.perf_counter()
    srv = serve.Server(storage=storage, rounding=rounding, chunk=args.serve_chunk, keep_results=False)
    done = srv.run(reqs)
    wall = _max_over_ranks(time.perf_counter() - t0, world)
    served = srv.stats(wall)
    served["LU_per_s"] = _sum_over_ranks(float(served["lattice_updates"]), world) / wall
    served["steady_state"] = steady(done)
    reqs = requests()
    torch.cuda.synchronize()
    _barrier(world)
    t0 = time.perf_counter()
    done_alone, alone = serve.serve_alone(reqs, storage=storage, rounding=rounding, keep_results=False)
    wall_alone = _max_over_ranks(time.perf_counter() - t0, world)
    alone["steady_state"] = steady(done_alone)
    alone["LU_per_s"] = _sum_over_ranks(float(alone["lattice_updates"]), world) / wall_alone
    return {"workload": f"serve_poisson_{args.serve_rate:g}per_s_{args.serve_duration:g}s",
            "requests_per_rank": len(trace), "ranks": world, "latencies": "rank 0",
            "nodes_total": int(sum(r["nx"] * r["ny"] for r in trace)), "wall_s": wall, "served": served,
            "alone": alone, "ratio_LU_per_s": served["LU_per_s"] / alone["LU_per_s"],
            "p99_ratio_alone_over_served": alone["p99_s"] / served["p99_s"],
            "storage": storage, "rounding": rounding, "chunk": args.serve_chunk,
            "steps_choices": list(args.serve_steps), "steady_frac": args.serve_steady_frac,
            "batching": "all lattices in one batched launch per step (TMA-fed strips from 128 columns)"}


def serve_run(args):
    import torch

    torch.cuda.set_device(0)
    from paper_1610_07114_gb300 import build as B

    B.build()
    print(json.dumps({"serving": bench_serve(args)}))
    return 0


def batch_run(args):
    import torch

    torch.cuda.set_device(0)
    from paper_1610_07114_gb300 import build as B

    B.build()
    from paper_1610_07114_gb300 import tclbm

    stream = torch.cuda.Stream()
    print(json.dumps({"batched": bench_batch(args, tclbm, stream)}))
    return 0


def bench_gpu(args):
    import torch

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1610_07114_gb300 import build as B

    B.build()
    from paper_1610_07114_gb300 import tclbm

    case, fields = _workload(args)
    n = case["nx"] * case["ny"]
    stream = torch.cuda.Stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    lat = tclbm.Lattice(case, fields, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        dev_fields = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in fields.items()}
    torch.cuda.synchronize()
    lat.init_fields(dev_fields)
    desc = lat.describe()

    def one_step(ev):
        ev[0].record(stream)
        lat.step(args.chunk)
        ev[1].record(stream)
        d = lat.diagnostics()  # FP64 Nusselt sum (synchronises the stream)
        ev[2].record(stream)
        return d

    for _ in range(args.warmup):
        one_step([torch.cuda.Event(enable_timing=True) for _ in range(3)])
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                _flush_l2(flush)
            d = one_step(evs[k])
        torch.cuda.synchronize()
    _barrier(world)
    t_step = sum(e[0].elapsed_time(e[1]) for e in evs) / 1e3
    t_diag = sum(e[1].elapsed_time(e[2]) for e in evs) / 1e3
    t_total = _max_over_ranks(t_step + t_diag, world)
    value = world * n * args.chunk * args.steps / t_total
    kernel_s = t_step / (args.chunk * args.steps)  # average step-kernel time (graph replays included)

    # Nusselt number (Section V.D): Nu = 1 + <u_y (T - T0)> H / (kappa dT)
    H = case["ny"] - 1
    kappa = case["visc"] / case["Pr"]
    nu_num = 1.0 + (d[5] / n) * H / (kappa * (case["T_bot"] - case["T_top"]))

    # ---- e2e: host fields in, host moments out, through the C ABI
    host_in = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in fields.items()}
    out = [np.zeros((case["ny"], case["nx"])) for _ in range(4)]
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lat.init_fields(host_in)
        lat.step(args.chunk)
        tclbm.tclbm_moments(lat.handle, *[o.ctypes.data for o in out], 0)
    torch.cuda.synchronize()
    t_e2e = _max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = world * n * args.chunk * e2e_steps / t_e2e
    lat.close()

    # ---- roofline probe: lattices far larger than L2 (step kernel alone, per launch)
    peak, peak_kind = _peaks()
    probes = []
    if not args.no_probe:
        from paper_1610_07114_gb300 import workloads as W

        sizes = [(args.probe_nx, args.probe_ny)]
        if not args.no_probe_large:
            sizes.append((2 * args.probe_nx, 2 * args.probe_ny))
        for (pnx, pny), storage in [(sz, st) for sz in sizes for st in args.probe_storages]:
            pc, pf = W.rayleigh_benard(pnx, pny, Ra=1e4, seed=2, storage=storage)
            pl = tclbm.Lattice(pc, pf, stream=stream.cuda_stream)
            pl.step(4)
            torch.cuda.synchronize()
            # the same bytes per probe at every size (at least 20 launches)
            reps = max(20, args.probe_steps * args.probe_nx * args.probe_ny // (pnx * pny))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pl.step(reps)
            e1.record(stream)
            torch.cuda.synchronize()
            dt = e0.elapsed_time(e1) / 1e3 / reps
            pn = pc["nx"] * pc["ny"]
            achieved = BYTES_PER_LU[storage] * pn / dt / 1e9
            key = f"rb_{pnx}x{pny}_{storage}"
            probes.append({"workload": key, "kernel": pl.describe(), "LU_per_s": pn / dt, "launches": reps,
                           "us_per_launch": dt * 1e6, "achieved_GBs": achieved, "peak_GBs": peak,
                           "frac": achieved / peak, "bytes_per_LU": BYTES_PER_LU[storage],
                           "traffic": _profiled_traffic(key)})
            pl.close()

    batched = None if args.no_batch else bench_batch(args, tclbm, stream)
    serving = None if args.no_serve else bench_serve(args)

    if rank != 0:
        return 0
    achieved = BYTES_PER_LU[args.storage] * n / kernel_s / 1e9
    wkey = f"rb_{args.nx}x{args.ny}_{args.storage}"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": _profiled_traffic(wkey), "peak_source": f"{peak_kind} hbm_gbs (copy)",
                "kernel": desc, "bytes_per_LU": BYTES_PER_LU[args.storage],
                "note": "the 4.7 MB state stays in L2 within a chunk; see roofline_probe for lattices >> L2"}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        threads = len(os.sched_getaffinity(0))
        r, s, dt = _oracle_rate(case, fields, args.cpu_budget, threads)
        cpu = {"value": r, "unit": "LU/s", "cores": threads, "kind": "oracle",
               "sample": f"{s} time steps of the {args.nx}x{args.ny} lattice in {dt:.1f} s (OpenMP, {threads} threads)"}
    clk = clocks.summary()
    line = {
        "metric": "lattice_updates_per_s", "value": value, "unit": "LU/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage == "fp32" else f"{args.storage}-dev/f32",
        "data": "synthetic",
        "config": {"workload": f"rayleigh_benard_{args.nx}x{args.ny}_Ra{args.ra:g}", "nx": args.nx, "ny": args.ny,
                   "Ra": args.ra, "chunk_steps": args.chunk,
                   "storage": args.storage, "l2": "flushed (256 MiB write) before every timed step; the state itself "
                                                 "is L2-resident within a step",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": "LU/s", "h2d_bytes_per_step": 4 * 8 * n, "d2h_bytes_per_step": 4 * 8 * n,
                "steps": e2e_steps},
        "roofline": roofline,
        "roofline_probe": probes,
        "batched": batched,
        "serving": serving,
        "cpu_baseline": cpu,
        "clocks": clk,
        "gpu_launches": args.steps * (args.chunk + 2),
        "nusselt": nu_num,
        "kernel_us": kernel_s * 1e6,
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tclbm", choices=["tclbm", "reference"])
    ap.add_argument("--chunk", type=int, default=1000, help="lattice time steps per bench step")
    ap.add_argument("--nx", type=int, default=256)
    ap.add_argument("--ny", type=int, default=128)
    ap.add_argument("--ra", type=float, default=1e4)
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--probe-nx", type=int, default=4096)
    ap.add_argument("--probe-ny", type=int, default=2048)
    ap.add_argument("--probe-steps", type=int, default=200)
    ap.add_argument("--probe-storages", nargs="*", default=["fp32", "bf16", "fp16"])
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--no-probe-large", action="store_true",
                    help="skip the second probe size (2 probe-nx x 2 probe-ny)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--profile-run", action="store_true",
                    help="only step one --probe-nx x --probe-ny lattice --probe-steps times (for ncu)")
    ap.add_argument("--tile", type=int, nargs=2, default=None, help="override (tx, rows per CTA)")
    ap.add_argument("--kernel", type=int, default=None, help="step kernel variant: 0 TMA-staged, 1 direct loads")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-storage", default="fp16", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--batch-steps", type=int, default=64)
    ap.add_argument("--batch-tune-steps", type=int, default=6)
    ap.add_argument("--batch-only", action="store_true", help="print only the batched-sweep measurement")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-duration", type=float, default=1.0, help="seconds of Poisson arrivals")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="mean arrivals per second")
    ap.add_argument("--serve-chunk", type=int, default=64)
    ap.add_argument("--serve-steps", type=int, nargs="+", default=[200, 500, 1000, 2000],
                    help="fixed step counts the requests draw from")
    ap.add_argument("--serve-steady-frac", type=float, default=0.0,
                    help="share of requests that ask for the steady state (Couette 32x128, nu 0.3)")
    ap.add_argument("--serve-steady-residual", type=float, default=1e-8)
    ap.add_argument("--serve-steady-max-steps", type=int, default=400000)
    ap.add_argument("--serve-storage", default="fp16", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--serve-only", action="store_true", help="print only the serving measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return bench_reference(args)
    if args.profile_run:
        return profile_run(args)
    if args.batch_only:
        return batch_run(args)
    if args.serve_only:
        return serve_run(args)
    return bench_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
