"""Continuous-batching serving loop for lattice simulations.

Requests arrive over time, each a lattice (case, initial fields) that asks for a fixed
number of time steps or for a steady state: the residual E_R of Section V.A (relative
L2 change of the velocity field over an interval, 1000 steps there and by default
here) below a target.

Every admitted lattice stays resident on the device.  Between chunks of steps the loop
  * admits arrived requests, first come first served, while their state fits in the
    device-memory budget (tclbm_state_bytes against the budget, or the free HBM the
    driver reports minus a reserve),
  * picks the lattices to step in the next chunk: least remaining work (nodes x steps
    left) first, until `node_budget` nodes -- enough to fill the GPU -- are chosen,
  * advances the chosen lattices together with one batched launch per time step
    (tclbm_batch_*; the lattice list is swapped by stream-ordered copies, nothing waits
    for the GPU): lattices at least `tma[0]` columns wide in TMA-fed strips (the
    single-lattice TMA kernel's code, one CTA per strip), narrower ones in direct-load
    strips, so large and small requests overlap in the same launch.  With tma=None,
    lattices from `own_launch_nodes` nodes take their own single-lattice launches on
    the same stream instead (the earlier policy, kept for comparison),
  * retires finished lattices: their read-back waits on an event recorded after
    their last step, on a separate stream, so the next chunk is already queued.
At most `max_in_flight` chunks are queued ahead of the GPU, so an arrival is stepped
within about two chunks of its admission.

Every step of every lattice runs in the library's kernels; this module only decides
what runs when.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import tclbm


@dataclasses.dataclass
class Request:
    rid: int
    case: dict
    fields: object  # dict of initial fields, or a callable returning one (built at admission)
    steps: int | None = None  # fixed step count, or
    residual: float | None = None  # steady state: residual below this ...
    max_steps: int = 1_000_000  # ... or this many steps, whichever comes first
    t_arrival: float = 0.0  # seconds after the start of the run
    # filled in by the server
    t_admit: float | None = None
    t_done: float | None = None
    steps_done: int = 0
    result: dict | None = None
    converged: bool | None = None

    @property
    def nodes(self) -> int:
        return self.case["nx"] * self.case["ny"]

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def _fields_of(req):
    return req.fields() if callable(req.fields) else req.fields


@dataclasses.dataclass
class _Active:
    req: Request
    lat: tclbm.Lattice
    remaining: int  # steps to the end (fixed) or to the next residual check
    bytes: int


class Server:
    """Admits, batches, steps and retires lattice requests on the current device."""

    def __init__(self, storage: str = "fp16", rounding: str = "stochastic", hbm_budget: int | None = None,
                 reserve_bytes: int = 4 << 30, chunk: int = 64, check_every: int = 1000, max_in_flight: int = 2,
                 tile=None, keep_results: bool = True, node_budget: int = 48 << 20,
                 own_launch_nodes: int = 1 << 17, tma=(128, 16)):
        import torch

        self.torch = torch
        self.storage = storage
        self.rounding = rounding
        self.hbm_budget = hbm_budget
        self.reserve = reserve_bytes
        self.chunk = chunk
        self.check_every = check_every
        self.max_in_flight = max_in_flight
        self.tile = tile
        self.keep_results = keep_results
        self.node_budget = node_budget
        self.own_launch_nodes = own_launch_nodes
        self.tma = tma
        self.stream = torch.cuda.Stream()  # batched steps
        self.admit_stream = torch.cuda.Stream()  # creation and initial fields
        self.readout = torch.cuda.Stream()  # results of retired lattices
        self.queue: collections.deque[Request] = collections.deque()
        self.active: list[_Active] = []
        self.retiring: list[tuple[_Active, object]] = []
        self.done: list[Request] = []
        self.batch: tclbm.Batch | None = None
        self._batch_lats: list = []
        self._chunks: collections.deque = collections.deque()
        self.used_bytes = 0
        self.lattice_updates = 0
        self.peak_resident = 0

    # ------------------------------------------------------------ admission
    def _fits(self, need: int) -> bool:
        if self.hbm_budget is not None:
            return self.used_bytes + need <= self.hbm_budget
        free, _ = self.torch.cuda.mem_get_info()
        cached = self.torch.cuda.memory_reserved() - self.torch.cuda.memory_allocated()
        return need <= free + cached - self.reserve

    def submit(self, req: Request):
        if req.steps is None and req.residual is None:
            raise ValueError("a request needs a step count or a residual target")
        self.queue.append(req)

    def _admit(self, now: float) -> bool:
        changed = False
        while self.queue and self.queue[0].t_arrival <= now:
            req = self.queue[0]
            case = dict(req.case, storage=self.storage, rounding=self.rounding)
            need = tclbm.tclbm_state_bytes(tclbm.params_from_case(case))
            if not self._fits(need):
                if not self.active and not self.retiring:
                    raise MemoryError(f"request {req.rid} needs {need} bytes, more than the whole budget")
                break  # first come, first served: wait for memory
            try:
                lat = tclbm.Lattice(case, None, stream=self.admit_stream.cuda_stream)
            except tclbm.TclbmError as e:
                # the free-memory estimate was optimistic (fragmentation): wait for a retirement
                if e.status != tclbm.ENOMEM or not (self.active or self.retiring):
                    raise
                break
            self.queue.popleft()
            lat.init_fields(_fields_of(req))  # host fields: synchronises the admission stream only
            lat.set_stream(self.stream.cuda_stream)
            req.t_admit = self._clock()
            first = req.steps if req.steps is not None else min(self.check_every, req.max_steps)
            if req.residual is not None:
                lat.snapshot_velocity()
            self.active.append(_Active(req, lat, first, need))
            self.used_bytes += need
            changed = True
        return changed

    # ------------------------------------------------------------ stepping
    def _work_left(self, a: _Active) -> int:
        left = a.req.steps - a.req.steps_done if a.req.steps is not None else a.req.max_steps - a.req.steps_done
        return a.req.nodes * left

    def _select(self) -> list:
        """Lattices stepped in the next chunk: least remaining work first, up to the node budget."""
        chosen, nodes = [], 0
        for a in sorted(self.active, key=self._work_left):
            if chosen and nodes + a.req.nodes > self.node_budget:
                break
            chosen.append(a)
            nodes += a.req.nodes
        return chosen

    def _own_launch(self, a) -> bool:
        return self.tma is None and a.req.nodes >= self.own_launch_nodes

    def _sync_batch(self, chosen):
        lats = [a.lat for a in chosen if not self._own_launch(a)]
        if lats == self._batch_lats:
            return
        if self.batch is None:
            if not lats:
                return
            self.batch = tclbm.Batch(lats, stream=self.stream.cuda_stream)
            if self.tile is not None:
                self.batch.set_tile(*self.tile)
            if self.tma is not None:
                self.batch.set_tma(*self.tma)
        else:
            self.batch.set_lattices(lats)
        self._batch_lats = lats

    def _step_chunk(self):
        torch = self.torch
        while len(self._chunks) >= self.max_in_flight:
            self._chunks.popleft().synchronize()
        chosen = self._select()
        self._sync_batch(chosen)
        k = min(self.chunk, min(a.remaining for a in chosen))
        if self._batch_lats:
            self.batch.step(k)
        for a in chosen:
            if self._own_launch(a):
                a.lat.step(k)
        ev = torch.cuda.Event()
        ev.record(self.stream)
        self._chunks.append(ev)
        self.lattice_updates += k * sum(a.req.nodes for a in chosen)
        stepped = set(id(a) for a in chosen)
        keep = [a for a in self.active if id(a) not in stepped]
        for a in chosen:
            a.remaining -= k
            a.req.steps_done += k
            if a.remaining > 0:
                keep.append(a)
            elif a.req.steps is not None:
                self._retire(a, ev)
            else:
                # residual check (synchronises the batch stream at this boundary)
                d = a.lat.diagnostics()
                res = float(np.sqrt(d[6] / d[7])) if d[7] > 0 else 0.0
                if res < a.req.residual or a.req.steps_done >= a.req.max_steps:
                    a.req.converged = res < a.req.residual
                    self._retire(a, ev)
                else:
                    a.lat.snapshot_velocity()
                    a.remaining = min(self.check_every, a.req.max_steps - a.req.steps_done)
                    keep.append(a)
        self.active = keep

    def _retire(self, a: _Active, ev):
        # the read-back waits for this chunk only, on its own stream
        self.readout.wait_event(ev)
        a.lat.set_stream(self.readout.cuda_stream)
        self.retiring.append((a, ev))

    def _collect(self, block: bool):
        left = []
        for a, ev in self.retiring:
            if block or ev.query():
                if self.keep_results:
                    a.req.result = a.lat.moments()
                else:
                    a.lat.diagnostics()  # a device->host read of the request's result
                a.lat.close()
                self.used_bytes -= a.bytes
                a.req.t_done = self._clock()
                self.done.append(a.req)
            else:
                left.append((a, ev))
        self.retiring = left

    # ------------------------------------------------------------ driver
    def _clock(self) -> float:
        return time.perf_counter() - self._t0

    def run(self, requests, realtime: bool = True):
        """Serve `requests` (arrival times relative to now); returns them completed.

        realtime=False admits every request at once (arrival times ignored)."""
        self._t0 = time.perf_counter()
        for r in sorted(requests, key=lambda r: r.t_arrival):
            if not realtime:
                r.t_arrival = 0.0
            self.submit(r)
        while self.queue or self.active or self.retiring:
            now = self._clock()
            self._admit(now)
            self.peak_resident = max(self.peak_resident, len(self.active) + len(self.retiring))
            if self.active:
                self._step_chunk()
                self._collect(block=False)
            elif self.retiring:
                self._collect(block=True)
            elif self.queue:
                wait = self.queue[0].t_arrival - self._clock()
                if wait > 0:
                    time.sleep(min(wait, 0.01))
        self.torch.cuda.synchronize()
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        return self.done

    def stats(self, wall_s: float | None = None) -> dict:
        lat = np.array([r.latency for r in self.done]) if self.done else np.zeros(1)
        out = {"requests": len(self.done), "p50_s": float(np.percentile(lat, 50)),
               "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
               "lattice_updates": int(self.lattice_updates), "peak_resident": self.peak_resident}
        if wall_s:
            out["LU_per_s"] = self.lattice_updates / wall_s
        return out


def serve_alone(requests, storage="fp16", rounding="stochastic", realtime=True, keep_results=True, kernel=None,
                check_every=1000):
    """The plain path: requests one at a time in arrival order, each lattice alone with
    the single-lattice kernels (its own launches; `kernel` forces the variant, 1 = the
    direct-load kernel whose strip code the batch shares).  Returns (requests, stats)."""
    import torch

    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    lu = 0
    done = []
    for r in sorted(requests, key=lambda r: r.t_arrival):
        if realtime:
            wait = r.t_arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        else:
            r.t_arrival = 0.0
        case = dict(r.case, storage=storage, rounding=rounding)
        lat = tclbm.Lattice(case, _fields_of(r), stream=stream.cuda_stream)
        if kernel is not None:
            lat.set_kernel(kernel)
        r.t_admit = time.perf_counter() - t0
        if r.steps is not None:
            lat.step(r.steps)
            r.steps_done = r.steps
        else:
            lat.snapshot_velocity()
            while True:
                n = min(check_every, r.max_steps - r.steps_done)
                lat.step(n)
                r.steps_done += n
                d = lat.diagnostics()
                res = float(np.sqrt(d[6] / d[7])) if d[7] > 0 else 0.0
                if res < r.residual or r.steps_done >= r.max_steps:
                    r.converged = res < r.residual
                    break
                lat.snapshot_velocity()
        lu += r.steps_done * r.nodes
        r.result = lat.moments() if keep_results else None
        if not keep_results:
            lat.diagnostics()
        lat.close()
        r.t_done = time.perf_counter() - t0
        done.append(r)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    lat_s = np.array([r.latency for r in done])
    return done, {"requests": len(done), "p50_s": float(np.percentile(lat_s, 50)),
                  "p99_s": float(np.percentile(lat_s, 99)), "mean_s": float(lat_s.mean()),
                  "lattice_updates": int(lu), "LU_per_s": lu / wall}
