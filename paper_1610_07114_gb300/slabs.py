"""Slab decomposition of one lattice along y, with a row exchange every k time steps.

The paper advances one lattice as a whole.  Split across devices, a lattice becomes
slabs of whole rows, each stepped by its own device, and the slabs swap the rows next
to their cut every few steps.  This module holds that split and exchange plan.  On one
device it runs the slabs as separate lattices and refreshes their ghost rows with
device-to-device row copies (tclbm_copy_rows).  A rank of a multi-device run would send
and receive the same rows.

Why 2k ghost rows give k steps.  Over one time step a node pulls from the rows next to
it.  It also needs the velocity of the next node on either side, for the central
differences of the correction term (Section IV), and those velocities are themselves
computed from the pulls one row further out.  So a row's new state depends on the two
rows on each side of it.

A slab lattice closes its outer edge with a boundary the whole lattice lacks there:
an equilibrium wall where the slab's other side is a real wall, or periodic wrap when
both sides are cut.  After one step, that edge row and the row next to it no longer
hold the whole lattice's state.  Each further step spoils two more rows.  With g = 2k
ghost rows beyond each cut, the owned rows stay exact for k steps, and the exchange
then overwrites every ghost row with its owner's current state.

An exchange also runs right after initialisation, because initialisation rebuilds
the artificial edge rows as walls.

Arithmetic per node does not change with the split, with two exceptions that each
depend on a node's global position:
  * the Taylor-Green force table, which is sized by the lattice's ny;
  * the stochastic-rounding bits of 16-bit storage, which hash the node index.
Slab lattices would see local positions, so both are refused here.  With everything
else, the owned rows evolve bit for bit as in the undivided lattice when every lattice
uses the same step kernel variant.
"""
from __future__ import annotations

import copy
import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Slab:
    lo: int  # first row of the whole lattice owned by the slab
    hi: int  # one past its last owned row
    below: int  # ghost rows under the owned rows (0 on a real wall)
    above: int  # ghost rows over them

    @property
    def own(self) -> int:
        return self.hi - self.lo

    @property
    def ny(self) -> int:
        return self.below + self.own + self.above

    def rows(self, ny_total: int) -> np.ndarray:
        """Row of the whole lattice held by each local row (periodic wrap)."""
        return (np.arange(self.ny) + self.lo - self.below) % ny_total


def plan(ny: int, parts: int, ghost: int, periodic: bool) -> list[Slab]:
    """Cut ny rows into `parts` slabs of nearly equal height, `ghost` rows at each cut."""
    if parts < 2:
        raise ValueError("a slab decomposition needs parts >= 2")
    if ghost < 2 or ghost % 2:
        raise ValueError("ghost must be an even number >= 2 (2 rows per step between exchanges)")
    bounds = [ny * k // parts for k in range(parts + 1)]
    slabs = []
    for k in range(parts):
        s = Slab(bounds[k], bounds[k + 1], ghost if (periodic or k > 0) else 0,
                 ghost if (periodic or k < parts - 1) else 0)
        # ghost rows come from one neighbour's owned rows; a real wall needs 3 owned rows
        if s.own < max(ghost, 3):
            raise ValueError(f"slab {k} owns {s.own} rows, fewer than max(ghost, 3) = {max(ghost, 3)}")
        slabs.append(s)
    return slabs


def exchanges(slabs: list[Slab], periodic: bool) -> list[tuple[int, int, int, int, int]]:
    """Row copies that refresh every ghost row: (dst slab, dst row, src slab, src row, rows),
    rows local to each slab."""
    faces = [(k, k + 1) for k in range(len(slabs) - 1)]
    if periodic:
        faces.append((len(slabs) - 1, 0))
    out = []
    for lo, hi in faces:  # slab `lo` lies under slab `hi`
        a, b = slabs[lo], slabs[hi]
        out.append((lo, a.below + a.own, hi, b.below, a.above))  # a's upper ghosts <- b's lowest owned rows
        out.append((hi, 0, lo, a.below + a.own - b.below, b.below))  # b's lower ghosts <- a's highest owned rows
    return out


def check_case(case: dict):
    if case["force"]["kind"] == "taylor_green":
        raise ValueError("the Taylor-Green force table depends on the whole lattice's ny")
    if case.get("storage", "fp32") != "fp32" and case.get("rounding", "nearest") == "stochastic":
        raise ValueError("stochastic-rounding bits depend on the node's index in the whole lattice")


def y_periodic(case: dict) -> bool:
    return case["walls"]["y-"]["kind"] == "periodic"


def slab_case(case: dict, s: Slab) -> dict:
    """Case of the slab lattice: the whole lattice's, with ny and the y sides of a cut replaced."""
    c = copy.deepcopy(case)
    c["ny"] = s.ny
    c["name"] = f"{case.get('name', 'lattice')}[{s.lo}:{s.hi}]"
    if not y_periodic(case):
        rest = {"kind": "equilibrium", "ux": 0.0, "uy": 0.0, "T": case["T0"], "rho": 1.0, "therm": "fixed"}
        if s.below and s.above:
            for side in ("y-", "y+"):
                c["walls"][side] = dict(rest, kind="periodic")
        elif s.below:
            c["walls"]["y-"] = rest
        elif s.above:
            c["walls"]["y+"] = dict(rest)
    return c


def slab_fields(fields: dict, s: Slab, ny: int) -> dict:
    rows = s.rows(ny)
    return {k: np.ascontiguousarray(np.asarray(v)[rows]) for k, v in fields.items()}


class Slabs:
    """One lattice advanced as `parts` slab lattices on the current device, the ghost
    rows refreshed by tclbm_copy_rows every `exchange_every` steps."""

    def __init__(self, case: dict, fields: dict | None = None, parts: int = 2, exchange_every: int = 1,
                 kernel: int | None = None, stream=None):
        from . import tclbm

        check_case(case)
        self.tclbm = tclbm
        self.case = case
        self.nx, self.ny = case["nx"], case["ny"]
        self.periodic = y_periodic(case)
        self.k = int(exchange_every)
        self.slabs = plan(self.ny, parts, 2 * self.k, self.periodic)
        self.copies = exchanges(self.slabs, self.periodic)
        self.lattices = [tclbm.Lattice(slab_case(case, s), None, stream=stream) for s in self.slabs]
        if kernel is not None:
            for lat in self.lattices:
                lat.set_kernel(kernel)
        self.steps_done = 0
        if fields is not None:
            self.init_fields(fields)

    def init_fields(self, fields: dict):
        for s, lat in zip(self.slabs, self.lattices):
            lat.init_fields(slab_fields(fields, s, self.ny))
        self.exchange()
        self.steps_done = 0

    def exchange(self):
        for d, dr, s, sr, n in self.copies:
            self.tclbm.tclbm_copy_rows(self.lattices[d].handle, dr, self.lattices[s].handle, sr, n)

    def step(self, n: int = 1):
        if n < 0:
            raise ValueError("n must be >= 0")
        while n > 0:
            k = min(self.k, n)
            for lat in self.lattices:
                lat.step(k)
            self.exchange()
            n -= k
            self.steps_done += k

    def _gather(self, parts, shape):
        out = np.zeros(shape)
        for s, a in zip(self.slabs, parts):
            out[..., s.lo:s.hi, :] = a[..., s.below:s.below + s.own, :]
        return out

    def moments(self) -> dict:
        ms = [lat.moments() for lat in self.lattices]
        return {k: self._gather([m[k] for m in ms], (self.ny, self.nx)) for k in ("rho", "ux", "uy", "T")}

    def populations(self):
        ps = [lat.populations() for lat in self.lattices]
        f = self._gather([p[0] for p in ps], (9, self.ny, self.nx))
        h = self._gather([p[1] for p in ps], (9, self.ny, self.nx)) if ps[0][1] is not None else None
        return f, h

    def close(self):
        for lat in self.lattices:
            lat.close()
        self.lattices = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
