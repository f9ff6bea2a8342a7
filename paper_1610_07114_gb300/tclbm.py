"""ctypes binding of libtclbm.so (include/tclbm.h): argument marshalling only.

Every step of the lattice update runs in the library's sm_103a kernels; PyTorch
supplies device memory (its caching allocator, through the create-time hooks) and
streams.  There is no CPU fallback: if the shared library is missing this module
raises on import.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtclbm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libtclbm.so not found at {LIB_PATH}; build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
NDIAG = 8
WALL = {"periodic": 0, "zouhe": 1, "nee": 2, "equilibrium": 3}
THERM = {"fixed": 0, "adiabatic": 1}
VISC = {"nu": 0, "mu": 1, "mu_T": 2, "w1": 3}
FORCE = {"none": 0, "accel": 1, "taylor_green": 2}
STORAGE = {"fp32": 0, "bf16": 1, "fp16": 2}
ROUNDING = {"nearest": 0, "stochastic": 1}
SIDES = ("x-", "x+", "y-", "y+")
DIAG_NAMES = ("mass", "momentum_x", "momentum_y", "energy", "kinetic", "nusselt_sum", "residual_num",
              "residual_den")


class TclbmError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: status {status}: {tclbm_last_error()}")
        self.status = status


class tclbm_wall(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("therm", ctypes.c_int32), ("rho", ctypes.c_double),
                ("ux", ctypes.c_double), ("uy", ctypes.c_double), ("T", ctypes.c_double)]


class tclbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("thermal", ctypes.c_int32), ("correction", ctypes.c_int32),
        ("visc_law", ctypes.c_int32), ("visc", ctypes.c_double),
        ("bgk", ctypes.c_int32), ("w2", ctypes.c_double), ("w3", ctypes.c_double), ("w4", ctypes.c_double),
        ("Pr", ctypes.c_double), ("gamma", ctypes.c_double), ("R", ctypes.c_double), ("T0", ctypes.c_double),
        ("force_kind", ctypes.c_int32), ("ax", ctypes.c_double), ("ay", ctypes.c_double), ("famp", ctypes.c_double),
        ("wall", tclbm_wall * 4),
        ("storage", ctypes.c_int32),
        ("T_ref", ctypes.c_double),
        ("rounding", ctypes.c_int32),
        ("work", ctypes.c_int32),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_P = ctypes.POINTER(tclbm_params)

_lib.tclbm_state_bytes.argtypes = [_P]
_lib.tclbm_state_bytes.restype = ctypes.c_size_t
_lib.tclbm_create.argtypes = [_P, ALLOC_FN, FREE_FN, _vp, _vp, ctypes.POINTER(_vp)]
_lib.tclbm_create.restype = ctypes.c_int
_lib.tclbm_init_fields.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int32]
_lib.tclbm_init_fields.restype = ctypes.c_int
_lib.tclbm_step.argtypes = [_vp, ctypes.c_int64]
_lib.tclbm_step.restype = ctypes.c_int
_lib.tclbm_moments.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int32]
_lib.tclbm_moments.restype = ctypes.c_int
_lib.tclbm_diagnostics.argtypes = [_vp, _dp]
_lib.tclbm_diagnostics.restype = ctypes.c_int
_lib.tclbm_snapshot_velocity.argtypes = [_vp]
_lib.tclbm_snapshot_velocity.restype = ctypes.c_int
_lib.tclbm_get_populations.argtypes = [_vp, _vp, _vp, ctypes.c_int32]
_lib.tclbm_get_populations.restype = ctypes.c_int
_lib.tclbm_set_populations.argtypes = [_vp, _vp, _vp, ctypes.c_int32]
_lib.tclbm_set_populations.restype = ctypes.c_int
_lib.tclbm_steps_done.argtypes = [_vp]
_lib.tclbm_steps_done.restype = ctypes.c_int64
_lib.tclbm_set_stream.argtypes = [_vp, _vp]
_lib.tclbm_set_stream.restype = ctypes.c_int
_lib.tclbm_destroy.argtypes = [_vp]
_lib.tclbm_destroy.restype = ctypes.c_int
_lib.tclbm_last_error.argtypes = []
_lib.tclbm_last_error.restype = ctypes.c_char_p
_lib.tclbm_describe.argtypes = [_vp]
_lib.tclbm_describe.restype = ctypes.c_char_p
_lib.tclbm_set_tile.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32]
_lib.tclbm_set_tile.restype = ctypes.c_int
_lib.tclbm_test_skip_row.argtypes = [_vp, ctypes.c_int32]
_lib.tclbm_test_skip_row.restype = ctypes.c_int
_lib.tclbm_test_rcp.argtypes = [_vp, _vp, ctypes.c_int64, _vp]
_lib.tclbm_test_rcp.restype = ctypes.c_int
_lib.tclbm_set_kernel.argtypes = [_vp, ctypes.c_int32]
_lib.tclbm_set_kernel.restype = ctypes.c_int
_lib.tclbm_copy_rows.argtypes = [_vp, ctypes.c_int32, _vp, ctypes.c_int32, ctypes.c_int32]
_lib.tclbm_copy_rows.restype = ctypes.c_int
_lib.tclbm_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, _vp, ctypes.POINTER(_vp)]
_lib.tclbm_batch_create.restype = ctypes.c_int
_lib.tclbm_batch_set_lattices.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.c_int32]
_lib.tclbm_batch_set_lattices.restype = ctypes.c_int
_lib.tclbm_batch_size.argtypes = [_vp]
_lib.tclbm_batch_size.restype = ctypes.c_int32
_lib.tclbm_batch_step.argtypes = [_vp, ctypes.c_int64]
_lib.tclbm_batch_step.restype = ctypes.c_int
_lib.tclbm_batch_set_tile.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
_lib.tclbm_batch_set_tile.restype = ctypes.c_int
_ip = ctypes.POINTER(ctypes.c_int32)
_lib.tclbm_batch_autotune.argtypes = [_vp, ctypes.c_int32, _ip, _ip, _ip, ctypes.POINTER(ctypes.c_float)]
_lib.tclbm_batch_autotune.restype = ctypes.c_int
_lib.tclbm_batch_set_tma.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32]
_lib.tclbm_batch_set_tma.restype = ctypes.c_int
_lib.tclbm_batch_tma_shape.argtypes = [_vp, _ip, _ip]
_lib.tclbm_batch_tma_shape.restype = ctypes.c_int
_lib.tclbm_batch_describe.argtypes = [_vp]
_lib.tclbm_batch_describe.restype = ctypes.c_char_p
_lib.tclbm_batch_steps_done.argtypes = [_vp]
_lib.tclbm_batch_steps_done.restype = ctypes.c_int64
_lib.tclbm_batch_destroy.argtypes = [_vp]
_lib.tclbm_batch_destroy.restype = ctypes.c_int

EXPORTED = [name for name in dir(_lib) if name.startswith("tclbm_")]


def library():
    return _lib


# ------------------------------------------------------------------ C-ABI names


def tclbm_last_error() -> str:
    return _lib.tclbm_last_error().decode()


def tclbm_state_bytes(params: tclbm_params) -> int:
    return int(_lib.tclbm_state_bytes(ctypes.byref(params)))


def _check(st, what):
    if st != OK:
        raise TclbmError(st, what)


def tclbm_create(params: tclbm_params, alloc=None, free=None, ctx=None, stream=None):
    """Returns a handle (ctypes void pointer).  `alloc`/`free` are ALLOC_FN/FREE_FN or None."""
    h = _vp()
    st = _lib.tclbm_create(ctypes.byref(params), alloc or ALLOC_FN(), free or FREE_FN(), ctx, stream,
                           ctypes.byref(h))
    _check(st, "tclbm_create")
    return h


def tclbm_init_fields(h, rho, ux, uy, T, on_device):
    _check(_lib.tclbm_init_fields(h, rho, ux, uy, T, int(on_device)), "tclbm_init_fields")


def tclbm_step(h, n):
    _check(_lib.tclbm_step(h, int(n)), "tclbm_step")


def tclbm_moments(h, rho, ux, uy, T, on_device):
    _check(_lib.tclbm_moments(h, rho, ux, uy, T, int(on_device)), "tclbm_moments")


def tclbm_diagnostics(h, out):
    _check(_lib.tclbm_diagnostics(h, out), "tclbm_diagnostics")


def tclbm_snapshot_velocity(h):
    _check(_lib.tclbm_snapshot_velocity(h), "tclbm_snapshot_velocity")


def tclbm_get_populations(h, f, hh, on_device):
    _check(_lib.tclbm_get_populations(h, f, hh, int(on_device)), "tclbm_get_populations")


def tclbm_set_populations(h, f, hh, on_device):
    _check(_lib.tclbm_set_populations(h, f, hh, int(on_device)), "tclbm_set_populations")


def tclbm_steps_done(h) -> int:
    return int(_lib.tclbm_steps_done(h))


def tclbm_set_stream(h, stream):
    _check(_lib.tclbm_set_stream(h, stream), "tclbm_set_stream")


def tclbm_set_tile(h, tx, ty):
    _check(_lib.tclbm_set_tile(h, int(tx), int(ty)), "tclbm_set_tile")


def tclbm_set_kernel(h, kind):
    _check(_lib.tclbm_set_kernel(h, int(kind)), "tclbm_set_kernel")


def tclbm_test_skip_row(h, row):
    _check(_lib.tclbm_test_skip_row(h, int(row)), "tclbm_test_skip_row")


def tclbm_test_rcp(x, y, n, stream=None):
    _check(_lib.tclbm_test_rcp(x, y, int(n), stream), "tclbm_test_rcp")


def tclbm_copy_rows(dst, dst_row, src, src_row, rows):
    _check(_lib.tclbm_copy_rows(dst, dst_row, src, src_row, rows), "tclbm_copy_rows")


def tclbm_describe(h) -> str:
    return _lib.tclbm_describe(h).decode()


def tclbm_destroy(h):
    _check(_lib.tclbm_destroy(h), "tclbm_destroy")


def tclbm_batch_create(handles, stream=None):
    arr = (_vp * len(handles))(*[h.value if isinstance(h, _vp) else h for h in handles])
    b = _vp()
    _check(_lib.tclbm_batch_create(arr, len(handles), stream, ctypes.byref(b)), "tclbm_batch_create")
    return b


def tclbm_batch_set_lattices(b, handles):
    arr = (_vp * max(1, len(handles)))(*[h.value if isinstance(h, _vp) else h for h in handles])
    _check(_lib.tclbm_batch_set_lattices(b, arr, len(handles)), "tclbm_batch_set_lattices")


def tclbm_batch_size(b) -> int:
    return int(_lib.tclbm_batch_size(b))


def tclbm_batch_step(b, n):
    _check(_lib.tclbm_batch_step(b, int(n)), "tclbm_batch_step")


def tclbm_batch_set_tile(b, tx, rows, persistent):
    _check(_lib.tclbm_batch_set_tile(b, int(tx), int(rows), int(persistent)), "tclbm_batch_set_tile")


def tclbm_batch_set_tma(b, tx, rows):
    _check(_lib.tclbm_batch_set_tma(b, int(tx), int(rows)), "tclbm_batch_set_tma")


def tclbm_batch_tma_shape(b):
    tx, rows = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.tclbm_batch_tma_shape(b, ctypes.byref(tx), ctypes.byref(rows)), "tclbm_batch_tma_shape")
    return tx.value, rows.value


def tclbm_batch_autotune(b, trial_steps):
    tx, rows, pers = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    us = ctypes.c_float()
    _check(_lib.tclbm_batch_autotune(b, int(trial_steps), ctypes.byref(tx), ctypes.byref(rows), ctypes.byref(pers),
                                     ctypes.byref(us)), "tclbm_batch_autotune")
    return tx.value, rows.value, pers.value, us.value


def tclbm_batch_describe(b) -> str:
    return _lib.tclbm_batch_describe(b).decode()


def tclbm_batch_steps_done(b) -> int:
    return int(_lib.tclbm_batch_steps_done(b))


def tclbm_batch_destroy(b):
    _check(_lib.tclbm_batch_destroy(b), "tclbm_batch_destroy")


# ------------------------------------------------------------------ case dict -> params


def params_from_case(case: dict) -> tclbm_params:
    p = tclbm_params()
    p.nx, p.ny = case["nx"], case["ny"]
    p.thermal = int(bool(case["thermal"]))
    p.correction = int(bool(case["correction"]))
    p.visc_law = VISC[case["visc_law"]]
    p.visc = case["visc"]
    p.w2, p.w3, p.w4 = case["w2"], case["w3"], case["w4"]
    p.Pr, p.gamma, p.R, p.T0 = case["Pr"], case["gamma"], case["R"], case["T0"]
    if case.get("w_equal"):
        # BGK limit with w1 fixed by the viscosity at T0 (Section V.A)
        if case["visc_law"] != "nu":
            raise ValueError("w_equal needs visc_law 'nu'")
        p.visc_law = VISC["w1"]
        p.visc = 1.0 / (case["visc"] / (case["R"] * case["T0"]) + 0.5)
        p.bgk = 1
    fk = case["force"]
    p.force_kind = FORCE[fk["kind"]]
    p.ax, p.ay, p.famp = fk.get("ax", 0.0), fk.get("ay", 0.0), fk.get("amp", 0.0)
    for i, s in enumerate(SIDES):
        w = case["walls"][s]
        p.wall[i].kind = WALL[w["kind"]]
        p.wall[i].therm = THERM[w.get("therm", "fixed")]
        p.wall[i].rho, p.wall[i].ux, p.wall[i].uy, p.wall[i].T = w["rho"], w["ux"], w["uy"], w["T"]
    p.storage = STORAGE[case.get("storage", "fp32")]
    p.T_ref = case.get("T_ref", case["T0"])
    p.rounding = ROUNDING[case.get("rounding", "nearest")]
    p.work = int(bool(case.get("work")))
    if case.get("adiabatic", "zero_gradient") != "zero_gradient":
        raise ValueError("the CUDA path's adiabatic walls are zero-gradient (T_w = T_f) only")
    return p


# ------------------------------------------------------------------ torch memory hooks


class _TorchMemory:
    """Device memory from torch's caching allocator (kept alive with the handle)."""

    def __init__(self, device):
        import torch

        self.torch = torch
        self.device = device

        def _alloc(nbytes, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0))
            except Exception:
                return None

        def _free(ptr, nbytes, stream, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


class Lattice:
    """One lattice resident on the current CUDA device (a tclbm_lattice handle)."""

    def __init__(self, case: dict, fields: dict | None = None, stream=None, memory: str = "torch"):
        import torch

        self.case = case
        self.params = params_from_case(case)
        self.nx, self.ny = case["nx"], case["ny"]
        self.thermal = bool(case["thermal"])
        self.device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self._mem = _TorchMemory(self.device) if memory == "torch" else None
        self.handle = tclbm_create(self.params, self._mem.alloc if self._mem else None,
                                   self._mem.free if self._mem else None, None, ctypes.c_void_p(stream))
        if fields is not None:
            self.init_fields(fields)

    # -- state
    def init_fields(self, fields: dict):
        arrs = []
        on_dev = not isinstance(fields["rho"], np.ndarray)
        for k in ("rho", "ux", "uy", "T"):
            a = fields[k]
            if on_dev:
                a = a.contiguous().double()
            else:
                a = np.ascontiguousarray(a, dtype=np.float64)
            arrs.append(a)
        self._keep = arrs
        tclbm_init_fields(self.handle, *[_ptr(a) for a in arrs], on_dev)

    def step(self, n: int = 1):
        tclbm_step(self.handle, n)

    def moments(self):
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        tclbm_moments(self.handle, *[_ptr(o) for o in out], 0)
        return dict(zip(("rho", "ux", "uy", "T"), out))

    def moments_device(self, out: dict):
        """Write rho, ux, uy, T into caller-owned float64 CUDA tensors [ny][nx]."""
        tclbm_moments(self.handle, *[_ptr(out.get(k)) for k in ("rho", "ux", "uy", "T")], 1)

    def diagnostics(self) -> np.ndarray:
        out = np.zeros(NDIAG)
        tclbm_diagnostics(self.handle, out.ctypes.data_as(_dp))
        return out

    def snapshot_velocity(self):
        tclbm_snapshot_velocity(self.handle)

    def populations(self):
        f = np.zeros((9, self.ny, self.nx))
        h = np.zeros((9, self.ny, self.nx)) if self.thermal else None
        tclbm_get_populations(self.handle, _ptr(f), _ptr(h), 0)
        return f, h

    def set_populations(self, f, h=None):
        f = np.ascontiguousarray(f, dtype=np.float64)
        h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
        tclbm_set_populations(self.handle, _ptr(f), _ptr(h), 0)

    @property
    def steps_done(self) -> int:
        return tclbm_steps_done(self.handle)

    def set_tile(self, tx=0, ty=0):
        tclbm_set_tile(self.handle, tx, ty)

    def set_kernel(self, kind: int):
        """0: TMA-staged rows; 1: direct loads, row strips; 2: direct loads, 2-D tiles
        (one node per thread).  The library picks by lattice size."""
        tclbm_set_kernel(self.handle, kind)

    def set_stream(self, stream):
        self.stream = stream
        tclbm_set_stream(self.handle, ctypes.c_void_p(stream))

    def describe(self) -> str:
        return tclbm_describe(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            tclbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Lattices advanced together by one batched launch per time step (a tclbm_batch)."""

    def __init__(self, lattices, stream=None):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.lattices = list(lattices)  # keeps the handles alive
        self.stream = stream
        # the batch allocates through the first lattice's allocator hooks: keep them alive
        self._mem = self.lattices[0]._mem if self.lattices else None
        self.handle = tclbm_batch_create([l.handle for l in self.lattices], ctypes.c_void_p(stream))

    def set_lattices(self, lattices):
        lattices = list(lattices)
        tclbm_batch_set_lattices(self.handle, [l.handle for l in lattices])
        self.lattices = lattices

    def __len__(self):
        return tclbm_batch_size(self.handle)

    def step(self, n: int = 1):
        tclbm_batch_step(self.handle, n)

    def set_tile(self, tx: int, rows: int, persistent: bool = True):
        tclbm_batch_set_tile(self.handle, tx, rows, 1 if persistent else 0)

    def set_tma(self, tx: int, rows: int = 16):
        """TMA-fed strips (tx 64 or 128; 0 = off) for the thermal lattices with the
        correction term at least tx wide; the others keep the direct-load strips."""
        tclbm_batch_set_tma(self.handle, tx, rows)

    def tma_shape(self):
        return tclbm_batch_tma_shape(self.handle)

    def autotune(self, trial_steps: int = 8):
        """(tx, rows, persistent, us_per_step) of the fastest direct-load work-list shape,
        now selected together with the fastest TMA-fed shape (tma_shape(); tx 0 if the
        direct-load strips alone were faster)."""
        tx, rows, pers, us = tclbm_batch_autotune(self.handle, trial_steps)
        return tx, rows, bool(pers), us

    @property
    def steps_done(self) -> int:
        return tclbm_batch_steps_done(self.handle)

    def describe(self) -> str:
        return tclbm_batch_describe(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            tclbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
