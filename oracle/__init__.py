"""FP64 CPU oracle of the thermal cascaded LBM (Fei & Luo, arXiv:1610.07114).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
reference legs of bench.py may import this package.  It shares no code with the
CUDA path: it loads its own C library (tclbm_oracle.c, plain loops in the paper's
order) and defines its own parameter struct.  Case dicts come from the shared
seeded-input module, which holds no method arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tclbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

WALL = {"periodic": 0, "zouhe": 1, "nee": 2, "equilibrium": 3}
THERM = {"fixed": 0, "adiabatic": 1}
VISC = {"nu": 0, "mu": 1, "mu_T": 2, "w1": 3}
FORCE = {"none": 0, "accel": 1, "taylor_green": 2}
SIDES = ("x-", "x+", "y-", "y+")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no contraction, OpenMP for the node loops)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        # plain IEEE operations (no fused multiply-add), so x86 and Arm hosts agree
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-o", _LIB, _SRC,
               "-lm"]
        subprocess.check_call(cmd)
    return _LIB


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("thermal", ctypes.c_int32), ("correction", ctypes.c_int32),
        ("visc_law", ctypes.c_int32), ("visc", ctypes.c_double),
        ("w2", ctypes.c_double), ("w3", ctypes.c_double), ("w4", ctypes.c_double),
        ("Pr", ctypes.c_double), ("gamma", ctypes.c_double), ("R", ctypes.c_double), ("T0", ctypes.c_double),
        ("force_kind", ctypes.c_int32), ("ax", ctypes.c_double), ("ay", ctypes.c_double), ("famp", ctypes.c_double),
        ("wall_kind", ctypes.c_int32 * 4), ("wall_therm", ctypes.c_int32 * 4),
        ("wall_rho", ctypes.c_double * 4), ("wall_ux", ctypes.c_double * 4),
        ("wall_uy", ctypes.c_double * 4), ("wall_T", ctypes.c_double * 4),
        ("work", ctypes.c_int32),
        ("adiabatic_flux", ctypes.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            pp = ctypes.POINTER(OracleParams)
            L.oracle_check.argtypes = [pp]
            L.oracle_init.argtypes = [pp, dp, dp, dp, dp, dp, dp]
            L.oracle_step.argtypes = [pp, dp, dp, ctypes.c_int]
            L.oracle_update_nodes.argtypes = [pp, dp, dp, ctypes.c_int, ip, ip, dp, dp]
            L.oracle_moments.argtypes = [pp, dp, dp, dp, dp, dp, dp]
            L.oracle_moments.restype = None
            L.oracle_collide_node.argtypes = [pp, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, dp, dp, dp, dp, dp, dp]
            L.oracle_collide_node.restype = None
            L.oracle_wall_node.argtypes = [pp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            L.oracle_wall_node.restype = None
            L.oracle_pop_from_moments.argtypes = [ctypes.c_double, dp, dp]
            L.oracle_pop_from_moments.restype = None
            L.oracle_feq.argtypes = [ctypes.c_double] * 4 + [dp]
            L.oracle_feq.restype = None
            L.oracle_heq.argtypes = [ctypes.c_double] * 5 + [dp]
            L.oracle_heq.restype = None
            L.oracle_source.argtypes = [ctypes.c_double] * 5 + [dp]
            L.oracle_source.restype = None
            L.oracle_correction.argtypes = [ctypes.c_double] * 5 + [dp]
            L.oracle_correction.restype = None
            L.oracle_velocities.argtypes = [ip, ip]
            L.oracle_velocities.restype = None
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            L.oracle_set_threads.restype = None
            L.oracle_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def params(case: dict) -> OracleParams:
    """The oracle's own parameter struct for a case dict."""
    p = OracleParams()
    p.nx, p.ny = case["nx"], case["ny"]
    p.thermal = 1 if case["thermal"] else 0
    p.correction = 1 if case["correction"] else 0
    p.visc_law = VISC[case["visc_law"]]
    p.visc = case["visc"]
    p.w2, p.w3, p.w4 = case["w2"], case["w3"], case["w4"]
    p.Pr, p.gamma, p.R, p.T0 = case["Pr"], case["gamma"], case["R"], case["T0"]
    fk = case["force"]
    p.force_kind = FORCE[fk["kind"]]
    p.ax, p.ay, p.famp = fk.get("ax", 0.0), fk.get("ay", 0.0), fk.get("amp", 0.0)
    for i, s in enumerate(SIDES):
        w = case["walls"][s]
        p.wall_kind[i] = WALL[w["kind"]]
        p.wall_therm[i] = THERM[w.get("therm", "fixed")]
        p.wall_rho[i], p.wall_ux[i], p.wall_uy[i], p.wall_T[i] = w["rho"], w["ux"], w["uy"], w["T"]
    p.work = 1 if case.get("work") else 0
    # adiabatic walls: "zero_gradient" (T_w = T_f, both paths) or "zero_flux" (oracle-only study)
    adiabatic = case.get("adiabatic", "zero_gradient")
    if adiabatic not in ("zero_gradient", "zero_flux"):
        raise ValueError(f"adiabatic must be 'zero_gradient' or 'zero_flux', not {adiabatic!r}")
    p.adiabatic_flux = 1 if adiabatic == "zero_flux" else 0
    if case.get("w_equal"):
        # BGK limit of Section V.A: w2 = w3 = w4 = w1 with w1 fixed from the viscosity.
        if case["visc_law"] != "nu":
            raise ValueError("w_equal needs visc_law 'nu'")
        w1 = 1.0 / (case["visc"] / (case["R"] * case["T0"]) + 0.5)
        p.visc_law = VISC["w1"]
        p.visc = w1
        p.w2 = p.w3 = p.w4 = w1
    return p


class Oracle:
    """A lattice held by the oracle: populations f[9][ny][nx], h[9][ny][nx] in FP64."""

    def __init__(self, case: dict, fields: dict | None = None, threads: int = 1):
        self.case = case
        self.p = params(case)
        rc = lib().oracle_check(ctypes.byref(self.p))
        if rc:
            raise ValueError(f"oracle rejects case {case.get('name')}: {rc}")
        self.threads = threads
        nx, ny = case["nx"], case["ny"]
        self.f = np.zeros((9, ny, nx))
        self.h = np.zeros((9, ny, nx))
        if fields is not None:
            self.init(fields)

    def init(self, fields):
        arrs = [np.ascontiguousarray(fields[k], dtype=np.float64) for k in ("rho", "ux", "uy", "T")]
        rc = lib().oracle_init(ctypes.byref(self.p), *[_dp(a) for a in arrs], _dp(self.f), _dp(self.h))
        if rc:
            raise RuntimeError("oracle_init failed")

    def step(self, n: int = 1):
        lib().oracle_set_threads(self.threads)
        rc = lib().oracle_step(ctypes.byref(self.p), _dp(self.f), _dp(self.h), int(n))
        if rc:
            raise RuntimeError(f"oracle_step failed: {rc}")

    def moments(self):
        ny, nx = self.case["ny"], self.case["nx"]
        out = [np.zeros((ny, nx)) for _ in range(4)]
        lib().oracle_moments(ctypes.byref(self.p), _dp(self.f), _dp(self.h), *[_dp(o) for o in out])
        return dict(zip(("rho", "ux", "uy", "T"), out))

    def set_populations(self, f, h=None):
        self.f[...] = f
        if h is not None:
            self.h[...] = h

    def update_nodes(self, xs, ys, f=None, h=None):
        """Populations at t+1 of the listed nodes, from state (f, h) at t (default: own state)."""
        f = self.f if f is None else np.ascontiguousarray(f, dtype=np.float64)
        h = self.h if h is None else np.ascontiguousarray(h, dtype=np.float64)
        xs = np.ascontiguousarray(xs, dtype=np.int32)
        ys = np.ascontiguousarray(ys, dtype=np.int32)
        n = len(xs)
        of = np.zeros((n, 9))
        oh = np.zeros((n, 9))
        lib().oracle_set_threads(self.threads)
        rc = lib().oracle_update_nodes(ctypes.byref(self.p), _dp(f), _dp(h), n, _ip(xs), _ip(ys), _dp(of), _dp(oh))
        if rc:
            raise RuntimeError("oracle_update_nodes failed")
        return of, oh


# ------------------------------------------------------------------ single-node entry points


def velocities():
    ex = np.zeros(9, dtype=np.int32)
    ey = np.zeros(9, dtype=np.int32)
    lib().oracle_velocities(_ip(ex), _ip(ey))
    return ex, ey


def pop_from_moments(rho, M):
    M = np.ascontiguousarray(M, dtype=np.float64)
    out = np.zeros(9)
    lib().oracle_pop_from_moments(float(rho), _dp(M), _dp(out))
    return out


def feq(rho, ux, uy, RT):
    out = np.zeros(9)
    lib().oracle_feq(float(rho), float(ux), float(uy), float(RT), _dp(out))
    return out


def heq(rho, ux, uy, RT, b):
    out = np.zeros(9)
    lib().oracle_heq(float(rho), float(ux), float(uy), float(RT), float(b), _dp(out))
    return out


def source(rho, ux, uy, ax, ay):
    out = np.zeros(9)
    lib().oracle_source(float(rho), float(ux), float(uy), float(ax), float(ay), _dp(out))
    return out


def correction(rho, ux, uy, dx, dy):
    out = np.zeros(9)
    lib().oracle_correction(float(rho), float(ux), float(uy), float(dx), float(dy), _dp(out))
    return out


def collide_node(case, fb, hb, F=(0.0, 0.0), dx=0.0, dy=0.0):
    """One node's collision; returns dict of fstar, S, C, fout, hout and macro (rho, ux, uy, T, w1)."""
    p = params(case)
    fb = np.ascontiguousarray(fb, dtype=np.float64)
    hb = np.ascontiguousarray(hb if hb is not None else np.zeros(9), dtype=np.float64)
    outs = {k: np.zeros(9) for k in ("fstar", "S", "C", "fout", "hout")}
    mac = np.zeros(5)
    lib().oracle_collide_node(ctypes.byref(p), _dp(fb), _dp(hb), float(F[0]), float(F[1]), float(dx), float(dy),
                              *[_dp(outs[k]) for k in ("fstar", "S", "C", "fout", "hout")], _dp(mac))
    outs["macro"] = dict(zip(("rho", "ux", "uy", "T", "w1"), mac))
    return outs


def wall_node(case, side, x, y, fb, hb, ff, hf):
    p = params(case)
    fb = np.ascontiguousarray(fb, dtype=np.float64).copy()
    hb = np.ascontiguousarray(hb, dtype=np.float64).copy()
    ff = np.ascontiguousarray(ff, dtype=np.float64)
    hf = np.ascontiguousarray(hf, dtype=np.float64)
    lib().oracle_wall_node(ctypes.byref(p), SIDES.index(side), int(x), int(y), _dp(fb), _dp(hb), _dp(ff), _dp(hf))
    return fb, hb


def max_threads():
    return lib().oracle_max_threads()
