"""Reduced-precision population storage: error of every stored format against the
FP64 oracle and the closed forms.

Formats: FP32 (deviations from the rest state), FP16 and BF16 deviations with FP32
arithmetic, each 16-bit format with round-to-nearest or stochastic rounding.
Errors are relative L2 on the velocity and on the rho and T deviations (tests/parity.py:
each normalised by its deviation from the mean, floored at sqrt(N) times the case's own
scale of that variation).  Tolerances come from the storage precision: a stored
deviation carries a relative rounding error of 2^-11 (FP16) or 2^-8 (BF16) per step, a
few ulps of which the fields accumulate over a few hundred to a few thousand steps.
They are set at about twice the largest error measured for each format and rounding;
round-to-nearest 16-bit storage freezes slow growth (below), which is what its larger
temperature bounds hold.

Near a steady state the per-step change of a population falls below half an ulp.
Round-to-nearest then freezes it: on Rayleigh-Benard convection the slow instability
never develops (Nu stays at 1.00 against the oracle's 2.52).  Stochastic rounding
keeps the expected stored value unbiased, and FP16 with it reproduces the FP64
Nusselt number to 0.5 %.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1610_07114_gb300 import workloads as W
from tests import riemann
from tests.parity import field_errors

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
VARIANTS = [("fp32", "nearest"), ("fp16", "nearest"), ("fp16", "stochastic"), ("bf16", "nearest"),
            ("bf16", "stochastic")]
# relative L2 tolerances on (rho deviation, u, T deviation) per stored format and rounding
TOL = {("fp32", "nearest"): (1e-5, 1e-5, 1e-5),
       ("fp16", "nearest"): (1e-2, 3e-3, 4e-2), ("fp16", "stochastic"): (1e-2, 1e-3, 6e-3),
       ("bf16", "nearest"): (5e-2, 3e-2, 8e-2), ("bf16", "stochastic"): (5e-2, 1e-2, 4e-2)}


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1610_07114_gb300 import build

    build.build()
    from paper_1610_07114_gb300 import tclbm

    return tclbm


def gpu_moments(T, case, fields, steps):
    lat = T.Lattice(case, fields)
    lat.step(steps)
    m = lat.moments()
    lat.close()
    return m


CASES = [
    ("rb_256x128", lambda: W.rayleigh_benard(256, 128), 2000),
    ("shock_4096x4", lambda: W.shock_tube(4096, 4), 2000),
    ("tg_64", lambda: W.taylor_green(64, F0=1e-5, nu=0.02), 3000),
    ("rand_70x37", lambda: W.random_periodic(70, 37, seed=1), 300),
]
_oracle_cache = {}


def _oracle(name, make, steps):
    if name not in _oracle_cache:
        case, fields = make()
        o = oracle.Oracle(case, fields, threads=os.cpu_count())
        o.step(steps)
        _oracle_cache[name] = o.moments()
    return _oracle_cache[name]


@pytest.mark.parametrize("storage,rounding", VARIANTS)
@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
def test_stored_format_against_fp64_oracle(T, name, make, steps, storage, rounding):
    case, fields = make()
    ref = _oracle(name, make, steps)
    case = dict(case, storage=storage, rounding=rounding)
    e = field_errors(gpu_moments(T, case, fields, steps), ref, case)
    print(name, storage, rounding, "rho %.2e u %.2e T %.2e" % (e["rho"], e["u"], e["T"]))
    tol = TOL[(storage, rounding)]
    assert e["rho"] <= tol[0] and e["u"] <= tol[1] and e["T"] <= tol[2], e


@pytest.mark.parametrize("storage,rounding", VARIANTS)
def test_taylor_green_closed_form_per_format(T, storage, rounding):
    # Section V.A steady state from the closed-form start: E2 (paper, Table 1: 1.55e-3 at 64^2)
    n, nu, u0 = 64, 0.02, 0.025
    k = 2 * math.pi / n
    case, _ = W.taylor_green(n, F0=2 * nu * k * k * u0, nu=nu)
    ua, va = W.taylor_green_fields(n, u0)
    fields = W.uniform_fields(n, n)
    fields["ux"], fields["uy"] = ua, va
    m = gpu_moments(T, dict(case, storage=storage, rounding=rounding), fields, 14000)
    e2 = math.sqrt(np.sum((m["ux"] - ua) ** 2 + (m["uy"] - va) ** 2) / np.sum(ua ** 2 + va ** 2))
    print(storage, rounding, "E2 %.3e" % e2)
    # with stochastic rounding the field is one draw of the rounding noise (BF16 SR measured
    # 7.2e-3 and 2.1e-2 on two builds whose FP32 arithmetic differed in the last bits)
    bound = {"fp32": 1.8e-3, "fp16": 3e-3, "bf16": 1.5e-2 if rounding == "nearest" else 3e-2}[storage]
    assert e2 < bound


@pytest.mark.parametrize("storage,rounding", VARIANTS)
def test_shock_tube_plateau_per_format(T, storage, rounding):
    # Section V.C against the exact Riemann solution: velocity between the waves
    nx, t = 1200, 300
    case, fields = W.shock_tube(nx, 1)
    R = case["R"]
    _, us = riemann.star_state(1.05, 0.0, 1.05 * R, 1.0, 0.0, R, 1.4)
    m = gpu_moments(T, dict(case, storage=storage, rounding=rounding), fields, t)
    xt = (np.arange(nx) - (nx / 2 - 0.5)) / t
    cs = math.sqrt(1.4 * R)
    sel = (np.abs(xt) > 0.2 * cs) & (np.abs(xt) < 0.8 * cs)
    u_plateau = float(np.mean(m["ux"][0][sel]))
    # Stochastic rounding makes the plateau one draw of the rounding noise; any change in
    # the FP32 arithmetic draws another.  Its u field is 4.5e-4 (relative L2) off the FP64
    # oracle, and the 174 plateau nodes share that noise over the acoustic scale, so
    # their mean is held to that level, not to the deterministic round-to-nearest bound.
    rel = {"fp32": 2e-5, "fp16": 2e-4 if rounding == "nearest" else 5e-4, "bf16": 3e-3}[storage]
    assert u_plateau == pytest.approx(us, rel=rel)


def _golden_nusselt():
    rows = {}
    with open(os.path.join(HERE, "golden", "rb_128x64_nusselt.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                s, nu = line.split()
                rows[int(s)] = float(nu)
    return rows


def _rb_nusselt(T, storage, rounding, steps):
    case, fields = W.rayleigh_benard(128, 64, Ra=1e4, seed=1, amp=1e-2)
    m = gpu_moments(T, dict(case, storage=storage, rounding=rounding), fields, steps)
    H = case["ny"] - 1
    kappa = case["visc"] / case["Pr"]
    return 1.0 + np.mean(m["uy"] * (m["T"] - case["T0"])) * H / (kappa * (case["T_bot"] - case["T_top"]))


@pytest.mark.parametrize("storage,rounding,bound", [("fp32", "nearest", 1e-4), ("fp16", "stochastic", 5e-3)])
def test_nusselt_number_against_fp64(T, storage, rounding, bound):
    # Section V.D: the Nusselt number of the reduced-storage run within 0.5 % of FP64
    gold = _golden_nusselt()
    for steps in (60000, 80000):
        nu = _rb_nusselt(T, storage, rounding, steps)
        print(storage, rounding, steps, "Nu %.5f (FP64 %.5f)" % (nu, gold[steps]))
        assert abs(nu / gold[steps] - 1.0) < bound


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_round_to_nearest_16bit_storage_freezes_slow_growth(T, storage):
    # The measured failure mode that stochastic rounding removes: with round-to-nearest
    # 16-bit deviations the convective instability stagnates and Nu stays near 1.
    gold = _golden_nusselt()
    nu = _rb_nusselt(T, storage, "nearest", 60000)
    assert nu < 1.05 < gold[60000]


def _tg_to_steady_state(T, case, fields, residual, check, max_steps):
    """Steps until E_R (Section V.A: relative L2 change of u over `check` steps, from the
    device FP64 sums) falls below `residual` or `max_steps` is reached."""
    lat = T.Lattice(case, fields)
    done, er = 0, 1.0
    lat.snapshot_velocity()
    while done < max_steps:
        lat.step(check)
        done += check
        d = lat.diagnostics()
        er = float(np.sqrt(d[6] / d[7]))
        if er < residual:
            break
        lat.snapshot_velocity()
    m = lat.moments()
    lat.close()
    return m, done, er


def test_taylor_green_512_per_format(T):
    # Taylor-Green on 512^2 at the Reynolds number of the Section V.A case (nu = 0.02,
    # u0 = 0.026 * 64 / 512 = 3.25e-3), started from the closed form and run for 10^6 steps
    # (3 e-foldings of the slowest mode, 1/(nu k^2) = 332 000 steps): E2 against the closed
    # form and the residual E_R (1000-step interval) of every stored format.  Measured:
    # FP32 2.26e-3 (E_R 2.2e-7), FP16 nearest 9.7e-3, FP16 stochastic 3.2e-3, BF16 nearest
    # 0.35, BF16 stochastic 1.05e-2.  FP32 settles but not to the closed form's second-order
    # error (2.4e-5): its roundings, partly systematic, are integrated by the slow mode into
    # an absolute velocity error of ~7e-6, and its residual floor is 2e-7, above 1e-8.
    # Round-to-nearest BF16 cannot follow the slow relaxation at all.  (With u0 held at
    # 0.026 instead, the 512^2 flow runs at 8 times that Reynolds number and is unstable:
    # a 1e-3 perturbation grows to O(1) within 500 000 steps.)
    n, nu, steps = 512, 0.02, 1_000_000
    k = 2 * math.pi / n
    u0 = 0.026 * 64.0 / n
    case, _ = W.taylor_green(n, F0=2 * nu * k * k * u0, nu=nu)
    ua, va = W.taylor_green_fields(n, u0)
    fields = W.uniform_fields(n, n)
    fields["ux"], fields["uy"] = ua, va

    def e2(m):
        return math.sqrt(np.sum((m["ux"] - ua) ** 2 + (m["uy"] - va) ** 2) / np.sum(ua ** 2 + va ** 2))

    bound = {("fp32", "nearest"): (5e-3, 1e-6), ("fp16", "nearest"): (2e-2, 3e-3),
             ("fp16", "stochastic"): (7e-3, 3e-3), ("bf16", "nearest"): (0.7, 0.1), ("bf16", "stochastic"): (2.5e-2, 3e-2)}
    for (storage, rounding), (b_e2, b_er) in bound.items():
        lat = T.Lattice(dict(case, storage=storage, rounding=rounding), fields)
        lat.step(steps - 1000)
        lat.snapshot_velocity()
        lat.step(1000)
        d = lat.diagnostics()
        m = lat.moments()
        lat.close()
        er = math.sqrt(d[6] / d[7])
        print("TG-512 %s %s after %d steps: E2 %.3e, E_R %.2e" % (storage, rounding, steps, e2(m), er))
        assert e2(m) < b_e2 and er < b_er


def _golden_nusselt_256():
    rows = {}
    with open(os.path.join(HERE, "golden", "rb_256x128_nusselt.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                s, nu = line.split()
                rows[int(s)] = float(nu)
    return rows


@pytest.mark.parametrize("storage,rounding,bound", [("fp32", "nearest", 1e-3)])
def test_rayleigh_benard_256x128_nusselt_history(T, storage, rounding, bound):
    # The bench workload (Section V.D set-up: 256 x 128, Ra = 1e4, perturbation 1e-4) over
    # 300 000 steps, the Nusselt number from the device FP64 sums every 25 000 steps
    # against the FP64 oracle's history.  Convection sets in
    # between 75 000 and 125 000 steps, where the Nusselt number rises from 1 to its
    # overshoot: there the onset time, not the arithmetic, sets the difference, so the
    # comparison is on the developed flow (from 150 000 steps) and, before the onset, on
    # the conduction state (Nu = 1 within 1e-3).  16-bit storage with stochastic rounding
    # is not compared here: from this 1e-4 seed its own rounding noise sets off the
    # convection (Nu 1.72 at 75 000 steps against 1.003) and the flow develops along
    # another path (Nu 2.24 at 150 000, 2.14 at 175 000) to the same steady state, which
    # test_rayleigh_benard_256x128_steady_nusselt_16bit compares at 300 000 steps.
    gold = _golden_nusselt_256()
    case, fields = W.rayleigh_benard(256, 128, Ra=1e4, seed=1)
    case = dict(case, storage=storage, rounding=rounding)
    lat = T.Lattice(case, fields)
    n = case["nx"] * case["ny"]
    H, kappa, dT = case["ny"] - 1, case["visc"] / case["Pr"], case["T_bot"] - case["T_top"]
    done = 0
    for steps in sorted(gold):
        lat.step(steps - done)
        done = steps
        d = lat.diagnostics()
        nu = 1.0 + d[5] / n * H / (kappa * dT)
        print(storage, rounding, steps, "Nu %.5f (FP64 %.5f)" % (nu, gold[steps]))
        if steps <= 50000:
            assert abs(nu - 1.0) < 1e-3 and abs(gold[steps] - 1.0) < 1e-3
        elif steps >= 150000:
            assert abs(nu / gold[steps] - 1.0) < bound
    lat.close()


@pytest.mark.parametrize("storage,bound", [("fp16", 5e-3), ("bf16", 1e-2)])
def test_rayleigh_benard_256x128_steady_nusselt_16bit(T, storage, bound):
    # 16-bit deviation storage with stochastic rounding on the bench workload: its own
    # rounding noise starts the convection early and through other roll patterns, but
    # after 300 000 steps the flow has settled into the FP64 oracle's steady state.  FP16
    # meets the 0.5 % reduced-storage target (measured 2.5163 against the oracle's
    # 2.5143, +0.08 %).  BF16 keeps 8 significand bits against FP16's 11, so its rounding
    # noise per stored deviation is 8 times larger, and its steady Nusselt number sits
    # 0.52 % low (2.5012): it misses the 0.5 % target, and is held to 1 % here.
    gold = _golden_nusselt_256()
    last = max(gold)
    case, fields = W.rayleigh_benard(256, 128, Ra=1e4, seed=1)
    case = dict(case, storage=storage, rounding="stochastic")
    lat = T.Lattice(case, fields)
    lat.step(last)
    d = lat.diagnostics()
    lat.close()
    n = case["nx"] * case["ny"]
    H, kappa, dT = case["ny"] - 1, case["visc"] / case["Pr"], case["T_bot"] - case["T_top"]
    nu = 1.0 + d[5] / n * H / (kappa * dT)
    print(storage, last, "Nu %.5f (FP64 %.5f)" % (nu, gold[last]))
    assert abs(nu / gold[last] - 1.0) < bound
