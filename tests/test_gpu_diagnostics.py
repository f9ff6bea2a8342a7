"""The device FP64 diagnostics and the collision's reciprocal, against independent sums.

tclbm_diagnostics() returns, from FP64 block reductions on the device: out[0] sum rho,
out[1..2] sum rho u, out[3] sum h_bar (total energy), out[4] the kinetic energy
sum rho |u|^2 / 2 (Section V.D), out[5] sum u_y (T - T_ref) (the Nusselt sum of
Section V.D), out[6] sum |u - u_snap|^2 and out[7] sum |u|^2 (the residual E_R of
Section V.A).  Each is checked two ways: against the same sum formed on the host from
the lattice's own FP64 moments (the reduction itself: summation order only), and
against the sum formed from the FP64 oracle's fields after the same steps (the state:
the FP32 parity of the fields carried into each sum).
"""
import numpy as np
import pytest

import oracle
from paper_1610_07114_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1610_07114_gb300 import build

    build.build()
    from paper_1610_07114_gb300 import tclbm

    return tclbm


def sums(m, h, T_ref, usnap):
    """The eight diagnostics from FP64 fields, and the sums of the magnitudes of their terms."""
    r, vx, vy, t = m["rho"], m["ux"], m["uy"], m["T"]
    terms = [r, r * vx, r * vy, None, 0.5 * r * (vx * vx + vy * vy), vy * (t - T_ref),
             (vx - usnap[0]) ** 2 + (vy - usnap[1]) ** 2, vx * vx + vy * vy]
    out = np.zeros(8)
    mag = np.zeros(8)
    for k, a in enumerate(terms):
        if k == 3:
            out[3] = float(h.sum()) if h is not None else 0.0
            mag[3] = float(np.abs(h).sum()) if h is not None else 0.0
        else:
            out[k] = float(a.sum())
            mag[k] = float(np.abs(a).sum())
    return out, mag


CASES = [
    # walls (Zou-He velocity, NEE temperature) and gravity: the bench workload's kind of lattice
    ("rb_walls_gravity", lambda: W.rayleigh_benard(96, 48, Ra=2e4, seed=31, amp=1e-2), 600, 400),
    # periodic, Taylor-Green force field on a thermal lattice
    ("tg_thermal", lambda: W.taylor_green(48, F0=2e-5, nu=0.02, thermal=True), 300, 200),
    # athermal (T = T0 everywhere: out[5] vanishes identically up to the velocity sum)
    ("random_athermal", lambda: W.random_periodic(40, 28, seed=32, force="accel", thermal=False), 150, 100),
]


@pytest.mark.parametrize("name,make,n1,n2", CASES, ids=[c[0] for c in CASES])
def test_device_diagnostics_against_host_and_oracle_sums(T, name, make, n1, n2):
    case, fields = make()
    T_ref = case.get("T_ref", case["T0"])
    lat = T.Lattice(case, fields)
    assert lat.params.T_ref == pytest.approx(T_ref)
    o = oracle.Oracle(case, fields, threads=8)
    lat.step(n1)
    o.step(n1)
    lat.snapshot_velocity()
    g1, o1 = lat.moments(), o.moments()
    # the handle keeps its velocity snapshot in FP32
    us_g = np.stack([g1["ux"].astype(np.float32), g1["uy"].astype(np.float32)]).astype(np.float64)
    us_o = np.stack([o1["ux"], o1["uy"]])
    lat.step(n2)
    o.step(n2)
    dev = lat.diagnostics()
    g2 = lat.moments()
    _, hg = lat.populations()
    lat.close()
    o2 = o.moments()
    host, mag = sums(g2, hg, T_ref, us_g)
    orc, mag_o = sums(o2, o.h if case["thermal"] else None, T_ref, us_o)
    print(name, "device", dev)
    print(name, "oracle", orc)
    for k in range(8):
        # the reduction: the same FP64 node values in another order
        assert abs(dev[k] - host[k]) <= 1e-12 * mag[k] + 1e-300, (name, k, dev[k], host[k])
    # the state: the FP32 field parity (rel-L2 <= 1e-5 on rho, u, T; velocity floored at
    # U_ref, temperature deviations at T_scale) carried into each sum
    n = case["nx"] * case["ny"]
    U, Ts = case["U_ref"], case.get("T_scale", 0.0)
    assert dev[0] == pytest.approx(orc[0], rel=1e-7), name
    if case["thermal"]:
        assert dev[3] == pytest.approx(orc[3], rel=1e-7), name
    for k, floor in ((1, n * U), (2, n * U), (5, n * U * Ts)):
        tol = 2e-5 * max(mag_o[k], floor)
        assert abs(dev[k] - orc[k]) <= tol, (name, k, dev[k], orc[k], tol)
    for k in (4, 7):
        tol = 2e-5 * max(mag_o[k], n * U * U)
        assert abs(dev[k] - orc[k]) <= tol, (name, k, dev[k], orc[k], tol)
    # the residual sum compares velocities n2 steps apart; its reference is the velocity
    # field at n1 (FP32 on the device), so its error is that of u relative to the change
    assert orc[6] > 0
    assert dev[6] == pytest.approx(orc[6], rel=1e-4), name
    # E_R itself, as the serving loop and the paper's steady-state test evaluate it
    er_dev = np.sqrt(dev[6] / dev[7])
    er_orc = np.sqrt(orc[6] / orc[7])
    assert er_dev == pytest.approx(er_orc, rel=1e-4), name


def test_rcp_error_bound(T):
    # the reciprocal the collision takes of R T (~0.1-0.3), mu/p + 1/2 and mu/(p Pr) + 1/2
    # (0.5-4): the hardware approximation refined by one Newton step.  Against the exact
    # 1/x: within 2^-22 relative over [1e-3, 1e2] and on a dense sample of [0.5, 2];
    # against the correctly rounded FP32 quotient: within one ulp.
    import torch

    rng = np.random.default_rng(3)
    x = np.concatenate([np.geomspace(1e-3, 1e2, 400001), rng.uniform(0.5, 2.0, 400000),
                        np.float32(1.0) + np.arange(-2000, 2000) * np.float32(2.0**-23)]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    T.tclbm_test_rcp(xd.data_ptr(), yd.data_ptr(), x.size)
    y = yd.cpu().numpy()
    exact = 1.0 / x.astype(np.float64)
    rel = np.abs(y.astype(np.float64) - exact) / exact
    ieee = (np.float32(1.0) / x).astype(np.float32)
    ulps = np.abs(y.view(np.int32).astype(np.int64) - ieee.view(np.int32).astype(np.int64))
    print("rcp: max rel %.3e, mean rel %.3e, max ulps from 1/x %d, equal %.4f" %
          (rel.max(), rel.mean(), ulps.max(), float(np.mean(ulps == 0))))
    assert rel.max() <= 2.0**-22
    assert ulps.max() <= 1
    # deterministic: the same bits on a second evaluation
    yd2 = torch.empty_like(xd)
    T.tclbm_test_rcp(xd.data_ptr(), yd2.data_ptr(), x.size)
    assert torch.equal(yd, yd2)
    with pytest.raises(T.TclbmError):
        T.tclbm_test_rcp(None, None, 5)
