"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance for FP32 population storage: relative L2 <= 1e-5 on the velocity vector
field, and on rho and T as deviations (tests/parity.py: each normalised by its
deviation from the mean, floored at sqrt(N) times the case's own scale of that
variation; the velocity norm is floored at sqrt(N) U_ref), after the stated step
counts, on the same seeded inputs.  One step from an identical state must agree
population by population to FP32 rounding of O(1) arithmetic (abs 2e-6).  Independent
tiles must give bit-identical states, since every node's arithmetic is the same
whatever the launch shape.
"""
import numpy as np
import pytest

import oracle
from paper_1610_07114_gb300 import workloads as W
from tests.parity import field_errors

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1610_07114_gb300 import build

    build.build()
    from paper_1610_07114_gb300 import tclbm

    return tclbm


def run_both(T, case, fields, steps, threads=8):
    lat = T.Lattice(case, fields)
    lat.step(steps)
    g = lat.moments()
    lat.close()
    o = oracle.Oracle(case, fields, threads=threads)
    o.step(steps)
    return g, o.moments()


def errors(T, case, fields, steps, threads=8):
    g, o = run_both(T, case, fields, steps, threads)
    return field_errors(g, o, case)


def _cases_small():
    out = []
    out.append(("rand_corr_accel_70x37", *W.random_periodic(70, 37, seed=1, force="accel")))
    out.append(("rand_thermal_tg_45x33", *W.random_periodic(45, 33, seed=2, force="taylor_green",
                                                             correction=False)))
    out.append(("rand_athermal_40x24", *W.random_periodic(40, 24, seed=3, force="accel", thermal=False)))
    out.append(("walls_y_nee", *W.with_walls(*W.random_periodic(53, 41, seed=4, force="accel"), axis="y",
                                             kind="nee")))
    out.append(("walls_y_zouhe", *W.with_walls(*W.random_periodic(53, 41, seed=5, force="accel"), axis="y",
                                               kind="zouhe")))
    out.append(("walls_x_equilibrium", *W.with_walls(*W.random_periodic(67, 9, seed=6, force="none"), axis="x",
                                                     kind="equilibrium")))
    out.append(("walls_x_nee", *W.with_walls(*W.random_periodic(67, 9, seed=7, force="accel"), axis="x",
                                             kind="nee")))
    out.append(("walls_x_zouhe", *W.with_walls(*W.random_periodic(35, 12, seed=8, force="taylor_green"), axis="x",
                                               kind="zouhe")))
    return out


SMALL = _cases_small()


@pytest.mark.parametrize("name,case,fields", SMALL, ids=[c[0] for c in SMALL])
def test_initial_state_matches_oracle(T, name, case, fields):
    lat = T.Lattice(case, fields)
    f, h = lat.populations()
    lat.close()
    o = oracle.Oracle(case, fields)
    np.testing.assert_allclose(f, o.f, rtol=0, atol=2.5e-7)
    if case["thermal"]:
        np.testing.assert_allclose(h, o.h, rtol=0, atol=2.5e-7)


@pytest.mark.parametrize("name,case,fields", SMALL, ids=[c[0] for c in SMALL])
def test_one_step_from_identical_state(T, name, case, fields):
    o = oracle.Oracle(case, fields)
    o.step(3)
    lat = T.Lattice(case, fields)
    lat.set_populations(o.f, o.h if case["thermal"] else None)
    f0, h0 = lat.populations()
    o.set_populations(f0, h0 if case["thermal"] else None)  # the oracle starts from the FP32-rounded state
    lat.step(1)
    f1, h1 = lat.populations()
    lat.close()
    o.step(1)
    np.testing.assert_allclose(f1, o.f, rtol=0, atol=2e-6)
    if case["thermal"]:
        np.testing.assert_allclose(h1, o.h, rtol=0, atol=2e-6)


@pytest.mark.parametrize("name,case,fields", SMALL, ids=[c[0] for c in SMALL])
def test_fields_after_many_steps(T, name, case, fields):
    e = errors(T, case, fields, 300)
    for k in ("rho", "u", "T"):
        assert e[k] <= REL_L2, (name, e)


# FP32 bounds per case (tests/parity.py): 1e-5, wider only for small-signal deviation
# fields (FP32 resolves rho and T to ~3e-8 absolute) and for the thermal Couette flow (a
# moving wall's O(U) populations rounded by 1-2 ulps per step and integrated by the slow
# shear mode); at 1000 steps, before that integration, its u is held to the common 1e-5.
from tests.parity import fp32_bounds  # noqa: E402


def test_thermal_couette_config(T):
    # thermal Couette 8 x 64, U = 0.05, nu = 0.05, Pr = 0.71, gamma = 1.4, 20 000 steps
    case, fields = W.couette(8, 64)
    b = fp32_bounds(case)
    assert b[1] == 5e-5
    e = errors(T, case, fields, 20000)
    print("couette", e)
    assert e["rho"] <= b[0] and e["u"] <= b[1] and e["T"] <= b[2], e
    e1 = errors(T, case, fields, 1000)
    print("couette 1000", e1)
    assert e1["u"] <= REL_L2, e1


def test_rayleigh_benard_config(T):
    # Rayleigh-Benard 256 x 128, Ra = 1e4: parity over 2 000 steps (chaotic growth limits longer parity)
    case, fields = W.rayleigh_benard(256, 128)
    e = errors(T, case, fields, 2000, threads=16)
    print("rb", e)
    for k in ("rho", "u", "T"):
        assert e[k] <= REL_L2, e


def test_shock_tube_config(T):
    case, fields = W.shock_tube(4096, 4)
    e = errors(T, case, fields, 2000, threads=16)
    print("shock", e)
    for k in ("rho", "u", "T"):
        assert e[k] <= REL_L2, e


def test_taylor_green_config(T):
    case, fields = W.taylor_green(64, F0=1e-5, nu=0.02)
    e = errors(T, case, fields, 3000)
    print("tg", e)
    for k in ("rho", "u"):
        assert e[k] <= REL_L2, e


CONFIGS_FULL = [
    ("rb_256x128_bench", lambda: W.rayleigh_benard(256, 128), "tclbm_step_tile"),
    ("taylor_green_512", lambda: W.taylor_green(512, F0=1.5625e-7, nu=0.02), "tclbm_step_plain"),
    ("couette_8x64", lambda: W.couette(8, 64), "tclbm_step"),
    ("shock_tube_4096x4", lambda: W.shock_tube(4096, 4), "tclbm_step"),
]


@pytest.mark.parametrize("name,make,kernel", CONFIGS_FULL, ids=[c[0] for c in CONFIGS_FULL])
def test_config_one_step_every_node(T, name, make, kernel):
    # each workload at its full size, in the kernel the library picks for it: one step
    # from a state both sides hold (the oracle's after 20 steps, rounded to FP32),
    # compared population by population at every node
    case, fields = make()
    o = oracle.Oracle(case, fields, threads=16)
    o.step(20)
    lat = T.Lattice(case, fields)
    assert lat.describe().startswith(kernel), lat.describe()
    lat.set_populations(o.f, o.h if case["thermal"] else None)
    f0, h0 = lat.populations()
    o.set_populations(f0, h0 if case["thermal"] else None)
    lat.step(1)
    f1, h1 = lat.populations()
    lat.close()
    o.step(1)
    np.testing.assert_allclose(f1, o.f, rtol=0, atol=2e-6)
    if case["thermal"]:
        np.testing.assert_allclose(h1, o.h, rtol=0, atol=2e-6)


@pytest.mark.parametrize("nx,ny,walls", [(1, 5, None), (2, 2, None), (3, 3, "y"), (5, 3, "x"), (33, 4, "y"),
                                         (129, 7, None), (31, 130, "y")])
def test_edge_sizes(T, nx, ny, walls):
    case, fields = W.random_periodic(nx, ny, seed=nx * 100 + ny, force="accel")
    if walls:
        case, fields = W.with_walls(case, fields, axis=walls, kind="nee")
    e = errors(T, case, fields, 40)
    for k in ("rho", "u", "T"):
        assert e[k] <= REL_L2, (nx, ny, e)


def test_launch_shapes_are_bit_identical(T):
    case, fields = W.with_walls(*W.random_periodic(150, 45, seed=9, force="accel"), axis="y", kind="zouhe")
    states = []
    for tx, ty in ((32, 4), (64, 7), (128, 16), (32, 45), (64, 5), (32, 1), (64, 2), (32, 3)):
        lat = T.Lattice(case, fields)
        lat.set_kernel(1)  # the marching kernel, whose row segments the tiles change
        lat.set_tile(tx, ty)
        lat.step(25)
        states.append(lat.populations())
        lat.close()
    for f, h in states[1:]:
        assert np.array_equal(f, states[0][0]) and np.array_equal(h, states[0][1])


def test_tma_rows_per_cta_are_bit_identical(T):
    # the TMA kernel's row segments change which CTA computes a node, not its
    # arithmetic: 16 rows on 2048 x 1024 is a grid of more than two waves, so its last
    # wave takes half-height segments (the first one absorbing the remainder); 7, 32 and
    # 48 rows are uniform segments
    case, fields = W.rayleigh_benard(2048, 1024, seed=5)
    states = []
    for ty in (16, 32, 7, 48):
        lat = T.Lattice(case, fields)
        lat.set_kernel(0)
        lat.set_tile(128, ty)
        assert ("last" in lat.describe()) == (ty == 16), lat.describe()
        lat.step(21)
        states.append(lat.populations())
        lat.close()
    for f, h in states[1:]:
        assert np.array_equal(f, states[0][0]) and np.array_equal(h, states[0][1])


@pytest.mark.parametrize("name,make,tile", [
    # walls in y, 16-row segments with the half-height last wave (more than two waves)
    ("rb_2048x1024_rows16", lambda: W.rayleigh_benard(2048, 1024, seed=5), (128, 16)),
    # a last strip of 104 columns, 32-row segments
    ("rb_1000x512_rows32", lambda: W.rayleigh_benard(1000, 512, seed=8), (128, 32)),
    # periodic in x and y: the neighbouring items of edge strips and segments wrap
    ("periodic_1024x1024_rows8", lambda: W.random_periodic(1024, 1024, seed=9, force="accel"), (64, 8)),
    # walls in x, periodic in y
    ("xwalls_768x1024_rows16", lambda: W.with_walls(*W.random_periodic(768, 1024, seed=10, force="accel"),
                                                    axis="x", kind="zouhe"), (128, 16)),
    # 16-bit storage with round-to-nearest
    ("rb_2048x1024_fp16_nearest", lambda: W.rayleigh_benard(2048, 1024, seed=5, storage="fp16"), (128, 32)),
], ids=["rb_2048x1024_rows16", "rb_1000x512_rows32", "periodic_1024x1024_rows8", "xwalls_768x1024_rows16",
        "rb_2048x1024_fp16_nearest"])
def test_chained_tma_launches_equal_whole_grid_waits(T, name, make, tile):
    # One call of 24 steps chains its launches (each work item waits for the nine items
    # around it in the previous launch); 24 calls of one step wait for the whole previous
    # grid every time.  The arithmetic is the same, so the states agree bit for bit.
    case, fields = make()
    if case.get("storage", "fp32") != "fp32":
        case = dict(case, rounding="nearest")
    states = []
    for chained in (False, True):
        lat = T.Lattice(case, fields)
        lat.set_kernel(0)
        lat.set_tile(*tile)
        assert "tclbm_step_tma_corr" in lat.describe(), lat.describe()
        if chained:
            lat.step(24)
        else:
            for _ in range(24):
                lat.step(1)
        states.append(lat.populations())
        lat.close()
    (fa, ha), (fb, hb) = states
    assert np.array_equal(fa, fb) and np.array_equal(ha, hb)


@pytest.mark.parametrize("name,make", [
    ("athermal_taylor_green_2048", lambda: W.taylor_green(2048, F0=1e-8, nu=0.02)),
    ("thermal_no_correction_2048x1024", lambda: W.random_periodic(2048, 1024, seed=31, force="accel",
                                                                   correction=False)),
], ids=["athermal_taylor_green_2048", "thermal_no_correction_2048x1024"])
def test_tma_plain_kernel_short_tail_equals_the_direct_kernel(T, name, make):
    # the TMA kernel without the correction term, 16-row segments on a grid of more than
    # two waves (its last wave half-height), against the direct-load kernel: periodic, so
    # bit for bit
    case, fields = make()
    states = []
    for kind in (0, 1):
        lat = T.Lattice(case, fields)
        lat.set_kernel(kind)
        if kind == 0:
            lat.set_tile(128, 16)
            assert "last" in lat.describe(), lat.describe()
        lat.step(21)
        states.append(lat.populations())
        lat.close()
    (fa, ha), (fb, hb) = states
    assert np.array_equal(fa, fb)
    if case["thermal"]:
        assert np.array_equal(ha, hb)


_PLAN_SCRIPT = """
import sys
sys.path.insert(0, {root!r})
from paper_1610_07114_gb300 import tclbm, workloads as W
if {warm}:
    tclbm.Lattice(*W.rayleigh_benard(64, 32)).close()
lat = tclbm.Lattice(*W.random_periodic(4096, 2048, seed=32, force="accel", correction=False))
print(lat.describe())
lat.close()
"""


def test_tma_plain_segment_plan_does_not_depend_on_the_first_lattice(T):
    # the plain TMA kernel's resident CTAs come from the occupancy calculator, asked (and
    # remembered) the first time a lattice's launch shape is chosen, which may be before
    # any lattice raised the kernel's shared-memory limit: a fresh process whose first
    # lattice is this one must plan the same segments as one that made another first
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = [subprocess.run([sys.executable, "-c", _PLAN_SCRIPT.format(root=root, warm=w)], capture_output=True,
                          text=True, timeout=600, check=True).stdout.strip().splitlines()[-1] for w in (False, True)]
    assert out[0] == out[1], out
    assert "last" in out[0], out[0]


KERNEL_CASES = [
    ("periodic_corr", *W.random_periodic(150, 45, seed=21, force="accel")),
    ("periodic_tg_nocorr", *W.random_periodic(97, 33, seed=22, force="taylor_green", correction=False)),
    ("athermal", *W.random_periodic(70, 20, seed=23, force="accel", thermal=False)),
    ("ywalls_zouhe", *W.with_walls(*W.random_periodic(130, 40, seed=24, force="accel"), axis="y", kind="zouhe")),
    ("ywalls_nee", *W.with_walls(*W.random_periodic(64, 9, seed=25, force="accel"), axis="y", kind="nee")),
    ("xwalls_eq", *W.with_walls(*W.random_periodic(129, 8, seed=26, force="none"), axis="x", kind="equilibrium")),
    ("tiny", *W.random_periodic(3, 5, seed=27, force="accel")),
]


@pytest.mark.parametrize("name,case,fields", KERNEL_CASES, ids=[c[0] for c in KERNEL_CASES])
@pytest.mark.parametrize("tile", [(32, 4), (64, 5), (128, 9), (32, 1), (64, 2)])
def test_tma_and_direct_kernels_agree(T, name, case, fields, tile):
    # Same arithmetic in both kernels; only the wall-node helpers, inlined into two
    # different kernels, may contract a multiply-add differently (one ulp at x walls).
    states = []
    for kind in (0, 1):
        lat = T.Lattice(case, fields)
        lat.set_kernel(kind)
        lat.set_tile(*tile)
        lat.step(30)
        states.append(lat.populations())
        assert lat.diagnostics() is not None  # also surfaces a pipeline timeout as an error
        lat.close()
    (fa, ha), (fb, hb) = states
    exact = "walls" not in name
    if exact:
        assert np.array_equal(fa, fb)
    np.testing.assert_allclose(fa, fb, rtol=0, atol=5e-7)
    if case["thermal"]:
        if exact:
            assert np.array_equal(ha, hb)
        np.testing.assert_allclose(ha, hb, rtol=0, atol=5e-7)


def test_graph_replay_equals_single_launches(T):
    case, fields = W.random_periodic(64, 40, seed=10, force="accel")
    a = T.Lattice(case, fields)
    a.step(129)  # odd start, then graph replays of 64 steps
    b = T.Lattice(case, fields)
    for _ in range(129):
        b.step(1)
    fa, ha = a.populations()
    fb, hb = b.populations()
    assert a.steps_done == b.steps_done == 129
    a.close()
    b.close()
    assert np.array_equal(fa, fb) and np.array_equal(ha, hb)


def test_device_diagnostics_conserve_mass_and_energy(T):
    case, fields = W.random_periodic(96, 64, seed=11, force="none")
    lat = T.Lattice(case, fields)
    d0 = lat.diagnostics()
    lat.step(500)
    d1 = lat.diagnostics()
    o = oracle.Oracle(case, fields, threads=8)
    m = o.moments()
    assert d0[0] == pytest.approx(m["rho"].sum(), rel=1e-7)
    assert d1[0] == pytest.approx(d0[0], rel=1e-6)
    assert d1[3] == pytest.approx(d0[3], rel=1e-6)
    assert d1[1] == pytest.approx(d0[1], abs=1e-4)
    lat.close()


def test_moments_into_device_tensors(T):
    import torch

    case, fields = W.random_periodic(40, 30, seed=12, force="accel")
    lat = T.Lattice(case, fields)
    lat.step(10)
    host = lat.moments()
    dev = {k: torch.empty((30, 40), dtype=torch.float64, device="cuda") for k in ("rho", "ux", "uy", "T")}
    lat.moments_device(dev)
    torch.cuda.synchronize()
    for k in dev:
        assert np.array_equal(dev[k].cpu().numpy(), host[k])
    lat.close()


def test_full_size_sampled_nodes(T):
    # the large Rayleigh-Benard-shaped lattice of the roofline measurement, in its
    # launch configuration: GPU step t -> t+1 against the oracle evaluated node by node
    case, fields = W.rayleigh_benard(4096, 2048, seed=5)
    lat = T.Lattice(case, fields)
    lat.step(3)
    f0, h0 = lat.populations()
    lat.step(1)
    f1, h1 = lat.populations()
    lat.close()
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.integers(0, 4096, 400), [0, 4095, 127, 128, 0, 4095]])
    ys = np.concatenate([rng.integers(0, 2048, 400), [0, 0, 2047, 2047, 1, 2046]])
    o = oracle.Oracle(case, None, threads=16)
    of, oh = o.update_nodes(xs, ys, f0, h0)
    np.testing.assert_allclose(f1[:, ys, xs].T, of, rtol=0, atol=2e-6)
    np.testing.assert_allclose(h1[:, ys, xs].T, oh, rtol=0, atol=2e-6)


def test_full_size_sampled_nodes_fp16_stochastic(T):
    # the same lattice in 16-bit deviation storage with stochastic rounding (the TMA
    # kernel's 16-bit build): one step from the stored state against the oracle; the
    # GPU output is a deviation from the rest state rounded to FP16 (stochastic: within
    # one ulp, 2^-10 of the deviation, which is smaller than the population itself),
    # hence relative 2^-10 of the population plus 1e-6
    case, fields = W.rayleigh_benard(4096, 2048, seed=6, storage="fp16")
    case = dict(case, rounding="stochastic")
    lat = T.Lattice(case, fields)
    lat.step(3)
    f0, h0 = lat.populations()
    lat.step(1)
    f1, h1 = lat.populations()
    lat.close()
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.integers(0, 4096, 400), [0, 4095, 127, 128, 0, 4095]])
    ys = np.concatenate([rng.integers(0, 2048, 400), [0, 0, 2047, 2047, 1, 2046]])
    o = oracle.Oracle(dict(case, storage="fp32"), None, threads=16)
    of, oh = o.update_nodes(xs, ys, f0, h0)
    np.testing.assert_allclose(f1[:, ys, xs].T, of, rtol=2.0**-10, atol=1e-6)
    np.testing.assert_allclose(h1[:, ys, xs].T, oh, rtol=2.0**-10, atol=1e-6)


def test_batched_sweep_full_size_sampled_nodes(T):
    # the 256-lattice sweep of the batched measurement (FP16 deviations, stochastic
    # rounding) in one batch with the shape the autotuner keeps there (32-wide strips,
    # 64 rows): one batch step against the oracle, node by node, on the largest and
    # smallest lattices
    cases = W.batched_rb_sweep(count=256, storage="fp16")
    lats = [T.Lattice(dict(c, rounding="stochastic"), f) for c, f in cases]
    b = T.Batch(lats)
    b.set_tile(32, 64, False)
    b.step(3)
    order = sorted(range(len(cases)), key=lambda i: cases[i][0]["nx"] * cases[i][0]["ny"])
    pick = order[:2] + order[-2:]
    before = {i: lats[i].populations() for i in pick}
    b.step(1)
    rng = np.random.default_rng(2)
    for i in pick:
        c = cases[i][0]
        nx, ny = c["nx"], c["ny"]
        xs = np.concatenate([rng.integers(0, nx, 100), [0, nx - 1, 0, nx - 1]])
        ys = np.concatenate([rng.integers(0, ny, 100), [0, 0, ny - 1, ny - 1]])
        f0, h0 = before[i]
        f1, h1 = lats[i].populations()
        of, oh = oracle.Oracle(dict(c, storage="fp32"), None, threads=16).update_nodes(xs, ys, f0, h0)
        np.testing.assert_allclose(f1[:, ys, xs].T, of, rtol=2.0**-10, atol=1e-6)  # FP16, as above
        np.testing.assert_allclose(h1[:, ys, xs].T, oh, rtol=2.0**-10, atol=1e-6)
    b.close()
    for l in lats:
        l.close()


TILE_CASES = [
    ("periodic_corr_partial", *W.random_periodic(150, 45, seed=71, force="accel")),
    ("periodic_tg_force", *W.random_periodic(70, 37, seed=72, force="taylor_green")),
    ("rb_zouhe", *W.rayleigh_benard(96, 48, Ra=2e4, seed=73)),
    ("ywalls_nee", *W.with_walls(*W.random_periodic(64, 19, seed=74, force="accel"), axis="y", kind="nee")),
    ("xwalls_eq", *W.with_walls(*W.random_periodic(130, 8, seed=75, force="none"), axis="x", kind="equilibrium")),
    ("couette_narrow", *W.couette()),
    ("tiny_periodic", *W.random_periodic(3, 5, seed=76, force="accel")),
]


@pytest.mark.parametrize("name,case,fields", TILE_CASES, ids=[c[0] for c in TILE_CASES])
def test_tile_kernel_agrees_with_the_marching_kernel(T, name, case, fields):
    # one node per thread on 32 x 4 tiles against row marching: the same per-node code;
    # wall helpers inlined into another kernel may differ by one ulp (5e-7 absolute)
    states = []
    for kind in (2, 1):
        lat = T.Lattice(case, fields)
        lat.set_kernel(kind)
        if kind == 2:
            assert lat.describe().startswith("tclbm_step_tile")
        lat.step(41)
        states.append(lat.populations())
        lat.close()
    (fa, ha), (fb, hb) = states
    walls = any(case["walls"][s]["kind"] != "periodic" for s in ("x-", "x+", "y-", "y+"))
    if not walls:
        assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
    np.testing.assert_allclose(fa, fb, rtol=0, atol=5e-7)
    np.testing.assert_allclose(ha, hb, rtol=0, atol=5e-7)


LATE_WAIT_CASES = [
    ("rb_512x256", lambda: W.rayleigh_benard(512, 256, Ra=1e4, seed=79, amp=1e-2)),
    ("periodic_512x256", lambda: W.random_periodic(512, 256, seed=80, force="accel")),
]


@pytest.mark.parametrize("name,make", LATE_WAIT_CASES, ids=[c[0] for c in LATE_WAIT_CASES])
def test_tile_kernel_on_grids_of_several_waves_agrees_with_the_marching_kernel(T, name, make):
    # 512 x 256 on 32 x 4 tiles is 1024 CTAs, more than one wave of resident CTAs, so the
    # tile kernel takes its instance that waits for the previous step's grid just before
    # the first load; the arithmetic is the same as on one wave
    case, fields = make()
    states = []
    for kind in (2, 1):
        lat = T.Lattice(case, fields)
        lat.set_kernel(kind)
        lat.step(41)
        lat.step(64)  # graph replay
        states.append(lat.populations())
        lat.close()
    (fa, ha), (fb, hb) = states
    walls = any(case["walls"][s]["kind"] != "periodic" for s in ("x-", "x+", "y-", "y+"))
    if not walls:
        assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
    np.testing.assert_allclose(fa, fb, rtol=0, atol=5e-7)
    np.testing.assert_allclose(ha, hb, rtol=0, atol=5e-7)


def test_tile_kernel_matches_the_oracle_and_is_the_small_lattice_default(T):
    case, fields = W.rayleigh_benard(72, 40, Ra=5e3, seed=77)
    lat = T.Lattice(case, fields)
    assert lat.describe().startswith("tclbm_step_tile")
    lat.step(300)
    g = lat.moments()
    lat.close()
    o = oracle.Oracle(case, fields, threads=8)
    o.step(300)
    e = field_errors(g, o.moments(), case)
    assert e["rho"] <= REL_L2 and e["u"] <= REL_L2 and e["T"] <= REL_L2, e


def test_tile_kernel_refuses_lattices_it_cannot_serve(T):
    # ny % 8 == 1 with y walls: a top-wall row would need a row outside the tile's halo
    case, fields = W.with_walls(*W.random_periodic(40, 17, seed=78), axis="y", kind="zouhe")
    lat = T.Lattice(case, fields)
    assert not lat.describe().startswith("tclbm_step_tile")
    with pytest.raises(T.TclbmError):
        lat.set_kernel(2)
    athermal = T.Lattice(*W.random_periodic(40, 16, seed=79, thermal=False))
    with pytest.raises(T.TclbmError):
        athermal.set_kernel(2)
    lat.close()
    athermal.close()


WORK_CASES = [
    ("periodic_accel", lambda: W.random_periodic(70, 37, seed=61, force="accel")),
    ("periodic_tg", lambda: W.random_periodic(45, 33, seed=62, force="taylor_green")),
    ("rb_zouhe_nee", lambda: W.rayleigh_benard(96, 48, Ra=1e4, seed=63, amp=1e-2)),
    ("ywalls_nee", lambda: W.with_walls(*W.random_periodic(53, 41, seed=64, force="accel"), axis="y", kind="nee")),
    ("xwalls_eq", lambda: W.with_walls(*W.random_periodic(67, 9, seed=65, force="accel"), axis="x",
                                       kind="equilibrium")),
]


@pytest.mark.parametrize("name,make", WORK_CASES, ids=[c[0] for c in WORK_CASES])
def test_work_term_matches_oracle(T, name, make):
    # the body force's power as a source of total energy (tclbm_params.work, an extension of
    # Eq. 22): every kernel variant against the FP64 oracle at the FP32 parity bar
    case, fields = make()
    case = dict(case, work=True)
    o = oracle.Oracle(case, fields, threads=8)
    o.step(300)
    om = o.moments()
    for kernel in (2, 1, 0):
        lat = T.Lattice(case, fields)
        try:
            lat.set_kernel(kernel)
        except T.TclbmError:
            lat.close()
            continue
        lat.step(300)
        e = field_errors(lat.moments(), om, case)
        lat.close()
        print(name, kernel, e)
        assert e["rho"] <= REL_L2 and e["u"] <= REL_L2 and e["T"] <= REL_L2, (name, kernel, e)
