"""Batched stepping (tclbm_batch_*): many lattices of different sizes, parameters and
collision variants advanced by one launch per time step.

The batch changes no arithmetic: every node runs the single-lattice strip code, so a
lattice stepped in a batch must equal the same lattice stepped alone with the
direct-load kernel -- bit for bit on periodic lattices; at walls the wall helpers,
inlined into a different kernel, may contract one multiply-add differently (one FP32
ulp of an O(0.1) population), hence the 5e-7 absolute bound there.  The batch result
is also compared with the FP64 oracle at the single-lattice tolerance.
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


def mixed_cases(storage="fp32", rounding="nearest"):
    cases = [
        ("periodic_corr_150x45", *W.random_periodic(150, 45, seed=31, force="accel")),
        ("rb_zouhe_96x48", *W.rayleigh_benard(96, 48, Ra=2e4, seed=32)),
        ("athermal_70x20", *W.random_periodic(70, 20, seed=33, force="accel", thermal=False)),
        ("tg_nocorr_97x33", *W.random_periodic(97, 33, seed=34, force="taylor_green", correction=False)),
        ("nee_walls_64x9", *W.with_walls(*W.random_periodic(64, 9, seed=35, force="accel"), axis="y", kind="nee")),
        ("eq_ends_129x8", *W.with_walls(*W.random_periodic(129, 8, seed=36, force="none"), axis="x",
                                        kind="equilibrium")),
        ("tiny_3x5", *W.random_periodic(3, 5, seed=37, force="accel")),
        ("couette_8x64", *W.couette()),
    ]
    return [(n, dict(c, storage=storage, rounding=rounding), f) for n, c, f in cases]


def has_walls(case):
    return any(case["walls"][s]["kind"] != "periodic" for s in ("x-", "x+", "y-", "y+"))


def alone(T, case, fields, steps):
    lat = T.Lattice(case, fields)
    lat.set_kernel(1)
    lat.step(steps)
    f, h = lat.populations()
    lat.close()
    return f, h


def assert_same(case, a, b):
    (fa, ha), (fb, hb) = a, b
    if not has_walls(case):
        assert np.array_equal(fa, fb)
        if ha is not None:
            assert np.array_equal(ha, hb)
    np.testing.assert_allclose(fa, fb, rtol=0, atol=5e-7)
    if ha is not None:
        np.testing.assert_allclose(ha, hb, rtol=0, atol=5e-7)


@pytest.mark.parametrize("shape", [(32, 1, True), (64, 4, True), (128, 3, False), (32, 64, False)])
def test_batch_equals_each_lattice_alone(T, shape):
    cases = mixed_cases()
    lats = [T.Lattice(c, f) for _, c, f in cases]
    with T.Batch(lats) as b:
        b.set_tile(*shape)
        b.step(37)
        assert b.steps_done == 37
    for (name, c, f), lat in zip(cases, lats):
        assert lat.steps_done == 37
        assert_same(c, lat.populations(), alone(T, c, f, 37))
        lat.close()


def test_batch_graph_replay_and_odd_parity(T):
    # 1 + 129 steps: single launches, then graph replays entered at odd batch parity
    cases = mixed_cases()[:4]
    lats = [T.Lattice(c, f) for _, c, f in cases]
    b = T.Batch(lats)
    b.step(1)
    b.step(129)
    for (name, c, f), lat in zip(cases, lats):
        assert_same(c, lat.populations(), alone(T, c, f, 130))
        lat.close()
    b.close()


def test_lattice_stepped_alone_between_batch_steps(T):
    # the batch re-reads each lattice's source copy when it changed behind its back
    cases = mixed_cases()[:3]
    lats = [T.Lattice(c, f) for _, c, f in cases]
    for l in lats:
        l.set_kernel(1)
    b = T.Batch(lats)
    b.step(10)
    lats[1].step(3)
    b.step(7)
    lats[0].init_fields(cases[0][2])
    b.step(5)
    expect_steps = [5, 25, 22]
    for (name, c, f), lat, s in zip(cases, lats, expect_steps):
        assert lat.steps_done == s
        assert_same(c, lat.populations(), alone(T, c, f, s))
    b.close()
    for l in lats:
        l.close()


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_batch_16bit_stochastic_rounding_equals_alone(T, storage):
    # the rounding bits depend on (node, population pair, step) only: same in a batch
    cases = mixed_cases(storage, "stochastic")[:5]
    lats = [T.Lattice(c, f) for _, c, f in cases]
    with T.Batch(lats) as b:
        b.step(70)
    for (name, c, f), lat in zip(cases, lats):
        got = lat.populations()
        ref = alone(T, c, f, 70)
        assert_same(c, got, ref)
        lat.close()


def test_autotune_keeps_the_state_and_picks_a_valid_shape(T):
    cases = mixed_cases()
    lats = [T.Lattice(c, f) for _, c, f in cases]
    b = T.Batch(lats)
    b.step(5)
    tx, rows, pers, us = b.autotune(trial_steps=4)
    assert tx in (32, 64, 128) and rows >= 1 and us > 0
    assert b.steps_done == 5 and all(l.steps_done == 5 for l in lats)
    assert f"<{tx}," in b.describe() and f"rows {rows}" in b.describe()
    b.step(6)
    for (name, c, f), lat in zip(cases, lats):
        assert_same(c, lat.populations(), alone(T, c, f, 11))
        lat.close()
    b.close()


def test_batch_matches_fp64_oracle(T):
    cases = mixed_cases()[:3]
    lats = [T.Lattice(c, f) for _, c, f in cases]
    with T.Batch(lats) as b:
        b.step(200)
    for (name, c, f), lat in zip(cases, lats):
        g = lat.moments()
        o = oracle.Oracle(c, f, threads=8)
        o.step(200)
        r = o.moments()
        for k in ("rho", "T"):
            assert np.linalg.norm(g[k] - r[k]) / np.linalg.norm(r[k]) <= 1e-5, (name, k)
        du = np.sqrt(np.sum((g["ux"] - r["ux"]) ** 2 + (g["uy"] - r["uy"]) ** 2))
        nu = max(np.sqrt(np.sum(r["ux"] ** 2 + r["uy"] ** 2)), np.sqrt(r["ux"].size) * c["U_ref"])
        assert du / nu <= 1e-5, name
        lat.close()


def test_batch_rejects_bad_arguments(T):
    a = T.Lattice(*W.random_periodic(16, 8, seed=1))
    c16 = dict(W.random_periodic(16, 8, seed=2)[0], storage="fp16")
    b16 = T.Lattice(c16)
    with pytest.raises(T.TclbmError):
        T.tclbm_batch_create([a.handle, b16.handle])  # mixed storage
    with pytest.raises(T.TclbmError):
        T.tclbm_batch_create([a.handle, a.handle])  # repeated handle
    with pytest.raises(T.TclbmError):
        T.tclbm_batch_create([])
    b = T.Batch([a])
    with pytest.raises(T.TclbmError):
        b.set_tile(48, 2)
    with pytest.raises(T.TclbmError):
        b.set_tile(32, 0)
    with pytest.raises(T.TclbmError):
        b.step(-1)
    b.close()
    a.close()
    b16.close()


def test_replacing_lattices_rebuilds_the_work_list(T):
    # A destroyed lattice's handle address can come back for a new lattice of another
    # size; the batch must rebuild its work list from sizes, not from handle addresses.
    keep = T.Lattice(*W.random_periodic(40, 24, seed=40))
    b = T.Batch([keep])
    sizes = [(24, 16), (70, 36), (16, 8), (96, 40), (33, 21), (64, 64)]
    prev = None
    for i, (nx, ny) in enumerate(sizes):
        case, fields = W.random_periodic(nx, ny, seed=50 + i)
        lat = T.Lattice(case, fields)
        lat.set_kernel(1)
        b.set_lattices([keep, lat])
        b.step(9)
        assert_same(case, lat.populations(), alone(T, case, fields, 9))
        b.set_lattices([keep])
        lat.close()  # frees the handle; the next iteration's handle may reuse its address
        prev = (nx, ny)
    assert prev is not None
    b.close()
    keep.close()


@pytest.mark.parametrize("storage,rounding", [("fp32", "nearest"), ("fp16", "stochastic")])
@pytest.mark.parametrize("tma", [(128, 16), (64, 8), (128, 3)])
def test_tma_fed_batch_equals_each_lattice_alone(T, tma, storage, rounding):
    # TMA-fed strips for the thermal lattices with the correction term at least tx wide
    # (the single-lattice TMA kernel's code, one CTA per strip); the others keep the
    # direct-load strips.  Both agree with the lattice stepped alone.
    cases = mixed_cases(storage, rounding) + [
        ("rb_256x64", *W.rayleigh_benard(256, 64, Ra=1e4, seed=38, storage=storage)),
        ("periodic_200x37", *W.random_periodic(200, 37, seed=39, force="taylor_green", storage=storage)),
    ]
    cases = [(n, dict(c, rounding=rounding), f) for n, c, f in cases]
    lats = [T.Lattice(c, f) for _, c, f in cases]
    with T.Batch(lats) as b:
        b.set_tma(*tma)
        assert b.tma_shape() == tma
        assert "tclbm_step_batch_tma" in b.describe()
        b.step(3)
        b.step(70)  # graph replay entered at odd parity
    for (name, c, f), lat in zip(cases, lats):
        assert lat.steps_done == 73
        got = lat.populations()
        assert lat.diagnostics() is not None  # an expired pipeline wait would surface here
        for kernel in (0, 1):
            ref = T.Lattice(c, f)
            try:
                ref.set_kernel(kernel)
            except T.TclbmError:
                ref.close()
                continue
            ref.step(73)
            exp = ref.populations()
            ref.close()
            assert_same(c, got, exp)
        lat.close()


def test_tma_fed_batch_with_a_half_height_last_wave_equals_each_lattice_alone(T):
    # 40 periodic thermal lattices of 512 x 256 in 128 x 16 TMA strips: 2,560 work items,
    # more than two waves, so the last wave of items (the last lattices in the list) is cut
    # to half height; every lattice still equals itself stepped alone, bit for bit
    cases = [W.random_periodic(512, 256, seed=300 + i, force="accel") for i in range(40)]
    lats = [T.Lattice(c, f) for c, f in cases]
    import torch

    wave = torch.cuda.get_device_properties(0).multi_processor_count * 3  # FP32 TMA CTAs per SM: 3
    with T.Batch(lats) as b:
        b.set_tma(128, 16)
        b.step(5)
        # 2,560 items, the last `wave` of them split in two
        assert "items %d " % (2560 + wave) in b.describe(), b.describe()
    for (c, f), lat in zip(cases, lats):
        got = lat.populations()
        ref = T.Lattice(c, f)
        ref.set_kernel(0)
        ref.step(5)
        exp = ref.populations()
        ref.close()
        assert np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1])
        lat.close()


def test_tma_fed_batch_matches_fp64_oracle(T):
    case, fields = W.rayleigh_benard(192, 96, Ra=1e4, seed=40, amp=1e-2)
    lat = T.Lattice(case, fields)
    with T.Batch([lat]) as b:
        b.set_tma(128, 16)
        b.step(300)
    g = lat.moments()
    lat.close()
    o = oracle.Oracle(case, fields, threads=8)
    o.step(300)
    from tests.parity import field_errors

    e = field_errors(g, o.moments(), case)
    assert e["rho"] <= 1e-5 and e["u"] <= 1e-5 and e["T"] <= 1e-5, e
