"""Slab decomposition on the GPU: one lattice advanced as slab lattices whose ghost rows
are refreshed by tclbm_copy_rows must equal the undivided lattice bit for bit on the
owned rows, when every lattice runs the same step kernel variant."""
import numpy as np
import pytest

from paper_1610_07114_gb300 import slabs as S
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


def whole_run(T, case, fields, steps, kernel):
    lat = T.Lattice(case, fields)
    if kernel is not None:
        lat.set_kernel(kernel)
    lat.step(steps)
    out = lat.populations(), lat.moments()
    lat.close()
    return out


CASES = [
    # name, make, parts, exchange_every, kernel variant (None: the library's choice), steps
    ("rb_256x128_tiles_every1", lambda: W.rayleigh_benard(256, 128), 2, 1, None, 200),
    ("rb_256x128_tiles_every4", lambda: W.rayleigh_benard(256, 128), 2, 4, 2, 203),
    ("rb_256x128_4parts_every2", lambda: W.rayleigh_benard(256, 128), 4, 2, 2, 130),
    ("rb_512x256_tma_every3", lambda: W.rayleigh_benard(512, 256, seed=2), 3, 3, 0, 100),
    ("periodic_150x45_direct", lambda: W.random_periodic(150, 45, seed=11, force="accel"), 3, 2, 1, 77),
    ("x_walls_129x24_direct", lambda: W.with_walls(*W.random_periodic(129, 24, seed=12, force="none"), axis="x",
                                                   kind="equilibrium"), 2, 1, 1, 50),
    ("couette_zouhe_8x64", lambda: W.couette(), 2, 2, 1, 300),
    ("rb_128x64_fp16_nearest", lambda: W.rayleigh_benard(128, 64, storage="fp16"), 2, 2, None, 120),
]


@pytest.mark.parametrize("name,make,parts,every,kernel,steps", CASES)
def test_slabs_equal_the_undivided_lattice(T, name, make, parts, every, kernel, steps):
    case, fields = make()
    (fw, hw), mw = whole_run(T, case, fields, steps, kernel)
    with S.Slabs(case, fields, parts=parts, exchange_every=every, kernel=kernel) as sl:
        sl.step(steps // 2)
        sl.step(steps - steps // 2)  # a partial chunk between calls, then the rest
        assert sl.steps_done == steps
        f, h = sl.populations()
        m = sl.moments()
    assert np.array_equal(f, fw), name
    assert np.array_equal(h, hw), name
    for k in ("rho", "ux", "uy", "T"):
        assert np.array_equal(m[k], mw[k]), (name, k)


def test_copy_rows_orders_streams(T):
    import torch

    case, fields = W.random_periodic(96, 64, seed=13, force="accel")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a = T.Lattice(case, fields, stream=s1.cuda_stream)
    b = T.Lattice(case, fields, stream=s2.cuda_stream)
    a.step(300)  # queued on s1; b's copy must wait for it
    T.tclbm_copy_rows(b.handle, 0, a.handle, 0, case["ny"])
    fb, hb = b.populations()
    fa, ha = a.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
    a.step(10)  # a's next steps follow the copy; b is untouched by them
    fb2, _ = b.populations()
    assert np.array_equal(fb2, fb)
    a.close()
    b.close()


def test_copy_rows_rejects_bad_arguments(T):
    c1, f1 = W.random_periodic(32, 16, seed=14)
    c2, f2 = W.random_periodic(48, 16, seed=15)
    c3 = dict(c1, storage="fp16")
    a, b, c = T.Lattice(c1, f1), T.Lattice(c2, f2), T.Lattice(c3, f1)
    for args in [(b.handle, 0, a.handle, 0, 2),  # nx differs
                 (c.handle, 0, a.handle, 0, 2),  # storage differs
                 (a.handle, 15, a.handle, 0, 2),  # destination past the last row
                 (a.handle, 0, a.handle, -1, 1),
                 (a.handle, 0, a.handle, 1, 2),  # overlapping rows of one lattice
                 (a.handle, 0, a.handle, 4, -1)]:
        with pytest.raises(T.TclbmError):
            T.tclbm_copy_rows(*args)
    before = a.populations()[0]
    T.tclbm_copy_rows(a.handle, 3, a.handle, 9, 0)  # nothing to copy
    T.tclbm_copy_rows(a.handle, 0, a.handle, 8, 8)  # disjoint rows of one lattice
    after = a.populations()[0]
    # populations() reads the streamed state, row y from stored rows y-1..y+1: rows 1..6
    # now pull only copied rows, rows 9..14 only untouched ones
    assert np.array_equal(after[:, 1:7], before[:, 9:15]) and np.array_equal(after[:, 9:15], before[:, 9:15])
    for l in (a, b, c):
        l.close()
