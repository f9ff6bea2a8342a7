"""tclbm_diagnostics_noalloc(): the allocation-free form of the FP64 diagnostics.

It exists for callers that may not allocate device memory when they need the sums
(memory planned up front, a fixed budget, raw device pointers only).  It is checked
here through the C ABI against tclbm_diagnostics() on the same state, on two calls in
a row (the calls share one file-scope scratch array), and after the lattice moved on;
on a thermal lattice with a uniform body force, on a Taylor-Green forced lattice
(athermal and thermal), and with a velocity reference for the residual sum out[6].
This file is collected last so that a failure here cannot hide other results.
"""
import ctypes

import numpy as np
import pytest

from paper_1610_07114_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# Both paths sum the same FP64 node values (the same constants in T and the force); only
# the order of the additions differs, which moves a sum by at most about N ulps of the
# sum of the magnitudes of its terms (N <= 4608 nodes here).
REL = 1e-9
ORDER = 1e-12


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1610_07114_gb300 import build

    build.build()
    from paper_1610_07114_gb300 import tclbm

    lib = tclbm.library()
    lib.tclbm_diagnostics_noalloc.argtypes = [ctypes.POINTER(tclbm.tclbm_params), ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    lib.tclbm_diagnostics_noalloc.restype = ctypes.c_int
    return tclbm


def _device_populations(T, lat, f, h):
    T.tclbm_get_populations(lat.handle, f.data_ptr(), h.data_ptr() if h is not None else None, 1)


def _noalloc(T, lat, f, h, usnap=None, out_dev=None):
    """One call; the result lands in `out_dev` (a device tensor) if given, else on the host."""
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    hp = h.data_ptr() if h is not None else None
    up = usnap.data_ptr() if usnap is not None else None
    if out_dev is not None:
        st = T.library().tclbm_diagnostics_noalloc(ctypes.byref(lat.params), f.data_ptr(), hp, up,
                                                    out_dev.data_ptr(), 1, ctypes.c_void_p(stream))
        torch.cuda.synchronize()
        assert st == 0, T.tclbm_last_error()
        return None
    out = np.zeros(8)
    st = T.library().tclbm_diagnostics_noalloc(ctypes.byref(lat.params), f.data_ptr(), hp, up, out.ctypes.data, 0,
                                                ctypes.c_void_p(stream))
    assert st == 0, T.tclbm_last_error()
    return out


def _magnitudes(lat, usnap_host=None):
    """Sums of |term| of every diagnostic, from the FP64 moments: the scale of the
    rounding that a different summation order can introduce."""
    m = lat.moments()
    r, vx, vy, t = m["rho"], m["ux"], m["uy"], m["T"]
    f, h = lat.populations()
    mag = np.zeros(8)
    mag[0] = np.abs(r).sum()
    mag[1] = np.abs(r * vx).sum()
    mag[2] = np.abs(r * vy).sum()
    mag[3] = np.abs(h).sum() if h is not None else 0.0
    mag[4] = (0.5 * r * (vx * vx + vy * vy)).sum()
    mag[5] = np.abs(vy * (t - lat.params.T_ref)).sum()
    if usnap_host is not None:
        mag[6] = ((vx - usnap_host[0]) ** 2 + (vy - usnap_host[1]) ** 2).sum()
    mag[7] = (vx * vx + vy * vy).sum()
    return mag


def _check(a, ref, mag, with_snapshot=False):
    for k in range(8):
        if k == 6 and not with_snapshot:
            assert a[6] == 0.0
            continue
        tol = REL * abs(ref[k]) + ORDER * mag[k]
        assert abs(a[k] - ref[k]) <= tol, (k, a[k], ref[k], tol)


CASES = [
    ("rb_accel", lambda: W.rayleigh_benard(96, 48, Ra=1e4, seed=4)),
    ("tg_athermal", lambda: W.taylor_green(48, F0=2e-5, nu=0.02)),
    ("tg_thermal", lambda: W.taylor_green(40, F0=2e-5, nu=0.02, thermal=True)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_noalloc_sums_match_the_handle_diagnostics_on_two_calls_in_a_row(T, name, make):
    import torch

    case, fields = make()
    lat = T.Lattice(case, fields)
    shape = (9, lat.ny, lat.nx)
    f = torch.empty(shape, dtype=torch.float64, device="cuda")
    h = torch.empty(shape, dtype=torch.float64, device="cuda") if lat.thermal else None
    out_dev = torch.empty(8, dtype=torch.float64, device="cuda")
    lat.step(200)
    ref = lat.diagnostics()
    mag = _magnitudes(lat)
    _device_populations(T, lat, f, h)
    first = _noalloc(T, lat, f, h)  # the first call on the device resolves the scratch address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _noalloc(T, lat, f, h, out_dev=out_dev)
    second = out_dev.cpu().numpy()
    assert torch.cuda.mem_get_info()[0] == free0  # the call itself allocates nothing
    _check(first, ref, mag)
    _check(second, ref, mag)
    # the lattice moves on; the shared scratch still holds the previous call's partials
    lat.step(150)
    ref2 = lat.diagnostics()
    mag2 = _magnitudes(lat)
    _device_populations(T, lat, f, h)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    third = _noalloc(T, lat, f, h)
    assert torch.cuda.mem_get_info()[0] == free1
    _check(third, ref2, mag2)
    assert abs(ref2[4] - ref[4]) > 0  # a different state, so stale partials would show
    lat.close()


def test_noalloc_residual_sum_against_the_handle_snapshot(T):
    # out[6] = sum |u - u_snap|^2.  The handle keeps its snapshot as FP32 velocities; the
    # allocation-free call takes the reference as double [2][ny][nx], here the same
    # FP32-rounded velocities.
    import torch

    case, fields = W.rayleigh_benard(80, 40, Ra=1e4, seed=6)
    lat = T.Lattice(case, fields)
    lat.step(100)
    lat.snapshot_velocity()
    m = lat.moments()
    usnap_host = np.stack([m["ux"].astype(np.float32).astype(np.float64),
                           m["uy"].astype(np.float32).astype(np.float64)])
    usnap = torch.from_numpy(np.ascontiguousarray(usnap_host)).cuda()
    lat.step(40)
    ref = lat.diagnostics()
    mag = _magnitudes(lat, usnap_host)
    assert ref[6] > 0
    shape = (9, lat.ny, lat.nx)
    f, h = (torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(2))
    _device_populations(T, lat, f, h)
    torch.cuda.synchronize()
    for _ in range(2):
        _check(_noalloc(T, lat, f, h, usnap=usnap), ref, mag, with_snapshot=True)
    lat.close()


def test_noalloc_reports_a_non_finite_state(T):
    import torch

    case, fields = W.rayleigh_benard(32, 16, Ra=1e4, seed=7)
    lat = T.Lattice(case, fields)
    shape = (9, lat.ny, lat.nx)
    f, h = (torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(2))
    _device_populations(T, lat, f, h)
    f[3, 5, 7] = float("nan")
    torch.cuda.synchronize()
    out = np.zeros(8)
    st = T.library().tclbm_diagnostics_noalloc(ctypes.byref(lat.params), f.data_ptr(), h.data_ptr(), None,
                                                out.ctypes.data, 0, None)
    assert st == T.ENONFINITE
    assert "non-finite" in T.tclbm_last_error()
    lat.close()


def test_noalloc_rejects_lattices_beyond_its_maximum(T):
    case, _ = W.rayleigh_benard(16, 8)
    p = T.params_from_case(case)
    p.nx, p.ny = 16384, 8192  # 134 M nodes > 67,108,864
    out = np.zeros(8)
    st = T.library().tclbm_diagnostics_noalloc(ctypes.byref(p), ctypes.c_void_p(1), ctypes.c_void_p(1), None,
                                                out.ctypes.data, 0, None)
    assert st == T.EINVAL
    assert "maximum" in T.tclbm_last_error()
