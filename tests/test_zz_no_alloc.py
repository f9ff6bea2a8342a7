"""tclbm_diagnostics_noalloc(): the allocation-free form of the FP64 diagnostics.

It exists for callers that may not allocate device memory when they need the sums
(memory planned up front, a fixed budget, raw device pointers only).  It is checked
here through the C ABI against tclbm_diagnostics() on the same state, on two calls in
a row (the calls share one file-scope scratch array), and after the lattice moved on.
This file is collected last so that a failure here cannot hide other results.
"""
import ctypes

import numpy as np
import pytest

from paper_1610_07114_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-9  # both paths sum the same FP64 node values; only the force tables may round differently


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
    T.tclbm_get_populations(lat.handle, f.data_ptr(), h.data_ptr(), 1)


def _noalloc(T, lat, f, h, out_dev=None):
    """One call; the result lands in `out_dev` (a device tensor) if given, else on the host."""
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    if out_dev is not None:
        st = T.library().tclbm_diagnostics_noalloc(ctypes.byref(lat.params), f.data_ptr(), h.data_ptr(), None,
                                                    out_dev.data_ptr(), 1, ctypes.c_void_p(stream))
        torch.cuda.synchronize()
        assert st == 0, T.tclbm_last_error()
        return None
    out = np.zeros(8)
    st = T.library().tclbm_diagnostics_noalloc(ctypes.byref(lat.params), f.data_ptr(), h.data_ptr(), None,
                                                out.ctypes.data, 0, ctypes.c_void_p(stream))
    assert st == 0, T.tclbm_last_error()
    return out


def _check(a, ref):
    for k in (0, 1, 2, 3, 4, 5, 7):  # out[6] needs a velocity reference, which is not passed here
        assert a[k] == pytest.approx(ref[k], rel=REL, abs=1e-12 * abs(ref[0])), (k, a[k], ref[k])
    assert a[6] == 0.0


def test_noalloc_sums_match_the_handle_diagnostics_on_two_calls_in_a_row(T):
    import torch

    case, fields = W.rayleigh_benard(96, 48, Ra=1e4, seed=4)
    lat = T.Lattice(case, fields)
    shape = (9, lat.ny, lat.nx)
    f, h = (torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(2))
    out_dev = torch.empty(8, dtype=torch.float64, device="cuda")
    lat.step(200)
    ref = lat.diagnostics()
    _device_populations(T, lat, f, h)
    first = _noalloc(T, lat, f, h)  # the first call on the device resolves the scratch address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _noalloc(T, lat, f, h, out_dev)
    second = out_dev.cpu().numpy()
    assert torch.cuda.mem_get_info()[0] == free0  # the call itself allocates nothing
    _check(first, ref)
    _check(second, ref)
    # the lattice moves on; the shared scratch still holds the previous call's partials
    lat.step(150)
    ref2 = lat.diagnostics()
    _device_populations(T, lat, f, h)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    third = _noalloc(T, lat, f, h)
    assert torch.cuda.mem_get_info()[0] == free1
    _check(third, ref2)
    assert abs(ref2[4] - ref[4]) > 0  # a different state, so stale partials would show
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
