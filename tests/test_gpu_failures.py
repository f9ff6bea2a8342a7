"""Failure paths, made to happen without faulting or hanging the GPU.

* A bounded wait that runs out: the TMA producer is told to skip one source row
  (tclbm_test_skip_row); the consumers' 1 s waits expire, the kernel records the failure
  and returns, and the next synchronising call reports TCLBM_ETIMEOUT.  The context
  stays usable: the same handle, re-initialised, steps correctly afterwards.
* An allocator hook that returns NULL: tclbm_create reports TCLBM_ENOMEM.
* A non-finite state: the FP64 diagnostics report TCLBM_ENONFINITE.
"""
import ctypes

import numpy as np
import pytest

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


def test_expired_pipeline_wait_is_reported_and_the_context_recovers(T):
    case, fields = W.rayleigh_benard(256, 64, Ra=1e4, seed=9)
    ref = T.Lattice(case, fields)
    ref.set_kernel(0)
    ref.step(5)
    f_ref, h_ref = ref.populations()
    ref.close()

    lat = T.Lattice(case, fields)
    lat.set_kernel(0)
    T.tclbm_test_skip_row(lat.handle, 30)
    lat.step(1)
    with pytest.raises(T.TclbmError) as err:
        lat.diagnostics()
    assert err.value.status == T.ETIMEOUT
    T.tclbm_test_skip_row(lat.handle, -1)
    lat.init_fields(fields)
    lat.step(5)
    f, h = lat.populations()
    lat.close()
    assert np.array_equal(f, f_ref) and np.array_equal(h, h_ref)


def test_expired_wait_in_a_chain_of_launches_is_reported_and_the_context_recovers(T):
    # three chained launches: the first one's CTA for row 30 never gets that row and
    # gives up after 1 s; the items of the next launches that wait for it see the error
    # word and return instead of waiting out their own limit
    case, fields = W.rayleigh_benard(1024, 512, Ra=1e4, seed=9)
    ref = T.Lattice(case, fields)
    ref.set_kernel(0)
    ref.set_tile(128, 16)
    ref.step(5)
    f_ref, h_ref = ref.populations()
    ref.close()

    lat = T.Lattice(case, fields)
    lat.set_kernel(0)
    lat.set_tile(128, 16)
    T.tclbm_test_skip_row(lat.handle, 30)
    lat.step(3)
    with pytest.raises(T.TclbmError) as err:
        lat.diagnostics()
    assert err.value.status == T.ETIMEOUT
    T.tclbm_test_skip_row(lat.handle, -1)
    lat.init_fields(fields)
    lat.step(5)
    f, h = lat.populations()
    lat.close()
    assert np.array_equal(f, f_ref) and np.array_equal(h, h_ref)


def test_allocator_returning_null_gives_enomem(T):
    case, _ = W.random_periodic(64, 32, seed=1)
    params = T.params_from_case(case)
    alloc = T.ALLOC_FN(lambda nbytes, stream, ctx: None)
    free = T.FREE_FN(lambda ptr, nbytes, stream, ctx: None)
    with pytest.raises(T.TclbmError) as err:
        T.tclbm_create(params, alloc, free, None, None)
    assert err.value.status == T.ENOMEM


def test_non_finite_state_is_reported(T):
    case, fields = W.random_periodic(64, 32, seed=2)
    fields = {k: np.array(v) for k, v in fields.items()}
    fields["rho"][5, 7] = np.nan
    lat = T.Lattice(case, fields)
    lat.step(2)
    with pytest.raises(T.TclbmError) as err:
        lat.diagnostics()
    assert err.value.status == T.ENONFINITE
    lat.close()


@pytest.mark.parametrize("name,make", [
    ("rb_walls", lambda: W.rayleigh_benard(96, 48, Ra=2e4, seed=11)),
    ("periodic", lambda: W.random_periodic(70, 37, seed=12, force="accel")),
    ("x_ends", lambda: W.with_walls(*W.random_periodic(66, 10, seed=13), axis="x", kind="equilibrium")),
])
def test_resume_from_populations_equals_an_uninterrupted_run(T, name, make):
    # checkpoint = the populations read out; resume = a new handle set from them
    case, fields = make()
    whole = T.Lattice(case, fields)
    whole.step(40)
    f_ref, h_ref = whole.populations()
    whole.close()
    first = T.Lattice(case, fields)
    first.step(17)
    f, h = first.populations()
    first.close()
    second = T.Lattice(case)
    second.set_populations(f, h)
    second.step(23)
    f2, h2 = second.populations()
    second.close()
    assert np.array_equal(f2, f_ref) and np.array_equal(h2, h_ref)
