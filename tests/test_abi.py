"""The C ABI without a GPU: the library loads, exports every symbol include/tclbm.h
declares, and rejects invalid parameter sets before touching CUDA."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def T():
    from paper_1610_07114_gb300 import build

    build.build()
    from paper_1610_07114_gb300 import tclbm

    return tclbm


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "tclbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tclbm_[a-z_]+)\s*\(", text)) - {"tclbm_alloc_fn", "tclbm_free_fn"})


def test_header_declares_the_paper_entry_points():
    syms = declared_symbols()
    for s in ("tclbm_create", "tclbm_init_fields", "tclbm_step", "tclbm_moments", "tclbm_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(T):
    lib = T.library()
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def _valid_case():
    from paper_1610_07114_gb300 import workloads as W

    return W.rayleigh_benard(32, 16)[0]


@pytest.mark.parametrize("mutate,status", [
    (lambda c: c.update(nx=0), -1),
    (lambda c: c.update(gamma=1.0), -1),
    (lambda c: c.update(Pr=0.0), -1),
    (lambda c: c.update(w2=2.5), -1),
    (lambda c: c.update(thermal=False), -1),  # correction without thermal
    (lambda c: c.update(thermal=False, correction=False, work=True), -1),  # work term without thermal
    (lambda c: c["walls"]["y+"].update(kind="periodic"), -1),  # one side periodic, its opposite a wall
    (lambda c: [c["walls"][s].update(kind="nee") for s in ("x-", "x+")], -6),  # walls on both axes
    (lambda c: c.update(ny=2), -1),  # walled axis too short
])
def test_invalid_parameters_are_rejected_before_any_device_work(T, mutate, status):
    case = _valid_case()
    mutate(case)
    p = T.params_from_case(case)
    with pytest.raises(T.TclbmError) as ei:
        T.tclbm_create(p)
    assert ei.value.status == status
    assert T.tclbm_last_error() != ""


def test_state_bytes_counts_both_population_copies(T):
    case = _valid_case()
    p = T.params_from_case(case)
    n_pitch = 32 * 16  # pitch rounds nx up to 32
    assert T.tclbm_state_bytes(p) >= 2 * 18 * n_pitch * 4
    case["storage"] = "fp16"
    assert T.tclbm_state_bytes(T.params_from_case(case)) >= 2 * 18 * n_pitch * 2


def test_zero_flux_adiabatic_walls_are_refused_by_the_cuda_path(T):
    # the zero-flux adiabatic wall is a study option of the oracle only; a case asking for
    # it must not run silently with the CUDA path's zero-gradient walls
    from paper_1610_07114_gb300 import workloads as W

    case, _ = W.couette_paper()
    T.params_from_case(case)
    with pytest.raises(ValueError):
        T.params_from_case(dict(case, adiabatic="zero_flux"))
