"""Onset of Rayleigh-Benard convection (Section V.D): the critical Rayleigh number.

The paper extrapolates the growth of the total kinetic energy e = sum rho |u|^2 / 2
over several Rayleigh numbers to the one where it neither grows nor decays, and finds
1707.07 against the linear-stability value 1707.76 for rigid walls.  Here, on the
paper's 200 x 100 mesh with its 6 % temperature difference: the start is the conduction
profile plus the shape of the critical mode (workloads.rb_onset), and after the start-up
the exponential rate of e (from the device FP64 sums, every 20 000 steps over the second
half of 600 000 steps) is fitted linearly in Ra; its zero is Ra_c.  Paper-literal model:
no work term of the body force in the total-energy equation (Eq. 22), total-energy h for
the temperature; the layer is kept weakly stratified (u_c = 0.005, g H / (R T0) = 2.5e-3).
"""
import numpy as np
import pytest

from paper_1610_07114_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RA_C_THEORY = 1707.76  # rigid-rigid linear stability, quoted in Section V.D


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1610_07114_gb300 import build

    build.build()
    from paper_1610_07114_gb300 import tclbm

    return tclbm


def growth_rate(T, Ra, total=600000, every=20000):
    case, fields = W.rb_onset(Ra)
    lat = T.Lattice(case, fields)
    ts, es = [], []
    done = 0
    while done < total:
        lat.step(every)
        done += every
        ts.append(done)
        es.append(lat.diagnostics()[4])
    lat.close()
    ts, es = np.array(ts), np.array(es)
    half = len(ts) // 2
    return 0.5 * np.polyfit(ts[half:], np.log(es[half:]), 1)[0]  # e ~ exp(2 sigma t)


def test_critical_rayleigh_number(T):
    ras = np.array([1400.0, 1600.0, 1800.0, 2000.0, 2200.0])
    sig = np.array([growth_rate(T, ra) for ra in ras])
    print("growth rates", dict(zip(ras.tolist(), sig.tolist())))
    assert sig[0] < 0 < sig[-1]  # decays below onset, grows above
    assert np.all(np.diff(sig) > 0)
    p = np.polyfit(ras, sig, 1)
    ra_c = -p[1] / p[0]
    print("Ra_c %.1f (theory %.2f, paper 1707.07)" % (ra_c, RA_C_THEORY))
    assert abs(ra_c / RA_C_THEORY - 1.0) < 0.01
