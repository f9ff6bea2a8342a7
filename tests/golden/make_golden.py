"""Writes the stored expected values that come from the FP64 oracle (and only from it).

    python tests/golden/make_golden.py

rb_128x64_nusselt.txt: Nusselt number (Section V.D definition, H = ny - 1,
kappa = nu / Pr, T0 = mean wall temperature) of Rayleigh-Benard convection on a
128 x 64 lattice, Ra = 1e4, Pr = 0.71, seeded temperature perturbation of amplitude
1e-2 (seed 1), after 60 000 and 80 000 time steps.

rb_256x128_nusselt.txt: the same on the 256 x 128 lattice of the bench workload
(perturbation amplitude 1e-4, seed 1, as the workload draws it), every 25 000 steps
up to 300 000.

table2_couette_oracle.txt: bottom-wall temperature of the paper's thermal Couette flow
(Section V.B, Table 2 rows: Pr = 5, 4; gamma = 5/3, 3/2; Ma = 0.35; 5 x 40 lattice)
after 60 000 steps.

    python tests/golden/make_golden.py [rb_128x64] [rb_256x128] [table2_couette_oracle]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1610_07114_gb300 import workloads as W  # noqa: E402


def nusselt(case, m):
    H = case["ny"] - 1
    kappa = case["visc"] / case["Pr"]
    dT = case["T_bot"] - case["T_top"]
    return 1.0 + np.mean(m["uy"] * (m["T"] - case["T0"])) * H / (kappa * dT)


def rb_128x64():
    case, fields = W.rayleigh_benard(128, 64, Ra=1e4, seed=1, amp=1e-2)
    o = oracle.Oracle(case, fields, threads=os.cpu_count())
    rows = []
    t0 = time.time()
    for steps, chunk in ((60000, 60000), (80000, 20000)):
        o.step(chunk)
        rows.append((steps, nusselt(case, o.moments())))
        print(f"  {steps} steps: Nu = {rows[-1][1]:.9f} ({time.time() - t0:.0f} s)", flush=True)
    with open(os.path.join(HERE, "rb_128x64_nusselt.txt"), "w") as fh:
        fh.write("# Nusselt number of the FP64 oracle: Rayleigh-Benard 128 x 64, Ra = 1e4, Pr = 0.71,\n")
        fh.write("# perturbation amplitude 1e-2 (seed 1); written by tests/golden/make_golden.py\n")
        fh.write("# columns: steps  Nu\n")
        for steps, nu in rows:
            fh.write(f"{steps} {nu:.12f}\n")


def rb_256x128():
    case, fields = W.rayleigh_benard(256, 128, Ra=1e4, seed=1)
    o = oracle.Oracle(case, fields, threads=os.cpu_count())
    rows = []
    t0 = time.time()
    for k in range(12):
        o.step(25000)
        rows.append(((k + 1) * 25000, nusselt(case, o.moments())))
        print(f"  {rows[-1][0]} steps: Nu = {rows[-1][1]:.9f} ({time.time() - t0:.0f} s)", flush=True)
    with open(os.path.join(HERE, "rb_256x128_nusselt.txt"), "w") as fh:
        fh.write("# Nusselt number of the FP64 oracle: Rayleigh-Benard 256 x 128, Ra = 1e4, Pr = 0.71,\n")
        fh.write("# perturbation amplitude 1e-4 (seed 1); written by tests/golden/make_golden.py\n")
        fh.write("# columns: steps  Nu\n")
        for steps, nu in rows:
            fh.write(f"{steps} {nu:.12f}\n")


def table2_couette_oracle():
    rows = []
    for Pr, gamma in ((5.0, 5.0 / 3.0), (5.0, 1.5), (4.0, 5.0 / 3.0), (4.0, 1.5)):
        case, fields = W.couette_paper(Pr=Pr, gamma=gamma)
        o = oracle.Oracle(case, fields, threads=4)
        o.step(60000)
        T_bottom = float(o.moments()["T"][0].mean())
        rows.append((Pr, gamma, T_bottom))
        print(f"  Pr {Pr:g} gamma {gamma:.4f}: T_bottom = {T_bottom:.9f}", flush=True)
    with open(os.path.join(HERE, "table2_couette_oracle.txt"), "w") as fh:
        fh.write("# Bottom-wall temperature of the FP64 oracle: thermal Couette flow of Section V.B (Table 2),\n")
        fh.write("# 5 x 40 lattice, Ma = 0.35, mu0 = 0.35, w2 = 1.1, w3 = 1.6, w4 = 0.3, 60 000 steps;\n")
        fh.write("# written by tests/golden/make_golden.py\n")
        fh.write("# columns: Pr  gamma  T_bottom\n")
        for Pr, gamma, Tb in rows:
            fh.write(f"{Pr:g} {gamma!r} {Tb:.12f}\n")


if __name__ == "__main__":
    which = sys.argv[1:] or ["rb_128x64", "rb_256x128", "table2_couette_oracle"]
    for name in which:
        globals()[name]()
