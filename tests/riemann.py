"""Exact solution of the Riemann problem for the 1-D Euler equations of an ideal gas.

Written from the textbook method (E. F. Toro, "Riemann Solvers and Numerical
Methods for Fluid Dynamics", ch. 4): Newton iteration on the star pressure with
the shock / rarefaction pressure functions, then sampling of the self-similar
solution.  Used to pin the oracle's low-Mach shock tube (Section V.C of the paper
compares against this solution).
"""
import math

import numpy as np


def _fK(p, rhoK, pK, cK, g):
    if p > pK:  # shock
        A = 2.0 / ((g + 1.0) * rhoK)
        B = (g - 1.0) / (g + 1.0) * pK
        f = (p - pK) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - (p - pK) / (2.0 * (B + p)))
    else:  # rarefaction
        f = 2.0 * cK / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rhoK * cK) * (p / pK) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rhoL, uL, pL, rhoR, uR, pR, g):
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    p = 0.5 * (pL + pR)
    for _ in range(100):
        fL, dL = _fK(p, rhoL, pL, cL, g)
        fR, dR = _fK(p, rhoR, pR, cR, g)
        dp = (fL + fR + uR - uL) / (dL + dR)
        p = max(1e-12, p - dp)
        if abs(dp) < 1e-14 * p:
            break
    fL, _ = _fK(p, rhoL, pL, cL, g)
    fR, _ = _fK(p, rhoR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def sample(x_over_t, rhoL, uL, pL, rhoR, uR, pR, g):
    """(rho, u, p) of the exact solution at similarity coordinate x/t (array)."""
    ps, us = star_state(rhoL, uL, pL, rhoR, uR, pR, g)
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    gm = (g - 1.0) / (g + 1.0)
    out = np.zeros((3, len(x_over_t)))
    for i, s in enumerate(np.asarray(x_over_t, dtype=float)):
        if s <= us:  # left of contact
            if ps > pL:
                rs = rhoL * ((ps / pL + gm) / (gm * ps / pL + 1.0))
                SL = uL - cL * math.sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
                st = (rhoL, uL, pL) if s <= SL else (rs, us, ps)
            else:
                rs = rhoL * (ps / pL) ** (1.0 / g)
                cs = cL * (ps / pL) ** ((g - 1.0) / (2.0 * g))
                SH, ST = uL - cL, us - cs
                if s <= SH:
                    st = (rhoL, uL, pL)
                elif s >= ST:
                    st = (rs, us, ps)
                else:
                    c = 2.0 / (g + 1.0) * (cL + (g - 1.0) / 2.0 * (uL - s))
                    st = (rhoL * (c / cL) ** (2.0 / (g - 1.0)), 2.0 / (g + 1.0) * (cL + (g - 1.0) / 2.0 * uL + s),
                          pL * (c / cL) ** (2.0 * g / (g - 1.0)))
        else:
            if ps > pR:
                rs = rhoR * ((ps / pR + gm) / (gm * ps / pR + 1.0))
                SR = uR + cR * math.sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
                st = (rhoR, uR, pR) if s >= SR else (rs, us, ps)
            else:
                rs = rhoR * (ps / pR) ** (1.0 / g)
                cs = cR * (ps / pR) ** ((g - 1.0) / (2.0 * g))
                SH, ST = uR + cR, us + cs
                if s >= SH:
                    st = (rhoR, uR, pR)
                elif s <= ST:
                    st = (rs, us, ps)
                else:
                    c = 2.0 / (g + 1.0) * (cR - (g - 1.0) / 2.0 * (uR - s))
                    st = (rhoR * (c / cR) ** (2.0 / (g - 1.0)), 2.0 / (g + 1.0) * (-cR + (g - 1.0) / 2.0 * uR + s),
                          pR * (c / cR) ** (2.0 * g / (g - 1.0)))
        out[:, i] = st
    return out
