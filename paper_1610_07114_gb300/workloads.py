"""Seeded synthetic workloads for the thermal cascaded LBM (Fei & Luo, arXiv:1610.07114).

This module is the only code shared by the CUDA path and the FP64 oracle.  It
holds problem set-up only -- lattice sizes, physical parameters, boundary
descriptions and initial macroscopic fields -- and none of the method's
arithmetic (no equilibria, no relaxation rates, no moments).  Each side turns a
case dict into its own parameter struct.

Case dict vocabulary (names follow the paper's notation):

    nx, ny            lattice nodes; x fastest in every [ny][nx] array
    thermal           True: total-energy distribution h evolved (Section IV)
                      False: athermal cascaded LBM with T = T0 (Sections II-III)
    correction        True: correction term C_a of Section IV included
    visc_law, visc    "nu" kinematic viscosity | "mu" dynamic viscosity |
                      "mu_T" mu = visc * T/T0 | "w1" fixed w1 (Eq. 29)
    w2, w3, w4        Eq. 8 rates; w_equal=True sets all four equal to w1 (BGK limit)
    Pr, gamma, R, T0  Prandtl number, specific-heat ratio, gas constant, reference T
    force             {"kind": "none"} | {"kind": "accel", "ax", "ay"} (F = rho a) |
                      {"kind": "taylor_green", "amp"}: F = amp (sin kx sin ky, cos kx cos ky)
    walls             {"x-","x+","y-","y+"} -> {"kind": "periodic"|"zouhe"|"nee"|"equilibrium",
                      "ux", "uy", "T", "rho", "therm": "fixed"|"adiabatic"}
    work              True: the body force's power F.u enters the total energy (an extension;
                      the paper's Eq. 22 has no force term)
    storage           "fp32" | "bf16" | "fp16" population storage of the CUDA path
    U_ref, rho_scale, T_scale
                      the case's own scales of velocity, density variation and temperature
                      variation (wall speed, imposed jumps, hydrostatic or heating
                      amplitudes): comparisons of fields normalise by them where a field
                      is nearly uniform
"""
from __future__ import annotations

import copy
import math

import numpy as np

# Gas constant in lattice units.  Section V.C normalises p0 = rho0 R T0 = 1/3, but with
# the local temperature in the total-energy equilibrium the D2Q9 scheme's linearised
# step then grows grid-scale two-dimensional modes (k = (pi, pi)) by a factor 1.8-4.8
# per step for every w1; R T0 <= 0.18 is stable for w1 <= 1.8.  Thermal cases therefore
# take R T0 = 1/6 (the correction term then cancels the defect rho u (1 - 3RT)); the
# athermal cascaded LBM (c_s^2 = R T0 = 1/3) and the paper's odd-width one-dimensional
# Couette case keep R = 1/3.
R_DEFAULT = 1.0 / 6.0
R_PAPER = 1.0 / 3.0
SIDES = ("x-", "x+", "y-", "y+")


def _periodic():
    return {"kind": "periodic", "ux": 0.0, "uy": 0.0, "T": 1.0, "rho": 1.0, "therm": "fixed"}


def _wall(kind, ux=0.0, uy=0.0, T=1.0, rho=1.0, therm="fixed"):
    return {"kind": kind, "ux": float(ux), "uy": float(uy), "T": float(T), "rho": float(rho), "therm": therm}


def base_case(nx, ny, **kw):
    case = {
        "name": "custom",
        "nx": int(nx),
        "ny": int(ny),
        "thermal": True,
        "correction": True,
        "visc_law": "nu",
        "visc": 0.05,
        "w2": 1.0,
        "w3": 1.0,
        "w4": 1.0,
        "w_equal": False,
        "Pr": 0.71,
        "gamma": 1.4,
        "R": R_DEFAULT,
        "T0": 1.0,
        "force": {"kind": "none", "ax": 0.0, "ay": 0.0, "amp": 0.0},
        "walls": {s: _periodic() for s in SIDES},
        "storage": "fp32",
    }
    for k, v in kw.items():
        case[k] = v
    return case


def uniform_fields(nx, ny, rho=1.0, ux=0.0, uy=0.0, T=1.0):
    shape = (ny, nx)
    return {
        "rho": np.full(shape, float(rho)),
        "ux": np.full(shape, float(ux)),
        "uy": np.full(shape, float(uy)),
        "T": np.full(shape, float(T)),
    }


# --------------------------------------------------------------------------- paper cases


def couette(nx=8, ny=64, U=0.05, nu=0.05, Pr=0.71, gamma=1.4, T_wall=1.0, storage="fp32", fields=True):
    """Thermal Couette flow with viscous heating (Section V.B set-up, isothermal walls).

    Periodic in x; y = 0 is a wall at rest and y = ny-1 moves with u = (U, 0); both
    walls use non-equilibrium bounce-back for velocity and non-equilibrium
    extrapolation for temperature (Section V.B), at T = T_wall.  Initial state rho = 1,
    u = 0, T = T_wall.  With constant mu and lambda the steady temperature is
    T = T_wall + Pr U^2 / (2 c_p) eta (1 - eta), eta = y / (ny - 1).
    """
    case = base_case(nx, ny, name=f"couette_{nx}x{ny}", visc_law="nu", visc=nu, Pr=Pr, gamma=gamma,
                     storage=storage)
    case["walls"]["y-"] = _wall("zouhe", 0.0, 0.0, T_wall)
    case["walls"]["y+"] = _wall("zouhe", U, 0.0, T_wall)
    case["U"] = U
    case["U_ref"] = U
    # peak viscous heating Pr U^2 / (8 c_p), c_p = R (b + 2) / 2; at uniform pressure the
    # density varies by the same fraction
    b = 2.0 / (gamma - 1.0)
    case["T_scale"] = Pr * U * U / (8.0 * case["R"] * (b + 2.0) / 2.0) * T_wall
    case["rho_scale"] = case["T_scale"] / T_wall
    return case, (uniform_fields(nx, ny, T=T_wall) if fields else None)


def couette_paper(Pr=5.0, gamma=5.0 / 3.0, nx=5, ny=40, Ma=0.35, mu0=0.35):
    """The paper's thermal Couette variant (Section V.B, Table 2): top wall moving at
    U = Ma sqrt(gamma R T0) with T = T0, bottom wall fixed and adiabatic, mu/mu0 = T/T0,
    w2 = 1.1, w3 = 1.6, w4 = 0.3."""
    U = Ma * math.sqrt(gamma * R_PAPER * 1.0)
    case = base_case(nx, ny, name=f"couette_paper_Pr{Pr}_g{gamma:.3f}", visc_law="mu_T", visc=mu0, Pr=Pr,
                     gamma=gamma, w2=1.1, w3=1.6, w4=0.3, R=R_PAPER)
    case["walls"]["y-"] = _wall("zouhe", 0.0, 0.0, 1.0, therm="adiabatic")
    case["walls"]["y+"] = _wall("zouhe", U, 0.0, 1.0)
    case["U"] = U
    case["U_ref"] = U
    case["Ma"] = Ma
    b = 2.0 / (gamma - 1.0)
    case["T_scale"] = Pr * U * U / (2.0 * R_PAPER * (b + 2.0) / 2.0)  # adiabatic-wall heating
    case["rho_scale"] = case["T_scale"]
    return case, uniform_fields(nx, ny)


def rb_gravity(Ra, ny, Pr=0.71, dT=0.02, u_c=0.03, T0=1.0):
    """Gravity and viscosity of a Rayleigh-Benard layer (Section V.D):
    Ra = g beta dT H^3 Pr / nu^2, u_c = sqrt(g beta dT H), beta = 1/T0, H = ny - 1."""
    H = ny - 1
    beta = 1.0 / T0
    g = u_c * u_c / (beta * dT * H)
    nu = math.sqrt(g * beta * dT * H ** 3 * Pr / Ra)
    return g, nu


def rayleigh_benard(nx=256, ny=128, Ra=1e4, Pr=0.71, gamma=1.4, T_bot=1.01, T_top=0.99, u_c=0.03,
                    seed=1, amp=1e-4, storage="fp32", fields=True):
    """Rayleigh-Benard convection with gravity as a direct body force (Section V.D).

    Periodic in x; walls at y = 0 (hot) and y = ny-1 (cold), at rest.  Velocity walls
    use non-equilibrium bounce-back and temperature walls non-equilibrium
    extrapolation (the Section V.B pairing): extrapolating the density as well lets
    mass through a wall under the body force.  Initial T: linear between the walls
    plus a seeded uniform perturbation of amplitude `amp` in the interior; initial
    rho: the discrete hydrostatic profile of that mean T, normalised to mean 1.
    """
    T0 = 0.5 * (T_bot + T_top)
    g, nu = rb_gravity(Ra, ny, Pr, T_bot - T_top, u_c, T0)
    case = base_case(nx, ny, name=f"rb_{nx}x{ny}_Ra{Ra:g}", visc_law="nu", visc=nu, Pr=Pr, gamma=gamma,
                     T0=T0, storage=storage)
    case["force"] = {"kind": "accel", "ax": 0.0, "ay": -g, "amp": 0.0}
    case["walls"]["y-"] = _wall("zouhe", 0.0, 0.0, T_bot)
    case["walls"]["y+"] = _wall("zouhe", 0.0, 0.0, T_top)
    case["T_ref"] = T0
    case["Ra"] = Ra
    case["g"] = g
    case["U_ref"] = u_c
    case["T_scale"] = T_bot - T_top
    case["rho_scale"] = g * (ny - 1) / (case["R"] * T0)  # hydrostatic variation across the layer
    case["T_bot"], case["T_top"] = T_bot, T_top
    if not fields:
        return case, None
    rng = np.random.default_rng(seed)
    y = np.arange(ny, dtype=np.float64)
    Tcol = T_bot + (T_top - T_bot) * y / (ny - 1)
    R = case["R"]
    rho_col = np.empty(ny)
    rho_col[0] = 1.0
    for j in range(ny - 1):  # p = rho R T, (p_{j+1} - p_j) = -g (rho_j + rho_{j+1}) / 2
        rho_col[j + 1] = rho_col[j] * (R * Tcol[j] - 0.5 * g) / (R * Tcol[j + 1] + 0.5 * g)
    rho_col /= rho_col.mean()
    T = np.repeat(Tcol[:, None], nx, axis=1)
    pert = rng.uniform(-amp, amp, size=(ny, nx))
    pert[0, :] = 0.0
    pert[-1, :] = 0.0
    T = T + pert
    out = {
        "rho": np.repeat(rho_col[:, None], nx, axis=1).copy(),
        "ux": np.zeros((ny, nx)),
        "uy": np.zeros((ny, nx)),
        "T": T,
    }
    return case, out


def rb_onset(Ra, nx=200, ny=100, dT=0.06, u_c=0.005, amp=1e-2, storage="fp32"):
    """Rayleigh-Benard layer for the onset of convection (Section V.D: the 200 x 100 mesh
    and the 6 % temperature difference of the paper): u_c = 0.005 keeps the layer weakly
    stratified (g H / (R T0) = 2.5e-3) with w1 <= 1.8 near Ra = 1708, and the start is the
    linear conduction profile plus the shape of the critical mode,
    T' = amp dT sin(pi y / H) cos(2 pi x / nx) (one wavelength across nx = 2 H, wave number
    close to the critical 3.117 / H)."""
    case, fields = rayleigh_benard(nx, ny, Ra=Ra, T_bot=1.0 + dT / 2, T_top=1.0 - dT / 2, u_c=u_c, seed=0, amp=0.0,
                                   storage=storage)
    y = np.arange(ny)[:, None]
    x = np.arange(nx)[None, :]
    fields["T"] = fields["T"] + amp * dT * np.sin(np.pi * y / (ny - 1)) * np.cos(2 * np.pi * x / nx)
    case["name"] = f"rb_onset_{nx}x{ny}_Ra{Ra:g}"
    return case, fields


TABLE3_MESH = {2500: 80, 5000: 80, 10000: 100, 30000: 100, 50000: 150}  # N_y of the paper's Table 3 runs


def rb_table3(Ra, dT=0.06, w1=1.78, seed=3, amp=1e-2, storage="fp32"):
    """Rayleigh-Benard layer of Table 3 (Section V.D): aspect ratio 2:1 on the paper's mesh
    for this Ra (TABLE3_MESH), its 6 % temperature difference, and the smallest u_c that
    keeps w1 at `w1` (nu = R T0 (1/w1 - 1/2), u_c = nu sqrt(Ra / Pr) / H): a weakly
    stratified layer (g H / (R T0) = 0.006 .. 0.05)."""
    ny = TABLE3_MESH[int(Ra)]
    nu = R_DEFAULT * 1.0 * (1.0 / w1 - 0.5)
    u_c = nu * math.sqrt(Ra / 0.71) / (ny - 1)
    case, fields = rayleigh_benard(2 * ny, ny, Ra=Ra, T_bot=1.0 + dT / 2, T_top=1.0 - dT / 2, u_c=max(u_c, 0.005),
                                   seed=seed, amp=amp, storage=storage)
    case["name"] = f"rb_table3_Ra{Ra:g}"
    return case, fields


def shock_tube(nx=4096, ny=4, rho_l=1.05, rho_r=1.0, T=1.0, w1=1.887, storage="fp32"):
    """Low-Mach shock tube (Section V.C): periodic in y, equilibrium distributions at
    x = 0 and x = nx-1 with the initial end states; gamma = 1.4, Pr = 0.71,
    w2 = w3 = w4 = 1.  The paper's w1 = 1.887 at its R T0 = 1/3 fixes the kinematic
    viscosity nu = (1/3)(1/w1 - 1/2); that viscosity is kept (w1 = 1.786 at R T0 = 1/6)."""
    nu = R_PAPER * (1.0 / w1 - 0.5)
    case = base_case(nx, ny, name=f"shock_{nx}x{ny}", visc_law="nu", visc=nu, Pr=0.71, gamma=1.4,
                     storage=storage)
    case["walls"]["x-"] = _wall("equilibrium", 0.0, 0.0, T, rho_l)
    case["walls"]["x+"] = _wall("equilibrium", 0.0, 0.0, T, rho_r)
    f = uniform_fields(nx, ny, T=T)
    f["rho"][:, : nx // 2] = rho_l
    f["rho"][:, nx // 2:] = rho_r
    case["rho_l"], case["rho_r"] = rho_l, rho_r
    # velocity scale of the weak waves: c_s d(rho)/rho with c_s = sqrt(gamma R T)
    case["U_ref"] = math.sqrt(1.4 * case["R"] * T) * abs(rho_l - rho_r) / (rho_l + rho_r) * 2.0
    case["rho_scale"] = abs(rho_l - rho_r)
    # adiabatic temperature change of the same density jump: (gamma - 1) T d(rho) / rho
    case["T_scale"] = (1.4 - 1.0) * T * abs(rho_l - rho_r) / (0.5 * (rho_l + rho_r))
    return case, f


def taylor_green(n=64, F0=1e-5, nu=0.02, thermal=False, storage="fp32", fields=True):
    """Steady forced Taylor-Green flow (Section V.A): periodic N x N lattice, node i at
    x = i * 2 pi / N, F = F0 (sin x sin y, cos x cos y), rho = 1 and u = 0 initially,
    w1 = w2 = w3 = w4 (BGK limit).  Closed form u = u0 (sin x sin y, cos x cos y) with
    u0 = F0 / (2 nu k^2), k = 2 pi / N."""
    case = base_case(n, n, name=f"tg_{n}", thermal=thermal, correction=thermal, visc_law="nu", visc=nu,
                     w_equal=True, storage=storage, R=R_DEFAULT if thermal else R_PAPER)
    case["force"] = {"kind": "taylor_green", "ax": 0.0, "ay": 0.0, "amp": F0}
    k = 2.0 * math.pi / n
    case["u0"] = F0 / (2.0 * nu * k * k)
    case["U_ref"] = case["u0"]
    # dynamic pressure over the squared sound speed; kinetic energy over c_p
    case["rho_scale"] = case["u0"] ** 2 / (case["R"] * case["T0"])
    b = 2.0 / (case["gamma"] - 1.0)
    case["T_scale"] = case["u0"] ** 2 / (case["R"] * (b + 2.0) / 2.0)
    return case, (uniform_fields(n, n) if fields else None)


def taylor_green_fields(n, u0):
    """Closed-form steady Taylor-Green velocity at the nodes (Section V.A)."""
    k = 2.0 * math.pi / n
    x = np.arange(n) * k
    X, Y = np.meshgrid(x, x, indexing="xy")  # arrays [y][x]
    return u0 * np.sin(X) * np.sin(Y), u0 * np.cos(X) * np.cos(Y)


def random_periodic(nx, ny, seed=0, thermal=True, force="accel", amp_rho=1e-2, amp_u=2e-2, amp_T=1e-2,
                    visc=0.03, storage="fp32", correction=None):
    """Seeded random smooth-ish state on a fully periodic lattice, for parity checks."""
    rng = np.random.default_rng(seed)
    case = base_case(nx, ny, name=f"rand_{nx}x{ny}_s{seed}", thermal=thermal,
                     correction=thermal if correction is None else correction, visc_law="nu", visc=visc,
                     w2=1.2, w3=1.1, w4=0.9, storage=storage)
    if force == "accel":
        case["force"] = {"kind": "accel", "ax": 1e-5, "ay": -2e-5, "amp": 0.0}
    elif force == "taylor_green":
        case["force"] = {"kind": "taylor_green", "ax": 0.0, "ay": 0.0, "amp": 1e-5}

    def field(amp):
        a = rng.uniform(-1.0, 1.0, size=(ny, nx))
        # one pass of a 5-point average keeps gradients moderate
        a = (a + np.roll(a, 1, 0) + np.roll(a, -1, 0) + np.roll(a, 1, 1) + np.roll(a, -1, 1)) / 5.0
        return amp * a

    case["U_ref"] = amp_u
    case["rho_scale"] = amp_rho
    case["T_scale"] = amp_T
    fields = {
        "rho": 1.0 + field(amp_rho),
        "ux": field(amp_u),
        "uy": field(amp_u),
        "T": 1.0 + (field(amp_T) if thermal else 0.0),
    }
    return case, fields


def with_walls(case, fields, axis="y", kind="nee", seed=0):
    """Copy of a random case with walls on one axis (for boundary parity checks)."""
    case = copy.deepcopy(case)
    lo, hi = ("y-", "y+") if axis == "y" else ("x-", "x+")
    rng = np.random.default_rng(seed + 17)
    if kind == "zouhe":
        t = "ux" if axis == "y" else "uy"
        u_lo, u_hi = {t: 0.0}, {t: 0.03}
    else:
        u_lo, u_hi = {}, {}
    case["walls"][lo] = _wall(kind, T=1.0 + 0.01 * rng.uniform(), rho=1.02, **u_lo)
    case["walls"][hi] = _wall(kind, T=1.0 - 0.01 * rng.uniform(), rho=0.99, **u_hi)
    case["name"] += f"_{axis}{kind}"
    return case, fields


# --------------------------------------------------------------------------- growth workloads


def rb_max_resolved_ra(ny, u_c=0.03, Pr=0.71, w1_max=1.8, RT0=R_DEFAULT):
    """Largest Rayleigh number a layer of ny rows resolves: the one whose viscosity
    (rb_gravity) puts w1 = 1 / (nu / RT0 + 1/2) at w1_max.  Ra = Pr (u_c H / nu)^2.
    Above w1 ~ 1.9 the FP64 oracle itself diverges within a few hundred steps
    (128 x 64 and 256 x 128 layers, u_c = 0.03 and 0.08); at w1 = 1.8 it runs through
    the onset into steady convection (64 x 32 and 128 x 64, 40 000 steps)."""
    nu_min = RT0 * (1.0 / w1_max - 0.5)
    return Pr * (u_c * (ny - 1) / nu_min) ** 2


def batched_rb_sweep(count=256, seed=1234, sizes=((64, 32), (128, 64), (256, 128), (512, 256), (1024, 512)),
                     ra_lo=2e3, ra_hi=1e6, storage="fp16"):
    """Batched Rayleigh-Benard sweep: `count` independent lattices, sizes uniform over
    `sizes` (aspect 2:1), Ra log-uniform in [ra_lo, ra_hi] and capped at the lattice's
    rb_max_resolved_ra (the drawn value is kept as case["Ra_drawn"]), Pr = 0.71."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx, ny = sizes[int(rng.integers(len(sizes)))]
        Ra = float(math.exp(rng.uniform(math.log(ra_lo), math.log(ra_hi))))
        case, fields = rayleigh_benard(nx, ny, Ra=min(Ra, rb_max_resolved_ra(ny)), seed=seed + i, storage=storage)
        case["Ra_drawn"] = Ra
        out.append((case, fields))
    return out


def serving_trace(duration_s=2.0, rate=200.0, seed=42, scale=1.0, max_nodes=None, steps_choices=(200, 500, 1000, 2000),
                  steady_frac=0.0, steady_residual=1e-8):
    """Poisson-arriving requests (mean `rate`/s) mixing thermal Couette (32 x 128),
    forced Taylor-Green (256^2 .. 2048^2) and Rayleigh-Benard (128x64 .. 4096x2048,
    Ra log-uniform up to 1e7, capped at rb_max_resolved_ra of the lattice).  Each request
    asks for a fixed step count drawn from `steps_choices`, except a share `steady_frac`
    of the Couette requests, which ask for the steady state: the residual E_R (Section
    V.A) below `steady_residual` (those take nu = 0.3, whose slowest shear mode on
    32 x 128 e-folds in ~5400 steps).  `scale` shrinks lattice sides (for small test
    runs); `max_nodes` caps lattice size."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration_s:
            break
        kind = int(rng.integers(3))
        if kind == 0:
            nx, ny = 32, 128
            case, fields = None, None
            spec = ("couette", nx, ny, {})
        elif kind == 1:
            n = int(2 ** rng.integers(8, 12))
            spec = ("taylor_green", n, n, {})
        else:
            e = int(rng.integers(7, 13))
            nx = 2 ** e
            Ra = float(math.exp(rng.uniform(math.log(2e3), math.log(1e7))))
            spec = ("rayleigh_benard", nx, nx // 2, {"Ra_drawn": Ra})
        name, nx, ny, extra = spec
        nx = max(8, int(nx * scale))
        ny = max(8, int(ny * scale))
        if max_nodes is not None:
            while nx * ny > max_nodes:
                nx //= 2
                ny //= 2
        if "Ra_drawn" in extra:  # capped at what the (possibly scaled) lattice resolves
            extra["Ra"] = min(extra["Ra_drawn"], rb_max_resolved_ra(ny))
        steps = int(rng.choice(list(steps_choices)))
        r = {"t_arrival": t, "kind": name, "nx": nx, "ny": ny, "steps": steps, "seed": len(reqs), **extra}
        if name == "couette" and steady_frac > 0 and rng.uniform() < 3.0 * steady_frac:
            r.update(steps=None, residual=steady_residual, nu=0.3)
        reqs.append(r)
    return reqs


def build_request(req, storage="fp16", fields=True):
    """Case and initial fields of one serving request (fields None with fields=False:
    a long trace builds each request's fields only when it is admitted)."""
    if req["kind"] == "couette":
        return couette(req["nx"], req["ny"], nu=req.get("nu", 0.05), storage=storage, fields=fields)
    if req["kind"] == "taylor_green":
        n = req["nx"]
        F0 = 1e-5 * (64.0 / n) ** 2  # keeps u0 at the Section V.A value of 0.026
        return taylor_green(n, F0=F0, nu=0.02, thermal=True, storage=storage, fields=fields)
    return rayleigh_benard(req["nx"], req["ny"], Ra=req.get("Ra", 1e4), seed=req["seed"], storage=storage,
                           fields=fields)
