/*
 * tclbm_oracle.c -- plain, slow FP64 CPU oracle of the thermal cascaded lattice
 * Boltzmann method (TCLBM) of Fei & Luo, "Thermal cascaded lattice Boltzmann
 * method" (arXiv:1610.07114), on the D2Q9 lattice.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py may load this library.  It shares no code, header,
 * table or helper with the CUDA path in paper_1610_07114_gb300/csrc; the two meet
 * only in the seeded initial fields that both receive.
 *
 * Everything is written in the paper's order and notation, one node at a time,
 * with no fusion or reordering:
 *   Section II   D2Q9 set, raw moments (Eq. 1-2), Eq. 3 (populations from raw
 *                moments), central moments by definition (Eq. 4), cascaded
 *                relaxation (Eq. 8), binomial back-transform (Eq. 9), streaming.
 *   Section III  transformed distribution f_bar = f - S/2 (Eq. 12), source moments
 *                (Eq. 15 and the raw list after it), forced post-collision raw
 *                moments (Eq. 18), macroscopic variables (Eq. 20).
 *   Section IV   thermal f^eq (Eq. 7 with local T), correction term C_a and its
 *                moments, Eq. 27, shifted equilibria for f_bar, viscosities
 *                (Eq. 29), total-energy equilibrium h^eq, transformed h_bar and
 *                K_a, the discrete h update, w_h and tau_hf, temperature.
 *   Section V    boundary schemes named there: periodic, non-equilibrium
 *                bounce-back (Zou-He) for velocity walls, non-equilibrium
 *                extrapolation for velocity and temperature walls, equilibrium
 *                distributions at open ends.
 *
 * Readings taken where the paper is silent or garbled (each also applies to the
 * CUDA path, which is written independently):
 *   - Eq. 6 / Section IV: the Maxwellian exponent "2 pi R T" is read as 2 R T;
 *     Eq. 7's values (E~eq = 2RT, M~22eq = (RT)^2) confirm it.
 *   - R = 1/3 and T0 = 1 by default (Section V.C: p0 = rho0 R T0 = 1/3).
 *   - Correction moments are normalised like Eq. 1: C_a = Eq. 3(rho, M^c) with
 *     E^c = d_x[u_x(1-theta)] + d_y[u_y(1-theta)], ...; theta = 3 R T, which is the
 *     paper's T/T0 when 3 R T0 = 1 (the defect it cancels is rho u (1 - 3RT - u^2)).
 *   - R is a parameter.  At the paper's R T0 = 1/3 the thermal scheme's linearised
 *     step amplifies the two-dimensional grid-scale mode k = (pi, pi); thermal
 *     two-dimensional cases run at R T0 = 1/6, the athermal scheme keeps 1/3.
 *   - Derivatives in C_a are taken at the same time level as the collision, by
 *     second-order central differences; at a wall node the wall-normal one is the
 *     one-sided second-order difference (-3 phi_0 + 4 phi_1 - phi_2)/2.
 *   - Eq. 18 first line: Pi_bar is read as the post-collision Pi_bar^*.
 *   - K_a uses f_bar_a (the subscript is missing in the paper).
 *   - lambda = mu c_p / Pr with c_p = R(b+2)/2, so 1/w_h = (1/w1 - 1/2)/Pr + 1/2;
 *     1/tau_hf = (Pr - 1)/(mu/p + 1/2) = (Pr - 1) w1 (finite at Pr = 1).
 *   - Initial state: f_bar = f^eq - S/2 (C = 0 at t = 0), h_bar = h^eq, so that
 *     Eq. 20 returns the prescribed fields.
 *   - Optional work term (not in the paper, whose total-energy equation Eq. 22 has no
 *     force term): the power of the body force F.u enters the h update as a source
 *     q_a = W_a F.u (D2Q9 weights, zeroth moment F.u, first moment zero) with the factor
 *     (1 - w_h/2), and the energy moment carries half a step of it, rho E =
 *     sum h_bar + F.u / 2, as Eq. 20 does for the momentum.  Initial h_bar = h^eq - q/2.
 *   - Adiabatic temperature walls (Section V.B names non-equilibrium extrapolation
 *     without saying how an adiabatic wall picks its temperature): T_w = T_f, the
 *     interior neighbour's temperature.  This zero-gradient choice is first order: at
 *     a wall at rest beside a sheared layer the total-energy distribution carries the
 *     flux mu u_f^2 / 2 of total enthalpy into the wall node each step and the rebuild
 *     removes it.  A study option (adiabatic_flux) takes instead the temperature at
 *     which conduction and viscous work across that link cancel.
 *   - Walls are "wet": the wall lies on the first/last node row (or column); the
 *     boundary scheme rebuilds that node's populations after streaming and the
 *     node then collides like any other.  Zou-He is written for transformed
 *     populations with the force terms kept (see wall_rebuild()).  Walls may sit
 *     on one axis only (x or y); the other axis is periodic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9
#define PI_ 3.14159265358979323846

/* Section II: e_0 = (0,0); e_a = (cos((a-1)pi/2), sin((a-1)pi/2)) for a = 1..4;
 * e_a = sqrt(2) (cos((a-9/2)pi/2), sin((a-9/2)pi/2)) for a = 5..8; c = 1. */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* D2Q9 weights (zeroth moment 1, first moment 0): the shape of the work source. */
static const double WQ[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

enum { SIDE_XM = 0, SIDE_XP = 1, SIDE_YM = 2, SIDE_YP = 3 };
enum { WALL_PERIODIC = 0, WALL_ZOUHE = 1, WALL_NEE = 2, WALL_EQUILIBRIUM = 3 };
enum { THERM_FIXED_T = 0, THERM_ADIABATIC = 1 };
enum { VISC_CONST_NU = 0, VISC_CONST_MU = 1, VISC_MU_PROP_T = 2, VISC_FIXED_W1 = 3 };
enum { FORCE_NONE = 0, FORCE_UNIFORM_ACCEL = 1, FORCE_TAYLOR_GREEN = 2 };

/* Inward unit normal of each side. */
static const int NRM_X[4] = {1, -1, 0, 0};
static const int NRM_Y[4] = {0, 0, 1, -1};

typedef struct {
    int32_t nx, ny;
    int32_t thermal;     /* 1: total-energy distribution h evolved (Section IV); 0: athermal CLBM, T = T0 */
    int32_t correction;  /* 1: correction term C_a of Section IV included */
    int32_t visc_law;    /* VISC_*: how w1 follows from the viscosity (Eq. 29) */
    double visc;         /* nu, mu, mu0 or w1, by visc_law */
    double w2, w3, w4;   /* Eq. 8 rates for E, (M21, M12), M22 */
    double Pr, gamma, R, T0;
    int32_t force_kind;  /* FORCE_* */
    double ax, ay;       /* FORCE_UNIFORM_ACCEL: F = rho (ax, ay) */
    double famp;         /* FORCE_TAYLOR_GREEN: F = famp (sin kx sin ky, cos kx cos ky), k = 2 pi / n */
    int32_t wall_kind[4];   /* per side x-, x+, y-, y+ : WALL_* */
    int32_t wall_therm[4];  /* THERM_* for the h populations of a wall */
    double wall_rho[4], wall_ux[4], wall_uy[4], wall_T[4];
    int32_t work;        /* 1: the body force's power F.u as a source of total energy (an extension:
                            the paper's Eq. 22 has none) */
    int32_t adiabatic_flux; /* adiabatic walls: 0 zero gradient, T_w = T_f (the reading both paths
                               take); 1 zero total-energy flux across the first link (a study of
                               that reading, oracle only: the CUDA path has no such option) */
} oracle_params;

typedef struct { double rho, ux, uy, T, Fx, Fy, ax, ay; } macro_t;

static int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }
static size_t at(const oracle_params* p, int a, int x, int y) {
    return ((size_t)a * p->ny + y) * p->nx + x;
}
static double b_dof(const oracle_params* p) { return 2.0 / (p->gamma - 1.0); } /* gamma = (b+2)/b */
static int x_periodic(const oracle_params* p) { return p->wall_kind[SIDE_XM] == WALL_PERIODIC; }
static int y_periodic(const oracle_params* p) { return p->wall_kind[SIDE_YM] == WALL_PERIODIC; }

/* ---------------------------------------------------------------- Section II */

/* Eq. 3: populations from the nine raw moments {M00, M10, M01, E, N, Pi, M21, M12, M22}
 * (normalised by rho as in Eq. 1).  The same form serves S_a, C_a and h^eq. */
void oracle_pop_from_moments(double rho, const double M[9], double out[9]) {
    const double M00 = M[0], M10 = M[1], M01 = M[2], E = M[3], N = M[4], Pi = M[5];
    const double M21 = M[6], M12 = M[7], M22 = M[8];
    out[0] = rho * (M00 - E + M22);
    out[1] = 0.5 * rho * (M10 + 0.5 * (E + N) - M12 - M22);
    out[2] = 0.5 * rho * (M01 + 0.5 * (E - N) - M21 - M22);
    out[3] = 0.5 * rho * (-M10 + 0.5 * (E + N) + M12 - M22);
    out[4] = 0.5 * rho * (-M01 + 0.5 * (E - N) + M21 - M22);
    out[5] = 0.25 * rho * (Pi + M21 + M12 + M22);
    out[6] = 0.25 * rho * (-Pi + M21 - M12 + M22);
    out[7] = 0.25 * rho * (Pi - M21 - M12 + M22);
    out[8] = 0.25 * rho * (-Pi - M21 + M12 + M22);
}

/* Eq. 4: central moment rho M~_pq = sum_a f_a (e_ax - ux)^p (e_ay - uy)^q, returned / rho. */
static double central_moment(const double f[9], double rho, double ux, double uy, int p, int q) {
    double s = 0.0;
    for (int a = 0; a < Q; ++a) {
        double cx = EX[a] - ux, cy = EY[a] - uy, w = 1.0;
        for (int i = 0; i < p; ++i) w *= cx;
        for (int i = 0; i < q; ++i) w *= cy;
        s += f[a] * w;
    }
    return s / rho;
}

/* Section IV: f^eq at local temperature.  Central moments from Eq. 7 with T0 -> T,
 * raw moments by the binomial theorem (Eq. 9), populations by Eq. 3. */
void oracle_feq(double rho, double ux, double uy, double RT, double out[9]) {
    const double Pit = 0.0, Nt = 0.0, M21t = 0.0, M12t = 0.0;
    const double Et = 2.0 * RT, M22t = RT * RT;
    const double uu = ux * ux + uy * uy;
    const double Pi = Pit + ux * uy;
    const double N = Nt + ux * ux - uy * uy;
    const double E = Et + ux * ux + uy * uy;
    const double M21 = M21t + 2.0 * ux * Pi + 0.5 * uy * (E + N) - 2.0 * ux * ux * uy;
    const double M12 = M12t + 2.0 * uy * Pi + 0.5 * ux * (E - N) - 2.0 * uy * uy * ux;
    const double M22 = M22t + 2.0 * ux * M12 + 2.0 * uy * M21 - 0.5 * uu * E
                     + 0.5 * (ux * ux - uy * uy) * N - 4.0 * ux * uy * Pi + 3.0 * ux * ux * uy * uy;
    const double M[9] = {1.0, ux, uy, E, N, Pi, M21, M12, M22};
    oracle_pop_from_moments(rho, M, out);
}

/* Section III: S_a = Eq. 3 applied to the raw source moments listed after Eq. 15
 * (third-order central moments of S dropped). */
void oracle_source(double rho, double ux, double uy, double ax, double ay, double out[9]) {
    const double M[9] = {
        0.0,
        ax,
        ay,
        2.0 * (ax * ux + ay * uy),
        2.0 * (ax * ux - ay * uy),
        ax * uy + ay * ux,
        ay * ux * ux + 2.0 * ax * ux * uy,
        ax * uy * uy + 2.0 * ay * ux * uy,
        2.0 * ax * ux * uy * uy + 2.0 * ay * uy * ux * ux,
    };
    oracle_pop_from_moments(rho, M, out);
}

/* Section IV: C_a = Eq. 3 applied to the correction raw moments; dx = d_x[u_x(1-theta)],
 * dy = d_y[u_y(1-theta)]. */
void oracle_correction(double rho, double ux, double uy, double dx, double dy, double out[9]) {
    const double M[9] = {0.0, 0.0, 0.0, dx + dy, dx - dy, 0.0, uy * dx, ux * dy, 0.0};
    oracle_pop_from_moments(rho, M, out);
}

/* Section IV: total-energy equilibrium, closed form printed after the h^eq moment list,
 * with the total energy Etot = (b R T + u^2)/2. */
void oracle_heq(double rho, double ux, double uy, double RT, double b, double out[9]) {
    const double uu = ux * ux + uy * uy;
    const double Etot = 0.5 * (b * RT + uu);
    out[0] = rho * (Etot - (Etot + 2.0 * RT) * uu - 2.0 * RT * (Etot + RT));
    for (int a = 1; a <= 4; ++a) {
        const double eu = EX[a] * ux + EY[a] * uy;
        const double e2u2 = (double)(EX[a] * EX[a]) * ux * ux + (double)(EY[a] * EY[a]) * uy * uy;
        out[a] = 0.5 * rho * ((Etot + RT) * eu + (Etot + 2.0 * RT) * e2u2 + RT * (Etot + RT));
    }
    for (int a = 5; a <= 8; ++a)
        out[a] = 0.25 * rho * ((Etot + 2.0 * RT) * EX[a] * EY[a] * ux * uy);
}

/* ------------------------------------------------------------ macroscopic */

static void force_field(const oracle_params* p, int x, int y, double* Fx, double* Fy) {
    const double kx = 2.0 * PI_ / p->nx, ky = 2.0 * PI_ / p->ny;
    *Fx = p->famp * sin(kx * x) * sin(ky * y);
    *Fy = p->famp * cos(kx * x) * cos(ky * y);
}

/* Eq. 20 and the temperature of Section IV: rho = sum f_bar, rho u = sum f_bar e + F/2,
 * T = 2/(bR) (sum h_bar / rho - u^2/2). */
static void macro_of(const oracle_params* p, const double fb[9], const double hb[9], int x, int y, macro_t* m) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < Q; ++a) { rho += fb[a]; jx += fb[a] * EX[a]; jy += fb[a] * EY[a]; }
    double Fx = 0.0, Fy = 0.0;
    if (p->force_kind == FORCE_UNIFORM_ACCEL) { Fx = rho * p->ax; Fy = rho * p->ay; }
    else if (p->force_kind == FORCE_TAYLOR_GREEN) force_field(p, x, y, &Fx, &Fy);
    m->rho = rho;
    m->Fx = Fx; m->Fy = Fy;
    m->ux = (jx + 0.5 * Fx) / rho;
    m->uy = (jy + 0.5 * Fy) / rho;
    m->ax = Fx / rho; m->ay = Fy / rho;
    if (p->thermal) {
        double sh = 0.0;
        for (int a = 0; a < Q; ++a) sh += hb[a];
        if (p->work) sh += 0.5 * (Fx * m->ux + Fy * m->uy); /* rho E = sum h_bar + F.u / 2 */
        m->T = 2.0 / (b_dof(p) * p->R) * (sh / rho - 0.5 * (m->ux * m->ux + m->uy * m->uy));
    } else {
        m->T = p->T0;
    }
}

static void gather(const oracle_params* p, const double* arr, int x, int y, double out[9]) {
    for (int a = 0; a < Q; ++a) out[a] = arr[at(p, a, x, y)];
}

static void macro_at(const oracle_params* p, const double* f, const double* h, int x, int y, macro_t* m) {
    double fb[9], hb[9];
    gather(p, f, x, y, fb);
    if (p->thermal) gather(p, h, x, y, hb);
    macro_of(p, fb, hb, x, y, m);
}

/* phi = u (1 - theta), the quantity differentiated in the correction term.  The
 * defect it removes is rho u_l (1 - 3 R T - u_l^2) (Section IV: D2Q9 gives
 * sum f^eq e_x^3 = rho u_x where the Maxwellian gives rho u_x (3 R T + u_x^2)), so
 * theta = 3 R T; this is the paper's T/T0 at its normalisation 3 R T0 = 1. */
static double phi_at(const oracle_params* p, const double* f, const double* h, int x, int y, int comp) {
    macro_t m;
    macro_at(p, f, h, x, y, &m);
    return (comp == 0 ? m.ux : m.uy) * (1.0 - 3.0 * p->R * m.T);
}

/* Second-order central differences at the collision's time level; one-sided
 * second-order at a wall node in the wall-normal direction. */
static void grad_at(const oracle_params* p, const double* f, const double* h, int x, int y, double* dx, double* dy) {
    const int nx = p->nx, ny = p->ny;
    if (x_periodic(p))
        *dx = 0.5 * (phi_at(p, f, h, wrap(x + 1, nx), y, 0) - phi_at(p, f, h, wrap(x - 1, nx), y, 0));
    else if (x == 0)
        *dx = 0.5 * (-3.0 * phi_at(p, f, h, 0, y, 0) + 4.0 * phi_at(p, f, h, 1, y, 0) - phi_at(p, f, h, 2, y, 0));
    else if (x == nx - 1)
        *dx = 0.5 * (3.0 * phi_at(p, f, h, nx - 1, y, 0) - 4.0 * phi_at(p, f, h, nx - 2, y, 0) + phi_at(p, f, h, nx - 3, y, 0));
    else
        *dx = 0.5 * (phi_at(p, f, h, x + 1, y, 0) - phi_at(p, f, h, x - 1, y, 0));
    if (y_periodic(p))
        *dy = 0.5 * (phi_at(p, f, h, x, wrap(y + 1, ny), 1) - phi_at(p, f, h, x, wrap(y - 1, ny), 1));
    else if (y == 0)
        *dy = 0.5 * (-3.0 * phi_at(p, f, h, x, 0, 1) + 4.0 * phi_at(p, f, h, x, 1, 1) - phi_at(p, f, h, x, 2, 1));
    else if (y == ny - 1)
        *dy = 0.5 * (3.0 * phi_at(p, f, h, x, ny - 1, 1) - 4.0 * phi_at(p, f, h, x, ny - 2, 1) + phi_at(p, f, h, x, ny - 3, 1));
    else
        *dy = 0.5 * (phi_at(p, f, h, x, y + 1, 1) - phi_at(p, f, h, x, y - 1, 1));
}

/* Eq. 29 (and the athermal nu = R T0 (1/w1 - 1/2) of Section II): 1/w1 = mu/p + 1/2. */
static double omega1(const oracle_params* p, double rho, double T) {
    const double pres = rho * p->R * T;
    double mu;
    switch (p->visc_law) {
    case VISC_CONST_NU: mu = rho * p->visc; break;
    case VISC_CONST_MU: mu = p->visc; break;
    case VISC_MU_PROP_T: mu = p->visc * T / p->T0; break;
    default: return p->visc; /* VISC_FIXED_W1 */
    }
    return 1.0 / (mu / pres + 0.5);
}

/* ----------------------------------------------------------- the collision */

/* One node's collision, in the paper's order.  Inputs: transformed populations
 * fb, hb at time t, force density (Fx, Fy) at the node (uniform acceleration
 * is handled by the caller through macro_of), and the correction derivatives
 * dx, dy.  Outputs: fstar = f_bar^*, S, C, fout = f_bar^* + S + C (Eq. 27),
 * hout = the updated h_bar (before streaming). */
static void collide(const oracle_params* p, const double fb[9], const double hb[9], const macro_t* m,
                    double dx, double dy, double fstar[9], double S[9], double C[9],
                    double fout[9], double hout[9]) {
    const double rho = m->rho, ux = m->ux, uy = m->uy, ax = m->ax, ay = m->ay;
    const double T = m->T, RT = p->R * T, uu = ux * ux + uy * uy;
    const double w1 = omega1(p, rho, T), w2 = p->w2, w3 = p->w3, w4 = p->w4;
    if (!(p->thermal && p->correction)) { dx = 0.0; dy = 0.0; }

    /* Eq. 4 on f_bar: central moments about u (the p+q >= 2 ones are relaxed). */
    const double k20 = central_moment(fb, rho, ux, uy, 2, 0);
    const double k02 = central_moment(fb, rho, ux, uy, 0, 2);
    const double k11 = central_moment(fb, rho, ux, uy, 1, 1);
    const double k21 = central_moment(fb, rho, ux, uy, 2, 1);
    const double k12 = central_moment(fb, rho, ux, uy, 1, 2);
    const double k22 = central_moment(fb, rho, ux, uy, 2, 2);
    const double Et = k20 + k02, Nt = k20 - k02, Pit = k11; /* Eq. 2 */

    /* Equilibrium central moments of f_bar (Section IV, shifted by C; Eq. 7 when C = 0). */
    const double Pieq = 0.0, M21eq = 0.0, M12eq = 0.0;
    const double Neq = 0.5 * dy - 0.5 * dx;
    const double Eeq = 2.0 * RT - 0.5 * dx - 0.5 * dy;
    const double M22eq = RT * RT;

    /* Eq. 8: cascaded relaxation. */
    const double Pis = w1 * Pieq + (1.0 - w1) * Pit;
    const double Ns = w1 * Neq + (1.0 - w1) * Nt;
    const double Es = w2 * Eeq + (1.0 - w2) * Et;
    const double M21s = w3 * M21eq + (1.0 - w3) * k21;
    const double M12s = w3 * M12eq + (1.0 - w3) * k12;
    const double M22s = w4 * M22eq + (1.0 - w4) * k22;

    /* Eq. 18: forced post-collision raw moments. */
    const double Pi = Pis + ux * uy - 0.5 * (ax * uy + ay * ux);
    const double N = Ns + ux * ux - uy * uy - (ax * ux - ay * uy);
    const double E = Es + ux * ux + uy * uy - (ax * ux + ay * uy);
    const double M21 = M21s + 2.0 * ux * Pi + 0.5 * uy * (E + N) - 2.0 * ux * ux * uy
                     + 0.5 * ay * ux * ux + ax * ux * uy;
    const double M12 = M12s + 2.0 * uy * Pi + 0.5 * ux * (E - N) - 2.0 * uy * uy * ux
                     + 0.5 * ax * uy * uy + ay * ux * uy;
    const double M22 = M22s + 2.0 * ux * M12 + 2.0 * uy * M21 - 0.5 * uu * E
                     + 0.5 * (ux * ux - uy * uy) * N - 4.0 * ux * uy * Pi + 3.0 * ux * ux * uy * uy
                     - ax * ux * uy * uy - ay * uy * ux * ux;

    /* Eq. 3 with the conserved moments of f_bar: M00 = 1, M10 = ux - ax/2, M01 = uy - ay/2. */
    const double Mpost[9] = {1.0, ux - 0.5 * ax, uy - 0.5 * ay, E, N, Pi, M21, M12, M22};
    oracle_pop_from_moments(rho, Mpost, fstar);
    oracle_source(rho, ux, uy, ax, ay, S);
    oracle_correction(rho, ux, uy, dx, dy, C);
    for (int a = 0; a < Q; ++a) fout[a] = fstar[a] + S[a] + C[a]; /* Eq. 27 */

    if (!p->thermal) return;

    /* Section IV: total-energy distribution. */
    const double b = b_dof(p);
    const double pres = rho * RT;
    const double mu_over_p = 1.0 / w1 - 0.5;                 /* Eq. 29 */
    const double cp = p->R * (b + 2.0) / 2.0;
    const double lambda = mu_over_p * pres * cp / p->Pr;     /* Pr = mu c_p / lambda */
    const double wh = 1.0 / (2.0 * lambda / (pres * p->R * (b + 2.0)) + 0.5);
    const double inv_tau_hf = (p->Pr - 1.0) / (mu_over_p + 0.5);
    double feq[9], heq[9];
    oracle_feq(rho, ux, uy, RT, feq);
    oracle_heq(rho, ux, uy, RT, b, heq);
    const double qw = p->work ? m->Fx * ux + m->Fy * uy : 0.0;   /* power of the body force */
    for (int a = 0; a < Q; ++a) {
        const double Z = EX[a] * ux + EY[a] * uy - 0.5 * uu;           /* Eq. 22 */
        const double K = Z * inv_tau_hf * (fb[a] - feq[a] + 0.5 * S[a] + 0.5 * C[a]);
        hout[a] = hb[a] - wh * (hb[a] - heq[a]) + (1.0 - 0.5 * wh) * (K + WQ[a] * qw);
    }
}

/* Post-collision populations of node (x, y) from the state (f, h) at time t. */
static void collide_at(const oracle_params* p, const double* f, const double* h, int x, int y,
                       double fout[9], double hout[9]) {
    double fb[9], hb[9] = {0}, fstar[9], S[9], C[9];
    gather(p, f, x, y, fb);
    if (p->thermal) gather(p, h, x, y, hb);
    macro_t m;
    macro_of(p, fb, hb, x, y, &m);
    double dx = 0.0, dy = 0.0;
    if (p->thermal && p->correction) grad_at(p, f, h, x, y, &dx, &dy);
    collide(p, fb, hb, &m, dx, dy, fstar, S, C, fout, hout);
}

/* ---------------------------------------------------------------- walls */

static int opposite(int a) {
    for (int b = 0; b < Q; ++b)
        if (EX[b] == -EX[a] && EY[b] == -EY[a]) return b;
    return -1;
}
static int dir_index(int cx, int cy) {
    for (int a = 0; a < Q; ++a)
        if (EX[a] == cx && EY[a] == cy) return a;
    return -1;
}

/* Rebuild the populations of wall node (x, y) on side `side` after streaming.
 * fb/hb: the node's streamed populations (entries that would have come from
 * outside the lattice are undefined on entry); ff/hf: the streamed populations of
 * the interior neighbour x_f = x_b + n (n = inward normal). */
static void wall_rebuild(const oracle_params* p, int side, int x, int y, double fb[9], double hb[9],
                         const double ff[9], const double hf[9]) {
    const int kind = p->wall_kind[side];
    const int nxv = NRM_X[side], nyv = NRM_Y[side];
    const int txv = nyv != 0 ? 1 : 0, tyv = nyv != 0 ? 0 : 1; /* tangent */
    const double uwx = p->wall_ux[side], uwy = p->wall_uy[side];
    const double b = b_dof(p);
    macro_t mf;
    macro_of(p, ff, hf, x + nxv, y + nyv, &mf);
    /* Adiabatic wall temperature.  Zero gradient: T_w = T_f.  Zero flux (study option):
     * conduction -lambda dT and viscous work -u.sigma across the link between the wall
     * node and x_f cancel when lambda (T_f - T_w) + mu (|u_f|^2 - |u_w|^2)/2 = 0, i.e.
     * T_w = T_f + Pr (|u_f|^2 - |u_w|^2) / (2 c_p) with lambda = mu c_p / Pr. */
    double T_adiabatic = mf.T;
    if (p->adiabatic_flux) {
        const double cp = p->R * (b + 2.0) / 2.0;
        T_adiabatic += p->Pr * ((mf.ux * mf.ux + mf.uy * mf.uy) - (uwx * uwx + uwy * uwy)) / (2.0 * cp);
    }
    const double Tw = p->thermal ? (p->wall_therm[side] == THERM_ADIABATIC ? T_adiabatic : p->wall_T[side]) : p->T0;

    if (kind == WALL_ZOUHE) {
        /* Non-equilibrium bounce-back (Zou-He) for a tangentially moving wall,
         * written for the transformed populations: the wall density and the two
         * momentum components of Eq. 20 are imposed, with the normal unknown closed
         * by bounce-back of its non-equilibrium part (f_bar^eq = f^eq - S/2). */
        double sumK = 0.0, sumI = 0.0;
        for (int a = 0; a < Q; ++a) {
            const int en = EX[a] * nxv + EY[a] * nyv;
            if (en == 0) sumK += fb[a];
            else if (en < 0) sumI += fb[a];
        }
        double Fxw = 0.0, Fyw = 0.0, an = 0.0, at_ = 0.0, rho_w;
        if (p->force_kind == FORCE_TAYLOR_GREEN) {
            force_field(p, x, y, &Fxw, &Fyw);
            rho_w = sumK + 2.0 * sumI - 0.5 * (Fxw * nxv + Fyw * nyv);
            an = (Fxw * nxv + Fyw * nyv) / rho_w;
            at_ = (Fxw * txv + Fyw * tyv) / rho_w;
        } else {
            if (p->force_kind == FORCE_UNIFORM_ACCEL) { an = p->ax * nxv + p->ay * nyv; at_ = p->ax * txv + p->ay * tyv; }
            rho_w = (sumK + 2.0 * sumI) / (1.0 + 0.5 * an);
        }
        const double Fn = rho_w * an, Ft = rho_w * at_;
        const double uwt = uwx * txv + uwy * tyv;
        const int in = dir_index(nxv, nyv), it = dir_index(txv, tyv), imt = dir_index(-txv, -tyv);
        const int ip = dir_index(nxv + txv, nyv + tyv), im = dir_index(nxv - txv, nyv - tyv);
        const double dn = -0.5 * rho_w * an * (1.0 - uwt * uwt); /* -(S_n - S_-n)/2 at the wall */
        fb[in] = fb[opposite(in)] + dn;
        fb[ip] = fb[opposite(ip)] - 0.5 * (fb[it] - fb[imt]) + 0.5 * rho_w * uwt - 0.25 * Ft - 0.25 * Fn - 0.5 * dn;
        fb[im] = fb[opposite(im)] + 0.5 * (fb[it] - fb[imt]) - 0.5 * rho_w * uwt + 0.25 * Ft - 0.25 * Fn - 0.5 * dn;
    } else if (kind == WALL_NEE) {
        /* Non-equilibrium extrapolation: f_b = f^eq(rho_f, u_w, T_w) + [f_f - f^eq(rho_f, u_f, T_f)]. */
        double eqw[9], eqf[9];
        oracle_feq(mf.rho, uwx, uwy, p->R * Tw, eqw);
        oracle_feq(mf.rho, mf.ux, mf.uy, p->R * mf.T, eqf);
        for (int a = 0; a < Q; ++a) fb[a] = eqw[a] + (ff[a] - eqf[a]);
    } else if (kind == WALL_EQUILIBRIUM) {
        /* Equilibrium distribution at the prescribed wall state, transformed by -S/2. */
        const double rw = p->wall_rho[side];
        double Fx = 0.0, Fy = 0.0;
        if (p->force_kind == FORCE_UNIFORM_ACCEL) { Fx = rw * p->ax; Fy = rw * p->ay; }
        else if (p->force_kind == FORCE_TAYLOR_GREEN) force_field(p, x, y, &Fx, &Fy);
        double eqw[9], S[9];
        oracle_feq(rw, uwx, uwy, p->R * (p->thermal ? p->wall_T[side] : p->T0), eqw);
        oracle_source(rw, uwx, uwy, Fx / rw, Fy / rw, S);
        for (int a = 0; a < Q; ++a) fb[a] = eqw[a] - 0.5 * S[a];
    }

    if (!p->thermal) return;
    if (kind == WALL_EQUILIBRIUM) {
        oracle_heq(p->wall_rho[side], uwx, uwy, p->R * p->wall_T[side], b, hb);
        if (p->work) {
            const double rw = p->wall_rho[side];
            double Fx = 0.0, Fy = 0.0;
            if (p->force_kind == FORCE_UNIFORM_ACCEL) { Fx = rw * p->ax; Fy = rw * p->ay; }
            else if (p->force_kind == FORCE_TAYLOR_GREEN) force_field(p, x, y, &Fx, &Fy);
            for (int a = 0; a < Q; ++a) hb[a] -= 0.5 * WQ[a] * (Fx * uwx + Fy * uwy);
        }
        return;
    }
    /* Temperature by non-equilibrium extrapolation: h_b = h^eq(rho_b, u_b, T_w) + [h_f - h^eq(rho_f, u_f, T_f)],
     * with (rho_b, u_b) the moments of the rebuilt f_b. */
    macro_t mb;
    macro_of(p, fb, hf, x, y, &mb);
    double eqw[9], eqf[9];
    oracle_heq(mb.rho, mb.ux, mb.uy, p->R * Tw, b, eqw);
    oracle_heq(mf.rho, mf.ux, mf.uy, p->R * mf.T, b, eqf);
    if (p->work) { /* the transformed equilibria h^eq - q/2 of both nodes */
        const double qb = mb.Fx * mb.ux + mb.Fy * mb.uy, qf = mf.Fx * mf.ux + mf.Fy * mf.uy;
        for (int a = 0; a < Q; ++a) { eqw[a] -= 0.5 * WQ[a] * qb; eqf[a] -= 0.5 * WQ[a] * qf; }
    }
    for (int a = 0; a < Q; ++a) hb[a] = eqw[a] + (hf[a] - eqf[a]);
}

/* Which side, if any, node (x, y) is a wall node of (walls sit on one axis only). */
static int wall_side_of(const oracle_params* p, int x, int y) {
    if (!x_periodic(p)) {
        if (x == 0) return SIDE_XM;
        if (x == p->nx - 1) return SIDE_XP;
    }
    if (!y_periodic(p)) {
        if (y == 0) return SIDE_YM;
        if (y == p->ny - 1) return SIDE_YP;
    }
    return -1;
}

/* ---------------------------------------------------------------- API */

int oracle_check(const oracle_params* p) {
    if (p->nx < 1 || p->ny < 1) return -1;
    if ((p->wall_kind[SIDE_XM] == WALL_PERIODIC) != (p->wall_kind[SIDE_XP] == WALL_PERIODIC)) return -1;
    if ((p->wall_kind[SIDE_YM] == WALL_PERIODIC) != (p->wall_kind[SIDE_YP] == WALL_PERIODIC)) return -1;
    if (!x_periodic(p) && !y_periodic(p)) return -2; /* walls on both axes: not supported */
    if (!x_periodic(p) && p->nx < 3) return -1;
    if (!y_periodic(p) && p->ny < 3) return -1;
    if (p->gamma <= 1.0 || p->Pr <= 0.0 || p->R <= 0.0 || p->T0 <= 0.0) return -1;
    if (p->work && !p->thermal) return -1;
    return 0;
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Initial populations from the fields (arrays [ny][nx]): f_bar = f^eq - S/2, h_bar = h^eq;
 * the wall nodes are then rebuilt by their wall scheme from the initial interior state,
 * so that the initial state satisfies the boundary conditions like every later one. */
int oracle_init(const oracle_params* p, const double* rho, const double* ux, const double* uy,
                const double* T, double* f, double* h) {
    if (oracle_check(p)) return -1;
    const double b = b_dof(p);
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const size_t i = (size_t)y * p->nx + x;
            const double Tn = p->thermal ? T[i] : p->T0;
            double Fx = 0.0, Fy = 0.0;
            if (p->force_kind == FORCE_UNIFORM_ACCEL) { Fx = rho[i] * p->ax; Fy = rho[i] * p->ay; }
            else if (p->force_kind == FORCE_TAYLOR_GREEN) force_field(p, x, y, &Fx, &Fy);
            double feq[9], S[9], heq[9];
            oracle_feq(rho[i], ux[i], uy[i], p->R * Tn, feq);
            oracle_source(rho[i], ux[i], uy[i], Fx / rho[i], Fy / rho[i], S);
            for (int a = 0; a < Q; ++a) f[at(p, a, x, y)] = feq[a] - 0.5 * S[a];
            if (p->thermal) {
                oracle_heq(rho[i], ux[i], uy[i], p->R * Tn, b, heq);
                const double qw = p->work ? Fx * ux[i] + Fy * uy[i] : 0.0;
                for (int a = 0; a < Q; ++a) h[at(p, a, x, y)] = heq[a] - 0.5 * WQ[a] * qw;
            }
        }
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const int side = wall_side_of(p, x, y);
            if (side < 0) continue;
            double fb[9], hb[9] = {0}, ff[9], hf[9] = {0};
            const int xf = x + NRM_X[side], yf = y + NRM_Y[side];
            gather(p, f, x, y, fb);
            gather(p, f, xf, yf, ff);
            if (p->thermal) { gather(p, h, x, y, hb); gather(p, h, xf, yf, hf); }
            wall_rebuild(p, side, x, y, fb, hb, ff, hf);
            for (int a = 0; a < Q; ++a) {
                f[at(p, a, x, y)] = fb[a];
                if (p->thermal) h[at(p, a, x, y)] = hb[a];
            }
        }
    return 0;
}

/* nsteps full time steps in place: collide every node, stream (Eq. 27 and the h
 * update), then rebuild the wall nodes. */
int oracle_step(const oracle_params* p, double* f, double* h, int nsteps) {
    if (oracle_check(p)) return -1;
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)Q * nx * ny;
    double* fn = (double*)malloc(n * sizeof(double));
    double* hn = p->thermal ? (double*)malloc(n * sizeof(double)) : NULL;
    if (!fn || (p->thermal && !hn)) { free(fn); free(hn); return -3; }
    for (int s = 0; s < nsteps; ++s) {
        for (size_t i = 0; i < n; ++i) { fn[i] = NAN; if (hn) hn[i] = NAN; }
        #pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double fo[9], ho[9];
                collide_at(p, f, h, x, y, fo, ho);
                for (int a = 0; a < Q; ++a) {
                    int xd = x + EX[a], yd = y + EY[a];
                    if (x_periodic(p)) xd = wrap(xd, nx); else if (xd < 0 || xd >= nx) continue;
                    if (y_periodic(p)) yd = wrap(yd, ny); else if (yd < 0 || yd >= ny) continue;
                    fn[at(p, a, xd, yd)] = fo[a];
                    if (hn) hn[at(p, a, xd, yd)] = ho[a];
                }
            }
        #pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int side = wall_side_of(p, x, y);
                if (side < 0) continue;
                double fb[9], hb[9] = {0}, ff[9], hf[9] = {0};
                const int xf = x + NRM_X[side], yf = y + NRM_Y[side];
                gather(p, fn, x, y, fb);
                gather(p, fn, xf, yf, ff);
                if (hn) { gather(p, hn, x, y, hb); gather(p, hn, xf, yf, hf); }
                wall_rebuild(p, side, x, y, fb, hb, ff, hf);
                for (int a = 0; a < Q; ++a) {
                    fn[at(p, a, x, y)] = fb[a];
                    if (hn) hn[at(p, a, x, y)] = hb[a];
                }
            }
        memcpy(f, fn, n * sizeof(double));
        if (hn) memcpy(h, hn, n * sizeof(double));
    }
    free(fn);
    free(hn);
    return 0;
}

/* Streamed populations of node (x, y) at t+1 before its own wall rebuild; entries
 * whose source lies outside the lattice are NaN. */
static void streamed_at(const oracle_params* p, const double* f, const double* h, int x, int y,
                        double fo[9], double ho[9]) {
    for (int a = 0; a < Q; ++a) {
        int xs = x - EX[a], ys = y - EY[a];
        int ok = 1;
        if (x_periodic(p)) xs = wrap(xs, p->nx); else if (xs < 0 || xs >= p->nx) ok = 0;
        if (y_periodic(p)) ys = wrap(ys, p->ny); else if (ys < 0 || ys >= p->ny) ok = 0;
        if (!ok) { fo[a] = NAN; ho[a] = NAN; continue; }
        double cf[9], ch[9] = {0};
        collide_at(p, f, h, xs, ys, cf, ch);
        fo[a] = cf[a];
        ho[a] = p->thermal ? ch[a] : 0.0;
    }
}

/* One time step evaluated only at the listed output nodes: out_f/out_h receive the
 * populations of those nodes at t+1 ([n][9]), computed from the full state at t.
 * Same arithmetic as oracle_step; used to check full-size lattices node by node. */
int oracle_update_nodes(const oracle_params* p, const double* f, const double* h, int n,
                        const int32_t* xs, const int32_t* ys, double* out_f, double* out_h) {
    if (oracle_check(p)) return -1;
    #pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < n; ++k) {
        const int x = xs[k], y = ys[k];
        double fb[9], hb[9] = {0};
        streamed_at(p, f, h, x, y, fb, hb);
        const int side = wall_side_of(p, x, y);
        if (side >= 0) {
            double ff[9], hf[9] = {0};
            streamed_at(p, f, h, x + NRM_X[side], y + NRM_Y[side], ff, hf);
            wall_rebuild(p, side, x, y, fb, hb, ff, hf);
        }
        for (int a = 0; a < Q; ++a) {
            out_f[(size_t)k * Q + a] = fb[a];
            if (out_h) out_h[(size_t)k * Q + a] = p->thermal ? hb[a] : 0.0;
        }
    }
    return 0;
}

/* Macroscopic fields (Eq. 20, temperature of Section IV), arrays [ny][nx]. */
void oracle_moments(const oracle_params* p, const double* f, const double* h, double* rho,
                    double* ux, double* uy, double* T) {
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            macro_t m;
            macro_at(p, f, h, x, y, &m);
            const size_t i = (size_t)y * p->nx + x;
            rho[i] = m.rho; ux[i] = m.ux; uy[i] = m.uy; T[i] = m.T;
        }
}

/* Single-node collision for unit checks: given f_bar, h_bar, the force density and
 * the correction derivatives, return f_bar^*, S, C, f_bar^* + S + C, the updated
 * h_bar, and the node's (rho, ux, uy, T, w1).  Uniform acceleration is taken from p. */
void oracle_collide_node(const oracle_params* p, const double fb[9], const double hb[9],
                         double Fx_field, double Fy_field, double dx, double dy,
                         double fstar[9], double S[9], double C[9], double fout[9], double hout[9],
                         double macro_out[5]) {
    macro_t m;
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < Q; ++a) { rho += fb[a]; jx += fb[a] * EX[a]; jy += fb[a] * EY[a]; }
    double Fx = Fx_field, Fy = Fy_field;
    if (p->force_kind == FORCE_UNIFORM_ACCEL) { Fx = rho * p->ax; Fy = rho * p->ay; }
    else if (p->force_kind == FORCE_NONE) { Fx = 0.0; Fy = 0.0; }
    m.rho = rho; m.Fx = Fx; m.Fy = Fy;
    m.ux = (jx + 0.5 * Fx) / rho; m.uy = (jy + 0.5 * Fy) / rho;
    m.ax = Fx / rho; m.ay = Fy / rho;
    if (p->thermal) {
        double sh = 0.0;
        for (int a = 0; a < Q; ++a) sh += hb[a];
        if (p->work) sh += 0.5 * (Fx * m.ux + Fy * m.uy);
        m.T = 2.0 / (b_dof(p) * p->R) * (sh / rho - 0.5 * (m.ux * m.ux + m.uy * m.uy));
    } else m.T = p->T0;
    double hzero[9] = {0};
    collide(p, fb, p->thermal ? hb : hzero, &m, dx, dy, fstar, S, C, fout, hout);
    macro_out[0] = m.rho; macro_out[1] = m.ux; macro_out[2] = m.uy; macro_out[3] = m.T;
    macro_out[4] = omega1(p, m.rho, m.T);
}

/* Wall rebuild of one node for unit checks (fb, hb modified in place). */
void oracle_wall_node(const oracle_params* p, int side, int x, int y, double fb[9], double hb[9],
                      const double ff[9], const double hf[9]) {
    wall_rebuild(p, side, x, y, fb, hb, ff, hf);
}

void oracle_velocities(int32_t ex[9], int32_t ey[9]) {
    for (int a = 0; a < Q; ++a) { ex[a] = EX[a]; ey[a] = EY[a]; }
}
