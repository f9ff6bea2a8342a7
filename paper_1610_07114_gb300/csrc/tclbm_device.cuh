// tclbm_device.cuh -- per-node arithmetic and the fused collide-and-stream kernel of
// the thermal cascaded lattice Boltzmann method (Fei & Luo, arXiv:1610.07114), D2Q9,
// written for sm_103a.
//
// Layout (structure of arrays): plane q in [0, 9) holds f_bar_q, plane 9 + q holds
// h_bar_q; each plane is ny rows of `pitch` elements, x fastest.  Two ping-pong
// copies; a step reads one and writes the other (pull streaming: the kernel gathers
// f_bar_q(x, t+1) = f_out_q(x - e_q, t) from the source copy and writes the node's
// own post-collision values at its own address).
//
// The kernel marches each CTA up a strip of TX columns, one row at a time, keeping
// the next row's streamed populations in registers.  That lookahead gives the
// moments of row r+1 before row r collides, which the correction term of Section IV
// needs (central differences of u(1 - theta) at the collision's time level); the
// x-neighbours come from a three-row shared-memory ring.  No tensor cores: the update
// is a memory-bound stencil.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace tclbm {

enum { SIDE_XM = 0, SIDE_XP = 1, SIDE_YM = 2, SIDE_YP = 3 };
enum { WALL_PERIODIC = 0, WALL_ZOUHE = 1, WALL_NEE = 2, WALL_EQUILIBRIUM = 3 };
enum { THERM_FIXED_T = 0, THERM_ADIABATIC = 1 };
enum { VISC_NU = 0, VISC_MU = 1, VISC_MU_PROP_T = 2, VISC_W1 = 3 };
enum { FORCE_NONE = 0, FORCE_ACCEL = 1, FORCE_TAYLOR_GREEN = 2 };

// Device-side constants of one lattice (derived on the host from tclbm_params).
struct DevParams {
    int nx, ny, pitch;
    long long plane;  // ny * pitch elements
    int xper, yper;   // 1 if the axis is periodic
    int visc_law;
    float visc, w2, w3, w4;
    int bgk;
    float R, T0, b, two_over_b, inv_R, inv_Pr, Pr_m1;
    float RTp, inv_RTp;   // R T0 (the athermal temperature) and its inverse
    float inv_w1_fixed;   // 1 / w1 for VISC_W1
    float RT0, Et0, cRT;  // rest state of the deviations (exact floats); cRT = (2/b) Et0 - RT0
    int force_kind;
    float ax, ay, famp;
    const float* sx;  // sin(2 pi x / nx), cos(...), sin(2 pi y / ny), cos(...)
    const float* cx;
    const float* sy;
    const float* cy;
    int wall_kind[4], wall_therm[4];
    float wall_rho[4], wall_ux[4], wall_uy[4], wall_T[4];
    // R T of each wall and its deviation R T - RT0, both formed in FP64 on the host: an
    // FP32 product R T (R = 1/6 is not a float) would shift the wall temperature by 3e-8
    float wall_RT[4], wall_dRT[4];
    float dRTp;  // R T0 - RT0, formed in FP64 (athermal lattices)
    float fbase[9], hbase[9];  // rest-state populations f^eq(1, 0, T0), h^eq(1, 0, T0)
    int rounding;              // 16-bit stores: 0 nearest, 1 stochastic
    unsigned* step_ctr;        // two step counters, alternated by launch parity
    int parity;                // index of the source copy of this launch
    int skip_row;              // test hook: the TMA producer never copies this source row (-1: off)
    // FP64 constants of the field conversions (moments, diagnostics): T = inv_bR2 (E - u^2/2)
    // with inv_bR2 = 2 / (b R), and T0, as the FP64 initialisation uses them
    double inv_bR2, T0d;
    int work;  // 1: the body force's power F.u is a source of total energy (rho E = sum h_bar + F.u/2)
};

// D2Q9 weights: the shape of the work source (zeroth moment 1, first moment 0).
constexpr float kW0 = 4.0f / 9.0f, kW1 = 1.0f / 9.0f, kW5 = 1.0f / 36.0f;

// Counter-based 32-bit mix of (node, pair, step): random bits for stochastic rounding.
__device__ __forceinline__ uint32_t sr_bits(uint32_t node, uint32_t pair, uint32_t step) {
    uint32_t h = node * 0x9E3779B1u ^ (step * 0x85EBCA77u + pair * 0xC2B2AE3Du);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return h;
}

// Random bits of population pair k from a node's seed: a Weyl step and a short
// multiply-xorshift finaliser (the seed is already fully mixed).
__device__ __forceinline__ uint32_t sr_pair_bits(uint32_t seed, uint32_t k) {
    uint32_t h = seed + k * 0x9E3779B9u;
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    return h;
}

template <class ST>
__device__ __forceinline__ uint32_t cvt_rs_pair(float a, float b, uint32_t rbits);
template <>
__device__ __forceinline__ uint32_t cvt_rs_pair<__half>(float a, float b, uint32_t rbits) {
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rbits));
    return d;
}
template <>
__device__ __forceinline__ uint32_t cvt_rs_pair<__nv_bfloat16>(float a, float b, uint32_t rbits) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rbits));
    return d;
}

// ---------------------------------------------------------------- storage formats
//
// Every format stores deviations from the rest state, df_q = f_bar_q - f^eq_q(1, 0, T0)
// and dh_q = h_bar_q - h^eq_q(1, 0, T0), and the collision is carried out on those
// deviations: the O(1) parts of moments and equilibria then cancel analytically
// instead of in FP32 arithmetic, so a per-step change far below one ulp of an O(1)
// population (viscous heating is ~1e-8 per step in a slow shear flow) is still
// represented.  16-bit formats use the same deviations, rounded to half or bfloat16.

template <class ST>
struct Store;
template <>
struct Store<float> {
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float ld_smem(const float* p) { return *p; }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <>
struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float ld_smem(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float ld_smem(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------- node arithmetic

// 1/x from the hardware approximation refined by one Newton step (relative error a few
// 1e-8); deterministic, so every inlined copy returns the same bits for the same x.
__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return __fmul_rn(r, __fmaf_rn(-x, r, 2.0f));
}

// Node state after Eq. 20, kept both whole and as deviations from the rest state
// (rho0 = 1, RT0 = R T0, Et0 = b RT0 / 2): Et = sum h_bar / rho is the total energy per
// unit mass and RT = (2/b)(Et - u^2/2).
struct Macro {
    float rho, drho, irho, ux, uy, ax, ay, RT, dRT, Et, dEt;
};

__device__ __forceinline__ void force_at(const DevParams& p, int x, int y, float rho, float& Fx, float& Fy) {
    if (p.force_kind == FORCE_ACCEL) {
        Fx = __fmul_rn(rho, p.ax);
        Fy = __fmul_rn(rho, p.ay);
    } else if (p.force_kind == FORCE_TAYLOR_GREEN) {
        Fx = __fmul_rn(__fmul_rn(p.famp, p.sx[x]), p.sy[y]);
        Fy = __fmul_rn(__fmul_rn(p.famp, p.cx[x]), p.cy[y]);
    } else {
        Fx = 0.f;
        Fy = 0.f;
    }
}

__device__ __forceinline__ float sum9(const float* v) {
    return __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(v[0], v[1]), __fadd_rn(v[2], v[3])),
                               __fadd_rn(__fadd_rn(v[4], v[5]), __fadd_rn(v[6], v[7]))),
                     v[8]);
}

// Eq. 20 and the temperature of Section IV from deviations df, dh.  Explicitly rounded
// operations: halo nodes evaluate this in other inlined copies, and the result must be
// bit-identical to the owner's so that the state does not depend on the launch shape.
template <bool THERMAL>
__device__ __forceinline__ Macro macro_of(const DevParams& p, const float* f, const float* h, int x, int y) {
    Macro m;
    m.drho = sum9(f);
    m.rho = __fadd_rn(1.0f, m.drho);
    const float jx = __fadd_rn(__fadd_rn(__fsub_rn(f[1], f[3]), __fsub_rn(f[5], f[6])), __fsub_rn(f[8], f[7]));
    const float jy = __fadd_rn(__fadd_rn(__fsub_rn(f[2], f[4]), __fsub_rn(f[5], f[7])), __fsub_rn(f[6], f[8]));
    float Fx, Fy;
    force_at(p, x, y, m.rho, Fx, Fy);
    const float irho = __frcp_rn(m.rho);  // correctly rounded: 1/rho feeds u, whose bias would accumulate
    m.irho = irho;
    m.ux = __fmul_rn(__fmaf_rn(0.5f, Fx, jx), irho);
    m.uy = __fmul_rn(__fmaf_rn(0.5f, Fy, jy), irho);
    m.ax = __fmul_rn(Fx, irho);
    m.ay = __fmul_rn(Fy, irho);
    if (THERMAL) {
        float sdh = sum9(h);
        // with the work term, rho E = sum h_bar + F.u / 2
        if (p.work) sdh = __fmaf_rn(0.5f, __fmaf_rn(Fx, m.ux, __fmul_rn(Fy, m.uy)), sdh);
        m.dEt = __fmul_rn(__fmaf_rn(-p.Et0, m.drho, sdh), irho);
        m.Et = __fadd_rn(p.Et0, m.dEt);
        const float ke = __fmul_rn(0.5f, __fmaf_rn(m.ux, m.ux, __fmul_rn(m.uy, m.uy)));
        m.dRT = __fmaf_rn(p.two_over_b, __fsub_rn(m.dEt, ke), p.cRT);
        m.RT = __fadd_rn(p.RT0, m.dRT);
    } else {
        m.RT = p.RTp;
        m.dRT = p.dRTp;
        m.dEt = 0.0f;
        m.Et = p.Et0;
    }
    return m;
}

// u (1 - 3 R T): the argument of the correction-term derivatives (Section IV; the
// paper's T/T0 at its normalisation 3 R T0 = 1).
__device__ __forceinline__ float phi_x(const Macro& m) { return __fmul_rn(m.ux, __fmaf_rn(-3.0f, m.RT, 1.0f)); }
__device__ __forceinline__ float phi_y(const Macro& m) { return __fmul_rn(m.uy, __fmaf_rn(-3.0f, m.RT, 1.0f)); }

// Eq. 3: populations from raw moments {M00, M10, M01, E, N, Pi, M21, M12, M22}.
__device__ __forceinline__ void eq3(float rho, float m00, float m10, float m01, float E, float N, float Pi,
                                    float M21, float M12, float M22, float* o) {
    const float hr = 0.5f * rho, qr = 0.25f * rho;
    const float ep = 0.5f * (E + N), em = 0.5f * (E - N);
    o[0] = rho * (m00 - E + M22);
    o[1] = hr * (m10 + ep - M12 - M22);
    o[2] = hr * (m01 + em - M21 - M22);
    o[3] = hr * (-m10 + ep + M12 - M22);
    o[4] = hr * (-m01 + em + M21 - M22);
    o[5] = qr * (Pi + M21 + M12 + M22);
    o[6] = qr * (-Pi + M21 - M12 + M22);
    o[7] = qr * (Pi - M21 - M12 + M22);
    o[8] = qr * (-Pi - M21 + M12 + M22);
}

// f^eq at local temperature is the product rho X(e_x; ux) Y(e_y; uy) with X_0 = 1 - RT - v^2,
// X_{+-1} = (RT + v^2 +- v)/2 (the Eq. 7 central moments).  dfeq returns
// f^eq(rho, u, RT) - f^eq(1, 0, RT0) without cancellation: with X = Xb + dX around
// (0, RT0), the difference is
// (rho - 1) Xb Yb + rho (dX Yb + Xb dY + dX dY).
__device__ __forceinline__ void dfeq(const DevParams& p, float rho, float drho, float ux, float uy, float dRT,
                                     float* o) {
    const float xb0 = 1.0f - p.RT0, xb1 = 0.5f * p.RT0;  // exact: RT0 is on a 2^-10 grid
    const float ux2 = ux * ux, uy2 = uy * uy;
    const float dx0 = -dRT - ux2, dxp = 0.5f * (dRT + ux2 + ux), dxm = 0.5f * (dRT + ux2 - ux);
    const float dy0 = -dRT - uy2, dyp = 0.5f * (dRT + uy2 + uy), dym = 0.5f * (dRT + uy2 - uy);
    // (a, b) -> rho (dX_a Yb_b + Xb_a dY_b + dX_a dY_b) + drho fbase
    auto term = [&](float dxa, float xba, float dyb, float ybb) { return rho * (dxa * ybb + xba * dyb + dxa * dyb); };
    o[0] = term(dx0, xb0, dy0, xb0);
    o[1] = term(dxp, xb1, dy0, xb0);
    o[2] = term(dx0, xb0, dyp, xb1);
    o[3] = term(dxm, xb1, dy0, xb0);
    o[4] = term(dx0, xb0, dym, xb1);
    o[5] = term(dxp, xb1, dyp, xb1);
    o[6] = term(dxm, xb1, dyp, xb1);
    o[7] = term(dxm, xb1, dym, xb1);
    o[8] = term(dxp, xb1, dym, xb1);
#pragma unroll
    for (int q = 0; q < 9; ++q) o[q] += drho * p.fbase[q];
}

// h^eq(rho, u, RT, Et) - h^eq(1, 0, RT0, Et0) without cancellation, with
// C = RT (Et + RT) - RT0 (Et0 + RT0) = dRT (Et + RT) + RT0 (dEt + dRT).
__device__ __forceinline__ void dheq(const DevParams& p, float rho, float drho, float ux, float uy, float RT,
                                     float dRT, float Et, float dEt, float* o) {
    const float ux2 = ux * ux, uy2 = uy * uy, uu = ux2 + uy2;
    const float A = Et + RT, B = Et + 2.0f * RT;
    const float dC = dRT * A + p.RT0 * (dEt + dRT);
    const float hr = 0.5f * rho, qb = 0.25f * rho * B * ux * uy;
    o[0] = drho * p.hbase[0] + rho * (dEt - B * uu - 2.0f * dC);
    const float axis_c = drho * p.hbase[1] + hr * dC;
    o[1] = axis_c + hr * (A * ux + B * ux2);
    o[2] = axis_c + hr * (A * uy + B * uy2);
    o[3] = axis_c + hr * (-A * ux + B * ux2);
    o[4] = axis_c + hr * (-A * uy + B * uy2);
    o[5] = qb;
    o[6] = -qb;
    o[7] = qb;
    o[8] = -qb;
}

// Lane pairs.  Blackwell issues two FP32 lanes per FADD2 / FMUL2 / FFMA2, each lane
// rounded like __fadd_rn / __fmul_rn / __fmaf_rn.  The collision keeps populations in
// the pairs (1,2), (3,4), (5,6), (7,8) from the raw moments to the store.
__device__ __forceinline__ float2 pr(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc(-1.0f), a); }  // b * -1 is exact

// Eq. 3 in lane pairs: o0 and P[k] = (o_{2k+1}, o_{2k+2}); m1 = (M10, M01), m3 = (M21, M12).
__device__ __forceinline__ void eq3_pairs(float rho, float m00, float2 m1, float E, float N, float Pi, float2 m3,
                                          float M22, float& o0, float2* P) {
    const float hr = 0.5f * rho, qr = 0.25f * rho;
    o0 = rho * (m00 - E + M22);
    const float2 e = fma2(bc(N), pr(0.5f, -0.5f), bc(0.5f * E));  // ((E + N) / 2, (E - N) / 2)
    const float2 c = sub2(e, bc(M22));
    const float2 mm = sub2(m1, pr(m3.y, m3.x));  // (M10 - M12, M01 - M21)
    P[0] = mul2(bc(hr), add2(c, mm));
    P[1] = mul2(bc(hr), sub2(c, mm));
    const float2 sd = fma2(bc(m3.y), pr(1.0f, -1.0f), bc(m3.x));  // (M21 + M12, M21 - M12)
    const float2 pm = fma2(bc(Pi), pr(1.0f, -1.0f), bc(M22));   // (M22 + Pi, M22 - Pi)
    P[2] = mul2(bc(qr), add2(pm, sd));
    P[3] = mul2(bc(qr), sub2(pm, sd));
}

// dheq in lane pairs: o0 and P[k] = (o_{2k+1}, o_{2k+2}); u = (ux, uy), u2 = (ux^2, uy^2).
__device__ __forceinline__ void dheq_pairs(const DevParams& p, float rho, float drho, float2 u, float2 u2, float RT,
                                           float dRT, float Et, float dEt, float& o0, float2* P) {
    const float uu = u2.x + u2.y;
    const float A = Et + RT, B = Et + 2.0f * RT;
    const float dC = dRT * A + p.RT0 * (dEt + dRT);
    const float hr = 0.5f * rho, qb = 0.25f * rho * B * u.x * u.y;
    o0 = drho * p.hbase[0] + rho * (dEt - B * uu - 2.0f * dC);
    const float2 axis = bc(drho * p.hbase[1] + hr * dC);
    const float2 bu2 = mul2(bc(B), u2);
    P[0] = fma2(bc(hr), fma2(bc(A), u, bu2), axis);
    P[1] = fma2(bc(hr), fma2(bc(-A), u, bu2), axis);
    P[2] = pr(qb, -qb);
    P[3] = pr(qb, -qb);
}

// Source populations S_a (Section III raw moments) at the given state.
__device__ __forceinline__ void source(float rho, float ux, float uy, float ax, float ay, float* o) {
    eq3(rho, 0.0f, ax, ay, 2.0f * (ax * ux + ay * uy), 2.0f * (ax * ux - ay * uy), ax * uy + ay * ux,
        ay * ux * ux + 2.0f * ax * ux * uy, ax * uy * uy + 2.0f * ay * ux * uy,
        2.0f * ax * ux * uy * uy + 2.0f * ay * uy * ux * ux, o);
}

// Eq. 29: 1/w1 = mu/p + 1/2 with p = rho R T; returns mu/p (= 1/w1 - 1/2).
__device__ __forceinline__ float mu_over_p(const DevParams& p, float irho, float RT) {
    switch (p.visc_law) {
        case VISC_NU: return p.visc * rcp(RT);
        case VISC_MU: return p.visc * irho * rcp(RT);
        case VISC_MU_PROP_T: return p.visc * irho * p.inv_RTp;
        default: return p.inv_w1_fixed - 0.5f;
    }
}

// One node's collision on deviations: (df, dh) at time t -> deviations of
// f_out = f_bar^* + S + C (Eq. 27) and of the updated h_bar (Section IV).
// dx, dy: d_x[u_x(1-theta)], d_y[u_y(1-theta)].
template <bool THERMAL>
__device__ __forceinline__ void collide(const DevParams& p, const float* f, const float* h, const Macro& m,
                                        float dx, float dy, float* fo, float* ho) {
    const float rho = m.rho, drho = m.drho, ux = m.ux, uy = m.uy, ax = m.ax, ay = m.ay;
    const float irho = m.irho;
    const float RT0 = p.RT0, RT = m.RT, dRT = m.dRT;
    const float2 u = pr(ux, uy), a = pr(ax, ay);
    const float2 u2 = mul2(u, u);
    const float ux2 = u2.x, uy2 = u2.y, uxy = ux * uy, uu = ux2 + uy2;
    const float mup = mu_over_p(p, irho, RT);
    const float w1 = p.visc_law == VISC_W1 ? p.visc : rcp(mup + 0.5f);
    const float w2 = p.bgk ? w1 : p.w2, w3 = p.bgk ? w1 : p.w3, w4 = p.bgk ? w1 : p.w4;

    // raw moments (Eq. 1) of the deviations; the rest state contributes 1, RT0, RT0^2.
    // Pairs hold (x, y) mirror images: (r20, r02), (r10, r01), (k21, k12), (M21, M12); usw = (uy, ux).
    const float2 s13 = add2(pr(f[1], f[2]), pr(f[3], f[4]));  // (f1 + f3, f2 + f4)
    const float2 a57 = add2(pr(f[5], f[6]), pr(f[7], f[8]));  // (f5 + f7, f6 + f8)
    const float2 d57 = sub2(pr(f[5], f[6]), pr(f[7], f[8]));  // (f5 - f7, f6 - f8)
    const float S22 = a57.x + a57.y, S11 = a57.x - a57.y;
    const float2 dr2 = mul2(fma2(bc(drho), bc(-RT0), add2(s13, bc(S22))), bc(irho));  // (r20, r02) - RT0
    const float dr22 = (S22 - RT0 * RT0 * drho) * irho;  // r22 - RT0^2
    const float r11 = S11 * irho;
    const float2 r3 = mul2(fma2(bc(d57.y), pr(1.0f, -1.0f), bc(d57.x)), bc(irho));  // (r21, r12)
    const float2 r2 = add2(dr2, bc(RT0));
    const float2 r1 = fma2(bc(-0.5f), a, u);  // (r10, r01)
    const float2 usw = pr(uy, ux), r1sw = pr(r1.y, r1.x);
    const float2 m2u = mul2(bc(-2.0f), u);

    // central moments about u by the binomial theorem (Eq. 4), k20, k02 less RT0, k22 less RT0^2
    const float2 dk2 = fma2(m2u, r1, add2(dr2, u2));  // (k20, k02) - RT0
    const float k11 = r11 - ux * r1.y - uy * r1.x + uxy;
    // k21 = r21 - 2 ux r11 - uy (r20 + ux^2) + ux^2 r01 + 2 ux uy r10, and its mirror k12
    const float2 k3 = fma2(bc(2.0f * uxy), r1,
                           fma2(u2, r1sw, fma2(mul2(bc(-1.0f), usw), add2(r2, u2), fma2(m2u, bc(r11), r3))));
    // k22 = r22 - 2 (ux r12 + uy r21) + ux^2 r02 + uy^2 r20 + 4 ux uy r11 - 2 ux uy (uy r10 + ux r01) + ux^2 uy^2
    const float2 v22 = fma2(mul2(bc(-2.0f), usw), r3, mul2(pr(uy2, ux2), r2));
    const float2 w22 = mul2(usw, r1);
    const float dk22 = dr22 + (v22.x + v22.y) + uxy * (4.0f * r11 - 2.0f * (w22.x + w22.y) + uxy);

    // Eq. 8 towards the equilibria of f_bar shifted by the correction term
    // (E~eq = 2RT - (dx+dy)/2, N~eq = (dy-dx)/2, M~22eq = RT^2; E, M22 kept less 2RT0, RT0^2)
    const float dRT2 = dRT * (2.0f * RT0 + dRT);  // RT^2 - RT0^2
    const float Pis = (1.0f - w1) * k11;
    const float Ns = w1 * (0.5f * (dy - dx)) + (1.0f - w1) * (dk2.x - dk2.y);
    const float dEs = w2 * (2.0f * dRT - 0.5f * (dx + dy)) + (1.0f - w2) * (dk2.x + dk2.y);
    const float2 m3s = mul2(bc(1.0f - w3), k3);  // (M21*, M12*) central
    const float dM22s = w4 * dRT2 + (1.0f - w4) * dk22;

    // raw moments of S (Section III) and of C (Section IV)
    const float2 au = mul2(a, u);  // (ax ux, ay uy)
    const float Es_ = 2.0f * (au.x + au.y), Ns_ = 2.0f * (au.x - au.y), Pis_ = ax * uy + ay * ux;
    const float2 m3s_ = fma2(pr(ay, ax), u2, mul2(bc(2.0f * uxy), a));  // (ay ux^2 + 2 ax ux uy, mirror)
    const float M22s_ = 2.0f * uxy * Pis_;
    const float Ec = dx + dy, Nc = dx - dy;
    const float2 m3c = mul2(usw, pr(dx, dy));  // (uy dx, ux dy)
    const float2 m3sc = add2(m3s_, m3c);

    // Eq. 18: raw post-collision moments of f_bar^*
    const float Pi = Pis + uxy - 0.5f * Pis_;
    const float N = Ns + ux2 - uy2 - (au.x - au.y);
    const float dE = dEs + uu - (au.x + au.y);
    const float E = 2.0f * RT0 + dE;
    // M21 = M21* + 2 ux Pi + uy (E + N) / 2 - 2 ux^2 uy + ay ux^2 / 2 + ax ux uy, and its mirror
    const float2 en = fma2(bc(N), pr(1.0f, -1.0f), bc(E));  // (E + N, E - N)
    const float2 m3 = fma2(a, bc(uxy),
                           fma2(mul2(bc(0.5f), pr(ay, ax)), u2,
                                fma2(mul2(bc(-2.0f), u2), usw,
                                     fma2(mul2(bc(0.5f), usw), en, fma2(bc(2.0f * Pi), u, m3s)))));
    const float2 w3m = mul2(usw, m3);  // (uy M21, ux M12)
    const float dM22 = dM22s + 2.0f * (w3m.x + w3m.y) - 0.5f * uu * E + 0.5f * (ux2 - uy2) * N - 4.0f * uxy * Pi
                     + 3.0f * ux2 * uy2 - uxy * Pis_;

    float2 FO[4];
    eq3_pairs(rho, 0.0f, fma2(bc(0.5f), a, u), dE + Es_ + Ec, N + Ns_ + Nc, Pi + Pis_, add2(m3, m3sc),
              dM22 + M22s_, fo[0], FO);
    fo[0] += drho * p.fbase[0];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 r = fma2(bc(drho), pr(p.fbase[2 * k + 1], p.fbase[2 * k + 2]), FO[k]);
        fo[2 * k + 1] = r.x;
        fo[2 * k + 2] = r.y;
    }

    if (THERMAL) {
        // g = f_bar + S/2 + C/2 - f^eq through its moments (M00, M10, M01 of g vanish)
        const float dEg = dr2.x + dr2.y + 0.5f * (Es_ + Ec) - 2.0f * dRT - uu;
        const float dNg = (dr2.x - dr2.y) + 0.5f * (Ns_ + Nc) - (ux2 - uy2);
        const float dPig = r11 + 0.5f * Pis_ - uxy;
        // (M21, M12) of g: r21 + (M21 of S + C) / 2 - uy (RT + ux^2), and its mirror
        const float2 m3g = fma2(mul2(bc(-1.0f), usw), add2(bc(RT), u2), fma2(bc(0.5f), m3sc, r3));
        const float dM22g = dr22 + 0.5f * M22s_ - (dRT2 + RT * uu + ux2 * uy2);
        float g0, he0;
        float2 G[4], HE[4];
        eq3_pairs(rho, 0.0f, bc(0.0f), dEg, dNg, dPig, m3g, dM22g, g0, G);
        // 1/w_h = (1/w1 - 1/2)/Pr + 1/2 (lambda = mu c_p / Pr); 1/tau_hf = (Pr - 1) w1
        const float wh = rcp(mup * p.inv_Pr + 0.5f);
        const float kc = p.Pr_m1 * w1 * (1.0f - 0.5f * wh);
        dheq_pairs(p, rho, drho, u, u2, RT, dRT, m.Et, m.dEt, he0, HE);
        // Z_a = e_a . u - |u|^2 / 2, in the lane pairs
        const float hu = 0.5f * uu;
        const float2 Z[4] = {sub2(u, bc(hu)), fma2(u, bc(-1.0f), bc(-hu)), fma2(bc(ux), pr(1.0f, -1.0f), bc(uy - hu)),
                             fma2(bc(ux), pr(-1.0f, 1.0f), bc(-uy - hu))};
        ho[0] = h[0] - wh * (h[0] - he0) - kc * hu * g0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 hp = pr(h[2 * k + 1], h[2 * k + 2]);
            const float2 r = fma2(mul2(bc(kc), Z[k]), G[k], fma2(bc(-wh), sub2(hp, HE[k]), hp));
            ho[2 * k + 1] = r.x;
            ho[2 * k + 2] = r.y;
        }
        if (p.work) {
            // the power of the body force, (1 - w_h / 2) W_a F.u
            const float cq = (1.0f - 0.5f * wh) * (rho * (ax * ux + ay * uy));
            ho[0] += kW0 * cq;
#pragma unroll
            for (int q = 1; q < 9; ++q) ho[q] += (q < 5 ? kW1 : kW5) * cq;
        }
    }
}

// ---------------------------------------------------------------- walls (Section V)

template <int SIDE>
struct SideIdx;
// in: normal (inward) direction, ip = n + t, im = n - t, it = t, imt = -t; o* = opposites
template <>
struct SideIdx<SIDE_YM> {
    enum { in = 2, ip = 5, im = 6, it = 1, imt = 3, on = 4, op = 7, om = 8, nxv = 0, nyv = 1, txv = 1, tyv = 0 };
};
template <>
struct SideIdx<SIDE_YP> {
    enum { in = 4, ip = 8, im = 7, it = 1, imt = 3, on = 2, op = 6, om = 5, nxv = 0, nyv = -1, txv = 1, tyv = 0 };
};
template <>
struct SideIdx<SIDE_XM> {
    enum { in = 1, ip = 5, im = 8, it = 2, imt = 4, on = 3, op = 7, om = 6, nxv = 1, nyv = 0, txv = 0, tyv = 1 };
};
template <>
struct SideIdx<SIDE_XP> {
    enum { in = 3, ip = 6, im = 7, it = 2, imt = 4, on = 1, op = 8, om = 5, nxv = -1, nyv = 0, txv = 0, tyv = 1 };
};

// Non-equilibrium bounce-back for a tangentially moving wall, on transformed populations:
// wall density and both momentum components of Eq. 20 imposed, normal unknown closed by
// bounce-back of its non-equilibrium part.  Works on deviations directly: the scheme is
// linear and opposite directions have equal rest weights, whose known/incoming sums
// (f_rest over K plus twice over I) add up to exactly 1.  The wall density is carried as
// 1 + drho_w: an O(1) FP32 rho_w would round away the low bits of the density deviation,
// and rho_w u_w would then force the moving wall by ~1e-9 every step.
template <int SIDE>
__device__ __forceinline__ void zouhe(const DevParams& p, int x, int y, float* f) {
    using S = SideIdx<SIDE>;
    const float dsum = (f[0] + f[S::it] + f[S::imt]) + 2.0f * (f[S::on] + f[S::op] + f[S::om]);
    float drho_w, an, at;
    if (p.force_kind == FORCE_TAYLOR_GREEN) {
        float Fx, Fy;
        force_at(p, x, y, 0.0f, Fx, Fy);
        const float Fn = Fx * S::nxv + Fy * S::nyv, Ft = Fx * S::txv + Fy * S::tyv;
        drho_w = dsum - 0.5f * Fn;
        const float irw = 1.0f / (1.0f + drho_w);
        an = Fn * irw;
        at = Ft * irw;
    } else {
        an = (p.force_kind == FORCE_ACCEL) ? (p.ax * S::nxv + p.ay * S::nyv) : 0.0f;
        at = (p.force_kind == FORCE_ACCEL) ? (p.ax * S::txv + p.ay * S::tyv) : 0.0f;
        // rho_w = (1 + dsum) / (1 + an / 2), i.e. drho_w = (dsum - an / 2) / (1 + an / 2)
        drho_w = (dsum - 0.5f * an) / (1.0f + 0.5f * an);
    }
    const float rho_w = 1.0f + drho_w;
    const float Fn = rho_w * an, Ft = rho_w * at;
    const float uwt = p.wall_ux[SIDE] * S::txv + p.wall_uy[SIDE] * S::tyv;
    const float dn = -0.5f * rho_w * an * (1.0f - uwt * uwt);
    const float tdiff = f[S::it] - f[S::imt];
    const float mom = 0.5f * uwt + 0.5f * drho_w * uwt;  // rho_w u_w / 2
    f[S::in] = f[S::on] + dn;
    f[S::ip] = f[S::op] - 0.5f * tdiff + mom - 0.25f * Ft - 0.25f * Fn - 0.5f * dn;
    f[S::im] = f[S::om] + 0.5f * tdiff - mom + 0.25f * Ft - 0.25f * Fn - 0.5f * dn;
}

// Wall rebuild on deviations (f, h of the wall node; ff, hf of its interior neighbour).
template <bool THERMAL, int SIDE>
__device__ __forceinline__ void wall_rebuild_side(const DevParams& p, int x, int y, float* f, float* h,
                                                  const float* ff, const float* hf) {
    using S = SideIdx<SIDE>;
    const int kind = p.wall_kind[SIDE];
    const float uwx = p.wall_ux[SIDE], uwy = p.wall_uy[SIDE];
    const Macro mf = macro_of<THERMAL>(p, ff, hf, x + S::nxv, y + S::nyv);
    const bool adiabatic = THERMAL && p.wall_therm[SIDE] == THERM_ADIABATIC;
    const float RTw = THERMAL ? (adiabatic ? mf.RT : p.wall_RT[SIDE]) : p.RTp;
    const float dRTw = THERMAL ? (adiabatic ? mf.dRT : p.wall_dRT[SIDE]) : p.dRTp;
    if (kind == WALL_ZOUHE) {
        zouhe<SIDE>(p, x, y, f);
    } else if (kind == WALL_NEE) {
        // f_b = f^eq(rho_f, u_w, T_w) + [f_f - f^eq(rho_f, u_f, T_f)]
        float ew[9], ef[9];
        dfeq(p, mf.rho, mf.drho, uwx, uwy, dRTw, ew);
        dfeq(p, mf.rho, mf.drho, mf.ux, mf.uy, mf.dRT, ef);
#pragma unroll
        for (int q = 0; q < 9; ++q) f[q] = ff[q] + (ew[q] - ef[q]);
    } else {  // WALL_EQUILIBRIUM: f^eq - S/2 at the wall state
        const float rw = p.wall_rho[SIDE];
        const float dRTe = THERMAL ? p.wall_dRT[SIDE] : p.dRTp;
        float Fx, Fy;
        force_at(p, x, y, rw, Fx, Fy);
        float sw[9];
        dfeq(p, rw, rw - 1.0f, uwx, uwy, dRTe, f);
        source(rw, uwx, uwy, Fx / rw, Fy / rw, sw);
#pragma unroll
        for (int q = 0; q < 9; ++q) f[q] -= 0.5f * sw[q];
    }
    if (!THERMAL) return;
    if (kind == WALL_EQUILIBRIUM) {
        const float rw = p.wall_rho[SIDE];
        const float RTe = p.wall_RT[SIDE], dRTe = p.wall_dRT[SIDE];
        const float Ete = 0.5f * (p.b * RTe + uwx * uwx + uwy * uwy);
        const float dEte = 0.5f * p.b * dRTe + 0.5f * (uwx * uwx + uwy * uwy) + (0.5f * p.b * p.RT0 - p.Et0);
        dheq(p, rw, rw - 1.0f, uwx, uwy, RTe, dRTe, Ete, dEte, h);
        if (p.work) {  // h_bar^eq = h^eq - q / 2 at the wall state
            float Fx, Fy;
            force_at(p, x, y, rw, Fx, Fy);
            const float hq = 0.5f * (Fx * uwx + Fy * uwy);
#pragma unroll
            for (int q = 0; q < 9; ++q) h[q] -= (q == 0 ? kW0 : (q < 5 ? kW1 : kW5)) * hq;
        }
        return;
    }
    // temperature by non-equilibrium extrapolation around the rebuilt node's rho and u:
    // h_b = h^eq(rho_b, u_b, T_w) + [h_f - h^eq(rho_f, u_f, T_f)]
    const Macro mb = macro_of<false>(p, f, f, x, y);
    const float ke = 0.5f * (mb.ux * mb.ux + mb.uy * mb.uy);
    const float Etw = 0.5f * p.b * RTw + ke;
    const float dEtw = 0.5f * p.b * dRTw + ke + (0.5f * p.b * p.RT0 - p.Et0);
    float ew[9], ef[9];
    dheq(p, mb.rho, mb.drho, mb.ux, mb.uy, RTw, dRTw, Etw, dEtw, ew);
    dheq(p, mf.rho, mf.drho, mf.ux, mf.uy, mf.RT, mf.dRT, mf.Et, mf.dEt, ef);
    if (p.work) {  // the transformed equilibria h^eq - q / 2 of both nodes
        float Fbx, Fby, Ffx, Ffy;
        force_at(p, x, y, mb.rho, Fbx, Fby);
        force_at(p, x + S::nxv, y + S::nyv, mf.rho, Ffx, Ffy);
        const float hqb = 0.5f * (Fbx * mb.ux + Fby * mb.uy), hqf = 0.5f * (Ffx * mf.ux + Ffy * mf.uy);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float w = q == 0 ? kW0 : (q < 5 ? kW1 : kW5);
            ew[q] -= w * hqb;
            ef[q] -= w * hqf;
        }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) h[q] = hf[q] + (ew[q] - ef[q]);
}

__device__ __forceinline__ int wall_side_of(const DevParams& p, int x, int y) {
    if (!p.yper) {
        if (y == 0) return SIDE_YM;
        if (y == p.ny - 1) return SIDE_YP;
    }
    if (!p.xper) {
        if (x == 0) return SIDE_XM;
        if (x == p.nx - 1) return SIDE_XP;
    }
    return -1;
}

// Streamed (pulled) populations of node (x, y) at t+1 from the source copy.  Sources
// outside a walled axis are clamped into range; the wall scheme replaces them.
template <bool THERMAL, class ST>
__device__ __forceinline__ void pull(const DevParams& p, const ST* __restrict__ src, int x, int y, float* f,
                                     float* h) {
    const int nx = p.nx, ny = p.ny;
    int xm = x - 1, xp = x + 1, ym = y - 1, yp = y + 1;
    if (p.xper) {
        xm = xm < 0 ? nx - 1 : xm;
        xp = xp >= nx ? 0 : xp;
    } else {
        xm = xm < 0 ? 0 : xm;
        xp = xp >= nx ? nx - 1 : xp;
    }
    if (p.yper) {
        ym = ym < 0 ? ny - 1 : ym;
        yp = yp >= ny ? 0 : yp;
    } else {
        ym = ym < 0 ? 0 : ym;
        yp = yp >= ny ? ny - 1 : yp;
    }
    const long long P = p.plane;
    const long long r0 = (long long)y * p.pitch, rm = (long long)ym * p.pitch, rp = (long long)yp * p.pitch;
    const long long idx[9] = {r0 + x, r0 + xm, rm + x, r0 + xp, rp + x, rm + xm, rm + xp, rp + xp, rp + xm};
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = Store<ST>::ld(src + q * P + idx[q]);
    if (THERMAL) {
#pragma unroll
        for (int q = 0; q < 9; ++q) h[q] = Store<ST>::ld(src + (9 + q) * P + idx[q]);
    }
}

template <bool THERMAL>
__device__ __forceinline__ void wall_rebuild(const DevParams& p, int side, int x, int y, float* f, float* h,
                                          const float* ff, const float* hf) {
    switch (side) {
        case SIDE_YM: wall_rebuild_side<THERMAL, SIDE_YM>(p, x, y, f, h, ff, hf); break;
        case SIDE_YP: wall_rebuild_side<THERMAL, SIDE_YP>(p, x, y, f, h, ff, hf); break;
        case SIDE_XM: wall_rebuild_side<THERMAL, SIDE_XM>(p, x, y, f, h, ff, hf); break;
        default: wall_rebuild_side<THERMAL, SIDE_XP>(p, x, y, f, h, ff, hf); break;
    }
}

// The same, out of line, for kernels whose interior loop must stay compact in the
// instruction cache (the TMA-fed kernels: wall code inlined at each of their five pull
// sites cost the FP32 kernel 10 % of its time in a wall-free comparison build; the
// direct-load kernels run faster with it inlined).  io holds f, h of the wall node and
// ff, hf of its interior neighbour (36 values); f, h are rewritten.
template <bool THERMAL>
__device__ __noinline__ void wall_rebuild_out_of_line(const DevParams* pp, int side, int x, int y, float* io) {
    float f[9], h[9], ff[9], hf[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        f[q] = io[q];
        h[q] = io[9 + q];
        ff[q] = io[18 + q];
        hf[q] = io[27 + q];
    }
    wall_rebuild<THERMAL>(*pp, side, x, y, f, h, ff, hf);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        io[q] = f[q];
        io[9 + q] = h[q];
    }
}

// Call site of the out-of-line rebuild: the node's values are copied into a scratch
// array, so only the wall branch touches local memory and f, h stay in registers.
// `p` must be addressable without a copy (a __grid_constant__ kernel parameter or
// shared memory).
template <bool THERMAL>
__device__ __forceinline__ void wall_rebuild_call(const DevParams& p, int side, int x, int y, float* f, float* h,
                                               const float* ff, const float* hf) {
    float io[36];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        io[q] = f[q];
        io[9 + q] = THERMAL ? h[q] : 0.0f;
        io[18 + q] = ff[q];
        io[27 + q] = THERMAL ? hf[q] : 0.0f;
    }
    wall_rebuild_out_of_line<THERMAL>(&p, side, x, y, io);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        f[q] = io[q];
        if (THERMAL) h[q] = io[9 + q];
    }
}

// Streamed populations of node (x, y) with its wall scheme applied (the state at t+1
// that Eq. 20 reads), as deviations from the rest state.
template <bool THERMAL, class ST>
__device__ __forceinline__ void load_node(const DevParams& p, const ST* __restrict__ src, int x, int y, float* f,
                                          float* h) {
    pull<THERMAL, ST>(p, src, x, y, f, h);
    const int side = wall_side_of(p, x, y);
    if (side >= 0) {
        const int nxv = side == SIDE_XM ? 1 : (side == SIDE_XP ? -1 : 0);
        const int nyv = side == SIDE_YM ? 1 : (side == SIDE_YP ? -1 : 0);
        float ff[9], hf[9];
        pull<THERMAL, ST>(p, src, x + nxv, y + nyv, ff, hf);
        wall_rebuild<THERMAL>(p, side, x, y, f, h, ff, hf);
    }
}

template <class ST>
__device__ __forceinline__ void store_node(const DevParams& p, ST* __restrict__ dst, int x, int y, const float* f,
                                           const float* h, bool thermal) {
    const long long P = p.plane, o = (long long)y * p.pitch + x;
    if (sizeof(ST) == 2 && p.rounding) {
        // stochastic rounding, two planes per conversion
        const uint32_t step = p.step_ctr[p.parity];
        const uint32_t node = (uint32_t)(y * p.nx + x);
        const uint32_t seed = sr_bits(node, 0u, step);  // one full mix per node
        float v[18];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            v[q] = f[q];
            v[9 + q] = thermal ? h[q] : 0.0f;
        }
        const int npl = thermal ? 18 : 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (2 * k >= npl) break;
            const uint32_t d = cvt_rs_pair<ST>(v[2 * k + 1], v[2 * k], sr_pair_bits(seed, (uint32_t)k));
            const unsigned short lo = (unsigned short)(d & 0xffffu), hi = (unsigned short)(d >> 16);
            reinterpret_cast<unsigned short*>(dst)[(2 * k) * P + o] = lo;
            if (2 * k + 1 < npl) reinterpret_cast<unsigned short*>(dst)[(2 * k + 1) * P + o] = hi;
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) Store<ST>::st(dst + q * P + o, f[q]);
    if (thermal) {
#pragma unroll
        for (int q = 0; q < 9; ++q) Store<ST>::st(dst + (9 + q) * P + o, h[q]);
    }
}

// Advances the stochastic-rounding step counter for the next launch (thread 0 of the
// one CTA that owns the lattice's first strip and row).
__device__ __forceinline__ void bump_step_counter(const DevParams& p) {
    if (p.rounding && threadIdx.x == 0) p.step_ctr[p.parity ^ 1] = p.step_ctr[p.parity] + 1u;
}

// ---------------------------------------------------------------- the fused step

// Strip [x0, x0 + TX) x rows [y0, y1) without the correction term: no neighbour
// moments, one row at a time.
template <int TX, bool THERMAL, class ST>
__device__ __forceinline__ void strip_plain(const DevParams& p, const ST* __restrict__ src, ST* __restrict__ dst,
                                            int x0, int y0, int y1) {
    const int x = x0 + threadIdx.x;
    if (x >= p.nx) return;
    for (int y = y0; y < y1; ++y) {
        float f[9], h[9], fo[9], ho[9];
        load_node<THERMAL, ST>(p, src, x, y, f, h);
        const Macro m = macro_of<THERMAL>(p, f, h, x, y);
        collide<THERMAL>(p, f, h, m, 0.0f, 0.0f, fo, ho);
        store_node<ST>(p, dst, x, y, fo, ho, THERMAL);
    }
}

// Strip with the correction term (thermal): lookahead of one row in registers, the
// x-derivative from a three-row ring of u_x(1-theta) in shared memory with a
// two-column halo on each side (computed by four designated threads).  Every thread
// of the CTA must call it (it synchronises once per row).
template <int TX, class ST>
__device__ __forceinline__ void strip_corr(const DevParams& p, const ST* __restrict__ src, ST* __restrict__ dst,
                                           int x0, int y0, int y1, float (*ring)[TX + 4]) {
    const int tid = threadIdx.x;
    const int nx = p.nx, ny = p.ny;

    // own column (slot tid + 2) and, for four threads, one halo slot
    const int xl = x0 + tid;
    const bool owns = xl < nx;
    const int xown = p.xper ? (xl % nx) : xl;
    const bool own_valid = p.xper || owns;
    int hslot = -1, xh = 0;
    bool h_valid = false;
    if ((tid % (TX / 4)) == 0) {
        const int k = tid / (TX / 4);  // 0..3 -> slots 0, 1, TX+2, TX+3
        hslot = k < 2 ? k : TX + k;
        const int xlh = x0 - 2 + hslot;
        if (p.xper) {
            xh = ((xlh % nx) + nx) % nx;
            h_valid = true;
        } else {
            xh = xlh;
            h_valid = xlh >= 0 && xlh < nx;
        }
    }
    const bool ywall = !p.yper;

    // phi_y ring in registers: rows r-2, r-1, r, r+1
    float py_m2 = 0.f, py_m1 = 0.f, py_0 = 0.f, py_p1 = 0.f;
    float fc[9], hc[9], fn[9], hn[9];
    Macro mc, mn;

    auto row_phys = [&](int r) { return p.yper ? ((r % ny) + ny) % ny : r; };
    auto compute_row = [&](int r, float* f, float* h, Macro& m, float& py, int buf) {
        const int yr = row_phys(r);
        if (own_valid) {
            load_node<true, ST>(p, src, xown, yr, f, h);
            m = macro_of<true>(p, f, h, xown, yr);
            ring[buf][tid + 2] = phi_x(m);
            py = phi_y(m);
        }
        if (hslot >= 0 && h_valid) {
            float fh[9], hh[9];
            load_node<true, ST>(p, src, xh, yr, fh, hh);
            const Macro mh = macro_of<true>(p, fh, hh, xh, yr);
            ring[buf][hslot] = phi_x(mh);
        }
    };
    auto phiy_only = [&](int r) -> float {
        const int yr = row_phys(r);
        if (!own_valid) return 0.f;
        float f[9], h[9];
        load_node<true, ST>(p, src, xown, yr, f, h);
        const Macro m = macro_of<true>(p, f, h, xown, yr);
        return phi_y(m);
    };

    // prologue; a top-wall row closer than two rows to the segment start reads phi_y(r-2)
    if (y0 > 0 || p.yper) py_m1 = phiy_only(y0 - 1);
    if (ywall && y1 == ny && y0 >= 2 && y1 - y0 < 3) py_m2 = phiy_only(y0 - 2);
    compute_row(y0, fc, hc, mc, py_0, y0 % 3);
    __syncthreads();  // the prologue's phi_x row is read by the first collision

    // the lookahead of row r+1 and the collision of row r share one block between
    // barriers (the collision reads the phi_x row published one barrier earlier)
    for (int r = y0; r < y1; ++r) {
        const bool has_next = (r + 1 < ny) || p.yper;
        if (has_next) compute_row(r + 1, fn, hn, mn, py_p1, (r + 1) % 3);
        float py_p2 = 0.f;
        if (ywall && r == 0) py_p2 = phiy_only(2);
        if (owns) {
            const float* rw = ring[r % 3];
            const int s = tid + 2;
            float dxv;
            if (!p.xper && xl == 0)
                dxv = 0.5f * (-3.0f * rw[s] + 4.0f * rw[s + 1] - rw[s + 2]);
            else if (!p.xper && xl == nx - 1)
                dxv = 0.5f * (3.0f * rw[s] - 4.0f * rw[s - 1] + rw[s - 2]);
            else
                dxv = 0.5f * (rw[s + 1] - rw[s - 1]);
            float dyv;
            if (ywall && r == 0)
                dyv = 0.5f * (-3.0f * py_0 + 4.0f * py_p1 - py_p2);
            else if (ywall && r == ny - 1)
                dyv = 0.5f * (3.0f * py_0 - 4.0f * py_m1 + py_m2);
            else
                dyv = 0.5f * (py_p1 - py_m1);
            float fo[9], ho[9];
            collide<true>(p, fc, hc, mc, dxv, dyv, fo, ho);
            store_node<ST>(p, dst, xl, r, fo, ho, true);
        }
        __syncthreads();  // phi_x of row r+1 complete; the buffer of row r-1 free again
        py_m2 = py_m1;
        py_m1 = py_0;
        py_0 = py_p1;
        mc = mn;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            fc[q] = fn[q];
            hc[q] = hn[q];
        }
    }
}

__device__ __forceinline__ void segment_rows(const DevParams& p, int rows_per_cta, int& y0, int& y1) {
    y0 = blockIdx.y * rows_per_cta;
    y1 = (blockIdx.y == gridDim.y - 1) ? p.ny : y0 + rows_per_cta;
}

template <int TX, bool THERMAL, class ST>
__global__ void __launch_bounds__(TX, 512 / TX) tclbm_step_plain(const DevParams p, const ST* __restrict__ src,
                                                                 ST* __restrict__ dst, int rows_per_cta) {
    int y0, y1;
    segment_rows(p, rows_per_cta, y0, y1);
    strip_plain<TX, THERMAL, ST>(p, src, dst, blockIdx.x * TX, y0, y1);
    if (blockIdx.x == 0 && blockIdx.y == 0) bump_step_counter(p);
}

template <int TX, class ST>
__global__ void __launch_bounds__(TX, 512 / TX) tclbm_step_corr(const DevParams p, const ST* __restrict__ src,
                                                                ST* __restrict__ dst, int rows_per_cta) {
    __shared__ float ring[3][TX + 4];
    int y0, y1;
    segment_rows(p, rows_per_cta, y0, y1);
    strip_corr<TX, ST>(p, src, dst, blockIdx.x * TX, y0, y1, ring);
    if (blockIdx.x == 0 && blockIdx.y == 0) bump_step_counter(p);
}

// ---------------------------------------------------------------- 2-D tiles

// The step with the correction term on BX x BY node tiles, one node per thread: each
// thread pulls its node and, for the 2 (BX + BY) threads with the highest indices, one
// halo node (the columns x0-1, x0+BX and rows y0-1, y0+BY around the tile) in the same
// phase, evaluates the moments and phi = u (1 - 3RT) into shared memory, and after one
// barrier takes the derivatives and collides.  No thread marches over rows, so a
// lattice of one short wave finishes its step after a single dependent chain of loads
// and arithmetic.  Threads of a partial tile on a periodic axis stand in for the
// wrapped column or row.  Requires nx % BX != 1 unless x is periodic, and ny % BY != 1
// unless y is periodic (the one-sided derivative at a wall then finds its two
// neighbours inside the tile or its halo).  Same per-node code as strip_corr.
// LATE_WAIT: the wait for the previous step's grid (programmatic dependent launch) comes
// just before the first load instead of at kernel entry (the caller then omits it).
template <int BX, int BY, class ST, bool LATE_WAIT = false>
__device__ __forceinline__ void tile_step(const DevParams& p, const ST* __restrict__ src, ST* __restrict__ dst,
                                          int x0, int y0, float (*phx)[BX + 2], float (*phy)[BX]) {
    static_assert(2 * (BX + BY) <= BX * BY, "every halo node needs a thread");
    static_assert(BX >= 3 && BY >= 3, "a wall's one-sided derivative reads two nodes inside the tile");
    const int nx = p.nx, ny = p.ny;
    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    const int x = x0 + tx, y = y0 + ty;
    const bool owns = x < nx && y < ny;
    const bool in_x = p.xper || x < nx, in_y = p.yper || y < ny;
    const int xw = x < nx ? x : x - nx, yw = y < ny ? y : y - ny;  // wrapped (periodic) position
    const bool node_valid = in_x && in_y && xw < nx && yw < ny;

    // halo node of this thread, taken by the last 2 (BX + BY) threads, so that the halo
    // columns of a wall row land in another warp than the wall row's own nodes: halo
    // index u < 2 BY -> column x0-1 / x0+BX at row y0 + u % BY; u < 2 (BX + BY) -> row
    // y0-1 / y0+BY at column x0 + (u - 2 BY) % BX
    const int u = (int)threadIdx.x - (BX * BY - 2 * (BX + BY));
    int hx = 0, hy = 0;
    bool h_col = false, h_row = false;
    if (u >= 0 && u < 2 * BY) {
        h_col = true;
        hx = u < BY ? x0 - 1 : x0 + BX;
        hy = y0 + u % BY;
    } else if (u >= 2 * BY) {
        h_row = true;
        const int v = u - 2 * BY;
        hx = x0 + v % BX;
        hy = v < BX ? y0 - 1 : y0 + BY;
    }
    bool h_valid = h_col || h_row;
    if (h_valid) {
        if (p.xper)
            hx = ((hx % nx) + nx) % nx;
        else
            h_valid = hx >= 0 && hx < nx;
        if (p.yper)
            hy = ((hy % ny) + ny) % ny;
        else
            h_valid = h_valid && hy >= 0 && hy < ny;
    }

    // every pull in one phase: own node, halo node, and the interior neighbours that
    // the wall schemes of a wall node (own or halo) read
    const int side_o = node_valid ? wall_side_of(p, xw, yw) : -1;
    const int side_h = h_valid ? wall_side_of(p, hx, hy) : -1;
    float f[9], h[9], fh[9], hh[9], fn[9], hn[9], fhn[9], hhn[9];
    // everything above reads only the parameters, so it may overlap the tail of the
    // previous step's grid, whose writes are this step's source
    if (LATE_WAIT) asm volatile("griddepcontrol.wait;" ::: "memory");
    if (node_valid) pull<true, ST>(p, src, xw, yw, f, h);
    if (h_valid) pull<true, ST>(p, src, hx, hy, fh, hh);
    if (side_o >= 0)
        pull<true, ST>(p, src, xw + (side_o == SIDE_XM ? 1 : (side_o == SIDE_XP ? -1 : 0)),
                       yw + (side_o == SIDE_YM ? 1 : (side_o == SIDE_YP ? -1 : 0)), fn, hn);
    if (side_h >= 0)
        pull<true, ST>(p, src, hx + (side_h == SIDE_XM ? 1 : (side_h == SIDE_XP ? -1 : 0)),
                       hy + (side_h == SIDE_YM ? 1 : (side_h == SIDE_YP ? -1 : 0)), fhn, hhn);
    Macro m;
    if (node_valid) {
        if (side_o >= 0) wall_rebuild<true>(p, side_o, xw, yw, f, h, fn, hn);
        m = macro_of<true>(p, f, h, xw, yw);
        phx[ty][tx + 1] = phi_x(m);
        phy[ty + 1][tx] = phi_y(m);
    }
    if (h_valid) {
        if (side_h >= 0) wall_rebuild<true>(p, side_h, hx, hy, fh, hh, fhn, hhn);
        const Macro mh = macro_of<true>(p, fh, hh, hx, hy);
        if (h_col)
            phx[u % BY][u < BY ? 0 : BX + 1] = phi_x(mh);
        else
            phy[u - 2 * BY < BX ? 0 : BY + 1][(u - 2 * BY) % BX] = phi_y(mh);
    }
    __syncthreads();
    if (owns) {
        const float* rw = phx[ty];
        const int s = tx + 1;
        float dxv;
        if (!p.xper && x == 0)
            dxv = 0.5f * (-3.0f * rw[s] + 4.0f * rw[s + 1] - rw[s + 2]);
        else if (!p.xper && x == nx - 1)
            dxv = 0.5f * (3.0f * rw[s] - 4.0f * rw[s - 1] + rw[s - 2]);
        else
            dxv = 0.5f * (rw[s + 1] - rw[s - 1]);
        const int r = ty + 1;
        float dyv;
        if (!p.yper && y == 0)
            dyv = 0.5f * (-3.0f * phy[r][tx] + 4.0f * phy[r + 1][tx] - phy[r + 2][tx]);
        else if (!p.yper && y == ny - 1)
            dyv = 0.5f * (3.0f * phy[r][tx] - 4.0f * phy[r - 1][tx] + phy[r - 2][tx]);
        else
            dyv = 0.5f * (phy[r + 1][tx] - phy[r - 1][tx]);
        float fo[9], ho[9];
        collide<true>(p, f, h, m, dxv, dyv, fo, ho);
        store_node<ST>(p, dst, x, y, fo, ho, true);
    }
}

// One lattice: CTA (bx, by) takes the tile at (bx BX, by BY).  Programmatic dependent
// launch: the kernel waits for the previous step's grid (its writes are this step's
// source) at entry, or with LATE_WAIT just before its first load, and lets the next
// step's grid be scheduled behind it.  Measured at 32 x 4: the late wait is 6 % faster
// on grids of more than one wave of resident CTAs (512 x 256) and 4 % slower on one
// short wave (256 x 128), where the next grid's early prologue competes with this one.
template <int BX, int BY, class ST, bool LATE_WAIT = false>
__global__ void __launch_bounds__(BX * BY, 512 / (BX * BY)) tclbm_step_tile(const DevParams p, const ST* __restrict__ src,
                                                              ST* __restrict__ dst) {
    __shared__ float phx[BY][BX + 2];  // phi_x of columns x0-1 .. x0+BX
    __shared__ float phy[BY + 2][BX];  // phi_y of rows y0-1 .. y0+BY
    if (!LATE_WAIT) asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    tile_step<BX, BY, ST, LATE_WAIT>(p, src, dst, blockIdx.x * BX, blockIdx.y * BY, phx, phy);
    if (blockIdx.x == 0 && blockIdx.y == 0) bump_step_counter(p);
}

}  // namespace tclbm
