// tclbm_api.cu -- host side of the C ABI declared in include/tclbm.h: parameter
// validation and derived constants, device memory, the step loop (CUDA graphs for
// short launches), field initialisation, moments, FP64 diagnostics and population
// transfer kernels.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdarg>
#include <cstring>
#include <type_traits>
#include <new>

#include "tclbm.h"
#include "tclbm_device.cuh"
#include "tclbm_internal.h"
#include "tclbm_launch.h"

using namespace tclbm;

namespace {
thread_local char g_err[512] = "";
}  // namespace

tclbm_status tclbm::fail(tclbm_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

tclbm_status tclbm::cuda_fail(cudaError_t e, const char* what) {
    return fail(TCLBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {
constexpr int kDiagBlock = 256;
constexpr int kDiagMaxBlocks = 1024;
}  // namespace

void tclbm::set_last_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

void* tclbm::dev_alloc(tclbm_lattice* L, size_t bytes) {
    if (bytes == 0) return nullptr;
    if (L->alloc) return L->alloc(bytes, (void*)L->stream, L->ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void tclbm::dev_free(tclbm_lattice* L, void* p, size_t bytes) {
    if (!p) return;
    if (L->free_fn)
        L->free_fn(p, bytes, (void*)L->stream, L->ctx);
    else
        cudaFree(p);
}

namespace {

bool walls_ok(const tclbm_params* p) {
    for (int s = 0; s < 4; ++s) {
        const int k = p->wall[s].kind;
        if (k < TCLBM_WALL_PERIODIC || k > TCLBM_WALL_EQUILIBRIUM) return false;
        if (p->wall[s].therm != TCLBM_THERM_FIXED_T && p->wall[s].therm != TCLBM_THERM_ADIABATIC) return false;
    }
    return true;
}

tclbm_status validate(const tclbm_params* p) {
    if (!p) return fail(TCLBM_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(TCLBM_EINVAL, "nx, ny must be >= 1 (got %d, %d)", p->nx, p->ny);
    if ((long long)p->nx * p->ny > (1LL << 34)) return fail(TCLBM_EINVAL, "lattice too large");
    if (!walls_ok(p)) return fail(TCLBM_EINVAL, "unknown wall kind or thermal treatment");
    const bool xper = p->wall[TCLBM_SIDE_XM].kind == TCLBM_WALL_PERIODIC;
    const bool yper = p->wall[TCLBM_SIDE_YM].kind == TCLBM_WALL_PERIODIC;
    if (xper != (p->wall[TCLBM_SIDE_XP].kind == TCLBM_WALL_PERIODIC) ||
        yper != (p->wall[TCLBM_SIDE_YP].kind == TCLBM_WALL_PERIODIC))
        return fail(TCLBM_EINVAL, "opposite sides must both be periodic or both walls");
    if (!xper && !yper) return fail(TCLBM_EUNSUPPORTED, "walls on both axes are not supported");
    if (!xper && p->nx < 3) return fail(TCLBM_EINVAL, "a walled x axis needs nx >= 3");
    if (!yper && p->ny < 3) return fail(TCLBM_EINVAL, "a walled y axis needs ny >= 3");
    if (!(p->gamma > 1.0) || !(p->Pr > 0.0) || !(p->R > 0.0) || !(p->T0 > 0.0))
        return fail(TCLBM_EINVAL, "gamma > 1, Pr > 0, R > 0, T0 > 0 required");
    if (p->visc_law < TCLBM_VISC_NU || p->visc_law > TCLBM_VISC_W1) return fail(TCLBM_EINVAL, "bad visc_law");
    if (p->visc_law == TCLBM_VISC_W1 ? !(p->visc > 0.0 && p->visc < 2.0) : !(p->visc > 0.0))
        return fail(TCLBM_EINVAL, "viscosity (or w1) out of range");
    if (!p->bgk)
        for (double w : {p->w2, p->w3, p->w4})
            if (!(w > 0.0 && w < 2.0)) return fail(TCLBM_EINVAL, "w2, w3, w4 must lie in (0, 2)");
    if (p->force_kind < TCLBM_FORCE_NONE || p->force_kind > TCLBM_FORCE_TAYLOR_GREEN)
        return fail(TCLBM_EINVAL, "bad force_kind");
    if (p->correction && !p->thermal) return fail(TCLBM_EINVAL, "the correction term needs thermal = 1");
    if (p->work && !p->thermal) return fail(TCLBM_EINVAL, "the work term needs thermal = 1");
    if (p->storage < TCLBM_STORE_FP32 || p->storage > TCLBM_STORE_FP16) return fail(TCLBM_EINVAL, "bad storage");
    if (p->rounding != TCLBM_ROUND_NEAREST && p->rounding != TCLBM_ROUND_STOCHASTIC)
        return fail(TCLBM_EINVAL, "bad rounding");
    return TCLBM_OK;
}

int pitch_of(int nx) { return (nx + 31) / 32 * 32; }

size_t elem_of(int storage) { return storage == TCLBM_STORE_FP32 ? 4 : 2; }

void derive(tclbm_lattice* L) {
    const tclbm_params& p = L->prm;
    DevParams& d = L->dp;
    memset(&d, 0, sizeof d);
    d.skip_row = -1;  // the timeout test hook is off
    d.nx = p.nx;
    d.ny = p.ny;
    d.pitch = pitch_of(p.nx);
    d.plane = (long long)p.ny * d.pitch;
    d.xper = p.wall[TCLBM_SIDE_XM].kind == TCLBM_WALL_PERIODIC;
    d.yper = p.wall[TCLBM_SIDE_YM].kind == TCLBM_WALL_PERIODIC;
    d.visc_law = p.visc_law;
    d.visc = (float)p.visc;
    d.w2 = (float)p.w2;
    d.w3 = (float)p.w3;
    d.w4 = (float)p.w4;
    d.bgk = p.bgk;
    const double b = 2.0 / (p.gamma - 1.0);
    d.R = (float)p.R;
    d.T0 = (float)p.T0;
    d.b = (float)b;
    d.two_over_b = (float)(2.0 / b);
    d.inv_R = (float)(1.0 / p.R);
    // Rest state of the deviations: RT0 and Et0 on a 2^-10 grid near R T0 and b R T0 / 2,
    // so that f^eq(1, 0, RT0), h^eq(1, 0, RT0) and their moment identities are exact in
    // float (each value needs at most 21 significant bits).
    const double RTb = std::max(1.0, std::round(p.R * p.T0 * 1024.0)) / 1024.0;
    const double Etb = std::max(1.0, std::round(0.5 * b * RTb * 1024.0)) / 1024.0;
    d.RT0 = (float)RTb;
    d.Et0 = (float)Etb;
    d.cRT = (float)(2.0 / b * Etb - RTb);
    d.RTp = (float)(p.R * p.T0);
    d.inv_RTp = (float)(1.0 / (p.R * p.T0));
    d.inv_w1_fixed = p.visc_law == TCLBM_VISC_W1 ? (float)(1.0 / p.visc) : 0.0f;
    d.inv_Pr = (float)(1.0 / p.Pr);
    d.Pr_m1 = (float)(p.Pr - 1.0);
    d.force_kind = p.force_kind;
    d.ax = (float)p.ax;
    d.ay = (float)p.ay;
    d.famp = (float)p.famp;
    d.rounding = p.storage != TCLBM_STORE_FP32 && p.rounding == TCLBM_ROUND_STOCHASTIC;
    for (int s = 0; s < 4; ++s) {
        d.wall_kind[s] = p.wall[s].kind;
        d.wall_therm[s] = p.wall[s].therm;
        d.wall_rho[s] = (float)p.wall[s].rho;
        d.wall_ux[s] = (float)p.wall[s].ux;
        d.wall_uy[s] = (float)p.wall[s].uy;
        d.wall_T[s] = (float)p.wall[s].T;
        d.wall_RT[s] = (float)(p.R * p.wall[s].T);
        d.wall_dRT[s] = (float)(p.R * p.wall[s].T - RTb);
    }
    d.dRTp = (float)(p.R * p.T0 - RTb);
    d.inv_bR2 = 2.0 / (b * p.R);  // the same FP64 expression tclbm_diagnostics_noalloc() takes
    d.work = p.thermal && p.work;
    d.T0d = p.T0;
    // rest-state populations f^eq(1, 0, RT0), h^eq(1, 0, RT0) with Et = Et0
    const double x0 = 1.0 - RTb, x1 = 0.5 * RTb;
    const double fr[9] = {x0 * x0, x1 * x0, x0 * x1, x1 * x0, x0 * x1, x1 * x1, x1 * x1, x1 * x1, x1 * x1};
    const double C0 = RTb * (Etb + RTb);
    const double hr[9] = {Etb - 2.0 * C0, 0.5 * C0, 0.5 * C0, 0.5 * C0, 0.5 * C0, 0, 0, 0, 0};
    for (int q = 0; q < 9; ++q) {
        d.fbase[q] = (float)fr[q];
        d.hbase[q] = p.thermal ? (float)hr[q] : 0.0f;
    }
}

// Lattices that fit in L2 are latency-bound: 2-D tiles of one node per thread (or the
// direct-load kernel with short strips where tiles do not apply) expose the most
// parallelism.  Larger lattices stream rows through the TMA ring with 128-wide strips
// of 16 or 32 rows per CTA (default_shape).
constexpr long long kSmallNodes = 1LL << 21;

// Launch shape a kernel variant gets by default: (tx, rows per CTA) for the marching
// kernels, the tile (BX, BY) for KERNEL_TILE.
void default_shape(const tclbm_params& p, int kernel, int& tx, int& ty) {
    if (kernel == KERNEL_TILE) {
        tx = kTileBX;
        ty = kTileBY;
    } else if (kernel == KERNEL_DIRECT) {
        tx = p.nx >= 96 ? 64 : 32;
        const long long strips = (p.nx + tx - 1) / tx;
        long long t = (long long)p.ny * strips / (8LL * 152);
        ty = (int)(t < 2 ? 2 : (t > 16 ? 16 : t));
    } else {
        // 16 rows per CTA, or 32 (fewer halo rows per node) where the last wave's tail
        // weighs little: where the 32-row grid spans more than two waves of the kernel's
        // resident CTAs, so its tail of half-height segments applies (ny a multiple of 8),
        // else where it spans at least 8 waves.  Measured with the short tail: 32 rows tie
        // 16 at 4096 x 2048 and beat it by 1 % at 2048 x 2048 (FP32) and by 4-5 % at
        // 8192 x 4096; 16 rows win by 12-20 % where the 32-row grid has no short tail
        // (FP16 2048 x 2048, athermal 2048 x 2048).
        tx = p.nx >= 512 ? 128 : (p.nx >= 96 ? 64 : 32);
        const long long strips = (p.nx + tx - 1) / tx;
        const long long resident = tma_resident(p.storage, tx, p.thermal && p.correction, p.thermal);
        // Chained launches (tclbm_step: the correction-term kernel, FP32 or 16-bit with
        // round-to-nearest) overlap consecutive steps, so the tail no longer sets the
        // segment height: the tallest of 96, 64 and 48 rows whose grid still spans three
        // waves of resident CTAs (measured against 16-96 rows: 4096 x 2048 FP32 takes 48
        // rows, 0.722 -> 0.740 of peak; 8192 x 4096 takes 96, FP32 0.738 -> 0.779, FP16
        // 0.389 -> 0.405); grids that reach three waves at none of them keep the rule below.
        const bool chained = p.thermal && p.correction &&
                             (p.storage == TCLBM_STORE_FP32 || p.rounding == TCLBM_ROUND_NEAREST);
        if (chained) {
            DevParams d = {};
            d.nx = p.nx;
            d.ny = p.ny;
            for (int rows : {96, 64, 48}) {
                const SegPlan plan = tma_seg_plan(d, tx, rows, resident);
                if (strips * (plan.full + plan.half) >= 3 * resident) {
                    ty = rows;
                    return;
                }
            }
        }
        if (p.ny % 8 == 0)
            ty = strips * (p.ny / 32) > 2 * resident ? 32 : 16;
        else
            ty = strips * ((p.ny + 31) / 32) >= 8 * resident ? 32 : 16;
    }
}

bool tile_fits(const tclbm_params& p, int bx, int by) {
    const bool xper = p.wall[TCLBM_SIDE_XM].kind == TCLBM_WALL_PERIODIC;
    const bool yper = p.wall[TCLBM_SIDE_YM].kind == TCLBM_WALL_PERIODIC;
    return tile_kernel_fits(p.nx, p.ny, xper, yper, p.thermal, p.correction, bx, by);
}

void default_launch(const tclbm_params& p, int& tx, int& ty, int& kernel) {
    const long long n = (long long)p.nx * p.ny;
    if (n <= kSmallNodes)
        kernel = tile_fits(p, kTileBX, kTileBY) ? KERNEL_TILE : KERNEL_DIRECT;
    else
        kernel = KERNEL_TMA;
    default_shape(p, kernel, tx, ty);
}

void default_tile(const tclbm_params& p, int kernel, int& tx, int& ty) { default_shape(p, kernel, tx, ty); }

// ------------------------------------------------------------------ small kernels

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// f_bar = f^eq - S/2, h_bar = h^eq at each node (FP64), written where the pull of the
// next step reads it: buffer_q(x - e_q) = value_q(x).
template <class ST>
__global__ void init_kernel(const DevParams p, const double* __restrict__ rho, const double* __restrict__ ux,
                            const double* __restrict__ uy, const double* __restrict__ T, ST* __restrict__ dst,
                            int thermal, double R, double T0, double b, int force_kind, double ax, double ay,
                            double famp) {
    const long long n = (long long)p.nx * p.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % p.nx), y = (int)(i / p.nx);
        const double r = rho[i], vx = ux[i], vy = uy[i], t = thermal ? T[i] : T0;
        double Fx = 0, Fy = 0;
        if (force_kind == FORCE_ACCEL) {
            Fx = r * ax;
            Fy = r * ay;
        } else if (force_kind == FORCE_TAYLOR_GREEN) {
            const double kx = 6.283185307179586 / p.nx, ky = 6.283185307179586 / p.ny;
            Fx = famp * sin(kx * x) * sin(ky * y);
            Fy = famp * cos(kx * x) * cos(ky * y);
        }
        const double Ax = Fx / r, Ay = Fy / r, RT = R * t;
        const double ux2 = vx * vx, uy2 = vy * vy;
        const double px[3] = {1.0 - RT - ux2, 0.5 * (RT + ux2 + vx), 0.5 * (RT + ux2 - vx)};  // e = 0, +1, -1
        const double py[3] = {1.0 - RT - uy2, 0.5 * (RT + uy2 + vy), 0.5 * (RT + uy2 - vy)};
        const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        // S by Eq. 3 of its raw moments
        const double sE = 2 * (Ax * vx + Ay * vy), sN = 2 * (Ax * vx - Ay * vy), sP = Ax * vy + Ay * vx;
        const double s21 = Ay * ux2 + 2 * Ax * vx * vy, s12 = Ax * uy2 + 2 * Ay * vx * vy;
        const double s22 = 2 * Ax * vx * uy2 + 2 * Ay * vy * ux2;
        const double S[9] = {r * (-sE + s22),
                             0.5 * r * (Ax + 0.5 * (sE + sN) - s12 - s22),
                             0.5 * r * (Ay + 0.5 * (sE - sN) - s21 - s22),
                             0.5 * r * (-Ax + 0.5 * (sE + sN) + s12 - s22),
                             0.5 * r * (-Ay + 0.5 * (sE - sN) + s21 - s22),
                             0.25 * r * (sP + s21 + s12 + s22),
                             0.25 * r * (-sP + s21 - s12 + s22),
                             0.25 * r * (sP - s21 - s12 + s22),
                             0.25 * r * (-sP - s21 + s12 + s22)};
        const double uu = ux2 + uy2, Et = 0.5 * (b * RT + uu), A = Et + RT, B = Et + 2 * RT, C = RT * A;
        for (int q = 0; q < 9; ++q) {
            const int ix = ex[q] == 0 ? 0 : (ex[q] > 0 ? 1 : 2), iy = ey[q] == 0 ? 0 : (ey[q] > 0 ? 1 : 2);
            const double fv = r * px[ix] * py[iy] - 0.5 * S[q];
            double hv = 0.0;
            if (thermal) {
                if (q == 0)
                    hv = r * (Et - B * uu - 2 * C);
                else if (q <= 4)
                    hv = 0.5 * r * (A * (ex[q] * vx + ey[q] * vy) + B * (ex[q] * ex[q] * ux2 + ey[q] * ey[q] * uy2) + C);
                else
                    hv = 0.25 * r * B * ex[q] * ey[q] * vx * vy;
                if (p.work)  // h_bar = h^eq - q / 2, q_a = W_a F.u
                    hv -= 0.5 * (q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0)) * (Fx * vx + Fy * vy);
            }
            int xs = x - ex[q], ys = y - ey[q];
            if (p.xper) xs = wrapi(xs, p.nx); else if (xs < 0 || xs >= p.nx) continue;
            if (p.yper) ys = wrapi(ys, p.ny); else if (ys < 0 || ys >= p.ny) continue;
            const long long o = (long long)ys * p.pitch + xs;
            Store<ST>::st(dst + q * p.plane + o, (float)(fv - (double)p.fbase[q]));
            if (thermal) Store<ST>::st(dst + (9 + q) * p.plane + o, (float)(hv - (double)p.hbase[q]));
        }
    }
}

// Arbitrary populations (double [9][ny][nx] each) written in the pull layout.
template <class ST>
__global__ void set_pops_kernel(const DevParams p, const double* __restrict__ f, const double* __restrict__ h,
                                ST* __restrict__ dst, int thermal) {
    const long long n = (long long)p.nx * p.ny;
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % p.nx), y = (int)(i / p.nx);
        for (int q = 0; q < 9; ++q) {
            int xs = x - ex[q], ys = y - ey[q];
            if (p.xper) xs = wrapi(xs, p.nx); else if (xs < 0 || xs >= p.nx) continue;
            if (p.yper) ys = wrapi(ys, p.ny); else if (ys < 0 || ys >= p.ny) continue;
            const long long o = (long long)ys * p.pitch + xs;
            Store<ST>::st(dst + q * p.plane + o, (float)(f[q * n + i] - (double)p.fbase[q]));
            if (thermal) Store<ST>::st(dst + (9 + q) * p.plane + o, (float)(h[q * n + i] - (double)p.hbase[q]));
        }
    }
}

// Observable state: streamed populations with wall schemes applied (double [9][ny][nx]).
template <bool THERMAL, class ST>
__global__ void get_pops_kernel(const DevParams p, const ST* __restrict__ src, double* __restrict__ f,
                                double* __restrict__ h) {
    const long long n = (long long)p.nx * p.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % p.nx), y = (int)(i / p.nx);
        float fv[9], hv[9];
        load_node<THERMAL, ST>(p, src, x, y, fv, hv);
        for (int q = 0; q < 9; ++q) {
            f[q * n + i] = (double)p.fbase[q] + fv[q];
            if (THERMAL && h) h[q * n + i] = (double)p.hbase[q] + hv[q];
        }
    }
}

// Eq. 20 and the temperature of Section IV in FP64 from the observable state.
template <bool THERMAL, class ST>
__device__ __forceinline__ void node_fields(const DevParams& p, const ST* __restrict__ src, int x, int y, double& rho,
                                            double& vx, double& vy, double& T, double& sh) {
    float fv[9], hv[9];
    load_node<THERMAL, ST>(p, src, x, y, fv, hv);
    double r = 0, jx = 0, jy = 0;
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int q = 0; q < 9; ++q) {
        const double fq = (double)p.fbase[q] + fv[q];
        r += fq;
        jx += fq * ex[q];
        jy += fq * ey[q];
    }
    double Fx = 0, Fy = 0;
    if (p.force_kind == FORCE_ACCEL) {
        Fx = r * (double)p.ax;
        Fy = r * (double)p.ay;
    } else if (p.force_kind == FORCE_TAYLOR_GREEN) {
        Fx = (double)p.famp * p.sx[x] * p.sy[y];
        Fy = (double)p.famp * p.cx[x] * p.cy[y];
    }
    rho = r;
    vx = (jx + 0.5 * Fx) / r;
    vy = (jy + 0.5 * Fy) / r;
    sh = 0;
    if (THERMAL) {
        for (int q = 0; q < 9; ++q) sh += (double)p.hbase[q] + hv[q];
        const double she = p.work ? sh + 0.5 * (Fx * vx + Fy * vy) : sh;  // rho E with the work term
        T = p.inv_bR2 * (she / r - 0.5 * (vx * vx + vy * vy));
    } else {
        T = p.T0d;
    }
}

template <bool THERMAL, class ST>
__global__ void moments_kernel(const DevParams p, const ST* __restrict__ src, double* __restrict__ rho,
                               double* __restrict__ ux, double* __restrict__ uy, double* __restrict__ T) {
    const long long n = (long long)p.nx * p.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % p.nx), y = (int)(i / p.nx);
        double r, vx, vy, t, sh;
        node_fields<THERMAL, ST>(p, src, x, y, r, vx, vy, t, sh);
        rho[i] = r;
        ux[i] = vx;
        uy[i] = vy;
        T[i] = t;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// FP64 sums (see tclbm_diagnostics) -> one partial per block, summed by diag_finish.
template <bool THERMAL, class ST>
__global__ void __launch_bounds__(kDiagBlock) diag_kernel(const DevParams p, const ST* __restrict__ src,
                                                          const float* __restrict__ usnap, double T_ref,
                                                          double* __restrict__ partial) {
    __shared__ double red[kDiagBlock / 32][TCLBM_NDIAG];
    double acc[TCLBM_NDIAG] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long n = (long long)p.nx * p.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % p.nx), y = (int)(i / p.nx);
        double r, vx, vy, t, sh;
        node_fields<THERMAL, ST>(p, src, x, y, r, vx, vy, t, sh);
        acc[0] += r;
        acc[1] += r * vx;
        acc[2] += r * vy;
        acc[3] += sh;
        acc[4] += 0.5 * r * (vx * vx + vy * vy);
        acc[5] += vy * (t - T_ref);
        if (usnap) {
            const double dx = vx - usnap[2 * i], dy = vy - usnap[2 * i + 1];
            acc[6] += dx * dx + dy * dy;
        }
        acc[7] += vx * vx + vy * vy;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < TCLBM_NDIAG; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) red[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < TCLBM_NDIAG) {
        double s = 0;
        for (int w = 0; w < kDiagBlock / 32; ++w) s += red[w][threadIdx.x];
        partial[blockIdx.x * TCLBM_NDIAG + threadIdx.x] = s;
    }
}

__global__ void diag_finish(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k < TCLBM_NDIAG) {
        double s = 0;
        for (int b = 0; b < nblocks; ++b) s += partial[b * TCLBM_NDIAG + k];
        out[k] = s;
    }
}

template <bool THERMAL, class ST>
__global__ void snapshot_kernel(const DevParams p, const ST* __restrict__ src, float* __restrict__ usnap) {
    const long long n = (long long)p.nx * p.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % p.nx), y = (int)(i / p.nx);
        double r, vx, vy, t, sh;
        node_fields<THERMAL, ST>(p, src, x, y, r, vx, vy, t, sh);
        usnap[2 * i] = (float)vx;
        usnap[2 * i + 1] = (float)vy;
    }
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

// ---------------------------------------------------------------- storage dispatch

template <class F>
tclbm_status with_storage(int storage, F&& fn) {
    switch (storage) {
        case TCLBM_STORE_FP32: return fn((float*)nullptr);
        case TCLBM_STORE_BF16: return fn((__nv_bfloat16*)nullptr);
        default: return fn((__half*)nullptr);
    }
}

tclbm_status ensure_maps(tclbm_lattice* L);

StepLaunch step_launch(tclbm_lattice* L, int src) {
    StepLaunch k;
    k.thermal = L->prm.thermal;
    k.correction = L->prm.correction;
    k.tx = L->tx;
    k.ty = L->ty;
    k.kernel = L->kernel;
    k.src_map = &L->maps[src];
    k.err = L->err;
    k.parity = src;
    return k;
}

tclbm_status launch_steps(tclbm_lattice* L, int64_t n) {
    if (n > 0 && L->kernel == KERNEL_TMA) {
        tclbm_status st = ensure_maps(L);
        if (st != TCLBM_OK) return st;
    }
    // TMA launches with the correction term publish per-item completion tickets; after the
    // first launch of this run the next one waits for each item's neighbours only (16-bit
    // stochastic rounding keeps whole-grid waits: its step counter is written by one CTA)
    const int tx = L->tx, nx = L->prm.nx;
    const bool tickets = L->kernel == KERNEL_TMA && L->prm.thermal && L->prm.correction;
    const bool chainable = tickets && !L->dp.rounding && L->ty >= 8 && (nx % tx == 0 || nx % tx >= 8);
    for (int64_t s = 0; s < n; ++s) {
        StepLaunch k = step_launch(L, L->cur);
        if (tickets) {
            k.seg_done = L->seg_done;
            k.seg_cap = (long long)(L->seg_bytes / sizeof(unsigned));
            k.ticket = ++L->ticket;
            k.chain = chainable && s > 0;
        }
        const cudaError_t e = launch_step_kernel(L->prm.storage, k, L->dp, L->buf[L->cur], L->buf[L->cur ^ 1], L->stream);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
        L->cur ^= 1;
        ++L->steps;
    }
    return TCLBM_OK;
}

tclbm_status build_graph(tclbm_lattice* L) {
    if (L->graph && L->graph_tx == L->tx && L->graph_ty == L->ty && L->graph_kernel == L->kernel) return TCLBM_OK;
    if (L->kernel == KERNEL_TMA) {
        tclbm_status st = ensure_maps(L);
        if (st != TCLBM_OK) return st;
    }
    if (L->graph) {
        cudaGraphExecDestroy(L->graph);
        L->graph = nullptr;
    }
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int s = 0; s < 2 * kGraphPairs && e == cudaSuccess; ++s)
            e = launch_step_kernel(L->prm.storage, step_launch(L, s & 1), L->dp, L->buf[s & 1], L->buf[(s & 1) ^ 1],
                                   cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&L->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        L->graph = nullptr;
        return cuda_fail(e, "step graph capture");
    }
    L->graph_tx = L->tx;
    L->graph_ty = L->ty;
    L->graph_kernel = L->kernel;
    return TCLBM_OK;
}

}  // namespace

// TMA descriptors of both copies of L for strips of tx columns: 3-D (x, y, plane), box
// (tx + 2M, 1, planes).
tclbm_status tclbm::encode_row_maps(const tclbm_lattice* L, int tx, CUtensorMap out[2]) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(TCLBM_ECUDA, "cuTensorMapEncodeTiled is not available");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const CUtensorMapDataType dt = L->prm.storage == TCLBM_STORE_FP32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : L->prm.storage == TCLBM_STORE_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)L->dp.pitch, (cuuint64_t)L->prm.ny, (cuuint64_t)L->nplanes};
    const cuuint64_t strides[2] = {(cuuint64_t)L->dp.pitch * L->elem, (cuuint64_t)L->dp.plane * L->elem};
    const cuuint32_t box[3] = {(cuuint32_t)tma_box_width(L->prm.storage, tx), 1u, (cuuint32_t)L->nplanes};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    for (int b = 0; b < 2; ++b) {
        const CUresult r = encode(&out[b], dt, 3, L->buf[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(TCLBM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    return TCLBM_OK;
}

namespace {

tclbm_status ensure_maps(tclbm_lattice* L) {
    if (L->maps_tx == L->tx) return TCLBM_OK;
    tclbm_status st = encode_row_maps(L, L->tx, L->maps);
    if (st != TCLBM_OK) return st;
    L->maps_tx = L->tx;
    return TCLBM_OK;
}

// Error word of the step kernels (a bounded wait expired): ETIMEOUT once, then cleared.
tclbm_status check_kernel_error(tclbm_lattice* L) {
    int v = 0;
    CK(cudaMemcpyAsync(&v, L->err, sizeof v, cudaMemcpyDeviceToHost, L->stream));
    CK(cudaStreamSynchronize(L->stream));
    if (v) {
        CK(cudaMemsetAsync(L->err, 0, sizeof(int), L->stream));
        return fail(TCLBM_ETIMEOUT, "a step kernel's pipeline wait expired (%d)", v);
    }
    return TCLBM_OK;
}

}  // namespace

// Entries of the completion-ticket array of the TMA kernel's work items: strips of at
// least 32 columns times segments of at least 4 rows (half-height segments of 8-row plans).
static size_t seg_entries(int nx, int ny) { return (size_t)((nx + 31) / 32) * (size_t)(ny / 4 + 2); }

// ==================================================================== C ABI

extern "C" {

const char* tclbm_last_error(void) { return g_err; }

size_t tclbm_state_bytes(const tclbm_params* p) {
    if (!p || p->nx < 1 || p->ny < 1) return 0;
    const size_t n = (size_t)p->nx * p->ny;
    const size_t planes = p->thermal ? 18 : 9;
    const size_t pops = 2 * planes * (size_t)p->ny * pitch_of(p->nx) * elem_of(p->storage);
    const size_t tables = sizeof(float) * 2 * ((size_t)p->nx + p->ny);
    const size_t diag = sizeof(double) * (kDiagMaxBlocks + 1) * TCLBM_NDIAG;
    return pops + tables + diag + n * 4 * sizeof(double) + seg_entries(p->nx, p->ny) * sizeof(unsigned);
}

tclbm_status tclbm_create(const tclbm_params* params, tclbm_alloc_fn alloc, tclbm_free_fn free_fn, void* ctx,
                          void* stream, tclbm_lattice** out) {
    if (!out) return fail(TCLBM_EINVAL, "out is NULL");
    *out = nullptr;
    tclbm_status st = validate(params);
    if (st != TCLBM_OK) return st;
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(TCLBM_EINVAL, "alloc and free must be given together");
    tclbm_lattice* L = new (std::nothrow) tclbm_lattice;
    if (!L) return fail(TCLBM_ENOMEM, "host allocation failed");
    L->prm = *params;
    L->alloc = alloc;
    L->free_fn = free_fn;
    L->ctx = ctx;
    L->stream = (cudaStream_t)stream;
    L->storage = params->storage;
    L->elem = elem_of(params->storage);
    L->nplanes = params->thermal ? 18 : 9;
    derive(L);
    default_launch(L->prm, L->tx, L->ty, L->kernel);
    const size_t n = (size_t)params->nx * params->ny;
    L->buf_bytes = (size_t)L->nplanes * L->dp.plane * L->elem;
    L->tables_bytes = sizeof(float) * 2 * ((size_t)params->nx + params->ny);
    L->diag_bytes = sizeof(double) * (kDiagMaxBlocks + 1) * TCLBM_NDIAG;
    L->stage_bytes = n * 4 * sizeof(double);
    L->buf[0] = dev_alloc(L, L->buf_bytes);
    L->buf[1] = dev_alloc(L, L->buf_bytes);
    L->tables = (float*)dev_alloc(L, L->tables_bytes);
    L->diag = (double*)dev_alloc(L, L->diag_bytes);
    L->stage = (double*)dev_alloc(L, L->stage_bytes);
    L->err = (int*)dev_alloc(L, 256);
    L->seg_bytes = seg_entries(params->nx, params->ny) * sizeof(unsigned);
    L->seg_done = (unsigned*)dev_alloc(L, L->seg_bytes);
    if (!L->buf[0] || !L->buf[1] || !L->tables || !L->diag || !L->stage || !L->err || !L->seg_done) {
        tclbm_destroy(L);
        return fail(TCLBM_ENOMEM, "device allocation of %zu bytes failed", tclbm_state_bytes(params));
    }
    // Taylor-Green force tables: sin/cos of 2 pi x / nx and 2 pi y / ny
    {
        const int nx = params->nx, ny = params->ny;
        float* h = new (std::nothrow) float[2 * ((size_t)nx + ny)];
        if (!h) {
            tclbm_destroy(L);
            return fail(TCLBM_ENOMEM, "host allocation failed");
        }
        for (int i = 0; i < nx; ++i) {
            h[i] = (float)std::sin(2.0 * M_PI * i / nx);
            h[nx + i] = (float)std::cos(2.0 * M_PI * i / nx);
        }
        for (int j = 0; j < ny; ++j) {
            h[2 * nx + j] = (float)std::sin(2.0 * M_PI * j / ny);
            h[2 * nx + ny + j] = (float)std::cos(2.0 * M_PI * j / ny);
        }
        cudaError_t e = cudaMemcpyAsync(L->tables, h, L->tables_bytes, cudaMemcpyHostToDevice, L->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
        delete[] h;
        if (e != cudaSuccess) {
            tclbm_destroy(L);
            return cuda_fail(e, "table upload");
        }
        L->dp.sx = L->tables;
        L->dp.cx = L->tables + nx;
        L->dp.sy = L->tables + 2 * nx;
        L->dp.cy = L->tables + 2 * nx + ny;
    }
    cudaError_t e = cudaMemsetAsync(L->buf[0], 0, L->buf_bytes, L->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->err, 0, 256, L->stream);
    L->dp.step_ctr = reinterpret_cast<unsigned*>(L->err) + 4;  // two counters after the error word
    if (e == cudaSuccess) e = cudaMemsetAsync(L->buf[1], 0, L->buf_bytes, L->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->seg_done, 0, L->seg_bytes, L->stream);  // tickets start at 1
    if (e != cudaSuccess) {
        tclbm_destroy(L);
        return cuda_fail(e, "state clear");
    }
    {
        // dynamic shared-memory limits of the TMA kernels, set before any launch or capture
        const cudaError_t pe = params->storage == TCLBM_STORE_FP32   ? prepare_step_fp32()
                               : params->storage == TCLBM_STORE_BF16 ? prepare_step_bf16()
                                                                     : prepare_step_fp16();
        if (pe != cudaSuccess) {
            tclbm_destroy(L);
            return cuda_fail(pe, "step kernel attributes");
        }
    }
    snprintf(L->desc, sizeof L->desc, "unset");
    *out = L;
    return TCLBM_OK;
}

tclbm_status tclbm_destroy(tclbm_lattice* L) {
    if (!L) return TCLBM_OK;
    if (L->graph) cudaGraphExecDestroy(L->graph);
    cudaStreamSynchronize(L->stream);  // work queued on the handle may still use its memory
    dev_free(L, L->buf[0], L->buf_bytes);
    dev_free(L, L->buf[1], L->buf_bytes);
    dev_free(L, L->tables, L->tables_bytes);
    dev_free(L, L->diag, L->diag_bytes);
    dev_free(L, L->usnap, L->usnap_bytes);
    dev_free(L, L->stage, L->stage_bytes);
    dev_free(L, L->err, 256);
    dev_free(L, L->seg_done, L->seg_bytes);
    if (L->copy_event) cudaEventDestroy(L->copy_event);
    delete L;
    return TCLBM_OK;
}

tclbm_status tclbm_set_stream(tclbm_lattice* L, void* stream) {
    if (!L) return fail(TCLBM_EINVAL, "lattice is NULL");
    L->stream = (cudaStream_t)stream;
    return TCLBM_OK;
}

int64_t tclbm_steps_done(const tclbm_lattice* L) { return L ? L->steps : -1; }

tclbm_status tclbm_set_tile(tclbm_lattice* L, int32_t tx, int32_t ty) {
    if (!L) return fail(TCLBM_EINVAL, "lattice is NULL");
    int dtx, dty;
    default_tile(L->prm, L->kernel, dtx, dty);
    const int ntx = tx ? tx : dtx, nty = ty ? ty : dty;
    if (L->kernel == KERNEL_TILE) {
        if (!tile_fits(L->prm, ntx, nty))
            return fail(TCLBM_EINVAL, "tile shape %dx%d is not available for this lattice", ntx, nty);
    } else {
        if (tx != 0 && tx != 32 && tx != 64 && tx != 128) return fail(TCLBM_EINVAL, "tx must be 0, 32, 64 or 128");
        if (ty < 0) return fail(TCLBM_EINVAL, "ty must be 0 or >= 1");
    }
    L->tx = ntx;
    L->ty = nty;
    return TCLBM_OK;
}

tclbm_status tclbm_test_skip_row(tclbm_lattice* L, int32_t row) {
    if (!L) return fail(TCLBM_EINVAL, "lattice is NULL");
    if (row < -1 || row >= L->prm.ny) return fail(TCLBM_EINVAL, "row must be -1 or in [0, ny)");
    L->dp.skip_row = row;
    if (L->graph) {  // a captured graph holds the old parameters
        cudaGraphExecDestroy(L->graph);
        L->graph = nullptr;
    }
    return TCLBM_OK;
}

namespace {
// The reciprocal the collision takes of R T, mu/p + 1/2 and the thermal rate's argument.
__global__ void rcp_kernel(const float* __restrict__ x, float* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = tclbm::rcp(x[i]);
}
}  // namespace

tclbm_status tclbm_test_rcp(const float* x, float* y, int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return fail(TCLBM_EINVAL, "x, y must be device arrays of n >= 0 floats");
    if (n == 0) return TCLBM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    rcp_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, y, n);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return TCLBM_OK;
}

tclbm_status tclbm_set_kernel(tclbm_lattice* L, int32_t kind) {
    if (!L) return fail(TCLBM_EINVAL, "lattice is NULL");
    if (kind != KERNEL_TMA && kind != KERNEL_DIRECT && kind != KERNEL_TILE)
        return fail(TCLBM_EINVAL, "kernel kind must be 0, 1 or 2");
    if (kind == KERNEL_TILE && !tile_fits(L->prm, kTileBX, kTileBY))
        return fail(TCLBM_EUNSUPPORTED,
                    "2-D tiles need the correction term, nx %% %d != 1 on a walled x axis and ny %% %d != 1 on a "
                    "walled y axis",
                    kTileBX, kTileBY);
    if (kind != L->kernel) default_shape(L->prm, kind, L->tx, L->ty);
    L->kernel = kind;
    return TCLBM_OK;
}

const char* tclbm_describe(const tclbm_lattice* L) {
    if (!L) return "";
    tclbm_lattice* M = const_cast<tclbm_lattice*>(L);
    describe_step_kernel(L->prm.storage, step_launch(M, 0), L->dp, M->desc, sizeof M->desc);
    return L->desc;
}

tclbm_status tclbm_init_fields(tclbm_lattice* L, const double* rho, const double* ux, const double* uy,
                               const double* T, int32_t on_device) {
    if (!L || !rho || !ux || !uy || (!T && L->prm.thermal)) return fail(TCLBM_EINVAL, "NULL argument");
    const size_t n = (size_t)L->prm.nx * L->prm.ny;
    const double* d[4] = {rho, ux, uy, T ? T : rho};
    if (!on_device) {
        for (int k = 0; k < 4; ++k) {
            if (k == 3 && !T) break;
            CK(cudaMemcpyAsync(L->stage + k * n, d[k], n * sizeof(double), cudaMemcpyHostToDevice, L->stream));
        }
        d[0] = L->stage;
        d[1] = L->stage + n;
        d[2] = L->stage + 2 * n;
        d[3] = T ? L->stage + 3 * n : L->stage;
    }
    const tclbm_params& p = L->prm;
    const double b = 2.0 / (p.gamma - 1.0);
    tclbm_status st = with_storage(p.storage, [&](auto* tag) -> tclbm_status {
        using ST = std::remove_pointer_t<decltype(tag)>;
        init_kernel<ST><<<grid_for((long long)n, 256), 256, 0, L->stream>>>(
            L->dp, d[0], d[1], d[2], d[3], (ST*)L->buf[0], p.thermal, p.R, p.T0, b, p.force_kind, p.ax, p.ay, p.famp);
        return TCLBM_OK;
    });
    if (st != TCLBM_OK) return st;
    CK(cudaGetLastError());
    L->cur = 0;
    L->steps = 0;
    if (!on_device) CK(cudaStreamSynchronize(L->stream));  // host arrays may be freed on return
    return TCLBM_OK;
}

tclbm_status tclbm_step(tclbm_lattice* L, int64_t nsteps) {
    if (!L) return fail(TCLBM_EINVAL, "lattice is NULL");
    if (nsteps < 0) return fail(TCLBM_EINVAL, "nsteps must be >= 0");
    int64_t left = nsteps;
    // long runs of short launches go through a captured graph of 2*kGraphPairs steps
    const long long nodes = (long long)L->prm.nx * L->prm.ny;
    if (left >= 2 * kGraphPairs && nodes <= (1LL << 22)) {
        if (L->cur != 0) {
            tclbm_status st = launch_steps(L, 1);
            if (st != TCLBM_OK) return st;
            --left;
        }
        tclbm_status st = build_graph(L);
        if (st != TCLBM_OK) return st;
        while (left >= 2 * kGraphPairs) {
            CK(cudaGraphLaunch(L->graph, L->stream));
            left -= 2 * kGraphPairs;
            L->steps += 2 * kGraphPairs;
        }
    }
    return launch_steps(L, left);
}

tclbm_status tclbm_moments(tclbm_lattice* L, double* rho, double* ux, double* uy, double* T, int32_t on_device) {
    if (!L) return fail(TCLBM_EINVAL, "lattice is NULL");
    const size_t n = (size_t)L->prm.nx * L->prm.ny;
    double* out[4] = {rho, ux, uy, T};
    double* dst[4];
    for (int k = 0; k < 4; ++k) dst[k] = (on_device && out[k]) ? out[k] : L->stage + k * n;
    tclbm_status st = with_storage(L->prm.storage, [&](auto* tag) -> tclbm_status {
        using ST = std::remove_pointer_t<decltype(tag)>;
        const ST* src = (const ST*)L->buf[L->cur];
        if (L->prm.thermal)
            moments_kernel<true, ST><<<grid_for((long long)n, 256), 256, 0, L->stream>>>(L->dp, src, dst[0], dst[1],
                                                                                         dst[2], dst[3]);
        else
            moments_kernel<false, ST><<<grid_for((long long)n, 256), 256, 0, L->stream>>>(L->dp, src, dst[0], dst[1],
                                                                                          dst[2], dst[3]);
        return TCLBM_OK;
    });
    if (st != TCLBM_OK) return st;
    CK(cudaGetLastError());
    if (!on_device)
        for (int k = 0; k < 4; ++k)
            if (out[k])
                CK(cudaMemcpyAsync(out[k], dst[k], n * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CK(cudaStreamSynchronize(L->stream));
    return check_kernel_error(L);
}

tclbm_status tclbm_snapshot_velocity(tclbm_lattice* L) {
    if (!L) return fail(TCLBM_EINVAL, "lattice is NULL");
    const size_t n = (size_t)L->prm.nx * L->prm.ny;
    if (!L->usnap) {
        L->usnap_bytes = 2 * n * sizeof(float);
        L->usnap = (float*)dev_alloc(L, L->usnap_bytes);
        if (!L->usnap) return fail(TCLBM_ENOMEM, "velocity snapshot allocation failed");
    }
    return with_storage(L->prm.storage, [&](auto* tag) -> tclbm_status {
        using ST = std::remove_pointer_t<decltype(tag)>;
        const ST* src = (const ST*)L->buf[L->cur];
        if (L->prm.thermal)
            snapshot_kernel<true, ST><<<grid_for((long long)n, 256), 256, 0, L->stream>>>(L->dp, src, L->usnap);
        else
            snapshot_kernel<false, ST><<<grid_for((long long)n, 256), 256, 0, L->stream>>>(L->dp, src, L->usnap);
        CK(cudaGetLastError());
        return TCLBM_OK;
    });
}

tclbm_status tclbm_diagnostics(tclbm_lattice* L, double out[TCLBM_NDIAG]) {
    if (!L || !out) return fail(TCLBM_EINVAL, "NULL argument");
    const long long n = (long long)L->prm.nx * L->prm.ny;
    long long nb = (n + kDiagBlock - 1) / kDiagBlock;
    if (nb > kDiagMaxBlocks) nb = kDiagMaxBlocks;
    double* res = L->diag + kDiagMaxBlocks * TCLBM_NDIAG;
    tclbm_status st = with_storage(L->prm.storage, [&](auto* tag) -> tclbm_status {
        using ST = std::remove_pointer_t<decltype(tag)>;
        const ST* src = (const ST*)L->buf[L->cur];
        if (L->prm.thermal)
            diag_kernel<true, ST><<<(int)nb, kDiagBlock, 0, L->stream>>>(L->dp, src, L->usnap, L->prm.T_ref, L->diag);
        else
            diag_kernel<false, ST><<<(int)nb, kDiagBlock, 0, L->stream>>>(L->dp, src, L->usnap, L->prm.T_ref, L->diag);
        diag_finish<<<1, 32, 0, L->stream>>>(L->diag, (int)nb, res);
        return TCLBM_OK;
    });
    if (st != TCLBM_OK) return st;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, res, TCLBM_NDIAG * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CK(cudaStreamSynchronize(L->stream));
    tclbm_status ks = check_kernel_error(L);
    if (ks != TCLBM_OK) return ks;
    for (int k = 0; k < TCLBM_NDIAG; ++k)
        if (!std::isfinite(out[k])) return fail(TCLBM_ENONFINITE, "non-finite diagnostic %d", k);
    return TCLBM_OK;
}

tclbm_status tclbm_get_populations(tclbm_lattice* L, double* f, double* h, int32_t on_device) {
    if (!L || !f) return fail(TCLBM_EINVAL, "NULL argument");
    const size_t n = (size_t)L->prm.nx * L->prm.ny;
    const size_t bytes = 9 * n * sizeof(double);
    double *df = f, *dh = h;
    double* tmp = nullptr;
    if (!on_device) {
        tmp = (double*)dev_alloc(L, 2 * bytes);
        if (!tmp) return fail(TCLBM_ENOMEM, "staging allocation failed");
        df = tmp;
        dh = tmp + 9 * n;
    }
    tclbm_status st = with_storage(L->prm.storage, [&](auto* tag) -> tclbm_status {
        using ST = std::remove_pointer_t<decltype(tag)>;
        const ST* src = (const ST*)L->buf[L->cur];
        if (L->prm.thermal)
            get_pops_kernel<true, ST><<<grid_for((long long)n, 256), 256, 0, L->stream>>>(L->dp, src, df, dh);
        else
            get_pops_kernel<false, ST><<<grid_for((long long)n, 256), 256, 0, L->stream>>>(L->dp, src, df, nullptr);
        return TCLBM_OK;
    });
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !on_device) {
        e = cudaMemcpyAsync(f, df, bytes, cudaMemcpyDeviceToHost, L->stream);
        if (e == cudaSuccess && h && L->prm.thermal) e = cudaMemcpyAsync(h, dh, bytes, cudaMemcpyDeviceToHost, L->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
    if (tmp) dev_free(L, tmp, 2 * bytes);
    if (st != TCLBM_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "get_populations");
    return check_kernel_error(L);
}

tclbm_status tclbm_set_populations(tclbm_lattice* L, const double* f, const double* h, int32_t on_device) {
    if (!L || !f || (L->prm.thermal && !h)) return fail(TCLBM_EINVAL, "NULL argument");
    const size_t n = (size_t)L->prm.nx * L->prm.ny;
    const size_t bytes = 9 * n * sizeof(double);
    const double *df = f, *dh = h;
    double* tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        tmp = (double*)dev_alloc(L, 2 * bytes);
        if (!tmp) return fail(TCLBM_ENOMEM, "staging allocation failed");
        e = cudaMemcpyAsync(tmp, f, bytes, cudaMemcpyHostToDevice, L->stream);
        if (e == cudaSuccess && L->prm.thermal) e = cudaMemcpyAsync(tmp + 9 * n, h, bytes, cudaMemcpyHostToDevice, L->stream);
        df = tmp;
        dh = tmp + 9 * n;
    }
    if (e == cudaSuccess) {
        with_storage(L->prm.storage, [&](auto* tag) -> tclbm_status {
            using ST = std::remove_pointer_t<decltype(tag)>;
            set_pops_kernel<ST><<<grid_for((long long)n, 256), 256, 0, L->stream>>>(L->dp, df, dh, (ST*)L->buf[L->cur],
                                                                                    L->prm.thermal);
            return TCLBM_OK;
        });
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
    if (tmp) dev_free(L, tmp, 2 * bytes);
    if (e != cudaSuccess) return cuda_fail(e, "set_populations");
    return TCLBM_OK;
}

// Slab decomposition along y: whole rows of every population plane, in the storage
// format as stored (post-collision values at their own node, ready for the next pull).
tclbm_status tclbm_copy_rows(tclbm_lattice* dst, int32_t dst_row, tclbm_lattice* src, int32_t src_row,
                             int32_t rows) {
    if (!dst || !src) return fail(TCLBM_EINVAL, "lattice is NULL");
    if (dst->prm.nx != src->prm.nx || dst->storage != src->storage || dst->nplanes != src->nplanes)
        return fail(TCLBM_EINVAL, "lattices differ in nx, storage format or thermal flag");
    if (rows < 0 || src_row < 0 || dst_row < 0 || (int64_t)src_row + rows > src->prm.ny ||
        (int64_t)dst_row + rows > dst->prm.ny)
        return fail(TCLBM_EINVAL, "rows [%d, %d) of %d and [%d, %d) of %d are not all inside the lattices", src_row,
                    src_row + rows, src->prm.ny, dst_row, dst_row + rows, dst->prm.ny);
    if (dst == src && dst_row < src_row + rows && src_row < dst_row + rows)
        return fail(TCLBM_EINVAL, "source and destination rows overlap");
    if (rows == 0) return TCLBM_OK;
    const size_t row_bytes = (size_t)dst->dp.pitch * dst->elem;
    const size_t width = (size_t)rows * row_bytes;
    const size_t dplane = (size_t)dst->dp.plane * dst->elem, splane = (size_t)src->dp.plane * src->elem;
    char* d = (char*)dst->buf[dst->cur] + (size_t)dst_row * row_bytes;
    const char* s = (const char*)src->buf[src->cur] + (size_t)src_row * row_bytes;
    const bool cross = dst->stream != src->stream;
    if (cross) {  // the copy follows work queued on the source's stream
        if (!src->copy_event) CK(cudaEventCreateWithFlags(&src->copy_event, cudaEventDisableTiming));
        if (!dst->copy_event) CK(cudaEventCreateWithFlags(&dst->copy_event, cudaEventDisableTiming));
        CK(cudaEventRecord(src->copy_event, src->stream));
        CK(cudaStreamWaitEvent(dst->stream, src->copy_event, 0));
    }
    if (dplane <= (size_t)INT32_MAX && splane <= (size_t)INT32_MAX) {
        CK(cudaMemcpy2DAsync(d, dplane, s, splane, width, (size_t)dst->nplanes, cudaMemcpyDeviceToDevice,
                             dst->stream));
    } else {
        for (int q = 0; q < dst->nplanes; ++q)
            CK(cudaMemcpyAsync(d + q * dplane, s + q * splane, width, cudaMemcpyDeviceToDevice, dst->stream));
    }
    if (cross) {  // and the source's later steps, which overwrite these rows, follow the copy
        CK(cudaEventRecord(dst->copy_event, dst->stream));
        CK(cudaStreamWaitEvent(src->stream, dst->copy_event, 0));
    }
    return TCLBM_OK;
}

}  // extern "C"
