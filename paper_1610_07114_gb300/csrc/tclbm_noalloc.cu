// tclbm_noalloc.cu -- tclbm_diagnostics_noalloc(): the FP64 global sums of
// tclbm_diagnostics() for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where
// they need the sums: a serving loop whose device memory is planned once up front and
// may not grow while requests are in flight, code running under a fixed memory budget
// or on a stream whose allocator is frozen, and embedders that hand the library raw
// device pointers only.  This entry point takes the populations and an output
// pointer from the caller and keeps its block partial sums in a fixed file-scope
// device array, so it allocates nothing.
//
// The scratch array is shared by every call in the process (one copy per device that
// loads the library, held until exit).  Calls whose kernels overlap on the GPU race on
// it: serialise them (one stream, or events).  Each call writes every partial it later
// reads, so nothing needs clearing between calls.
//
// On the first call on a device, with that device current, the host resolves the
// array's device address with cudaGetSymbolAddress (the array's name in host code is
// a host-side stand-in, not a device address) and caches it per device.  Make that
// first call before any stream capture on the device.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "tclbm.h"
#include "tclbm_launch.h"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxBlocks = 1024;
constexpr int kMaxDevices = 64;
constexpr long long kMaxNodesPerThread = 256;
// Largest lattice this path accepts: bounded work per thread (1024 blocks x 256 threads
// x 256 nodes = 67,108,864 nodes, e.g. 8192 x 8192).
constexpr long long kMaxNodes = (long long)kMaxBlocks * kBlock * kMaxNodesPerThread;

// Block partials [kMaxBlocks][8] followed by the 8 final sums (65,600 bytes).
static __device__ __align__(256) double g_noalloc_scratch[(kMaxBlocks + 1) * TCLBM_NDIAG];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

tclbm_status fail(tclbm_status st, const char* msg) {
    tclbm::set_last_error(msg);
    return st;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Per-node macroscopic values from FP64 populations (Eq. 20 and the temperature of
// Section IV), summed like tclbm_diagnostics(): T = 2 / (b R) (E - u^2/2) and T0 in FP64,
// the body force with the FP32-rounded constants the step kernels advance the state with,
// and the Taylor-Green force with its sines rounded to FP32 like the handle's tables.
__global__ void __launch_bounds__(kBlock) noalloc_sums(const double* __restrict__ f, const double* __restrict__ h,
                                                       const double* __restrict__ usnap, long long n, int nx, int ny,
                                                       int thermal, int force_kind, double ax, double ay, double famp,
                                                       double bR, double T0, double T_ref, int work, double* partial) {
    __shared__ double red[kBlock / 32][TCLBM_NDIAG];
    double acc[TCLBM_NDIAG] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)(i / nx);
        double r = 0, jx = 0, jy = 0, sh = 0;
        for (int q = 0; q < 9; ++q) {
            const double v = f[q * n + i];
            r += v;
            jx += v * ex[q];
            jy += v * ey[q];
            if (thermal) sh += h[q * n + i];
        }
        double Fx = 0, Fy = 0;
        if (force_kind == TCLBM_FORCE_ACCEL) {
            Fx = r * ax;
            Fy = r * ay;
        } else if (force_kind == TCLBM_FORCE_TAYLOR_GREEN) {
            const double ax_ = 6.283185307179586 * x / nx, ay_ = 6.283185307179586 * y / ny;
            Fx = famp * (double)(float)sin(ax_) * (double)(float)sin(ay_);
            Fy = famp * (double)(float)cos(ax_) * (double)(float)cos(ay_);
        }
        const double vx = (jx + 0.5 * Fx) / r, vy = (jy + 0.5 * Fy) / r;
        const double she = work ? sh + 0.5 * (Fx * vx + Fy * vy) : sh;  // rho E with the work term
        const double T = thermal ? 2.0 / bR * (she / r - 0.5 * (vx * vx + vy * vy)) : T0;
        acc[0] += r;
        acc[1] += r * vx;
        acc[2] += r * vy;
        acc[3] += sh;
        acc[4] += 0.5 * r * (vx * vx + vy * vy);
        acc[5] += vy * (T - T_ref);
        if (usnap) {
            const double dx = vx - usnap[i], dy = vy - usnap[n + i];
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
        for (int w = 0; w < kBlock / 32; ++w) s += red[w][threadIdx.x];
        partial[blockIdx.x * TCLBM_NDIAG + threadIdx.x] = s;
    }
}

__global__ void noalloc_finish(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k < TCLBM_NDIAG) {
        double s = 0;
        for (int b = 0; b < nblocks; ++b) s += partial[b * TCLBM_NDIAG + k];
        out[k] = s;
    }
}

// Device address of the scratch array on the current device (resolved once per device).
tclbm_status scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(TCLBM_ECUDA, "cudaGetDevice failed");
    }
    if (dev < 0 || dev >= kMaxDevices) return fail(TCLBM_EUNSUPPORTED, "device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(TCLBM_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed");
        }
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return TCLBM_OK;
}

}  // namespace

extern "C" tclbm_status tclbm_diagnostics_noalloc(const tclbm_params* params, const double* f, const double* h,
                                                  const double* u_snap, double* out, int32_t out_on_device,
                                                  void* stream) {
    if (!params || !f || !out || (params->thermal && !h)) return fail(TCLBM_EINVAL, "NULL argument");
    if (params->nx < 1 || params->ny < 1) return fail(TCLBM_EINVAL, "nx, ny must be >= 1");
    if (!(params->gamma > 1.0) || !(params->R > 0.0)) return fail(TCLBM_EINVAL, "gamma > 1 and R > 0 required");
    const long long n = (long long)params->nx * params->ny;
    if (n > kMaxNodes) {
        char msg[160];
        snprintf(msg, sizeof msg, "lattice of %lld nodes exceeds the %lld-node maximum of tclbm_diagnostics_noalloc",
                 n, kMaxNodes);
        return fail(TCLBM_EINVAL, msg);
    }
    double* scratch = nullptr;
    tclbm_status st = scratch_for_current_device(&scratch);
    if (st != TCLBM_OK) return st;
    long long nb = (n + kBlock - 1) / kBlock;
    if (nb > kMaxBlocks) nb = kMaxBlocks;
    cudaStream_t s = (cudaStream_t)stream;
    const double bR = 2.0 / (params->gamma - 1.0) * params->R;  // the handle's FP64 b R
    double* result = scratch + kMaxBlocks * TCLBM_NDIAG;
    noalloc_sums<<<(int)nb, kBlock, 0, s>>>(f, params->thermal ? h : nullptr, u_snap, n, params->nx, params->ny,
                                           params->thermal, params->force_kind, (double)(float)params->ax,
                                           (double)(float)params->ay, (double)(float)params->famp, bR,
                                           params->T0, params->T_ref, params->thermal && params->work, scratch);
    noalloc_finish<<<1, 32, 0, s>>>(scratch, (int)nb, out_on_device ? out : result);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !out_on_device)
        e = cudaMemcpyAsync(out, result, TCLBM_NDIAG * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && !out_on_device) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        char msg[160];
        snprintf(msg, sizeof msg, "tclbm_diagnostics_noalloc: %s", cudaGetErrorString(e));
        return fail(TCLBM_ECUDA, msg);
    }
    // a NaN or Inf anywhere in the state reaches the sums; report it as tclbm_diagnostics() does
    if (!out_on_device)
        for (int k = 0; k < TCLBM_NDIAG; ++k)
            if (!std::isfinite(out[k])) {
                char msg[96];
                snprintf(msg, sizeof msg, "tclbm_diagnostics_noalloc: non-finite diagnostic %d", k);
                return fail(TCLBM_ENONFINITE, msg);
            }
    return TCLBM_OK;
}
