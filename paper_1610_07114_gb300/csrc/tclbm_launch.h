// tclbm_launch.h -- launch entry points of the fused step kernel, one translation unit
// per population storage format (compiled in parallel).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "tclbm_device.cuh"

namespace tclbm {
// Sets the thread-local message returned by tclbm_last_error().
void set_last_error(const char* msg);

cudaError_t launch_step_fp32(int thermal, int correction, int tx, int ty, const DevParams& p, const void* src,
                             void* dst, cudaStream_t s);
cudaError_t launch_step_bf16(int thermal, int correction, int tx, int ty, const DevParams& p, const void* src,
                             void* dst, cudaStream_t s);
cudaError_t launch_step_fp16(int thermal, int correction, int tx, int ty, const DevParams& p, const void* src,
                             void* dst, cudaStream_t s);

inline cudaError_t launch_step_kernel(int storage, int thermal, int correction, int tx, int ty, const DevParams& p,
                                      const void* src, void* dst, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_step_fp32(thermal, correction, tx, ty, p, src, dst, s);
        case 1: return launch_step_bf16(thermal, correction, tx, ty, p, src, dst, s);
        default: return launch_step_fp16(thermal, correction, tx, ty, p, src, dst, s);
    }
}

inline dim3 step_grid(const DevParams& p, int tx, int ty) {
    int nseg = p.ny / ty;
    if (nseg < 1) nseg = 1;
    return dim3((unsigned)((p.nx + tx - 1) / tx), (unsigned)nseg, 1);
}

inline void describe_step_kernel(int storage, int thermal, int correction, int tx, int ty, const DevParams& p,
                                 char* out, size_t len) {
    const char* st = storage == 0 ? "float" : (storage == 1 ? "bf16" : "half");
    const dim3 g = step_grid(p, tx, ty);
    snprintf(out, len, "%s<%d,%s%s> grid (%u, %u) block (%d) rows/cta %d",
             (thermal && correction) ? "tclbm_step_corr" : "tclbm_step_plain", tx,
             (thermal && correction) ? "" : (thermal ? "thermal," : "athermal,"), st, g.x, g.y, tx, ty);
}
}  // namespace tclbm
