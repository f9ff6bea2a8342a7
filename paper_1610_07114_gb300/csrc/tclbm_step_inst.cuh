// tclbm_step_inst.cuh -- instantiates the step kernels for one storage type ST and
// defines its launch function LAUNCH_FN (included by tclbm_step_<format>.cu).
#include <cstdio>

#include "tclbm_launch.h"

namespace tclbm {

template <int TX>
static cudaError_t launch_tx(int thermal, int correction, int ty, const DevParams& p, const void* src, void* dst,
                             cudaStream_t s) {
    const dim3 grid = step_grid(p, TX, ty);
    const ST* in = static_cast<const ST*>(src);
    ST* out = static_cast<ST*>(dst);
    if (thermal && correction)
        tclbm_step_corr<TX, ST><<<grid, TX, 0, s>>>(p, in, out, ty);
    else if (thermal)
        tclbm_step_plain<TX, true, ST><<<grid, TX, 0, s>>>(p, in, out, ty);
    else
        tclbm_step_plain<TX, false, ST><<<grid, TX, 0, s>>>(p, in, out, ty);
    return cudaGetLastError();
}

cudaError_t LAUNCH_FN(int thermal, int correction, int tx, int ty, const DevParams& p, const void* src, void* dst,
                      cudaStream_t s) {
    switch (tx) {
        case 32: return launch_tx<32>(thermal, correction, ty, p, src, dst, s);
        case 64: return launch_tx<64>(thermal, correction, ty, p, src, dst, s);
        default: return launch_tx<128>(thermal, correction, ty, p, src, dst, s);
    }
}

}  // namespace tclbm
