// tclbm_step_inst.cuh -- instantiates the step kernels for one storage type ST and
// defines its launch function LAUNCH_FN (included by tclbm_step_<format>.cu).
#include <cstdio>

#include "tclbm_launch.h"
#include "tclbm_tma.cuh"

namespace tclbm {

template <class K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// CTAs of tclbm_step_tile<BX, BY> the current device holds resident at once (0 if the
// query fails).
template <int BX, int BY, bool LATE>
static long long tile_wave() {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tclbm_step_tile<BX, BY, ST, LATE>, BX * BY, 0)) {
        cudaGetLastError();
        return 0;
    }
    return (long long)sms * per_sm;
}

template <int BX, int BY>
static cudaError_t launch_tile_shape(const DevParams& p, const ST* in, ST* out, cudaStream_t s) {
    // programmatic dependent launch: the next step's grid is scheduled while this one
    // runs (the kernel waits for its predecessor before touching memory); 32 x 4 tiles
    // wait late on grids of more than one wave
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nx + BX - 1) / BX, (p.ny + BY - 1) / BY, 1);
    cfg.blockDim = dim3(BX * BY, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if constexpr (BX == 32 && BY == 4) {
        static const long long wave = tile_wave<BX, BY, true>();
        if (wave > 0 && (long long)cfg.gridDim.x * cfg.gridDim.y > wave) {
            const cudaError_t e = cudaLaunchKernelEx(&cfg, tclbm_step_tile<BX, BY, ST, true>, p, in, out);
            return e != cudaSuccess ? e : cudaGetLastError();
        }
    }
    const cudaError_t e = cudaLaunchKernelEx(&cfg, tclbm_step_tile<BX, BY, ST, false>, p, in, out);
    return e != cudaSuccess ? e : cudaGetLastError();
}

static cudaError_t launch_tile(int bx, int by, const DevParams& p, const ST* in, ST* out, cudaStream_t s) {
    if (bx == 16 && by == 4) return launch_tile_shape<16, 4>(p, in, out, s);
    if (bx == 16 && by == 8) return launch_tile_shape<16, 8>(p, in, out, s);
    if (bx == 32 && by == 8) return launch_tile_shape<32, 8>(p, in, out, s);
    if (bx == 32 && by == 16) return launch_tile_shape<32, 16>(p, in, out, s);
    if (bx == 64 && by == 4) return launch_tile_shape<64, 4>(p, in, out, s);
    if (bx == 64 && by == 8) return launch_tile_shape<64, 8>(p, in, out, s);
    if (bx == 128 && by == 4) return launch_tile_shape<128, 4>(p, in, out, s);
    return launch_tile_shape<32, 4>(p, in, out, s);
}

// One launch of a TMA-fed step kernel (signature of tclbm_step_tma_corr / _plain) under the
// segment plan for `resident` CTAs, with programmatic dependent launch.
template <class K>
static cudaError_t launch_tma(K kernel, int tx, size_t smem, long long resident, const StepLaunch& k, const DevParams& p,
                              const ST* in, ST* out, cudaStream_t s) {
    const SegPlan plan = tma_seg_plan(p, tx, k.ty, resident);
    // completion tickets only where every item has an entry
    const long long items = (long long)((p.nx + tx - 1) / tx) * (plan.full + plan.half);
    unsigned* seg_done = items <= k.seg_cap ? k.seg_done : nullptr;
    const int chain = seg_done ? k.chain : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((p.nx + tx - 1) / tx), (unsigned)(plan.full + plan.half), 1);
    cfg.blockDim = dim3(tx, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, p, *k.src_map, in, out, k.ty, plan.full, plan.extra, k.err, seg_done,
                              k.ticket, chain);
}

// CTAs of tclbm_step_tma_plain<TX, THERMAL> the current device holds resident at once
// (the kernel's dynamic shared-memory limit is raised first: the query may come before
// PREPARE_FN, and the answer is kept).
template <int TX, bool THERMAL>
static long long plain_resident() {
    static const long long n = [] {
        int per_sm = 0;
        const size_t smem = tma_smem_bytes<TX, THERMAL, ST>(false);
        if (allow_smem(tclbm_step_tma_plain<TX, THERMAL, ST>, smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tclbm_step_tma_plain<TX, THERMAL, ST>, TX, smem) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        return (long long)sm_count() * per_sm;
    }();
    return n;
}

template <int TX>
static cudaError_t launch_tx(const StepLaunch& k, const DevParams& p0, const void* src, void* dst, cudaStream_t s) {
    DevParams p = p0;
    p.parity = k.parity;
    const dim3 grid = step_grid(p, TX, k.ty);
    const ST* in = static_cast<const ST*>(src);
    ST* out = static_cast<ST*>(dst);
    const bool corr = k.thermal && k.correction;
    if (k.kernel == KERNEL_TMA) {
        cudaError_t e;
        if (corr) {
            static const long long resident = (long long)sm_count() * (CorrShape<ST>::kThreadsPerSM / TX);
            e = launch_tma(tclbm_step_tma_corr<TX, ST>, TX, tma_smem_bytes<TX, true, ST>(true), resident, k, p, in, out, s);
        } else if (k.thermal) {
            e = launch_tma(tclbm_step_tma_plain<TX, true, ST>, TX, tma_smem_bytes<TX, true, ST>(false),
                           plain_resident<TX, true>(), k, p, in, out, s);
        } else {
            e = launch_tma(tclbm_step_tma_plain<TX, false, ST>, TX, tma_smem_bytes<TX, false, ST>(false),
                           plain_resident<TX, false>(), k, p, in, out, s);
        }
        if (e != cudaSuccess) return e;
    } else if (k.kernel == KERNEL_TILE && corr) {
        return launch_tile(k.tx, k.ty, p, in, out, s);
    } else {
        if (corr)
            tclbm_step_corr<TX, ST><<<grid, TX, 0, s>>>(p, in, out, k.ty);
        else if (k.thermal)
            tclbm_step_plain<TX, true, ST><<<grid, TX, 0, s>>>(p, in, out, k.ty);
        else
            tclbm_step_plain<TX, false, ST><<<grid, TX, 0, s>>>(p, in, out, k.ty);
    }
    return cudaGetLastError();
}

template <int TX>
static cudaError_t prepare_tx() {
    cudaError_t e = allow_smem(tclbm_step_tma_corr<TX, ST>, tma_smem_bytes<TX, true, ST>(true));
    if (e == cudaSuccess) e = allow_smem(tclbm_step_batch_tma<TX, ST>, tma_smem_bytes<TX, true, ST>(true));
    if (e == cudaSuccess) e = allow_smem(tclbm_step_tma_plain<TX, true, ST>, tma_smem_bytes<TX, true, ST>(false));
    if (e == cudaSuccess) e = allow_smem(tclbm_step_tma_plain<TX, false, ST>, tma_smem_bytes<TX, false, ST>(false));
    return e;
}

// Dynamic shared-memory limits of every TMA kernel of this format (current device).
cudaError_t PREPARE_FN() {
    cudaError_t e = prepare_tx<32>();
    if (e == cudaSuccess) e = prepare_tx<64>();
    if (e == cudaSuccess) e = prepare_tx<128>();
    return e;
}

// Resident CTAs the TMA launcher plans the segments for (see launch_tma).
long long TMA_RESIDENT_FN(int tx, int corr, int thermal) {
    if (corr) return (long long)sm_count() * (CorrShape<ST>::kThreadsPerSM / tx);
    switch (tx) {
        case 32: return thermal ? plain_resident<32, true>() : plain_resident<32, false>();
        case 64: return thermal ? plain_resident<64, true>() : plain_resident<64, false>();
        default: return thermal ? plain_resident<128, true>() : plain_resident<128, false>();
    }
}

cudaError_t LAUNCH_FN(const StepLaunch& k, const DevParams& p, const void* src, void* dst, cudaStream_t s) {
    switch (k.tx) {
        case 32: return launch_tx<32>(k, p, src, dst, s);
        case 64: return launch_tx<64>(k, p, src, dst, s);
        default: return launch_tx<128>(k, p, src, dst, s);
    }
}

template <int TX>
static cudaError_t launch_batch_tx(int kind, unsigned grid, const BatchLattice* lats, const BatchItem* items,
                                   int nitems, int step_parity, cudaStream_t s) {
    switch (kind) {
        case BATCH_THERMAL_CORR:
            tclbm_step_batch<TX, ST, BATCH_THERMAL_CORR><<<grid, TX, 0, s>>>(lats, items, nitems, step_parity);
            break;
        case BATCH_THERMAL:
            tclbm_step_batch<TX, ST, BATCH_THERMAL><<<grid, TX, 0, s>>>(lats, items, nitems, step_parity);
            break;
        default: tclbm_step_batch<TX, ST, BATCH_ATHERMAL><<<grid, TX, 0, s>>>(lats, items, nitems, step_parity);
    }
    return cudaGetLastError();
}

cudaError_t BATCH_FN(int tx, int kind, unsigned grid, const BatchLattice* lats, const BatchItem* items, int nitems,
                     int step_parity, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    switch (tx) {
        case 32: return launch_batch_tx<32>(kind, grid, lats, items, nitems, step_parity, s);
        case 64: return launch_batch_tx<64>(kind, grid, lats, items, nitems, step_parity, s);
        default: return launch_batch_tx<128>(kind, grid, lats, items, nitems, step_parity, s);
    }
}

template <int TX>
static int occupancy_tx(int kind) {
    int n = 0;
    cudaError_t e;
    if (kind == BATCH_THERMAL_CORR)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tclbm_step_batch<TX, ST, BATCH_THERMAL_CORR>, TX, 0);
    else if (kind == BATCH_THERMAL)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tclbm_step_batch<TX, ST, BATCH_THERMAL>, TX, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tclbm_step_batch<TX, ST, BATCH_ATHERMAL>, TX, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

cudaError_t BATCH_TMA_FN(int tx, unsigned grid, const BatchLattice* lats, const BatchItem* items, int nitems,
                         int step_parity, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    if (tx == 64)
        tclbm_step_batch_tma<64, ST><<<grid, 64, tma_smem_bytes<64, true, ST>(true), s>>>(lats, items, nitems,
                                                                                          step_parity);
    else
        tclbm_step_batch_tma<128, ST><<<grid, 128, tma_smem_bytes<128, true, ST>(true), s>>>(lats, items, nitems,
                                                                                             step_parity);
    return cudaGetLastError();
}

int BATCH_OCC_FN(int tx, int kind) {
    switch (tx) {
        case 32: return occupancy_tx<32>(kind);
        case 64: return occupancy_tx<64>(kind);
        default: return occupancy_tx<128>(kind);
    }
}

}  // namespace tclbm
