// tclbm_launch.h -- launch entry points of the fused step kernel, one translation unit
// per population storage format (compiled in parallel).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <cuda.h>

#include "tclbm_batch.cuh"
#include "tclbm_device.cuh"

namespace tclbm {
// Sets the thread-local message returned by tclbm_last_error().
void set_last_error(const char* msg);

// Kernel variants: the TMA-fed ring (default) and the direct-load marching kernel.
// Kernel variants: the TMA-fed ring, the direct-load marching kernel, and 2-D tiles of
// one node per thread (small lattices with the correction term).
enum { KERNEL_TMA = 0, KERNEL_DIRECT = 1, KERNEL_TILE = 2 };

// Tile shapes of KERNEL_TILE (set through tclbm_set_tile as (BX, BY)), and whether a
// lattice can use one (one-sided wall derivatives need nx % BX != 1 on a walled x axis
// and ny % BY != 1 on a walled y axis).
constexpr int kTileBX = 32, kTileBY = 4;  // default shape (fastest from 256x128 to 2048x1024)
inline bool tile_shape_valid(int bx, int by) {
    return (bx == 16 && (by == 4 || by == 8)) || (bx == 32 && (by == 4 || by == 8 || by == 16)) ||
           (bx == 64 && (by == 4 || by == 8)) || (bx == 128 && by == 4);
}
inline bool tile_kernel_fits(int nx, int ny, bool xper, bool yper, bool thermal, bool correction, int bx = kTileBX,
                             int by = kTileBY) {
    return thermal && correction && tile_shape_valid(bx, by) && (xper || nx % bx != 1) && (yper || ny % by != 1);
}
struct StepLaunch {
    int thermal, correction, tx, ty, kernel;
    const CUtensorMap* src_map;  // tensor map of the source copy (KERNEL_TMA)
    int* err;                    // device error word (bounded waits that expired)
    int parity;                  // index of the source copy (selects the step counter)
    // chained TMA launches (tclbm_step_tma_corr): per-item completion tickets (nullptr:
    // none), their capacity, this launch's ticket, and whether to wait for the previous
    // launch's neighbouring items instead of its whole grid
    unsigned* seg_done = nullptr;
    long long seg_cap = 0;
    unsigned ticket = 0;
    int chain = 0;
};

cudaError_t launch_step_fp32(const StepLaunch& k, const DevParams& p, const void* src, void* dst, cudaStream_t s);
cudaError_t launch_step_bf16(const StepLaunch& k, const DevParams& p, const void* src, void* dst, cudaStream_t s);
cudaError_t launch_step_fp16(const StepLaunch& k, const DevParams& p, const void* src, void* dst, cudaStream_t s);
// Batched step of the items of one collision variant (BATCH_*).
cudaError_t launch_batch_fp32(int tx, int kind, unsigned grid, const BatchLattice* lats, const BatchItem* items,
                              int nitems, int step_parity, cudaStream_t s);
cudaError_t launch_batch_bf16(int tx, int kind, unsigned grid, const BatchLattice* lats, const BatchItem* items,
                              int nitems, int step_parity, cudaStream_t s);
cudaError_t launch_batch_fp16(int tx, int kind, unsigned grid, const BatchLattice* lats, const BatchItem* items,
                              int nitems, int step_parity, cudaStream_t s);
// TMA-fed batched step of thermal lattices with the correction term (tx 64 or 128; one
// CTA per item).
cudaError_t launch_batch_tma_fp32(int tx, unsigned grid, const BatchLattice* lats, const BatchItem* items, int nitems,
                                  int step_parity, cudaStream_t s);
cudaError_t launch_batch_tma_bf16(int tx, unsigned grid, const BatchLattice* lats, const BatchItem* items, int nitems,
                                  int step_parity, cudaStream_t s);
cudaError_t launch_batch_tma_fp16(int tx, unsigned grid, const BatchLattice* lats, const BatchItem* items, int nitems,
                                  int step_parity, cudaStream_t s);
inline cudaError_t launch_batch_tma_kernel(int storage, int tx, unsigned grid, const BatchLattice* lats,
                                           const BatchItem* items, int nitems, int step_parity, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_batch_tma_fp32(tx, grid, lats, items, nitems, step_parity, s);
        case 1: return launch_batch_tma_bf16(tx, grid, lats, items, nitems, step_parity, s);
        default: return launch_batch_tma_fp16(tx, grid, lats, items, nitems, step_parity, s);
    }
}
// Resident CTAs per SM of the batched kernel for a tile width and variant (occupancy calculator).
int batch_occupancy_fp32(int tx, int kind);
int batch_occupancy_bf16(int tx, int kind);
int batch_occupancy_fp16(int tx, int kind);
inline int batch_ctas_per_sm(int storage, int tx, int kind) {
    return storage == 0 ? batch_occupancy_fp32(tx, kind)
                        : storage == 1 ? batch_occupancy_bf16(tx, kind) : batch_occupancy_fp16(tx, kind);
}
cudaError_t prepare_step_fp32();
cudaError_t prepare_step_bf16();
cudaError_t prepare_step_fp16();

inline cudaError_t launch_step_kernel(int storage, const StepLaunch& k, const DevParams& p, const void* src,
                                      void* dst, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_step_fp32(k, p, src, dst, s);
        case 1: return launch_step_bf16(k, p, src, dst, s);
        default: return launch_step_fp16(k, p, src, dst, s);
    }
}

inline cudaError_t launch_batch_kernel(int storage, int tx, int kind, unsigned grid, const BatchLattice* lats,
                                       const BatchItem* items, int nitems, int step_parity, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_batch_fp32(tx, kind, grid, lats, items, nitems, step_parity, s);
        case 1: return launch_batch_bf16(tx, kind, grid, lats, items, nitems, step_parity, s);
        default: return launch_batch_fp16(tx, kind, grid, lats, items, nitems, step_parity, s);
    }
}

// Box width (elements) of the TMA row copy for a strip of tx columns.
inline int tma_box_width(int storage, int tx) { return tx + 2 * (storage == 0 ? 4 : 8); }

// Multiprocessors of the current device (152 if the query fails).
inline int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n < 1) {
        cudaGetLastError();
        return 152;
    }
    return n;
}

// Row segments of the TMA kernel with the correction term: `full` segments of ty rows
// (the first one `extra` rows taller), then `half` segments of ty / 2 rows.  The block
// scheduler dispatches blocks in index order, so the short segments run last: about
// one wave of them makes the launch's tail out of half-length CTAs.  Used where the
// grid spans more than two waves of `resident` CTAs, ty is a multiple of 16 and ny a
// multiple of 8 (segment starts stay on multiples of 8 rows); otherwise the plan is
// uniform (full = ny / ty, the last segment taking the remainder, half = extra = 0).
struct SegPlan {
    int full, half, extra;
};
inline SegPlan tma_seg_plan(const DevParams& p, int tx, int ty, long long resident) {
    const int strips = (p.nx + tx - 1) / tx;
    int nseg = p.ny / ty;
    if (nseg < 1) nseg = 1;
    SegPlan s{nseg, 0, 0};
    if (ty % 16 != 0 || p.ny % 8 != 0 || (long long)nseg * strips <= 2 * resident) return s;
    const int half = (int)((resident + strips - 1) / strips);
    const int full = (p.ny - half * (ty / 2)) / ty;
    if (full < 2) return s;
    s.full = full;
    s.half = half;
    s.extra = p.ny - full * ty - half * (ty / 2);
    return s;
}

// CTAs per SM the TMA kernels with the correction term are sized for (threads per SM of
// CorrShape in tclbm_tma.cuh: 384 for FP32 rows, 512 for 16-bit rows), for strips of tx.
inline int tma_corr_ctas_per_sm(int storage, int tx) { return (storage == 0 ? 384 : 512) / tx; }

// Resident CTAs the TMA launcher of each format plans its segments for.
long long tma_resident_fp32(int tx, int corr, int thermal);
long long tma_resident_bf16(int tx, int corr, int thermal);
long long tma_resident_fp16(int tx, int corr, int thermal);
inline long long tma_resident(int storage, int tx, int corr, int thermal) {
    return storage == 0 ? tma_resident_fp32(tx, corr, thermal)
                        : storage == 1 ? tma_resident_bf16(tx, corr, thermal) : tma_resident_fp16(tx, corr, thermal);
}

inline dim3 step_grid(const DevParams& p, int tx, int ty) {
    int nseg = p.ny / ty;
    if (nseg < 1) nseg = 1;
    return dim3((unsigned)((p.nx + tx - 1) / tx), (unsigned)nseg, 1);
}

inline void describe_step_kernel(int storage, const StepLaunch& k, const DevParams& p, char* out, size_t len) {
    const char* st = storage == 0 ? "float" : (storage == 1 ? "bf16" : "half");
    const dim3 g = step_grid(p, k.tx, k.ty);
    const bool corr = k.thermal && k.correction;
    if (k.kernel == KERNEL_TILE && corr) {
        snprintf(out, len, "tclbm_step_tile<%d,%d,%s> grid (%d, %d) block (%d)", k.tx, k.ty, st,
                 (p.nx + k.tx - 1) / k.tx, (p.ny + k.ty - 1) / k.ty, k.tx * k.ty);
        return;
    }
    const char* base = k.kernel == KERNEL_TMA ? (corr ? "tclbm_step_tma_corr" : "tclbm_step_tma_plain")
                                              : (corr ? "tclbm_step_corr" : "tclbm_step_plain");
    if (k.kernel == KERNEL_TMA) {
        const SegPlan plan = tma_seg_plan(p, k.tx, k.ty, tma_resident(storage, k.tx, corr, k.thermal));
        if (plan.half > 0) {
            snprintf(out, len, "%s<%d,%s%s> grid (%u, %d) block (%d) rows/cta %d, last %d segments of %d", base, k.tx,
                     corr ? "" : (k.thermal ? "thermal," : "athermal,"), st, g.x, plan.full + plan.half, k.tx, k.ty,
                     plan.half, k.ty / 2);
            return;
        }
    }
    snprintf(out, len, "%s<%d,%s%s> grid (%u, %u) block (%d) rows/cta %d", base, k.tx,
             corr ? "" : (k.thermal ? "thermal," : "athermal,"), st, g.x, g.y, k.tx, k.ty);
}
}  // namespace tclbm
