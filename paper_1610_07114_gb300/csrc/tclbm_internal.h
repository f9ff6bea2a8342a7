// tclbm_internal.h -- host-side state of a lattice handle and helpers shared by the
// translation units of the C ABI (not part of the public interface).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "tclbm.h"
#include "tclbm_device.cuh"
#include "tclbm_launch.h"

namespace tclbm {
constexpr int kGraphPairs = 32;  // a captured step graph holds 2 * kGraphPairs launches
}  // namespace tclbm

using tclbm::DevParams;
using tclbm::KERNEL_TMA;

struct tclbm_lattice {
    tclbm_params prm;
    DevParams dp;
    cudaStream_t stream = nullptr;
    tclbm_alloc_fn alloc = nullptr;
    tclbm_free_fn free_fn = nullptr;
    void* ctx = nullptr;
    int storage = TCLBM_STORE_FP32;
    size_t elem = 4;
    int nplanes = 18;
    void* buf[2] = {nullptr, nullptr};
    size_t buf_bytes = 0;
    float* tables = nullptr;
    size_t tables_bytes = 0;
    double* diag = nullptr;  // [kDiagMaxBlocks * TCLBM_NDIAG] partials + TCLBM_NDIAG result
    size_t diag_bytes = 0;
    float* usnap = nullptr;  // 2 * nx * ny
    size_t usnap_bytes = 0;
    double* stage = nullptr;  // 4 * nx * ny doubles (or 18 * nx * ny for populations)
    size_t stage_bytes = 0;
    int cur = 0;
    int64_t steps = 0;
    int tx = 0, ty = 0;
    int kernel = KERNEL_TMA;
    CUtensorMap maps[2];  // TMA descriptors of the two copies for box width of tx
    int maps_tx = 0;
    int* err = nullptr;  // device error word of the step kernels
    // completion tickets of the TMA kernel's work items (chained launches) and the
    // ticket of the last launch that published them
    unsigned* seg_done = nullptr;
    size_t seg_bytes = 0;
    unsigned ticket = 0;
    char desc[256] = "";
    // CUDA graph of 2 * kGraphPairs step launches (parity preserved)
    cudaGraphExec_t graph = nullptr;
    int graph_tx = 0, graph_ty = 0, graph_kernel = -1;
    // orders row copies between lattices on different streams (created on first use)
    cudaEvent_t copy_event = nullptr;
};

namespace tclbm {
// Records a printf-style message for tclbm_last_error() and returns `st`.
tclbm_status fail(tclbm_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
tclbm_status cuda_fail(cudaError_t e, const char* what);
// TMA row descriptors of both copies of L for strips of tx columns (box tx + 2M wide).
tclbm_status encode_row_maps(const tclbm_lattice* L, int tx, CUtensorMap out[2]);
// Device memory through the handle's allocator hooks (cudaMalloc / cudaFree without them).
void* dev_alloc(tclbm_lattice* L, size_t bytes);
void dev_free(tclbm_lattice* L, void* p, size_t bytes);
}  // namespace tclbm

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return tclbm::cuda_fail(e_, #call); \
    } while (0)
