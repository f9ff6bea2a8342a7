// tclbm_batch.cuh -- the batched step kernel: many independent lattices advance one
// time step in one launch, each work item a strip of one lattice updated by the same
// strip code as the single-lattice direct kernel.
#pragma once
#include <cuda.h>
#include <stddef.h>

#include "tclbm_device.cuh"

namespace tclbm {

// Collision variants a lattice of a batch can use.
enum { BATCH_ATHERMAL = 0, BATCH_THERMAL = 1, BATCH_THERMAL_CORR = 2 };

// One lattice of a batch: its constants (p.parity = index of its source copy at the
// batch's step 0), its two population copies, its collision variant, and for the
// TMA-fed batch kernel the row tensor maps of both copies and its error word.
struct BatchLattice {
    CUtensorMap map[2];  // 64-byte aligned: the first member
    DevParams p;
    const void* buf[2];
    int* err;
    int kind;
};

// One unit of work: a TX-wide strip of rows [y0, y1) of lattice `lat`, segmented like
// the single-lattice kernel (row segments of the same strip recompute their halo rows).
struct BatchItem {
    int lat, x0, y0, y1;
};

// Advances the lattices of one collision variant of a batch by one time step (one
// launch per variant present; usually one).  CTA b takes items b, b + grid, b + 2 grid,
// ... (a persistent grid of one wave, or one CTA per item); `step_parity` flips the
// source copy of every lattice at once.  All lattices share the storage format; each
// runs the single-lattice strip code, so it evolves bit-identically alone or in a batch.
template <int TX, class ST, int KIND>
__global__ void __launch_bounds__(TX, 512 / TX) tclbm_step_batch(const BatchLattice* __restrict__ lats,
                                                                 const BatchItem* __restrict__ items, int nitems,
                                                                 int step_parity) {
    __shared__ DevParams sp;
    __shared__ float ring[3][TX + 4];
    constexpr int kWords = (int)(sizeof(DevParams) / sizeof(int));
    constexpr int kParityWord = (int)(offsetof(DevParams, parity) / sizeof(int));
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
        const BatchItem it = items[i];
        const BatchLattice* L = lats + it.lat;
        __syncthreads();  // the previous item is done with sp and the ring
        {
            const int* s = reinterpret_cast<const int*>(&L->p);
            int* d = reinterpret_cast<int*>(&sp);
            for (int w = threadIdx.x; w < kWords; w += TX) d[w] = w == kParityWord ? (s[w] ^ step_parity) : s[w];
        }
        __syncthreads();
        const int par = sp.parity;
        const ST* src = static_cast<const ST*>(L->buf[par]);
        ST* dst = static_cast<ST*>(const_cast<void*>(L->buf[par ^ 1]));
        if (KIND == BATCH_THERMAL_CORR)
            strip_corr<TX, ST>(sp, src, dst, it.x0, it.y0, it.y1, ring);
        else
            strip_plain<TX, KIND == BATCH_THERMAL, ST>(sp, src, dst, it.x0, it.y0, it.y1);
        if (it.x0 == 0 && it.y0 == 0) bump_step_counter(sp);
    }
}

}  // namespace tclbm
