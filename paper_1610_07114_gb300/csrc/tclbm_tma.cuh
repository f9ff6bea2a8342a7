// tclbm_tma.cuh -- the fused step with TMA-fed row staging (sm_103a).
//
// One thread per CTA streams whole source rows -- all 9 or 18 planes of columns
// [x0 - M, x0 + TX + M) -- from HBM into a shared-memory ring (7 FP32 / 8 16-bit slots)
// with cp.async.bulk.tensor (one 3-D box per row), signalling an mbarrier per slot.  The
// compute threads pull their node's populations from the ring (f_q(x, t+1) =
// f_out_q(x - e_q, t) is a shifted shared-memory read), collide, and store their own
// node to the destination copy.  Rows are staged several rows ahead of use, so HBM
// latency is hidden by the copy engine rather than by registers or occupancy.
//
// While output row r is processed: its pull needs source rows r-1..r+1, a top-wall
// node also its interior neighbour's pulls (r-2..r), the correction-term lookahead row
// r+1 sources up to r+2, and a bottom-wall node the one-sided stencil's row 2 (sources
// up to 3).  The correction kernel keeps the lookahead row's pulled populations in
// registers, so its collision reads no ring row and a slot is free one row after its
// last lookahead use; the plain kernel pulls at collision time and frees slots later.
// A launch that finds the error word set returns at once.  Periodic wrap in x: strips whose
// box crosses x = 0 or x = nx patch the wrapped columns from global memory after the
// row lands; in y the producer requests the wrapped (or clamped) row directly.
//
// Every wait is bounded by the global timer; on expiry the CTA records an error code,
// drains its own outstanding copies (again bounded) and returns.
#pragma once

#include <cuda.h>

#include "tclbm_batch.cuh"
#include "tclbm_device.cuh"

namespace tclbm {

constexpr long long kWaitNs = 1000000000LL;  // 1 s per wait

// Ring slots: FP32 rows are twice the bytes of 16-bit rows; 7 FP32 slots (69 KB) keep
// three CTAs per SM, 8 16-bit slots (43 KB) five.
template <class ST>
struct RingSlots {
    static constexpr int N = sizeof(ST) == 4 ? 7 : 8;
};

__device__ __forceinline__ long long globaltimer_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait: true when the phase with this parity completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long deadline = globaltimer_ns() + kWaitNs;
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() > deadline) return false;
    return true;
}

// Row copy: box (BOXW, 1, NP) at (x, y, 0) into `dst`, completing on `bar`.
__device__ __forceinline__ void tma_row(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                        uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(0), "r"(smem_u32(bar))
        : "memory");
}

template <class ST>
struct TmaGeom {
    static constexpr int M = 16 / (int)sizeof(ST);  // halo columns each side; keeps x * size on 16 B
};

// Shared-memory pull of node column `xi` (index in the box) for target row t, whose
// source rows t-1, t, t+1 sit at ring slots sm1, s0, sp1.
template <bool THERMAL, class ST, int BOXW, int SLOT>
__device__ __forceinline__ void pull_ring(const ST* ring, int sm1, int s0, int sp1, int xi, float* f, float* h) {
    // plane q comes from source row t - e_qy and column x - e_qx
    const ST* r_m = ring + sm1 * SLOT;  // row t-1 (e_y = +1: planes 2, 5, 6)
    const ST* r_0 = ring + s0 * SLOT;   // row t   (planes 0, 1, 3)
    const ST* r_p = ring + sp1 * SLOT;  // row t+1 (planes 4, 7, 8)
    auto ld = [](const ST* p) { return Store<ST>::ld_smem(p); };
    f[0] = ld(r_0 + 0 * BOXW + xi);
    f[1] = ld(r_0 + 1 * BOXW + xi - 1);
    f[2] = ld(r_m + 2 * BOXW + xi);
    f[3] = ld(r_0 + 3 * BOXW + xi + 1);
    f[4] = ld(r_p + 4 * BOXW + xi);
    f[5] = ld(r_m + 5 * BOXW + xi - 1);
    f[6] = ld(r_m + 6 * BOXW + xi + 1);
    f[7] = ld(r_p + 7 * BOXW + xi + 1);
    f[8] = ld(r_p + 8 * BOXW + xi - 1);
    if (THERMAL) {
        h[0] = ld(r_0 + 9 * BOXW + xi);
        h[1] = ld(r_0 + 10 * BOXW + xi - 1);
        h[2] = ld(r_m + 11 * BOXW + xi);
        h[3] = ld(r_0 + 12 * BOXW + xi + 1);
        h[4] = ld(r_p + 13 * BOXW + xi);
        h[5] = ld(r_m + 14 * BOXW + xi - 1);
        h[6] = ld(r_m + 15 * BOXW + xi + 1);
        h[7] = ld(r_p + 16 * BOXW + xi + 1);
        h[8] = ld(r_p + 17 * BOXW + xi - 1);
    }
}

// Pipeline bookkeeping shared by the two kernels below.
template <int TX, bool THERMAL, class ST>
struct RowRing {
    static constexpr int M = TmaGeom<ST>::M;
    static constexpr int BOXW = TX + 2 * M;
    static constexpr int NP = THERMAL ? 18 : 9;
    static constexpr uint32_t ROW_BYTES = (uint32_t)(BOXW * NP * sizeof(ST));     // bytes one copy delivers
    static constexpr uint32_t SLOT_BYTES = (ROW_BYTES + 127u) / 128u * 128u;       // slots start 128-byte aligned
    static constexpr int SLOT_ELEMS = (int)(SLOT_BYTES / sizeof(ST));
    static constexpr int NS = RingSlots<ST>::N;
    static constexpr size_t RING_BYTES = (size_t)NS * SLOT_BYTES;

    ST* ring;
    uint64_t* bar;
    const CUtensorMap* map;
    int s_first, s_last;  // source rows this CTA stages
    int issued_to;        // highest source row issued
    int ready_to;         // highest source row waited for (and patched)
    int freed_to;         // highest source row whose slot was handed back for a refill
    bool patch;           // strip box crosses x = 0 or x = nx on a periodic x axis
    int xb;               // logical column of box index 0

    __device__ __forceinline__ int slot(int s) const { return (s - s_first) % NS; }
    __device__ __forceinline__ uint32_t parity(int s) const { return (uint32_t)(((s - s_first) / NS) & 1); }
    __device__ __forceinline__ int phys_row(const DevParams& p, int s) const {
        if (p.yper) return ((s % p.ny) + p.ny) % p.ny;
        return s < 0 ? 0 : (s >= p.ny ? p.ny - 1 : s);
    }
    // thread 0 only
    __device__ __forceinline__ void issue(const DevParams& p, int s) {
        // test hook (tclbm_test_skip_row, FP32 builds only: in the 16-bit builds its register
        // cost measured 3 %): leave this row's barrier phase open, so the bounded wait on it
        // expires and the error path runs.  Source rows below 0 exist (wrapped or clamped).
        if (sizeof(ST) != 4 || p.skip_row < 0 || s != p.skip_row)
            tma_row(ring + (size_t)slot(s) * SLOT_ELEMS, map, bar + slot(s), xb, phys_row(p, s), ROW_BYTES);
        issued_to = s;
    }
    // every thread: make sources up to `s_need` available; false on timeout
    __device__ __forceinline__ bool acquire(const DevParams& p, const ST* __restrict__ src, int s_need) {
        if (s_need > s_last) s_need = s_last;
        bool ok = true;
        bool patched = false;
        while (ready_to < s_need) {
            const int s = ready_to + 1;
            ok = mbar_wait(bar + slot(s), parity(s)) && ok;
            if (patch) {
                // wrapped columns of a periodic x axis, straight from global memory: the
                // box columns left of x = 0 (n_left of them) and right of nx - 1 (n_right)
                ST* row = ring + (size_t)slot(s) * SLOT_ELEMS;
                const ST* srow = src + (long long)phys_row(p, s) * p.pitch;
                const int n_left = xb < 0 ? -xb : 0;
                const int c_right = p.nx - xb;  // first box column with x >= nx
                const int n_right = c_right < BOXW ? BOXW - c_right : 0;
                const int ncol = n_left + n_right;
                for (int i = threadIdx.x; i < ncol * NP; i += blockDim.x) {
                    const int q = i / ncol, k = i - q * ncol;
                    const int c = k < n_left ? k : c_right + (k - n_left);
                    int xp = xb + c;
                    xp = xp < 0 ? xp + p.nx : xp - p.nx;
                    if (xp < 0 || xp >= p.nx) xp = ((xp % p.nx) + p.nx) % p.nx;  // nx smaller than the halo
                    row[q * BOXW + c] = srow[(long long)q * p.plane + xp];
                }
                patched = true;
            }
            ready_to = s;
        }
        if (patched) __syncthreads();
        return ok;
    }
    // every thread, after a timeout was agreed on: wait (bounded) for copies still in flight
    __device__ __forceinline__ void drain() {
        for (int s = ready_to + 1; s <= issued_to; ++s) mbar_wait(bar + slot(s), parity(s));
    }
};

// Ring slots of source rows t-2 .. t+2 around a target row t (computed once per row).
struct Slots5 {
    int m2, m1, z, p1, p2;
};

// Streamed populations of the node at box index xi, physical (x, y), target row t,
// with its wall scheme applied when `maybe_wall` (its row or column is a wall): the
// wall neighbour is read from the ring as well (rows t +- 1, sources t-2 .. t+2).
template <int TX, bool THERMAL, class ST>
__device__ __forceinline__ void load_node_ring(const DevParams& p, const RowRing<TX, THERMAL, ST>& R, const Slots5& sl,
                                               int xi, int x, int y, bool maybe_wall, float* f, float* h) {
    using RR = RowRing<TX, THERMAL, ST>;
    pull_ring<THERMAL, ST, RR::BOXW, RR::SLOT_ELEMS>(R.ring, sl.m1, sl.z, sl.p1, xi, f, h);
    if (maybe_wall) {
        const int side = wall_side_of(p, x, y);
        if (side >= 0) {
            float ff[9], hf[9];
            if (side == SIDE_YM)
                pull_ring<THERMAL, ST, RR::BOXW, RR::SLOT_ELEMS>(R.ring, sl.z, sl.p1, sl.p2, xi, ff, hf);
            else if (side == SIDE_YP)
                pull_ring<THERMAL, ST, RR::BOXW, RR::SLOT_ELEMS>(R.ring, sl.m2, sl.m1, sl.z, xi, ff, hf);
            else
                pull_ring<THERMAL, ST, RR::BOXW, RR::SLOT_ELEMS>(R.ring, sl.m1, sl.z, sl.p1,
                                                                  xi + (side == SIDE_XM ? 1 : -1), ff, hf);
            wall_rebuild_call<THERMAL>(p, side, x, y, f, h, ff, hf);
        }
    }
}

template <int NS>
__device__ __forceinline__ Slots5 slots_around(int st) {  // st = ring slot of row t
    Slots5 s;
    s.z = st;
    s.m1 = st == 0 ? NS - 1 : st - 1;
    s.m2 = s.m1 == 0 ? NS - 1 : s.m1 - 1;
    s.p1 = st == NS - 1 ? 0 : st + 1;
    s.p2 = s.p1 == NS - 1 ? 0 : s.p1 + 1;
    return s;
}

template <int TX, bool THERMAL, class ST>
__device__ __forceinline__ void ring_setup(RowRing<TX, THERMAL, ST>& R, unsigned char* smem, const CUtensorMap* map,
                                           int x0, int s_first, int s_last, const DevParams& p) {
    using RR = RowRing<TX, THERMAL, ST>;
    R.ring = reinterpret_cast<ST*>(smem);
    R.bar = reinterpret_cast<uint64_t*>(smem + RR::RING_BYTES);  // 8 barrier words reserved
    R.map = map;
    R.s_first = s_first;
    R.s_last = s_last;
    R.issued_to = s_first - 1;
    R.ready_to = s_first - 1;
    R.freed_to = s_first - 1;
    R.xb = x0 - RR::M;
    R.patch = p.xper && (R.xb < 0 || R.xb + RR::BOXW > p.nx);
    if (threadIdx.x == 0) {
        for (int k = 0; k < RR::NS; ++k) mbar_init(R.bar + k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int last = s_first + RR::NS - 1 < s_last ? s_first + RR::NS - 1 : s_last;
        for (int s = s_first; s <= last; ++s) R.issue(p, s);
    }
}

// thread 0: reuse the slots of source rows up to `s_free` that nobody reads any more
// (called after a barrier); each freed slot takes the row NS further on.
template <int TX, bool THERMAL, class ST>
__device__ __forceinline__ void ring_refill(RowRing<TX, THERMAL, ST>& R, const DevParams& p, int s_free) {
    constexpr int NS = RowRing<TX, THERMAL, ST>::NS;
    if (threadIdx.x != 0 || s_free <= R.freed_to) return;
    // generic-proxy reads (and wrap patches) of these slots happened before the barrier
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int s = R.freed_to + 1; s <= s_free; ++s) {
        const int s_new = s + NS;
        if (s_new <= R.s_last && s_new > R.issued_to) R.issue(p, s_new);
    }
    R.freed_to = s_free;
}

// Rows [y0, y1) of this CTA's segment (blockIdx.y) under the host's segment plan
// (tma_seg_plan): seg_full segments of `rows` rows, the first one seg_extra rows taller,
// then half-height segments; the last segment ends at ny.
__device__ __forceinline__ void tma_segment(const DevParams& p, int rows, int seg_full, int seg_extra, int& y0,
                                            int& y1) {
    const int j = blockIdx.y;
    if (j < seg_full) {
        y0 = j == 0 ? 0 : seg_extra + j * rows;
        y1 = seg_extra + (j + 1) * rows;
    } else {
        const int h = rows / 2;
        y0 = seg_extra + seg_full * rows + (j - seg_full) * h;
        y1 = y0 + h;
    }
    if (j == (int)gridDim.y - 1) y1 = p.ny;
}

// Without the correction term (athermal, or thermal with C off).
template <int TX, bool THERMAL, class ST>
__global__ void __launch_bounds__(TX, 512 / TX) tclbm_step_tma_plain(const __grid_constant__ DevParams p, const __grid_constant__ CUtensorMap map,
                                                           const ST* __restrict__ src, ST* __restrict__ dst,
                                                           int rows_per_cta, int seg_full, int seg_extra,
                                                           int* __restrict__ err, unsigned* __restrict__ /*seg_done*/,
                                                           unsigned /*ticket*/, int /*chain*/) {
    extern __shared__ __align__(128) unsigned char smem[];
    using RR = RowRing<TX, THERMAL, ST>;
    RR R;
    // programmatic dependent launch, as in tclbm_step_tma_corr
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (*(volatile int*)err) return;  // an earlier launch gave up: do not queue more waits
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX;
    int y0, y1;
    tma_segment(p, rows_per_cta, seg_full, seg_extra, y0, y1);
    // output row r pulls sources r-1..r+1; a wall row's neighbour reaches r-2 / r+2
    ring_setup<TX, THERMAL, ST>(R, smem, &map, x0, y0 - 2, y1 + 1, p);
    const int x = x0 + tid;
    const bool owns = x < p.nx;
    const int xi = tid + RR::M;
    const bool col_wall = !p.xper && (x == 0 || x == p.nx - 1);
    int st = R.slot(y0);
    for (int r = y0; r < y1; ++r) {
        const bool ok = R.acquire(p, src, r + 2);
        if (owns) {
            const Slots5 sl = slots_around<RR::NS>(st);
            const bool maybe_wall = col_wall || (!p.yper && (r == 0 || r == p.ny - 1));
            float f[9], h[9], fo[9], ho[9];
            load_node_ring<TX, THERMAL, ST>(p, R, sl, xi, x, r, maybe_wall, f, h);
            const Macro m = macro_of<THERMAL>(p, f, h, x, r);
            collide<THERMAL>(p, f, h, m, 0.0f, 0.0f, fo, ho);
            store_node<ST>(p, dst, x, r, fo, ho, THERMAL);
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            R.drain();
            return;
        }
        ring_refill<TX, THERMAL, ST>(R, p, r - 2);
        st = st == RR::NS - 1 ? 0 : st + 1;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0) bump_step_counter(p);
}

// With the correction term: lookahead of one row for the same-time moments, x halo of
// two columns each side from the ring, the x-derivative through a three-row ring of
// u_x (1 - theta) in shared memory.
// Threads per SM the register budget is sized for: FP32 rows fill the shared memory
// at three CTAs per SM (160 registers each); 16-bit rows run four CTAs of 128.
template <class ST>
struct CorrShape {
    static constexpr int kThreadsPerSM = sizeof(ST) == 4 ? 384 : 512;
};

// One strip: columns [x0, x0 + TX) of rows [y0, y1), every thread of the CTA.  `p` is a
// kernel parameter or a shared-memory copy; `map` the source copy's tensor map (in
// parameter or global memory); `smem` the dynamic shared memory of tma_smem_bytes().
// Returns false after a bounded wait expired (the error word is then set).
template <int TX, class ST>
__device__ __forceinline__ bool tma_corr_strip(const DevParams& p, const CUtensorMap* map, const ST* __restrict__ src,
                                               ST* __restrict__ dst, int x0, int y0, int y1, int* __restrict__ err,
                                               unsigned char* smem) {
    using RR = RowRing<TX, true, ST>;
    RR R;
    float(*phix)[TX + 4] = reinterpret_cast<float(*)[TX + 4]>(smem + RR::RING_BYTES + 8 * sizeof(uint64_t));
    const int tid = threadIdx.x;
    const int nx = p.nx, ny = p.ny;
    const bool ywall = !p.yper;
    // sources: the phi_y of row y0-1 needs y0-2; the lookahead of row y1 needs y1+1;
    // the bottom wall's one-sided stencil needs row 3 (inside the first ring fill); a
    // top-wall row within two rows of the segment start also needs phi_y(y0-2) (y0-3)
    const bool short_top = ywall && y1 == ny && y0 >= 2 && y1 - y0 < 3;
    const int s_first = short_top ? y0 - 3 : y0 - 2;
    int s_last = y1 + 1;
    if (ywall && y0 == 0 && s_last < 3) s_last = 3;
    ring_setup<TX, true, ST>(R, smem, map, x0, s_first, s_last, p);

    const int xl = x0 + tid;  // logical column of this thread
    const bool owns = xl < nx;
    const int xown = p.xper ? (xl % nx) : xl;
    const bool own_valid = p.xper || owns;
    const int xi = tid + RR::M;
    // the four halo slots (columns x0-2, x0-1, x0+TX, x0+TX+1) go to lanes 0..3 of the last warp
    int hslot = -1, xh = 0, xih = 0;
    bool h_valid = false;
    const int hl = tid - (TX - 32);
    if (hl >= 0 && hl < 4) {
        hslot = hl < 2 ? hl : TX + hl;
        const int xlh = x0 - 2 + hslot;
        xih = hslot - 2 + RR::M;
        if (p.xper) {
            xh = ((xlh % nx) + nx) % nx;
            h_valid = true;
        } else {
            xh = xlh;
            h_valid = xlh >= 0 && xlh < nx;
        }
    }

    const bool col_wall_own = !p.xper && (xl == 0 || xl == nx - 1);
    const bool col_wall_halo = !p.xper && (xh == 0 || xh == nx - 1);
    float py_m2 = 0.f, py_m1 = 0.f, py_0 = 0.f, py_p1 = 0.f;
    Macro mc, mn;
    float fc[9], hc[9], fn[9], hn[9];  // pulled populations of rows r and r+1
    // moments of row t (physical row yr, ring slot st): own column (kept, with its pulled
    // populations) and, for four lanes, a halo column
    auto moments_row = [&](int t, int yr, int st, Macro& m, float& py, int buf, float* fk, float* hk) {
        const Slots5 sl = slots_around<RR::NS>(st);
        const bool row_wall = ywall && (t == 0 || t == ny - 1);
        if (own_valid) {
            float f[9], h[9];
            load_node_ring<TX, true, ST>(p, R, sl, xi, xown, yr, row_wall || col_wall_own, f, h);
            m = macro_of<true>(p, f, h, xown, yr);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                fk[q] = f[q];
                hk[q] = h[q];
            }
            phix[buf][tid + 2] = phi_x(m);
            py = phi_y(m);
        }
        if (hslot >= 0 && h_valid) {
            float f[9], h[9];
            load_node_ring<TX, true, ST>(p, R, sl, xih, xh, yr, row_wall || col_wall_halo, f, h);
            phix[buf][hslot] = phi_x(macro_of<true>(p, f, h, xh, yr));
        }
    };
    auto phiy_row = [&](int t, int yr, int st) -> float {
        if (!own_valid) return 0.f;
        const Slots5 sl = slots_around<RR::NS>(st);
        const bool row_wall = ywall && (t == 0 || t == ny - 1);
        float f[9], h[9];
        load_node_ring<TX, true, ST>(p, R, sl, xi, xown, yr, row_wall || col_wall_own, f, h);
        return phi_y(macro_of<true>(p, f, h, xown, yr));
    };
    auto next_slot = [](int st) { return st == RR::NS - 1 ? 0 : st + 1; };
    auto prev_slot = [](int st) { return st == 0 ? RR::NS - 1 : st - 1; };

    bool ok = true;
    // prologue: phi_y of row y0-1 (if it exists) and the moments of row y0
    ok = R.acquire(p, src, y0 + 2) && ok;  // a bottom-wall row y0 reads its neighbour's sources up to y0+2
    int st = R.slot(y0);                    // ring slot of row r (collision row)
    int yr_next = p.yper ? (y0 + 1 == ny ? 0 : y0 + 1) : y0 + 1;  // physical row r + 1
    if (y0 > 0 || p.yper) py_m1 = phiy_row(y0 - 1, y0 == 0 ? ny - 1 : y0 - 1, prev_slot(st));
    if (short_top) py_m2 = phiy_row(y0 - 2, y0 - 2, prev_slot(prev_slot(st)));
    moments_row(y0, y0, st, mc, py_0, ((y0 % 3) + 3) % 3, fc, hc);
    int buf_c = ((y0 % 3) + 3) % 3;

    __syncthreads();  // the prologue's phi_x row is read by the first collision

    // Row r: the lookahead of row r+1 (pull, moments, phi) and the collision of row r
    // (from registers and the phi_x row published one barrier earlier) share one block
    // between barriers, so the two independent chains interleave.
    for (int r = y0; r < y1; ++r) {
        const bool has_next = (r + 1 < ny) || p.yper;
        const int buf_n = buf_c == 2 ? 0 : buf_c + 1;
        int need = r + 2;
        if (ywall && r == 0) need = 3;
        ok = R.acquire(p, src, need) && ok;
        if (has_next) moments_row(r + 1, yr_next, next_slot(st), mn, py_p1, buf_n, fn, hn);
        float py_p2 = 0.f;
        if (ywall && r == 0) py_p2 = phiy_row(2, 2, next_slot(next_slot(st)));
        if (owns && ok) {
            const float* rw = phix[buf_c];
            const int s = tid + 2;
            float dxv;
            if (col_wall_own && xl == 0)
                dxv = 0.5f * (-3.0f * rw[s] + 4.0f * rw[s + 1] - rw[s + 2]);
            else if (col_wall_own)
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
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            R.drain();
            return false;
        }
        // later rows read sources from r on (a top-wall row r+2 reads its neighbour's
        // r..r+2): the slot of r-1 is free
        ring_refill<TX, true, ST>(R, p, r - 1);
        py_m2 = py_m1;
        py_m1 = py_0;
        py_0 = py_p1;
        mc = mn;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            fc[q] = fn[q];
            hc[q] = hn[q];
        }
        st = next_slot(st);
        buf_c = buf_n;
        yr_next = (p.yper && yr_next == ny - 1) ? 0 : yr_next + 1;
    }
    return true;
}

// ---------------------------------------------------------------- chained launches
//
// Consecutive launches of the kernel below on one lattice can be chained: instead of
// waiting for the whole previous grid (griddepcontrol.wait), a CTA waits only for the
// nine work items around its own (strip +-1, segment +-1, wrapped on periodic axes) to
// have finished the previous step.  Those items wrote every source row this CTA reads
// (rows y0-3 .. y1+1 and columns x0-M .. x0+TX+M, inside those items where every segment
// has at least 4 rows and the last strip at least M columns: the host chains only such
// plans) and were the only readers of the rows it overwrites, so the wait covers both
// orders.  Each item
// publishes, once all its stores are issued, the launch's ticket (a per-lattice counter
// that only grows) in seg_done[blockIdx.y * gridDim.x + blockIdx.x]; the next launch
// (ticket + 1) proceeds once the nine entries reach ticket.  The next grid is released
// when every CTA of this one has started (griddepcontrol.launch_dependents at entry), so
// every item waited on is already resident or finished: the waits cannot deadlock.  The
// first launch of a chain, and every launch of a captured graph, waits for the previous
// grid as before.

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Every thread: true once the nine items around this CTA's reached `need` (false after
// the error word was set, by this wait expiring (code 2) or by another CTA).
__device__ __forceinline__ bool seg_wait_neighbours(const DevParams& p, const unsigned* __restrict__ seg_done,
                                                    unsigned need, int* __restrict__ err) {
    int fail = 0;
    const int t = threadIdx.x;
    if (t < 9) {
        const int gx = (int)gridDim.x, gy = (int)gridDim.y;
        int ix = (int)blockIdx.x + t % 3 - 1, iy = (int)blockIdx.y + t / 3 - 1;
        bool use = true;
        if (ix < 0 || ix >= gx) {
            if (p.xper) ix = ix < 0 ? ix + gx : ix - gx;
            else use = false;
        }
        if (iy < 0 || iy >= gy) {
            if (p.yper) iy = iy < 0 ? iy + gy : iy - gy;
            else use = false;
        }
        if (use) {
            const unsigned* f = seg_done + (size_t)iy * gx + ix;
            if ((int)(ld_acquire_gpu(f) - need) < 0) {
                const long long deadline = globaltimer_ns() + kWaitNs;
                while ((int)(ld_acquire_gpu(f) - need) < 0) {
                    if (*(volatile int*)err) {
                        fail = 1;
                        break;
                    }
                    if (globaltimer_ns() > deadline) {
                        atomicExch(err, 2);
                        fail = 1;
                        break;
                    }
                    __nanosleep(128);
                }
            }
        }
    }
    fail = __syncthreads_or(fail);
    // the rows the neighbours stored through the generic proxy are read next by TMA
    if (!fail) asm volatile("fence.proxy.async.global;" ::: "memory");
    return !fail;
}

// Every thread, after its last store: publish this item's completion of launch `ticket`
// (the release store is cumulative over the stores the barrier ordered before it).
__device__ __forceinline__ void seg_mark_done(unsigned* __restrict__ seg_done, unsigned ticket) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0)
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(seg_done + (size_t)blockIdx.y * gridDim.x + blockIdx.x),
                     "r"(ticket)
                     : "memory");
}

// seg_done: completion tickets of the work items (nullptr: none published); chain: wait
// for the neighbouring items of launch ticket - 1 instead of the whole previous grid.
template <int TX, class ST>
__global__ void __launch_bounds__(TX, CorrShape<ST>::kThreadsPerSM / TX) tclbm_step_tma_corr(const __grid_constant__ DevParams p, const __grid_constant__ CUtensorMap map,
                                                          const ST* __restrict__ src, ST* __restrict__ dst,
                                                          int rows_per_cta, int seg_full, int seg_extra,
                                                          int* __restrict__ err, unsigned* __restrict__ seg_done,
                                                          unsigned ticket, int chain) {
    extern __shared__ __align__(128) unsigned char smem[];
    // programmatic dependent launch: this grid's CTAs take the slots the previous step's
    // grid frees and wait here for its completion (its writes are this step's source),
    // or, chained, for the previous step's items around their own
    if (!chain) asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (*(volatile int*)err) return;  // an earlier launch gave up: do not queue more waits
    int y0, y1;
    tma_segment(p, rows_per_cta, seg_full, seg_extra, y0, y1);
    if (chain && !seg_wait_neighbours(p, seg_done, ticket - 1u, err)) return;
    if (!tma_corr_strip<TX, ST>(p, &map, src, dst, blockIdx.x * TX, y0, y1, err, smem)) return;
    if (seg_done) seg_mark_done(seg_done, ticket);
    if (blockIdx.x == 0 && blockIdx.y == 0) bump_step_counter(p);
}

// Batched form of the kernel above (thermal lattices with the correction term): CTA b
// takes work item b, a strip of TX columns by rows [y0, y1) of one lattice, whose
// constants it copies to shared memory (parity flipped by `step_parity`) and whose row
// tensor map it reads from the lattice's descriptor in global memory.  Every node runs
// the same code as in the single-lattice kernel, so a lattice evolves bit for bit as it
// does alone with that kernel.  A lattice whose error word is set is skipped; an
// expired wait sets it.
template <int TX, class ST>
__global__ void __launch_bounds__(TX, CorrShape<ST>::kThreadsPerSM / TX) tclbm_step_batch_tma(
    const BatchLattice* __restrict__ lats, const BatchItem* __restrict__ items, int nitems, int step_parity) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ DevParams sp;
    const BatchItem it = items[blockIdx.x];
    const BatchLattice* L = lats + it.lat;
    if (*(volatile int*)L->err) return;  // an earlier launch on this lattice gave up
    constexpr int kWords = (int)(sizeof(DevParams) / sizeof(int));
    constexpr int kParityWord = (int)(offsetof(DevParams, parity) / sizeof(int));
    {
        const int* s = reinterpret_cast<const int*>(&L->p);
        int* d = reinterpret_cast<int*>(&sp);
        for (int w = threadIdx.x; w < kWords; w += TX) d[w] = w == kParityWord ? (s[w] ^ step_parity) : s[w];
    }
    __syncthreads();
    const int par = sp.parity;
    const CUtensorMap* map = &L->map[par];
    // the descriptor was written through the generic proxy (a host copy); the TMA unit
    // reads it through the tensor-map proxy
    if (threadIdx.x == 0) asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
    const ST* src = static_cast<const ST*>(L->buf[par]);
    ST* dst = static_cast<ST*>(const_cast<void*>(L->buf[par ^ 1]));
    if (!tma_corr_strip<TX, ST>(sp, map, src, dst, it.x0, it.y0, it.y1, L->err, smem)) return;
    if (it.x0 == 0 && it.y0 == 0) bump_step_counter(sp);
}

// Dynamic shared memory of the TMA kernels.
template <int TX, bool THERMAL, class ST>
constexpr size_t tma_smem_bytes(bool corr) {
    return RowRing<TX, THERMAL, ST>::RING_BYTES + 8 * sizeof(uint64_t) + (corr ? 3 * (TX + 4) * sizeof(float) : 0);
}

}  // namespace tclbm
