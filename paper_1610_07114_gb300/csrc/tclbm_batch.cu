// tclbm_batch.cu -- many independent lattices advanced together: one launch of the
// batched step kernel per time step over a work list of strips of every lattice,
// CUDA-graph capture of long runs, and an autotuner of the work-list shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "tclbm.h"
#include "tclbm_internal.h"

using namespace tclbm;

struct tclbm_batch {
    std::vector<tclbm_lattice*> lats;
    cudaStream_t stream = nullptr;
    // allocator hooks copied from the first lattice at creation (the batch's own
    // memory does not depend on any lattice staying alive)
    tclbm_alloc_fn alloc = nullptr;
    tclbm_free_fn free_fn = nullptr;
    void* ctx = nullptr;
    int storage = 0;
    int sms = 0;
    // work-list shape of the direct-load strip kernel
    int tx = 64, rows = 4, persistent = 1;
    // TMA-fed strips for thermal lattices with the correction term at least tma_tx wide
    // (tma_tx = 0: off; one CTA per item)
    int tma_tx = 0, tma_rows = 16;
    // device arrays: descriptors and work items
    BatchLattice* d_lats = nullptr;
    size_t d_lats_bytes = 0;
    BatchItem* d_items = nullptr;
    size_t d_items_bytes = 0;
    int nitems = 0;
    // items grouped by kernel: groups 0..2 the direct-load kernel for each collision
    // variant (BATCH_*), group 3 the TMA-fed kernel; [first[g], first[g] + count[g]),
    // grid[g] CTAs
    int first[4] = {0, 0, 0, 0}, count[4] = {0, 0, 0, 0};
    unsigned grid[4] = {0, 0, 0, 0};
    // pinned staging of uploads, two generations: uploads are stream-ordered copies,
    // so the host never waits for the kernels in flight
    struct Staging {
        void* host = nullptr;
        size_t bytes = 0;
        cudaEvent_t used = nullptr;  // the copy out of `host` has executed
    } stage[2];
    int gen = 0;
    std::vector<BatchLattice> h_lats;  // last uploaded descriptors
    int64_t steps = 0;                 // batch steps taken (parity of the next launch)
    bool items_valid = false;
    // what the uploaded work list was built from: (nx, ny, variant) per lattice in list
    // order and the shape; a handle's address says nothing (a destroyed lattice's
    // address can come back for a new one of another size)
    std::vector<int> items_sig;
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    cudaEvent_t ev = nullptr;
    char desc[256] = "";
};

namespace {

int kind_of(const tclbm_lattice* L) {
    if (!L->prm.thermal) return BATCH_ATHERMAL;
    return L->prm.correction ? BATCH_THERMAL_CORR : BATCH_THERMAL;
}

long long nodes_of(const tclbm_lattice* L) { return (long long)L->prm.nx * L->prm.ny; }

constexpr int kGroupTma = 3;

// Whether lattice L steps in the TMA-fed group.
bool tma_item(const tclbm_batch* B, const tclbm_lattice* L) {
    return B->tma_tx > 0 && kind_of(L) == BATCH_THERMAL_CORR && L->prm.nx >= B->tma_tx;
}

// Work items for the current shape, grouped by kernel (the TMA-fed group first, then
// the direct-load groups by collision variant): within a group, lattices by decreasing
// size (longest work first); within a lattice row segments of `rows` rows (the last one
// takes the remainder, as in the single-lattice kernel) and strips of tx columns, strip
// index fastest.
void make_items(tclbm_batch* B, std::vector<BatchItem>& items) {
    std::vector<int> order(B->lats.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return nodes_of(B->lats[a]) > nodes_of(B->lats[b]); });
    items.clear();
    for (int g : {kGroupTma, (int)BATCH_THERMAL_CORR, (int)BATCH_THERMAL, (int)BATCH_ATHERMAL}) {
        B->first[g] = (int)items.size();
        for (int li : order) {
            const tclbm_lattice* L = B->lats[li];
            const bool tma = tma_item(B, L);
            if (g == kGroupTma ? !tma : (tma || kind_of(L) != g)) continue;
            const int tx = tma ? B->tma_tx : B->tx, rows = tma ? B->tma_rows : B->rows;
            const tclbm_params& p = L->prm;
            int nseg = p.ny / rows;
            if (nseg < 1) nseg = 1;
            const int nstrip = (p.nx + tx - 1) / tx;
            for (int sg = 0; sg < nseg; ++sg) {
                const int y0 = sg * rows;
                const int y1 = sg == nseg - 1 ? p.ny : y0 + rows;
                for (int c = 0; c < nstrip; ++c) items.push_back(BatchItem{li, c * tx, y0, y1});
            }
        }
        if (g == kGroupTma) {
            // as in the single-lattice TMA kernel: blocks run in index order, so where the
            // group spans more than two waves its last wave of items is cut to half height
            // (at a multiple of 8 rows) and the launch's tail is made of short CTAs
            const long long wave = (long long)B->sms * tma_corr_ctas_per_sm(B->storage, B->tma_tx);
            const long long n = (long long)items.size() - B->first[g];
            if (n > 2 * wave) {
                std::vector<BatchItem> tail(items.end() - wave, items.end());
                items.resize(items.size() - wave);
                for (const BatchItem& it : tail) {
                    const int cut = it.y0 + (it.y1 - it.y0) / 16 * 8;
                    if (cut - it.y0 >= 8 && it.y1 - cut >= 8) {
                        items.push_back(BatchItem{it.lat, it.x0, it.y0, cut});
                        items.push_back(BatchItem{it.lat, it.x0, cut, it.y1});
                    } else {
                        items.push_back(it);
                    }
                }
            }
        }
        B->count[g] = (int)items.size() - B->first[g];
    }
}

void* batch_alloc(tclbm_batch* B, size_t bytes) {
    if (bytes == 0) return nullptr;
    if (B->alloc) return B->alloc(bytes, (void*)B->stream, B->ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void release(tclbm_batch* B, void*& p, size_t& bytes) {
    if (p) {
        if (B->free_fn)
            B->free_fn(p, bytes, (void*)B->stream, B->ctx);
        else
            cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
}

// Copies `bytes` from `src` into the device array `dst` (grown if needed) on the batch
// stream, through the pinned staging buffer of this generation.  The previous user of
// that buffer is two uploads back; its copy has normally long executed.
tclbm_status upload(tclbm_batch* B, void*& dst, size_t& dst_bytes, const void* src, size_t bytes) {
    if (bytes == 0) return TCLBM_OK;
    if (bytes > dst_bytes) {
        release(B, dst, dst_bytes);  // stream-ordered (caching allocator) or device-synchronising (cudaFree)
        dst = batch_alloc(B, bytes);
        if (!dst) return fail(TCLBM_ENOMEM, "batch device allocation of %zu bytes failed", bytes);
        dst_bytes = bytes;
    }
    tclbm_batch::Staging& st = B->stage[B->gen & 1];
    ++B->gen;
    CK(cudaEventSynchronize(st.used));
    if (bytes > st.bytes) {
        if (st.host) cudaFreeHost(st.host);
        st.host = nullptr;
        st.bytes = 0;
        CK(cudaMallocHost(&st.host, bytes));
        st.bytes = bytes;
    }
    std::memcpy(st.host, src, bytes);
    CK(cudaMemcpyAsync(dst, st.host, bytes, cudaMemcpyHostToDevice, B->stream));
    CK(cudaEventRecord(st.used, B->stream));
    return TCLBM_OK;
}

std::vector<int> items_signature(const tclbm_batch* B) {
    std::vector<int> sig;
    sig.reserve(3 * B->lats.size() + 3);
    sig.push_back(B->tx);
    sig.push_back(B->rows);
    sig.push_back(B->persistent);
    sig.push_back(B->tma_tx);
    sig.push_back(B->tma_rows);
    for (const tclbm_lattice* L : B->lats) {
        sig.push_back(L->prm.nx);
        sig.push_back(L->prm.ny);
        sig.push_back(kind_of(L));
    }
    return sig;
}

tclbm_status upload_items(tclbm_batch* B) {
    if (B->items_valid) return TCLBM_OK;
    std::vector<int> sig = items_signature(B);
    if (!B->items_sig.empty() && sig == B->items_sig) {  // same work list as uploaded
        B->items_valid = true;
        return TCLBM_OK;
    }
    std::vector<BatchItem> items;
    make_items(B, items);
    void* d = B->d_items;
    tclbm_status st = upload(B, d, B->d_items_bytes, items.data(), items.size() * sizeof(BatchItem));
    B->d_items = (BatchItem*)d;
    if (st != TCLBM_OK) return st;
    B->nitems = (int)items.size();
    for (int k = 0; k < 3; ++k) {
        const long long wave = (long long)B->sms * batch_ctas_per_sm(B->storage, B->tx, k);
        B->grid[k] = (unsigned)(B->persistent ? std::min<long long>(wave, B->count[k]) : B->count[k]);
    }
    B->grid[kGroupTma] = (unsigned)B->count[kGroupTma];
    B->items_valid = true;
    B->items_sig.swap(sig);
    B->graph_valid = false;
    return TCLBM_OK;
}

// Descriptors from the handles' current state: lattice i reads copy L->cur at the
// batch's current parity.  Re-uploaded only when something changed (a lattice stepped
// or re-initialised on its own between batch calls).
tclbm_status upload_lattices(tclbm_batch* B) {
    const int n = (int)B->lats.size();
    const int par = (int)(B->steps & 1);
    std::vector<BatchLattice> h(n);
    bool same = (int)B->h_lats.size() == n;
    for (int i = 0; i < n; ++i) {
        const tclbm_lattice* L = B->lats[i];
        std::memset(&h[i], 0, sizeof h[i]);
        h[i].p = L->dp;
        h[i].p.parity = L->cur ^ par;
        h[i].buf[0] = L->buf[0];
        h[i].buf[1] = L->buf[1];
        h[i].err = L->err;
        h[i].kind = kind_of(L);
        if (tma_item(B, L)) {
            tclbm_status ms = encode_row_maps(L, B->tma_tx, h[i].map);
            if (ms != TCLBM_OK) return ms;
        }
        if (same && std::memcmp(&h[i], &B->h_lats[i], sizeof h[i]) != 0) same = false;
    }
    if (same) return TCLBM_OK;
    void* d = B->d_lats;
    const size_t old_bytes = B->d_lats_bytes;
    tclbm_status st = upload(B, d, B->d_lats_bytes, h.data(), n * sizeof(BatchLattice));
    B->d_lats = (BatchLattice*)d;
    if (st != TCLBM_OK) return st;
    if (B->d_lats_bytes != old_bytes) B->graph_valid = false;  // the array moved
    B->h_lats.swap(h);
    return TCLBM_OK;
}

// Orders the batch stream after work queued on each lattice's own stream, or the
// reverse (after = true).
tclbm_status join_streams(tclbm_batch* B, bool after) {
    for (tclbm_lattice* L : B->lats) {
        if (L->stream == B->stream) continue;
        cudaStream_t from = after ? B->stream : L->stream;
        cudaStream_t to = after ? L->stream : B->stream;
        CK(cudaEventRecord(B->ev, from));
        CK(cudaStreamWaitEvent(to, B->ev, 0));
    }
    return TCLBM_OK;
}

// One batch step: a launch per kernel group present.
cudaError_t launch_one_step(const tclbm_batch* B, int parity, cudaStream_t s) {
    if (B->count[kGroupTma] > 0) {
        const cudaError_t e = launch_batch_tma_kernel(B->storage, B->tma_tx, B->grid[kGroupTma], B->d_lats,
                                                      B->d_items + B->first[kGroupTma], B->count[kGroupTma], parity, s);
        if (e != cudaSuccess) return e;
    }
    for (int k = 2; k >= 0; --k) {
        if (B->count[k] == 0) continue;
        const cudaError_t e = launch_batch_kernel(B->storage, B->tx, k, B->grid[k], B->d_lats,
                                                  B->d_items + B->first[k], B->count[k], parity, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

tclbm_status launch_batch_steps(tclbm_batch* B, int64_t n) {
    for (int64_t s = 0; s < n; ++s) {
        const cudaError_t e = launch_one_step(B, (int)(B->steps & 1), B->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batched step kernel launch");
        ++B->steps;
    }
    return TCLBM_OK;
}

tclbm_status build_batch_graph(tclbm_batch* B) {
    if (B->graph_valid) return TCLBM_OK;
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int s = 0; s < 2 * kGraphPairs && e == cudaSuccess; ++s)
            e = launch_one_step(B, s & 1, cs);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        B->graph = nullptr;
        return cuda_fail(e, "batched step graph capture");
    }
    B->graph_valid = true;
    return TCLBM_OK;
}

// Advances the batch by n steps on its stream (graphs for runs of 2 * kGraphPairs).
tclbm_status run_steps(tclbm_batch* B, int64_t n) {
    if (n >= 2 * kGraphPairs) {
        if (B->steps & 1) {
            tclbm_status st = launch_batch_steps(B, 1);
            if (st != TCLBM_OK) return st;
            --n;
        }
        tclbm_status st = build_batch_graph(B);
        if (st != TCLBM_OK) return st;
        while (n >= 2 * kGraphPairs) {
            CK(cudaGraphLaunch(B->graph, B->stream));
            B->steps += 2 * kGraphPairs;
            n -= 2 * kGraphPairs;
        }
    }
    return launch_batch_steps(B, n);
}

tclbm_status check_lattices(tclbm_lattice* const* lattices, int count, int storage) {
    for (int i = 0; i < count; ++i) {
        if (!lattices[i]) return fail(TCLBM_EINVAL, "lattice %d is NULL", i);
        if (lattices[i]->storage != storage)
            return fail(TCLBM_EINVAL, "lattice %d has another storage format than the batch", i);
        for (int j = 0; j < i; ++j)
            if (lattices[j] == lattices[i]) return fail(TCLBM_EINVAL, "lattice %d appears twice", i);
    }
    return TCLBM_OK;
}

bool valid_shape(int tx, int rows) { return (tx == 32 || tx == 64 || tx == 128) && rows >= 1; }

}  // namespace

extern "C" {

tclbm_status tclbm_batch_create(tclbm_lattice* const* lattices, int32_t count, void* stream, tclbm_batch** out) {
    if (!out) return fail(TCLBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!lattices || count < 1) return fail(TCLBM_EINVAL, "a batch needs at least one lattice");
    tclbm_status vs = check_lattices(lattices, count, lattices[0]->storage);
    if (vs != TCLBM_OK) return vs;
    tclbm_batch* B = new (std::nothrow) tclbm_batch;
    if (!B) return fail(TCLBM_ENOMEM, "host allocation failed");
    B->lats.assign(lattices, lattices + count);
    B->stream = (cudaStream_t)stream;
    B->storage = lattices[0]->storage;
    B->alloc = lattices[0]->alloc;
    B->free_fn = lattices[0]->free_fn;
    B->ctx = lattices[0]->ctx;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&B->stage[k].used, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete B;
        return cuda_fail(e, "batch setup");
    }
    // default shape: narrow strips and short segments for batches of small lattices
    long long total = 0;
    for (tclbm_lattice* L : B->lats) total += nodes_of(L);
    const long long avg = total / count;
    B->tx = avg <= (1LL << 16) ? 32 : 64;
    B->rows = avg <= (1LL << 16) ? 2 : 4;
    B->persistent = 1;
    tclbm_status st = upload_items(B);
    if (st == TCLBM_OK) st = upload_lattices(B);
    if (st != TCLBM_OK) {
        tclbm_batch_destroy(B);
        return st;
    }
    *out = B;
    return TCLBM_OK;
}

tclbm_status tclbm_batch_set_lattices(tclbm_batch* B, tclbm_lattice* const* lattices, int32_t count) {
    if (!B) return fail(TCLBM_EINVAL, "batch is NULL");
    if (count < 0 || (count > 0 && !lattices)) return fail(TCLBM_EINVAL, "bad lattice list");
    tclbm_status st = check_lattices(lattices, count, B->storage);
    if (st != TCLBM_OK) return st;
    // always rebuilt from the handles' current sizes (upload_items skips identical lists)
    B->lats.assign(lattices, lattices + count);
    B->items_valid = false;
    st = upload_items(B);
    if (st == TCLBM_OK) st = upload_lattices(B);
    return st;
}

int32_t tclbm_batch_size(const tclbm_batch* B) { return B ? (int32_t)B->lats.size() : -1; }

tclbm_status tclbm_batch_step(tclbm_batch* B, int64_t nsteps) {
    if (!B) return fail(TCLBM_EINVAL, "batch is NULL");
    if (nsteps < 0) return fail(TCLBM_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0) return TCLBM_OK;
    if (B->lats.empty()) {
        B->steps += nsteps;
        return TCLBM_OK;
    }
    tclbm_status st = join_streams(B, false);
    if (st == TCLBM_OK) st = upload_items(B);
    if (st == TCLBM_OK) st = upload_lattices(B);
    if (st == TCLBM_OK) st = run_steps(B, nsteps);
    if (st != TCLBM_OK) return st;
    for (tclbm_lattice* L : B->lats) {
        L->cur ^= (int)(nsteps & 1);
        L->steps += nsteps;
    }
    return join_streams(B, true);
}

tclbm_status tclbm_batch_set_tile(tclbm_batch* B, int32_t tx, int32_t rows, int32_t persistent) {
    if (!B) return fail(TCLBM_EINVAL, "batch is NULL");
    if (!valid_shape(tx, rows)) return fail(TCLBM_EINVAL, "tx must be 32, 64 or 128 and rows >= 1");
    if (tx != B->tx || rows != B->rows || (persistent != 0) != (B->persistent != 0)) {
        B->tx = tx;
        B->rows = rows;
        B->persistent = persistent != 0;
        B->items_valid = false;
    }
    return upload_items(B);
}

tclbm_status tclbm_batch_set_tma(tclbm_batch* B, int32_t tx, int32_t rows) {
    if (!B) return fail(TCLBM_EINVAL, "batch is NULL");
    if (!(tx == 0 || tx == 64 || tx == 128) || rows < 1)
        return fail(TCLBM_EINVAL, "TMA strips: tx must be 0 (off), 64 or 128 and rows >= 1");
    if (tx != B->tma_tx || rows != B->tma_rows) {
        B->tma_tx = tx;
        B->tma_rows = rows;
        B->items_valid = false;
    }
    tclbm_status st = upload_items(B);
    if (st == TCLBM_OK) st = upload_lattices(B);
    return st;
}

tclbm_status tclbm_batch_tma_shape(const tclbm_batch* B, int32_t* tx, int32_t* rows) {
    if (!B) return fail(TCLBM_EINVAL, "batch is NULL");
    if (tx) *tx = B->tma_tx;
    if (rows) *rows = B->tma_rows;
    return TCLBM_OK;
}

tclbm_status tclbm_batch_autotune(tclbm_batch* B, int32_t trial_steps, int32_t* best_tx, int32_t* best_rows,
                                  int32_t* best_persistent, float* best_us) {
    if (!B) return fail(TCLBM_EINVAL, "batch is NULL");
    if (trial_steps < 2) return fail(TCLBM_EINVAL, "trial_steps must be >= 2");
    trial_steps += trial_steps & 1;  // even: every lattice ends on the copy it started from
    tclbm_status st = join_streams(B, false);
    if (st == TCLBM_OK) st = upload_items(B);
    if (st == TCLBM_OK) st = upload_lattices(B);
    if (st != TCLBM_OK) return st;
    // keep the current state (source copy and stochastic-rounding counters) of every lattice
    size_t total = 0;
    for (tclbm_lattice* L : B->lats) total += L->buf_bytes + 256;
    void* backup_mem = batch_alloc(B, total);
    char* backup = (char*)backup_mem;
    if (!backup) return fail(TCLBM_ENOMEM, "autotune backup of %zu bytes failed", total);
    {
        size_t off = 0;
        for (tclbm_lattice* L : B->lats) {
            CK(cudaMemcpyAsync(backup + off, L->buf[L->cur], L->buf_bytes, cudaMemcpyDeviceToDevice, B->stream));
            CK(cudaMemcpyAsync(backup + off + L->buf_bytes, L->err, 256, cudaMemcpyDeviceToDevice, B->stream));
            off += L->buf_bytes + 256;
        }
    }
    const int keep_tx = B->tx, keep_rows = B->rows, keep_p = B->persistent;
    const int keep_ttx = B->tma_tx, keep_trows = B->tma_rows;
    const int64_t keep_steps = B->steps;
    int bt = keep_tx, br = keep_rows, bp = keep_p, btt = keep_ttx, btr = keep_trows;
    float best = 1e30f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    int max_ny = 1;
    bool any_tma = false;
    for (tclbm_lattice* L : B->lats) {
        max_ny = std::max(max_ny, L->prm.ny);
        any_tma = any_tma || (kind_of(L) == BATCH_THERMAL_CORR && L->prm.nx >= 64);
    }
    // one trial of the current shape: true if it was timed
    auto trial = [&](int tx, int rows, int pers, int ttx, int trows) {
        B->tx = tx;
        B->rows = rows;
        B->persistent = pers;
        B->tma_tx = ttx;
        B->tma_rows = trows;
        B->items_valid = false;
        st = upload_items(B);
        if (st == TCLBM_OK) st = upload_lattices(B);
        if (st == TCLBM_OK) st = launch_batch_steps(B, 2);  // warm-up
        if (st != TCLBM_OK) return;
        cudaEventRecord(e0, B->stream);
        st = launch_batch_steps(B, trial_steps);
        cudaEventRecord(e1, B->stream);
        if (st != TCLBM_OK) return;
        if ((ce = cudaEventSynchronize(e1)) != cudaSuccess) return;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        const float us = 1e3f * ms / trial_steps;
        if (us < best) {
            best = us;
            bt = tx;
            br = rows;
            bp = pers;
            btt = ttx;
            btr = trows;
        }
    };
    static const int kTx[] = {32, 64, 128};
    static const int kRows[] = {1, 2, 4, 8, 16, 32, 64};
    // direct-load strips for every lattice
    for (int t = 0; t < 3 && ce == cudaSuccess && st == TCLBM_OK; ++t)
        for (int r = 0; r < 7 && ce == cudaSuccess && st == TCLBM_OK; ++r)
            for (int pers = 0; pers < 2 && ce == cudaSuccess && st == TCLBM_OK; ++pers) {
                if (kRows[r] > max_ny) continue;
                trial(kTx[t], kRows[r], pers, 0, keep_trows);
            }
    // TMA-fed strips for the wide thermal lattices with the correction term, the others
    // on the best direct-load shape
    static const int kTmaTx[] = {64, 128};
    static const int kTmaRows[] = {8, 16, 32, 48, 64};
    const int dtx = bt, drows = br, dpers = bp;
    for (int t = 0; t < 2 && any_tma && ce == cudaSuccess && st == TCLBM_OK; ++t)
        for (int r = 0; r < 5 && ce == cudaSuccess && st == TCLBM_OK; ++r) {
            if (kTmaRows[r] > max_ny) continue;
            trial(dtx, drows, dpers, kTmaTx[t], kTmaRows[r]);
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // restore the state; the batch's parity is back where it was (even trial lengths)
    cudaError_t re = cudaSuccess;  // first failure of the restore copies
    {
        size_t off = 0;
        for (tclbm_lattice* L : B->lats) {
            cudaError_t e1 = cudaMemcpyAsync(L->buf[L->cur], backup + off, L->buf_bytes, cudaMemcpyDeviceToDevice,
                                             B->stream);
            cudaError_t e2 = cudaMemcpyAsync(L->err, backup + off + L->buf_bytes, 256, cudaMemcpyDeviceToDevice,
                                             B->stream);
            if (re == cudaSuccess) re = e1 != cudaSuccess ? e1 : e2;
            off += L->buf_bytes + 256;
        }
    }
    cudaError_t se = cudaStreamSynchronize(B->stream);
    if (se == cudaSuccess) se = re;
    release(B, backup_mem, total);
    B->steps = keep_steps;
    if (st != TCLBM_OK) return st;
    if (ce != cudaSuccess) return cuda_fail(ce, "autotune timing");
    if (se != cudaSuccess) return cuda_fail(se, "autotune restore");
    B->tx = bt;
    B->rows = br;
    B->persistent = bp;
    B->tma_tx = btt;
    B->tma_rows = btr;
    B->items_valid = false;
    st = upload_items(B);
    if (st == TCLBM_OK) st = upload_lattices(B);
    if (st != TCLBM_OK) return st;
    if (best_tx) *best_tx = bt;
    if (best_rows) *best_rows = br;
    if (best_persistent) *best_persistent = bp;
    if (best_us) *best_us = best;
    return join_streams(B, true);
}

const char* tclbm_batch_describe(const tclbm_batch* B) {
    if (!B) return "";
    tclbm_batch* M = const_cast<tclbm_batch*>(B);
    const char* st = B->storage == 0 ? "float" : (B->storage == 1 ? "bf16" : "half");
    int n = snprintf(M->desc, sizeof M->desc,
                     "tclbm_step_batch<%d,%s> lattices %zu items %d (corr %d, thermal %d, athermal %d) grid (%u,%u,%u) "
                     "block (%d) rows %d%s",
                     B->tx, st, B->lats.size(), B->nitems - B->count[kGroupTma], B->count[2], B->count[1], B->count[0],
                     B->grid[2], B->grid[1], B->grid[0], B->tx, B->rows, B->persistent ? " persistent" : "");
    if (B->count[kGroupTma] > 0 && n > 0 && n < (int)sizeof M->desc)
        snprintf(M->desc + n, sizeof M->desc - n, "; tclbm_step_batch_tma<%d,%s> items %d rows %d", B->tma_tx, st,
                 B->count[kGroupTma], B->tma_rows);
    return B->desc;
}

int64_t tclbm_batch_steps_done(const tclbm_batch* B) { return B ? B->steps : -1; }

tclbm_status tclbm_batch_destroy(tclbm_batch* B) {
    if (!B) return TCLBM_OK;
    cudaStreamSynchronize(B->stream);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->ev) cudaEventDestroy(B->ev);
    for (auto& st : B->stage) {
        if (st.used) cudaEventDestroy(st.used);
        if (st.host) cudaFreeHost(st.host);
    }
    void* p = B->d_items;
    release(B, p, B->d_items_bytes);
    p = B->d_lats;
    release(B, p, B->d_lats_bytes);
    delete B;
    return TCLBM_OK;
}

}  // extern "C"
