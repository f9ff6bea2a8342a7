/*
 * tclbm.h -- C ABI of the GB300 thermal cascaded lattice Boltzmann library
 * (Fei & Luo, "Thermal cascaded lattice Boltzmann method", arXiv:1610.07114).
 *
 * One handle = one D2Q9 lattice resident in device memory: two ping-pong copies of
 * the transformed populations f_bar (Section III, Eq. 12 and Eq. 27) and h_bar
 * (Section IV), structure-of-arrays, x fastest.  tclbm_step() advances it by whole
 * time steps with the fused collide-and-stream kernel: macroscopic moments (Eq. 20
 * and the temperature of Section IV), correction-term gradients (Section IV),
 * cascaded collision of f_bar (Eq. 8 with the shifted equilibria, Eq. 18, Eq. 3,
 * plus S_a and C_a), BGK collision of h_bar with its K_a coupling (Section IV),
 * pull streaming and the wall schemes of Section V.
 *
 * Conventions for every entry point:
 *   - Returns a tclbm_status; never aborts, never prints.  tclbm_last_error() gives a
 *     thread-local message for the last non-OK status of the calling thread.
 *   - Field arrays are double, [ny][nx] row-major (x fastest).  `on_device` = 1 means
 *     the pointer is device memory of the handle's device, 0 means host memory.
 *     Caller-owned arrays are read or written only during the call.
 *   - Work is queued on the handle's CUDA stream; calls that return data to the
 *     caller (moments, diagnostics, populations) synchronise that stream.  CUDA
 *     errors raised asynchronously surface at the next synchronising call as
 *     TCLBM_ECUDA.
 *   - Calls on one handle are not thread-safe; distinct handles are independent.
 */
#ifndef TCLBM_H
#define TCLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TCLBM_OK = 0,
    TCLBM_EINVAL = -1,         /* invalid argument or parameter set */
    TCLBM_ENOMEM = -2,         /* device allocation failed (allocator returned NULL) */
    TCLBM_ECUDA = -3,          /* a CUDA runtime call or kernel failed */
    TCLBM_ENONFINITE = -4,     /* a non-finite value was found in the state */
    TCLBM_ETIMEOUT = -5,       /* a bounded device wait gave up */
    TCLBM_EUNSUPPORTED = -6    /* valid request the library does not implement */
} tclbm_status;

/* Sides of the lattice, in this order in tclbm_params.wall[]. */
enum { TCLBM_SIDE_XM = 0, TCLBM_SIDE_XP = 1, TCLBM_SIDE_YM = 2, TCLBM_SIDE_YP = 3 };

/* Wall schemes of Section V.  Walls are wet: the wall lies on the first/last node row
 * (or column); after streaming that node's populations are rebuilt and it then
 * collides like any other node.  Opposite sides must both be periodic or both walls,
 * and walls may sit on one axis only. */
enum {
    TCLBM_WALL_PERIODIC = 0,
    TCLBM_WALL_ZOUHE = 1,       /* non-equilibrium bounce-back, tangential wall velocity */
    TCLBM_WALL_NEE = 2,         /* non-equilibrium extrapolation of f_bar (and h_bar) */
    TCLBM_WALL_EQUILIBRIUM = 3  /* equilibrium distributions at (rho, u, T) of the wall */
};
/* Temperature treatment of a ZOUHE or NEE wall (h_bar by non-equilibrium extrapolation). */
enum { TCLBM_THERM_FIXED_T = 0, TCLBM_THERM_ADIABATIC = 1 };
/* How w1 follows from the viscosity, Eq. 29: 1/w1 = mu/p + 1/2, p = rho R T. */
enum {
    TCLBM_VISC_NU = 0,       /* visc = kinematic nu, mu = rho nu (w1 per node) */
    TCLBM_VISC_MU = 1,       /* visc = dynamic mu */
    TCLBM_VISC_MU_PROP_T = 2,/* mu = visc * T / T0 (Section V.B) */
    TCLBM_VISC_W1 = 3        /* visc = w1, fixed */
};
/* Body force of Section III (force density F; acceleration a = F / rho). */
enum {
    TCLBM_FORCE_NONE = 0,
    TCLBM_FORCE_ACCEL = 1,       /* F = rho (ax, ay): gravity as a direct force (Section V.D) */
    TCLBM_FORCE_TAYLOR_GREEN = 2 /* F = famp (sin kx sin ky, cos kx cos ky), k = 2 pi / n (Section V.A) */
};
/* Population storage.  Every format stores the deviation of f_bar and h_bar from a rest
 * state near (rho, u, T) = (1, 0, T0) and the kernels collide on those deviations in
 * FP32; the 16-bit formats round the stored deviations to bfloat16 or half. */
enum { TCLBM_STORE_FP32 = 0, TCLBM_STORE_BF16 = 1, TCLBM_STORE_FP16 = 2 };
/* Rounding of 16-bit stores.  Near a steady state the per-step change of a population
 * falls below half an ulp and round-to-nearest freezes it; stochastic rounding (random
 * bits from a counter-based hash of node, plane and step) keeps the expected stored
 * value equal to the FP32 one. */
enum { TCLBM_ROUND_NEAREST = 0, TCLBM_ROUND_STOCHASTIC = 1 };

typedef struct {
    int32_t kind;   /* TCLBM_WALL_* */
    int32_t therm;  /* TCLBM_THERM_* (ZOUHE / NEE walls of a thermal lattice) */
    double rho;     /* wall density (EQUILIBRIUM walls) */
    double ux, uy;  /* wall velocity; ZOUHE walls move tangentially only */
    double T;       /* wall temperature */
} tclbm_wall;

typedef struct {
    int32_t nx, ny;       /* nodes; >= 1 on periodic axes, >= 3 on a walled axis */
    int32_t thermal;      /* 1: h_bar evolved, T local (Section IV); 0: athermal, T = T0 */
    int32_t correction;   /* 1: correction term C_a (Section IV); needs thermal */
    int32_t visc_law;     /* TCLBM_VISC_* */
    double visc;          /* see visc_law */
    int32_t bgk;          /* 1: w2 = w3 = w4 = w1 (the BGK limit of Section V.A) */
    double w2, w3, w4;    /* Eq. 8 rates of E, (M21, M12), M22; each in (0, 2) */
    double Pr;            /* Prandtl number (> 0) */
    double gamma;         /* specific-heat ratio (> 1); b = 2 / (gamma - 1) */
    double R, T0;         /* gas constant and reference temperature (> 0) */
    int32_t force_kind;   /* TCLBM_FORCE_* */
    double ax, ay;        /* TCLBM_FORCE_ACCEL */
    double famp;          /* TCLBM_FORCE_TAYLOR_GREEN */
    tclbm_wall wall[4];   /* indexed by TCLBM_SIDE_* */
    int32_t storage;      /* TCLBM_STORE_* */
    double T_ref;         /* reference temperature of the Nusselt sum in diagnostics */
    int32_t rounding;     /* 16-bit storage: TCLBM_ROUND_NEAREST or TCLBM_ROUND_STOCHASTIC */
    int32_t work;         /* 1: the body force's power F.u is a source of total energy (thermal only;
                             an extension, the paper's Eq. 22 has no force term): the h update
                             gains (1 - w_h/2) W_a F.u (D2Q9 weights W_a) and the energy moment
                             is rho E = sum h_bar + F.u / 2; 0: paper-literal */
} tclbm_params;

/* Device allocator hooks.  alloc(bytes, stream, ctx) returns device memory or NULL;
 * free(ptr, bytes, stream, ctx) releases it.  Both may be NULL: the library then uses
 * cudaMalloc / cudaFree. */
typedef void* (*tclbm_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*tclbm_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

typedef struct tclbm_lattice tclbm_lattice;

/* Number of doubles written by tclbm_diagnostics(). */
#define TCLBM_NDIAG 8

/* Device bytes one lattice of these parameters holds (state, tables, scratch). */
size_t tclbm_state_bytes(const tclbm_params* params);

/* Validate params, derive constants, allocate the state on the current device.
 * `stream` is a cudaStream_t (NULL = legacy default stream).  No kernel runs.
 * EINVAL on bad parameters, ENOMEM if the allocator fails; *out is NULL on error. */
tclbm_status tclbm_create(const tclbm_params* params, tclbm_alloc_fn alloc, tclbm_free_fn free_fn, void* ctx,
                          void* stream, tclbm_lattice** out);

/* Set the populations from macroscopic fields: f_bar = f^eq(rho, u, T) - S/2 (the
 * correction term is taken as zero at t = 0) and h_bar = h^eq(rho, u, T), so that
 * Eq. 20 and the temperature formula return the given fields.  Resets the step count. */
tclbm_status tclbm_init_fields(tclbm_lattice* lat, const double* rho, const double* ux, const double* uy,
                               const double* T, int32_t on_device);

/* Advance `nsteps` >= 0 time steps (asynchronous on the handle's stream).  Under kernel
 * variant 0 with the correction term (and round-to-nearest for 16-bit storage, rows per
 * CTA >= 8), the launches of one call are chained: each work item of a launch waits
 * only for the nine items around it in the previous launch, so consecutive steps
 * overlap on the device; the first launch of a call waits for whatever precedes it on
 * the stream.  The states are bit-identical to one step per call.  A chained wait that
 * expires is reported like the other bounded waits (TCLBM_ETIMEOUT at the next
 * synchronising call). */
tclbm_status tclbm_step(tclbm_lattice* lat, int64_t nsteps);

/* Macroscopic fields of the current state (Eq. 20; T per Section IV, T0 if athermal),
 * each [ny][nx]; any pointer may be NULL.  Synchronises the stream. */
tclbm_status tclbm_moments(tclbm_lattice* lat, double* rho, double* ux, double* uy, double* T, int32_t on_device);

/* FP64 global sums of the current state, reduced on the device:
 * out[0] sum rho, out[1] sum rho ux, out[2] sum rho uy, out[3] sum h_bar (total energy),
 * out[4] sum rho |u|^2 / 2 (kinetic energy, Section V.D), out[5] sum uy (T - T_ref)
 * (the Nusselt sum of Section V.D), out[6] sum |u - u_snap|^2, out[7] sum |u|^2
 * (steady-state residual of Section V.A against the last tclbm_snapshot_velocity()).
 * Synchronises the stream. */
tclbm_status tclbm_diagnostics(tclbm_lattice* lat, double out[TCLBM_NDIAG]);

/* Allocation-free form of the sums of tclbm_diagnostics() (no counterpart in the paper).
 * For callers that may not allocate device memory when they need the sums -- a serving
 * loop whose memory is planned up front, code under a fixed memory budget, embedders
 * that only pass raw device pointers.  Inputs: the lattice's parameters, and device
 * pointers f, h to FP64 populations in the layout of tclbm_get_populations() (double
 * [9][ny][nx] each; h may be NULL for athermal lattices), u_snap: NULL or a device
 * double [2][ny][nx] velocity reference for out[6] (0 when NULL).  out: 8 doubles, on
 * the device if out_on_device, else on the host (then the call synchronises `stream`).
 * Block partial sums live in a fixed 65,600-byte file-scope device array held by every
 * device that loads the library; no cudaMalloc, cudaFree or other allocating call is
 * made.  Lattices above 67,108,864 nodes are rejected with TCLBM_EINVAL.  The first call
 * on a device resolves the array's address with that device current; make it before
 * any stream capture.  All calls share the array: calls that overlap on the GPU race.
 * With host output a non-finite sum returns TCLBM_ENONFINITE, as tclbm_diagnostics()
 * does; with device output the sums are not inspected (the call does not synchronise). */
tclbm_status tclbm_diagnostics_noalloc(const tclbm_params* params, const double* f, const double* h,
                                       const double* u_snap, double* out, int32_t out_on_device, void* stream);

/* Store the current velocity field as the reference of out[6] in tclbm_diagnostics(). */
tclbm_status tclbm_snapshot_velocity(tclbm_lattice* lat);

/* Copy the populations out of / into the current state as double [9][ny][nx] each
 * (f_bar, then h_bar; h may be NULL for athermal lattices).  Synchronising. */
tclbm_status tclbm_get_populations(tclbm_lattice* lat, double* f, double* h, int32_t on_device);
tclbm_status tclbm_set_populations(tclbm_lattice* lat, const double* f, const double* h, int32_t on_device);

/* Row exchange of a slab decomposition along y (no counterpart in the paper, which
 * steps one lattice as a whole).  One lattice cut into slabs of whole rows, each slab a
 * lattice that also holds `g` rows of its neighbours, stays equal row for row to the
 * undivided lattice for g/2 steps (a node's update reads the rows next to it and the
 * correction-term gradient of Section IV reads the velocity one row further); this
 * call refreshes those rows.  It copies rows [src_row, src_row + rows) of src's
 * current state into rows [dst_row, dst_row + rows) of dst's, every population plane,
 * in the storage format as stored (a device-to-device copy; nothing is converted).
 * Both lattices need the same nx, storage format and thermal flag, and both row ranges
 * must lie inside their lattices (the same lattice is allowed with disjoint ranges);
 * EINVAL otherwise.  rows = 0 does nothing.  Asynchronous: queued on dst's stream after
 * the work already queued on src's stream, and later work on src's stream waits for the
 * copy.  The copy changes no step count. */
tclbm_status tclbm_copy_rows(tclbm_lattice* dst, int32_t dst_row, tclbm_lattice* src, int32_t src_row,
                             int32_t rows);

/* Time steps taken since the last init. */
int64_t tclbm_steps_done(const tclbm_lattice* lat);

/* Replace the handle's stream (cudaStream_t). */
tclbm_status tclbm_set_stream(tclbm_lattice* lat, void* stream);

/* Release the handle and its device memory; NULL is accepted. */
tclbm_status tclbm_destroy(tclbm_lattice* lat);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* tclbm_last_error(void);

/* Name of the step kernel variant and its launch shape for this handle, for
 * profiling ("tclbm_step_kernel<...> grid (gx, gy) block (bx)"). */
const char* tclbm_describe(const tclbm_lattice* lat);

/* Test hook for the timeout path (no counterpart in the paper): with row in [0, ny) the
 * TMA-fed kernel (variant 0, FP32 storage; other formats ignore the hook) never copies
 * that source row, so the bounded waits on it
 * expire after 1 s, the kernel records the failure and returns, and the next
 * synchronising call returns TCLBM_ETIMEOUT (the state is then invalid; re-initialise
 * it).  row = -1 turns the hook off.  EINVAL for other rows. */
tclbm_status tclbm_test_skip_row(tclbm_lattice* lat, int32_t row);

/* Test hook for the collision's reciprocal (no counterpart in the paper): y[i] = the
 * reciprocal the step kernels take of R T, mu/p + 1/2 and mu/(p Pr) + 1/2 (the hardware
 * approximation refined by one Newton step), for n floats at device pointers x, y.
 * Queued on `stream` (a cudaStream_t, NULL = legacy default), which it synchronises.
 * EINVAL on n < 0 or NULL arrays with n > 0. */
tclbm_status tclbm_test_rcp(const float* x, float* y, int64_t n, void* stream);

/* Launch-shape override for tuning; 0 keeps the library's choice.  Kernel variants 0
 * and 1: strip width tx (32, 64 or 128 nodes) and rows per CTA ty (>= 1); under variant 0,
 * where the grid spans more than two waves of resident CTAs, ty is a multiple of 16 and
 * ny a multiple of 8, about the last wave of row segments takes ty / 2 rows (and the
 * first segment the remainder), so that the launch ends on short CTAs.  Variant 2:
 * the tile (tx, ty) = (BX, BY), one of 16x4, 16x8, 32x4, 32x8, 32x16, 64x4, 64x8,
 * 128x4, subject to the variant's size rule (EINVAL otherwise). */
tclbm_status tclbm_set_tile(tclbm_lattice* lat, int32_t tx, int32_t ty);

/* Step kernel variant: 0 = rows staged into shared memory by the tensor-memory
 * accelerator, 1 = direct loads marching up strips of rows, 2 = direct loads on 2-D
 * tiles, one node per thread (thermal lattices with the correction term; on a walled x
 * axis nx % BX != 1 and on a walled y axis ny % BY != 1, else TCLBM_EUNSUPPORTED).  The
 * library picks per lattice size: 2 (or 1 where 2 does not apply) up to 2,097,152
 * nodes, 0 above.  Interior nodes evolve bit-identically under all variants; wall
 * nodes may differ in the last bit (multiply-add contraction).  Changing the variant
 * resets the launch shape to that variant's default.  EINVAL for other values. */
tclbm_status tclbm_set_kernel(tclbm_lattice* lat, int32_t kind);

/* ------------------------------------------------------------------ batches
 * A batch advances many independent lattices together: one launch of the batched step
 * kernel per time step over a work list of strips of every lattice (tx columns by
 * `rows` rows each, largest lattices first), captured in CUDA graphs for long runs.
 * The paper treats one lattice at a time; a batch changes no arithmetic: every node
 * is updated by the same code as in tclbm_step(), so each lattice evolves exactly as
 * it does alone with the direct-load kernel (tclbm_set_kernel(lat, 1)).
 *
 * The batch borrows its lattices; they must stay alive for every batch call except
 * tclbm_batch_destroy, which touches no lattice.  They must share the storage
 * format and may differ in size, parameters, walls and collision variant (athermal,
 * thermal, thermal with the correction term).  Stepping or re-initialising a lattice
 * on its own between batch calls is allowed.  Device memory for the work list comes
 * from the allocator hooks the first lattice was created with. */
typedef struct tclbm_batch tclbm_batch;

/* `stream` is a cudaStream_t (NULL = legacy default stream); batch steps are ordered
 * after work already queued on each lattice's own stream, and later work on those
 * streams after the batch steps.  EINVAL on count < 1, a NULL or repeated handle, or
 * mixed storage formats; ENOMEM if the work list cannot be allocated. */
tclbm_status tclbm_batch_create(tclbm_lattice* const* lattices, int32_t count, void* stream, tclbm_batch** out);

/* Replace the batch's lattices (count >= 0; same storage format as at creation), keeping
 * its work-list shape.  Nothing waits for the GPU: the new work list and descriptors
 * are stream-ordered copies on the batch stream, so steps already queued finish on the
 * old list.  For serving loops whose set of resident lattices changes while the GPU is
 * busy.  EINVAL on a NULL or repeated handle or another storage format. */
tclbm_status tclbm_batch_set_lattices(tclbm_batch* batch, tclbm_lattice* const* lattices, int32_t count);

/* Number of lattices in the batch (-1 for NULL). */
int32_t tclbm_batch_size(const tclbm_batch* batch);

/* Advance every lattice of the batch by `nsteps` >= 0 time steps (asynchronous). */
tclbm_status tclbm_batch_step(tclbm_batch* batch, int64_t nsteps);

/* Work-list shape: strip width tx (32, 64 or 128), rows per work item (>= 1) and
 * persistent != 0 for a grid of one wave of resident CTAs that loops over the work
 * list (else one CTA per item).  EINVAL on other values. */
tclbm_status tclbm_batch_set_tile(tclbm_batch* batch, int32_t tx, int32_t rows, int32_t persistent);

/* TMA-fed strips: thermal lattices with the correction term at least tx columns wide
 * step in strips of tx (64 or 128) columns by `rows` rows, each staged row by row into
 * shared memory by the tensor-memory accelerator (the single-lattice kernel variant 0,
 * one CTA per strip); the other lattices keep the direct-load strips.  tx = 0 turns it
 * off (the default).  Those lattices then evolve exactly as alone with kernel variant 0
 * (bit for bit on periodic lattices, as variants 0 and 1 agree there; at walls within
 * the last bit).  A bounded wait that expires sets the lattice's error word: its next
 * synchronising call returns TCLBM_ETIMEOUT.  EINVAL on other tx or rows < 1. */
tclbm_status tclbm_batch_set_tma(tclbm_batch* batch, int32_t tx, int32_t rows);
/* Current TMA-fed strip shape (tx 0 = off). */
tclbm_status tclbm_batch_tma_shape(const tclbm_batch* batch, int32_t* tx, int32_t* rows);

/* Time every shape (tx in {32, 64, 128}, rows in {1, 2, 4, ..., 64} up to the tallest
 * lattice, persistent or not), then with the fastest of those every TMA-fed shape (tx
 * in {64, 128}, rows in {8, 16, 32, 48, 64}) where the batch has lattices for it, over
 * `trial_steps` (>= 2, rounded up to even) steps each; keep the fastest combination and
 * report the direct-load shape through the non-NULL out pointers (best_us: device
 * microseconds per batch step; the TMA-fed shape through tclbm_batch_tma_shape).  The
 * lattices' state is saved before and restored after, so the call changes no results;
 * it needs device memory for one copy of every lattice's state and synchronises the
 * stream. */
tclbm_status tclbm_batch_autotune(tclbm_batch* batch, int32_t trial_steps, int32_t* best_tx, int32_t* best_rows,
                                  int32_t* best_persistent, float* best_us);

/* Kernel name and work-list shape, for profiling. */
const char* tclbm_batch_describe(const tclbm_batch* batch);

/* Batch steps taken since creation (-1 for NULL). */
int64_t tclbm_batch_steps_done(const tclbm_batch* batch);

/* Release the batch (not its lattices); NULL is accepted.  Synchronises the stream. */
tclbm_status tclbm_batch_destroy(tclbm_batch* batch);

#ifdef __cplusplus
}
#endif
#endif /* TCLBM_H */
