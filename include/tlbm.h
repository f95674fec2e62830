/*
 * tlbm: GB300 (sm_103a) thermal lattice Boltzmann step, C ABI.
 *
 * The library advances the double-distribution-function (DDF) thermal lattice
 * Boltzmann model of Xu & Li, "Multi-GPU thermal lattice Boltzmann simulations
 * using OpenACC and MPI" (IJHMT 2022):
 *   - flow populations f on D2Q9 / D3Q19 with the MRT collision of Eq. (5)
 *     and the Guo forcing term of Eq. (6a)/(6b);
 *   - temperature populations g on D2Q5 / D3Q7 with the MRT collision of Eq. (7);
 *   - Boussinesq buoyancy F = rho g beta (T - T0) along +y (2D) or +z (3D), §2.2;
 *   - macroscopic rho = sum f, u = (sum e f + F/2)/rho, T = sum g, §2.2;
 *   - half-way bounce-back (no-slip), half-way anti-bounce-back (isothermal,
 *     omega = (4 + a_T)/10 or (6 + a_T)/21) and bounce-back of g (adiabatic), §2.2;
 *   - collision and streaming, Eqs. (10)-(11), fused into one pull kernel.
 * Parameters follow the free-fall scaling of Eqs. (2)-(4): H = cell height (ny in
 * 2D, nz in 3D), dT = Th - Tc = 1, U = Ma/sqrt(3), nu = U H sqrt(Pr/Ra),
 * alpha = U H / sqrt(Pr Ra), g beta = U^2 / (H dT).
 *
 * Conventions shared by every call:
 *   - Every function returns TLBM_OK (0) or a negative TLBM_ERR_* code; the text
 *     of the last error is kept per handle (tlbm_last_error).
 *   - Kernels run asynchronously on the handle's stream.  A call that returns a
 *     host value (nusselt, energy, status, get_populations) synchronises that
 *     stream.  A device fault from an earlier asynchronous call is reported by
 *     the next synchronising call as TLBM_ERR_CUDA.
 *   - Device memory: the caller owns it.  tlbm_required_bytes() gives the size
 *     of one block that holds both population buffers plus the library's
 *     scratch; tlbm_bind_memory() hands it to the handle.  The library never
 *     allocates or frees device memory for a handle.
 *   - Arrays exchanged with the caller are dense, x fastest:
 *     node n = x + nx*(y + ny*z); population i of a set at [i*N + n], N = nx*ny*nz.
 *   - The state "after t steps" is the pre-collision population set at time t.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef TLBM_H
#define TLBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TLBM_API __attribute__((visibility("default")))
#else
#define TLBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- constants */
enum tlbm_status_code {
    TLBM_OK = 0,
    TLBM_ERR_ARG = -1,         /* invalid argument (bad size, NULL, out of range) */
    TLBM_ERR_OOM = -2,         /* bound memory too small / host allocation failed */
    TLBM_ERR_CUDA = -3,        /* a CUDA runtime call or a kernel failed */
    TLBM_ERR_DIVERGED = -4,    /* non-finite or |u| > 0.5 found in the state */
    TLBM_ERR_TIMEOUT = -5,     /* a bounded device wait gave up */
    TLBM_ERR_UNBOUND = -6,     /* device memory not bound yet */
    TLBM_ERR_UNSUPPORTED = -7  /* combination not built (e.g. unknown precision) */
};

enum tlbm_lattice { TLBM_D2Q9_D2Q5 = 0, TLBM_D3Q19_D3Q7 = 1 };

/* Storage precision of the populations.  FP32, FP16 and BF16 storage keep
 * the flow deviations f_i - w_i and g_i (temperature, T0 = 0), FP16/BF16
 * ("offset" storage) scaled by a power of two; collision then runs in FP32.
 * FP64 storage keeps f_i and g_i and collides in FP64. */
enum tlbm_prec { TLBM_FP64 = 0, TLBM_FP32 = 1, TLBM_FP16_OFFSET = 2, TLBM_BF16_OFFSET = 3 };

/* Wall configuration.  RB: hot bottom (Th), cold top (Tc), adiabatic sides.
 * SIDE_HEATED (§2.3): hot left wall (x = -1/2), cold right wall, others adiabatic.
 * Every non-periodic face is a no-slip wall. */
enum tlbm_walls { TLBM_RB = 0, TLBM_SIDE_HEATED = 1 };

/* Output element type for tlbm_macros. */
enum tlbm_dtype { TLBM_OUT_F64 = 0, TLBM_OUT_F32 = 1 };

/* Streaming scheme (the same method, two memory layouts).  PULL: two population
 * buffers, each step reads one and writes the other.  INPLACE: one buffer,
 * steps alternate between a half that reads and writes every node's own slots
 * (storing each post-collision value in the slot of the opposite direction) and
 * a half that reads from the neighbours and writes to them (the "AA" access
 * pattern); the same bytes per lattice update, half the device memory.  The
 * in-place scheme runs on the register kernels only (tlbm_set_staged and
 * multi-row variants return TLBM_ERR_UNSUPPORTED) and not in batches. */
enum tlbm_streaming { TLBM_STREAM_PULL = 0, TLBM_STREAM_INPLACE = 1 };

/* Optional parameters.  Initialise with tlbm_default_params(); every double left
 * as NaN is derived from (Ra, Pr, Ma) as stated at the top of this file:
 *   s_nu = 1/(3 nu + 1/2) on all even non-conserved flow moments (s_e, s_eps, s_pi),
 *   s_q = s_m = 8(2 - s_nu)/(8 - s_nu) on all odd non-conserved ones,
 *   s_rho = s_j = 1 (they do not change the result),
 *   a_T = -2/3 (D2Q5) or -3/4 (D3Q7), q_j from alpha = omega (1/q_j - 1/2),
 *   q_e = q_v from (1/q_j - 1/2)(1/q_e - 1/2) = 1/4.
 * periodic_mask (bit0 x, bit1 y, bit2 z) and body_force (a constant
 * acceleration; force density rho*a) exist for validation cases. */
typedef struct {
    int walls;
    int periodic_mask;
    int u_is_ma;            /* 1: U = Ma instead of Ma/sqrt(3) */
    double a_T;
    double nu, alpha, gbeta;
    double s_rho, s_e, s_eps, s_j, s_q, s_pi, s_m;
    double q_e, q_v;
    double body_force[3];
    double Th, Tc;
    double store_scale;     /* FP16/BF16 storage scale (power of two); NaN = default */
    int streaming;          /* TLBM_STREAM_PULL (0, default) or TLBM_STREAM_INPLACE */
} tlbm_params;

typedef struct tlbm_s* tlbm_t;

/* One instance of a batched ensemble (same lattice and precision for all). */
typedef struct {
    int nx, ny, nz;
    double Ra, Pr, Ma;
    uint64_t seed;
} tlbm_instance;

/* ---------------------------------------------------------------- lifecycle */

/* Fill *p with the defaults described above (all derivable doubles NaN). */
TLBM_API void tlbm_default_params(tlbm_params* p);

/* Create a handle for an nx x ny (x nz) cell.  nz is ignored (1) for D2Q9_D2Q5.
 * Errors: TLBM_ERR_ARG for nx, ny < 3, nz < 3 in 3D, Ra/Pr/Ma <= 0, an unknown
 * lattice/precision/walls value, or tau - 1/2 = 3 nu <= 1e-6.  *out is set to
 * NULL on error.  The handle owns host memory only. */
TLBM_API int tlbm_create(tlbm_t* out, int nx, int ny, int nz, int lattice, double Ra, double Pr,
                double Ma, int precision, const tlbm_params* p);

/* Bytes of device memory the handle needs (both population buffers and
 * scratch), 256-byte aligned. */
TLBM_API int tlbm_required_bytes(tlbm_t h, size_t* bytes);

/* Bind a caller-owned device block of at least tlbm_required_bytes() bytes,
 * 256-byte aligned.  The library never frees it; it must outlive the handle's
 * use.  Re-binding moves nothing: call tlbm_init or tlbm_set_populations after.
 * The block starts with two population buffers of B bytes each, then scratch:
 *   P = 32 * ceil((nx + 16) / 32),  R = (ny + 2) * (nz + 2) in 3D, ny + 2 in 2D,
 *   plane = 64 * ceil((128 + R * P) / 64) elements,
 *   B = 256 * ceil((qf + qg) * plane * element_bytes / 256),
 * with (qf, qg) = (9, 5) or (19, 7) and element_bytes 8, 4, 2, 2 for FP64, FP32,
 * FP16, BF16.  The current state is buffer 0 after tlbm_init or
 * tlbm_set_populations and after every even number of steps since; buffer 1
 * after an odd number. */
TLBM_API int tlbm_bind_memory(tlbm_t h, void* dev_ptr, size_t bytes);

/* Stream for all later work (a cudaStream_t; NULL = legacy default stream). */
TLBM_API int tlbm_set_stream(tlbm_t h, void* cuda_stream);

/* Initial state (t = 0): f = f_eq(rho = 1, u = 0) and g = g_eq(T, 0) with the
 * conductive profile between the isothermal walls plus noise_amp*(2r - 1),
 * r = (splitmix64(seed ^ splitmix64(n)) >> 11) * 2^-53 for node n. */
TLBM_API int tlbm_init(tlbm_t h, uint64_t seed, double noise_amp);

/* Initial state (t = 0) from given device FP32 fields of nx*ny*nz values (x
 * fastest): f = f_eq(rho = 1, u), g = g_eq(T, u) (a warm start).  T is
 * required; a NULL velocity component is 0.  Asynchronous. */
TLBM_API int tlbm_init_fields(tlbm_t h, const float* T, const float* ux, const float* uy, const float* uz);

/* Advance n >= 0 time steps (Eqs. (10)-(11), fused).  Asynchronous.  Whole
 * blocks of graph_steps steps (tlbm_set_graph, default 16) are replayed from a
 * CUDA graph captured at the first such block; the rest are plain launches. */
TLBM_API int tlbm_step(tlbm_t h, int64_t n);

/* Steps per CUDA graph replay in tlbm_step (even, <= 4096; 0 = plain launches
 * only).  The graph is captured on a private stream the first time it is needed
 * and dropped when the variant, the staged setting or the bound memory change. */
TLBM_API int tlbm_set_graph(tlbm_t h, int steps);

/* Macroscopic fields of the current state into caller device arrays of
 * nx*ny*nz elements (x fastest), element type out_dtype.  NULL skips a field;
 * uz is ignored in 2D.  Asynchronous. */
TLBM_API int tlbm_macros(tlbm_t h, void* rho, void* ux, void* uy, void* uz, void* T, int out_dtype);

/* Nusselt number of the current state, FP64 deterministic reduction:
 * Nu = 1 + L <u_h T> / (alpha dT), u_h the velocity component along the
 * heat-flux axis (vertical for RB, x for side-heated) and L the cell extent
 * along it.  Synchronises the stream.  TLBM_ERR_DIVERGED (the value still
 * written) if the same reduction finds a non-finite value or |u| > 0.5. */
TLBM_API int tlbm_nusselt(tlbm_t h, double* nu);

/* Kinetic energy sum 1/2 rho |u|^2 and mass sum rho, FP64.  Synchronises.
 * TLBM_ERR_DIVERGED (the values still written) as for tlbm_nusselt. */
TLBM_API int tlbm_energy(tlbm_t h, double* ekin, double* mass);

/* Copy the canonical pre-collision populations (FP64, dense layout above) to
 * host arrays f[qf*N], g[qg*N] (either may be NULL).  Synchronises. */
TLBM_API int tlbm_get_populations(tlbm_t h, double* host_f, double* host_g);

/* Same for the box [x0, x0+wx) x [y0, y0+wy) x [z0, z0+wz) of the cell (z0 = 0,
 * wz = 1 in 2D); the host arrays hold qf (qg) planes of wx*wy*wz values, x
 * fastest.  TLBM_ERR_ARG if the box leaves the cell.  Synchronises. */
TLBM_API int tlbm_get_populations_window(tlbm_t h, int x0, int y0, int z0, int wx, int wy, int wz,
                                         double* host_f, double* host_g);

/* Replace the state by host FP64 populations in the same layout (rounded to the
 * storage precision).  Both pointers are required.  Synchronises. */
TLBM_API int tlbm_set_populations(tlbm_t h, const double* host_f, const double* host_g);

/* Checkpoint the state to the file `path` (host I/O; synchronises): a header
 * (magic "TLBMCKP1", format version 1, byte-order mark, lattice, nx, ny, nz,
 * storage precision, walls, periodic axes, Ra, Pr, Ma, Th, Tc, storage scale,
 * body force, the derived parameters of tlbm_derived, the step counter, the
 * node count) followed by the pre-collision populations in FP64 in the layout
 * of tlbm_get_populations (flow planes, then thermal planes, each nx*ny*nz
 * values, x fastest), native byte order; with FP32, FP16 or BF16 storage the
 * flow planes hold the deviations f_i - w_i (a header flag says so), the exact
 * FP64 image of what the storage holds.  Written in chunks through the scratch
 * of the bound block (no full host copy).  TLBM_ERR_ARG if path is NULL or
 * cannot be written. */
TLBM_API int tlbm_save(tlbm_t h, const char* path);
/* Restore a file written by tlbm_save into a handle created with the same
 * lattice, size, storage precision and physical parameters (TLBM_ERR_ARG
 * otherwise, and for a file that is not a checkpoint or is shorter or longer
 * than its header says); the step counter is restored too.  The file holds
 * every stored value exactly, so stepping on after tlbm_load gives bitwise the
 * states of the uninterrupted run.  The streaming scheme of the handle may
 * differ from the saving one's.  Synchronises. */
TLBM_API int tlbm_load(tlbm_t h, const char* path);

/* *diverged = 1 if the state holds a non-finite value or |u| > 0.5; *step =
 * current time step.  Runs a reduction; synchronises.  Either output may be
 * NULL.  Reports divergence through *diverged, returning TLBM_OK. */
TLBM_API int tlbm_status(tlbm_t h, int* diverged, int64_t* step);

/* Derived parameters: out[0..6] = U, H, nu, alpha, gbeta, a_T, omega, then the
 * flow rates S[qf] and thermal rates Q[qg].  Returns the count written (<= cap)
 * through *count. */
TLBM_API int tlbm_derived(tlbm_t h, double* out, int cap, int* count);

/* Choose the step kernel variant: vec = nodes per thread (0 = default),
 * rows = consecutive rows per thread (0 or 1: one; 2 or 4: software-pipelined,
 * the next row's loads are issued before the current row is collided; those
 * variants exist for the two-relaxation-time form),
 * form = 0 automatic (two-relaxation-time evaluation when the rates allow it,
 * else the general MRT), 1 general MRT, 2 two-relaxation-time (TLBM_ERR_ARG if
 * the rates are not of that form); block_x (multiple of 32) x block_y threads
 * per block (0 = the tuned default of the lattice and precision).  All variants compute the same collision;
 * TLBM_ERR_UNSUPPORTED if the variant is not compiled. */
TLBM_API int tlbm_set_variant(tlbm_t h, int vec, int form, int block_x, int block_y, int rows);
/* Use the shared-memory staged step kernel instead: a persistent grid whose
 * blocks move each tile (one row segment of tile_width nodes) with TMA bulk
 * copies: one warp copies the tile's source row of every population into
 * shared memory (completing on mbarriers), 4 or 8 warps (2D) or 4 or 7 warps
 * (3D) collide two nodes per thread and store them straight to global memory;
 * `stages` tiles are in flight per block.  Handles with FP16/BF16 storage and
 * two-relaxation-time rates start on this kernel (whole rows; stages automatic
 * in 2D, 2 in 3D) unless tlbm_set_variant was called.
 * tile_width: a multiple of 16 bytes' worth of elements, at most 512 in 2D and
 * 448 in 3D (0 = whole rows up to that width, else that width); stages: 2 .. 8 (0 = the most tiles in
 * flight per SM, blocks x stages, up to six, more blocks first).  FP32/FP16/BF16 storage with two-relaxation-time rates
 * only (TLBM_ERR_UNSUPPORTED otherwise).  A block that waits too long for its
 * copies gives up; the next synchronising call then returns TLBM_ERR_TIMEOUT.
 * tlbm_set_variant switches back to the register kernels. */
TLBM_API int tlbm_set_staged(tlbm_t h, int tile_width, int stages);
/* How long a block of the staged kernel waits for a copy (or a free stage)
 * before it gives up (default 0.2 s; 0 gives up at the first wait that has not
 * completed when first tested, which makes the timeout path testable).  seconds in [0, 10], else
 * TLBM_ERR_ARG.  A block that gives up first waits (at most 10 ms) for the
 * copies it has in flight; the next synchronising call returns
 * TLBM_ERR_TIMEOUT, and keeps doing so until tlbm_init, tlbm_init_fields or
 * tlbm_set_populations replaces the state. */
TLBM_API int tlbm_set_wait_limit(tlbm_t h, double seconds);
/* Accesses that left the population buffers, counted by a library built with
 * TLBM_DEBUG_BOUNDS (libtlbm_debug.so): there every global load and store of
 * the step, in-place, staged, batch, transfer, initial-state and reduction
 * kernels is checked against the handle's population buffers; an access
 * outside them is counted and redirected into them (never trapped).  The count
 * covers everything since tlbm_bind_memory.  Synchronises.  The release
 * library returns TLBM_ERR_UNSUPPORTED. */
TLBM_API int tlbm_bounds_violations(tlbm_t h, int64_t* count);
/* The staged kernel's configuration as chosen (all 0 when the register kernels
 * are in use): tile width in nodes, stages per block, and the persistent grid
 * (blocks per SM x SMs).  Outputs may be NULL. */
TLBM_API int tlbm_get_staged(tlbm_t h, int* tile_width, int* stages, int* blocks);
/* Current variant (form reported as 1 MRT or 2 TRT; vec 0 for the staged
 * kernel).  Outputs may be NULL. */
TLBM_API int tlbm_get_variant(tlbm_t h, int* vec, int* form, int* block_x, int* block_y, int* rows);

/* ---------------------------------------------------------------- batched ensemble
 * n independent cells with their own sizes, (Ra, Pr, Ma) and seeds, one lattice
 * and precision.  One flattened launch advances every instance by one step;
 * blocks of graph_steps steps are replayed as one CUDA graph launch.  Each
 * instance is an ordinary handle bound to its own slice of the batch's block
 * (tlbm_batch_instance), so the single-cell calls (macros, populations,
 * reductions) apply to it; it must not be destroyed, re-bound or stepped on its
 * own.  Errors as for the single-cell calls, text in tlbm_batch_last_error. */
typedef struct tlbm_batch_s* tlbm_batch_t;

/* Create (host memory only).  p applies to every instance (NULL = defaults). */
TLBM_API int tlbm_batch_create(tlbm_batch_t* out, int n, const tlbm_instance* instances, int lattice,
                               int precision, const tlbm_params* p);
/* Device bytes for all instances plus the launch tables, 256-byte aligned. */
TLBM_API int tlbm_batch_required_bytes(tlbm_batch_t b, size_t* bytes);
/* Bind a caller-owned, 256-byte aligned device block (never freed by the library). */
TLBM_API int tlbm_batch_bind_memory(tlbm_batch_t b, void* dev_ptr, size_t bytes);
TLBM_API int tlbm_batch_set_stream(tlbm_batch_t b, void* cuda_stream);
/* tlbm_init of every instance with its own tlbm_instance.seed. */
TLBM_API int tlbm_batch_init(tlbm_batch_t b, double noise_amp);
/* Advance every instance by n steps.  Asynchronous. */
TLBM_API int tlbm_batch_step(tlbm_batch_t b, int64_t n);
/* Launch shape of the batched kernel (0 keeps the current value; form as in
 * tlbm_set_variant) and the steps per graph launch (even; 0 = no graph). */
TLBM_API int tlbm_batch_set_variant(tlbm_batch_t b, int vec, int form, int block_x, int block_y,
                                    int graph_steps);
/* Persistent form: steps_per_launch > 0 makes tlbm_batch_step run up to that
 * many steps per launch of one cooperative kernel whose blocks (as many as fit
 * on the device at once) work through the tiles of every instance in a fixed
 * order and meet at a grid barrier between steps; 0 returns to one flattened
 * launch per step (graph-captured).  The barrier's waits are bounded: a block
 * that waits too long gives up, and tlbm_batch_status then returns
 * TLBM_ERR_TIMEOUT.  TLBM_ERR_UNSUPPORTED without cooperative launch. */
TLBM_API int tlbm_batch_set_persistent(tlbm_batch_t b, int steps_per_launch);
/* How long a block of the persistent kernel waits at the grid barrier, and a
 * block of the staged form for its copies or a free stage, before it gives up
 * (default 0.5 s; 0 gives up at once unless the barrier is already open or the
 * copies have landed, which makes the timeout path testable).  seconds in
 * [0, 10], else TLBM_ERR_ARG.  The timeout stays reported by tlbm_batch_status
 * until tlbm_batch_init. */
TLBM_API int tlbm_batch_set_wait_limit(tlbm_batch_t b, double seconds);
TLBM_API int tlbm_batch_get_variant(tlbm_batch_t b, int* vec, int* form, int* block_x, int* block_y,
                                    int* graph_steps);
/* Rows per thread of the flattened launch: 1, or 2 (the software-pipelined
 * body: the next row's loads are issued before the current row is collided;
 * two-relaxation-time rates, TLBM_ERR_UNSUPPORTED where not compiled).  The
 * persistent form always runs one row per thread.  tlbm_batch_set_variant
 * falls back to 1 for a vector width without the 2-row variant;
 * tlbm_batch_autotune tries both. */
TLBM_API int tlbm_batch_set_rows(tlbm_batch_t b, int rows);
TLBM_API int tlbm_batch_get_rows(tlbm_batch_t b, int* rows);
/* Shared-memory staged form of the flattened launch (the single-cell staged
 * kernel's pipeline, tlbm_set_staged, over the tiles of every instance):
 * consumer_warps 4 or 8 in 2D, 4 or 7 in 3D, 0 turns it off; a tile is a
 * stretch of 64 x consumer_warps elements of one z-plane's interior rows of an
 * instance, which lie contiguously at the row pitch (tiles run over row ends;
 * the lanes on padding and ghost columns idle); stages 0 chooses the tiles in
 * flight per block, else 2 .. 8.  FP32,
 * FP16 or BF16 storage with two-relaxation-time rates in every instance
 * (TLBM_ERR_UNSUPPORTED otherwise, and for the persistent form).
 * tlbm_batch_set_variant turns it off; tlbm_batch_autotune times it against
 * the register-kernel shapes.  A block that waits longer than the wait limit
 * for its copies gives up; tlbm_batch_status then returns TLBM_ERR_TIMEOUT. */
TLBM_API int tlbm_batch_set_staged(tlbm_batch_t b, int consumer_warps, int stages);
/* The staged form's consumer warps (0: off), stages and tiles per step. */
TLBM_API int tlbm_batch_get_staged(tlbm_batch_t b, int* consumer_warps, int* stages, long long* tiles);
/* Time the compiled launch shapes (nodes per thread x rows per thread x block
 * shape, then tiles per block, then the staged form where it applies: 4 or the
 * most consumer warps x 2 to 4 stages; trials launches each) on the bound
 * state and keep the fastest.  The state is not changed. */
TLBM_API int tlbm_batch_autotune(tlbm_batch_t b, int trials);
/* (trials < 0: reuse the shape this process tuned for the same lattice, storage,
 * collision form and size class floor(log2(total nodes)), if any.) */
/* Borrow instance idx as a single-cell handle (owned by the batch). */
TLBM_API int tlbm_batch_instance(tlbm_batch_t b, int idx, tlbm_t* out);
/* Per-instance Nusselt numbers / divergence flags into nu[n] / diverged[n].
 * tlbm_batch_nusselt writes every value and returns TLBM_ERR_DIVERGED if any
 * instance has diverged (tlbm_batch_status says which). */
TLBM_API int tlbm_batch_nusselt(tlbm_batch_t b, double* nu);
TLBM_API int tlbm_batch_status(tlbm_batch_t b, int* diverged);
/* tlbm_macros of instance idx. */
TLBM_API int tlbm_batch_macros(tlbm_batch_t b, int idx, void* rho, void* ux, void* uy, void* uz, void* T,
                               int out_dtype);
TLBM_API int tlbm_batch_launch_count(tlbm_batch_t b, int64_t* count);
TLBM_API const char* tlbm_batch_last_error(tlbm_batch_t b);
TLBM_API void tlbm_batch_destroy(tlbm_batch_t b);

/* ---------------------------------------------------------------- learned warm start
 * Layers of a small convolutional surrogate that predicts a statistically
 * steady T/u/v field from (Ra, Pr) to start the solver from (no counterpart in
 * the paper).  3x3 convolutions, stride 1, zero padding 1, NCHW, at most 32
 * channels; BF16 operands on the 5th-generation tensor cores (tcgen05.mma),
 * FP32 accumulation in tensor memory.  All pointers
 * are device pointers owned by the caller; every call is asynchronous on
 * `stream` (a cudaStream_t, NULL = legacy stream) and returns TLBM_ERR_ARG for
 * bad shapes or NULL pointers. */

/* Elements (BF16) of the packed weight operand of a layer with cin input
 * channels: 4608 * ceil(cin / 16); 0 for cin outside 1..32. */
TLBM_API int tlbm_conv3x3_weight_elems(int cin);
/* FP32 weights w[cout][cin][3][3] -> the BF16 tensor-core operand a of
 * tlbm_conv3x3_weight_elems(cin) elements, in the tile order the forward
 * kernel stages in shared memory: for tap t = 3 di + dj and 16-channel chunk
 * h (CH = ceil(cin / 16) chunks), element
 *   512 (t CH + h) + 256 (c' / 8) + 64 (m / 8) + 8 (m % 8) + c' % 8
 * holds w[m][16 h + c'][di][dj], zero for m >= cout or 16 h + c' >= cin. */
TLBM_API int tlbm_conv3x3_pack_weights(const float* w, int cout, int cin, void* a, void* stream);
/* y[B][cout][H][W] (FP32) = bias + conv(x, w); x BF16 [B][cin][H][W]; a from
 * tlbm_conv3x3_pack_weights; bias FP32 [cout] or NULL; y_act (BF16, optional)
 * = relu(y) when relu != 0, else y.  Runs as a tcgen05 implicit GEMM (128
 * pixels x 32 channels per CTA, FP32 accumulator in tensor memory); a CTA whose
 * MMAs do not complete within 0.5 s writes nothing and counts itself in
 * tlbm_conv3x3_status. */
TLBM_API int tlbm_conv3x3_forward(const void* x, const void* a, const float* bias, float* y, void* y_act, int B,
                                  int cin, int cout, int H, int W, int relu, void* stream);
/* dx[B][cin][H][W] (FP32) = gradient w.r.t. the input of the convolution with
 * BF16 weights w_bf16[cout][cin][3][3], given dy (BF16 [B][cout][H][W]): the
 * same tensor-core kernel as the forward with the flipped, transposed weights
 * (written to at_workspace, BF16 scratch of 32 * 288 elements). */
TLBM_API int tlbm_conv3x3_backward_data(const void* dy, const void* w_bf16, float* dx, int B, int cin, int cout,
                                        int H, int W, void* at_workspace, void* stream);
/* Number of convolution CTAs (forward, data or weight gradient) since load that
 * gave up waiting for their tensor-core MMAs (0 in a healthy run); synchronous. */
TLBM_API int tlbm_conv3x3_status(unsigned long long* timeouts);
/* Bytes of workspace tlbm_conv3x3_backward_weight needs for this shape on the
 * current device (one FP32 partial of 32 x 288 per CTA of the persistent
 * weight-gradient kernel, whose count follows the device's SM count). */
TLBM_API int tlbm_conv3x3_workspace_bytes(int B, int cin, int cout, int H, int W, size_t* bytes);
/* dw[cout][cin][3][3] (FP32) = sum over pixels of dy * patches(x), summed in a
 * fixed order (tcgen05 GEMMs per CTA, the CTAs' partials added in CTA order:
 * the same bits on every call on a given device); db[cout] = sum of dy (FP32 dy,
 * optional; two fixed-order levels).  x, dy_bf16: BF16.  A CTA whose MMAs do
 * not complete within 0.5 s writes NaN partials and counts itself in
 * tlbm_conv3x3_status. */
TLBM_API int tlbm_conv3x3_backward_weight(const void* x, const void* dy_bf16, const float* dy, float* dw, float* db,
                                          int B, int cin, int cout, int H, int W, void* workspace,
                                          size_t workspace_bytes, void* stream);
/* g = dx where y > 0 else 0, as FP32 and BF16 (n elements). */
TLBM_API int tlbm_relu_backward(const float* dx, const float* y, long long n, float* g, void* g_bf16, void* stream);
/* BF16 copy of an FP32 array. */
TLBM_API int tlbm_to_bf16(const float* a, long long n, void* b, void* stream);
/* Mean squared error of y against target (n elements): *loss_dev (FP64) and
 * its gradient 2 (y - target) / n as FP32 and BF16; partial_dev holds 1024
 * FP64 block sums (deterministic order). */
TLBM_API int tlbm_mse_loss(const float* y, const float* target, long long n, float* g, void* g_bf16,
                           double* loss_dev, double* partial_dev, void* stream);
/* One Adam step (Kingma & Ba 2015) on FP32 weights w with moments m, v; t >= 1. */
TLBM_API int tlbm_adam_step(float* w, const float* g, float* m, float* v, long long n, float lr, float b1,
                            float b2, float eps, int t, void* stream);
/* Vertex-aligned bilinear upsampling of `channels` planes of h x w to
 * ((h-1) factor + 1) x ((w-1) factor + 1); coarse node (i, j) lands on fine node
 * (factor i, factor j). */
TLBM_API int tlbm_upsample_bilinear(const float* in, int channels, int h, int w, int factor, float* out,
                                    void* stream);

/* FP64 diagnostic sums of a population state without any device memory from
 * the caller beyond the state itself (the paper has no counterpart; this is a
 * library service).  For callers that hold a state but cannot allocate device
 * memory: e.g. a monitoring process that maps a running simulation's state
 * through CUDA IPC on a GPU whose memory that simulation has taken, or an
 * application whose device memory is all held by its own pool allocator, so
 * that the scratch block of tlbm_bind_memory cannot be had.
 *   h:     handle describing the cell, precision, streaming scheme and
 *          parameters; it needs bound memory only when state is NULL.
 *   state: device pointer to a population buffer laid out as described at
 *          tlbm_bind_memory for a handle created with the same arguments, or
 *          NULL for h's current state.  It is read in the storage order of h's
 *          own current state: the pull layout for two-buffer handles; for
 *          in-place handles (TLBM_STREAM_INPLACE) the natural order when h has
 *          taken an even number of steps (a fresh handle included) and the
 *          swapped order after an odd number.  A state in the other order gives
 *          wrong sums without an error.
 *   out:   host array of 6 doubles: sum u_h T, sum 1/2 rho |u|^2, sum rho,
 *          max |u|^2, non-finite flag (1.0 if any), sum T; u_h as in tlbm_nusselt.
 * The block partial sums live in a static device array compiled into the
 * library (8192 slots, 384 KiB per device that loads the library, kept until
 * the process exits), so the call allocates nothing; cells of more than
 * 8192 * 16384 = 134,217,728 nodes are rejected with TLBM_ERR_ARG.  The first
 * call on a device looks up that array's device address, so make it before any
 * stream capture.  Every call shares the array: calls that overlap on the GPU
 * (other streams, handles or threads) race.  Runs on h's stream and
 * synchronises it. */
TLBM_API int tlbm_reduce_noalloc(tlbm_t h, const void* state, double* out);

/* Measured FP64 arithmetic roof of the current device (the paper has no
 * counterpart; it is the roofline of the FP64 storage path, which the FP64
 * pipes bind before HBM does on GB300): FLOP/s of independent FP64 fused
 * multiply-adds (2 FLOP each) over every SM, best of a few launches of about
 * 20 ms timed with CUDA events on `stream` (a cudaStream_t; NULL = legacy
 * stream), which it synchronises.  Allocates nothing.  TLBM_ERR_ARG if
 * flops_per_second is NULL, TLBM_ERR_CUDA on a CUDA error. */
TLBM_API int tlbm_fp64_fma_rate(void* stream, double* flops_per_second);

/* Text of the last error on this handle ("" if none); valid until the next call
 * on the handle.  A NULL handle returns the last error of a failed tlbm_create
 * in this thread. */
TLBM_API const char* tlbm_last_error(tlbm_t h);

/* Number of kernels this handle has launched so far (for accounting). */
TLBM_API int tlbm_launch_count(tlbm_t h, int64_t* count);

TLBM_API void tlbm_destroy(tlbm_t h);

#ifdef __cplusplus
}
#endif
#endif /* TLBM_H */
