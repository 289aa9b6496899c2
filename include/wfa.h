/*
 * wfa.h — C ABI of the GB300 explicit finite-volume field-equation library.
 *
 * The library advances a scalar field T on a 3D structured grid with the
 * explicit (forward-time) finite-volume update of arXiv 2209.13768, Sec. 1.1.1
 * (Eq. expl_form), written in conservative face-flux form so that it also
 * covers per-cell conductivity (harmonic-mean face conductivity) and
 * first-order upwind advection with a constant velocity:
 *
 *   T'_C = T_C + dt * [ sum_f K_f (T_D - T_C) / h_a^2  +  sum_a (F_a- - F_a+) / h_a ]
 *   K_f  = 2 k_C k_D / (k_C + k_D)                  (interior face)
 *   F    = max(u_a,0) T_lower + min(u_a,0) T_upper   (upwind face flux)
 *
 * With uniform k, no advection and the boundary cells held at a constant this
 * is exactly the paper's T' = w sum_{D in N(C)} T_D + (1 - 6w) T_C,
 * w = alpha dt / dl^2. Heat capacity is 1, so alpha = k.
 *
 * Conventions for every entry point:
 *   - returns WFA_OK (0) or a negative wfa_status; nothing is thrown across
 *     the ABI; wfa_last_error() gives a message for the calling thread;
 *   - host buffers belong to the caller and are copied before the call
 *     returns (reads) or filled before it returns (writes);
 *   - device memory belongs to the grid handle and is freed by
 *     wfa_destroy_grid;
 *   - work is queued on the CUDA stream given at creation; calls that hand
 *     data back to the host synchronise that stream;
 *   - a handle is not thread-safe; distinct handles on distinct streams are.
 *
 * Host arrays are dense, x fastest: element (x, y, z) is at x + nx*(y + ny*z).
 */
#ifndef WFA_H
#define WFA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wfa_grid_s* wfa_grid;

enum wfa_status {
    WFA_OK = 0,
    WFA_ERR_ARG = -1,      /* bad argument (null pointer, size, enum value)          */
    WFA_ERR_OOM = -2,      /* device or pinned-host allocation failed                */
    WFA_ERR_BC = -3,       /* inconsistent boundary conditions                       */
    WFA_ERR_UNSTABLE = -4, /* dt above the stability (positivity) limit              */
    WFA_ERR_CUDA = -5,     /* a CUDA call failed; the message names it               */
    WFA_ERR_TIMEOUT = -6,  /* a device-side wait gave up after its iteration limit   */
    WFA_ERR_STATE = -7,    /* call out of order (e.g. step before field / dt is set) */
    WFA_ERR_BUDGET = -8    /* request larger than the server's memory budget         */
};

enum wfa_storage { WFA_F32 = 0, WFA_BF16 = 1 };

enum wfa_bc_kind {
    WFA_BC_DIRICHLET = 0,      /* value on the boundary face, half a cell from the centre */
    WFA_BC_ZEROFLUX = 1,       /* no diffusive and no advective flux through the face     */
    WFA_BC_PERIODIC = 2,       /* must be set on both faces of an axis                    */
    WFA_BC_DIRICHLET_CELL = 3, /* outer cell layer held at the value (Eq. expl_form, C in bc) */
    WFA_BC_EXCHANGE = 4        /* z faces only: the face between two slabs of one grid split
                                  along z; the neighbour slab's cells are copied into the halo
                                  plane beyond the face before every step (wfa_exchange) */
};

enum wfa_face { WFA_XLO = 0, WFA_XHI = 1, WFA_YLO = 2, WFA_YHI = 3, WFA_ZLO = 4, WFA_ZHI = 5 };

/* ---------------------------------------------------------------- grids -- */

/* Create a grid of nx*ny*nz cells of size hx*hy*hz (Sec. 1.1, control volumes;
 * Sec. 2.1, uniform Cartesian grid). storage: WFA_F32 or WFA_BF16 (field stored
 * in bf16, arithmetic in fp32, rounded to nearest-even after every step).
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 * Each edge must be >= 2, the cell count <= 2^40, and 16 (a + 16)(b + 16) <
 * 2^32 for every pair of edges a, b (a face with its halo layers is indexed in
 * 32 bits). Boundary faces start as
 * zero-flux; the field starts at 0. Errors: WFA_ERR_ARG, WFA_ERR_OOM, WFA_ERR_CUDA. */
int wfa_create_grid(int nx, int ny, int nz, double hx, double hy, double hz, int storage,
                    void* cuda_stream, wfa_grid* out);

/* Free the handle and its device memory (synchronises its stream). NULL is a
 * no-op. The handle is this library's counterpart of a WSE_Array (Sec. 2.1,
 * Example Code): the field and its coefficients resident on the device for
 * the whole solve, released here. */
int wfa_destroy_grid(wfa_grid g);

/* Copy a dense host field (nx*ny*nz floats) in (Sec. 2.1: T_init -> WSE_Array).
 * bf16 grids round each value to nearest-even. Held boundary layers
 * (WFA_BC_DIRICHLET_CELL) are overwritten with their value at the next step. */
int wfa_set_field(wfa_grid g, const float* host_dense);

/* Conductivity and velocity (Eq. diff_eq with alpha = k; constant advection).
 * k_host: nx*ny*nz floats, >= 0 and finite, or NULL to use k_uniform (>= 0).
 * u: constant velocity in length units per time unit.
 * Errors: WFA_ERR_ARG for a negative or non-finite value. */
int wfa_set_coeffs(wfa_grid g, const float* k_host, double k_uniform, double ux, double uy,
                   double uz);

/* Boundary condition of one face (enum wfa_face; Sec. 1.1.1, Eq. expl_form
 * holds the boundary cells at a constant: WFA_BC_DIRICHLET_CELL; the face
 * Dirichlet, zero-flux, periodic and exchange kinds have no counterpart in
 * the paper). value: the face value for
 * WFA_BC_DIRICHLET, the held cell value for WFA_BC_DIRICHLET_CELL (which needs
 * an edge >= 3 on that axis), ignored otherwise. A periodic face whose
 * opposite face is not periodic makes the next wfa_step fail with WFA_ERR_BC. */
int wfa_set_bc(wfa_grid g, int face, int kind, double value);

/* Largest stable time step, computed on the device in fp64:
 * dt_max = 1 / max_C D_C over the cells that are not held, where D_C sums the
 * face conductances / h^2 (2 k_C / h^2 on a Dirichlet face, 0 on a zero-flux
 * face) and |u_a| / h_a for each outflow face that carries flux; every weight
 * of the update is then >= 0 (Sec. 1.1.1: stable for omega < 1/6).
 * Writes +inf when nothing couples. Synchronises the stream. Needs the
 * coefficients (WFA_ERR_STATE otherwise). */
int wfa_stability_dt(wfa_grid g, double* dt_max);

/* Set the time step (Sec. 1.1.1: omega = alpha dt / dl^2 in Eq. expl_form).
 * dt must be > 0 and <= dt_max (WFA_ERR_UNSTABLE otherwise). */
int wfa_set_dt(wfa_grid g, double dt);

/* Force a kernel configuration instead of the tuned one (no counterpart in
 * the paper, whose step is one fused program per tile, Sec. 2.1).
 * depth: time steps fused per pass over the grid (1..8; 0 = automatic).
 * variant: 0 = automatic; 1..2 = one of the compiled tile shapes of the
 * tiled TMA kernel (depth steps per pass); 3 = the column-march kernel (one
 * step per pass, register queue along z, no shared memory; boundary cells by
 * ghost layers or a short fix-up launch); 4 = the two-step column-march
 * kernel (uniform k; two steps per pass, shared-memory stage plane; with
 * per-cell k it acts as 3); 5 = the column-march kernel with boundary cells
 * and periodic copies inside the pass (one launch per step; for small
 * grids); 6 = the column-march kernel with 8 cells a thread (16 for bf16
 * fields with uniform k); 7 = two steps per pass with TMA-staged input
 * planes (uniform k; with per-cell k it acts as 3); -1 = the plain
 * one-thread-per-column kernel (one step per pass; a
 * second, independent realisation of the same per-cell arithmetic).
 * Results do not depend on the choice: every kernel evaluates the same fixed
 * per-cell expression, so fields are bit-identical. */
int wfa_set_tuning(wfa_grid g, int depth, int variant);

/* Planes per z chunk of the column-march kernels (variants 3 and 5): each
 * block of those kernels marches one chunk of the z extent, neighbouring
 * chunks in opposite directions. planes = 0 (the default) lets the tuned or
 * automatic choice stand. A tuning aid with no counterpart in the paper:
 * results do not depend on it (fields are bit-identical).
 * Errors: WFA_ERR_ARG for a NULL grid or planes < 0. */
int wfa_set_zchunk(wfa_grid g, int planes);

/* No counterpart in the paper (a tuning aid, like wfa_set_tuning).
 * The kernel configuration the next wfa_step of this grid uses (after
 * wfa_set_tuning, wfa_set_zchunk and wfa_autotune): fused depth, variant
 * (as in wfa_set_tuning) and planes per z chunk (0 = automatic). Any output
 * pointer may be NULL. Errors: WFA_ERR_ARG for a NULL grid. */
int wfa_get_tuning(wfa_grid g, int* depth, int* variant, int* zchunk);

/* No counterpart in the paper (its step has one mapping, a column per tile,
 * Sec. 2.1). Time the compiled kernel configurations (the column-march kernels 3 to 7,
 * kernel 3 also with z chunks of 8, 12, 32, 64, 128 planes and of half the
 * z extent, kernel 6 with chunks of 12 and 32; the tiled TMA kernel at
 * depths 1..8 and two tile shapes) on this grid and use the fastest from
 * now on. The trials run on a scratch copy of the field: the field and the step
 * count are left as they were, and results never depend on the choice. The
 * choice is also remembered for later grids of the same size class (device
 * compute capability and SM count, storage,
 * conductivity mode, advection, log2 of each edge) in this process, and in
 * the file named by the environment variable WFA_TUNE_CACHE if it is set.
 * Synchronises the stream; needs one extra field of device memory while it
 * runs. *depth / *variant (may be NULL) receive the choice. */
int wfa_autotune(wfa_grid g, int* depth, int* variant);

/* Advance n >= 0 time steps (asynchronous on the grid's stream): n
 * applications of Eq. expl_form (Sec. 1.1.1, the explicit time step, T^n ->
 * T^{n+1} for every cell from the values of step n), in the face-flux form
 * given at the top of this file. The paper's fused kernel runs one step per
 * RPC (Sec. 2.1, Example Code); here a step is one pass of a kernel over the
 * grid, or several steps per pass with temporal blocking.
 * Errors: WFA_ERR_STATE before the field, coefficients and dt are set,
 * WFA_ERR_BC for an unpaired periodic face, WFA_ERR_CUDA. */
int wfa_step(wfa_grid g, long long n);

/* Number of steps taken since the last wfa_set_field: the time index n of
 * T^n in Eq. expl_form, counted from the field that was set. */
int wfa_steps_done(wfa_grid g, long long* n);

/* Copy the field out as dense fp32 (nx*ny*nz floats). Synchronises the
 * stream. The counterpart of reading a WSE_Array back into a NumPy array
 * (Sec. 2.1, Example Code), where the WFA's validation mode compares results. */
int wfa_read_field(wfa_grid g, float* host_dense);

/* Total heat E = sum_C T_C hx hy hz, summed on the device in fp64 in a fixed
 * order (bit-reproducible for a given grid). Synchronises the stream.
 * Sec. 3, reduction of a field to one value. */
int wfa_total_heat(wfa_grid g, double* e);

/* Sum of a caller-owned dense device array of n floats, in fp64, times scale
 * (the reduction of wfa_total_heat), written to *d_out (device memory), queued
 * on `stream` (a cudaStream_t; NULL = the legacy default stream). The paper
 * has no counterpart: this entry point exists for callers that cannot
 * allocate device memory (a process that reserves all device memory in its
 * own pool, a real-time loop that cannot afford an allocation's implicit
 * synchronisation, a plug-in inside a framework that owns every buffer). It
 * allocates nothing: its scratch, one fp64 partial per 16384 elements, is a
 * fixed 64 KiB array in the library's device image, held by every GPU that
 * loads the library until the process exits. Hence n <= 2^27 (134,217,728);
 * larger n is rejected with WFA_ERR_ARG. Every call writes all the scratch it
 * reads (nothing carries over), but all calls share the array: calls that may
 * overlap on the GPU (on different streams without ordering) race. The first
 * call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins. The address is kept per device and
 * context: after a cudaDeviceReset the next call looks it up again (so make
 * that call, too, outside a capture). Bit-reproducible for a given n.
 * Errors: WFA_ERR_ARG (null pointer, negative or too large n), WFA_ERR_CUDA. */
int wfa_sum_f32_noalloc(const float* d_x, long long n, double scale, double* d_out, void* stream);

/* Implicit time steps (Sec. 1.1.2, Eq. impl_form): n >= 0 backward-Euler
 * steps of size dt >= 0 (no stability limit; dt of wfa_set_dt is not used),
 * each solving, for every cell that is not held,
 *   T'_C - dt * [ sum_f K_f (T'_D - T'_C) / h_a^2
 *                 + sum_{Dirichlet faces} 2 k_C (Tb - T'_C) / h_a^2 ] = T_C
 * (the explicit step's face terms taken at the new time; held layers keep
 * their value) by classic conjugate gradients, two inner products per
 * iteration, started from T. Uniform k = k0, h = 1 and held layers on every
 * face give Eq. impl_form with omega = k0 dt. A step stops when
 * ||r|| <= rtol ||b|| (the recursively updated residual; rtol = 0 runs
 * max_iter iterations) or after max_iter iterations. A call is one graph
 * launch (device-side loops over the steps and iterations) and one wait.
 * Work vectors (four fp32 fields, seven for WFA_CG_PIPELINED) are allocated
 * on the first call and kept with the grid.
 * *iters (may be NULL) receives the CG iterations of all n steps,
 * *rel_res (may be NULL) the last step's ||r|| / ||b||. Synchronises the
 * stream. Needs fp32 storage and no advection (with u != 0 the system is not
 * symmetric): WFA_ERR_ARG otherwise, or for dt < 0, n < 0, rtol < 0,
 * max_iter < 0; WFA_ERR_STATE before the field and coefficients are set;
 * WFA_ERR_BC for a periodic face paired with a non-periodic one. */
int wfa_implicit_step(wfa_grid g, double dt, long long n, double rtol, int max_iter, long long* iters,
                      double* rel_res);

/* CG variant of wfa_implicit_step (the iterates are the same in exact
 * arithmetic; the default is WFA_CG_CLASSIC):
 *   WFA_CG_CLASSIC    classic CG, two inner products and two kernels an
 *                     iteration (Sec. 1.1.2);
 *   WFA_CG_PIPELINED  Chronopoulos and Gear's CG, both inner products in one
 *                     reduction and one kernel an iteration (the
 *                     reduction-limited variant Sec. 3.2 points to); w = A r
 *                     and s = A p by recurrence, three more fp32 work fields.
 * Errors: WFA_ERR_ARG for a NULL grid or another value. */
enum { WFA_CG_CLASSIC = 0, WFA_CG_PIPELINED = 1 };
int wfa_set_cg_method(wfa_grid g, int method);

/* Heat that one time step from the current field brings in through the
 * Dirichlet faces (Sec. 3's reduction, applied to the boundary), in fp64:
 * dt * hx*hy*hz * sum over the cells on Dirichlet faces of
 * 2 k_C (T_b - T_C) / h^2 plus the upwind advective flux (T_b upwind for
 * inflow, T_C for outflow). With zero-flux and periodic faces elsewhere,
 * E(n+1) - E(n) equals it up to the rounding of the step. Synchronises the
 * stream. Errors: WFA_ERR_STATE before field, coefficients and dt are set;
 * WFA_ERR_BC with held layers (they are cells, not faces). No counterpart
 * call in the paper. */
int wfa_boundary_flux(wfa_grid g, double* flux);

/* Bytes of one padded field buffer and of one padded k (or 1/k) buffer of
 * this grid, for callers that own the device memory (below). No counterpart
 * in the paper (the WFA's arrays live in each tile's own memory, Sec. 1). */
int wfa_grid_buffer_bytes(wfa_grid g, size_t* field_bytes, size_t* k_bytes);

/* No counterpart in the paper (the WFA's arrays live in each tile's own memory, Sec. 1).
 * Let caller-owned device memory hold the grid's data (e.g. tensors of a
 * framework that manages all device memory): d_Ta and d_Tb, field_bytes
 * each, take the two field buffers; d_k and d_r, k_bytes each (both or both
 * NULL), take the per-cell conductivity and its reciprocal, now if the grid
 * has per-cell k and from the next wfa_set_coeffs with k otherwise. All
 * must be distinct, 256-byte aligned device memory; the grid's current
 * contents are copied in and its own buffers released. The caller keeps the
 * buffers alive until wfa_destroy_grid, which does not free them; their
 * layout is the library's padded layout (opaque to the caller).
 * Synchronises the stream. Errors: WFA_ERR_ARG, WFA_ERR_CUDA. */
int wfa_grid_attach_buffers(wfa_grid g, void* d_Ta, void* d_Tb, float* d_k, float* d_r);

/* Wait for the grid's queued work; reports a device-side error. The host
 * side of Sec. 2's control flow: the program runs on the device without host
 * interaction until the host collects the result. */
int wfa_sync(wfa_grid g);

/* Kernel timing, a profiling aid with no counterpart in the paper.
 * wfa_set_kernel_timing(g, every): every > 0 records a CUDA event pair on the
 * grid's stream just before and just after the main sweep kernel of every
 * every-th pass that wfa_step launches from now on (a pass's boundary fix-up
 * and periodic-copy kernels fall outside the pair; autotuning trials are not
 * sampled; on small grids, where wfa_step replays captured runs of 32 passes
 * as CUDA graphs, a sample brackets a whole run and counts as 32 launches);
 * 0 turns timing off and frees the events. At most 4096 pairs are
 * held; later passes go unsampled until wfa_kernel_time reads them.
 * Errors: WFA_ERR_ARG for a NULL grid or every < 0. */
int wfa_set_kernel_timing(wfa_grid g, int every);

/* Number of kernels the sweeps of this grid have launched (wfa_step,
 * autotuning trials included), a profiling aid with no counterpart in the
 * paper. */
int wfa_launch_count(wfa_grid g, long long* n);

/* Synchronise the stream, then give the summed duration in milliseconds and
 * the number of the sampled kernel launches since the last call (0 and 0 when
 * timing is off), and start counting afresh. A profiling aid with no
 * counterpart in the paper (it feeds the bandwidth model of Sec. 3.1.3,
 * Eqs. A_eff and t_it_min, with measured kernel times). */
int wfa_kernel_time(wfa_grid g, double* ms, long long* launches);

/* Message of the last failed call on this thread ("" if none). Error
 * reporting of this C ABI; no counterpart in the paper. */
const char* wfa_last_error(void);

/* Host-side fault injection for testing the out-of-memory paths, with no
 * counterpart in the paper: after n >= 0 further successful device
 * allocations from the grid memory pool (field, conductivity, staging and
 * reduction buffers of wfa_create_grid, wfa_set_coeffs, wfa_set_field and
 * the autotuner), the next one fails once as if the device were out of
 * memory, so that call returns WFA_ERR_OOM and leaves the grid as it was;
 * n < 0 disarms a pending failure. Process-wide; nothing is injected on the
 * device. The environment variable WFA_FAULT_ALLOC_AT=n (n >= 1), read at the
 * first device allocation, arms the same failure for the n-th allocation of
 * the process. Returns WFA_OK. */
int wfa_inject_alloc_failure(int n);

/* ------------------------------------------------ slabs (z decomposition) -- */
/* One grid split along z into slabs, each an ordinary grid (Sec. 1, Fig. 1b:
 * domain decomposition; Sec. 2.1: each WSE tile owns a column of cells;
 * Sec. 3: neighbour values come over the fabric for every product; Eq. iteration_time_model: a step's
 * time is its computation or its halo exchange, whichever is longer, plus the
 * boundary work). A slab holds planes [z0, z1) of the whole grid: nx, ny, the
 * cell size, storage, x / y faces, conductivity (its planes), velocity and dt
 * as the whole grid; its z faces towards neighbouring slabs are
 * WFA_BC_EXCHANGE faces, its other z faces the whole grid's (a periodic z
 * axis: exchange faces at both ends, the last slab's +z face meeting the
 * first slab's -z face). Before every step the outermost plane of each slab
 * is copied into the halo plane beyond the neighbour's exchange face; each
 * cell then sees the operands it has in the whole grid, so the slabs' fields
 * are bitwise the whole grid's. Slabs step with the column-march kernels
 * (variants 3 and 5) or the one-column kernel, one step per pass; batched and
 * implicit steps reject exchange faces (WFA_ERR_BC). The stability limit of a
 * slab counts its exchange faces as interior faces and needs the
 * neighbours' conductivity planes (wfa_exchange with WFA_PLANES_K) first: the
 * whole grid's limit is the minimum over its slabs. Total heat: the sum over
 * slabs. */
enum { WFA_PLANES_FIELD = 0, WFA_PLANES_K = 1, WFA_PLANES_RECIP_K = 2 };

/* Sec. 3: a tile's column receives its neighbours' values for every
 * product (Sec. 2.1: a column of cells per tile); here one
 * slab's boundary plane with the next slab's (Sec. 1, Fig. 1b's partition).
 * Device addresses of the planes an exchange face moves, for callers that
 * move them themselves (slabs on several GPUs or processes, e.g. NCCL send /
 * receive into the receiving GPU's own memory). face: WFA_ZLO or WFA_ZHI,
 * which must be an exchange face. what: WFA_PLANES_FIELD (the buffer that
 * holds the current field: the addresses change with every step),
 * WFA_PLANES_K or WFA_PLANES_RECIP_K (per-cell k and 1/k; both must be moved
 * after every wfa_set_coeffs). *send: the slab's own outermost plane next to
 * the face (z = 0 or nz - 1); *recv: the halo plane beyond the face (z = -1
 * or nz), where the neighbour's outermost plane goes; *plane_bytes: the size
 * of one such plane (whole padded planes, contiguous). Any output may be NULL.
 * Queued halo and coefficient set-up work of the grid is issued first (on its
 * stream), so that nothing overwrites a received plane later. Errors:
 * WFA_ERR_ARG, WFA_ERR_BC (not an exchange face), WFA_ERR_STATE (k planes of
 * a grid with uniform k). */
int wfa_exchange_planes(wfa_grid g, int face, int what, void** send, void** recv, size_t* plane_bytes);

/* The neighbour exchange (Sec. 3) between two slabs on one device (Sec. 1,
 * Fig. 1b's partition along z): lower's +z exchange face
 * meets upper's -z exchange face (lower == upper: one slab whose z axis wraps
 * around). what: WFA_PLANES_FIELD (the current fields) or WFA_PLANES_K
 * (per-cell k and 1/k; nothing for uniform k). Copies are queued on lower's
 * stream after upper's queued work, and upper's later work waits for them.
 * Errors: WFA_ERR_ARG (different nx, ny or storage, different devices),
 * WFA_ERR_BC (not exchange faces), WFA_ERR_CUDA. */
int wfa_exchange(wfa_grid lower, wfa_grid upper, int what);

/* Eq. expl_form on a grid partitioned into z slabs (Sec. 1, Fig. 1b), with
 * the neighbour exchange (Sec. 3) before every step.
 * Advance the slabs gs[0 .. count-1] (in z order, one device) by n steps:
 * the conductivity planes are exchanged once, then before every step the
 * field planes of each pair of neighbouring slabs (and of the last and the
 * first, when the z axis wraps), then every slab takes one step. The slabs
 * need one dt. Errors: WFA_ERR_ARG, WFA_ERR_STATE (a slab without field,
 * coefficients or dt), WFA_ERR_BC (neighbours that do not meet at exchange
 * faces), WFA_ERR_CUDA. */
int wfa_slabs_step(wfa_grid* gs, int count, long long n);

/* ----------------------------------------------------------- batching -- */

/* Advance many grids in one go (Sec. 3.1.2: iteration rate at small
 * workloads per processor). gs[i] advances steps[i] >= 0 steps; grids may mix
 * storage types and conductivity modes. All grids must share the stream of
 * gs[0], appear once, and have their field, coefficients and dt set. Round
 * r advances every grid with more than r steps by one step, one multi-grid
 * launch per class of grid; all rounds are captured into one CUDA graph and
 * launched once. The environment variable WFA_BATCH_MODE selects
 * "persistent" (all rounds in one persistent kernel whose blocks meet at a
 * grid-wide barrier with a bounded spin) or "stream" (the per-round launches
 * without a graph). Results are bitwise identical to calling wfa_step on
 * each grid, in every mode. Returns after the work is done (synchronises the
 * stream).
 * Errors: WFA_ERR_ARG (NULL or repeated grid, negative steps, different
 * streams, more steps than the barrier counter holds), WFA_ERR_STATE (a grid
 * not ready to step), WFA_ERR_TIMEOUT (a device-side wait gave up; the fields
 * of the grids are then undefined), WFA_ERR_CUDA. */
int wfa_batch_run(wfa_grid* gs, const long long* steps, int count);

/* ------------------------------------------------------------- serving -- */
/* Serving has no counterpart call in the paper. It applies Sec. 3.1.2's
 * point about small workloads per processor (the explicit step keeps its rate
 * down to about 50 cells per WSE tile, where a distributed code needs
 * thousands) to a stream of independent small solves: many grids resident on
 * the device at once, advanced together by the batched sweep. A request
 * carries its own inputs (not a wfa_grid) because the server owns the device
 * memory of resident requests: it allocates a grid only when the request fits
 * the HBM budget, and frees it when the result is back on the host. */

typedef struct wfa_server_s* wfa_server;

/* A transient solve submitted to the server. The server reads T0_host and
 * k_host when it admits the request (it moves them to the device on its own
 * thread, beside the running work) and writes out_host when the request is
 * done: all three must stay valid until the ticket is done. dt <= 0 selects
 * 0.9 * dt_max. */
typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
    int storage;              /* WFA_F32 / WFA_BF16 */
    const float* T0_host;     /* nx*ny*nz */
    const float* k_host;      /* nx*ny*nz, or NULL for k_uniform */
    double k_uniform;
    double ux, uy, uz;
    int bc_kind[6];
    double bc_value[6];
    double dt;
    long long steps;
    float* out_host;          /* nx*ny*nz, written when the ticket is done */
} wfa_request;

typedef struct {
    long long submitted, admitted, completed, rejected;
    long long ticks;           /* scheduler iterations that launched work */
    double cell_updates;       /* total cell-updates performed */
    double busy_seconds;       /* wall time with work on the device */
    double p50_latency_s, p99_latency_s, mean_latency_s;  /* submit -> result on host */
    size_t resident_bytes, peak_resident_bytes;
} wfa_server_stats;

/* Start a continuous-batching server on its own scheduler thread (many
 * small workloads sharing one processor, Sec. 3.1.2; the paper has no
 * server).
 * hbm_budget_bytes: admission limit on the device memory of resident
 * requests; max_resident: most requests on the device at once (0 = 1024);
 * quantum: steps a resident request advances per scheduler tick (0 = 64).
 * Requests that arrive while others run are admitted at the next tick as
 * memory and slots free up. A tick takes the residents with the least
 * remaining work (cells x steps) until about 64 M cells are in it, plus any
 * resident passed over 8 ticks in a row, and advances each by up to quantum
 * steps (all of them when fewer than two quanta are left), together in one
 * batched launch (wfa_batch_run). Four more threads move inputs to the
 * device and results back, each on its own stream, while the ticks run. A
 * request's result is bitwise the result of running it alone. */
int wfa_server_create(size_t hbm_budget_bytes, int max_resident, long long quantum,
                      wfa_server* out);

/* Queue a request (one transient solve: Eq. expl_form for r->steps steps on
 * its own grid; see the serving note above); *ticket identifies it.
 * WFA_ERR_BUDGET if it can never fit. */
int wfa_server_submit(wfa_server s, const wfa_request* r, long long* ticket);

/* *done = 1 once out_host holds the result (0 while queued or running;
 * -1 if the request failed, with the reason in wfa_last_error()). Serving
 * (see the note above); no counterpart call in the paper. */
int wfa_server_poll(wfa_server s, long long ticket, int* done);

/* Block until the ticket is done or timeout_s passes (WFA_ERR_TIMEOUT).
 * Serving (see the note above); no counterpart call in the paper. */
int wfa_server_wait(wfa_server s, long long ticket, double timeout_s);

/* Latency of a finished request: seconds from its wfa_server_submit to its
 * result in out_host. WFA_ERR_STATE while it is not done (or if it failed),
 * WFA_ERR_ARG for an unknown ticket. Serving metrics (see the note above); no
 * counterpart call in the paper. */
int wfa_server_latency(wfa_server s, long long ticket, double* seconds);

/* Counters and latency percentiles of the server so far (see
 * wfa_server_stats). Serving (see the note above); the iteration-rate and
 * latency figures the paper reports for single solves (Sec. 3) become
 * throughput and p50 / p99 latency of a request stream here. */
int wfa_server_stats_get(wfa_server s, wfa_server_stats* st);

/* Stop the scheduler (finishing resident work first) and free everything.
 * Serving (see the note above); no counterpart call in the paper. */
int wfa_server_destroy(wfa_server s);

#ifdef __cplusplus
}
#endif

#endif /* WFA_H */
