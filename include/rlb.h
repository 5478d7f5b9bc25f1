/*
 * rlb.h -- C ABI of librlb: the relativistic lattice Boltzmann (RLB) step of
 * Mendoza, Boghosian, Herrmann and Succi, "Lattice Boltzmann scheme for
 * relativistic fluids" (arXiv:0912.2913), on one NVIDIA GB300 (sm_103a).
 *
 * The scheme: two D3Q19 population sets per cell, f_i (particle number) and
 * g_i (energy-momentum) (Fig. 2 and the paragraph that introduces f_i and
 * g_i); each step streams the populations one cell along their velocity and
 * relaxes them to the ultra-relativistic equilibria with BGK time tau
 * (Eqs. lbe1, lbe2, equil1s, equil2as, equil2bs); the macroscopic fields n,
 * eps, beta come from the moment constraints n gamma = sum f_i,
 * (4/3) eps (gamma^2 - 1/4) = sum g_i, (4/3) eps gamma^2 u = sum g_i c_i
 * with eps = 3P.  Optionally (rlb_eos) the general equilibria of Eqs. equil1,
 * equil2a, equil2b with (eps + P) gamma^2 - P = sum g_i,
 * (eps + P) gamma^2 u = sum g_i c_i and an ideal-gas equation of state.
 *
 * Conventions common to every entry point:
 *  - Lattice: nx * ny * nz cells, x fastest; cell = (z*ny + y)*nx + x.  y and
 *    z are periodic; x is periodic, or has ghost planes (rlb_xbc).
 *  - Field arrays (n, eps, dL/dn, ...) are float64, N = nx*ny*nz values in
 *    cell order; beta-like arrays are three consecutive planes of N values
 *    (x, y, z components).  solid is N bytes, non-zero = solid cell.
 *  - A "state" is one set of populations in device memory: 38 planes
 *    (f_0..f_18, g_0..g_18), plane q starting at element q * plane_stride
 *    (rlb_state_layout), element type float64 (RLB_FP64) or float32
 *    (RLB_FP32_DEV: deviations from the rest equilibrium of n_ref, eps_ref).
 *    Velocity i follows this order: 0 rest; 1..6 = +x, -x, +y, -y, +z, -z;
 *    7..18 = (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1),
 *    (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).
 *    Solid cells hold a NaN-payload marker in every plane.
 *  - Pointers marked "device" must be device memory of the context's GPU,
 *    aligned to 16 bytes; the caller owns every array it passes; nothing is
 *    retained after the call returns (the context keeps only its own
 *    workspace).  Work is enqueued on the context's CUDA stream; a call
 *    returns before the GPU finishes unless it says it synchronises.
 *  - Errors are status codes, never aborts.  A CUDA error is latched in the
 *    context and returned by every later call on it (rlb_last_error gives the
 *    text).  Unphysical cells (failed recovery) do not stop a run: values are
 *    written as computed and the cells are counted (rlb_stats).
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef RLB_H
#define RLB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RLB_API __attribute__((visibility("default")))
#else
#define RLB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlb_ctx rlb_ctx;

typedef enum {
    RLB_OK = 0,
    RLB_ERR_ARG = 1,         /* invalid argument (null pointer, size, parameter range) */
    RLB_ERR_OOM = 2,         /* a device or host allocation failed                      */
    RLB_ERR_CUDA = 3,        /* a CUDA call failed; latched in the context              */
    RLB_ERR_UNPHYSICAL = 4,  /* outputs written, but some cell failed the recovery      */
    RLB_ERR_STATE = 5        /* call out of order (e.g. step before init)               */
} rlb_status;

typedef enum { RLB_FP64 = 0, RLB_FP32_DEV = 1 } rlb_precision;

/* x boundary.  Periodic; or an inflow ghost plane x = 0 held at the
 * equilibrium of (n_in, eps_in, beta_in) plus an outflow ghost x = nx-1 that
 * copies x = nx-2 after each step; or outflow copies at both ends
 * (x = 0 <- x = 1, x = nx-1 <- x = nx-2).  Ghost planes are not collided. */
typedef enum { RLB_BC_PERIODIC = 0, RLB_BC_INFLOW_OUTFLOW = 1, RLB_BC_OUTFLOW_BOTH = 2 } rlb_xbc;

typedef enum { RLB_HOST = 0, RLB_DEVICE = 1 } rlb_where;

/* Equation of state.  RLB_EOS_ULTRA: eps = 3P, the equilibria of Eqs.
 * (equil1s), (equil2as), (equil2bs) with the closed-form recovery.
 * RLB_EOS_GAMMA_LAW: an ideal gas with rest mass, P = (eos_gamma - 1)
 * (eps - n eos_mass), the general equilibria of Eqs. (equil1), (equil2a),
 * (equil2b) and the macroscopic constraints after Fig. 2, inverted by a
 * Newton iteration on P; FP64 states only, no discrete adjoint.            */
typedef enum { RLB_EOS_ULTRA = 0, RLB_EOS_GAMMA_LAW = 1 } rlb_eos;

/* z boundary (not in the paper: the decomposition of one lattice into z
 * slabs).  RLB_ZBC_PERIODIC: the lattice is periodic in z.  RLB_ZBC_HALO: the
 * context holds one z slab of a larger lattice, its planes z = 0 and
 * z = nz-1 are ghost copies of the neighbouring slabs' edge planes, which the
 * steps neither collide nor write, and rlb_halo_exchange refills them after
 * every step; only z = 1 .. nz-2 are updated (nz >= 3).  The eps = 3P
 * equation of state only; the adjoint entry points refuse such contexts.    */
typedef enum { RLB_ZBC_PERIODIC = 0, RLB_ZBC_HALO = 1 } rlb_zbc;

typedef struct {
    int32_t nx, ny, nz;   /* lattice size; nx >= 3 unless periodic; N <= 2^31 - 2^21   */
    int32_t prec;         /* rlb_precision                                              */
    int32_t xbc;          /* rlb_xbc                                                    */
    int32_t eos;          /* rlb_eos                                                    */
    double tau;           /* BGK relaxation time in steps, tau > 1/2 (Eqs. lbe1, lbe2)  */
    double c_l;           /* lattice speed dx/dt in units of c (c_l > 1: "tachyons")    */
    double n_in, eps_in;  /* inflow state (RLB_BC_INFLOW_OUTFLOW)                       */
    double beta_in[3];
    double n_ref, eps_ref;/* RLB_FP32_DEV reference: populations are stored as
                             f - f^eq(n_ref, eps_ref, beta = 0); must be > 0           */
    double eos_gamma;     /* RLB_EOS_GAMMA_LAW: adiabatic index, 1 < Gamma <= 2         */
    double eos_mass;      /* RLB_EOS_GAMMA_LAW: particle rest mass m >= 0               */
    int32_t zbc;          /* rlb_zbc                                                    */
    int32_t reserved;     /* must be 0                                                  */
} rlb_params;

/* Size of one state: plane stride in elements and element size in bytes;
 * bytes = 38 * plane_stride * elem_bytes.  The adjoint variables lambda use
 * the same layout and element type.                                         */
RLB_API rlb_status rlb_state_layout(const rlb_params* p, int64_t* plane_stride, int32_t* elem_bytes, size_t* bytes);

/* Bytes of device workspace a context needs (two states, counters and
 * reduction buffers).                                                       */
RLB_API rlb_status rlb_workspace_bytes(const rlb_params* p, size_t* bytes);

/* Create a context on the current CUDA device.  stream: a cudaStream_t (NULL
 * = legacy default stream).  workspace: device memory of at least
 * rlb_workspace_bytes, owned by the caller and kept by the context until
 * rlb_destroy; or NULL, in which case the context allocates it with
 * cudaMallocAsync on the stream and frees it in rlb_destroy.
 * Errors: RLB_ERR_ARG (bad parameters), RLB_ERR_OOM, RLB_ERR_CUDA.        */
RLB_API rlb_status rlb_create(const rlb_params* p, void* stream, void* workspace, size_t workspace_bytes, rlb_ctx** out);
RLB_API rlb_status rlb_destroy(rlb_ctx* ctx);

/* Initial condition (the shock-tube paragraph: both sides start as
 * "thermodynamically equilibrated matter"): every fluid cell starts at
 * f^eq, g^eq of its fields; the inflow plane at the inflow state; solid
 * cells take the solid marker.  n, eps: N values; beta: 3N; solid: N bytes
 * or NULL.  where = RLB_HOST (copied in, synchronises) or RLB_DEVICE.
 * Solid cells may not lie on the planes x = 0, 1, nx-2, nx-1 of a
 * non-periodic lattice (RLB_ERR_ARG).  Resets the step counter and stats.  */
RLB_API rlb_status rlb_init_fields(rlb_ctx* ctx, const double* n, const double* eps, const double* beta,
                           const uint8_t* solid, rlb_where where);

/* Enqueue nsteps time steps of Eqs. (lbe1), (lbe2) on the context's state
 * (fused pull streaming with link bounce-back, moments, eps = 3P recovery,
 * equilibria Eqs. (equil1s, equil2as, equil2bs), BGK relaxation, boundary
 * planes; under RLB_EOS_GAMMA_LAW the Newton recovery and Eqs. (equil1,
 * equil2a, equil2b)).  Asynchronous, except that the first call on an RLB_FP32_DEV
 * context times its launch variants (bit-identical results) on the
 * context's second buffer and synchronises once; make that first call
 * before any stream capture.  nsteps >= 0.                                  */
RLB_API rlb_status rlb_step(rlb_ctx* ctx, int32_t nsteps);

/* One time step from the device state src into the device state dst (both
 * caller-owned, rlb_state_layout bytes, distinct); every cell of dst is
 * written.  Does not touch the context's own state or its statistics.      */
RLB_API rlb_status rlb_step_into(rlb_ctx* ctx, const void* src, void* dst);

/* As rlb_step_into, and the update counts in the context's statistics as its
 * next time step (steps, n_unphysical, first_bad, n_nonpositive_eq): a run
 * that keeps its states in caller buffers (the stored tail of a checkpointed
 * gradient run) reports the statistics of rlb_step.  The context's own state
 * is not touched.  RLB_ERR_STATE before rlb_init_fields (the statistics start
 * there), RLB_ERR_ARG for NULL or equal buffers.  Not in the paper.        */
RLB_API rlb_status rlb_step_into_counted(rlb_ctx* ctx, const void* src, void* dst);

/* Device pointer of the context's current state (valid until the next
 * rlb_step / rlb_init_fields / rlb_load_state / rlb_destroy).               */
RLB_API rlb_status rlb_state_ptr(rlb_ctx* ctx, void** state);

/* Copy the current state to / from caller device memory (same layout).     */
RLB_API rlb_status rlb_save_state(rlb_ctx* ctx, void* dst);
RLB_API rlb_status rlb_load_state(rlb_ctx* ctx, const void* src);

/* Macroscopic fields of a state (the moment constraints solved with
 * eps = 3P, or by the Newton recovery under RLB_EOS_GAMMA_LAW): n, eps (N
 * values each) and beta (3N); NaN at solid cells.
 * state = NULL means the context's current state.  where = RLB_DEVICE
 * (device outputs) or RLB_HOST (host outputs).  Synchronises; returns
 * RLB_ERR_UNPHYSICAL when a non-solid cell of the state fails the recovery
 * or the run so far counted an unphysical update (outputs still written).  */
RLB_API rlb_status rlb_macro(rlb_ctx* ctx, const void* state, double* n, double* eps, double* beta, rlb_where where);

/* Statistics since rlb_init_fields.  Synchronises.  steps: steps taken;
 * n_unphysical: cell updates whose recovery failed; first_bad: smallest
 * step*N + cell of such an update, -1 if none; n_nonpositive_eq: cell
 * updates whose equilibrium had a non-positive population (the positivity
 * condition c_i.u < c_l^2/3 stated for the tachyon runs, decided in
 * binary32).  Any pointer may be NULL.                                      */
RLB_API rlb_status rlb_stats(rlb_ctx* ctx, int64_t* steps, int64_t* n_unphysical, int64_t* first_bad,
                     int64_t* n_nonpositive_eq);

/* ---- discrete adjoint (transpose of the exact Jacobian of the step) ----
 * Not in the paper: the transpose of the Jacobian of one step of Eqs. (lbe1),
 * (lbe2) with the eps = 3P equilibria and recovery, boundary planes and
 * bounce-back included.  Every adjoint entry point returns RLB_ERR_ARG on a
 * NULL or aliased buffer and on an RLB_EOS_GAMMA_LAW context.               */

/* lambda_T = (d macro / d state)^T (dL/dn, dL/deps, dL/dbeta) at the device
 * state 'state': device inputs of N, N and 3N float64; lam_out a device
 * state-layout buffer.  Zero at solid cells.                                */
RLB_API rlb_status rlb_adjoint_macro(rlb_ctx* ctx, const void* state, const double* dL_dn, const double* dL_deps,
                             const double* dL_dbeta, void* lam_out);

/* One adjoint step: given the state A_t the forward step started from
 * (device), lam_in = dL/dA_{t+1} and lam_out = dL/dA_t (device, distinct,
 * every element written).  Adds dL/dtau of the step to *dL_dtau_accum and
 * dL/dbeta_in to dL_dbeta_in_accum[3] (device float64; the sums are taken
 * in a fixed order, so results do not depend on scheduling).               */
RLB_API rlb_status rlb_adjoint_step(rlb_ctx* ctx, const void* state_t, const void* lam_in, void* lam_out,
                            double* dL_dtau_accum, double* dL_dbeta_in_accum);

/* rlb_adjoint_step without any device allocation.  The paper has no
 * counterpart: this is an interface for callers that cannot allocate device
 * memory at the point of the call -- code running under a caching allocator
 * or memory pool that owns all device memory, or a real-time loop that must
 * not synchronise (cudaMalloc/cudaFree can synchronise the device).
 * Same arguments, results and errors as rlb_adjoint_step, and the same
 * kernels: FP64 the persistent register kernel (SMs x 2 blocks), FP32 the
 * persistent shared-memory staged kernel (SMs x 3 blocks of 128; with
 * RLB_ADJ_PIPE=0 or 1 the persistent register kernel, SMs x 4 blocks), grids
 * capped at N/128 blocks.  The per-warp partial sums live in one static
 * device array of 32768 doubles (256 KiB) per device: a launch that would
 * need more (16 doubles per block) returns RLB_ERR_ARG and enqueues nothing;
 * every launch writes all the slots it reads, so nothing needs to start at
 * zero.  The first call on each device (and the first after the device's
 * context was reset) does the set-up: it takes the array's address and loads
 * every kernel this entry point launches, which may allocate and
 * synchronise, so make that first call before any stream capture and before
 * the code that must not allocate; later calls allocate nothing.  The
 * context's device must be current.  Calls that overlap in time on one
 * device (different streams or contexts) share the array and race:
 * serialise them.                                                          */
RLB_API rlb_status rlb_adjoint_step_noalloc(rlb_ctx* ctx, const void* state_t, const void* lam_in, void* lam_out,
                                            double* dL_dtau_accum, double* dL_dbeta_in_accum);

/* Halo exchange between two z slabs of one lattice (the paper has no
 * counterpart: this is the data movement of a z decomposition, one slab per
 * context, on one device).  lower and upper: contexts with zbc =
 * RLB_ZBC_HALO, the same nx, ny, precision and device; upper's slab lies
 * directly above lower's (lower's last updated plane z = nz_l - 2 and upper's
 * first updated plane z = 1 are neighbours in the whole lattice; for a
 * lattice periodic in z, the last slab's upper neighbour is the first slab,
 * and a single slab is its own neighbour: lower == upper).  In the current
 * states of both contexts it copies the 10 populations with e_z = +1 (5 of
 * f, 5 of g) of lower's plane z = nz_l - 2 into upper's ghost plane z = 0,
 * and the 10 with e_z = -1 of upper's plane z = 1 into lower's ghost plane
 * z = nz_l - 1: exactly what the next step pulls across the two faces.  One
 * kernel launch on lower's stream; when upper's stream is another one, the
 * copy is ordered after the work already enqueued there and before any work
 * enqueued there later.  Call it after every step (rlb_step with nsteps = 1)
 * of every slab and before the next step.  Errors: RLB_ERR_ARG for contexts
 * that do not fit together, RLB_ERR_STATE before rlb_init_fields.          */
RLB_API rlb_status rlb_halo_exchange(rlb_ctx* lower, rlb_ctx* upper);

/* Gradient with respect to the initial fields of rlb_init_fields, given
 * lam0 = dL/dA_0 (device): writes dL/dn0, dL/deps0 (N) and dL/dbeta0 (3N),
 * zero at solid cells and at the inflow plane, whose dependence on beta_in
 * is added to dL_dbeta_in_accum[3].  All pointers device.                   */
RLB_API rlb_status rlb_adjoint_fields(rlb_ctx* ctx, const double* n0, const double* eps0, const double* beta0,
                              const void* lam0, double* dL_dn0, double* dL_deps0, double* dL_dbeta0,
                              double* dL_dbeta_in_accum);

/* Diagnostic: the integer-pipe binary32 <-> binary64 conversions that the
 * FP32 deviation kernels use in their recovery, applied elementwise on the
 * current device (legacy default stream, synchronises): f2d_out[k] =
 * (double)f_in[k], d2f_out[k] = (float)d_in[k] rounded to nearest even.  All
 * pointers device, n >= 0.  Exact for values whose results are normal
 * numbers, zero, inf or NaN; binary32 subnormal results flush to zero.      */
RLB_API rlb_status rlb_selftest_conversions(const float* f_in, const double* d_in, int64_t n, double* f2d_out,
                                            float* d2f_out);

/* Debug: out-of-range state-buffer indices the step, adjoint and general-EOS
 * kernels met since the last call (the bounds-checking build, compiled with
 * RLB_CHECK_BOUNDS, counts them and keeps every access inside its buffer;
 * not in the paper).  Synchronises the current device.  The release build
 * sets *count = -1 and returns RLB_ERR_STATE.                              */
RLB_API rlb_status rlb_debug_bounds_violations(int64_t* count);

/* Debug: runs the bounds build's index check on one index in a kernel on the
 * legacy default stream (no memory is accessed with the index) and stores the
 * checked index in *checked: `index` itself when 0 <= index < n, else 0, and
 * the violation is counted as by the kernels.  The release build sets
 * *checked = -1 and returns RLB_ERR_STATE.                                   */
RLB_API rlb_status rlb_debug_bounds_selftest(int64_t index, int64_t n, int64_t* checked);

/* Wait for the context's stream; returns a latched or new CUDA error.       */
RLB_API rlb_status rlb_sync(rlb_ctx* ctx);

RLB_API const char* rlb_status_str(rlb_status s);

/* Text of the last error recorded on ctx (or globally when ctx is NULL).    */
RLB_API const char* rlb_last_error(rlb_ctx* ctx);

/* Number of kernel launches this context has enqueued (for accounting).     */
RLB_API int64_t rlb_launch_count(rlb_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RLB_H */
