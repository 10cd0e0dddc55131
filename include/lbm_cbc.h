/*
 * lbm_cbc.h -- C ABI of the GB300 (sm_103a) thermal lattice Boltzmann solver
 * with the layer-wise characteristic boundary condition of Klass, Gabbana &
 * Bartel, "Characteristic Boundary Condition for Thermal Lattice Boltzmann
 * Methods" (arXiv 2307.16766).
 *
 * One time step (Fig. flowchart-lbm-algo) is a fused pull-stream + BGK
 * collide over the bulk (Eqs. lbe, bgk, macro, feq-3/feq-4) followed by the
 * boundary solver of Sec. 3: characteristic analysis on each of the M boundary
 * layers (Eq. thermal_WAV), incoming amplitudes by Eqs. PNR / LODI-Relax /
 * CBC-PNR / CBC-Relax (Tab. CBCs), RK4 in time (Sec. 3.3) and a mesoscopic
 * Dirichlet write (equilibrium or Eq. NEEP).  Zero gradient (Eq. zg-bc) and a
 * fixed inflow equilibrium are available per side; corners use LODI along the
 * outward diagonal (Sec. 3.3, Fig. Layer-Multispeed-BC).
 *
 * Conventions
 *  - Every function returns LBM_OK (0) or a negative LBM_ERR_* code; the text
 *    of the last error of a handle is available from lbm_last_error().
 *  - Grid arrays are row-major [ny][nx], x fastest, double precision.
 *  - Sides are indexed W (-x) = 0, E (+x) = 1, S (-y) = 2, N (+y) = 3.
 *  - T is the dimensionless temperature (T~ = c_s^2 T, reference T0 = 1).
 *  - The library owns every device buffer it allocates; with lbm_create_in()
 *    the caller owns the workspace and must keep it alive until
 *    lbm_destroy().  Caller arrays passed to a call are only borrowed for the
 *    duration of that call.
 *  - Work is issued on the handle's CUDA stream (default: the legacy default
 *    stream; see lbm_set_stream()).  lbm_step() is asynchronous; the calls
 *    that return data to the caller synchronise the stream.  A step's
 *    kernels all go on the handle's stream (the bulk kernel behind the band
 *    kernel with programmatic stream serialization, so the two run side by
 *    side), so work issued afterwards on that stream sees the whole step.
 *    Only with the timing hook of lbm_set_kernel_events() does a step fork
 *    onto the handle's internal stream and join back (legal under stream
 *    capture).
 *  - A handle must not be used from two threads at once.
 */
#ifndef LBM_CBC_H
#define LBM_CBC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK              0
#define LBM_ERR_ARG        -1   /* invalid argument or configuration            */
#define LBM_ERR_ALLOC      -2   /* device or host allocation failed             */
#define LBM_ERR_CUDA       -3   /* a CUDA call failed (message has the reason)  */
#define LBM_ERR_NUMERICAL  -4   /* non-finite macroscopic values were produced  */
#define LBM_ERR_STATE      -5   /* call out of order (e.g. step before init)    */
#define LBM_ERR_TIMEOUT    -6   /* a bounded device-side wait gave up           */

/* Velocity sets (Appendix B): D2Q9 (M = 1, isothermal, second-order
 * equilibrium), D2Q37 (M = 3, fourth-order Hermite equilibrium, Eq. feq-4)
 * and D2Q17 (M = 3, third-order equilibrium, Eq. feq-3). */
enum lbm_lattice { LBM_D2Q9 = 0, LBM_D2Q37 = 1, LBM_D2Q17 = 2 };

/* Storage of the populations, always shifted by the rest state,
 * g_i = f_i - w_i rho0.  F64: double, FP64 arithmetic.  F32: float, FP32
 * arithmetic.  F16: half holding g_i / w_i, FP32 arithmetic.  The boundary
 * solver always runs in FP64. */
enum lbm_storage { LBM_F64 = 0, LBM_F32 = 1, LBM_F16 = 2 };

enum lbm_side_kind {
    LBM_SIDE_PERIODIC = 0,   /* both sides of an axis must be periodic or neither */
    LBM_SIDE_CBC      = 1,   /* characteristic boundary condition (Sec. 3)       */
    LBM_SIDE_INFLOW   = 2,   /* equilibrium of the fixed inflow state            */
    LBM_SIDE_ZG       = 3    /* zero gradient, Eq. zg-bc                         */
};

/* Incoming-wave treatment of a CBC side (Tab. CBCs). */
enum lbm_scheme { LBM_LODI = 0, LBM_LODI_RELAX = 1, LBM_CBC = 2, LBM_CBC_RELAX = 3 };

/* Viscous vector V of the CBC schemes: mesoscopic (Eqs. LaplaceU, LaplaceT,
 * with the one-sided stencil starting M nodes below x_f, at the first node
 * none of whose populations was streamed from a boundary layer; a
 * characteristic side then needs 3 M + 3 nodes across), finite differences
 * of the macros ("-FD" of Sec. 4.2), or none. */
enum lbm_viscous { LBM_VISCOUS_MESO = 0, LBM_VISCOUS_FD = 1, LBM_VISCOUS_OFF = 2 };

/* Mesoscopic Dirichlet condition (Sec. 3.3): equilibrium, Eq. NEEP, or NEEP
 * with the non-equilibrium part of x_f projected onto the Hermite
 * polynomials of orders 2 (D2Q9) or 2 and 3 (D2Q17, D2Q37) -- a regularised
 * scheme the paper names for future work (Sec. 5). */
enum lbm_dirichlet { LBM_DIRICHLET_EQ = 0, LBM_DIRICHLET_NEEP = 1, LBM_DIRICHLET_REG = 2 };

typedef struct lbm_cbc_params {
    int    side[4];     /* enum lbm_side_kind per side (W, E, S, N)                   */
    int    scheme[4];   /* enum lbm_scheme per CBC side                                */
    int    viscous;     /* enum lbm_viscous                                            */
    int    dirichlet;   /* enum lbm_dirichlet                                          */
    double alpha_T;     /* alpha of Eqs. CBC-Relax / LODI-Relax: transversal relaxation */
    double beta_P;      /* beta of Eqs. CBC-Relax / LODI-Relax: pressure relaxation     */
    double t_inf;       /* target transversal amplitude T^inf (the paper uses 0)        */
    double p_inf[4];    /* target pressure Z_inf = P_inf per side, P = rho c_s^2 T      */
    double inflow[4];   /* rho, ux, uy, T imposed on LBM_SIDE_INFLOW sides              */
    int    storage;     /* enum lbm_storage                                             */
    double rho0;        /* reference density of the population shift                   */
    double alpha_V;     /* relaxation of the viscous term towards 0 in Eq. CBC-Relax:
                           L_i = T_i + V_i + alpha_T (T_inf - T_i) + alpha_V (0 - V_i)
                           + beta_P (P - P_inf) on incoming waves (an extension; 0 is
                           the paper's equation; other schemes ignore it)            */
    double u_ref[2];    /* reference velocity of the stored populations: they are held
                           as f - f^eq(rho0, u_ref, T = 1) instead of f - w rho0, and
                           every equilibrium is formed as its difference from that one.
                           Exact for any value (|u_ref| < c_s); a value near the flow's
                           mean velocity keeps the stored values, and with them the
                           FP32/FP16 rounding, small.  (0, 0): the plain shift.  Not
                           supported by the gradient calls or in batches; a saved state
                           restores only into a solver with the same u_ref.         */
    int    band_ctas;   /* CTAs of the band launch with FP32 / FP16 storage, each taking
                           every band_ctas-th boundary tile (a tile holds a whole SM,
                           which the bulk kernel beside it then lacks).  0: as few as
                           keep the band within about half the bulk kernel's expected
                           time; above the tile count: one per tile.  Results do not
                           depend on it.  Ignored with FP64 storage and in batches.  */
} lbm_cbc_params;

typedef struct lbm_handle lbm_handle;

/* Fill p with defaults: all sides periodic, CBC-RELAX, mesoscopic viscous
 * terms, equilibrium Dirichlet, alpha_T = beta_P = t_inf = alpha_V = 0,
 * p_inf = rho0 c_s^2 (set per lattice by lbm_create when left at 0),
 * inflow = (1, 0, 0, 1), F32 storage, rho0 = 1, u_ref = (0, 0). */
int lbm_params_default(lbm_cbc_params* p);

/* Bytes of device workspace a configuration needs (for lbm_create_in). */
int lbm_workspace_bytes(int lattice, int nx, int ny, const lbm_cbc_params* p, size_t* bytes);

/* Create a solver for an nx x ny grid with BGK relaxation time tau > 1/2
 * (Eq. bgk).  Non-periodic axes need at least 2M + 3 nodes (3M + 3 across
 * a CBC side with the mesoscopic viscous vector); when both axes are
 * non-periodic, either all four sides are CBC or none is.  Allocates its
 * device memory with cudaMalloc on the current device. */
int lbm_create(int lattice, int nx, int ny, double tau, const lbm_cbc_params* p,
               lbm_handle** out);

/* As lbm_create, but carves every device buffer out of the caller's
 * workspace (device pointer, 256-byte aligned, at least
 * lbm_workspace_bytes()).  No device memory is allocated. */
int lbm_create_in(int lattice, int nx, int ny, double tau, const lbm_cbc_params* p,
                  void* dev_workspace, size_t workspace_bytes, lbm_handle** out);

/* Issue all further work on stream (a cudaStream_t; NULL = legacy default). */
int lbm_set_stream(lbm_handle* h, void* stream);

/* Initialise f = f^eq(rho, u, T) on every node (Sec. 2) and the boundary
 * state from the same fields.  Arrays are [ny][nx] doubles, on the device
 * when on_device != 0, else in host memory (copied in on the handle's stream).
 * For D2Q9, T is ignored (isothermal).  Resets the step counter and clears
 * the status of earlier steps (a wait that gave up, non-finite values). */
int lbm_init_fields(lbm_handle* h, const double* rho, const double* ux,
                    const double* uy, const double* T, int on_device);

/* Advance n time steps (asynchronous on the handle's stream).  Per step the
 * band kernel (strip nodes and the boundary solver) is launched first and the
 * bulk kernel (every bulk node) behind it on the same stream with
 * programmatic stream serialization, so the two run side by side; the
 * zero-gradient copies and the next step follow in stream order.  The result
 * is identical to phase 0 followed by phase 1. */
int lbm_step(lbm_handle* h, int n);

/* Issue one phase of one step on the handle's stream, without overlap:
 * 0 = bulk stream-collide, 1 = boundary conditions (band kernel,
 * zero-gradient copies; ends the step).  Used to time the phases
 * separately; a step is phase 0 then phase 1. */
int lbm_step_phase(lbm_handle* h, int phase);

/* Timing hook: record the caller's CUDA events (cudaEvent_t, created by the
 * caller with timing enabled) around the launches of every following
 * lbm_step() / lbm_step_phase() call, so that the dominant kernel can be
 * timed while the boundary phase runs beside it.  n = 0 turns the hook off;
 * n = 2 or 5:
 *   events[0], events[1]  before / after the bulk launch;
 *   events[2]             at the start of the step;
 *   events[3], events[4]  before / after the band launch (with the inflow
 *                         write of the first steps);
 * all on the handle's stream except events[3..4] in lbm_step(), which go
 * on the internal stream with the band launch.  The events stay owned by the
 * caller, who must keep them alive while the hook is set; with several steps
 * per call only the last step's records remain.  A NULL entry among the
 * first n is LBM_ERR_ARG. */
int lbm_set_kernel_events(lbm_handle* h, void* const* events, int n);

/* Limit of the bulk kernel's wait for each tensor copy (TMA) of its
 * populations, in seconds (default 1; 0 to 60; 0 tests once without
 * waiting, so that nearly every copy counts as late).  When a wait runs out the
 * kernel records it, waits again -- at most 1 s, whatever this limit -- for
 * the copies still in flight, so that none lands in the shared memory of a
 * CTA that has left, and leaves that row segment unwritten; the next
 * lbm_get_macros returns LBM_ERR_TIMEOUT.  The band kernel's cluster
 * exchanges (FP64 storage) keep their fixed 1 s limit: a CTA that gave up on
 * one could still receive other CTAs' stores after leaving.  A batch (lbm_batch_create)
 * takes the limit its runs have when it is created.  Synchronises the
 * stream. */
int lbm_set_wait_limit(lbm_handle* h, double seconds);

/* Macroscopic fields of the current populations (Eq. macro): absolute rho,
 * ux, uy and T ([ny][nx] doubles; T = 1 for D2Q9).  Device or host arrays as
 * on_device says.  Synchronises the stream.  Returns LBM_ERR_NUMERICAL (after
 * filling the arrays) if any value is not finite. */
int lbm_get_macros(lbm_handle* h, double* rho, double* ux, double* uy, double* T,
                   int on_device);

/* Checkpoint / resume: the populations, the boundary state and the step
 * counter, as an opaque host buffer of lbm_state_bytes() bytes.  Restoring a
 * state reproduces the continuation bit for bit. */
int lbm_state_bytes(const lbm_handle* h, size_t* bytes);
int lbm_get_state(lbm_handle* h, void* host_buf, size_t bytes);
int lbm_set_state(lbm_handle* h, const void* host_buf, size_t bytes);

/* Steps taken since lbm_init_fields (or restored with lbm_set_state). */
long long lbm_steps_done(const lbm_handle* h);

/* Text of the last error on h (never NULL; empty when none). */
const char* lbm_last_error(const lbm_handle* h);

/* Free everything the handle owns.  NULL is ignored. */
void lbm_destroy(lbm_handle* h);

/* ---------------------------------------------------------------------- */
/* Gradients with respect to the relaxation parameters                    */
/* ---------------------------------------------------------------------- */

/* The incoming-wave relaxation of Eqs. LODI-Relax and CBC-Relax has free
 * parameters the paper leaves to be chosen by hand: alpha_T (the transversal
 * terms), beta_P (P - P_inf on the acoustic waves), the target pressure P_inf
 * and the target transversal amplitude t_inf, and this library adds alpha_V
 * (the viscous term's relaxation towards 0).  These calls advance a handle by
 * tangent-linear steps: the step of the method (strip macros, RK4 of the
 * characteristic boundary state, equilibrium Dirichlet write, pull-stream +
 * BGK collide) evaluated together with its derivatives along three
 * directions in theta = (alpha_T, beta_P, P_inf, alpha_V, t_inf) (P_inf
 * moved on every characteristic side together), and accumulate the pressure
 * loss
 *     J = sum over the steps and over the nodes off the M boundary layers of
 *         (P - c_s^2 rho0 - dP_ref)^2,   P = rho c_s^2 T (D2Q9: rho c_s^2)
 * with its three directional derivatives.  Derivatives are exact up to
 * rounding (forward mode), in FP64 for the boundary state; populations and
 * their derivatives are held in the handle's storage precision.
 *
 * Supported: FP64 or FP32 storage, every viscous form (the vector frozen at
 * time t as in the ordinary step), the equilibrium Dirichlet condition,
 * characteristic and periodic sides (otherwise LBM_ERR_ARG).  Gradient steps use the handle's stream and
 * steps counter; afterwards the handle's ordinary step state (strips,
 * boundary state) is behind: lbm_step, lbm_step_phase, lbm_get_state and
 * batch steps return LBM_ERR_STATE until lbm_init_fields or lbm_set_state.
 * lbm_get_macros reads the populations the gradient steps produced. */

/* Allocate the derivative state (cudaMalloc: about 3 x the populations),
 * zero the derivatives and the sums, starting from the current state; the
 * three directions are d/dalpha_T, d/dbeta_P and d/dP_inf. */
int lbm_grad_begin(lbm_handle* h);

/* As lbm_grad_begin, with direction k = dirs[5 k .. 5 k + 4], a vector in
 * theta = (alpha_T, beta_P, P_inf, alpha_V, t_inf) (host array of 15
 * finite doubles, row-major [3][5]; NULL = the first three unit vectors). */
int lbm_grad_begin_along(lbm_handle* h, const double* dirs);

/* n tangent-linear steps (asynchronous).  dP_ref: NULL (reference 0) or a
 * device array holding, for step i of this call, the [ny][nx] doubles of
 * P_ref - c_s^2 rho0 at dP_ref + i * ref_stride. */
int lbm_grad_step(lbm_handle* h, int n, const double* dP_ref, long long ref_stride);

/* J and dJ[k] = the derivative of J along direction k (k = 0, 1, 2)
 * accumulated since lbm_grad_begin (synchronises the handle's stream). */
int lbm_grad_result(lbm_handle* h, double* J, double* dJ);

/* Free the derivative state.  NULL-safe on a handle without one. */
int lbm_grad_end(lbm_handle* h);

/* Reverse-mode (adjoint) gradients with segment checkpointing.  The same
 * pressure loss J as above, and its gradient with respect to all five
 * parameters theta = (alpha_T, beta_P, P_inf, alpha_V, t_inf) (P_inf moved
 * on every characteristic side together) in one backward pass.
 *
 * lbm_adj_forward advances the handle n ordinary steps (Fig.
 * flowchart-lbm-algo) and accumulates J, keeping a checkpoint of the state
 * every checkpoint_every steps.  lbm_adj_backward then sweeps the steps
 * backwards, segment by segment from the last: it restores the segment's
 * checkpoint, recomputes its steps keeping their macros, boundary states and
 * strips, and runs the adjoint of each step -- the Dirichlet write, the RK4
 * of the characteristic boundary state (Sec. 3.3; its right-hand side
 * differentiated in forward mode per boundary unknown), the viscous vector,
 * the strips, and the pull-stream + BGK collision of every bulk node
 * (Eqs. lbe, bgk) -- and leaves the handle in the state after the n steps.
 * Memory: one state per checkpoint plus the macros of checkpoint_every
 * steps, so long runs fit in device memory.  The gradient is exact up to
 * rounding; the boundary solver's arithmetic and the adjoint populations
 * are in the storage's precision (FP32 with FP32 storage), the parameter
 * gradient is accumulated in FP64.
 *
 * Supported: FP64 or FP32 storage, every viscous form, the equilibrium
 * Dirichlet condition, characteristic and periodic sides (otherwise
 * LBM_ERR_ARG).  Ordinary steps stay available: the forward pass is made of
 * them. */

/* Allocate the checkpoints and the adjoint state (cudaMalloc) for up to
 * max_steps forward steps with a checkpoint every checkpoint_every steps. */
int lbm_adj_begin(lbm_handle* h, int checkpoint_every, int max_steps);

/* n ordinary steps (n <= max_steps) with checkpoints; *J = the loss over
 * them (synchronises).  dP_ref: NULL (reference 0) or a device array holding,
 * for step i, the [ny][nx] doubles of P_ref - c_s^2 rho0 at dP_ref + i *
 * ref_stride; it is read again by lbm_adj_backward and must stay valid
 * until that returns. */
int lbm_adj_forward(lbm_handle* h, int n, const double* dP_ref, long long ref_stride, double* J);

/* dJ[0..4] = dJ/d(alpha_T, beta_P, P_inf, alpha_V, t_inf) of the last
 * lbm_adj_forward (synchronises); the handle ends in the state after the
 * forward steps. */
int lbm_adj_backward(lbm_handle* h, double* dJ);

/* Free the checkpoints and the adjoint state.  NULL-safe on a handle
 * without them. */
int lbm_adj_end(lbm_handle* h);

/* ---------------------------------------------------------------------- */
/* Batches: many independent runs stepped together                        */
/* ---------------------------------------------------------------------- */

typedef struct lbm_batch lbm_batch;

/* Create a batch of n independent runs -- lattices, grids, relaxation times
 * and boundary parameters may all differ (the paper tunes its relaxation
 * coefficients by such scans) -- each as lbm_create(lattice[r], nx[r],
 * ny[r], tau[r], &params[r]) would.  Every step of the batch then issues,
 * per lattice and storage, one band launch covering the boundary tiles of
 * all its runs and one persistent bulk launch whose CTAs loop over the row
 * segments of all its runs; after the first two steps each parity's step
 * is captured once as a CUDA graph and replayed.  The persistent kernel's
 * CTAs per SM are autotuned on the first step (fastest of 1..5) and cached
 * per device, lattice, storage and size bucket in the text file named by
 * the environment variable LBM_AUTOTUNE_CACHE (default
 * ~/.cache/lbm_cbc_autotune.txt; an empty value turns the cache off).  At
 * most 256 runs per lattice and storage.  Allocates with cudaMalloc. */
int lbm_batch_create(int n, const int* lattice, const int* nx, const int* ny, const double* tau,
                     const lbm_cbc_params* params, lbm_batch** out);

/* The handle of run r (owned by the batch): use it with lbm_init_fields,
 * lbm_get_macros, lbm_get_state and lbm_steps_done; stepping it alone
 * (lbm_step) puts it out of step with the batch, which lbm_batch_step then
 * rejects. */
int lbm_batch_run(lbm_batch* b, int r, lbm_handle** h);

/* Issue the batch's work, and that of every run, on stream (cudaStream_t). */
int lbm_batch_set_stream(lbm_batch* b, void* stream);

/* Advance every run n steps (asynchronous).  Every run must have been
 * initialised. */
int lbm_batch_step(lbm_batch* b, int n);

/* The autotuned CTAs per SM of the persistent bulk kernel for the runs of
 * one lattice and storage (0 before the first step or if there are none). */
int lbm_batch_ctas_per_sm(const lbm_batch* b, int lattice, int storage);

const char* lbm_batch_last_error(const lbm_batch* b);

/* Free the batch and its runs.  NULL is ignored. */
void lbm_batch_destroy(lbm_batch* b);

/* Allocation-free boundary step for one side.  The paper has no counterpart:
 * this exists for callers that cannot allocate device memory -- code running
 * inside another framework's memory pool, under a no-allocation policy, or
 * where cudaMalloc is not allowed at all -- but that hold the boundary data
 * themselves.  It advances the characteristic boundary state of ONE straight
 * CBC side (side index as above) whose tangential axis is periodic by one
 * time step: the same four RK4 stages lbm_step() runs, without writing
 * populations.
 *
 *   Ub        device, [length][M][4] doubles, in/out: the state of layers
 *             j = 1..M at each tangential position, as deviations
 *             (rho - rho0, u_x, u_y, T - 1); time t in, t + 1 out.
 *   strip_t   device, [3][length][4]: the same quantities on the bulk nodes
 *             at depths 0, 1, 2 inside the layers (x_f, x_f - n, x_f - 2n)
 *             at time t;  strip_t1: the same at time t + 1.
 *   neq_t     device, [3][length][9]: the nodes of the mesoscopic stencil,
 *             depths M, M + 1, M + 2 inside the layers (x_f - M n, ...), at
 *             time t: sigma'_xx, sigma'_xy, sigma'_yy, q_x, q_y, then
 *             rho - rho0, u_x, u_y, T - 1.  sigma' = -(1 - 1/(2 tau))
 *             sum_i c_i c_i (f_i - f_i^eq) and q = +(1 - 1/(2 tau)) 1/2
 *             sum_i (f_i - f_i^eq) |c_i - u|^2 (c_i - u), from the node's
 *             pulled (pre-collision) populations -- not the raw
 *             non-equilibrium moments.  Needed only when p->viscous is
 *             LBM_VISCOUS_MESO, otherwise may be NULL.
 *   stream    cudaStream_t (NULL = legacy default); the call is asynchronous.
 * tau is the BGK relaxation time.  Of p, only scheme[side], viscous,
 * alpha_T, beta_P, t_inf, alpha_V, p_inf[side] and rho0 are read.
 * length * M may not exceed 12288 (4096 positions on D2Q37 and D2Q17, 12288
 * on D2Q9); larger sides are rejected with LBM_ERR_ARG and a message on
 * stderr.
 *
 * Nothing is allocated: the RK4 stage scratch lives in one fixed ~1.6 MB
 * device array inside the library, held by every GPU that loads it until the
 * process exits.  The first call in a CUDA context looks that array's
 * address up (cudaGetSymbolAddress) and keeps it for that context, so make
 * that first call before any stream capture; a device reset that recreates
 * the primary context at the same address is not supported.  All calls share
 * the array and it keeps the last call's contents (every value a stage reads
 * is written earlier in the same call, so nothing needs clearing); calls
 * that overlap on the GPU -- on different streams, or from different
 * threads -- race on it and must be serialised by the caller. */
int lbm_cbc_side_step_noalloc(int lattice, int side, int length, double tau,
                              const lbm_cbc_params* p, double* Ub, const double* strip_t,
                              const double* strip_t1, const double* neq_t, void* stream);

/* Measured FP64 FMA throughput of the current device, in flop/s (an FMA
 * counts two): one timed launch of 8 CTAs of 256 threads per SM, each
 * thread running 8 independent register chains of `iters` FMAs (1 to 2^24),
 * after a short warm-up launch, on `stream` (a cudaStream_t; NULL = legacy
 * default).  The roof of the FP64 storage's ALU-bound bulk update.
 * Synchronises the stream; LBM_ERR_CUDA if a launch fails. */
int lbm_fp64_fma_rate(int iters, void* stream, double* flops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* LBM_CBC_H */
