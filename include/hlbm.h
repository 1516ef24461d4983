/*
 * hlbm.h -- C ABI of the B300 (sm_103a) HLBM mean-flow adjoint hot path.
 *
 * The library computes, on one GPU, the three steps of the paper's
 * Algorithm 1 (Ito et al., "Mean-Flow Adjoint Sensitivity Analysis of
 * Unsteady Flow Around Porous Cylinders Using a Homogenized Lattice
 * Boltzmann Method"):
 *   1. the primal homogenized LBM (Sec. 2.1, Eq. hlbm with the porous
 *      equilibrium; BGK or the recursive regularised collision of Sec. 2.2,
 *      Smagorinsky tau_eff) with on-device tracking averages (Sec. 3.3,
 *      Eq. averageObjective);
 *   2. the steady / mean-flow adjoint LBM (Eq. adjoint_steady,
 *      Eq. adjoint_unsteady), exact or frozen-turbulence (Sec. 5.4), by its
 *      fixed-point iteration or by restarted GMRES on the same fixed point;
 *   3. the gradient contraction dJ/dd (Eq. gradients_steady,
 *      Eq. gradients_unsteady)
 * for the far-field drag J_FFA (Sec. 4.2), the dissipation J_DISS
 * (Sec. 4.3) and the momentum-exchange drag J_MEA (Sec. 4.1); plus the
 * tangent-linear primal step of the exact transient sensitivities (App. C).
 *
 * Conventions (all entry points):
 *  - Lattice units (dx = dt = 1).  Grids are (nx, ny, nz), nz = 1 for D2Q9;
 *    cell index = x + nx*(y + ny*z) ("canonical order").  x = 0 is an
 *    equilibrium inflow node (uniform u_in, or the profile inflow_ux),
 *    x = nx-1 an outflow node; y and z are periodic.  nx >= 4, ny >= 1,
 *    nz >= 1, ny and nz <= 65535, nx * ny * nz < 2^31 - 64.
 *  - Multi-component fields are component-major: component c of cell k is
 *    at [c*N + k], N = nx*ny*nz.
 *  - Every call returns a status: HLBM_OK (0), HLBM_NOT_CONVERGED (1, a
 *    warning), or a negative error.  After an error other than HLBM_ECUDA
 *    the context stays usable; hlbm_last_error() gives a message.
 *  - Host pointers are only read/written during the call; no caller pointer
 *    is retained.  Device pointers (on_device = 1) must be device memory of
 *    the context's GPU, readable/writable by the context's stream.
 *  - A context is not thread-safe; it issues all work on one CUDA stream
 *    (the caller's, or its own).  Calls return after their GPU work is
 *    complete unless stated otherwise.
 *  - The library allocates device memory with cudaMalloc (or the caller's
 *    allocator hooks) at create time and lazily at the first adjoint solve.
 */
#ifndef HLBM_H
#define HLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hlbm_ctx hlbm_ctx;

enum { HLBM_D2Q9 = 9, HLBM_D3Q19 = 19 };

/* population storage (precision forms of the populations) */
enum {
  HLBM_FP64 = 0,    /* double storage and double arithmetic */
  HLBM_FP32 = 1,    /* float storage, float arithmetic */
  HLBM_FP16DEV = 2, /* IEEE half storage of f_i - w_i, float arithmetic */
  HLBM_BF16DEV = 3  /* bfloat16 storage of f_i - w_i, float arithmetic */
};

/* objectives: bit mask for accumulation, single value for solve/gradient.
 * HLBM_OBJ_DRAG_MEA is the momentum-exchange drag of Sec. 4.1 over the
 * fluid-side surface nodes (d >= 1/2 next to d < 1/2), flow direction x,
 * normalised by the number of surface nodes; it is linear in f, so its
 * average is taken as J(f_bar) and its derivative is constant (averaging it
 * turns on average_full_f); the surface set is held fixed (dJ/dd = 0). */
enum { HLBM_OBJ_DRAG_FFA = 1, HLBM_OBJ_DISSIPATION = 2, HLBM_OBJ_DRAG_MEA = 4 };

/* collision model: BGK (Sec. 2.1, Eq. 2; Smagorinsky tau_eff when Cs > 0) or
 * the third-order recursive regularised collision of the turbulent model
 * (Sec. 2.2, Eq. HRRLBM): f* = f^eq3(rho, u~) + (1 - 1/tau_eff) f^(1), f^eq3
 * the third-order Hermite equilibrium and f^(1) the non-equilibrium part
 * expanded to third order with the recursive third-order coefficient
 * u~ (x) Pi.  Its averages keep the second moments of f instead of f itself,
 * and its adjoint reads only (rho, u, Pi) of f_bar.  The tangent-linear step
 * supports BGK only. */
enum { HLBM_COLL_BGK = 0, HLBM_COLL_RR = 1 };

/* adjoint linearisation: full Jacobian or frozen turbulence (Sec. 5.4) */
enum { HLBM_ADJ_EXACT = 0, HLBM_ADJ_FTA = 1 };

/* element types of caller buffers */
enum { HLBM_DTYPE_F64 = 0, HLBM_DTYPE_F32 = 1 };

/* fields for hlbm_get_field / hlbm_set_field */
enum {
  HLBM_FIELD_RHO = 0,    /* get: density of the current canonical state (N) */
  HLBM_FIELD_U = 1,      /* get: velocity u = sum xi f / rho (dim x N) */
  HLBM_FIELD_F = 2,      /* get/set: canonical populations (q x N) */
  HLBM_FIELD_FBAR = 3,   /* get/set: averaged populations (q x N); get needs
                            average_full_f or Cs > 0 */
  HLBM_FIELD_GBAR_FFA = 4,   /* get/set: averaged dJ_FFA/df (q x N) */
  HLBM_FIELD_GBAR_DISS = 5,  /* get/set: averaged dJ_DISS/df (q x N); both are kept
                                as coefficients of a quadratic polynomial in xi
                                (the form every objective derivative has), so a
                                set value is projected onto that form */
  HLBM_FIELD_DJDD_FFA = 6,   /* get/set: averaged dJ_FFA/dd (N) */
  HLBM_FIELD_DJDD_DISS = 7,  /* get/set: averaged dJ_DISS/dd (N) */
  HLBM_FIELD_TAU_T = 8,      /* get/set: averaged tau_eff - tau0 (N) */
  HLBM_FIELD_LAMBDA = 9,     /* get: mu = S^T B^T lambda (q x N), the adjoint pulled
                                back through streaming and the boundary nodes, i.e.
                                the vector contracted with dC/dd in the gradient */
  HLBM_FIELD_POROSITY = 10   /* get: porosity d (N) */
};

enum {
  HLBM_OK = 0,
  HLBM_NOT_CONVERGED = 1, /* adjoint hit max_iter; results are the last iterate */
  HLBM_EINVAL = -1,       /* bad argument */
  HLBM_ENOMEM = -2,       /* device allocation failed */
  HLBM_ESTATE = -3,       /* call out of order (e.g. adjoint before primal) */
  HLBM_ECUDA = -4,        /* CUDA runtime error; context unusable */
  HLBM_ENONFINITE = -5,   /* NaN/Inf or non-positive density detected */
  HLBM_EDIVERGED = -6,    /* adjoint residual grew by > 1e6 over its minimum */
  HLBM_ETIMEOUT = -7,     /* reserved: bounded device wait expired */
  HLBM_ESCRATCH = -8      /* problem needs more than a fixed scratch area holds */
};

typedef struct {
  int storage;          /* HLBM_FP64 / FP32 / FP16DEV / BF16DEV (default FP32) */
  double u_in;          /* inflow velocity (default 0.05) */
  double u_solid[3];    /* solid velocity u_s blended by (1 - d) (default 0) */
  double tau_adj;       /* adjoint relaxation time replacing tau0 in the
                           linearised operator (Sec. 5.4); 0 = tau0 */
  int objectives;       /* mask of objectives averaged during the window */
  int ffa_x;            /* x index of the far-field plane Gamma_J */
  int ffa_y0, ffa_y1;   /* y extent [y0, y1) of Gamma_J */
  int ffa_z0, ffa_z1;   /* z extent [z0, z1) of Gamma_J */
  int diss_box[6];      /* Omega_J: x0, x1, y0, y1, z0, z1 (half-open) */
  int design_box[6];    /* Omega_alpha: region returned by hlbm_gradient */
  int accum_stride;     /* sample every k-th step of the window (>= 1) */
  int check_every;      /* adjoint residual check interval, even (>= 2) */
  int average_full_f;   /* 1: also average all q populations (HLBM_FIELD_FBAR);
                           always on when Cs > 0, where the exact LES adjoint
                           linearises at f_bar itself.  Otherwise only the
                           density and momentum of f are averaged, which is
                           all the BGK / frozen-turbulence linearisation reads */
  int block_x;          /* threads per block along x of the step kernels: 32, 64
                           or 128; 0 = chosen from the grid size */
  int adjoint_solver;   /* 0: the paper's fixed-point iteration of the adjoint
                           sweep; 1: restarted GMRES on the same fixed point
                           (operator = two sweeps), same stopping criterion */
  int gmres_restart;    /* Krylov basis size of solver 1 (default 30, <= 64) */
  int gmres_inner;      /* pairs of sweeps per operator application of solver 1
                           (>= 1; default 100): GMRES then solves
                           (I - M^(2k)) mu = c_k, the same fixed point with the
                           fast modes pre-damped */
  void* stream;         /* cudaStream_t to issue work on; NULL = own stream */
  void* (*dev_alloc)(size_t bytes, void* user); /* NULL = cudaMalloc */
  void (*dev_free)(void* ptr, void* user);      /* NULL = cudaFree */
  void* alloc_user;
  int collision;        /* HLBM_COLL_BGK (default) or HLBM_COLL_RR; fixed at
                           hlbm_create (hlbm_configure rejects a change) */
  const double* inflow_ux; /* optional host array of ny * nz values (y fastest):
                           u_x of the inflow node f^eq(1, u_x e_x) per row, e.g.
                           a parabolic channel profile; NULL = uniform u_in.
                           Copied by hlbm_create / hlbm_configure (|u_x| < 0.5,
                           else HLBM_EINVAL); u_in stays the reference velocity
                           of J_FFA. */
  int adjoint_warm_start; /* 1: an adjoint solve starts from the adjoint array as
                           the previous solve on this context left it (its
                           lambda for another porosity, Re or window) instead of
                           from lambda = 0: the same fixed point and stopping
                           criterion, reached from a nearby start when a stream
                           of similar problems runs on one context.  No effect
                           before the context's first solve.  Default 0. */
} hlbm_options;

/* Velocity set of the library's direction order: xi (q x 3 ints, may be
 * NULL) and weights w (q doubles, may be NULL).  Returns q (9 or 19) or
 * HLBM_EINVAL.  Population fields (HLBM_FIELD_F, FBAR, GBAR_*, LAMBDA) are
 * indexed in this order. */
int hlbm_velocity_set(int lattice, int* xi, double* w);

/* Fill *opt with defaults for a grid of dims[3] (regions: Gamma_J at
 * x = nx/2 over the full height, Omega_J and Omega_alpha the whole domain,
 * both objectives, stride 1, check every 100 iterations). */
void hlbm_default_options(hlbm_options* opt, const int dims[3]);

/* Create a context: lattice HLBM_D2Q9 or HLBM_D3Q19, grid dims[3],
 * molecular relaxation time tau > 0.5 (nu = (tau - 1/2)/3, Sec. 2.1),
 * Smagorinsky constant Cs >= 0 (0 = plain BGK; Sec. 2.2).  The state is
 * set to f = f^eq(1, u_in e_x) and the porosity to 1.  opt may be NULL
 * (defaults).  On error *out is NULL. */
int hlbm_create(hlbm_ctx** out, int lattice, const int dims[3], double tau,
                double Cs, const hlbm_options* opt);

/* Change the physical parameters of an existing context without
 * reallocating it: relaxation time tau, Smagorinsky constant Cs and, from
 * opt (may be NULL), u_in, u_solid, tau_adj, objectives, the regions,
 * accum_stride, check_every, average_full_f, the adjoint solver settings
 * (adjoint_solver, gmres_*, adjoint_warm_start) and the inflow profile (NULL
 * restores the uniform inflow); storage, stream, allocator, block_x and
 * collision keep their creation values (a different collision is
 * HLBM_EINVAL).  Clears the averages and the adjoint result (the adjoint
 * array itself stays, as the start of a warm-started solve); the state and
 * the porosity are kept.  Arguments are checked before anything changes,
 * so an HLBM_EINVAL leaves the context as it was.  Lets a server reuse a
 * context (and its captured graphs) for a new request of the same grid. */
int hlbm_configure(hlbm_ctx* ctx, double tau, double Cs, const hlbm_options* opt);

/* Set the lattice porosity d(x) in [0, 1] (Sec. 2.1; the control of
 * Sec. 3.1), N values of dtype, host or device.  Values outside [0, 1]
 * or non-finite give HLBM_EINVAL (checked on the device). */
int hlbm_set_porosity(hlbm_ctx* ctx, const void* d, int dtype, int on_device);

/* Initialise the state to f = f^eq(rho, u) with the inflow/outflow nodes
 * applied.  rho (N) may be NULL (= 1); u (dim x N) may be NULL
 * (= u_in e_x).  Clears averages and the step counter. */
int hlbm_init_equilibrium(hlbm_ctx* ctx, const void* rho, const void* u,
                          int dtype, int on_device);

/* Advance `steps` time steps.  The last `avg_window` steps (1 <= avg_window
 * <= steps; 0 = no averaging) sample the canonical state they start from
 * every accum_stride-th step into the running averages of f, J, dJ/df,
 * dJ/dd and tau_eff - tau0 (a new window restarts the averages).
 * avg_window = 1 is the steady case.  Returns HLBM_ENONFINITE if the state
 * became non-finite. */
int hlbm_run_primal(hlbm_ctx* ctx, long steps, long avg_window);

/* Forward (tangent-linear) sensitivity along the primal trajectory, the
 * quantity whose growth App. C of the paper studies: advances the state
 * `steps` steps together with its derivative f' = (df/dd) . delta along the
 * porosity direction delta (N values of dtype, host or device), from f' = 0,
 * and writes to jdot_out[n] (host, `steps` doubles) the derivative
 * dJ/dd . delta of the instantaneous objective at the canonical state each
 * step starts from.  The state advances as in hlbm_run_primal; averages and
 * the adjoint are cleared. */
int hlbm_run_tangent(hlbm_ctx* ctx, long steps, const void* delta, int dtype, int on_device,
                     int objective, double* jdot_out);

/* Time-averaged objective J_bar over the last window (HLBM_ESTATE if the
 * objective was not in the accumulation mask or no window was run). */
int hlbm_objective(hlbm_ctx* ctx, int objective, double* J_out);

/* Solve the adjoint lambda = A^T lambda + g_bar, A the step Jacobian at
 * the averaged state (Eq. adjoint_unsteady; Eq. adjoint_steady for window
 * 1), from lambda = 0, until ||lambda^{k+1} - lambda^k||_2 / ||g_bar||_2
 * <= tol (checked every check_every iterations) or max_iter iterations.
 * With opt.adjoint_solver = 1 the fixed point is reached by restarted GMRES
 * (max_iter then bounds the adjoint sweeps it applies, 2 gmres_inner per
 * Krylov step; restarts that take less than 5 % off the true residual over
 * 4000 sweeps end the pass) and the criterion is evaluated on its result; when it
 * misses tol, GMRES goes on from that iterate with a proportionally tighter
 * Krylov tolerance until the criterion holds, max_iter is reached or a pass
 * no longer halves it (the rounding floor: HLBM_NOT_CONVERGED).
 * mode is HLBM_ADJ_EXACT or HLBM_ADJ_FTA.  iters_out / residual_out may
 * be NULL.  Returns HLBM_NOT_CONVERGED at max_iter, HLBM_EDIVERGED or
 * HLBM_ENONFINITE on blow-up. */
int hlbm_solve_adjoint(hlbm_ctx* ctx, int objective, int mode, double tol,
                       long max_iter, long* iters_out, double* residual_out);

/* Gradient dJ/dd over the design box, x fastest (Eq. gradients_unsteady),
 * for the objective of the last solve: dJ/dd_bar + sum_i mu_i dC_i/dd.
 * out holds box-volume values of dtype, host or device. */
int hlbm_gradient(hlbm_ctx* ctx, void* out, int dtype, int on_device);

/* Read a field (see HLBM_FIELD_*) in canonical order into out. */
int hlbm_get_field(hlbm_ctx* ctx, int which, void* out, int dtype, int on_device);

/* Overwrite the state (HLBM_FIELD_F) or an averaged field (FBAR, GBAR_*,
 * DJDD_*, TAU_T; the sample count becomes 1).  Used to feed the same
 * averaged state to the adjoint that another implementation produced. */
int hlbm_set_field(hlbm_ctx* ctx, int which, const void* data, int dtype, int on_device);

/* Counters of the work done so far and the GPU time of the two hot loops,
 * measured with CUDA events on the context's stream. */
typedef struct {
  long primal_steps;      /* total primal steps run */
  long adjoint_iters;     /* adjoint iterations of the last solve */
  double primal_ms;       /* GPU time of the last hlbm_run_primal */
  double adjoint_ms;      /* GPU time of the last hlbm_solve_adjoint */
  long primal_launches;   /* kernel launches of the last run_primal */
  long adjoint_launches;  /* kernel launches of the last solve */
  double primal_bytes_per_lup_plain;  /* algorithmic bytes of a plain step */
  double adjoint_bytes_per_lup;       /* algorithmic bytes of an iteration */
  long kernels_total;     /* all kernels this context launched since creation */
} hlbm_stats;
int hlbm_get_stats(const hlbm_ctx* ctx, hlbm_stats* out);

/* Checkpoint the state, averages and step counter to a file / restore them
 * into a context created with the same lattice, dims and storage. */
int hlbm_save(hlbm_ctx* ctx, const char* path);
int hlbm_load(hlbm_ctx* ctx, const char* path);

/* Message of the last error on this context (never NULL). */
const char* hlbm_last_error(const hlbm_ctx* ctx);

/* Release all device memory and the own stream.  NULL is a no-op. */
void hlbm_destroy(hlbm_ctx* ctx);

/* ---------------------------------------------------------------------
 * Batched stepping (the serving form of the path).  Several contexts, each
 * with its own grid, porosity, parameters and device state, advance together:
 * every primal step (adjoint sweep) of all of them is one kernel launch over a
 * device work list of (context, x-block, y, z) tiles, each block reading its
 * context's arguments from a device table.  Small grids that cannot fill the
 * GPU alone then share launches, and a launch's fixed cost is paid once per
 * step for the whole batch.  Per context, the arithmetic, the order of every
 * reduction and the block decomposition are those of the single-context
 * calls, so a context's results are bitwise the same whether it is stepped
 * alone (hlbm_run_primal / hlbm_solve_adjoint) or in any batch.
 *
 * A batch holds contexts created on the batch's stream with the batch's
 * lattice, FP32 storage, BGK collision with Cs = 0, block_x = 128,
 * accum_stride 1, the fixed-point adjoint solver, no J_MEA and averages of
 * the moments only (average_full_f = 0), all at the same AA phase (every
 * context that has run the same parity of steps; an even number of steps
 * keeps it); others give HLBM_EINVAL.  The batch owns only its tables and work
 * list (device memory it allocates as it grows); the contexts keep their
 * state.
 *
 * hlbm_batch_create: lattice HLBM_D2Q9 or HLBM_D3Q19, stream (cudaStream_t,
 *   not NULL) that the member contexts were created on.
 * hlbm_batch_run_primal: hlbm_run_primal(ctx, steps, avg_window) for each of
 *   ctxs[0..n), in one launch per step.  Returns HLBM_ENONFINITE if any
 *   state became non-finite (that context's last error says so).
 * hlbm_batch_solve_adjoint: hlbm_solve_adjoint(ctxs[k], objectives[k], mode,
 *   tol, max_iter) for each k, in one launch per sweep over the contexts still
 *   iterating (a context leaves the work list when it converges, diverges or
 *   becomes non-finite; the residual is checked every check_every sweeps of
 *   ctxs[0]).  iters_out, residual_out, status_out (n entries each, may be
 *   NULL) receive each context's results; the return value is the worst
 *   status (a negative one, else HLBM_NOT_CONVERGED if any, else HLBM_OK).
 *   hlbm_gradient then reads each context's gradient.
 * --------------------------------------------------------------------- */
typedef struct hlbm_batch hlbm_batch;
int hlbm_batch_create(hlbm_batch** out, int lattice, void* stream);
int hlbm_batch_run_primal(hlbm_batch* batch, hlbm_ctx* const* ctxs, int n, long steps,
                          long avg_window);
int hlbm_batch_solve_adjoint(hlbm_batch* batch, hlbm_ctx* const* ctxs, int n,
                             const int* objectives, int mode, double tol, long max_iter,
                             long* iters_out, double* residual_out, int* status_out);
void hlbm_batch_destroy(hlbm_batch* batch);

/* ---------------------------------------------------------------------
 * Objective evaluation without allocation.  The paper has no counterpart
 * to this entry point; it exists for callers that must not allocate device
 * memory (a component inside a fixed memory arena or pool that may not
 * grow, a latency-critical loop where an allocation's implicit device
 * synchronisation is not acceptable, or a plug-in host that forbids its
 * plug-ins to allocate).  It needs no context.
 *
 * Evaluates objective HLBM_OBJ_DRAG_FFA or HLBM_OBJ_DISSIPATION of the
 * canonical population field f (q x N doubles, device, direction order of
 * hlbm_velocity_set) with porosity d (N doubles, device) over `region`
 * (x0, x1, y0, y1, z0, z1, half-open; for the drag a plane, x1 = x0 + 1),
 * with the same definitions as the averages of hlbm_run_primal.  Writes J
 * (one double, device) and, when not NULL, dJ/df (q x N, device) and dJ/dd
 * (N, device) at the cells of the region; other cells are not written.
 * tau, Cs, u_in and u_solid (may be NULL = 0) are as in hlbm_create.  Work
 * is enqueued on `stream` (cudaStream_t, NULL = legacy default stream); the
 * call returns without waiting for it.
 *
 * No cudaMalloc / cudaFree or other allocating call is made.  Scratch is a
 * fixed device array of HLBM_NOALLOC_MAX_BLOCKS doubles (512 KiB per GPU,
 * held until the process exits) shared by all calls: a region of more than
 * HLBM_NOALLOC_MAX_BLOCKS blocks (ceil((x1-x0)/128) * (y1-y0) * (z1-z0))
 * returns HLBM_ESCRATCH.  Calls that overlap on the GPU race on the scratch
 * array; order them on one stream.  The first call on a device looks up
 * the scratch address (cudaGetSymbolAddress, that device current); make it
 * before any stream capture.  The address is kept for the life of the
 * process: after a cudaDeviceReset of that device the kept address is stale,
 * so do not call this entry point on a device that has been reset.  Errors: HLBM_EINVAL (bad argument),
 * HLBM_ESCRATCH, HLBM_ECUDA.
 * --------------------------------------------------------------------- */
#define HLBM_NOALLOC_MAX_BLOCKS 65536
int hlbm_objective_noalloc(int lattice, const int dims[3], double tau, double Cs, double u_in,
                           const double u_solid[3], int objective, const int region[6],
                           const double* f, const double* d, double* J, double* dJdf,
                           double* dJdd, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HLBM_H */
