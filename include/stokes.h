/*
 * stokes.h -- C ABI of libstokes_gb300, a single-GPU (GB300, sm_103a) solver
 * for the variable-density, variable-viscosity staggered-grid Stokes system
 *
 *     M x = b,   M = [ A  G ]      A = theta rho - L_mu,   theta = 1/dt
 *                    [ -D 0 ]
 *
 * of Cai, Nonaka, Bell, Griffith & Donev, "Efficient Variable-Coefficient
 * Finite-Volume Stokes Solvers" (arXiv:1308.4605), Eq. Saddle_sys of Sec. 2
 * with the MAC discretisation of Sec. 3.1, solved by GMRES (Sec. 3.2, Sec. 4)
 * preconditioned by the block preconditioners P1..P5 of Sec. 2, each of
 * which applies one geometric-multigrid V-cycle (App. C) to the velocity and
 * to the pressure subproblem.
 *
 * Data layout (all arrays are caller-owned DEVICE memory, FP64, contiguous):
 *   cell arrays   nz * ny * nx doubles, x fastest (nz = 1 in 2D);
 *                 cell (i,j,k) is centred at ((i+1/2)h, (j+1/2)h, (k+1/2)h).
 *   face arrays   one per velocity component a; same shape except that the
 *                 extent along axis a is n_a + 1 when axis a has walls (faces
 *                 0 and n_a lie on the walls; the library writes zeros there
 *                 and ignores what it finds there) and n_a when it is
 *                 periodic.  Face i of component a lies at x_a = i h.
 * Right-hand side convention (Eq. Saddle_sys):  b_u = rho u^n / dt + f,
 * b_p = -g where g is the prescribed velocity divergence.
 *
 * Every call returns STK_OK (0) or a negative STK_ERR_* code; the message of
 * the last failure on a handle is returned by stk_last_error.  Calls are
 * asynchronous on the given stream (a cudaStream_t passed as void*, NULL for
 * the legacy default stream) except stk_create, stk_destroy,
 * stk_set_coefficients (which validates its inputs) and stk_solve (which
 * returns when the solve is finished and info is written).
 * The library owns all workspace (multigrid hierarchy, Krylov basis) and
 * allocates it in stk_create / stk_set_coefficients / the first stk_solve.
 * A handle is used from one host thread at a time.
 */
#ifndef STOKES_GB300_H
#define STOKES_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

/* boundary condition codes, one per side: x_lo, x_hi, y_lo, y_hi, z_lo, z_hi
 * (Sec. 3.1: periodic, no-slip u = 0, free-slip u.n = 0 with zero tangential
 * stress).  Periodic must be set on both sides of an axis. */
#define STK_PERIODIC 0
#define STK_NOSLIP   1
#define STK_FREESLIP 2

/* return codes */
#define STK_OK                 0
#define STK_ERR_ARG           -1  /* bad argument (null pointer, bad code)       */
#define STK_ERR_SIZE          -2  /* n_a not a power of two >= 2                 */
#define STK_ERR_CUDA          -3  /* a CUDA runtime call failed                  */
#define STK_ERR_NOT_CONVERGED -4  /* maxit reached; x holds the last iterate     */
#define STK_ERR_NONFINITE     -5  /* NaN/Inf in coefficients or in the iteration */
#define STK_ERR_TIMEOUT       -6  /* a bounded device wait expired               */
#define STK_ERR_STATE         -7  /* coefficients not set                        */

/* preconditioners (Sec. 2.1-2.4) */
#define STK_P1 1  /* projection, Eq. P1_practical        */
#define STK_P2 2  /* lower triangular, Eq. CC_Pre_lower  */
#define STK_P3 3  /* upper triangular, Eq. CC_Pre_upper  */
#define STK_P4 4  /* block diagonal, Eq. CC_Pre_diagonal */
#define STK_P5 5  /* Uzawa-like, Sec. 2.4                */

/* precision of the solve */
#define STK_FP64  0  /* left-preconditioned GMRES(m), everything in FP64 (Sec. 3.2)      */
#define STK_MIXED 1  /* flexible GMRES(m) in FP64 around an FP32 preconditioner (Sec. 4) */

typedef struct stk_handle stk_handle;

typedef struct {
    int    precond;    /* STK_P1..STK_P5                                            */
    int    restart;    /* GMRES restart length m (paper: 10, Sec. 4.2.2), 1..32     */
    double rtol;       /* stop when ||b - M x||_2 <= rtol ||b||_2                   */
    int    maxit;      /* maximum number of Arnoldi steps                           */
    int    precision;  /* STK_FP64 or STK_MIXED                                     */
    int    nu;         /* smoothing sweeps before and after the coarse correction (2) */
    int    ncoarse;    /* sweeps on the coarsest level (8, App. C).  The 8 sweeps
                        * from zero are a fixed linear map; with at most 1024
                        * coarsest unknowns it is formed at stk_set_coefficients
                        * and applied as a matrix (the same map up to rounding);
                        * other counts sweep                                      */
    int    vcycles_u;  /* V-cycles per velocity subsolve (1; 1..64): the first from
                        * zero, each further one on the residual, x += V(r - A x)
                        * (the number of multigrid cycles of Sec. 4.1.2)           */
    int    vcycles_p;  /* the same for the pressure subsolve (1; 1..64), residual
                        * projected onto mean-zero vectors                         */
} stk_solver_params;

typedef struct {
    int    iterations;     /* Arnoldi steps (= applications of M and of P^{-1})     */
    int    restarts;       /* GMRES cycles                                           */
    int    converged;      /* 1 when ||b - M x|| <= rtol ||b||                       */
    int    status;         /* return code of the solve                               */
    double true_residual;  /* final ||b - M x|| / ||b|| (computed in FP64)           */
    double est_residual;   /* last Arnoldi residual estimate                         */
    double scalar_vcycles; /* cost proxy of Sec. 4: d per velocity, 1 per pressure V-cycle */
    double solve_ms;       /* wall time of the solve on the stream                   */
} stk_solve_info;

/* Default parameters: P1, m = 10, rtol = 1e-10, maxit = 1000, FP64, nu = 2,
 * ncoarse = 8, one V-cycle per subsolve (Sec. 4.1.1, 4.1.2, 4.2.2, App. C). */
void stk_default_params(stk_solver_params* p);

/* Create a grid of dim (2 or 3) dimensions with n[0..dim-1] cells per axis,
 * spacing h > 0 and boundary codes bc[0..2*dim-1].  Each n_a must be a power
 * of two >= 2 so that coarsening by 2 reaches 2 cells along the shortest
 * axis (App. C).  Uses the current CUDA device.  *out is NULL on failure. */
int stk_create(int dim, const int* n, double h, const int* bc, stk_handle** out);

/* Stacked batch: `count` independent 2D systems on the same grid (n, h, bc
 * as in stk_create, dim must be 2), each with its own coefficients and
 * right-hand side, stored as instances along a third array axis: every face
 * and cell array of the handle holds the count instances one after another
 * (instance i of the a-face array at i * stk_face_length(h, a) / count, of
 * a cell array at i * stk_cell_length(h) / count).  No stencil couples two
 * instances, so each is the 2D system of Sec. 3.1 on its own: every kernel
 * of a V-cycle, of the operator and of the preconditioner runs once over
 * all instances, the reductions and the GMRES least-squares problems
 * (Sec. 3.2) per instance, and an instance's results equal those of a
 * handle made by stk_create for it alone: bitwise for the operator,
 * V-cycles, preconditioners and solves whenever the coarsest level runs in
 * the coarse-level kernel (as in the default schedules: each instance then
 * applies its own precomputed coarse-solve matrix, like a single handle) or
 * sweeps (ncoarse != 8); to rounding when a stacked handle sweeps a
 * coarsest level that a single handle applies as a matrix.  stk_solve on the handle solves every instance, one
 * CUDA graph launch per GMRES cycle for all of them; an instance that has
 * converged sits out the rest of the solve and its solution is final.  The
 * solve's info summarises the instances (iterations, restarts, residuals
 * and V-cycles: the largest; converged: all of them); stk_stack_info gives
 * each.  x receives every instance's final iterate also when the solve
 * returns STK_ERR_NONFINITE or STK_ERR_TIMEOUT for one of them (the others
 * are unaffected).  1 <= count <= STK_MAX_STACK.  Not available on a stacked handle:
 * stk_set_bulk_viscosity, stk_subtract_boundary_terms, stk_gradient and the
 * persistent multi-block V-cycle (schedule grid_level). */
#define STK_MAX_STACK 1024
int stk_create_stacked(int dim, const int* n, double h, const int* bc, int count, stk_handle** out);
/* Instances of a stacked handle (1 for a handle from stk_create). */
int stk_stack_count(const stk_handle* h);
/* The last solve's record of one instance (0 <= instance < count):
 * converged, iterations, restarts, residuals, V-cycles and status of that
 * instance, solve_ms of the whole solve.  STK_ERR_STATE before any solve. */
int stk_stack_info(const stk_handle* h, int instance, stk_solve_info* info);
/* stk_solve_history for one instance. */
int stk_stack_history(const stk_handle* h, int instance, int kind, double* out, int cap);

/* Free the handle and every device allocation it owns. */
int stk_destroy(stk_handle* h);

/* Message of the last failure on h (h may be NULL for a failed stk_create). */
const char* stk_last_error(const stk_handle* h);

/* Number of doubles in the face array of component a (0 <= a < dim) and in a
 * cell array. */
long long stk_face_length(const stk_handle* h, int a);
long long stk_cell_length(const stk_handle* h);

/* Set the cell-centred density rho > 0 and viscosity mu >= 0 (device arrays,
 * copied) and dt (theta = 1/dt; dt = +INFINITY gives steady flow, theta = 0).
 * Builds the face densities (Sec. 3.1: mean of the two adjacent cells), the
 * node/edge viscosities (mean of the surrounding in-domain cells) and the
 * coarse-level coefficients of the velocity and pressure multigrid hierarchy
 * (App. C), in FP64 and FP32.  Synchronises the stream.  Returns
 * STK_ERR_NONFINITE / STK_ERR_ARG for non-finite or non-positive inputs. */
int stk_set_coefficients(stk_handle* h, const double* rho, const double* mu, double dt,
                         void* stream);

/* Bulk-viscosity stress form (Sec. 2): tau = mu (grad u + grad u^T) +
 * (gamma - 2/3 mu)(div u) I, for flows with div u = g != 0.  gamma: device
 * cell array of bulk viscosities >= 0 (copied), or NULL to return to the
 * stress form without the bulk term.  Call after stk_set_coefficients; the
 * setting persists through later stk_set_coefficients calls.  The operator,
 * the smoothers (coarse levels average lam = gamma - 2/3 mu over the fine
 * cells, like mu) and the Schur approximation -theta L_rho^{-1} +
 * (gamma + 4/3 mu) (Eq. Schur_app_bulk) all use it; stk_gradient then
 * returns STK_ERR_STATE.  Errors: STK_ERR_STATE (no coefficients),
 * STK_ERR_NONFINITE, STK_ERR_ARG (gamma < 0).  Synchronises the stream. */
int stk_set_bulk_viscosity(stk_handle* h, const double* gamma, void* stream);

/* y = M x  (Eq. Saddle_sys): y_u = theta rho_f x_u - L_mu x_u + G x_p and
 * y_p = -D x_u, with the stress-form viscous operator of Eq. div_stress.
 * x_u[a], y_u[a] are face arrays, x_p, y_p cell arrays; y must not alias x. */
int stk_apply_operator(stk_handle* h, const double* const* x_u, const double* x_p,
                       double* const* y_u, double* y_p, void* stream);

/* x = P^{-1} b for which = STK_P1..STK_P5 (Sec. 2.1-2.4) in FP64: one velocity
 * V-cycle per velocity subsolve, one pressure V-cycle per pressure subsolve,
 * zero initial guesses (Sec. 3.2), S~^{-1} = -theta L~_rho^{-1} + 2 mu
 * (Eq. Schur_app_varDen_varVis).  The mean of every Poisson right-hand side
 * and of x_p is removed. */
int stk_apply_preconditioner(stk_handle* h, int which, const double* const* b_u,
                             const double* b_p, double* const* x_u, double* x_p,
                             void* stream);

/* The same with the subsolver settings of params (precond, precision, nu,
 * ncoarse, vcycles_u, vcycles_p; the Krylov fields are ignored).  With
 * precision STK_MIXED the preconditioner runs in FP32 on the FP32
 * coefficient hierarchy (inputs rounded to FP32, outputs widened to FP64),
 * as inside the flexible solve. */
int stk_apply_preconditioner_params(stk_handle* h, const stk_solver_params* params,
                                    const double* const* b_u, const double* b_p,
                                    double* const* x_u, double* x_p, void* stream);

/* One velocity V-cycle for A x = r (x = A~^{-1} r, zero initial guess, App. C)
 * and one pressure V-cycle for L_rho x = r (x = L~_rho^{-1} r), in FP64. */
int stk_velocity_vcycle(stk_handle* h, const double* const* r_u, double* const* x_u,
                        void* stream);
int stk_pressure_vcycle(stk_handle* h, const double* r_p, double* x_p, void* stream);

/* Solve M x = b with restarted GMRES (Sec. 3.2, Sec. 4).  x_u, x_p hold the
 * initial guess on entry and the solution on exit.  info may be NULL.
 * Returns STK_OK, STK_ERR_NOT_CONVERGED (x holds the last iterate) or an
 * error code.  Synchronises the stream. */
int stk_solve(stk_handle* h, const stk_solver_params* params, const double* const* b_u,
              const double* b_p, double* const* x_u, double* x_p, stk_solve_info* info,
              void* stream);

/* Inhomogeneous velocity boundary conditions (Sec. 3.2: the viscous
 * stencils next to a wall use the prescribed values, so the operator is
 * affine; the Krylov solver works on the homogeneous problem after the
 * boundary terms are subtracted from the right-hand side):
 *   b_u -= c_u,  b_p -= c_p,   with M x + c the operator with boundary data,
 * for the Stokes operator and coefficients set on h (bulk term included).
 * u_wall: NULL, or dim face arrays whose wall faces (the a-faces at index 0
 *   and n_a of a non-periodic axis a) hold the prescribed normal velocity;
 *   other entries are ignored (a NULL entry means zero).
 * u_tan: NULL, or 18 pointers, u_tan[3 * (2 d + side) + a] for the wall of
 *   axis d (side 0 low, 1 high) and component a != d: the prescribed
 *   tangential velocity on that wall at the positions of the a-faces, an
 *   array with the extents of the a-face array with axis d removed (x
 *   fastest); NULL means zero.  Only no-slip walls use it (a free-slip wall
 *   has zero shear stress).
 * The solution of M x = b' is then the interior field; its wall faces are
 * the prescribed normal velocities.  With walls all around, the net normal
 * flux must match the integral of g (the pressure right-hand side must have
 * zero mean).  Stream-ordered, no synchronisation. */
int stk_subtract_boundary_terms(stk_handle* h, const double* const* u_wall,
                                const double* const* u_tan, double* const* b_u, double* b_p,
                                void* stream);

/* Momentum right-hand side of one backward-Euler time step (Sec. 2, Eq.
 * Stokes_eqn: rho (u^{n+1} - u^n)/dt + grad p^{n+1} = div tau(u^{n+1}) +
 * f^{n+1}, div u^{n+1} = g^{n+1}): b_u = (rho_f / dt) u^n + f on every
 * unknown face and 0 on wall faces, with rho_f / dt = theta rho_f the face
 * coefficient of the last stk_set_coefficients (dt finite, else
 * STK_ERR_STATE).  u_n, f, b_u: device face arrays of length
 * stk_face_length(h, a); f may be NULL (no forcing); b_u may be u_n.  The
 * step then solves M x = (b_u, -g^{n+1}) with stk_solve, x = u^n a good
 * initial guess.  Stream-ordered, no synchronisation. */
int stk_backward_euler_rhs(stk_handle* h, const double* const* u_n, const double* const* f,
                           double* const* b_u, void* stream);

/* Gradient of a loss L(u) of the velocity with respect to the cell
 * log-viscosity and density, by the adjoint method: given the forward
 * velocity u (solution of M x = b) and the adjoint velocity lambda (solution
 * of M^T lambda = (dL/du, 0); M is symmetric, so stk_solve computes it),
 *   dL/dlog mu_c = mu_c lambda^T (dL_mu/dmu_c) u,
 *   dL/drho_c    = -theta lambda^T (d rho_f/d rho_c) u,
 * for the stress-form L_mu of Eq. div_stress (edge viscosities are the mean
 * of the surrounding in-domain cells, face densities the mean of the two
 * adjacent cells, Sec. 3.1) with the coefficients last set on h.  u, lambda:
 * face arrays; dL_dlogmu, dL_drho: cell arrays (written). */
int stk_gradient(stk_handle* h, const double* const* u, const double* const* lambda,
                 double* dL_dlogmu, double* dL_drho, void* stream);

/* y = x widened from FP32 to FP64 (n elements, device arrays, no handle),
 * with the exact conversion the flexible solve applies to its FP32
 * preconditioner outputs: integer instructions build the binary64 encoding
 * (GB300's FP64 pipe, which the conversion instruction would occupy, stays
 * free); bitwise equal to the conversion instruction for every input.
 * Stream-ordered.  Returns STK_OK, STK_ERR_ARG or STK_ERR_CUDA. */
int stk_widen(const float* x, double* y, long long n, void* stream);

/* Bound of every device-side wait of h's kernels (the grid barriers of the
 * persistent multi-block V-cycle), in clock64() cycles of the SM clock
 * (default 2e9, about one second).  A wait that runs out writes
 * STK_ERR_TIMEOUT to h's device status word and the launch ends at its next
 * barriers without faulting or hanging; stk_solve then returns
 * STK_ERR_TIMEOUT (its result is not a solution).  stk_wait_status returns
 * STK_OK or STK_ERR_TIMEOUT for the work issued so far (synchronises the
 * device; reset != 0 clears the word; stk_solve clears it when it starts). */
int stk_set_wait_budget(stk_handle* h, long long cycles);
int stk_wait_status(stk_handle* h, int reset);

/* CUDA graphs on (enable = 1, the default) or off (0) for h.  With graphs on,
 * every preconditioner application outside a solve is one graph launch and a
 * single stk_solve runs each GMRES cycle as one graph whose phases are gated
 * on the device; with graphs off every kernel is launched from the host and
 * the host gates the phases (for tools that do not follow kernels inside
 * graphs, and for debugging).  The results are bitwise the same. */
int stk_set_graphs(stk_handle* h, int enable);
/* 1 while h uses graphs, 0 once they are off (stk_set_graphs, or a graph the
 * library could not build, after which it launches from the host). */
int stk_graphs_in_use(const stk_handle* h);

/* Residual history of the last stk_solve / stk_solve_batched on h (Sec. 3.2
 * distinguishes the true residual r = b - M x from the preconditioned one):
 * kind 0: the true relative residual ||b - M x|| / ||b|| at the start of every
 * GMRES cycle and at the end (at most 256 kept); kind 1: the Arnoldi residual
 * estimate divided by ||b|| after every Arnoldi step (the preconditioned
 * residual of the left form, the true residual of the flexible form; at
 * most 2048 kept).  Copies min(cap, count) values to the host array out (out
 * may be NULL) and returns the count, or STK_ERR_ARG.  A stacked handle:
 * instance 0 (stk_stack_history gives the others). */
int stk_solve_history(const stk_handle* h, int kind, double* out, int cap);

/* y_p = x_p - mean(x_p): projection of a cell array onto mean-zero vectors,
 * the complement of the constant-pressure null space of M (Sec. 3.2: the
 * pressure is determined up to a constant with periodic, no-slip and
 * free-slip boundaries, so a pressure right-hand side must have zero mean,
 * e.g. the pressure part of an adjoint right-hand side).  x_p, y_p: device
 * cell arrays; y_p may be x_p.  Stream-ordered, no synchronisation. */
int stk_remove_mean(stk_handle* h, const double* x_p, double* y_p, void* stream);

/* Batched solve: count independent systems, each on its own handle (any
 * grid size, boundary conditions and coefficients), solved together with
 * the same parameters.  A batch of at most 8 handles (e.g. one stacked
 * handle per grid size) runs each handle's GMRES cycles as graph launches,
 * every handle at its own pace (the host waits once per cycle and handle);
 * larger batches advance in lockstep (one host synchronisation per GMRES
 * phase -- stopping test, first basis vector, each Arnoldi step, update --
 * for the whole batch)
 * and each instance's kernels and preconditioner graphs run on its handle's
 * own stream, forked from and joined back into `stream`, so the instances
 * share the GPU.  io[i] holds instance i's right-hand side and its initial
 * guess / solution (layouts as in stk_solve); infos (may be NULL) receives
 * count records.  A handle may appear once per batch.  Returns STK_OK when
 * every instance converged, else the first error (STK_ERR_NOT_CONVERGED when
 * that is the only kind). */
typedef struct {
    const double* const* b_u;
    const double* b_p;
    double* const* x_u;
    double* x_p;
} stk_batch_io;
int stk_solve_batched(int count, stk_handle* const* hs, const stk_solver_params* params,
                      const stk_batch_io* io, stk_solve_info* infos, void* stream);

/* Multigrid schedule of one precision (STK_FP64: the FP64 preconditioner of
 * left GMRES; STK_MIXED: the FP32 one of the flexible form).  Levels
 * coarse_level and coarser run as one single-block kernel (all of their
 * smoothing and transfers in one launch); finer levels run as grid-wide
 * kernels.  On those, levels pair_level and coarser smooth with one launch
 * per sweep and component doing both colours (each block recomputes the
 * red points of a one-point halo around its tile); finer levels launch once
 * per colour with `threads` threads per block (64, 128, 256 or 512).
 * Levels grid_level and coarser, down to coarse_level, run as one persistent
 * multi-block launch (cooperative, all blocks resident, grid-wide barriers
 * between the stages instead of kernel boundaries; the levels from
 * coarse_level on are then done by one of its blocks); grid_level >=
 * coarse_level switches it off.  Each barrier wait is bounded (see
 * stk_set_wait_budget).  Levels cluster_level and coarser, down to
 * coarse_level, run as one thread-block cluster (up to 16 blocks of 1024
 * threads on one GPC, hardware cluster barriers between the stages; it takes
 * precedence over grid_level); cluster_level >= coarse_level switches it off.
 * Stacked handles use neither.
 * 0 <= pair_level, coarse_level, grid_level, cluster_level <= number of levels.  The arithmetic does
 * not depend on the schedule, except that with coarse_level = 0 the finest
 * level's FP64 residual is evaluated point by point instead of through the
 * stresses of the grid kernels (equal up to rounding).  stk_autotune times one velocity + one
 * pressure V-cycle (as a captured graph) for every admissible schedule
 * (grid_level excepted: measured slower than cluster_level everywhere),
 * applies the fastest and returns it; stk_set_schedule applies a known one
 * (e.g. cached from an earlier run). */
typedef struct {
    int coarse_level;
    int threads;
    int pair_level;
    int grid_level;
    int cluster_level;
} stk_schedule;
int stk_get_schedule(const stk_handle* h, int precision, stk_schedule* out);
int stk_set_schedule(stk_handle* h, int precision, const stk_schedule* sc);
int stk_autotune(stk_handle* h, int precision, stk_schedule* best, void* stream);

/* Per-kernel timing of the calls above with CUDA events on the call's
 * stream (event nodes inside the preconditioner graphs).  stk_profile(h, 1)
 * starts collecting (and clears), 0 stops.  stk_profile_read returns, for
 * kernel family k (0 <= k < STK_NPROF), its name, its number of launches, its
 * summed device time in ms, the algorithmic bytes it moved (reads of every
 * input word and writes of every output word, once per launch) and, for the
 * Gauss-Seidel families, its floating-point operations.  Level-0 smoothing
 * has families of its own.  Returns -1 when k is out of range. */
#define STK_NPROF 24
int stk_profile(stk_handle* h, int enable);
/* Number of CUDA kernels this handle has launched since it was created:
 * coefficient setup (stk_set_coefficients, stk_set_bulk_viscosity), solves,
 * preconditioner and operator applications (graph replays count the kernels
 * they contain). */
long long stk_kernel_launches(const stk_handle* h);
int stk_profile_read(stk_handle* h, int k, const char** name, long long* launches,
                     double* ms, double* bytes, double* flops);

/* Bounds-checked builds (compiled with -DSTK_BOUNDS_CHECK: `python -m
 * paper_1308_4605_gb300.build --bounds-check` writes libstokes_gb300_check.so
 * beside the release library): every array index the stencil, transfer and
 * coarse-level kernels form is checked against the length of its array; an
 * index out of range is counted and the access goes to element 0 instead, so
 * nothing traps or faults.  stk_bounds_violations returns the number counted
 * since the library was loaded or last reset (reset != 0 clears it), with the
 * kind of the first (1 face, 2 cell, 3 edge, 4 shared memory) and its value
 * (either pointer may be NULL); it synchronises the device.  Release builds
 * return -1.  stk_bounds_selftest launches a kernel that checks the index 7
 * against the length 7 without accessing memory (one count of kind 2);
 * release builds return STK_ERR_STATE. */
long long stk_bounds_violations(long long* first_kind, long long* first_index, int reset);
int stk_bounds_selftest(void* stream);

/* Pressure V-cycle for callers that cannot allocate device memory.
 * (No counterpart in the paper: this is a deployment variant of
 * stk_pressure_vcycle.)  Callers whose device memory is wholly owned by another
 * allocator, or whose loop cannot afford the implicit synchronisation of
 * cudaMalloc, cannot create an stk_handle; this call needs none.  It computes
 * x_p = L~_rho^{-1} r_p: one multigrid V-cycle with zero initial guess for the
 * density-weighted Poisson equation div (1/rho_f) grad x = r (two red-black
 * Gauss-Seidel sweeps before and after each coarse correction, eight on the
 * coarsest grid), the same V-cycle as stk_pressure_vcycle on a handle whose
 * coefficients were set from the same rho, equal to it up to rounding, for the
 * grid (dim, n, h, bc) described as in stk_create.  rho, r_p (inputs) and x_p
 * (output) are caller-owned device cell arrays.
 * Workspace: a file-scope device array of 2,097,152 doubles (16 MiB) that every
 * GPU using this call holds until the process exits; grids needing more
 * (about 6 doubles per cell: 2D up to 512^2, 3D up to 64^3 fit) are rejected
 * with STK_ERR_SIZE before any device work.  No cudaMalloc, cudaFree or other
 * allocating call is made by the call itself, but with CUDA's lazy module
 * loading (the default) the array and the code of the kernels it uses are
 * placed in device memory during the first call on each device: make that
 * first call (a warm-up on a small grid) before the caller's allocator
 * reserves the device memory, and before any stream capture (it also looks
 * up the array's device address, with that device current).  Later calls
 * leave the device's free memory unchanged.  All calls on a device share that
 * device's one array and leave their workspace in it; each call writes every
 * value it later reads, so a call does not depend on what an earlier call
 * left.  Calls whose work overlaps on the same GPU (issued on different
 * streams, or from different host threads, without ordering between them)
 * race on the array: serialise them.  Returns STK_OK, STK_ERR_ARG,
 * STK_ERR_SIZE or STK_ERR_CUDA (also when a CUDA error from earlier work is
 * already pending; it is left pending); no message is recorded for
 * stk_last_error. */
int stk_pressure_vcycle_noalloc(int dim, const int* n, double h, const int* bc,
                                const double* rho, const double* r_p, double* x_p,
                                void* stream);

#ifdef __cplusplus
}
#endif
#endif /* STOKES_GB300_H */
