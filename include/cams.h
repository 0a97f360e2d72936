/*
 * cams.h -- C-ABI of the GB300 (sm_103a) C-AMS pressure solver.
 *
 * The library solves one implicit time step of single-phase compressible
 * flow in heterogeneous porous media (Sec. 2, Eqs. 1-6) with the adaptive
 * algebraic multiscale solver C-AMS (Sec. 3, Table 1) inside a Newton loop
 * with linear-system update adaptivity (Sec. 4.1.1) and adaptive multiscale
 * operator updates (Sec. 4.1.2).  Every step runs in the library's own CUDA
 * kernels on one GPU; there is no CPU fallback: without a usable CUDA device
 * every entry point that needs one returns CAMS_ECUDA.
 *
 * Conventions shared by all entry points
 *   - Cartesian grid of nx*ny*nz cells, cell index i = x + nx*(y + ny*z),
 *     x fastest.  All fields are float64 arrays of N = nx*ny*nz entries in
 *     that order.  A direction with one cell is inactive (2D: nz = 1).
 *   - Pointers given to the library are HOST pointers when
 *     cams_options.memspace == CAMS_HOST and DEVICE pointers (on the
 *     handle's device) when memspace == CAMS_DEVICE.  The caller keeps
 *     ownership of every buffer it passes; inputs are copied at the call
 *     and never retained.  Outputs are written before the call returns.
 *   - The handle owns all device memory it allocates (cudaMalloc at
 *     cams_setup and at the first use of an optional feature).
 *   - Every entry point returns CAMS_OK (0) or a negative CAMS_E* code and
 *     never aborts the process or throws; the message of the last failure
 *     is returned by cams_last_error.  A handle is not thread-safe.
 *   - Work is issued on the handle's stream (default stream unless set with
 *     cams_set_stream) and completed before the call returns.
 */
#ifndef CAMS_H
#define CAMS_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CAMS_OK          0
#define CAMS_EINVAL     -1  /* bad argument: sizes, coarse size not dividing the grid, k/phi/dt <= 0 */
#define CAMS_ENOMEM     -2  /* device or host allocation failed */
#define CAMS_ECUDA      -3  /* CUDA runtime error (message carries cudaGetErrorString) */
#define CAMS_ENOCONV    -4  /* max_newton reached; p_inout holds the last iterate */
#define CAMS_ESINGULAR  -5  /* zero or non-finite pivot in a local or coarse factorisation */
#define CAMS_ETIMEOUT   -6  /* a device-side wait exceeded its iteration limit */
#define CAMS_ENAN       -7  /* a non-finite value appeared in a norm */

/* memory spaces */
#define CAMS_HOST   0
#define CAMS_DEVICE 1

/* density laws (Sec. 4): rho = rho0 exp(c p)  or  rho = rho0 (1 + eta p) */
#define CAMS_RHO_EXP    0
#define CAMS_RHO_LINEAR 1

typedef struct cams_handle cams_handle;

/* Fine grid (Sec. 4: Delta x / alpha = Delta y = Delta z). */
typedef struct {
  int nx, ny, nz;
  double dx, dy, dz;
} cams_grid;

/* Fluid and rock: density law and its coefficient (c or eta), rho0,
 * viscosity mu, porosity phi (constant, d phi/dp = 0). */
typedef struct {
  int law;
  double c_or_eta;
  double rho0;
  double mu;
  double phi;
} cams_fluid;

/* Boundary conditions and sources.  dirichlet != 0 fixes p = p_west on the
 * west faces (x = 0) and p = p_east on the east faces (x = nx-1); every
 * other face is no-flow.  n_src point sources: src_cell[k] is a cell index,
 * src_rate[k] the integrated volumetric rate q_i dV_i of Eq. 6 (positive =
 * injection).  src_cell/src_rate follow cams_options.memspace and may be
 * NULL when n_src == 0.  Repeated cells add up.
 *
 * n_fix prescribed cell-centre pressures (Test Case 2 of Sec. 4.2.2 fixes
 * two vertical columns of cells): cell fix_cell[k] holds p = fix_value[k];
 * a cell listed more than once takes its last value.  The fixed cells are
 * eliminated symmetrically: their entries of the iterate are set to the
 * prescribed values on entry (and returned so in p_inout), each fixed row
 * of A reads p_i = fix_value (unit diagonal, no couplings), the couplings of
 * the free neighbours move to their right-hand side, Eq. 19 is not imposed
 * there (eps = 0), and the basis operators are eliminated the same way, so
 * the basis values of a fixed cell are 0.  A fixed cell may not be a
 * coarse node (CAMS_EINVAL), since that would remove a coarse unknown.
 * fix_cell/fix_value follow cams_options.memspace and may be NULL when
 * n_fix == 0; they are read during the call only. */
typedef struct {
  int dirichlet;
  double p_west, p_east;
  int n_src;
  const int* src_cell;
  const double* src_rate;
  int n_fix;
  const int* fix_cell;
  const double* fix_value;
} cams_bc;

/* Solver options (Table 1 and Sec. 4.1). */
typedef struct {
  int coarse[3];       /* primal-coarse block size per direction; must divide
                          the grid; >= 2 on active directions, 1 on inactive */
  int basis;           /* 1..4: basis equation (B1)..(B4) (Eqs. 8-11) */
  int restriction;     /* 0 = MSFE (R = P^T), 1 = MSFV (Eq. 7), 2 = MSFE iterations, then,
                          once the step's Newton loop has converged, one MSFV coarse
                          correction of the last linearisation for mass conservation
                          (Sec. 4.3) */
  int n_pre, n_post;   /* ILU(0) pre- / post-smoothing steps per iteration */
  double lin_rtol;     /* inner stop: ||r^i|| / ||r^0|| < lin_rtol (0.1 in Sec. 4.1.1) */
  double nl_tol;       /* outer stop: ||eps|| < nl_tol * ||eps at p^n|| (or absolute) */
  int tol_abs;         /* nonzero: ||eps|| < nl_tol (the paper's absolute test) */
  double adapt_theta;  /* relative-change threshold of the adaptive basis update;
                          < 0 rebuilds every entity at every linearisation */
  int max_newton;      /* linearisations per time step (<= 64) */
  int max_cams;        /* C-AMS iterations per linearisation */
  int memspace;        /* CAMS_HOST or CAMS_DEVICE for every pointer argument */
  int precision;       /* CAMS_PREC_FP64: every stage in FP64.  CAMS_PREC_MIXED: the
                          multiscale preconditioner (basis solves and P, the products of
                          R A P, restriction and prolongation, ILU(0) factor and sweeps) runs
                          in FP32 on the correction equation A delta = r inside FP64 iterative
                          refinement (block sums of R A P and of R r in FP64); assembly, the
                          residual r = f - A p, the update p += delta and the coarse-system
                          factorisation stay FP64.  The symmetric (MSFE) coarse system is then
                          solved in FP32 as Z^T D^{-1} Z R r, Z = L^{-1} of the factor's FP32
                          copy formed once per factorisation, where that costs at most 2e10
                          FMAs and 1 GiB (environment variable CAMS_COARSE_INV=0 at setup: FP32
                          substitution with the factor's copy); the MSFV coarse system is
                          factored and solved in FP64.
                          Converges to the same fixed point (the FP64 residual decides the
                          stopping tests). */
  int cf;              /* 1: correction functions (Sec. 3; Table 1 step 4) open every C-AMS
                          iteration: p += Psi, Psi solving the basis stages' local problems
                          with the residual f - A p as the source (zero on the vertices),
                          before any ILU(0) pre-smoothing.  Costs one set of local solves per
                          iteration (the paper leaves them out, Sec. 4.1.4).  0: off. */
  int jacobian;        /* 0: the Newton step of Eq. 3 (flux density lagged).  1: the full
                          Jacobian of the paper's equation (Eq. 2 over rho), the flux
                          density and the flux term's 1/rho differentiated too, rows scaled
                          by V rho as for Eq. 3; A is then not symmetric: the MSFE coarse
                          matrix is factorised by band LU.  Both steps have the same root. */
} cams_options;

#define CAMS_PREC_FP64  0
#define CAMS_PREC_MIXED 1

/* Per-step statistics filled by cams_solve. */
typedef struct {
  int newton_its;           /* linearisations performed */
  int cams_its;             /* C-AMS iterations, all linearisations */
  int basis_rebuilt;        /* local entities rebuilt, all linearisations */
  int converged;            /* 1 if the outer stopping test was met */
  int cams_per_newton[64];
  double eps_hist[65];      /* ||eps||_2 at each linearisation point */
  double res_final;         /* ||f - A p||_2 after the last inner loop */
  double t_assemble, t_precond, t_iterate, t_total;   /* milliseconds */
} cams_stats;

/* Quantities readable with cams_get / cams_get_int (debug and tests). */
#define CAMS_Q_TRANS      1  /* double 3N: Tx, Ty, Tz; T_d[i] couples i and i - stride_d (0 on the low face) */
#define CAMS_Q_MATRIX     2  /* double 4N: diag, then the couplings a_{i,i-1}, a_{i,i-nx}, a_{i,i-nx*ny} (0 when absent);
                                with jacobian = 0 A is symmetric and these are also a_{i-1,i} ... */
#define CAMS_Q_RHS        3  /* double N: f of Eq. 6 (rows scaled by V rho) */
#define CAMS_Q_EPS        4  /* double N: nonlinear error of Eq. 19 at the linearisation point */
#define CAMS_Q_PRESSURE   5  /* double N: the handle's current iterate p */
#define CAMS_Q_PROLONG    6  /* double 8N: P values, slot-major (slot s, cell i at s*N + i);
                                the FP32 values widened in mixed precision */
#define CAMS_Q_PROLONG_J  7  /* int 8N: coarse column of each P slot, -1 where the slot is unused */
#define CAMS_Q_COARSE     8  /* double 27*Nc: R A P as a 27-point coarse stencil, row I at 27*I,
                                neighbour (dx,dy,dz) in {-1,0,1}^3 at (dx+1) + 3(dy+1) + 9(dz+1) */
#define CAMS_Q_ILU_DIAG   9  /* double N: ILU(0) pivots d~_i (the only entries ILU(0) changes);
                                of the FP32 copy of A in mixed precision */
#define CAMS_Q_RESIDUAL  10  /* double N: f - A p for the current p */
#define CAMS_Q_SIZES     11  /* int 8: N, Nc, ncx, ncy, ncz, entities, entities rebuilt by the last update,
                                interiors supplied by the surrogate in the last update */
#define CAMS_Q_PROFILE   12  /* double 3*CAMS_PROF_CLASSES: per kernel class {launches, total ms,
                                kernels}; accumulated while profiling is on (cams_profile) */
#define CAMS_Q_LAUNCHES  13  /* double 1: kernels launched by this handle since cams_setup */
#define CAMS_Q_SURR_RATIO 14  /* double n (n = full interiors, cams_surrogate_data with 0): the
                                surrogate's gate ratio of each full interior in the last build that
                                used it (CAMS_EINVAL without a surrogate) */
#define CAMS_Q_MATRIX_UPPER 15  /* double 3N: the transposed couplings a_{i-1,i}, a_{i-nx,i},
                                a_{i-nx*ny,i} stored at cell i (0 when absent); equal to the
                                couplings of CAMS_Q_MATRIX when jacobian = 0 */
#define CAMS_Q_COARSE_FACTOR 16 /* double Nc*(m+1): the FP64 L D L^T of R A P (Sec. 3) in the
                                band order of CAMS_Q_COARSE_ORDER, column-major band: column q at
                                q*(m+1) holds d_q, then l_{q+1,q} .. l_{q+m,q} (rows past Nc-1 are
                                not defined); CAMS_EINVAL unless the last update factored R A P
                                by L D L^T (MSFE of a symmetric A) */
#define CAMS_Q_COARSE_ORDER  17 /* int Nc+1 (cams_get_int): the band half-width m, then the band
                                position of each natural coarse index I (x fastest) */

/* kernel classes of CAMS_Q_PROFILE */
#define CAMS_PROF_ASSEMBLE      0   /* density + linear-system population (a2) */
#define CAMS_PROF_BASIS_OP      1   /* basis operator of Eqs. 8-11 */
#define CAMS_PROF_ADAPT         2   /* adaptive-update flags (a3) */
#define CAMS_PROF_BASIS         3   /* vertex/edge/face/interior local solves (a4-a7) */
#define CAMS_PROF_GALERKIN      4   /* R A P (a8) */
#define CAMS_PROF_COARSE_FACTOR 5   /* band fill + LDL^T / LU of R A P (a9) */
#define CAMS_PROF_ILU_FACTOR    6   /* ILU(0) pivots (a10) */
#define CAMS_PROF_RESIDUAL      7   /* r = f - A p with its norm */
#define CAMS_PROF_RESTRICT      8   /* R r */
#define CAMS_PROF_COARSE_SOLVE  9   /* band substitution, or Z^T D^{-1} Z (mixed) */
#define CAMS_PROF_PROLONG      10   /* p += P p_c (FP64), delta = P p_c (mixed precision) */
#define CAMS_PROF_ILU_FWD      11   /* ILU(0) forward wavefront sweep */
#define CAMS_PROF_ILU_BWD      12   /* ILU(0) backward wavefront sweep */
#define CAMS_PROF_ILU_RESID    13   /* D^{-1}(f - A p) feeding the forward sweep */
#define CAMS_PROF_UPDATE       14   /* p += delta (mixed precision) */
#define CAMS_PROF_ILU_APPLY    15   /* x += z after the backward sweep */
#define CAMS_PROF_COARSE_INV   16   /* Z = L^{-1} of the FP32 copy of the FP64 coarse factor (mixed) */
#define CAMS_PROF_CLASSES      17

/* (a1) Set up a solver for one grid and permeability field.
 * kx, ky, kz: permeability per cell (> 0, finite); ky and kz may alias kx.
 * Computes the static TPFA transmissibilities (harmonic average of the
 * half-cell conductances; half-cell distance to Dirichlet faces), the
 * primal/dual-coarse wirebasket tables (Sec. 3, Fig. 1; coarse nodes at
 * offset floor(b/2) in each primal block) and allocates every buffer.
 * On success *out receives a handle to release with cams_destroy; on failure
 * *out is NULL and the status tells why (cams_last_error(NULL) gives the
 * message). */
int cams_setup(const cams_grid* grid, const cams_fluid* fluid, const cams_options* opt,
               const double* kx, const double* ky, const double* kz, cams_handle** out);

/* (a1) Replace the permeability field of an existing handle: recompute the
 * static transmissibilities and mark every basis function for rebuilding at
 * the next cams_update_basis / cams_solve (as on a fresh handle).  Same
 * argument rules as cams_setup; no allocation. */
int cams_set_permeability(cams_handle* h, const double* kx, const double* ky, const double* kz);

/* Turn per-kernel-class timing on (enable != 0) or off.  While on, CUDA
 * events bracket every kernel class on the handle's stream and
 * CAMS_Q_PROFILE accumulates launches and milliseconds; turning it on resets
 * the totals. */
int cams_profile(cams_handle* h, int enable);

/* Self-test of the bounded device-side waits used by the wavefront sweeps:
 * launches one wait on a counter that nothing sets.  The wait gives up after
 * its iteration limit (well under a few seconds), the kernel returns and the
 * call returns CAMS_ETIMEOUT; the handle stays usable.  Any other result
 * means the timeout path is broken. */
int cams_selftest_wait(cams_handle* h);

/* Run the handle's work on the given cudaStream_t (passed as void*; NULL =
 * default stream).  The stream must belong to the handle's device. */
int cams_set_stream(cams_handle* h, void* stream);

/* Choose between the handle's equivalent kernel schedules (for an autotuner;
 * setup picks defaults):
 *   ilu_cta         ILU(0) wavefront sweeps: 0 = one 8x4-row tile per warp,
 *                   1 = 2x2 tiles per CTA with the edges inside a block in
 *                   shared memory (the same arithmetic; results are bitwise
 *                   equal); -1 = unchanged
 *   coarse_cluster  symmetric (MSFE) coarse solve: 0 = one CTA, 1 = across a
 *                   thread-block cluster (a different summation order); -1 =
 *                   unchanged.  The general band solve has one schedule.
 * Waits for the handle's stream and drops its captured iteration graph (it
 * is captured again at the next iteration).  Errors: CAMS_EINVAL (null
 * handle, a value outside {-1, 0, 1}, a schedule this GPU or grid cannot run,
 * the level-scheduled sweeps of CAMS_ILU_LEVEL=1), CAMS_ECUDA. */
int cams_set_schedule(cams_handle* h, int ilu_cta, int coarse_cluster);

/* The handle's current schedule (the values of cams_set_schedule); either
 * pointer may be NULL. */
int cams_get_schedule(cams_handle* h, int* ilu_cta, int* coarse_cluster);

/* (a2) Linear-system population (Table 1, step 1): from p_nu (iterate) and
 * p_n (previous time level) build A = C + A~ and f (Eq. 6, Eqs. 3-5, rows
 * scaled by V rho^nu), the error eps of Eq. 19 and its 2-norm.  The handle's
 * current iterate becomes p_nu.  eps_norm_out may be NULL. */
int cams_assemble(cams_handle* h, const double* p_nu, const double* p_n, double dt,
                  const cams_bc* bc, double* eps_norm_out);

/* (a3-a10) Update the operators of the two-stage preconditioner for the
 * system of the last cams_assemble: adaptively rebuild the basis functions
 * (Sec. 4.1.2; force != 0 rebuilds all), form R A P (Eq. 13, MSFE or MSFV)
 * and factorise it, and factorise ILU(0).  *n_rebuilt_out (may be NULL)
 * receives the number of local entities rebuilt. */
int cams_update_basis(cams_handle* h, int force, int* n_rebuilt_out);

/* (a11) Run n C-AMS iterations (Table 1 steps 4-7) on the current system
 * from the handle's current iterate.  res_norms (may be NULL; n+1 doubles,
 * host memory always) receives ||f - A p||_2 before and after each one. */
int cams_iterate(cams_handle* h, int n, double* res_norms);

/* (a2-a12) One implicit time step from p_n: Newton loop of Sec. 4.1.1 with
 * the C-AMS inner loop, adaptive basis updates and the stopping tests of
 * cams_options.  p_inout: initial guess on entry (normally p_n), p^{n+1} on
 * return (also when CAMS_ENOCONV is returned).  stats may be NULL (host). */
int cams_solve(cams_handle* h, const double* p_n, double dt, const cams_bc* bc,
               double* p_inout, cams_stats* stats);

/* Ensemble of independent time steps (batches of realisations, such as the
 * statistically equivalent permeability fields the paper averages over,
 * Sec. 4): for k < n the same as
 *   status[k] = cams_solve(h[k], p_n[k], dt[k], bc[k], p_inout[k], &stats[k]),
 * with the members run concurrently on the GPU.  n_workers host threads
 * (0: one per hardware thread; never more than n) each take the next member
 * in index order and run it on a stream of their own, so the kernels of
 * different members overlap.  A member's result is bit-for-bit the one
 * cams_solve gives: no kernel depends on the stream or on what else runs.
 * The handles must be distinct and each follows its own memspace rule for
 * its pointers; work already queued on a handle's stream is completed
 * before its member starts and the handle's stream is restored afterwards.
 * dt, bc, status (n entries) and stats (n entries, may be NULL) are host
 * arrays.  Returns CAMS_OK when every member returned CAMS_OK, else the
 * status of the lowest-index member that did not; bad arguments give
 * CAMS_EINVAL before any member runs (message in cams_last_error(NULL)).
 * cams_get(CAMS_Q_LAUNCHES) counts the launches of all handles that ran
 * meanwhile. */
int cams_ensemble_solve(int n, cams_handle* const* h, const double* const* p_n, const double* dt,
                        const cams_bc* const* bc, double* const* p_inout, cams_stats* stats,
                        int* status, int n_workers);

/* ---- Learned basis surrogate (interior stage of the basis construction) ----
 *
 * A small 3D convolutional network predicts the basis functions of each full
 * dual-block interior (the (b-1)^3 cells between the vertex planes of a
 * dual block of (b+1)^3 cells, cubic coarse blocks of size b) from the
 * block's basis-operator coefficients and the exact edge and face values of
 * its 8 corner functions.  Input channels (CAMS_NET_IN, on the (b+1)^3
 * patch): the logs of the three lower-face couplings of A_b minus their patch
 * mean, the relative accumulation term (A_b diagonal minus the coupling sum,
 * over the coupling sum), and for each corner function its deviation from
 * the multilinear interpolant of the corner values on the patch boundary (0
 * inside).  Output (CAMS_NET_OUT channels): the deviation from that
 * interpolant, used on the interior cells.  Layers: 3x3x3 convolutions with
 * zero padding, CAMS_NET_IN -> CAMS_NET_HID -> CAMS_NET_HID -> CAMS_NET_HID
 * -> CAMS_NET_OUT, ReLU between them.  Parameters (CAMS_NET_PARAMS floats):
 * w1, b1, w2, b2, w3, b3, w4, b4 in that order; w_l is [co][ci][27] with
 * tap t = (dx+1) + 3(dy+1) + 9(dz+1).  A prediction is kept only when the
 * residual of the interior equations it leaves, scaled by the diagonal
 * (D^{-1} A_b P on the interior cells, 2-norm, worst of the 8 corner
 * functions), is at most gate_tol times the norm of the boundary data's
 * scaled contribution; otherwise the exact local solve runs. */
#define CAMS_NET_IN      12
#define CAMS_NET_HID     32
#define CAMS_NET_OUT      8
#define CAMS_NET_PARAMS  72680

/* Enable the surrogate on a 3D handle with cubic coarse blocks: params
 * (host, CAMS_NET_PARAMS floats) are copied; gate_tol > 0 is the residual
 * threshold.  gate_tol <= 0 (params may be NULL) disables it.  The surrogate
 * is used whenever every local entity is rebuilt (first build, forced or
 * theta < 0); adaptive partial rebuilds use the exact solves.  CAMS_Q_SIZES[7]
 * reports the interiors it supplied in the last build. */
int cams_set_surrogate(cams_handle* h, const float* params, double gate_tol);

/* Training data from the handle's current basis (after cams_update_basis
 * with exact solves): for the first n = min(max_patches, number of full
 * interiors) patches, x (n x CAMS_NET_IN x (b+1)^3), target (n x
 * CAMS_NET_OUT x (b+1)^3: the deviation from the multilinear interpolant)
 * and mask (same shape: 1 on interior cells, 0 elsewhere).  Device pointers,
 * FP32.  *n_out receives n; with max_patches <= 0 nothing is written and
 * *n_out receives the number of full interiors. */
int cams_surrogate_data(cams_handle* h, int max_patches, float* x, float* target, float* mask,
                        int* n_out);

/* Layer kernels of the network, used for training and by the engine
 * (device pointers, FP32; work is queued on `stream`, a cudaStream_t or
 * NULL, and the call returns after queueing; CAMS_ECUDA on a launch error).
 * Activations are [B][C][S][S][S], x fastest.
 *   forward:  y = conv(x; w, bias), then ReLU when relu != 0.
 *   backward: with gy = dL/dy (of the pre-ReLU output), gw = dL/dw,
 *             gbias = dL/dbias and, when gx != NULL, gx = dL/dx multiplied
 *             by the ReLU mask xact > 0 of the layer's input when xact !=
 *             NULL (the gradient with respect to the previous layer's
 *             pre-activation).  gw and gbias are overwritten.
 *   mse:      loss = sum(mask (pred - target)^2) / count into *loss (device
 *             double), grad = 2 mask (pred - target) / count; scratch holds
 *             512 doubles.
 *   energy:   the energy norm of the interior error, the norm in which a
 *             basis function's error costs the coarse space: e = mask
 *             (pred - target) on B patches of C channels, relative face
 *             couplings w = exp(x[b][d]) from channels d = 0, 1, 2 of the
 *             network input x (cx channels; channel d at a cell is the log
 *             coupling to its lower neighbour along d), loss = sum over the
 *             patch's faces of w (e_u - e_v)^2 / count into *loss, grad = mask
 *             d loss / d pred; scratch holds 512 doubles.
 *   adam:     one Adam step (Kingma and Ba) at step number step >= 1. */
int cams_net_conv_forward(int B, int S, int ci, int co, const float* x, const float* w,
                          const float* bias, int relu, float* y, void* stream);
int cams_net_conv_backward(int B, int S, int ci, int co, const float* x, const float* w,
                           const float* gy, const float* xact, float* gx, float* gw,
                           float* gbias, void* stream);
int cams_net_mse(long long n, const float* pred, const float* target, const float* mask,
                 double count, float* grad, double* loss, double* scratch, void* stream);
int cams_net_energy(int B, int S, int C, int cx, const float* pred, const float* target,
                    const float* mask, const float* x, double count, float* grad, double* loss,
                    double* scratch, void* stream);
int cams_net_adam(long long n, float* p, const float* g, float* m, float* v, float lr,
                  float beta1, float beta2, float eps, int step, void* stream);

/* The network on the tensor cores (tcgen05 MMAs: BF16 operands, FP32
 * accumulation in tensor memory), the form the engine uses for inference
 * whenever a patch fits (cubic coarse blocks up to b = 10, S = b + 1 <= 11).
 * Each 3x3x3 layer is an implicit GEMM over the zero-padded patch: the 27
 * taps are 27 shifted views of the patch's rows in shared memory.  Inputs,
 * weights and hidden activations are rounded to BF16 (nearest, ties to
 * even); biases, accumulation and the outputs below are FP32.  Device
 * pointers; `work` is caller-owned device memory of at least
 * cams_net_tc_work_bytes(B, S) bytes (cleared and used by the call).  The
 * calls queue their work on `stream` and return when it is done.
 *   conv_forward_tc: one layer, x [B][ci][S^3] -> y [B][co][S^3] FP32
 *                    (ci, co <= CAMS_NET_HID), ReLU when relu != 0.
 *   forward_tc:      the whole network (parameters as for cams_set_surrogate),
 *                    x [B][CAMS_NET_IN][S^3] -> y [B][CAMS_NET_OUT][S^3].
 * Errors: CAMS_EINVAL (sizes, a workspace that is too small, a patch too
 * large for shared memory), CAMS_ETIMEOUT (an MMA completion wait gave up),
 * CAMS_ECUDA; the message is cams_last_error(NULL). */
long long cams_net_tc_work_bytes(int B, int S);
int cams_net_conv_forward_tc(int B, int S, int ci, int co, const float* x, const float* w,
                             const float* bias, int relu, float* y, void* work,
                             long long work_bytes, void* stream);
int cams_net_forward_tc(int B, int S, const float* x, const float* params, float* y, void* work,
                        long long work_bytes, void* stream);

/* Copy an internal quantity (CAMS_Q_*) to dst (memspace of the handle, except
 * CAMS_Q_SIZES which is always host).  dst must hold the documented size. */
int cams_get(cams_handle* h, int what, double* dst);
int cams_get_int(cams_handle* h, int what, int* dst);

/* Residual r = f - A p and ||r||_2 of a symmetric 7-point system, without
 * allocating any device memory.  The paper has no counterpart: this is a
 * service for callers that cannot call cudaMalloc -- frameworks that give
 * all device memory to their own pool or arena (an allocation behind the
 * pool's back can fail or fragment it) and time-critical loops that cannot
 * afford the device-wide synchronisation cudaMalloc/cudaFree imply.  The
 * reduction's scratch is a file-scope static device array of 32769 doubles
 * (256 KiB), present on every GPU that loads the library until the process
 * exits.
 *   nx, ny, nz       grid (cell i = x + nx*(y + ny*z)); at most 268,435,456
 *                    cells (32768 partial sums of 8192 cells), else
 *                    CAMS_EINVAL with a message naming the limit
 *   diag, ax, ay, az A in the CAMS_Q_MATRIX layout (diagonal, then the
 *                    couplings a_{i,i-1}, a_{i,i-nx}, a_{i,i-nx*ny}, stored
 *                    at the upper cell, 0 where absent); DEVICE pointers
 *   f, p             right-hand side and iterate; DEVICE pointers
 *   r                output residual (DEVICE, N doubles) or NULL
 *   norm_out         HOST double receiving ||r||_2, or NULL (not both NULL)
 *   stream           cudaStream_t (NULL = default stream) of the current device
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and so does the first
 * call after the device's current context has changed (cudaDeviceReset
 * reloads the module); make the first call on a device before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race
 * and must be serialised by the caller.  The call returns when the result
 * is ready.  Errors: CAMS_EINVAL (sizes, null pointers), CAMS_ECUDA; the
 * message is cams_last_error(NULL). */
int cams_residual_norm_noalloc(int nx, int ny, int nz, const double* diag, const double* ax,
                               const double* ay, const double* az, const double* f,
                               const double* p, double* r, double* norm_out, void* stream);

/* Message of the last failure on h (or of the last failed cams_setup when h
 * is NULL).  Never NULL; owned by the library. */
const char* cams_last_error(cams_handle* h);

/* Release every resource of h.  NULL is ignored. */
void cams_destroy(cams_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* CAMS_H */
