/*
 * rr.h -- C ABI of the GB300 randomized-resolvent library (librr.so).
 *
 * Randomized resolvent analysis (Ribeiro, Yeh & Taira, arXiv:1902.01458):
 * for a discretised linearised flow operator L (Sec. II.A, Eq. 1) and a
 * complex shift s = i*omega (+ beta for the discounted resolvent, Sec. II.A),
 * the weighted resolvent is
 *
 *     R = W^{1/2} (s I - L)^{-1} W^{-1/2}                    (Eq. 4)
 *
 * and Algorithm 1 (Sec. II.B) approximates its leading singular triplets
 * (Eq. 5) from k solves with a Gaussian test matrix, k adjoint solves and k
 * recovery solves (Eq. 8), all reusing one factorisation per shift
 * (Sec. III.A).  W is diagonal and positive (identity when not given).
 *
 * Conventions for every entry point
 *  - Every call returns rr_status and never aborts; rr_last_error() gives a
 *    one-line message for the calling thread's most recent failure.
 *  - Complex numbers are interleaved (re, im) pairs of doubles (complex128).
 *  - Unknowns are ordered by streamwise column, n = ((ix*ny)+iy)*q + c, so
 *    the operator is block-tridiagonal with b x b blocks, b = q*ny.
 *  - Batches: a factors object holds F shifts ("problems").  Block vectors
 *    are device arrays laid out [F][N][k] (row-major; column j of problem f
 *    is the strided vector x[f*N*k + n*k + j]).
 *  - Device pointers must be on the operator's device; host pointers are
 *    read before the call returns.  The caller owns every pointer it
 *    passes; the library owns the opaque handles, which are created and
 *    destroyed in pairs.
 *  - Work is issued on the stream given to rr_factor (or rr_apply/rr_phi).
 *    Calls that iterate (refinement) or report rr_info synchronise that
 *    stream before returning; the others return once the work is queued.
 */
#ifndef RR_H
#define RR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RR_OK = 0,
  RR_ERR_ARG = 1,         /* invalid argument (null, size, kind, range)      */
  RR_ERR_NOMEM = 2,       /* device allocation failed                        */
  RR_ERR_SINGULAR = 3,    /* zero pivot in the block factorisation           */
  RR_ERR_NOCONV = 4,      /* refinement hit max_refine above refine_tol      */
  RR_ERR_RANK = 5,        /* CholeskyQR breakdown even with the shift        */
  RR_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up              */
  RR_ERR_CUDA = 7,        /* CUDA runtime error (message in rr_last_error)   */
  RR_ERR_UNSUPPORTED = 8  /* valid request the library does not implement   */
} rr_status;

/* Arithmetic of the block factorisation and the block sweeps.  FP64 runs
 * everything in complex double.  FP32 stores the factors in complex float,
 * runs the factorisation's rank-128 updates and the sweep products on the
 * tensor cores (tcgen05 kind::tf32 with each operand split into a TF32 part
 * and its remainder, hi.hi + hi.lo + lo.hi: FP32-level products, FP32
 * accumulation; the pivoted panels and the rank-16 updates inside a
 * 128-column slab run in FP32 on the CUDA cores) and wins accuracy back by
 * iterative refinement against an FP64 residual.
 * FP32_BF16X3 and FP32_BF16X6 are the same with the operands split into
 * BF16 pieces on tcgen05 kind::f16: two pieces and three products (about 16
 * bits of each product) or three pieces and six products (hi.hi, hi.mid,
 * mid.hi, hi.lo, mid.mid, lo.hi: FP32-level).  FP32_SIMT is FP32 with every
 * product on the FP32 CUDA cores.  QR, SVD, norms and the refinement
 * residual stay FP64 in every mode. */
typedef enum {
  RR_FP64 = 0,
  RR_FP32 = 1,
  RR_FP32_SIMT = 2,
  RR_FP32_BF16X3 = 3,
  RR_FP32_BF16X6 = 4
} rr_precision;

/* Operator kinds (q = unknowns per grid point). */
enum { RR_ADVDIFF_SCALAR = 1, RR_ISO_NS2D = 3, RR_ISO_NS2D_KZ = 4 };

/* Uniform grid of nx x ny interior nodes on [x0,x1] x [y0,y1].
 * Dirichlet directions have spacing L/(n+1) and zero ghost nodes; a periodic
 * y direction (periodic_y != 0) has spacing (y1-y0)/ny and nodes y0+j*dy.
 *  RR_ADVDIFF_SCALAR: L phi = -U phi_x - V phi_y + (1/re) lap phi - s_s phi
 *  RR_ISO_NS2D: isothermal compressible Navier-Stokes in (rho', u', v')
 *    linearised about (rho, U, V), p = rho / mach^2, Reynolds number re,
 *    second-order central differences (4-corner cross derivative).
 * Sponge s_s = sponge_max * xi^2 on the outer sponge_frac of each
 * (non-periodic) boundary, xi the normalised depth into the layer.
 * Boundary closure per side (Sec. III.A: Dirichlet velocities and Neumann
 * pressure at the far field, Neumann for every variable at the outlet):
 * neumann[side] is a bit mask over the q variables (bit c = variable c,
 * in the order rho', u', v'), sides x0, x1, y0, y1.  A set bit makes the
 * ghost node of that variable equal to the adjacent interior node (the
 * coefficient folds onto it); a clear bit keeps the zero (Dirichlet) ghost.
 * All zero is the homogeneous Dirichlet operator; the paper's closure for
 * RR_ISO_NS2D is {1, 7, 1, 1} (p' = rho'/mach^2, so Neumann pressure is
 * Neumann rho').  The y masks must be zero when periodic_y is set.
 *  RR_ISO_NS2D_KZ: the bi-global form of RR_ISO_NS2D (Sec. III.A/B, the
 *    spanwise wavenumbers k_z): perturbations (rho', u', v', w') varying as
 *    exp(i kz z) about the same z-invariant base flow with no spanwise
 *    velocity, so d/dz -> i kz (continuity gains -rho i kz w', the
 *    Laplacians -kz^2, the divergence i kz w', and the w' equation is
 *    advection, -(c^2/rho) i kz rho' and the viscous terms).  L(kz) is
 *    complex; with D = diag(1, 1, 1, i) per point, D^{-1} L D is real, and
 *    the library factors and sweeps that real operator (R = D R~ D^{-1}
 *    has the same singular values; every entry point takes and returns the
 *    vectors of L itself).  q = 4, Neumann masks over 4 variables. */
typedef struct {
  int kind;
  int nx, ny;
  int periodic_y;
  double x0, x1, y0, y1;
  double re;
  double mach;
  double sponge_max;
  double sponge_frac;
  int neumann[4];
  double kz;        /* spanwise wavenumber (RR_ISO_NS2D_KZ only) */
} rr_grid;

/* Base-flow fields on the interior nodes, host pointers to nx*ny doubles
 * each, point index ix*ny + iy.  rho may be NULL for RR_ADVDIFF_SCALAR. */
typedef struct {
  const double* rho;
  const double* u;
  const double* v;
} rr_baseflow;

typedef struct rr_operator rr_operator; /* device copy of L's stencil      */
typedef struct rr_factors rr_factors;   /* block factors of F shifts       */

/* Diagnostics of one rr_solve / rr_sketch / rr_modes call. */
typedef struct {
  int refine_iters;       /* largest refinement count over all solves      */
  double refine_residual; /* largest final ||b - A x|| / ||b|| per column  */
  double cqr_cond;        /* largest condition estimate of a CholeskyQR R  */
  int cqr_shifted;        /* 1 if a shifted CholeskyQR fallback was used   */
  int refine_stagnated;   /* 1 if refinement stopped above refine_tol
                             because a correction removed less than a
                             tenth of the residual (the floor of the FP64
                             residual or of the factors' accuracy)         */
  double first_residual;  /* largest ||b - A x|| / ||b|| per column after
                             the first, uncorrected solve (the accuracy of
                             the factors themselves)                       */
  long long problem_solves; /* block solves run, summed over the call's
                             solves: each solve counts its problems, each
                             correction the problems it was applied to     */
} rr_info;

const char* rr_last_error(void);
const char* rr_status_string(rr_status s);

/* Build the stencil of L (Sec. II.A, Eq. 1; the discrete operator of the
 * grid kind above) on `device` from host base-flow fields.  weights: NULL
 * (identity) or N = nx*ny*q positive doubles (host), the diagonal of W.
 * Errors: RR_ERR_ARG (kind, nx or ny < 3, b = q*ny > 1024, non-positive
 * weight, re <= 0, mach <= 0 for NS), RR_ERR_NOMEM, RR_ERR_CUDA. */
rr_status rr_create_operator(const rr_grid* grid, const rr_baseflow* flow,
                             const double* weights, int device,
                             rr_operator** out);
rr_status rr_destroy_operator(rr_operator* op);

/* Sizes of an operator: N unknowns, block size b, q, nx, ny. */
rr_status rr_operator_dims(const rr_operator* op, int* n, int* b, int* q,
                           int* nx, int* ny);

/* y = (s_f I - L) x for F shifts (adjoint != 0: y = (s_f I - L)^H x).
 * shifts: host, 2*F doubles (re, im).  x, y: device complex128 [F][N][k],
 * distinct buffers.  This is the FP64 residual operator of the refinement
 * (Sec. II.A's operator applied, no solve). */
rr_status rr_apply(rr_operator* op, int nshift, const double* shifts, int k,
                   int adjoint, const void* x, void* y, void* stream);

/* Allocation-free variant of rr_apply.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory once
 * they are running -- for example a host framework that owns the whole GPU
 * through its own memory pool, or a time-critical loop where cudaMalloc's
 * implicit device synchronisation is not allowed.  Same arguments, result
 * and errors as rr_apply, but the F shifts are staged in a fixed array
 * compiled into the library (RR_APPLY_STATIC_MAX_SHIFTS complex doubles,
 * 64 KB, held on every GPU that loads the library until the process exits)
 * instead of a cudaMalloc'd buffer; nshift above the maximum is rejected with
 * RR_ERR_ARG.  The call allocates nothing.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress, under a host lock)
 * with that device current and keeps it for the process; a cudaDeviceReset
 * of that device invalidates the kept address, so do not call this entry
 * point after resetting a device.  Every call copies the shifts from host
 * memory and synchronises its stream before returning, so it must not be
 * called on a capturing stream: it checks and returns RR_ERR_ARG.  All calls
 * share the one array, so calls that overlap on the GPU (other streams or
 * host threads) race on it.  RR_ISO_NS2D_KZ operators: RR_ERR_UNSUPPORTED
 * (their application goes through a temporary; use rr_apply). */
#define RR_APPLY_STATIC_MAX_SHIFTS 4096
rr_status rr_apply_static(rr_operator* op, int nshift, const double* shifts, int k,
                          int adjoint, const void* x, void* y, void* stream);

/* Eq. (9): Phi_j = ||grad v||_F at every grid point, repeated over the q
 * variables.  phi: device, N doubles. */
rr_status rr_phi(rr_operator* op, double* phi, void* stream);

/* Factor s_f I - L for F shifts (Sec. III.A: one factorisation per shift,
 * reused by all solves).  shifts: host, 2*F doubles.  Block LU over the
 * streamwise columns with an explicit inverse of every Schur block by
 * Gauss-Jordan elimination with partial pivoting.  stream: a cudaStream_t
 * (NULL = default stream) used by every later call on the factors.
 * Errors: RR_ERR_ARG, RR_ERR_NOMEM, RR_ERR_SINGULAR (exact zero pivot in some
 * Schur block; the factors are still returned), RR_ERR_CUDA. */
rr_status rr_factor(rr_operator* op, int nshift, const double* shifts,
                    rr_precision prec, void* stream, rr_factors** out);
rr_status rr_destroy_factors(rr_factors* f);

/* x = R b (adjoint = 0) or x = R^H b (adjoint != 0) for every problem: the
 * solve of Algorithm 1's second, fourth and sixth steps.  b, x: device
 * complex128 [F][N][k], distinct.  refine_tol / max_refine drive the
 * iterative refinement x <- x + solve(b - A x) with the residual in FP64
 * (FP64 factors too, when refine_tol > 0): it stops once every column's
 * ||b - A x|| / ||b|| <= refine_tol or a correction removes less than a
 * tenth of the residual.  With FP32 factors on the tensor-core sweep (even
 * k <= 32, even block >= 128) each problem is refined on its own and leaves
 * the set of corrected problems when it stops.  info may be NULL.  Errors:
 * RR_ERR_ARG, RR_ERR_NOCONV (x still written), RR_ERR_CUDA. */
rr_status rr_solve(rr_factors* f, int k, int adjoint, const void* b, void* x,
                   double refine_tol, int max_refine, rr_info* info);

/* Algorithm 1, first five steps, for every problem: Omega = randn(N, k)
 * (Philox-4x32-10 with key seeds[f], counter (n, j, 0, 0), Box-Muller),
 * optionally Omega_p = diag(phi) Omega (Eq. 9; phi: device, N doubles, or
 * NULL); Y = R Omega; Q = qr(Y) (FP64 CholeskyQR2); B^H = R^H Q; the SVD of
 * B from CholeskyQR2 of B^H and a k x k one-sided Jacobi SVD.
 * seeds: host, F values.  Outputs (device): V [F][N][k] forcing modes and
 * sigma_halko [F][k] (singular values of B, descending).  1 <= k <= 64,
 * k <= N.  Errors: RR_ERR_ARG, RR_ERR_NOCONV, RR_ERR_RANK, RR_ERR_CUDA. */
rr_status rr_sketch(rr_factors* f, int k, const uint64_t* seeds,
                    const double* phi, double refine_tol, int max_refine,
                    void* V, double* sigma_halko, rr_info* info);

/* Test matrices of Sec. II.B.2, all drawn from one Philox-4x32-10 block per
 * entry (key seeds[f], counter (n, j, 0, 0); words w0..w3):
 *  RR_OMEGA_GAUSSIAN          Box-Muller N(0, 1) as described at rr_sketch;
 *  RR_OMEGA_RADEMACHER        -1 if bit 0 of w0 is set, else +1;
 *  RR_OMEGA_SPARSE_RADEMACHER nonzero iff w1 < floor(density * 2^32), then
 *                             +-1/sqrt(density) with the Rademacher sign
 *                             (mean 0, variance 1; density 1/3 is
 *                             Achlioptas' sparse projection);
 *  RR_OMEGA_ORTHONORMAL       the Q factor (CholeskyQR2, R with a real
 *                             positive diagonal) of diag(phi) times the
 *                             Gaussian matrix.
 * Every kind is scaled by phi (Eq. 9) when phi is given. */
typedef enum {
  RR_OMEGA_GAUSSIAN = 0,
  RR_OMEGA_RADEMACHER = 1,
  RR_OMEGA_SPARSE_RADEMACHER = 2,
  RR_OMEGA_ORTHONORMAL = 3
} rr_omega_kind;

/* Options of rr_sketch_ex.  power_iters = q runs q subspace iterations
 * (Sec. II.B.1; Halko, Martinsson & Tropp 2011, Alg. 4.4) after the sketch:
 * q times { Z = qr(R^H Q); Q = qr(R Z) }, every QR a CholeskyQR2, every
 * solve reusing the factors (2k extra solves per iteration).  density is
 * read only for RR_OMEGA_SPARSE_RADEMACHER. */
typedef struct {
  int omega_kind;   /* rr_omega_kind                       */
  double density;   /* in (0, 1]                           */
  int power_iters;  /* 0 .. 64                             */
} rr_sketch_opts;

/* rr_sketch with a choice of test matrix and subspace iterations.  opts NULL
 * is rr_sketch (Gaussian, no iterations).  Errors as rr_sketch, plus
 * RR_ERR_ARG for an unknown kind, a density outside (0, 1] or power_iters
 * outside [0, 64]. */
rr_status rr_sketch_ex(rr_factors* f, int k, const uint64_t* seeds,
                       const double* phi, const rr_sketch_opts* opts,
                       double refine_tol, int max_refine, void* V,
                       double* sigma_halko, rr_info* info);

/* Algorithm 1, last steps (Eq. 8): U Sigma = R V, sigma_j = ||(U Sigma)_j||,
 * u_j = (U Sigma)_j / sigma_j; with orthogonalize != 0 also the optional
 * SVD(U Sigma) = U Sigma Vt^H and V <- V Vt.  Results are sorted by sigma
 * descending and each v_j is phase-normalised (largest-modulus entry, lowest
 * index on ties, real positive; u_j takes the same phase).  V is in/out
 * [F][N][k]; U [F][N][k]; sigma [F][k]; all device.  Errors as rr_sketch. */
rr_status rr_modes(rr_factors* f, int k, void* V, void* U, double* sigma,
                   int orthogonalize, double refine_tol, int max_refine,
                   rr_info* info);

/* Algorithm 1, first step: the test matrix alone.  omega[f][n][j] =
 * phi[n] * g(seeds[f], n, j) (phi NULL: 1), g the Philox-4x32-10 + Box-Muller
 * normal deviate described at rr_sketch; imaginary parts are zero.  seeds:
 * host, nshift values; phi, omega: device (omega complex128 [F][N][k]). */
rr_status rr_gaussian(int nshift, int n, int k, const uint64_t* seeds, const double* phi,
                      void* omega, void* stream);

/* The test matrix alone for the Philox kinds (RR_OMEGA_GAUSSIAN,
 * RR_OMEGA_RADEMACHER, RR_OMEGA_SPARSE_RADEMACHER; see rr_omega_kind):
 * omega[f][n][j] = phi[n] * entry(seeds[f], n, j), imaginary parts zero.
 * rr_gaussian is this call with RR_OMEGA_GAUSSIAN.  Errors: RR_ERR_ARG
 * (null, sizes < 1, other kinds, density outside (0, 1]), RR_ERR_CUDA. */
rr_status rr_test_matrix(int nshift, int n, int k, const uint64_t* seeds,
                         const double* phi, int kind, double density,
                         void* omega, void* stream);

/* Gradient of the summed leading gains with respect to the base flow (no
 * counterpart in the paper; it differentiates Eq. 5):
 *
 *   grad += d/d(rho, U, V) sum_f sum_{j<J} sigma_{f,j}^2
 *         = sum_f sum_{j<J} 2 sigma_j Re(a_j^H (dL/dtheta) b_j),
 *   a_j = A^{-H} W^{1/2} u_j,  b_j = A^{-1} W^{-1/2} v_j,  A = s_f I - L,
 *
 * the first-order perturbation of a simple singular value with singular
 * vectors u_j, v_j (d sigma_j = Re(u_j^H dR v_j)).  The 2J solves reuse the
 * factors (with FP64 refinement for FP32 factors); dL/dtheta is the exact
 * derivative of the discrete operator of rr_create_operator with respect to
 * the nodal base-flow values, the base flow the operator was built from.
 * U, V: device [F][N][k] with unit columns (as returned by rr_modes), of
 * which the first J are used; sigma: device [F][k]; grad: device, 3*nx*ny
 * doubles laid out [rho | U | V], each field point-indexed ix*ny + iy,
 * ACCUMULATED into (zero it first; the rho part stays untouched for
 * RR_ADVDIFF_SCALAR).  The result is the gradient of the true leading gains
 * to the accuracy of the given triplets: exact triplets give the exact
 * gradient.  RR_ISO_NS2D_KZ operators: RR_ERR_UNSUPPORTED.
 * Errors: RR_ERR_ARG (J outside [1, k], k outside [1, 64], null),
 * RR_ERR_NOCONV (grad still accumulated), RR_ERR_CUDA. */
rr_status rr_gain_grad(rr_factors* f, int k, int J, const void* U, const void* V,
                       const double* sigma, double refine_tol, int max_refine,
                       double* grad, rr_info* info);

/* Re-factor an existing factors object for F new shifts (same operator,
 * count and precision), reusing its device storage: the per-frequency loop of
 * a frequency sweep without reallocation.  Errors as rr_factor. */
rr_status rr_refactor(rr_factors* f, const double* shifts);

/* ------------------------------------------------------------ batch plans
 * Many resolvent problems of uneven size (grids, shifts, k) as one CUDA
 * graph.  The paper sweeps the frequency (Sec. III.B) with one factorisation
 * per frequency (Sec. III.A); the frequencies are independent problems, so a
 * plan runs them together:
 *  - problems that share an operator form a group with ONE batched block
 *    factorisation over the group's shifts (as rr_factor);
 *  - each group is split by k into sub-batches that run Algorithm 1 (as
 *    rr_sketch then rr_modes with orthogonalize = 0) on the shared factors;
 *  - rr_batch_create runs every problem once eagerly (calibration), records
 *    the data-dependent host decisions of that run (the number of FP64
 *    refinement corrections of every solve, the shifted-CholeskyQR choice of
 *    every QR), then records the same launch sequence under stream capture,
 *    with the groups spread over concurrent stream lanes (longest first),
 *    and instantiates it: rr_batch_run is one cudaGraphLaunch;
 *  - with opts->tune = 1 the plan is tuned on the device by timing the
 *    candidates: the trailing-update kernel of each group's factorisation
 *    (128 x 64 tensor-core tiles or 64 x 64 CUDA-core tiles, on its first
 *    columns), the K-split (1..4 or the built-in choice) of each
 *    sub-batch's tensor-core sweep, and the number of lanes (2, 4, 8, all
 *    groups, and 1 for plans of at most two groups; whole-graph runs).
 * A run reproduces the calibration run's arithmetic (same kernels, same
 * order); after it, the factor flags and a device log of every solve's
 * final residual and every QR's breakdown flag are checked on the host.
 *
 * Problem i: op (problems may share operators; all on one device), shift
 * s = s_re + i s_im, k in [1, min(64, N)], Philox key seed (the test
 * matrix of rr_sketch, scaled by the operator's Phi of Eq. 9 when
 * opts->use_phi), outputs V, U (device complex128 [N][k]), sigma and
 * sigma_halko (device [k]; sigma_halko may be NULL) as rr_sketch /
 * rr_modes define them.  The plan keeps the problems' pointers: outputs are
 * written on every run, and the operators must outlive the plan. */
typedef struct rr_batch rr_batch;

typedef struct {
  rr_operator* op;
  double s_re, s_im;
  int k;
  uint64_t seed;
  void* V;
  void* U;
  double* sigma;
  double* sigma_halko;
} rr_problem;

typedef struct {
  int use_phi;        /* 1: test matrix scaled by Phi (Eq. 9)              */
  double refine_tol;  /* FP64 refinement tolerance (FP32 factors)          */
  int max_refine;     /* refinement cap per solve                          */
  int tune;           /* 1: time candidate schedules on the device         */
  int lanes;          /* concurrent lanes; 0: tuned, or min(groups, 4)     */
} rr_batch_opts;

typedef struct {
  int groups;             /* operators (one factorisation each)             */
  int views;              /* (operator, k) sub-batches                      */
  int lanes;              /* stream lanes of the captured graph             */
  int graph_nodes;        /* nodes of the graph                             */
  int kernel_nodes;       /* kernel launches per rr_batch_run               */
  int cuda_core_updates;  /* groups tuned to the CUDA-core trailing update  */
  double plan_ms;         /* host wall time of rr_batch_create, of which:   */
  double calib_ms;        /*   calibration (eager factor + Algorithm 1)     */
  double tune_ms;         /*   kernel and lane tuning                       */
  double capture_ms;      /*   final capture + instantiation               */
  double tuned_ms;        /* best whole-graph time seen by the lane tuner   */
} rr_batch_desc;

/* Build a plan (calibration run, optional tuning, capture, one validation
 * run).  opts NULL = {use_phi 1, refine_tol 1e-10, max_refine 10, tune 0,
 * lanes 0}.  Errors: RR_ERR_ARG (no problems, null pointers, k out of
 * range, operators on different devices, non-finite shifts, lanes outside
 * [0, 64]), RR_ERR_NOMEM, RR_ERR_SINGULAR, RR_ERR_RANK, RR_ERR_TIMEOUT,
 * RR_ERR_CUDA; *out is NULL on error. */
rr_status rr_batch_create(int nprob, const rr_problem* probs, rr_precision prec,
                          const rr_batch_opts* opts, rr_batch** out);

/* Run the plan's graph on stream (NULL: the plan's own stream), wait for it
 * and check it: RR_ERR_SINGULAR / RR_ERR_TIMEOUT from the factor flags,
 * RR_ERR_RANK from a QR breakdown, RR_ERR_NOCONV when some solve's final
 * relative residual exceeds both refine_tol and 4x the one the calibration
 * run reached (possible only after rr_batch_set_shifts: rebuild the plan).
 * info (may be NULL): largest residual, corrections and condition estimate. */
rr_status rr_batch_run(rr_batch* b, void* stream, rr_info* info);

/* Replace the shifts of all problems (host, 2*nprob doubles, problem order)
 * for later runs: the graph reads them from device memory, so a frequency
 * sweep reuses one plan.  The refinement schedule stays the calibrated one
 * (checked by rr_batch_run). */
rr_status rr_batch_set_shifts(rr_batch* b, const double* shifts);

rr_status rr_batch_describe(const rr_batch* b, rr_batch_desc* desc);
rr_status rr_batch_destroy(rr_batch* b);

/* Instrumentation (no counterpart in the paper).  rr_launch_count: kernels
 * launched by this library in this process since the last rr_profile_start.
 * rr_profile_start(mask): reset the counters and time every later launch of
 * the kernel classes whose bit is set in mask with a CUDA event pair on the
 * launching stream.  Classes: 0 Schur update, 1 pivoted panel, 2 row block,
 * 3 trailing update (tensor cores), 4 finalize (inverse + X), 5 block sweep
 * step, 6 FP64 residual, 7 Gram, 8 right multiply, 9 small k x k kernels,
 * 10 inner slab update of the wide factorisation (CUDA cores).
 * rr_profile_read(cls): summed event time (ms) and launches of a class. */
long long rr_launch_count(void);
rr_status rr_profile_start(unsigned mask);
rr_status rr_profile_read(int cls, double* ms, long long* launches);

/* Diagnostics of the bounded device-side waits (no counterpart in the paper;
 * for tests of the RR_ERR_TIMEOUT path).  Every mbarrier wait of the
 * tensor-core kernels polls at most `tries` times (0 restores the default,
 * 2^22) before the kernel records a timeout, drains what it has in flight,
 * frees its tensor memory and returns; the call that launched it then
 * returns RR_ERR_TIMEOUT.  stall_launches > 0 makes that many of the next
 * tensor-core sweep launches stall on purpose: the control thread of their
 * first CTA issues no copy and no MMA, so that CTA's first wait runs out with
 * nothing in flight.  Process-wide, not thread-safe; for tests only. */
rr_status rr_debug_waits(unsigned tries, int stall_launches);

/* Measured arithmetic peaks for roofline fractions (no counterpart in the
 * paper).  Runs a microbenchmark whose operands stay on chip on `device` and
 * returns the best of five timed launches (after a warm-up) in TFLOP/s:
 * kind 0 tcgen05.mma kind::tf32 (128 x 256 tiles, FP32 accumulation in
 * TMEM), 1 tcgen05.mma kind::f16 with BF16 operands, 2 FP64 FMA and 3 FP32
 * FMA on the CUDA cores (2 flops per FMA).  Synchronous.  Errors:
 * RR_ERR_ARG, RR_ERR_TIMEOUT, RR_ERR_CUDA. */
rr_status rr_measure_peak(int kind, int device, double* tflops);

/* Number of problems (shifts) and precision of a factors object. */
rr_status rr_factors_dims(const rr_factors* f, int* nshift, int* prec);

#ifdef __cplusplus
}
#endif
#endif /* RR_H */
