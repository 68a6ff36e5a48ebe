/*
 * pmg.h -- C ABI of the GB300-native p-multigrid solver for nodal IP/LDG
 * discretisations of the Poisson equation on Cartesian grids.
 *
 * Method: J. Stiller, "Robust multigrid for high-order discontinuous Galerkin
 * methods: a fast Poisson solver suitable for high-aspect ratio Cartesian
 * grids", arXiv 1603.02524.  Section, equation and algorithm numbers below
 * refer to that paper.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Vectors are contiguous fp64 arrays (fp32 nowhere crosses the ABI) in the
 *    element-major layout u[e_z][e_y][e_x][k][j][i]: elements in x-fastest
 *    lexicographic order, inside an element the (P+1)^dim GLL nodal values with
 *    x fastest.  In 2-D drop e_z and k.  Level l has order P_l = 2^l and
 *    n_elem_x * n_elem_y [* n_elem_z] * (P_l + 1)^dim entries.
 *  - Pointers named *_dev are device pointers on the current CUDA device; the
 *    caller allocates and owns them.  The library owns only the grid/hierarchy
 *    objects and their internal workspace (allocated in pmg_hierarchy_build,
 *    freed in pmg_hierarchy_destroy).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls enqueue work on that stream and return without synchronising,
 *    except pmg_solve / pmg_solve_host / pmg_batch_solve, which synchronise
 *    before returning (the first pmg_solve of a hierarchy once per CG
 *    iteration, later ones and batches once per call).
 *  - Every call returns a pmg_status (0 = PMG_OK) and never throws.  Invalid
 *    arguments are rejected before any work is enqueued.  Kernel launch errors
 *    return PMG_ECUDA.  Conditions detected on the device (a non-finite residual,
 *    CG breakdown, a bounded device wait that gave up) are written to the
 *    hierarchy's device status word: pmg_solve / pmg_solve_host / pmg_batch_solve
 *    stop the iteration and return them (PMG_ENAN, PMG_EBREAKDOWN, PMG_ETIMEOUT)
 *    after their synchronisation; the asynchronous calls (pmg_smooth, pmg_vcycle,
 *    pmg_schwarz_sweep) leave them there for pmg_device_status.
 *  - A hierarchy object is not thread safe: calls that use it must not run
 *    concurrently (they share its workspace).
 */
#ifndef PMG_H_
#define PMG_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pmg_grid_s* pmg_grid;
typedef struct pmg_hier_s* pmg_hier;
typedef struct pmg_batch_s* pmg_batch;

typedef enum {
  PMG_OK = 0,
  PMG_EINVAL = -1,       /* invalid argument or unsupported configuration */
  PMG_ENOMEM = -2,       /* device or host allocation failed */
  PMG_ECUDA = -3,        /* CUDA runtime / launch error */
  PMG_ENOCONV = -4,      /* pmg_solve: tolerance not reached within max_iter */
  PMG_EBREAKDOWN = -5,   /* pmg_solve: p^T A p <= 0 or delta <= 0 */
  PMG_ENAN = -6,         /* pmg_solve: non-finite residual */
  PMG_ETIMEOUT = -7      /* a bounded device wait gave up (tcgen05 patch kernel, PMG_PREC_MIXED_TF32):
                            the corrections of that sweep are incomplete */
} pmg_status;

/* Smoother (Sec. 3.1): additive element-centred (EA) or face-centred (FA). */
enum { PMG_SMOOTHER_EA = 0, PMG_SMOOTHER_FA = 1 };
/* Overlap policy N_o (Sec. 4.3): 0 -> none; LEVEL -> 1 + round(P_l/8)
 * (reproduces Tables 2-3); LEVEL_FLOOR -> 1 + floor(P_l/8) as printed. */
enum { PMG_OVERLAP_ZERO = 0, PMG_OVERLAP_LEVEL = 1, PMG_OVERLAP_LEVEL_FLOOR = 2 };
/* Weighting of the additive update, Eqs. (weight function:ec/fc). */
enum { PMG_WEIGHT_UNWEIGHTED = 0, PMG_WEIGHT_ARITHMETIC = 1, PMG_WEIGHT_CUBIC = 3,
       PMG_WEIGHT_QUINTIC = 5 };
/* Arithmetic of the V-cycle: FP64 everywhere; or an fp32 V-cycle (smoother,
 * residuals, transfers) inside the FP64 flexible CG (spec extension), with
 * the patch transforms on the SIMT cores (MIXED) or on the tensor cores (MIXED_TC:
 * mma.sync TF32 with the 3xTF32 split, i.e. fp32-level products and fp32
 * accumulation; 3-D patches of at most 32 nodes per axis, others stay SIMT). */
enum { PMG_PREC_FP64 = 0, PMG_PREC_MIXED = 1, PMG_PREC_MIXED_TC = 2, PMG_PREC_MIXED_TF32 = 3 };
/* PMG_PREC_MIXED_TF32: one TF32 product per multiply-add (10-bit operand
 * mantissas, fp32 accumulation), the patch line passes as tcgen05 MMAs with the
 * operands in shared memory and the accumulators in tensor memory (3-D patches
 * of at most 32 nodes per axis; others stay SIMT): a lower-precision
 * preconditioner whose effect on the iteration count the flexible CG absorbs. */
/* Preconditioner of the CG iteration (Algorithm 2). */
enum { PMG_PC_VCYCLE = 0, PMG_PC_NONE = 1 };
/* Arithmetic of the CG's operator apply (spec extension): FP64, or
 * emulated FP64 in double-float (DF: each value the sum of two fp32 words,
 * about 48 significant bits, products split exactly by FMA and sums by TwoSum)
 * on the FP32 pipes, which on GB300 issue ~60x the FP64 rate.  DF needs the
 * vector and operator magnitudes within fp32's exponent range (~1e-30..1e30). */
enum { PMG_OUTER_FP64 = 0, PMG_OUTER_DF = 1 };

typedef struct {
  int smoother;        /* PMG_SMOOTHER_*                                  (default EA) */
  int overlap;         /* PMG_OVERLAP_*                                   (default LEVEL) */
  int weighting;       /* PMG_WEIGHT_*                                    (default QUINTIC) */
  int ns_pre, ns_post; /* smoothing steps per level                       (default 1, 1) */
  int variable_v;      /* 1: n_s,l = n_s * 2^(L-l) (variable V-cycle)     (default 0) */
  double omega;        /* damping of the additive update                  (default 1) */
  int precision;       /* PMG_PREC_*                                      (default FP64) */
  int max_iter;        /* MGCG iteration cap (Algorithm 2, i_max)         (default 100) */
  /* Per-level smoother parameters (index = level l = 1..L; entry 0 unused), e.g.
   * from a learned model; 0 selects the default.  omega_level: damping of level l
   * (default omega).  tau_level in (0, 1]: width of the weight transition zone
   * relative to the paper's (w_H over tau * dxi_O; w_F = 1/2 [1 + phi((1-|xi_F|)/tau)]);
   * default 1 = the paper's weights.  Any tau in (0, 1] keeps the weights a
   * partition of unity. */
  double omega_level[8];
  double tau_level[8];
  int preconditioner;  /* PMG_PC_*: the V-cycle of Algorithm 1 (default), or none:
                          z = r, i.e. plain CG, the paper's reference method of Sec. 4 */
  int outer_apply;     /* PMG_OUTER_*: arithmetic of the CG's own operator apply
                          (residual g - A u and q = A p of Algorithm 2) (default FP64) */
  int nrhs;            /* right-hand sides solved together, 1..64 (default 1): every
                          vector of the hierarchy then holds nrhs vectors of the grid back
                          to back (vector r at offset r * n, n = the grid's unknowns at that
                          level), pmg_level_info reports nrhs * n, and each kernel launch
                          covers all of them with one copy of the tables.  Internally the
                          copies are stacked along the grid's last axis with walls between
                          them, hence homogeneous Dirichlet grids only (periodic: EINVAL).
                          pmg_solve runs nrhs independent CG iterations (own scalars,
                          convergence test and result each) in one loop until all have
                          stopped; stats then points to nrhs entries. */
} pmg_options;

typedef struct {
  int iterations;      /* CG iterations performed (= V-cycles applied)     */
  double r0;           /* ||g - A u_0||_2                                    */
  double rn;           /* ||r|| at exit                                      */
  double* history;     /* optional host array of max_iter+1 entries, or NULL */
  int status;          /* pmg_status of this solve (pmg_solve also returns it) */
  int device_loop;     /* 1: the iterations ran as a device-side loop inside one
                          CUDA graph launch; 0: host-driven iterations        */
} pmg_stats;

/* Fill *opt with the defaults listed above. */
void pmg_options_default(pmg_options* opt);

/*
 * Create a Cartesian grid description (Sec. 2.2).
 *   dim       2 or 3.
 *   P         polynomial order, a power of two, 1 <= P <= 32
 *             (levels P_l = 2^l, Sec. 3.2).
 *   n_elem    elements per axis (n_elem[2] ignored in 2-D); each >= 1, and >= 2
 *             when periodic.
 *   spacing   host arrays: spacing[d][m] = width of element m along axis d (> 0).
 *   periodic  1: periodic domain (the paper's Sec. 2.1 setting); 0: homogeneous
 *             Dirichlet walls (odd-reflection ghost element, symmetric Nitsche).
 *   mu_star   penalty factor, mu = mu0 (1 + mu_star) (Sec. 2.4); the paper uses 1.
 *   beta      LDG auxiliary parameter per axis (Eq. flux:num:sigma); 0 -> interior
 *             penalty (IP), 1/2 -> LDG as in Table 2.  NULL = all zero.
 * The host arrays are copied; *out receives a handle freed by pmg_grid_destroy.
 */
int pmg_grid_create(int dim, int P, const int n_elem[3], const double* const spacing[3],
                    int periodic, double mu_star, const double beta[3], pmg_grid* out);
void pmg_grid_destroy(pmg_grid g);

/*
 * Node coordinates (host): out[m*(P+1)+i] = physical coordinate of GLL node i
 * of element m along axis `axis` at the grid's finest order P.  `out` must hold
 * n_elem[axis]*(P+1) doubles.
 */
int pmg_grid_coords(pmg_grid g, int axis, double* out);

/*
 * Build the p-multigrid hierarchy (Sec. 3.2): for every level P_l = 2^l the
 * re-discretised operator tables (Eq. L:generic), the Schwarz patch
 * eigen-tables (Sec. 3.1, fast diagonalisation), the interpolation I_l and
 * the level vectors; the coarse P = 1 problem is solved exactly (see
 * pmg_coarse_solve).  Allocates device memory on the current device.
 * opt == NULL uses the defaults.  *out is freed by pmg_hierarchy_destroy.
 */
int pmg_hierarchy_build(pmg_grid g, const pmg_options* opt, pmg_hier* out);
void pmg_hierarchy_destroy(pmg_hier h);

/* Number of levels L+1 and, per level, order and vector length (nrhs vectors of
 * the grid for a hierarchy with several right-hand sides). */
int pmg_num_levels(pmg_hier h);
int pmg_level_info(pmg_hier h, int level, int* P_l, long long* ndof);

/* Au_dev = A_l u_dev  (Eq. discrete problem; 3-D tensor form). level in 0..L.
 * On the finest level L this is the CG's own apply, in the hierarchy's
 * outer_apply arithmetic (FP64 by default); coarser levels are FP64. */
int pmg_apply(pmg_hier h, int level, const double* u_dev, double* Au_dev, void* stream);

/* r_dev = f_dev - A_l u_dev (arithmetic as pmg_apply). */
int pmg_residual(pmg_hier h, int level, const double* u_dev, const double* f_dev, double* r_dev,
                 void* stream);

/* g_dev = M f_nodal_dev: the discrete right-hand side g = M f (Sec. 2.4). */
int pmg_rhs(pmg_hier h, const double* f_nodal_dev, double* g_dev, void* stream);

/*
 * `nsteps` Schwarz iterations on level l >= 1 (Sec. 3.1): each EA step is
 * r = f - A u followed by u += omega * sum_s R_s^T (w_s A_ss^{-1} R_s r); each
 * FA step does one such sweep per direction with the residual recomputed in
 * between.  u_dev is updated in place.  Runs in the hierarchy's precision
 * (mixed: fp32 arithmetic, fp64 in and out).
 */
int pmg_smooth(pmg_hier h, int level, double* u_dev, const double* f_dev, int nsteps,
               void* stream);

/* fc_dev = I_l^T rf_dev: restriction from level l to l-1 (Sec. 3.2), l >= 1. */
int pmg_restrict(pmg_hier h, int level, const double* rf_dev, double* fc_dev, void* stream);

/* uf_dev += I_l uc_dev: prolongation (embedded interpolation) from l-1 to l. */
int pmg_prolong(pmg_hier h, int level, const double* uc_dev, double* uf_dev, void* stream);

/*
 * u0_dev = A_0^+ f0_dev at P = 1 (Algorithm 1, coarse-grid solution).  Solved
 * exactly by a global tensor-product fast diagonalisation (the coarse operator
 * has the same Kronecker structure as A_ss); on periodic grids the right-hand
 * side is projected onto range(A_0) and the zero mode dropped.
 */
int pmg_coarse_solve(pmg_hier h, const double* f0_dev, double* u0_dev, void* stream);

/*
 * pmg_coarse_solve without any device workspace of its own (the paper has no
 * counterpart; this is a library-integration entry point).  Same arguments,
 * same result as pmg_coarse_solve; the call allocates nothing.  Its two scratch
 * vectors live in a fixed 4 MiB device array compiled into the library, so it
 * suits callers that cannot call cudaMalloc while they solve: code inside a host
 * framework whose own allocator owns all device memory and forbids side
 * allocations, or a caller that has reserved its memory up front and must not
 * grow it mid-run.
 *  - Limit: the P = 1 problem may have at most 262 144 unknowns (32^3 elements in
 *    3-D); larger hierarchies get PMG_EINVAL and a message in pmg_last_error.
 *  - The first call on each device looks up the array's device address; make that
 *    first call before any stream capture.
 *  - All calls in the process share the one array per device: calls that may run
 *    concurrently on the GPU (different streams, different hierarchies) race and
 *    must be serialised by the caller.
 * The hierarchy itself (tables, f0/u0 sizes) comes from pmg_hierarchy_build.
 */
int pmg_coarse_solve_static(pmg_hier h, const double* f0_dev, double* u0_dev, void* stream);

/* u_dev = MultigridCycle(0, f_dev): one V-cycle of Algorithm 1 on the finest level. */
int pmg_vcycle(pmg_hier h, const double* f_dev, double* u_dev, void* stream);

/*
 * Inexact multigrid-preconditioned CG (Algorithm 2; beta by Golub-Ye,
 * z^T (r - r_old) / delta).  g_dev: right-hand side (periodic grids: projected
 * onto zero mean internally).  u_dev: initial guess in, solution out; the solve checks on
 * the device whether the guess is all zero and then takes r_0 = g without an operator apply.
 * Stops when ||r||_2 <= rtol * ||r_0||_2 or after opt.max_iter iterations
 * (PMG_ENOCONV, u holds the last iterate).  stats may be NULL.  A hierarchy with
 * nrhs > 1 solves its nrhs right-hand sides (g_dev, u_dev: nrhs vectors back to back),
 * each with its own test; stats[0..nrhs) receive their statistics and the call returns
 * the status of the first right-hand side that failed, else PMG_OK.
 */
int pmg_solve(pmg_hier h, const double* g_dev, double* u_dev, double rtol, pmg_stats* stats,
              void* stream);

/*
 * As pmg_solve, but g_host / u_host are host arrays (pinned memory is fastest):
 * the host->device copies of g and u, the solve and the device->host copy of u
 * all run inside this call, on the hierarchy's internal device buffers (with
 * nrhs > 1: nrhs vectors back to back in each array, stats as for pmg_solve).
 */
int pmg_solve_host(pmg_hier h, const double* g_host, double* u_host, double rtol,
                   pmg_stats* stats, void* stream);

/*
 * Batched solves (spec extension; the paper solves one problem at a
 * time).  pmg_batch_create records `count` independent MGCG solves (Algorithm
 * 2), solve i on hierarchy hiers[i] with right-hand side g_dev[i] and initial
 * guess / solution u_dev[i], into one CUDA graph: one branch per solve, each
 * with its iterations in a device-side loop and its own convergence test
 * ||r||_2 <= rtol ||r_0||_2 (cap: that hierarchy's max_iter).  Grids may differ
 * in size, order, spacing, options and number of right-hand sides (a hierarchy
 * built with nrhs > 1 solves all of its right-hand sides in its branch: g_dev[i]
 * and u_dev[i] then hold nrhs vectors each); the hierarchies must be distinct
 * (else PMG_EINVAL), since a hierarchy holds one solve's workspace.  The vectors
 * are the caller's and are bound to the batch: pmg_batch_solve reads g_dev[i]
 * and u_dev[i] where they are at that call.
 *   pmg_batch_solve  runs all solves with one graph launch on `stream`,
 *                    synchronises once, fills stats (may be NULL; history
 *                    arrays optional) with one entry per right-hand side, solve
 *                    by solve, and returns PMG_OK or the status of the first
 *                    right-hand side (in that order) that failed.
 *   pmg_batch_destroy  frees the graph; destroy a batch before its hierarchies.
 * Creation runs one V-cycle on each hierarchy that has not run yet (kernel
 * set-up) and synchronises the device.  Not thread safe with respect to the
 * hierarchies it holds.
 */
int pmg_batch_create(int count, const pmg_hier* hiers, const double* const* g_dev,
                     double* const* u_dev, double rtol, pmg_batch* out);
int pmg_batch_solve(pmg_batch b, pmg_stats* stats, void* stream);
void pmg_batch_destroy(pmg_batch b);
/* Text of the last error recorded on a batch ("" if none). */
const char* pmg_batch_last_error(pmg_batch b);

/*
 * Autotuner (spec extension): times the Schwarz patch kernel of every
 * level with each candidate CTA size (multiples of 32 from 64 to 512) on the
 * level's own work vectors and keeps the fastest; a line pass strides over its
 * lines by the CTA size, so every candidate computes the same result.  Results
 * are cached per patch shape and patch count for the process.  Enqueues on
 * `stream` and synchronises it; overwrites the hierarchy's level work vectors.
 * Call it before pmg_batch_create: a batch keeps the launch shapes it captured.
 * pmg_tuned_threads returns the CTA size in use for (level >= 1, family as in
 * pmg_schwarz_sweep), 0 = the kernel's default, or PMG_EINVAL.
 */
int pmg_hierarchy_autotune(pmg_hier h, void* stream);
int pmg_tuned_threads(pmg_hier h, int level, int family);

/*
 * One additive Schwarz sweep without the residual (Sec. 3.1, Eq.
 * correction:global): u_dev += omega * sum_s R_s^T (w_s A_ss^{-1} R_s r_dev)
 * over one subdomain family of level l >= 1.  family = -1: the element-centred
 * subdomains (hierarchy built with the EA smoother); family = d in 0..dim-1:
 * the face-centred subdomains normal to axis d (FA smoother).  fp64 in and
 * out; in mixed precision the sweep runs in fp32 on staged copies.
 */
int pmg_schwarz_sweep(pmg_hier h, int level, int family, const double* r_dev, double* u_dev,
                      void* stream);

/*
 * Learned smoother parameters (spec extension; the paper fixes omega = 1
 * and the weight transition): a small fp32 MLP mapping the features of one level
 * (log2 P_l, N_o, three log2 element aspect ratios, l/L) to two raw outputs,
 * which paper_1603_02524_gb300.learned maps to (omega_l, tau_l) for
 * pmg_options.omega_level / tau_level.  Network 6 -> 64 tanh -> 64 tanh -> 2;
 * parameters theta packed as W1[6][64], b1[64], W2[64][64], b2[64], W3[64][2], b3[2]
 * (PMG_MLP_NPARAM floats).  All pointers are device pointers; row-major batches.
 */
#define PMG_MLP_IN 6
#define PMG_MLP_HIDDEN 64
#define PMG_MLP_OUT 2
#define PMG_MLP_NPARAM 4738
/* y[batch][2] = MLP(x[batch][6]); h1, h2 (batch x 64, may be NULL) keep the hidden
 * activations for pmg_mlp_backward. */
int pmg_mlp_forward(const float* theta, const float* x, int batch, float* y, float* h1, float* h2,
                    void* stream);
/* grad[PMG_MLP_NPARAM] = d loss / d theta and *loss (device scalar, may be NULL) for
 * loss = (1/batch) sum_b weight_b sum_o (y_bo - target_bo)^2 (weight may be NULL = 1),
 * from the activations of pmg_mlp_forward.  work: batch x PMG_MLP_NPARAM floats of
 * scratch (per-sample gradients, summed in a fixed order: deterministic). */
int pmg_mlp_backward(const float* theta, const float* x, const float* h1, const float* h2,
                     const float* y, const float* target, const float* weight, int batch, float* grad,
                     float* loss, float* work, void* stream);
/* One Adam step (bias-corrected, step >= 1) on n parameters with moments m, v. */
int pmg_mlp_adam(float* theta, const float* grad, float* m, float* v, int n, int step, float lr,
                 float beta1, float beta2, float eps, void* stream);

/* Text for a status code; last error detail of a hierarchy (may be ""). */
const char* pmg_status_string(int status);
const char* pmg_last_error(pmg_hier h);

/* Benchmark hook: one sweep of (level, family) in the hierarchy's own
 * arithmetic (fp32 in mixed precision) on its internal level buffers, whose
 * contents are arbitrary; no staging copies, nothing the caller owns is read
 * or written.  For timing the patch kernel alone. */
int pmg_schwarz_sweep_native(pmg_hier h, int level, int family, void* stream);

/* Multiply-adds one pmg_schwarz_sweep of (level, family) executes in its six
 * eigenvector line passes, as implemented (even-odd split on centro-symmetric
 * axes): the figure the benchmark's roofline uses.  Host only. */
int pmg_schwarz_sweep_fma(pmg_hier h, int level, int family, double* fma);

/* Benchmark hook (not part of the paper's method): enqueues on `stream` one launch
 * of a multiply-add throughput probe on the FP64 (fp64 != 0) or FP32 pipes, every
 * resident thread of every SM running independent multiply-add chains for `iters`
 * loop trips, and stores in *flops the floating-point operations of that launch
 * (2 per multiply-add).  Timing the launch with CUDA events on `stream` gives the
 * measured peak that the roofline fractions of ALU-bound kernels divide by.
 * Allocates nothing.  PMG_EINVAL for iters < 1 or a null flops, PMG_ECUDA on a
 * launch error. */
int pmg_fma_probe(int fp64, int iters, void* stream, double* flops);

/* Number of CUDA kernels this library has launched in this process so far
 * (all hierarchies, all devices); for counting launches in a timed region. */
unsigned long long pmg_kernel_launches(void);

/* Number of thread blocks of the tcgen05 patch kernel (PMG_PREC_MIXED_TF32)
 * that gave up waiting for their tensor-core MMAs (each wait is bounded at about
 * one second; such a block stops early and its corrections are incomplete) since
 * the last call, on the current device; the count is reset.  Synchronises the
 * device.  Returns PMG_OK, or PMG_EINVAL for a null pointer, PMG_ECUDA on a CUDA
 * error. */
int pmg_tc_timeouts(unsigned int* count);

/*
 * Device status word of a hierarchy (see the conventions at the top): enqueues its
 * read on `stream`, synchronises that stream, stores the value in *status (PMG_OK,
 * or PMG_ENAN / PMG_EBREAKDOWN / PMG_ETIMEOUT left by an earlier call on this
 * hierarchy) and resets it to PMG_OK.  pmg_solve resets the word when it starts.
 * Returns PMG_OK, PMG_EINVAL (null argument) or PMG_ECUDA.
 */
int pmg_device_status(pmg_hier h, void* stream, int* status);

/*
 * Test hook for the failure path of the bounded device waits (not part of the
 * paper's method).  limit_us > 0: every block of this hierarchy's tcgen05 patch
 * kernels (PMG_PREC_MIXED_TF32, 3-D patches of 13^3 nodes and more) waits after its
 * first MMAs on an mbarrier that nothing completes, gives up after limit_us
 * microseconds, lets its MMAs finish (bounded wait of about one second), frees its
 * tensor memory and stops, counting itself in pmg_tc_timeouts and setting
 * PMG_ETIMEOUT in the hierarchy's device status word; no fault, trap or unbounded
 * wait is involved.  limit_us = 0 restores normal operation.  Captured graphs of
 * the hierarchy are discarded (synchronises the device).  PMG_EINVAL for a null
 * hierarchy or limit_us > 10^6.
 */
int pmg_test_stall_tc_waits(pmg_hier h, unsigned int limit_us);

#ifdef __cplusplus
}
#endif
#endif /* PMG_H_ */
