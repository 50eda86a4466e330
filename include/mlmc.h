/*
 * mlmc.h -- C ABI of the GB300 (sm_103a) multilevel Monte Carlo multigrid library.
 *
 * The library computes the data-parallel hot path of the multilevel Monte Carlo
 * method of Gmeiner, Drzisga, Ruede, Scheichl and Wohlmuth, "Scheduling massively
 * parallel multigrid for multilevel Monte Carlo methods": samples
 * Y_l = Q_l - Q_{l-1} of the level differences (Sec. 2.2, Eq. 8, Algorithm 1), where
 * both Q's of one sample come from solves of the model problem -div(k grad u) = f on
 * D = (0,1)^3 with homogeneous Dirichlet data (Sec. 3, Eq. 16) on the SAME
 * realisation of a lognormal coefficient k = exp(Z) (Sec. 3.2), by geometric
 * multigrid on structured grids.
 *
 * Discretisation (fixed by this library; the paper's P1 finite elements and SPDE
 * field sampler are replaced):
 *   grid     nodes (i h, j h, k h), i,j,k = 0..n-1, n = 2^p + 1 (p >= 2), h = 1/(n-1);
 *            u = 0 on boundary nodes;
 *   operator (A u)_p = h^-2 sum_{q in N(p)} k_pq (u_p - u_q), 7-point, harmonic-mean
 *            faces k_pq = 2 k_p k_q / (k_p + k_q) of the nodal coefficient;
 *   field    log k(x) = sigma sqrt(2/M) sum_m cos(w_m . x + b_m), random Fourier features
 *            of a stationary covariance: w_m ~ N(0, I/ell^2) for the Gaussian covariance
 *            sigma^2 exp(-r^2 / (2 ell^2)) (MLMC_COV_GAUSS), w_m ~ multivariate Cauchy,
 *            density proportional to (1 + ell^2 |w|^2)^-2, for the exponential
 *            covariance sigma^2 exp(-r / ell) of Sec. 3.2 (MLMC_COV_EXP);
 *            b_m ~ U[0, 2 pi), drawn by Philox4x32-10 keyed by (run_seed, sample_id):
 *            key = (seed low, seed high), counter = (id low, id high, m, c), c = 0,1,2;
 *            the 12 words give six 53-bit uniforms U = ((a>>5) 2^26 + (b>>6) + 1/2) 2^-53
 *            from consecutive word pairs; Box-Muller on (U1,U2), (U3,U4) gives
 *            g1, g2 (cos, sin of the first pair) and g3 (cos of the second);
 *            w_m = (g1, g2, g3) / ell (Gaussian) or (g1, g2, g3) / (ell |g4|) with g4
 *            the sin of the second pair (exponential), b_m = 2 pi U5;
 *   solver   V(nu1, nu2) cycles: red ((i+j+k) even) then black Gauss-Seidel sweeps,
 *            full weighting (1/64)(1,2,1)^3, trilinear prolongation, rediscretised
 *            coarse operators (k injected), exact solve on the 5^3 grid; cycles repeat
 *            until ||f - A u||_2 / ||f||_2 over interior nodes <= rtol;
 *   QoI      Q = mean of u over [0.25, 0.75]^3 by the tensor trapezoid rule.
 *
 * Memory layout of every grid array: batch-outermost, then z, y, x with x fastest:
 *   element (s, z, y, x) at offset ((s * n + z) * n + y) * n + x, n^3 per sample,
 *   boundary nodes included.
 *
 * Conventions:
 *   - Every call returns an int status: MLMC_OK (0) or a negative MLMC_ERR_* code;
 *     mlmc_last_error_string() then describes the failure (thread-local).
 *   - Device buffers passed in are owned by the caller and must stay valid until the
 *     stream work of the call has completed; the library never frees them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Calls that say "blocking" synchronise `stream` before returning; the others only
 *     enqueue work, except where host-side outputs are requested.
 *   - Only one GPU is used: the device current on the calling thread.
 *   - There is no CPU fallback: without a usable CUDA device every compute call
 *     returns MLMC_ERR_CUDA.
 */
#ifndef MLMC_GB300_H
#define MLMC_GB300_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define MLMC_OK 0
#define MLMC_PENDING 1
#define MLMC_ERR_INVALID (-1)
#define MLMC_ERR_OOM (-2)
#define MLMC_ERR_NOT_CONVERGED (-3)
#define MLMC_ERR_TIMEOUT (-4)
#define MLMC_ERR_CUDA (-5)
#define MLMC_ERR_BUSY (-6)
#define MLMC_ERR_NOT_FOUND (-7)
#define MLMC_ERR_CANCELLED (-8)

/* ---- element types of grid buffers ---- */
#define MLMC_F64 0
#define MLMC_F32 1

/* ---- solver precision ---- */
#define MLMC_PREC_F64 0   /* every step in FP64 */
#define MLMC_PREC_MIXED 1 /* FP32 faces, FP32 V-cycle as correction; FP64 residual and update */

/* ---- covariance of log k ---- */
#define MLMC_COV_GAUSS 0 /* sigma^2 exp(-|x-y|^2 / (2 ell^2)) */
#define MLMC_COV_EXP 1   /* sigma^2 exp(-|x-y| / ell), the paper's covariance (Sec. 3.2) */
#define MLMC_COV_SPDE 2  /* the paper's sampler for that covariance (Sec. 3.2): log k =
                            sqrt(8 pi kappa sigma^2) Z, (kappa^2 - Laplace) Z = W, kappa =
                            1/ell, W white noise; cell-centred finite volumes on the
                            zero-flux box (-1/2 - h/2, 3/2 - h/2)^3 of 2(n-1) cells of side
                            h = 1/(n-1) per axis (D's node j at the centre of cell
                            j + (n-1)/2); W(cell) sums one Philox normal (Marsaglia's polar
                            method, FP32, correctly rounded steps and an atanh-series log)
                            per octant of side h_f/2, h_f the spacing of the pair's fine
                            grid, so both grids of a level pair share one W; each grid's
                            system solved by cell-centred multigrid to a relative residual
                            of 1e-12. M is not used. Grids up to 1025 nodes per axis. */

/* Parameters of the lognormal random field (Sec. 3.2; Fourier-feature form above).
   A zero-initialised `cov` selects the Gaussian covariance. */
typedef struct {
  uint64_t run_seed; /* Philox key */
  double sigma2;     /* variance of log k, >= 0 */
  double ell;        /* correlation length, > 0 */
  int M;             /* number of Fourier features, >= 1 */
  int cov;           /* MLMC_COV_GAUSS or MLMC_COV_EXP */
} mlmc_field_cfg;

/* Smoother implementations (all compute the same red-black sweep, bit for bit). */
#define MLMC_SMOOTH_AUTO 0      /* the tuned choice for the grid size (mlmc_autotune), else a default */
#define MLMC_SMOOTH_TWO_PASS 1  /* one kernel per colour */
#define MLMC_SMOOTH_FUSED_32x8 2  /* both colours in one z-marching pass, 32x8 x-y tiles */
#define MLMC_SMOOTH_FUSED_32x16 3
#define MLMC_SMOOTH_FUSED_64x8 4
#define MLMC_SMOOTH_BULK_32x8 5   /* fused, plane rows staged by TMA bulk copies on mbarriers */
#define MLMC_SMOOTH_BULK_32x16 6
#define MLMC_SMOOTH_BULK_64x8 7
#define MLMC_SMOOTH_NODAL 8      /* two colour passes that read the nodal coefficient instead of the
                                    stored faces, recomputing the six harmonic faces, D and 1/D of
                                    each updated node with fast reciprocals (faces within a few ulps
                                    of the stored ones, 4 instead of 7 words per node and sweep).
                                    FP32 correction cycles only (MLMC_PREC_MIXED), where the FP64
                                    outer residual on the stored faces fixes the solution: results
                                    agree with the other smoothers to the solve tolerance, not bit
                                    for bit. An FP64 solve uses MLMC_SMOOTH_TWO_PASS. */
#define MLMC_SMOOTH_SPLIT 9      /* the hierarchy stored colour-split: per sample the red
                                    ((x+y+z) even) and the black nodes form two blocks of n x n
                                    rows of (n+1)/2 slots rounded up to a multiple of 4 (node x
                                    at slot x/2), so that a colour pass streams only the rows of
                                    the colour it updates and of the other colour it reads. In
                                    FP32 correction cycles (MLMC_PREC_MIXED) the sweep is
                                    MLMC_SMOOTH_NODAL's (bit for bit the same iterates; 2.5
                                    instead of 4 words per node at cache-line granularity); in
                                    FP64 stationary and FMG cycles (MLMC_ACCEL_NONE, _FMG; finite
                                    volumes or P1 elements) it is the stored-face sweep of
                                    MLMC_SMOOTH_TWO_PASS (bit for bit the same iterates, cycles
                                    and residuals; 5 instead of ~7 words per node and pass).
                                    n <= 1025 only. Chosen for the
                                    finest grid, it applies to every grid of the hierarchy; on a
                                    coarser grid alone, or where it does not apply, it means
                                    MLMC_SMOOTH_NODAL (FP32) or MLMC_SMOOTH_TWO_PASS (FP64). */

/* Outer iteration around the V-cycle. */
#define MLMC_ACCEL_NONE 0 /* stationary: repeat V-cycles (FP64), or FP32 V-cycles as corrections of
                             FP64 residuals (iterative refinement, MLMC_PREC_MIXED) */
#define MLMC_ACCEL_CG 1   /* flexible preconditioned conjugate gradients, FP64 recurrences, one
                             V-cycle (FP64 or FP32) as the preconditioner per iteration */
#define MLMC_ACCEL_FMG 2  /* one full-multigrid cycle (the paper's FMG-2V(4,4), Sec. 7, with
                             nu1 = nu2 = 4 and max_cycles = 2): the exact solve on the coarsest
                             grid, then on each finer grid the interpolated coarser solution and
                             max_cycles V(nu1, nu2) cycles. Fixed work: rtol is not used (the
                             statistics report the final relative residual). FP64 and f = 1. */

/* Discretisation of -div(k grad u) = f. */
#define MLMC_DISC_FV 0 /* vertex-centred finite volumes, harmonic-mean faces; full weighting
                          and trilinear interpolation between grids */
#define MLMC_DISC_FE 1 /* P1 finite elements (Sec. 3.1) on the mesh that cuts every grid cube
                          into the six tetrahedra {O, O+e_a, O+e_a+e_b, O+(1,1,1)}, stiffness
                          with the four-vertex quadrature of k; on this mesh the operator is
                          the seven-point stencil with face K_a(P) = (k_P + k_{P+a})/4 +
                          (k_{P+a+b} + k_{P+a+c} + k_{P+a+b+c} + k_{P-b} + k_{P-c} +
                          k_{P-b-c})/12 ({a,b,c} = {x,y,z}); P1 interpolation between grids and
                          its transpose. FP64, stored-face smoothers. */

/* Execution engine of a solve (no counterpart in the paper; same results bit for bit).
 * MLMC_ENGINE_BATCHED: every phase of the cycle is a kernel over the whole batch, one
 * convergence test per cycle on the host. MLMC_ENGINE_CTA (finite volumes, stationary
 * cycles, refinement or CG, grids up to 33^3; otherwise the batched engine runs): one
 * persistent launch for the whole solve, each CTA taking the next sample from a device
 * counter and running all of its cycles, the convergence tests and the CG recurrences
 * with block barriers; the sums follow the batched kernels' partitions and trees, so
 * iterates, cycle counts and residuals are identical. MLMC_ENGINE_AUTO: the CTA engine
 * for grids up to 17^3 (where the batched engine waits on launches and host round trips)
 * and for 33^3 grids in batches of at least 1024 samples, the batched engine otherwise;
 * the environment variable MLMC_ENGINE=1 or 2 overrides the automatic choice. */
#define MLMC_ENGINE_AUTO 0
#define MLMC_ENGINE_BATCHED 1
#define MLMC_ENGINE_CTA 2

/* Multigrid parameters. */
typedef struct {
  int nu1;        /* pre-smoothing red-black sweeps, 0..8 (nu1 = nu2 = 0: the tuned count, else 2) */
  int nu2;        /* post-smoothing red-black sweeps, 0..8 */
  double rtol;    /* stop when ||f - A u|| / ||f|| <= rtol; rtol <= 0 runs exactly max_cycles */
  int max_cycles; /* 1..1000 */
  int precision;  /* MLMC_PREC_F64 or MLMC_PREC_MIXED */
  int smoother;   /* MLMC_SMOOTH_* */
  int accel;      /* MLMC_ACCEL_NONE, MLMC_ACCEL_CG or MLMC_ACCEL_FMG */
  int disc;       /* MLMC_DISC_FV (zero-initialised) or MLMC_DISC_FE */
  int engine;     /* MLMC_ENGINE_AUTO (zero-initialised), MLMC_ENGINE_BATCHED or MLMC_ENGINE_CTA */
} mg_cfg;

/* Per-sample solve statistics. */
typedef struct {
  int cycles;     /* V-cycles performed (mixed refinement and CG: outer steps, one V-cycle each) */
  double rel_res; /* final ||f - A u||_2 / ||f||_2 over interior nodes (FP64) */
} mg_stats;

/*
 * mlmc_field_eval -- the coefficient of the realisations `sample_ids_host[0..batch)`
 * (the coefficient of one realisation in Algorithm 1) at the n^3 nodes of
 * one grid. Writes k = exp(log k) into k_out (device, batch * n^3 elements of type
 * `dtype`: MLMC_F64, or MLMC_F32 = the FP64 value rounded to FP32). The phase is
 * always evaluated in FP64; the sum over the M features runs as exact products of bf16
 * slices of the phasors on the tensor cores (tcgen05 from n = 65, the warp-level MMA
 * below; grids with n - 1 a multiple of 16, others in double-float), within ~1e-13 of the
 * FP64 sum relative in k. sample_ids_host is host memory, read before return.
 * Errors: MLMC_ERR_INVALID for n not 2^p+1 (5 <= n <= 4097), batch < 1, M < 1,
 * ell <= 0, sigma2 < 0, unknown cov or dtype, or NULL pointers; MLMC_ERR_OOM / _CUDA;
 * MLMC_ERR_TIMEOUT if a bounded wait of the tensor-core kernel ran out (its nodes hold NaN;
 * see mlmc_set_wait_budget). Returns after the stream has drained.
 */
int mlmc_field_eval(const mlmc_field_cfg* cfg, const uint64_t* sample_ids_host, int batch, int n, int dtype,
                    void* k_out, void* stream);

/*
 * mlmc_field_eval_pair -- as mlmc_field_eval, for grid n as one grid of the level pair
 * whose fine grid is n_fine (n_fine = n: the fine grid itself; n_fine = 2n - 1: the
 * coarse grid of the pair, solved on the same realisation in Algorithm 1). Fourier-
 * feature fields are functions of x, so the result does not depend on n_fine; the SPDE
 * field of the coarse grid solves the coarse discretisation with the fine grid's white
 * noise. Errors: as mlmc_field_eval, and MLMC_ERR_INVALID for another n_fine;
 * MLMC_ERR_NOT_CONVERGED if an SPDE solve misses its tolerance in 60 cycles.
 */
int mlmc_field_eval_pair(const mlmc_field_cfg* cfg, const uint64_t* sample_ids_host, int batch, int n, int n_fine,
                         int dtype, void* k_out, void* stream);

/*
 * mg_solve_batch -- solve A u = f for `batch` independent samples on one grid size n
 * (the deterministic solves inside every sample of Algorithm 1) by V(nu1,nu2) cycles.
 *   k  device, FP64, batch * n^3: nodal coefficient (all nodes used, k > 0);
 *   f  device, FP64, batch * n^3: right-hand side at interior nodes, or NULL for f = 1;
 *   u  device, FP64, batch * n^3: initial guess in, solution out (boundary set to 0);
 *   stats_host  host array of `batch` entries, or NULL.
 * Each sample stops independently when its relative residual reaches cfg->rtol, so a
 * sample's result does not depend on the other samples of the batch.
 * On a created stream (not the legacy default stream) with nu1 + nu2 even, the first
 * V-cycle of the call is captured as a CUDA graph and the others replay it (same
 * kernels, same results); per-launch event timing (mlmc_profile_enable) or the
 * environment variable MLMC_NO_GRAPHS=1 keeps every launch direct.
 * Blocking: synchronises `stream`. Returns MLMC_ERR_NOT_CONVERGED if any sample
 * reached max_cycles without meeting rtol (u is still written); MLMC_ERR_INVALID for
 * bad sizes / parameters / NULL k or u; MLMC_ERR_OOM; MLMC_ERR_CUDA.
 */
int mg_solve_batch(const mg_cfg* cfg, int batch, int n, const double* k, const double* f, double* u,
                   mg_stats* stats_host, void* stream);

/*
 * mg_solve_batch_noalloc -- mg_solve_batch for callers that cannot allocate device
 * memory: code running inside another framework whose memory pool or allocator hooks
 * own every device allocation, or an embedded runtime with a fixed device-memory budget
 * set at start-up. The paper has no counterpart; this is an interface variant only, with
 * the same arguments,
 * numerics and results as mg_solve_batch, except that the FMG cycle (MLMC_ACCEL_FMG) is
 * not offered here (MLMC_ERR_INVALID).
 * The workspace is a fixed 32 MiB array in the library's device image (every GPU that
 * loads the library keeps it until the process exits); the call makes no cudaMalloc,
 * cudaMallocAsync or cudaFree and no torch allocation. Sizes whose workspace exceeds
 * 32 MiB (about 50 samples at 17^3, 8 at 33^3, 1 at 65^3 in FP64) return
 * MLMC_ERR_INVALID with the required size in mlmc_last_error_string().
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * once for that device and keeps it for the life of the process (not refreshed after
 * cudaDeviceReset); make that first call before any stream capture.
 * Every call reuses the same array, which keeps the previous call's contents; the
 * solver initialises every part it reads. Blocking: the call synchronises `stream`
 * (also when it fails), and it reads convergence data back to the host once per cycle.
 * Calls in one process are serialised by a lock; calls whose GPU work overlapped would
 * race on the shared array.
 */
int mg_solve_batch_noalloc(const mg_cfg* cfg, int batch, int n, const double* k, const double* f, double* u,
                           mg_stats* stats_host, void* stream);

/* Configuration of an MLMC level computation. */
/* Quantity of interest of a solve. */
#define MLMC_QOI_MEAN 0  /* mean of u over [1/4, 3/4]^3, tensor trapezoid rule */
#define MLMC_QOI_POINT 1 /* u(1/4, 1/4, 1/4) (Sec. 7; a grid node) */
#define MLMC_QOI_FLUX 2  /* flux of k du/dx_2 across the plane x_2 = 1/4 (Sec. 7): the mean of
                            k du/dx_2 over the layer of tetrahedra (the P1 mesh above) between
                            x_2 = 1/4 - h and 1/4, k the vertex mean per element */

typedef struct {
  mlmc_field_cfg field;
  mg_cfg mg;
  int n0;        /* nodes per axis of MLMC level 0 (17 gives 17, 33, 65, ... for levels 0, 1, 2, ...) */
  int max_batch; /* samples per device batch, 0 = choose from free HBM */
  void* stream;  /* cudaStream_t, NULL = default */
  int qoi;       /* MLMC_QOI_MEAN (zero-initialised), MLMC_QOI_POINT or MLMC_QOI_FLUX */
} mlmc_cfg;

/* Statistics of one MLMC level (Sec. 2.3: Y-hat_l, s_l^2, C_l). */
typedef struct {
  int64_t N;               /* samples */
  double mean;             /* Y-hat_l = (1/N) sum Y */
  double var_biased;       /* s_l^2 with 1/N (Sec. 2.3) */
  double var_unbiased;     /* with 1/(N-1) (0 for N < 2) */
  double sum;              /* Kahan-compensated sum of Y */
  double sum_comp;         /* its compensation term */
  double M2;               /* sum (Y - mean)^2 (Welford / Chan) */
  double mean_cycles_fine; /* mean V-cycles of the fine solve */
  double mean_cycles_coarse;
  int max_cycles_seen;
  double seconds;          /* wall time of the call */
  double cost_per_sample;  /* seconds / N, the C_l estimate of Eq. 15 */
} mlmc_level_stats;

/*
 * mlmc_level_estimate -- N samples of Y_level with realisation ids first_id ..
 * first_id + N - 1 (Algorithm 1 for one level: the samples, and their mean and
 * variance in `out`).
 * For level 0, Y = Q_0 on grid n0; for level l >= 1 the fine grid has
 * n_l = (n0 - 1) 2^l + 1 nodes and the coarse grid n_{l-1}, both solved on the field
 * of the same id; the coarse solve runs first and the trilinear interpolation of its
 * solution is the initial guess of the fine solve (nested iteration, the first step of
 * the full multigrid of Sec. 7.1), which saves about two fine cycles and changes Q_l only
 * within the solve tolerance. Y_host, Qf_host, Qc_host: host arrays of N doubles or NULL
 * (Qc = 0 for level 0). Blocking. Errors as mg_solve_batch; MLMC_ERR_NOT_CONVERGED
 * if any solve missed rtol (the outputs are still written).
 */
int mlmc_level_estimate(const mlmc_cfg* cfg, int level, uint64_t first_id, int N, double* Y_host, double* Qf_host,
                        double* Qc_host, mlmc_level_stats* out);

/*
 * mlmc_level_run -- the device-resident form of mlmc_level_estimate: the N realisation
 * ids are read from DEVICE memory (ids_dev) and the per-sample results are written to
 * DEVICE arrays of N doubles (Y_dev, Qf_dev, Qc_dev; each may be NULL). `out` (host,
 * may be NULL) receives the level statistics; they are accumulated on the device in
 * id order, so they are identical to mlmc_level_estimate's for the same ids. Blocking
 * (the cycle loop synchronises cfg->stream once per V-cycle to test convergence).
 * Errors as mlmc_level_estimate; MLMC_ERR_INVALID for ids_dev == NULL.
 */
int mlmc_level_run(const mlmc_cfg* cfg, int level, const uint64_t* ids_dev, int N, double* Y_dev, double* Qf_dev,
                   double* Qc_dev, mlmc_level_stats* out);

/*
 * Adaptive MLMC (Algorithm 2 of Sec. 2.4) on levels 0..L, with optional level growth.
 *
 * Each round (mlmc_adaptive_step) computes the missing samples of every level -- sample i
 * of level l is the realisation id (l << 48) | i, in order, through the level pipeline of
 * mlmc_level_estimate with cfg.level (or through a caller's sampler, below) -- folds them
 * into the level's running record (Chan's merge of (N, mean, M2): Y-hat_l and s_l^2 of
 * Sec. 2.3, s_l^2 with 1/(N-1)), takes C_l (measured wall seconds per sample, or the node
 * count n_l^3 + n_{l-1}^3), and sets N_l = ceil(eps_s^-2 (sum_k sqrt(s_k^2 C_k))
 * sqrt(s_l^2 / C_l)), at least 2 (Eqs. 11 / 15; eps_s^2 = theta eps^2, eps_b^2 = (1 - theta)
 * eps^2, Eq. 6). Samples already computed are kept (N_l never decreases). With
 * max_level > L0 the bias estimate |Y-hat_L| / (8^alpha - 1) of Eq. 14 is compared with
 * eps_b after each round; while it is larger and L < max_level, level L + 1 joins with its
 * pilot count. A round that changes neither N_l nor L ends the run (*finished = 1).
 * alpha: cfg.alpha if > 0, else minus the least-squares slope of log_8 |Y-hat_l| over the
 * levels l >= 1 with samples (M_l ~ 8^l), alpha0 while fewer than two such levels exist,
 * never below alpha_floor; beta and gamma (Eq. 12) are fitted the same way from s_l^2 and
 * C_l and only reported (NAN where no fit exists).
 * With lanes > 1 the levels of a round run concurrently, one host thread and one stream
 * per lane (lane_streams[k]; lane 0 uses cfg.level.stream when lane_streams[0] is NULL),
 * levels placed longest first (count x node cost) onto the least-loaded lane; the records
 * do not depend on the lanes. Blocking calls; one handle must not be stepped from two
 * threads at once.
 */
#define MLMC_MAX_LEVELS 9
#define MLMC_COST_MEASURED 0 /* C_l = wall seconds per sample of the level's calls */
#define MLMC_COST_NODES 1    /* C_l = n_l^3 + n_{l-1}^3 (deterministic decisions) */

typedef struct {
  mlmc_cfg level;                   /* field, solver, n0, max_batch, stream and QoI of the level calls */
  int L0;                           /* levels 0..L0 at the start, 0 <= L0 <= 8 */
  int max_level;                    /* L0 <= max_level <= 8; > L0 enables level growth (then L0 >= 1) */
  int64_t N_init[MLMC_MAX_LEVELS];  /* pilot count per level (>= 1 for 0..L0; a grown level without
                                       an entry (0) takes the previous level's) */
  double eps;                       /* RMS tolerance, > 0 */
  double theta;                     /* 0 < theta < 1 (Eq. 6) */
  int cost_model;                   /* MLMC_COST_MEASURED or MLMC_COST_NODES */
  double alpha;                     /* > 0: fixed; <= 0: fitted online */
  double alpha0;                    /* alpha before two levels l >= 1 have samples (fitted mode), > 0 */
  double alpha_floor;               /* lower bound of the fitted alpha, >= 0 */
  int lanes;                        /* 0 or 1: levels in sequence; up to 8 concurrent lanes */
  void* lane_streams[8];            /* cudaStream_t per lane (lanes 1.. must be created streams) */
} mlmc_adaptive_cfg;

/* One round of the run (what the round saw and decided). */
typedef struct {
  int round, L, grow;
  int64_t have[MLMC_MAX_LEVELS];   /* samples per level after the round's computation */
  int64_t N_next[MLMC_MAX_LEVELS]; /* Eq. 15 counts from the round's statistics */
  double alpha, bias;              /* alpha used by the bias test, the Eq. 14 estimate */
} mlmc_adaptive_round;

/* Result of the run so far. */
typedef struct {
  int L, rounds, bias_ok;          /* bias_ok: the Eq. 14 estimate <= eps_b */
  double Q_hat;                    /* sum of the level means (Eq. 8), compensated sum */
  double sampling_var;             /* sum_l s_l^2 / N_l (Eq. 10) */
  double eps_s2;                   /* theta eps^2 */
  double alpha, beta, gamma, bias;
  int64_t N[MLMC_MAX_LEVELS];
  double mean[MLMC_MAX_LEVELS], var[MLMC_MAX_LEVELS], M2[MLMC_MAX_LEVELS];
  double cost[MLMC_MAX_LEVELS], seconds[MLMC_MAX_LEVELS];
} mlmc_adaptive_summary;

/* Resumable state (plain data: the caller may store it anywhere). The round log is not
 * part of it. */
typedef struct {
  uint32_t magic, version;
  int L, rounds;
  int64_t have[MLMC_MAX_LEVELS], target[MLMC_MAX_LEVELS];
  double N[MLMC_MAX_LEVELS], mean[MLMC_MAX_LEVELS], M2[MLMC_MAX_LEVELS], seconds[MLMC_MAX_LEVELS];
} mlmc_adaptive_state;

/* A caller's sampler of level l, used instead of the library's level pipeline: the
 * record (N = count, mean, M2 = sum of squared deviations) of samples first_index ..
 * first_index + count - 1 of level l. Returns MLMC_OK or a negative status (the step
 * then fails with it). */
typedef int (*mlmc_level_sampler)(void* user, int level, uint64_t first_index, int64_t count, double* N,
                                  double* mean, double* M2);

typedef struct mlmc_adaptive mlmc_adaptive;

/* Eq. 11 / Eq. 15 on their own: N_out[l] = ceil(eps_s^-2 (sum_k sqrt(var_k cost_k))
 * sqrt(var_l / cost_l)), at least 2, eps_s = sqrt(theta) eps (Eq. 6), for `levels` levels
 * (1..64) with positive variances and costs. Host-only. */
int mlmc_sample_sizes(const double* var, const double* cost, int levels, double eps, double theta, int64_t* N_out);
/* Chan et al.'s pairwise merge, in the given order, of `count` records (N, mean, M2) of
 * disjoint sample sets (records: count x 3 doubles) into out[3] = (N, mean, M2): how the
 * level records of replicas, lanes or chunks are combined. Host-only. */
int mlmc_merge_records(const double* records, int count, double* out);

/* NULL on an invalid cfg (mlmc_last_error_string says why). Host-only. */
mlmc_adaptive* mlmc_adaptive_create(const mlmc_adaptive_cfg* cfg);
void mlmc_adaptive_destroy(mlmc_adaptive* est);
/* fn = NULL restores the library's level pipeline. */
int mlmc_adaptive_set_sampler(mlmc_adaptive* est, mlmc_level_sampler fn, void* user);
/* One round; *finished = 1 when it changed neither N_l nor L. Errors of the level calls
 * (MLMC_ERR_NOT_CONVERGED, _OOM, _CUDA, ...) or of the sampler are returned. */
int mlmc_adaptive_step(mlmc_adaptive* est, int* finished);
/* Rounds until finished or max_rounds (>= 1); *finished may be NULL. */
int mlmc_adaptive_run(mlmc_adaptive* est, int max_rounds, int* finished);
int mlmc_adaptive_result(const mlmc_adaptive* est, mlmc_adaptive_summary* out);
int mlmc_adaptive_log_count(const mlmc_adaptive* est);
int mlmc_adaptive_log_get(const mlmc_adaptive* est, int index, mlmc_adaptive_round* out);
/* Checkpoint / resume: a state taken after any round, set into a handle created with the
 * same cfg, continues exactly as the uninterrupted run (same ids, same records).
 * MLMC_ERR_INVALID for a state that does not fit the handle's cfg. */
int mlmc_adaptive_get_state(const mlmc_adaptive* est, mlmc_adaptive_state* out);
int mlmc_adaptive_set_state(mlmc_adaptive* est, const mlmc_adaptive_state* state);

/*
 * Launch accounting (no counterpart in the paper; measurement support). The library
 * counts every kernel launch per kernel class with the algorithmic bytes and flops of
 * that launch. After mlmc_profile_enable(1) it also records a CUDA event pair around
 * each launch on the launching stream. mlmc_profile_get(i, ...) synchronises on the
 * recorded events and returns class i's name, launches, launches with timing, total
 * device milliseconds, algorithmic bytes and flops. mlmc_profile_reset() clears all
 * classes. mlmc_profile_total_launches() counts launches since the last reset.
 */
int mlmc_profile_enable(int on);
int mlmc_profile_reset(void);
int mlmc_profile_count(void);
int64_t mlmc_profile_total_launches(void);
int mlmc_profile_get(int index, char* name, int name_len, int64_t* launches, int64_t* timed_launches, double* ms,
                     double* bytes, double* flops);
/* Measured FMA throughput of the current device: *tflops = 2 x FMAs per second / 1e12 of
 * a probe kernel with 8 independent FMA chains per thread on 8 CTAs of 256 threads per SM,
 * best of four timed launches (CUDA events on the legacy default stream). precision:
 * MLMC_PREC_F64 (FP64 FMA) or MLMC_PREC_MIXED (FP32 FMA). Blocking. */
int mlmc_profile_fma_peak(int precision, double* tflops);

/*
 * Solve service with continuous batching (the single-GPU counterpart of the paper's
 * schedulers, Secs. 4-5, whose dynamic variants hand the next sample to whichever
 * process group is free). Requests (level, realisation id) are queued per level;
 * `workers` host threads, each with its own CUDA stream, repeatedly take the level
 * whose oldest request has waited longest, batch up to max_batch requests of it (fewer
 * once the oldest has waited batch_wait_ms), admit the batch only while the device
 * bytes of all running batches stay within hbm_budget_bytes, and run the level pipeline
 * for it. A request's result does not depend on its batch. All requests share the
 * service's field and solver configuration.
 */
typedef struct {
  mlmc_field_cfg field;
  mg_cfg mg;
  int n0;                  /* nodes per axis of level 0 */
  int max_level;           /* levels 0..max_level accepted (fine grid <= 1025) */
  int max_batch;           /* samples per batch, 1..65535 */
  int workers;             /* concurrent batches (streams), 1..16 */
  int queue_capacity;      /* pending requests before mlmc_submit returns MLMC_ERR_BUSY */
  size_t hbm_budget_bytes; /* device bytes the running batches may hold together */
  double batch_wait_ms;    /* longest wait for batch-mates before a partial batch runs */
} mlmc_service_cfg;

typedef struct {
  int level;
  uint64_t sample_id;
} mlmc_request;

typedef struct {
  int status;          /* MLMC_PENDING, MLMC_OK, or an MLMC_ERR_* of the batch */
  int level;
  uint64_t sample_id;
  double Y, Qf, Qc;    /* Y = Qf - Qc; Qc = 0 on level 0 */
  int cycles_fine, cycles_coarse;
  double t_submit, t_start, t_done; /* host steady-clock seconds */
} mlmc_result;

typedef struct {
  int64_t submitted, completed, rejected, pending;
  int64_t cancelled;         /* requests withdrawn by mlmc_cancel before they ran */
  int inflight_batches;
  size_t bytes_in_use;
  double samples_per_s;      /* completed / (last completion - first submission) */
  int64_t count[9];          /* completed requests per level */
  double p50_ms[9], p99_ms[9]; /* latency (done - submit) per level */
} mlmc_service_report;

typedef struct mlmc_service mlmc_service;

/* Starts the worker threads on the current device; NULL on invalid cfg (see
 * mlmc_last_error_string). */
mlmc_service* mlmc_service_create(const mlmc_service_cfg* cfg);
/* Stops after the running batches finish; queued requests are dropped. */
void mlmc_service_destroy(mlmc_service* svc);
/* Non-blocking. MLMC_ERR_BUSY when queue_capacity requests are pending (backpressure);
 * MLMC_ERR_INVALID for a level outside 0..max_level. */
int mlmc_submit(mlmc_service* svc, const mlmc_request* req, uint64_t* ticket);
/* MLMC_PENDING while queued or running; MLMC_OK once (the result is then released);
 * MLMC_ERR_NOT_FOUND for an unknown or already delivered ticket. */
int mlmc_poll(mlmc_service* svc, uint64_t ticket, mlmc_result* res);
/* Blocks up to timeout_ms; MLMC_ERR_TIMEOUT if still pending. */
int mlmc_wait(mlmc_service* svc, uint64_t ticket, double timeout_ms, mlmc_result* res);
/* Withdraws a request that is still queued: it will not run, and mlmc_poll / mlmc_wait
 * then deliver it once with status MLMC_ERR_CANCELLED (so no waiter is left blocked).
 * Returns MLMC_OK if it was withdrawn; MLMC_ERR_BUSY if its batch is already running or
 * finished (its result is delivered as usual); MLMC_ERR_NOT_FOUND for an unknown or
 * already delivered ticket. Non-blocking; no counterpart in the paper. */
int mlmc_cancel(mlmc_service* svc, uint64_t ticket);
int mlmc_service_stats(mlmc_service* svc, mlmc_service_report* out);

/* One measurement of mlmc_autotune. */
typedef struct {
  int smoother;              /* MLMC_SMOOTH_* */
  int nu;                    /* sweeps per side, V(nu, nu) */
  double seconds_per_sample; /* wall time of the level pipeline per sample */
  double mean_cycles;        /* fine-grid cycles per sample */
} mlmc_tune_entry;

/*
 * mlmc_autotune -- picks the smoother implementation (two-pass on stored faces, two-pass
 * on the nodal coefficient in the plain or the colour-split storage, or fused with 32x8,
 * 32x16 or 64x8 tiles staged by cp.async or by TMA bulk copies: 9 candidates for FP32
 * correction cycles on finite volumes; 8 for FP64 stationary or FMG cycles (the
 * colour-split stored-face sweep, no nodal-coefficient sweep); 7 for FP64 CG) and the sweep count
 * nu in {1,2,3,4} of V(nu, nu) for MLMC level
 * `level` under cfg (no counterpart in the paper; the paper fixes its cycle, Sec. 7.1).
 * Each candidate runs the whole level pipeline on the batched engine
 * (MLMC_ENGINE_BATCHED) once untimed and once timed on `samples` realisations
 * first_id .. first_id + samples - 1; the fastest by wall time
 * per sample is stored in a process-wide table for the level's fine grid size and
 * precision, where MLMC_SMOOTH_AUTO and nu1 = nu2 = 0 find it. With nu1 = nu2 > 0 in
 * cfg->mg only the smoother is tuned, at that nu. Every candidate solves
 * to the same rtol, so the choice changes speed, not results beyond rtol.
 * table: host array of table_len entries (may be NULL) for the measurements; *n_entries,
 * *best_smoother, *best_nu (each may be NULL) receive the count and the choice.
 * Blocking. Errors as mlmc_level_estimate.
 */
int mlmc_autotune(const mlmc_cfg* cfg, int level, uint64_t first_id, int samples, mlmc_tune_entry* table,
                  int table_len, int* n_entries, int* best_smoother, int* best_nu);

/*
 * mlmc_tune_set -- stores a tuning choice in the process-wide table that mlmc_autotune
 * fills: grids of n^3 nodes solved at `precision` with MLMC_SMOOTH_AUTO use `smoother`,
 * and with nu1 = nu2 = 0 the cycle V(nu, nu). For restoring a table measured earlier
 * (for example in a run without a profiler attached) without measuring again. No
 * counterpart in the paper. Host-only, thread-safe, no device work. Errors:
 * MLMC_ERR_INVALID for n not 2^p+1 (5 <= n <= 4097), an unknown precision, smoother
 * outside MLMC_SMOOTH_TWO_PASS .. MLMC_SMOOTH_SPLIT, or nu outside 1..8.
 */
int mlmc_tune_set(int n, int precision, int smoother, int nu);

/*
 * Failure-path controls (no counterpart in the paper; for tests of the error paths, and
 * process-wide).
 *
 * mlmc_set_wait_budget -- every bounded wait inside a kernel (the mbarrier waits of the
 * TMA bulk-copy smoothers and of the tcgen05 field kernel) gives up after `clocks` SM clocks: the kernel then records an
 * error word, waits (bounded by about one second, whatever `clocks` is) for the copies it
 * still has in flight, and returns; the solve reports MLMC_ERR_TIMEOUT and the context
 * stays usable. Default 2e9 clocks (about one second). clocks = 0 gives up at the first
 * wait that finds its data not yet arrived. Read at each launch (a V-cycle captured as a
 * CUDA graph keeps the budget of its capture). *previous (may be NULL) receives the old
 * value. MLMC_ERR_INVALID for clocks < 0. Host-only.
 *
 * mlmc_inject_alloc_failure -- host-side fault injection: after `after` more successful
 * device allocations of the library, every later one fails with MLMC_ERR_OOM without
 * calling the CUDA allocator, until the next call; after = -1 turns it off (the
 * default). MLMC_ERR_INVALID for after < -1. Host-only.
 *
 * mlmc_inject_wait_failure -- host-side fault injection for the tensor-core field (the
 * tcgen05 volume kernel, grids from 65^3): each of the next `launches` launches of that
 * kernel also waits, in its issuing thread, on an mbarrier that nothing arrives on, so the
 * wait runs out after the wait budget (mlmc_set_wait_budget); the blocks then drain their
 * copies and products, write NaN to their nodes, free their tensor memory and return, and
 * mlmc_field_eval (or the level call) reports MLMC_ERR_TIMEOUT. launches = 0 turns it off
 * (the default). MLMC_ERR_INVALID for launches < 0. Host-only.
 */
int mlmc_set_wait_budget(int64_t clocks, int64_t* previous);
int mlmc_inject_alloc_failure(int64_t after);
int mlmc_inject_wait_failure(int launches);

/* Text of the last error on the calling thread ("" if none). Never NULL. */
const char* mlmc_last_error_string(void);

/* Library version string. */
const char* mlmc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MLMC_GB300_H */
