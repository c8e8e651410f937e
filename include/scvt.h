/*
 * scvt.h -- C ABI of the GB300 spherical centroidal Voronoi tessellation
 * (SCVT) engine: Lloyd-preconditioned LBFGS (Yang, Gunzburger and Ju,
 * "Fast spherical centroidal Voronoi mesh generation: a Lloyd-preconditioned
 * LBFGS method in parallel").
 *
 * Problem (Sec. 2.1): for generators z_1..z_N on the unit sphere S^2 and a
 * point density rho > 0, the spherical Voronoi region of z_i is
 *     V_i = { x in S^2 : |x - z_i| < |x - z_j| for all j != i }
 * (Euclidean distance restricted to the sphere) and the energy is
 *     F(Z) = sum_i int_{V_i} |y - z_i|^2 rho(y) dsigma(y).
 * With m_i = int_{V_i} rho and c_i = int_{V_i} y rho, the tangential gradient
 * is g_i = 2 (c_i . z_i) z_i - 2 c_i and the Lloyd preconditioner is
 * h_i = 1 / (2 c_i . z_i) (Sec. 3.1, spherical form).
 *
 * Conventions for every entry point below:
 *   - Arrays of points or vectors are contiguous row-major N x 3 doubles
 *     (x, y, z of point 0, then point 1, ...); per-point scalars are N doubles.
 *   - The caller owns every array.  A pointer may be device memory or host
 *     memory (pageable or pinned); host pointers are staged through the
 *     handle's device buffers inside the call.
 *   - All device work is ordered on the CUDA stream given to scvt_create.
 *     Calls that return host scalars synchronise that stream.
 *   - Errors are returned as scvt_status, never thrown or aborted; after an
 *     error the outputs are unspecified and the handle remains usable.
 *     scvt_last_error() then gives a one-line description.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef SCVT_H
#define SCVT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SCVT_OK = 0,
    SCVT_ERR_INVALID = 1,       /* bad argument: N < 4, non-finite or non-unit point (| |z|-1 | > 1e-12),
                                   duplicate points, null pointer, unsupported option */
    SCVT_ERR_DEGENERATE = 2,    /* origin not strictly inside the hull of Z (some cell leaves its
                                   hemisphere), c_i . z_i <= 0, or neighbouring cells that disagree
                                   on a Voronoi vertex (four or more cocircular generators) */
    SCVT_ERR_OOM = 3,           /* device allocation failed */
    SCVT_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    SCVT_ERR_KNN_EXHAUSTED = 5, /* a cell could not be certified (security radius) with any neighbour count */
    SCVT_ERR_LINESEARCH = 6,    /* the line search found no decrease from a Lloyd direction (rounding floor) */
    SCVT_ERR_TIMEOUT = 7,       /* a bounded device wait ran out */
    SCVT_ERR_UNIMPLEMENTED = 8  /* option not available in this build */
} scvt_status;

/* Point densities of Sec. 4.  TANH_CAP: rho = (1-gamma)/2 (tanh((beta - d)/alpha) + 1) + gamma with
 * d the geodesic distance to xc (radians), evaluated as (1-gamma)/(1 + exp(-2(beta - d)/alpha))
 * + gamma (equal; no cancellation far from the cap); POLAR_X3: rho = (1-gamma) z^4 + gamma;
 * TANH_CAP_POW4: the TANH_CAP value raised to the 4th power. */
typedef enum {
    SCVT_RHO_UNIFORM = 0,
    SCVT_RHO_POLAR_X3 = 1,
    SCVT_RHO_TANH_CAP = 2,
    SCVT_RHO_TANH_CAP_POW4 = 3
} scvt_rho_kind;

typedef struct {
    int kind;           /* scvt_rho_kind */
    double gamma;       /* minimum density (rho >= gamma > 0) */
    double alpha;       /* transition width (radians), TANH kinds */
    double beta;        /* cap radius (radians), TANH kinds */
    double xc[3];       /* cap centre (unit vector), TANH kinds */
} scvt_density;

typedef struct {
    int64_t n;          /* number of generators, >= 4 */
    scvt_density rho;
    int quad_points;    /* points per sub-triangle; 7 (Radon degree-5 rule) is the only value */
    int precision;      /* Arithmetic of the geometry.  The topology (neighbour sets) is the same
                           in every form: clipping decisions are filtered in FP32 and taken in
                           FP64 where the filter cannot decide.  Sums over edges and cells and all
                           LBFGS vectors are FP64 in every form.
                           0 = FP64 form (parity mode): Voronoi corners and the rule points in
                             double-float arithmetic (pairs of FP32 values, about 48 bits)
                             relative to z_i, from FP64 offsets; corners that are poorly
                             conditioned or far from z_i, and edges reaching beyond chord 0.03
                             of z_i, in FP64; the tanh-cap density from a table of FP64 Taylor
                             series in x_c.p built once per handle (direct formula where no
                             series is validated over the edge's range).
                             Results within 1e-12 (relative) of an FP64 evaluation.
                           1 = mixed: corners and quadrature in FP32 local coordinates (offsets
                             from z_i), density in FP32; error stated per quantity (about 1e-5
                             relative for m_i, c_i and F_i).
                           2 = plain FP64: corners, rule points and density in FP64 arithmetic
                             (the density from the same FP64 series table / direct formula). */
    int lbfgs_m;        /* number of (s, y) pairs kept, 0..32 (the paper uses 7) */
    int knn_k0;         /* first-pass neighbour count, 0 = default (32); 8..32 */
    int knn_kmax;       /* largest neighbour count of the retry passes, 0 = default (128) */
    int decomposition;  /* 0: per Voronoi edge the two signed sub-triangles (z_i, v_a, mu), (z_i, mu, v_b)
                           through the Delaunay-edge midpoint mu (Sec. 3.2.2, the paper's six
                           sub-triangles per Delaunay triangle).  1: the fan, one triangle
                           (z_i, v_a, v_b) per Voronoi edge. */
} scvt_config;

typedef struct {
    int max_iter;         /* LBFGS iterations (accepted steps) at most */
    double grad_tol;      /* stop when ||g||_2 <= grad_tol (2-norm over all 3N components) */
    double rel_grad_tol;  /* stop when ||g||/F <= rel_grad_tol (0 = off; the paper uses 5e-4) */
    double rel_df_tol;    /* stop when |F_k - F_{k-1}|/F_{k-1} < rel_df_tol (0 = off; paper 1e-7) */
    double step_tol;      /* stop when max_i |z_i^{k+1} - z_i^k| <= step_tol (0 = off; paper 5e-4) */
    int ls_max_evals;     /* function evaluations per line search, 0 = default (10, Sec. 4) */
    double c1, c2;        /* strong Wolfe constants, 0 = defaults (1e-4, 0.9) */
    int warm_start;       /* 0: start at z with an empty history.
                             1: continue from the handle's state left by the previous
                                scvt_lbfgs_solve (iterate, gradient and history); z's input
                                value is ignored and z receives the result.
                             2: as 1 if z holds exactly the iterate the previous solve
                                returned (checked on the device), else as 0. */
    int method;           /* 0: Lloyd-preconditioned LBFGS (Sec. 3.1).  1: plain LBFGS, H0 = gamma_n I
                             with gamma_n = y.s / y.y of the newest stored pair, I with an empty
                             memory (Sec. 2.2.2).  2: Lloyd's iteration (Sec. 2.2.1), taken as the
                             unit step along q = -h g, whose trial point normalize(z - h g) is
                             c / |c|, with no line search and no memory. */
} scvt_solve_opts;

typedef struct {
    int iters;          /* accepted LBFGS steps in this call */
    int fevals;         /* energy/gradient evaluations in this call */
    int resets;         /* history resets (no descent, line-search trouble) */
    int skipped;        /* pairs skipped by the curvature test */
    int knn_retries;    /* cells that needed a retry pass, summed over evaluations */
    double energy;      /* F at the returned iterate */
    double grad_norm;   /* ||g||_2 at the returned iterate */
    int converged;      /* 1 if a stopping tolerance was met */
    int status;         /* scvt_status of the call */
} scvt_solve_report;

typedef struct {
    int64_t evaluations;        /* energy/gradient evaluations since creation */
    int64_t cell_launches;      /* launches of the cell kernel (first pass + retries) */
    int64_t kernel_launches;    /* all kernel launches of this handle */
    int64_t knn_retries;        /* cells sent to a retry pass */
    int64_t ambiguous;          /* clip decisions within rounding of zero (0 on generic input) */
    double cell_kernel_ms;      /* device time of the first-pass cell kernel (profiling on) */
    double eval_ms;             /* device time of whole evaluations (profiling on) */
    double lbfgs_ms;            /* device time of the two-loop / update kernels (profiling on) */
    int64_t cell_kernel_timed;  /* first-pass launches included in cell_kernel_ms */
    int64_t bytes_device;       /* device memory held by the handle */
    int64_t series_edges;       /* FP64 forms: quadrature edges whose density came from the density
                                   table's Taylor series (the others evaluate it directly) */
    int64_t series_terms;       /* ... and the sum of those series' lengths */
    double topo_kernel_ms;      /* device time of the first topology pass (profiling on, one pipeline) */
    int64_t topo_kernel_timed;  /* first topology passes included in topo_kernel_ms */
} scvt_stats;

typedef struct scvt_handle scvt_handle;

/* Create an engine for N generators.  cuda_stream: a cudaStream_t (NULL = the
 * legacy default stream).  Allocates all device workspace for N, including
 * the LBFGS history (2 * lbfgs_m * N * 3 doubles).  *out is set on success.
 * Errors: INVALID (bad config), OOM, CUDA. */
scvt_status scvt_create(const scvt_config *cfg, void *cuda_stream, scvt_handle **out);

/* Destroy the engine and free its device memory.  NULL-safe. */
void scvt_destroy(scvt_handle *h);

/* Energy and gradient at z (Sec. 2.1 energy, Sec. 3.1 gradient).
 * z: N x 3.  energy: host double (required).  grad: N x 3 (nullable).
 * mass: N, m_i (nullable).  moment: N x 3, c_i (nullable).  Synchronises. */
scvt_status scvt_energy_grad(scvt_handle *h, const double *z, double *energy, double *grad,
                             double *mass, double *moment);

/* Everything one evaluation produces.  Any array pointer may be NULL. */
typedef struct {
    double *grad;        /* N x 3, g_i = 2 (c_i.z_i) z_i - 2 c_i */
    double *precond;     /* N, h_i = 1 / (2 c_i.z_i) */
    double *mass;        /* N, m_i */
    double *moment;      /* N x 3, c_i */
    double *cell_energy; /* N, F_i = int_{V_i} |y - z_i|^2 rho */
    double energy;       /* out: F = sum_i F_i */
    double grad_norm;    /* out: ||g||_2 */
} scvt_eval_out;

scvt_status scvt_evaluate(scvt_handle *h, const double *z, scvt_eval_out *out);

/* One Lloyd iteration (Sec. 2.2.1 on S^2): z_out_i = c_i / |c_i|.
 * z_out may alias z_in.  Synchronises. */
scvt_status scvt_lloyd_step(scvt_handle *h, const double *z_in, double *z_out);

/* Lloyd-preconditioned LBFGS (Sec. 3.1; serial core of the algorithm of
 * Sec. 3.3): two-loop recursion with diag(h) as initial inverse Hessian,
 * strong-Wolfe line search from step 1 on alpha -> F(normalize(Z + alpha q)),
 * re-projection onto S^2.  z: N x 3 in/out.  opts: NULL = defaults
 * (200 iterations, grad_tol 1e-8).  report: host (nullable).
 * Returns OK when a tolerance or max_iter ends the solve, LINESEARCH when no
 * decrease can be found from a Lloyd direction (z then holds the last
 * accepted iterate). */
scvt_status scvt_lbfgs_solve(scvt_handle *h, double *z, const scvt_solve_opts *opts,
                             scvt_solve_report *report);

/* Voronoi topology (Sec. 2.1): deg[i] and the neighbour ids of cell i in
 * counter-clockwise order seen from outside, nbr[i * max_deg + t],
 * t < deg[i].  deg: N ints, nbr: N * max_deg ints (device or host).
 * INVALID if a cell has more than max_deg neighbours.  Synchronises. */
scvt_status scvt_voronoi(scvt_handle *h, const double *z, int *deg, int *nbr, int max_deg);

/* LBFGS direction on caller-provided pairs (Sec. 2.2.2 two-loop with the
 * Sec. 3.1 preconditioner): q = -H g with H0 = diag(h) applied per generator.
 * S, Y: count x N x 3, oldest pair first; requires y_k . s_k > 0.
 * g, h, q: N x 3, N, N x 3.  count <= 64.  Synchronises. */
scvt_status scvt_lbfgs_direction(scvt_handle *h, const double *g, const double *hdiag, int count,
                                 const double *S, const double *Y, double *q);

/* Energy and gradient for callers that cannot allocate device memory (a
 * memory budget fixed up front, an allocator that must not be re-entered, a
 * host that forbids cudaMalloc after start-up).  The paper has no
 * counterpart: this is a deployment variant of scvt_energy_grad.
 * It needs no handle and allocates nothing: its scratch is one fixed array
 * in device memory (about 16.4 MB, held on every GPU that loads the library
 * until the process exits), sized for n <= SCVT_STATIC_MAX_N.
 * n: generators (4 <= n <= SCVT_STATIC_MAX_N, else SCVT_ERR_INVALID before
 * any device work).  rho: host.  z: N x 3 device.  cuda_stream: cudaStream_t
 * (NULL = legacy default stream).  energy: host double (required).  grad
 * (N x 3), mass (N), moment (N x 3): device, nullable.  Host pointers for
 * z/grad/mass/moment are rejected (SCVT_ERR_INVALID).  Synchronises the
 * stream.  The first call on a device looks up the array's device address
 * with that device current and keeps it until the process exits; make that
 * call before any stream capture, and do not call this entry point on a
 * device after cudaDeviceReset (the kept address is then stale).  All calls
 * share the one array and it keeps the previous call's contents; each call
 * clears what must start at zero.  Calls whose GPU work overlaps (other
 * streams or host threads) race on the array: serialise them. */
#define SCVT_STATIC_MAX_N 16384
scvt_status scvt_energy_grad_static(int64_t n, const scvt_density *rho, const double *z, void *cuda_stream,
                                    double *energy, double *grad, double *mass, double *moment);

/* Launch shape and search parameters of an evaluation (not in the paper:
 * GPU scheduling).  None of them changes a result -- a cell is unique, its
 * corners come from its neighbour triples and its sums are taken in its own
 * edge order -- only the time.  Defaults: 2, 24, 4, 16, 256, 32, 3. */
typedef struct {
    int bin_load;           /* target generators per cube-map bin, 1..16: G = ceil(sqrt(N / (6 bin_load)))
                               bins per face edge */
    int knn_target;         /* candidates the first search radius aims at when a cell has no radius
                               from a previous evaluation, 8..64 */
    int topo_warps;         /* warps per block of the topology pass (one warp per cell): 2, 4 or 8 */
    int topo_blocks_per_sm; /* grid cap of the topology pass in blocks per SM, 1..64 */
    int quad_block;         /* threads per block of the per-edge quadrature: 128, 256 or 512 */
    int topo_cell_lanes;    /* lanes per cell in the topology pass: 32 (one cell per warp) or 16 (two) */
    int chunks;             /* cell pipelines run concurrently on forked streams, 1..4 */
} scvt_tuning;

/* Set / read the tuning of a handle.  INVALID when a field is out of range. */
scvt_status scvt_set_tuning(scvt_handle *h, const scvt_tuning *t);
scvt_status scvt_get_tuning(const scvt_handle *h, scvt_tuning *t);
/* Autotuner: times evaluations at z (N x 3, device or host) over a grid of
 * tunings, one coordinate at a time (concurrent chunks 1/2/3/4; topology
 * lanes per cell 32/16; bin
 * load 1/2/4/8; topology warps per block 2/4/8; topology grid cap 8/16/32
 * blocks per SM; quadrature block 128/256/512; first-pass target
 * 16/24/32/48, the last compared on
 * evaluations without radius hints), keeps the fastest and returns it in
 * *chosen (nullable).  About 30 evaluations.  Synchronises. */
scvt_status scvt_tune(scvt_handle *h, const double *z, scvt_tuning *chosen);

/* ---- Batches of independent problems ------------------------------------
 * Many problems of Sec. 2.1 (uneven N, each with its own density) solved
 * together on one GPU.  The paper solves one problem at a time; a batch is
 * a deployment form of the same computation: every evaluation covers all
 * problems' cells in one launch sequence (captured once as a CUDA graph and
 * replayed), and the LBFGS of Sec. 3.1 runs for all problems in lockstep,
 * each with its own line search, history, preconditioner and stopping test.
 * Each problem's results equal, bit for bit, those of a single-problem
 * handle with the same configuration (the tuning does not matter).
 *
 * Layout: problem b's generators are rows [off_b, off_b + n_b) of one
 * concatenated N_tot x 3 array, off_b = n_0 + ... + n_(b-1); the same for
 * gradients.  Per-problem scalars are host arrays of `count` entries.
 * The batch owns a CUDA stream of its own; every call first waits for the
 * work queued on the stream given at creation and synchronises before it
 * returns. */
typedef struct scvt_batch scvt_batch;

/* cfgs: `count` configurations (1 <= count <= 65535).  All must share
 * precision and lbfgs_m.  Allocates the workspace for N_tot = sum n_b
 * generators (the LBFGS history included).  Errors: INVALID, OOM, CUDA. */
scvt_status scvt_batch_create(const scvt_config *cfgs, int count, void *cuda_stream, scvt_batch **out);
void scvt_batch_destroy(scvt_batch *b);  /* NULL-safe */

/* Energies (host, count) and gradients (N_tot x 3, nullable) of every
 * problem at z (N_tot x 3).  Device or host pointers.  The status is that of
 * the first problem that failed (all problems are evaluated). */
scvt_status scvt_batch_energy_grad(scvt_batch *b, const double *z, double *energy, double *grad);

/* Lockstep Lloyd-preconditioned LBFGS of every problem, with the options of
 * scvt_lbfgs_solve (warm_start 0 or 1; 1 continues every problem from the
 * batch's previous solve).  z: N_tot x 3 in/out.  reports: host, count
 * entries (required); reports[b].status is problem b's outcome.  Returns OK
 * when every problem ended with OK or LINESEARCH, else the status of the
 * first problem that failed (the others are still solved). */
scvt_status scvt_batch_lbfgs_solve(scvt_batch *b, double *z, const scvt_solve_opts *opts,
                                   scvt_solve_report *reports);

/* Autotuner: as scvt_tune, on evaluations of the whole batch at z
 * (N_tot x 3).  Results of later calls do not depend on the choice. */
scvt_status scvt_batch_tune(scvt_batch *b, const double *z, scvt_tuning *chosen);
scvt_status scvt_batch_set_tuning(scvt_batch *b, const scvt_tuning *t);
scvt_status scvt_batch_get_tuning(const scvt_batch *b, scvt_tuning *t);

/* Counters of the batch (evaluations count batch evaluations). */
scvt_status scvt_batch_get_stats(const scvt_batch *b, scvt_stats *out);
scvt_status scvt_batch_reset_stats(scvt_batch *b);
const char *scvt_batch_last_error(const scvt_batch *b);

/* ---- Serving: continuous batching of solve requests ----------------------
 * A request loop for many independent problems arriving over time (a
 * deployment form; the paper solves one problem at a time).  Submitted jobs
 * wait in a FIFO queue; each scvt_server_step() first admits queued jobs in
 * order while the device-memory budget, the workspace rows and the job
 * slots allow, then advances every job on the device by one LBFGS iteration
 * (newly admitted jobs get their first evaluation in the same evaluation
 * round), and retires the jobs that stopped.  A job's generators, gradient,
 * preconditioner and LBFGS history stay resident on the device from
 * admission to retirement; all jobs' evaluations share one launch sequence
 * (the batch workspace above, re-laid out when the set of jobs changes).
 * Each job's result equals, bit for bit, a single-problem scvt_lbfgs_solve
 * with the same configuration and options from the same start.
 * All calls are on the thread that owns the server. */
typedef struct scvt_server scvt_server;

typedef struct {
    int64_t memory_budget;   /* device bytes for the workspace plus resident jobs; 0 = 80 % of the free
                                memory at creation */
    int64_t max_generators;  /* most generators on the device at once (sum of N of running jobs) */
    int max_jobs;            /* most jobs on the device at once, 1..65535 */
    int precision;           /* as scvt_config.precision, for every job */
    int lbfgs_m;             /* as scvt_config.lbfgs_m, for every job */
} scvt_server_config;

typedef enum {
    SCVT_JOB_QUEUED = 0,
    SCVT_JOB_RUNNING = 1,
    SCVT_JOB_DONE = 2,      /* stopped by a tolerance or max_iter (report.status OK or LINESEARCH) */
    SCVT_JOB_FAILED = 3,    /* report.status holds the problem's error */
    SCVT_JOB_FETCHED = 4    /* result handed out by scvt_server_fetch */
} scvt_job_state;

typedef struct {
    int state;                     /* scvt_job_state */
    int64_t n;
    double t_submit, t_admit, t_done;  /* seconds on the server clock; -1 = not yet */
    int64_t bytes_resident;        /* device bytes the job holds while running */
    scvt_solve_report report;      /* progress so far; final once DONE or FAILED */
} scvt_job_info;

/* Errors: INVALID (bad config; workspace larger than the budget), OOM, CUDA. */
scvt_status scvt_server_create(const scvt_server_config *cfg, void *cuda_stream, scvt_server **out);
void scvt_server_destroy(scvt_server *s);  /* NULL-safe; drops queued and running jobs */
/* Queue a job: n generators with density rho, start z0 (n x 3, host or
 * device; copied before return), solve options as scvt_lbfgs_solve
 * (warm_start must be 0; NULL = defaults).  INVALID when n exceeds
 * max_generators, when the job alone exceeds the memory budget, or on a bad
 * density or option.  *job_id receives the id (ids count from 0). */
scvt_status scvt_server_submit(scvt_server *s, int64_t n, const scvt_density *rho, const double *z0,
                               const scvt_solve_opts *opts, int64_t *job_id);
/* One scheduling step (admit, one iteration of every running job, retire).
 * running / queued (nullable) receive the counts after the step. */
scvt_status scvt_server_step(scvt_server *s, int *running, int *queued);
/* State and timing of a job. */
scvt_status scvt_server_job(const scvt_server *s, int64_t job_id, scvt_job_info *info);
/* Copy a finished job's generators (n x 3, host or device) and release them.
 * INVALID if the job is not DONE or FAILED. */
scvt_status scvt_server_fetch(scvt_server *s, int64_t job_id, double *z_out);
/* Seconds since the server was created (the clock of scvt_job_info). */
double scvt_server_clock(const scvt_server *s);
scvt_status scvt_server_get_stats(const scvt_server *s, scvt_stats *out);
const char *scvt_server_last_error(const scvt_server *s);

/* Bisection refinement (Sec. 4.3: the optimisation-bisection procedure
 * that initialises the large meshes): z_out receives the N generators z
 * followed by the midpoints normalize(z_i + z_j) of all Delaunay edges
 * i < j, in lexicographic (i, j) order -- 4N - 6 points for a full
 * triangulation.  z: N x 3; z_out: cap x 3 (device or host).  *n_out (host)
 * receives the count; INVALID if it exceeds cap or a cell has more than 32
 * neighbours.  Synchronises. */
scvt_status scvt_bisect(scvt_handle *h, const double *z, double *z_out, int64_t cap, int64_t *n_out);

/* Mesh quality measures of Sec. 4: cellq[i] = min / max great-circle length
 * of the edges of Voronoi cell i (N values, nullable); triq = (a+b-c)(b+c-a)
 * (c+a-b)/(abc) of every Delaunay triangle with arc lengths a, b, c (1 for
 * an equilateral triangle), triangles (i < j < k) in lexicographic order,
 * up to tri_cap values (nullable).  *n_tri (host) receives the number of
 * triangles (2N - 4); INVALID if it exceeds tri_cap or a cell has more than
 * 32 neighbours.  Device or host arrays.  Synchronises. */
scvt_status scvt_mesh_quality(scvt_handle *h, const double *z, double *cellq, double *triq, int64_t tri_cap,
                              int64_t *n_tri);

/* Monte Carlo initialisation by the density (Sec. 4.1 starts its serial
 * tests from it): candidate k is kept when u_k * rho_max^e <= rho(cand_k)^e,
 * rho_max the density's largest value (1 for rho = 1 and X3, the cap centre
 * for the tanh kinds); the first n_target kept candidates, in candidate
 * order, are written to z_out.  exponent e in (0, 4]: 1 samples by rho,
 * 1/2 by rho^(1/2), the asymptotic CVT generator density on a surface.  cand: m x 3 unit vectors (the caller draws
 * them uniformly on S^2), u: m values in [0, 1), z_out: n_target x 3 -- each
 * device or host.  *n_out (host) receives the number written, below
 * n_target if the candidates run out.  1 <= m < 2^31.  Allocates and frees
 * temporaries on the stream; synchronises it. */
scvt_status scvt_sample_density(const scvt_density *rho, double exponent, const double *cand, const double *u,
                                int64_t m, int64_t n_target, double *z_out, int64_t *n_out, void *cuda_stream);

/* Per-handle counters and (with profiling on) device times. */
scvt_status scvt_get_stats(const scvt_handle *h, scvt_stats *out);
scvt_status scvt_reset_stats(scvt_handle *h);
/* Profiling: record CUDA events around the cell kernel and evaluations. */
scvt_status scvt_set_profiling(scvt_handle *h, int enabled);

const char *scvt_status_string(scvt_status s);
/* Description of the handle's last error ("" if none); owned by the handle. */
const char *scvt_last_error(const scvt_handle *h);
/* Library build string (compute capability, precision modes). */
const char *scvt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SCVT_H */
