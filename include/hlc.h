/*
 * hlc.h -- C ABI of the GB300 H-matrix Gaussian log-likelihood library.
 *
 * One evaluation of the joint Gaussian log-likelihood of a zero-mean Matern
 * random field observed at n scattered 2-D locations (arXiv:1709.08625):
 *
 *   L(theta) = -n/2 log(2 pi) - 1/2 log det C(theta) - 1/2 z^T C(theta)^-1 z   (eq. 1)
 *
 * computed with a hierarchical (H-) matrix approximation C~ of the covariance
 * (Sec. 2.2), its H-Cholesky factor L~, log det C~ = 2 sum log L~_ii and the
 * triangular solve L~ v = z (eq. 2), with the quadratic form refined against
 * C~ in FP64.  The covariance is the Matern function of eq. (3),
 *
 *   C(h) = sigma2 / (2^(nu-1) Gamma(nu)) (h/ell)^nu K_nu(h/ell),
 *
 * plus the nugget tau^2 on the diagonal (Sec. 4.1, eq. 4).
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: HLC_OK (0) or a negative HLC_ERR_*
 *     code; hlc_serve_poll may also return HLC_PENDING (1).  Functions never
 *     abort the process; hlc_strerror(status) gives a one-line description.
 *   - Outputs go through out-parameters.  Opaque handles are owned by the
 *     caller and released with the matching *_free / hlc_destroy.
 *   - Array arguments are borrowed for the duration of the call only.  A
 *     pointer may point to host memory or to device memory of the context's
 *     device (detected per call); results are written to the same kind of
 *     memory the caller passed.
 *   - Points and data vectors are in the caller's order; the tree
 *     permutation stays internal.
 *   - A non-positive pivot in the factorisation (the NaN failure described in
 *     Sec. 3) is reported as HLC_ERR_NOT_SPD; no NaN is returned.
 *   - All device work of a context runs on the context's stream; calls on one
 *     context must not overlap from several host threads.
 *
 * Environment switches (read once per process; the defaults are the product
 * path, the others serve measurement and comparison):
 *   HLC_ACCUMULATE=1  defer the updates of a low-rank block and truncate them
 *                     together before its next use (default: every update is
 *                     truncated at once)
 *   HLC_PERSISTENT=0  run triangular solves and matvecs wave by wave instead of
 *                     as one cooperative launch
 *   HLC_FACTOR_FLOW=0 replay the H-Cholesky's waves from a CUDA graph instead of
 *                     running it as one dependency-driven cooperative launch
 *                     (same result, bit for bit)
 *   HLC_FLOW=0        in that cooperative launch, separate the waves by a grid
 *                     barrier instead of starting every op once its own
 *                     producers are done (same result, bit for bit)
 *   HLC_GRAPHS=0      launch the op waves directly instead of replaying CUDA
 *                     graphs
 *   HLC_CHAINS=1      plan the solve of every small diagonal block as one
 *                     chain op run by one CTA instead of op by op (same
 *                     result, bit for bit)
 *   HLC_PROFILE=1     time every op launch (synchronising) and print a summary
 *                     at exit
 *   HLC_PHASES=1      count clock cycles per phase of the truncation kernel
 *                     (separately for batches of at most 32 columns and wider
 *                     ones) and print them when the context is destroyed
 *   HLC_FACTOR_TRACE=<path>  record the dependency-driven factorisation's
 *                     timeline (per op: taken, ready, done, CTA, releasing
 *                     producer) and write it to <path> after every
 *                     factorisation (paper_1709_08625_gb300/factor_trace.py
 *                     reads it)
 *   HLC_SOLVE_TRACE=<path>   the same timeline for every dependency-driven
 *                     solve or matvec, written to <path>.fwd, <path>.bwd and
 *                     <path>.mv (the last run of each plan)
 */
#ifndef HLC_H
#define HLC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define HLC_OK 0
#define HLC_PENDING 1
#define HLC_ERR_ARG (-1)       /* invalid argument (null pointer, n <= 0, bad theta ...) */
#define HLC_ERR_OOM (-2)       /* device or host allocation failed */
#define HLC_ERR_NOT_SPD (-3)   /* non-positive pivot in the H-Cholesky factorisation */
#define HLC_ERR_TIMEOUT (-4)   /* a bounded device wait expired */
#define HLC_ERR_CUDA (-5)      /* a CUDA runtime call failed */
#define HLC_ERR_RANK (-6)      /* a low-rank block needed more than kmax columns */
#define HLC_ERR_STATE (-7)     /* call out of order (e.g. factor before assemble) */
#define HLC_ERR_UNSUPPORTED (-8)
#define HLC_ERR_NUMERIC (-9)   /* numerical breakdown (NaN in a factor or a sum) */
#define HLC_ERR_SCRATCH (-10)  /* the tree needs more than the fixed buffer of hlc_matvec_noalloc */

/* ---- precision modes ---------------------------------------------------- */
#define HLC_FP64 0         /* every stage in FP64 */
#define HLC_MIXED 1        /* FP32 low-rank panels, updates and recompression
                              core (QRCP, Jacobi SVD, coefficients); FP64 leaf
                              POTRF, log-det and refinement */
#define HLC_MIXED_SVD64 2  /* as HLC_MIXED, with the recompression core in FP64 */

typedef struct hlc_ctx hlc_ctx;   /* device, stream, workspaces; owns device memory */
typedef struct hlc_tree hlc_tree; /* cluster tree + block-cluster tree of one point set */
typedef struct hlc_hmat hlc_hmat; /* an assembled C~ or a factor L~ (device resident) */

/* theta = (ell, nu, sigma2) of eq. (3) and the nugget tau^2 of eq. (4). */
typedef struct {
  double sigma2; /* variance, > 0 */
  double ell;    /* range, > 0 */
  double nu;     /* smoothness, > 0 */
  double nugget; /* tau^2 >= 0, added to the diagonal */
} hlc_theta;

/* ---- block structure variants (Sec. 2.2, App. A) -------------------------- */
#define HLC_ADM_STANDARD 0  /* admissible iff dist > 0 and min(diam) <= eta dist (App. A) */
#define HLC_ADM_MAXDIAM 1   /* admissible iff dist > 0 and max(diam) <= eta dist (App. A) */
#define HLC_ADM_WEAK 2      /* every block of two distinct clusters is admissible */
#define HLC_SPLIT_GEOMETRIC 0   /* bisect the longest bounding-box axis at its midpoint */
#define HLC_SPLIT_CARDINALITY 1 /* split the points at the median of the longest axis:
                                   two equal-sized sub-sets (Sec. 2.2) */

typedef struct {
  int leaf;           /* n_min: largest leaf cluster (Sec. 2.2), 1..128 */
  double eta;         /* admissibility parameter (App. A), > 0 */
  double eps;         /* block accuracy of C~ and of the H-arithmetic (Sec. 2.2) */
  int precision;      /* HLC_FP64, HLC_MIXED or HLC_MIXED_SVD64 */
  double refine_tol;  /* stop the solve when |z - C~ x| <= refine_tol |z| */
  int refine_maxit;   /* at most this many preconditioned CG iterations */
  int kmax;           /* rank capacity of a low-rank block, 1..128 */
  int admissibility;  /* HLC_ADM_STANDARD (default), HLC_ADM_MAXDIAM or HLC_ADM_WEAK */
  int split;          /* HLC_SPLIT_GEOMETRIC (default) or HLC_SPLIT_CARDINALITY */
  int fixed_rank;     /* 0: adaptive rank (accuracy eps); k > 0: fixed-rank mode
                         (Tables 2 and 3): every low-rank block -- ACA and every
                         truncation -- keeps at most k columns (those with
                         sigma_i > eps sigma_1), without an error; k <= kmax */
} hlc_params;

typedef struct {
  double loglik;       /* L~(theta), eq. (2) with the refined quadratic form */
  double logdet;       /* 2 sum log L~_ii */
  double quad;         /* z^T x, x refined against C~ */
  double quad_factor;  /* v^T v with L~ v = z (eq. 2 as printed) */
  int refine_iters;    /* preconditioned CG iterations */
  double rel_residual; /* |z - C~ x| / |z| at exit */
  double est_rel_err;  /* estimate of |I - (L~ L~^T)^-1 C~|_2 (Table 5's last
                          column): the largest distance from 1 of the Ritz
                          values that the CG iterations give for the
                          preconditioned operator (Lanczos); a lower bound
                          that tightens with refine_iters; -1 without an
                          iteration.  The factor's error against C~ in the
                          2-norm; the refined quadratic form itself is exact
                          to rel_residual times the condition of C~. */
  size_t bytes_C;      /* storage of C~ (actual ranks) */
  size_t bytes_L;      /* storage of L~ (actual ranks) */
  int max_rank_C, max_rank_L;
  double ms_assemble, ms_factor, ms_solve; /* device time per phase */
  double ms_total;     /* served requests: submit-to-completion wall time */
} hlc_result;

/* Defaults: leaf 64, eta 2, eps 1e-6, HLC_FP64, refine_tol 1e-12,
 * refine_maxit 100, kmax 64, standard admissibility, geometric split,
 * adaptive rank. */
void hlc_default_params(hlc_params* p);

/* Description of a status code (static string, never NULL). */
const char* hlc_strerror(int status);

/* Create a context on CUDA device `device` (its own stream and workspaces).
 * HLC_ERR_CUDA if the device is absent. */
int hlc_create(hlc_ctx** out, int device);
/* Destroy a context.  Free its trees and H-matrices first: they refer to it. */
void hlc_destroy(hlc_ctx* ctx);

/*
 * Cluster tree and block-cluster tree of n points (Sec. 2.2, Def. 2.2, App. A).
 * xy: n x 2 row-major FP64 (x0, y0, x1, y1, ...), host or device.
 * The points are Morton-sorted over their bounding box and bisected
 * (p->split: geometrically, the longest axis of the tight bounding box at its
 * midpoint; or by cardinality, at the median along that axis) down to
 * clusters of at most p->leaf points; block pairs of the lower triangle that
 * are admissible under p->admissibility are low-rank, other pairs with a
 * leaf cluster are dense.  Runs on the device.
 * The parameters are copied into the tree and used by every later call on it.
 */
int hlc_build_tree(hlc_ctx* ctx, const double* xy, int64_t n, const hlc_params* p,
                   hlc_tree** out);
void hlc_tree_free(hlc_tree* t);

/* info[8] = {n, clusters, leaf clusters, dense leaves, low-rank leaves,
 *            depth, plan ops, plan waves}. */
int hlc_tree_info(const hlc_tree* t, int64_t* info);
/* Device memory a tree holds, in bytes (host array of 6): out[0] one
 * H-matrix arena (blocks at their rank capacity, and the rank words),
 * out[1] H-matrices kept as the tree's evaluation workspace (0..2; both
 * after the first hlc_loglik), out[2] plan temporaries, out[3] vectors and
 * point / block descriptors, out[4] op programs, out[5] the total
 * out[0] * out[1] + out[2] + out[3] + out[4].  Plans and workspaces appear
 * once built (the first hlc_loglik on the tree builds all of them). */
int hlc_tree_memory(const hlc_tree* t, int64_t* out);
/* perm[i] = caller index of the point at tree position i (host array of n). */
int hlc_tree_perm(const hlc_tree* t, int32_t* perm);
/* Leaf blocks, 5 int64 each {row lo, row hi, col lo, col hi, type (0 dense,
 * 1 low-rank)} in tree positions, depth-first order; host array. */
int hlc_tree_leaf_blocks(const hlc_tree* t, int64_t* out);

/*
 * Assemble C~(theta) (Sec. 2.2): dense leaves exactly, admissible leaves by
 * ACA with partial pivoting (App. B) recompressed by QR+SVD to block
 * accuracy eps (Remark A.1).  The result is owned by the caller.
 */
int hlc_assemble(hlc_ctx* ctx, hlc_tree* t, const hlc_theta* th, hlc_hmat** C);

/* H-Cholesky C~ = L~ L~^T (Table 1) with truncation at eps; C is kept. */
int hlc_cholesky(hlc_ctx* ctx, const hlc_hmat* C, hlc_hmat** L);

/* y = C~ x (C~ symmetric, Table 1 matvec); x, y: n values in caller order. */
int hlc_matvec(hlc_ctx* ctx, const hlc_hmat* C, const double* x, double* y);

/*
 * Product with the H-Cholesky factor L~ (from hlc_cholesky): y = L~ x
 * (trans = 0) or y = L~^T x (trans = 1), FP64 arithmetic.  In caller order
 * this is P L~ P^T x with P the tree permutation, so that L~ L~^T is C~ in
 * caller order.  x, y: n values, host or device.  Synchronous.
 */
int hlc_factor_apply(hlc_ctx* ctx, const hlc_hmat* L, int trans, const double* x, double* y);

/*
 * Synthetic data of Sec. 5.1: the H-Cholesky factorisation C~(theta) = L~ L~^T
 * on the tree (in the tree's precision mode), then z = L~ xi in caller order,
 * so that z ~ N(0, C~(theta)) when xi ~ N(0, I).  xi, z: n values, host or
 * device; the caller draws xi.  Uses the tree's evaluation workspace (a later
 * hlc_loglik on the tree overwrites it).  Synchronous.
 */
int hlc_sample(hlc_ctx* ctx, hlc_tree* t, const hlc_theta* th, const double* xi, double* z);

/*
 * Accuracy diagnostics of the H-approximation at theta (Sec. 3: Tables 2, 3
 * and 5): assembles C~(theta) and its factor L~ on the tree (the tree's
 * evaluation workspace), then estimates with `iters` power iterations from
 * seeded random starts (FP64, tree order):
 *   out[0] |C - C~|_2      (C the exact covariance, evaluated on the fly)
 *   out[1] |C|_2
 *   out[2] |C~ - L~ L~^T|_2
 *   out[3] |I - (L~ L~^T)^-1 C~|_2 (Table 5's last column; power iteration
 *          on A^T A)
 *   out[4] KLD(C, C~) of Sec. 3 (zero means), to second order
 *          1/4 |L~^-1 (C - C~) L~^-T|_F^2, estimated with `probes` Gaussian
 *          probes (0: not estimated)
 *   out[5] |C~|_2
 * Power-iteration values approach the norms from below.  out[0], out[1] and
 * out[4] need O(n^2) covariance evaluations per product and are computed for
 * n <= 131072 only; -1 marks a value not computed.  Allocates a few vectors
 * of n doubles for the call.  Synchronous.
 */
int hlc_diagnostics(hlc_ctx* ctx, hlc_tree* t, const hlc_theta* th, int iters, int probes, uint64_t seed,
                    double* out);

/*
 * y = C~ x without allocating device memory (the paper has no counterpart:
 * this is an interface for callers that may not allocate during a call).
 * Same result, bit for bit, as hlc_matvec on the same C~ and x.  Like every
 * plan run, it executes as one persistent launch unless the context is a
 * serve slot or HLC_PERSISTENT=0 (or the cooperative launch is unavailable),
 * and wave by wave otherwise.
 *   x, y      device pointers, n doubles each in caller order (host pointers
 *             -> HLC_ERR_ARG); borrowed for the call, synchronous.
 *   scratch   one fixed buffer of hlc_matvec_noalloc_capacity() doubles
 *             (64 MiB) per device and process, part of the library module.
 *             A tree needs 3 n + (matvec temporaries) doubles of it, about
 *             n <= 3e5 at leaf 64 and kmax 64; larger -> HLC_ERR_SCRATCH.
 *   preconditions  the matvec plan of C's tree exists: call hlc_matvec or
 *             hlc_loglik on that tree once first, else HLC_ERR_STATE.
 *   concurrency  calls whose device work overlaps (other host threads,
 *             contexts or streams on the same device) share the buffer and
 *             corrupt each other's results: serialise them.
 *   first call  the first call on a device looks the buffer up (and may load
 *             the module there); make it before any stream capture begins.
 */
int hlc_matvec_noalloc(hlc_ctx* ctx, const hlc_hmat* C, const double* x, double* y);
/* Capacity in doubles of the fixed buffer of hlc_matvec_noalloc. */
int64_t hlc_matvec_noalloc_capacity(void);

/*
 * Self-test of the bounded device waits (no counterpart in the paper).  The
 * persistent solve kernel separates its waves by a grid barrier whose wait is
 * limited to 2 s; past the limit every CTA leaves the kernel and the call
 * returns HLC_ERR_TIMEOUT.  This call makes two CTAs wait at a barrier that
 * expects one arrival more than there are CTAs, so that only the limit can
 * end the wait: it returns HLC_ERR_TIMEOUT after about 2 s, and the context
 * stays usable.  Synchronous.
 */
int hlc_selftest_barrier_timeout(hlc_ctx* ctx);

/*
 * Host-only self-test of the planner's dataflow programs (no device, no
 * context; no counterpart in the paper).  Builds a synthetic cluster tree
 * (midpoint bisection of the index interval [0, n) down to `leaf` points;
 * boxes: geometry 0 the intervals themselves, geometry 1 the tight boxes of
 * a square grid's points numbered in Morton order, n <= 2^26) and
 * block-cluster tree (admissible iff min(diam) <= eta * dist), the
 * H-Cholesky (a7, also with accumulated updates), forward and backward solve
 * (a9, a10), matvec and factor-product (f2) plans at rank capacity kmax, and
 * checks what the dependency-driven kernels rely on:
 * plans inside their buffers, dependency edges pointing forward, predecessor
 * counts, group truncations as consecutive parts with edges on the first,
 * the ready list, products joined into TRSMs, and a model run of the
 * factorisation kernel's ready-queue protocol with `ctas` CTAs (> 8) and
 * op durations drawn from `seed`.  stats (up to 15 entries): factorisation
 * ops, edges, groups, initially ready ops; forward ops, joined products;
 * backward ops, joined products; matvec ops; model makespan; leaves; rank
 * slots; milliseconds of planning the factorisation; a hash of the
 * factorisation's op program and one of the solve and matvec programs (equal
 * hashes: the same programs).  Returns HLC_OK,
 * HLC_ERR_STATE with the first violation in msg (msglen bytes,
 * NUL-terminated), HLC_ERR_ARG or HLC_ERR_OOM.
 */
int hlc_selftest_plans(int64_t n, int leaf, double eta, int geometry, int kmax, int ctas, uint64_t seed,
                       int64_t* stats, int nstats, char* msg, int msglen);

/* Dense expansion of C~ (symmetric) or L~ (lower) into an n x n column-major
 * host array in caller order; for small n only (n <= 16384). */
int hlc_hmat_expand(hlc_ctx* ctx, const hlc_hmat* M, double* out);

/* Ranks of the low-rank leaves in hlc_tree_leaf_blocks order (-1 for dense). */
int hlc_hmat_ranks(hlc_ctx* ctx, const hlc_hmat* M, int32_t* out);

void hlc_hmat_free(hlc_hmat* M);

/*
 * One likelihood evaluation on an existing tree: assemble C~(theta), factor,
 * log det, forward solve (eq. 2), C~^-1 z by conjugate gradients preconditioned
 * with the factor (App. B), in FP64; assemble L.
 * z: n values in caller order (host or device).  Uses the tree's cached
 * workspace; no device allocation after the first call on a tree.
 */
int hlc_loglik(hlc_ctx* ctx, hlc_tree* t, const hlc_theta* th, const double* z,
               hlc_result* out);

/* ---- identification of theta (Sec. 5, App. B) ------------------------------ */
/* Objective of hlc_nelder_mead: f(x, user) for x of the call's dimension;
 * NaN counts as +inf. */
typedef double (*hlc_objective)(const double* x, void* user);

/*
 * The simplex method of Nelder and Mead (Comput. J. 7, 1965, in the form of
 * Lagarias et al., SIAM J. Optim. 9, 1998), the minimiser of the App. B
 * listing; host code, no device work.  Coefficients: reflection 1, expansion
 * 2, contraction 1/2, shrink 1/2.  Starts from the simplex x, x + step_i e_i
 * and iterates until the simplex size (root mean square distance of the
 * vertices from their centroid) is below size_tol or max_iter iterations
 * have run.  x (dim values, 1 <= dim <= 64) is overwritten with the best
 * vertex; *fmin, *iters (either may be NULL) get its value and the
 * iterations run.
 */
int hlc_nelder_mead(int dim, double* x, const double* step, double size_tol, int max_iter, hlc_objective f,
                    void* user, double* fmin, int* iters);

typedef struct {
  double step[3];   /* initial simplex steps for (nu, ell, sigma2) */
  double size_tol;  /* stop below this simplex size */
  int max_iter;     /* iteration limit */
  int free_mask;    /* parameters identified: bit 0 nu, 1 ell, 2 sigma2 (7 = all
                       three, as in the paper); the others stay at start */
} hlc_fit_opts;

/* The App. B settings: steps 0.02 (nu), 0.04 (ell), 0.01 (sigma2), size
 * tolerance 1e-5, 200 iterations, all three parameters free. */
void hlc_default_fit_opts(hlc_fit_opts* o);

typedef struct {
  hlc_theta theta;   /* identified parameters (nugget as given in start) */
  double loglik;     /* L~ at theta */
  int iterations;    /* simplex iterations */
  int evaluations;   /* likelihood evaluations (each one hlc_loglik) */
  int failed_evals;  /* evaluations outside the parameter domain or whose
                        factorisation failed (counted as L = -inf) */
  int converged;     /* 1: stopped by the size tolerance, 0: by max_iter */
  int traced;        /* rows written to trace */
  double ms_total;   /* wall time of the whole fit */
} hlc_fit_result;

/*
 * Maximum-likelihood identification of theta = (nu, ell, sigma2) on one
 * tree (Sec. 5; the App. B listing): Nelder-Mead on -L~(theta), each
 * evaluation a full hlc_loglik (assembly, H-Cholesky, log det, solve) on the
 * device with the tree's parameters.  z: n values in caller order, host or
 * device.  start: the initial guess (its nugget stays fixed).  opts may be
 * NULL for the App. B settings.  trace (optional, trace_cap rows of 5
 * doubles): every evaluation as {nu, ell, sigma2, loglik, status}.
 * A point outside the domain (a parameter <= 0, nu >= 20) or whose
 * factorisation fails (HLC_ERR_NOT_SPD / NUMERIC / RANK) counts as
 * L = -inf; any other error ends the fit and is returned.
 */
int hlc_fit(hlc_ctx* ctx, hlc_tree* t, const double* z, const hlc_theta* start, const hlc_fit_opts* opts,
            double* trace, int trace_cap, hlc_fit_result* out);

/* ---- measurement ---------------------------------------------------------- */
/* The context's CUDA stream (cudaStream_t) in *stream, for timing with events
 * recorded on the stream the kernels run on. */
int hlc_ctx_stream(hlc_ctx* ctx, void** stream);
/* on = 1: count kernel launches, time every launch of the op kernels with
 * CUDA events and accumulate their algorithmic flops (small overhead);
 * on = 0: counting only. */
int hlc_ctx_set_profiling(hlc_ctx* ctx, int on);
/* Counters since the last reset (reset = 1 clears them after reading):
 * out[0] kernel launches of the library,
 * out[1 + 3*t .. 3 + 3*t] for op type t in {0 potrf, 1 trsm, 2 gemm,
 *   3 truncation (one CTA), 4 truncation (cluster), 5 chain (a small
 *   diagonal block's solve run by one CTA)}: launches, device ms (profiling
 *   on), algorithmic flops (chains: counted under trsm and gemm),
 * out[19] launches of the persistent solve kernel (one per triangular solve,
 *   product with the factor or matvec; their ops are not counted per type).
 * 20 doubles. */
int hlc_ctx_counters(hlc_ctx* ctx, int reset, double* out);

/* ---- serving: continuous batching of likelihood requests ------------------ */
/* Start the request loop with a device-memory budget and a slot limit.
 * max_slots slot workers (each its own context, stream and workspaces) admit
 * queued requests in arrival order as soon as a slot is free and the
 * request's estimated device footprint fits in what the budget has left;
 * admitted requests run concurrently on the device. */
int hlc_serve_start(hlc_ctx* ctx, size_t hbm_budget_bytes, int max_slots);
/* Queue one request (copies host arrays xy (n x 2 row-major) and z; p may be
 * NULL for the defaults); returns its id in *req_id.  A request in a mixed
 * mode whose factorisation meets a non-positive pivot or a NaN is evaluated
 * again in HLC_FP64 before its result is posted. */
int hlc_serve_submit(hlc_ctx* ctx, const double* xy, const double* z, int64_t n,
                     const hlc_theta* th, const hlc_params* p, uint64_t* req_id);
/* HLC_PENDING until done; then the request's status with *out filled
 * (ms_total = submit-to-completion wall time).  A finished request is
 * forgotten once polled. */
int hlc_serve_poll(hlc_ctx* ctx, uint64_t req_id, hlc_result* out);
/* Finish every queued request, then stop the loop. */
int hlc_serve_stop(hlc_ctx* ctx);

/* The device footprint (bytes) the request loop charges against its budget
 * for one request of n points with parameters p (NULL: defaults): two arenas
 * of n (3 leaf + 7.5 log2(n/leaf) kmax) doubles each, temporaries and
 * vectors.  0 for invalid arguments.  Host only. */
size_t hlc_serve_footprint(int64_t n, const hlc_params* p);

/* Host-only replay of the request loop's admission rule (no device work, no
 * context): nreq requests queued at time 0 in index order, request i holding
 * footprint[i] bytes for duration[i] time units once admitted, max_slots
 * slots and a budget of `budget` bytes.  The rule is the one the slot
 * workers apply: the head of the queue is admitted when a slot is free and
 * its footprint fits in what is left of the budget, or when nothing runs.
 * Outputs start[i] (admission time of request i) and *peak (largest sum of
 * footprints running at once).  HLC_ERR_ARG for invalid arguments. */
int hlc_serve_admission_replay(size_t budget, int max_slots, int64_t nreq, const size_t* footprint,
                               const double* duration, double* start, size_t* peak);

#ifdef __cplusplus
}
#endif
#endif /* HLC_H */
