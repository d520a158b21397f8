/*
 * fkt.h -- C ABI of the GB300-native Fast Kernel Transform (arXiv 2106.04487).
 *
 * The library computes the approximate kernel matrix-vector product
 *
 *     y = Ktilde(X, X) w,        y_i ~ sum_j K(|x_i - x_j|) w_j          (eq. nbody, Sec. 3)
 *
 * for an isotropic kernel K with the paper's tree code (Algorithm 1, Sec. 3.2):
 * a binary space partitioning tree over the points (Sec. 3.1), dense kernel
 * blocks between each target and the leaves it is near to, and for every
 * (target, node) pair that passes the far-field criterion of eq. accparam
 *
 *     max_{x' in node} |x' - c_node| / |x - c_node| < theta
 *
 * the order-p truncation of the generalized multipole expansion of Theorem 3.1
 * (eq. finaltrunc, eq. kdef): source-to-multipole (s2m) coefficients per node
 * and their multipole-to-target (m2t) evaluation.
 *
 * Conventions for every entry point:
 *   - Array pointers are DEVICE pointers unless the name ends in _host.
 *     The caller owns them; the library never frees or retains them past the call,
 *     except that fkt_plan copies the points into the plan.
 *   - Layouts: points row-major [N][d] float32 in the caller's order;
 *     weights w, results y, right-hand sides b and solutions x are RHS-major
 *     [nrhs][N] float32, in the caller's original point order.
 *   - Work is enqueued on the plan's CUDA stream (given at fkt_plan) and is
 *     asynchronous unless stated otherwise; fkt_plan, fkt_solve and the _host
 *     calls synchronize that stream before returning.
 *   - Every call returns an int status (FKT_OK = 0).  No C++ exception crosses
 *     the ABI.  A plan is not thread-safe: calls on one plan must not overlap.
 *   - Parameters that the paper leaves open are fixed as follows: the tree
 *     splits boxes at the midpoint cycling the axes (Sec. 3.1 rules (a),(b)); the
 *     node centre is the box midpoint and the node radius the largest distance
 *     from a point of the node to it; the far test is evaluated per target point
 *     in float64 as rho^2 < theta^2 |x - c|^2; singular kernels (Laplace) skip
 *     exact r = 0 pairs, all other kernels include K(0) w_i.
 */
#ifndef FKT_H
#define FKT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FKT_OK                0
#define FKT_ERR_INVALID_ARG   1  /* an argument is out of range (see each call) */
#define FKT_ERR_CUDA          2  /* a CUDA runtime call or kernel launch failed */
#define FKT_ERR_OOM           3  /* device memory allocation failed */
#define FKT_ERR_NOT_CONVERGED 4  /* fkt_solve reached max_iter above tol */
#define FKT_ERR_TIMEOUT       5  /* a bounded device-side wait ran out */
#define FKT_ERR_UNSUPPORTED   6  /* a valid request this build does not implement */
#define FKT_ERR_INTERNAL      7  /* an internal consistency check failed (a library bug) */
#define FKT_ERR_SCRATCH_LIMIT 8  /* the request needs more than fkt_mvm_noalloc's fixed scratch */

typedef struct fkt_plan_s* fkt_plan_t;

/* Isotropic kernels.  l = lengthscale, a = alpha, s = scale (a multiplier):
 *   FKT_GAUSSIAN     s exp(-r^2 / (2 l^2))
 *   FKT_EXPONENTIAL  s exp(-r / l)                              (Table 1, Matern nu=1/2)
 *   FKT_MATERN32     s (1 + sqrt3 r/l) exp(-sqrt3 r/l)          (Table 1)
 *   FKT_MATERN52     s (1 + sqrt5 r/l + 5 r^2/(3 l^2)) exp(-sqrt5 r/l)
 *   FKT_CAUCHY       s / (1 + r^2 / l^2)                        (Table 1, l = sigma)
 *   FKT_RATQUAD      s (1 + r^2 / (2 a l^2))^(-a)               (Table 1 has a = 1/2)
 *   FKT_LAPLACE      s / r      (Green's function: s = 1/(4 pi) in d = 3; r = 0 pairs skipped) */
typedef enum {
    FKT_GAUSSIAN = 0,
    FKT_EXPONENTIAL = 1,
    FKT_MATERN32 = 2,
    FKT_MATERN52 = 3,
    FKT_CAUCHY = 4,
    FKT_RATQUAD = 5,
    FKT_LAPLACE = 6
} fkt_kernel_kind;

typedef struct {
    int kind;            /* fkt_kernel_kind */
    double lengthscale;  /* l > 0 */
    double alpha;        /* a > 0, used by FKT_RATQUAD only */
    double scale;        /* s, any finite value */
} fkt_kernel;

/* Plan statistics.  Pair counts are exact and fixed by the method (they count
 * what Algorithm 1 evaluates for this tree and theta), not by the implementation. */
typedef struct {
    int64_t N;
    int32_t d, p;
    int32_t nterms;          /* expansion size binom(p+d, d) (Sec. 4.2) */
    int32_t leaf_size;
    int32_t depth;           /* deepest level; the root is level 0 */
    int64_t nodes, leaves;
    int64_t target_blocks;   /* groups of <= 128 consecutive targets of one leaf */
    int64_t far_entries, near_entries, masks;
    int64_t far_pairs;       /* (target, far node) pairs: m2t evaluations */
    int64_t near_pairs;      /* (target, source) pairs evaluated densely */
    int64_t s2m_pairs;       /* (source, node) pairs: s2m basis evaluations */
    int64_t s2m_nodes;       /* nodes whose coefficients some target uses */
    double plan_ms;          /* wall time of fkt_plan */
    double last_near_ms, last_far_ms, last_s2m_ms, last_total_ms; /* last fkt_mvm, if timing is on */
    int32_t coarse_columns;  /* columns of fkt_solve's coarse space after its last set-up (0: none) */
    int32_t coarse_dropped;  /* eigen-directions of its coarse operator E left out of E^+ */
} fkt_stats;

/* Build a plan (Sec. 3.1 tree, far/near sets of Sec. 3.1-3.2, expansion tables of Theorem 3.1).
 *   points     device [N][d] float32, finite
 *   N          1 <= N < 2^31
 *   d          2, 3 or 4.  d = 2 takes the circular harmonics cos k phi, sin k phi with the
 *              Chebyshev T_k as zonal functions (the alpha = 0 limit of the Gegenbauer form
 *              of Sec. A.1); its far field runs on the CUDA cores only (far_precision other
 *              than "fp32" makes fkt_mvm return FKT_ERR_UNSUPPORTED), and the batch entry
 *              points take d = 3 and 4 only.
 *   kernel     see fkt_kernel; lengthscale > 0 (alpha > 0 for FKT_RATQUAD)
 *   p          truncation order, 0 <= p <= 10 for d = 2 and 3, 0 <= p <= 8 for d = 4
 *   leaf_size  largest number of points in a leaf that may still split, 1 <= leaf_size <= 4096
 *   theta      far-field parameter of eq. accparam, 0 < theta < 1
 *   cuda_stream  cudaStream_t to enqueue on, or NULL for the default stream
 *   out        receives the plan; set to NULL on failure
 * Errors: FKT_ERR_INVALID_ARG for the ranges above or non-finite points;
 *         FKT_ERR_OOM / FKT_ERR_CUDA.  Synchronizes the stream. */
int fkt_plan(const float* points, int64_t N, int d, fkt_kernel kernel, int p, int leaf_size,
             double theta, void* cuda_stream, fkt_plan_t* out);

/* y = Ktilde w  (Algorithm 1), overwriting y.  w, y device [nrhs][N] float32, 1 <= nrhs <= 64;
 * w and y must not overlap.  Asynchronous on the plan's stream.
 * Errors: FKT_ERR_INVALID_ARG (null plan/pointers, nrhs out of range), FKT_ERR_OOM, FKT_ERR_CUDA. */
int fkt_mvm(fkt_plan_t plan, const float* w, float* y, int nrhs);

/* Same as fkt_mvm with HOST buffers: copies w to the device, runs the MVM and copies y back.
 * Pinned host memory gives the fastest copies.  Synchronizes the plan's stream. */
int fkt_mvm_host(fkt_plan_t plan, const float* w_host, float* y_host, int nrhs);

/* Exact dense product y_i = sum_j K(|x_i - x_j|) w_j (eq. nbody) on the GPU in float32 over the
 * plan's points (same r = 0 rule).  Device [nrhs][N] buffers as for fkt_mvm.  O(N^2) work. */
int fkt_dense_mvm(fkt_plan_t plan, const float* w, float* y, int nrhs);

/* ---- Gaussian-process style solves:  (Ktilde + sigma2 I) x = b  ----
 *
 * The paper uses the FKT product to evaluate GP posterior means, which need
 * Sigma^{-1} (y - mu) with Sigma = K + sigma_y^2 I (Sec. C, eq. gp_posterior), computed
 * through matrix-vector products only.  fkt_solve runs preconditioned conjugate gradients
 * with one fkt_mvm per iteration (all right-hand sides at once): iterates x and residuals r
 * in float64, inner products in float64, search directions and products in float32.
 * The preconditioner is block-Jacobi over the plan's target blocks (<= 128 consecutive
 * points of one leaf): each diagonal block K(X_b, X_b) + sigma2 I is factored (Cholesky)
 * and inverted in float32 on the GPU. */
typedef struct {
    int iterations;             /* CG iterations run */
    int converged;              /* 1 if every right-hand side reached tol */
    int used_fallback;          /* 1 if a learned correction was rejected for plain block-Jacobi */
    int pad;
    double rel_residual;        /* max over right-hand sides of |r_k| / |b| from the recurrence */
    double true_rel_residual;   /* max over right-hand sides of |b - (Ktilde + sigma2 I) x| / |b|,
                                   recomputed with one more fkt_mvm */
} fkt_solve_info;

/* Build the block-Jacobi preconditioner for (Ktilde + sigma2 I) (sigma2 > 0).  Called by
 * fkt_solve when needed; call it directly to time or inspect it.  Synchronizes. */
int fkt_precond_setup(fkt_plan_t plan, double sigma2);

/* z = M^{-1} r with the current preconditioner; r, z device [nrhs][N] float32 in the
 * caller's order, 1 <= nrhs <= 64.  FKT_ERR_INVALID_ARG if no preconditioner is set up. */
int fkt_precond_apply(fkt_plan_t plan, const float* r, float* z, int nrhs);

/* ---- Learned low-rank correction of the block-Jacobi preconditioner ----
 * For each target block b (points X_b) with neighbourhood y = up to 32 trailing points of block
 * b-1 and 32 leading points of block b+1 (neighbours in tree order), the teacher is the coupling of
 * the block to its neighbours folded into the block,
 *     T_b = A_by A_yy^{-1} A_yb  (positive semidefinite),  A = K + sigma2 I,
 * so that the corrected block A_bb + T_b acts on locally smooth vectors like the rows of A do
 * (the idea behind lumping dropped couplings into the diagonal in modified incomplete
 * factorisations).  A small network maps the block's points and its neighbours' points (relative
 * to the block's centroid, divided by the lengthscale) to V_b (n_b x rank):
 *     phi(u) = tanh(W2^T tanh(W1^T u + b1) + b2)                      (per point, width H)
 *     g = mean_{i in X_b} phi(u_i),  h = mean_{j in neighbours} phi(u_j)
 *     V_i = Wo^T [phi(u_i); g; h] + bo,
 * trained on the GPU (hand-written forward/backward kernels, Adam) to minimise
 *     L = sum_b |beta^2 V_b V_b^T - T_b|_F^2 / sum_b |T_b|_F^2
 * over a subset of blocks.  The preconditioner block is (A_bb + beta^2 V_b V_b^T)^{-1}, a rank-r
 * update of the block-Jacobi block, symmetric positive definite by construction.  Parameters are
 * one flat float32 vector: W1 [d][H], b1 [H], W2 [H][H], b2 [H], Wo [3H][rank], bo [rank], beta. */
typedef struct {
    int rank;          /* columns of V_b, 1..16 (default 8) */
    int hidden;        /* H, 8..64 (default 32) */
    int steps;         /* Adam steps (default 300) */
    float lr;          /* Adam learning rate (default 3e-3) */
    int train_blocks;  /* blocks used for training, every (nblocks / train_blocks)-th (default 512) */
    int seed;          /* initialisation seed */
    int install_teacher;  /* 1: install (A_bb + T_b)^{-1} itself (every block must be a training block,
                             train_blocks >= blocks): the target the network approximates, for
                             comparison; 0 (default): the network's correction */
} fkt_learn_opts;

typedef struct {
    int nparams;
    int ntrain;                 /* training blocks */
    double loss_initial;        /* L at the initial parameters */
    double loss_final;          /* L after training */
    double train_ms;            /* teacher generation + training + installation */
} fkt_learn_info;

/* Build the teacher data for sigma2, train the network, compute V_b for every block and install
 * the corrected preconditioner (used by fkt_solve with option "preconditioner" = "learned").
 * opts may be NULL for the defaults.  Synchronizes. */
int fkt_precond_learn(fkt_plan_t plan, double sigma2, const fkt_learn_opts* opts, fkt_learn_info* info);

/* The trained parameters (host, *nparams floats).  params may be NULL to query *nparams. */
int fkt_learn_params(fkt_plan_t plan, float* params, int* nparams);

/* Loss L and its gradient at the given parameters (host buffers of nparams floats) on the
 * training blocks of the last fkt_precond_learn, computed by the GPU forward/backward kernels. */
int fkt_learn_eval(fkt_plan_t plan, const float* params, double* loss, float* grad);

/* The training blocks' indices (host [ntrain]) and their teachers T_b (host [ntrain][128][128],
 * rows and columns beyond the block's size are zero).  Either pointer may be NULL. */
int fkt_learn_teacher(fkt_plan_t plan, int64_t* blocks, float* D);

/* Random Fourier frequencies of a kernel (host only, no device work): omega [R][d] and phase [R]
 * (row-major, caller-allocated host buffers) such that E[cos(omega . delta)] = K(|delta|) / K(0)
 * (Bochner's theorem), phase ~ U[0, 2 pi), drawn with a 64-bit Mersenne Twister seeded by seed.
 * Spectral densities: Gaussian N(0, I/l^2); exponential and Matern-nu (nu = 1/2, 3/2, 5/2)
 * multivariate Student t with 2 nu degrees of freedom and scale 1/l; rational quadratic and
 * Cauchy Gaussian scale mixtures (precision tau/l^2 with tau ~ Gamma(a, rate a), Cauchy: a = 1
 * and l^2/2); Laplace 1/r has no normalisable density, so it gets the Gaussian's at l.  These
 * are the features of fkt_solve's coarse space (option "coarse_rank").  The paper has no
 * counterpart.  1 <= d <= 8, 1 <= R <= 2^24; FKT_ERR_INVALID_ARG otherwise. */
int fkt_spectral_sample(fkt_kernel kernel, int d, int R, uint64_t seed, double* omega, double* phase);

/* Solve (Ktilde + sigma2 I) x = b.  b, x device [nrhs][N] float32 (x is output only),
 * 1 <= nrhs <= 64, sigma2 > 0, 0 < tol < 1, max_iter >= 1.  Synchronizes.
 * Returns FKT_OK when every right-hand side reached |r| <= tol |b|, FKT_ERR_NOT_CONVERGED
 * after max_iter iterations otherwise (x then holds the last iterate); info may be NULL. */
int fkt_solve(fkt_plan_t plan, double sigma2, const float* b, float* x, int nrhs, double tol, int max_iter,
              fkt_solve_info* info);

/* fkt_solve with the solution returned in float64: x device [nrhs][N] float64 (output only).
 * The CG iterates are float64; fkt_solve rounds them to float32.  Here x keeps the float64
 * iterate, and info->true_rel_residual is recomputed with two products, Ktilde x = Ktilde hi +
 * Ktilde lo (x = hi + lo, both float32), so that the rounding of x does not enter.  What limits
 * the true residual |b - (Ktilde + sigma2 I) x| / |b| either way is the float32 arithmetic of the
 * products CG runs on: the recurrence residual drifts from the true one by their errors (measured
 * for a GP system with sigma2 = 1e-2, N = 2000: recurrence 1e-7, true residual 9e-5 for both the
 * float64 and the float32 x).  Arguments, errors and synchronisation as for fkt_solve. */
int fkt_solve_f64(fkt_plan_t plan, double sigma2, const float* b, double* x, int nrhs, double tol, int max_iter,
                  fkt_solve_info* info);

/* ---- Batches of independent problems (one product over all of them) ----
 * Each problem has its own points and kernel; all share d, p and theta.  The batch plan builds
 * every problem's tree, lists and expansion, then merges them into one arena so each stage of the
 * product runs as one launch over the whole batch (near-field blocks grouped by kernel kind and
 * ordered by work, largest first), and captures the whole product as one CUDA graph that later
 * calls with the same buffers replay. */
typedef struct fkt_batch_s* fkt_batch_t;
typedef struct {
    const float* points;   /* device [N][d] float32 */
    int64_t N;             /* >= 1 */
    fkt_kernel kernel;
} fkt_problem;

/* leaf_size > 0 uses it for every problem; leaf_size = 0 autotunes it per size class (problems
 * whose N has the same power of two) by timing candidate plans (64, 128, 256, 512 points) on the
 * device with 8 right-hand sides (fkt_autotune_leaf).  Other arguments as for fkt_plan. */
int fkt_batch_plan(int nprob, const fkt_problem* probs, int d, int p, int leaf_size, double theta,
                   void* cuda_stream, fkt_batch_t* out);

/* y = Ktilde_i w for every problem i at once.  w, y device [nrhs][N_total] float32 where
 * N_total = sum N_i and problem i occupies columns [offset_i, offset_i + N_i) (fkt_batch_info),
 * each in its caller's point order.  The first call with given (w, y, nrhs) runs the product and
 * captures it as a CUDA graph; calls with the same buffers replay the graph.  Asynchronous. */
int fkt_batch_mvm(fkt_batch_t batch, const float* w, float* y, int nrhs);

/* fkt_set_option for every problem of the batch (drops the captured graph). */
int fkt_batch_set_option(fkt_batch_t batch, const char* key, const char* value);

/* offsets [nprob+1] (column offsets), leaf_sizes [nprob], totals; any pointer may be NULL. */
int fkt_batch_info(fkt_batch_t batch, int64_t* offsets, int32_t* leaf_sizes, fkt_stats* total);

/* Autotuner of the kernel variants for products with nrhs right-hand sides: times the batch
 * product (CUDA events, best of 3 after a warm-up) for each value of one option at a time and keeps
 * the fastest -- the tensor-core far field's CTA shape ("far_kernel": one far entry per thread at
 * four CTAs per SM, one with the row held in registers at three, or two per thread at two; BF16
 * forms, d = 3), the near field of
 * 32-wide passes ("near_precision": register-tiled CUDA cores, TF32 or FP16 tensor-core operands,
 * all float32-level accurate) and the single-RHS near kernel's targets per thread.  The far
 * precision, which sets the accuracy, is left as it is.  chosen (may be NULL) receives
 * "key=value;..." (at most len bytes with the terminating zero).  Synchronizes; drops the captured
 * graph. */
int fkt_batch_autotune(fkt_batch_t batch, int nrhs, char* chosen, int len);

/* fkt_check for the batch. */
int fkt_batch_check(fkt_batch_t batch);

void fkt_batch_destroy(fkt_batch_t batch);

/* Autotuner: build a plan for each candidate leaf size, time fkt_mvm with nrhs right-hand sides
 * (best of 3 after a warm-up, CUDA events), and return the fastest leaf size (and its time in
 * milliseconds if best_ms is not NULL).  Synchronizes. */
int fkt_autotune_leaf(const float* points, int64_t N, int d, fkt_kernel kernel, int p, double theta, int nrhs,
                      const int* candidates, int ncand, void* cuda_stream, int* best_leaf, double* best_ms);

/* Options (all take effect on the next call):
 *   "timing"    "0" | "1"   record per-stage CUDA-event times of fkt_mvm in fkt_stats
 *   "far_precision"  "fp32" (default) | "tf32" | "bf16" | "bf16x3"  arithmetic of the far-field
 *               contraction: fp32 on CUDA cores; otherwise on the tensor cores (tcgen05.mma,
 *               float32 accumulation in tensor memory) with operands in TF32, BF16, or BF16
 *               split into hi + lo parts (three products, about 16 significant bits); the
 *               near field's kernel values stay float32.  Right-hand sides go 32 per pass.
 *   "near_precision"  "fp32" (default) | "tf32x3"  arithmetic of the near-field contraction of
 *               passes of 17-32 right-hand sides: fp32 on CUDA cores, or on the tensor cores
 *               (tcgen05.mma kind::tf32, A = float32 kernel values in tensor memory) with each
 *               factor split into TF32 hi + lo parts (three products, about 20 significant bits
 *               per product) and the accumulator added into float32 registers every 128 sources;
 *               kernel values are float32 either way.  fkt_dense_mvm always uses fp32.
 *   "preconditioner" "block_jacobi" (default) | "learned" | "none"   preconditioner of fkt_solve;
 *               "learned" needs fkt_precond_learn first and falls back to block_jacobi when
 *               CG with the correction does not converge (fkt_solve_info.used_fallback)
 *   "coarse_rank"  "0" (default) | R in 1..256  adds a two-level coarse correction to fkt_solve's
 *               preconditioner: the coarse space spans R random Fourier features of the kernel
 *               (frequencies from fkt_spectral_sample), orthonormalised; with A = Ktilde + sigma2 I,
 *               W = A Q and E = Q^T W the preconditioner becomes
 *               Q E^-1 Q^T + (I - Q E^-1 W^T) M (I - W E^-1 Q^T), M = the "preconditioner" option
 *               (balancing two-level form; symmetric positive semi-definite).  It targets the
 *               smooth global modes that make CG slow for long-range kernels and small sigma2,
 *               which no block-diagonal M can represent.  Set-up per (sigma2, R, seed): R / 64
 *               fkt_mvm products plus float64 R x R factorisations on the host; per iteration
 *               two skinny N x R products each way.  Needs N >= 4 R and a single-problem plan
 *               (FKT_ERR_INVALID_ARG / FKT_ERR_UNSUPPORTED otherwise); fkt_solve returns
 *               FKT_ERR_INVALID_ARG if Ktilde + sigma2 I is not positive definite on the coarse
 *               space.  The paper has no counterpart (its GP solves run plain CG, Sec. C).
 *   "coarse_seed"  unsigned integer (default 1): seed of the coarse space's frequencies
 *   "near_targets_per_thread"  "2" (default) | "4"  register blocking of the near-field kernel
 *               (4 applies to one right-hand side; results are identical up to rounding order)
 *   "far_kernel"  "single" (default) | "pairs" | "held"  tensor-core far field of d = 3 in the BF16
 *               forms: each target thread generates its basis rows for one far entry at a time
 *               (four CTAs per SM at p <= 6); for two far entries at once in packed float32 pairs
 *               ("pairs", where the tensor memory allows: BF16 hi/lo up to p = 6, BF16 up to p = 9;
 *               two CTAs per SM); or for one entry, holding the first 64 terms of the row in
 *               registers until the previous entry's MMAs complete ("held", three CTAs per SM).
 *               Results agree up to rounding order.
 *   "wait_limit_cycles"  "default" | an integer 0..2000000000  limit, in SM clocks, of the
 *               pipeline waits of the tensor-core near and far kernels (a source-record or
 *               multipole copy landing, the hand-off of a chunk or entry to the MMA issuer).
 *               The default (about one second) is reached only by a fault; a wait that runs out
 *               stops that CTA's work, and fkt_check reports FKT_ERR_TIMEOUT.  A small value makes
 *               the waits give up early on valid work: a test hook for the failure path (0 = a
 *               single poll).  The waits that drain copies and MMAs in flight before a CTA exits
 *               keep the default.
 * Errors: FKT_ERR_INVALID_ARG for an unknown key or value. */
int fkt_set_option(fkt_plan_t plan, const char* key, const char* value);

/* Copy the plan's statistics into *out. */
int fkt_plan_stats(fkt_plan_t plan, fkt_stats* out);

/* Export the tree (Sec. 3.1), nodes in breadth-first order, host buffers sized from fkt_plan_stats:
 *   perm [N]           sorted position -> caller's point index
 *   begin, end [nodes] point range [begin, end) in sorted order
 *   level, leaf [nodes], child [nodes][2] (-1 = none)
 *   centre [nodes][d] float64, rho2 [nodes] float64
 * Any pointer may be NULL to skip that array.  Synchronizes the stream. */
int fkt_plan_tree(fkt_plan_t plan, int64_t* perm, int64_t* begin, int64_t* end, int32_t* level,
                  int32_t* leaf, int64_t* child, double* centre, double* rho2);

/* Export the interaction lists per target block (host buffers sized from fkt_plan_stats):
 *   block_range [blocks][2]  sorted target range [lo, hi) of each block (hi - lo <= 128)
 *   far_off [blocks+1], far_node [far_entries], far_mask [far_entries]
 *   near_off [blocks+1], near_leaf [near_entries], near_mask [near_entries]
 *   masks [masks][4] uint32: bit t of mask m is set when target lo+t takes the entry;
 *   an entry whose mask index is -1 applies to every target of its block.
 * Any pointer may be NULL.  Synchronizes the stream. */
int fkt_plan_lists(fkt_plan_t plan, int64_t* block_range, int64_t* far_off, int32_t* far_node,
                   int32_t* far_mask, int64_t* near_off, int32_t* near_leaf, int32_t* near_mask,
                   uint32_t* masks);

/* ---- Target-sharded product over several processes (one GPU each) ----
 * The product shards by targets with one exchange step.  Every rank builds the same plan from all
 * the points (the tree and lists of Sec. 3.1 are deterministic).  The target blocks, in tree
 * (Morton) order, are split into one contiguous range per rank, balanced by their work (near
 * pairs plus far pairs weighted by the cost of a basis row).  Each target keeps its own far and
 * near sets (eq. accparam), so every (target, source) pair is evaluated exactly once, by the rank
 * owning the target.  A rank owns the sources of its target range too: fkt_mvm_shard_begin
 * computes the partial multipoles (s2m, Algorithm 1) of those sources for every node, the caller
 * sums them over the ranks (one allreduce), and fkt_mvm_shard_end evaluates the far field
 * (m2t) and the near field of the rank's targets.  s2m is linear in the weights, so the sum is
 * the full product's multipoles.  w must hold all N weights on every rank (the near field reads
 * any source); y receives the rank's targets only.  One pass: 1 <= nrhs <= 32.  The paper's code
 * is single-process; this is the partition of its Algorithm 1 by targets. */

/* Host only, no device work: split nblocks blocks of the given non-negative work into nranks
 * contiguous ranges; bounds [nranks+1] receives the first block of each rank and nblocks.  A
 * block goes to the rank whose share of the total work contains the block's cumulative midpoint.
 * FKT_ERR_INVALID_ARG for nranks outside 1..4096, negative or NaN work, or null pointers. */
int fkt_shard_partition(int64_t nblocks, const double* work, int nranks, int64_t* bounds);

/* The work of each target block (host [target_blocks], from fkt_plan_stats) that the partition
 * balances, near pairs plus 50 x far pairs, with the blocks in target order (sorted by their first
 * target; fkt_plan_lists lists them leaf by leaf).  Synchronizes.  FKT_ERR_UNSUPPORTED for batch
 * plans. */
int fkt_shard_block_work(fkt_plan_t plan, double* work);

/* Select this process's share: rank in 0..nranks-1.  Partitions the blocks (fkt_shard_partition
 * over fkt_shard_block_work) and cuts the s2m work to the rank's sources.  Synchronizes. */
int fkt_shard_set(fkt_plan_t plan, int nranks, int rank);

/* The selected share: target blocks [block_lo, block_hi) in target order, sorted targets [target_lo, target_hi)
 * (positions in tree order; fkt_plan_tree's perm maps them to the caller's indices), and the size
 * in floats of the multipole array that fkt_mvm_shard_begin fills for nrhs right-hand sides.
 * Any pointer may be NULL.  FKT_ERR_INVALID_ARG before fkt_shard_set. */
int fkt_shard_info(fkt_plan_t plan, int nrhs, int64_t* block_lo, int64_t* block_hi, int64_t* target_lo,
                   int64_t* target_hi, int64_t* mult_floats);

/* Phase 1: w device [nrhs][N] float32 (all points, caller order); mult device float32 of
 * fkt_shard_info's mult_floats, overwritten with this rank's partial multipoles.  The caller then
 * sums mult over the ranks (e.g. an NCCL allreduce) before phase 2.  Asynchronous. */
int fkt_mvm_shard_begin(fkt_plan_t plan, const float* w, float* mult, int nrhs);

/* Phase 2: mult = the multipoles summed over all ranks; y device [nrhs][N] float32 (caller
 * order) receives the product for this rank's targets, other entries untouched.  Uses the source
 * records of the last fkt_mvm_shard_begin on this plan (same w, same nrhs).  Asynchronous. */
int fkt_mvm_shard_end(fkt_plan_t plan, const float* mult, float* y, int nrhs);

/* fkt_mvm without any device allocation.
 *
 * fkt_mvm grows per-call work buffers with cudaMalloc the first time it sees a larger nrhs.
 * Some callers cannot allow that: code recording a CUDA graph (an allocation during stream
 * capture invalidates the capture), latency-critical loops (cudaMalloc can synchronise the
 * whole device), and hosts whose memory is owned by another allocator, such as a framework's
 * caching pool, where a raw cudaMalloc can fail or fragment memory the pool already holds.
 * This entry point computes exactly what fkt_mvm computes, with the same kernels, but takes
 * its work buffers from a fixed array in device memory that the library declares statically;
 * it calls no cudaMalloc, cudaFree or other allocating routine.  The paper has no counterpart;
 * the result is the same product that fkt_mvm computes.
 *
 *   plan, w, y, nrhs  as for fkt_mvm (device buffers, [nrhs][N], 1 <= nrhs <= 64).
 *   The device that was current at fkt_plan must be current at the call (FKT_ERR_INVALID_ARG
 *   otherwise).
 *
 * Limits and behaviour:
 *   - The array holds FKT_NOALLOC_SCRATCH_BYTES (48 MiB) and is part of the library image:
 *     every GPU that loads libfkt.so holds it until the process exits.  A call with one
 *     right-hand side needs 4 * (6 N + nterms * (nodes + s2m chunks)) bytes, about 35 MB at
 *     N = 1M, d = 3, p = 6, leaf 256 (each part rounded up to 256 bytes); more right-hand
 *     sides need proportionally more, and passes of 17-32 right-hand sides on the TF32 near
 *     kernel also need the pass's near-field image, about 272 bytes per point.  Requests that
 *     do not fit return FKT_ERR_SCRATCH_LIMIT and enqueue nothing.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current; make that first call before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents.  Nothing in it
 *     needs to start at zero: every value a call reads was written earlier in the same call.
 *     Calls whose GPU work overlaps (two streams, two plans, two host threads) race on the
 *     array and give wrong results; order them on one stream or synchronise between them.
 *   - Asynchronous on the plan's stream, like fkt_mvm. */
#define FKT_NOALLOC_SCRATCH_BYTES (48u << 20)
int fkt_mvm_noalloc(fkt_plan_t plan, const float* w, float* y, int nrhs);

/* Measurement helper (not part of the method): lane-operation throughput of one arithmetic pipe
 * on the current device -- op 0 FP32 FMA, 1 MUFU ex2.approx, 2 MUFU rsqrt.approx, 3 MUFU
 * sqrt.approx, 4 MUFU rcp.approx, 5 packed FP32x2 FMA (two lane-ops per instruction) -- from a
 * grid of 8 x 256-thread CTAs per SM running 8 independent chains of iters operations per thread,
 * timed with CUDA events.  It is the denominator of the near and far kernels' ALU rooflines.
 * 1 <= iters <= 2^32.  Synchronizes the device. */
int fkt_probe_pipe_rate(int op, int64_t iters, double* lane_ops_per_second);

/* Failure detection: synchronise the plan's stream, then report FKT_ERR_TIMEOUT if any
 * bounded device-side wait of this plan's kernels ran out since the last check (the kernel
 * recorded it and stopped instead of hanging; results of that call are invalid), or
 * FKT_ERR_CUDA for a pending CUDA error.  Clears the record.  FKT_OK otherwise. */
int fkt_check(fkt_plan_t plan);

/* Release the plan and all device memory it owns.  NULL is ignored. */
void fkt_destroy(fkt_plan_t plan);

/* Static string for a status code. */
const char* fkt_error_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* FKT_H */
