/*
 * kf.h -- C ABI of the GB300 hierarchical kernel-matrix solver.
 *
 * Method: Yu, March, Biros, "An N log N Parallel Fast Direct Solver for Kernel
 * Matrices" (arXiv 1701.02324).  Given N points x_i in R^d, the Gaussian kernel
 * K_ij = exp(-||x_i - x_j||^2 / (2 h^2)) (Eq. e:gaussian) and lambda >= 0, the
 * library builds the ball tree and interpolative-decomposition skeletons of
 * Sec. II-A (Algorithm 1), factorizes the hierarchical approximation
 * lambda I + K~ level by level with the Sherman-Morrison-Woodbury formula
 * (Eqs. e:smw, e:hodlr, e:blocksmw, e:invtelescope; Algorithm 2), and applies
 * its inverse (Algorithm 3), its transpose, the operator itself and the
 * gradient of a loss through the solve.
 *
 * Conventions shared by every entry point:
 *  - Status: every function returns kf_status; nothing aborts.  A message for
 *    the last failure of a context is available from kf_last_error().
 *  - Pointers: "device or host" arguments may point to device memory or to
 *    ordinary/pinned host memory; the library looks the pointer up with
 *    cudaPointerGetAttributes and stages host data through device buffers.
 *    The caller keeps ownership of everything it passes in.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Work is enqueued on that stream.  Calls whose outputs
 *    land in host memory synchronize the stream before returning.
 *  - Point order: X rows, right-hand sides and solutions are in the caller's
 *    ORIGINAL point order; the tree permutation is internal.
 *  - Matrices of right-hand sides are column-major: column j of B starts at
 *    B + j*ld (elements), ld >= N.
 *  - Sizes: N < 2^31, 1 <= d <= 1024, 1 <= m, 1 <= s_max <= 512.
 *  - Handles own the device memory they allocate, drawn through the
 *    allocator given to kf_create (cudaMallocAsync/cudaFreeAsync on the call's
 *    stream when NULL).  A factor
 *    keeps a pointer to its tree: free factors before their tree.  *_free(NULL)
 *    is a no-op.
 *  - Device-side errors (ill-conditioned pivots, bounded waits that ran out)
 *    are written to a device status word and returned by the next call that
 *    synchronizes (kf_factor_status, kf_solve with info, *_free) or at once
 *    when kf_opts.sync_errors is set.
 */
#ifndef KF_H
#define KF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KF_OK = 0,
  KF_EINVAL = 1,        /* bad argument (NaN/Inf input, h <= 0, lambda < 0, sizes) */
  KF_ENOMEM = 2,        /* the allocator returned NULL */
  KF_ECUDA = 3,         /* a CUDA runtime call failed */
  KF_EILLCOND = 4,      /* a leaf block or reduced system Z is numerically singular
                           (Sec. III "Stability": detectable instability) */
  KF_ENOTCONV = 5,      /* refinement did not reach the requested residual */
  KF_ETIMEOUT = 6,      /* a bounded device-side wait ran out */
  KF_EUNSUPPORTED = 7   /* valid request the library does not support */
} kf_status;

typedef enum { KF_F32 = 0, KF_F64 = 1 } kf_dtype;

typedef enum {
  KF_PREC_FP64 = 0,     /* every step in FP64 */
  KF_PREC_MIXED = 1     /* FP32 factors, tensor-core contractions, FP64 pivoted QR,
                           FP64 reduced-system LU and FP64 refinement residual */
} kf_precision;

typedef enum {
  KF_V_STORED = 0,      /* keep the skeleton rows K_{b~ a} of every level for the solve */
  KF_V_RECOMPUTE = 1    /* evaluate them on the fly in the solve (matrix-free, Sec. II-D) */
} kf_vstorage;

/* Device memory allocator.  alloc returns a device pointer of at least `bytes`
 * bytes usable on `stream` (or NULL on failure); free releases it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, size_t bytes, void* stream, void* user);
  void* user;
} kf_alloc;

/* Options of kf_factorize.  Zero-initialise, then set fields; n_samp = 0 means
 * 2*s_max, seed = 0 means 0x1701. */
typedef struct {
  int32_t precision;      /* kf_precision */
  int32_t n_samp;         /* |S'|: sampled rows per ID (Sec. II-A), capped by N - |node| */
  uint64_t seed;          /* sampler seed */
  int32_t v_storage;      /* kf_vstorage */
  int32_t sync_errors;    /* nonzero: synchronize and report device status at once */
  double refine_tol;      /* target relative residual (0 = 1e-10) */
  int32_t refine_max_iter;/* max refinement iterations (0 = 100, mixed path only; > 0 also turns
                             refinement on for the FP64 path; -1 = no refinement) */
  int32_t no_tensor_cores;/* mixed path: 1 = CUDA-core FP32 products instead of tcgen05 3xTF32 */
  int32_t fp64_operator;  /* keep FP64 V blocks and leaf blocks so that the refinement residual and
                             kf_matvec use an FP64-accurate operator: 0 = default (on for the mixed
                             path), 1 = on, -1 = off */
  int32_t gmres_restart;  /* refinement method: 0 = GMRES(50), m > 0 = GMRES(m) (m <= 64) in FP64,
                             right-preconditioned by the factorization; -1 = x += M^-1 r */
  int32_t no_cluster_kernels; /* 1 = one CTA per node everywhere (no thread-block clusters for the
                             pivoted QR and reduced-system LU of the upper tree levels) */
  int32_t tc_tile_n;      /* mixed path: tile width of the tcgen05 products, 128 or 256 (0 = 256) */
  int32_t zinv_max_nodes; /* tree levels with at most this many nodes keep the explicit inverse of
                             their reduced systems Z for the solve sweep (a product spread over many
                             CTAs instead of a latency-bound LU solve per node), computed after each
                             level's LU at 2 z^3 FP64 flops a node: 0 = default (64; in
                             kf_factorize_batched none for factors whose solves are not refined,
                             whose single sweep the concurrent problems hide), -1 = none */
  int32_t hybrid_level;   /* 0 = the direct solver (Algorithm 2 up to the root).  L >= 1: the hybrid
                             level-restricted solver of Sec. II-C (Algorithms 6-8) with its frontier
                             at level L (1 <= L <= depth): the subtrees of the 2^L nodes of level L
                             are skeletonized and factorized (the frontier nodes' own IDs included),
                             nothing above them is compressed, and the reduced system I + VW of the
                             frontier skeletons, (VW)[a~, b~] = K_{a~ b} P^_b for frontier nodes
                             a != b, is formed in FP64 and LU-factored (2^L s_max <= 1024, else
                             KF_EUNSUPPORTED).  kf_solve (transpose = 0) and kf_matvec then apply
                             (D + UV)^-1 and D + UV, D = blockdiag(lambda I + K~_aa); transpose
                             solves and kf_grad return KF_EUNSUPPORTED.  kf_factorize only. */
  int32_t knn_kappa;      /* near-field sampling of S' (the ASKIT sampling the paper uses, Sec. II-A,
                             with kappa neighbours, Sec. IV): 0 = uniform sampling (default); kappa in
                             1..32: every point's kappa nearest points are found by knn_trees
                             randomized projection trees with leaves of at most knn_leaf points
                             (FP32 squared distances of the FP32 coordinates, sequential fused
                             multiply-adds, ties to the smaller tree position); every node lists the
                             positions outside it that its points' lists name most often (a parent
                             adds its children's lists), keeps n_samp / 2 of them, and S' takes the
                             first min(list length, floor(n_s / 2)) of those and draws the rest
                             uniformly.  Needs leaf size x kappa <= 16384 (else KF_EUNSUPPORTED). */
  int32_t knn_trees;      /* projection trees of the neighbour search (0 = 4) */
  int32_t knn_leaf;       /* their leaf size, 2..1024 (0 = 512) */
  int32_t zoff_fused;     /* mixed path with tcgen05 products: 0 = the Z off-diagonal blocks K_{l~ r} P^_r
                             read the stored V blocks (default); 1 = they evaluate their kernel entries
                             inside the product (kernel summation fused with the weights, Sec. II-D):
                             FP32 squared distances of the FP32 coordinates and a fast exponential,
                             so the entries carry ~1e-6 relative error instead of FP32 rounding, and
                             the reduced systems no longer wait for the V blocks */
  int32_t w_recompute;    /* 1 = memory-lean W (Sec. III, storage): P^ is kept for the leaves only, with
                             T = Z^-1 P_c of every node (z x s each); the solve applies P^ of a level
                             as P^_leaf times the telescoped T's (Eq. e:invtelescope), pushed down
                             the tree, and the transpose sweep gathers up the same way.  Storage of P^
                             falls from D N s_max to 3 N s_max values (two levels alternate during the
                             factorization).  Not with the hybrid solver (KF_EUNSUPPORTED);
                             kf_factor_Phat then returns the leaves' P^ only.  With
                             v_storage = KF_V_RECOMPUTE the factorization also keeps only three
                             levels of V blocks, used in turn. */
  int32_t tc_operator;    /* mixed path with fp64_operator: 1 = also keep the V blocks, the leaf blocks,
                             the leaves' P and every P_c as exact BF16 integer digits (7 per entry,
                             14 bytes; Ozaki splitting; P and P_c with rows scaled by powers of two),
                             so that the FP64-accurate operator over 16 to 4096 right-hand sides
                             (its leaf blocks, V pass of Eq. e:blocksmw, pushes through P_c and the
                             leaves' P update) runs as tcgen05 products with exact FP32 accumulation
                             (about 2^-49 of the column's scale per product, against the
                             double-float kernels' 2^-46 of each product); refined solves of such
                             blocks use it.  0 = double-float CUDA-core passes only (default) */
} kf_opts;

/* Filled by kf_solve when non-NULL (synchronizes the stream). */
typedef struct {
  double eps_r;           /* ||b - (lambda I + K~) x|| / ||b|| (Eq. e:errors), max over RHS;
                             -1 when not computed (FP64 path without refinement) */
  int32_t iters;          /* refinement steps taken */
  int32_t status;         /* device status at the end of the solve */
} kf_solve_info;

typedef struct kf_ctx kf_ctx;
typedef struct kf_tree kf_tree;
typedef struct kf_factor kf_factor;

/* Context: allocator and error message.  alloc may be NULL. */
kf_status kf_create(kf_ctx** out, const kf_alloc* alloc);
kf_status kf_destroy(kf_ctx* ctx);
const char* kf_status_string(kf_status s);
const char* kf_last_error(const kf_ctx* ctx);

/* Ball tree of Sec. II-A "Partitioning the matrix".  X: N x d row-major,
 * original order, device or host, dtype KF_F32 or KF_F64.  Depth
 * D = ceil(log2(N/m)); each node splits into floor(n/2) and ceil(n/2) points by
 * the order of (projection on the farthest-pair direction, original index).
 * The tree copies and permutes X; the caller keeps X.  Errors: KF_EINVAL for
 * non-finite coordinates or bad sizes. */
kf_status kf_tree_build(kf_ctx* ctx, const void* X, int32_t dtype, int64_t N, int32_t d, int32_t m,
                        void* stream, kf_tree** out);
/* perm[i] = original index of the point at tree position i (device or host, N int64). */
kf_status kf_tree_perm(const kf_tree* t, int64_t* perm, void* stream);
/* Sizes of the tree; any output pointer may be NULL. */
kf_status kf_tree_info(const kf_tree* t, int64_t* N, int32_t* d, int32_t* m, int32_t* depth);
kf_status kf_tree_free(kf_tree* t);

/* Skeletonize (Algorithm 1, ID of Eq. e:id with sampled rows S') and factorize
 * (Algorithm 2) lambda I + K~.  h > 0, lambda >= 0, tau >= 0 (rank rule
 * sigma_{s+1}/sigma_1 < tau estimated by |R_kk|/|R_00| of a pivoted QR),
 * 1 <= s_max <= 512.  opts may be NULL (FP64, |S'| = 2 s_max, seed 0x1701,
 * stored V).  Errors: KF_EINVAL, KF_ENOMEM, KF_EILLCOND (also later, see the
 * device status convention above). */
kf_status kf_factorize(kf_tree* t, double h, double lambda, double tau, int32_t s_max,
                       const kf_opts* opts, void* stream, kf_factor** out);
/* Device status word of the factorization (synchronizes the stream). */
kf_status kf_factor_status(kf_factor* f, void* stream);
kf_status kf_factor_free(kf_factor* f);

/* X = (lambda I + K~)^-1 B (transpose = 0, Algorithm 3) or
 * X = (lambda I + K~)^-T B (transpose = 1).  B, X: N x nrhs column-major with
 * leading dimension ld, device or host, dtype KF_F32 or KF_F64; B and X may
 * alias.  When refinement is on (mixed path by default, refine_max_iter > 0)
 * the solve is refined against the hierarchical operator, with FP64
 * accumulation, until the relative residual (Eq. e:errors) is below
 * opts.refine_tol: by x += M^-1 r or by GMRES(m) (opts.gmres_restart; the
 * columns of B run their own GMRES iterations in lockstep, sharing every
 * sweep and operator launch), M being
 * the factorization.  A transpose solve is refined the same way against the
 * transposed operator, M^-T being the transpose sweep.  The operator is
 * FP64-accurate when opts.fp64_operator is set (or on the FP64 path);
 * otherwise the mixed path evaluates it in FP32.  KF_ENOTCONV when the
 * refinement stops above refine_tol (X is then left unwritten). */
kf_status kf_solve(kf_factor* f, const void* B, void* X, int64_t nrhs, int64_t ld, int32_t dtype,
                   int32_t transpose, void* stream, kf_solve_info* info);
/* Y = (lambda I + K~) X with the operator the factorization inverts
 * (second form of Eq. e:uv): leaf blocks lambda I + K_aa, off-diagonal blocks
 * P_{l l~} K_{l~ r} and P_{r r~} K_{r~ l}.  Layout as kf_solve.  With
 * opts.tc_operator and 16 <= nrhs <= 4096 the call holds the BF16 digits of X
 * (14 bytes per entry) for its duration; KF_ENOMEM when they do not fit
 * (Y then unspecified; a smaller block of columns fits). */
kf_status kf_matvec(kf_factor* f, const void* X, void* Y, int64_t nrhs, int64_t ld, int32_t dtype, void* stream);
/* Gradient of a loss L through x = (lambda I + K~)^-1 b given x and dL/dx:
 * a = (lambda I + K~)^-T dL/dx; dL/db = a; dL/dlambda = -sum a.x;
 * dL/dh = -sum a.(dK~/dh) x with skeletons and P held fixed.  The adjoint
 * solve for a is refined like kf_solve(transpose = 1) whenever the factor's
 * solves are refined (mixed path by default); dK~/dh is evaluated from the FP64
 * coordinates on both paths.  x, dLdx, dLdb: N x nrhs (ld), device or host,
 * FP64.  dLdlambda, dLdh: host, one value summed over the RHS columns.  Not in
 * the paper: the adjoint of Algorithm 3 through the factorization of
 * Eq. (e:smw). */
kf_status kf_grad(kf_factor* f, const void* x, const void* dLdx, void* dLdb, double* dLdlambda,
                  double* dLdh, int64_t nrhs, int64_t ld, void* stream);

/* ---- many independent problems ------------------------------------------------ */
/* Skeletonize and factorize nprob independent problems (one tree each, uneven
 * N and ranks) with ONE CUDA-graph launch: the factors are allocated first,
 * then every problem's kernel sequence is captured into one graph whose
 * branches run concurrently on up to 16 streams, and the graph is launched
 * once on `stream` (no counterpart in the paper, which solves one problem at
 * a time; Algorithms 1-2 per problem).  h, lambda, tau: host arrays of nprob
 * values; s_max and opts are shared (opts.zinv_max_nodes = 0 means no explicit
 * Z^-1 here unless the factors' solves are refined).  out: host array of nprob factor handles (NULL on failure).
 * Synchronizes `stream`; returns the worst per-problem status (KF_EILLCOND
 * leaves the factors in place).  Scratch memory inside the graph comes from
 * cudaMallocAsync even when the context has an allocator. */
kf_status kf_factorize_batched(kf_tree* const* trees, int32_t nprob, const double* h, const double* lambda,
                               const double* tau, int32_t s_max, const kf_opts* opts, void* stream, kf_factor** out);
/* X_i = (lambda_i I + K~_i)^-1 B_i for nprob factors: the direct sweeps of
 * every problem in one CUDA-graph launch (Algorithm 3 per problem).  When the
 * factors refine (the mixed path by default, see kf_solve), the batch is then
 * refined as a whole: each step is one graph launch for the residuals
 * b - (lambda I + K~) x of every unconverged problem (FP64-accurate operator)
 * and one for x += M^-1 r, with one host synchronization per step to read the
 * residual norms; a problem leaves the batch once its relative residual
 * (Eq. e:errors, max over its columns) is at most its refine_tol, and a problem
 * whose residual falls by less than half in a step finishes with GMRES(m) on
 * its columns, as kf_solve does.  B, X: host arrays of DEVICE pointers; nrhs, ld:
 * host arrays.  info: NULL or a host array of nprob records (eps_r: the final
 * relative residual, max over the problem's columns, -1 when the problem was
 * not refined; iters: refinement steps plus GMRES iterations, max over
 * columns; status: KF_OK or KF_ENOTCONV for that problem).  Synchronizes
 * `stream`.  KF_ENOTCONV when a problem ends above its refine_tol (X is
 * written all the same). */
kf_status kf_solve_batched(kf_factor* const* f, int32_t nprob, const void* const* B, void* const* X,
                           const int64_t* nrhs, const int64_t* ld, int32_t dtype, void* stream,
                           kf_solve_info* info);

/* ---- inspection (host outputs; they synchronize the stream) -------------- */
/* Heap-numbered nodes: root 1, children 2a and 2a+1, level l holds nodes
 * 2^l .. 2^(l+1)-1.  Ranks of nodes 0..2^(D+1)-1 (entry 0 and the root are 0). */
kf_status kf_factor_ranks(const kf_factor* f, int32_t* ranks, void* stream);
/* Stability diagnostic (Sec. III "Stability": the instability is detectable):
 * for every node, the smallest pivot over the largest of its factorization --
 * squared Cholesky pivots over the largest diagonal entry at a leaf, |u_jj|
 * of the LU of Z at an internal node.  ratios: host, 2^(D+1) entries (entry 0
 * unused). */
kf_status kf_factor_pivot_ratios(const kf_factor* f, double* ratios, void* stream);
/* Skeleton of a non-root node: s tree positions in pivot order. */
kf_status kf_factor_skeleton(const kf_factor* f, int32_t node, int64_t* skel, void* stream);
/* Interpolation matrix of a non-root node's ID, s x c row-major FP64, with
 * c = |node| (leaf) or s_l + s_r (internal). */
kf_status kf_factor_P(const kf_factor* f, int32_t node, double* P, void* stream);
/* P^_node = K~_node^-1 P_{node node~}, |node| x s row-major FP64. */
kf_status kf_factor_Phat(const kf_factor* f, int32_t node, double* Phat, void* stream);

/* Near-field sampling (kf_opts.knn_kappa > 0): every point's neighbour list,
 * nbr: host, N x kappa int32 tree positions (-1 pads a short list); and the
 * list of a non-root node: pos and cnt host arrays of n_samp / 2 entries, the
 * first *len of them used, positions by decreasing count.  KF_EINVAL when
 * near-field sampling is off. */
kf_status kf_factor_knn(const kf_factor* f, int32_t* nbr, void* stream);
kf_status kf_factor_near(const kf_factor* f, int32_t node, int32_t* pos, int32_t* cnt, int32_t* len, void* stream);

/* Test hook: factorize with skeletons and interpolation matrices supplied by
 * the caller instead of computing them, so that the factorization can be
 * compared with a reference that used the same IDs.  ranks: host int32
 * [2^(D+1)]; skel: host int64, node a's list at skel + a*s_max; P: host FP64,
 * node a's s x c matrix at P + a*s_max*cmax with cmax = max(max leaf size,
 * 2*s_max).  Otherwise as kf_factorize. */
kf_status kf_factorize_with_ids(kf_tree* t, double h, double lambda, int32_t s_max, const int32_t* ranks,
                                const int64_t* skel, const double* P, const kf_opts* opts, void* stream,
                                kf_factor** out);

/* ---- allocation-free variant ------------------------------------------------------ */
/* Ball-tree permutation (the same tree as kf_tree_build) computed without
 * allocating any device memory.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate, for example code that runs
 * inside a device-memory allocator's own callback (re-entering the allocator
 * would deadlock or recurse), latency-bound loops in which cudaMalloc would
 * synchronize the device, or processes whose device memory is entirely
 * reserved by another framework's pool, where a cudaMalloc fails.
 *
 * X:    device, N x d FP64 row-major, original order (read only).
 * Xt:   device output, N x d FP64, the points in tree order.
 * perm: device output, N int64, perm[i] = original index of tree position i.
 * Limits: 1 <= N <= 65536, 1 <= d <= 1024 (as kf_tree_build), N * d <= 2^19,
 * m >= 1; larger sizes are rejected with KF_EINVAL and a message in
 * kf_last_error(NULL); a current device index above 63 gives KF_EUNSUPPORTED.
 * X is checked for non-finite coordinates before anything is written: on
 * that KF_EINVAL, Xt and perm are left untouched.
 * Scratch: one 12 MiB file-scope device array that every GPU loading the
 * library holds until the process exits.  Every call shares it and it keeps
 * the previous call's contents (the call initializes what it reads), so calls
 * whose GPU work overlaps (different streams, devices used concurrently from
 * several threads) race and must be serialized by the caller.  The first call
 * on each device looks up the array's device address on the current device;
 * make that first call before any stream capture.  The call synchronizes
 * `stream` once to read the finiteness check of X. */
kf_status kf_tree_perm_noalloc(const double* X, int64_t N, int32_t d, int32_t m, double* Xt, int64_t* perm,
                               void* stream);

/* Kernel-variant autotuner (no counterpart in the paper; an implementation
 * knob).  Factorizes the given problem once per candidate and keeps the
 * fastest: one CTA per node or thread-block clusters for the upper tree levels
 * (no_cluster_kernels), and on the mixed path CUDA-core or tcgen05 products
 * (no_tensor_cores) with tcgen05 tiles of 256 or 128 columns (tc_tile_n).
 * After one untimed factorization with `base`, each candidate is timed with
 * CUDA events on `stream` (two factorizations, the faster counts).  `best`
 * receives `base` with the fastest choice; ms (nullable, KF_AUTOTUNE_MAX
 * entries) the candidates' times in milliseconds in the order above, and
 * *ncand (nullable) their number.  The choice changes no result beyond
 * rounding (the skeletons come from the same FP64 QR).  Synchronizes
 * `stream`.  Errors: those of kf_factorize. */
#define KF_AUTOTUNE_MAX 8
kf_status kf_autotune(kf_tree* t, double h, double lambda, double tau, int32_t s_max, const kf_opts* base,
                      void* stream, kf_opts* best, float* ms, int32_t* ncand);

/* Test hook of the device-side time-out path (no counterpart in the paper).
 * polls > 0: every CTA of the tensor-core products of the mixed path (the Z
 * off-diagonal blocks and the telescoping) first polls an mbarrier that
 * nothing arrives at, at most `polls` times, and then takes the path of a
 * bounded wait that ran out: it flags KF_ETIMEOUT in the factor's device
 * status word, skips its product, frees its tensor memory and returns, so the
 * context stays usable.  polls = 0 (the default) turns the probe off.
 * Process-wide for the current device; synchronous.  KF_EINVAL for polls < 0. */
kf_status kf_test_tc_wait_probe(int64_t polls);

/* ---- diagnostics ------------------------------------------------------------- */
/* Number of kernel launches this process has made through the library. */
int64_t kf_launch_count(void);
/* Per-phase timing: while on, every launch is bracketed by CUDA events on its
 * stream (adds two event records per launch).  Process-wide. */
kf_status kf_profile_enable(int32_t on);
/* Totals since the last read: ms[i] and launches[i] for phase i, nphase >=
 * KF_PHASE_COUNT.  Synchronizes the recorded events.  Phases, in order: tree,
 * sample, eval_A, qr, leaf_assemble, leaf_cholesky, leaf_phat, eval_V, zoff,
 * z_lu, z_solve_pc, telescope, solve_leaf, solve_colsum, solve_zsolve,
 * solve_rowupd, matvec_leaf, matvec_push, misc, qr_cluster (the pivoted QR of
 * the upper levels on thread-block clusters and its R11^-1 R12 step), qr_leaf
 * (the pivoted QR of the leaf level; "qr" holds the other one-CTA-per-node
 * levels), matvec_colsum and matvec_rowupd (the V-block passes of kf_matvec
 * and of the refinement's operator; solve_colsum and solve_rowupd are those of
 * the solve sweep), z_inv (the explicit Z^-1 of the upper levels, see
 * kf_opts.zinv_max_nodes), hybrid (the reduced system of the hybrid solver:
 * its coupling blocks, LU and products, kf_opts.hybrid_level), near (the
 * neighbour lists of near-field sampling, kf_opts.knn_kappa). */
#define KF_PHASE_COUNT 26
kf_status kf_profile_read(double* ms, int64_t* launches, int32_t nphase);
/* Per-launch timeline of the launches recorded since the last kf_profile_read
 * (which it leaves in place): for launch q < *n, its start and end in ms
 * relative to the start of the first recorded launch, its phase and the
 * index of its stream in order of first appearance.  Host arrays of cap
 * entries; *n receives the number of records (entries past cap are not
 * written).  Synchronizes the recorded events.  KF_EINVAL on a null pointer
 * or a negative cap. */
kf_status kf_profile_timeline(double* t0_ms, double* t1_ms, int32_t* phase, int32_t* stream, int64_t cap,
                              int64_t* n);

#ifdef __cplusplus
}
#endif
#endif /* KF_H */
