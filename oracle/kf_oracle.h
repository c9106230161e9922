/*
 * kf_oracle.h -- plain FP64 CPU oracle for the hierarchical factorization and
 * solve of lambda*I + K (Yu, March, Biros, "An N log N Parallel Fast Direct
 * Solver for Kernel Matrices", arXiv 1701.02324).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header, table
 * or helper with the CUDA library.
 *
 * All matrices are row-major FP64.  Point indices of the tree are "tree
 * positions" (0..N-1 after the ball-tree permutation) unless stated otherwise.
 * Tree nodes use heap numbering: root = 1, children of a are 2a and 2a+1, the
 * nodes of level l are 2^l .. 2^(l+1)-1.
 */
#ifndef KF_ORACLE_H
#define KF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kfo kfo;

/* status values */
#define KFO_OK 0
#define KFO_EINVAL 1
#define KFO_EILLCOND 4

/* Ball tree (Sec. II-A "Partitioning the matrix").  X is N x d in ORIGINAL
 * order; the oracle copies it.  Returns NULL on bad arguments. */
kfo* kfo_create(const double* X, int64_t N, int32_t d, int32_t m);
void kfo_free(kfo* o);
int32_t kfo_depth(const kfo* o);
/* perm[i] = original index of the point at tree position i. */
void kfo_perm(const kfo* o, int64_t* perm);
void kfo_node_range(const kfo* o, int32_t node, int64_t* lo, int64_t* hi);

/* Sampled rows S' of a non-root node (reading of Sec. II-A, sampling of S). */
int32_t kfo_sample(const kfo* o, int32_t node, int32_t n_samp, uint64_t seed, int64_t* out);

/* Near-field sampling (reading of the ASKIT sampling the paper uses, Sec.
 * II-A and the parameter kappa of Sec. IV).  kfo_knn: for every tree position
 * the kappa nearest positions found by ntrees randomized projection trees with
 * leaves of at most `leaf` points (FP32 squared distances of the FP32-rounded
 * coordinates; -1 pads a short list); nbr: N x kappa.  kfo_set_near: node
 * lists of at most near_cap positions built from nbr; from then on
 * kfo_sample (and the skeletonizations) take the first min(list length,
 * floor(n_s / 2)) of the node's list and draw the rest uniformly.  nbr = NULL
 * turns it off.  kfo_node_near: the node's list and counts; returns its length. */
int32_t kfo_knn(const kfo* o, int32_t kappa, int32_t ntrees, int32_t leaf, uint64_t seed, int64_t* nbr);
int32_t kfo_set_near(kfo* o, const int64_t* nbr, int32_t kappa, int32_t near_cap);
int32_t kfo_node_near(const kfo* o, int32_t a, int64_t* pos, int32_t* cnt);

/* Skeletonization, Algorithm 1 with the ID of Eq. (e:id).  n_samp = |S'| cap. */
int32_t kfo_skeletonize(kfo* o, double h, double tau, int32_t s_max, int32_t n_samp, uint64_t seed);
int32_t kfo_rank(const kfo* o, int32_t node);
int32_t kfo_ncols(const kfo* o, int32_t node);         /* columns of the node's ID */
void kfo_skel(const kfo* o, int32_t node, int64_t* out); /* s tree positions, pivot order */
void kfo_P(const kfo* o, int32_t node, double* out);     /* s x ncols interpolation */
/* Replace the ID of one node (for tests that hold skeletons fixed).  The
 * caller must set children before parents, since ncols of a parent follows
 * the children's ranks. */
int32_t kfo_set_id(kfo* o, int32_t node, int32_t s, const int64_t* skel, const double* P);
/* The telescoped P_{alpha, alpha~} of Eq. (e:innerid): |alpha| x s. */
void kfo_P_full(const kfo* o, int32_t node, double* out);

/* Factorization, Algorithm 2.  variant 0 = telescoping (Eq. e:invtelescope),
 * variant 1 = the log^2 N predecessor (full recursive solve for P^). */
int32_t kfo_factorize(kfo* o, double lambda, int32_t variant);
void kfo_Phat(const kfo* o, int32_t node, double* out); /* |alpha| x s */
void kfo_Z(const kfo* o, int32_t node, double* out);    /* (s_l+s_r)^2, before LU */
/* The literal form u - W Z^-1 V u (u = W P_c) and the push-through form
 * W Z^-1 P_c of P^_alpha, for the identity check (|alpha| x s each). */
int32_t kfo_Phat_forms(const kfo* o, int32_t node, double* literal, double* pushed);

/* Solve, Algorithm 3 (transpose = 0) or its transpose sweep (transpose = 1).
 * b and x are N-vectors in ORIGINAL order. */
int32_t kfo_solve(const kfo* o, const double* b, double* x, int32_t transpose);
/* y = (lambda I + K~) x (deriv = 0) or y = (dK~/dh) x with P held fixed
 * (deriv = 1); ORIGINAL order. */
int32_t kfo_matvec(const kfo* o, const double* x, double* y, int32_t deriv);
/* Gradient of L through x = (lambda I + K~)^-1 b: given x and g = dL/dx,
 * returns dL/db (N), dL/dlambda and dL/dh. */
int32_t kfo_grad(const kfo* o, const double* x, const double* g, double* dLdb, double* dLdlambda, double* dLdh);

/* Algorithms 1 and 2 restricted to the disjoint subtrees under the given
 * roots: each of their nodes gets the skeleton, P, Z and P^ that
 * kfo_skeletonize + kfo_factorize would give it; other nodes are untouched
 * (their accessors then return nothing meaningful).  For checks of sampled
 * nodes at sizes where the whole tree takes too long.  KFO_EINVAL when a
 * root is out of range or lies inside another root's subtree. */
int32_t kfo_subtrees(kfo* o, const int32_t* roots, int32_t nroots, double h, double tau, int32_t s_max,
                     int32_t n_samp, uint64_t seed, double lambda);

/* Hybrid level-restricted solver (Sec. II-C, Algorithms 6-8): the subtrees
 * of the 2^L frontier nodes of level L (1 <= L <= D) are skeletonized and
 * factorized (the frontier nodes' IDs included); above them nothing is
 * compressed, and the reduced system I + VW of the frontier skeletons is
 * formed and factored with LU.  Replaces any earlier skeletons or factors of
 * those subtrees.  KFO_EILLCOND when a pivot is tiny. */
int32_t kfo_hybrid(kfo* o, int32_t L, double h, double tau, int32_t s_max, int32_t n_samp, uint64_t seed,
                   double lambda);
/* x = (D + U V)^-1 b (Algorithm 6) and y = (D + U V) x, ORIGINAL order. */
int32_t kfo_hybrid_solve(const kfo* o, const double* b, double* x);
int32_t kfo_hybrid_matvec(const kfo* o, const double* x, double* y);

/* splitmix64 output function (used by the sampler); exposed for its pin. */
uint64_t kfo_splitmix64(uint64_t x);

#ifdef __cplusplus
}
#endif
#endif
