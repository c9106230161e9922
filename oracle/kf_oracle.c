/*
 * kf_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Restates the method of arXiv 1701.02324 step by step, in the paper's order:
 * ball tree (Sec. II-A), interpolative decomposition skeletons (Eq. e:id,
 * Algorithm 1), the N log N factorization (Eqs. e:hodlr, e:blocksmw,
 * e:innerid, e:invtelescope, Algorithm 2), the direct solve (Algorithm 3),
 * the O(N log^2 N) predecessor factorization for comparison, the
 * hierarchical matvec with lambda*I + K~, its transpose solve and the
 * gradient with respect to b, lambda and h.
 *
 * Compiled with -ffp-contract=off: every a*b+c below is two roundings unless
 * written as fma().  No blocking, fusion or reordering beyond the formulas.
 * OpenMP is used only to run independent tree nodes at the same time; each
 * node's arithmetic is the same sequential loop either way.
 *
 * Readings of points the paper leaves open are marked READING.
 */
#include "kf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t s;      /* rank s_alpha */
  int32_t c;      /* columns of the ID: |alpha| (leaf) or s_l + s_r */
  int64_t* skel;  /* s tree positions, pivot order */
  double* P;      /* s x c */
  double* Pfull;  /* |alpha| x s, Eq. e:innerid */
  /* factorization */
  double* LU;     /* leaf: |alpha|^2 LU of lambda I + K_aa */
  int64_t* piv;   /* leaf row pivots */
  double* Phat;   /* |alpha| x s */
  double* Vl;     /* internal: K_{l~ r}, s_l x |r| */
  double* Vr;     /* internal: K_{r~ l}, s_r x |l| */
  double* Z;      /* internal: Z before LU */
  double* ZLU;    /* internal: LU of Z */
  int64_t* Zpiv;
} node_t;

struct kfo {
  int64_t N;
  int32_t d, m, D;
  int32_t nnodes; /* 2^(D+1) - 1 */
  double* X;      /* N x d, tree order */
  int64_t* perm;  /* tree position -> original index */
  int64_t* lo;    /* indexed by heap id */
  int64_t* hi;
  double h, c_exp, lambda;
  int32_t skeletonized, factorized, variant;
  /* hybrid level-restricted solver (kfo_hybrid): frontier level, offsets of
   * the frontier skeleton blocks, LU of the reduced system I + VW */
  int32_t hyb_ready, hyb_L;
  int64_t* hyb_off;
  double* hyb_lu;
  int64_t* hyb_piv;
  int32_t illcond;
  node_t* nd;     /* indexed by heap id */
  /* near-field sampling (kfo_set_near): per node, at most near_cap neighbour
   * positions outside the node, by decreasing count (ties: smaller position),
   * with their counts; near_on = 0 means uniform sampling */
  int32_t near_on, near_cap;
  int64_t** near_pos;
  int32_t** near_cnt;
  int32_t* near_len;
};

static int is_leaf(const kfo* o, int32_t a) { return a >= (1 << o->D); }
static int64_t nsz(const kfo* o, int32_t a) { return o->hi[a] - o->lo[a]; }

/* Gaussian kernel, Eq. (e:gaussian): exp(-||x-y||^2 / (2 h^2)).  The squared
 * distance is a sequential sum over the coordinates; c_exp = -0.5/(h*h). */
static double kern(const kfo* o, int64_t i, int64_t j) {
  const double* x = o->X + i * o->d;
  const double* y = o->X + j * o->d;
  double d2 = 0.0;
  for (int32_t k = 0; k < o->d; ++k) {
    double t = x[k] - y[k];
    d2 = d2 + t * t;
  }
  return exp(d2 * o->c_exp);
}

/* dK/dh of the Gaussian kernel: K * ||x-y||^2 / h^3. */
static double dkern_dh(const kfo* o, int64_t i, int64_t j) {
  const double* x = o->X + i * o->d;
  const double* y = o->X + j * o->d;
  double d2 = 0.0;
  for (int32_t k = 0; k < o->d; ++k) {
    double t = x[k] - y[k];
    d2 = d2 + t * t;
  }
  double h3 = o->h * o->h * o->h;
  return exp(d2 * o->c_exp) * (d2 / h3);
}

/* ------------------------------------------------------------------------ */
/* Small dense helpers (plain loops).                                        */

/* C (n x k) = A (n x p) * B (p x k), all row-major. */
static void matmul(const double* A, const double* B, double* C, int64_t n, int64_t p, int64_t k) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < k; ++j) {
      double acc = 0.0;
      for (int64_t t = 0; t < p; ++t) acc = acc + A[i * p + t] * B[t * k + j];
      C[i * k + j] = acc;
    }
}

/* LU with partial pivoting (LAPACK GETRF semantics; ties in |pivot| go to the
 * lowest row).  Returns the smallest |u_kk| relative to max |a_ij|. */
static double lu_factor(double* A, int64_t* piv, int64_t n) {
  double amax = 0.0;
  for (int64_t i = 0; i < n * n; ++i) if (fabs(A[i]) > amax) amax = fabs(A[i]);
  double minpiv = INFINITY;
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = k;
    double best = fabs(A[k * n + k]);
    for (int64_t i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); p = i; }
    piv[k] = p;
    if (p != k)
      for (int64_t j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
    double ukk = A[k * n + k];
    if (fabs(ukk) < minpiv) minpiv = fabs(ukk);
    if (ukk == 0.0) continue;
    for (int64_t i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / ukk;
      A[i * n + k] = l;
      for (int64_t j = k + 1; j < n; ++j) A[i * n + j] = A[i * n + j] - l * A[k * n + j];
    }
  }
  return (n == 0 || amax == 0.0) ? 1.0 : minpiv / amax;
}

/* Solve A X = B (trans = 0) or A^T X = B (trans = 1) in place, B is n x k. */
static void lu_solve(const double* LU, const int64_t* piv, int64_t n, double* B, int64_t k, int trans) {
  if (!trans) {
    for (int64_t i = 0; i < n; ++i)
      if (piv[i] != i)
        for (int64_t j = 0; j < k; ++j) { double t = B[i * k + j]; B[i * k + j] = B[piv[i] * k + j]; B[piv[i] * k + j] = t; }
    for (int64_t i = 0; i < n; ++i)          /* L y = Pb, unit lower */
      for (int64_t t = 0; t < i; ++t)
        for (int64_t j = 0; j < k; ++j) B[i * k + j] = B[i * k + j] - LU[i * n + t] * B[t * k + j];
    for (int64_t i = n - 1; i >= 0; --i) {   /* U x = y */
      for (int64_t t = i + 1; t < n; ++t)
        for (int64_t j = 0; j < k; ++j) B[i * k + j] = B[i * k + j] - LU[i * n + t] * B[t * k + j];
      for (int64_t j = 0; j < k; ++j) B[i * k + j] = B[i * k + j] / LU[i * n + i];
    }
  } else {
    for (int64_t i = 0; i < n; ++i) {        /* U^T y = b */
      for (int64_t t = 0; t < i; ++t)
        for (int64_t j = 0; j < k; ++j) B[i * k + j] = B[i * k + j] - LU[t * n + i] * B[t * k + j];
      for (int64_t j = 0; j < k; ++j) B[i * k + j] = B[i * k + j] / LU[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i)     /* L^T z = y */
      for (int64_t t = i + 1; t < n; ++t)
        for (int64_t j = 0; j < k; ++j) B[i * k + j] = B[i * k + j] - LU[t * n + i] * B[t * k + j];
    for (int64_t i = n - 1; i >= 0; --i)     /* x = P^T z */
      if (piv[i] != i)
        for (int64_t j = 0; j < k; ++j) { double t = B[i * k + j]; B[i * k + j] = B[piv[i] * k + j]; B[piv[i] * k + j] = t; }
  }
}

/* ------------------------------------------------------------------------ */
/* Ball tree, Sec. II-A "Partitioning the matrix".
 * READING: the splitting hyperplane is not specified.  For the points of a
 * node: a = the point with the smallest original index; p = the point
 * farthest from a; q = the point farthest from p (ties: smallest original
 * index); every point is projected on q - p, proj_i = sum_k (x_ik - x_pk) *
 * (x_qk - x_pk); the points are ordered by (proj, original index) and the
 * left child takes the first floor(n/2).  Depth D = ceil(log2(N/m)) so that
 * the leaves sit at level D = log2(N/m) as the paper states. */

typedef struct { double key; int64_t orig; int64_t pos; } sortrec;

static int cmp_sortrec(const void* A, const void* B) {
  const sortrec* a = (const sortrec*)A;
  const sortrec* b = (const sortrec*)B;
  if (a->key < b->key) return -1;
  if (a->key > b->key) return 1;
  return (a->orig < b->orig) ? -1 : (a->orig > b->orig);
}

static double sqdist_rows(const double* x, const double* y, int32_t d) {
  double acc = 0.0;
  for (int32_t k = 0; k < d; ++k) { double t = x[k] - y[k]; acc = acc + t * t; }
  return acc;
}

static void split_node(kfo* o, int32_t a, int32_t level) {
  int64_t lo = o->lo[a], hi = o->hi[a], n = hi - lo;
  if (level == o->D) return;
  int32_t d = o->d;
  if (n >= 2) {
    int64_t ia = lo;
    for (int64_t i = lo + 1; i < hi; ++i) if (o->perm[i] < o->perm[ia]) ia = i;
    int64_t ip = lo; double best = -1.0;
    for (int64_t i = lo; i < hi; ++i) {
      double dd = sqdist_rows(o->X + i * d, o->X + ia * d, d);
      if (dd > best || (dd == best && o->perm[i] < o->perm[ip])) { best = dd; ip = i; }
    }
    int64_t iq = lo; best = -1.0;
    for (int64_t i = lo; i < hi; ++i) {
      double dd = sqdist_rows(o->X + i * d, o->X + ip * d, d);
      if (dd > best || (dd == best && o->perm[i] < o->perm[iq])) { best = dd; iq = i; }
    }
    sortrec* r = (sortrec*)malloc(sizeof(sortrec) * n);
    const double* xp = o->X + ip * d;
    const double* xq = o->X + iq * d;
    for (int64_t i = lo; i < hi; ++i) {
      const double* xi = o->X + i * d;
      double acc = 0.0;
      for (int32_t k = 0; k < d; ++k) acc = acc + (xi[k] - xp[k]) * (xq[k] - xp[k]);
      r[i - lo].key = acc; r[i - lo].orig = o->perm[i]; r[i - lo].pos = i;
    }
    qsort(r, n, sizeof(sortrec), cmp_sortrec);
    double* xs = (double*)malloc(sizeof(double) * n * d);
    for (int64_t i = 0; i < n; ++i) memcpy(xs + i * d, o->X + r[i].pos * d, sizeof(double) * d);
    memcpy(o->X + lo * d, xs, sizeof(double) * n * d);
    for (int64_t i = 0; i < n; ++i) o->perm[lo + i] = r[i].orig;
    free(xs); free(r);
  }
  int64_t mid = lo + n / 2;
  o->lo[2 * a] = lo; o->hi[2 * a] = mid;
  o->lo[2 * a + 1] = mid; o->hi[2 * a + 1] = hi;
  split_node(o, 2 * a, level + 1);
  split_node(o, 2 * a + 1, level + 1);
}

kfo* kfo_create(const double* X, int64_t N, int32_t d, int32_t m) {
  if (!X || N < 1 || d < 1 || m < 1) return NULL;
  for (int64_t i = 0; i < N * d; ++i) if (!isfinite(X[i])) return NULL;
  kfo* o = (kfo*)calloc(1, sizeof(kfo));
  o->N = N; o->d = d; o->m = m;
  int32_t D = 0;
  while (((int64_t)m << D) < N) ++D;
  o->D = D;
  o->nnodes = (1 << (D + 1)) - 1;
  o->X = (double*)malloc(sizeof(double) * N * d);
  memcpy(o->X, X, sizeof(double) * N * d);
  o->perm = (int64_t*)malloc(sizeof(int64_t) * N);
  for (int64_t i = 0; i < N; ++i) o->perm[i] = i;
  o->lo = (int64_t*)calloc(o->nnodes + 1, sizeof(int64_t));
  o->hi = (int64_t*)calloc(o->nnodes + 1, sizeof(int64_t));
  o->lo[1] = 0; o->hi[1] = N;
  split_node(o, 1, 0);
  o->nd = (node_t*)calloc(o->nnodes + 1, sizeof(node_t));
  return o;
}

static void free_factor(kfo* o) {
  for (int32_t a = 1; a <= o->nnodes; ++a) {
    node_t* n = &o->nd[a];
    free(n->LU); free(n->piv); free(n->Phat); free(n->Vl); free(n->Vr);
    free(n->Z); free(n->ZLU); free(n->Zpiv);
    n->LU = n->Phat = n->Vl = n->Vr = n->Z = n->ZLU = NULL; n->piv = n->Zpiv = NULL;
  }
  o->factorized = 0;
}

static void free_skel(kfo* o) {
  for (int32_t a = 1; a <= o->nnodes; ++a) {
    node_t* n = &o->nd[a];
    free(n->skel); free(n->P); free(n->Pfull);
    n->skel = NULL; n->P = n->Pfull = NULL; n->s = 0; n->c = 0;
  }
  o->skeletonized = 0;
}

static void free_near(kfo* o) {
  if (o->near_pos)
    for (int32_t a = 0; a <= o->nnodes; ++a) { free(o->near_pos[a]); free(o->near_cnt[a]); }
  free(o->near_pos); free(o->near_cnt); free(o->near_len);
  o->near_pos = NULL; o->near_cnt = NULL; o->near_len = NULL;
  o->near_on = 0;
}

void kfo_free(kfo* o) {
  if (!o) return;
  free_factor(o);
  free_skel(o);
  free(o->hyb_off); free(o->hyb_lu); free(o->hyb_piv);
  free_near(o);
  free(o->nd); free(o->X); free(o->perm); free(o->lo); free(o->hi);
  free(o);
}

int32_t kfo_depth(const kfo* o) { return o->D; }
void kfo_perm(const kfo* o, int64_t* perm) { memcpy(perm, o->perm, sizeof(int64_t) * o->N); }
void kfo_node_range(const kfo* o, int32_t a, int64_t* lo, int64_t* hi) { *lo = o->lo[a]; *hi = o->hi[a]; }

/* ------------------------------------------------------------------------ */
/* Sampling of S' (Sec. II-A: "sampling a small subset S' of S").
 * READING: the paper defers the sampler to ASKIT.  Here S' is n_s =
 * min(N - |alpha|, n_samp) distinct positions drawn uniformly from the
 * complement of alpha: draw j gives u = splitmix64(seed ^ (node << 32) ^ j),
 * c = u mod (N - |alpha|); c is skipped if already drawn; c maps to the tree
 * position c (c < lo) or c + |alpha| (c >= lo).  When n_s equals the
 * complement size the whole complement is taken.  The result is ascending. */

/* splitmix64 (Steele, Lea, Flood 2014): add the golden-ratio increment, then
 * the xor-shift-multiply finalizer. */
uint64_t kfo_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static int cmp_i64(const void* A, const void* B) {
  int64_t a = *(const int64_t*)A, b = *(const int64_t*)B;
  return (a > b) - (a < b);
}

/* With near-field sampling on (kfo_set_near): the first min(|near list|,
 * floor(n_s / 2)) entries of the node's near list are taken, and the rest of
 * S' is drawn as above, a draw also being skipped when its position is one of
 * the near entries taken. */
int32_t kfo_sample(const kfo* o, int32_t a, int32_t n_samp, uint64_t seed, int64_t* out) {
  int64_t lo = o->lo[a], sz = nsz(o, a), M = o->N - sz;
  int64_t ns = M < n_samp ? M : n_samp;
  if (ns == M) {
    int64_t t = 0;
    for (int64_t i = 0; i < o->N; ++i) if (i < lo || i >= lo + sz) out[t++] = i;
    return (int32_t)ns;
  }
  int64_t got = 0, n1 = 0;
  if (o->near_on) {
    n1 = o->near_len[a] < ns / 2 ? o->near_len[a] : ns / 2;
    for (int64_t t = 0; t < n1; ++t) out[got++] = o->near_pos[a][t];
  }
  for (uint64_t j = 0; got < ns; ++j) {
    uint64_t u = kfo_splitmix64(seed ^ ((uint64_t)a << 32) ^ j);
    int64_t c = (int64_t)(u % (uint64_t)M);
    int64_t pos = c < lo ? c : c + sz;
    int dup = 0;
    for (int64_t t = 0; t < got; ++t) if (out[t] == pos) { dup = 1; break; }
    if (!dup) out[got++] = pos;
  }
  qsort(out, ns, sizeof(int64_t), cmp_i64);
  return (int32_t)ns;
}

/* ------------------------------------------------------------------------ */
/* Near-field sampling.  READING: the paper samples S' as ASKIT does, whose
 * sampling draws on the kappa nearest neighbours of the node's points (the
 * paper's parameter kappa, Sec. IV) and fills up with uniform samples.  Here:
 *  1. Neighbours by randomized projection trees: tree t over the tree
 *     positions splits every node like the ball tree (depth
 *     ceil(log2(N / leaf)), floor(n/2) points to the left child) by the order
 *     of (projection on x_q - x_p, position), with p and q the points at
 *     offsets splitmix64(seed ^ (t << 56) ^ (node << 1) ^ k) mod n, k = 0, 1,
 *     of the node's current list (projections in FP64 as the ball tree's).
 *     Within a leaf every point's candidates are the leaf's other points, at
 *     the FP32 squared distance of the FP32-rounded coordinates (sequential
 *     fmaf over the coordinates of u = x_ik - x_jk).  A point keeps the kappa
 *     best (distance, position) pairs over all trees, distinct positions.
 *  2. Node lists: a leaf counts how often each position outside it occurs in
 *     its points' neighbour lists; an internal node adds up its children's
 *     lists (counts of equal positions summed, positions inside it dropped).
 *     Each keeps the near_cap positions of largest count (ties: smaller
 *     position), in that order.
 *  3. kfo_sample takes the first min(list length, floor(n_s / 2)) of them. */
typedef struct { float d; int64_t j; } nbr_t;

static int cmp_nbr(const void* A, const void* B) {
  const nbr_t* a = (const nbr_t*)A;
  const nbr_t* b = (const nbr_t*)B;
  if (a->d != b->d) return a->d < b->d ? -1 : 1;
  return (a->j > b->j) - (a->j < b->j);
}

typedef struct { int64_t pos; int64_t cnt; } cnt_t;

static int cmp_cnt_pos(const void* A, const void* B) {
  const cnt_t* a = (const cnt_t*)A;
  const cnt_t* b = (const cnt_t*)B;
  return (a->pos > b->pos) - (a->pos < b->pos);
}
static int cmp_cnt_rank(const void* A, const void* B) {
  const cnt_t* a = (const cnt_t*)A;
  const cnt_t* b = (const cnt_t*)B;
  if (a->cnt != b->cnt) return a->cnt > b->cnt ? -1 : 1;
  return (a->pos > b->pos) - (a->pos < b->pos);
}

typedef struct { double key; int64_t pos; } proj_t;
static int cmp_proj(const void* A, const void* B) {
  const proj_t* a = (const proj_t*)A;
  const proj_t* b = (const proj_t*)B;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return (a->pos > b->pos) - (a->pos < b->pos);
}

static float dist32(const float* x, const float* y, int32_t d) {
  float acc = 0.0f;
  for (int32_t k = 0; k < d; ++k) {
    float u = x[k] - y[k];
    acc = fmaf(u, u, acc);
  }
  return acc;
}

/* Orders positions ord[0..N) by randomized projection tree t; leaves of the
 * complete tree of depth Dk are contiguous ranges (node ranges as the ball
 * tree's). */
static void rp_tree(const kfo* o, int32_t t, int32_t Dk, uint64_t seed, int64_t* ord) {
  const int64_t N = o->N;
  const int32_t d = o->d;
  int64_t nn = (int64_t)1 << (Dk + 1);
  int64_t* lo = (int64_t*)malloc(sizeof(int64_t) * nn);
  int64_t* hi = (int64_t*)malloc(sizeof(int64_t) * nn);
  lo[1] = 0; hi[1] = N;
  for (int64_t a = 1; a < ((int64_t)1 << Dk); ++a) {
    int64_t n = hi[a] - lo[a], mid = lo[a] + n / 2;
    lo[2 * a] = lo[a]; hi[2 * a] = mid; lo[2 * a + 1] = mid; hi[2 * a + 1] = hi[a];
  }
  for (int64_t i = 0; i < N; ++i) ord[i] = i;
  for (int32_t l = 0; l < Dk; ++l) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = (int64_t)1 << l; a < ((int64_t)1 << (l + 1)); ++a) {
      int64_t n = hi[a] - lo[a];
      if (n < 2) continue;
      int64_t* L = ord + lo[a];
      uint64_t key = seed ^ ((uint64_t)t << 56) ^ ((uint64_t)a << 1);
      const double* xp = o->X + L[kfo_splitmix64(key ^ 0) % (uint64_t)n] * d;
      const double* xq = o->X + L[kfo_splitmix64(key ^ 1) % (uint64_t)n] * d;
      proj_t* pr = (proj_t*)malloc(sizeof(proj_t) * n);
      for (int64_t i = 0; i < n; ++i) {
        const double* xi = o->X + L[i] * d;
        double acc = 0.0;
        for (int32_t k = 0; k < d; ++k) acc = acc + (xi[k] - xp[k]) * (xq[k] - xp[k]);
        pr[i].key = acc;
        pr[i].pos = L[i];
      }
      qsort(pr, n, sizeof(proj_t), cmp_proj);
      for (int64_t i = 0; i < n; ++i) L[i] = pr[i].pos;
      free(pr);
    }
  }
  free(lo); free(hi);
}

int32_t kfo_knn(const kfo* o, int32_t kappa, int32_t ntrees, int32_t leaf, uint64_t seed, int64_t* nbr) {
  if (!o || kappa < 1 || ntrees < 1 || leaf < 2) return KFO_EINVAL;
  const int64_t N = o->N;
  const int32_t d = o->d;
  int32_t Dk = 0;
  while (((int64_t)leaf << Dk) < N) ++Dk;
  float* xf = (float*)malloc(sizeof(float) * (size_t)N * d);
  for (int64_t i = 0; i < N * d; ++i) xf[i] = (float)o->X[i];
  nbr_t* best = (nbr_t*)malloc(sizeof(nbr_t) * (size_t)N * kappa);
  int32_t* nbest = (int32_t*)calloc((size_t)N, sizeof(int32_t));
  int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * N);
  int64_t nleaf = (int64_t)1 << Dk;
  for (int32_t t = 0; t < ntrees; ++t) {
    rp_tree(o, t, Dk, seed, ord);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t f = 0; f < nleaf; ++f) {
      /* leaf range of the complete tree: the same halving as rp_tree */
      int64_t lo = 0, hi = N;
      for (int32_t l = Dk - 1; l >= 0; --l) {
        int64_t mid = lo + (hi - lo) / 2;
        if ((f >> l) & 1) lo = mid; else hi = mid;
      }
      int64_t n = hi - lo;
      nbr_t* cand = (nbr_t*)malloc(sizeof(nbr_t) * (size_t)(n + kappa));
      for (int64_t ii = lo; ii < hi; ++ii) {
        int64_t i = ord[ii];
        int64_t c = 0;
        for (int32_t q = 0; q < nbest[i]; ++q) cand[c++] = best[i * kappa + q];
        for (int64_t jj = lo; jj < hi; ++jj) {
          int64_t j = ord[jj];
          if (j == i) continue;
          int dup = 0;
          for (int32_t q = 0; q < nbest[i]; ++q) if (best[i * kappa + q].j == j) { dup = 1; break; }
          if (dup) continue;
          cand[c].d = dist32(xf + i * d, xf + j * d, d);
          cand[c].j = j;
          ++c;
        }
        qsort(cand, c, sizeof(nbr_t), cmp_nbr);
        int32_t keep = c < kappa ? (int32_t)c : kappa;
        for (int32_t q = 0; q < keep; ++q) best[i * kappa + q] = cand[q];
        nbest[i] = keep;
      }
      free(cand);
    }
  }
  for (int64_t i = 0; i < N; ++i)
    for (int32_t q = 0; q < kappa; ++q) nbr[i * kappa + q] = q < nbest[i] ? best[i * kappa + q].j : -1;
  free(xf); free(best); free(nbest); free(ord);
  return KFO_OK;
}

/* top near_cap of a (pos, cnt) multiset: merge equal positions, rank */
static int32_t near_select(cnt_t* e, int64_t n, int32_t cap, int64_t** pos_out, int32_t** cnt_out) {
  qsort(e, n, sizeof(cnt_t), cmp_cnt_pos);
  int64_t u = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (u > 0 && e[u - 1].pos == e[i].pos) e[u - 1].cnt += e[i].cnt;
    else e[u++] = e[i];
  }
  qsort(e, u, sizeof(cnt_t), cmp_cnt_rank);
  int32_t keep = u < cap ? (int32_t)u : cap;
  *pos_out = (int64_t*)malloc(sizeof(int64_t) * (keep > 0 ? keep : 1));
  *cnt_out = (int32_t*)malloc(sizeof(int32_t) * (keep > 0 ? keep : 1));
  for (int32_t q = 0; q < keep; ++q) { (*pos_out)[q] = e[q].pos; (*cnt_out)[q] = (int32_t)e[q].cnt; }
  return keep;
}

int32_t kfo_set_near(kfo* o, const int64_t* nbr, int32_t kappa, int32_t near_cap) {
  if (!o) return KFO_EINVAL;
  free_near(o);
  if (!nbr) return KFO_OK;
  if (kappa < 1 || near_cap < 0) return KFO_EINVAL;
  o->near_cap = near_cap;
  o->near_pos = (int64_t**)calloc((size_t)o->nnodes + 1, sizeof(int64_t*));
  o->near_cnt = (int32_t**)calloc((size_t)o->nnodes + 1, sizeof(int32_t*));
  o->near_len = (int32_t*)calloc((size_t)o->nnodes + 1, sizeof(int32_t));
  for (int32_t l = o->D; l >= 1; --l) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t a = 1 << l; a < (1 << (l + 1)); ++a) {
      int64_t lo = o->lo[a], hi = o->hi[a];
      cnt_t* e;
      int64_t n = 0;
      if (l == o->D) {
        e = (cnt_t*)malloc(sizeof(cnt_t) * (size_t)((hi - lo) * kappa + 1));
        for (int64_t i = lo; i < hi; ++i)
          for (int32_t q = 0; q < kappa; ++q) {
            int64_t j = nbr[i * kappa + q];
            if (j >= 0 && (j < lo || j >= hi)) { e[n].pos = j; e[n].cnt = 1; ++n; }
          }
      } else {
        int32_t c0 = 2 * a, c1 = 2 * a + 1;
        e = (cnt_t*)malloc(sizeof(cnt_t) * (size_t)(o->near_len[c0] + o->near_len[c1] + 1));
        for (int32_t cc = c0; cc <= c1; ++cc)
          for (int32_t q = 0; q < o->near_len[cc]; ++q) {
            int64_t j = o->near_pos[cc][q];
            if (j < lo || j >= hi) { e[n].pos = j; e[n].cnt = o->near_cnt[cc][q]; ++n; }
          }
      }
      o->near_len[a] = near_select(e, n, near_cap, &o->near_pos[a], &o->near_cnt[a]);
      free(e);
    }
  }
  o->near_on = 1;
  return KFO_OK;
}

int32_t kfo_node_near(const kfo* o, int32_t a, int64_t* pos, int32_t* cnt) {
  if (!o || !o->near_on || a < 2 || a > o->nnodes) return 0;
  int32_t n = o->near_len[a];
  if (pos) memcpy(pos, o->near_pos[a], sizeof(int64_t) * n);
  if (cnt) memcpy(cnt, o->near_cnt[a], sizeof(int32_t) * n);
  return n;
}

/* ------------------------------------------------------------------------ */
/* Interpolative decomposition, Eq. (e:id): K_{S' C} ~ K_{S' C~} P_{C~ C}.
 * Pivoted Householder QR (Businger-Golub) of A = K_{S' C}: at step k the
 * squared norms of the trailing columns (rows k..) are recomputed and the
 * largest is the pivot (ties: lowest column).  Rank rule of Sec. II-A with the
 * diagonal of R as the singular-value estimate: s = the smallest k >= 1 with
 * |R_kk| < tau |R_00| (0-based), capped by min(s_max, n_s, c); s = 0 when
 * |R_00| = 0.  C~ = the first s pivots; P = [I, R11^-1 R12] with the columns
 * put back in their original order.
 * READING: the paper writes P = K_{S C~}^+ K_{S C}; on the sampled rows this
 * is R11^-1 R12 of the truncated QR, the standard ID form it cites. */
static void id_node(kfo* o, int32_t a, const int64_t* cols, int32_t c, double tau, int32_t s_max,
                    int32_t n_samp, uint64_t seed) {
  node_t* nd = &o->nd[a];
  nd->c = c;
  int64_t* S = (int64_t*)malloc(sizeof(int64_t) * (n_samp > 0 ? n_samp : 1));
  int32_t ns = kfo_sample(o, a, n_samp, seed, S);
  int32_t kmax = s_max;
  if (ns < kmax) kmax = ns;
  if (c < kmax) kmax = c;
  double* A = (double*)malloc(sizeof(double) * (size_t)(ns > 0 ? ns : 1) * (c > 0 ? c : 1));
  for (int32_t i = 0; i < ns; ++i)
    for (int32_t j = 0; j < c; ++j) A[(int64_t)i * c + j] = kern(o, S[i], cols[j]);
  int32_t* pv = (int32_t*)malloc(sizeof(int32_t) * (c > 0 ? c : 1));
  for (int32_t j = 0; j < c; ++j) pv[j] = j;
  double* v = (double*)malloc(sizeof(double) * (ns > 0 ? ns : 1));
  int32_t s = kmax;
  double r00 = 0.0;
  for (int32_t k = 0; k < kmax; ++k) {
    int32_t p = k; double best = -1.0;
    for (int32_t j = k; j < c; ++j) {
      double nrm = 0.0;
      for (int32_t i = k; i < ns; ++i) nrm = nrm + A[(int64_t)i * c + j] * A[(int64_t)i * c + j];
      if (nrm > best) { best = nrm; p = j; }
    }
    double rkk = sqrt(best);
    if (k == 0) {
      r00 = rkk;
      if (r00 == 0.0) { s = 0; break; }
    } else if (rkk < tau * r00) { s = k; break; }
    if (p != k) {
      for (int32_t i = 0; i < ns; ++i) { double t = A[(int64_t)i * c + k]; A[(int64_t)i * c + k] = A[(int64_t)i * c + p]; A[(int64_t)i * c + p] = t; }
      int32_t t = pv[k]; pv[k] = pv[p]; pv[p] = t;
    }
    /* Householder reflector H = I - beta v v^T with H x = alpha e_0. */
    double x0 = A[(int64_t)k * c + k];
    double alpha = (x0 >= 0.0) ? -rkk : rkk;
    double vtv = 0.0;
    for (int32_t i = k; i < ns; ++i) {
      v[i] = A[(int64_t)i * c + k];
      if (i == k) v[i] = x0 - alpha;
      vtv = vtv + v[i] * v[i];
    }
    double beta = (vtv > 0.0) ? 2.0 / vtv : 0.0;
    for (int32_t j = k + 1; j < c; ++j) {
      double w = 0.0;
      for (int32_t i = k; i < ns; ++i) w = w + v[i] * A[(int64_t)i * c + j];
      w = beta * w;
      for (int32_t i = k; i < ns; ++i) A[(int64_t)i * c + j] = A[(int64_t)i * c + j] - w * v[i];
    }
    A[(int64_t)k * c + k] = alpha;
    for (int32_t i = k + 1; i < ns; ++i) A[(int64_t)i * c + k] = 0.0;
  }
  /* T = R11^-1 R12 by back substitution (s x (c - s)). */
  int32_t nc = c - s;
  double* T = (double*)malloc(sizeof(double) * (size_t)(s > 0 ? s : 1) * (nc > 0 ? nc : 1));
  for (int32_t j = 0; j < nc; ++j)
    for (int32_t i = s - 1; i >= 0; --i) {
      double acc = A[(int64_t)i * c + s + j];
      for (int32_t t = i + 1; t < s; ++t) acc = acc - A[(int64_t)i * c + t] * T[(int64_t)t * nc + j];
      T[(int64_t)i * nc + j] = acc / A[(int64_t)i * c + i];
    }
  nd->s = s;
  nd->skel = (int64_t*)malloc(sizeof(int64_t) * (s > 0 ? s : 1));
  nd->P = (double*)calloc((size_t)(s > 0 ? s : 1) * (c > 0 ? c : 1), sizeof(double));
  for (int32_t i = 0; i < s; ++i) nd->skel[i] = cols[pv[i]];
  for (int32_t i = 0; i < s; ++i) {
    nd->P[(int64_t)i * c + pv[i]] = 1.0;
    for (int32_t j = 0; j < nc; ++j) nd->P[(int64_t)i * c + pv[s + j]] = T[(int64_t)i * nc + j];
  }
  free(T); free(v); free(pv); free(A); free(S);
}

/* Columns of a node's ID: its points (leaf) or [l~ r~] (internal). */
static int32_t id_columns(const kfo* o, int32_t a, int64_t** cols) {
  if (is_leaf(o, a)) {
    int32_t c = (int32_t)nsz(o, a);
    *cols = (int64_t*)malloc(sizeof(int64_t) * (c > 0 ? c : 1));
    for (int32_t j = 0; j < c; ++j) (*cols)[j] = o->lo[a] + j;
    return c;
  }
  const node_t* l = &o->nd[2 * a];
  const node_t* r = &o->nd[2 * a + 1];
  int32_t c = l->s + r->s;
  *cols = (int64_t*)malloc(sizeof(int64_t) * (c > 0 ? c : 1));
  for (int32_t j = 0; j < l->s; ++j) (*cols)[j] = l->skel[j];
  for (int32_t j = 0; j < r->s; ++j) (*cols)[l->s + j] = r->skel[j];
  return c;
}

/* P_{alpha alpha~} telescoped, Eq. (e:innerid):
 * P_{alpha alpha~} = diag(P_{l l~}, P_{r r~}) P_{[l~ r~] alpha~}. */
static void build_pfull(kfo* o, int32_t a) {
  node_t* nd = &o->nd[a];
  int64_t n = nsz(o, a);
  int32_t s = nd->s;
  free(nd->Pfull);
  nd->Pfull = (double*)calloc((size_t)(n > 0 ? n : 1) * (s > 0 ? s : 1), sizeof(double));
  if (is_leaf(o, a)) {
    for (int64_t i = 0; i < n; ++i)
      for (int32_t j = 0; j < s; ++j) nd->Pfull[i * s + j] = nd->P[(int64_t)j * nd->c + i];
    return;
  }
  const node_t* l = &o->nd[2 * a];
  const node_t* r = &o->nd[2 * a + 1];
  int64_t nl = nsz(o, 2 * a), nr = nsz(o, 2 * a + 1);
  for (int64_t i = 0; i < nl; ++i)
    for (int32_t j = 0; j < s; ++j) {
      double acc = 0.0;
      for (int32_t t = 0; t < l->s; ++t) acc = acc + l->Pfull[i * l->s + t] * nd->P[(int64_t)j * nd->c + t];
      nd->Pfull[i * s + j] = acc;
    }
  for (int64_t i = 0; i < nr; ++i)
    for (int32_t j = 0; j < s; ++j) {
      double acc = 0.0;
      for (int32_t t = 0; t < r->s; ++t) acc = acc + r->Pfull[i * r->s + t] * nd->P[(int64_t)j * nd->c + l->s + t];
      nd->Pfull[(nl + i) * s + j] = acc;
    }
}

/* Algorithm 1, Skeletonize(alpha): children first, then the ID of the node. */
static void skeletonize_rec(kfo* o, int32_t a, double tau, int32_t s_max, int32_t n_samp, uint64_t seed) {
  if (!is_leaf(o, a)) {
#pragma omp task if (nsz(o, a) > 4096)
    skeletonize_rec(o, 2 * a, tau, s_max, n_samp, seed);
#pragma omp task if (nsz(o, a) > 4096)
    skeletonize_rec(o, 2 * a + 1, tau, s_max, n_samp, seed);
#pragma omp taskwait
  }
  if (a == 1) return; /* the root is not skeletonized */
  int64_t* cols;
  int32_t c = id_columns(o, a, &cols);
  id_node(o, a, cols, c, tau, s_max, n_samp, seed);
  free(cols);
  build_pfull(o, a);
}

int32_t kfo_skeletonize(kfo* o, double h, double tau, int32_t s_max, int32_t n_samp, uint64_t seed) {
  if (!(h > 0.0) || !(tau >= 0.0) || s_max < 0 || n_samp < 0) return KFO_EINVAL;
  o->hyb_ready = 0;
  free_factor(o);
  free_skel(o);
  o->h = h;
  o->c_exp = -0.5 / (h * h);
#pragma omp parallel
#pragma omp single
  skeletonize_rec(o, 1, tau, s_max, n_samp, seed);
  o->skeletonized = 1;
  return KFO_OK;
}

int32_t kfo_rank(const kfo* o, int32_t a) { return o->nd[a].s; }
int32_t kfo_ncols(const kfo* o, int32_t a) { return o->nd[a].c; }
void kfo_skel(const kfo* o, int32_t a, int64_t* out) { memcpy(out, o->nd[a].skel, sizeof(int64_t) * o->nd[a].s); }
void kfo_P(const kfo* o, int32_t a, double* out) {
  memcpy(out, o->nd[a].P, sizeof(double) * (size_t)o->nd[a].s * o->nd[a].c);
}
void kfo_P_full(const kfo* o, int32_t a, double* out) {
  memcpy(out, o->nd[a].Pfull, sizeof(double) * (size_t)nsz(o, a) * o->nd[a].s);
}

int32_t kfo_set_id(kfo* o, int32_t a, int32_t s, const int64_t* skel, const double* P) {
  if (a < 2 || a > o->nnodes) return KFO_EINVAL;
  free_factor(o);
  node_t* nd = &o->nd[a];
  int32_t c = is_leaf(o, a) ? (int32_t)nsz(o, a) : o->nd[2 * a].s + o->nd[2 * a + 1].s;
  if (s < 0 || s > c) return KFO_EINVAL;
  free(nd->skel); free(nd->P);
  nd->s = s; nd->c = c;
  nd->skel = (int64_t*)malloc(sizeof(int64_t) * (s > 0 ? s : 1));
  nd->P = (double*)malloc(sizeof(double) * (size_t)(s > 0 ? s : 1) * (c > 0 ? c : 1));
  memcpy(nd->skel, skel, sizeof(int64_t) * s);
  memcpy(nd->P, P, sizeof(double) * (size_t)s * c);
  build_pfull(o, a);
  /* ancestors' telescoped P depend on this node */
  for (int32_t b = a / 2; b >= 2; b /= 2)
    if (o->nd[b].c == o->nd[2 * b].s + o->nd[2 * b + 1].s && o->nd[b].P) build_pfull(o, b);
  return KFO_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3, Solve(alpha, u, do_recur), applied in place to the n x k block
 * U (rows = the node's tree positions).  Internal node: after the (optional)
 * recursion on the children, w = v - W Z^-1 V v with
 * V v = [K_{l~ r} v_r ; K_{r~ l} v_l] and W = diag(P^_l, P^_r) (Eq. e:blocksmw).
 * READING: the printed last line uses u where the recursively solved v must
 * stand; with do_recur = false the two coincide. */
static void solve_rec(const kfo* o, int32_t a, double* U, int64_t k, int do_recur) {
  const node_t* nd = &o->nd[a];
  int64_t n = nsz(o, a);
  if (is_leaf(o, a)) {
    lu_solve(nd->LU, nd->piv, n, U, k, 0);
    return;
  }
  int32_t l = 2 * a, r = 2 * a + 1;
  int64_t nl = nsz(o, l), nr = nsz(o, r);
  double* Ul = U;
  double* Ur = U + nl * k;
  if (do_recur) {
#pragma omp task if (n > 4096)
    solve_rec(o, l, Ul, k, 1);
#pragma omp task if (n > 4096)
    solve_rec(o, r, Ur, k, 1);
#pragma omp taskwait
  }
  int32_t sl = o->nd[l].s, sr = o->nd[r].s, z = sl + sr;
  if (z == 0) return;
  double* t = (double*)malloc(sizeof(double) * z * k);
  matmul(nd->Vl, Ur, t, sl, nr, k);            /* K_{l~ r} v_r */
  matmul(nd->Vr, Ul, t + (int64_t)sl * k, sr, nl, k); /* K_{r~ l} v_l */
  lu_solve(nd->ZLU, nd->Zpiv, z, t, k, 0);     /* Z^-1 V v */
  const double* Pl = o->nd[l].Phat;
  const double* Pr = o->nd[r].Phat;
  for (int64_t i = 0; i < nl; ++i)
    for (int64_t j = 0; j < k; ++j) {
      double acc = 0.0;
      for (int32_t q = 0; q < sl; ++q) acc = acc + Pl[i * sl + q] * t[(int64_t)q * k + j];
      Ul[i * k + j] = Ul[i * k + j] - acc;
    }
  for (int64_t i = 0; i < nr; ++i)
    for (int64_t j = 0; j < k; ++j) {
      double acc = 0.0;
      for (int32_t q = 0; q < sr; ++q) acc = acc + Pr[i * sr + q] * t[(int64_t)(sl + q) * k + j];
      Ur[i * k + j] = Ur[i * k + j] - acc;
    }
  free(t);
}

/* W P_c with P_c = P_{[l~ r~] alpha~} = (P_{alpha~ [l~ r~]})^T:
 * rows of l get P^_l P_c[top], rows of r get P^_r P_c[bottom]. */
static double* w_times_pc(const kfo* o, int32_t a) {
  const node_t* nd = &o->nd[a];
  int32_t l = 2 * a, r = 2 * a + 1, s = nd->s, sl = o->nd[l].s, sr = o->nd[r].s;
  int64_t nl = nsz(o, l), nr = nsz(o, r);
  double* u = (double*)calloc((size_t)(nl + nr) * (s > 0 ? s : 1), sizeof(double));
  for (int64_t i = 0; i < nl; ++i)
    for (int32_t j = 0; j < s; ++j) {
      double acc = 0.0;
      for (int32_t q = 0; q < sl; ++q) acc = acc + o->nd[l].Phat[i * sl + q] * nd->P[(int64_t)j * nd->c + q];
      u[i * s + j] = acc;
    }
  for (int64_t i = 0; i < nr; ++i)
    for (int32_t j = 0; j < s; ++j) {
      double acc = 0.0;
      for (int32_t q = 0; q < sr; ++q) acc = acc + o->nd[r].Phat[i * sr + q] * nd->P[(int64_t)j * nd->c + sl + q];
      u[(nl + i) * s + j] = acc;
    }
  return u;
}

/* Algorithm 2, Factorize(alpha), postorder. */
static void factorize_rec(kfo* o, int32_t a) {
  node_t* nd = &o->nd[a];
  int64_t n = nsz(o, a);
  if (is_leaf(o, a)) {
    /* LU of lambda I + K_aa (lambda enters only the leaf blocks). */
    nd->LU = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n * n : 1));
    nd->piv = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j)
        nd->LU[i * n + j] = kern(o, o->lo[a] + i, o->lo[a] + j) + (i == j ? o->lambda : 0.0);
    double rel = lu_factor(nd->LU, nd->piv, n);
    if (rel < 1e-14) {
#pragma omp atomic write
      o->illcond = 1;
    }
    /* base case: P^_alpha = (lambda I + K_aa)^-1 P_{alpha alpha~} */
    if (a != 1) {
      int32_t s = nd->s;
      nd->Phat = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (s > 0 ? s : 1));
      memcpy(nd->Phat, nd->Pfull, sizeof(double) * (size_t)n * s);
      lu_solve(nd->LU, nd->piv, n, nd->Phat, s, 0);
    }
    return;
  }
  int32_t l = 2 * a, r = 2 * a + 1;
#pragma omp task if (n > 4096)
  factorize_rec(o, l);
#pragma omp task if (n > 4096)
  factorize_rec(o, r);
#pragma omp taskwait
  int32_t sl = o->nd[l].s, sr = o->nd[r].s, z = sl + sr;
  int64_t nl = nsz(o, l), nr = nsz(o, r);
  /* V_alpha blocks K_{l~ r} and K_{r~ l} (second form of Eq. e:uv). */
  nd->Vl = (double*)malloc(sizeof(double) * (size_t)(sl > 0 ? sl : 1) * (nr > 0 ? nr : 1));
  nd->Vr = (double*)malloc(sizeof(double) * (size_t)(sr > 0 ? sr : 1) * (nl > 0 ? nl : 1));
  for (int32_t i = 0; i < sl; ++i)
    for (int64_t j = 0; j < nr; ++j) nd->Vl[i * nr + j] = kern(o, o->nd[l].skel[i], o->lo[r] + j);
  for (int32_t i = 0; i < sr; ++i)
    for (int64_t j = 0; j < nl; ++j) nd->Vr[i * nl + j] = kern(o, o->nd[r].skel[i], o->lo[l] + j);
  /* Reduced system of Eq. (e:blocksmw): Z = [[I, K_{l~r} P^_r], [K_{r~l} P^_l, I]]. */
  size_t zz = (size_t)(z > 0 ? z : 1) * (z > 0 ? z : 1);
  nd->Z = (double*)calloc(zz, sizeof(double));
  for (int32_t i = 0; i < z; ++i) nd->Z[(int64_t)i * z + i] = 1.0;
  double* tmp = (double*)malloc(sizeof(double) * zz);
  matmul(nd->Vl, o->nd[r].Phat, tmp, sl, nr, sr);
  for (int32_t i = 0; i < sl; ++i)
    for (int32_t j = 0; j < sr; ++j) nd->Z[(int64_t)i * z + sl + j] = tmp[(int64_t)i * sr + j];
  matmul(nd->Vr, o->nd[l].Phat, tmp, sr, nl, sl);
  for (int32_t i = 0; i < sr; ++i)
    for (int32_t j = 0; j < sl; ++j) nd->Z[(int64_t)(sl + i) * z + j] = tmp[(int64_t)i * sl + j];
  free(tmp);
  nd->ZLU = (double*)malloc(sizeof(double) * zz);
  memcpy(nd->ZLU, nd->Z, sizeof(double) * zz);
  nd->Zpiv = (int64_t*)malloc(sizeof(int64_t) * (z > 0 ? z : 1));
  double rel = lu_factor(nd->ZLU, nd->Zpiv, z);
  if (rel < 1e-14) {
#pragma omp atomic write
    o->illcond = 1;
  }
  if (a == 1) return;
  int32_t s = nd->s;
  if (o->variant == 0) {
    /* Eq. (e:invtelescope): P^_alpha = Solve(alpha, W P_c, false). */
    double* u = w_times_pc(o, a);
    solve_rec(o, a, u, s, 0);
    nd->Phat = u;
  } else {
    /* log^2 N predecessor: P^_alpha = K~_aa^-1 P_{alpha alpha~} by a full
     * recursive solve with the telescoped P of Eq. (e:innerid). */
    double* u = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (s > 0 ? s : 1));
    memcpy(u, nd->Pfull, sizeof(double) * (size_t)n * s);
    solve_rec(o, a, u, s, 1);
    nd->Phat = u;
  }
}

int32_t kfo_factorize(kfo* o, double lambda, int32_t variant) {
  if (!o->skeletonized) return KFO_EINVAL;
  if (!(lambda >= 0.0) || (variant != 0 && variant != 1)) return KFO_EINVAL;
  free_factor(o);
  o->hyb_ready = 0;
  o->lambda = lambda;
  o->variant = variant;
  o->illcond = 0;
#pragma omp parallel
#pragma omp single
  factorize_rec(o, 1);
  o->factorized = 1;
  return o->illcond ? KFO_EILLCOND : KFO_OK;
}

void kfo_Phat(const kfo* o, int32_t a, double* out) {
  memcpy(out, o->nd[a].Phat, sizeof(double) * (size_t)nsz(o, a) * o->nd[a].s);
}

void kfo_Z(const kfo* o, int32_t a, double* out) {
  int32_t z = o->nd[2 * a].s + o->nd[2 * a + 1].s;
  memcpy(out, o->nd[a].Z, sizeof(double) * (size_t)z * z);
}

int32_t kfo_Phat_forms(const kfo* o, int32_t a, double* literal, double* pushed) {
  if (!o->factorized || is_leaf(o, a) || a == 1) return KFO_EINVAL;
  const node_t* nd = &o->nd[a];
  int32_t s = nd->s, l = 2 * a, r = 2 * a + 1, sl = o->nd[l].s, sr = o->nd[r].s, z = sl + sr;
  int64_t n = nsz(o, a), nl = nsz(o, l);
  double* u = w_times_pc(o, a);
  memcpy(literal, u, sizeof(double) * (size_t)n * s);
  solve_rec(o, a, literal, s, 0);
  free(u);
  /* W Z^-1 P_c */
  double* T = (double*)malloc(sizeof(double) * (size_t)(z > 0 ? z : 1) * (s > 0 ? s : 1));
  for (int32_t i = 0; i < z; ++i)
    for (int32_t j = 0; j < s; ++j) T[(int64_t)i * s + j] = nd->P[(int64_t)j * nd->c + i];
  lu_solve(nd->ZLU, nd->Zpiv, z, T, s, 0);
  matmul(o->nd[l].Phat, T, pushed, nl, sl, s);
  matmul(o->nd[r].Phat, T + (int64_t)sl * s, pushed + nl * s, n - nl, sr, s);
  free(T);
  return KFO_OK;
}

/* ------------------------------------------------------------------------ */
/* Transpose solve: K~_aa^-1 = (I - W Z^-1 V) D^-1 (Eq. e:smw), so
 * K~_aa^-T = D^-T (I - V^T Z^-T W^T): first t = Z^-T [P^_l^T u_l ; P^_r^T u_r],
 * u_l -= K_{r~ l}^T t_r, u_r -= K_{l~ r}^T t_l, then recurse. */
static void tsolve_rec(const kfo* o, int32_t a, double* u) {
  const node_t* nd = &o->nd[a];
  int64_t n = nsz(o, a);
  if (is_leaf(o, a)) {
    lu_solve(nd->LU, nd->piv, n, u, 1, 1);
    return;
  }
  int32_t l = 2 * a, r = 2 * a + 1, sl = o->nd[l].s, sr = o->nd[r].s, z = sl + sr;
  int64_t nl = nsz(o, l), nr = nsz(o, r);
  double* ul = u;
  double* ur = u + nl;
  if (z > 0) {
    double* t = (double*)calloc(z, sizeof(double));
    for (int32_t q = 0; q < sl; ++q) {
      double acc = 0.0;
      for (int64_t i = 0; i < nl; ++i) acc = acc + o->nd[l].Phat[i * sl + q] * ul[i];
      t[q] = acc;
    }
    for (int32_t q = 0; q < sr; ++q) {
      double acc = 0.0;
      for (int64_t i = 0; i < nr; ++i) acc = acc + o->nd[r].Phat[i * sr + q] * ur[i];
      t[sl + q] = acc;
    }
    lu_solve(nd->ZLU, nd->Zpiv, z, t, 1, 1);
    for (int64_t j = 0; j < nl; ++j) {
      double acc = 0.0;
      for (int32_t q = 0; q < sr; ++q) acc = acc + nd->Vr[(int64_t)q * nl + j] * t[sl + q];
      ul[j] = ul[j] - acc;
    }
    for (int64_t j = 0; j < nr; ++j) {
      double acc = 0.0;
      for (int32_t q = 0; q < sl; ++q) acc = acc + nd->Vl[(int64_t)q * nr + j] * t[q];
      ur[j] = ur[j] - acc;
    }
    free(t);
  }
#pragma omp task if (n > 4096)
  tsolve_rec(o, l, ul);
#pragma omp task if (n > 4096)
  tsolve_rec(o, r, ur);
#pragma omp taskwait
}

int32_t kfo_solve(const kfo* o, const double* b, double* x, int32_t transpose) {
  if (!o->factorized) return KFO_EINVAL;
  int64_t N = o->N;
  double* u = (double*)malloc(sizeof(double) * N);
  for (int64_t i = 0; i < N; ++i) u[i] = b[o->perm[i]];
#pragma omp parallel
#pragma omp single
  {
    if (transpose) tsolve_rec(o, 1, u);
    else solve_rec(o, 1, u, 1, 1);
  }
  for (int64_t i = 0; i < N; ++i) x[o->perm[i]] = u[i];
  free(u);
  return KFO_OK;
}

/* ------------------------------------------------------------------------ */
/* Hierarchical matvec with the operator the factorization inverts:
 * K~_aa = [[K~_ll, P_{l l~} K_{l~ r}], [P_{r r~} K_{r~ l}, K~_rr]]
 * (second form of Eq. e:uv), lambda I + K_aa at the leaves.  The skeleton
 * blocks are evaluated on the fly, independent of the factorization.  With
 * deriv = 1 every kernel entry is replaced by dK/dh and lambda by 0 (the
 * derivative of the operator with the skeletons and P held fixed). */
static void matvec_rec(const kfo* o, int32_t a, const double* x, double* y, int deriv) {
  int64_t n = nsz(o, a), lo = o->lo[a];
  if (is_leaf(o, a)) {
    for (int64_t i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int64_t j = 0; j < n; ++j)
        acc = acc + (deriv ? dkern_dh(o, lo + i, lo + j) : kern(o, lo + i, lo + j)) * x[j];
      y[i] = (deriv ? 0.0 : o->lambda * x[i]) + acc;
    }
    return;
  }
  int32_t l = 2 * a, r = 2 * a + 1;
  int64_t nl = nsz(o, l);
#pragma omp task if (n > 4096)
  matvec_rec(o, l, x, y, deriv);
#pragma omp task if (n > 4096)
  matvec_rec(o, r, x + nl, y + nl, deriv);
#pragma omp taskwait
  for (int side = 0; side < 2; ++side) {
    int32_t c = side == 0 ? l : r, sib = side == 0 ? r : l;
    const node_t* cn = &o->nd[c];
    int64_t nc = nsz(o, c), nsib = nsz(o, sib);
    const double* xs = x + (o->lo[sib] - lo);
    double* yc = y + (o->lo[c] - lo);
    double* zt = (double*)calloc(cn->s > 0 ? cn->s : 1, sizeof(double));
    for (int32_t q = 0; q < cn->s; ++q) {   /* K_{c~ sib} x_sib */
      double acc = 0.0;
      for (int64_t j = 0; j < nsib; ++j)
        acc = acc + (deriv ? dkern_dh(o, cn->skel[q], o->lo[sib] + j) : kern(o, cn->skel[q], o->lo[sib] + j)) * xs[j];
      zt[q] = acc;
    }
    for (int64_t i = 0; i < nc; ++i) {      /* P_{c c~} (...) */
      double acc = 0.0;
      for (int32_t q = 0; q < cn->s; ++q) acc = acc + cn->Pfull[i * cn->s + q] * zt[q];
      yc[i] = yc[i] + acc;
    }
    free(zt);
  }
}

int32_t kfo_matvec(const kfo* o, const double* x, double* y, int32_t deriv) {
  if (!o->skeletonized) return KFO_EINVAL;
  int64_t N = o->N;
  double* u = (double*)malloc(sizeof(double) * N);
  double* v = (double*)malloc(sizeof(double) * N);
  for (int64_t i = 0; i < N; ++i) u[i] = x[o->perm[i]];
#pragma omp parallel
#pragma omp single
  matvec_rec(o, 1, u, v, deriv);
  for (int64_t i = 0; i < N; ++i) y[o->perm[i]] = v[i];
  free(u); free(v);
  return KFO_OK;
}

/* Gradient through x = A^-1 b with A = lambda I + K~(h):
 * a = A^-T g; dL/db = a; dL/dlambda = -a^T x; dL/dh = -a^T (dK~/dh) x. */
int32_t kfo_grad(const kfo* o, const double* x, const double* g, double* dLdb, double* dLdlambda, double* dLdh) {
  if (!o->factorized) return KFO_EINVAL;
  int64_t N = o->N;
  kfo_solve(o, g, dLdb, 1);
  double* dx = (double*)malloc(sizeof(double) * N);
  kfo_matvec(o, x, dx, 1);
  double sl = 0.0, sh = 0.0;
  for (int64_t i = 0; i < N; ++i) { sl = sl + dLdb[i] * x[i]; sh = sh + dLdb[i] * dx[i]; }
  *dLdlambda = -sl;
  *dLdh = -sh;
  free(dx);
  return KFO_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithms 1 and 2 on chosen subtrees only.  The ID of a node reads its own
 * columns and its sampled rows S' (drawn from the complement in the whole
 * tree), and Z, P^ and the leaf factors of a node read only its descendants'
 * skeletons and factors; so every node under the given roots gets exactly the
 * values kfo_skeletonize followed by kfo_factorize give it (a root that is the
 * tree root gets no ID and no P^, as there).  The rest of the tree is not
 * touched.  This checks single nodes of trees too large for a whole run. */
static void clear_node(node_t* n) {
  free(n->skel); free(n->P); free(n->Pfull);
  free(n->LU); free(n->piv); free(n->Phat); free(n->Vl); free(n->Vr);
  free(n->Z); free(n->ZLU); free(n->Zpiv);
  memset(n, 0, sizeof(node_t));
}

static int is_ancestor_or_self(int32_t a, int32_t b) {
  while (b > a) b >>= 1;
  return a == b;
}

int32_t kfo_subtrees(kfo* o, const int32_t* roots, int32_t nroots, double h, double tau, int32_t s_max,
                     int32_t n_samp, uint64_t seed, double lambda) {
  if (!o || !roots || nroots < 1 || !(h > 0.0) || !(tau >= 0.0) || s_max < 0 || n_samp < 0 || !(lambda >= 0.0))
    return KFO_EINVAL;
  for (int32_t i = 0; i < nroots; ++i) {
    if (roots[i] < 1 || roots[i] > o->nnodes) return KFO_EINVAL;
    for (int32_t j = 0; j < nroots; ++j)
      if (i != j && (is_ancestor_or_self(roots[i], roots[j]) || is_ancestor_or_self(roots[j], roots[i])))
        return KFO_EINVAL;  /* subtrees must be disjoint */
  }
  o->hyb_ready = 0;
  for (int32_t i = 0; i < nroots; ++i)
    for (int32_t lv = 0; ((int64_t)roots[i] << lv) <= o->nnodes; ++lv)
      for (int64_t b = (int64_t)roots[i] << lv; b < ((int64_t)roots[i] + 1) << lv; ++b) clear_node(&o->nd[b]);
  o->h = h;
  o->c_exp = -0.5 / (h * h);
  o->lambda = lambda;
  o->variant = 0;
  o->illcond = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t i = 0; i < nroots; ++i) {
    skeletonize_rec(o, roots[i], tau, s_max, n_samp, seed);
    factorize_rec(o, roots[i]);
  }
  if (nroots == 1 && roots[0] == 1) o->skeletonized = o->factorized = 1; /* the whole tree */
  return o->illcond ? KFO_EILLCOND : KFO_OK;
}

/* ------------------------------------------------------------------------ */
/* Hybrid level-restricted solver (Sec. II-C "Fast hybrid solver",
 * Algorithms 6-8).  The frontier A is the set of the 2^L nodes of level L
 * (1 <= L <= D): their subtrees are skeletonized and factorized by
 * Algorithms 1-2, the frontier nodes' own IDs and P^ included; the nodes above
 * A are neither compressed nor factorized.  The operator is
 *   lambda I + K~ = D + U V,   D = blockdiag(lambda I + K~_aa),
 *   U = blockdiag(P_{a a~}),   V[a~, b] = K_{a~ b} for frontier nodes b != a
 *   (and 0 for b = a),
 * so the block between two frontier subtrees is P_{a a~} K_{a~ b} (the second
 * form of Eq. e:uv).  With W = D^-1 U = blockdiag(P^_a), Eq. (e:smw) gives
 *   x = D^-1 u - W (I + V W)^-1 V D^-1 u          (Algorithm 6).
 * The paper solves the reduced system I + VW (size sum_a s_a) by a Krylov
 * method with the products of Algorithms 7 (MatVecW) and 8 (MatVecV); the
 * oracle forms it, (VW)[a~, b~] = K_{a~ b} P^_b, and factors it with LU.
 * READING: the last line of Algorithm 6 is printed w = u - MatVecW(root, w, A);
 * the vector the correction is subtracted from is D^-1 u of its first line,
 * as Eq. (e:smw) requires. */
static int32_t frontier_s(const kfo* o, int32_t a) { return o->nd[a].s; }

/* t[a~] = sum over frontier b != a of K_{a~ b} y_b (Algorithm 8 over A). */
static void hyb_apply_v(const kfo* o, const double* y, double* t) {
  int32_t nA = 1 << o->hyb_L;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t ia = 0; ia < nA; ++ia) {
    int32_t a = nA + ia;
    const node_t* na = &o->nd[a];
    for (int32_t q = 0; q < na->s; ++q) {
      double acc = 0.0;
      for (int32_t ib = 0; ib < nA; ++ib) {
        int32_t b = nA + ib;
        if (b == a) continue;
        for (int64_t j = o->lo[b]; j < o->hi[b]; ++j) acc = acc + kern(o, na->skel[q], j) * y[j];
      }
      t[o->hyb_off[ia] + q] = acc;
    }
  }
}

int32_t kfo_hybrid(kfo* o, int32_t L, double h, double tau, int32_t s_max, int32_t n_samp, uint64_t seed,
                   double lambda) {
  if (!o || L < 1 || L > o->D) return KFO_EINVAL;
  int32_t nA = 1 << L;
  int32_t* roots = (int32_t*)malloc(sizeof(int32_t) * nA);
  for (int32_t i = 0; i < nA; ++i) roots[i] = nA + i;
  int32_t st = kfo_subtrees(o, roots, nA, h, tau, s_max, n_samp, seed, lambda);
  free(roots);
  if (st != KFO_OK && st != KFO_EILLCOND) return st;
  free(o->hyb_off); free(o->hyb_lu); free(o->hyb_piv);
  o->hyb_L = L;
  o->hyb_off = (int64_t*)malloc(sizeof(int64_t) * (nA + 1));
  o->hyb_off[0] = 0;
  for (int32_t i = 0; i < nA; ++i) o->hyb_off[i + 1] = o->hyb_off[i] + frontier_s(o, nA + i);
  int64_t S = o->hyb_off[nA];
  o->hyb_lu = (double*)calloc((size_t)(S > 0 ? S * S : 1), sizeof(double));
  o->hyb_piv = (int64_t*)malloc(sizeof(int64_t) * (S > 0 ? S : 1));
  double* M = o->hyb_lu;
  for (int64_t i = 0; i < S; ++i) M[i * S + i] = 1.0;
  /* (VW)[a~, b~] = K_{a~ b} P^_b for frontier nodes a != b */
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t ia = 0; ia < nA; ++ia) {
    const node_t* na = &o->nd[nA + ia];
    for (int32_t ib = 0; ib < nA; ++ib) {
      if (ib == ia) continue;
      int32_t b = nA + ib;
      const node_t* nb = &o->nd[b];
      int64_t n = nsz(o, b);
      double* Kab = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (na->s > 0 ? na->s : 1));
      for (int32_t q = 0; q < na->s; ++q)
        for (int64_t j = 0; j < n; ++j) Kab[q * n + j] = kern(o, na->skel[q], o->lo[b] + j);
      for (int32_t q = 0; q < na->s; ++q)
        for (int32_t t = 0; t < nb->s; ++t) {
          double acc = 0.0;
          for (int64_t j = 0; j < n; ++j) acc = acc + Kab[q * n + j] * nb->Phat[j * nb->s + t];
          M[(o->hyb_off[ia] + q) * S + o->hyb_off[ib] + t] += acc;
        }
      free(Kab);
    }
  }
  double rel = S > 0 ? lu_factor(M, o->hyb_piv, S) : 1.0;
  o->hyb_ready = 1;
  return (st == KFO_EILLCOND || rel < 1e-14) ? KFO_EILLCOND : KFO_OK;
}

int32_t kfo_hybrid_solve(const kfo* o, const double* b, double* x) {
  if (!o || !o->hyb_ready) return KFO_EINVAL;
  int64_t N = o->N;
  int32_t nA = 1 << o->hyb_L;
  int64_t S = o->hyb_off[nA];
  double* y = (double*)malloc(sizeof(double) * N);
  double* t = (double*)calloc((size_t)(S > 0 ? S : 1), sizeof(double));
  for (int64_t i = 0; i < N; ++i) y[i] = b[o->perm[i]];
  /* y = D^-1 u: the direct solve of every frontier subtree (Algorithm 3) */
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t ia = 0; ia < nA; ++ia) solve_rec(o, nA + ia, y + o->lo[nA + ia], 1, 1);
  hyb_apply_v(o, y, t);                                   /* t = V y */
  if (S > 0) lu_solve(o->hyb_lu, o->hyb_piv, S, t, 1, 0); /* z = (I + V W)^-1 t */
  for (int32_t ia = 0; ia < nA; ++ia) {                   /* x = y - W z */
    const node_t* na = &o->nd[nA + ia];
    for (int64_t i = 0; i < nsz(o, nA + ia); ++i) {
      double acc = 0.0;
      for (int32_t q = 0; q < na->s; ++q) acc = acc + na->Phat[i * na->s + q] * t[o->hyb_off[ia] + q];
      y[o->lo[nA + ia] + i] = y[o->lo[nA + ia] + i] - acc;
    }
  }
  for (int64_t i = 0; i < N; ++i) x[o->perm[i]] = y[i];
  free(y); free(t);
  return KFO_OK;
}

int32_t kfo_hybrid_matvec(const kfo* o, const double* x, double* y) {
  if (!o || !o->hyb_ready) return KFO_EINVAL;
  int64_t N = o->N;
  int32_t nA = 1 << o->hyb_L;
  int64_t S = o->hyb_off[nA];
  double* u = (double*)malloc(sizeof(double) * N);
  double* v = (double*)malloc(sizeof(double) * N);
  double* t = (double*)calloc((size_t)(S > 0 ? S : 1), sizeof(double));
  for (int64_t i = 0; i < N; ++i) u[i] = x[o->perm[i]];
  /* D u: the hierarchical operator of every frontier subtree */
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t ia = 0; ia < nA; ++ia) matvec_rec(o, nA + ia, u + o->lo[nA + ia], v + o->lo[nA + ia], 0);
  hyb_apply_v(o, u, t);                                   /* V u */
  for (int32_t ia = 0; ia < nA; ++ia) {                   /* + U (V u) */
    const node_t* na = &o->nd[nA + ia];
    for (int64_t i = 0; i < nsz(o, nA + ia); ++i) {
      double acc = 0.0;
      for (int32_t q = 0; q < na->s; ++q) acc = acc + na->Pfull[i * na->s + q] * t[o->hyb_off[ia] + q];
      v[o->lo[nA + ia] + i] = v[o->lo[nA + ia] + i] + acc;
    }
  }
  for (int64_t i = 0; i < N; ++i) y[o->perm[i]] = v[i];
  free(u); free(v); free(t);
  return KFO_OK;
}
