// kf_internal.cuh -- internal types and device helpers of the CUDA library.
//
// Storage layout in HBM (all fixed-capacity, strides in elements):
//   tree:   X64 N x d (tree order), X32 N x d, perm N, node ranges lo/hi per
//           heap id (root 1, children 2a, 2a+1; level l = 2^l .. 2^(l+1)-1).
//   skel:   rank[node], skel[node * s_max + q] (tree positions, pivot order).
//   Pleaf:  N x s_max (FP64): row i holds P_{a a~}[i, :] of the leaf owning i.
//   Pc:     internal node a: (2 s_max) x s_max FP64 at a * 2 s_max * s_max,
//           P_c = P_{[l~ r~] a~} (rows: ID columns [l~ r~], cols: skeleton).
//   Phat:   level l in [1, D]: N x s_max of type T at (l-1) * N * s_max; row i
//           holds P^_{b b~}[i, :] of the level-l node b owning i (Eq. e:hodlr).
//   VT:     level l in [1, D]: N x s_max of type T; row i holds
//           K(x_i, x_{skel(sib)[q]}) where sib is the sibling of the level-l
//           node owning i, so that K_{sib~ b} = VT[b rows, :s_sib]^T (Eq. e:uv).
//   L:      leaf j: leaf_max x leaf_max of type T (Cholesky factor, row-major).
//   ZLU:    internal node a: (2 s_max)^2 FP64 LU of Z_a, Zpiv (2 s_max) int32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/kf.h"

#define KF_MAX_SMAX 512
#define KF_MAX_D 1024

struct kf_ctx {
  kf_alloc alloc;
  int has_alloc = 0;
  int capturing = 0;  // inside a batched graph capture: scratch comes from cudaMallocAsync
  std::string err;
  void* dalloc(size_t bytes, cudaStream_t s);
  void dfree(void* p, size_t bytes, cudaStream_t s);
};

struct kf_tree {
  kf_ctx* ctx = nullptr;
  int64_t N = 0;
  int32_t d = 0, m = 0, D = 0, nnodes = 0, leaf_max = 0;
  std::vector<int32_t> lo, hi;  // host copy, heap indexed, size nnodes + 1
  int32_t* d_lo = nullptr;
  int32_t* d_hi = nullptr;
  double* X64 = nullptr;
  float* X32 = nullptr;
  float* X32lo = nullptr;  // fp32(X64 - X32): the low half of a double-float copy
  float2* exp_tab = nullptr;  // 2^(j/64), j < 64, as double-float pairs (kf_exp_df)
  int64_t* perm = nullptr;
  std::vector<std::pair<void*, size_t>> allocs;
};

// default: levels with at most this many nodes keep Z^-1 for the solve sweep
// (measured at N = 2^20, s_max = 256: the direct sweep 18% faster on the mixed
// path and 9% on the FP64 path, the factorization within 1.5%)
constexpr int kZinvDefaultMaxNodes = 64;

struct kf_factor {
  kf_tree* t = nullptr;
  kf_ctx* ctx = nullptr;
  double h = 1, lambda = 0, tau = 0, c_exp = 0;
  float c_exp_hi = 0, c_exp_lo = 0;  // c_exp as a double-float pair
  int32_t s_max = 0, n_samp = 0, cmax = 0, prec = 0, vstore = 0, sync_errors = 0;
  int32_t use_tc = 1;  // mixed path: tcgen05 products (0: CUDA-core FP32)
  int32_t fused_zoff = 0;  // mixed path with tcgen05: 1 = Z blocks evaluate their kernel entries (no V read)
  // memory-lean W (kf_opts.w_recompute): P^ of the leaves and two alternating
  // levels only (3 N s_max); Tw holds T = Z^-1 P_c of every internal node
  // (ldz x s_max each, by node, in the factor precision)
  int32_t w_lean = 0;
  void* Tw = nullptr;
  int32_t tc_bn = 256; // tile width of the tcgen05 products: 128 or 256 columns
  int32_t use_cluster_qr = 1;  // upper tree levels: cluster QR in distributed shared memory
  int32_t use_cluster_lu = 1;  // upper tree levels: reduced-system LU and T on a CTA cluster per node
  int32_t fp64_op = 0;  // keep the FP64-accurate operator data (VTdf, Kdf)
  int32_t gmres_m = 0;  // refinement: 0 = Richardson, m > 0 = GMRES(m)
  int32_t refine_user = 0;  // refinement explicitly requested (enables it on the FP64 path)
  // FP64-accurate operator (fp64_op), stored as double-float pairs (hi, lo):
  float2* VTdf = nullptr;  // mixed path: D x N x s_max V blocks
  float2* Kdf = nullptr;   // leaf blocks lambda-free K_aa, leaf_max^2 each
  // mixed path: Pleaf and Pc as pairs, for the operator's passes over several
  // right-hand sides (split once at the end of the factorization)
  float2* Pleafdf = nullptr;
  float2* Pcdf = nullptr;
  // mixed path: the reduced systems' LU factors as pairs (by node, like ZLU) for
  // the levels that keep no Z^-1, read by the sweep over several right-hand sides
  float2* ZLUdf = nullptr;
  double refine_tol = 1e-10;
  int32_t refine_max_iter = 8;
  uint64_t seed = 0x1701;
  int32_t* rank = nullptr;
  int32_t* skel = nullptr;
  double* Pleaf = nullptr;
  double* Pc = nullptr;
  void* Phat = nullptr;
  void* VT = nullptr;
  void* L = nullptr;
  float* Pleaf32 = nullptr;
  double* ZLU = nullptr;
  int32_t* Zpiv = nullptr;
  // explicit Z^-1 of the nodes of levels 0..zinv_top (ldz^2 each, by node):
  // there the sweep's LU solves, one CTA per node, are latency bound, while a
  // product with Z^-1 spreads over many CTAs
  double* Zinv = nullptr;
  int32_t zinv_top = -1;
  int32_t zinv_max_nodes = kZinvDefaultMaxNodes;  // -1: none
  // hybrid level-restricted solver (Sec. II-C): frontier level hyb_L >= 1, or
  // 0 for the direct solver.  Vh: per frontier node a, s_max rows of N FP64
  // entries K(x_{a~q}, x_j) (zero for j in a and for q >= s_a).  The reduced
  // system I + VW is stored as node 1 of a two-node Z array (HM: 2 hyb_scap^2,
  // node 1 at offset hyb_scap^2; Hpiv: 2 hyb_scap), with Hrank = {0, 0, S, 0}
  // so that the reduced-system LU and solve kernels see one node whose first
  // child has rank S = sum of the frontier ranks; Hoff: prefix sums of the
  // frontier ranks (2^L + 1 entries).
  int32_t hyb_L = 0;
  int32_t hyb_scap = 0;
  double* Vh = nullptr;
  double* HM = nullptr;
  int32_t* Hpiv = nullptr;
  int32_t* Hrank = nullptr;
  int32_t* Hoff = nullptr;
  double* Hpivr = nullptr;
  // near-field sampling (knn_kappa > 0): every point's kappa neighbours (tree
  // positions, N x kappa, -1 padding) and every node's list of at most
  // near_cap = n_samp / 2 positions (node * near_cap + i), counts, lengths
  int32_t knn_kappa = 0, knn_trees = 4, knn_leaf = 512, near_cap = 0;
  int32_t* nbr = nullptr;
  int32_t* near_pos = nullptr;
  int32_t* near_cnt = nullptr;
  int32_t* near_len = nullptr;
  // mixed path with tcgen05 products: inverses of the leaves' 128 x 128
  // diagonal Cholesky blocks (leaf, panel) and per-leaf pivot tracking
  float* Dinv = nullptr;
  double* ltrack = nullptr;
  int32_t* status = nullptr;
  double* pivr = nullptr;
  // mixed path, FP64-accurate operator with tc_operator: the V blocks as exact
  // BF16 integer digits for the tensor-core V pass of blocks of right-hand
  // sides (oz_op.cu): tiles of 128 rows x 128 skeleton columns x 7 digits, by
  // level (element offsets oz_off[l]) and 128-row window (oz_wbase: first
  // window of each node within its level, heap indexed)
  int32_t use_oz = 0;
  uint16_t* VTsl = nullptr;
  uint16_t* Ksl = nullptr;  // the leaf blocks' digits: (leaf, row tile, column window) tiles
  // the leaves' P as row-scaled 7-digit tiles (row windows x skeleton
  // windows) for the operator's row update (row exponents PLrexp)
  uint16_t* PLsl = nullptr;
  int32_t* PLrexp = nullptr;
  // P_c of the internal nodes the same way (node, row window, skeleton window),
  // row exponents PCrexp[node 2 s_max + i], for the operator's pushes
  uint16_t* PCsl = nullptr;
  int32_t* PCrexp = nullptr;
  int32_t* oz_wbase = nullptr;
  std::vector<int64_t> oz_off;
  std::vector<int32_t> oz_wbase_h;  // per node: smallest / largest pivot of its leaf Cholesky or Z LU
  std::vector<std::pair<void*, size_t>> allocs;
  size_t tsize() const { return prec == KF_PREC_FP64 ? 8 : 4; }
};

// tensor-core V pass of the FP64-accurate operator (oz_op.cu)
constexpr int kOzTileElems = 128 * 128;  // one BF16 digit tile: 128 skeleton columns x 128 rows
constexpr int kOzChunkRows = 1024;       // rows of one partial sum
struct kf_oz_x {                         // the digits of one B operand
  uint16_t* xsl = nullptr;               // nd x kpad x ldx BF16 digits
  unsigned long long* xmax = nullptr;
  int32_t* xexp = nullptr;               // scales 2^xexp (per column, or per node and column)
  int64_t ldx = 0, k = 0, nexp = 0;
  int kpad = 0, nc = 0;
  size_t bytes = 0;
};
kf_status kf_oz_alloc(kf_factor* f, cudaStream_t s);
kf_status kf_oz_slice_v(kf_factor* f, int lv, cudaStream_t s);
kf_status kf_oz_slice_leaf(kf_factor* f, cudaStream_t s);
kf_status kf_oz_leaf(kf_factor* f, const kf_oz_x& oz, int64_t k, double lambda, const double* x, double* y,
                     cudaStream_t s);
kf_status kf_oz_prepare_x(kf_factor* f, const double* x, int64_t k, kf_oz_x* oz, cudaStream_t s);
kf_status kf_oz_prepare_t(kf_factor* f, int lv, const double* Vt, int64_t k, kf_oz_x* oz, cudaStream_t s);
kf_status kf_oz_slice_rows(kf_factor* f, cudaStream_t s);
kf_status kf_oz_rowupd(kf_factor* f, const kf_oz_x& td, int64_t k, double* y, double sign, cudaStream_t s);
kf_status kf_oz_push(kf_factor* f, int lv, const kf_oz_x& td, int64_t k, double* G, cudaStream_t s);
void kf_oz_release_x(kf_factor* f, kf_oz_x* oz, cudaStream_t s);
kf_status kf_oz_colsum_level(kf_factor* f, int l, const kf_oz_x& oz, int64_t k, double* parts, int* nchunk,
                             cudaStream_t s);

// device status bits
#define KF_DEV_ILLCOND 1
#define KF_DEV_TIMEOUT 2
#define KF_DEV_BADARG 4

// ---- error helpers ----------------------------------------------------------
kf_status kf_set_err(kf_ctx* c, kf_status s, const char* fmt, ...);
#define KF_CUDA(ctx, call)                                                               \
  do {                                                                                   \
    cudaError_t _e = (call);                                                             \
    if (_e != cudaSuccess) return kf_set_err((ctx), KF_ECUDA, "%s: %s (%s:%d)", #call,   \
                                             cudaGetErrorString(_e), __FILE__, __LINE__); \
  } while (0)
#define KF_LAUNCH_CHECK(ctx) KF_CUDA(ctx, cudaGetLastError())

// ---- device helpers ---------------------------------------------------------
// Squared distance and Gaussian kernel in FP64 with two roundings per term
// (no FMA contraction), the operation order of the definition in Eq. e:gaussian.
__device__ __forceinline__ double kf_sqdist64(const double* __restrict__ x, const double* __restrict__ y, int d) {
  double acc = 0.0;
  for (int k = 0; k < d; ++k) {
    double t = __dsub_rn(x[k], y[k]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}
__device__ __forceinline__ double kf_kern64(const double* x, const double* y, int d, double c_exp) {
  return exp(__dmul_rn(kf_sqdist64(x, y, d), c_exp));
}
__device__ __forceinline__ float kf_kern32(const float* __restrict__ x, const float* __restrict__ y, int d, float c_exp) {
  float acc = 0.f;
  for (int k = 0; k < d; ++k) {
    float t = x[k] - y[k];
    acc = fmaf(t, t, acc);
  }
  return __expf(acc * c_exp);
}

// ---- double-float arithmetic on the FP32 pipes ------------------------------------
// Every coordinate is also held as hi + lo (hi = fp32(x), lo = fp32(x - hi)):
// differences, squares and sums then carry an error term through exact
// two-sum / two-product steps, giving about 46 significant bits.
__device__ __forceinline__ void kf_two_sum(float a, float b, float& s, float& e) {
  // round-to-nearest intrinsics: never contracted, so the error term is exact
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// A double-float value is the unevaluated sum hi + lo of two floats, |lo| at
// most half an ulp of hi (Dekker 1971).  two_sum (Knuth) and two_prod (by
// FMA) are error-free; the rest is built from them.
__device__ __forceinline__ void kf_two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ void kf_fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// exp(y), y = yh + yl in [-20, 0], to about 2^-46 relative, on the FP32 pipes:
// Tang's table-driven method (ACM TOMS 15(2), 1989).  y = n ln2/64 + r with n
// an integer and |r| <= ln2/128, ln2/64 split Cody-Waite style into L1 (12
// significant bits, so n L1 is exact for |n| < 4096) + L2 + L3;
// exp(y) = 2^(n >> 6) 2^((n & 63)/64) (1 + q), q = r + r^2/2 + ... + r^5/120
// (the r^6 term is below 4e-17).  tab[j] = 2^(j/64) as a double-float pair.
__device__ __forceinline__ float2 kf_exp_df(float yh, float yl, const float2* __restrict__ tab) {
  const float kInvL = 0x1.715476p+6f;  // 64 / ln 2
  const float L1 = 0x1.62ep-7f, L2 = 0x1.0bfbe8p-21f, L3 = 0x1.cf79acp-46f;
  const float n = rintf(__fmul_rn(yh, kInvL));
  const float t1 = fmaf(-n, L1, yh);  // exact: yh and n L1 agree in their leading bits
  float p, pe, s, e, s2, e2, rh, rl;
  kf_two_prod(n, L2, p, pe);          // n L2 = p + pe
  kf_two_sum(t1, -p, s, e);           // t1 - p = s + e
  kf_two_sum(s, yl, s2, e2);
  e2 = __fadd_rn(e2, __fsub_rn(__fsub_rn(e, pe), __fmul_rn(n, L3)));
  kf_fast_two_sum(s2, e2, rh, rl);    // r = rh + rl
  float sq, sqe;
  kf_two_prod(rh, rh, sq, sqe);
  sqe = fmaf(2.f * rh, rl, sqe);      // r^2 = sq + sqe
  const float tail = __fmul_rn(__fmul_rn(sq, rh), fmaf(rh, fmaf(rh, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f));
  float a, ae;
  kf_two_sum(rh, 0.5f * sq, a, ae);   // q = a + ae
  ae = __fadd_rn(ae, __fadd_rn(rl, __fadd_rn(0.5f * sqe, tail)));
  const int ni = __float2int_rn(n);
  const float2 T = __ldg(tab + (ni & 63));
  float u, ue, v, ve;
  kf_two_prod(T.x, a, u, ue);         // T q = u + ue
  ue = fmaf(T.x, ae, fmaf(T.y, a, ue));
  kf_two_sum(T.x, u, v, ve);          // T + T q
  ve = __fadd_rn(ve, __fadd_rn(T.y, ue));
  float hi, lo;
  kf_fast_two_sum(v, ve, hi, lo);
  const float sc = __int_as_float(((ni >> 6) + 127) << 23);  // 2^(n >> 6), exact
  return make_float2(__fmul_rn(hi, sc), __fmul_rn(lo, sc));
}

// squared distance as a double-float pair (ah, al); y's coordinates are ys apart
__device__ __forceinline__ void kf_sqdist_df2(const float* __restrict__ xh, const float* __restrict__ xl,
                                              const float* __restrict__ yh, const float* __restrict__ yl, int ys,
                                              int d, float& ah, float& al) {
  ah = 0.f;
  al = 0.f;
  for (int k = 0; k < d; ++k) {
    float th, te;
    kf_two_sum(xh[k], -yh[k * ys], th, te);
    const float tl = te + (xl[k] - yl[k * ys]);
    const float p = __fmul_rn(th, th);
    const float q = fmaf(th, th, -p) + 2.f * th * tl;
    float sh, se;
    kf_two_sum(ah, p, sh, se);
    se = __fadd_rn(se, __fadd_rn(al, q));
    ah = __fadd_rn(sh, se);
    al = __fsub_rn(se, __fsub_rn(ah, sh));
  }
}

// Kernel entry exp(c |x - y|^2) as a double-float pair, to about 2^-46
// relative with no FP64 arithmetic, from the squared distance ah + al
// (kf_sqdist_df2 of coordinates held as pairs X32 + X32lo) and c = ch + cl.
// Arguments below -20 (entries below 2e-9) take the FP32 exponential, whose
// absolute error there is below 1e-16.
__device__ __forceinline__ float2 kf_kern_from_df(float ah, float al, float ch, float cl,
                                                  const float2* __restrict__ tab) {
  float y, ye;
  kf_two_prod(ah, ch, y, ye);
  ye = fmaf(ah, cl, fmaf(al, ch, ye));
  float zh, zl;
  kf_fast_two_sum(y, ye, zh, zl);
  if (zh < -20.f) return make_float2(__expf(zh), 0.f);
  return kf_exp_df(zh, zl, tab);
}

// (sh, sl) += (ah + al)(bh + bl) in double-float arithmetic (about 2^-46 relative)
__device__ __forceinline__ void kf_df_fma(float ah, float al, float bh, float bl, float& sh, float& sl) {
  float p, e, s, t;
  kf_two_prod(ah, bh, p, e);
  e = fmaf(ah, bl, fmaf(al, bh, e));
  kf_two_sum(sh, p, s, t);
  t = __fadd_rn(t, __fadd_rn(sl, e));
  kf_fast_two_sum(s, t, sh, sl);
}

// y <- y - s for double-float pairs (y as hi, lo; s as hi, lo)
__device__ __forceinline__ void kf_df_sub(float& yh, float& yl, float sh, float sl) {
  float t, e;
  kf_two_sum(yh, -sh, t, e);
  e = __fadd_rn(e, __fsub_rn(yl, sl));
  kf_fast_two_sum(t, e, yh, yl);
}

// a double as a double-float pair (two conversions, off the hot loops)
__device__ __forceinline__ float2 kf_split_df(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}



template <typename T> struct kf_kern;
template <> struct kf_kern<double> {
  static __device__ __forceinline__ double eval(const double* X64, const float*, int64_t i, int64_t j, int d, double c) {
    return kf_kern64(X64 + i * d, X64 + j * d, d, c);
  }
};
template <> struct kf_kern<float> {
  static __device__ __forceinline__ float eval(const double*, const float* X32, int64_t i, int64_t j, int d, double c) {
    return kf_kern32(X32 + i * d, X32 + j * d, d, (float)c);
  }
};

__host__ __device__ inline int kf_level_of(int a) { return 31 - __builtin_clz((unsigned)a); }

// splitmix64 (Steele, Lea, Flood 2014): golden-ratio increment then the
// xor-shift-multiply finalizer; used as a counter-based generator.
__host__ __device__ inline uint64_t kf_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// ---- launchers implemented in the .cu files ------------------------------------
struct kf_skel_scratch {
  double* A = nullptr;
  int32_t* samp = nullptr;
  int32_t* nsamp = nullptr;
  size_t a_elems = 0;
};
kf_status kf_tree_build_device(kf_tree* t, cudaStream_t s);
kf_status kf_skeletonize_device(kf_factor* f, cudaStream_t s);
kf_status kf_skel_begin(kf_factor* f, kf_skel_scratch* sc, cudaStream_t s);
kf_status kf_skel_level(kf_factor* f, int l, kf_skel_scratch* sc, cudaStream_t s);
void kf_skel_end(kf_factor* f, kf_skel_scratch* sc, cudaStream_t s);
kf_status kf_factorize_device(kf_factor* f, cudaStream_t s);
// factorization in steps: leaves (after skeleton level D), then level l (after
// skeleton levels l + 1 and l); Tm is the T = Z^-1 P_c scratch of
// kf_factor_tm_elems() doubles.
size_t kf_factor_tm_elems(const kf_factor* f);
size_t kf_factor_tm_bytes(const kf_factor* f);
// the split-K partials of the Z-block products inside that scratch (cap bytes)
void* kf_factor_zparts(const kf_factor* f, double* Tm, size_t* cap);
// part 0: all; 1: leaf blocks and their Cholesky factors; 2: P^ = A^-1 P
kf_status kf_factorize_leaves(kf_factor* f, cudaStream_t s, bool with_k64, int part);
kf_status kf_leaf_k64_launch(kf_factor* f, cudaStream_t s);
// Pleaf and Pc as double-float pairs (mixed path with the FP64-accurate operator)
kf_status kf_split_p_df(kf_factor* f, cudaStream_t s);
// the LU factors of the levels without Z^-1 as double-float pairs (mixed path)
kf_status kf_split_z_df(kf_factor* f, cudaStream_t s);
kf_status kf_factorize_level(kf_factor* f, int l, double* Tm, cudaStream_t s);
kf_status kf_factorize_level_v(kf_factor* f, int l, cudaStream_t s);
kf_status kf_factorize_level_z(kf_factor* f, int l, double* Tm, cudaStream_t s);
// skeletonize and factorize with the two interleaved on two streams
kf_status kf_skel_factorize_pipelined(kf_factor* f, cudaStream_t s);
kf_status kf_solve_device(kf_factor* f, double* W, int64_t nrhs, int transpose, cudaStream_t s);
kf_status kf_matvec_device(kf_factor* f, const double* Xin, double* Y, int64_t nrhs, int deriv, cudaStream_t s);
// Z^-1 of the nodes of level l (l <= f->zinv_top) from their LU; stream order
// after the level's LU.
kf_status kf_z_inverse_level(kf_factor* f, int l, cudaStream_t s);

// y = (lambda I + K~)^T x (tree order, N x nrhs FP64), with the same operator
// data as kf_matvec_device (FP64-accurate on the mixed path when it is stored).
kf_status kf_matvec_transpose_device(kf_factor* f, const double* Xin, double* Y, int64_t nrhs, cudaStream_t s);

// ---- hybrid level-restricted solver (hybrid.cu) ------------------------------------
// After the frontier subtrees are factorized: offsets of the frontier ranks,
// the coupling rows Vh, the reduced system I + VW and its LU (stream order).
kf_status kf_hybrid_reduced_system(kf_factor* f, cudaStream_t s);
// W (tree order, N x k FP64, point-major) <- W - W_L (I + VW)^-1 V W: the
// top of Algorithm 6, applied after the frontier subtrees' direct solves.
kf_status kf_hybrid_top_solve(kf_factor* f, double* W, int64_t k, cudaStream_t s);
// G (per node, (node * s_max + q) * k + c) of the frontier nodes <- V x: the
// coupling between frontier subtrees in the operator D + UV (Algorithm 8).
kf_status kf_hybrid_top_apply(kf_factor* f, const double* x, double* G, int64_t k, cudaStream_t s);
// launchers of kernels that live with the direct solver's reduced systems
// (factor.cu, solve.cu), for the one synthetic node of the hybrid system
kf_status kf_z_factor_one_launch(const int32_t* rank, int ldz, double* Z, int32_t* piv, int32_t* status,
                                 double* pivr, cudaStream_t s);
kf_status kf_zsolve_one_launch(const int32_t* rank, int ldz, const double* ZLU, const int32_t* piv, const double* in,
                               double* out, int k, cudaStream_t s);
// W -= rows of P^ (level l, type of the factor) times the per-node vector V
kf_status kf_rowupd_level_launch(kf_factor* f, int l, const double* V, double* W, int64_t k, cudaStream_t s);

// ---- near-field sampling (tree.cu, knn.cu) ------------------------------------------
// order of the tree positions under randomized projection tree tidx of depth Dk
kf_status kf_rp_order(kf_tree* t, int tidx, int Dk, uint64_t seed, int64_t* ord, cudaStream_t s);
// f->nbr and the node lists f->near_* from the tree (stream order)
kf_status kf_near_field_lists(kf_factor* f, cudaStream_t s);

// whether the Z off-diagonal blocks evaluate their kernel entries inside the
// tcgen05 product (mixed path) instead of reading the stored V blocks
// offset (elements) of P^ of level l (1..D) in f->Phat: N x s_max per level, or
// with memory-lean W the leaves in slot 0 and levels D-1, D-2, .. alternating
// in slots 1 and 2
inline int64_t kf_phat_level_off(const kf_factor* f, int l) {
  const int D = f->t->D;
  const int64_t per = f->t->N * (int64_t)f->s_max;
  if (!f->w_lean) return (int64_t)(l - 1) * per;
  return (l == D ? 0 : 1 + ((D - 1 - l) & 1)) * per;
}

// offset (elements) of the V blocks of level l (1..D) in f->VT: N x s_max per
// level, or, when the sweeps evaluate V on the fly (KF_V_RECOMPUTE), three
// slots used in turn (level l needs the V blocks of level l + 1 only)
inline int64_t kf_vt_level_off(const kf_factor* f, int l) {
  const int64_t per = f->t->N * (int64_t)f->s_max;
  return f->vstore == KF_V_RECOMPUTE ? (int64_t)(l % 3) * per : (int64_t)(l - 1) * per;
}

inline bool kf_zoff_fused(const kf_factor* f) { return f->prec == KF_PREC_MIXED && f->use_tc && f->fused_zoff; }
