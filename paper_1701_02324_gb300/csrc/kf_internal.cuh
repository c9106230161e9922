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
  int64_t* perm = nullptr;
  std::vector<std::pair<void*, size_t>> allocs;
};

struct kf_factor {
  kf_tree* t = nullptr;
  kf_ctx* ctx = nullptr;
  double h = 1, lambda = 0, tau = 0, c_exp = 0;
  int32_t s_max = 0, n_samp = 0, cmax = 0, prec = 0, vstore = 0, sync_errors = 0;
  int32_t use_tc = 1;  // mixed path: tcgen05 products (0: CUDA-core FP32)
  int32_t use_cluster_qr = 1;  // upper tree levels: cluster QR in distributed shared memory
  int32_t fp64_op = 0;  // keep FP64 operator data (VT64, K64)
  int32_t gmres_m = 0;  // refinement: 0 = Richardson, m > 0 = GMRES(m)
  int32_t refine_user = 0;  // refinement explicitly requested (enables it on the FP64 path)
  double* VT64 = nullptr;  // mixed path with fp64_op: D x N x s_max FP64 V blocks
  double* K64 = nullptr;   // fp64_op: leaf blocks lambda-free K_aa, leaf_max^2 each
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
  int32_t* status = nullptr;
  double* pivr = nullptr;  // per node: smallest / largest pivot of its leaf Cholesky or Z LU
  std::vector<std::pair<void*, size_t>> allocs;
  size_t tsize() const { return prec == KF_PREC_FP64 ? 8 : 4; }
};

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

// Squared distance in double-float arithmetic on the FP32 pipes: every
// coordinate is held as hi + lo (hi = fp32(x), lo = fp32(x - hi)); the
// difference, its square and the running sum carry an error term through
// exact two-sum / two-product steps, giving about 44 significant bits.
__device__ __forceinline__ void kf_two_sum(float a, float b, float& s, float& e) {
  // round-to-nearest intrinsics: never contracted, so the error term is exact
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ double kf_sqdist_df(const float* __restrict__ xh, const float* __restrict__ xl,
                                              const float* __restrict__ yh, const float* __restrict__ yl, int d) {
  float ah = 0.f, al = 0.f;
  for (int k = 0; k < d; ++k) {
    float th, te;
    kf_two_sum(xh[k], -yh[k], th, te);
    const float tl = te + (xl[k] - yl[k]);
    const float p = __fmul_rn(th, th);
    const float q = fmaf(th, th, -p) + 2.f * th * tl;  // th^2 - p exactly, plus the cross term
    float sh, se;
    kf_two_sum(ah, p, sh, se);
    se = __fadd_rn(se, __fadd_rn(al, q));
    ah = __fadd_rn(sh, se);
    al = __fsub_rn(se, __fsub_rn(ah, sh));
  }
  return (double)ah + (double)al;
}

// FP64-accurate kernel entry at FP32 cost for the small ones: entries below
// 2^-24 are taken from the FP32 evaluation (their absolute error stays below
// about 1e-12); larger ones take the double-float distance and an FP64 exp.
__device__ __forceinline__ double kf_kern_hybrid(const float* X32, const float* X32lo, int64_t i, int64_t j, int d,
                                                 double c_exp) {
  const float k32 = kf_kern32(X32 + i * d, X32 + j * d, d, (float)c_exp);
  if (k32 < 5.9604645e-8f) return (double)k32;
  return exp(kf_sqdist_df(X32 + i * d, X32lo + i * d, X32 + j * d, X32lo + j * d, d) * c_exp);
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
kf_status kf_factorize_leaves(kf_factor* f, cudaStream_t s);
kf_status kf_factorize_level(kf_factor* f, int l, double* Tm, cudaStream_t s);
// skeletonize and factorize with the two interleaved on two streams
kf_status kf_skel_factorize_pipelined(kf_factor* f, cudaStream_t s);
kf_status kf_solve_device(kf_factor* f, double* W, int64_t nrhs, int transpose, cudaStream_t s);
kf_status kf_matvec_device(kf_factor* f, const double* Xin, double* Y, int64_t nrhs, int deriv, cudaStream_t s);
