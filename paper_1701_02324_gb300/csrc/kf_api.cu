// kf_api.cu -- the C ABI declared in include/kf.h: argument checks, device
// memory, staging of host or device buffers, the permutation into tree order
// and the mixed-precision refinement loop around the solve.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "kf_internal.cuh"
#include "prof.cuh"

kf_status kf_to_f64_launch(const float* in, double* out, int64_t n, cudaStream_t s);
kf_status kf_to_f32_launch(const double* in, float* out, int64_t n, cudaStream_t s);
kf_status kf_check_finite_launch(const double* x, int64_t n, int32_t* bad, cudaStream_t s);
kf_status kf_split_lo_launch(const double* in, const float* hi, float* lo, int64_t n, cudaStream_t s);

static thread_local std::string g_err;

kf_status kf_set_err(kf_ctx* c, kf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  g_err = buf;
  return s;
}

void* kf_ctx::dalloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (has_alloc && !capturing) return alloc.alloc(bytes, (void*)s, alloc.user);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void kf_ctx::dfree(void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  if (has_alloc && !capturing) alloc.free(p, bytes, (void*)s, alloc.user);
  else cudaFreeAsync(p, s);
}

namespace {

inline int grid_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// B (original order, column-major, ld, F32/F64) -> W (tree order, N x k row-major, FP64)
__global__ void k_gather_in(const void* __restrict__ B, int dtype, int64_t ld, const int64_t* __restrict__ perm,
                            int64_t N, int64_t k, double* __restrict__ W) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * k; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / k, r = e % k;
    int64_t src = perm[i] + r * ld;
    W[e] = dtype == KF_F64 ? ((const double*)B)[src] : (double)((const float*)B)[src];
  }
}
__global__ void k_scatter_out(const double* __restrict__ W, const int64_t* __restrict__ perm, int64_t N, int64_t k,
                              void* __restrict__ X, int dtype, int64_t ld) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * k; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / k, r = e % k;
    int64_t dst = perm[i] + r * ld;
    if (dtype == KF_F64) ((double*)X)[dst] = W[e];
    else ((float*)X)[dst] = (float)W[e];
  }
}
// ---- deterministic reductions ------------------------------------------------------
// A fixed grid of kRedBlocks blocks: every block forms its partial sums in a
// fixed order (thread-strided sums, then a fixed tree in shared memory) and
// writes them to part[block][e]; k_sum_parts adds the partials in block order.
// The results do not depend on the order in which blocks run.
constexpr int kRedBlocks = 256, kRedThreads = 256;

__device__ __forceinline__ double block_tree_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}
// part[block][r] = the block's share of sum_i W[i][r]^2 (W: N x k point-major)
__global__ void __launch_bounds__(kRedThreads) k_colnorm2_part(const double* __restrict__ W, int64_t N, int64_t k,
                                                                double* __restrict__ part) {
  __shared__ double sh[kRedThreads];
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = 0; r < k; ++r) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += T) acc += W[i * k + r] * W[i * k + r];
    const double t = block_tree_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x * k + r] = t;
  }
}
__global__ void __launch_bounds__(kRedThreads) k_dot_part(const double* __restrict__ a, const double* __restrict__ b,
                                                           int64_t n, double* __restrict__ part) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  const double t = block_tree_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}
// out[e] = sum over blocks b (in order) of part[b][e]
__global__ void k_sum_parts(const double* __restrict__ part, int nblk, int64_t len, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    double sum = 0.0;
    for (int b = 0; b < nblk; ++b) sum += part[(int64_t)b * len + e];
    out[e] = sum;
  }
}
// host side of the deterministic reductions (partials from the context's allocator)
static kf_status red_colnorm2(kf_ctx* c, const double* W, int64_t N, int64_t k, double* out, cudaStream_t s) {
  const size_t pb = sizeof(double) * kRedBlocks * (size_t)k;
  double* part = (double*)c->dalloc(pb, s);
  if (!part) return kf_set_err(c, KF_ENOMEM, "reduction: allocation failed");
  KF_PHASE(KF_PH_MISC, s, k_colnorm2_part<<<kRedBlocks, kRedThreads, 0, s>>>(W, N, k, part));
  KF_PHASE(KF_PH_MISC, s, k_sum_parts<<<(unsigned)std::min<int64_t>(64, (k + 255) / 256), 256, 0, s>>>(
                              part, kRedBlocks, k, out));
  c->dfree(part, pb, s);
  return KF_OK;
}
static kf_status red_dot(kf_ctx* c, const double* a, const double* b, int64_t n, double* out, cudaStream_t s) {
  const size_t pb = sizeof(double) * kRedBlocks;
  double* part = (double*)c->dalloc(pb, s);
  if (!part) return kf_set_err(c, KF_ENOMEM, "reduction: allocation failed");
  KF_PHASE(KF_PH_MISC, s, k_dot_part<<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, part));
  KF_PHASE(KF_PH_MISC, s, k_sum_parts<<<1, 256, 0, s>>>(part, kRedBlocks, 1, out));
  c->dfree(part, pb, s);
  return KF_OK;
}

// r = b - y
__global__ void k_sub(const double* __restrict__ b, const double* __restrict__ y, double* __restrict__ r, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - y[i];
}
__global__ void k_add(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += d[i];
}

// ---- GMRES helpers ----------------------------------------------------------------
// Dot products, updates and scalings of Krylov vectors for k columns at once.
// k columns stored point-major (element (i, c) at i * k + c), so that k
// independent GMRES iterations share every launch:
// part[block][j][c] = the block's share of sum_i V_j[i * k + c] w[i * k + c],
// j < J.  Each thread keeps one column (the grid stride is a multiple of k);
// a block adds its threads' sums per column in thread order (shared memory).
__global__ void __launch_bounds__(kRedThreads) k_multidot_part(const double* __restrict__ V, int64_t ldv, int J,
                                                                const double* __restrict__ w, int64_t n, int k,
                                                                double* __restrict__ part) {
  __shared__ double sh[kRedThreads];
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t stride = (T / k) * k;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int j = 0; j < J; ++j) {
    double acc = 0.0;
    if (gid < stride) {
      const double* v = V + (int64_t)j * ldv;
      for (int64_t e = gid; e < n * k; e += stride) acc = fma(v[e], w[e], acc);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int q = threadIdx.x; q < k; q += blockDim.x) {
      double sum = 0.0;
      for (int t = 0; t < (int)blockDim.x; ++t)
        if ((blockIdx.x * (int64_t)blockDim.x + t) % k == q && blockIdx.x * (int64_t)blockDim.x + t < stride)
          sum += sh[t];
      part[((int64_t)blockIdx.x * J + j) * k + q] = sum;
    }
    __syncthreads();
  }
}
// h[j * k + c] = sum_i V_j[i * k + c] w[i * k + c], j < J (deterministic)
static kf_status red_multidot(kf_ctx* c, const double* V, int64_t ldv, int J, const double* w, int64_t n, int k,
                              double* h, cudaStream_t s) {
  const size_t pb = sizeof(double) * kRedBlocks * (size_t)J * k;
  double* part = (double*)c->dalloc(pb, s);
  if (!part) return kf_set_err(c, KF_ENOMEM, "reduction: allocation failed");
  KF_PHASE(KF_PH_MISC, s, k_multidot_part<<<kRedBlocks, kRedThreads, 0, s>>>(V, ldv, J, w, n, k, part));
  const int64_t len = (int64_t)J * k;
  KF_PHASE(KF_PH_MISC, s, k_sum_parts<<<(unsigned)std::min<int64_t>(64, (len + 255) / 256), 256, 0, s>>>(
                              part, kRedBlocks, len, h));
  c->dfree(part, pb, s);
  return KF_OK;
}
// w[i * k + c] -= sum_j h[j * k + c] V_j[i * k + c]
__global__ void k_multiaxpy_k(const double* __restrict__ V, int64_t ldv, int J, const double* __restrict__ h,
                              double* __restrict__ w, int64_t n, int k) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % k);
    double acc = w[e];
    for (int j = 0; j < J; ++j) acc = fma(-h[(int64_t)j * k + c], V[(int64_t)j * ldv + e], acc);
    w[e] = acc;
  }
}
// x[i * k + c] += sum_j y[j * k + c] Z_j[i * k + c]
__global__ void k_zupdate_k(const double* __restrict__ Z, int64_t ldz, int J, const double* __restrict__ y,
                            double* __restrict__ x, int64_t n, int k) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % k);
    double acc = x[e];
    for (int j = 0; j < J; ++j) acc = fma(y[(int64_t)j * k + c], Z[(int64_t)j * ldz + e], acc);
    x[e] = acc;
  }
}
// b[i * k + c] = a[i * k + c] * sc[c]
__global__ void k_scale_cols(const double* __restrict__ a, const double* __restrict__ sc, double* __restrict__ b,
                             int64_t n, int k) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = a[e] * sc[e % k];
}

struct Staged {
  kf_ctx* c;
  void* dev = nullptr;
  size_t bytes = 0;
  bool owned = false;
  cudaStream_t s;
  ~Staged() {
    if (owned) c->dfree(dev, bytes, s);
  }
};

// Make a device view of a caller buffer of `bytes` bytes (copy in if host).
kf_status stage_in(kf_ctx* c, const void* p, size_t bytes, cudaStream_t s, Staged& out) {
  out.c = c;
  out.s = s;
  out.bytes = bytes;
  if (is_device_ptr(p)) {
    out.dev = const_cast<void*>(p);
    return KF_OK;
  }
  out.dev = c->dalloc(bytes, s);
  if (!out.dev) return kf_set_err(c, KF_ENOMEM, "staging: allocation of %zu bytes failed", bytes);
  out.owned = true;
  KF_CUDA(c, cudaMemcpyAsync(out.dev, p, bytes, cudaMemcpyHostToDevice, s));
  return KF_OK;
}

template <typename T>
T* falloc(kf_factor* f, size_t n, cudaStream_t s) {
  size_t b = sizeof(T) * n;
  void* p = f->ctx->dalloc(b, s);
  if (p) {
    f->allocs.push_back({p, b});
    cudaMemsetAsync(p, 0, b, s);
  }
  return (T*)p;
}

kf_status alloc_factor(kf_tree* t, double h, double lambda, double tau, int32_t s_max, const kf_opts* opts,
                       cudaStream_t s, kf_factor** out) {
  kf_ctx* c = t->ctx;
  if (!(h > 0.0) || !isfinite(h)) return kf_set_err(c, KF_EINVAL, "h must be > 0 (got %g)", h);
  if (!(lambda >= 0.0) || !isfinite(lambda)) return kf_set_err(c, KF_EINVAL, "lambda must be >= 0 (got %g)", lambda);
  if (!(tau >= 0.0) || !isfinite(tau)) return kf_set_err(c, KF_EINVAL, "tau must be >= 0 (got %g)", tau);
  if (s_max < 1 || s_max > KF_MAX_SMAX) return kf_set_err(c, KF_EINVAL, "s_max must be in [1, %d]", KF_MAX_SMAX);
  kf_factor* f = new kf_factor();
  f->t = t;
  f->ctx = c;
  f->h = h;
  f->lambda = lambda;
  f->tau = tau;
  f->c_exp = -0.5 / (h * h);
  f->c_exp_hi = (float)f->c_exp;
  f->c_exp_lo = (float)(f->c_exp - (double)f->c_exp_hi);
  f->s_max = s_max;
  f->n_samp = 2 * s_max;
  // defaults: the mixed path refines with GMRES(20) against an FP64-accurate
  // operator; the FP64 path solves directly
  const int32_t prec0 = opts ? opts->precision : KF_PREC_FP64;
  f->fp64_op = prec0 == KF_PREC_MIXED ? 1 : 0;
  f->gmres_m = 50;
  f->refine_max_iter = 100;
  if (opts) {
    f->prec = opts->precision;
    if (opts->n_samp > 0) f->n_samp = opts->n_samp;
    if (opts->seed) f->seed = opts->seed;
    f->vstore = opts->v_storage;
    f->sync_errors = opts->sync_errors;
    if (opts->refine_tol > 0) f->refine_tol = opts->refine_tol;
    if (opts->refine_max_iter > 0) f->refine_max_iter = opts->refine_max_iter;
    f->refine_user = opts->refine_max_iter > 0 ? 1 : 0;
    if (opts->refine_max_iter < 0) f->refine_max_iter = 0;
    f->use_tc = opts->no_tensor_cores ? 0 : 1;
    if (opts->fp64_operator != 0) f->fp64_op = opts->fp64_operator > 0 ? 1 : 0;
    if (opts->gmres_restart != 0) f->gmres_m = opts->gmres_restart > 0 ? std::min(opts->gmres_restart, 64) : 0;
    if (opts->no_cluster_kernels) f->use_cluster_qr = f->use_cluster_lu = 0;
    if (opts->zinv_max_nodes != 0) f->zinv_max_nodes = opts->zinv_max_nodes > 0 ? opts->zinv_max_nodes : -1;
    f->hyb_L = opts->hybrid_level;
    f->knn_kappa = opts->knn_kappa;
    f->fused_zoff = opts->zoff_fused ? 1 : 0;
    f->w_lean = opts->w_recompute ? 1 : 0;
    f->use_oz = opts->tc_operator > 0 ? 1 : 0;
    if (opts->knn_trees > 0) f->knn_trees = opts->knn_trees;
    if (opts->knn_leaf > 0) f->knn_leaf = opts->knn_leaf;
    if (opts->tc_tile_n == 128) f->tc_bn = 128;
    else if (opts->tc_tile_n != 0 && opts->tc_tile_n != 256) {
      delete f;
      return kf_set_err(c, KF_EINVAL, "tc_tile_n must be 128 or 256");
    }
  }
  if (f->prec != KF_PREC_FP64 && f->prec != KF_PREC_MIXED) {
    delete f;
    return kf_set_err(c, KF_EINVAL, "unknown precision %d", opts ? opts->precision : -1);
  }
  if (f->vstore != KF_V_STORED && f->vstore != KF_V_RECOMPUTE) {
    delete f;
    return kf_set_err(c, KF_EINVAL, "unknown v_storage");
  }
  if (f->n_samp > 1024) {
    delete f;
    return kf_set_err(c, KF_EINVAL, "n_samp must be <= 1024");
  }
  if (f->knn_kappa < 0 || f->knn_kappa > 32 || f->knn_trees < 1 || f->knn_trees > 64 || f->knn_leaf < 2 ||
      f->knn_leaf > 1024) {
    delete f;
    return kf_set_err(c, KF_EINVAL, "near-field sampling: knn_kappa in 0..32, knn_trees in 1..64, knn_leaf in "
                      "2..1024");
  }
  if (f->knn_kappa > 0 && (int64_t)t->leaf_max * f->knn_kappa > 16384) {
    delete f;
    return kf_set_err(c, KF_EUNSUPPORTED, "near-field sampling: leaf size x knn_kappa = %lld exceeds 16384",
                      (long long)t->leaf_max * f->knn_kappa);
  }
  if (f->hyb_L < 0 || f->hyb_L > t->D) {
    const int Lbad = f->hyb_L;
    delete f;
    return kf_set_err(c, KF_EINVAL, "hybrid_level %d outside [0, %d] (the tree depth)", Lbad, t->D);
  }
  if (f->hyb_L > 0 && f->w_lean) {
    delete f;
    return kf_set_err(c, KF_EUNSUPPORTED, "memory-lean W (w_recompute) is not available with the hybrid solver");
  }
  if (f->hyb_L > 0 && ((int64_t)s_max << f->hyb_L) > 2 * KF_MAX_SMAX) {
    const int Lbad = f->hyb_L;
    delete f;
    return kf_set_err(c, KF_EUNSUPPORTED, "hybrid reduced system of up to 2^%d * s_max = %lld rows; at most %d "
                      "are supported", Lbad, (long long)s_max << Lbad, 2 * KF_MAX_SMAX);
  }
  const int64_t N = t->N;
  const int D = t->D;
  f->cmax = std::max(t->leaf_max, 2 * s_max);
  const size_t nn = (size_t)t->nnodes + 1;
  const size_t ts = f->tsize();
  f->rank = falloc<int32_t>(f, nn, s);
  f->skel = falloc<int32_t>(f, nn * s_max, s);
  f->status = falloc<int32_t>(f, 1, s);
  f->pivr = falloc<double>(f, nn, s);
  f->Pleaf = falloc<double>(f, (size_t)N * s_max, s);
  if (D > 0) {
    f->Pc = falloc<double>(f, (size_t)(1 << D) * 2 * s_max * s_max, s);
    f->ZLU = falloc<double>(f, (size_t)(1 << D) * 4 * s_max * s_max, s);
    f->Zpiv = falloc<int32_t>(f, (size_t)(1 << D) * 2 * s_max, s);
    // levels 0..zinv_top (at most zinv_max_nodes nodes each) keep Z^-1
    int zt = f->zinv_max_nodes >= 1 ? 0 : -1;
    while (zt >= 0 && zt + 1 <= D - 1 && (1 << (zt + 1)) <= f->zinv_max_nodes) ++zt;
    f->zinv_top = zt;
    if (zt >= 0) f->Zinv = falloc<double>(f, (size_t)(2 << zt) * 4 * s_max * s_max, s);
    if (f->prec == KF_PREC_MIXED && zt + 1 <= D - 1) {
      f->ZLUdf = falloc<float2>(f, (size_t)(1 << D) * 4 * s_max * s_max, s);
      if (!f->ZLUdf) {
        kf_factor_free(f);
        return kf_set_err(c, KF_ENOMEM, "factorize: device allocation of the reduced systems' pairs failed");
      }
    }
    f->Phat = falloc<char>(f, (size_t)(f->w_lean ? std::min(D, 3) : D) * N * s_max * ts, s);
    if (f->w_lean) f->Tw = falloc<char>(f, (size_t)(1 << D) * 2 * s_max * s_max * ts, s);
    f->VT = falloc<char>(f, (size_t)(f->vstore == KF_V_RECOMPUTE ? std::min(D + 1, 3) : D) * N * s_max * ts, s);
  }
  f->L = falloc<char>(f, (size_t)(1 << D) * t->leaf_max * t->leaf_max * ts, s);
  if (f->fp64_op) {
    f->Kdf = falloc<float2>(f, (size_t)(1 << D) * t->leaf_max * t->leaf_max, s);
    if (D > 0 && f->prec != KF_PREC_FP64) {
      f->VTdf = falloc<float2>(f, (size_t)D * N * s_max, s);
      f->Pleafdf = falloc<float2>(f, (size_t)N * s_max, s);
      f->Pcdf = falloc<float2>(f, (size_t)(1 << D) * 2 * s_max * s_max, s);
    }
    if (!f->Kdf || (D > 0 && f->prec != KF_PREC_FP64 && (!f->VTdf || !f->Pleafdf || !f->Pcdf))) {
      kf_factor_free(f);
      return kf_set_err(c, KF_ENOMEM, "factorize: device allocation of the FP64 operator failed");
    }
    if (f->use_oz && f->use_tc && f->VTdf) {  // BF16 digits of the V blocks (tc_operator)
      kf_status zs = kf_oz_alloc(f, s);
      if (zs != KF_OK) {
        kf_factor_free(f);
        return zs;
      }
    }
  }
  if (f->prec == KF_PREC_MIXED && f->use_tc) {  // leaf factorization on the tensor cores
    const size_t npan = ((size_t)t->leaf_max + 127) / 128;
    f->Dinv = falloc<float>(f, ((size_t)1 << D) * npan * 128 * 128, s);
    f->ltrack = falloc<double>(f, ((size_t)1 << D) * 2, s);
    if (!f->Dinv || !f->ltrack) {
      kf_factor_free(f);
      return kf_set_err(c, KF_ENOMEM, "factorize: device allocation of the leaf panels failed");
    }
  }
  if (f->knn_kappa > 0) {
    f->near_cap = f->n_samp / 2;
    f->nbr = falloc<int32_t>(f, (size_t)N * f->knn_kappa, s);
    f->near_pos = falloc<int32_t>(f, nn * (size_t)std::max(1, f->near_cap), s);
    f->near_cnt = falloc<int32_t>(f, nn * (size_t)std::max(1, f->near_cap), s);
    f->near_len = falloc<int32_t>(f, nn, s);
    if (!f->nbr || !f->near_pos || !f->near_cnt || !f->near_len) {
      kf_factor_free(f);
      return kf_set_err(c, KF_ENOMEM, "factorize: device allocation of the near-field lists failed");
    }
  }
  if (f->hyb_L > 0) {
    const int nA = 1 << f->hyb_L;
    f->hyb_scap = s_max << f->hyb_L;
    const size_t sc = (size_t)f->hyb_scap;
    f->Vh = falloc<double>(f, (size_t)nA * s_max * N, s);
    f->HM = falloc<double>(f, 2 * sc * sc, s);
    f->Hpiv = falloc<int32_t>(f, 2 * sc, s);
    f->Hrank = falloc<int32_t>(f, 4, s);
    f->Hoff = falloc<int32_t>(f, (size_t)nA + 1, s);
    f->Hpivr = falloc<double>(f, 2, s);
    if (!f->Vh || !f->HM || !f->Hpiv || !f->Hrank || !f->Hoff || !f->Hpivr) {
      kf_factor_free(f);
      return kf_set_err(c, KF_ENOMEM, "factorize: device allocation of the hybrid reduced system failed");
    }
  }
  bool ok = f->rank && f->skel && f->status && f->pivr && f->Pleaf && f->L &&
            (D == 0 || (f->Pc && f->ZLU && f->Zpiv && (f->Zinv || f->zinv_top < 0) && f->Phat && f->VT &&
                        (f->Tw || !f->w_lean)));
  if (!ok) {
    kf_factor_free(f);
    return kf_set_err(c, KF_ENOMEM, "factorize: device allocation failed");
  }
  *out = f;
  return KF_OK;
}

kf_status read_status(kf_factor* f, cudaStream_t s) {
  int32_t st = 0;
  KF_CUDA(f->ctx, cudaMemcpyAsync(&st, f->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaStreamSynchronize(s));
  if (st & KF_DEV_TIMEOUT) return kf_set_err(f->ctx, KF_ETIMEOUT, "a bounded device wait ran out");
  if (st & KF_DEV_ILLCOND)
    return kf_set_err(f->ctx, KF_EILLCOND, "ill-conditioned leaf block or reduced system (small pivot)");
  return KF_OK;
}

}  // namespace

extern "C" {

const char* kf_status_string(kf_status s) {
  switch (s) {
    case KF_OK: return "KF_OK";
    case KF_EINVAL: return "KF_EINVAL";
    case KF_ENOMEM: return "KF_ENOMEM";
    case KF_ECUDA: return "KF_ECUDA";
    case KF_EILLCOND: return "KF_EILLCOND";
    case KF_ENOTCONV: return "KF_ENOTCONV";
    case KF_ETIMEOUT: return "KF_ETIMEOUT";
    case KF_EUNSUPPORTED: return "KF_EUNSUPPORTED";
  }
  return "KF_UNKNOWN";
}

kf_status kf_create(kf_ctx** out, const kf_alloc* alloc) {
  if (!out) return KF_EINVAL;
  kf_ctx* c = new kf_ctx();
  if (alloc) {
    if (!alloc->alloc || !alloc->free) {
      delete c;
      return kf_set_err(nullptr, KF_EINVAL, "allocator needs alloc and free");
    }
    c->alloc = *alloc;
    c->has_alloc = 1;
  }
  *out = c;
  return KF_OK;
}

kf_status kf_destroy(kf_ctx* c) {
  delete c;
  return KF_OK;
}

const char* kf_last_error(const kf_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

// 2^(j/64), j < 64, split into double-float pairs (hi = fp32(v), lo = fp32(v - hi))
// for the table-driven exponential of the kernel entries
static const float2* exp2_table() {
  static const std::vector<float2> tab = [] {
    std::vector<float2> v(64);
    for (int j = 0; j < 64; ++j) {
      const double e = std::exp2((double)j / 64.0);
      v[j].x = (float)e;
      v[j].y = (float)(e - (double)v[j].x);
    }
    return v;
  }();
  return tab.data();
}

kf_status kf_tree_build(kf_ctx* c, const void* X, int32_t dtype, int64_t N, int32_t d, int32_t m, void* stream,
                        kf_tree** out) {
  if (!c || !out) return KF_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (!X) return kf_set_err(c, KF_EINVAL, "X is NULL");
  if (N < 1 || N >= (int64_t)INT32_MAX) return kf_set_err(c, KF_EINVAL, "N must be in [1, 2^31)");
  if (d < 1 || d > KF_MAX_D) return kf_set_err(c, KF_EINVAL, "d must be in [1, %d]", KF_MAX_D);
  if (m < 1) return kf_set_err(c, KF_EINVAL, "m must be >= 1");
  if (dtype != KF_F32 && dtype != KF_F64) return kf_set_err(c, KF_EINVAL, "dtype must be KF_F32 or KF_F64");
  kf_tree* t = new kf_tree();
  t->ctx = c;
  t->N = N;
  t->d = d;
  t->m = m;
  int D = 0;
  while (((int64_t)m << D) < N) ++D;
  if (D > 24) {
    delete t;
    return kf_set_err(c, KF_EINVAL, "tree deeper than 24 levels (N/m too large)");
  }
  t->D = D;
  t->nnodes = (1 << (D + 1)) - 1;
  t->lo.assign(t->nnodes + 1, 0);
  t->hi.assign(t->nnodes + 1, 0);
  t->lo[1] = 0;
  t->hi[1] = (int32_t)N;
  for (int a = 1; a < (1 << D); ++a) {
    int32_t n = t->hi[a] - t->lo[a], mid = t->lo[a] + n / 2;
    t->lo[2 * a] = t->lo[a];
    t->hi[2 * a] = mid;
    t->lo[2 * a + 1] = mid;
    t->hi[2 * a + 1] = t->hi[a];
  }
  t->leaf_max = 0;
  for (int a = 1 << D; a < (2 << D); ++a) t->leaf_max = std::max(t->leaf_max, t->hi[a] - t->lo[a]);
  if (t->leaf_max < 1) t->leaf_max = 1;
  auto talloc = [&](size_t b) {
    void* p = c->dalloc(b, s);
    if (p) t->allocs.push_back({p, b});
    return p;
  };
  t->X64 = (double*)talloc(sizeof(double) * N * d);
  t->X32 = (float*)talloc(sizeof(float) * N * d);
  t->X32lo = (float*)talloc(sizeof(float) * N * d);
  t->exp_tab = (float2*)talloc(sizeof(float2) * 64);
  t->perm = (int64_t*)talloc(sizeof(int64_t) * N);
  t->d_lo = (int32_t*)talloc(sizeof(int32_t) * (t->nnodes + 1));
  t->d_hi = (int32_t*)talloc(sizeof(int32_t) * (t->nnodes + 1));
  int32_t* bad = (int32_t*)talloc(sizeof(int32_t));
  if (!t->X64 || !t->X32 || !t->X32lo || !t->exp_tab || !t->perm || !t->d_lo || !t->d_hi || !bad) {
    kf_tree_free(t);
    return kf_set_err(c, KF_ENOMEM, "tree: device allocation failed");
  }
  kf_status st = KF_OK;
  {
    Staged xs;
    size_t xb = (dtype == KF_F64 ? 8 : 4) * (size_t)N * d;
    st = stage_in(c, X, xb, s, xs);
    if (st == KF_OK) {
      if (dtype == KF_F64) cudaMemcpyAsync(t->X64, xs.dev, xb, cudaMemcpyDeviceToDevice, s);
      else kf_to_f64_launch((const float*)xs.dev, t->X64, N * d, s);
      cudaMemcpyAsync(t->d_lo, t->lo.data(), sizeof(int32_t) * (t->nnodes + 1), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(t->d_hi, t->hi.data(), sizeof(int32_t) * (t->nnodes + 1), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(t->exp_tab, exp2_table(), sizeof(float2) * 64, cudaMemcpyHostToDevice, s);
      cudaMemsetAsync(bad, 0, sizeof(int32_t), s);
      kf_check_finite_launch(t->X64, N * d, bad, s);
      int32_t hb = 0;
      cudaMemcpyAsync(&hb, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = kf_set_err(c, KF_ECUDA, "tree: %s", cudaGetErrorString(e));
      else if (hb) st = kf_set_err(c, KF_EINVAL, "X has non-finite coordinates");
    }
  }
  if (st == KF_OK) st = kf_tree_build_device(t, s);
  if (st == KF_OK) st = kf_to_f32_launch(t->X64, t->X32, N * d, s);
  if (st == KF_OK) st = kf_split_lo_launch(t->X64, t->X32, t->X32lo, N * d, s);
  if (st != KF_OK) {
    kf_tree_free(t);
    return st;
  }
  *out = t;
  return KF_OK;
}

kf_status kf_tree_perm(const kf_tree* t, int64_t* perm, void* stream) {
  if (!t || !perm) return KF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  KF_CUDA(t->ctx, cudaMemcpyAsync(perm, t->perm, sizeof(int64_t) * t->N, cudaMemcpyDefault, s));
  if (!is_device_ptr(perm)) KF_CUDA(t->ctx, cudaStreamSynchronize(s));
  return KF_OK;
}

kf_status kf_tree_info(const kf_tree* t, int64_t* N, int32_t* d, int32_t* m, int32_t* depth) {
  if (!t) return KF_EINVAL;
  if (N) *N = t->N;
  if (d) *d = t->d;
  if (m) *m = t->m;
  if (depth) *depth = t->D;
  return KF_OK;
}

kf_status kf_tree_free(kf_tree* t) {
  if (!t) return KF_OK;
  for (auto& a : t->allocs) t->ctx->dfree(a.first, a.second, 0);
  cudaDeviceSynchronize();
  delete t;
  return KF_OK;
}

kf_status kf_factorize(kf_tree* t, double h, double lambda, double tau, int32_t s_max, const kf_opts* opts,
                       void* stream, kf_factor** out) {
  if (!t || !out) return KF_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  kf_factor* f = nullptr;
  kf_status st = alloc_factor(t, h, lambda, tau, s_max, opts, s, &f);
  if (st != KF_OK) return st;
  st = kf_skel_factorize_pipelined(f, s);
  if (st == KF_OK && f->sync_errors) st = read_status(f, s);
  if (st != KF_OK && st != KF_EILLCOND) {
    kf_factor_free(f);
    return st;
  }
  *out = f;
  return st;
}

kf_status kf_autotune(kf_tree* t, double h, double lambda, double tau, int32_t s_max, const kf_opts* base,
                      void* stream, kf_opts* best, float* ms, int32_t* ncand) {
  if (!t || !best) return KF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  kf_ctx* c = t->ctx;
  kf_opts b0 = {};
  if (base) b0 = *base;
  if (b0.hybrid_level != 0) return kf_set_err(c, KF_EUNSUPPORTED, "kf_autotune: the direct solver only");
  b0.sync_errors = 0;
  std::vector<kf_opts> cand;
  for (int cl = 0; cl < 2; ++cl) {
    kf_opts o = b0;
    o.no_cluster_kernels = cl;
    if (b0.precision == KF_PREC_MIXED) {
      for (int tile : {256, 128}) {
        o.no_tensor_cores = 0;
        o.tc_tile_n = tile;
        cand.push_back(o);
      }
      o.no_tensor_cores = 1;
      o.tc_tile_n = 0;
      cand.push_back(o);
    } else {
      cand.push_back(o);
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KF_CUDA(c, cudaEventCreate(&e0));
  KF_CUDA(c, cudaEventCreate(&e1));
  auto run = [&](const kf_opts& o, float* t_ms) -> kf_status {
    kf_factor* f = nullptr;
    cudaEventRecord(e0, s);
    kf_status st = kf_factorize(t, h, lambda, tau, s_max, &o, stream, &f);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (f) kf_factor_free(f);
    if (st != KF_OK && st != KF_EILLCOND) return st;
    if (e != cudaSuccess) return kf_set_err(c, KF_ECUDA, "autotune: %s", cudaGetErrorString(e));
    if (t_ms) cudaEventElapsedTime(t_ms, e0, e1);
    return KF_OK;
  };
  kf_status st = run(b0, nullptr);  // warm-up: module loading, allocator pools
  int bi = 0;
  float bt = 0.f;
  for (size_t i = 0; i < cand.size() && st == KF_OK; ++i) {
    float t1 = 0.f, t2 = 0.f;
    st = run(cand[i], &t1);
    if (st == KF_OK) st = run(cand[i], &t2);
    const float tm = std::min(t1, t2);
    if (ms && i < KF_AUTOTUNE_MAX) ms[i] = tm;
    if (st == KF_OK && (i == 0 || tm < bt)) { bt = tm; bi = (int)i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != KF_OK) return st;
  *best = cand[bi];
  if (base) best->sync_errors = base->sync_errors;
  if (ncand) *ncand = (int32_t)cand.size();
  return KF_OK;
}

kf_status kf_factorize_with_ids(kf_tree* t, double h, double lambda, int32_t s_max, const int32_t* ranks,
                                const int64_t* skel, const double* P, const kf_opts* opts, void* stream,
                                kf_factor** out) {
  if (!t || !out || !ranks || !skel || !P) return KF_EINVAL;
  *out = nullptr;
  if (opts && opts->hybrid_level != 0)
    return kf_set_err(t->ctx, KF_EUNSUPPORTED, "kf_factorize_with_ids: the hybrid solver is kf_factorize only");
  cudaStream_t s = (cudaStream_t)stream;
  kf_factor* f = nullptr;
  kf_status st = alloc_factor(t, h, lambda, 0.0, s_max, opts, s, &f);
  if (st != KF_OK) return st;
  const int D = t->D, nn = t->nnodes;
  const int cmax = f->cmax;
  std::vector<int32_t> hr(nn + 1, 0), hs((size_t)(nn + 1) * s_max, -1);
  std::vector<double> hpl((size_t)t->N * s_max, 0.0), hpc(D > 0 ? (size_t)(1 << D) * 2 * s_max * s_max : 1, 0.0);
  // ranks first (children before parents: a node's column count is the sum
  // of its children's ranks)
  for (int a = nn; a >= 2 && st == KF_OK; --a) {
    const bool leaf = a >= (1 << D);
    const int sa = ranks[a];
    const int c = leaf ? t->hi[a] - t->lo[a] : hr[2 * a] + hr[2 * a + 1];
    if (sa < 0 || sa > s_max || sa > c) st = kf_set_err(t->ctx, KF_EINVAL, "import: bad rank %d at node %d", sa, a);
    hr[a] = sa;
  }
  // children must be set before parents: ranks of children define c
  for (int a = nn; a >= 2 && st == KF_OK; --a) {
    bool leaf = a >= (1 << D);
    int sa = hr[a];
    int c = leaf ? t->hi[a] - t->lo[a] : hr[2 * a] + hr[2 * a + 1];
    const double* Pa = P + (size_t)a * s_max * cmax;
    for (int q = 0; q < sa; ++q) {
      int64_t sk = skel[(size_t)a * s_max + q];
      if (sk < t->lo[a] || sk >= t->hi[a]) {
        st = kf_set_err(t->ctx, KF_EINVAL, "import: skeleton point outside node %d", a);
        break;
      }
      hs[(size_t)a * s_max + q] = (int32_t)sk;
      for (int j = 0; j < c; ++j) {
        double v = Pa[(size_t)q * c + j];
        if (leaf) hpl[(size_t)(t->lo[a] + j) * s_max + q] = v;
        else hpc[((size_t)a * 2 * s_max + j) * s_max + q] = v;
      }
    }
  }
  if (st == KF_OK) {
    cudaMemcpyAsync(f->rank, hr.data(), sizeof(int32_t) * (nn + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(f->skel, hs.data(), sizeof(int32_t) * hs.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(f->Pleaf, hpl.data(), sizeof(double) * hpl.size(), cudaMemcpyHostToDevice, s);
    if (D > 0) cudaMemcpyAsync(f->Pc, hpc.data(), sizeof(double) * hpc.size(), cudaMemcpyHostToDevice, s);
    cudaError_t e = cudaStreamSynchronize(s);  // host vectors go out of scope
    if (e != cudaSuccess) st = kf_set_err(t->ctx, KF_ECUDA, "import: %s", cudaGetErrorString(e));
  }
  if (st == KF_OK) st = kf_factorize_device(f, s);
  if (st == KF_OK && f->sync_errors) st = read_status(f, s);
  if (st != KF_OK && st != KF_EILLCOND) {
    kf_factor_free(f);
    return st;
  }
  *out = f;
  return st;
}

kf_status kf_factor_status(kf_factor* f, void* stream) {
  if (!f) return KF_EINVAL;
  return read_status(f, (cudaStream_t)stream);
}

kf_status kf_factor_free(kf_factor* f) {
  if (!f) return KF_OK;
  for (auto& a : f->allocs) f->ctx->dfree(a.first, a.second, 0);
  cudaDeviceSynchronize();
  delete f;
  return KF_OK;
}

}  // extern "C"

static kf_status check_rhs(kf_factor* f, const void* B, const void* X, int64_t nrhs, int64_t ld, int32_t dtype) {
  if (!f) return KF_EINVAL;
  if (!B || !X) return kf_set_err(f->ctx, KF_EINVAL, "NULL vector");
  if (nrhs < 1) return kf_set_err(f->ctx, KF_EINVAL, "nrhs must be >= 1");
  if (ld < f->t->N) return kf_set_err(f->ctx, KF_EINVAL, "ld must be >= N");
  if (dtype != KF_F32 && dtype != KF_F64) return kf_set_err(f->ctx, KF_EINVAL, "dtype must be KF_F32 or KF_F64");
  return KF_OK;
}

// Copy a caller matrix in, run fn on the tree-order FP64 block, copy out.
template <typename Fn>
static kf_status with_vectors(kf_factor* f, const void* B, void* X, int64_t nrhs, int64_t ld, int32_t dtype,
                              cudaStream_t s, Fn fn) {
  kf_ctx* c = f->ctx;
  const int64_t N = f->t->N;
  const size_t es = dtype == KF_F64 ? 8 : 4;
  const size_t bb = es * (size_t)(ld * (nrhs - 1) + N);
  Staged bs;
  kf_status st = stage_in(c, B, bb, s, bs);
  if (st != KF_OK) return st;
  const bool xdev = is_device_ptr(X);
  void* xd = X;
  if (!xdev) {
    xd = c->dalloc(bb, s);
    if (!xd) return kf_set_err(c, KF_ENOMEM, "staging: allocation failed");
    if (ld > N) cudaMemcpyAsync(xd, X, bb, cudaMemcpyHostToDevice, s);  // keep the gaps of X
  }
  double* W = (double*)c->dalloc(sizeof(double) * N * nrhs, s);
  if (!W) {
    if (!xdev) c->dfree(xd, bb, s);
    return kf_set_err(c, KF_ENOMEM, "solve: allocation failed");
  }
  KF_PHASE(KF_PH_MISC, s, k_gather_in<<<grid_for(N * nrhs, 256), 256, 0, s>>>(bs.dev, dtype, ld, f->t->perm, N, nrhs, W));
  st = fn(W);
  if (st == KF_OK) {
    KF_PHASE(KF_PH_MISC, s, k_scatter_out<<<grid_for(N * nrhs, 256), 256, 0, s>>>(W, f->t->perm, N, nrhs, xd, dtype, ld));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = kf_set_err(c, KF_ECUDA, "%s", cudaGetErrorString(e));
  }
  if (!xdev && st == KF_OK) {
    cudaMemcpyAsync(X, xd, bb, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
  }
  c->dfree(W, sizeof(double) * N * nrhs, s);
  if (!xdev) c->dfree(xd, bb, s);
  return st;
}

// max over columns of ||r_j|| / ||b_j||
// y = A x or A^T x with A = lambda I + K~ (the operator the refinement uses).
static kf_status apply_op(kf_factor* f, const double* x, double* y, int64_t k, int transpose, cudaStream_t s) {
  return transpose ? kf_matvec_transpose_device(f, x, y, k, s) : kf_matvec_device(f, x, y, k, 0, s);
}

static kf_status rel_residual(kf_factor* f, const double* Bt, const double* Xt, int64_t k, double* R, double* Y,
                              double* nrm, int transpose, cudaStream_t s, double* out) {
  kf_ctx* c = f->ctx;
  const int64_t N = f->t->N;
  kf_status st = apply_op(f, Xt, Y, k, transpose, s);
  if (st != KF_OK) return st;
  KF_PHASE(KF_PH_MISC, s, k_sub<<<grid_for(N * k, 256), 256, 0, s>>>(Bt, Y, R, N * k));
  KF_CUDA(c, cudaMemsetAsync(nrm, 0, sizeof(double) * 2 * k, s));
  if ((st = red_colnorm2(c, R, N, k, nrm, s)) != KF_OK) return st;
  if ((st = red_colnorm2(c, Bt, N, k, nrm + k, s)) != KF_OK) return st;
  std::vector<double> h(2 * k);
  KF_CUDA(c, cudaMemcpyAsync(h.data(), nrm, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, s));
  KF_CUDA(c, cudaStreamSynchronize(s));
  double worst = 0.0;
  for (int64_t j = 0; j < k; ++j) worst = std::max(worst, h[k + j] > 0 ? sqrt(h[j] / h[k + j]) : sqrt(h[j]));
  *out = worst;
  return KF_OK;
}

// GMRES(m) for (lambda I + K~) X = B (or the transpose system), k columns in
// lockstep: k independent Krylov iterations (each column its own basis,
// Hessenberg matrix and Givens rotations, on the host) that share every
// launch -- one k-column preconditioner sweep (z_j = M^-1 v_j, or M^-T v_j,
// kept) and one k-column operator product per iteration, classical
// Gram-Schmidt applied twice, four host synchronizations per iteration for
// all columns together (the two Gram-Schmidt passes' coefficients and the new
// vector's norm come to the host, the column scales go back).  FP64 basis, right preconditioning by the factorization,
// the true residual recomputed at every restart.  B, X: N x k point-major;
// X holds the initial guess.  bnorm: host, ||b_c||.  A column stops
// contributing once its residual estimate is below tol ||b_c|| (later steps
// of the shared iteration leave its solution as it is).
static kf_status gmres_block(kf_factor* f, const double* b, double* x, const double* bnorm, int k, int m, int maxit,
                             double tol, int transpose, cudaStream_t s, double* eps_out, int* iters_out) {
  kf_ctx* c = f->ctx;
  const int64_t N = f->t->N, nk = N * (int64_t)k;
  const size_t vb = sizeof(double) * (size_t)nk;
  double* V = (double*)c->dalloc(vb * (m + 1), s);
  double* Zb = (double*)c->dalloc(vb * m, s);
  double* w = (double*)c->dalloc(vb, s);
  double* h = (double*)c->dalloc(sizeof(double) * (size_t)(m + 2) * k, s);
  double* dsc = (double*)c->dalloc(sizeof(double) * (size_t)k, s);
  kf_status st = (V && Zb && w && h && dsc) ? KF_OK : kf_set_err(c, KF_ENOMEM, "gmres: allocation failed");
  const int g = grid_for(nk, 256, 304);
  std::vector<double> H((size_t)k * (m + 1) * m), cs((size_t)k * m), sn((size_t)k * m), gg((size_t)k * (m + 1));
  std::vector<double> hh((size_t)(m + 2) * k), y((size_t)m * k), sc(k), beta(k), eps(k, 0.0);
  std::vector<int> jc(k), done(k);
  auto Hc = [&](int col, int r, int q) -> double& { return H[((size_t)col * (m + 1) + r) * m + q]; };
  auto fetch = [&](size_t cnt) -> kf_status {
    KF_CUDA(c, cudaMemcpyAsync(hh.data(), h, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
    KF_CUDA(c, cudaStreamSynchronize(s));
    return KF_OK;
  };
  auto upload_sc = [&]() -> kf_status {
    KF_CUDA(c, cudaMemcpyAsync(dsc, sc.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
    KF_CUDA(c, cudaStreamSynchronize(s));  // sc is rewritten on the host before the next use
    return KF_OK;
  };
  int it = 0;
  double worst = 0.0;
  while (st == KF_OK) {
    // R = B - A X, beta_c = ||r_c||
    st = apply_op(f, x, w, k, transpose, s);
    if (st != KF_OK) break;
    KF_PHASE(KF_PH_MISC, s, k_sub<<<g, 256, 0, s>>>(b, w, w, nk));
    if ((st = red_colnorm2(c, w, N, k, h, s)) != KF_OK) break;
    if ((st = fetch(k)) != KF_OK) break;
    worst = 0.0;
    for (int col = 0; col < k; ++col) {
      beta[col] = sqrt(hh[col]);
      eps[col] = bnorm[col] > 0 ? beta[col] / bnorm[col] : beta[col];
      worst = std::max(worst, eps[col]);
      done[col] = !(eps[col] > tol) || beta[col] == 0.0;
      sc[col] = done[col] ? 0.0 : 1.0 / beta[col];
      jc[col] = 0;
      std::fill(gg.begin() + (size_t)col * (m + 1), gg.begin() + (size_t)(col + 1) * (m + 1), 0.0);
      gg[(size_t)col * (m + 1)] = done[col] ? 0.0 : beta[col];
    }
    if (worst <= tol || it >= maxit) break;
    if ((st = upload_sc()) != KF_OK) break;
    KF_PHASE(KF_PH_MISC, s, k_scale_cols<<<g, 256, 0, s>>>(w, dsc, V, N, k));
    int j = 0;
    for (; j < m && it < maxit; ++j) {
      double* zj = Zb + (int64_t)j * nk;
      KF_CUDA(c, cudaMemcpyAsync(zj, V + (int64_t)j * nk, vb, cudaMemcpyDeviceToDevice, s));
      if ((st = kf_solve_device(f, zj, k, transpose, s)) != KF_OK) break;  // z_j = M^-1 v_j (M^-T v_j)
      if ((st = apply_op(f, zj, w, k, transpose, s)) != KF_OK) break;     // w = A z_j (A^T z_j)
      for (int pass = 0; pass < 2; ++pass) {                            // CGS2
        if ((st = red_multidot(c, V, nk, j + 1, w, N, k, h, s)) != KF_OK) break;
        KF_PHASE(KF_PH_MISC, s, k_multiaxpy_k<<<g, 256, 0, s>>>(V, nk, j + 1, h, w, N, k));
        if ((st = fetch((size_t)(j + 1) * k)) != KF_OK) break;
        for (int col = 0; col < k; ++col)
          for (int q = 0; q <= j; ++q) Hc(col, q, j) = (pass == 0 ? 0.0 : Hc(col, q, j)) + hh[(size_t)q * k + col];
      }
      if (st != KF_OK) break;
      if ((st = red_colnorm2(c, w, N, k, h, s)) != KF_OK) break;
      if ((st = fetch(k)) != KF_OK) break;
      bool all_done = true;
      for (int col = 0; col < k; ++col) {
        const double hn = sqrt(hh[col]);
        sc[col] = (!done[col] && hn > 0) ? 1.0 / hn : 0.0;
        if (done[col]) continue;
        double* gc = gg.data() + (size_t)col * (m + 1);
        double* csc = cs.data() + (size_t)col * m;
        double* snc = sn.data() + (size_t)col * m;
        Hc(col, j + 1, j) = hn;
        for (int q = 0; q < j; ++q) {  // previous rotations on the new column
          const double a = Hc(col, q, j), bq = Hc(col, q + 1, j);
          Hc(col, q, j) = csc[q] * a + snc[q] * bq;
          Hc(col, q + 1, j) = -snc[q] * a + csc[q] * bq;
        }
        const double a = Hc(col, j, j), bq = Hc(col, j + 1, j);
        const double r = hypot(a, bq);
        csc[j] = r > 0 ? a / r : 1.0;
        snc[j] = r > 0 ? bq / r : 0.0;
        Hc(col, j, j) = r;
        Hc(col, j + 1, j) = 0.0;
        gc[j + 1] = -snc[j] * gc[j];
        gc[j] = csc[j] * gc[j];
        jc[col] = j + 1;
        if (fabs(gc[j + 1]) <= tol * bnorm[col] * 0.5 || hn == 0.0 || r == 0.0) done[col] = 1;
        all_done = all_done && done[col];
      }
      ++it;
      if (all_done) { ++j; break; }
      if ((st = upload_sc()) != KF_OK) break;
      KF_PHASE(KF_PH_MISC, s, k_scale_cols<<<g, 256, 0, s>>>(w, dsc, V + (int64_t)(j + 1) * nk, N, k));
    }
    if (st != KF_OK) break;
    // per column: y = H^-1 g (upper triangular, its own jc steps), then X += Z Y
    std::fill(y.begin(), y.end(), 0.0);
    int J = 0;
    for (int col = 0; col < k; ++col) {
      const double* gc = gg.data() + (size_t)col * (m + 1);
      for (int q = jc[col] - 1; q >= 0; --q) {
        double acc = gc[q];
        for (int t2 = q + 1; t2 < jc[col]; ++t2) acc -= Hc(col, q, t2) * y[(size_t)t2 * k + col];
        y[(size_t)q * k + col] = Hc(col, q, q) != 0.0 ? acc / Hc(col, q, q) : 0.0;
      }
      J = std::max(J, jc[col]);
    }
    if (J > 0) {
      KF_CUDA(c, cudaMemcpyAsync(h, y.data(), sizeof(double) * (size_t)J * k, cudaMemcpyHostToDevice, s));
      KF_PHASE(KF_PH_MISC, s, k_zupdate_k<<<g, 256, 0, s>>>(Zb, nk, J, h, x, N, k));
    }
    KF_CUDA(c, cudaStreamSynchronize(s));  // y lives on the host
  }
  *eps_out = worst;
  *iters_out = it;
  c->dfree(V, vb * (m + 1), s);
  c->dfree(Zb, vb * m, s);
  c->dfree(w, vb, s);
  c->dfree(h, sizeof(double) * (size_t)(m + 2) * k, s);
  c->dfree(dsc, sizeof(double) * (size_t)k, s);
  return st;
}

// Columns [c0, c0 + kg) of the point-major N x k matrix W <-> a point-major N x kg block.
__global__ void k_get_cols(const double* __restrict__ W, int64_t k, int64_t c0, int kg, double* __restrict__ out,
                           int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kg; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = W[(e / kg) * k + c0 + e % kg];
}
__global__ void k_put_cols(const double* __restrict__ in, int64_t k, int64_t c0, int kg, double* __restrict__ W,
                           int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kg; e += (int64_t)gridDim.x * blockDim.x)
    W[(e / kg) * k + c0 + e % kg] = in[e];
}

// GMRES(m) (lockstep, gmres_block) on groups of columns whose bases (2m + 2
// vectors each) take at most 4 GB, in place on W (N x nrhs, tree order).
// Bsrc = nullptr: W holds the right-hand sides on entry and each group starts
// from their direct solve; otherwise Bsrc holds them and W the initial guess.
// eps: the worst final relative residual; iters: the most iterations.
static kf_status gmres_columns(kf_factor* f, double* W, int64_t nrhs, int transpose, cudaStream_t s, double* eps,
                               int* iters, const double* Bsrc = nullptr) {
  kf_ctx* c = f->ctx;
  const int64_t N = f->t->N;
  const int m = f->gmres_m > 0 ? f->gmres_m : 50;
  const double budget = 4e9;
  const int64_t kg_max = std::max<int64_t>(1, std::min<int64_t>(nrhs, (int64_t)(budget / ((2.0 * m + 2) * 8.0 * N))));
  const size_t gb = sizeof(double) * (size_t)N * kg_max;
  double* bg = (double*)c->dalloc(gb, s);
  double* xg = (double*)c->dalloc(gb, s);
  double* nb = (double*)c->dalloc(sizeof(double) * (size_t)kg_max, s);
  kf_status r = (bg && xg && nb) ? KF_OK : kf_set_err(c, KF_ENOMEM, "gmres: allocation failed");
  double worst = 0.0;
  int most = 0;
  std::vector<double> hb(kg_max);
  for (int64_t c0 = 0; c0 < nrhs && r == KF_OK; c0 += kg_max) {
    const int kg = (int)std::min<int64_t>(kg_max, nrhs - c0);
    const int64_t ne = N * kg;
    if (Bsrc) {
      KF_PHASE(KF_PH_MISC, s, k_get_cols<<<grid_for(ne, 256), 256, 0, s>>>(Bsrc, nrhs, c0, kg, bg, N));
      KF_PHASE(KF_PH_MISC, s, k_get_cols<<<grid_for(ne, 256), 256, 0, s>>>(W, nrhs, c0, kg, xg, N));
    } else {
      KF_PHASE(KF_PH_MISC, s, k_get_cols<<<grid_for(ne, 256), 256, 0, s>>>(W, nrhs, c0, kg, bg, N));
      cudaMemcpyAsync(xg, bg, sizeof(double) * (size_t)ne, cudaMemcpyDeviceToDevice, s);
      if ((r = kf_solve_device(f, xg, kg, transpose, s)) != KF_OK) break;
    }
    if ((r = red_colnorm2(c, bg, N, kg, nb, s)) != KF_OK) break;
    cudaMemcpyAsync(hb.data(), nb, sizeof(double) * kg, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (int q = 0; q < kg; ++q) hb[q] = sqrt(hb[q]);
    double e = 0.0;
    int its = 0;
    r = gmres_block(f, bg, xg, hb.data(), kg, m, f->refine_max_iter, f->refine_tol, transpose, s, &e, &its);
    worst = std::max(worst, e);
    most = std::max(most, its);
    KF_PHASE(KF_PH_MISC, s, k_put_cols<<<grid_for(ne, 256), 256, 0, s>>>(xg, nrhs, c0, kg, W, N));
  }
  cudaStreamSynchronize(s);
  c->dfree(bg, gb, s);
  c->dfree(xg, gb, s);
  c->dfree(nb, sizeof(double) * (size_t)kg_max, s);
  *eps = worst;
  *iters = most;
  return r;
}

// Solve in place, W: N x nrhs FP64 in tree order.  The direct sweep of the
// factorization (Algorithm 3 or its transpose); with refine, GMRES(m) (or
// x += M^-1 r when gmres_m <= 0) against the operator A (A^T for transpose)
// until eps_r <= refine_tol; want_eps alone computes the residual of the
// direct sweep.  Shared by kf_solve and the adjoint solve of kf_grad.
static kf_status solve_refined(kf_factor* f, double* W, int64_t nrhs, int transpose, bool refine, bool want_eps,
                               cudaStream_t s, double* eps_out, int* iters_out) {
  kf_ctx* c = f->ctx;
  const int64_t N = f->t->N;
  int iters = 0;
  double eps = -1.0;
  auto richardson = [&]() -> kf_status {
    if (!refine && !want_eps) return kf_solve_device(f, W, nrhs, transpose, s);
    const size_t vb = sizeof(double) * N * nrhs;
    double* Bt = (double*)c->dalloc(vb, s);
    double* R = (double*)c->dalloc(vb, s);
    double* Y = (double*)c->dalloc(vb, s);
    double* nrm = (double*)c->dalloc(sizeof(double) * 2 * nrhs, s);
    kf_status r = (Bt && R && Y && nrm) ? KF_OK : kf_set_err(c, KF_ENOMEM, "refinement: allocation failed");
    if (r == KF_OK) {
      cudaMemcpyAsync(Bt, W, vb, cudaMemcpyDeviceToDevice, s);
      r = kf_solve_device(f, W, nrhs, transpose, s);
      if (r == KF_OK) {
        r = rel_residual(f, Bt, W, nrhs, R, Y, nrm, transpose, s, &eps);
        while (r == KF_OK && refine && eps > f->refine_tol && iters < f->refine_max_iter) {
          r = kf_solve_device(f, R, nrhs, transpose, s);  // correction M^-1 r (M^-T r)
          if (r != KF_OK) break;
          KF_PHASE(KF_PH_MISC, s, k_add<<<grid_for(N * nrhs, 256), 256, 0, s>>>(W, R, N * nrhs));
          ++iters;
          r = rel_residual(f, Bt, W, nrhs, R, Y, nrm, transpose, s, &eps);
        }
        if (r == KF_OK && refine && eps > f->refine_tol)
          r = kf_set_err(c, KF_ENOTCONV, "refinement stopped at eps_r = %.3e after %d steps", eps, iters);
      }
    }
    c->dfree(Bt, vb, s);
    c->dfree(R, vb, s);
    c->dfree(Y, vb, s);
    c->dfree(nrm, sizeof(double) * 2 * nrhs, s);
    return r;
  };
  auto gmres_path = [&]() -> kf_status {
    // GMRES(m) from the direct solve of the factorization, the columns in
    // lockstep groups whose Krylov bases fit a fixed memory budget
    kf_status r = gmres_columns(f, W, nrhs, transpose, s, &eps, &iters);
    if (r == KF_OK && eps > f->refine_tol)
      r = kf_set_err(c, KF_ENOTCONV, "GMRES stopped at eps_r = %.3e after %d iterations", eps, iters);
    return r;
  };
  kf_status r = (refine && f->gmres_m > 0) ? gmres_path() : richardson();
  if (eps_out) *eps_out = eps;
  if (iters_out) *iters_out = iters;
  return r;
}

// Whether solves with this factor are refined: the mixed path by default, the
// FP64 path when the caller asked for it; refine_max_iter <= 0 turns it off.
static bool refines(const kf_factor* f) {
  return (f->prec == KF_PREC_MIXED || f->refine_user) && f->refine_max_iter > 0;
}

extern "C" {

kf_status kf_solve(kf_factor* f, const void* B, void* X, int64_t nrhs, int64_t ld, int32_t dtype, int32_t transpose,
                   void* stream, kf_solve_info* info) {
  kf_status st = check_rhs(f, B, X, nrhs, ld, dtype);
  if (st != KF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int iters = 0;
  double eps = -1.0;
  st = with_vectors(f, B, X, nrhs, ld, dtype, s, [&](double* W) -> kf_status {
    return solve_refined(f, W, nrhs, transpose ? 1 : 0, refines(f), info != nullptr, s, &eps, &iters);
  });
  if (info) {
    info->eps_r = eps;
    info->iters = iters;
    int32_t dst = 0;
    cudaMemcpyAsync(&dst, f->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    info->status = dst;
  }
  if (st == KF_OK && f->sync_errors) st = read_status(f, s);
  return st;
}

kf_status kf_matvec(kf_factor* f, const void* Xin, void* Y, int64_t nrhs, int64_t ld, int32_t dtype, void* stream) {
  kf_status st = check_rhs(f, Xin, Y, nrhs, ld, dtype);
  if (st != KF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  kf_ctx* c = f->ctx;
  const int64_t N = f->t->N;
  return with_vectors(f, Xin, Y, nrhs, ld, dtype, s, [&](double* W) -> kf_status {
    double* Yt = (double*)c->dalloc(sizeof(double) * N * nrhs, s);
    if (!Yt) return kf_set_err(c, KF_ENOMEM, "matvec: allocation failed");
    kf_status r = kf_matvec_device(f, W, Yt, nrhs, 0, s);
    cudaMemcpyAsync(W, Yt, sizeof(double) * N * nrhs, cudaMemcpyDeviceToDevice, s);
    c->dfree(Yt, sizeof(double) * N * nrhs, s);
    return r;
  });
}

kf_status kf_grad(kf_factor* f, const void* x, const void* dLdx, void* dLdb, double* dLdlambda, double* dLdh,
                  int64_t nrhs, int64_t ld, void* stream) {
  kf_status st = check_rhs(f, x, dLdx, nrhs, ld, KF_F64);
  if (st != KF_OK) return st;
  if (!dLdb || !dLdlambda || !dLdh) return kf_set_err(f->ctx, KF_EINVAL, "NULL gradient output");
  if (f->hyb_L > 0) return kf_set_err(f->ctx, KF_EUNSUPPORTED, "kf_grad: not available for the hybrid solver");
  cudaStream_t s = (cudaStream_t)stream;
  kf_ctx* c = f->ctx;
  const int64_t N = f->t->N;
  const size_t vb = sizeof(double) * N * nrhs;
  Staged xs;
  st = stage_in(c, x, sizeof(double) * (size_t)(ld * (nrhs - 1) + N), s, xs);
  if (st != KF_OK) return st;
  double* Xt = (double*)c->dalloc(vb, s);
  double* DX = (double*)c->dalloc(vb, s);
  double* sums = (double*)c->dalloc(sizeof(double) * 2, s);
  if (!Xt || !DX || !sums) {
    c->dfree(Xt, vb, s);
    c->dfree(DX, vb, s);
    c->dfree(sums, 16, s);
    return kf_set_err(c, KF_ENOMEM, "grad: allocation failed");
  }
  KF_PHASE(KF_PH_MISC, s, k_gather_in<<<grid_for(N * nrhs, 256), 256, 0, s>>>(xs.dev, KF_F64, ld, f->t->perm, N, nrhs, Xt));
  kf_status r = kf_matvec_device(f, Xt, DX, nrhs, 1, s);  // (dK~/dh) x
  double hs[2] = {0, 0};
  if (r == KF_OK)
    r = with_vectors(f, dLdx, dLdb, nrhs, ld, KF_F64, s, [&](double* A) -> kf_status {
      // a = (lambda I + K~)^-T dL/dx, refined like the forward solve (GMRES on the
      // transpose system against A^T) where the factor's solves are refined
      kf_status q = solve_refined(f, A, nrhs, 1, refines(f), false, s, nullptr, nullptr);
      if (q != KF_OK) return q;
      if ((q = red_dot(c, A, Xt, N * nrhs, sums, s)) != KF_OK) return q;
      if ((q = red_dot(c, A, DX, N * nrhs, sums + 1, s)) != KF_OK) return q;
      cudaMemcpyAsync(hs, sums, sizeof(double) * 2, cudaMemcpyDeviceToHost, s);
      return KF_OK;
    });
  cudaStreamSynchronize(s);
  *dLdlambda = -hs[0];
  *dLdh = -hs[1];
  c->dfree(Xt, vb, s);
  c->dfree(DX, vb, s);
  c->dfree(sums, 16, s);
  return r;
}

kf_status kf_factor_ranks(const kf_factor* f, int32_t* ranks, void* stream) {
  if (!f || !ranks) return KF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  KF_CUDA(f->ctx, cudaMemcpyAsync(ranks, f->rank, sizeof(int32_t) * (f->t->nnodes + 1), cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaStreamSynchronize(s));
  return KF_OK;
}

kf_status kf_factor_pivot_ratios(const kf_factor* f, double* ratios, void* stream) {
  if (!f || !ratios) return KF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  KF_CUDA(f->ctx, cudaMemcpyAsync(ratios, f->pivr, sizeof(double) * (f->t->nnodes + 1), cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaStreamSynchronize(s));
  return KF_OK;
}

static kf_status node_ok(const kf_factor* f, int32_t node) {
  if (node < 2 || node > f->t->nnodes) return kf_set_err(f->ctx, KF_EINVAL, "node %d is not a non-root node", node);
  return KF_OK;
}

kf_status kf_factor_knn(const kf_factor* f, int32_t* nbr, void* stream) {
  if (!f || !nbr) return KF_EINVAL;
  if (f->knn_kappa <= 0) return kf_set_err(f->ctx, KF_EINVAL, "kf_factor_knn: near-field sampling is off");
  cudaStream_t s = (cudaStream_t)stream;
  KF_CUDA(f->ctx, cudaMemcpyAsync(nbr, f->nbr, sizeof(int32_t) * (size_t)f->t->N * f->knn_kappa,
                                  cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaStreamSynchronize(s));
  return KF_OK;
}

kf_status kf_factor_near(const kf_factor* f, int32_t node, int32_t* pos, int32_t* cnt, int32_t* len, void* stream) {
  if (!f || !pos || !cnt || !len) return KF_EINVAL;
  if (f->knn_kappa <= 0) return kf_set_err(f->ctx, KF_EINVAL, "kf_factor_near: near-field sampling is off");
  kf_status st = node_ok(f, node);
  if (st != KF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t cap = (size_t)f->near_cap;
  KF_CUDA(f->ctx, cudaMemcpyAsync(len, f->near_len + node, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaMemcpyAsync(pos, f->near_pos + node * cap, sizeof(int32_t) * cap, cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaMemcpyAsync(cnt, f->near_cnt + node * cap, sizeof(int32_t) * cap, cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaStreamSynchronize(s));
  return KF_OK;
}

kf_status kf_factor_skeleton(const kf_factor* f, int32_t node, int64_t* skel, void* stream) {
  if (!f || !skel) return KF_EINVAL;
  kf_status st = node_ok(f, node);
  if (st != KF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> r(f->t->nnodes + 1), sk(f->s_max);
  KF_CUDA(f->ctx, cudaMemcpyAsync(r.data(), f->rank, sizeof(int32_t) * r.size(), cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaMemcpyAsync(sk.data(), f->skel + (size_t)node * f->s_max, sizeof(int32_t) * f->s_max,
                                  cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaStreamSynchronize(s));
  for (int q = 0; q < r[node]; ++q) skel[q] = sk[q];
  return KF_OK;
}

kf_status kf_factor_P(const kf_factor* f, int32_t node, double* P, void* stream) {
  if (!f || !P) return KF_EINVAL;
  kf_status st = node_ok(f, node);
  if (st != KF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const kf_tree* t = f->t;
  const int s_max = f->s_max;
  std::vector<int32_t> r(t->nnodes + 1);
  KF_CUDA(f->ctx, cudaMemcpyAsync(r.data(), f->rank, sizeof(int32_t) * r.size(), cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaStreamSynchronize(s));
  const bool leaf = node >= (1 << t->D);
  const int sa = r[node];
  const int c = leaf ? t->hi[node] - t->lo[node] : r[2 * node] + r[2 * node + 1];
  std::vector<double> buf((size_t)std::max(c, 1) * s_max);
  const double* src = leaf ? f->Pleaf + (size_t)t->lo[node] * s_max : f->Pc + (size_t)node * 2 * s_max * s_max;
  KF_CUDA(f->ctx, cudaMemcpyAsync(buf.data(), src, sizeof(double) * (size_t)c * s_max, cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaStreamSynchronize(s));
  for (int q = 0; q < sa; ++q)
    for (int j = 0; j < c; ++j) P[(size_t)q * c + j] = buf[(size_t)j * s_max + q];
  return KF_OK;
}

kf_status kf_factor_Phat(const kf_factor* f, int32_t node, double* Phat, void* stream) {
  if (!f || !Phat) return KF_EINVAL;
  kf_status st = node_ok(f, node);
  if (st != KF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const kf_tree* t = f->t;
  const int s_max = f->s_max, l = kf_level_of(node);
  std::vector<int32_t> r(t->nnodes + 1);
  KF_CUDA(f->ctx, cudaMemcpyAsync(r.data(), f->rank, sizeof(int32_t) * r.size(), cudaMemcpyDeviceToHost, s));
  const int n = t->hi[node] - t->lo[node];
  if (f->w_lean && l != t->D)
    return kf_set_err(f->ctx, KF_EUNSUPPORTED, "memory-lean W keeps P^ of the leaves only (node %d)", node);
  const size_t off = (size_t)kf_phat_level_off(f, l) + (size_t)t->lo[node] * s_max;
  std::vector<char> buf((size_t)std::max(n, 1) * s_max * f->tsize());
  KF_CUDA(f->ctx, cudaMemcpyAsync(buf.data(), (const char*)f->Phat + off * f->tsize(), (size_t)n * s_max * f->tsize(),
                                  cudaMemcpyDeviceToHost, s));
  KF_CUDA(f->ctx, cudaStreamSynchronize(s));
  const int sa = r[node];
  for (int i = 0; i < n; ++i)
    for (int q = 0; q < sa; ++q)
      Phat[(size_t)i * sa + q] = f->prec == KF_PREC_FP64 ? ((const double*)buf.data())[(size_t)i * s_max + q]
                                                         : (double)((const float*)buf.data())[(size_t)i * s_max + q];
  return KF_OK;
}

}  // extern "C"

// ---- batched: many independent problems in one graph launch -------------------------
namespace {

// Runs enq(i, stream) for every problem inside one captured CUDA graph whose
// branches are spread over `nstreams` streams, launches it once on s and
// waits for it.  Scratch allocations inside use stream-ordered allocation.
template <typename Enq>
kf_status run_batched_graph(kf_ctx* c, int32_t nprob, cudaStream_t s, Enq enq) {
  const int nstreams = std::max(1, std::min<int>(nprob, 16));
  std::vector<cudaStream_t> ss(nstreams);
  std::vector<cudaEvent_t> ev(nstreams + 1);
  for (int i = 0; i < nstreams; ++i) KF_CUDA(c, cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking));
  for (int i = 0; i <= nstreams; ++i) KF_CUDA(c, cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
  cudaStream_t cs = s;
  bool own_stream = false;
  if (cs == 0) {  // the legacy stream cannot be captured
    KF_CUDA(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    own_stream = true;
  }
  kf_status st = KF_OK;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  c->capturing = 1;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaEventRecord(ev[nstreams], cs);
    for (int i = 0; i < nstreams; ++i) cudaStreamWaitEvent(ss[i], ev[nstreams], 0);
    for (int32_t i = 0; i < nprob && st == KF_OK; ++i) st = enq(i, ss[i % nstreams]);
    for (int i = 0; i < nstreams; ++i) {
      cudaEventRecord(ev[i], ss[i]);
      cudaStreamWaitEvent(cs, ev[i], 0);
    }
    e = cudaStreamEndCapture(cs, &graph);
  }
  c->capturing = 0;
  if (st == KF_OK && e != cudaSuccess) st = kf_set_err(c, KF_ECUDA, "batched capture: %s", cudaGetErrorString(e));
  if (st == KF_OK) {
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) st = kf_set_err(c, KF_ECUDA, "batched graph: %s", cudaGetErrorString(e));
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  for (auto& x : ss) cudaStreamDestroy(x);
  for (auto& x : ev) cudaEventDestroy(x);
  if (own_stream) cudaStreamDestroy(cs);
  cudaGetLastError();
  return st;
}

// Many problems solved and refined together: the direct sweeps of all
// problems in one graph launch, then refinement steps x += M^-1 (b - A x) for
// the whole batch, each step two graph launches (the residuals of every
// unconverged problem against its operator, then the sweeps of those
// residuals), with one host synchronization per step to read the residual
// norms.  A problem leaves the batch once its relative residual (Eq. e:errors,
// max over its columns) is at most its refine_tol; a problem whose residual
// falls by less than half in a step (or that reaches refine_max_iter steps)
// finishes column by column with GMRES(m) from where it stands, like kf_solve.
// Problems whose factors do not refine get the direct sweep only.
kf_status solve_batched_refined(kf_factor* const* f, int32_t nprob, const void* const* B, void* const* X,
                                const int64_t* nrhs, const int64_t* ld, int32_t dtype, cudaStream_t s,
                                kf_solve_info* info) {
  kf_ctx* c = f[0]->ctx;
  struct Prob {
    double *Bt = nullptr, *Wt = nullptr, *R = nullptr, *Y = nullptr;
    size_t vb = 0;
    double eps = INFINITY;
    int steps = 0;
    int state = 0;  // 0 refining, 1 converged, 2 to GMRES, 3 direct only
  };
  std::vector<Prob> P(nprob);
  int64_t ktot = 0;
  std::vector<int64_t> koff(nprob + 1, 0);
  for (int32_t i = 0; i < nprob; ++i) koff[i + 1] = koff[i] + nrhs[i];
  ktot = koff[nprob];
  double* nrm = (double*)c->dalloc(sizeof(double) * 2 * ktot, s);
  kf_status st = nrm ? KF_OK : kf_set_err(c, KF_ENOMEM, "batched solve: allocation failed");
  for (int32_t i = 0; i < nprob && st == KF_OK; ++i) {
    Prob& q = P[i];
    q.vb = sizeof(double) * (size_t)f[i]->t->N * nrhs[i];
    q.Bt = (double*)c->dalloc(q.vb, s);
    q.Wt = (double*)c->dalloc(q.vb, s);
    q.R = (double*)c->dalloc(q.vb, s);
    q.Y = (double*)c->dalloc(q.vb, s);
    if (!q.Bt || !q.Wt || !q.R || !q.Y) st = kf_set_err(c, KF_ENOMEM, "batched solve: allocation failed");
    q.state = refines(f[i]) ? 0 : 3;
  }
  std::vector<int32_t> act;
  auto run_on = [&](const std::vector<int32_t>& ids, auto enq) -> kf_status {
    if (ids.empty()) return KF_OK;
    return run_batched_graph(c, (int32_t)ids.size(), s,
                             [&](int32_t j, cudaStream_t si) -> kf_status { return enq(ids[j], si); });
  };
  std::vector<int32_t> all(nprob);
  for (int32_t i = 0; i < nprob; ++i) all[i] = i;
  // b in tree order, x = M^-1 b
  if (st == KF_OK)
    st = run_on(all, [&](int32_t i, cudaStream_t si) -> kf_status {
      const int64_t N = f[i]->t->N, k = nrhs[i];
      KF_PHASE(KF_PH_MISC, si, k_gather_in<<<grid_for(N * k, 256), 256, 0, si>>>(B[i], dtype, ld[i], f[i]->t->perm,
                                                                                  N, k, P[i].Bt));
      KF_CUDA(c, cudaMemcpyAsync(P[i].Wt, P[i].Bt, P[i].vb, cudaMemcpyDeviceToDevice, si));
      return kf_solve_device(f[i], P[i].Wt, k, 0, si);
    });
  for (int32_t i = 0; i < nprob; ++i)
    if (P[i].state == 0) act.push_back(i);
  std::vector<double> hn(2 * ktot);
  while (st == KF_OK && !act.empty()) {
    // r = b - A x and the column norms of r and b
    KF_CUDA(c, cudaMemsetAsync(nrm, 0, sizeof(double) * 2 * ktot, s));
    KF_CUDA(c, cudaStreamSynchronize(s));
    st = run_on(act, [&](int32_t i, cudaStream_t si) -> kf_status {
      const int64_t N = f[i]->t->N, k = nrhs[i];
      kf_status r = apply_op(f[i], P[i].Wt, P[i].Y, k, 0, si);
      if (r != KF_OK) return r;
      KF_PHASE(KF_PH_MISC, si, k_sub<<<grid_for(N * k, 256), 256, 0, si>>>(P[i].Bt, P[i].Y, P[i].R, N * k));
      if ((r = red_colnorm2(c, P[i].R, N, k, nrm + 2 * koff[i], si)) != KF_OK) return r;
      if ((r = red_colnorm2(c, P[i].Bt, N, k, nrm + 2 * koff[i] + k, si)) != KF_OK) return r;
      return KF_OK;
    });
    if (st != KF_OK) break;
    KF_CUDA(c, cudaMemcpy(hn.data(), nrm, sizeof(double) * 2 * ktot, cudaMemcpyDeviceToHost));
    std::vector<int32_t> next;
    for (int32_t i : act) {
      const int64_t k = nrhs[i];
      double e = 0.0;
      for (int64_t j = 0; j < k; ++j) {
        const double rr = hn[2 * koff[i] + j], bb = hn[2 * koff[i] + k + j];
        e = std::max(e, bb > 0 ? sqrt(rr / bb) : sqrt(rr));
      }
      Prob& q = P[i];
      const double prev = q.eps;
      q.eps = e;
      if (e <= f[i]->refine_tol) q.state = 1;
      else if (q.steps >= f[i]->refine_max_iter || !(e <= 0.5 * prev)) q.state = 2;
      else next.push_back(i);
    }
    act.swap(next);
    if (act.empty()) break;
    // x += M^-1 r
    st = run_on(act, [&](int32_t i, cudaStream_t si) -> kf_status {
      const int64_t N = f[i]->t->N, k = nrhs[i];
      kf_status r = kf_solve_device(f[i], P[i].R, k, 0, si);
      if (r != KF_OK) return r;
      KF_PHASE(KF_PH_MISC, si, k_add<<<grid_for(N * k, 256), 256, 0, si>>>(P[i].Wt, P[i].R, N * k));
      ++P[i].steps;
      return KF_OK;
    });
  }
  // the problems the steps did not settle: GMRES(m) on all their columns in
  // lockstep, from the current x
  kf_status worst = KF_OK;
  for (int32_t i = 0; i < nprob && st == KF_OK; ++i) {
    if (P[i].state != 2) continue;
    double pe = 0.0;
    int pits = 0;
    st = gmres_columns(f[i], P[i].Wt, nrhs[i], 0, s, &pe, &pits, P[i].Bt);
    P[i].eps = pe;
    P[i].steps += pits;
    if (st == KF_OK && pe > f[i]->refine_tol && worst == KF_OK)
      worst = kf_set_err(c, KF_ENOTCONV, "batched solve: problem %d stopped at eps_r = %.3e", i, pe);
  }
  if (info)
    for (int32_t i = 0; i < nprob; ++i) {
      info[i].eps_r = P[i].state == 3 ? -1.0 : P[i].eps;
      info[i].iters = P[i].steps;
      info[i].status = (P[i].state != 3 && P[i].eps > f[i]->refine_tol) ? KF_ENOTCONV : KF_OK;
    }
  // x back to the caller's order and type
  if (st == KF_OK)
    st = run_on(all, [&](int32_t i, cudaStream_t si) -> kf_status {
      const int64_t N = f[i]->t->N, k = nrhs[i];
      KF_PHASE(KF_PH_MISC, si, k_scatter_out<<<grid_for(N * k, 256), 256, 0, si>>>(P[i].Wt, f[i]->t->perm, N, k, X[i],
                                                                                   dtype, ld[i]));
      return KF_OK;
    });
  if (st == KF_OK) KF_CUDA(c, cudaStreamSynchronize(s));
  for (auto& q : P) {
    if (q.Bt) c->dfree(q.Bt, q.vb, s);
    if (q.Wt) c->dfree(q.Wt, q.vb, s);
    if (q.R) c->dfree(q.R, q.vb, s);
    if (q.Y) c->dfree(q.Y, q.vb, s);
  }
  if (nrm) c->dfree(nrm, sizeof(double) * 2 * ktot, s);
  return st == KF_OK ? worst : st;
}

}  // namespace

extern "C" {

kf_status kf_factorize_batched(kf_tree* const* trees, int32_t nprob, const double* h, const double* lambda,
                               const double* tau, int32_t s_max, const kf_opts* opts, void* stream, kf_factor** out) {
  if (!trees || nprob < 1 || !h || !lambda || !tau || !out) return kf_set_err(nullptr, KF_EINVAL, "batched: bad arguments");
  for (int32_t i = 0; i < nprob; ++i) {
    out[i] = nullptr;
    if (!trees[i]) return kf_set_err(nullptr, KF_EINVAL, "batched: tree %d is NULL", i);
    if (trees[i]->ctx != trees[0]->ctx) return kf_set_err(nullptr, KF_EINVAL, "batched: trees of different contexts");
  }
  kf_ctx* c = trees[0]->ctx;
  if (opts && opts->hybrid_level != 0)
    return kf_set_err(c, KF_EUNSUPPORTED, "batched: the hybrid solver is kf_factorize only");
  cudaStream_t s = (cudaStream_t)stream;
  // A single direct sweep of the batch hides the latency of the per-node LU
  // solves in its concurrent graph branches, so factors that are not refined
  // form no Z^-1 by default (measured on 256 problems of 2,048-32,768 points:
  // Z^-1 on levels of <= 64 nodes cost 37% more factorization time for 33%
  // less time of one solve).  Refined factors (the mixed path by default) run
  // several sweeps of all right-hand sides per solve, and there the LU solves,
  // one column after another on one CTA per node, dominated (11 of 23 s of
  // refined 64-RHS solves of that batch); they keep the default of kf_factorize.
  kf_opts ob = opts ? *opts : kf_opts{};
  const bool refined = ob.refine_max_iter > 0 || (ob.precision == KF_PREC_MIXED && ob.refine_max_iter == 0);
  if (ob.zinv_max_nodes == 0 && !refined) ob.zinv_max_nodes = -1;
  kf_status st = KF_OK;
  for (int32_t i = 0; i < nprob && st == KF_OK; ++i) st = alloc_factor(trees[i], h[i], lambda[i], tau[i], s_max, &ob, s, &out[i]);
  if (st == KF_OK) KF_CUDA(c, cudaStreamSynchronize(s));  // buffers zeroed before the graph runs
  if (st == KF_OK)
    st = run_batched_graph(c, nprob, s, [&](int32_t i, cudaStream_t si) -> kf_status {
      kf_status r = kf_skeletonize_device(out[i], si);
      return r == KF_OK ? kf_factorize_device(out[i], si) : r;
    });
  kf_status worst = st;
  if (st == KF_OK)
    for (int32_t i = 0; i < nprob; ++i) {
      kf_status r = read_status(out[i], s);
      if (r != KF_OK && r != KF_EILLCOND) worst = r;
      if (r == KF_EILLCOND && worst == KF_OK) worst = r;
    }
  if (st != KF_OK) {
    for (int32_t i = 0; i < nprob; ++i) {
      kf_factor_free(out[i]);
      out[i] = nullptr;
    }
    return st;
  }
  return worst;
}

kf_status kf_solve_batched(kf_factor* const* f, int32_t nprob, const void* const* B, void* const* X,
                           const int64_t* nrhs, const int64_t* ld, int32_t dtype, void* stream,
                           kf_solve_info* info) {
  if (!f || nprob < 1 || !B || !X || !nrhs || !ld) return kf_set_err(nullptr, KF_EINVAL, "batched solve: bad arguments");
  for (int32_t i = 0; i < nprob; ++i) {
    kf_status r = check_rhs(f[i], B[i], X[i], nrhs[i], ld[i], dtype);
    if (r != KF_OK) return r;
    if (!is_device_ptr(B[i]) || !is_device_ptr(X[i]))
      return kf_set_err(f[i]->ctx, KF_EINVAL, "batched solve: B and X must be device pointers");
  }
  kf_ctx* c = f[0]->ctx;
  bool any_refined = false;
  for (int32_t i = 0; i < nprob; ++i) any_refined = any_refined || refines(f[i]);
  if (any_refined) return solve_batched_refined(f, nprob, B, X, nrhs, ld, dtype, (cudaStream_t)stream, info);
  if (info)
    for (int32_t i = 0; i < nprob; ++i) info[i] = kf_solve_info{-1.0, 0, KF_OK};
  return run_batched_graph(c, nprob, (cudaStream_t)stream, [&](int32_t i, cudaStream_t si) -> kf_status {
    return with_vectors(f[i], B[i], X[i], nrhs[i], ld[i], dtype, si,
                        [&](double* W) { return kf_solve_device(f[i], W, nrhs[i], 0, si); });
  });
}

}  // extern "C"
