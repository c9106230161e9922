// tree.cu -- ball-tree partition of Sec. II-A ("Partitioning the matrix").
//
// Level by level, every node of the level is split at once:
//   a = the point with the smallest original index,
//   p = the point farthest from a, q = the point farthest from p (ties: the
//       smaller original index),
//   proj_i = sum_k (x_ik - x_pk)(x_qk - x_pk),
//   the node's points are ordered by (proj, original index) and the left child
//   takes the first floor(n/2).
// All FP64 arithmetic uses round-to-nearest intrinsics with no contraction so
// that the permutation is bit-identical to a sequential evaluation of the same
// formulas.  Per-node reductions run over fixed chunks of the node; the
// per-node sort is a bitonic network over segments padded to a power of two.
#include <algorithm>
#include <atomic>
#include <vector>

#include "kf_internal.cuh"
#include "prof.cuh"

namespace {

constexpr int kChunk = 4096;   // points per CTA in the per-node reductions
constexpr int kRedThreads = 256;
constexpr int kSortTile = 2048;  // elements sorted in shared memory per CTA

struct Cand {
  double v;
  int64_t orig;
  int32_t pos;
};

__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
  return a.v > b.v || (a.v == b.v && a.orig < b.orig);
}

__device__ __forceinline__ Cand shfl_cand(const Cand& c, int src_lane_delta) {
  Cand o;
  o.v = __shfl_down_sync(0xffffffffu, c.v, src_lane_delta);
  o.orig = __shfl_down_sync(0xffffffffu, c.orig, src_lane_delta);
  o.pos = __shfl_down_sync(0xffffffffu, c.pos, src_lane_delta);
  return o;
}

// Block-wide arg-reduction; result valid in thread 0.
__device__ Cand block_best(Cand c) {
  __shared__ Cand sh[32];
  for (int off = 16; off > 0; off >>= 1) {
    Cand o = shfl_cand(c, off);
    if (better(o, c)) c = o;
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = c;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
    c = lane < nw ? sh[lane] : Cand{-INFINITY, INT64_MAX, -1};
    for (int off = 16; off > 0; off >>= 1) {
      Cand o = shfl_cand(c, off);
      if (better(o, c)) c = o;
    }
  }
  return c;
}

// Phase 1 of a per-node arg-max.  mode 0: v = -orig (argmin of the original
// index); mode 1: v = ||x_i - x_ref(node)||^2.
__global__ void k_node_argmax_partial(const double* __restrict__ X, const int64_t* __restrict__ perm, int d,
                                      const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, int node0,
                                      int chunks_per_node, int mode, const int32_t* __restrict__ ref,
                                      Cand* __restrict__ partial) {
  int nl = blockIdx.y, node = node0 + nl, ch = blockIdx.x;
  int64_t b = lo[node], e = hi[node], n = e - b;
  int64_t cb = b + (n * ch) / chunks_per_node, ce = b + (n * (ch + 1)) / chunks_per_node;
  Cand best{-INFINITY, INT64_MAX, -1};
  const double* xr = nullptr;
  if (mode == 1) xr = X + (int64_t)ref[nl] * d;
  for (int64_t i = cb + threadIdx.x; i < ce; i += blockDim.x) {
    Cand c;
    c.orig = perm[i];
    c.pos = (int32_t)i;
    c.v = (mode == 0) ? -(double)c.orig : kf_sqdist64(X + i * d, xr, d);
    if (better(c, best)) best = c;
  }
  best = block_best(best);
  if (threadIdx.x == 0) partial[(int64_t)nl * chunks_per_node + ch] = best;
}

// Phase 2: one warp per node reduces its chunks; writes the winning position.
__global__ void k_node_argmax_final(const Cand* __restrict__ partial, int nnodes_level, int chunks_per_node,
                                    int32_t* __restrict__ out) {
  int nl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (nl >= nnodes_level) return;
  Cand best{-INFINITY, INT64_MAX, -1};
  for (int c = lane; c < chunks_per_node; c += 32) {
    Cand o = partial[(int64_t)nl * chunks_per_node + c];
    if (better(o, best)) best = o;
  }
  for (int off = 16; off > 0; off >>= 1) {
    Cand o = shfl_cand(best, off);
    if (better(o, best)) best = o;
  }
  if (lane == 0) out[nl] = best.pos;
}

// Projection keys, written into the padded sort segments.
__global__ void k_proj_keys(const double* __restrict__ X, const int64_t* __restrict__ perm, int d,
                            const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, int node0, int64_t seg,
                            const int32_t* __restrict__ pidx, const int32_t* __restrict__ qidx,
                            double* __restrict__ key, int64_t* __restrict__ orig, int32_t* __restrict__ pos) {
  int nl = blockIdx.y;
  int node = node0 + nl;
  int64_t b = lo[node], n = hi[node] - b;
  const double* xp = X + (int64_t)pidx[nl] * d;
  const double* xq = X + (int64_t)qidx[nl] * d;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < seg; j += (int64_t)gridDim.x * blockDim.x) {
    int64_t v = (int64_t)nl * seg + j;
    if (j < n) {
      int64_t i = b + j;
      const double* xi = X + i * d;
      double acc = 0.0;
      for (int k = 0; k < d; ++k) acc = __dadd_rn(acc, __dmul_rn(__dsub_rn(xi[k], xp[k]), __dsub_rn(xq[k], xp[k])));
      key[v] = acc;
      orig[v] = perm[i];
      pos[v] = (int32_t)i;
    } else {
      key[v] = INFINITY;
      orig[v] = INT64_MAX;
      pos[v] = -1;
    }
  }
}

__device__ __forceinline__ bool key_less(double ka, int64_t oa, double kb, int64_t ob) {
  return ka < kb || (ka == kb && oa < ob);
}

// One global compare-exchange pass (stride j within bitonic stage k).
__global__ void k_bitonic_global(double* __restrict__ key, int64_t* __restrict__ orig, int32_t* __restrict__ pos,
                                 int64_t total, int64_t seg, int64_t k, int64_t j) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < total; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t w = v ^ j;
    if (w <= v) continue;
    bool asc = ((v & (seg - 1)) & k) == 0;  // direction from the index inside the segment
    double kv = key[v], kw = key[w];
    int64_t ov = orig[v], ow = orig[w];
    bool swap = asc ? key_less(kw, ow, kv, ov) : key_less(kv, ov, kw, ow);
    if (swap) {
      key[v] = kw; key[w] = kv;
      orig[v] = ow; orig[w] = ov;
      int32_t t = pos[v]; pos[v] = pos[w]; pos[w] = t;
    }
  }
}

// Shared-memory passes: stages k <= kmax_stage (or the tail of a larger stage)
// for strides j < kSortTile, tile by tile.
__global__ void k_bitonic_shared(double* __restrict__ key, int64_t* __restrict__ orig, int32_t* __restrict__ pos,
                                 int64_t total, int64_t seg, int64_t k_begin, int64_t k_end, int64_t j_first) {
  __shared__ double sk[kSortTile];
  __shared__ int64_t so[kSortTile];
  __shared__ int32_t sp[kSortTile];
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int t = threadIdx.x; t < kSortTile; t += blockDim.x) {
    int64_t v = base + t;
    sk[t] = v < total ? key[v] : INFINITY;
    so[t] = v < total ? orig[v] : INT64_MAX;
    sp[t] = v < total ? pos[v] : -1;
  }
  __syncthreads();
  for (int64_t k = k_begin; k <= k_end; k <<= 1) {
    int64_t j0 = (k == k_begin) ? j_first : (k >> 1);
    for (int64_t j = j0; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < kSortTile; t += blockDim.x) {
        int u = t ^ (int)j;
        if (u <= t) continue;
        int64_t v = base + t;
        bool asc = ((v & (seg - 1)) & k) == 0;
        bool swap = asc ? key_less(sk[u], so[u], sk[t], so[t]) : key_less(sk[t], so[t], sk[u], so[u]);
        if (swap) {
          double a = sk[t]; sk[t] = sk[u]; sk[u] = a;
          int64_t b = so[t]; so[t] = so[u]; so[u] = b;
          int32_t c = sp[t]; sp[t] = sp[u]; sp[u] = c;
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < kSortTile; t += blockDim.x) {
    int64_t v = base + t;
    if (v < total) { key[v] = sk[t]; orig[v] = so[t]; pos[v] = sp[t]; }
  }
}

__global__ void k_gather_rows(const double* __restrict__ Xin, const int64_t* __restrict__ pin, int d,
                              const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, int node0, int64_t seg,
                              const int32_t* __restrict__ pos, double* __restrict__ Xout, int64_t* __restrict__ pout) {
  int nl = blockIdx.y;
  int node = node0 + nl;
  int64_t b = lo[node], n = hi[node] - b;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    int64_t src = pos[(int64_t)nl * seg + j];
    for (int k = 0; k < d; ++k) Xout[(b + j) * d + k] = Xin[src * d + k];
    pout[b + j] = pin[src];
  }
}

__global__ void k_to_f64(const float* __restrict__ in, double* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}
__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
// node ranges of the complete tree of depth D over N points (floor(n/2) to
// the left child), heap numbered
__global__ void k_node_ranges(int64_t N, int D, int32_t* __restrict__ lo, int32_t* __restrict__ hi) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  lo[1] = 0;
  hi[1] = (int32_t)N;
  for (int a = 1; a < (1 << D); ++a) {
    int32_t n = hi[a] - lo[a], mid = lo[a] + n / 2;
    lo[2 * a] = lo[a];
    hi[2 * a] = mid;
    lo[2 * a + 1] = mid;
    hi[2 * a + 1] = hi[a];
  }
}

// Randomized projection tree `tidx` (near-field sampling): the split points p
// and q of every node of a level, at offsets splitmix64(seed ^ (tidx << 56) ^
// (node << 1) ^ k) mod n (k = 0, 1) of the node's current list.
__global__ void k_rp_pairs(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, int node0, int nn,
                           uint64_t seed, int tidx, int32_t* __restrict__ ip, int32_t* __restrict__ iq) {
  for (int nl = blockIdx.x * blockDim.x + threadIdx.x; nl < nn; nl += gridDim.x * blockDim.x) {
    const int a = node0 + nl;
    const int64_t n = hi[a] - lo[a];
    const uint64_t key = seed ^ ((uint64_t)tidx << 56) ^ ((uint64_t)a << 1);
    ip[nl] = lo[a] + (n > 0 ? (int32_t)(kf_splitmix64(key ^ 0) % (uint64_t)n) : 0);
    iq[nl] = lo[a] + (n > 0 ? (int32_t)(kf_splitmix64(key ^ 1) % (uint64_t)n) : 0);
  }
}

__global__ void k_iota64(int64_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = i;
}
__global__ void k_check_finite(const double* __restrict__ x, int64_t n, int32_t* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicOr(bad, 1);
}

inline int grid_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

}  // namespace

kf_status kf_to_f64_launch(const float* in, double* out, int64_t n, cudaStream_t s) {
  KF_PHASE(KF_PH_MISC, s, k_to_f64<<<grid_for(n, 256), 256, 0, s>>>(in, out, n));
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ECUDA;
}
__global__ void k_split_lo(const double* __restrict__ in, const float* __restrict__ hi, float* __restrict__ lo, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    lo[i] = (float)(in[i] - (double)hi[i]);
}
kf_status kf_split_lo_launch(const double* in, const float* hi, float* lo, int64_t n, cudaStream_t s) {
  KF_PHASE(KF_PH_MISC, s, k_split_lo<<<grid_for(n, 256), 256, 0, s>>>(in, hi, lo, n));
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ECUDA;
}
kf_status kf_to_f32_launch(const double* in, float* out, int64_t n, cudaStream_t s) {
  KF_PHASE(KF_PH_MISC, s, k_to_f32<<<grid_for(n, 256), 256, 0, s>>>(in, out, n));
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ECUDA;
}
kf_status kf_check_finite_launch(const double* x, int64_t n, int32_t* bad, cudaStream_t s) {
  KF_PHASE(KF_PH_MISC, s, k_check_finite<<<grid_for(n, 256), 256, 0, s>>>(x, n, bad));
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ECUDA;
}

// Builds the tree on t->X64 (original order on entry, tree order on exit).
kf_status kf_tree_build_device(kf_tree* t, cudaStream_t s) {
  kf_ctx* c = t->ctx;
  const int64_t N = t->N;
  const int d = t->d;
  KF_PHASE(KF_PH_TREE, s, k_iota64<<<grid_for(N, 256), 256, 0, s>>>(t->perm, N));
  KF_LAUNCH_CHECK(c);
  if (t->D == 0) return KF_OK;
  int64_t segmax = 1;
  while (segmax < N) segmax <<= 1;
  const int64_t vcap = 2 * segmax;
  const int maxnodes = 1 << (t->D - 1);
  const int cpn_max = (int)((N + kChunk - 1) / kChunk) + 1;
  size_t bytes_X = sizeof(double) * N * d, bytes_p = sizeof(int64_t) * N;
  double* X2 = (double*)c->dalloc(bytes_X, s);
  int64_t* p2 = (int64_t*)c->dalloc(bytes_p, s);
  double* key = (double*)c->dalloc(sizeof(double) * vcap, s);
  int64_t* orig = (int64_t*)c->dalloc(sizeof(int64_t) * vcap, s);
  int32_t* pos = (int32_t*)c->dalloc(sizeof(int32_t) * vcap, s);
  Cand* part = (Cand*)c->dalloc(sizeof(Cand) * (size_t)maxnodes * cpn_max, s);
  int32_t* ia = (int32_t*)c->dalloc(sizeof(int32_t) * 3 * maxnodes, s);
  kf_status st = KF_OK;
  if (!X2 || !p2 || !key || !orig || !pos || !part || !ia) {
    st = kf_set_err(c, KF_ENOMEM, "tree build: allocation failed");
  } else {
    int32_t* ip = ia + maxnodes;
    int32_t* iq = ia + 2 * maxnodes;
    double* Xa = t->X64;
    int64_t* pa = t->perm;
    double* Xb = X2;
    int64_t* pb = p2;
    for (int l = 0; l < t->D && st == KF_OK; ++l) {
      int node0 = 1 << l, nn = 1 << l;
      int64_t nmax = 0;
      for (int a = node0; a < 2 * node0; ++a) nmax = std::max<int64_t>(nmax, t->hi[a] - t->lo[a]);
      int cpn = (int)((nmax + kChunk - 1) / kChunk);
      if (cpn < 1) cpn = 1;
      dim3 g(cpn, nn);
      KF_PHASE(KF_PH_TREE, s, k_node_argmax_partial<<<g, kRedThreads, 0, s>>>(Xa, pa, d, t->d_lo, t->d_hi, node0, cpn, 0, nullptr, part));
      KF_PHASE(KF_PH_TREE, s, k_node_argmax_final<<<(nn + 7) / 8, 256, 0, s>>>(part, nn, cpn, ia));
      KF_PHASE(KF_PH_TREE, s, k_node_argmax_partial<<<g, kRedThreads, 0, s>>>(Xa, pa, d, t->d_lo, t->d_hi, node0, cpn, 1, ia, part));
      KF_PHASE(KF_PH_TREE, s, k_node_argmax_final<<<(nn + 7) / 8, 256, 0, s>>>(part, nn, cpn, ip));
      KF_PHASE(KF_PH_TREE, s, k_node_argmax_partial<<<g, kRedThreads, 0, s>>>(Xa, pa, d, t->d_lo, t->d_hi, node0, cpn, 1, ip, part));
      KF_PHASE(KF_PH_TREE, s, k_node_argmax_final<<<(nn + 7) / 8, 256, 0, s>>>(part, nn, cpn, iq));
      int64_t seg = 1;
      while (seg < nmax) seg <<= 1;
      if (seg < 2) seg = 2;
      int64_t total = seg * nn;
      dim3 gk((unsigned)std::min<int64_t>((seg + 255) / 256, 4096), nn);
      KF_PHASE(KF_PH_TREE, s, k_proj_keys<<<gk, 256, 0, s>>>(Xa, pa, d, t->d_lo, t->d_hi, node0, seg, ip, iq, key, orig, pos));
      // bitonic sort of every segment of length seg
      int tiles = (int)((total + kSortTile - 1) / kSortTile);
      int64_t ktile = std::min<int64_t>(seg, kSortTile);
      KF_PHASE(KF_PH_TREE, s, k_bitonic_shared<<<tiles, 512, 0, s>>>(key, orig, pos, total, seg, 2, ktile, 1));
      for (int64_t k = 2 * kSortTile; k <= seg; k <<= 1) {
        for (int64_t j = k >> 1; j >= kSortTile; j >>= 1)
          KF_PHASE(KF_PH_TREE, s, k_bitonic_global<<<grid_for(total, 256), 256, 0, s>>>(key, orig, pos, total, seg, k, j));
        KF_PHASE(KF_PH_TREE, s, k_bitonic_shared<<<tiles, 512, 0, s>>>(key, orig, pos, total, seg, k, k, kSortTile / 2));
      }
      KF_PHASE(KF_PH_TREE, s, k_gather_rows<<<gk, 256, 0, s>>>(Xa, pa, d, t->d_lo, t->d_hi, node0, seg, pos, Xb, pb));
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) st = kf_set_err(c, KF_ECUDA, "tree build level %d: %s", l, cudaGetErrorString(e));
      std::swap(Xa, Xb);
      std::swap(pa, pb);
    }
    if (st == KF_OK && Xa != t->X64) {
      cudaMemcpyAsync(t->X64, Xa, bytes_X, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(t->perm, pa, bytes_p, cudaMemcpyDeviceToDevice, s);
    }
  }
  c->dfree(X2, bytes_X, s);
  c->dfree(p2, bytes_p, s);
  c->dfree(key, sizeof(double) * vcap, s);
  c->dfree(orig, sizeof(int64_t) * vcap, s);
  c->dfree(pos, sizeof(int32_t) * vcap, s);
  c->dfree(part, sizeof(Cand) * (size_t)maxnodes * cpn_max, s);
  c->dfree(ia, sizeof(int32_t) * 3 * maxnodes, s);
  return st;
}

// ---- allocation-free variant of the tree build ------------------------------------
//
// Near-field sampling: the order of the tree positions under randomized
// projection tree `tidx` of depth Dk (every node split like the ball tree's,
// by the order of (projection on x_q - x_p, position), p and q from
// k_rp_pairs); the leaves are the contiguous ranges of the complete tree of
// depth Dk.  ord: device, N int64.  The same projection, sort and gather
// kernels as the ball tree; coordinates from the tree's FP64 copy.
kf_status kf_rp_order(kf_tree* t, int tidx, int Dk, uint64_t seed, int64_t* ord, cudaStream_t s) {
  kf_ctx* c = t->ctx;
  const int64_t N = t->N;
  const int d = t->d;
  KF_PHASE(KF_PH_NEAR, s, k_iota64<<<grid_for(N, 256), 256, 0, s>>>(ord, N));
  KF_LAUNCH_CHECK(c);
  if (Dk == 0) return KF_OK;
  int64_t segmax = 1;
  while (segmax < N) segmax <<= 1;
  const int64_t vcap = 2 * segmax;
  const int maxnodes = 1 << (Dk - 1);
  const int nn_all = 2 << Dk;
  std::vector<int32_t> hlo(nn_all, 0), hhi(nn_all, 0);
  hlo[1] = 0;
  hhi[1] = (int32_t)N;
  for (int a = 1; a < (1 << Dk); ++a) {
    int32_t n = hhi[a] - hlo[a], mid = hlo[a] + n / 2;
    hlo[2 * a] = hlo[a]; hhi[2 * a] = mid; hlo[2 * a + 1] = mid; hhi[2 * a + 1] = hhi[a];
  }
  size_t bytes_X = sizeof(double) * N * d, bytes_p = sizeof(int64_t) * N;
  double* Xa = (double*)c->dalloc(bytes_X, s);
  double* Xb = (double*)c->dalloc(bytes_X, s);
  int64_t* pb = (int64_t*)c->dalloc(bytes_p, s);
  double* key = (double*)c->dalloc(sizeof(double) * vcap, s);
  int64_t* orig = (int64_t*)c->dalloc(sizeof(int64_t) * vcap, s);
  int32_t* pos = (int32_t*)c->dalloc(sizeof(int32_t) * vcap, s);
  int32_t* ia = (int32_t*)c->dalloc(sizeof(int32_t) * 2 * maxnodes, s);
  int32_t* rlo = (int32_t*)c->dalloc(sizeof(int32_t) * nn_all, s);
  int32_t* rhi = (int32_t*)c->dalloc(sizeof(int32_t) * nn_all, s);
  kf_status st = KF_OK;
  if (!Xa || !Xb || !pb || !key || !orig || !pos || !ia || !rlo || !rhi) {
    st = kf_set_err(c, KF_ENOMEM, "near-field sampling: allocation failed");
  } else {
    cudaMemcpyAsync(Xa, t->X64, bytes_X, cudaMemcpyDeviceToDevice, s);
    KF_PHASE(KF_PH_NEAR, s, k_node_ranges<<<1, 1, 0, s>>>(N, Dk, rlo, rhi));
    int32_t* ip = ia;
    int32_t* iq = ia + maxnodes;
    int64_t* pa = ord;
    for (int l = 0; l < Dk && st == KF_OK; ++l) {
      const int node0 = 1 << l, nn = 1 << l;
      int64_t nmax = 0;
      for (int a = node0; a < 2 * node0; ++a) nmax = std::max<int64_t>(nmax, hhi[a] - hlo[a]);
      KF_PHASE(KF_PH_NEAR, s, k_rp_pairs<<<(nn + 127) / 128, 128, 0, s>>>(rlo, rhi, node0, nn, seed, tidx, ip, iq));
      int64_t seg = 1;
      while (seg < nmax) seg <<= 1;
      if (seg < 2) seg = 2;
      const int64_t total = seg * nn;
      dim3 gk((unsigned)std::min<int64_t>((seg + 255) / 256, 4096), nn);
      KF_PHASE(KF_PH_NEAR, s, k_proj_keys<<<gk, 256, 0, s>>>(Xa, pa, d, rlo, rhi, node0, seg, ip, iq, key, orig, pos));
      const int tiles = (int)((total + kSortTile - 1) / kSortTile);
      const int64_t ktile = std::min<int64_t>(seg, kSortTile);
      KF_PHASE(KF_PH_NEAR, s, k_bitonic_shared<<<tiles, 512, 0, s>>>(key, orig, pos, total, seg, 2, ktile, 1));
      for (int64_t k = 2 * kSortTile; k <= seg; k <<= 1) {
        for (int64_t j = k >> 1; j >= kSortTile; j >>= 1)
          KF_PHASE(KF_PH_NEAR, s, k_bitonic_global<<<grid_for(total, 256), 256, 0, s>>>(key, orig, pos, total, seg, k, j));
        KF_PHASE(KF_PH_NEAR, s, k_bitonic_shared<<<tiles, 512, 0, s>>>(key, orig, pos, total, seg, k, k, kSortTile / 2));
      }
      KF_PHASE(KF_PH_NEAR, s, k_gather_rows<<<gk, 256, 0, s>>>(Xa, pa, d, rlo, rhi, node0, seg, pos, Xb, pb));
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) st = kf_set_err(c, KF_ECUDA, "projection tree level %d: %s", l, cudaGetErrorString(e));
      std::swap(Xa, Xb);
      std::swap(pa, pb);
    }
    if (st == KF_OK && pa != ord) cudaMemcpyAsync(ord, pa, bytes_p, cudaMemcpyDeviceToDevice, s);
    // the ping-pong may have swapped the caller's buffer into pb: free the other one
    if (pb == ord) pb = pa;
  }
  c->dfree(Xa, bytes_X, s);
  c->dfree(Xb, bytes_X, s);
  c->dfree(pb, bytes_p, s);
  c->dfree(key, sizeof(double) * vcap, s);
  c->dfree(orig, sizeof(int64_t) * vcap, s);
  c->dfree(pos, sizeof(int32_t) * vcap, s);
  c->dfree(ia, sizeof(int32_t) * 2 * maxnodes, s);
  c->dfree(rlo, sizeof(int32_t) * nn_all, s);
  c->dfree(rhi, sizeof(int32_t) * nn_all, s);
  return st;
}

// kf_tree_perm_noalloc runs the same kernels as kf_tree_build_device but takes
// every scratch buffer from one file-scope device array instead of the
// allocator, and uses the caller's outputs as the other half of each
// ping-pong pair.  Limits: N <= 65536 and N * d <= 2^19, which keep the
// array at 12 MiB (held by every GPU that loads the library until exit).
namespace {

constexpr int64_t kNoAllocMaxN = 65536;
constexpr int64_t kNoAllocMaxND = int64_t(1) << 19;
constexpr size_t kNoAllocBytes = size_t(12) << 20;
constexpr int kNoAllocMaxDevices = 64;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

static __device__ __align__(256) unsigned char kf_noalloc_tree_scratch[kNoAllocBytes];

extern "C" kf_status kf_tree_perm_noalloc(const double* X, int64_t N, int32_t d, int32_t m, double* Xt,
                                          int64_t* perm, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!X || !Xt || !perm) return kf_set_err(nullptr, KF_EINVAL, "kf_tree_perm_noalloc: NULL pointer");
  if (N < 1 || N > kNoAllocMaxN)
    return kf_set_err(nullptr, KF_EINVAL, "kf_tree_perm_noalloc: N = %lld outside [1, %lld]", (long long)N,
                      (long long)kNoAllocMaxN);
  if (d < 1 || d > KF_MAX_D)
    return kf_set_err(nullptr, KF_EINVAL, "kf_tree_perm_noalloc: d = %d outside [1, %d]", d, KF_MAX_D);
  if ((int64_t)N * d > kNoAllocMaxND)
    return kf_set_err(nullptr, KF_EINVAL, "kf_tree_perm_noalloc: N * d = %lld exceeds %lld", (long long)N * d,
                      (long long)kNoAllocMaxND);
  if (m < 1) return kf_set_err(nullptr, KF_EINVAL, "kf_tree_perm_noalloc: m must be >= 1");
  // Device address of the scratch array, looked up once per device.  Each
  // entry is atomic, so first calls from several host threads (on the same or
  // different devices) at worst look the same address up twice.
  static std::atomic<void*> dev_ptr[kNoAllocMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0)
    return kf_set_err(nullptr, KF_ECUDA, "kf_tree_perm_noalloc: no current device");
  if (dev >= kNoAllocMaxDevices)
    return kf_set_err(nullptr, KF_EUNSUPPORTED, "kf_tree_perm_noalloc: device index %d, only devices 0..%d are "
                      "supported", dev, kNoAllocMaxDevices - 1);
  if (!dev_ptr[dev].load(std::memory_order_acquire)) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, kf_noalloc_tree_scratch);
    if (e != cudaSuccess)
      return kf_set_err(nullptr, KF_ECUDA, "kf_tree_perm_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    dev_ptr[dev].store(p, std::memory_order_release);
  }
  int D = 0;
  while (((int64_t)m << D) < N) ++D;
  const int nnodes = (1 << (D + 1)) - 1;
  int64_t segmax = 1;
  while (segmax < N) segmax <<= 1;
  const int64_t vcap = 2 * segmax;
  const int maxnodes = D > 0 ? 1 << (D - 1) : 1;
  const int64_t part_cap = (N + kChunk - 1) / kChunk + 2 + 2 * (int64_t)maxnodes;
  // carve the scratch array
  unsigned char* base = (unsigned char*)dev_ptr[dev].load(std::memory_order_acquire);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* q = base + off;
    off = align256(off + bytes);
    return q;
  };
  double* Xb = (double*)take(sizeof(double) * N * d);
  int64_t* pb = (int64_t*)take(sizeof(int64_t) * N);
  double* key = (double*)take(sizeof(double) * vcap);
  int64_t* orig = (int64_t*)take(sizeof(int64_t) * vcap);
  int32_t* pos = (int32_t*)take(sizeof(int32_t) * vcap);
  Cand* part = (Cand*)take(sizeof(Cand) * part_cap);
  int32_t* ia = (int32_t*)take(sizeof(int32_t) * 3 * maxnodes);
  int32_t* lo = (int32_t*)take(sizeof(int32_t) * (nnodes + 1));
  int32_t* hi = (int32_t*)take(sizeof(int32_t) * (nnodes + 1));
  int32_t* bad = (int32_t*)take(sizeof(int32_t));
  if (off > kNoAllocBytes)
    return kf_set_err(nullptr, KF_EINVAL, "kf_tree_perm_noalloc: scratch of %zu bytes needed, %zu available", off,
                      kNoAllocBytes);
  // check X before any output is written (Xt and perm stay untouched when it
  // holds a non-finite coordinate), then copy it, node ranges, identity order
  if (cudaMemsetAsync(bad, 0, sizeof(int32_t), s) != cudaSuccess)
    return kf_set_err(nullptr, KF_ECUDA, "kf_tree_perm_noalloc: %s", cudaGetErrorString(cudaGetLastError()));
  KF_PHASE(KF_PH_MISC, s, k_check_finite<<<grid_for(N * d, 256), 256, 0, s>>>(X, N * d, bad));
  int32_t hbad = 0;
  if (cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return kf_set_err(nullptr, KF_ECUDA, "kf_tree_perm_noalloc: %s", cudaGetErrorString(cudaGetLastError()));
  if (hbad) return kf_set_err(nullptr, KF_EINVAL, "kf_tree_perm_noalloc: X has non-finite coordinates");
  if (cudaMemcpyAsync(Xt, X, sizeof(double) * N * d, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return kf_set_err(nullptr, KF_ECUDA, "kf_tree_perm_noalloc: %s", cudaGetErrorString(cudaGetLastError()));
  KF_PHASE(KF_PH_TREE, s, k_node_ranges<<<1, 1, 0, s>>>(N, D, lo, hi));
  KF_PHASE(KF_PH_TREE, s, k_iota64<<<grid_for(N, 256), 256, 0, s>>>(perm, N));
  int32_t* ip = ia + maxnodes;
  int32_t* iq = ia + 2 * maxnodes;
  double* Xa = Xt;
  int64_t* pa = perm;
  double* Xc = Xb;
  int64_t* pc = pb;
  for (int l = 0; l < D; ++l) {
    const int node0 = 1 << l, nn = 1 << l;
    const int64_t nmax = (N + (int64_t(1) << l) - 1) >> l;  // ceil(N / 2^l): the largest node of the level
    int cpn = (int)((nmax + kChunk - 1) / kChunk);
    if (cpn < 1) cpn = 1;
    dim3 g(cpn, nn);
    KF_PHASE(KF_PH_TREE, s, k_node_argmax_partial<<<g, kRedThreads, 0, s>>>(Xa, pa, d, lo, hi, node0, cpn, 0, nullptr, part));
    KF_PHASE(KF_PH_TREE, s, k_node_argmax_final<<<(nn + 7) / 8, 256, 0, s>>>(part, nn, cpn, ia));
    KF_PHASE(KF_PH_TREE, s, k_node_argmax_partial<<<g, kRedThreads, 0, s>>>(Xa, pa, d, lo, hi, node0, cpn, 1, ia, part));
    KF_PHASE(KF_PH_TREE, s, k_node_argmax_final<<<(nn + 7) / 8, 256, 0, s>>>(part, nn, cpn, ip));
    KF_PHASE(KF_PH_TREE, s, k_node_argmax_partial<<<g, kRedThreads, 0, s>>>(Xa, pa, d, lo, hi, node0, cpn, 1, ip, part));
    KF_PHASE(KF_PH_TREE, s, k_node_argmax_final<<<(nn + 7) / 8, 256, 0, s>>>(part, nn, cpn, iq));
    int64_t seg = 1;
    while (seg < nmax) seg <<= 1;
    if (seg < 2) seg = 2;
    const int64_t total = seg * nn;
    dim3 gk((unsigned)std::min<int64_t>((seg + 255) / 256, 4096), nn);
    KF_PHASE(KF_PH_TREE, s, k_proj_keys<<<gk, 256, 0, s>>>(Xa, pa, d, lo, hi, node0, seg, ip, iq, key, orig, pos));
    const int tiles = (int)((total + kSortTile - 1) / kSortTile);
    const int64_t ktile = std::min<int64_t>(seg, kSortTile);
    KF_PHASE(KF_PH_TREE, s, k_bitonic_shared<<<tiles, 512, 0, s>>>(key, orig, pos, total, seg, 2, ktile, 1));
    for (int64_t k = 2 * kSortTile; k <= seg; k <<= 1) {
      for (int64_t j = k >> 1; j >= kSortTile; j >>= 1)
        KF_PHASE(KF_PH_TREE, s, k_bitonic_global<<<grid_for(total, 256), 256, 0, s>>>(key, orig, pos, total, seg, k, j));
      KF_PHASE(KF_PH_TREE, s, k_bitonic_shared<<<tiles, 512, 0, s>>>(key, orig, pos, total, seg, k, k, kSortTile / 2));
    }
    KF_PHASE(KF_PH_TREE, s, k_gather_rows<<<gk, 256, 0, s>>>(Xa, pa, d, lo, hi, node0, seg, pos, Xc, pc));
    std::swap(Xa, Xc);
    std::swap(pa, pc);
  }
  if (Xa != Xt) {
    cudaMemcpyAsync(Xt, Xa, sizeof(double) * N * d, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(perm, pa, sizeof(int64_t) * N, cudaMemcpyDeviceToDevice, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return kf_set_err(nullptr, KF_ECUDA, "kf_tree_perm_noalloc: %s", cudaGetErrorString(e));
  return KF_OK;
}
