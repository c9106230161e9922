// knn.cu -- near-field sampling of S' (Sec. II-A samples the rows of a node's
// ID as ASKIT does, from the kappa nearest neighbours of the node's points,
// the paper's parameter kappa of Sec. IV, filled up with uniform samples).
//
//  1. Neighbours: knn_trees randomized projection trees over the tree
//     positions (kf_rp_order in tree.cu: every node split like the ball
//     tree's, by the order of (projection on x_q - x_p, position) with a
//     random pair p, q of the node's points).  Inside each leaf every point
//     compares itself with the leaf's other points at the FP32 squared
//     distance of the FP32 coordinates (sequential fused multiply-adds of
//     u = x_k - y_k), and keeps, over all trees, the kappa best (distance,
//     position) pairs with distinct positions (k_leaf_knn: one CTA per leaf,
//     the leaf's coordinates in shared memory, the query's coordinates and
//     its sorted list in registers).
//  2. Node lists (k_near_lists, one CTA per node of a level): a leaf counts
//     how often each position outside it occurs in its points' lists; a parent
//     adds its children's lists (counts of equal positions summed, positions
//     inside it dropped); each keeps the near_cap positions of largest count
//     (ties: smaller position), by two bitonic sorts in shared memory.
//  3. The sampler (skel.cu) takes the first min(list length, floor(n_s / 2))
//     entries of the node's list and draws the rest uniformly.
// Integer results throughout: the CUDA path and the oracle agree bit for bit.
#include <algorithm>

#include "kf_internal.cuh"
#include "prof.cuh"

namespace {

constexpr int kKnnThreads = 256;
constexpr int kKnnMaxD = 64;        // coordinates a query keeps in registers
constexpr int kNearThreads = 512;
constexpr int kNearMaxEntries = 16384;

inline int grid_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

__global__ void k_knn_init(float* __restrict__ bd, int32_t* __restrict__ bj, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    bd[i] = INFINITY;
    bj[i] = INT32_MAX;
  }
}

// One leaf of projection tree depth Dk per CTA; list width K >= kappa (the
// kappa best of the top-K lists are the kappa best of everything seen).
template <int K, bool REG>
__global__ void __launch_bounds__(kKnnThreads) k_leaf_knn(const float* __restrict__ X32, int d,
                                                          const int64_t* __restrict__ ord, int64_t N, int Dk,
                                                          float* __restrict__ bd, int32_t* __restrict__ bj) {
  extern __shared__ float sx[];  // nmax x d coordinates, then nmax positions
  const int64_t f = blockIdx.x;
  int64_t lo = 0, hi = N;
  for (int l = Dk - 1; l >= 0; --l) {  // the leaf's range: the halving of the complete tree
    const int64_t mid = lo + (hi - lo) / 2;
    if ((f >> l) & 1) lo = mid; else hi = mid;
  }
  const int n = (int)(hi - lo);
  int32_t* sp = (int32_t*)(sx + (size_t)n * d);
  for (int64_t e = threadIdx.x; e < (int64_t)n * d; e += blockDim.x) {
    const int64_t i = e / d;
    sx[e] = X32[ord[lo + i] * d + e % d];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) sp[i] = (int32_t)ord[lo + i];
  __syncthreads();
  for (int ii = threadIdx.x; ii < n; ii += blockDim.x) {
    const int32_t i = sp[ii];
    float dl[K];
    int32_t jl[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      dl[q] = bd[(int64_t)i * K + q];
      jl[q] = bj[(int64_t)i * K + q];
    }
    float xi[REG ? kKnnMaxD : 1];
    if (REG) {
#pragma unroll
      for (int k = 0; k < (REG ? kKnnMaxD : 1); ++k) xi[k] = k < d ? sx[(size_t)ii * d + k] : 0.f;
    }
    for (int jj = 0; jj < n; ++jj) {
      if (jj == ii) continue;
      const float* xj = sx + (size_t)jj * d;
      float acc = 0.f;
      if (REG) {
#pragma unroll
        for (int k = 0; k < (REG ? kKnnMaxD : 1); ++k) {
          if (k < d) {
            const float u = __fsub_rn(xi[k], xj[k]);
            acc = __fmaf_rn(u, u, acc);
          }
        }
      } else {
        for (int k = 0; k < d; ++k) {
          const float u = __fsub_rn(sx[(size_t)ii * d + k], xj[k]);
          acc = __fmaf_rn(u, u, acc);
        }
      }
      const int32_t j = sp[jj];
      if (acc < dl[K - 1] || (acc == dl[K - 1] && j < jl[K - 1])) {
        bool dup = false;
#pragma unroll
        for (int q = 0; q < K; ++q) dup |= (jl[q] == j);
        if (!dup) {  // insertion into the sorted list; the last entry falls off
          float cd = acc;
          int32_t cj = j;
#pragma unroll
          for (int q = 0; q < K; ++q) {
            const bool less = cd < dl[q] || (cd == dl[q] && cj < jl[q]);
            const float td = less ? dl[q] : cd;
            const int32_t tj = less ? jl[q] : cj;
            dl[q] = less ? cd : dl[q];
            jl[q] = less ? cj : jl[q];
            cd = td;
            cj = tj;
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      bd[(int64_t)i * K + q] = dl[q];
      bj[(int64_t)i * K + q] = jl[q];
    }
  }
}

// nbr[i][q] (q < kappa) from the width-K lists; empty slots become -1
__global__ void k_knn_finish(const int32_t* __restrict__ bj, int K, int kappa, int64_t N, int32_t* __restrict__ nbr) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * kappa;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = bj[(e / kappa) * K + e % kappa];
    nbr[e] = j == INT32_MAX ? -1 : j;
  }
}

__device__ void block_bitonic(unsigned long long* keys, int P) {
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < P; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          const bool asc = (t & k) == 0;
          const unsigned long long a = keys[t], b = keys[u];
          if ((a > b) == asc) {
            keys[t] = b;
            keys[u] = a;
          }
        }
      }
      __syncthreads();
    }
}

// Node lists of one level (one CTA per node).  mode 0 (leaves): entries
// (position, 1) from the points' neighbour lists; mode 1: (position, count)
// from the children's lists.  Entries inside the node are dropped.  Keys
// (position << 32 | weight) are sorted, runs of one position summed, then
// ((0xFFFFFFFF - count) << 32 | position) sorted and the first near_cap kept.
__global__ void __launch_bounds__(kNearThreads) k_near_lists(int mode, const int32_t* __restrict__ lo,
                                                             const int32_t* __restrict__ hi, int node0,
                                                             const int32_t* __restrict__ nbr, int kappa, int cap,
                                                             int32_t* __restrict__ near_pos,
                                                             int32_t* __restrict__ near_cnt,
                                                             int32_t* __restrict__ near_len, int pmax,
                                                             int32_t* __restrict__ status) {
  extern __shared__ unsigned long long keys[];  // pmax
  __shared__ int tsum[kNearThreads + 1];
  __shared__ int n_sh;
  const int node = node0 + blockIdx.x, tid = threadIdx.x;
  const int32_t b = lo[node], e = hi[node];
  if (tid == 0) n_sh = 0;
  __syncthreads();
  if (mode == 0) {
    for (int64_t x = tid; x < (int64_t)(e - b) * kappa; x += blockDim.x) {
      const int32_t j = nbr[(int64_t)b * kappa + x];
      if (j >= 0 && (j < b || j >= e)) {
        const int slot = atomicAdd(&n_sh, 1);
        if (slot < pmax) keys[slot] = ((unsigned long long)j << 32) | 1ull;
      }
    }
  } else {
    for (int c = 0; c < 2; ++c) {
      const int child = 2 * node + c, len = near_len[child];
      for (int q = tid; q < len; q += blockDim.x) {
        const int32_t j = near_pos[(int64_t)child * cap + q];
        if (j < b || j >= e) {
          const int slot = atomicAdd(&n_sh, 1);
          if (slot < pmax)
            keys[slot] = ((unsigned long long)j << 32) | (unsigned)near_cnt[(int64_t)child * cap + q];
        }
      }
    }
  }
  __syncthreads();
  if (n_sh > pmax) {  // excluded by the host's size check; flagged, never written out of bounds
    if (tid == 0) {
      atomicOr(status, KF_DEV_BADARG);
      near_len[node] = 0;
    }
    return;
  }
  const int n = n_sh;
  int P = 1;
  while (P < n) P <<= 1;
  for (int t = n + tid; t < P; t += blockDim.x) keys[t] = ~0ull;
  __syncthreads();
  block_bitonic(keys, P);
  // runs of equal positions: thread tid owns entries [t0, t1)
  const int E = (P + (int)blockDim.x - 1) / (int)blockDim.x;
  const int t0 = min(n, tid * E), t1 = min(n, t0 + E);
  int starts = 0;
  for (int t = t0; t < t1; ++t) starts += (t == 0 || (keys[t] >> 32) != (keys[t - 1] >> 32));
  tsum[tid] = starts;
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int q = 0; q < (int)blockDim.x; ++q) {
      const int v = tsum[q];
      tsum[q] = acc;
      acc += v;
    }
    tsum[blockDim.x] = acc;
  }
  __syncthreads();
  const int nu = tsum[blockDim.x];
  unsigned long long loc[kNearMaxEntries / kNearThreads];
  int nl = 0;
  for (int t = t0; t < t1; ++t) {
    if (!(t == 0 || (keys[t] >> 32) != (keys[t - 1] >> 32))) continue;
    const unsigned long long pos = keys[t] >> 32;
    unsigned long long sum = 0;
    for (int r = t; r < n && (keys[r] >> 32) == pos; ++r) sum += keys[r] & 0xFFFFFFFFull;
    if (sum > 0xFFFFFFFFull) sum = 0xFFFFFFFFull;
    loc[nl++] = ((0xFFFFFFFFull - sum) << 32) | pos;
  }
  __syncthreads();
  for (int q = 0; q < nl; ++q) keys[tsum[tid] + q] = loc[q];
  int P2 = 1;
  while (P2 < nu) P2 <<= 1;
  for (int t = nu + tid; t < P2; t += blockDim.x) keys[t] = ~0ull;
  __syncthreads();
  block_bitonic(keys, P2);
  const int keep = min(nu, cap);
  for (int q = tid; q < keep; q += blockDim.x) {
    near_pos[(int64_t)node * cap + q] = (int32_t)(keys[q] & 0xFFFFFFFFull);
    near_cnt[(int64_t)node * cap + q] = (int32_t)(0xFFFFFFFFull - (keys[q] >> 32));
  }
  if (tid == 0) near_len[node] = keep;
}

}  // namespace

kf_status kf_near_field_lists(kf_factor* f, cudaStream_t s) {
  kf_tree* t = f->t;
  kf_ctx* c = f->ctx;
  const int64_t N = t->N;
  const int d = t->d, kappa = f->knn_kappa, D = t->D;
  const int K = kappa <= 8 ? 8 : (kappa <= 16 ? 16 : 32);
  int Dk = 0;
  while (((int64_t)f->knn_leaf << Dk) < N) ++Dk;
  const int64_t nmax = (N + ((int64_t)1 << Dk) - 1) >> Dk;  // largest projection-tree leaf
  const size_t smem = (sizeof(float) * d + sizeof(int32_t)) * (size_t)nmax;
  if (smem > 227 * 1024)
    return kf_set_err(c, KF_EUNSUPPORTED, "near-field sampling: leaves of %lld points in %d dimensions exceed "
                      "shared memory (lower knn_leaf)", (long long)nmax, d);
  float* bdist = (float*)c->dalloc(sizeof(float) * (size_t)N * K, s);
  int32_t* bidx = (int32_t*)c->dalloc(sizeof(int32_t) * (size_t)N * K, s);
  int64_t* ord = (int64_t*)c->dalloc(sizeof(int64_t) * (size_t)N, s);
  kf_status st = (bdist && bidx && ord) ? KF_OK : kf_set_err(c, KF_ENOMEM, "near-field sampling: allocation failed");
  if (st == KF_OK) {
    KF_PHASE(KF_PH_NEAR, s, k_knn_init<<<grid_for(N * K, 256), 256, 0, s>>>(bdist, bidx, N * K));
    const bool reg = d <= kKnnMaxD;
    auto launch = [&](auto kern) -> kf_status {
      KF_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      KF_PHASE(KF_PH_NEAR, s, kern<<<(unsigned)(1u << Dk), kKnnThreads, smem, s>>>(t->X32, d, ord, N, Dk, bdist, bidx));
      KF_LAUNCH_CHECK(c);
      return KF_OK;
    };
    for (int tidx = 0; tidx < f->knn_trees && st == KF_OK; ++tidx) {
      st = kf_rp_order(t, tidx, Dk, f->seed, ord, s);
      if (st != KF_OK) break;
      if (K == 8) st = reg ? launch(k_leaf_knn<8, true>) : launch(k_leaf_knn<8, false>);
      else if (K == 16) st = reg ? launch(k_leaf_knn<16, true>) : launch(k_leaf_knn<16, false>);
      else st = reg ? launch(k_leaf_knn<32, true>) : launch(k_leaf_knn<32, false>);
    }
    if (st == KF_OK)
      KF_PHASE(KF_PH_NEAR, s, k_knn_finish<<<grid_for(N * kappa, 256), 256, 0, s>>>(bidx, K, kappa, N, f->nbr));
  }
  if (st == KF_OK && D > 0) {
    int pl = 1;
    while (pl < t->leaf_max * kappa) pl <<= 1;
    int pi = 1;
    while (pi < 2 * f->near_cap) pi <<= 1;
    const size_t sl = sizeof(unsigned long long) * pl, si = sizeof(unsigned long long) * pi;
    KF_CUDA(c, cudaFuncSetAttribute(k_near_lists, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)std::max(sl, si)));
    KF_PHASE(KF_PH_NEAR, s, k_near_lists<<<(unsigned)(1u << D), kNearThreads, sl, s>>>(
                                0, t->d_lo, t->d_hi, 1 << D, f->nbr, kappa, f->near_cap, f->near_pos, f->near_cnt,
                                f->near_len, pl, f->status));
    for (int l = D - 1; l >= 1; --l)
      KF_PHASE(KF_PH_NEAR, s, k_near_lists<<<(unsigned)(1u << l), kNearThreads, si, s>>>(
                                  1, t->d_lo, t->d_hi, 1 << l, f->nbr, kappa, f->near_cap, f->near_pos, f->near_cnt,
                                  f->near_len, pi, f->status));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = kf_set_err(c, KF_ECUDA, "near-field lists: %s", cudaGetErrorString(e));
  }
  c->dfree(bdist, sizeof(float) * (size_t)N * K, s);
  c->dfree(bidx, sizeof(int32_t) * (size_t)N * K, s);
  c->dfree(ord, sizeof(int64_t) * (size_t)N, s);
  return st;
}
