// solve.cu -- Algorithm 3 (solve), its transpose, the hierarchical operator
// lambda I + K~ (second form of Eq. e:uv) and dK~/dh, all level by level.
//
// Vectors live in tree order as N x k row-major blocks.  Per level l+1 the
// sweeps are two streaming passes over N x s_max matrices:
//   colsum:  u[b] = M[b rows, :cnt]^T w[b rows]      (segmented reduction)
//   rowupd:  w[b rows] += sign * M[b rows, :cnt] v[b] (per-row dot products)
// with M = VT (the V blocks K_{sib~ b}) or P^ (the W blocks), stored or
// evaluated on the fly, and a small FP64 solve with Z per parent in between.
//
// Forward solve (Algorithm 3, bottom-up): w = L^-T L^-1 b at the leaves; for
//   each level: g[l] = K_{l~ r} w_r, g[r] = K_{r~ l} w_l; t = Z^-1 [g_l; g_r];
//   w_l -= P^_l t_top; w_r -= P^_r t_bot.
// Transpose solve (top-down): t = Z^-T [P^_l^T w_l; P^_r^T w_r];
//   w_l -= K_{r~ l}^T t_bot; w_r -= K_{l~ r}^T t_top; then the leaves.
// Operator: leaves (lambda I + K_aa) x; g[c] = K_{c~ sib} x_sib for every
//   non-root c; pushed down g[children] += P_c g[parent]; y += P_{leaf} g.
// Transposed operator: leaves as above (K_aa is symmetric); g[leaf] =
//   P_{leaf}^T x; gathered up g[parent] += P_c^T [g[l]; g[r]]; then for every
//   non-root c, y_c += K_{c sib~} g[sib] (the transpose of K~_{sib c} =
//   P_{sib sib~} K_{sib~ c}).
#include <algorithm>
#include <cstring>

#include "kf_internal.cuh"
#include "prof.cuh"

namespace {

inline int grid_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

enum Src { SRC_STORED = 0, SRC_KERNEL = 1, SRC_DKERNEL = 2 };

// Kernel entry (or its h-derivative) between tree positions i and j, FP32
// evaluation for float matrices, FP64 for double.
template <typename TM>
__device__ __forceinline__ double eval_src(int src, const double* X64, const float* X32, int64_t i, int64_t j, int d,
                                           double c_exp, double inv_h3) {
  if (sizeof(TM) == 8) {
    double d2 = kf_sqdist64(X64 + i * d, X64 + j * d, d);
    double k = exp(d2 * c_exp);
    return src == SRC_DKERNEL ? k * d2 * inv_h3 : k;
  } else {
    const float* x = X32 + i * d;
    const float* y = X32 + j * d;
    float acc = 0.f;
    for (int t = 0; t < d; ++t) {
      float u = x[t] - y[t];
      acc = fmaf(u, u, acc);
    }
    float k = __expf(acc * (float)c_exp);
    return src == SRC_DKERNEL ? (double)(k * acc * (float)inv_h3) : (double)k;
  }
}

// ---- leaf triangular solves: Y <- L^-T L^-1 Y, Y rows = the leaf's points ----
// Blocks of 32 rows: warp 0 solves the diagonal block with shuffles (lane i
// holds row kb + i), then every thread updates one row of the rest of the
// leaf with the solved block (two barriers per block).
// y[i] -= sum_{j < nb} M[i][kb + j] x[j] for rows [r0, r1) of a row-major
// matrix (row i at rowp(i)): a warp takes 32 rows at a time, loads the 32 x 32
// tile row by row (each row one coalesced segment) into its shared-memory
// tile, then lane q forms row q's dot product.  x has 32 entries (zero past nb).
template <typename TM, typename TV, typename RowPtr, typename Out>
__device__ __forceinline__ void warp_tile_rowupd(int r0, int r1, int kb, int nb, RowPtr rowp, const TV* x,
                                                 Out out, TM (*tile)[33]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = r0 + warp * 32; i0 < r1; i0 += nw * 32) {
    TM v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = (i0 + q < r1 && lane < nb) ? rowp(i0 + q)[kb + lane] : (TM)0;
#pragma unroll
    for (int q = 0; q < 32; ++q) tile[q][lane] = v[q];
    __syncwarp();
    if (i0 + lane < r1) {
      TV acc = (TV)0;
#pragma unroll
      for (int j = 0; j < 32; ++j) acc += (TV)tile[lane][j] * x[j];
      out(i0 + lane, acc);
    }
    __syncwarp();
  }
}

// 128 threads a CTA, 8 (FP32) or 4 (FP64) CTAs an SM: with 256 threads and
// half as many CTAs, 1024 leaves took 1.7 rounds of the 608 slots (FP32) and
// the second round ran two thirds full.
constexpr int kLeafSolveThreads = 128;
template <typename TM, typename TV>
__global__ void __launch_bounds__(kLeafSolveThreads, sizeof(TM) == 4 ? 8 : 4) k_leaf_solve(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                    int leaf0, int ldL, const TM* __restrict__ Lall,
                                                    TV* __restrict__ W, int k) {
  constexpr int NB = 32, NQ = NB * NB / kLeafSolveThreads;  // diagonal-block entries per thread
  __shared__ TV xb[NB];
  __shared__ TM db[NB][NB + 1];  // the staged diagonal block
  __shared__ TV dinv[NB];        // reciprocals of its diagonal (divisions in parallel)
  extern __shared__ unsigned char lsm[];
  TM (*wtile)[33] = (TM (*)[33])lsm;  // one 32 x 32 row tile per warp (row updates), dynamic
  const int lf = blockIdx.x, node = leaf0 + lf;
  const int b = lo[node], n = hi[node] - b;
  const TM* L = Lall + (int64_t)lf * ldL * ldL;
  TV* Y = W + (int64_t)b * k;
  const int tid = threadIdx.x, lane = tid & 31;
  // diagonal blocks fetched into registers one block ahead, then committed
  // to shared memory; warp 0 forms the reciprocals of the diagonal
  TM pre[NQ];
  auto fetch = [&](int kb, int nb) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int e = q * kLeafSolveThreads + tid, i = e >> 5, j = e & 31;
      pre[q] = (i < nb && j <= i) ? L[(int64_t)(kb + i) * ldL + kb + j] : (TM)0;
    }
  };
  auto commit = [&](int nb) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int e = q * kLeafSolveThreads + tid;
      db[e >> 5][e & 31] = pre[q];
    }
    __syncthreads();
    if (tid < NB) {
      dinv[lane] = lane < nb ? (TV)1 / (TV)db[lane][lane] : (TV)0;
      __syncwarp();
    }
  };
  const int top = n > 0 ? ((n - 1) / NB) * NB : 0;
  for (int r = 0; r < k; ++r) {
    // forward: L y = b
    if (n > 0) fetch(0, min(NB, n));
    for (int kb = 0; kb < n; kb += NB) {
      const int nb = min(NB, n - kb);
      commit(nb);
      if (tid < 32) {
        TV yi = lane < nb ? Y[(int64_t)(kb + lane) * k + r] : (TV)0;
        for (int j = 0; j < nb; ++j) {
          if (lane == j) yi *= dinv[j];
          const TV yj = __shfl_sync(0xffffffffu, yi, j);
          if (lane > j && lane < nb) yi -= (TV)db[lane][j] * yj;
        }
        xb[lane] = lane < nb ? yi : (TV)0;
        if (lane < nb) Y[(int64_t)(kb + lane) * k + r] = yi;
      }
      __syncthreads();
      if (kb + NB < n) fetch(kb + NB, min(NB, n - kb - NB));
      warp_tile_rowupd<TM, TV>(kb + nb, n, kb, nb, [&](int i) { return L + (int64_t)i * ldL; }, xb,
                               [&](int i, TV acc) { Y[(int64_t)i * k + r] -= acc; }, wtile + (tid >> 5) * 32);
      __syncthreads();
    }
    // backward: L^T x = y
    if (n > 0) fetch(top, n - top);
    for (int kb = top; kb >= 0 && n > 0; kb -= NB) {
      const int nb = min(NB, n - kb);
      commit(nb);
      if (tid < 32) {
        TV xi = lane < nb ? Y[(int64_t)(kb + lane) * k + r] : (TV)0;
        for (int j = nb - 1; j >= 0; --j) {
          if (lane == j) xi *= dinv[j];
          const TV xj = __shfl_sync(0xffffffffu, xi, j);
          if (lane < j) xi -= (TV)db[j][lane] * xj;
        }
        xb[lane] = lane < nb ? xi : (TV)0;
        if (lane < nb) Y[(int64_t)(kb + lane) * k + r] = xi;
      }
      __syncthreads();
      if (kb >= NB) fetch(kb - NB, NB);
      for (int i = tid; i < kb; i += blockDim.x) {
        TM v[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) v[j] = j < nb ? L[(int64_t)(kb + j) * ldL + i] : (TM)0;
        TV acc = (TV)0;
#pragma unroll
        for (int j = 0; j < NB; ++j) acc += (TV)v[j] * xb[j];
        Y[(int64_t)i * k + r] -= acc;
      }
      __syncthreads();
    }
  }
}

// Several right-hand sides per pass (k >= 2): the leaf's KC columns of the
// right-hand side stay in shared memory for the whole forward and backward
// sweep, so that L is streamed once per KC columns instead of once per column
// and every loaded entry of L serves KC products.  Per 32-row block the
// diagonal block is staged in shared memory and each warp solves KC / 8 of its
// columns with shuffles; then every thread updates one row of the rest of the
// leaf for all KC columns (forward: row i of L, entries kb..kb+31; backward:
// column i of L, a coalesced read across the threads).  Per column the
// operations and their order are those of k_leaf_solve.  Shared-memory rows
// are KC + 16 / sizeof(TV) values long (a 16-byte multiple that makes the
// threads' 16-byte row accesses conflict-free); rows n .. n rounded up to 32
// are zero.  grid = (leaves, column chunks of KC).
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

template <typename TV, int KC>
constexpr int leaf_multi_stride() { return KC + 16 / (int)sizeof(TV); }

// y_i -= sum_{j < 32} l_j x_{kb+j} for all KC columns of row i of a block of
// right-hand sides held in shared memory (row r at ys[r * RS], RS a multiple
// of 16 bytes): the l_j in registers, the rows kb.. read as 16-byte
// broadcasts (one address in every lane), the sums formed in j order.
template <typename TM, typename TV, int KC, int RS>
__device__ __forceinline__ void block_row_update(TV* ys, int i, int kb, const TM (&lv)[32]) {
  constexpr int VW = 16 / (int)sizeof(TV);
  using V16 = typename Vec16<TV>::type;
  TV acc[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) acc[c] = (TV)0;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const TV l = (TV)lv[j];
    const V16* xj = (const V16*)(ys + (kb + j) * RS);
#pragma unroll
    for (int q = 0; q < KC / VW; ++q) {
      TV x[VW];
      const V16 v = xj[q];
      memcpy(x, &v, 16);
#pragma unroll
      for (int u = 0; u < VW; ++u) acc[q * VW + u] += l * x[u];
    }
  }
  V16* yr = (V16*)(ys + i * RS);
#pragma unroll
  for (int q = 0; q < KC / VW; ++q) {
    TV y[VW];
    V16 v = yr[q];
    memcpy(y, &v, 16);
#pragma unroll
    for (int u = 0; u < VW; ++u) y[u] -= acc[q * VW + u];
    memcpy(&v, y, 16);
    yr[q] = v;
  }
}

template <typename TM, typename TV, int KC>
__global__ void __launch_bounds__(256) k_leaf_solve_multi(const int32_t* __restrict__ lo,
                                                          const int32_t* __restrict__ hi, int leaf0, int ldL,
                                                          const TM* __restrict__ Lall, TV* __restrict__ W, int k) {
  static_assert(KC % 8 == 0, "KC: a multiple of 8");
  constexpr int NB = 32, RS = leaf_multi_stride<TV, KC>();
  extern __shared__ __align__(16) unsigned char lsm[];
  TV* ys = (TV*)lsm;  // ((n + 31) / 32 * 32) x RS
  __shared__ TM db[NB][NB + 1];
  __shared__ TV dinv[NB];
  const int lf = blockIdx.x, node = leaf0 + lf;
  const int b = lo[node], n = hi[node] - b;
  const int c0 = blockIdx.y * KC;
  if (c0 >= k || n <= 0) return;
  const int kc = min(KC, k - c0), npad = (n + NB - 1) / NB * NB;
  const TM* L = Lall + (int64_t)lf * ldL * ldL;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < npad * RS; e += blockDim.x) {
    const int i = e / RS, c = e % RS;
    ys[e] = (i < n && c < kc) ? W[(int64_t)(b + i) * k + c0 + c] : (TV)0;
  }
  auto stage = [&](int kb, int nb) {
    __syncthreads();
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      const int i = e >> 5, j = e & 31;
      db[i][j] = (i < nb && j <= i) ? L[(int64_t)(kb + i) * ldL + kb + j] : (TM)0;
    }
    __syncthreads();
    if (tid < NB) dinv[lane] = lane < nb ? (TV)1 / (TV)db[lane][lane] : (TV)0;
    __syncthreads();
  };
  auto update = [&](int i, int kb, const TM (&lv)[NB]) { block_row_update<TM, TV, KC, RS>(ys, i, kb, lv); };
  const bool vec_rows = (ldL * (int)sizeof(TM)) % 16 == 0;
  // forward: L y = b
  for (int kb = 0; kb < n; kb += NB) {
    const int nb = min(NB, n - kb);
    stage(kb, nb);
    for (int c = warp; c < KC; c += 8) {
      TV yi = lane < nb ? ys[(kb + lane) * RS + c] : (TV)0;
      for (int j = 0; j < nb; ++j) {
        if (lane == j) yi *= dinv[j];
        const TV yj = __shfl_sync(0xffffffffu, yi, j);
        if (lane > j && lane < nb) yi -= (TV)db[lane][j] * yj;
      }
      if (lane < nb) ys[(kb + lane) * RS + c] = yi;
    }
    __syncthreads();
    // rows below the block (they exist only when nb = 32): the thread's 32
    // entries of row i as 16-byte loads where the rows are 16-byte aligned
    for (int i = kb + nb + tid; i < n; i += blockDim.x) {
      const TM* Li = L + (int64_t)i * ldL + kb;
      TM lv[NB];
      if (vec_rows) {
        using VM = typename Vec16<TM>::type;
        constexpr int VWM = 16 / (int)sizeof(TM);
#pragma unroll
        for (int q = 0; q < NB / VWM; ++q) {
          const VM v = ((const VM*)Li)[q];
          memcpy(lv + q * VWM, &v, 16);
        }
      } else {
#pragma unroll
        for (int j = 0; j < NB; ++j) lv[j] = j < nb ? Li[j] : (TM)0;
      }
      update(i, kb, lv);
    }
  }
  // backward: L^T x = y
  for (int kb = (n - 1) / NB * NB; kb >= 0; kb -= NB) {
    const int nb = min(NB, n - kb);
    stage(kb, nb);
    for (int c = warp; c < KC; c += 8) {
      TV xi = lane < nb ? ys[(kb + lane) * RS + c] : (TV)0;
      for (int j = nb - 1; j >= 0; --j) {
        if (lane == j) xi *= dinv[j];
        const TV xj = __shfl_sync(0xffffffffu, xi, j);
        if (lane < j) xi -= (TV)db[j][lane] * xj;
      }
      if (lane < nb) ys[(kb + lane) * RS + c] = xi;
    }
    __syncthreads();
    for (int i = tid; i < kb; i += blockDim.x) {
      TM lv[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) lv[j] = j < nb ? L[(int64_t)(kb + j) * ldL + i] : (TM)0;
      update(i, kb, lv);
    }
  }
  __syncthreads();
  for (int e = tid; e < n * RS; e += blockDim.x) {
    const int i = e / RS, c = e % RS;
    if (c < kc) W[(int64_t)(b + i) * k + c0 + c] = ys[e];
  }
}

// ---- segmented column sums -------------------------------------------------------
// For every node b of a level (grid.y) and a chunk of its rows (grid.x):
// u[dst(b)][q][r] += sum_i M[i][q] w[i][r], q < cnt(b).  Sibling mode: the
// columns are the sibling's skeleton (cnt = rank[sib], dst = sib); own mode:
// cnt = rank[b], dst = b.  u is FP64 [node][s_max][k].
// ROWS rows per CTA (128; 512 for several right-hand sides).  The sums are
// deterministic: each CTA writes its partial sums to parts[node][chunk][q][c]
// (chunk = blockIdx.x, s_max x k per chunk) and colsum_reduce adds them in a
// fixed order into u[dst], so the result does not depend on the order in
// which the CTAs run.
constexpr int kRowsPerChunk = 128;

// The partial sums of a column-sum launch (parts[node][chunk][q][c], chunk =
// blockIdx.x of that launch, nchunk_stride chunks a node) added in a fixed
// order by two more launches: groups of kColsumGroup consecutive chunks first
// (parts2[node][group][q][c]), then the groups into u[dst].  Both spread the
// node's cnt x k sums over many threads and CTAs.
constexpr int kColsumGroup = 32;

__global__ void __launch_bounds__(256) k_colsum_reduce1(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                        const int32_t* __restrict__ rank, int node0, int sibling,
                                                        int rows_per_chunk, int nchunk_stride, int s_max, int k,
                                                        const double* __restrict__ parts, double* __restrict__ parts2,
                                                        int ngroup_stride) {
  const int nl = blockIdx.y, node = node0 + nl, g = blockIdx.z;
  const int cnt = sibling ? rank[node ^ 1] : rank[node];
  const int nch = (hi[node] - lo[node] + rows_per_chunk - 1) / rows_per_chunk;
  const int c0 = g * kColsumGroup, c1 = min(nch, c0 + kColsumGroup);
  if (c0 >= c1) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt * k; e += gridDim.x * blockDim.x) {
    const int q = e / k, c = e % k;
    double sum = 0.0;
    for (int ch = c0; ch < c1; ++ch) sum += parts[(((int64_t)nl * nchunk_stride + ch) * s_max + q) * k + c];
    parts2[(((int64_t)nl * ngroup_stride + g) * s_max + q) * k + c] = sum;
  }
}

__global__ void __launch_bounds__(256) k_colsum_reduce2(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                        const int32_t* __restrict__ rank, int node0, int sibling,
                                                        int rows_per_chunk, int s_max, int k,
                                                        const double* __restrict__ parts2, int ngroup_stride,
                                                        double* __restrict__ U) {
  const int nl = blockIdx.y, node = node0 + nl;
  const int cnt = sibling ? rank[node ^ 1] : rank[node], dst = sibling ? node ^ 1 : node;
  const int nch = (hi[node] - lo[node] + rows_per_chunk - 1) / rows_per_chunk;
  const int ng = (nch + kColsumGroup - 1) / kColsumGroup;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt * k; e += gridDim.x * blockDim.x) {
    const int q = e / k, c = e % k;
    double sum = 0.0;
    for (int g = 0; g < ng; ++g) sum += parts2[(((int64_t)nl * ngroup_stride + g) * s_max + q) * k + c];
    U[((int64_t)dst * s_max + q) * k + c] += sum;
  }
}

// the two reductions after a column-sum launch of grid g (g.x chunks of
// rows_per_chunk rows, g.y nodes)
inline void colsum_reduce(dim3 g, cudaStream_t s, const int32_t* lo, const int32_t* hi, const int32_t* rank,
                          int node0, int sibling, int rows_per_chunk, int s_max, int k, const double* parts,
                          double* parts2, double* U, int phase) {
  const int ng = ((int)g.x + kColsumGroup - 1) / kColsumGroup;
  const unsigned ex = (unsigned)std::min<int64_t>(64, ((int64_t)s_max * k + 255) / 256);
  KF_PHASE(phase, s, k_colsum_reduce1<<<dim3(ex, g.y, ng), 256, 0, s>>>(lo, hi, rank, node0, sibling, rows_per_chunk,
                                                                         (int)g.x, s_max, k, parts, parts2, ng));
  KF_PHASE(phase, s, k_colsum_reduce2<<<dim3(ex, g.y), 256, 0, s>>>(lo, hi, rank, node0, sibling, rows_per_chunk,
                                                                     s_max, k, parts2, ng, U));
}

// A bound on the partial sums of any column-sum launch of one sweep or
// operator product over N points (chunks of at least `rows` rows; at most
// 2^D nodes a level, each with one partly filled chunk).
inline size_t colsum_parts_bound(int64_t N, int D, int s_max, int64_t k, int rows) {
  return (size_t)(N / rows + ((int64_t)2 << D) + 4) * s_max * k;
}

template <typename TM, typename TV, int kMaxK, int ROWS = kRowsPerChunk>
__global__ void __launch_bounds__(256) k_colsum(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                const int32_t* __restrict__ rank, const int32_t* __restrict__ skel,
                                                int node0, int s_max, int sibling_mode, int src,
                                                const TM* __restrict__ M, const double* __restrict__ X64,
                                                const float* __restrict__ X32, int d, double c_exp, double inv_h3,
                                                const TV* __restrict__ W, int k, double* __restrict__ parts) {
  __shared__ TV ws[ROWS][kMaxK];
  const int nl = blockIdx.y, node = node0 + nl, sib = node ^ 1;
  const int b = lo[node], n = hi[node] - b;
  const int cnt = sibling_mode ? rank[sib] : rank[node];
  const int r0 = blockIdx.x * ROWS;
  if (r0 >= n || cnt == 0) return;
  const int r1 = min(n, r0 + ROWS);
  const int32_t* sk = skel + (int64_t)sib * s_max;
  for (int kb = 0; kb < k; kb += kMaxK) {
    const int kk = min(kMaxK, k - kb);
    __syncthreads();
    for (int e = threadIdx.x; e < (r1 - r0) * kMaxK; e += blockDim.x) {
      int i = e / kMaxK, r = e % kMaxK;
      ws[i][r] = r < kk ? W[(int64_t)(b + r0 + i) * k + kb + r] : (TV)0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      TV acc[kMaxK];
#pragma unroll
      for (int r = 0; r < kMaxK; ++r) acc[r] = (TV)0;
      if (src == SRC_STORED) {
        // 8 rows' loads in flight before their products (the same order of sums)
        const TM* Mq = M + (int64_t)(b + r0) * s_max + q;
        const int nr = r1 - r0;
        int i = 0;
        for (; i + 8 <= nr; i += 8) {
          TM mv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) mv[u] = Mq[(int64_t)(i + u) * s_max];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const TV m = (TV)mv[u];
#pragma unroll
            for (int r = 0; r < kMaxK; ++r) acc[r] += m * ws[i + u][r];
          }
        }
        for (; i < nr; ++i) {
          const TV m = (TV)Mq[(int64_t)i * s_max];
#pragma unroll
          for (int r = 0; r < kMaxK; ++r) acc[r] += m * ws[i][r];
        }
      } else {
        for (int i = r0; i < r1; ++i) {
          const TV m = (TV)eval_src<TM>(src, X64, X32, b + i, sk[q], d, c_exp, inv_h3);
#pragma unroll
          for (int r = 0; r < kMaxK; ++r) acc[r] += m * ws[i - r0][r];
        }
      }
      double* out = parts + (((int64_t)nl * gridDim.x + blockIdx.x) * s_max + q) * k + kb;
#pragma unroll
      for (int r = 0; r < kMaxK; ++r)  // static indices keep acc in registers
        if (r < kk) out[r] = (double)acc[r];
    }
  }
}

template <typename TM, typename TV>
void launch_colsum(dim3 g, cudaStream_t s, const int32_t* lo, const int32_t* hi, const int32_t* rank,
                   const int32_t* skel, int node0, int s_max, int sib, int src, const TM* M, const double* X64,
                   const float* X32, int d, double c_exp, double inv_h3, const TV* W, int k, double* U,
                   double* parts, double* parts2, int phase = KF_PH_S_COLSUM) {
  if (k == 1) {
    KF_PHASE(phase, s, k_colsum<TM, TV, 1><<<g, 256, 0, s>>>(lo, hi, rank, skel, node0, s_max, sib, src, M, X64, X32, d, c_exp, inv_h3,
                                          W, k, parts));
    colsum_reduce(g, s, lo, hi, rank, node0, sib, kRowsPerChunk, s_max, k, parts, parts2, U, phase);
  } else {
    // g.x counts 128-row chunks; several right-hand sides take 512 rows a CTA
    // (64 columns a pass over 128-row chunks measured slower: 24.1 against
    // 17.9 ms per sweep of 64 columns at N = 2^20, the partial sums of four
    // times as many chunks written and reduced)
    const dim3 g4((g.x + 3) / 4, g.y);
    bool done = false;
    if constexpr (sizeof(TV) == 4) {
      if (k > 8) {  // 16 columns a pass: each loaded entry of M serves 16 products
        KF_PHASE(phase, s, k_colsum<TM, TV, 16, 512><<<g4, 256, 0, s>>>(lo, hi, rank, skel, node0, s_max, sib, src, M,
                                                                        X64, X32, d, c_exp, inv_h3, W, k, parts));
        done = true;
      }
    }
    if (!done)
      KF_PHASE(phase, s, k_colsum<TM, TV, 8, 512><<<g4, 256, 0, s>>>(lo, hi, rank, skel, node0, s_max, sib, src, M, X64,
                                                                     X32, d, c_exp, inv_h3, W, k, parts));
    colsum_reduce(g4, s, lo, hi, rank, node0, sib, 512, s_max, k, parts, parts2, U, phase);
  }
}

// ---- row updates: w[i][r] += sign * sum_q M[i][q] v[src(b)][q][r] ------------------
// A CTA takes a chunk of rows of one node; the node's vector v (cnt x k) is
// staged in shared memory in the vector precision; one warp per row, lanes
// over q, products in the vector precision (FP32 on the mixed path).
constexpr int kRowUpdRows = 256;

template <typename TM, typename TV, int KB>
__global__ void __launch_bounds__(256) k_rowupd(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                const int32_t* __restrict__ rank, const int32_t* __restrict__ skel,
                                                int node0, int nnodes_level, int s_max, int sibling_mode, int src,
                                                const TM* __restrict__ M, const double* __restrict__ X64,
                                                const float* __restrict__ X32, int d, double c_exp, double inv_h3,
                                                const double* __restrict__ V, double sign, TV* __restrict__ W, int k) {
  __shared__ TV vs[KF_MAX_SMAX * KB];
  const int nl = blockIdx.y, node = node0 + nl, sib = node ^ 1;
  const int b = lo[node], n = hi[node] - b;
  const int cnt = sibling_mode ? rank[sib] : rank[node];
  const int from = sibling_mode ? sib : node;
  const int r0 = blockIdx.x * kRowUpdRows;
  if (cnt == 0 || r0 >= n) return;
  const int r1 = min(n, r0 + kRowUpdRows);
  const int32_t* sk = skel + (int64_t)sib * s_max;
  const double* v = V + (int64_t)from * s_max * k;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int kb = 0; kb < k; kb += KB) {
    const int kk = min(KB, k - kb);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * KB; e += blockDim.x) {
      const int q = e / KB, r = e % KB;
      vs[e] = r < kk ? (TV)v[(int64_t)q * k + kb + r] : (TV)0;
    }
    __syncthreads();
    for (int i = r0 + warp; i < r1; i += 8) {
      TV acc[KB];
#pragma unroll
      for (int r = 0; r < KB; ++r) acc[r] = (TV)0;
      if (src == SRC_STORED) {
        // a row's 8 loads per lane in flight before their products (the same order of sums)
        const TM* Mi = M + (int64_t)(b + i) * s_max;
        int q = lane;
        for (; q + 32 * 7 < cnt; q += 32 * 8) {
          TM mv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) mv[u] = Mi[q + 32 * u];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const TV m = (TV)mv[u];
#pragma unroll
            for (int r = 0; r < KB; ++r) acc[r] += m * vs[(q + 32 * u) * KB + r];
          }
        }
        for (; q < cnt; q += 32) {
          const TV m = (TV)Mi[q];
#pragma unroll
          for (int r = 0; r < KB; ++r) acc[r] += m * vs[q * KB + r];
        }
      } else {
        for (int q = lane; q < cnt; q += 32) {
          const TV m = (TV)eval_src<TM>(src, X64, X32, b + i, sk[q], d, c_exp, inv_h3);
#pragma unroll
          for (int r = 0; r < KB; ++r) acc[r] += m * vs[q * KB + r];
        }
      }
#pragma unroll
      for (int r = 0; r < KB; ++r)
        for (int off = 16; off > 0; off >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off);
      if (lane < kk) {
        TV a = acc[0];
#pragma unroll
        for (int r = 1; r < KB; ++r)
          if (lane == r) a = acc[r];
        W[(int64_t)(b + i) * k + kb + lane] += (TV)sign * a;
      }
    }
  }
}

// One right-hand side, stored M: a warp takes 32 rows and walks the columns
// in 32-wide tiles, each tile loaded row by row (coalesced) into the warp's
// shared-memory tile and read back transposed, so that lane q accumulates row
// q's dot product with no cross-lane reduction.  Every FMA is then a useful
// one: on the FP64 path this pass is bound by the FP64 pipe (one FMA per 8
// bytes of M), and the shuffle reductions of k_rowupd cost it another 60%.
template <typename TM, typename TV>
__global__ void __launch_bounds__(256) k_rowupd_tile(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                     const int32_t* __restrict__ rank, int node0, int s_max,
                                                     int sibling_mode, const TM* __restrict__ M,
                                                     const double* __restrict__ V, double sign, TV* __restrict__ W) {
  __shared__ TV vs[KF_MAX_SMAX + 32];
  extern __shared__ __align__(16) unsigned char rt_smem[];
  TM(*tile)[32][33] = (TM(*)[32][33])rt_smem;  // 8 warps x 32 x 33, dynamic
  const int nl = blockIdx.y, node = node0 + nl, sib = node ^ 1;
  const int b = lo[node], n = hi[node] - b;
  const int cnt = sibling_mode ? rank[sib] : rank[node];
  const int from = sibling_mode ? sib : node;
  const int r0 = blockIdx.x * kRowUpdRows;
  if (cnt == 0 || r0 >= n) return;
  const int r1 = min(n, r0 + kRowUpdRows);
  const double* v = V + (int64_t)from * s_max;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cpad = (cnt + 31) & ~31;
  for (int q = threadIdx.x; q < cpad; q += blockDim.x) vs[q] = q < cnt ? (TV)v[q] : (TV)0;
  __syncthreads();
  TM(*t)[33] = tile[warp];
  for (int i0 = r0 + warp * 32; i0 < r1; i0 += 8 * 32) {
    TV acc = (TV)0;
    for (int q0 = 0; q0 < cnt; q0 += 32) {
      TM x[32];
#pragma unroll
      for (int rr = 0; rr < 32; ++rr)
        x[rr] = (i0 + rr < r1 && q0 + lane < cnt) ? M[(int64_t)(b + i0 + rr) * s_max + q0 + lane] : (TM)0;
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) t[rr][lane] = x[rr];
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 32; ++j) acc += (TV)t[lane][j] * vs[q0 + j];
      __syncwarp();
    }
    if (i0 + lane < r1) W[b + i0 + lane] += (TV)sign * acc;
  }
}

// Several right-hand sides, stored M: a warp takes 32 rows and walks the
// node's columns in 32-wide tiles, each loaded row by row (coalesced) into the
// warp's shared-memory tile; lane q then forms row q's products with all KB
// staged columns of v (16-byte broadcast reads), so that every FMA is a useful
// one and no cross-lane reduction is needed.  v is staged in the vector
// precision, cnt rounded up to 32 rows of KB values, zero past cnt and k.
template <typename TM, typename TV, int KB>
__global__ void __launch_bounds__(256) k_rowupd_multi(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                      const int32_t* __restrict__ rank, int node0, int s_max,
                                                      int sibling_mode, const TM* __restrict__ M,
                                                      const double* __restrict__ V, double sign,
                                                      TV* __restrict__ W, int k) {
  constexpr int VW = 16 / (int)sizeof(TV);
  static_assert(KB % VW == 0, "KB: a multiple of the 16-byte vector");
  using V16 = typename Vec16<TV>::type;
  extern __shared__ __align__(16) unsigned char rm_smem[];
  const int vrows = (s_max + 31) & ~31;
  TV* vs = (TV*)rm_smem;  // vrows x KB
  TM(*tile)[32][33] = (TM(*)[32][33])(rm_smem + sizeof(TV) * vrows * KB);  // 8 warps x 32 x 33
  const int nl = blockIdx.y, node = node0 + nl, sib = node ^ 1;
  const int b = lo[node], n = hi[node] - b;
  const int cnt = sibling_mode ? rank[sib] : rank[node];
  const int from = sibling_mode ? sib : node;
  const int r0 = blockIdx.x * kRowUpdRows;
  if (cnt == 0 || r0 >= n) return;
  const int r1 = min(n, r0 + kRowUpdRows);
  const double* v = V + (int64_t)from * s_max * k;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cpad = (cnt + 31) & ~31;
  TM(*t)[33] = tile[warp];
  for (int kb = 0; kb < k; kb += KB) {
    const int kk = min(KB, k - kb);
    __syncthreads();
    for (int e = threadIdx.x; e < cpad * KB; e += blockDim.x) {
      const int q = e / KB, r = e % KB;
      vs[e] = (q < cnt && r < kk) ? (TV)v[(int64_t)q * k + kb + r] : (TV)0;
    }
    __syncthreads();
    for (int i0 = r0 + warp * 32; i0 < r1; i0 += 8 * 32) {
      TV acc[KB];
#pragma unroll
      for (int r = 0; r < KB; ++r) acc[r] = (TV)0;
      for (int q0 = 0; q0 < cnt; q0 += 32) {
        TM x[32];
#pragma unroll
        for (int rr = 0; rr < 32; ++rr)
          x[rr] = (i0 + rr < r1 && q0 + lane < cnt) ? M[(int64_t)(b + i0 + rr) * s_max + q0 + lane] : (TM)0;
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) t[rr][lane] = x[rr];
        __syncwarp();
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
          const TV m = (TV)t[lane][j];
          const V16* vj = (const V16*)(vs + (q0 + j) * KB);
#pragma unroll
          for (int qq = 0; qq < KB / VW; ++qq) {
            TV y[VW];
            const V16 w = vj[qq];
            memcpy(y, &w, 16);
#pragma unroll
            for (int u = 0; u < VW; ++u) acc[qq * VW + u] += m * y[u];
          }
        }
        __syncwarp();
      }
      if (i0 + lane < r1) {
        TV* wr = W + (int64_t)(b + i0 + lane) * k + kb;
#pragma unroll
        for (int r = 0; r < KB; ++r)
          if (r < kk) wr[r] += (TV)sign * acc[r];
      }
    }
  }
}

template <typename TM, typename TV, int KB>
size_t rowupd_multi_smem(int s_max) {
  return sizeof(TV) * (size_t)((s_max + 31) & ~31) * KB + sizeof(TM) * 8 * 32 * 33;
}

template <typename TM, typename TV>
void launch_rowupd(int64_t rows, int nnodes, cudaStream_t s, const int32_t* lo, const int32_t* hi, const int32_t* rank,
                   const int32_t* skel, int node0, int s_max, int sib, int src, const TM* M, const double* X64,
                   const float* X32, int d, double c_exp, double inv_h3, const double* V, double sign, TV* W, int k,
                   int phase = KF_PH_S_ROWUPD) {
  dim3 g((unsigned)((rows + kRowUpdRows - 1) / kRowUpdRows), nnodes);
  // FP64 M: the tiled form (FP64-pipe bound); FP32 M: the warp-per-row form,
  // which streams at about 75% of HBM bandwidth
  if constexpr (sizeof(TM) == 8) {
    if (k == 1 && src == SRC_STORED) {
      const int smem = (int)(sizeof(TM) * 8 * 32 * 33);
      static bool attr_set = false;  // per instantiation; setting it twice is harmless
      if (!attr_set) {
        cudaFuncSetAttribute(k_rowupd_tile<TM, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr_set = true;
      }
      KF_PHASE(phase, s, k_rowupd_tile<TM, TV><<<g, 256, smem, s>>>(lo, hi, rank, node0, s_max, sib, M, V, sign, W));
      return;
    }
  }
  if (k >= 2 && src == SRC_STORED) {
    // several right-hand sides: the tiled form, 16 FP32 (8 FP64) columns a
    // pass, or 64 FP32 columns for k > 32 (M read once per 64 columns)
    constexpr int KB = sizeof(TV) == 4 ? 16 : 8;
    constexpr int KW = sizeof(TV) == 4 ? 64 : 8;
    const int mode = (sizeof(TV) == 4 && k > 32) ? 2 : (k > 8 ? 1 : 0);
    const size_t smem = mode == 2 ? rowupd_multi_smem<TM, TV, KW>(s_max)
                                  : (mode == 1 ? rowupd_multi_smem<TM, TV, KB>(s_max) : rowupd_multi_smem<TM, TV, 8>(s_max));
    if (mode == 2) {
      cudaFuncSetAttribute(k_rowupd_multi<TM, TV, KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      KF_PHASE(phase, s, k_rowupd_multi<TM, TV, KW><<<g, 256, smem, s>>>(lo, hi, rank, node0, s_max, sib, M, V, sign,
                                                                        W, k));
    } else if (mode == 1) {
      cudaFuncSetAttribute(k_rowupd_multi<TM, TV, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      KF_PHASE(phase, s, k_rowupd_multi<TM, TV, KB><<<g, 256, smem, s>>>(lo, hi, rank, node0, s_max, sib, M, V, sign,
                                                                        W, k));
    } else {
      cudaFuncSetAttribute(k_rowupd_multi<TM, TV, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      KF_PHASE(phase, s, k_rowupd_multi<TM, TV, 8><<<g, 256, smem, s>>>(lo, hi, rank, node0, s_max, sib, M, V, sign,
                                                                       W, k));
    }
    return;
  }
  if (k == 1)
    KF_PHASE(phase, s, k_rowupd<TM, TV, 1><<<g, 256, 0, s>>>(lo, hi, rank, skel, node0, nnodes, s_max, sib, src, M,
                                                                     X64, X32, d, c_exp, inv_h3, V, sign, W, k));
  else
    KF_PHASE(phase, s, k_rowupd<TM, TV, 8><<<g, 256, 0, s>>>(lo, hi, rank, skel, node0, nnodes, s_max, sib, src, M,
                                                                     X64, X32, d, c_exp, inv_h3, V, sign, W, k));
}

// ---- reduced systems: out[l], out[r] <- Z^-1 [in[l]; in[r]] (or Z^-T) ---------------
// P Z = L U with implicit pivoting: logical row i of L and U is stored in row
// pm[i] of ZLU, and (P b)[i] = b[pm[i]].  Blocked by 32 rows: the 32 x 32
// diagonal block is staged in shared memory, warp 0 solves it with shuffles,
// then all threads update the remaining rows with it.
// acc - sum_{j < nb} A[rows[j]][i] x[j]: fully unrolled with predicated loads, so
// that the 32 loads are in flight together
// column i of rows rows[0..nb) of A (row stride lda)
__device__ __forceinline__ double col_update(const double* __restrict__ A, int lda, const int* rows, int i, int nb,
                                             const double* x, double acc) {
  double v[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = j < nb ? A[(int64_t)rows[j] * lda + i] : 0.0;
#pragma unroll
  for (int j = 0; j < 32; ++j) acc = fma(-v[j], x[j], acc);
  return acc;
}

__global__ void __launch_bounds__(256) k_zsolve(const int32_t* __restrict__ rank, int node0, int ldz, int s_max,
                                                const double* __restrict__ ZLU, const int32_t* __restrict__ piv,
                                                const double* __restrict__ in, double* __restrict__ out, int k,
                                                int transpose) {
  extern __shared__ double zsm[];
  double* t = zsm;                   // ldz
  double* u = t + ldz;               // ldz
  int* pm = (int*)(u + ldz);         // ldz
  double (*wtile)[33] = (double (*)[33])(zsm + 2 * ldz + (ldz + 1) / 2);  // 8 warps x 32 x 33: row tiles
  __shared__ double db[32][33];
  __shared__ double dinv[32];  // reciprocals of the diagonal of the staged block
  __shared__ double xb[32];
  const int nl = blockIdx.x, node = node0 + nl;
  const int l = 2 * node, r = l + 1, sl = rank[l], sr = rank[r], z = sl + sr;
  const double* A = ZLU + (int64_t)node * ldz * ldz;
  const int32_t* pv = piv + (int64_t)node * ldz;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < z; i += blockDim.x) pm[i] = pv[i];
  __syncthreads();
  // The 32 x 32 diagonal block of logical rows kb..kb+nb: fetched into
  // registers one block ahead (its loads fly while the previous block's rows
  // are updated), then committed to shared memory.  Warp 0 forms the
  // reciprocals of its diagonal, one division per lane in parallel (an FP64
  // division inside the dependent chain would cost about 1000 cycles).
  double pre[4];
  auto fetch = [&](int kb, int nb) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = q * 256 + tid, i = e >> 5, j = e & 31;
      pre[q] = (i < nb && j < nb) ? A[(int64_t)pm[kb + i] * ldz + kb + j] : 0.0;
    }
  };
  auto commit = [&](int nb, bool recip) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = q * 256 + tid;
      db[e >> 5][e & 31] = pre[q];
    }
    __syncthreads();
    if (recip && tid < 32) {
      dinv[lane] = lane < nb ? 1.0 / db[lane][lane] : 0.0;
      __syncwarp();
    }
  };
  const int top = z > 0 ? ((z - 1) / 32) * 32 : 0;
  // right-hand sides c = blockIdx.y, blockIdx.y + gridDim.y, ...: several CTAs
  // of one node solve different columns at once
  for (int c = blockIdx.y; c < k; c += gridDim.y) {
    for (int i = tid; i < z; i += blockDim.x)
      u[i] = i < sl ? in[((int64_t)l * s_max + i) * k + c] : in[((int64_t)r * s_max + (i - sl)) * k + c];
    __syncthreads();
    if (!transpose) {
      for (int i = tid; i < z; i += blockDim.x) t[i] = u[pm[i]];
      __syncthreads();
      // L (unit lower)
      if (z > 0) fetch(0, min(32, z));
      for (int kb = 0; kb < z; kb += 32) {
        const int nb = min(32, z - kb);
        commit(nb, false);
        if (tid < 32) {
          double yi = lane < nb ? t[kb + lane] : 0.0;
          for (int j = 0; j < nb; ++j) {
            double yj = __shfl_sync(0xffffffffu, yi, j);
            if (lane > j && lane < nb) yi = fma(-db[lane][j], yj, yi);
          }
          if (lane < nb) { xb[lane] = yi; t[kb + lane] = yi; } else { xb[lane] = 0.0; }
        }
        __syncthreads();
        if (kb + 32 < z) fetch(kb + 32, min(32, z - kb - 32));
        warp_tile_rowupd<double, double>(kb + nb, z, kb, nb, [&](int i) { return A + (int64_t)pm[i] * ldz; }, xb,
                                         [&](int i, double acc) { t[i] -= acc; }, wtile + (tid >> 5) * 32);
        __syncthreads();
      }
      // U
      if (z > 0) fetch(top, z - top);
      for (int kb = top; kb >= 0 && z > 0; kb -= 32) {
        const int nb = min(32, z - kb);
        commit(nb, true);
        if (tid < 32) {
          double xi = lane < nb ? t[kb + lane] : 0.0;
          for (int j = nb - 1; j >= 0; --j) {
            if (lane == j) xi *= dinv[j];
            double xj = __shfl_sync(0xffffffffu, xi, j);
            if (lane < j) xi = fma(-db[lane][j], xj, xi);
          }
          if (lane < nb) { xb[lane] = xi; t[kb + lane] = xi; } else { xb[lane] = 0.0; }
        }
        __syncthreads();
        if (kb >= 32) fetch(kb - 32, 32);
        warp_tile_rowupd<double, double>(0, kb, kb, nb, [&](int i) { return A + (int64_t)pm[i] * ldz; }, xb,
                                         [&](int i, double acc) { t[i] -= acc; }, wtile + (tid >> 5) * 32);
        __syncthreads();
      }
    } else {
      for (int i = tid; i < z; i += blockDim.x) t[i] = u[i];
      __syncthreads();
      // U^T y = b (forward)
      if (z > 0) fetch(0, min(32, z));
      for (int kb = 0; kb < z; kb += 32) {
        const int nb = min(32, z - kb);
        commit(nb, true);
        if (tid < 32) {
          double yi = lane < nb ? t[kb + lane] : 0.0;
          for (int j = 0; j < nb; ++j) {
            if (lane == j) yi *= dinv[j];
            double yj = __shfl_sync(0xffffffffu, yi, j);
            if (lane > j && lane < nb) yi = fma(-db[j][lane], yj, yi);
          }
          if (lane < nb) { xb[lane] = yi; t[kb + lane] = yi; } else { xb[lane] = 0.0; }
        }
        __syncthreads();
        if (kb + 32 < z) fetch(kb + 32, min(32, z - kb - 32));
        for (int i = kb + nb + tid; i < z; i += blockDim.x) t[i] = col_update(A, ldz, pm + kb, i, nb, xb, t[i]);
        __syncthreads();
      }
      // L^T x = y (backward, unit diagonal)
      if (z > 0) fetch(top, z - top);
      for (int kb = top; kb >= 0 && z > 0; kb -= 32) {
        const int nb = min(32, z - kb);
        commit(nb, false);
        if (tid < 32) {
          double xi = lane < nb ? t[kb + lane] : 0.0;
          for (int j = nb - 1; j >= 0; --j) {
            double xj = __shfl_sync(0xffffffffu, xi, j);
            if (lane < j) xi = fma(-db[j][lane], xj, xi);
          }
          if (lane < nb) { xb[lane] = xi; t[kb + lane] = xi; } else { xb[lane] = 0.0; }
        }
        __syncthreads();
        if (kb >= 32) fetch(kb - 32, 32);
        for (int i = tid; i < kb; i += blockDim.x) t[i] = col_update(A, ldz, pm + kb, i, nb, xb, t[i]);
        __syncthreads();
      }
      // x = P w: x[pm[i]] = w[i]
      for (int i = tid; i < z; i += blockDim.x) u[pm[i]] = t[i];
      __syncthreads();
      for (int i = tid; i < z; i += blockDim.x) t[i] = u[i];
      __syncthreads();
    }
    for (int i = tid; i < z; i += blockDim.x) {
      if (i < sl) out[((int64_t)l * s_max + i) * k + c] = t[i];
      else out[((int64_t)r * s_max + (i - sl)) * k + c] = t[i];
    }
    __syncthreads();
  }
}

// The reduced systems for several right-hand sides (k >= 2): KC columns of
// [in_l; in_r] per CTA held in shared memory (row i at ts[i * RS]) through
// all four triangular sweeps, so that the LU is read once per KC columns
// instead of once per column.  Per 32-row block the diagonal block is staged
// in shared memory and each warp solves KC / 8 columns with shuffles; then
// every thread updates one row of the rest for all KC columns: from row pm[i]
// of the LU (L and U sweeps, entries kb..kb+31) or from column i of rows
// pm[kb..kb+31] (the transposed sweeps, coalesced across the threads).
// grid = (nodes of the level, column chunks of KC).
template <int KC>
__global__ void __launch_bounds__(256) k_zsolve_multi(const int32_t* __restrict__ rank, int node0, int ldz,
                                                      int s_max, const double* __restrict__ ZLU,
                                                      const int32_t* __restrict__ piv, const double* __restrict__ in,
                                                      double* __restrict__ out, int k, int transpose) {
  constexpr int RS = leaf_multi_stride<double, KC>();
  extern __shared__ __align__(16) unsigned char zm_smem[];
  const int nl = blockIdx.x, node = node0 + nl;
  const int l = 2 * node, r = l + 1, sl = rank[l], sr = rank[r], z = sl + sr;
  const int c0 = blockIdx.y * KC;
  if (c0 >= k || z == 0) return;
  const int kc = min(KC, k - c0), zpad = (z + 31) / 32 * 32;
  double* ts = (double*)zm_smem;       // zpad x RS
  int* pm = (int*)(ts + (size_t)zpad * RS);  // z
  __shared__ double db[32][33];
  __shared__ double dinv[32];
  const double* A = ZLU + (int64_t)node * ldz * ldz;
  const int32_t* pv = piv + (int64_t)node * ldz;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto dst = [&](int i) -> int64_t { return i < sl ? (int64_t)l * s_max + i : (int64_t)r * s_max + (i - sl); };
  for (int i = tid; i < z; i += blockDim.x) pm[i] = pv[i];
  __syncthreads();
  // the right-hand sides, permuted by P for the L U sweeps
  for (int e = tid; e < zpad * RS; e += blockDim.x) {
    const int i = e / RS, c = e % RS;
    ts[e] = (i < z && c < kc) ? in[dst(transpose ? i : pm[i]) * k + c0 + c] : 0.0;
  }
  auto stage = [&](int kb, int nb, bool recip) {
    __syncthreads();
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
      const int i = e >> 5, j = e & 31;
      db[i][j] = (i < nb && j < nb) ? A[(int64_t)pm[kb + i] * ldz + kb + j] : 0.0;
    }
    __syncthreads();
    if (recip && tid < 32) dinv[lane] = lane < nb ? 1.0 / db[lane][lane] : 0.0;
    __syncthreads();
  };
  auto update = [&](int i, int kb, const double (&lv)[32]) { block_row_update<double, double, KC, RS>(ts, i, kb, lv); };
  const int top = (z - 1) / 32 * 32;
  if (!transpose) {
    // L (unit lower): forward
    for (int kb = 0; kb < z; kb += 32) {
      const int nb = min(32, z - kb);
      stage(kb, nb, false);
      for (int c = warp; c < KC; c += 8) {
        double yi = lane < nb ? ts[(kb + lane) * RS + c] : 0.0;
        for (int j = 0; j < nb; ++j) {
          const double yj = __shfl_sync(0xffffffffu, yi, j);
          if (lane > j && lane < nb) yi = fma(-db[lane][j], yj, yi);
        }
        if (lane < nb) ts[(kb + lane) * RS + c] = yi;
      }
      __syncthreads();
      for (int i = kb + nb + tid; i < z; i += blockDim.x) {
        const double* Ai = A + (int64_t)pm[i] * ldz + kb;
        double lv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) lv[j] = j < nb ? Ai[j] : 0.0;
        update(i, kb, lv);
      }
    }
    // U: backward
    for (int kb = top; kb >= 0; kb -= 32) {
      const int nb = min(32, z - kb);
      stage(kb, nb, true);
      for (int c = warp; c < KC; c += 8) {
        double xi = lane < nb ? ts[(kb + lane) * RS + c] : 0.0;
        for (int j = nb - 1; j >= 0; --j) {
          if (lane == j) xi *= dinv[j];
          const double xj = __shfl_sync(0xffffffffu, xi, j);
          if (lane < j) xi = fma(-db[lane][j], xj, xi);
        }
        if (lane < nb) ts[(kb + lane) * RS + c] = xi;
      }
      __syncthreads();
      for (int i = tid; i < kb; i += blockDim.x) {
        const double* Ai = A + (int64_t)pm[i] * ldz + kb;
        double lv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) lv[j] = j < nb ? Ai[j] : 0.0;
        update(i, kb, lv);
      }
    }
  } else {
    // U^T: forward
    for (int kb = 0; kb < z; kb += 32) {
      const int nb = min(32, z - kb);
      stage(kb, nb, true);
      for (int c = warp; c < KC; c += 8) {
        double yi = lane < nb ? ts[(kb + lane) * RS + c] : 0.0;
        for (int j = 0; j < nb; ++j) {
          if (lane == j) yi *= dinv[j];
          const double yj = __shfl_sync(0xffffffffu, yi, j);
          if (lane > j && lane < nb) yi = fma(-db[j][lane], yj, yi);
        }
        if (lane < nb) ts[(kb + lane) * RS + c] = yi;
      }
      __syncthreads();
      for (int i = kb + nb + tid; i < z; i += blockDim.x) {
        double lv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) lv[j] = j < nb ? A[(int64_t)pm[kb + j] * ldz + i] : 0.0;
        update(i, kb, lv);
      }
    }
    // L^T (unit): backward
    for (int kb = top; kb >= 0; kb -= 32) {
      const int nb = min(32, z - kb);
      stage(kb, nb, false);
      for (int c = warp; c < KC; c += 8) {
        double xi = lane < nb ? ts[(kb + lane) * RS + c] : 0.0;
        for (int j = nb - 1; j >= 0; --j) {
          const double xj = __shfl_sync(0xffffffffu, xi, j);
          if (lane < j) xi = fma(-db[j][lane], xj, xi);
        }
        if (lane < nb) ts[(kb + lane) * RS + c] = xi;
      }
      __syncthreads();
      for (int i = tid; i < kb; i += blockDim.x) {
        double lv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) lv[j] = j < nb ? A[(int64_t)pm[kb + j] * ldz + i] : 0.0;
        update(i, kb, lv);
      }
    }
  }
  __syncthreads();
  // x = P^T w for the transposed solve: x[pm[i]] = w[i]
  for (int e = tid; e < z * RS; e += blockDim.x) {
    const int i = e / RS, c = e % RS;
    if (c < kc) out[dst(transpose ? pm[i] : i) * k + c0 + c] = ts[e];
  }
}

inline size_t zsolve_multi_smem(int ldz) {
  const int zpad = (ldz + 31) / 32 * 32;
  return sizeof(double) * (size_t)zpad * leaf_multi_stride<double, 8>() + sizeof(int) * (size_t)ldz;
}

// y_i -= sum_{j < 32} l_j x_{kb+j} for all KC columns of row i, everything as
// double-float pairs (rows of ts are RS pairs long, a 16-byte multiple; the
// rows kb.. read as 16-byte broadcasts), on the FP32 pipes.
template <int KC, int RS>
__device__ __forceinline__ void block_row_update_df(float2* ts, int i, int kb, const float2 (&lv)[32]) {
  static_assert(KC % 2 == 0 && (RS * 8) % 16 == 0, "pairs in 16-byte groups");
  float sh[KC], sl[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) sh[c] = sl[c] = 0.f;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float2 l = lv[j];
    const float4* xj = (const float4*)(ts + (kb + j) * RS);
#pragma unroll
    for (int q = 0; q < KC / 2; ++q) {
      const float4 v = xj[q];
      kf_df_fma(l.x, l.y, v.x, v.y, sh[2 * q], sl[2 * q]);
      kf_df_fma(l.x, l.y, v.z, v.w, sh[2 * q + 1], sl[2 * q + 1]);
    }
  }
  float4* yr = (float4*)(ts + i * RS);
#pragma unroll
  for (int q = 0; q < KC / 2; ++q) {
    float4 y = yr[q];
    kf_df_sub(y.x, y.y, sh[2 * q], sl[2 * q]);
    kf_df_sub(y.z, y.w, sh[2 * q + 1], sl[2 * q + 1]);
    yr[q] = y;
  }
}

// The reduced systems of the mixed path's sweep for several right-hand sides:
// the structure of k_zsolve_multi, with the KC columns held as double-float
// pairs and the row updates formed from the pairs of the LU factors (ZLUdf)
// in double-float arithmetic on the FP32 pipes, which have about 60 times the
// FP64 pipe's rate (the FP64 updates, z^2 k multiply-adds per node and sweep,
// bounded this step).  The 32 x 32 diagonal blocks stay FP64: their entries
// come from ZLU, each warp converts its column of the block to FP64, solves it
// with shuffles and splits the result back.
template <int KC>
__global__ void __launch_bounds__(256) k_zsolve_df(const int32_t* __restrict__ rank, int node0, int ldz, int s_max,
                                                   const double* __restrict__ ZLU, const float2* __restrict__ ZLUdf,
                                                   const int32_t* __restrict__ piv, const double* __restrict__ in,
                                                   double* __restrict__ out, int k, int transpose) {
  constexpr int RS = KC + 2;
  extern __shared__ __align__(16) unsigned char zd_smem[];
  const int nl = blockIdx.x, node = node0 + nl;
  const int l = 2 * node, r = l + 1, sl = rank[l], sr = rank[r], z = sl + sr;
  const int c0 = blockIdx.y * KC;
  if (c0 >= k || z == 0) return;
  const int kc = min(KC, k - c0), zpad = (z + 31) / 32 * 32;
  float2* ts = (float2*)zd_smem;                 // zpad x RS pairs
  int* pm = (int*)(ts + (size_t)zpad * RS);      // z
  __shared__ double db[32][33];
  __shared__ double dinv[32];
  const double* A = ZLU + (int64_t)node * ldz * ldz;
  const float2* Ad = ZLUdf + (int64_t)node * ldz * ldz;
  const int32_t* pv = piv + (int64_t)node * ldz;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto dst = [&](int i) -> int64_t { return i < sl ? (int64_t)l * s_max + i : (int64_t)r * s_max + (i - sl); };
  for (int i = tid; i < z; i += blockDim.x) pm[i] = pv[i];
  __syncthreads();
  for (int e = tid; e < zpad * RS; e += blockDim.x) {
    const int i = e / RS, c = e % RS;
    ts[e] = (i < z && c < kc) ? kf_split_df(in[dst(transpose ? i : pm[i]) * k + c0 + c]) : make_float2(0.f, 0.f);
  }
  auto stage = [&](int kb, int nb, bool recip) {
    __syncthreads();
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
      const int i = e >> 5, j = e & 31;
      db[i][j] = (i < nb && j < nb) ? A[(int64_t)pm[kb + i] * ldz + kb + j] : 0.0;
    }
    __syncthreads();
    if (recip && tid < 32) dinv[lane] = lane < nb ? 1.0 / db[lane][lane] : 0.0;
    __syncthreads();
  };
  auto get = [&](int i, int c) -> double {
    const float2 v = ts[i * RS + c];
    return (double)v.x + (double)v.y;
  };
  auto update = [&](int i, int kb, const float2 (&lv)[32]) { block_row_update_df<KC, RS>(ts, i, kb, lv); };
  const float2 zero2 = make_float2(0.f, 0.f);
  const int top = (z - 1) / 32 * 32;
  if (!transpose) {
    for (int kb = 0; kb < z; kb += 32) {  // L (unit lower): forward
      const int nb = min(32, z - kb);
      stage(kb, nb, false);
      for (int c = warp; c < KC; c += 8) {
        double yi = lane < nb ? get(kb + lane, c) : 0.0;
        for (int j = 0; j < nb; ++j) {
          const double yj = __shfl_sync(0xffffffffu, yi, j);
          if (lane > j && lane < nb) yi = fma(-db[lane][j], yj, yi);
        }
        if (lane < nb) ts[(kb + lane) * RS + c] = kf_split_df(yi);
      }
      __syncthreads();
      for (int i = kb + nb + tid; i < z; i += blockDim.x) {
        const float2* Ai = Ad + (int64_t)pm[i] * ldz + kb;
        float2 lv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) lv[j] = j < nb ? Ai[j] : zero2;
        update(i, kb, lv);
      }
    }
    for (int kb = top; kb >= 0; kb -= 32) {  // U: backward
      const int nb = min(32, z - kb);
      stage(kb, nb, true);
      for (int c = warp; c < KC; c += 8) {
        double xi = lane < nb ? get(kb + lane, c) : 0.0;
        for (int j = nb - 1; j >= 0; --j) {
          if (lane == j) xi *= dinv[j];
          const double xj = __shfl_sync(0xffffffffu, xi, j);
          if (lane < j) xi = fma(-db[lane][j], xj, xi);
        }
        if (lane < nb) ts[(kb + lane) * RS + c] = kf_split_df(xi);
      }
      __syncthreads();
      for (int i = tid; i < kb; i += blockDim.x) {
        const float2* Ai = Ad + (int64_t)pm[i] * ldz + kb;
        float2 lv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) lv[j] = j < nb ? Ai[j] : zero2;
        update(i, kb, lv);
      }
    }
  } else {
    for (int kb = 0; kb < z; kb += 32) {  // U^T: forward
      const int nb = min(32, z - kb);
      stage(kb, nb, true);
      for (int c = warp; c < KC; c += 8) {
        double yi = lane < nb ? get(kb + lane, c) : 0.0;
        for (int j = 0; j < nb; ++j) {
          if (lane == j) yi *= dinv[j];
          const double yj = __shfl_sync(0xffffffffu, yi, j);
          if (lane > j && lane < nb) yi = fma(-db[j][lane], yj, yi);
        }
        if (lane < nb) ts[(kb + lane) * RS + c] = kf_split_df(yi);
      }
      __syncthreads();
      for (int i = kb + nb + tid; i < z; i += blockDim.x) {
        float2 lv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) lv[j] = j < nb ? Ad[(int64_t)pm[kb + j] * ldz + i] : zero2;
        update(i, kb, lv);
      }
    }
    for (int kb = top; kb >= 0; kb -= 32) {  // L^T (unit): backward
      const int nb = min(32, z - kb);
      stage(kb, nb, false);
      for (int c = warp; c < KC; c += 8) {
        double xi = lane < nb ? get(kb + lane, c) : 0.0;
        for (int j = nb - 1; j >= 0; --j) {
          const double xj = __shfl_sync(0xffffffffu, xi, j);
          if (lane < j) xi = fma(-db[j][lane], xj, xi);
        }
        if (lane < nb) ts[(kb + lane) * RS + c] = kf_split_df(xi);
      }
      __syncthreads();
      for (int i = tid; i < kb; i += blockDim.x) {
        float2 lv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) lv[j] = j < nb ? Ad[(int64_t)pm[kb + j] * ldz + i] : zero2;
        update(i, kb, lv);
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < z * RS; e += blockDim.x) {
    const int i = e / RS, c = e % RS;
    if (c < kc) out[dst(transpose ? pm[i] : i) * k + c0 + c] = (double)ts[e].x + (double)ts[e].y;
  }
}

template <int KC>
inline size_t zsolve_df_smem(int ldz) {
  const int zpad = (ldz + 31) / 32 * 32;
  return sizeof(float2) * (size_t)zpad * (KC + 2) + sizeof(int) * (size_t)ldz;
}

// The same product for several right-hand sides at once: a 32 x 64 tile of
// out (32 entries of the node's vector x 64 columns) per CTA, the reduction
// over the node's z entries in chunks of 32 with the Z^-1 block (or its
// transpose) and the input block staged in shared memory, so that Z^-1 is
// read once per 64 columns instead of once per column.  Thread (ty, tx)
// forms rows ty*4..+3 of columns tx and tx + 32.
__global__ void __launch_bounds__(256) k_zinv_apply_multi(const int32_t* __restrict__ rank, int node0, int ldz,
                                                          int s_max, const double* __restrict__ Zinv,
                                                          const double* __restrict__ in, double* __restrict__ out,
                                                          int k, int transpose) {
  __shared__ double sa[32][33];
  __shared__ double su[32][65];
  const int node = node0 + blockIdx.x, l = 2 * node, r = l + 1, sl = rank[l], sr = rank[r], z = sl + sr;
  const int e0 = blockIdx.y * 32, c0 = blockIdx.z * 64;
  if (e0 >= z || c0 >= k) return;
  const double* A = Zinv + (int64_t)node * ldz * ldz;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  auto dst = [&](int i) -> int64_t { return i < sl ? (int64_t)l * s_max + i : (int64_t)r * s_max + (i - sl); };
  double acc[4][2] = {};
  for (int j0 = 0; j0 < z; j0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ii = ty * 4 + q, i = e0 + ii, j = j0 + tx;
      // row i of Z^-1 (or column i, for Z^-T), entries j0..j0+31
      sa[ii][tx] = (i < z && j < z) ? (transpose ? A[(int64_t)j * ldz + i] : A[(int64_t)i * ldz + j]) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int jj = ty * 4 + q, j = j0 + jj;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int c = c0 + tx + 32 * h2;
        su[jj][tx + 32 * h2] = (j < z && c < k) ? in[dst(j) * k + c] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < 32; ++jj) {
      const double u0 = su[jj][tx], u1 = su[jj][tx + 32];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double a = sa[ty * 4 + q][jj];
        acc[q][0] = fma(a, u0, acc[q][0]);
        acc[q][1] = fma(a, u1, acc[q][1]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = e0 + ty * 4 + q;
    if (i >= z) continue;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int c = c0 + tx + 32 * h2;
      if (c < k) out[dst(i) * k + c] = acc[q][h2];
    }
  }
}

// ---- operator pieces ------------------------------------------------------------
// Leaf blocks: y_i = lambda x_i + sum_j K(x_i, x_j) x_j (or dK/dh, no lambda).
// ---- reduced systems by the explicit inverse (upper levels) -------------------
// out[l], out[r] <- Z^-1 [in[l]; in[r]] (transpose = 0) or Z^-T [...] (1) for
// the levels that keep Z^-1: the LU solve of such a node is a chain of 2 z/32
// dependent blocks on one CTA, while this product spreads a node over z/32
// CTAs.  blockIdx.x = node of the level, blockIdx.y = a block of 32 output
// entries.  Z^-1: warp w forms entries w, w + 8, .. of the block, lanes over
// the columns (a row is one coalesced segment), 16 loads in flight per lane,
// shuffle reduction.  Z^-T: lane q forms entry q of the block (column q of
// Z^-1: a row's 32 entries are one coalesced segment), the warps split the
// rows and add their partial sums in shared memory.
constexpr int kZinvChunk = 16;
__global__ void __launch_bounds__(256) k_zinv_apply(const int32_t* __restrict__ rank, int node0, int ldz, int s_max,
                                                    const double* __restrict__ Zinv, const double* __restrict__ in,
                                                    double* __restrict__ out, int k, int transpose) {
  __shared__ double u[2 * KF_MAX_SMAX];
  __shared__ double part[8][33];
  const int node = node0 + blockIdx.x, l = 2 * node, r = l + 1, sl = rank[l], sr = rank[r], z = sl + sr;
  const int e0 = blockIdx.y * 32;
  if (e0 >= z) return;
  const double* A = Zinv + (int64_t)node * ldz * ldz;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto dst = [&](int i) -> int64_t { return i < sl ? (int64_t)l * s_max + i : (int64_t)r * s_max + (i - sl); };
  for (int c = 0; c < k; ++c) {
    __syncthreads();
    for (int i = tid; i < z; i += blockDim.x) u[i] = in[dst(i) * k + c];
    __syncthreads();
    if (!transpose) {
      for (int q = warp; q < 32; q += 8) {
        const int i = e0 + q;
        if (i >= z) break;  // warp-uniform
        const double* Ai = A + (int64_t)i * ldz;
        double acc = 0.0;
        for (int j0 = 0; j0 < z; j0 += 32 * kZinvChunk) {
          double v[kZinvChunk];
#pragma unroll
          for (int t = 0; t < kZinvChunk; ++t) {
            const int j = j0 + 32 * t + lane;
            v[t] = j < z ? Ai[j] : 0.0;
          }
#pragma unroll
          for (int t = 0; t < kZinvChunk; ++t) {
            const int j = j0 + 32 * t + lane;
            if (j < z) acc = fma(v[t], u[j], acc);
          }
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) out[dst(i) * k + c] = acc;
      }
    } else {
      const int j = e0 + lane;
      double acc = 0.0;
      if (j < z) {
        for (int i0 = warp; i0 < z; i0 += 8 * kZinvChunk) {
          double v[kZinvChunk];
#pragma unroll
          for (int t = 0; t < kZinvChunk; ++t) {
            const int i = i0 + 8 * t;
            v[t] = i < z ? A[(int64_t)i * ldz + j] : 0.0;
          }
#pragma unroll
          for (int t = 0; t < kZinvChunk; ++t) {
            const int i = i0 + 8 * t;
            if (i < z) acc = fma(v[t], u[i], acc);
          }
        }
      }
      part[warp][lane] = acc;
      __syncthreads();
      if (warp == 0 && j < z) {
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) sum += part[w][lane];
        out[dst(j) * k + c] = sum;
      }
    }
  }
}

template <typename TM>
__global__ void __launch_bounds__(128) k_leaf_mv(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                 int leaf0, const double* __restrict__ X64,
                                                 const float* __restrict__ X32, int d, double c_exp, double inv_h3,
                                                 int src, double lambda, const double* __restrict__ x,
                                                 double* __restrict__ y, int k) {
  const int lf = blockIdx.y, node = leaf0 + lf;
  const int b = lo[node], n = hi[node] - b;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int r = 0; r < k; ++r) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc += eval_src<TM>(src, X64, X32, b + i, b + j, d, c_exp, inv_h3) * x[(int64_t)(b + j) * k + r];
    y[(int64_t)(b + i) * k + r] = (src == SRC_DKERNEL ? 0.0 : lambda * x[(int64_t)(b + i) * k + r]) + acc;
  }
}

// Leaf blocks from the stored FP64-accurate copy (double-float pairs):
// y_i = lambda x_i + sum_j K[i][j] x_j, the products and sums in double-float
// arithmetic on the FP32 pipes.  The leaf's x is split into pairs once per
// CTA in shared memory; one warp per row, lanes over j.
// RB right-hand sides r0 .. r0 + RB - 1 (those below k) per launch: each row of
// Kdf is read once for all of them; per right-hand side the arithmetic and its
// order are those of RB = 1.
template <int RB>
__global__ void __launch_bounds__(512) k_leaf_mv_df(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                    int leaf0, int ldL, const float2* __restrict__ Kdf,
                                                    double lambda, const double* __restrict__ x,
                                                    const float2* __restrict__ xdf, double* __restrict__ y, int k,
                                                    int r0) {
  extern __shared__ float2 xs[];  // RB x n: the lanes' consecutive j are consecutive words
  const int lf = blockIdx.y, node = leaf0 + lf;
  const int b = lo[node], n = hi[node] - b;
  const int nr = min(RB, k - r0);
  for (int e = threadIdx.x; e < n * RB; e += blockDim.x) {
    const int j = e / RB, q = e % RB;
    xs[q * n + j] = q < nr ? xdf[(int64_t)(b + j) * k + r0 + q] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < n; i += (gridDim.x * blockDim.x) >> 5) {
    const float2* Ki = Kdf + ((int64_t)lf * ldL + i) * ldL;
    float sh[RB], sl[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) sh[q] = sl[q] = 0.f;
    // four entries of the row in flight before their products (the same order of sums)
    int j = lane;
    for (; j + 96 < n; j += 128) {
      float2 m[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) m[u] = Ki[j + 32 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < RB; ++q) {
          const float2 v = xs[q * n + j + 32 * u];
          kf_df_fma(m[u].x, m[u].y, v.x, v.y, sh[q], sl[q]);
        }
    }
    for (; j < n; j += 32) {
      const float2 m = Ki[j];
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const float2 v = xs[q * n + j];
        kf_df_fma(m.x, m.y, v.x, v.y, sh[q], sl[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      for (int off = 16; off > 0; off >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, sh[q], off), ol = __shfl_xor_sync(0xffffffffu, sl[q], off);
        float t, e;
        kf_two_sum(sh[q], oh, t, e);
        e = __fadd_rn(e, __fadd_rn(sl[q], ol));
        kf_fast_two_sum(t, e, sh[q], sl[q]);
      }
      if (lane == 0 && q < nr)
        y[(int64_t)(b + i) * k + r0 + q] =
            lambda * x[(int64_t)(b + i) * k + r0 + q] + ((double)sh[q] + (double)sl[q]);
    }
  }
}

// V pass of the FP64-accurate operator: u[sib][q][r] += sum_i V[i][q] w[i][r]
// over the rows of every node of a level, V as double-float pairs, in
// double-float arithmetic on the FP32 pipes (the same partition as k_colsum,
// one thread per skeleton column, the chunk's w split into pairs in shared
// memory, 8 rows' loads in flight).
template <int KB, int ROWS = kRowsPerChunk>
__global__ void __launch_bounds__(256) k_colsum_df(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                   const int32_t* __restrict__ rank, int node0, int s_max,
                                                   const float2* __restrict__ M, const float2* __restrict__ W, int k,
                                                   double* __restrict__ parts) {
  __shared__ float2 ws[ROWS][KB];
  const int nl = blockIdx.y, node = node0 + nl, sib = node ^ 1;
  const int b = lo[node], n = hi[node] - b;
  const int cnt = rank[sib];
  const int r0 = blockIdx.x * ROWS;
  if (r0 >= n || cnt == 0) return;
  const int r1 = min(n, r0 + ROWS), nr = r1 - r0;
  for (int kb = 0; kb < k; kb += KB) {
    const int kk = min(KB, k - kb);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * KB; e += blockDim.x) {
      const int i = e / KB, c = e % KB;
      ws[i][c] = c < kk ? W[(int64_t)(b + r0 + i) * k + kb + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      float sh[KB], sl[KB];
#pragma unroll
      for (int c = 0; c < KB; ++c) sh[c] = sl[c] = 0.f;
      const float2* Mq = M + (int64_t)(b + r0) * s_max + q;
      int i = 0;
      for (; i + 8 <= nr; i += 8) {
        float2 m[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) m[u] = Mq[(int64_t)(i + u) * s_max];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int c = 0; c < KB; ++c) kf_df_fma(m[u].x, m[u].y, ws[i + u][c].x, ws[i + u][c].y, sh[c], sl[c]);
      }
      for (; i < nr; ++i) {
        const float2 m = Mq[(int64_t)i * s_max];
#pragma unroll
        for (int c = 0; c < KB; ++c) kf_df_fma(m.x, m.y, ws[i][c].x, ws[i][c].y, sh[c], sl[c]);
      }
      double* out = parts + (((int64_t)nl * gridDim.x + blockIdx.x) * s_max + q) * k + kb;
      for (int c = 0; c < kk; ++c) out[c] = (double)sh[c] + (double)sl[c];
    }
  }
}

// Push skeleton coefficients down: g[l] += P_c[:s_l] g[a], g[r] += P_c[s_l:] g[a].
// blockIdx.x = node of the level, blockIdx.y = a block of 32 rows of P_c:
// warp w forms rows w, w + 8, .. of the block, lanes over the columns (a row
// of P_c is contiguous), shuffle reduction; a node spreads over z/32 CTAs.
// Also the memory-lean sweep's push of reduced-system solutions through
// T = Z^-1 P_c (same layout, FP32 on the mixed path): Gin and G may differ.
template <typename TP>
__global__ void __launch_bounds__(256) k_push_down(const int32_t* __restrict__ rank, int node0, int s_max,
                                                   const TP* __restrict__ Pc, const double* __restrict__ Gin,
                                                   double* __restrict__ G, int k) {
  const int node = node0 + blockIdx.x;
  const int l = 2 * node, r = l + 1, sl = rank[l], sr = rank[r], s = rank[node], z = sl + sr;
  const int i0 = blockIdx.y * 32;
  if (i0 >= z || s == 0) return;
  const TP* P = Pc + (int64_t)node * 2 * s_max * s_max;
  const double* ga = Gin + (int64_t)node * s_max * k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int w = warp; w < 32; w += 8) {
    const int i = i0 + w;
    if (i >= z) break;  // warp-uniform
    const TP* Pi = P + (int64_t)i * s_max;
    double* dst = i < sl ? G + ((int64_t)l * s_max + i) * k : G + ((int64_t)r * s_max + (i - sl)) * k;
    for (int c = 0; c < k; ++c) {
      double acc = 0.0;
      for (int q = lane; q < s; q += 32) acc = fma((double)Pi[q], ga[(int64_t)q * k + c], acc);
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) dst[c] += acc;
    }
  }
}

// The same push for several right-hand sides: a 32 x 64 tile of the
// children's rows (32 rows of P_c x 64 columns) per CTA, the reduction over
// the parent's s entries in chunks of 32 with the P_c block and g[a] staged in
// shared memory (P_c read once per 64 columns).  Thread (ty, tx) forms rows
// ty*4..+3 of columns tx and tx + 32.  grid = (nodes, z / 32, k / 64).
template <typename TP>
__global__ void __launch_bounds__(256) k_push_down_multi(const int32_t* __restrict__ rank, int node0, int s_max,
                                                         const TP* __restrict__ Pc, const double* __restrict__ Gin,
                                                         double* __restrict__ G, int k) {
  __shared__ double sa[32][33];
  __shared__ double su[32][65];
  const int node = node0 + blockIdx.x;
  const int l = 2 * node, r = l + 1, sl = rank[l], sr = rank[r], s = rank[node], z = sl + sr;
  const int e0 = blockIdx.y * 32, c0 = blockIdx.z * 64;
  if (e0 >= z || c0 >= k || s == 0) return;
  const TP* P = Pc + (int64_t)node * 2 * s_max * s_max;
  const double* ga = Gin + (int64_t)node * s_max * k;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  double acc[4][2] = {};
  for (int j0 = 0; j0 < s; j0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ii = ty * 4 + q, i = e0 + ii, j = j0 + tx;
      sa[ii][tx] = (i < z && j < s) ? (double)P[(int64_t)i * s_max + j] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int jj = ty * 4 + q, j = j0 + jj;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int c = c0 + tx + 32 * h2;
        su[jj][tx + 32 * h2] = (j < s && c < k) ? ga[(int64_t)j * k + c] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < 32; ++jj) {
      const double u0 = su[jj][tx], u1 = su[jj][tx + 32];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double a = sa[ty * 4 + q][jj];
        acc[q][0] = fma(a, u0, acc[q][0]);
        acc[q][1] = fma(a, u1, acc[q][1]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = e0 + ty * 4 + q;
    if (i >= z) continue;
    double* dst = i < sl ? G + ((int64_t)l * s_max + i) * k : G + ((int64_t)r * s_max + (i - sl)) * k;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int c = c0 + tx + 32 * h2;
      if (c < k) dst[c] += acc[q][h2];
    }
  }
}

// Several right-hand sides on the mixed path's FP64-accurate operator:
// out[i][c] += sum_q M[i][q] v[q][c] for the rows of a matrix stored as
// double-float pairs, in double-float arithmetic on the FP32 pipes (the FP64
// pipe would bound these passes at 2 k FP64 flops per entry, and splitting
// FP64 entries here would bound them at the FP64 pipe's conversions).  MODE 0:
// the rows of the leaf interpolation P of a leaf (grid.y) into y from v =
// g[leaf]; 1 (PUSH): the rows of P_c of a node of the level, pushed into its
// children's skeleton weights g[l], g[r] from v = g[node]; 2: the rows of the
// V blocks of a level, K(x_i, sib~), in the transposed operator (v = g[sib]).
// A warp takes 32 rows and walks the columns in 32-wide tiles staged row by
// row (coalesced); lane q forms row q's KB sums.  v is split into pairs once
// per CTA (dynamic shared memory: KF_MAX_SMAX x KB pairs, then the warps'
// tiles).
template <int KB, int MODE>
__global__ void __launch_bounds__(256) k_rows_df(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                 const int32_t* __restrict__ rank, int node0, int s_max,
                                                 const float2* __restrict__ M, const double* __restrict__ V,
                                                 double* __restrict__ out, int k) {
  extern __shared__ __align__(16) unsigned char rd_smem[];
  float2* vs = (float2*)rd_smem;                                                   // KF_MAX_SMAX x KB
  float2(*tile)[32][33] = (float2(*)[32][33])(rd_smem + sizeof(float2) * KF_MAX_SMAX * KB);  // 8 warps
  constexpr bool PUSH = MODE == 1;
  const int node = node0 + blockIdx.y, from = MODE == 2 ? node ^ 1 : node;
  int nrows, cnt, sl = 0;
  const float2* Mb;
  if (PUSH) {
    sl = rank[2 * node];
    nrows = sl + rank[2 * node + 1];
    cnt = rank[node];
    Mb = M + (int64_t)node * 2 * s_max * s_max;
  } else {
    nrows = hi[node] - lo[node];
    cnt = rank[from];
    Mb = M + (int64_t)lo[node] * s_max;
  }
  const int r0 = blockIdx.x * kRowUpdRows;
  if (cnt == 0 || r0 >= nrows) return;
  const int r1 = min(nrows, r0 + kRowUpdRows);
  const double* v = V + (int64_t)from * s_max * k;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cpad = (cnt + 31) & ~31;
  float2(*t)[33] = tile[warp];
  auto dst = [&](int i) -> double* {
    if (PUSH) return out + ((int64_t)(i < sl ? 2 * node : 2 * node + 1) * s_max + (i < sl ? i : i - sl)) * k;
    return out + (int64_t)(lo[node] + i) * k;
  };
  for (int kb = 0; kb < k; kb += KB) {
    const int kk = min(KB, k - kb);
    __syncthreads();
    for (int e = threadIdx.x; e < cpad * KB; e += blockDim.x) {
      const int q = e / KB, r = e % KB;
      vs[e] = (q < cnt && r < kk) ? kf_split_df(v[(int64_t)q * k + kb + r]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int i0 = r0 + warp * 32; i0 < r1; i0 += 8 * 32) {
      float sh[KB], sl2[KB];
#pragma unroll
      for (int r = 0; r < KB; ++r) sh[r] = sl2[r] = 0.f;
      for (int q0 = 0; q0 < cnt; q0 += 32) {
        float2 x[32];
#pragma unroll
        for (int rr = 0; rr < 32; ++rr)
          x[rr] = (i0 + rr < r1 && q0 + lane < cnt) ? Mb[(int64_t)(i0 + rr) * s_max + q0 + lane]
                                                    : make_float2(0.f, 0.f);
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) t[rr][lane] = x[rr];
        __syncwarp();
        for (int j = 0; j < 32; ++j) {
          const float2 m = t[lane][j];
          const float2* vj = vs + (q0 + j) * KB;  // one address in every lane: a broadcast
#pragma unroll
          for (int r = 0; r < KB; ++r) kf_df_fma(m.x, m.y, vj[r].x, vj[r].y, sh[r], sl2[r]);
        }
        __syncwarp();
      }
      if (i0 + lane < r1) {
        double* o = dst(i0 + lane) + kb;
#pragma unroll
        for (int r = 0; r < KB; ++r)
          if (r < kk) o[r] += (double)sh[r] + (double)sl2[r];
      }
    }
  }
}

template <int KB>
constexpr size_t rows_df_smem() { return sizeof(float2) * (KF_MAX_SMAX * KB + 8 * 32 * 33); }

// The memory-lean sweep's push of reduced-system solutions, one right-hand
// side: g[l], g[r] += T g[a] with T = Z^-1 P_c, in the factor's precision (the
// sweep's: FP32 on the mixed path, where FP64 products would bound this push
// at the FP64 pipe's rate), g[a] staged in shared memory once per CTA;
// blockIdx.x = node, blockIdx.y = a block of 32 rows of T, a warp per row.
template <typename TP>
__global__ void __launch_bounds__(256) k_push_down_lean(const int32_t* __restrict__ rank, int node0, int s_max,
                                                        const TP* __restrict__ Tw, const double* __restrict__ Gin,
                                                        double* __restrict__ G) {
  __shared__ TP gs[KF_MAX_SMAX];
  const int node = node0 + blockIdx.x;
  const int l = 2 * node, r = l + 1, sl = rank[l], sr = rank[r], s = rank[node], z = sl + sr;
  const int i0 = blockIdx.y * 32;
  if (i0 >= z || s == 0) return;
  const TP* P = Tw + (int64_t)node * 2 * s_max * s_max;
  for (int q = threadIdx.x; q < s; q += blockDim.x) gs[q] = (TP)Gin[(int64_t)node * s_max + q];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int w = warp; w < 32; w += 8) {
    const int i = i0 + w;
    if (i >= z) break;  // warp-uniform
    const TP* Pi = P + (int64_t)i * s_max;
    TP acc = (TP)0;
    for (int q = lane; q < s; q += 32) acc += Pi[q] * gs[q];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) (i < sl ? G[(int64_t)l * s_max + i] : G[(int64_t)r * s_max + (i - sl)]) += (double)acc;
  }
}

// Gather skeleton weights up (transposed operator): g[a] += P_c^T [g[l]; g[r]].
// blockIdx.x = node of the level, blockIdx.y = a block of 32 columns of P_c:
// lane q forms column q of the block (a row's 32 entries are one coalesced
// segment), the warps split the rows and add their partial sums in shared
// memory.
template <typename TP>
__global__ void __launch_bounds__(256) k_push_up(const int32_t* __restrict__ rank, int node0, int s_max,
                                                 const TP* __restrict__ Pc, const double* __restrict__ Gin,
                                                 double* __restrict__ G, int k) {
  __shared__ double part[8][33];
  const int node = node0 + blockIdx.x;
  const int l = 2 * node, r = l + 1, sl = rank[l], sr = rank[r], s = rank[node], z = sl + sr;
  const int q0 = blockIdx.y * 32;
  if (q0 >= s) return;
  const TP* P = Pc + (int64_t)node * 2 * s_max * s_max;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, q = q0 + lane;
  for (int c = 0; c < k; ++c) {
    double acc = 0.0;
    if (q < s)
      for (int i = warp; i < z; i += 8) {
        const double gi = i < sl ? Gin[((int64_t)l * s_max + i) * k + c] : Gin[((int64_t)r * s_max + (i - sl)) * k + c];
        acc = fma((double)P[(int64_t)i * s_max + q], gi, acc);
      }
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && q < s) {
      double sum = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) sum += part[w][lane];
      G[((int64_t)node * s_max + q) * k + c] += sum;
    }
    __syncthreads();
  }
}

// The same gather for several right-hand sides: a 32 x 64 tile of g[a]
// (32 of its s entries x 64 columns) per CTA, the reduction over the z rows
// of P_c in chunks of 32 with the P_c block and the children's weights
// staged in shared memory.  grid = (nodes, s / 32, k / 64).
template <typename TP>
__global__ void __launch_bounds__(256) k_push_up_multi(const int32_t* __restrict__ rank, int node0, int s_max,
                                                       const TP* __restrict__ Pc, const double* __restrict__ Gin,
                                                       double* __restrict__ G, int k) {
  __shared__ double sa[32][33];
  __shared__ double su[32][65];
  const int node = node0 + blockIdx.x;
  const int l = 2 * node, r = l + 1, sl = rank[l], sr = rank[r], s = rank[node], z = sl + sr;
  const int q0 = blockIdx.y * 32, c0 = blockIdx.z * 64;
  if (q0 >= s || c0 >= k) return;
  const TP* P = Pc + (int64_t)node * 2 * s_max * s_max;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  auto gch = [&](int i) -> const double* {
    return i < sl ? Gin + ((int64_t)l * s_max + i) * k : Gin + ((int64_t)r * s_max + (i - sl)) * k;
  };
  double acc[4][2] = {};
  for (int i0 = 0; i0 < z; i0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // sa[qq][ii] = P[i0 + ii][q0 + qq]: row i0 + ii read along q
      const int ii = ty * 4 + q, i = i0 + ii, qq = q0 + tx;
      sa[tx][ii] = (i < z && qq < s) ? (double)P[(int64_t)i * s_max + qq] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ii = ty * 4 + q, i = i0 + ii;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int c = c0 + tx + 32 * h2;
        su[ii][tx + 32 * h2] = (i < z && c < k) ? gch(i)[c] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int ii = 0; ii < 32; ++ii) {
      const double u0 = su[ii][tx], u1 = su[ii][tx + 32];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double a = sa[ty * 4 + q][ii];
        acc[q][0] = fma(a, u0, acc[q][0]);
        acc[q][1] = fma(a, u1, acc[q][1]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int qq = q0 + ty * 4 + q;
    if (qq >= s) continue;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int c = c0 + tx + 32 * h2;
      if (c < k) G[((int64_t)node * s_max + qq) * k + c] += acc[q][h2];
    }
  }
}

// V pass of the transposed FP64-accurate operator: w[i][r] += sum_q V[i][q]
// g[sib][q][r] for the rows of every node of a level, V as double-float pairs
// (row i of node c: K(x_i, sib~)), in double-float arithmetic on the FP32
// pipes: one warp per row, lanes over q, the lanes' pairs combined with exact
// two-sums; g[sib] split into pairs in shared memory.
__global__ void __launch_bounds__(256) k_rowupd_df(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                   const int32_t* __restrict__ rank, int node0, int s_max,
                                                   const float2* __restrict__ M, const double* __restrict__ G, int k,
                                                   double* __restrict__ W) {
  __shared__ float2 gs[KF_MAX_SMAX];
  const int nl = blockIdx.y, node = node0 + nl, sib = node ^ 1;
  const int b = lo[node], n = hi[node] - b;
  const int cnt = rank[sib];
  const int r0 = blockIdx.x * kRowUpdRows;
  if (cnt == 0 || r0 >= n) return;
  const int r1 = min(n, r0 + kRowUpdRows);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = 0; r < k; ++r) {
    __syncthreads();
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) gs[q] = kf_split_df(G[((int64_t)sib * s_max + q) * k + r]);
    __syncthreads();
    for (int i = r0 + warp; i < r1; i += 8) {
      const float2* Mi = M + (int64_t)(b + i) * s_max;
      float sh = 0.f, sl = 0.f;
      for (int q = lane; q < cnt; q += 32) {
        const float2 m = Mi[q], v = gs[q];
        kf_df_fma(m.x, m.y, v.x, v.y, sh, sl);
      }
      for (int off = 16; off > 0; off >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, sh, off), ol = __shfl_xor_sync(0xffffffffu, sl, off);
        float t, e;
        kf_two_sum(sh, oh, t, e);
        e = __fadd_rn(e, __fadd_rn(sl, ol));
        kf_fast_two_sum(t, e, sh, sl);
      }
      if (lane == 0) W[(int64_t)(b + i) * k + r] += (double)sh + (double)sl;
    }
  }
}

// x as double-float pairs, once per operator product (the FP64 pipe that the
// split needs is far too narrow to split it again in every CTA that reads it)
__global__ void k_split_vec(const double* __restrict__ a, float2* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = kf_split_df(a[i]);
}

template <typename TV>
__global__ void k_axpy_cast(const double* __restrict__ a, TV* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (TV)a[i];
}
template <typename TV>
__global__ void k_cast_back(const TV* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// ---- drivers -------------------------------------------------------------------------
template <typename TM, typename TV>
kf_status solve_t(kf_factor* f, TV* W, int64_t k, int transpose, double* U, double* Vb, double* parts, double* parts2,
                  cudaStream_t s) {
  kf_tree* t = f->t;
  kf_ctx* c = f->ctx;
  const int D = t->D, s_max = f->s_max, ldz = 2 * s_max;
  const int64_t N = t->N;
  const TM* L = (const TM*)f->L;
  const TM* Phat = (const TM*)f->Phat;
  const TM* VT = (const TM*)f->VT;
  auto lvl = [&](const TM* base, int l) { return base + (int64_t)(l - 1) * N * s_max; };
  const int leaf0 = 1 << D;
  const size_t ubytes = sizeof(double) * (size_t)(t->nnodes + 1) * s_max * k;
  const double inv_h3 = 1.0 / (f->h * f->h * f->h);
  const int vsrc = f->vstore == KF_V_STORED ? SRC_STORED : SRC_KERNEL;
  // dynamic shared memory: the warps' 32 x 33 row tiles (plus the Z solve's vectors and row map)
  const size_t ls_smem = sizeof(TM) * (kLeafSolveThreads / 32) * 32 * 33;
  const size_t zs_smem = sizeof(double) * (2 * (size_t)ldz + (ldz + 1) / 2 + 8 * 32 * 33);
  KF_CUDA(c, cudaFuncSetAttribute(k_leaf_solve<TM, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ls_smem));
  KF_CUDA(c, cudaFuncSetAttribute(k_zsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zs_smem));
  const size_t zm_smem = zsolve_multi_smem(ldz);
  const size_t zd16_smem = zsolve_df_smem<16>(ldz), zd8_smem = zsolve_df_smem<8>(ldz);
  if (k >= 2) {
    KF_CUDA(c, cudaFuncSetAttribute(k_zsolve_multi<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zm_smem));
    KF_CUDA(c, cudaFuncSetAttribute(k_zsolve_df<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zd16_smem));
    KF_CUDA(c, cudaFuncSetAttribute(k_zsolve_df<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zd8_smem));
  }
  // t = Z^-1 [u_l; u_r] (or Z^-T) for the nodes of level l: the explicit
  // inverse where the factorization kept it, else the LU
  auto zsolve = [&](int l, int tr) {
    if (l <= f->zinv_top && f->Zinv) {
      dim3 gz(1u << l, (unsigned)((ldz + 31) / 32));
      if (k >= 4) {
        dim3 gm(1u << l, (unsigned)((ldz + 31) / 32), (unsigned)((k + 63) / 64));
        KF_PHASE(KF_PH_S_ZSOLVE, s, k_zinv_apply_multi<<<gm, 256, 0, s>>>(f->rank, 1 << l, ldz, s_max, f->Zinv, U, Vb,
                                                                          (int)k, tr));
      } else {
        KF_PHASE(KF_PH_S_ZSOLVE, s, k_zinv_apply<<<gz, 256, 0, s>>>(f->rank, 1 << l, ldz, s_max, f->Zinv, U, Vb,
                                                                   (int)k, tr));
      }
    } else if (k >= 2 && f->ZLUdf) {  // mixed path: double-float row updates
      if (k > 8)
        KF_PHASE(KF_PH_S_ZSOLVE, s, k_zsolve_df<16><<<dim3(1u << l, (unsigned)((k + 15) / 16)), 256, zd16_smem,
                                                       s>>>(f->rank, 1 << l, ldz, s_max, f->ZLU, f->ZLUdf, f->Zpiv,
                                                            U, Vb, (int)k, tr));
      else
        KF_PHASE(KF_PH_S_ZSOLVE, s, k_zsolve_df<8><<<dim3(1u << l, 1u), 256, zd8_smem, s>>>(
                                        f->rank, 1 << l, ldz, s_max, f->ZLU, f->ZLUdf, f->Zpiv, U, Vb, (int)k, tr));
    } else if (k >= 2) {
      KF_PHASE(KF_PH_S_ZSOLVE, s, k_zsolve_multi<8><<<dim3(1u << l, (unsigned)((k + 7) / 8)), 256, zm_smem, s>>>(
                                      f->rank, 1 << l, ldz, s_max, f->ZLU, f->Zpiv, U, Vb, (int)k, tr));
    } else {
      KF_PHASE(KF_PH_S_ZSOLVE, s, k_zsolve<<<dim3(1u << l, 1u), 256, zs_smem, s>>>(f->rank, 1 << l, ldz, s_max,
                                                                                  f->ZLU, f->Zpiv, U, Vb, (int)k, tr));
    }
  };
  // leaf blocks: one column per pass (k = 1), else KC columns per pass with
  // the columns in shared memory (16 FP32 or 8 FP64 columns; 8 FP32 columns
  // for k <= 8), when the leaf's columns fit
  const int npad = (t->leaf_max + 31) / 32 * 32;
  constexpr int KCm = sizeof(TV) == 4 ? 16 : 8;
  // 16 columns a CTA only for k > 16: two CTAs of 8 columns per leaf for k <= 16
  // (the leaf's chain of 32-row blocks is latency bound; more CTAs hide it)
  const bool wide = sizeof(TV) == 4 && k > 16;
  const size_t lm_smem = sizeof(TV) * (size_t)npad *
                         (wide ? leaf_multi_stride<TV, KCm>() : leaf_multi_stride<TV, 8>());
  const bool leaf_multi = k >= 2 && lm_smem <= 200 * 1024;
  if (leaf_multi) {
    if (wide)
      KF_CUDA(c, cudaFuncSetAttribute(k_leaf_solve_multi<TM, TV, KCm>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)lm_smem));
    else
      KF_CUDA(c, cudaFuncSetAttribute(k_leaf_solve_multi<TM, TV, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)lm_smem));
  }
  auto leaf_solve = [&]() {
    if (!leaf_multi) {
      KF_PHASE(KF_PH_S_LEAF, s, k_leaf_solve<TM, TV><<<1 << D, kLeafSolveThreads, ls_smem, s>>>(
                                    t->d_lo, t->d_hi, leaf0, t->leaf_max, L, W, (int)k));
    } else if (wide) {
      const dim3 g(1u << D, (unsigned)((k + KCm - 1) / KCm));
      KF_PHASE(KF_PH_S_LEAF, s, k_leaf_solve_multi<TM, TV, KCm><<<g, 256, lm_smem, s>>>(
                                    t->d_lo, t->d_hi, leaf0, t->leaf_max, L, W, (int)k));
    } else {
      const dim3 g(1u << D, (unsigned)((k + 7) / 8));
      KF_PHASE(KF_PH_S_LEAF, s, k_leaf_solve_multi<TM, TV, 8><<<g, 256, lm_smem, s>>>(
                                    t->d_lo, t->d_hi, leaf0, t->leaf_max, L, W, (int)k));
    }
  };
  // the column sums and row updates of one level (sib: the columns / vector of
  // the sibling's skeleton)
  auto colsum = [&](int c0, int nc, int sib, int src, const TM* M, dim3 gc) {
    launch_colsum<TM, TV>(gc, s, t->d_lo, t->d_hi, f->rank, f->skel, c0, s_max, sib, src, M, t->X64, t->X32, t->d,
                          f->c_exp, inv_h3, W, (int)k, U, parts, parts2);
  };
  auto rowupd = [&](int c0, int nc, int64_t rows, int sib, int src, const TM* M, const double* V) {
    launch_rowupd<TM, TV>(rows, nc, s, t->d_lo, t->d_hi, f->rank, f->skel, c0, s_max, sib, src, M, t->X64, t->X32,
                          t->d, f->c_exp, inv_h3, V, -1.0, W, (int)k);
  };
  // memory-lean W: P^ of a level is P^_leaf times the T = Z^-1 P_c of the
  // nodes below it (Eq. e:invtelescope).  Forward: the reduced-system solution
  // t of the nodes of level l + 1 (in Vb) is pushed down through the T's to
  // the leaves (into U, whose entries below level l + 1 are zero), then one
  // leaf-level row update.  Transpose: the leaves' P^^T w (into U), gathered
  // up through the T's to level l + 1.
  const TM* Tw = (const TM*)f->Tw;
  const TM* Pleafh = Phat + kf_phat_level_off(f, D);
  const int64_t leaf_rows = (N >> D) + 1;
  const unsigned gpz = (unsigned)((2 * s_max + 31) / 32), gps = (unsigned)((s_max + 31) / 32);
  const unsigned gpk = (unsigned)((k + 63) / 64);
  auto lean_down = [&](int l) {
    const double* gin = Vb;
    for (int lev = l + 1; lev < D; ++lev) {
      if (k >= 2)
        KF_PHASE(KF_PH_S_ROWUPD, s, k_push_down_multi<TM><<<dim3(1u << lev, gpz, gpk), 256, 0, s>>>(
                                        f->rank, 1 << lev, s_max, Tw, gin, U, (int)k));
      else
        KF_PHASE(KF_PH_S_ROWUPD, s, k_push_down_lean<TM><<<dim3(1u << lev, gpz), 256, 0, s>>>(f->rank, 1 << lev,
                                                                                             s_max, Tw, gin, U));
      gin = U;
    }
    rowupd(leaf0, 1 << D, leaf_rows, 0, SRC_STORED, Pleafh, gin);
  };
  auto lean_up = [&](int l) {
    const dim3 gcl((unsigned)((leaf_rows + kRowsPerChunk - 1) / kRowsPerChunk), 1u << D);
    colsum(leaf0, 1 << D, 0, SRC_STORED, Pleafh, gcl);
    for (int lev = D - 1; lev >= l + 1; --lev) {
      if (k >= 2)
        KF_PHASE(KF_PH_S_COLSUM, s, k_push_up_multi<TM><<<dim3(1u << lev, gps, gpk), 256, 0, s>>>(
                                        f->rank, 1 << lev, s_max, Tw, U, U, (int)k));
      else
        KF_PHASE(KF_PH_S_COLSUM, s, k_push_up<TM><<<dim3(1u << lev, gps), 256, 0, s>>>(f->rank, 1 << lev, s_max, Tw,
                                                                                      U, U, (int)k));
    }
  };
  const bool lean = f->w_lean && Tw;
  if (!transpose) {
    leaf_solve();
    // the hybrid solver stops at its frontier level (the reduced system above
    // it is applied by kf_hybrid_top_solve); the direct solver goes to the root
    for (int l = D - 1; l >= f->hyb_L; --l) {
      const int c0 = 1 << (l + 1), nc = 1 << (l + 1);
      const int64_t rows = (N >> (l + 1)) + 1;
      KF_CUDA(c, cudaMemsetAsync(U, 0, ubytes, s));
      dim3 gc((unsigned)((rows + kRowsPerChunk - 1) / kRowsPerChunk), nc);
      colsum(c0, nc, 1, vsrc, VT + kf_vt_level_off(f, l + 1), gc);
      zsolve(l, 0);
      if (lean) lean_down(l);
      else rowupd(c0, nc, rows, 0, SRC_STORED, Phat + kf_phat_level_off(f, l + 1), Vb);
    }
  } else {
    for (int l = 0; l < D; ++l) {
      const int c0 = 1 << (l + 1), nc = 1 << (l + 1);
      const int64_t rows = (N >> (l + 1)) + 1;
      KF_CUDA(c, cudaMemsetAsync(U, 0, ubytes, s));
      dim3 gc((unsigned)((rows + kRowsPerChunk - 1) / kRowsPerChunk), nc);
      if (lean) lean_up(l);
      else colsum(c0, nc, 0, SRC_STORED, Phat + kf_phat_level_off(f, l + 1), gc);
      zsolve(l, 1);
      rowupd(c0, nc, rows, 1, vsrc, VT + kf_vt_level_off(f, l + 1), Vb);
    }
    leaf_solve();
  }
  KF_LAUNCH_CHECK(c);
  return KF_OK;
}

template <typename TM>
kf_status matvec_t(kf_factor* f, const double* x, double* y, int64_t k, int deriv, int transpose, double* G,
                   float2* xdf, double* parts, double* parts2, cudaStream_t s) {
  kf_tree* t = f->t;
  kf_ctx* c = f->ctx;
  const int D = t->D, s_max = f->s_max;
  const int64_t N = t->N;
  // stored V blocks are read only when src is SRC_STORED (never for dK~/dh,
  // which the FP64 instantiation also serves on the mixed path)
  const TM* VT = deriv ? nullptr : (const TM*)f->VT;
  const int leaf0 = 1 << D;
  const double inv_h3 = 1.0 / (f->h * f->h * f->h);
  const int src = deriv ? SRC_DKERNEL : (f->vstore == KF_V_STORED ? SRC_STORED : SRC_KERNEL);
  auto vt_level = [&](int l) { return VT ? VT + kf_vt_level_off(f, l) : nullptr; };
  const bool split = xdf && f->Kdf && !deriv;
  if (split) KF_PHASE(KF_PH_MISC, s, k_split_vec<<<grid_for(N * k, 256), 256, 0, s>>>(x, xdf, N * k));
  // 16 or more right-hand sides on factors with BF16 digits (tc_operator): the
  // leaf blocks and the V pass on the tensor cores (oz_op.cu), from the digits
  // of x formed once here
  kf_oz_x oz;
  if ((f->Ksl || (f->VTsl && !transpose && D > f->hyb_L)) && !deriv && k >= 16 && k <= 4096) {
    kf_status zs = kf_oz_prepare_x(f, x, k, &oz, s);
    if (zs != KF_OK) return zs;
  }
  if (oz.xsl && f->Ksl) {
    kf_status zs = kf_oz_leaf(f, oz, k, f->lambda, x, y, s);
    if (zs != KF_OK) {
      kf_oz_release_x(f, &oz, s);
      return zs;
    }
  } else if (f->Kdf && !deriv) {
    if (k == 1) {
      dim3 gl((unsigned)std::max(1, std::min(64, (t->leaf_max * 32 + 255) / 256)), 1 << D);
      const size_t xsm = sizeof(float2) * t->leaf_max;
      KF_CUDA(c, cudaFuncSetAttribute(k_leaf_mv_df<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm));
      KF_PHASE(KF_PH_MV_LEAF, s, k_leaf_mv_df<1><<<gl, 256, xsm, s>>>(t->d_lo, t->d_hi, leaf0, t->leaf_max, f->Kdf,
                                                                     f->lambda, x, xdf, y, (int)k, 0));
    } else {  // eight right-hand sides per pass over the leaf blocks, 8 CTAs of 16 warps a leaf
      dim3 gl((unsigned)std::max(1, std::min(8, (t->leaf_max * 32 + 511) / 512)), 1 << D);
      const size_t xsm = sizeof(float2) * t->leaf_max * 8;
      KF_CUDA(c, cudaFuncSetAttribute(k_leaf_mv_df<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm));
      for (int r = 0; r < k; r += 8)
        KF_PHASE(KF_PH_MV_LEAF, s, k_leaf_mv_df<8><<<gl, 512, xsm, s>>>(t->d_lo, t->d_hi, leaf0, t->leaf_max, f->Kdf,
                                                                       f->lambda, x, xdf, y, (int)k, r));
    }
  } else {
    dim3 gl((t->leaf_max + 127) / 128, 1 << D);
    KF_PHASE(KF_PH_MV_LEAF, s, k_leaf_mv<TM><<<gl, 128, 0, s>>>(t->d_lo, t->d_hi, leaf0, t->X64, t->X32, t->d, f->c_exp, inv_h3,
                                     deriv ? SRC_DKERNEL : SRC_KERNEL, f->lambda, x, y, (int)k));
  }
  if (oz.xsl && (D == 0 || transpose || !f->VTsl)) kf_oz_release_x(f, &oz, s);  // only the leaf pass used them
  if (D == 0) { KF_LAUNCH_CHECK(c); return KF_OK; }
  KF_CUDA(c, cudaMemsetAsync(G, 0, sizeof(double) * (size_t)(t->nnodes + 1) * s_max * k, s));
  if (transpose) {
    // g[leaf] = P_leaf^T x, then up the tree, then y_c += K_{c sib~} g[sib] on every level
    const int64_t lrows = (N >> D) + 1;
    dim3 gcl((unsigned)((lrows + kRowsPerChunk - 1) / kRowsPerChunk), 1 << D);
    launch_colsum<double, double>(gcl, s, t->d_lo, t->d_hi, f->rank, f->skel, leaf0, s_max, 0, SRC_STORED, f->Pleaf,
                                  t->X64, t->X32, t->d, f->c_exp, inv_h3, x, (int)k, G, parts, parts2,
                                  KF_PH_MV_ROWUPD);
    for (int l = D - 1; l >= 1; --l) {
      if (k >= 2)
        KF_PHASE(KF_PH_MV_PUSH, s, k_push_up_multi<double><<<dim3(1u << l, (unsigned)((s_max + 31) / 32),
                                                                  (unsigned)((k + 63) / 64)), 256, 0, s>>>(
                                       f->rank, 1 << l, s_max, f->Pc, G, G, (int)k));
      else
        KF_PHASE(KF_PH_MV_PUSH, s, k_push_up<double><<<dim3(1u << l, (unsigned)((s_max + 31) / 32)), 256, 0, s>>>(
                                       f->rank, 1 << l, s_max, f->Pc, G, G, (int)k));
    }
    if (f->VTdf && k >= 2)
      KF_CUDA(c, cudaFuncSetAttribute(k_rows_df<8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)rows_df_smem<8>()));
    for (int l = 1; l <= D; ++l) {
      const int64_t rows = (N >> l) + 1;
      if (f->VTdf && k >= 2) {  // several right-hand sides: double-float row passes
        KF_PHASE(KF_PH_MV_COLSUM, s, k_rows_df<8, 2><<<dim3((unsigned)((rows + kRowUpdRows - 1) / kRowUpdRows),
                                                            1u << l), 256, rows_df_smem<8>(), s>>>(
                                         t->d_lo, t->d_hi, f->rank, 1 << l, s_max,
                                         f->VTdf + (int64_t)(l - 1) * N * s_max, G, y, (int)k));
      } else if (f->VTdf) {
        dim3 g((unsigned)((rows + kRowUpdRows - 1) / kRowUpdRows), 1 << l);
        KF_PHASE(KF_PH_MV_COLSUM, s, k_rowupd_df<<<g, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, 1 << l, s_max,
                                                                     f->VTdf + (int64_t)(l - 1) * N * s_max, G,
                                                                     (int)k, y));
      } else {
        launch_rowupd<TM, double>(rows, 1 << l, s, t->d_lo, t->d_hi, f->rank, f->skel, 1 << l, s_max, 1, src,
                                  vt_level(l), t->X64, t->X32, t->d, f->c_exp, inv_h3, G, 1.0, y, (int)k,
                                  KF_PH_MV_COLSUM);
      }
    }
    KF_LAUNCH_CHECK(c);
    return KF_OK;
  }
  // sibling couplings inside the frontier subtrees of the hybrid solver
  // (levels below its frontier), or at every level of the direct solver
  for (int l = f->hyb_L + 1; l <= D; ++l) {
    const int64_t rows = (N >> l) + 1;
    dim3 gc((unsigned)((rows + kRowsPerChunk - 1) / kRowsPerChunk), 1 << l);
    if (oz.xsl && f->VTsl) {
      int nch = 0;
      kf_status zs = kf_oz_colsum_level(f, l, oz, k, parts, &nch, s);
      if (zs != KF_OK) {
        kf_oz_release_x(f, &oz, s);
        return zs;
      }
      colsum_reduce(dim3((unsigned)nch, 1u << l), s, t->d_lo, t->d_hi, f->rank, 1 << l, 1, kOzChunkRows, s_max,
                    (int)k, parts, parts2, G, KF_PH_MV_COLSUM);
    } else if (f->VTdf && !deriv) {  // FP64-accurate operator of the mixed path
      const float2* Vl = f->VTdf + (int64_t)(l - 1) * N * s_max;
      // several right-hand sides: 256 rows a CTA (16 columns a pass for k > 8)
      const dim3 g2((gc.x + 1) / 2, gc.y);
      if (k == 1)
        KF_PHASE(KF_PH_MV_COLSUM, s, k_colsum_df<1><<<gc, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, 1 << l, s_max, Vl, xdf,
                                                                        (int)k, parts));
      else if (k <= 4)
        KF_PHASE(KF_PH_MV_COLSUM, s, k_colsum_df<4, 256><<<g2, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, 1 << l, s_max,
                                                                             Vl, xdf, (int)k, parts));
      else if (k <= 8)
        KF_PHASE(KF_PH_MV_COLSUM, s, k_colsum_df<8, 256><<<g2, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, 1 << l, s_max,
                                                                             Vl, xdf, (int)k, parts));
      else
        KF_PHASE(KF_PH_MV_COLSUM, s, k_colsum_df<16, 256><<<g2, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, 1 << l, s_max,
                                                                              Vl, xdf, (int)k, parts));
      if (k == 1)
        colsum_reduce(gc, s, t->d_lo, t->d_hi, f->rank, 1 << l, 1, kRowsPerChunk, s_max, (int)k, parts, parts2, G,
                      KF_PH_MV_COLSUM);
      else
        colsum_reduce(g2, s, t->d_lo, t->d_hi, f->rank, 1 << l, 1, 256, s_max, (int)k, parts, parts2, G,
                      KF_PH_MV_COLSUM);
    } else
      launch_colsum<TM, double>(gc, s, t->d_lo, t->d_hi, f->rank, f->skel, 1 << l, s_max, 1, src, vt_level(l),
                                t->X64, t->X32, t->d, f->c_exp, inv_h3, x, (int)k, G, parts, parts2, KF_PH_MV_COLSUM);
  }
  if (oz.xsl) kf_oz_release_x(f, &oz, s);
  // the hybrid solver's frontier nodes couple with every other frontier node
  // (V of Algorithm 8), pushed down from the frontier like a sibling coupling
  if (f->hyb_L > 0) {
    kf_status hs = kf_hybrid_top_apply(f, x, G, k, s);
    if (hs != KF_OK) return hs;
  }
  const dim3 gpd(1, (unsigned)((2 * s_max + 31) / 32));
  // several right-hand sides on the FP64-accurate operator: double-float passes over P_c and P
  const bool rows_df = f->VTdf && f->Pcdf && f->Pleafdf && !deriv && k >= 2;
  if (rows_df) {
    KF_CUDA(c, cudaFuncSetAttribute(k_rows_df<8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)rows_df_smem<8>()));
    KF_CUDA(c, cudaFuncSetAttribute(k_rows_df<8, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)rows_df_smem<8>()));
  }
  const bool oz_push = f->PCsl && f->VTsl && !deriv && k >= 16 && k <= 4096;
  for (int l = std::max(1, f->hyb_L); l < D; ++l) {
    if (oz_push) {  // g_children += P_c g_a on the tensor cores (digits of g_a formed per level)
      kf_oz_x td;
      kf_status zs = kf_oz_prepare_t(f, l, G, k, &td, s);
      if (zs == KF_OK) zs = kf_oz_push(f, l, td, k, G, s);
      kf_oz_release_x(f, &td, s);
      if (zs != KF_OK) return zs;
    } else if (rows_df)
      KF_PHASE(KF_PH_MV_PUSH, s, k_rows_df<8, 1><<<dim3((unsigned)((2 * s_max + kRowUpdRows - 1) / kRowUpdRows),
                                                          1u << l), 256, rows_df_smem<8>(), s>>>(
                                     t->d_lo, t->d_hi, f->rank, 1 << l, s_max, f->Pcdf, G, G, (int)k));
    else if (k >= 2)
      KF_PHASE(KF_PH_MV_PUSH, s, k_push_down_multi<double><<<dim3(1u << l, gpd.y, (unsigned)((k + 63) / 64)), 256, 0, s>>>(
                                     f->rank, 1 << l, s_max, f->Pc, G, G, (int)k));
    else
      KF_PHASE(KF_PH_MV_PUSH, s, k_push_down<double><<<dim3(1u << l, gpd.y), 256, 0, s>>>(f->rank, 1 << l, s_max, f->Pc, G,
                                                                                          G, (int)k));
  }
  const int64_t rows = (N >> D) + 1;
  if (f->PLsl && f->VTsl && !deriv && k >= 16 && k <= 4096) {  // y += P g of the leaves on the tensor cores
    kf_oz_x td;
    kf_status zs = kf_oz_prepare_t(f, D, G, k, &td, s);
    if (zs == KF_OK) zs = kf_oz_rowupd(f, td, k, y, 1.0, s);
    kf_oz_release_x(f, &td, s);
    if (zs != KF_OK) return zs;
  } else if (rows_df)
    KF_PHASE(KF_PH_MV_ROWUPD, s, k_rows_df<8, 0><<<dim3((unsigned)((rows + kRowUpdRows - 1) / kRowUpdRows),
                                                           1u << D), 256, rows_df_smem<8>(), s>>>(
                                     t->d_lo, t->d_hi, f->rank, leaf0, s_max, f->Pleafdf, G, y, (int)k));
  else
    launch_rowupd<double, double>(rows, 1 << D, s, t->d_lo, t->d_hi, f->rank, f->skel, leaf0, s_max, 0, SRC_STORED,
                                  f->Pleaf, t->X64, t->X32, t->d, f->c_exp, inv_h3, G, 1.0, y, (int)k,
                                  KF_PH_MV_ROWUPD);
  KF_LAUNCH_CHECK(c);
  return KF_OK;
}

}  // namespace

// Scratch of the deterministic column sums: the partial sums of a launch
// (parts) and of its chunk groups (parts2), bounded over the launches of one
// sweep or operator product with chunks of at least `rows` rows.
struct ColsumScratch {
  double* parts = nullptr;
  double* parts2 = nullptr;
  size_t pb = 0, pb2 = 0;
  kf_ctx* c = nullptr;
  cudaStream_t s = nullptr;
  bool alloc(kf_ctx* ctx, const kf_factor* f, int64_t k, int rows, cudaStream_t st) {
    c = ctx;
    s = st;
    pb = sizeof(double) * colsum_parts_bound(f->t->N, f->t->D, f->s_max, k, rows);
    pb2 = sizeof(double) * colsum_parts_bound(f->t->N, f->t->D, f->s_max, k, rows * kColsumGroup);
    parts = (double*)c->dalloc(pb, s);
    parts2 = (double*)c->dalloc(pb2, s);
    return parts && parts2;
  }
  ~ColsumScratch() {
    if (parts) c->dfree(parts, pb, s);
    if (parts2) c->dfree(parts2, pb2, s);
  }
};

// W: N x k FP64 in tree order; solved in place.  The mixed path runs the sweep
// on an FP32 copy.
kf_status kf_solve_device(kf_factor* f, double* W, int64_t k, int transpose, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  const int64_t N = f->t->N;
  const size_t ub = sizeof(double) * (size_t)(f->t->nnodes + 1) * f->s_max * k;
  double* U = (double*)c->dalloc(ub, s);
  double* Vb = (double*)c->dalloc(ub, s);
  if (!U || !Vb) {
    c->dfree(U, ub, s);
    c->dfree(Vb, ub, s);
    return kf_set_err(c, KF_ENOMEM, "solve: allocation failed");
  }
  kf_status st;
  if (f->hyb_L > 0 && transpose) {
    c->dfree(U, ub, s);
    c->dfree(Vb, ub, s);
    return kf_set_err(c, KF_EUNSUPPORTED, "transpose solves of the hybrid solver are not supported");
  }
  ColsumScratch cs;
  if (!cs.alloc(c, f, k, k == 1 ? kRowsPerChunk : 512, s)) {
    c->dfree(U, ub, s);
    c->dfree(Vb, ub, s);
    return kf_set_err(c, KF_ENOMEM, "solve: allocation failed");
  }
  if (f->prec == KF_PREC_FP64) {
    st = solve_t<double, double>(f, W, k, transpose, U, Vb, cs.parts, cs.parts2, s);
  } else {
    float* W32 = (float*)c->dalloc(sizeof(float) * N * k, s);
    if (!W32) {
      st = kf_set_err(c, KF_ENOMEM, "solve: allocation failed");
    } else {
      KF_PHASE(KF_PH_MISC, s, k_axpy_cast<float><<<grid_for(N * k, 256), 256, 0, s>>>(W, W32, N * k));
      st = solve_t<float, float>(f, W32, k, transpose, U, Vb, cs.parts, cs.parts2, s);
      KF_PHASE(KF_PH_MISC, s, k_cast_back<float><<<grid_for(N * k, 256), 256, 0, s>>>(W32, W, N * k));
      c->dfree(W32, sizeof(float) * N * k, s);
    }
  }
  c->dfree(U, ub, s);
  c->dfree(Vb, ub, s);
  // Algorithm 6 above the frontier: w = D^-1 u - W (I + V W)^-1 V D^-1 u
  if (st == KF_OK && f->hyb_L > 0) st = kf_hybrid_top_solve(f, W, k, s);
  return st;
}

static kf_status matvec_any(kf_factor* f, const double* x, double* y, int64_t k, int deriv, int transpose,
                            cudaStream_t s) {
  kf_ctx* c = f->ctx;
  if (f->hyb_L > 0 && (deriv || transpose))
    return kf_set_err(c, KF_EUNSUPPORTED, "the hybrid solver's operator has no transpose or h-derivative here");
  const size_t gb = sizeof(double) * (size_t)(f->t->nnodes + 1) * f->s_max * k;
  double* G = (double*)c->dalloc(gb, s);
  if (!G) return kf_set_err(c, KF_ENOMEM, "matvec: allocation failed");
  // x as double-float pairs for the FP64-accurate operator's leaf and V passes
  const size_t xb = f->Kdf && !deriv ? sizeof(float2) * (size_t)f->t->N * k : 0;
  float2* xdf = xb ? (float2*)c->dalloc(xb, s) : nullptr;
  if (xb && !xdf) {
    c->dfree(G, gb, s);
    return kf_set_err(c, KF_ENOMEM, "matvec: allocation failed");
  }
  // dK~/dh (deriv) is evaluated from the FP64 coordinates on both paths: the
  // gradient's -a^T (dK~/dh) x cancels heavily (the sum of |terms| is often
  // 10^3-10^4 times the result), so FP32 entries would leave it at ~1e-4
  ColsumScratch cs;
  if (!cs.alloc(c, f, k, k == 1 ? kRowsPerChunk : 256, s)) {
    if (xdf) c->dfree(xdf, xb, s);
    c->dfree(G, gb, s);
    return kf_set_err(c, KF_ENOMEM, "matvec: allocation failed");
  }
  kf_status st = (f->prec == KF_PREC_FP64 || deriv)
                     ? matvec_t<double>(f, x, y, k, deriv, transpose, G, xdf, cs.parts, cs.parts2, s)
                     : matvec_t<float>(f, x, y, k, deriv, transpose, G, xdf, cs.parts, cs.parts2, s);
  if (xdf) c->dfree(xdf, xb, s);
  c->dfree(G, gb, s);
  return st;
}

kf_status kf_matvec_device(kf_factor* f, const double* x, double* y, int64_t k, int deriv, cudaStream_t s) {
  return matvec_any(f, x, y, k, deriv, 0, s);
}

kf_status kf_matvec_transpose_device(kf_factor* f, const double* x, double* y, int64_t k, cudaStream_t s) {
  return matvec_any(f, x, y, k, 0, 1, s);
}

// Solve with one reduced system stored as node 1 of a two-node array (see
// kf_z_factor_one_launch): in/out hold its S entries contiguously at
// (2 ldz + i) * k + c, the layout k_zsolve reads for a node whose first
// child has rank S at a row stride of ldz.
kf_status kf_zsolve_one_launch(const int32_t* rank, int ldz, const double* ZLU, const int32_t* piv, const double* in,
                               double* out, int k, cudaStream_t s) {
  if (ldz < 1 || ldz > 2 * KF_MAX_SMAX) return KF_EINVAL;
  const size_t zs_smem = sizeof(double) * (2 * (size_t)ldz + (ldz + 1) / 2 + 8 * 32 * 33);
  if (cudaFuncSetAttribute(k_zsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zs_smem) != cudaSuccess)
    return KF_ECUDA;
  KF_PHASE(KF_PH_HYBRID, s, k_zsolve<<<dim3(1, (unsigned)std::min(k, 16)), 256, zs_smem, s>>>(rank, 1, ldz, ldz, ZLU,
                                                                                              piv, in, out, k, 0));
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ECUDA;
}

kf_status kf_rowupd_level_launch(kf_factor* f, int l, const double* V, double* W, int64_t k, cudaStream_t s) {
  kf_tree* t = f->t;
  const int64_t N = t->N;
  const int64_t rows = (N >> l) + 1;
  const double inv_h3 = 1.0 / (f->h * f->h * f->h);
  const int64_t off = (int64_t)(l - 1) * N * f->s_max;
  if (f->prec == KF_PREC_FP64)
    launch_rowupd<double, double>(rows, 1 << l, s, t->d_lo, t->d_hi, f->rank, f->skel, 1 << l, f->s_max, 0,
                                  SRC_STORED, (const double*)f->Phat + off, t->X64, t->X32, t->d, f->c_exp, inv_h3, V,
                                  -1.0, W, (int)k, KF_PH_HYBRID);
  else
    launch_rowupd<float, double>(rows, 1 << l, s, t->d_lo, t->d_hi, f->rank, f->skel, 1 << l, f->s_max, 0,
                                 SRC_STORED, (const float*)f->Phat + off, t->X64, t->X32, t->d, f->c_exp, inv_h3, V,
                                 -1.0, W, (int)k, KF_PH_HYBRID);
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ECUDA;
}
