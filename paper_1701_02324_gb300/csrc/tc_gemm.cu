// tc_gemm.cu -- 5th-generation tensor-core (tcgen05) products of the mixed
// path: the off-diagonal blocks of the reduced systems, K_{l~ r} P^_r and
// K_{r~ l} P^_l (Eq. e:blocksmw), and the telescoping P^_a = [P^_l T_top;
// P^_r T_bot] (Eq. e:invtelescope).
//
// One CTA (16 warps) computes a 128 x BN tile of D = A B:
//   * operands are staged by all threads from global memory into shared
//     memory in the canonical K-major, no-swizzle core-matrix layout (8 rows x
//     16 bytes per core matrix; LBO = 128 B between core matrices along K,
//     SBO = 1024 B between 8-row groups), split into tf32 hi and lo parts;
//   * one thread issues tcgen05.mma kind::tf32 for A_hi B_hi + A_hi B_lo +
//     A_lo B_hi (3xTF32, about 2^-22 relative) into an FP32 accumulator in
//     tensor memory -- or, for problems with three operand pieces, the six
//     products that reach the FP32 rounding level -- and tcgen05.commit
//     arrives on an mbarrier;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w reads lane
//     quadrant w mod 4, rows 32(w mod 4)..+31, and a quarter of the columns)
//     and hands each value to the problem's store.
// Every wait is bounded; on time-out the kernel flags KF_DEV_TIMEOUT, waits
// once more, frees its tensor memory and returns.
#include <algorithm>

#include "kf_internal.cuh"
#include "prof.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace kf_tc;

constexpr int kBM = 128;  // rows per tile (tcgen05 M for cta_group::1)
constexpr int kBK = 32;   // K elements staged per round (4 MMAs of K = 8)

// Test hook of the time-out path (kf_test_tc_wait_probe): when positive, each
// CTA of k_tc_gemm first polls an mbarrier that nothing arrives at, at most
// this many times, and on giving up takes the path of a wait that ran out:
// it flags KF_DEV_TIMEOUT, issues no MMA, stores nothing, frees its tensor
// memory and returns.  Zero (no probe) in normal use.
__device__ long long g_tc_probe_polls = 0;


// element (r, k) of a tile with 32 K-elements per row, in floats
__device__ __forceinline__ int core_off(int r, int k) { return (r >> 3) * 256 + (k >> 2) * 32 + (r & 7) * 4 + (k & 3); }

struct Tile {
  int m0, n0, k0, k1, M, N;  // tile origin, K range, valid extents (absolute indices)
  int node, side, base;      // problem-specific
  int tl, ks;                // split-K products: output tile index and part of K
  bool skip;
};

// Generic tile driver.  Problem provides: tile(bx, by, bz) -> Tile;
// loadA(tile, m, k) and loadB(tile, k, n) (valid indices only; FP32);
// a_m_fastest / b_n_fastest (staging order for coalescing); store(tile, m, n, v).
// Two shared-memory stages: the threads stage chunk c + 1 (global loads and
// the tf32 split) while the tensor core works on chunk c; an mbarrier per
// stage, armed by tcgen05.commit, says when a stage may be overwritten.
constexpr int kThreads = 512;  // 16 warps: all stage operands, 4 per TMEM lane quadrant in the epilogue

// Element e of a (rows x 32) operand tile.  32 consecutive e fill one
// 8-row x 4-k slice of a core matrix, i.e. 32 consecutive shared-memory words
// (no bank conflicts); inside the slice the row index runs fastest when the
// operand is contiguous along rows in global memory, else the k index.
template <bool kRowsFastest>
__device__ __forceinline__ void tile_coord(int e, int rows, int& r, int& k) {
  const int g = e >> 5;
  const int rl = kRowsFastest ? (e & 7) : ((e >> 2) & 7);
  const int kl = kRowsFastest ? ((e >> 3) & 3) : (e & 3);
  const int rg = rows >> 3;
  r = (g % rg) * 8 + rl;
  k = (g / rg) * 4 + kl;
}

// Operand pieces: Problem::kPieces = 2 splits every value into tf32 hi + lo
// (3 MMAs per product: hi hi + hi lo + lo hi, about 2^-22 relative); 3 splits
// it into hi + mid + lo (6 MMAs: hi hi + hi mid + mid hi + hi lo + lo hi +
// mid mid, the FP32 rounding level) for the products whose errors the
// factorization amplifies most (the leaves).  A stage holds the pieces of A
// then those of B, each kBM x kBK (A) or BN x kBK (B) floats.
template <class Problem, int BN>
__device__ __forceinline__ void stage_chunk(const Problem& prob, const Tile& t, int kc, float* As, float* Bs) {
  constexpr int P = Problem::kPieces;
  const int tid = threadIdx.x;
  const int kn = min(kBK, t.k1 - kc);
  // all global loads of the chunk first (in flight together), then the split
  constexpr int NA = kBM * kBK / kThreads, NB = BN * kBK / kThreads;
  float va[NA], vb[NB];
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    int m, k;
    tile_coord<Problem::a_m_fastest>(tid + q * kThreads, kBM, m, k);
    va[q] = (m < t.M - t.m0 && k < kn) ? prob.loadA(t, t.m0 + m, kc + k) : 0.f;
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    int n, k;
    tile_coord<Problem::b_n_fastest>(tid + q * kThreads, BN, n, k);
    vb[q] = (n < t.N - t.n0 && k < kn) ? prob.loadB(t, kc + k, t.n0 + n) : 0.f;
  }
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    int m, k;
    tile_coord<Problem::a_m_fastest>(tid + q * kThreads, kBM, m, k);
    const int o = core_off(m, k);
    const float hi = to_tf32(va[q]), r1 = va[q] - hi;  // r1 exact
    if (P == 2) {
      As[o] = hi;
      As[kBM * kBK + o] = to_tf32(r1);
    } else {
      const float mid = to_tf32(r1);
      As[o] = hi;
      As[kBM * kBK + o] = mid;
      As[2 * kBM * kBK + o] = to_tf32(r1 - mid);
    }
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    int n, k;
    tile_coord<Problem::b_n_fastest>(tid + q * kThreads, BN, n, k);
    const int o = core_off(n, k);
    const float hi = to_tf32(vb[q]), r1 = vb[q] - hi;
    if (P == 2) {
      Bs[o] = hi;
      Bs[BN * kBK + o] = to_tf32(r1);
    } else {
      const float mid = to_tf32(r1);
      Bs[o] = hi;
      Bs[BN * kBK + o] = mid;
      Bs[2 * BN * kBK + o] = to_tf32(r1 - mid);
    }
  }
}

template <int P, int BN>
__device__ __forceinline__ void issue_chunk(uint32_t tmem, uint32_t as, uint32_t bs, uint32_t idesc, bool first) {
  constexpr uint32_t sa = kBM * kBK * 4, sb = BN * kBK * 4;  // bytes between pieces
#pragma unroll
  for (int kk = 0; kk < kBK / 8; ++kk) {
    const uint32_t off = kk * 256;  // two core matrices along K per MMA (K = 8 tf32)
    const uint64_t a0 = smem_desc(as + off, 128, 1024), a1 = smem_desc(as + sa + off, 128, 1024);
    const uint64_t b0 = smem_desc(bs + off, 128, 1024), b1 = smem_desc(bs + sb + off, 128, 1024);
    mma_tf32(tmem, a0, b0, idesc, (first && kk == 0) ? 0u : 1u);
    mma_tf32(tmem, a0, b1, idesc, 1u);
    mma_tf32(tmem, a1, b0, idesc, 1u);
    if (P == 3) {
      const uint64_t a2 = smem_desc(as + 2 * sa + off, 128, 1024), b2 = smem_desc(bs + 2 * sb + off, 128, 1024);
      mma_tf32(tmem, a0, b2, idesc, 1u);
      mma_tf32(tmem, a2, b0, idesc, 1u);
      mma_tf32(tmem, a1, b1, idesc, 1u);
    }
  }
}

template <int BN, class Problem>
__global__ void __launch_bounds__(kThreads) k_tc_gemm(Problem prob, int32_t* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int P = Problem::kPieces;
  constexpr int kStage = P * kBM * kBK + P * BN * kBK;  // floats per stage
  __shared__ __align__(8) uint64_t mbar[3];  // two stages; [2] only for the time-out probe
  __shared__ uint32_t tmem_base;
  __shared__ int probe_timed_out;
  const Tile t = prob.tile(blockIdx.x, blockIdx.y, blockIdx.z);
  if (t.skip) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_base, BN);
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_init(&mbar[2], 1);
    probe_timed_out = 0;
    const long long polls = g_tc_probe_polls;
    if (polls > 0) {
      bool arrived = false;
      for (long long i = 0; i < polls && !arrived; ++i) arrived = mbar_try_wait(&mbar[2], 0u);
      if (!arrived) {
        probe_timed_out = 1;
        atomicOr(status, KF_DEV_TIMEOUT);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_tf32(kBM, BN);
  uint32_t uses[2] = {0u, 0u};  // commits issued per stage
  bool ok = probe_timed_out == 0;
  int c = 0;
  for (int kc = t.k0; kc < t.k1 && ok; kc += kBK, ++c) {
    const int st = c & 1;
    float* As = (float*)smem_raw + st * kStage;
    float* Bs = As + P * kBM * kBK;
    if (uses[st] > 0) {  // the MMAs that read this stage two chunks ago must be done
      if (!mbar_wait(&mbar[st], (uses[st] - 1) & 1u)) {
        ok = false;
        if (tid == 0) atomicOr(status, KF_DEV_TIMEOUT);
        break;
      }
    }
    stage_chunk<Problem, BN>(prob, t, kc, As, Bs);
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      issue_chunk<P, BN>(tmem, smem_u32(As), smem_u32(Bs), idesc, kc == t.k0);
      mma_commit(&mbar[st]);
    }
    ++uses[st];
  }
  // drain: wait for the last commit of each stage (a second bounded wait on time-out)
  for (int st = 0; st < 2; ++st)
    if (uses[st] > 0 && !mbar_wait(&mbar[st], (uses[st] - 1) & 1u)) {
      ok = false;
      if (tid == 0) atomicOr(status, KF_DEV_TIMEOUT);
      mbar_wait(&mbar[st], (uses[st] - 1) & 1u);
    }
  fence_after_sync();
  __syncthreads();
  if (ok) {
    // accumulator -> shared memory (the operand stages are idle now), then
    // stored row by row so that a warp's stores are contiguous.  Warp w reads
    // TMEM lane quadrant w % 4 (rows 32(w % 4) + lane); the four warps of a
    // quadrant split the columns.  Row stride BN + 1 words: conflict-free.
    float* Cs = (float*)smem_raw;
    const int quad = warp & 3, part = warp >> 2, nparts = kThreads / 128;
#pragma unroll 1
    for (int c0 = part * 32; c0 < BN; c0 += 32 * nparts) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
      float* row = Cs + (size_t)(quad * 32 + lane) * (BN + 1) + c0;
#pragma unroll
      for (int j = 0; j < 32; ++j) row[j] = v[j];
    }
    __syncthreads();
    const int nrow = min(kBM, t.M - t.m0), ncol = min(BN, t.N - t.n0);
    for (int r = warp; r < nrow; r += kThreads / 32) {
      const float* row = Cs + (size_t)r * (BN + 1);
      for (int cidx = lane; cidx < ncol; cidx += 32) prob.store(t, t.m0 + r, t.n0 + cidx, row[cidx]);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
}

// ---- Z off-diagonal blocks: Z[blk] += VT_c[:, :s_a]^T P^_c[:, :s_b] -------------
// side 0: rows of r, block Z[0:s_l, s_l:] = K_{l~ r} P^_r
// side 1: rows of l, block Z[s_l:, 0:s_l] = K_{r~ l} P^_l
// The long reduction over the child's rows is split over blockIdx.y; partial
// tiles are added into the FP64 Z with atomics.
// Split over K (ksplit > 1): each CTA writes its FP32 partial tile to
// parts[tile][ks] and k_zoff_reduce adds the ksplit partials of an entry in
// the order ks = 0, 1, .. into Z, so that Z does not depend on the order in
// which the CTAs run; with ksplit = 1 a CTA adds its tile into Z directly
// (one writer per entry).
struct ZoffProblem {
  static constexpr int kPieces = 2;
  static constexpr bool a_m_fastest = true;   // VT rows are contiguous in m
  static constexpr bool b_n_fastest = true;   // P^ rows are contiguous in n
  const int32_t* lo;
  const int32_t* hi;
  const int32_t* rank;
  int node0, s_max, ldz, ksplit, ntile_n, tile_n;
  const float* VT;
  const float* Ph;
  double* Z;
  float* parts;
  __device__ Tile tile(int bx, int by, int bz) const {
    Tile t;
    t.side = bz & 1;
    t.node = node0 + (bz >> 1);
    const int l = 2 * t.node, r = l + 1, sl = rank[l], sr = rank[r];
    const int c = t.side == 0 ? r : l;
    t.M = t.side == 0 ? sl : sr;
    t.N = t.side == 0 ? sr : sl;
    t.base = sl;
    t.m0 = (bx / ntile_n) * kBM;
    t.n0 = (bx % ntile_n) * tile_n;
    t.tl = bz * ((s_max + kBM - 1) / kBM) * ntile_n + bx;
    t.ks = by;
    const int rb = lo[c], rn = hi[c] - rb;
    const int chunk = ((rn + ksplit - 1) / ksplit + kBK - 1) / kBK * kBK;
    t.k0 = rb + by * chunk;
    t.k1 = min(hi[c], t.k0 + chunk);
    t.skip = t.M == 0 || t.N == 0 || t.m0 >= t.M || t.n0 >= t.N || t.k0 >= t.k1;
    return t;
  }
  __device__ float loadA(const Tile&, int m, int k) const { return VT[(int64_t)k * s_max + m]; }
  __device__ float loadB(const Tile&, int k, int n) const { return Ph[(int64_t)k * s_max + n]; }
  __device__ void store(const Tile& t, int m, int n, float v) const {
    if (ksplit > 1) {
      parts[((int64_t)(t.tl * ksplit + t.ks) * kBM + (m - t.m0)) * tile_n + (n - t.n0)] = v;
      return;
    }
    const int roff = t.side == 0 ? 0 : t.base, coff = t.side == 0 ? t.base : 0;
    Z[(int64_t)t.node * ldz * ldz + (int64_t)(roff + m) * ldz + coff + n] += (double)v;
  }
};

// Z blocks += the ksplit partial tiles of each entry, added in ks order
// (FP64 sums of the FP32 partials).  grid = (tiles of a block, 2 x nodes), the
// tile numbering of ZoffProblem::tile.
__global__ void __launch_bounds__(256) k_zoff_reduce(const int32_t* __restrict__ rank, int node0, int s_max, int ldz,
                                                     int ksplit, int ntile_n, int tile_n,
                                                     const float* __restrict__ parts, double* __restrict__ Z) {
  const int bx = blockIdx.x, bz = blockIdx.y, side = bz & 1, node = node0 + (bz >> 1);
  const int sl = rank[2 * node], sr = rank[2 * node + 1];
  const int M = side == 0 ? sl : sr, N = side == 0 ? sr : sl;
  const int m0 = (bx / ntile_n) * kBM, n0 = (bx % ntile_n) * tile_n;
  if (m0 >= M || n0 >= N) return;
  const int roff = side == 0 ? 0 : sl, coff = side == 0 ? sl : 0;
  const int64_t tl = (int64_t)bz * gridDim.x + bx;
  double* Zb = Z + (int64_t)node * ldz * ldz;
  for (int e = threadIdx.x; e < kBM * tile_n; e += blockDim.x) {
    const int mi = e / tile_n, ni = e % tile_n;
    if (m0 + mi >= M || n0 + ni >= N) continue;
    double sum = 0.0;
    for (int ks = 0; ks < ksplit; ++ks) sum += (double)parts[((tl * ksplit + ks) * kBM + mi) * tile_n + ni];
    Zb[(int64_t)(roff + m0 + mi) * ldz + coff + n0 + ni] += sum;
  }
}

// ---- Z off-diagonal blocks with the kernel entries evaluated in the product ----------
// The same blocks as ZoffProblem, K_{l~ r} P^_r and K_{r~ l} P^_l, but the A
// operand K(x_{sib~ m}, x_k) is evaluated while the operand is staged (FP32
// squared distance of the FP32 coordinates, sequential fused multiply-adds,
// then exp), as kernel summation fuses the kernel evaluation into the product
// with the weights (Sec. II-D): the V blocks are neither read nor needed
// before the reduced systems.
struct ZoffFusedProblem : ZoffProblem {
  const float* X32;
  const int32_t* skel;
  int d;
  float c_exp;
  __device__ float loadA(const Tile& t, int m, int k) const {
    const int sib = t.side == 0 ? 2 * t.node : 2 * t.node + 1;  // the skeleton's node
    const float* xs = X32 + (int64_t)skel[(int64_t)sib * s_max + m] * d;
    const float* xk = X32 + (int64_t)k * d;
    float acc = 0.f;
    for (int q = 0; q < d; ++q) {
      const float u = __fsub_rn(xs[q], xk[q]);
      acc = __fmaf_rn(u, u, acc);
    }
    return __expf(acc * c_exp);
  }
};

// ---- telescoping: P^_a[rows of c, :s_a] = P^_c[:, :s_c] T[c block, :s_a] ---------
struct TelescopeProblem {
  static constexpr int kPieces = 2;
  static constexpr bool a_m_fastest = false;  // P^_c rows are contiguous in k
  static constexpr bool b_n_fastest = true;   // T rows are contiguous in n
  const int32_t* lo;
  const int32_t* hi;
  const int32_t* rank;
  int node0, s_max, ldz, ntile_n, tile_n;
  const float* Pc_hat;
  const float* Tm;  // T = Z^-1 P_c, FP32 copy
  float* Pa_hat;
  __device__ Tile tile(int bx, int by, int bz) const {
    Tile t;
    t.side = bz & 1;
    t.node = node0 + (bz >> 1);
    t.base = bz >> 1;  // node-local index into T
    const int c = 2 * t.node + t.side;
    t.M = hi[c];       // absolute row range [lo[c], hi[c])
    t.N = rank[t.node];
    t.m0 = lo[c] + bx * kBM;
    t.n0 = by * tile_n;
    t.k0 = 0;
    t.k1 = rank[c];
    t.skip = t.N == 0 || t.m0 >= t.M || t.n0 >= t.N || t.k1 == 0;
    return t;
  }
  __device__ float loadA(const Tile&, int m, int k) const { return Pc_hat[(int64_t)m * s_max + k]; }
  __device__ float loadB(const Tile& t, int k, int n) const {
    const int koff = t.side == 0 ? 0 : rank[2 * t.node];
    return Tm[(int64_t)t.base * ldz * s_max + (int64_t)(koff + k) * s_max + n];
  }
  __device__ void store(const Tile&, int m, int n, float v) const { Pa_hat[(int64_t)m * s_max + n] = v; }
};

// ---- leaf factorization on the tensor cores (mixed path) --------------------------
// The leaf blocks A = lambda I + K_aa are factorized A = L L^T by 128-column
// panels kb: the panel's diagonal block L11 and its inverse Linv are formed on
// CUDA cores (k_chol_panel, factor.cu); these products do the rest.  Leaf lf's
// matrix is L + lf * ldL^2 (row-major, lower triangle); its panels' inverses
// are Dinv + (lf * npan + kb / 128) * 128^2 (row-major, 128 x 128).
struct LeafPanel {
  static constexpr int kPieces = 3;  // FP32-level products: the leaves' errors are the most amplified
  const int32_t* lo;
  const int32_t* hi;
  int leaf0, ldL, kb, npan;
  float* L;
  const float* Dinv;
  __device__ int size(int lf) const { return hi[leaf0 + lf] - lo[leaf0 + lf]; }
  __device__ float* Lm(int lf) const { return L + (int64_t)lf * ldL * ldL; }
  __device__ const float* Di(int lf) const { return Dinv + ((int64_t)lf * npan + kb / kBM) * kBM * kBM; }
};

// L21 = A21 Linv^T: rows kb + nb .. n - 1 of the panel columns, in place
struct LeafTrsmProblem : LeafPanel {
  static constexpr bool a_m_fastest = false;
  static constexpr bool b_n_fastest = false;
  __device__ Tile tile(int bx, int, int bz) const {
    Tile t;
    t.node = bz;
    const int n = size(bz), nb = min(kBM, n - kb);
    t.base = nb;
    t.M = n - kb - nb;
    t.N = nb;
    t.m0 = bx * kBM;
    t.n0 = 0;
    t.k0 = 0;
    t.k1 = nb;
    t.skip = nb <= 0 || t.M <= 0 || t.m0 >= t.M;
    return t;
  }
  __device__ float loadA(const Tile& t, int m, int k) const {
    return Lm(t.node)[(int64_t)(kb + t.base + m) * ldL + kb + k];
  }
  __device__ float loadB(const Tile& t, int k, int n) const { return Di(t.node)[n * kBM + k]; }
  __device__ void store(const Tile& t, int m, int n, float v) const {
    Lm(t.node)[(int64_t)(kb + t.base + m) * ldL + kb + n] = v;
  }
};

// A22 -= L21 L21^T on the lower triangle (tiles wholly above the diagonal skipped)
struct LeafSyrkProblem : LeafPanel {
  static constexpr bool a_m_fastest = false;
  static constexpr bool b_n_fastest = false;
  int tile_n;
  __device__ Tile tile(int bx, int by, int bz) const {
    Tile t;
    t.node = bz;
    const int n = size(bz), nb = min(kBM, n - kb);
    t.base = nb;
    t.M = t.N = n - kb - nb;
    t.m0 = bx * kBM;
    t.n0 = by * tile_n;
    t.k0 = 0;
    t.k1 = nb;
    t.skip = nb <= 0 || t.M <= 0 || t.m0 >= t.M || t.n0 >= t.N || t.n0 > t.m0 + kBM - 1;
    return t;
  }
  __device__ float loadA(const Tile& t, int m, int k) const {
    return Lm(t.node)[(int64_t)(kb + t.base + m) * ldL + kb + k];
  }
  __device__ float loadB(const Tile& t, int k, int n) const {
    return Lm(t.node)[(int64_t)(kb + t.base + n) * ldL + kb + k];
  }
  __device__ void store(const Tile& t, int m, int n, float v) const {
    if (n <= m) Lm(t.node)[(int64_t)(kb + t.base + m) * ldL + kb + t.base + n] -= v;
  }
};

// P^ = L^-T L^-1 P on Y = the leaf rows of P^ (stride s_max, rank s columns):
// Y_i = Linv_i Y_i (TRANS: Linv_i^T Y_i), in place on the panel's rows
template <bool TRANS>
struct PhatDinvProblem : LeafPanel {
  static constexpr bool a_m_fastest = TRANS;
  static constexpr bool b_n_fastest = true;
  const int32_t* rank;
  int s_max, tile_n;
  float* Y;
  __device__ Tile tile(int, int by, int bz) const {
    Tile t;
    t.node = bz;
    const int n = size(bz), nb = min(kBM, n - kb);
    t.base = lo[leaf0 + bz];
    t.M = nb;
    t.N = rank[leaf0 + bz];
    t.m0 = 0;
    t.n0 = by * tile_n;
    t.k0 = 0;
    t.k1 = nb;
    t.skip = nb <= 0 || t.N <= 0 || t.n0 >= t.N;
    return t;
  }
  __device__ float loadA(const Tile& t, int m, int k) const {
    return TRANS ? Di(t.node)[k * kBM + m] : Di(t.node)[m * kBM + k];
  }
  __device__ float loadB(const Tile& t, int k, int n) const { return Y[(int64_t)(t.base + kb + k) * s_max + n]; }
  __device__ void store(const Tile& t, int m, int n, float v) const { Y[(int64_t)(t.base + kb + m) * s_max + n] = v; }
};

// ABOVE = false: Y[kb+nb+m] -= L[kb+nb+m][kb..kb+nb) Y_i (forward substitution);
// ABOVE = true:  Y[m] -= L[kb..kb+nb)[m]^T Y_i for m < kb (backward)
template <bool ABOVE>
struct PhatUpdateProblem : LeafPanel {
  static constexpr bool a_m_fastest = ABOVE;
  static constexpr bool b_n_fastest = true;
  const int32_t* rank;
  int s_max, tile_n;
  float* Y;
  __device__ Tile tile(int bx, int by, int bz) const {
    Tile t;
    t.node = bz;
    const int n = size(bz), nb = min(kBM, n - kb);
    t.base = lo[leaf0 + bz];
    t.M = ABOVE ? kb : n - kb - nb;
    t.N = rank[leaf0 + bz];
    t.m0 = bx * kBM;
    t.n0 = by * tile_n;
    t.k0 = 0;
    t.k1 = nb;
    t.skip = nb <= 0 || t.M <= 0 || t.N <= 0 || t.m0 >= t.M || t.n0 >= t.N;
    return t;
  }
  __device__ float loadA(const Tile& t, int m, int k) const {
    const int nb = min(kBM, size(t.node) - kb);
    return ABOVE ? Lm(t.node)[(int64_t)(kb + k) * ldL + m] : Lm(t.node)[(int64_t)(kb + nb + m) * ldL + kb + k];
  }
  __device__ float loadB(const Tile& t, int k, int n) const { return Y[(int64_t)(t.base + kb + k) * s_max + n]; }
  __device__ void store(const Tile& t, int m, int n, float v) const {
    const int nb = min(kBM, size(t.node) - kb);
    const int row = ABOVE ? m : kb + nb + m;
    Y[(int64_t)(t.base + row) * s_max + n] -= v;
  }
};

}  // namespace

// ---- launchers ---------------------------------------------------------------------
static size_t tc_smem_bytes(int BN, int pieces = 2) {
  return 2 * sizeof(float) * (size_t)pieces * (kBM * kBK + BN * kBK);
}

template <int BN, class Problem>
static kf_status tc_launch(const Problem& p, dim3 g, int phase, int32_t* status, cudaStream_t s) {
  const size_t smem = tc_smem_bytes(BN, Problem::kPieces);
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<BN, Problem>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return KF_ECUDA;
  KF_PHASE(phase, s, k_tc_gemm<BN, Problem><<<g, kThreads, smem, s>>>(p, status));
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ECUDA;
}

// ksplit of the Z-block products: enough CTAs to fill the GPU, the reduction
// split over the child's rows
static int zoff_ksplit(int64_t tiles, int64_t rows_per_child) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((rows_per_child + 1023) / 1024, (2 * 152 + tiles - 1) / tiles));
}

// the split-K partials, zeroed (a part of K left empty writes nothing), then
// the product, then their sum in ks order
template <int BN, typename Problem>
static kf_status zoff_run(Problem& p, int nn, int mt, float* parts, size_t parts_cap, int32_t* status,
                          cudaStream_t s) {
  const dim3 g(mt * p.ntile_n, p.ksplit, 2 * nn);
  p.parts = parts;
  if (p.ksplit > 1) {
    const size_t pb = sizeof(float) * (size_t)g.x * g.z * p.ksplit * kBM * BN;
    if (!parts || pb > parts_cap) return KF_EINVAL;
    if (cudaMemsetAsync(parts, 0, pb, s) != cudaSuccess) return KF_ECUDA;
  }
  kf_status st = tc_launch<BN>(p, g, KF_PH_ZOFF, status, s);
  if (st != KF_OK || p.ksplit == 1) return st;
  KF_PHASE(KF_PH_ZOFF, s, k_zoff_reduce<<<dim3(g.x, g.z), 256, 0, s>>>(p.rank, p.node0, p.s_max, p.ldz, p.ksplit,
                                                                       p.ntile_n, BN, parts, p.Z));
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ECUDA;
}

template <int BN>
static kf_status tc_zoff_bn(const int32_t* lo, const int32_t* hi, const int32_t* rank, int node0, int nn, int s_max,
                            const float* VT, const float* Ph, int ldz, double* Z, int64_t rows_per_child,
                            float* parts, size_t parts_cap, int32_t* status, cudaStream_t s) {
  ZoffProblem p;
  p.lo = lo; p.hi = hi; p.rank = rank; p.node0 = node0; p.s_max = s_max; p.ldz = ldz;
  p.ntile_n = (s_max + BN - 1) / BN;
  p.tile_n = BN;
  p.VT = VT; p.Ph = Ph; p.Z = Z;
  const int mt = (s_max + kBM - 1) / kBM;
  p.ksplit = zoff_ksplit((int64_t)mt * p.ntile_n * 2 * nn, rows_per_child);
  return zoff_run<BN>(p, nn, mt, parts, parts_cap, status, s);
}

template <int BN>
static kf_status tc_telescope_bn(const int32_t* lo, const int32_t* hi, const int32_t* rank, int node0, int nn,
                                 int s_max, const float* Pc_hat, const float* Tm, int ldz, float* Pa_hat,
                                 int64_t rows_per_child, int32_t* status, cudaStream_t s) {
  TelescopeProblem p;
  p.lo = lo; p.hi = hi; p.rank = rank; p.node0 = node0; p.s_max = s_max; p.ldz = ldz;
  p.ntile_n = (s_max + BN - 1) / BN;
  p.tile_n = BN;
  p.Pc_hat = Pc_hat; p.Tm = Tm; p.Pa_hat = Pa_hat;
  const size_t smem = tc_smem_bytes(BN);
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<BN, TelescopeProblem>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return KF_ECUDA;
  dim3 g((unsigned)((rows_per_child + kBM - 1) / kBM), p.ntile_n, 2 * nn);
  KF_PHASE(KF_PH_TELESCOPE, s, k_tc_gemm<BN, TelescopeProblem><<<g, kThreads, smem, s>>>(p, status));
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ECUDA;
}

template <int BN>
static kf_status tc_zoff_fused_bn(const int32_t* lo, const int32_t* hi, const int32_t* rank, const int32_t* skel,
                                  const float* X32, int d, float c_exp, int node0, int nn, int s_max, const float* Ph,
                                  int ldz, double* Z, int64_t rows_per_child, float* parts, size_t parts_cap,
                                  int32_t* status, cudaStream_t s) {
  ZoffFusedProblem p;
  p.lo = lo; p.hi = hi; p.rank = rank; p.node0 = node0; p.s_max = s_max; p.ldz = ldz;
  p.ntile_n = (s_max + BN - 1) / BN;
  p.tile_n = BN;
  p.VT = nullptr; p.Ph = Ph; p.Z = Z;
  p.X32 = X32; p.skel = skel; p.d = d; p.c_exp = c_exp;
  const int mt = (s_max + kBM - 1) / kBM;
  p.ksplit = zoff_ksplit((int64_t)mt * p.ntile_n * 2 * nn, rows_per_child);
  return zoff_run<BN>(p, nn, mt, parts, parts_cap, status, s);
}

// tile_n: the tile width BN of the products, 128 or 256 columns
kf_status kf_tc_zoff_fused(const int32_t* lo, const int32_t* hi, const int32_t* rank, const int32_t* skel,
                           const float* X32, int d, float c_exp, int node0, int nn, int s_max, const float* Ph,
                           int ldz, double* Z, int64_t rows_per_child, float* parts, size_t parts_cap,
                           int32_t* status, cudaStream_t s, int tile_n) {
  return tile_n == 128 ? tc_zoff_fused_bn<128>(lo, hi, rank, skel, X32, d, c_exp, node0, nn, s_max, Ph, ldz, Z,
                                               rows_per_child, parts, parts_cap, status, s)
                       : tc_zoff_fused_bn<256>(lo, hi, rank, skel, X32, d, c_exp, node0, nn, s_max, Ph, ldz, Z,
                                               rows_per_child, parts, parts_cap, status, s);
}

// bytes of split-K partials the Z blocks of a level need (0: no split)
size_t kf_tc_zoff_parts_bytes(int s_max, int tile_n, int nn, int64_t rows_per_child) {
  const int mt = (s_max + kBM - 1) / kBM, nt = (s_max + tile_n - 1) / tile_n;
  const int64_t tiles = (int64_t)mt * nt * 2 * nn;
  const int ks = zoff_ksplit(tiles, rows_per_child);
  return ks > 1 ? sizeof(float) * (size_t)tiles * ks * kBM * tile_n : 0;
}

// tile_n: the tile width BN of the products, 128 or 256 columns
kf_status kf_tc_zoff(const int32_t* lo, const int32_t* hi, const int32_t* rank, int node0, int nn, int s_max,
                     const float* VT, const float* Ph, int ldz, double* Z, int64_t rows_per_child, float* parts,
                     size_t parts_cap, int32_t* status, cudaStream_t s, int tile_n) {
  return tile_n == 128 ? tc_zoff_bn<128>(lo, hi, rank, node0, nn, s_max, VT, Ph, ldz, Z, rows_per_child, parts,
                                         parts_cap, status, s)
                       : tc_zoff_bn<256>(lo, hi, rank, node0, nn, s_max, VT, Ph, ldz, Z, rows_per_child, parts,
                                         parts_cap, status, s);
}

kf_status kf_tc_telescope(const int32_t* lo, const int32_t* hi, const int32_t* rank, int node0, int nn, int s_max,
                          const float* Pc_hat, const float* Tm, int ldz, float* Pa_hat, int64_t rows_per_child,
                          int32_t* status, cudaStream_t s, int tile_n) {
  return tile_n == 128
             ? tc_telescope_bn<128>(lo, hi, rank, node0, nn, s_max, Pc_hat, Tm, ldz, Pa_hat, rows_per_child, status, s)
             : tc_telescope_bn<256>(lo, hi, rank, node0, nn, s_max, Pc_hat, Tm, ldz, Pa_hat, rows_per_child, status, s);
}


// Panel kb of the leaves' Cholesky factorization after k_chol_panel: the
// panel rows below the diagonal block (L21 = A21 Linv^T), then the trailing
// update A22 -= L21 L21^T.  nleaf leaves of at most ldL rows.
kf_status kf_tc_leaf_panel(const int32_t* lo, const int32_t* hi, int leaf0, int nleaf, int ldL, int kb, float* L,
                           const float* Dinv, int32_t* status, cudaStream_t s) {
  const int npan = (ldL + kBM - 1) / kBM;
  const int rows = ldL - kb - kBM;  // the most rows below the panel
  if (rows <= 0) return KF_OK;
  const unsigned mt = (unsigned)((rows + kBM - 1) / kBM);
  LeafTrsmProblem pt;
  pt.lo = lo; pt.hi = hi; pt.leaf0 = leaf0; pt.ldL = ldL; pt.kb = kb; pt.npan = npan; pt.L = L; pt.Dinv = Dinv;
  kf_status st = tc_launch<128>(pt, dim3(mt, 1, (unsigned)nleaf), KF_PH_LEAF_CHOL, status, s);
  if (st != KF_OK) return st;
  LeafSyrkProblem py;
  static_cast<LeafPanel&>(py) = pt;
  py.tile_n = 128;
  return tc_launch<128>(py, dim3(mt, mt, (unsigned)nleaf), KF_PH_LEAF_CHOL, status, s);
}

// P^ = L^-T L^-1 P for the leaves on the tensor cores: Y (the leaf rows of P^
// of the leaf level, FP32, holding P on entry) is solved in place panel by
// panel, forward then backward.
kf_status kf_tc_leaf_phat(const int32_t* lo, const int32_t* hi, const int32_t* rank, int leaf0, int nleaf, int ldL,
                          float* L, const float* Dinv, int s_max, float* Y, int32_t* status, cudaStream_t s) {
  const int npan = (ldL + kBM - 1) / kBM;
  const int BN = 128;
  const unsigned nt = (unsigned)((s_max + BN - 1) / BN);
  LeafPanel base;
  base.lo = lo; base.hi = hi; base.leaf0 = leaf0; base.ldL = ldL; base.npan = npan; base.L = L; base.Dinv = Dinv;
  kf_status st = KF_OK;
  for (int pi = 0; pi < npan && st == KF_OK; ++pi) {  // forward: L Y = P
    base.kb = pi * kBM;
    PhatDinvProblem<false> pd;
    static_cast<LeafPanel&>(pd) = base;
    pd.rank = rank; pd.s_max = s_max; pd.tile_n = BN; pd.Y = Y;
    st = tc_launch<128>(pd, dim3(1, nt, (unsigned)nleaf), KF_PH_LEAF_PHAT, status, s);
    const int rows = ldL - base.kb - kBM;
    if (st != KF_OK || rows <= 0) continue;
    PhatUpdateProblem<false> pu;
    static_cast<LeafPanel&>(pu) = base;
    pu.rank = rank; pu.s_max = s_max; pu.tile_n = BN; pu.Y = Y;
    st = tc_launch<128>(pu, dim3((unsigned)((rows + kBM - 1) / kBM), nt, (unsigned)nleaf), KF_PH_LEAF_PHAT, status, s);
  }
  for (int pi = npan - 1; pi >= 0 && st == KF_OK; --pi) {  // backward: L^T X = Y
    base.kb = pi * kBM;
    PhatDinvProblem<true> pd;
    static_cast<LeafPanel&>(pd) = base;
    pd.rank = rank; pd.s_max = s_max; pd.tile_n = BN; pd.Y = Y;
    st = tc_launch<128>(pd, dim3(1, nt, (unsigned)nleaf), KF_PH_LEAF_PHAT, status, s);
    if (st != KF_OK || base.kb == 0) continue;
    PhatUpdateProblem<true> pu;
    static_cast<LeafPanel&>(pu) = base;
    pu.rank = rank; pu.s_max = s_max; pu.tile_n = BN; pu.Y = Y;
    st = tc_launch<128>(pu, dim3((unsigned)((base.kb + kBM - 1) / kBM), nt, (unsigned)nleaf), KF_PH_LEAF_PHAT,
                        status, s);
  }
  return st;
}

extern "C" kf_status kf_test_tc_wait_probe(int64_t polls) {
  if (polls < 0) return kf_set_err(nullptr, KF_EINVAL, "kf_test_tc_wait_probe: polls must be >= 0");
  long long v = (long long)polls;
  cudaError_t e = cudaMemcpyToSymbol(g_tc_probe_polls, &v, sizeof(v));
  if (e != cudaSuccess)
    return kf_set_err(nullptr, KF_ECUDA, "kf_test_tc_wait_probe: %s", cudaGetErrorString(e));
  return KF_OK;
}
