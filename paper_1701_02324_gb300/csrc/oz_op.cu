// oz_op.cu -- the V pass of the mixed path's FP64-accurate operator for
// blocks of right-hand sides on the tensor cores, exact in integer
// arithmetic.  The pass forms, for every node of a level, the column sums of
// its sibling coupling (Eq. e:blocksmw, the K_{sib~ node} x_node of the
// hierarchical matvec)
//
//   u[sib][q][r] += sum_{i in node} V[i][q] x[i][r],   V[i][q] = K(x_i, x_{sib~ q}),
//
// which the double-float CUDA-core kernel (k_colsum_df) computes at about 15
// FP32 instructions per multiply-add.  Here the products run as BF16 tensor-core
// MMAs on integer slices of both operands, the error-free splitting of Ozaki,
// Ogita, Oishi and Rump (Numer. Algorithms 59, 2012):
//
//   * V entries are kernel values in [0, 1].  Each is rounded to a multiple of
//     2^-49 and cut into 7 unsigned 7-bit digits a_p (a_0 <= 128), V = sum_p
//     a_p 2^-7(p+1); the digits are stored as BF16 (integers of at most 8
//     significant bits are exact) once per factorization, in tiles of 128 rows
//     x 128 skeleton columns laid out as the tensor core reads them, so that a
//     tile is one bulk copy.
//   * Every column r of x is scaled by tau_r = 2^e_r >= max_i |x_ir|, rounded to
//     a multiple of 2^-49 tau_r and cut into 7 balanced digits d_q (|d_0| <=
//     128, |d_q| <= 64), per operator call.
//   * A product of digits is an integer below 2^14 in magnitude; the group sums
//     acc_g = sum_{p+q=g} sum_i a_p d_q over a window of 128 rows stay below
//     2^24, so the FP32 accumulation in tensor memory is exact.  The 34 digit
//     pairs with p + q <= 7 are formed; the dropped pairs (below 2^-54 tau_r)
//     and the two roundings (2^-50 each) leave about 2^-49 tau_r per product.
//   * A CTA takes 8 windows (1024 rows) of one node, 128 skeleton columns and
//     NC right-hand sides.  The windows' group sums, exact integers, are summed
//     in two int64 accumulators (groups 0-3 and 4-7), and the chunk writes its
//     FP64 partial sum tau_r 2^-63 (2^28 hi + lo) (one rounding) for the
//     fixed-order reduction of the column sums.
//
// Roles (256 threads): warp 0 issues the bulk copies of the V digit tiles
// into a ring of shared-memory stages; warp 1 issues the MMAs (one thread):
// per window and V digit p one MMA chain with B = the x digit tiles d_0 ..
// d_min(6, 7-p) side by side (N up to 8 NC) into the accumulator columns
// from group p on, so that digit pair (p, q) lands in group p + q (for p = 0
// a zero tile after d_6 clears group 7);
// warps 2-3 stage the x digits of the next window; warps 4-7 read the
// accumulators out of tensor memory (two buffers, so that a window's MMAs
// overlap the previous window's read-out).  Every wait is bounded; on time-out
// the kernel flags KF_DEV_TIMEOUT, waits for its own MMAs once more, frees
// its tensor memory and returns.
#include <algorithm>

#include "kf_internal.cuh"
#include "prof.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace kf_tc;

constexpr int kOzSlices = 7;                      // digits per operand
constexpr int kOzGroups = 8;                      // digit pairs p + q = 0 .. 7
constexpr int kOzWin = 128;                       // rows per window (exact accumulation)
constexpr int kOzWinPerChunk = kOzChunkRows / kOzWin;
constexpr int kOzQ = 128;                         // skeleton columns per CTA (MMA M)
constexpr int kOzTileBytes = kOzTileElems * 2;    // one BF16 digit tile
constexpr int kOzThreads = 256;

inline int grid_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

// BF16 bit pattern of a small integer (|d| <= 256: exact)
__device__ __forceinline__ uint32_t oz_bf16(int d) { return __float_as_uint((float)d) >> 16; }

// round(x 2^49) for a float |x| < 2, as an integer
__device__ __forceinline__ int64_t oz_fixed_f(float x) {
  const uint32_t b = __float_as_uint(x);
  const int ex = (int)((b >> 23) & 0xFFu);
  if (ex == 0) return 0;  // zero or below 2^-126
  const int64_t m = (int64_t)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = ex - 150 + 49;  // x = m 2^(ex - 150)
  int64_t r;
  if (sh >= 0) r = m << sh;
  else if (sh > -62) r = (m + ((int64_t)1 << (-sh - 1))) >> (-sh);
  else r = 0;
  return (b >> 31) ? -r : r;
}

// round(x 2^s) for a double with |x 2^s| < 2^49, as an integer
__device__ __forceinline__ int64_t oz_fixed_d(double x, int s) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FFu);
  if (ex == 0) return 0;  // zero or below 2^-1022
  const int64_t m = (int64_t)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int sh = ex - 1075 + s;  // x 2^s = m 2^sh, sh <= -4 in range
  int64_t r;
  if (sh >= 0) r = 0;  // out of range (tau_r below |x|): not produced by the exponents below
  else if (sh > -62) r = (m + ((int64_t)1 << (-sh - 1))) >> (-sh);
  else r = 0;
  return (b >> 63) ? -r : r;
}

// ---- factorization: V digit tiles of one level ----------------------------------
// grid = (windows of the largest node, nodes of the level, skeleton tiles).
// Thread item (qq, ig): skeleton column t*128 + qq, rows 8 ig .. 8 ig + 7 of
// the window; the 8 digits of a slice land in one 16-byte row of a core
// matrix (K-major: element (m = qq, k = ii) of a tile at
// ((qq / 8) * 16 + ii / 8) * 64 + (qq % 8) * 8 + ii % 8).
__global__ void __launch_bounds__(256) k_oz_slice_v(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                    const int32_t* __restrict__ rank, int node0, int s_max, int qt,
                                                    const float2* __restrict__ Vdf,
                                                    const int32_t* __restrict__ wbase, uint16_t* __restrict__ Asl) {
  const int nl = blockIdx.y, node = node0 + nl, sib = node ^ 1, w = blockIdx.x, t = blockIdx.z;
  const int b = lo[node], n = hi[node] - b;
  if (w * kOzWin >= n) return;
  const int cnt = rank[sib];
  uint16_t* base = Asl + ((int64_t)(wbase[nl] + w) * qt + t) * kOzSlices * kOzTileElems;
  for (int item = threadIdx.x; item < kOzQ * (kOzWin / 8); item += blockDim.x) {
    const int qq = item % kOzQ, ig = item / kOzQ;
    const int q = t * kOzQ + qq;
    uint32_t pk[kOzSlices][4];
#pragma unroll
    for (int p = 0; p < kOzSlices; ++p) pk[p][0] = pk[p][1] = pk[p][2] = pk[p][3] = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int ii = w * kOzWin + ig * 8 + j;
      int64_t V = 0;
      if (q < cnt && ii < n) {
        const float2 v = Vdf[(int64_t)(b + ii) * s_max + q];
        V = oz_fixed_f(v.x) + oz_fixed_f(v.y);
        V = V < 0 ? 0 : (V > ((int64_t)1 << 49) ? ((int64_t)1 << 49) : V);
      }
#pragma unroll
      for (int p = 0; p < kOzSlices; ++p) {
        const int a = p == 0 ? (int)(V >> 42) : (int)((V >> (7 * (6 - p))) & 127);
        pk[p][j >> 1] |= oz_bf16(a) << (16 * (j & 1));
      }
    }
    const int off = ((qq >> 3) * 16 + ig) * 64 + (qq & 7) * 8;
#pragma unroll
    for (int p = 0; p < kOzSlices; ++p)
      *(uint4*)(base + (int64_t)p * kOzTileElems + off) = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
  }
}

// ---- factorization: digit tiles of the leaf blocks ----------------------------
// grid = (column windows, leaves, row tiles).  K_aa (row-major, leading
// dimension ldL, entries in [0, 1]) as tiles of 128 rows x 128 columns x 7
// digits, (leaf, row tile t, column window w) in order; thread item (m, kg):
// row 128 t + m, columns 128 w + 8 kg .. + 7 (64 contiguous bytes of pairs).
__global__ void __launch_bounds__(256) k_oz_slice_leaf(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                       int leaf0, int ldL, int tpl, const float2* __restrict__ Kdf,
                                                       uint16_t* __restrict__ Ksl) {
  const int lf = blockIdx.y, w = blockIdx.x, t = blockIdx.z;
  const int n = hi[leaf0 + lf] - lo[leaf0 + lf];
  if (w * kOzWin >= n || t * kOzQ >= n) return;
  const float2* Kb = Kdf + (int64_t)lf * ldL * ldL;
  uint16_t* base = Ksl + (((int64_t)lf * tpl + t) * tpl + w) * kOzSlices * kOzTileElems;
  for (int item = threadIdx.x; item < kOzQ * (kOzWin / 8); item += blockDim.x) {
    const int kg = item % (kOzWin / 8), m = item / (kOzWin / 8);
    const int i = t * kOzQ + m;
    uint32_t pk[kOzSlices][4];
#pragma unroll
    for (int p = 0; p < kOzSlices; ++p) pk[p][0] = pk[p][1] = pk[p][2] = pk[p][3] = 0u;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = w * kOzWin + kg * 8 + jj;
      int64_t V = 0;
      if (i < n && j < n) {
        const float2 v = Kb[(int64_t)i * ldL + j];
        V = oz_fixed_f(v.x) + oz_fixed_f(v.y);
        V = V < 0 ? 0 : (V > ((int64_t)1 << 49) ? ((int64_t)1 << 49) : V);
      }
#pragma unroll
      for (int p = 0; p < kOzSlices; ++p) {
        const int a = p == 0 ? (int)(V >> 42) : (int)((V >> (7 * (6 - p))) & 127);
        pk[p][jj >> 1] |= oz_bf16(a) << (16 * (jj & 1));
      }
    }
    const int off = ((m >> 3) * 16 + kg) * 64 + (m & 7) * 8;
#pragma unroll
    for (int p = 0; p < kOzSlices; ++p)
      *(uint4*)(base + (int64_t)p * kOzTileElems + off) = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
  }
}

// ---- operator call: x digits ----------------------------------------------------
// column maxima of |x| as FP64 bit patterns (non-negative doubles order like
// their bit patterns, so integer maxima are exact and order-independent)
__global__ void __launch_bounds__(256) k_oz_colmax(const double* __restrict__ x, int64_t N, int k,
                                                   unsigned long long* __restrict__ mx) {
  extern __shared__ unsigned long long smx[];
  for (int r = threadIdx.x; r < k; r += blockDim.x) smx[r] = 0ull;
  __syncthreads();
  const int64_t nk = N * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x)
    atomicMax(&smx[e % k], (unsigned long long)__double_as_longlong(fabs(x[e])));
  __syncthreads();
  for (int r = threadIdx.x; r < k; r += blockDim.x)
    if (smx[r]) atomicMax(&mx[r], smx[r]);
}

// e_r with 2^e_r > max |x_r| (0 for a zero column; a non-finite column gets
// kOzBadExp, which makes its sums NaN)
constexpr int kOzBadExp = -100000;
__global__ void k_oz_exponents(const unsigned long long* __restrict__ mx, int k, int32_t* __restrict__ xexp) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x) {
    const int ef = (int)((mx[r] >> 52) & 0x7FFu);
    xexp[r] = ef == 0x7FF ? kOzBadExp : (mx[r] == 0ull ? 0 : ef - 1023 + 1);
  }
}

// xsl[(p kpad + r) ldx + i]: digit p of round(x_ir 2^(49 - e_r)), balanced
// (each of d_6 .. d_1 in [-64, 63], d_0 the rest, |d_0| <= 128)
__global__ void __launch_bounds__(256) k_oz_slice_x(const double* __restrict__ x, int64_t N, int k, int kpad,
                                                    int64_t ldx, const int32_t* __restrict__ xexp,
                                                    uint16_t* __restrict__ xsl) {
  const int64_t nk = N * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / N);
    const int64_t i = e % N;  // consecutive threads: consecutive rows of one column (coalesced digit stores)
    const int ex = xexp[r];
    int64_t v = ex == kOzBadExp ? 0 : oz_fixed_d(x[i * k + r], 49 - ex);
    int dg[kOzSlices];
#pragma unroll
    for (int p = kOzSlices - 1; p >= 1; --p) {
      const int64_t d = ((v + 64) & 127) - 64;
      dg[p] = (int)d;
      v = (v - d) >> 7;
    }
    dg[0] = (int)v;
#pragma unroll
    for (int p = 0; p < kOzSlices; ++p) xsl[((int64_t)p * kpad + r) * ldx + i] = (uint16_t)oz_bf16(dg[p]);
  }
}

// ---- the V pass -----------------------------------------------------------------
template <int NC>
struct OzCfg {
  static constexpr int kStages = NC == 16 ? 4 : 3;              // V digit tiles in flight
  static constexpr int kBBytes = (kOzSlices + 1) * NC * kOzWin * 2;  // x digits of one window + a zero tile
  static constexpr int kSmem = kStages * kOzTileBytes + 2 * kBBytes;
  static constexpr int kAccCols = kOzGroups * NC;               // one buffer of group sums
  static constexpr uint32_t kTmemCols = 2 * kAccCols <= 256 ? 256u : 512u;
};

// V pass (LEAF = false): grid = (1024-row chunks of the largest node, nodes,
// skeleton tiles x column groups); CTA (ch, node, t) sums rows 1024 ch ..
// of the node against skeleton columns 128 t .. of its sibling into parts.
// Leaf blocks (LEAF = true, leaves of at most 1024 points): grid = (1,
// leaves, row tiles x column groups); CTA (0, leaf, t) forms rows 128 t ..
// of y = lambda x + K_aa x over all of the leaf's columns, in place of the
// skeleton columns: the same products with A = the leaf block's digits.
template <int NC, bool LEAF>
__global__ void __launch_bounds__(kOzThreads, 1)
    k_colsum_oz(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, const int32_t* __restrict__ rank,
                int node0, int s_max, int qt, const uint16_t* __restrict__ Asl, const int32_t* __restrict__ wbase,
                const uint16_t* __restrict__ xsl, int64_t ldx, int kpad, const int32_t* __restrict__ xexp, int k,
                int nchunk, double* __restrict__ parts, double lambda, const double* __restrict__ x,
                double* __restrict__ y, int32_t* __restrict__ status) {
  using C = OzCfg<NC>;
  constexpr int ST = C::kStages;
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  __shared__ __align__(8) uint64_t a_full[ST], a_empty[ST], b_full[2], b_empty[2], acc_full[2], acc_empty[2], done;
  __shared__ uint32_t tmem_base;
  const int nl = blockIdx.y, node = node0 + nl, sib = node ^ 1;
  const int b = lo[node], n = hi[node] - b;
  const int cnt = LEAF ? n : rank[sib];  // rows of the product (M)
  const int t = blockIdx.z % qt, c0 = (blockIdx.z / qt) * NC;
  const int ch = blockIdx.x, w0 = ch * kOzWinPerChunk;
  const int nw = min(kOzWinPerChunk, (n + kOzWin - 1) / kOzWin - w0);
  if (nw <= 0 || cnt <= t * kOzQ || c0 >= k) return;  // uniform over the CTA
  uint16_t* As = (uint16_t*)oz_smem;
  uint16_t* Bs = (uint16_t*)(oz_smem + ST * kOzTileBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_base, C::kTmemCols);
  if (tid == 32) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&a_full[s], 1);
      mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&b_full[s], 64);
      mbar_init(&b_empty[s], 1);
      mbar_init(&acc_full[s], 1);
      mbar_init(&acc_empty[s], 128);
    }
    mbar_init(&done, 1);
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  const int nunits = nw * kOzSlices;  // (window, V digit) pairs, in order
  if (warp == 0) {
    // bulk copies of the V digit tiles
    if (lane == 0) {
      // V: tiles by (window of the level, skeleton tile); leaf: by (leaf, row tile, window)
      const uint16_t* tiles = LEAF ? Asl + ((int64_t)nl * qt + t) * qt * kOzSlices * kOzTileElems
                                   : Asl + ((int64_t)(wbase[nl] + w0) * qt + t) * kOzSlices * kOzTileElems;
      const int64_t wstride = (int64_t)(LEAF ? 1 : qt) * kOzSlices * kOzTileElems;  // elements between windows
      for (int u = 0; u < nunits; ++u) {
        const int st = u % ST;
        if (u >= ST && !mbar_wait(&a_empty[st], (uint32_t)((u / ST) - 1) & 1u)) {
          atomicOr(status, KF_DEV_TIMEOUT);
          break;
        }
        mbar_arrive_expect_tx(&a_full[st], kOzTileBytes);
        bulk_g2s(As + st * kOzTileElems, tiles + (u / kOzSlices) * wstride + (int64_t)(u % kOzSlices) * kOzTileElems,
                 kOzTileBytes, &a_full[st]);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // MMAs: window w, V digit p against x digits q <= 7 - p into group p + q
    if (lane == 0) {
      bool ok = true;
      int issued = 0;
      for (int w = 0; w < nw && ok; ++w) {
        const int buf = w & 1;
        ok = mbar_wait(&b_full[buf], (uint32_t)(w >> 1) & 1u);
        if (ok && w >= 2) ok = mbar_wait(&acc_empty[buf], (uint32_t)((w >> 1) - 1) & 1u);
        if (!ok) break;
        fence_after_sync();
        const uint32_t bs0 = smem_u32(Bs + buf * (C::kBBytes / 2));
        for (int p = 0; p < kOzSlices; ++p) {
          const int u = w * kOzSlices + p, st = u % ST;
          if (!(ok = mbar_wait(&a_full[st], (uint32_t)(u / ST) & 1u))) break;
          fence_after_sync();
          const uint32_t as = smem_u32(As + st * kOzTileElems);
          // p = 0: d_0 .. d_6 and the zero tile (groups 0-7, overwritten);
          // p >= 1: d_0 .. d_min(6, 7-p) (groups p .. 7, accumulated)
          const int nq = p == 0 ? kOzSlices + 1 : min(kOzSlices, kOzGroups - p);
          const uint32_t idesc = idesc_bf16(kOzQ, nq * NC);
          const uint32_t dt = tmem + (uint32_t)(buf * C::kAccCols + p * NC);
#pragma unroll
          for (int ks = 0; ks < kOzWin / 16; ++ks)  // K = 16 BF16: two core matrices
            mma_bf16(dt, smem_desc(as + ks * 256, 128, 2048), smem_desc(bs0 + ks * 256, 128, 2048), idesc,
                     (p == 0 && ks == 0) ? 0u : 1u);
          ++issued;
          mma_commit(&a_empty[st]);
        }
        if (!ok) break;
        mma_commit(&b_empty[buf]);
        mma_commit(&acc_full[buf]);
      }
      if (!ok) atomicOr(status, KF_DEV_TIMEOUT);
      if (issued > 0) {  // every MMA of this CTA complete before tensor memory is freed
        mma_commit(&done);
        if (!mbar_wait(&done, 0u)) atomicOr(status, KF_DEV_TIMEOUT);
      }
    }
    __syncwarp();
  } else if (warp < 4) {
    // x digits of window w into buffer w & 1 (K-major: element (m = r, k = ii)
    // of digit q at ((r / 8) * 16 + ii / 8) * 64 + (r % 8) * 8 + ii % 8)
    const int sid = tid - 64;
    for (int e = sid; e < NC * kOzWin / 8; e += 64)  // the zero tile after d_6, in both buffers
      for (int bb = 0; bb < 2; ++bb)
        *(uint4*)(Bs + bb * (C::kBBytes / 2) + kOzSlices * NC * kOzWin + e * 8) = make_uint4(0u, 0u, 0u, 0u);
    for (int w = 0; w < nw; ++w) {
      const int buf = w & 1;
      if (w >= 2 && !mbar_wait(&b_empty[buf], (uint32_t)((w >> 1) - 1) & 1u)) {
        atomicOr(status, KF_DEV_TIMEOUT);
        break;
      }
      const int ib = (w0 + w) * kOzWin, nr = min(kOzWin, n - ib);
      const int64_t i0 = (int64_t)b + ib;
      uint16_t* B = Bs + buf * (C::kBBytes / 2);
      for (int e = sid; e < kOzSlices * NC * (kOzWin / 8); e += 64) {
        const int ig = e % (kOzWin / 8), r = (e / (kOzWin / 8)) % NC, q = e / (NC * (kOzWin / 8));
        const uint16_t* src = xsl + ((int64_t)q * kpad + c0 + r) * ldx + i0 + ig * 8;
        uint16_t* dst = B + q * NC * kOzWin + ((r >> 3) * 16 + ig) * 64 + (r & 7) * 8;
        if ((i0 & 7) == 0 && ig * 8 + 8 <= nr) {
          cp_async16(dst, src);  // all of the thread's copies in flight together
        } else {                 // a node start off the 8-row grid, or the window's ragged end
          uint32_t pk[4] = {0u, 0u, 0u, 0u};
          for (int j = 0; j < 8; ++j)
            if (ig * 8 + j < nr) pk[j >> 1] |= (uint32_t)src[j] << (16 * (j & 1));
          *(uint4*)dst = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
      }
      cp_async_wait_all();
      fence_proxy_async();
      mbar_arrive(&b_full[buf]);
    }
  } else {
    // read-out: thread = accumulator row (skeleton column) t*128 + 32 (warp % 4) + lane
    const int quad = warp & 3;
    int64_t hi64[NC], lo64[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) hi64[c] = lo64[c] = 0;
    bool ok = true;
    for (int w = 0; w < nw; ++w) {
      const int buf = w & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (uint32_t)(w >> 1) & 1u))) {  // warp-uniform
        if (lane == 0) atomicOr(status, KF_DEV_TIMEOUT);
        ok = false;
        break;
      }
      fence_after_sync();
#pragma unroll 1
      for (int g = 0; g < kOzGroups; ++g) {
        const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * C::kAccCols + g * NC);
        float v[NC];
        if constexpr (NC == 16) {
          tmem_ld16(ta, v);
        } else {
          tmem_ld32(ta, v);
        }
        const int sh = g <= 3 ? 7 * (3 - g) : 7 * (7 - g);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int64_t a = (int64_t)__float2int_rn(v[c]) << sh;  // exact: |v| < 2^24
          if (g <= 3) hi64[c] += a;
          else lo64[c] += a;
        }
      }
      fence_before_sync();
      mbar_arrive(&acc_empty[buf]);
    }
    const int q = t * kOzQ + quad * 32 + lane;
    if (ok && q < cnt) {
      double* out = LEAF ? y + ((int64_t)b + q) * k : parts + (((int64_t)nl * nchunk + ch) * s_max + q) * k;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int col = c0 + c;
        if (col >= k) break;
        const int ex = xexp[col];
        const double v = ex == kOzBadExp ? __longlong_as_double(0x7FF8000000000000ll)
                                         : ldexp((double)hi64[c], ex - 35) + ldexp((double)lo64[c], ex - 63);
        if (LEAF) out[col] = lambda * x[((int64_t)b + q) * k + col] + v;
        else out[col] = v;
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, C::kTmemCols);
}

}  // namespace

// Windows of 128 rows per node, level by level, and the BF16 digit tiles of
// the V blocks (7 per window and 128 skeleton columns).  A failed allocation
// leaves the pass to the double-float kernels.
kf_status kf_oz_alloc(kf_factor* f, cudaStream_t s) {
  kf_tree* t = f->t;
  const int D = t->D, qt = (f->s_max + kOzQ - 1) / kOzQ;
  if (D == 0 || !f->VTdf) return KF_OK;
  f->oz_wbase_h.assign((size_t)2 << D, 0);
  f->oz_off.assign((size_t)D + 2, 0);
  int64_t tiles = 0;
  for (int l = 1; l <= D; ++l) {
    f->oz_off[l] = tiles * kOzTileElems;
    int64_t wc = 0;
    for (int a = 1 << l; a < (2 << l); ++a) {
      f->oz_wbase_h[a] = (int32_t)wc;
      wc += (t->hi[a] - t->lo[a] + kOzWin - 1) / kOzWin;
    }
    tiles += wc * qt * kOzSlices;
  }
  f->oz_off[D + 1] = tiles * kOzTileElems;
  const size_t vb = sizeof(uint16_t) * (size_t)tiles * kOzTileElems, wb = sizeof(int32_t) * ((size_t)2 << D);
  void* p = f->ctx->dalloc(vb, s);
  void* q = p ? f->ctx->dalloc(wb, s) : nullptr;
  if (!p || !q) {
    if (p) f->ctx->dfree(p, vb, s);
    cudaGetLastError();
    return KF_OK;
  }
  f->allocs.push_back({p, vb});
  f->allocs.push_back({q, wb});
  f->VTsl = (uint16_t*)p;
  f->oz_wbase = (int32_t*)q;
  KF_CUDA(f->ctx, cudaMemcpyAsync(f->oz_wbase, f->oz_wbase_h.data(), wb, cudaMemcpyHostToDevice, s));
  // the leaf blocks' digits (leaves of at most one 1024-row chunk)
  if (f->Kdf && t->leaf_max <= kOzChunkRows) {
    const int64_t tpl = (t->leaf_max + kOzQ - 1) / kOzQ;
    const size_t kb = sizeof(uint16_t) * (size_t)((int64_t)1 << D) * tpl * tpl * kOzSlices * kOzTileElems;
    void* r = f->ctx->dalloc(kb, s);
    if (r) {
      f->allocs.push_back({r, kb});
      f->Ksl = (uint16_t*)r;
    } else {
      cudaGetLastError();
    }
  }
  return KF_OK;
}

// digit tiles of the leaf blocks (after their double-float pairs are written)
kf_status kf_oz_slice_leaf(kf_factor* f, cudaStream_t s) {
  kf_tree* t = f->t;
  if (!f->Ksl) return KF_OK;
  const int tpl = (t->leaf_max + kOzQ - 1) / kOzQ;
  dim3 g((unsigned)tpl, 1u << t->D, (unsigned)tpl);
  KF_PHASE(KF_PH_LEAF_ASM, s, k_oz_slice_leaf<<<g, 256, 0, s>>>(t->d_lo, t->d_hi, 1 << t->D, t->leaf_max, tpl,
                                                                f->Kdf, f->Ksl));
  KF_LAUNCH_CHECK(f->ctx);
  return KF_OK;
}

// V digit tiles of level lv (after its double-float V blocks are written)
kf_status kf_oz_slice_v(kf_factor* f, int lv, cudaStream_t s) {
  kf_tree* t = f->t;
  if (!f->VTsl || lv < 1 || lv > t->D) return KF_OK;
  const int qt = (f->s_max + kOzQ - 1) / kOzQ;
  int maxn = 0;
  for (int a = 1 << lv; a < (2 << lv); ++a) maxn = std::max(maxn, t->hi[a] - t->lo[a]);
  if (maxn == 0) return KF_OK;
  dim3 g((unsigned)((maxn + kOzWin - 1) / kOzWin), 1u << lv, (unsigned)qt);
  KF_PHASE(KF_PH_EVAL_V, s, k_oz_slice_v<<<g, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, 1 << lv, f->s_max, qt,
                                                           f->VTdf + (int64_t)(lv - 1) * t->N * f->s_max,
                                                           f->oz_wbase + (1 << lv), f->VTsl + f->oz_off[lv]));
  KF_LAUNCH_CHECK(f->ctx);
  return KF_OK;
}

// x of one operator call as digits (k >= 2 right-hand sides, N x k point-major)
kf_status kf_oz_prepare_x(kf_factor* f, const double* x, int64_t k, kf_oz_x* oz, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  const int64_t N = f->t->N;
  oz->k = k;
  oz->nc = k > 16 ? 32 : 16;
  oz->kpad = (int)((k + oz->nc - 1) / oz->nc) * oz->nc;
  oz->ldx = (N + 7) / 8 * 8;
  oz->bytes = sizeof(uint16_t) * (size_t)kOzSlices * oz->kpad * oz->ldx;
  oz->xsl = (uint16_t*)c->dalloc(oz->bytes, s);
  oz->xmax = (unsigned long long*)c->dalloc(sizeof(unsigned long long) * (size_t)k, s);
  oz->xexp = (int32_t*)c->dalloc(sizeof(int32_t) * (size_t)k, s);
  if (!oz->xsl || !oz->xmax || !oz->xexp) {
    kf_oz_release_x(f, oz, s);
    return kf_set_err(c, KF_ENOMEM, "matvec: allocation of the x digits failed");
  }
  KF_CUDA(c, cudaMemsetAsync(oz->xsl, 0, oz->bytes, s));
  KF_CUDA(c, cudaMemsetAsync(oz->xmax, 0, sizeof(unsigned long long) * (size_t)k, s));
  const int smx = (int)(sizeof(unsigned long long) * (size_t)k);
  KF_PHASE(KF_PH_MV_COLSUM, s, k_oz_colmax<<<grid_for(N * k, 256, 1024), 256, smx, s>>>(x, N, (int)k, oz->xmax));
  KF_PHASE(KF_PH_MV_COLSUM, s, k_oz_exponents<<<grid_for(k, 256), 256, 0, s>>>(oz->xmax, (int)k, oz->xexp));
  KF_PHASE(KF_PH_MV_COLSUM, s, k_oz_slice_x<<<grid_for(N * k, 256), 256, 0, s>>>(x, N, (int)k, oz->kpad, oz->ldx,
                                                                                oz->xexp, oz->xsl));
  KF_LAUNCH_CHECK(c);
  return KF_OK;
}

void kf_oz_release_x(kf_factor* f, kf_oz_x* oz, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  if (oz->xsl) c->dfree(oz->xsl, oz->bytes, s);
  if (oz->xmax) c->dfree(oz->xmax, sizeof(unsigned long long) * (size_t)oz->k, s);
  if (oz->xexp) c->dfree(oz->xexp, sizeof(int32_t) * (size_t)oz->k, s);
  *oz = kf_oz_x{};
}

// The V pass of level l: FP64 partial sums of 1024-row chunks into parts
// (the layout of k_colsum's, nchunk chunks a node); the caller reduces them.
kf_status kf_oz_colsum_level(kf_factor* f, int l, const kf_oz_x& oz, int64_t k, double* parts, int* nchunk,
                             cudaStream_t s) {
  kf_tree* t = f->t;
  const int qt = (f->s_max + kOzQ - 1) / kOzQ;
  int maxn = 0;
  for (int a = 1 << l; a < (2 << l); ++a) maxn = std::max(maxn, t->hi[a] - t->lo[a]);
  const int nch = std::max(1, (maxn + kOzChunkRows - 1) / kOzChunkRows);
  *nchunk = nch;
  dim3 g((unsigned)nch, 1u << l, (unsigned)(qt * (oz.kpad / oz.nc)));
  const uint16_t* Asl = f->VTsl + f->oz_off[l];
  const int32_t* wb = f->oz_wbase + (1 << l);
  if (oz.nc == 16) {
    KF_CUDA(f->ctx, cudaFuncSetAttribute(k_colsum_oz<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         OzCfg<16>::kSmem));
    KF_PHASE(KF_PH_MV_COLSUM, s, k_colsum_oz<16, false><<<g, kOzThreads, OzCfg<16>::kSmem, s>>>(
                                     t->d_lo, t->d_hi, f->rank, 1 << l, f->s_max, qt, Asl, wb, oz.xsl, oz.ldx,
                                     oz.kpad, oz.xexp, (int)k, nch, parts, 0.0, nullptr, nullptr, f->status));
  } else {
    KF_CUDA(f->ctx, cudaFuncSetAttribute(k_colsum_oz<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         OzCfg<32>::kSmem));
    KF_PHASE(KF_PH_MV_COLSUM, s, k_colsum_oz<32, false><<<g, kOzThreads, OzCfg<32>::kSmem, s>>>(
                                     t->d_lo, t->d_hi, f->rank, 1 << l, f->s_max, qt, Asl, wb, oz.xsl, oz.ldx,
                                     oz.kpad, oz.xexp, (int)k, nch, parts, 0.0, nullptr, nullptr, f->status));
  }
  KF_LAUNCH_CHECK(f->ctx);
  return KF_OK;
}

// Leaf blocks: y = lambda x + K_aa x for every leaf (x, y: N x k, tree order)
kf_status kf_oz_leaf(kf_factor* f, const kf_oz_x& oz, int64_t k, double lambda, const double* x, double* y,
                     cudaStream_t s) {
  kf_tree* t = f->t;
  const int tpl = (t->leaf_max + kOzQ - 1) / kOzQ;
  dim3 g(1u, 1u << t->D, (unsigned)(tpl * (oz.kpad / oz.nc)));
  if (oz.nc == 16) {
    KF_CUDA(f->ctx, cudaFuncSetAttribute(k_colsum_oz<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         OzCfg<16>::kSmem));
    KF_PHASE(KF_PH_MV_LEAF, s, k_colsum_oz<16, true><<<g, kOzThreads, OzCfg<16>::kSmem, s>>>(
                                   t->d_lo, t->d_hi, f->rank, 1 << t->D, f->s_max, tpl, f->Ksl, nullptr, oz.xsl,
                                   oz.ldx, oz.kpad, oz.xexp, (int)k, 1, nullptr, lambda, x, y, f->status));
  } else {
    KF_CUDA(f->ctx, cudaFuncSetAttribute(k_colsum_oz<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         OzCfg<32>::kSmem));
    KF_PHASE(KF_PH_MV_LEAF, s, k_colsum_oz<32, true><<<g, kOzThreads, OzCfg<32>::kSmem, s>>>(
                                   t->d_lo, t->d_hi, f->rank, 1 << t->D, f->s_max, tpl, f->Ksl, nullptr, oz.xsl,
                                   oz.ldx, oz.kpad, oz.xexp, (int)k, 1, nullptr, lambda, x, y, f->status));
  }
  KF_LAUNCH_CHECK(f->ctx);
  return KF_OK;
}
