// oz_op.cu -- the mixed path's FP64-accurate operator for blocks of
// right-hand sides on the tensor cores, exact in integer arithmetic: the
// leaf blocks K_aa x_a, the pushes of the skeleton weights through P_c, the
// leaves' row update P g, and the V pass, which forms for every node of a
// level the column sums of
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
// Order-preserving key of |x| (non-negative doubles order like their bit
// patterns, so integer maxima are exact and order-independent)
__device__ __forceinline__ unsigned long long oz_key(double x) {
  return (unsigned long long)__double_as_longlong(fabs(x));
}

// column maxima of |x| (N x k point-major) as keys
__global__ void __launch_bounds__(256) k_oz_colmax(const double* __restrict__ x, int64_t N, int k,
                                                   unsigned long long* __restrict__ mx) {
  extern __shared__ unsigned long long smx[];
  for (int r = threadIdx.x; r < k; r += blockDim.x) smx[r] = 0ull;
  __syncthreads();
  const int64_t nk = N * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x)
    atomicMax(&smx[e % k], oz_key(x[e]));
  __syncthreads();
  for (int r = threadIdx.x; r < k; r += blockDim.x)
    if (smx[r]) atomicMax(&mx[r], smx[r]);
}

// e with 2^e > the key's value (0 for zero; a non-finite value gets
// kOzBadExp, which makes the sums NaN)
constexpr int kOzBadExp = -100000;
__device__ __forceinline__ int oz_exp_of(unsigned long long key) {
  const int ef = (int)((key >> 52) & 0x7FFu);
  return ef == 0x7FF ? kOzBadExp : (key == 0ull ? 0 : ef - 1023 + 1);
}
__global__ void k_oz_exponents(const unsigned long long* __restrict__ mx, int k, int32_t* __restrict__ xexp) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x) xexp[r] = oz_exp_of(mx[r]);
}

// the ND balanced digits of v (|v| <= 2^(7 ND)): each of d_(ND-1) .. d_1 in
// [-64, 63], d_0 the rest (|d_0| <= 128), as BF16 bit patterns
template <int ND>
__device__ __forceinline__ void oz_digits(int64_t v, uint16_t (&dg)[ND]) {
#pragma unroll
  for (int p = ND - 1; p >= 1; --p) {
    const int64_t d = ((v + 64) & 127) - 64;
    dg[p] = (uint16_t)oz_bf16((int)d);
    v = (v - d) >> 7;
  }
  dg[0] = (uint16_t)oz_bf16((int)v);
}

// xsl[(p kpad + r) ldx + i]: digit p of round(x_ir 2^(7 ND - e_r))
template <int ND>
__global__ void __launch_bounds__(256) k_oz_slice_x(const double* __restrict__ x, int64_t N, int k, int kpad,
                                                    int64_t ldx, const int32_t* __restrict__ xexp,
                                                    uint16_t* __restrict__ xsl) {
  const int64_t nk = N * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / N);
    const int64_t i = e % N;  // consecutive threads: consecutive rows of one column (coalesced digit stores)
    const int ex = xexp[r];
    uint16_t dg[ND];
    oz_digits<ND>(ex == kOzBadExp ? 0 : oz_fixed_d(x[i * k + r], 7 * ND - ex), dg);
#pragma unroll
    for (int p = 0; p < ND; ++p) xsl[((int64_t)p * kpad + r) * ldx + i] = dg[p];
  }
}

// The skeleton vectors t_a of the nodes of a level (Vt[(node s_max + q) k + r],
// q < rank[node]) as digits for the row updates: per node and column a scale
// 2^e (xexp[nl k + r]) and xsl[(p kpad + r) ldx + nl s_pad + q].  One CTA a
// node; smem: k keys.
template <int ND>
__global__ void __launch_bounds__(256) k_oz_slice_t(const int32_t* __restrict__ rank, int node0, int s_max,
                                                    int s_pad, const double* __restrict__ Vt, int k, int kpad,
                                                    int64_t ldx, int32_t* __restrict__ xexp,
                                                    uint16_t* __restrict__ xsl) {
  extern __shared__ unsigned long long tmx[];
  const int nl = blockIdx.x, node = node0 + nl, sa = rank[node];
  for (int r = threadIdx.x; r < k; r += blockDim.x) tmx[r] = 0ull;
  __syncthreads();
  const double* T = Vt + (int64_t)node * s_max * k;
  for (int e = threadIdx.x; e < sa * k; e += blockDim.x) atomicMax(&tmx[e % k], oz_key(T[e]));
  __syncthreads();
  for (int r = threadIdx.x; r < k; r += blockDim.x) xexp[(int64_t)nl * k + r] = oz_exp_of(tmx[r]);
  __syncthreads();
  for (int e = threadIdx.x; e < sa * k; e += blockDim.x) {
    const int q = e / k, r = e % k;
    const int ex = xexp[(int64_t)nl * k + r];
    uint16_t dg[ND];
    oz_digits<ND>(ex == kOzBadExp ? 0 : oz_fixed_d(T[e], 7 * ND - ex), dg);
#pragma unroll
    for (int p = 0; p < ND; ++p) xsl[((int64_t)p * kpad + r) * ldx + (int64_t)nl * s_pad + q] = dg[p];
  }
}

// ---- factorization: row-scaled digit tiles of the leaves' P (operator) ----------
// rexp[i] = e with 2^e > max_{q < rank[node]} |M[i][q]| for the rows of the
// nodes of a level; one warp a row
__global__ void __launch_bounds__(256) k_oz_row_exp(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                    const int32_t* __restrict__ rank, int node0, int s_max,
                                                    const double* __restrict__ M, int32_t* __restrict__ rexp) {
  const int node = node0 + blockIdx.y, b = lo[node], n = hi[node] - b, sa = rank[node];
  const int lane = threadIdx.x & 31;
  for (int i = blockIdx.x * 8 + (threadIdx.x >> 5); i < n; i += gridDim.x * 8) {
    unsigned long long m = 0ull;
    for (int q = lane; q < sa; q += 32) m = max(m, oz_key(M[(int64_t)(b + i) * s_max + q]));
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) rexp[b + i] = oz_exp_of(m);
  }
}

// tiles (window of the level's rows, skeleton window, digit): element (m =
// row in the window, k = skeleton in the window), K-major as the V tiles;
// grid = (windows of the largest node, nodes, skeleton windows)
template <int ND>
__global__ void __launch_bounds__(256) k_oz_slice_rows(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                       const int32_t* __restrict__ rank, int node0, int s_max,
                                                       int qw, const double* __restrict__ M,
                                                       const int32_t* __restrict__ rexp,
                                                       const int32_t* __restrict__ wbase, uint16_t* __restrict__ tiles) {
  const int nl = blockIdx.y, node = node0 + nl, w = blockIdx.x, t = blockIdx.z;
  const int b = lo[node], n = hi[node] - b, sa = rank[node];
  if (w * kOzWin >= n) return;
  uint16_t* base = tiles + ((int64_t)(wbase[nl] + w) * qw + t) * ND * kOzTileElems;
  for (int item = threadIdx.x; item < kOzWin * (kOzQ / 8); item += blockDim.x) {
    const int kg = item % (kOzQ / 8), m = item / (kOzQ / 8);
    const int i = w * kOzWin + m;
    const int ex = i < n ? rexp[b + i] : 0;
    uint32_t pk[ND][4];
#pragma unroll
    for (int p = 0; p < ND; ++p) pk[p][0] = pk[p][1] = pk[p][2] = pk[p][3] = 0u;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int q = t * kOzQ + kg * 8 + jj;
      int64_t v = 0;
      if (i < n && q < sa && ex != kOzBadExp) v = oz_fixed_d(M[(int64_t)(b + i) * s_max + q], 7 * ND - ex);
      uint16_t dg[ND];
      oz_digits<ND>(v, dg);
#pragma unroll
      for (int p = 0; p < ND; ++p) pk[p][jj >> 1] |= (uint32_t)dg[p] << (16 * (jj & 1));
    }
    const int off = ((m >> 3) * 16 + kg) * 64 + (m & 7) * 8;
#pragma unroll
    for (int p = 0; p < ND; ++p)
      *(uint4*)(base + (int64_t)p * kOzTileElems + off) = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
  }
}

// P_c of every internal node a (FP64, rows i < s_l + s_r of (2 s_max) x s_max
// blocks, columns q < s_a) as row-scaled digit tiles: rexp[a 2 s_max + i] and
// tiles (node, row window, skeleton window, digit); grid = (row windows,
// internal nodes 1 .. 2^D - 1, skeleton windows)
template <int ND>
__global__ void __launch_bounds__(256) k_oz_slice_pc(const int32_t* __restrict__ rank, int s_max, int rw, int qw,
                                                     const double* __restrict__ Pc, int32_t* __restrict__ rexp,
                                                     uint16_t* __restrict__ tiles) {
  const int node = 1 + blockIdx.y, w = blockIdx.x, t = blockIdx.z;
  const int z = rank[2 * node] + rank[2 * node + 1], sa = rank[node];
  if (w * kOzWin >= z || t * kOzQ >= sa) return;
  const double* M = Pc + (int64_t)node * 2 * s_max * s_max;
  // every CTA of a row window forms its rows' exponents (cheap; no order between CTAs needed)
  __shared__ int ex_s[kOzWin];
  const int lane = threadIdx.x & 31;
  for (int m = threadIdx.x >> 5; m < kOzWin; m += blockDim.x >> 5) {
    const int i = w * kOzWin + m;
    unsigned long long key = 0ull;
    if (i < z)
      for (int q = lane; q < sa; q += 32) key = max(key, oz_key(M[(int64_t)i * s_max + q]));
    for (int off = 16; off > 0; off >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, off));
    if (lane == 0) {
      ex_s[m] = oz_exp_of(key);
      if (t == 0 && i < z) rexp[(int64_t)node * 2 * s_max + i] = ex_s[m];
    }
  }
  __syncthreads();
  uint16_t* base = tiles + (((int64_t)node * rw + w) * qw + t) * ND * kOzTileElems;
  for (int item = threadIdx.x; item < kOzWin * (kOzQ / 8); item += blockDim.x) {
    const int kg = item % (kOzQ / 8), m = item / (kOzQ / 8);
    const int i = w * kOzWin + m;
    const int ex = ex_s[m];
    uint32_t pk[ND][4];
#pragma unroll
    for (int p = 0; p < ND; ++p) pk[p][0] = pk[p][1] = pk[p][2] = pk[p][3] = 0u;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int q = t * kOzQ + kg * 8 + jj;
      int64_t v = 0;
      if (i < z && q < sa && ex != kOzBadExp) v = oz_fixed_d(M[(int64_t)i * s_max + q], 7 * ND - ex);
      uint16_t dg[ND];
      oz_digits<ND>(v, dg);
#pragma unroll
      for (int p = 0; p < ND; ++p) pk[p][jj >> 1] |= (uint32_t)dg[p] << (16 * (jj & 1));
    }
    const int off = ((m >> 3) * 16 + kg) * 64 + (m & 7) * 8;
#pragma unroll
    for (int p = 0; p < ND; ++p)
      *(uint4*)(base + (int64_t)p * kOzTileElems + off) = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
  }
}

// ---- the tensor-core passes ----------------------------------------------------
// 7 digits per operand: the digit pairs p + q <= 7 in 8 groups (a zero tile
// after the x digit d_6 clears group 7, which has no pair with p = 0)
constexpr int kOzGroups = 8;

template <int NC>
struct OzCfg {
  static_assert(NC == 16 || NC == 32, "column group");
  static constexpr int kGroups = kOzGroups;
  static constexpr int kStages = NC == 16 ? 4 : 3;             // A digit tiles in flight
  static constexpr int kBBytes = kGroups * NC * kOzWin * 2;    // x digits of one window (+ zero tiles)
  static constexpr int kSmem = kStages * kOzTileBytes + 2 * kBBytes;
  static constexpr int kAccCols = kGroups * NC;                // one buffer of group sums
  static constexpr uint32_t kTmemCols = 2 * kAccCols <= 256 ? 256u : 512u;
};

enum { kOzColsum = 0, kOzLeaf = 1, kOzRowupd = 2, kOzPush = 3 };

// MODE kOzColsum (V passes): grid = (1024-row chunks of the largest node,
// nodes, skeleton tiles x column groups); CTA (ch, node, t) sums rows
// 1024 ch .. of the node against skeleton columns 128 t .. of its sibling:
// partial sums into parts.
// MODE kOzLeaf (leaves of at most 1024 points): grid = (1, leaves, row
// tiles x column groups); CTA (0, leaf, t) forms rows 128 t .. of
// y = lambda x + K_aa x over all of the leaf's columns.
// MODE kOzRowupd (the row update y_i += sign P_i g_a of the leaves, P's rows
// scaled by 2^rexp[i]): grid = (1, leaves, row windows x column groups); CTA
// (0, leaf, t) updates rows 128 t .. of the leaf from its skeleton weights
// g_a (digits per leaf and column, scales 2^xexp[leaf k + r]); its skeleton
// windows of 128 are read out like the V pass's row windows.
// MODE kOzPush (the operator's push through P_c: g_children += P_c g_a for
// the nodes a of a level, P_c's rows scaled by 2^rexp[a 2 s_max + i]): grid =
// (1, nodes, row windows of P_c x column groups); CTA (0, a, t) forms rows
// 128 t .. of P_c g_a, row i landing in slot i of the left child (i < s_l)
// or slot i - s_l of the right one.
template <int NC, int MODE, typename TY>
__global__ void __launch_bounds__(kOzThreads, 1)
    k_oz(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, const int32_t* __restrict__ rank,
         int node0, int s_max, int qt, const uint16_t* __restrict__ Asl, const int32_t* __restrict__ wbase,
         const uint16_t* __restrict__ xsl, int64_t ldx, int kpad, const int32_t* __restrict__ xexp, int k,
         int nchunk, double* __restrict__ parts, double lambda, const double* __restrict__ x, TY* __restrict__ y,
         const int32_t* __restrict__ rexp, double sign, int32_t* __restrict__ status) {
  using C = OzCfg<NC>;
  constexpr int ST = C::kStages, G = C::kGroups, ND = kOzSlices;
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  __shared__ __align__(8) uint64_t a_full[ST], a_empty[ST], b_full[2], b_empty[2], acc_full[2], acc_empty[2], done;
  __shared__ uint32_t tmem_base;
  const int nl = blockIdx.y, node = node0 + nl, sib = node ^ 1;
  const int b = lo[node], n = hi[node] - b;
  // rows of the product (M): skeletons of the sibling, points, or P_c's rows
  const int cnt = MODE == kOzColsum ? rank[sib] : (MODE == kOzPush ? rank[2 * node] + rank[2 * node + 1] : n);
  const int t = blockIdx.z % qt, c0 = (blockIdx.z / qt) * NC;
  const int ch = blockIdx.x, w0 = ch * kOzWinPerChunk;
  constexpr bool kSkel = MODE == kOzRowupd || MODE == kOzPush;  // contraction over the node's skeletons
  const int s_a = kSkel ? rank[node] : 0;
  const int nw = kSkel ? (s_a + kOzWin - 1) / kOzWin : min(kOzWinPerChunk, (n + kOzWin - 1) / kOzWin - w0);
  if (nw <= 0 || cnt <= t * kOzQ || c0 >= k) return;  // uniform over the CTA
  const int s_pad = (s_max + kOzWin - 1) / kOzWin * kOzWin;
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
  const int nunits = nw * ND;  // (window, A digit) pairs, in order
  if (warp == 0) {
    // bulk copies of the A digit tiles.  V: (window of the level, skeleton
    // tile); leaf blocks: (leaf, row tile, window); row updates: (row window
    // of the level, skeleton window); 7 digit tiles each
    if (lane == 0) {
      const uint16_t* tiles;
      int64_t wstride;
      if (MODE == kOzColsum) {
        tiles = Asl + ((int64_t)(wbase[nl] + w0) * qt + t) * kOzSlices * kOzTileElems;
        wstride = (int64_t)qt * kOzSlices * kOzTileElems;
      } else if (MODE == kOzLeaf) {
        tiles = Asl + ((int64_t)nl * qt + t) * qt * kOzSlices * kOzTileElems;
        wstride = (int64_t)kOzSlices * kOzTileElems;
      } else if (MODE == kOzRowupd) {
        tiles = Asl + (int64_t)(wbase[nl] + t) * (s_pad / kOzWin) * ND * kOzTileElems;
        wstride = (int64_t)ND * kOzTileElems;
      } else {  // P_c of node a: (node, row window, skeleton window) tiles, qt row windows a node
        tiles = Asl + ((int64_t)node * qt + t) * (s_pad / kOzWin) * ND * kOzTileElems;
        wstride = (int64_t)ND * kOzTileElems;
      }
      for (int u = 0; u < nunits; ++u) {
        const int st = u % ST;
        if (u >= ST && !mbar_wait(&a_empty[st], (uint32_t)((u / ST) - 1) & 1u)) {
          atomicOr(status, KF_DEV_TIMEOUT);
          break;
        }
        mbar_arrive_expect_tx(&a_full[st], kOzTileBytes);
        bulk_g2s(As + st * kOzTileElems, tiles + (u / ND) * wstride + (int64_t)(u % ND) * kOzTileElems, kOzTileBytes,
                 &a_full[st]);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // MMAs: per window and A digit p one chain with B = x digits d_0 .. into
    // the accumulator columns from group p on (pair (p, q) -> group p + q)
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
        for (int p = 0; p < ND; ++p) {
          const int u = w * ND + p, st = u % ST;
          if (!(ok = mbar_wait(&a_full[st], (uint32_t)(u / ST) & 1u))) break;
          fence_after_sync();
          const uint32_t as = smem_u32(As + st * kOzTileElems);
          // p = 0: every group (overwritten; the zero tile for group 7);
          // p >= 1: groups p .. 7 (accumulated)
          const int nq = p == 0 ? G : min(ND, G - p);
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
        *(uint4*)(Bs + bb * (C::kBBytes / 2) + ND * NC * kOzWin + e * 8) = make_uint4(0u, 0u, 0u, 0u);
    for (int w = 0; w < nw; ++w) {
      const int buf = w & 1;
      if (w >= 2 && !mbar_wait(&b_empty[buf], (uint32_t)((w >> 1) - 1) & 1u)) {
        atomicOr(status, KF_DEV_TIMEOUT);
        break;
      }
      // rows of x (V, leaf: the node's rows of the window) or of t_a (row updates: skeletons)
      int64_t i0;
      int nr;
      if (kSkel) {
        i0 = (int64_t)nl * s_pad + w * kOzWin;
        nr = min(kOzWin, s_a - w * kOzWin);
      } else {
        const int ib = (w0 + w) * kOzWin;
        i0 = (int64_t)b + ib;
        nr = min(kOzWin, n - ib);
      }
      uint16_t* B = Bs + buf * (C::kBBytes / 2);
      for (int e = sid; e < ND * NC * (kOzWin / 8); e += 64) {
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
    // read-out: thread = accumulator row t*128 + 32 (warp % 4) + lane
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
      for (int g = 0; g < G; ++g) {
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
    // value = 2^e (2^-35 hi + 2^-63 lo): e = the x column's exponent (plus the row's)
    const int q = t * kOzQ + quad * 32 + lane;
    if (ok && q < cnt) {
      int64_t row = (int64_t)b + q;
      if (MODE == kOzPush) {  // P_c's row q: a slot of the left or the right child
        const int sl = rank[2 * node];
        row = q < sl ? (int64_t)(2 * node) * s_max + q : (int64_t)(2 * node + 1) * s_max + (q - sl);
      }
      const int rx = MODE == kOzRowupd ? rexp[(int64_t)b + q] : (MODE == kOzPush ? rexp[(int64_t)node * 2 * s_max + q] : 0);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int col = c0 + c;
        if (col >= k) break;
        const int ex = kSkel ? xexp[(int64_t)nl * k + col] : xexp[col];
        const double v = ex == kOzBadExp ? __longlong_as_double(0x7FF8000000000000ll)
                                         : ldexp((double)hi64[c], ex + rx - 35) + ldexp((double)lo64[c], ex + rx - 63);
        if (MODE == kOzColsum)
          parts[(((int64_t)nl * nchunk + ch) * s_max + q) * k + col] = v;
        else if (MODE == kOzLeaf)
          y[row * k + col] = (TY)(lambda * x[row * k + col] + v);
        else
          y[row * k + col] = (TY)((double)y[row * k + col] + sign * v);
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
  // row-scaled digits of the leaves' P (7 digits)
  const int qw = (f->s_max + kOzWin - 1) / kOzWin;
  auto grab = [&](size_t bytes) -> void* {
    void* m = f->ctx->dalloc(bytes, s);
    if (m) f->allocs.push_back({m, bytes});
    else cudaGetLastError();
    return m;
  };
  int64_t wD = 0;
  for (int a = 1 << D; a < (2 << D); ++a) wD += (t->hi[a] - t->lo[a] + kOzWin - 1) / kOzWin;
  f->PLsl = (uint16_t*)grab(sizeof(uint16_t) * (size_t)wD * qw * 7 * kOzTileElems);
  f->PLrexp = f->PLsl ? (int32_t*)grab(sizeof(int32_t) * (size_t)t->N) : nullptr;
  if (!f->PLrexp) f->PLsl = nullptr;
  // P_c of the internal nodes (7 digits, rows scaled), for the operator's pushes
  if (D >= 2) {
    const int rw = (2 * f->s_max + kOzWin - 1) / kOzWin;
    f->PCsl = (uint16_t*)grab(sizeof(uint16_t) * ((size_t)1 << D) * rw * qw * 7 * kOzTileElems);
    f->PCrexp = f->PCsl ? (int32_t*)grab(sizeof(int32_t) * ((size_t)1 << D) * 2 * f->s_max) : nullptr;
    if (!f->PCrexp) f->PCsl = nullptr;
  }
  return KF_OK;
}

// row exponents and digit tiles of one matrix M (point-major N x s_max) over
// the rows of the nodes of level lv
void oz_rows_level(kf_factor* f, int lv, const double* M, int32_t* rexp, uint16_t* tiles, cudaStream_t s) {
  kf_tree* t = f->t;
  const int qw = (f->s_max + kOzWin - 1) / kOzWin;
  int maxn = 0;
  for (int a = 1 << lv; a < (2 << lv); ++a) maxn = std::max(maxn, t->hi[a] - t->lo[a]);
  if (maxn == 0) return;
  dim3 ge((unsigned)std::min(64, (maxn + 7) / 8), 1u << lv);
  KF_PHASE(KF_PH_MISC, s, k_oz_row_exp<<<ge, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, 1 << lv, f->s_max, M, rexp));
  dim3 g((unsigned)((maxn + kOzWin - 1) / kOzWin), 1u << lv, (unsigned)qw);
  KF_PHASE(KF_PH_MISC, s, k_oz_slice_rows<kOzSlices><<<g, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, 1 << lv, f->s_max, qw,
                                                                    M, rexp, f->oz_wbase + (1 << lv), tiles));
}

// the row-scaled digits of the leaves' P, once the factorization is complete
kf_status kf_oz_slice_rows(kf_factor* f, cudaStream_t s) {
  kf_tree* t = f->t;
  const int D = t->D;
  if (D == 0 || !f->oz_wbase) return KF_OK;
  if (f->PLsl) oz_rows_level(f, D, f->Pleaf, f->PLrexp, f->PLsl, s);
  if (f->PCsl) {  // and P_c of the internal nodes that push (levels 1 .. D-1; node 1 is sliced too)
    const int rw = (2 * f->s_max + kOzWin - 1) / kOzWin, qw = (f->s_max + kOzWin - 1) / kOzWin;
    dim3 g((unsigned)rw, (unsigned)((1 << D) - 1), (unsigned)qw);
    KF_PHASE(KF_PH_MISC, s, k_oz_slice_pc<kOzSlices><<<g, 256, 0, s>>>(f->rank, f->s_max, rw, qw, f->Pc, f->PCrexp,
                                                                        f->PCsl));
  }
  KF_LAUNCH_CHECK(f->ctx);
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

// x of one operator call (N x k point-major) as 7 digits a column
kf_status kf_oz_prepare_x(kf_factor* f, const double* x, int64_t k, kf_oz_x* oz, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  const int64_t N = f->t->N;
  oz->k = k;
  oz->nc = k > 16 ? 32 : 16;
  oz->kpad = (int)((k + oz->nc - 1) / oz->nc) * oz->nc;
  oz->ldx = (N + 7) / 8 * 8;
  oz->bytes = sizeof(uint16_t) * (size_t)kOzSlices * oz->kpad * oz->ldx;
  oz->nexp = k;
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
  KF_PHASE(KF_PH_MV_COLSUM, s, k_oz_slice_x<kOzSlices><<<grid_for(N * k, 256), 256, 0, s>>>(
                                   x, N, (int)k, oz->kpad, oz->ldx, oz->xexp, oz->xsl));
  KF_LAUNCH_CHECK(c);
  return KF_OK;
}

// the skeleton weights of the nodes of level lv (Vt, by node) as 7 digits for
// a row update
kf_status kf_oz_prepare_t(kf_factor* f, int lv, const double* Vt, int64_t k, kf_oz_x* oz, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  const int nodes = 1 << lv, s_pad = (f->s_max + kOzWin - 1) / kOzWin * kOzWin;
  oz->k = k;
  oz->nc = k > 16 ? 32 : 16;
  oz->kpad = (int)((k + oz->nc - 1) / oz->nc) * oz->nc;
  oz->ldx = (int64_t)nodes * s_pad;
  oz->bytes = sizeof(uint16_t) * (size_t)kOzSlices * oz->kpad * oz->ldx;
  oz->nexp = (int64_t)nodes * k;
  oz->xsl = (uint16_t*)c->dalloc(oz->bytes, s);
  oz->xexp = (int32_t*)c->dalloc(sizeof(int32_t) * (size_t)oz->nexp, s);
  if (!oz->xsl || !oz->xexp) {
    kf_oz_release_x(f, oz, s);
    return kf_set_err(c, KF_ENOMEM, "matvec: allocation of the skeleton-weight digits failed");
  }
  KF_CUDA(c, cudaMemsetAsync(oz->xsl, 0, oz->bytes, s));
  const int smx = (int)(sizeof(unsigned long long) * (size_t)k);
  KF_PHASE(KF_PH_MV_ROWUPD, s, k_oz_slice_t<kOzSlices><<<nodes, 256, smx, s>>>(
                                   f->rank, nodes, f->s_max, s_pad, Vt, (int)k, oz->kpad, oz->ldx, oz->xexp, oz->xsl));
  KF_LAUNCH_CHECK(c);
  return KF_OK;
}

void kf_oz_release_x(kf_factor* f, kf_oz_x* oz, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  if (oz->xsl) c->dfree(oz->xsl, oz->bytes, s);
  if (oz->xmax) c->dfree(oz->xmax, sizeof(unsigned long long) * (size_t)oz->k, s);
  if (oz->xexp) c->dfree(oz->xexp, sizeof(int32_t) * (size_t)oz->nexp, s);
  *oz = kf_oz_x{};
}

template <int NC, int MODE, typename TY>
kf_status oz_launch(kf_factor* f, dim3 g, int phase, cudaStream_t s, int node0, int qt, const uint16_t* Asl,
                    const int32_t* wb, const uint16_t* xsl, int64_t ldx, int kpad, const int32_t* xexp, int k,
                    int nchunk, double* parts, double lambda, const double* x, TY* y, const int32_t* rexp,
                    double sign) {
  kf_tree* t = f->t;
  using C = OzCfg<NC>;
  KF_CUDA(f->ctx, cudaFuncSetAttribute(k_oz<NC, MODE, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem));
  KF_PHASE(phase, s, k_oz<NC, MODE, TY><<<g, kOzThreads, C::kSmem, s>>>(
                         t->d_lo, t->d_hi, f->rank, node0, f->s_max, qt, Asl, wb, xsl, ldx, kpad, xexp, k, nchunk,
                         parts, lambda, x, y, rexp, sign, f->status));
  KF_LAUNCH_CHECK(f->ctx);
  return KF_OK;
}

// The V pass of level l: FP64 partial sums of 1024-row chunks into parts
// (the layout of k_colsum's, nchunk chunks a node); the caller reduces them.
// oz.nd = 7: the FP64-accurate operator; 4: the FP32 sweep.
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
#define OZ_ARGS g, KF_PH_MV_COLSUM, s, 1 << l, qt, Asl, wb, oz.xsl, oz.ldx, oz.kpad, oz.xexp, (int)k, nch, parts, 0.0, \
                nullptr, (double*)nullptr, nullptr, 0.0
  if (oz.nc == 16) return oz_launch<16, kOzColsum, double>(f, OZ_ARGS);
  return oz_launch<32, kOzColsum, double>(f, OZ_ARGS);
#undef OZ_ARGS
}

// Leaf blocks: y = lambda x + K_aa x for every leaf (x, y: N x k, tree order)
kf_status kf_oz_leaf(kf_factor* f, const kf_oz_x& oz, int64_t k, double lambda, const double* x, double* y,
                     cudaStream_t s) {
  kf_tree* t = f->t;
  const int tpl = (t->leaf_max + kOzQ - 1) / kOzQ;
  dim3 g(1u, 1u << t->D, (unsigned)(tpl * (oz.kpad / oz.nc)));
#define OZ_ARGS g, KF_PH_MV_LEAF, s, 1 << t->D, tpl, f->Ksl, nullptr, oz.xsl, oz.ldx, oz.kpad, oz.xexp, (int)k, 1, \
                nullptr, lambda, x, y, nullptr, 0.0
  if (oz.nc == 16) return oz_launch<16, kOzLeaf, double>(f, OZ_ARGS);
  return oz_launch<32, kOzLeaf, double>(f, OZ_ARGS);
#undef OZ_ARGS
}

// The operator's row update of the leaves from their skeleton weights (digits
// in td): y += sign P g (7 digits of the leaves' P)
kf_status kf_oz_rowupd(kf_factor* f, const kf_oz_x& td, int64_t k, double* y, double sign, cudaStream_t s) {
  kf_tree* t = f->t;
  const int lv = t->D;
  int maxn = 0;
  for (int a = 1 << lv; a < (2 << lv); ++a) maxn = std::max(maxn, t->hi[a] - t->lo[a]);
  const int nwin = std::max(1, (maxn + kOzWin - 1) / kOzWin);
  dim3 g(1u, 1u << lv, (unsigned)(nwin * (td.kpad / td.nc)));
  const int32_t* wb = f->oz_wbase + (1 << lv);
#define OZ_ARGS g, KF_PH_MV_ROWUPD, s, 1 << lv, nwin, f->PLsl, wb, td.xsl, td.ldx, td.kpad, td.xexp, (int)k, 1, \
                nullptr, 0.0, nullptr, y, f->PLrexp, sign
  if (td.nc == 16) return oz_launch<16, kOzRowupd, double>(f, OZ_ARGS);
  return oz_launch<32, kOzRowupd, double>(f, OZ_ARGS);
#undef OZ_ARGS
}

// The operator's push of level lv: g_children += P_c g_a for the nodes a of
// level lv (skeleton weights of the nodes by node in G; digits of g_a in td)
kf_status kf_oz_push(kf_factor* f, int lv, const kf_oz_x& td, int64_t k, double* G, cudaStream_t s) {
  const int rw = (2 * f->s_max + kOzWin - 1) / kOzWin;
  dim3 g(1u, 1u << lv, (unsigned)(rw * (td.kpad / td.nc)));
#define OZ_ARGS g, KF_PH_MV_PUSH, s, 1 << lv, rw, f->PCsl, nullptr, td.xsl, td.ldx, td.kpad, td.xexp, (int)k, 1, \
                nullptr, 0.0, nullptr, G, f->PCrexp, 1.0
  if (td.nc == 16) return oz_launch<16, kOzPush, double>(f, OZ_ARGS);
  return oz_launch<32, kOzPush, double>(f, OZ_ARGS);
#undef OZ_ARGS
}
