// skel.cu -- skeletonization (Algorithm 1) with the interpolative
// decomposition of Eq. e:id on sampled rows S' (Sec. II-A).
//
// For each level from the leaves up, every node of the level at once:
//  1. S' : n_s = min(N - |a|, n_samp) distinct complement positions drawn with
//     the counter-based splitmix64 (draw j: splitmix64(seed ^ (node << 32) ^ j)
//     mod (N - |a|), duplicates skipped, mapped past the node's range), sorted;
//     the whole complement when it is not larger than n_samp.
//  2. A = K(S', C) in FP64 (C = the node's points at a leaf, [l~ r~] above).
//  3. Column-pivoted Householder QR of A (one CTA per node), stopping at the
//     first k with |R_kk| < tau |R_00| or at min(s_max, n_s, |C|); the squared
//     norms of the trailing columns are downdated by each new row of R and
//     evaluated exactly again whenever they have fallen 16x since their last
//     exact value, so they stay within rounding of the recomputed norms.
//  4. P = [I, R11^-1 R12] with the columns in their original order.
#include <cooperative_groups.h>

#include <algorithm>

#include "kf_internal.cuh"
#include "prof.cuh"

namespace {

// ---- 1. sampling: one warp per node ------------------------------------------
// With near-field sampling (near_pos != nullptr) the first min(list length,
// floor(n_s / 2)) entries of the node's near list are accepted before the
// draws, which then also skip them (knn.cu).
__global__ void k_sample(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, int64_t N, int node0,
                         int nn, int n_samp, uint64_t seed, const int32_t* __restrict__ near_pos,
                         const int32_t* __restrict__ near_len, int near_cap, int32_t* __restrict__ samp,
                         int32_t* __restrict__ ns_out, int32_t* __restrict__ status) {
  extern __shared__ int32_t acc[];  // n_samp accepted candidates
  int nl = blockIdx.x;
  if (nl >= nn) return;
  int node = node0 + nl;
  int lane = threadIdx.x;
  int64_t b = lo[node], sz = hi[node] - b, M = N - sz;
  int64_t ns = M < n_samp ? M : n_samp;
  int32_t* out = samp + (int64_t)nl * n_samp;
  if (ns == M) {  // whole complement, already ascending
    for (int64_t t = lane; t < ns; t += 32) out[t] = (int32_t)(t < b ? t : t + sz);
    if (lane == 0) ns_out[nl] = (int32_t)ns;
    return;
  }
  int got = 0;
  if (near_pos) {  // near entries first, as complement indices (the draws' space)
    const int n1 = (int)((int64_t)near_len[node] < ns / 2 ? (int64_t)near_len[node] : ns / 2);
    for (int t = lane; t < n1; t += 32) {
      const int32_t p = near_pos[(int64_t)node * near_cap + t];
      acc[t] = (int32_t)(p < b ? p : p - sz);
    }
    got = n1;
    __syncwarp();
  }
  // bounded: with n_s < N - |a| distinct values exist; the cap only guards
  // against a generator defect and flags it instead of spinning
  for (uint64_t j0 = 0; got < ns; j0 += 32) {
    if (j0 > (1ull << 30)) {
      if (lane == 0) atomicOr(status, KF_DEV_TIMEOUT);
      break;
    }
    uint64_t u = kf_splitmix64(seed ^ ((uint64_t)node << 32) ^ (j0 + lane));
    int32_t cand = (int32_t)(u % (uint64_t)M);
    bool dup = false;
    for (int t = 0; t < got; ++t) dup |= (acc[t] == cand);
    // accept in draw order; a candidate equal to an earlier accepted lane of
    // this round is a duplicate as well
    bool mine_acc = false;
    for (int t = 0; t < 32 && got < ns; ++t) {
      int32_t ct = __shfl_sync(0xffffffffu, cand, t);
      bool dt = __shfl_sync(0xffffffffu, dup, t);
      unsigned same = __ballot_sync(0xffffffffu, mine_acc && cand == ct && lane < t);
      if (!dt && same == 0) {
        if (lane == 0) acc[got] = ct;
        if (lane == t) mine_acc = true;
        ++got;
      }
    }
    __syncwarp();
  }
  ns = got;
  // map and rank-sort (values are distinct)
  for (int t = lane; t < ns; t += 32) {
    int32_t v = acc[t];
    int r = 0;
    for (int q = 0; q < ns; ++q) r += acc[q] < v;
    out[r] = (int32_t)(v < b ? v : v + sz);
  }
  if (lane == 0) ns_out[nl] = (int32_t)ns;
}

// ID columns of node a: position of column j.
__device__ __forceinline__ int32_t id_col(int node, bool leaf, const int32_t* lo, const int32_t* rank,
                                          const int32_t* skel, int s_max, int j) {
  if (leaf) return lo[node] + j;
  int sl = rank[2 * node];
  return j < sl ? skel[(int64_t)(2 * node) * s_max + j] : skel[(int64_t)(2 * node + 1) * s_max + (j - sl)];
}

__device__ __forceinline__ int id_ncols(int node, bool leaf, const int32_t* lo, const int32_t* hi, const int32_t* rank) {
  return leaf ? hi[node] - lo[node] : rank[2 * node] + rank[2 * node + 1];
}

// ---- 2. A = K(S', C), column-major, ld = n_samp ---------------------------------
__global__ void k_eval_A(const double* __restrict__ X, int d, double c_exp, const int32_t* __restrict__ lo,
                         const int32_t* __restrict__ hi, const int32_t* __restrict__ rank,
                         const int32_t* __restrict__ skel, int s_max, int node0, bool leaf, int n_samp, int cmax,
                         const int32_t* __restrict__ samp, const int32_t* __restrict__ nsamp, double* __restrict__ A) {
  int nl = blockIdx.z, node = node0 + nl;
  int c = id_ncols(node, leaf, lo, hi, rank);
  int ns = nsamp[nl];
  int j = blockIdx.y;
  if (j >= c) return;
  int32_t col = id_col(node, leaf, lo, rank, skel, s_max, j);
  const double* xc = X + (int64_t)col * d;
  double* Aj = A + ((int64_t)nl * cmax + j) * n_samp;
  const int32_t* S = samp + (int64_t)nl * n_samp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x)
    Aj[i] = kf_kern64(X + (int64_t)S[i] * d, xc, d, c_exp);
}

// T = R11^-1 R12 in place over R12 (rows 0..s-1 of the columns s..c-1 of the
// factored block Ab, column-major with stride n_samp), by 32-row blocks from
// the bottom: the upper-triangular diagonal block is staged in shared memory
// (reciprocal pivots formed once) and solved with shuffles, a warp per column;
// the rows above are then updated for all columns at once by 64 x 64 FP64
// tiles staged in shared memory (thread: 4 consecutive rows x 2 columns, so
// that a warp's stores to the column-major block are contiguous).
struct IdSolveShared {
  double du[32][33];
  double rd[32];
  double ta[32][64];  // R11[ti + r][kb + t] at [t][r]
  double tb[32][65];  // X[kb + t][tj + j] at [t][j]
};

__device__ void id_solve_t(double* __restrict__ Ab, int n_samp, int s, int c, IdSolveShared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int nc = c - s;
  if (s == 0 || nc <= 0) return;
  const int tx = tid & 15, ty = tid >> 4;  // 16 x (blockDim / 16)
  const int nty = blockDim.x >> 4;
  for (int kb = ((s - 1) / 32) * 32; kb >= 0; kb -= 32) {
    const int nb = min(32, s - kb);
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
      const int i = e & 31, t = e >> 5;
      sh.du[i][t] = (i < nb && t < nb && i <= t) ? Ab[(int64_t)(kb + t) * n_samp + kb + i] : 0.0;
    }
    __syncthreads();
    if (tid < 32) sh.rd[tid] = tid < nb ? 1.0 / sh.du[tid][tid] : 0.0;
    __syncthreads();
    for (int jj = warp; jj < nc; jj += nw) {
      double* col = Ab + (int64_t)(s + jj) * n_samp + kb;
      double bi = lane < nb ? col[lane] : 0.0;
      for (int t = nb - 1; t >= 0; --t) {
        if (lane == t) bi *= sh.rd[t];
        const double xt = __shfl_sync(0xffffffffu, bi, t);
        if (lane < t) bi = fma(-sh.du[lane][t], xt, bi);
      }
      if (lane < nb) col[lane] = bi;
    }
    __syncthreads();
    // rows above: X[0:kb, :] -= R11[0:kb, kb:kb+nb] X[kb:kb+nb, :]
    for (int ti = 0; ti < kb; ti += 64)
      for (int tj = 0; tj < nc; tj += 2 * nty) {
        for (int e = tid; e < 32 * 64; e += blockDim.x) {
          const int r = e & 63, t = e >> 6;
          sh.ta[t][r] = (ti + r < kb && t < nb) ? Ab[(int64_t)(kb + t) * n_samp + ti + r] : 0.0;
          const int t2 = e & 31, j2 = e >> 5;
          if (j2 < 2 * nty) sh.tb[t2][j2] = (t2 < nb && tj + j2 < nc) ? Ab[(int64_t)(s + tj + j2) * n_samp + kb + t2] : 0.0;
        }
        __syncthreads();
        double acc[4][2] = {};
#pragma unroll 8
        for (int t = 0; t < 32; ++t) {
          double av[4], bv[2];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = sh.ta[t][tx * 4 + a];
#pragma unroll
          for (int bq = 0; bq < 2; ++bq) bv[bq] = sh.tb[t][ty * 2 + bq];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int bq = 0; bq < 2; ++bq) acc[a][bq] = fma(av[a], bv[bq], acc[a][bq]);
        }
#pragma unroll
        for (int bq = 0; bq < 2; ++bq) {
          const int j = tj + ty * 2 + bq;
          if (j >= nc) continue;
          double* colj = Ab + (int64_t)(s + j) * n_samp;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = ti + tx * 4 + a;
            if (i < kb) colj[i] -= acc[a][bq];
          }
        }
        __syncthreads();
      }
  }
}

// P, the skeleton list and the rank from the factored block (columns in
// position order, piv[q] = ID column at position q, s = rank):
// P[j * ldP + q]: ID column j, skeleton q.  Leaves write their rows of the
// N x s_max matrix (base lo[node]); internal nodes have fixed-size blocks.
__device__ void id_finish(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                          int32_t* __restrict__ rank, int32_t* __restrict__ skel, int s_max, int node, int nl,
                          bool leaf, int n_samp, int c, double* __restrict__ Ab, const int* piv, int s,
                          double* __restrict__ Pout, int ldP, int64_t P_node_stride, IdSolveShared& ish) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  id_solve_t(Ab, n_samp, s, c, ish);  // R12 now holds T = R11^-1 R12
  __syncthreads();
  double* P = leaf ? Pout + (int64_t)lo[node] * ldP : Pout + (int64_t)nl * P_node_stride;
  for (int j = s + warp; j < c; j += nwarps) {
    const double* tj = Ab + (int64_t)j * n_samp;
    double* Pj = P + (int64_t)piv[j] * ldP;
    for (int q = lane; q < s_max; q += 32) Pj[q] = q < s ? tj[q] : 0.0;
  }
  for (int j = warp; j < s; j += nwarps) {
    double* Pj = P + (int64_t)piv[j] * ldP;
    for (int q = lane; q < s_max; q += 32) Pj[q] = (q == j) ? 1.0 : 0.0;
  }
  // rows of P beyond c (internal nodes: up to 2 s_max) are zero
  if (!leaf)
    for (int j = c + warp; j < 2 * s_max; j += nwarps)
      for (int q = lane; q < s_max; q += 32) P[(int64_t)j * ldP + q] = 0.0;
  if (threadIdx.x == 0) rank[node] = s;
  int32_t* sk = skel + (int64_t)node * s_max;
  for (int q = threadIdx.x; q < s_max; q += blockDim.x)
    sk[q] = q < s ? id_col(node, leaf, lo, rank, skel, s_max, piv[q]) : -1;
}

// ---- 3/4. pivoted QR and P ------------------------------------------------------
// RPL: rows per lane held in registers (n_samp <= 32 * RPL); NT threads
template <int RPL, int NT>
__global__ void __launch_bounds__(NT, 1) k_pivoted_qr(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                    int32_t* __restrict__ rank, int32_t* __restrict__ skel, int s_max,
                                                    int node0, bool leaf, int n_samp, int cmax,
                                                    const int32_t* __restrict__ nsamp, double tau,
                                                    double* __restrict__ A, double* __restrict__ Pout, int ldP,
                                                    int64_t P_node_stride) {
  extern __shared__ double sm[];
  double* norms = sm;                          // cmax
  double* v = norms + cmax;                    // n_samp
  double* nref = v + n_samp;                   // cmax: 1/16 of the norm at its last exact evaluation
  int* piv = (int*)(nref + cmax);              // cmax
  __shared__ double red_v[32];
  __shared__ long long red_k[32];
  __shared__ int red_i[32];
  __shared__ int s_final, step_p;
  __shared__ double step_rkk, step_beta;
  __shared__ bool step_stop;
  const int nl = blockIdx.x, node = node0 + nl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int c = id_ncols(node, leaf, lo, hi, rank);
  const int ns = nsamp[nl];
  double* Ab = A + (int64_t)nl * cmax * n_samp;
  int kmax = min(s_max, min(ns, c));
  // initial squared column norms
  for (int j = warp; j < c; j += nwarps) {
    const double* col = Ab + (int64_t)j * n_samp;
    double acc = 0.0;
    for (int i = lane; i < ns; i += 32) acc = fma(col[i], col[i], acc);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) { norms[j] = acc; nref[j] = acc * 0.0625; }
  }
  for (int j = threadIdx.x; j < c; j += blockDim.x) piv[j] = j;
  if (threadIdx.x == 0) s_final = kmax;
  __syncthreads();
  double r00 = 0.0;
  for (int k = 0; k < kmax; ++k) {
    // pivot: largest trailing norm, ties to the lowest column.  The keys are
    // the norms' bit patterns (non-negative doubles order like their bits;
    // a negative rounding residue counts as 0), compared on the integer
    // pipes; the scalar FP64 work of the step runs in one thread
    long long bv = -1;
    int bi = c;
    for (int j = k + threadIdx.x; j < c; j += blockDim.x) {
      const long long key = max(__double_as_longlong(norms[j]), 0ll);
      if (key > bv) { bv = key; bi = j; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const long long ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { red_k[warp] = bv; red_i[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long b2 = -1;
      int i2 = c;
      for (int w = 0; w < nwarps; ++w)
        if (red_k[w] > b2 || (red_k[w] == b2 && red_i[w] < i2)) { b2 = red_k[w]; i2 = red_i[w]; }
      const double rkk = sqrt(__longlong_as_double(b2));
      if (k == 0) r00 = rkk;
      step_p = i2;
      step_rkk = rkk;
      step_stop = (k == 0) ? (r00 == 0.0) : (rkk < tau * r00);
    }
    __syncthreads();
    const int p = step_p;
    const double rkk = step_rkk;
    const bool stop = step_stop;
    if (stop) {
      if (threadIdx.x == 0) s_final = k;
      break;
    }
    if (p != k) {  // swap columns k and p (all rows) and their bookkeeping
      double* ck = Ab + (int64_t)k * n_samp;
      double* cp = Ab + (int64_t)p * n_samp;
      for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        double t = ck[i]; ck[i] = cp[i]; cp[i] = t;
      }
      if (threadIdx.x == 0) {
        double t = norms[k]; norms[k] = norms[p]; norms[p] = t;
        t = nref[k]; nref[k] = nref[p]; nref[p] = t;
        int ti = piv[k]; piv[k] = piv[p]; piv[p] = ti;
      }
    }
    __syncthreads();
    // Householder vector of column k, rows k..ns-1
    const double* ck = Ab + (int64_t)k * n_samp;
    const double x0 = ck[k];
    const double alpha = (x0 >= 0.0) ? -rkk : rkk;
    double part = 0.0;
    for (int i = k + threadIdx.x; i < ns; i += blockDim.x) {
      double vi = (i == k) ? x0 - alpha : ck[i];
      v[i] = vi;
      part = fma(vi, vi, part);
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    __syncthreads();
    if (lane == 0) red_v[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double vtv = 0.0;
      for (int w = 0; w < nwarps; ++w) vtv += red_v[w];
      step_beta = vtv > 0.0 ? 2.0 / vtv : 0.0;
    }
    __syncthreads();
    const double beta = step_beta;
    const int nr = (ns - k + 31) >> 5;  // 32-row chunks of rows k..ns-1
    // apply H to the trailing columns; their squared norms over rows > k are
    // downdated by the new row-k entry, and evaluated exactly again once they
    // have fallen by 16x since the last exact value (rounding stays near
    // machine precision relative to the current norm).
    // A warp takes the trailing columns two at a time (k+1+2q, k+2+2q), both
    // held in registers (their 2 x RPL independent loads per lane keep enough
    // requests in flight; loading the next pair ahead measured no faster).
    // Every FP64 warp instruction costs the same whatever its active
    // lanes, so the per-column scalar work is shared by the pair: one
    // butterfly reduces both dot products (lanes 0-15 end with the first
    // column's, lanes 16-31 with the second's), one multiply forms both
    // Householder weights and one fma downdates both norms (lanes 0 and 1).
    const int npair = (c - k) >> 1;  // ceil((c - k - 1) / 2) trailing pairs
    for (int q = warp; q < npair; q += nwarps) {
      const int j0 = k + 1 + 2 * q, j1 = j0 + 1;
      const bool has1 = j1 < c;
      double* c0 = Ab + (int64_t)j0 * n_samp;
      double* c1 = c0 + n_samp;
      double a[RPL], b[RPL];
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        if (r >= nr) break;
        const int i = k + lane + 32 * r;
        a[r] = (i < ns) ? c0[i] : 0.0;
        b[r] = (has1 && i < ns) ? c1[i] : 0.0;
      }
      double d0 = 0.0, d1 = 0.0;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        if (r >= nr) break;  // slots past the last row chunk hold nothing
        const int i = k + lane + 32 * r;
        if (i < ns) {
          const double vi = v[i];
          d0 = fma(vi, a[r], d0);
          d1 = fma(vi, b[r], d1);
        }
      }
      const bool upper = lane & 16;
      double dsum = (upper ? d1 : d0) + __shfl_xor_sync(0xffffffffu, upper ? d0 : d1, 16);
      for (int off = 8; off > 0; off >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, off);
      const double wl = beta * dsum;
      const double w0 = __shfl_sync(0xffffffffu, wl, 0), w1 = __shfl_sync(0xffffffffu, wl, 16);
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        if (r >= nr) break;
        const int i = k + lane + 32 * r;
        if (i < ns) {
          const double vi = v[i];
          a[r] = fma(-w0, vi, a[r]);
          b[r] = fma(-w1, vi, b[r]);
          c0[i] = a[r];
          if (has1) c1[i] = b[r];
        }
      }
      // row k sits in lane 0, slot 0 of both columns
      const double x0 = __shfl_sync(0xffffffffu, a[0], 0), x1 = __shfl_sync(0xffffffffu, b[0], 0);
      const int jl = (lane & 1) ? j1 : j0;
      const bool mine = lane < 2 && jl < c;
      double nrm = 0.0;
      bool redo = false;
      if (mine) {
        const double akj = (lane & 1) ? x1 : x0;
        nrm = fma(-akj, akj, norms[jl]);
        // nref holds 1/16 of the last exact value; the bit patterns of a
        // non-negative threshold and of nrm compare like the values (a
        // negative nrm compares below), which keeps the test off the FP64 pipe
        redo = !(__double_as_longlong(nrm) > __double_as_longlong(nref[jl]));
      }
      const unsigned rm = __ballot_sync(0xffffffffu, redo);
      if (rm & 1u) {
        double e = 0.0;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          if (r >= nr) break;
          const int i = k + lane + 32 * r;
          if (i > k && i < ns) e = fma(a[r], a[r], e);
        }
        for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
        if (lane == 0) { nrm = e; nref[j0] = e * 0.0625; }
      }
      if (rm & 2u) {
        double e = 0.0;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          if (r >= nr) break;
          const int i = k + lane + 32 * r;
          if (i > k && i < ns) e = fma(b[r], b[r], e);
        }
        for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
        if (lane == 1) { nrm = e; nref[j1] = e * 0.0625; }
      }
      __syncwarp();
      if (mine) norms[jl] = nrm;
    }
    __syncthreads();
    if (threadIdx.x == 0) Ab[(int64_t)k * n_samp + k] = alpha;
    for (int i = k + 1 + threadIdx.x; i < ns; i += blockDim.x) Ab[(int64_t)k * n_samp + i] = 0.0;
    __syncthreads();
  }
  __syncthreads();
  __shared__ IdSolveShared ish;
  id_finish(lo, hi, rank, skel, s_max, node, nl, leaf, n_samp, c, Ab, piv, s_final, Pout, ldP, P_node_stride, ish);
}

// ---- 3b. pivoted QR of an internal node on a 16-CTA cluster -------------------
// The node's sample block lives in the distributed shared memory of its
// cluster: CTA r holds the ID columns j with j % 16 == r for the whole
// factorization.  Per Householder step: each CTA proposes its best trailing
// column (largest norm, ties to the lowest current position), the proposals
// are read across the cluster, the owner of the pivot publishes v, every CTA
// copies v and updates its own columns (norms downdated as in the single-CTA
// kernel).  Columns are not moved; their current positions are tracked so
// that the pivot order and tie rule equal those of the column-swapping QR.
// At the end the columns are written to global memory in position order and
// k_id_finish computes T = R11^-1 R12 and P.
constexpr int kQC = 16;  // CTAs per cluster

struct QrCand {
  double v;
  int pos;
  int phys;
};

__global__ void __cluster_dims__(kQC, 1, 1) __launch_bounds__(256)
    k_qr_cluster(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, const int32_t* __restrict__ rank,
                 int s_max, int node0, int n_samp, int cmax, const int32_t* __restrict__ nsamp, double tau,
                 double* __restrict__ A, int32_t* __restrict__ pivpos, int32_t* __restrict__ sout) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) double qsm[];
  const int W = (cmax + kQC - 1) / kQC;
  double* Aloc = qsm;                        // W x n_samp, column-major
  double* norms = Aloc + (size_t)W * n_samp; // W
  double* nref = norms + W;                  // W
  double* vloc = nref + W;                   // n_samp
  double* vbuf = vloc + n_samp;              // n_samp: published Householder vector
  int* posof = (int*)(vbuf + n_samp);        // cmax: position of each column
  int* physat = posof + cmax;                // cmax: column at each position
  int* done = physat + cmax;                 // W
  __shared__ QrCand wcand[8];
  __shared__ QrCand cand;                    // this CTA's proposal
  __shared__ double pub[2];                  // beta of the published vector
  __shared__ QrCand best;
  __shared__ int s_final;
  const int cr = (int)cluster.block_rank();
  const int nl = blockIdx.x / kQC, node = node0 + nl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = rank[2 * node] + rank[2 * node + 1];
  const int ns = nsamp[nl];
  const int kmax = min(s_max, min(ns, c));
  double* Ab = A + (int64_t)nl * cmax * n_samp;
  // load my columns, exact norms
  for (int lj = warp; lj < W; lj += 8) {
    const int j = lj * kQC + cr;
    double acc = 0.0;
    if (j < c) {
      for (int i = lane; i < ns; i += 32) {
        const double a = Ab[(int64_t)j * n_samp + i];
        Aloc[(size_t)lj * n_samp + i] = a;
        acc = fma(a, a, acc);
      }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) { norms[lj] = acc; nref[lj] = acc * 0.0625; done[lj] = (j < c) ? 0 : 1; }
  }
  for (int j = tid; j < c; j += blockDim.x) { posof[j] = j; physat[j] = j; }
  if (tid == 0) s_final = kmax;
  __syncthreads();
  double r00 = 0.0;
  for (int k = 0; k < kmax; ++k) {
    // 1. my proposal
    QrCand mine{-1.0, c, -1};
    for (int lj = tid; lj < W; lj += blockDim.x) {
      if (done[lj]) continue;
      const int j = lj * kQC + cr;
      const double v = norms[lj];
      const int p = posof[j];
      if (v > mine.v || (v == mine.v && p < mine.pos)) mine = {v, p, j};
    }
    for (int off = 16; off > 0; off >>= 1) {
      QrCand o;
      o.v = __shfl_xor_sync(0xffffffffu, mine.v, off);
      o.pos = __shfl_xor_sync(0xffffffffu, mine.pos, off);
      o.phys = __shfl_xor_sync(0xffffffffu, mine.phys, off);
      if (o.v > mine.v || (o.v == mine.v && o.pos < mine.pos)) mine = o;
    }
    if (lane == 0) wcand[warp] = mine;
    __syncthreads();
    if (tid == 0) {
      QrCand b = wcand[0];
      for (int w = 1; w < 8; ++w)
        if (wcand[w].v > b.v || (wcand[w].v == b.v && wcand[w].pos < b.pos)) b = wcand[w];
      cand = b;
    }
    cluster.sync();  // (A) proposals visible
    if (warp == 0) {  // lane r reads CTA r's proposal; positions are distinct, so the max is unique
      QrCand b{-1.0, c, -1};
      if (lane < kQC) b = *cluster.map_shared_rank(&cand, lane);
      for (int off = 16; off > 0; off >>= 1) {
        QrCand o;
        o.v = __shfl_xor_sync(0xffffffffu, b.v, off);
        o.pos = __shfl_xor_sync(0xffffffffu, b.pos, off);
        o.phys = __shfl_xor_sync(0xffffffffu, b.phys, off);
        if (o.v > b.v || (o.v == b.v && o.pos < b.pos)) b = o;
      }
      if (lane == 0) best = b;
    }
    __syncthreads();
    const double rkk = sqrt(best.v);
    if (k == 0) r00 = rkk;
    const bool stop = (k == 0) ? (r00 == 0.0) : (rkk < tau * r00);
    if (stop) {
      if (tid == 0) s_final = k;
      break;  // uniform over the cluster: every CTA saw the same proposals
    }
    const int p = best.phys, P = best.pos;
    const int owner = p % kQC, lp = p / kQC;
    // 2. bookkeeping of positions (replicated): swap positions k and P
    if (tid == 0) {
      const int jk = physat[k];
      physat[k] = p;
      physat[P] = jk;
      posof[p] = k;
      posof[jk] = P;
    }
    // 3. the owner publishes v = x - alpha e_k over rows k.. and beta
    if (cr == owner) {
      double* x = Aloc + (size_t)lp * n_samp;
      const double x0 = x[k];
      const double alpha = (x0 >= 0.0) ? -rkk : rkk;
      const double vtv = 2.0 * rkk * (rkk + fabs(x0));
      for (int i = k + tid; i < ns; i += blockDim.x) vbuf[i] = (i == k) ? x0 - alpha : x[i];
      if (tid == 0) pub[0] = vtv > 0.0 ? 2.0 / vtv : 0.0;
      __syncthreads();
      if (tid == 0) { x[k] = alpha; done[lp] = 1; }
      for (int i = k + 1 + tid; i < ns; i += blockDim.x) x[i] = 0.0;
    }
    cluster.sync();  // (B) v and beta visible
    {
      const double* rv = cluster.map_shared_rank(vbuf, owner);
      for (int i = k + tid; i < ns; i += blockDim.x) vloc[i] = rv[i];
      if (tid == 0) pub[1] = *cluster.map_shared_rank(&pub[0], owner);
    }
    __syncthreads();
    const double beta = pub[1];
    // 4. update my trailing columns, two per warp (local columns lj and
    // lj + 8) as in k_pivoted_qr: one butterfly for both dot products, one
    // multiply for both weights, one fma for both norm downdates
    for (int lj0 = warp; lj0 < W; lj0 += 16) {
      const int lj1 = lj0 + 8;
      const bool u0 = !done[lj0], u1 = lj1 < W && !done[lj1];
      if (!u0 && !u1) continue;
      double* c0 = Aloc + (size_t)lj0 * n_samp;
      double* c1 = Aloc + (size_t)lj1 * n_samp;
      double d0 = 0.0, d1 = 0.0;
      for (int i = k + lane; i < ns; i += 32) {
        const double vi = vloc[i];
        if (u0) d0 = fma(vi, c0[i], d0);
        if (u1) d1 = fma(vi, c1[i], d1);
      }
      const bool upper = lane & 16;
      double dsum = (upper ? d1 : d0) + __shfl_xor_sync(0xffffffffu, upper ? d0 : d1, 16);
      for (int off = 8; off > 0; off >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, off);
      const double wl = beta * dsum;
      const double w0 = __shfl_sync(0xffffffffu, wl, 0), w1 = __shfl_sync(0xffffffffu, wl, 16);
      for (int i = k + lane; i < ns; i += 32) {
        const double vi = vloc[i];
        if (u0) c0[i] = fma(-w0, vi, c0[i]);
        if (u1) c1[i] = fma(-w1, vi, c1[i]);
      }
      __syncwarp();
      // lane 0: column lj0, lane 1: column lj1.  nref holds 1/16 of the last
      // exact norm; non-negative doubles compare like their bit patterns
      const int ljl = (lane & 1) ? lj1 : lj0;
      const bool mine = (lane == 0 && u0) || (lane == 1 && u1);
      double nrm = 0.0;
      bool redo = false;
      if (mine) {
        const double akj = (lane & 1) ? c1[k] : c0[k];
        nrm = fma(-akj, akj, norms[ljl]);
        redo = !(__double_as_longlong(nrm) > __double_as_longlong(nref[ljl]));
      }
      const unsigned rm = __ballot_sync(0xffffffffu, redo);
      for (int h = 0; h < 2; ++h) {
        if (!(rm & (1u << h))) continue;
        const double* ch = h ? c1 : c0;
        double e = 0.0;
        for (int i = k + 1 + lane; i < ns; i += 32) e = fma(ch[i], ch[i], e);
        for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
        if (lane == h) { nrm = e; nref[ljl] = e * 0.0625; }
      }
      __syncwarp();
      if (mine) norms[ljl] = nrm;
    }
    __syncthreads();
  }
  cluster.sync();
  // write my columns back in position order
  for (int lj = warp; lj < W; lj += 8) {
    const int j = lj * kQC + cr;
    if (j >= c) continue;
    const int p = posof[j];
    for (int i = lane; i < ns; i += 32) Ab[(int64_t)p * n_samp + i] = Aloc[(size_t)lj * n_samp + i];
  }
  if (cr == 0) {
    for (int q = tid; q < c; q += blockDim.x) pivpos[(int64_t)nl * cmax + q] = physat[q];
    if (tid == 0) sout[nl] = s_final;
  }
}

// Finishing step after the cluster QR: one CTA per node.
__global__ void __launch_bounds__(512) k_id_finish(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                   int32_t* __restrict__ rank, int32_t* __restrict__ skel, int s_max,
                                                   int node0, int n_samp, int cmax, double* __restrict__ A,
                                                   const int32_t* __restrict__ pivpos, const int32_t* __restrict__ sout,
                                                   double* __restrict__ Pout, int ldP, int64_t P_node_stride) {
  extern __shared__ int pv[];  // cmax
  __shared__ IdSolveShared ish;
  const int nl = blockIdx.x, node = node0 + nl;
  const int c = rank[2 * node] + rank[2 * node + 1];
  for (int q = threadIdx.x; q < c; q += blockDim.x) pv[q] = pivpos[(int64_t)nl * cmax + q];
  __syncthreads();
  id_finish(lo, hi, rank, skel, s_max, node, nl, false, n_samp, c, A + (int64_t)nl * cmax * n_samp, pv, sout[nl],
            Pout, ldP, P_node_stride, ish);
}

}  // namespace

// Skeletonize every non-root node, leaves first, in three parts so that the
// factorization can follow level by level on another stream.
kf_status kf_skel_begin(kf_factor* f, kf_skel_scratch* sc, cudaStream_t s) {
  kf_tree* t = f->t;
  kf_ctx* c = f->ctx;
  KF_CUDA(c, cudaMemsetAsync(f->rank, 0, sizeof(int32_t) * (t->nnodes + 1), s));
  sc->A = nullptr;
  sc->samp = sc->nsamp = nullptr;
  if (t->D == 0) return KF_OK;
  const int maxnodes = 1 << t->D;
  sc->a_elems = std::max((size_t)maxnodes * t->leaf_max, (size_t)(maxnodes / 2) * 2 * f->s_max) * f->n_samp;
  sc->a_elems += (size_t)maxnodes * 2 * f->s_max + maxnodes;  // tail: cluster-QR positions and ranks
  sc->A = (double*)c->dalloc(sizeof(double) * sc->a_elems, s);
  // S' of every non-root node (heap order from node 2), drawn here at once:
  // the draws depend on the tree only, and a level's sampling launch would
  // otherwise wait for a free SM behind the reduced-system kernels
  const size_t nsampled = 2 * (size_t)maxnodes - 2;
  sc->samp = (int32_t*)c->dalloc(sizeof(int32_t) * nsampled * f->n_samp, s);
  sc->nsamp = (int32_t*)c->dalloc(sizeof(int32_t) * nsampled, s);
  if (!sc->A || !sc->samp || !sc->nsamp)
    return kf_set_err(c, KF_ENOMEM, "skeletonize: allocation of %zu bytes failed", sizeof(double) * sc->a_elems);
  if (f->knn_kappa > 0) {
    kf_status st = kf_near_field_lists(f, s);
    if (st != KF_OK) return st;
  }
  KF_PHASE(KF_PH_SAMPLE, s, k_sample<<<(unsigned)nsampled, 32, sizeof(int32_t) * f->n_samp, s>>>(
                                t->d_lo, t->d_hi, t->N, 2, (int)nsampled, f->n_samp, f->seed,
                                f->knn_kappa > 0 ? f->near_pos : nullptr, f->near_len, f->near_cap, sc->samp,
                                sc->nsamp, f->status));
  KF_LAUNCH_CHECK(c);
  return KF_OK;
}

void kf_skel_end(kf_factor* f, kf_skel_scratch* sc, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  const int maxnodes = 1 << f->t->D;
  c->dfree(sc->A, sizeof(double) * sc->a_elems, s);
  c->dfree(sc->samp, sizeof(int32_t) * (2 * (size_t)maxnodes - 2) * f->n_samp, s);
  c->dfree(sc->nsamp, sizeof(int32_t) * (2 * (size_t)maxnodes - 2), s);
  sc->A = nullptr;
  sc->samp = sc->nsamp = nullptr;
}

kf_status kf_skel_level(kf_factor* f, int l, kf_skel_scratch* sc, cudaStream_t s) {
  kf_tree* t = f->t;
  kf_ctx* c = f->ctx;
  const int D = t->D;
  const int n_samp = f->n_samp, s_max = f->s_max;
  const int cleaf = t->leaf_max, cint = 2 * s_max;
  const int rpl = (n_samp + 31) / 32;
  double* A = sc->A;
  const int node0 = 1 << l, nn = 1 << l;
  int32_t* samp = sc->samp + (size_t)(node0 - 2) * n_samp;  // drawn in kf_skel_begin
  int32_t* nsamp = sc->nsamp + (node0 - 2);
  const bool leaf = (l == D);
  const int cmax = leaf ? cleaf : cint;
  dim3 ga((n_samp + 127) / 128, cmax, nn);
  // FP64 entries on both paths: late pivots of the QR hinge on downdated norms
  // whose relative error is far above that of the entries, so any change of
  // the entries' rounding can change the skeletons
  KF_PHASE(KF_PH_EVAL_A, s, k_eval_A<<<ga, 128, 0, s>>>(t->X64, t->d, f->c_exp, t->d_lo, t->d_hi, f->rank, f->skel, s_max, node0, leaf,
                              n_samp, cmax, samp, nsamp, A));
  double* Pout = leaf ? f->Pleaf : f->Pc + (int64_t)node0 * cint * s_max;
  int64_t pstride = leaf ? 0 : (int64_t)cint * s_max;
  // upper levels (few nodes): one 16-CTA cluster per node, the block in distributed shared memory
  // (at 16 nodes and more, one CTA per node is faster inside the overlapped
  // factorization: a 16-CTA cluster waits for 16 free SMs of one GPC, which
  // the reduced-system kernels running beside it rarely leave)
  if (!leaf && nn <= 8 && f->use_cluster_qr) {
    const int W = (cmax + kQC - 1) / kQC;
    const size_t qsmem = sizeof(double) * ((size_t)W * n_samp + 2 * W + 2 * n_samp) + sizeof(int) * (2 * cmax + W);
    if (qsmem <= 200 * 1024) {
      cudaError_t e1 = cudaFuncSetAttribute(k_qr_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      cudaError_t e2 = cudaFuncSetAttribute(k_qr_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsmem);
      if (e1 == cudaSuccess && e2 == cudaSuccess) {
        // positions and ranks from the tail of the A scratch
        int32_t* pp = (int32_t*)(A + (size_t)nn * cmax * n_samp);
        int32_t* so = pp + (size_t)nn * cmax;
        KF_PHASE(KF_PH_QR_CLUSTER, s, k_qr_cluster<<<nn * kQC, 256, qsmem, s>>>(t->d_lo, t->d_hi, f->rank, s_max, node0,
                                                                       n_samp, cmax, nsamp, f->tau, A, pp, so));
        KF_CUDA(c, cudaFuncSetAttribute(k_id_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(int) * cmax)));
        KF_PHASE(KF_PH_QR_CLUSTER, s, k_id_finish<<<nn, 512, sizeof(int) * cmax, s>>>(t->d_lo, t->d_hi, f->rank, f->skel,
                                                                            s_max, node0, n_samp, cmax, A, pp, so,
                                                                            Pout, s_max, pstride));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return kf_set_err(c, KF_ECUDA, "cluster QR level %d: %s", l, cudaGetErrorString(e));
        return KF_OK;
      }
      cudaGetLastError();
    }
  }
  size_t smem = sizeof(double) * (2 * cmax + n_samp) + sizeof(int) * cmax;
  // the static part (the blocked R11^-1 R12 tiles) plus this may pass 48 KiB
#define KF_QR_GO(R, NT)                                                                                          \
  do {                                                                                                          \
    KF_CUDA(c, cudaFuncSetAttribute(k_pivoted_qr<R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    KF_PHASE(leaf ? KF_PH_QR_LEAF : KF_PH_QR, s,                                                                \
             (k_pivoted_qr<R, NT><<<nn, NT, smem, s>>>(t->d_lo, t->d_hi, f->rank, f->skel, s_max, node0, leaf,     \
                                                      n_samp, cmax, nsamp, f->tau, A, Pout, s_max, pstride)));       \
  } while (0)
  // 512 threads (16 warps) while two columns of RPL rows fit in 128 registers
  if (rpl <= 8)
    KF_QR_GO(8, 512);
  else if (rpl <= 16)
    KF_QR_GO(16, 512);
  else
    KF_QR_GO(32, 256);
#undef KF_QR_GO
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return kf_set_err(c, KF_ECUDA, "skeletonize level %d: %s", l, cudaGetErrorString(e));
  return KF_OK;
}

kf_status kf_skeletonize_device(kf_factor* f, cudaStream_t s) {
  kf_skel_scratch sc;
  kf_status st = kf_skel_begin(f, &sc, s);
  for (int l = f->t->D; l >= 1 && st == KF_OK; --l) st = kf_skel_level(f, l, &sc, s);
  kf_skel_end(f, &sc, s);
  return st;
}
