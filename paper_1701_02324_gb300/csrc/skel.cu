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
//     first k with |R_kk| < tau |R_00| or at min(s_max, n_s, |C|); the column
//     norms of the trailing block are accumulated from the updated entries
//     at every step (no downdating).
//  4. P = [I, R11^-1 R12] with the columns in their original order.
#include <algorithm>

#include "kf_internal.cuh"
#include "prof.cuh"

namespace {

// ---- 1. sampling: one warp per node ------------------------------------------
__global__ void k_sample(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, int64_t N, int node0,
                         int nn, int n_samp, uint64_t seed, int32_t* __restrict__ samp, int32_t* __restrict__ ns_out,
                         int32_t* __restrict__ status) {
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

// ---- 3/4. pivoted QR and P ------------------------------------------------------
template <int RPL>  // rows per lane held in registers (n_samp <= 32 * RPL)
__global__ void __launch_bounds__(512) k_pivoted_qr(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                    int32_t* __restrict__ rank, int32_t* __restrict__ skel, int s_max,
                                                    int node0, bool leaf, int n_samp, int cmax,
                                                    const int32_t* __restrict__ nsamp, double tau,
                                                    double* __restrict__ A, double* __restrict__ Pout, int ldP,
                                                    int64_t P_node_stride) {
  extern __shared__ double sm[];
  double* norms = sm;                          // cmax
  double* v = norms + cmax;                    // n_samp
  int* piv = (int*)(v + n_samp);               // cmax
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_final;
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
    if (lane == 0) norms[j] = acc;
  }
  for (int j = threadIdx.x; j < c; j += blockDim.x) piv[j] = j;
  if (threadIdx.x == 0) s_final = kmax;
  __syncthreads();
  double r00 = 0.0;
  for (int k = 0; k < kmax; ++k) {
    // pivot: largest trailing norm, ties to the lowest column
    double bv = -1.0;
    int bi = c;
    for (int j = k + threadIdx.x; j < c; j += blockDim.x)
      if (norms[j] > bv) { bv = norms[j]; bi = j; }
    for (int off = 16; off > 0; off >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, bv, off);
      int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = bv; red_i[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      bv = lane < nwarps ? red_v[lane] : -1.0;
      bi = lane < nwarps ? red_i[lane] : c;
      for (int off = 16; off > 0; off >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, off);
        int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (lane == 0) { red_v[0] = bv; red_i[0] = bi; }
    }
    __syncthreads();
    const int p = red_i[0];
    const double rkk = sqrt(red_v[0]);
    if (k == 0) r00 = rkk;
    bool stop = (k == 0) ? (r00 == 0.0) : (rkk < tau * r00);
    __syncthreads();
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
    double vtv = 0.0;
    for (int w = 0; w < nwarps; ++w) vtv += red_v[w];
    const double beta = vtv > 0.0 ? 2.0 / vtv : 0.0;
    // apply H to the trailing columns; accumulate their new norms (rows > k)
    for (int j = k + 1 + warp; j < c; j += nwarps) {
      double* cj = Ab + (int64_t)j * n_samp;
      double a[RPL];
      double dot = 0.0;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        int i = k + lane + 32 * r;
        a[r] = (i < ns) ? cj[i] : 0.0;
        if (i < ns) dot = fma(v[i], a[r], dot);
      }
      for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
      const double w = beta * dot;
      double nrm = 0.0;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        int i = k + lane + 32 * r;
        if (i < ns) {
          a[r] = fma(-w, v[i], a[r]);
          cj[i] = a[r];
          if (i > k) nrm = fma(a[r], a[r], nrm);
        }
      }
      for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
      if (lane == 0) norms[j] = nrm;
    }
    __syncthreads();
    if (threadIdx.x == 0) Ab[(int64_t)k * n_samp + k] = alpha;
    for (int i = k + 1 + threadIdx.x; i < ns; i += blockDim.x) Ab[(int64_t)k * n_samp + i] = 0.0;
    __syncthreads();
  }
  __syncthreads();
  const int s = s_final;
  // T = R11^-1 R12 (warp per column of R12), written straight into P
  // P[j * ldP + q]: ID column j, skeleton q.  Leaves write their rows of the
  // N x s_max matrix (base lo[node]); internal nodes have fixed-size blocks.
  double* P = leaf ? Pout + (int64_t)lo[node] * ldP : Pout + (int64_t)nl * P_node_stride;
  for (int j = s + warp; j < c; j += nwarps) {
    const double* cj = Ab + (int64_t)j * n_samp;
    double b[KF_MAX_SMAX / 32];
#pragma unroll
    for (int r = 0; r < KF_MAX_SMAX / 32; ++r) {
      int i = lane + 32 * r;
      b[r] = (i < s) ? cj[i] : 0.0;
    }
    for (int t = s - 1; t >= 0; --t) {
      const double* ct = Ab + (int64_t)t * n_samp;
      double bt = 0.0;
#pragma unroll
      for (int r = 0; r < KF_MAX_SMAX / 32; ++r)
        if (lane + 32 * r == t) bt = b[r];
      bt = __shfl_sync(0xffffffffu, bt, t & 31);
      double xt = bt / ct[t];
#pragma unroll
      for (int r = 0; r < KF_MAX_SMAX / 32; ++r) {
        int i = lane + 32 * r;
        if (i == t) b[r] = xt;
        else if (i < t) b[r] = fma(-ct[i], xt, b[r]);
      }
    }
    double* Pj = P + (int64_t)piv[j] * ldP;
#pragma unroll
    for (int r = 0; r < KF_MAX_SMAX / 32; ++r) {
      int q = lane + 32 * r;
      if (q < s) Pj[q] = b[r];
      else if (q < s_max) Pj[q] = 0.0;
    }
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
  sc->A = (double*)c->dalloc(sizeof(double) * sc->a_elems, s);
  sc->samp = (int32_t*)c->dalloc(sizeof(int32_t) * (size_t)maxnodes * f->n_samp, s);
  sc->nsamp = (int32_t*)c->dalloc(sizeof(int32_t) * maxnodes, s);
  if (!sc->A || !sc->samp || !sc->nsamp)
    return kf_set_err(c, KF_ENOMEM, "skeletonize: allocation of %zu bytes failed", sizeof(double) * sc->a_elems);
  return KF_OK;
}

void kf_skel_end(kf_factor* f, kf_skel_scratch* sc, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  const int maxnodes = 1 << f->t->D;
  c->dfree(sc->A, sizeof(double) * sc->a_elems, s);
  c->dfree(sc->samp, sizeof(int32_t) * (size_t)maxnodes * f->n_samp, s);
  c->dfree(sc->nsamp, sizeof(int32_t) * maxnodes, s);
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
  int32_t* samp = sc->samp;
  int32_t* nsamp = sc->nsamp;
  const int node0 = 1 << l, nn = 1 << l;
  const bool leaf = (l == D);
  const int cmax = leaf ? cleaf : cint;
  KF_PHASE(KF_PH_SAMPLE, s, k_sample<<<nn, 32, sizeof(int32_t) * n_samp, s>>>(t->d_lo, t->d_hi, t->N, node0, nn, n_samp, f->seed, samp, nsamp,
                                                    f->status));
  dim3 ga((n_samp + 127) / 128, cmax, nn);
  KF_PHASE(KF_PH_EVAL_A, s, k_eval_A<<<ga, 128, 0, s>>>(t->X64, t->d, f->c_exp, t->d_lo, t->d_hi, f->rank, f->skel, s_max, node0, leaf,
                              n_samp, cmax, samp, nsamp, A));
  double* Pout = leaf ? f->Pleaf : f->Pc + (int64_t)node0 * cint * s_max;
  int64_t pstride = leaf ? 0 : (int64_t)cint * s_max;
  size_t smem = sizeof(double) * (cmax + n_samp) + sizeof(int) * cmax;
  if (rpl <= 8)
    KF_PHASE(KF_PH_QR, s, k_pivoted_qr<8><<<nn, 512, smem, s>>>(t->d_lo, t->d_hi, f->rank, f->skel, s_max, node0, leaf, n_samp, cmax,
                                          nsamp, f->tau, A, Pout, s_max, pstride));
  else if (rpl <= 16)
    KF_PHASE(KF_PH_QR, s, k_pivoted_qr<16><<<nn, 512, smem, s>>>(t->d_lo, t->d_hi, f->rank, f->skel, s_max, node0, leaf, n_samp, cmax,
                                           nsamp, f->tau, A, Pout, s_max, pstride));
  else
    KF_PHASE(KF_PH_QR, s, k_pivoted_qr<32><<<nn, 512, smem, s>>>(t->d_lo, t->d_hi, f->rank, f->skel, s_max, node0, leaf, n_samp, cmax,
                                           nsamp, f->tau, A, Pout, s_max, pstride));
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
