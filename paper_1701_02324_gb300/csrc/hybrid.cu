// hybrid.cu -- the reduced system of the hybrid level-restricted solver
// (Sec. II-C "Fast hybrid solver", Algorithms 6-8).
//
// With the frontier A = the 2^L nodes of level L, the subtrees below A are
// skeletonized and factorized like the direct solver's (Algorithms 1-2, the
// frontier nodes' own IDs and P^ included) and nothing above A is compressed:
//   lambda I + K~ = D + U V,  D = blockdiag(lambda I + K~_aa) over a in A,
//   U = blockdiag(P_{a a~}),  V[a~, b] = K_{a~ b} (b != a), 0 (b = a),
// so that with W = D^-1 U = blockdiag(P^_a), Eq. (e:smw) gives
//   x = D^-1 u - W (I + V W)^-1 V D^-1 u                    (Algorithm 6).
// The paper applies V W inside a Krylov method (Algorithms 7-8); here the
// reduced system I + V W (S = sum of the frontier ranks rows, S <= 1024) is
// formed once in FP64, (V W)[a~, b~] = K_{a~ b} P^_b, and LU-factored by the
// reduced-system kernels of the direct solver, so that the solve is direct.
//
// Data: Vh holds, for frontier node a and q < s_max, the row K(x_{a~ q}, x_j)
// over all tree positions j (zero for j in a and for q >= s_a), FP64.
// The LU lives as node 1 of a two-node Z array with rank {0, 0, S, 0}.
#include <algorithm>

#include "kf_internal.cuh"
#include "prof.cuh"

namespace {

constexpr int kVhChunk = 1 << 16;  // tree positions per partial sum of V x

// offsets of the frontier ranks; Hrank = {0, 0, S, 0}
__global__ void k_hyb_offsets(const int32_t* __restrict__ rank, int nA, int scap, int32_t* __restrict__ off,
                              int32_t* __restrict__ hrank, int32_t* __restrict__ status) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int acc = 0;
  for (int a = 0; a < nA; ++a) {
    off[a] = acc;
    acc += rank[nA + a];
  }
  off[nA] = acc;
  if (acc > scap) {  // cannot happen: each rank is at most s_max and scap = nA s_max
    atomicOr(status, KF_DEV_BADARG);
    acc = 0;
  }
  hrank[0] = hrank[1] = hrank[3] = 0;
  hrank[2] = acc;
}

// Vh[a][q][j] = K(x_{a~ q}, x_j) for j outside a, q < s_a; 0 otherwise (FP64,
// the operation order of Eq. e:gaussian: sequential sum of squared differences)
__global__ void __launch_bounds__(256) k_hyb_eval_vh(const double* __restrict__ X64, int d, double c_exp,
                                                     const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                     const int32_t* __restrict__ rank, const int32_t* __restrict__ skel,
                                                     int nA, int s_max, int64_t N, double* __restrict__ Vh) {
  __shared__ double xs[KF_MAX_D];
  const int row = blockIdx.y, a = row / s_max, q = row % s_max, node = nA + a;
  const int sa = rank[node];
  double* out = Vh + (int64_t)row * N;
  const int64_t b0 = lo[node], b1 = hi[node];
  if (q >= sa) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x)
      out[j] = 0.0;
    return;
  }
  const int64_t p = skel[(int64_t)node * s_max + q];
  for (int t = threadIdx.x; t < d; t += blockDim.x) xs[t] = X64[p * d + t];
  __syncthreads();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = (j >= b0 && j < b1) ? 0.0 : kf_kern64(xs, X64 + j * d, d, c_exp);
}

// M = I on the S x S reduced system (node 1 of the two-node array, row stride scap)
__global__ void k_hyb_identity(const int32_t* __restrict__ hrank, int scap, double* __restrict__ M) {
  const int S = hrank[2];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x)
    M[(int64_t)i * scap + i] = 1.0;
}

// (V W)[a~, b~] = K_{a~ b} P^_b for a != b: a 32 x 32 tile (rows q0.., columns
// t0..) per CTA, the reduction over the points of b in chunks of 32 staged in
// shared memory (Vh rows coalesced along j, P^ rows coalesced along t).
template <typename TP>
__global__ void __launch_bounds__(256) k_hyb_vw(const double* __restrict__ Vh, const TP* __restrict__ PhatL,
                                                const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                const int32_t* __restrict__ rank, const int32_t* __restrict__ off,
                                                int nA, int s_max, int64_t N, int scap, double* __restrict__ M) {
  __shared__ double va[32][33];
  __shared__ double pb[32][33];
  const int a = blockIdx.z / nA, b = blockIdx.z % nA;
  if (a == b) return;
  const int na = nA + a, nb = nA + b;
  const int sa = rank[na], sb = rank[nb];
  const int q0 = blockIdx.y * 32, t0 = blockIdx.x * 32;
  if (q0 >= sa || t0 >= sb) return;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;  // 8 row groups of 4 rows
  const int64_t j0 = lo[nb], j1 = hi[nb];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t jc = j0; jc < j1; jc += 32) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int qq = ty * 4 + r;
      const int64_t j = jc + tx;
      va[qq][tx] = (q0 + qq < sa && j < j1) ? Vh[((int64_t)a * s_max + q0 + qq) * N + j] : 0.0;
      pb[qq][tx] = (jc + qq < j1 && t0 + tx < sb) ? (double)PhatL[(jc + qq) * s_max + t0 + tx] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < 32; ++jj) {
      const double p = pb[jj][tx];
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] = fma(va[ty * 4 + r][jj], p, acc[r]);
    }
    __syncthreads();
  }
  if (t0 + tx >= sb) return;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int q = q0 + ty * 4 + r;
    if (q < sa) M[(int64_t)(off[a] + q) * scap + off[b] + t0 + tx] = acc[r];
  }
}

// partial sums of V x: part[((row * nchunk) + chunk) * k + c] = sum over the
// chunk's tree positions j of Vh[row][j] x[j * k + c] (vectors are N x k,
// point-major, as everywhere in the solve); one warp per row
__global__ void __launch_bounds__(256) k_hyb_vpart(const double* __restrict__ Vh, const int32_t* __restrict__ rank,
                                                   int nA, int s_max, int64_t N, const double* __restrict__ x, int k,
                                                   int nchunk, double* __restrict__ part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.y * 8 + warp;
  if (row >= nA * s_max) return;
  const int a = row / s_max, q = row % s_max;
  if (q >= rank[nA + a]) return;
  const int chunk = blockIdx.x;
  const int64_t j0 = (int64_t)chunk * kVhChunk, j1 = (N < j0 + kVhChunk) ? N : j0 + kVhChunk;
  const double* v = Vh + (int64_t)row * N;
  for (int c = 0; c < k; ++c) {
    double acc = 0.0;
    for (int64_t j = j0 + lane; j < j1; j += 32) acc = fma(v[j], x[j * k + c], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[((int64_t)row * nchunk + chunk) * k + c] = acc;
  }
}

// the partial sums added in chunk order.  mode 0: contiguous reduced-system
// layout out[(2 scap + off_a + q) * k + c]; mode 1: per-node layout
// out[((nA + a) * s_max + q) * k + c]
__global__ void k_hyb_vsum(const double* __restrict__ part, const int32_t* __restrict__ rank,
                           const int32_t* __restrict__ off, int nA, int s_max, int k, int nchunk, int scap, int mode,
                           double* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nA * s_max * k) return;
  const int c = (int)(e % k);
  const int row = (int)(e / k), a = row / s_max, q = row % s_max;
  if (q >= rank[nA + a]) return;
  double acc = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) acc += part[((int64_t)row * nchunk + ch) * k + c];
  if (mode == 0)
    out[((int64_t)2 * scap + off[a] + q) * k + c] = acc;
  else
    out[((int64_t)(nA + a) * s_max + q) * k + c] = acc;
}

// contiguous reduced-system vector -> per-node layout of the frontier nodes
__global__ void k_hyb_scatter(const double* __restrict__ z, const int32_t* __restrict__ rank,
                              const int32_t* __restrict__ off, int nA, int s_max, int k, int scap,
                              double* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nA * s_max * k) return;
  const int c = (int)(e % k);
  const int row = (int)(e / k), a = row / s_max, q = row % s_max;
  out[((int64_t)(nA + a) * s_max + q) * k + c] =
      q < rank[nA + a] ? z[((int64_t)2 * scap + off[a] + q) * k + c] : 0.0;
}

inline int grid_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

// V x of the frontier (Algorithm 8 over A) into `out` (mode as k_hyb_vsum)
kf_status hyb_apply_v(kf_factor* f, const double* x, int64_t k, int mode, double* out, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  const int nA = 1 << f->hyb_L, s_max = f->s_max;
  const int64_t N = f->t->N;
  const int nchunk = (int)((N + kVhChunk - 1) / kVhChunk);
  const size_t pb = sizeof(double) * (size_t)nA * s_max * nchunk * k;
  double* part = (double*)c->dalloc(pb, s);
  if (!part) return kf_set_err(c, KF_ENOMEM, "hybrid: allocation failed");
  dim3 g((unsigned)nchunk, (unsigned)((nA * s_max + 7) / 8));
  KF_PHASE(KF_PH_HYBRID, s, k_hyb_vpart<<<g, 256, 0, s>>>(f->Vh, f->rank, nA, s_max, N, x, (int)k, nchunk, part));
  const int64_t ne = (int64_t)nA * s_max * k;
  KF_PHASE(KF_PH_HYBRID, s, k_hyb_vsum<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(
                                 part, f->rank, f->Hoff, nA, s_max, (int)k, nchunk, f->hyb_scap, mode, out));
  cudaError_t e = cudaGetLastError();
  c->dfree(part, pb, s);
  if (e != cudaSuccess) return kf_set_err(c, KF_ECUDA, "hybrid V x: %s", cudaGetErrorString(e));
  return KF_OK;
}

}  // namespace

kf_status kf_hybrid_reduced_system(kf_factor* f, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  kf_tree* t = f->t;
  const int L = f->hyb_L, nA = 1 << L, s_max = f->s_max, scap = f->hyb_scap;
  const int64_t N = t->N;
  KF_PHASE(KF_PH_HYBRID, s, k_hyb_offsets<<<1, 32, 0, s>>>(f->rank, nA, scap, f->Hoff, f->Hrank, f->status));
  dim3 gv((unsigned)std::min<int64_t>((N + 255) / 256, 64), (unsigned)(nA * s_max));
  KF_PHASE(KF_PH_HYBRID, s, k_hyb_eval_vh<<<gv, 256, 0, s>>>(t->X64, t->d, f->c_exp, t->d_lo, t->d_hi, f->rank,
                                                             f->skel, nA, s_max, N, f->Vh));
  double* M = f->HM + (size_t)scap * scap;
  KF_CUDA(c, cudaMemsetAsync(f->HM, 0, sizeof(double) * 2 * (size_t)scap * scap, s));
  KF_PHASE(KF_PH_HYBRID, s, k_hyb_identity<<<grid_for(scap, 256), 256, 0, s>>>(f->Hrank, scap, M));
  dim3 gw((unsigned)((s_max + 31) / 32), (unsigned)((s_max + 31) / 32), (unsigned)(nA * nA));
  const int64_t lvlL = (int64_t)(L - 1) * N * s_max;
  if (f->prec == KF_PREC_FP64)
    KF_PHASE(KF_PH_HYBRID, s, k_hyb_vw<double><<<gw, 256, 0, s>>>(f->Vh, (const double*)f->Phat + lvlL, t->d_lo,
                                                                  t->d_hi, f->rank, f->Hoff, nA, s_max, N, scap, M));
  else
    KF_PHASE(KF_PH_HYBRID, s, k_hyb_vw<float><<<gw, 256, 0, s>>>(f->Vh, (const float*)f->Phat + lvlL, t->d_lo,
                                                                 t->d_hi, f->rank, f->Hoff, nA, s_max, N, scap, M));
  KF_LAUNCH_CHECK(c);
  return kf_z_factor_one_launch(f->Hrank, scap, f->HM, f->Hpiv, f->status, f->Hpivr, s);
}

kf_status kf_hybrid_top_solve(kf_factor* f, double* W, int64_t k, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  const int nA = 1 << f->hyb_L, s_max = f->s_max, scap = f->hyb_scap;
  const size_t rb = sizeof(double) * 3 * (size_t)scap * k;
  const size_t vb = sizeof(double) * (size_t)(f->t->nnodes + 1) * s_max * k;
  double* tvec = (double*)c->dalloc(rb, s);
  double* zvec = (double*)c->dalloc(rb, s);
  double* znode = (double*)c->dalloc(vb, s);
  kf_status st = KF_OK;
  if (!tvec || !zvec || !znode) st = kf_set_err(c, KF_ENOMEM, "hybrid solve: allocation failed");
  if (st == KF_OK) st = hyb_apply_v(f, W, k, 0, tvec, s);                                   // t = V D^-1 u
  if (st == KF_OK)
    st = kf_zsolve_one_launch(f->Hrank, scap, f->HM, f->Hpiv, tvec, zvec, (int)k, s);     // z = (I + VW)^-1 t
  if (st == KF_OK) {
    const int64_t ne = (int64_t)nA * s_max * k;
    KF_PHASE(KF_PH_HYBRID, s, k_hyb_scatter<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(zvec, f->rank, f->Hoff, nA,
                                                                                        s_max, (int)k, scap, znode));
    if (cudaGetLastError() != cudaSuccess) st = kf_set_err(c, KF_ECUDA, "hybrid solve: launch failed");
  }
  if (st == KF_OK) st = kf_rowupd_level_launch(f, f->hyb_L, znode, W, k, s);              // w -= W z
  c->dfree(tvec, rb, s);
  c->dfree(zvec, rb, s);
  c->dfree(znode, vb, s);
  return st;
}

kf_status kf_hybrid_top_apply(kf_factor* f, const double* x, double* G, int64_t k, cudaStream_t s) {
  return hyb_apply_v(f, x, k, 1, G, s);
}
