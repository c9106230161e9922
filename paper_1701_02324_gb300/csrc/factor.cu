// factor.cu -- the N log N factorization, Algorithm 2, run level by level.
//
// Leaves (base case of Eq. e:invtelescope): A = lambda I + K_aa, Cholesky
// A = L L^T (the paper uses LU; A is symmetric positive definite), and
// P^_a = A^-1 P_{a a~}.
// Internal node a with children l, r (Eqs. e:hodlr, e:blocksmw):
//   V blocks  K_{l~ r}, K_{r~ l}            (stored as VT rows of the children)
//   Z_a     = [[I, K_{l~ r} P^_r], [K_{r~ l} P^_l, I]]   (FP64), LU with
//             partial pivoting (GETRF semantics)
//   P^_a    = W_a Z_a^-1 P_c = [P^_l T_top ; P^_r T_bot], T = Z_a^-1 P_c.
// The last line is Solve(a, W P_c, false) of Algorithm 2 after the identity
// u - W Z^-1 V u = W Z^-1 P_c for u = W P_c (since V W = Z - I).
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "kf_internal.cuh"
#include "prof.cuh"

kf_status kf_tc_zoff(const int32_t* lo, const int32_t* hi, const int32_t* rank, int node0, int nn, int s_max,
                     const float* VT, const float* Ph, int ldz, double* Z, int64_t rows_per_child, float* parts,
                     size_t parts_cap, int32_t* status, cudaStream_t s, int tile_n);
size_t kf_tc_zoff_parts_bytes(int s_max, int tile_n, int nn, int64_t rows_per_child);
kf_status kf_tc_telescope(const int32_t* lo, const int32_t* hi, const int32_t* rank, int node0, int nn, int s_max,
                          const float* Pc_hat, const float* Tm, int ldz, float* Pa_hat, int64_t rows_per_child,
                          int32_t* status, cudaStream_t s, int tile_n);
kf_status kf_tc_zoff_fused(const int32_t* lo, const int32_t* hi, const int32_t* rank, const int32_t* skel,
                           const float* X32, int d, float c_exp, int node0, int nn, int s_max, const float* Ph,
                           int ldz, double* Z, int64_t rows_per_child, float* parts, size_t parts_cap,
                           int32_t* status, cudaStream_t s, int tile_n);
kf_status kf_tc_leaf_panel(const int32_t* lo, const int32_t* hi, int leaf0, int nleaf, int ldL, int kb, float* L,
                           const float* Dinv, int32_t* status, cudaStream_t s);
kf_status kf_tc_leaf_phat(const int32_t* lo, const int32_t* hi, const int32_t* rank, int leaf0, int nleaf, int ldL,
                          float* L, const float* Dinv, int s_max, float* Y, int32_t* status, cudaStream_t s);

namespace {

template <typename T> struct Acc;
template <> struct Acc<double> { using type = double; };
template <> struct Acc<float> { using type = float; };

// split over K of the CUDA-core Z-block products (64 x 64 tiles): enough CTAs
// for the GPU, at least 512 rows a part
inline int zoff64_ksplit(int64_t rows, int nn, int tiles) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(rows / 512, (152 * 8) / std::max(1, 2 * nn * tiles) + 1));
}

inline int grid_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

// ---- leaves --------------------------------------------------------------------
template <typename T>
__global__ void k_leaf_assemble(const double* __restrict__ X64, const float* __restrict__ X32, int d, double c_exp,
                                double lambda, const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                int leaf0, int ldL, T* __restrict__ L) {
  int lf = blockIdx.z, node = leaf0 + lf;
  int b = lo[node], n = hi[node] - b;
  int i = blockIdx.y;
  if (i >= n) return;
  T* Li = L + ((int64_t)lf * ldL + i) * ldL;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= i; j += gridDim.x * blockDim.x) {
    T kij = kf_kern<T>::eval(X64, X32, b + i, b + j, d, c_exp);
    Li[j] = (i == j) ? (T)((double)kij + lambda) : kij;
  }
}

// Blocked right-looking Cholesky of one leaf per CTA (lower triangle, in
// place).  nb = 32 column panels; the trailing update is tiled 64 x 64.
template <typename T>
__global__ void __launch_bounds__(256) k_leaf_cholesky(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                       int leaf0, int ldL, T* __restrict__ Lall,
                                                       int32_t* __restrict__ status, double* __restrict__ pivr) {
  constexpr int NB = 32, TS = 64;
  __shared__ T dg[NB][NB + 1];
  __shared__ T pa[TS][NB + 1];
  __shared__ T pb[TS][NB + 1];
  __shared__ double amax_sh;
  const int lf = blockIdx.x, node = leaf0 + lf;
  const int n = hi[node] - lo[node];
  T* L = Lall + (int64_t)lf * ldL * ldL;
  __shared__ double dinv[NB];  // reciprocals of the factored diagonal block
  __shared__ float red[8];
  const int tid = threadIdx.x;
  {  // max |diagonal| (FP32 compare; only a scale for the pivot test)
    float mx = 0.f;
    for (int i = tid; i < n; i += blockDim.x) mx = fmaxf(mx, fabsf((float)L[(int64_t)i * ldL + i]));
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
      float m2 = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmaxf(m2, red[w]);
      amax_sh = (double)m2;
    }
    __syncthreads();
  }
  const double amax = amax_sh;
  bool bad = false;
  double minpiv = INFINITY;
  for (int kb = 0; kb < n; kb += NB) {
    const int nb = min(NB, n - kb);
    // 1. diagonal block in shared memory, unblocked Cholesky by warp 0
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      dg[i][j] = (i < nb && j <= i) ? L[(int64_t)(kb + i) * ldL + kb + j] : (T)0;
    }
    __syncthreads();
    if (tid < 32) {
      const int lane = tid;
      for (int k = 0; k < nb; ++k) {
        T dkk = dg[k][k];
        minpiv = fmin(minpiv, (double)dkk);
        if (!((double)dkk > 1e-14 * amax)) { bad = true; dkk = (T)(1e-14 * amax + 1e-300); }
        T lkk = sqrt(dkk);
        __syncwarp();
        if (lane == k) dg[k][k] = lkk;
        if (lane > k && lane < nb) dg[lane][k] = dg[lane][k] / lkk;
        __syncwarp();
        if (lane > k && lane < nb)
          for (int j = k + 1; j <= lane; ++j) dg[lane][j] -= dg[lane][k] * dg[j][k];
        __syncwarp();
      }
    }
    if (tid < NB) dinv[tid] = tid < nb ? 1.0 / (double)dg[tid][tid] : 0.0;  // divisions in parallel
    __syncthreads();
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      if (i < nb && j <= i) L[(int64_t)(kb + i) * ldL + kb + j] = dg[i][j];
    }
    // 2. panel rows below: X L_kk^T = A  (row-wise forward substitution)
    for (int i = kb + nb + tid; i < n; i += blockDim.x) {
      T* row = L + (int64_t)i * ldL + kb;
      T x[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) x[j] = j < nb ? row[j] : (T)0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j < nb) {
          T acc = x[j];
          for (int t = 0; t < j; ++t) acc -= x[t] * dg[j][t];
          x[j] = acc * (T)dinv[j];
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (j < nb) row[j] = x[j];
    }
    __syncthreads();
    // 3. trailing update A[i][j] -= sum_t L[i][kb+t] L[j][kb+t], j <= i
    const int t0 = kb + nb;
    for (int ti = t0; ti < n; ti += TS) {
      for (int tj = t0; tj <= ti; tj += TS) {
#pragma unroll
        for (int e0 = 0; e0 < TS * NB; e0 += 256) {  // all loads in flight together
          const int e = e0 + tid, r = e / NB, cc = e % NB;
          pa[r][cc] = (ti + r < n && cc < nb) ? L[(int64_t)(ti + r) * ldL + kb + cc] : (T)0;
          pb[r][cc] = (tj + r < n && cc < nb) ? L[(int64_t)(tj + r) * ldL + kb + cc] : (T)0;
        }
        __syncthreads();
        // 256 threads x 16 entries (4 x 4)
        const int ty = tid / 16, tx = tid % 16;
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int bq = 0; bq < 4; ++bq) acc[a][bq] = (T)0;
        for (int t = 0; t < NB; ++t) {
          T av[4], bv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = pa[ty * 4 + a][t];
#pragma unroll
          for (int bq = 0; bq < 4; ++bq) bv[bq] = pb[tx * 4 + bq][t];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int bq = 0; bq < 4; ++bq) acc[a][bq] += av[a] * bv[bq];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int bq = 0; bq < 4; ++bq) {
            int i = ti + ty * 4 + a, j = tj + tx * 4 + bq;
            if (i < n && j <= i) L[(int64_t)i * ldL + j] -= acc[a][bq];
          }
        __syncthreads();
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(status, KF_DEV_ILLCOND);
  if (tid == 0) pivr[node] = (n == 0 || amax == 0.0) ? 1.0 : fmax(minpiv, 0.0) / amax;
}

// ---- leaves on the tensor cores (mixed path) ---------------------------------------
// Panel kb (128 columns) of every leaf's Cholesky factorization, one CTA per
// leaf: the diagonal block L11 by an unblocked right-looking Cholesky in
// shared memory, written back in place, and its inverse Linv = L11^-1 (lower;
// column j by forward substitution) into the leaf's panel slot of Dinv, for
// the tcgen05 products that form the panel rows below and the trailing update
// (kf_tc_leaf_panel) and P^ (kf_tc_leaf_phat).  Pivots as k_leaf_cholesky: a
// pivot at most 1e-14 times the largest diagonal entry flags KF_DEV_ILLCOND;
// track[2 lf] keeps that entry, track[2 lf + 1] the smallest pivot so far.
constexpr int kPanel = 128;
__global__ void __launch_bounds__(256) k_chol_panel(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                    int leaf0, int ldL, float* __restrict__ Lall, int kb, int npan,
                                                    float* __restrict__ Dinv, double* __restrict__ track,
                                                    int32_t* __restrict__ status, double* __restrict__ pivr) {
  extern __shared__ float pan[];
  float(*Dm)[kPanel + 1] = (float(*)[kPanel + 1])pan;                         // L11
  float(*Im)[kPanel + 1] = (float(*)[kPanel + 1])(pan + kPanel * (kPanel + 1));  // L11^-1
  __shared__ float red[8];
  __shared__ float lkk_sh;
  __shared__ double amax_sh, minpiv_sh;
  __shared__ int bad_sh;
  const int lf = blockIdx.x, node = leaf0 + lf, tid = threadIdx.x;
  const int n = hi[node] - lo[node], nb = min(kPanel, n - kb);
  if (nb <= 0) return;
  float* L = Lall + (int64_t)lf * ldL * ldL;
  if (kb == 0) {  // max |diagonal| of A (FP32 compare; only a scale for the pivot test)
    float mx = 0.f;
    for (int i = tid; i < n; i += blockDim.x) mx = fmaxf(mx, fabsf(L[(int64_t)i * ldL + i]));
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
      float m2 = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmaxf(m2, red[w]);
      amax_sh = (double)m2;
      minpiv_sh = INFINITY;
    }
  } else if (tid == 0) {
    amax_sh = track[2 * lf];
    minpiv_sh = track[2 * lf + 1];
  }
  if (tid == 0) bad_sh = 0;
  for (int e = tid; e < kPanel * kPanel; e += blockDim.x) {
    const int i = e / kPanel, j = e % kPanel;
    Dm[i][j] = (i < nb && j <= i) ? L[(int64_t)(kb + i) * ldL + kb + j] : 0.f;
    Im[i][j] = 0.f;
  }
  __syncthreads();
  const double amax = amax_sh;
  for (int k = 0; k < nb; ++k) {
    if (tid == 0) {
      float dkk = Dm[k][k];
      minpiv_sh = fmin(minpiv_sh, (double)dkk);
      if (!((double)dkk > 1e-14 * amax)) {
        bad_sh = 1;
        dkk = (float)(1e-14 * amax + 1e-30);
      }
      lkk_sh = sqrtf(dkk);
      Dm[k][k] = lkk_sh;
    }
    __syncthreads();
    const float lkk = lkk_sh;
    for (int i = k + 1 + tid; i < nb; i += blockDim.x) Dm[i][k] = Dm[i][k] / lkk;
    __syncthreads();
    const int w = nb - k - 1;
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int i = k + 1 + e / w, j = k + 1 + e % w;
      if (j <= i) Dm[i][j] -= Dm[i][k] * Dm[j][k];
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    if (j <= i) L[(int64_t)(kb + i) * ldL + kb + j] = Dm[i][j];
  }
  if (tid < nb) {  // column tid of L11^-1
    const int j = tid;
    Im[j][j] = 1.f / Dm[j][j];
    for (int i = j + 1; i < nb; ++i) {
      float acc = 0.f;
      for (int t = j; t < i; ++t) acc = fmaf(Dm[i][t], Im[t][j], acc);
      Im[i][j] = -acc / Dm[i][i];
    }
  }
  __syncthreads();
  float* Di = Dinv + ((int64_t)lf * npan + kb / kPanel) * kPanel * kPanel;
  for (int e = tid; e < kPanel * kPanel; e += blockDim.x) Di[e] = Im[e / kPanel][e % kPanel];
  if (tid == 0) {
    if (bad_sh) atomicOr(status, KF_DEV_ILLCOND);
    track[2 * lf] = amax;
    track[2 * lf + 1] = minpiv_sh;
    if (kb + nb >= n) pivr[node] = (n == 0 || amax == 0.0) ? 1.0 : fmax(minpiv_sh, 0.0) / amax;
  }
}

__global__ void k_to_f32_rows(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// P^ = L^-T L^-1 P for one leaf per CTA; rhs = Pleaf rows of the leaf (FP64,
// N x s_max), out = Phat level D rows (type T).  Blocked by 32 rows: the
// diagonal block is solved with one thread per column, the rest of the
// matrix is updated with 64 x 64 register-tiled products.
template <typename T>
__device__ __forceinline__ void tile_update(T (*sa)[33], T (*sb)[65], int ty, int tx, int nb, T* Y, int ldy,
                                            int ti, int tj, int rows, int cols) {
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
#pragma unroll 8
  for (int t = 0; t < 32; ++t) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = sa[ty * 4 + a][t];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = sb[t][tx * 4 + b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = ti + ty * 4 + a, j = tj + tx * 4 + b;
      if (i < rows && j < cols) Y[(int64_t)i * ldy + j] -= acc[a][b];
    }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_leaf_phat(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                   const int32_t* __restrict__ rank, int leaf0, int ldL,
                                                   const T* __restrict__ Lall, const double* __restrict__ Pleaf,
                                                   int s_max, T* __restrict__ Phat) {
  constexpr int NB = 32, TS = 64;
  __shared__ T sa[TS][NB + 1];
  __shared__ T sb[NB][TS + 1];
  __shared__ T rdg[NB];  // reciprocals of the staged diagonal block
  const int lf = blockIdx.x, node = leaf0 + lf;
  const int b = lo[node], n = hi[node] - b, s = rank[node];
  const T* L = Lall + (int64_t)lf * ldL * ldL;
  T* Y = Phat + (int64_t)b * s_max;
  const double* P = Pleaf + (int64_t)b * s_max;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  for (int64_t e = tid; e < (int64_t)n * s_max; e += blockDim.x) {
    int i = (int)(e / s_max), q = (int)(e % s_max);
    Y[(int64_t)i * s_max + q] = q < s ? (T)P[(int64_t)i * s_max + q] : (T)0;
  }
  __syncthreads();
  if (s == 0) return;
  // forward: L y = p
  for (int kb = 0; kb < n; kb += NB) {
    const int nb = min(NB, n - kb);
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      sa[i][j] = (i < nb && j <= i) ? L[(int64_t)(kb + i) * ldL + kb + j] : (T)0;
    }
    __syncthreads();
    if (tid < NB) rdg[tid] = tid < nb ? (T)1 / sa[tid][tid] : (T)0;
    __syncthreads();
    for (int q = tid; q < s; q += blockDim.x) {
      T x[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) x[i] = i < nb ? Y[(int64_t)(kb + i) * s_max + q] : (T)0;
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < nb) {
          T acc = x[i];
#pragma unroll
          for (int t = 0; t < i; ++t) acc = fma(-sa[i][t], x[t], acc);
          x[i] = acc * rdg[i];
        }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < nb) Y[(int64_t)(kb + i) * s_max + q] = x[i];
    }
    __syncthreads();
    for (int ti = kb + nb; ti < n; ti += TS)
      for (int tj = 0; tj < s; tj += TS) {
#pragma unroll
        for (int e0 = 0; e0 < TS * NB; e0 += 256) {  // all loads in flight together
          const int e = e0 + tid, r = e / NB, cc = e % NB;
          sa[r][cc] = (ti + r < n && cc < nb) ? L[(int64_t)(ti + r) * ldL + kb + cc] : (T)0;
          const int rr = e / TS, c2 = e % TS;
          sb[rr][c2] = (rr < nb && tj + c2 < s) ? Y[(int64_t)(kb + rr) * s_max + tj + c2] : (T)0;
        }
        __syncthreads();
        tile_update<T>(sa, sb, ty, tx, nb, Y, s_max, ti, tj, n, s);
        __syncthreads();
      }
  }
  // backward: L^T x = y
  for (int kb = ((n - 1) / NB) * NB; kb >= 0; kb -= NB) {
    const int nb = min(NB, n - kb);
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      sa[i][j] = (i < nb && j <= i) ? L[(int64_t)(kb + i) * ldL + kb + j] : (T)0;
    }
    __syncthreads();
    if (tid < NB) rdg[tid] = tid < nb ? (T)1 / sa[tid][tid] : (T)0;
    __syncthreads();
    for (int q = tid; q < s; q += blockDim.x) {
      T x[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) x[i] = i < nb ? Y[(int64_t)(kb + i) * s_max + q] : (T)0;
#pragma unroll
      for (int i = NB - 1; i >= 0; --i)
        if (i < nb) {
          T acc = x[i];
#pragma unroll
          for (int t = i + 1; t < NB; ++t) acc = fma(-sa[t][i], x[t], acc);
          x[i] = acc * rdg[i];
        }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < nb) Y[(int64_t)(kb + i) * s_max + q] = x[i];
    }
    __syncthreads();
    // rows above: y[0:kb] -= L[kb:kb+nb, 0:kb]^T x_block
    for (int ti = 0; ti < kb; ti += TS)
      for (int tj = 0; tj < s; tj += TS) {
#pragma unroll
        for (int e0 = 0; e0 < TS * NB; e0 += 256) {  // all loads in flight together
          const int e = e0 + tid, r = e % TS, cc = e / TS;   // coalesced over r (contiguous in a row of L)
          sa[r][cc] = (ti + r < kb && cc < nb) ? L[(int64_t)(kb + cc) * ldL + ti + r] : (T)0;
          const int rr = e / TS, c2 = e % TS;
          sb[rr][c2] = (rr < nb && tj + c2 < s) ? Y[(int64_t)(kb + rr) * s_max + tj + c2] : (T)0;
        }
        __syncthreads();
        tile_update<T>(sa, sb, ty, tx, nb, Y, s_max, ti, tj, kb, s);
        __syncthreads();
      }
  }
}

// ---- V blocks: VT rows of every point of the level -------------------------------
// VT[i][q] = K(x_i, x_{skel(sib)[q]}) for the points i of every node of the
// level (FP64 path).  The sibling's skeleton coordinates are staged transposed
// in shared memory (yT[k][q]); one warp per row, lanes over q, coalesced stores.
template <typename T>
__global__ void __launch_bounds__(256) k_eval_vt(const double* __restrict__ X64, const float* __restrict__ X32, int d,
                                                 double c_exp, const int32_t* __restrict__ lo,
                                                 const int32_t* __restrict__ hi, const int32_t* __restrict__ rank,
                                                 const int32_t* __restrict__ skel, int s_max, int node0, int rows_per_cta,
                                                 int qchunk, T* __restrict__ VT) {
  extern __shared__ unsigned char smraw[];
  T* yT = (T*)smraw;                       // d x qchunk
  T* xs = yT + (size_t)d * qchunk;         // 8 warps x d
  const int nl = blockIdx.y, node = node0 + nl, sib = node ^ 1;
  const int b = lo[node], n = hi[node] - b, ss = rank[sib];
  const int r0 = blockIdx.x * rows_per_cta;
  if (r0 >= n || ss == 0) return;
  const int r1 = min(n, r0 + rows_per_cta);
  const int32_t* sk = skel + (int64_t)sib * s_max;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* xw = xs + warp * d;
  const T c = (T)c_exp;
  for (int q0 = 0; q0 < ss; q0 += qchunk) {
    const int qn = min(qchunk, ss - q0);
    __syncthreads();
    for (int e = threadIdx.x; e < d * qn; e += blockDim.x) {
      int k = e / qn, q = e % qn;
      int64_t src = (int64_t)sk[q0 + q] * d + k;
      yT[(size_t)k * qn + q] = sizeof(T) == 8 ? (T)X64[src] : (T)X32[src];
    }
    __syncthreads();
    for (int i = r0 + warp; i < r1; i += 8) {
      for (int k = lane; k < d; k += 32)
        xw[k] = sizeof(T) == 8 ? (T)X64[(int64_t)(b + i) * d + k] : (T)X32[(int64_t)(b + i) * d + k];
      __syncwarp();
      T* out = VT + (int64_t)(b + i) * s_max + q0;
      for (int q = lane; q < qn; q += 32) {
        T acc = (T)0;
        for (int k = 0; k < d; ++k) {
          T t = xw[k] - yT[(size_t)k * qn + q];
          acc = fma(t, t, acc);
        }
        out[q] = sizeof(T) == 8 ? (T)exp((double)(acc * c)) : (T)__expf((float)(acc * c));
      }
      __syncwarp();
    }
  }
}

// Mixed path: the same V blocks in FP32, plus (VTdf != nullptr) their FP64-
// accurate operator copy as double-float pairs, tiled 64 points x 64 skeleton
// columns per CTA with both
// coordinate tiles (hi and lo halves) staged transposed in shared memory and
// 4 x 4 entries per thread.  The FP32 value is exp(c |x - y|^2) of the FP32
// coordinates (as k_eval_vt); entries at or above 2^-24 of the operator copy
// take the double-float evaluation, which also replaces the FP32 value.
constexpr int kVT = 64;
__global__ void __launch_bounds__(256) k_eval_vt_tiled(const float* __restrict__ X32, const float* __restrict__ X32lo,
                                                       int d, double c_exp, const int32_t* __restrict__ lo,
                                                       const int32_t* __restrict__ hi,
                                                       const int32_t* __restrict__ rank,
                                                       const int32_t* __restrict__ skel, int s_max, int node0,
                                                       float* __restrict__ VT, float2* __restrict__ VTdf, float ch,
                                                       float cl, const float2* __restrict__ tab) {
  extern __shared__ float vts[];  // x hi, x lo, y hi, y lo: d x 64 each
  const int nl = blockIdx.z, node = node0 + nl, sib = node ^ 1;
  const int b = lo[node], n = hi[node] - b, ss = rank[sib];
  const int r0 = blockIdx.x * kVT, q0 = blockIdx.y * kVT;
  if (r0 >= n || q0 >= ss) return;
  const int32_t* sk = skel + (int64_t)sib * s_max;
  float* xh = vts;
  float* xl = xh + d * kVT;
  float* yh = xl + d * kVT;
  float* yl = yh + d * kVT;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool df = VTdf != nullptr;
  for (int e = tid; e < d * kVT; e += blockDim.x) {
    const int k = e % d, r = e / d;
    const int pi = r0 + r, pq = q0 + r;
    const int64_t xi = (int64_t)(b + min(pi, n - 1)) * d + k;
    const int64_t yi = (int64_t)sk[min(pq, ss - 1)] * d + k;
    xh[k * kVT + r] = X32[xi];
    yh[k * kVT + r] = X32[yi];
    if (df) {
      xl[k * kVT + r] = X32lo[xi];
      yl[k * kVT + r] = X32lo[yi];
    }
  }
  __syncthreads();
  float a32[4][4], ah[4][4], al[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) a32[a][c] = ah[a][c] = al[a][c] = 0.f;
  if (df) {
    for (int k = 0; k < d; ++k) {
      const float4 x4h = *(const float4*)(xh + k * kVT + ty * 4), x4l = *(const float4*)(xl + k * kVT + ty * 4);
      const float4 y4h = *(const float4*)(yh + k * kVT + tx * 4), y4l = *(const float4*)(yl + k * kVT + tx * 4);
      const float xhv[4] = {x4h.x, x4h.y, x4h.z, x4h.w}, xlv[4] = {x4l.x, x4l.y, x4l.z, x4l.w};
      const float yhv[4] = {y4h.x, y4h.y, y4h.z, y4h.w}, ylv[4] = {y4l.x, y4l.y, y4l.z, y4l.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float th, te;
          kf_two_sum(xhv[a], -yhv[c], th, te);  // th = fl(x - y): the FP32 difference
          a32[a][c] = fmaf(th, th, a32[a][c]);
          const float tl = te + (xlv[a] - ylv[c]);
          const float p = __fmul_rn(th, th);
          const float q = fmaf(th, th, -p) + 2.f * th * tl;
          float sh, se;
          kf_two_sum(ah[a][c], p, sh, se);
          se = __fadd_rn(se, __fadd_rn(al[a][c], q));
          ah[a][c] = __fadd_rn(sh, se);
          al[a][c] = __fsub_rn(se, __fsub_rn(ah[a][c], sh));
        }
    }
  } else {
    for (int k = 0; k < d; ++k) {
      const float4 x4 = *(const float4*)(xh + k * kVT + ty * 4);
      const float4 y4 = *(const float4*)(yh + k * kVT + tx * 4);
      const float xv[4] = {x4.x, x4.y, x4.z, x4.w}, yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float t = xv[a] - yv[c];
          a32[a][c] = fmaf(t, t, a32[a][c]);
        }
    }
  }
  const float c32 = (float)c_exp;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = r0 + ty * 4 + a;
    if (i >= n) continue;
    const int64_t row = (int64_t)(b + i) * s_max;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int q = q0 + tx * 4 + c;
      if (q >= ss) continue;
      float kv = __expf(a32[a][c] * c32);
      if (df) {
        float2 kd = make_float2(kv, 0.f);
        if (kv >= 5.9604645e-8f) kd = kf_kern_from_df(ah[a][c], al[a][c], ch, cl, tab);
        VTdf[row + q] = kd;
        kv = kd.x;  // hi is the pair rounded to FP32
      }
      VT[row + q] = kv;
    }
  }
}

// ---- Z = I + [[0, K_{l~r} P^_r], [K_{r~l} P^_l, 0]] --------------------------------
__global__ void k_z_init(const int32_t* __restrict__ rank, int node0, int ldz, double* __restrict__ Z) {
  const int nl = blockIdx.y, node = node0 + nl;
  const int z = rank[2 * node] + rank[2 * node + 1];
  double* Zb = Z + (int64_t)node * ldz * ldz;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)ldz * ldz;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / ldz), j = (int)(e % ldz);
    Zb[e] = (i == j && i < z) ? 1.0 : 0.0;
  }
}

// Off-diagonal blocks by a "TN" product with a long reduction over the
// child's rows: C (s_a x s_b) += VT_c[:, :s_a]^T P^_c[:, :s_b], c = the child
// whose rows are summed.  Tiles of 64 x 64, split over the rows; FP64 atomics.
template <typename T>
__global__ void __launch_bounds__(256) k_zoff(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                              const int32_t* __restrict__ rank, int node0, int s_max,
                                              const T* __restrict__ VT, const T* __restrict__ Ph, int ldz,
                                              double* __restrict__ Z, int ksplit, double* __restrict__ parts) {
  using A = typename Acc<T>::type;
  constexpr int TS = 64, KC = 16;
  __shared__ T sa[KC][TS];
  __shared__ T sb[KC][TS];
  const int side = blockIdx.z & 1, nl = blockIdx.z >> 1, node = node0 + nl;
  const int l = 2 * node, r = l + 1;
  const int sl = rank[l], sr = rank[r];
  // side 0: rows of r, M = s_l (VT cols), N = s_r (P^ cols), block Z[0:sl, sl:]
  // side 1: rows of l, M = s_r, N = s_l, block Z[sl:, 0:sl]
  const int c = side == 0 ? r : l;
  const int M = side == 0 ? sl : sr, Nn = side == 0 ? sr : sl;
  const int tm = blockIdx.x / ((Nn + TS - 1) / TS + (Nn == 0)), tn = blockIdx.x % ((Nn + TS - 1) / TS + (Nn == 0));
  if (M == 0 || Nn == 0 || tm * TS >= M || tn * TS >= Nn) return;
  const int rb = lo[c], rn = hi[c] - rb;
  const int kchunk = (rn + ksplit - 1) / ksplit;
  const int k0 = blockIdx.y * kchunk, k1 = min(rn, k0 + kchunk);
  if (k0 >= k1) return;
  const T* Ab = VT + (int64_t)rb * s_max;
  const T* Bb = Ph + (int64_t)rb * s_max;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  A acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (A)0;
  for (int kk = k0; kk < k1; kk += KC) {
    for (int e = tid; e < KC * TS; e += blockDim.x) {
      int kr = e / TS, cc = e % TS;
      int row = kk + kr;
      int ca = tm * TS + cc, cb = tn * TS + cc;
      sa[kr][cc] = (row < k1 && ca < M) ? Ab[(int64_t)row * s_max + ca] : (T)0;
      sb[kr][cc] = (row < k1 && cb < Nn) ? Bb[(int64_t)row * s_max + cb] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < KC; ++t) {
      A av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = (A)sa[t][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = (A)sb[t][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
  // one writer per entry without a split; with one, the partial tile goes to
  // parts[tile][ks] and k_zoff_reduce64 adds the parts in ks order
  double* Zb = Z + (int64_t)node * ldz * ldz;
  double* pt = parts + (((int64_t)blockIdx.z * gridDim.x + blockIdx.x) * ksplit + blockIdx.y) * TS * TS;
  const int roff = side == 0 ? 0 : sl, coff = side == 0 ? sl : 0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = tm * TS + ty * 4 + a, j = tn * TS + tx * 4 + b;
      if (i < M && j < Nn) {
        if (ksplit == 1) Zb[(int64_t)(roff + i) * ldz + coff + j] += (double)acc[a][b];
        else pt[(ty * 4 + a) * TS + tx * 4 + b] = (double)acc[a][b];
      }
    }
}

// the split-K parts of k_zoff added in ks order (the same tile mapping)
__global__ void __launch_bounds__(256) k_zoff_reduce64(const int32_t* __restrict__ rank, int node0, int ldz,
                                                       int ksplit, const double* __restrict__ parts,
                                                       double* __restrict__ Z) {
  constexpr int TS = 64;
  const int side = blockIdx.y & 1, node = node0 + (blockIdx.y >> 1);
  const int sl = rank[2 * node], sr = rank[2 * node + 1];
  const int M = side == 0 ? sl : sr, Nn = side == 0 ? sr : sl;
  const int nt = (Nn + TS - 1) / TS + (Nn == 0);
  const int tm = blockIdx.x / nt, tn = blockIdx.x % nt;
  if (M == 0 || Nn == 0 || tm * TS >= M || tn * TS >= Nn) return;
  const double* pt = parts + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * ksplit * TS * TS;
  double* Zb = Z + (int64_t)node * ldz * ldz;
  const int roff = side == 0 ? 0 : sl, coff = side == 0 ? sl : 0;
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
    const int i = tm * TS + e / TS, j = tn * TS + e % TS;
    if (i >= M || j >= Nn) continue;
    double sum = 0.0;
    for (int ks = 0; ks < ksplit; ++ks) sum += pt[(int64_t)ks * TS * TS + e];
    Zb[(int64_t)(roff + i) * ldz + coff + j] += sum;
  }
}

// Blocked LU with partial pivoting of Z (FP64) followed, for non-root nodes,
// by T = Z^-1 P_c.  Row pivoting is implicit: rm[i] is the row of Z that
// holds logical row i of the factorization (P Z = L U with (P Z)[i] =
// Z[rm[i]]), so a pivot interchange swaps two entries of rm and no data.
//   panel:    32 columns at a time; per column an arg-max over the logical
//             rows (ties: lowest), the interchange, scaling, and the rank-1
//             update restricted to the panel;
//   U12:      L11^-1 A12 by the 32 x 32 unit-lower block;
//   trailing: A22 -= L21 U12, 64 x 64 register-tiled FP64 tiles;
// then X[i] = P_c[rm[i]], L y = x and U t = y by 32-row blocks (diagonal
// block per column thread, off-block updates tiled).  rm is stored per node
// (the solve sweep reads it).
// k_z_factor runs one CTA per node.  k_z_factor_cluster spreads a node over
// a thread-block cluster for the upper levels (few nodes): CTA 0 factors each
// panel, the cluster shares U12 and the trailing tiles (a cluster barrier
// between the phases), and each CTA solves its own slice of the columns of
// P_c.  Z is read with L2-only loads there, since other CTAs write it between
// the phases.
constexpr int kZNB = 32, kZTS = 64;

struct ZShared {
  double sa[kZTS][kZNB + 1];
  double sb[kZNB][kZTS + 1];
  double sinv[kZNB];  // reciprocals of a staged diagonal block
  double prow[kZNB];
  double pinv;  // 1 / pivot of the current panel column
  int rm[2 * KF_MAX_SMAX];
  double rv[8];
  int ri[8];
  int pk;
  double amax;
};

// L2 selects L2-only loads (the cluster kernel: other CTAs write Z between phases)
template <bool L2>
__device__ __forceinline__ double zld(const double* p) {
  if (L2) return __ldcg(p);
  return *p;
}

template <bool L2>
__device__ double z_absmax(const double* A, int ldz, int z, ZShared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the bit patterns of |v| order like the values: integer max keeps this off the FP64 pipe
  long long mx = 0;
  for (int i = tid / 32; i < z; i += blockDim.x / 32)
    for (int c = lane; c < z; c += 32) mx = max(mx, __double_as_longlong(zld<L2>(A + (int64_t)i * ldz + c)) & 0x7fffffffffffffffll);
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if (lane == 0) sh.rv[warp] = __longlong_as_double(mx);
  __syncthreads();
  if (tid == 0) {
    long long m2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = max(m2, __double_as_longlong(sh.rv[w]));
    sh.amax = __longlong_as_double(m2);
  }
  __syncthreads();
  return sh.amax;
}

// columns kb..kb+nb-1 of logical rows kb..z-1, one CTA
template <bool L2>
__device__ void zlu_panel(double* A, int ldz, int z, int kb, int nb, double amax, bool& bad, double& umin,
                          double& umax, ZShared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int* rm = sh.rm;
  for (int j = kb; j < kb + nb; ++j) {
    // arg-max of |A| by integer compares of the bit patterns (same order)
    long long bv = -1;
    int bi = z;
    for (int i = j + tid; i < z; i += blockDim.x) {
      const long long v = __double_as_longlong(zld<L2>(A + (int64_t)rm[i] * ldz + j)) & 0x7fffffffffffffffll;
      if (v > bv) { bv = v; bi = i; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const long long ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { sh.rv[warp] = __longlong_as_double(bv); sh.ri[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      long long b2 = -1;
      int i2 = z;
      for (int w = 0; w < nw; ++w) {
        const long long v = __double_as_longlong(sh.rv[w]);
        if (v > b2 || (v == b2 && sh.ri[w] < i2)) { b2 = v; i2 = sh.ri[w]; }
      }
      const int t = rm[j];
      rm[j] = rm[i2];
      rm[i2] = t;
    }
    __syncthreads();
    const double* Aj = A + (int64_t)rm[j] * ldz;
    for (int c = j + tid; c < kb + nb; c += blockDim.x) {
      const double a = zld<L2>(Aj + c);
      sh.prow[c - kb] = a;
      if (c == j) {  // thread 0: the pivot; one FP64 division for the whole CTA
        umin = fmin(umin, fabs(a));
        umax = fmax(umax, fabs(a));
        if (!(fabs(a) > 1e-14 * amax)) bad = true;
        sh.pinv = a != 0.0 ? 1.0 / a : 0.0;
      }
    }
    __syncthreads();
    const double inv = sh.pinv;
    const int jj = j - kb;
    for (int i = j + 1 + tid; i < z; i += blockDim.x) {
      double* Ai = A + (int64_t)rm[i] * ldz + kb;
      double v[kZNB];
#pragma unroll
      for (int c = 0; c < kZNB; ++c) v[c] = (c > jj && c < nb) ? zld<L2>(Ai + c) : 0.0;
      const double l = zld<L2>(Ai + jj) * inv;
#pragma unroll
      for (int c = 0; c < kZNB; ++c)
        if (c > jj && c < nb) Ai[c] = fma(-l, sh.prow[c], v[c]);
      Ai[jj] = l;
    }
    __syncthreads();
  }
}

// U12 = L11^-1 A12 for the columns of part `part` of `nparts` (thread per column)
template <bool L2>
__device__ void zlu_trsm(double* A, int ldz, int z, int kb, int nb, int part, int nparts, ZShared& sh) {
  const int tid = threadIdx.x;
  const int* rm = sh.rm;
#pragma unroll 4
  for (int e = tid; e < kZNB * kZNB; e += blockDim.x) {
    int i = e / kZNB, j = e % kZNB;
    sh.sa[i][j] = (i < nb && j < i) ? zld<L2>(A + (int64_t)rm[kb + i] * ldz + kb + j) : 0.0;
  }
  __syncthreads();
  for (int c = kb + nb + part * (int)blockDim.x + tid; c < z; c += nparts * (int)blockDim.x) {
    double x[kZNB];
#pragma unroll
    for (int r = 0; r < kZNB; ++r) x[r] = r < nb ? zld<L2>(A + (int64_t)rm[kb + r] * ldz + c) : 0.0;
#pragma unroll
    for (int r = 1; r < kZNB; ++r) {
      double acc = x[r];
#pragma unroll
      for (int t = 0; t < r; ++t) acc = fma(-sh.sa[r][t], x[t], acc);
      x[r] = acc;
    }
#pragma unroll
    for (int r = 1; r < kZNB; ++r)
      if (r < nb) A[(int64_t)rm[kb + r] * ldz + c] = x[r];
  }
  __syncthreads();
}

// C[r0 + i][q0 + j] -= sum_t Lp[i][t] Rp[t][j] over a 64 x TC tile, t < nb:
// Lp rows from A (row stride ldz, columns k0..k0+nb), Rp rows k0..k0+nb of B
// (row stride ldb); mA, mB, mC map logical rows to stored rows (nullptr:
// identity).  Rows < rlim and columns < climit are valid.  256 threads: 16
// row groups of 4 rows x 16 column groups of TC/16 columns.
template <int TC, bool L2>
__device__ void z_tile_sub(const double* A, int ldz, const int* mA, const double* B, int ldb, const int* mB,
                           double* C, int ldc, const int* mC, int r0, int rlim, int q0, int climit, int k0, int nb,
                           ZShared& sh) {
  constexpr int CB = TC / 16;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
#pragma unroll
  for (int e0 = 0; e0 < kZTS * kZNB; e0 += 256) {
    const int e = e0 + tid, r = e / kZNB, cc = e % kZNB;
    const int row = r0 + r;
    sh.sa[r][cc] = (row < rlim && cc < nb) ? zld<L2>(A + (int64_t)(mA ? mA[row] : row) * ldz + k0 + cc) : 0.0;
  }
#pragma unroll
  for (int e0 = 0; e0 < kZNB * TC; e0 += 256) {
    const int e = e0 + tid, rr = e / TC, c2 = e % TC;
    if (rr < kZNB) {
      const int row = k0 + rr;
      sh.sb[rr][c2] = (rr < nb && q0 + c2 < climit) ? zld<L2>(B + (int64_t)(mB ? mB[row] : row) * ldb + q0 + c2) : 0.0;
    }
  }
  __syncthreads();
  double acc[4][CB] = {};
#pragma unroll 8
  for (int t = 0; t < kZNB; ++t) {
    double av[4], bv[CB];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = sh.sa[ty * 4 + a][t];
#pragma unroll
    for (int b = 0; b < CB; ++b) bv[b] = sh.sb[t][tx * CB + b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < CB; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = r0 + ty * 4 + a;
    if (i >= rlim) continue;
    double* Ci = C + (int64_t)(mC ? mC[i] : i) * ldc;
#pragma unroll
    for (int b = 0; b < CB; ++b) {
      const int j = q0 + tx * CB + b;
      if (j < climit) Ci[j] = zld<L2>(Ci + j) - acc[a][b];
    }
  }
  __syncthreads();
}

// A22 -= L21 U12 for the tiles of part `part` of `nparts`
template <bool L2>
__device__ void zlu_update(double* A, int ldz, int z, int kb, int nb, int part, int nparts, ZShared& sh) {
  const int c0 = kb + nb;
  const int nt = (z - c0 + kZTS - 1) / kZTS;
  for (int t = part; t < nt * nt; t += nparts) {
    const int ti = c0 + (t / nt) * kZTS, tj = c0 + (t % nt) * kZTS;
    z_tile_sub<kZTS, L2>(A, ldz, sh.rm, A, ldz, sh.rm, A, ldz, sh.rm, ti, z, tj, z, kb, nb, sh);
  }
}

// X[:, q0:q1) = Z^-1 B[:, q0:q1) from the LU in A (columns >= s are zero;
// B = nullptr stands for the identity, so that X is Z^-1); s_max is the row
// stride of B and X
template <int TC, bool L2>
__device__ void z_solve_cols_impl(const double* A, int ldz, int z, const double* B, double* X, int s_max, int s,
                                  int q0, int q1, ZShared& sh);

// ... and, when X32 is given, an FP32 copy of the same columns (the mixed
// path's telescoping reads T in FP32)
template <int TC, bool L2>
__device__ void z_solve_cols(const double* A, int ldz, int z, const double* B, double* X, float* X32, int s_max,
                             int s, int q0, int q1, ZShared& sh) {
  z_solve_cols_impl<TC, L2>(A, ldz, z, B, X, s_max, s, q0, q1, sh);
  if (X32 == nullptr) return;
  __syncthreads();
  const int qw = q1 - q0;
  for (int64_t e = threadIdx.x; e < (int64_t)ldz * qw; e += blockDim.x) {
    const int64_t o = (e / qw) * s_max + q0 + e % qw;
    X32[o] = (float)X[o];
  }
}

template <int TC, bool L2>
__device__ void z_solve_cols_impl(const double* A, int ldz, int z, const double* B, double* X, int s_max, int s,
                                  int q0, int q1, ZShared& sh) {
  const int tid = threadIdx.x;
  const int qw = q1 - q0;
  const int* rm = sh.rm;
  for (int64_t e = tid; e < (int64_t)ldz * qw; e += blockDim.x) {
    int i = (int)(e / qw), q = q0 + (int)(e % qw);
    X[(int64_t)i * s_max + q] = (i < z && q < s) ? (B ? B[(int64_t)rm[i] * s_max + q] : (rm[i] == q ? 1.0 : 0.0))
                                                 : 0.0;
  }
  __syncthreads();
  const int qe = min(q1, s);
  if (qe <= q0 || z == 0) return;
  // forward: L (unit lower)
  for (int kb = 0; kb < z; kb += kZNB) {
    const int nb = min(kZNB, z - kb);
#pragma unroll 4
    for (int e = tid; e < kZNB * kZNB; e += blockDim.x) {
      int i = e / kZNB, j = e % kZNB;
      sh.sa[i][j] = (i < nb && j < i) ? zld<L2>(A + (int64_t)rm[kb + i] * ldz + kb + j) : 0.0;
    }
    __syncthreads();
    for (int q = q0 + tid; q < qe; q += blockDim.x) {
      double x[kZNB];
#pragma unroll
      for (int r = 0; r < kZNB; ++r) x[r] = r < nb ? X[(int64_t)(kb + r) * s_max + q] : 0.0;
#pragma unroll
      for (int r = 1; r < kZNB; ++r) {
        double acc = x[r];
#pragma unroll
        for (int t = 0; t < r; ++t) acc = fma(-sh.sa[r][t], x[t], acc);
        x[r] = acc;
      }
#pragma unroll
      for (int r = 1; r < kZNB; ++r)
        if (r < nb) X[(int64_t)(kb + r) * s_max + q] = x[r];
    }
    __syncthreads();
    for (int ti = kb + nb; ti < z; ti += kZTS)
      for (int tj = q0; tj < qe; tj += TC)
        z_tile_sub<TC, L2>(A, ldz, rm, X, s_max, nullptr, X, s_max, nullptr, ti, z, tj, qe, kb, nb, sh);
  }
  // backward: U
  for (int kb = ((z - 1) / kZNB) * kZNB; kb >= 0; kb -= kZNB) {
    const int nb = min(kZNB, z - kb);
#pragma unroll 4
    for (int e = tid; e < kZNB * kZNB; e += blockDim.x) {
      int i = e / kZNB, j = e % kZNB;
      sh.sa[i][j] = (i < nb && j < nb && j >= i) ? zld<L2>(A + (int64_t)rm[kb + i] * ldz + kb + j) : 0.0;
    }
    __syncthreads();
    if (tid < kZNB) sh.sinv[tid] = tid < nb ? 1.0 / sh.sa[tid][tid] : 0.0;  // divisions in parallel
    __syncthreads();
    for (int q = q0 + tid; q < qe; q += blockDim.x) {
      double x[kZNB];
#pragma unroll
      for (int r = 0; r < kZNB; ++r) x[r] = r < nb ? X[(int64_t)(kb + r) * s_max + q] : 0.0;
#pragma unroll
      for (int r = kZNB - 1; r >= 0; --r) {
        if (r < nb) {
          double acc = x[r];
#pragma unroll
          for (int t = r + 1; t < kZNB; ++t) acc = fma(-sh.sa[r][t], x[t], acc);
          x[r] = acc * sh.sinv[r];
        }
      }
#pragma unroll
      for (int r = 0; r < kZNB; ++r)
        if (r < nb) X[(int64_t)(kb + r) * s_max + q] = x[r];
    }
    __syncthreads();
    // rows above: X[0:kb] -= U[0:kb, kb:kb+nb] X[kb:kb+nb]
    for (int ti = 0; ti < kb; ti += kZTS)
      for (int tj = q0; tj < qe; tj += TC)
        z_tile_sub<TC, L2>(A, ldz, rm, X, s_max, nullptr, X, s_max, nullptr, ti, kb, tj, qe, kb, nb, sh);
  }
}

__global__ void __launch_bounds__(256) k_z_factor(const int32_t* __restrict__ rank, int node0, int ldz, int s_max,
                                                  double* __restrict__ Z, int32_t* __restrict__ piv,
                                                  const double* __restrict__ Pc, double* __restrict__ T,
                                                  float* __restrict__ T32, int solve_pc, int32_t* __restrict__ status,
                                                  double* __restrict__ pivr) {
  __shared__ ZShared sh;
  const int nl = blockIdx.x, node = node0 + nl;
  const int z = rank[2 * node] + rank[2 * node + 1];
  double* A = Z + (int64_t)node * ldz * ldz;
  int32_t* pv = piv + (int64_t)node * ldz;
  for (int i = threadIdx.x; i < z; i += blockDim.x) sh.rm[i] = i;
  const double amax = z_absmax<false>(A, ldz, z, sh);
  bool bad = false;
  double umin = INFINITY, umax = 0.0;
  for (int kb = 0; kb < z; kb += kZNB) {
    const int nb = min(kZNB, z - kb);
    zlu_panel<false>(A, ldz, z, kb, nb, amax, bad, umin, umax, sh);
    if (kb + nb >= z) break;
    zlu_trsm<false>(A, ldz, z, kb, nb, 0, 1, sh);
    zlu_update<false>(A, ldz, z, kb, nb, 0, 1, sh);
  }
  for (int i = threadIdx.x; i < z; i += blockDim.x) pv[i] = sh.rm[i];
  if (bad && threadIdx.x == 0) atomicOr(status, KF_DEV_ILLCOND);
  if (threadIdx.x == 0) pivr[node] = (z == 0 || umax == 0.0) ? 1.0 : umin / umax;
  if (!solve_pc) return;
  z_solve_cols<kZTS, false>(A, ldz, z, Pc + (int64_t)node * ldz * s_max, T + (int64_t)nl * ldz * s_max,
                            T32 ? T32 + (int64_t)nl * ldz * s_max : nullptr, s_max, rank[node], 0, s_max, sh);
}

// Z^-1 of the nodes of a level from their LU (rows stored in pivot order,
// row map piv): blockIdx.x = node, blockIdx.y = a block of qw columns of the
// identity, solved with the tiled L and U sweeps of z_solve_cols.
__global__ void __launch_bounds__(256) k_z_inverse(const int32_t* __restrict__ rank, int node0, int ldz,
                                                   const double* __restrict__ ZLU, const int32_t* __restrict__ piv,
                                                   double* __restrict__ Zinv, int qw) {
  __shared__ ZShared sh;
  const int node = node0 + blockIdx.x;
  const int z = rank[2 * node] + rank[2 * node + 1];
  const int q0 = blockIdx.y * qw;
  if (q0 >= z) return;
  for (int i = threadIdx.x; i < z; i += blockDim.x) sh.rm[i] = piv[(int64_t)node * ldz + i];
  __syncthreads();
  z_solve_cols_impl<16, false>(ZLU + (int64_t)node * ldz * ldz, ldz, z, nullptr, Zinv + (int64_t)node * ldz * ldz,
                               ldz, z, q0, min(q0 + qw, ldz), sh);
}

// cluster size is set at launch (cudaLaunchAttributeClusterDimension)
__global__ void __launch_bounds__(256) k_z_factor_cluster(const int32_t* __restrict__ rank, int node0, int ldz,
                                                          int s_max, double* __restrict__ Z,
                                                          int32_t* __restrict__ piv, const double* __restrict__ Pc,
                                                          double* __restrict__ T, float* __restrict__ T32,
                                                          int solve_pc, int32_t* __restrict__ status,
                                                          double* __restrict__ pivr) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ ZShared sh;
  const int cr = (int)cluster.block_rank(), nc = (int)cluster.num_blocks();
  const int nl = blockIdx.x / nc, node = node0 + nl;
  const int z = rank[2 * node] + rank[2 * node + 1];
  double* A = Z + (int64_t)node * ldz * ldz;
  int32_t* pv = piv + (int64_t)node * ldz;
  for (int i = threadIdx.x; i < z; i += blockDim.x) sh.rm[i] = i;
  double amax = 0.0;
  if (cr == 0) amax = z_absmax<true>(A, ldz, z, sh);
  bool bad = false;
  double umin = INFINITY, umax = 0.0;
  // CTA 0 owns the row map; the others take it from pv after each panel
  for (int kb = 0; kb < z; kb += kZNB) {  // the same trip count in every CTA of the cluster
    const int nb = min(kZNB, z - kb);
    if (cr == 0) {
      zlu_panel<true>(A, ldz, z, kb, nb, amax, bad, umin, umax, sh);
      for (int i = kb + threadIdx.x; i < z; i += blockDim.x) pv[i] = sh.rm[i];
    }
    cluster.sync();
    if (cr != 0) {
      for (int i = kb + threadIdx.x; i < z; i += blockDim.x) sh.rm[i] = __ldcg(pv + i);
      __syncthreads();
    }
    if (kb + nb >= z) break;
    zlu_trsm<true>(A, ldz, z, kb, nb, cr, nc, sh);
    cluster.sync();
    zlu_update<true>(A, ldz, z, kb, nb, cr, nc, sh);
    cluster.sync();
  }
  if (cr == 0 && threadIdx.x == 0) {
    if (bad) atomicOr(status, KF_DEV_ILLCOND);
    pivr[node] = (z == 0 || umax == 0.0) ? 1.0 : umin / umax;
  }
  if (!solve_pc) return;
  const int qn = (s_max + nc - 1) / nc;
  const int q0 = min(s_max, cr * qn), q1 = min(s_max, q0 + qn);
  z_solve_cols<16, true>(A, ldz, z, Pc + (int64_t)node * ldz * s_max, T + (int64_t)nl * ldz * s_max,
                         T32 ? T32 + (int64_t)nl * ldz * s_max : nullptr, s_max, rank[node], q0, q1, sh);
}

// Telescoping GEMM: P^_a[rows of c, :s_a] = P^_c[:, :s_c] T[c block, :s_a].
template <typename T>
__global__ void __launch_bounds__(256) k_telescope(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                   const int32_t* __restrict__ rank, int node0, int s_max,
                                                   const T* __restrict__ Pc_hat, const double* __restrict__ Tm,
                                                   int ldz, T* __restrict__ Pa_hat) {
  using A = typename Acc<T>::type;
  constexpr int TM = 64, TN = 64, KC = 16;
  __shared__ T sa[TM][KC + 1];
  __shared__ T sb[KC][TN];
  const int side = blockIdx.z & 1, nl = blockIdx.z >> 1, node = node0 + nl;
  const int c = 2 * node + side;
  const int sc = rank[c], sa_ = rank[node], sl = rank[2 * node];
  const int rb = lo[c], rn = hi[c] - rb;
  const int tm = blockIdx.x, tn = blockIdx.y;
  if (tm * TM >= rn || tn * TN >= sa_) return;
  const T* Ab = Pc_hat + (int64_t)rb * s_max;
  const double* Bb = Tm + (int64_t)nl * ldz * s_max + (int64_t)(side == 0 ? 0 : sl) * s_max;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  A acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (A)0;
  for (int kk = 0; kk < sc; kk += KC) {
    for (int e = tid; e < TM * KC; e += blockDim.x) {
      int rr = e / KC, kc = e % KC;
      int row = tm * TM + rr, k = kk + kc;
      sa[rr][kc] = (row < rn && k < sc) ? Ab[(int64_t)row * s_max + k] : (T)0;
    }
    for (int e = tid; e < KC * TN; e += blockDim.x) {
      int kr = e / TN, cc = e % TN;
      int k = kk + kr, col = tn * TN + cc;
      sb[kr][cc] = (k < sc && col < sa_) ? (T)Bb[(int64_t)k * s_max + col] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < KC; ++t) {
      A av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = (A)sa[ty * 4 + a][t];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = (A)sb[t][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = tm * TM + ty * 4 + a, j = tn * TN + tx * 4 + b;
      if (i < rn && j < sa_) Pa_hat[(int64_t)(rb + i) * s_max + j] = (T)acc[a][b];
    }
}

// FP64-accurate copy of the leaf kernel blocks (no lambda) as double-float
// pairs, both triangles, for the operator.  One CTA per 64 x 64 tile (I, J) of a leaf block
// with I <= J, written to (I, J) and, transposed, to (J, I); the tile's
// coordinates (double-float, hi + lo) are staged in shared memory, transposed
// so that a thread's 4 rows and 4 columns are 4 consecutive words.  Entries
// below 2^-24 take the FP32 value exp(c d_hi), the rest kf_kern_from_df.
constexpr int kK64T = 64;
__global__ void __launch_bounds__(256) k_leaf_k64(const float* __restrict__ X32lo, const float* __restrict__ X32,
                                                  int d, double c_exp, const int32_t* __restrict__ lo,
                                                  const int32_t* __restrict__ hi, int leaf0, int ldL,
                                                  float2* __restrict__ Kdf, float ch, float cl,
                                                  const float2* __restrict__ tab) {
  extern __shared__ float k64s[];  // 4 arrays of d x 64: x hi, x lo, y hi, y lo
  const int lf = blockIdx.y, node = leaf0 + lf;
  const int b = lo[node], n = hi[node] - b;
  const int nt = (n + kK64T - 1) / kK64T;
  // tile index -> (I, J), I <= J, row by row of the upper triangle
  int t = blockIdx.x, I = 0;
  while (I < nt && t >= nt - I) { t -= nt - I; ++I; }
  if (I >= nt) return;
  const int J = I + t;
  float* xh = k64s;
  float* xl = xh + d * kK64T;
  float* yh = xl + d * kK64T;
  float* yl = yh + d * kK64T;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < d * kK64T; e += blockDim.x) {
    const int k = e % d, r = e / d;  // coalesced over (point, dim)
    const int pi = I * kK64T + r, pj = J * kK64T + r;
    xh[k * kK64T + r] = pi < n ? X32[(int64_t)(b + pi) * d + k] : 0.f;
    xl[k * kK64T + r] = pi < n ? X32lo[(int64_t)(b + pi) * d + k] : 0.f;
    yh[k * kK64T + r] = pj < n ? X32[(int64_t)(b + pj) * d + k] : 0.f;
    yl[k * kK64T + r] = pj < n ? X32lo[(int64_t)(b + pj) * d + k] : 0.f;
  }
  __syncthreads();
  float ah[4][4], al[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) ah[a][c] = al[a][c] = 0.f;
  for (int k = 0; k < d; ++k) {
    const float4 x4h = *(const float4*)(xh + k * kK64T + ty * 4), x4l = *(const float4*)(xl + k * kK64T + ty * 4);
    const float4 y4h = *(const float4*)(yh + k * kK64T + tx * 4), y4l = *(const float4*)(yl + k * kK64T + tx * 4);
    const float xhv[4] = {x4h.x, x4h.y, x4h.z, x4h.w}, xlv[4] = {x4l.x, x4l.y, x4l.z, x4l.w};
    const float yhv[4] = {y4h.x, y4h.y, y4h.z, y4h.w}, ylv[4] = {y4l.x, y4l.y, y4l.z, y4l.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float th, te;
        kf_two_sum(xhv[a], -yhv[c], th, te);
        const float tl = te + (xlv[a] - ylv[c]);
        const float p = __fmul_rn(th, th);
        const float q = fmaf(th, th, -p) + 2.f * th * tl;
        float sh, se;
        kf_two_sum(ah[a][c], p, sh, se);
        se = __fadd_rn(se, __fadd_rn(al[a][c], q));
        ah[a][c] = __fadd_rn(sh, se);
        al[a][c] = __fsub_rn(se, __fsub_rn(ah[a][c], sh));
      }
  }
  const float c32 = (float)c_exp;
  float2* Kb = Kdf + (int64_t)lf * ldL * ldL;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = I * kK64T + ty * 4 + a, j = J * kK64T + tx * 4 + c;
      if (i >= n || j >= n) continue;
      const float k32 = __expf(ah[a][c] * c32);
      const float2 kv = k32 < 5.9604645e-8f ? make_float2(k32, 0.f) : kf_kern_from_df(ah[a][c], al[a][c], ch, cl, tab);
      Kb[(int64_t)i * ldL + j] = kv;
      if (I != J) Kb[(int64_t)j * ldL + i] = kv;
    }
}

template <typename T>
kf_status leaves_t(kf_factor* f, cudaStream_t s, bool with_k64, int part) {
  kf_tree* t = f->t;
  kf_ctx* c = f->ctx;
  const int D = t->D, s_max = f->s_max;
  const int64_t N = t->N;
  const int ldL = t->leaf_max;
  T* L = (T*)f->L;
  T* Phat = (T*)f->Phat;
  const int leaf0 = 1 << D, nleaf = 1 << D;
  dim3 g((ldL + 127) / 128, ldL, nleaf);
  if (part != 2) {
    KF_PHASE(KF_PH_LEAF_ASM, s, k_leaf_assemble<T><<<g, 128, 0, s>>>(t->X64, t->X32, t->d, f->c_exp, f->lambda, t->d_lo, t->d_hi, leaf0, ldL, L));
    if (f->Kdf && with_k64) {
      kf_status r = kf_leaf_k64_launch(f, s);
      if (r != KF_OK) return r;
    }
    if (sizeof(T) == 4 && f->Dinv) {  // mixed path on the tensor cores: 128-column panels
      const size_t psm = sizeof(float) * 2 * kPanel * (kPanel + 1);
      KF_CUDA(c, cudaFuncSetAttribute(k_chol_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
      const int npan = (ldL + kPanel - 1) / kPanel;
      for (int kb = 0; kb < ldL; kb += kPanel) {
        KF_PHASE(KF_PH_LEAF_CHOL, s, k_chol_panel<<<nleaf, 256, psm, s>>>(t->d_lo, t->d_hi, leaf0, ldL, (float*)L,
                                                                        kb, npan, f->Dinv, f->ltrack, f->status,
                                                                        f->pivr));
        KF_LAUNCH_CHECK(c);
        if (kf_tc_leaf_panel(t->d_lo, t->d_hi, leaf0, nleaf, ldL, kb, (float*)L, f->Dinv, f->status, s) != KF_OK)
          return kf_set_err(c, KF_ECUDA, "leaf panel products: %s", cudaGetErrorString(cudaGetLastError()));
      }
    } else {
      KF_PHASE(KF_PH_LEAF_CHOL, s, k_leaf_cholesky<T><<<nleaf, 256, 0, s>>>(t->d_lo, t->d_hi, leaf0, ldL, L, f->status, f->pivr));
    }
  }
  if (D > 0 && part != 1) {
    T* PhD = Phat + kf_phat_level_off(f, D);
    if (sizeof(T) == 4 && f->Dinv) {
      KF_PHASE(KF_PH_LEAF_PHAT, s, k_to_f32_rows<<<grid_for(N * s_max, 256), 256, 0, s>>>(f->Pleaf, (float*)PhD,
                                                                                        N * s_max));
      if (kf_tc_leaf_phat(t->d_lo, t->d_hi, f->rank, leaf0, nleaf, ldL, (float*)L, f->Dinv, s_max, (float*)PhD,
                          f->status, s) != KF_OK)
        return kf_set_err(c, KF_ECUDA, "leaf P^ products: %s", cudaGetErrorString(cudaGetLastError()));
    } else {
      KF_PHASE(KF_PH_LEAF_PHAT, s, k_leaf_phat<T><<<nleaf, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, leaf0, ldL, L,
                                                                        f->Pleaf, s_max, PhD));
    }
  }
  KF_LAUNCH_CHECK(c);
  return KF_OK;
}

// V blocks of the children of level l (rows of level l + 1): they need the
// skeletons of level l + 1 only, so the pipelined driver runs them ahead on
// a stream of their own.
template <typename T>
kf_status level_eval_v(kf_factor* f, int l, cudaStream_t s) {
  kf_tree* t = f->t;
  kf_ctx* c = f->ctx;
  const int s_max = f->s_max;
  const int64_t N = t->N;
  T* VT = (T*)f->VT;
  auto lvl = [&](T* base, int lv) { return base + (int64_t)(lv - 1) * N * s_max; };
  const int nn = 1 << l;
  const int child0 = 1 << (l + 1);
  // V blocks of the children's level
  const int vt_rows = 64;
  dim3 gv((unsigned)(((N >> (l + 1)) + vt_rows) / vt_rows), 2 * nn);
  // skeleton coordinates of up to qchunk columns per pass, at most 96 KiB of shared memory
  // skeleton coordinates of up to qchunk columns per pass, at most 96 KiB of shared memory
  const int qchunk = (int)std::max<int64_t>(1, std::min<int64_t>(s_max, (96 * 1024 / (int64_t)sizeof(T) - 8 * t->d) / t->d));
  const size_t vt_smem = sizeof(T) * ((size_t)t->d * qchunk + 8 * t->d);
  if (sizeof(T) == 4) {  // mixed path: register-tiled FP32 (+ double-float) evaluation
    const size_t ts = sizeof(float) * 4 * (size_t)t->d * kVT;
    KF_CUDA(c, cudaFuncSetAttribute(k_eval_vt_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ts));
    const int64_t rows = (N >> (l + 1)) + 1;
    dim3 gt((unsigned)((rows + kVT - 1) / kVT), (unsigned)((s_max + kVT - 1) / kVT), 2 * nn);
    KF_PHASE(KF_PH_EVAL_V, s, k_eval_vt_tiled<<<gt, 256, ts, s>>>(t->X32, t->X32lo, t->d, f->c_exp, t->d_lo, t->d_hi,
                                                                f->rank, f->skel, s_max, child0,
                                                                (float*)(VT + kf_vt_level_off(f, l + 1)),
                                                                f->VTdf ? f->VTdf + (int64_t)l * N * s_max : nullptr,
                                                                f->c_exp_hi, f->c_exp_lo, t->exp_tab));
    if (f->VTsl) {
      kf_status zs = kf_oz_slice_v(f, l + 1, s);
      if (zs != KF_OK) return zs;
    }
  } else {
    KF_CUDA(c, cudaFuncSetAttribute(k_eval_vt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vt_smem));
    KF_PHASE(KF_PH_EVAL_V, s, k_eval_vt<T><<<gv, 256, vt_smem, s>>>(t->X64, t->X32, t->d, f->c_exp, t->d_lo, t->d_hi,
                                                                   f->rank, f->skel, s_max, child0, vt_rows, qchunk,
                                                                   VT + kf_vt_level_off(f, l + 1)));
  }
  KF_LAUNCH_CHECK(c);
  return KF_OK;
}

// Z, its LU, T = Z^-1 P_c and the telescoped P^ of level l
template <typename T>
kf_status level_reduce(kf_factor* f, int l, double* Tm, cudaStream_t s) {
  float* Tm32 = f->prec == KF_PREC_FP64 ? nullptr : (float*)(Tm + kf_factor_tm_elems(f));
  size_t zp_cap = 0;
  void* zparts = kf_factor_zparts(f, Tm, &zp_cap);
  kf_tree* t = f->t;
  kf_ctx* c = f->ctx;
  const int s_max = f->s_max, ldz = 2 * s_max;
  const int64_t N = t->N;
  T* Phat = (T*)f->Phat;
  T* VT = (T*)f->VT;
  auto phl = [&](int lv) { return Phat + kf_phat_level_off(f, lv); };
  const int node0 = 1 << l, nn = 1 << l;
  // Z
  KF_PHASE(KF_PH_ZOFF, s, k_z_init<<<dim3(grid_for((int64_t)ldz * ldz, 256, 64), nn), 256, 0, s>>>(f->rank, node0, ldz, f->ZLU));
  const int tiles = ((s_max + 63) / 64) * ((s_max + 63) / 64);
  const int64_t rows = N >> (l + 1);
  const int ksplit = zoff64_ksplit(rows, nn, tiles);
  if (sizeof(T) == 4 && f->use_tc && f->fused_zoff) {  // kernel entries evaluated inside the product
    kf_status r = kf_tc_zoff_fused(t->d_lo, t->d_hi, f->rank, f->skel, t->X32, t->d, f->c_exp_hi, node0, nn, s_max,
                                   (const float*)phl(l + 1), ldz, f->ZLU, rows, (float*)zparts, zp_cap, f->status, s,
                                   f->tc_bn);
    if (r != KF_OK) return kf_set_err(c, r, "tensor-core Z blocks failed at level %d", l);
  } else if (sizeof(T) == 4 && f->use_tc) {
    kf_status r = kf_tc_zoff(t->d_lo, t->d_hi, f->rank, node0, nn, s_max, (const float*)(VT + kf_vt_level_off(f, l + 1)),
                             (const float*)phl(l + 1), ldz, f->ZLU, rows, (float*)zparts, zp_cap, f->status, s,
                             f->tc_bn);
    if (r != KF_OK) return kf_set_err(c, r, "tensor-core Z blocks failed at level %d", l);
  } else {
    const dim3 gz(tiles, ksplit, 2 * nn);
    if (ksplit > 1) {
      const size_t pb = sizeof(double) * (size_t)gz.x * gz.y * gz.z * 64 * 64;
      if (pb > zp_cap) return kf_set_err(c, KF_EINVAL, "Z blocks: split-K scratch too small at level %d", l);
      KF_CUDA(c, cudaMemsetAsync(zparts, 0, pb, s));
    }
    KF_PHASE(KF_PH_ZOFF, s, k_zoff<T><<<gz, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, node0, s_max,
                                                          VT + kf_vt_level_off(f, l + 1), phl(l + 1), ldz, f->ZLU,
                                                          ksplit, (double*)zparts));
    if (ksplit > 1)
      KF_PHASE(KF_PH_ZOFF, s, k_zoff_reduce64<<<dim3(tiles, 2 * nn), 256, 0, s>>>(f->rank, node0, ldz, ksplit,
                                                                                (const double*)zparts, f->ZLU));
  }
  // few nodes: a cluster of CTAs per node (one CTA per SM: the kernel takes
  // 255 registers a thread), the largest size whose nn clusters are all
  // resident at once (16-CTA clusters need 16 free SMs of one GPC, and only a
  // few GPCs offer them); a level that does not fit one wave keeps one CTA
  // per node
  int zc = 1;
  if (f->use_cluster_lu && (int64_t)nn * 2 <= 152) {
    cudaError_t ea = cudaFuncSetAttribute(k_z_factor_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int cand = 16; cand >= 2 && ea == cudaSuccess; cand >>= 1) {
      if ((int64_t)nn * cand > 152) continue;
      cudaLaunchConfig_t qc = {};
      qc.gridDim = dim3((unsigned)(nn * cand));
      qc.blockDim = dim3(256);
      cudaLaunchAttribute qa[1];
      qa[0].id = cudaLaunchAttributeClusterDimension;
      qa[0].val.clusterDim.x = (unsigned)cand;
      qa[0].val.clusterDim.y = 1;
      qa[0].val.clusterDim.z = 1;
      qc.attrs = qa;
      qc.numAttrs = 1;
      int act = 0;
      if (cudaOccupancyMaxActiveClusters(&act, k_z_factor_cluster, &qc) == cudaSuccess && act >= nn) {
        zc = cand;
        break;
      }
    }
    cudaGetLastError();
  }
  if (zc > 1) {
    KF_CUDA(c, cudaFuncSetAttribute(k_z_factor_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nn * zc));
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)zc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int solve = l >= 1 ? 1 : 0;
    cudaError_t le = cudaSuccess;
    KF_PHASE(KF_PH_ZLU, s, le = cudaLaunchKernelEx(&cfg, k_z_factor_cluster, (const int32_t*)f->rank, node0, ldz,
                                                   s_max, f->ZLU, f->Zpiv, (const double*)f->Pc, Tm, Tm32, solve,
                                                   f->status, f->pivr));
    if (le != cudaSuccess)
      return kf_set_err(c, KF_ECUDA, "reduced-system LU (cluster of %d) at level %d: %s", zc, l, cudaGetErrorString(le));
  } else {
    KF_PHASE(KF_PH_ZLU, s, k_z_factor<<<nn, 256, 0, s>>>(f->rank, node0, ldz, s_max, f->ZLU, f->Zpiv, f->Pc, Tm, Tm32,
                                                         l >= 1 ? 1 : 0, f->status, f->pivr));
  }
  if (l >= 1 && f->Tw) {  // memory-lean W: keep T = Z^-1 P_c of the level's nodes for the solve
    const size_t tb = sizeof(T) * (size_t)nn * ldz * s_max;
    const void* src = sizeof(T) == 4 ? (const void*)Tm32 : (const void*)Tm;
    KF_CUDA(c, cudaMemcpyAsync((char*)f->Tw + sizeof(T) * (size_t)node0 * ldz * s_max, src, tb,
                               cudaMemcpyDeviceToDevice, s));
  }
  if (l >= 1) {
    const int64_t cmax_rows = (N >> (l + 1)) + 1;
    dim3 gt((unsigned)((cmax_rows + 63) / 64), (s_max + 63) / 64, 2 * nn);
    if (sizeof(T) == 4 && f->use_tc) {
      kf_status r = kf_tc_telescope(t->d_lo, t->d_hi, f->rank, node0, nn, s_max, (const float*)phl(l + 1), Tm32,
                                    ldz, (float*)phl(l), cmax_rows, f->status, s, f->tc_bn);
      if (r != KF_OK) return kf_set_err(c, r, "tensor-core telescoping failed at level %d", l);
    } else {
      KF_PHASE(KF_PH_TELESCOPE, s, k_telescope<T><<<gt, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, node0, s_max, phl(l + 1), Tm, ldz,
                                        phl(l)));
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return kf_set_err(c, KF_ECUDA, "factorize level %d: %s", l, cudaGetErrorString(e));
  return KF_OK;
}

}  // namespace

// T = Z^-1 P_c of one level (FP64) and, on the mixed path, its FP32 copy right after it
// the Z-block products' split-K partials of the largest level
static size_t zoff_parts_bytes(const kf_factor* f) {
  size_t need = 0;
  const int s_max = f->s_max, tiles = ((s_max + 63) / 64) * ((s_max + 63) / 64);
  for (int l = 0; l < f->t->D; ++l) {
    const int nn = 1 << l;
    const int64_t rows = f->t->N >> (l + 1);
    size_t b;
    if (f->prec != KF_PREC_FP64 && f->use_tc) {
      b = kf_tc_zoff_parts_bytes(s_max, f->tc_bn, nn, rows);
    } else {
      const int ks = zoff64_ksplit(rows, nn, tiles);
      b = ks > 1 ? sizeof(double) * (size_t)tiles * 2 * nn * ks * 64 * 64 : 0;
    }
    need = std::max(need, b);
  }
  return need;
}

static size_t tm_core_bytes(const kf_factor* f) {
  const size_t b = (sizeof(double) + (f->prec == KF_PREC_FP64 ? 0 : sizeof(float))) * kf_factor_tm_elems(f);
  return (b + 255) / 256 * 256;
}

size_t kf_factor_tm_bytes(const kf_factor* f) { return tm_core_bytes(f) + zoff_parts_bytes(f); }

void* kf_factor_zparts(const kf_factor* f, double* Tm, size_t* cap) {
  *cap = zoff_parts_bytes(f);
  return *cap ? (void*)((char*)Tm + tm_core_bytes(f)) : nullptr;
}

size_t kf_factor_tm_elems(const kf_factor* f) {
  const int D = f->t->D;
  return D > 0 ? (size_t)(1 << (D - 1)) * 2 * f->s_max * f->s_max : 1;
}

kf_status kf_leaf_k64_launch(kf_factor* f, cudaStream_t s) {
  kf_tree* t = f->t;
  const int nt = (t->leaf_max + kK64T - 1) / kK64T;
  const size_t smem = sizeof(float) * 4 * (size_t)t->d * kK64T;
  KF_CUDA(f->ctx, cudaFuncSetAttribute(k_leaf_k64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 g((unsigned)(nt * (nt + 1) / 2), 1u << t->D);
  KF_PHASE(KF_PH_LEAF_ASM, s, k_leaf_k64<<<g, 256, smem, s>>>(t->X32lo, t->X32, t->d, f->c_exp, t->d_lo, t->d_hi,
                                                              1 << t->D, t->leaf_max, f->Kdf, f->c_exp_hi,
                                                              f->c_exp_lo, t->exp_tab));
  KF_LAUNCH_CHECK(f->ctx);
  return kf_oz_slice_leaf(f, s);  // their BF16 digits, when the factors keep them (tc_operator)
}

__global__ void k_split_df_array(const double* __restrict__ a, float2* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = kf_split_df(a[i]);
}

kf_status kf_split_p_df(kf_factor* f, cudaStream_t s) {
  if (!f->Pleafdf || !f->Pcdf) return KF_OK;
  const int64_t nl = f->t->N * (int64_t)f->s_max, nc = ((int64_t)1 << f->t->D) * 2 * f->s_max * f->s_max;
  KF_PHASE(KF_PH_MISC, s, k_split_df_array<<<grid_for(nl, 256), 256, 0, s>>>(f->Pleaf, f->Pleafdf, nl));
  KF_PHASE(KF_PH_MISC, s, k_split_df_array<<<grid_for(nc, 256), 256, 0, s>>>(f->Pc, f->Pcdf, nc));
  KF_LAUNCH_CHECK(f->ctx);
  return KF_OK;
}

kf_status kf_split_z_df(kf_factor* f, cudaStream_t s) {
  if (!f->ZLUdf) return KF_OK;
  const int64_t ldz2 = 4 * (int64_t)f->s_max * f->s_max;
  const int64_t first = ((int64_t)2 << f->zinv_top) * ldz2, last = ((int64_t)1 << f->t->D) * ldz2;
  if (last > first)
    KF_PHASE(KF_PH_MISC, s, k_split_df_array<<<grid_for(last - first, 256), 256, 0, s>>>(f->ZLU + first,
                                                                                      f->ZLUdf + first, last - first));
  KF_LAUNCH_CHECK(f->ctx);
  return KF_OK;
}

kf_status kf_factorize_leaves(kf_factor* f, cudaStream_t s, bool with_k64, int part) {
  return f->prec == KF_PREC_FP64 ? leaves_t<double>(f, s, with_k64, part) : leaves_t<float>(f, s, with_k64, part);
}

kf_status kf_factorize_level_v(kf_factor* f, int l, cudaStream_t s) {
  return f->prec == KF_PREC_FP64 ? level_eval_v<double>(f, l, s) : level_eval_v<float>(f, l, s);
}

kf_status kf_factorize_level_z(kf_factor* f, int l, double* Tm, cudaStream_t s) {
  return f->prec == KF_PREC_FP64 ? level_reduce<double>(f, l, Tm, s) : level_reduce<float>(f, l, Tm, s);
}

kf_status kf_factorize_level(kf_factor* f, int l, double* Tm, cudaStream_t s) {
  kf_status st = kf_factorize_level_v(f, l, s);
  return st == KF_OK ? kf_factorize_level_z(f, l, Tm, s) : st;
}

kf_status kf_z_inverse_level(kf_factor* f, int l, cudaStream_t s) {
  if (l > f->zinv_top) return KF_OK;
  const int ldz = 2 * f->s_max, qw = 16;
  dim3 g(1u << l, (unsigned)((ldz + qw - 1) / qw));
  KF_PHASE(KF_PH_ZINV, s, k_z_inverse<<<g, 256, 0, s>>>(f->rank, 1 << l, ldz, f->ZLU, f->Zpiv, f->Zinv, qw));
  KF_LAUNCH_CHECK(f->ctx);
  return KF_OK;
}

kf_status kf_factorize_device(kf_factor* f, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  kf_status st = kf_factorize_leaves(f, s, true, 0);
  if (st != KF_OK || f->t->D == 0) return st;
  const size_t tb = kf_factor_tm_bytes(f);
  double* Tm = (double*)c->dalloc(tb, s);
  if (!Tm) return kf_set_err(c, KF_ENOMEM, "factorize: allocation failed");
  for (int l = f->t->D - 1; l >= 0 && st == KF_OK; --l) {
    st = kf_factorize_level(f, l, Tm, s);
    if (st == KF_OK) st = kf_z_inverse_level(f, l, s);
  }
  c->dfree(Tm, tb, s);
  if (st == KF_OK) st = kf_split_p_df(f, s);
  if (st == KF_OK) st = kf_split_z_df(f, s);
  if (st == KF_OK) st = kf_oz_slice_rows(f, s);  // digits of P^ and P (tc_operator)
  return st;
}

// Skeletonization and factorization interleaved on five streams: level l of
// the factorization needs the skeletons of levels l + 1 and l only, so the
// pivoted QRs of the upper levels run while the lower levels are factorized
// (s1: skeletons; s4: the leaf blocks and their Cholesky factors, which need
// no skeleton and start at once; s2: P^ of the leaves and the reduced
// systems; s3: V blocks, then the FP64 operator's leaf blocks; s5: Z^-1 of the
// upper levels, each after its level's LU).  Events order
// the streams; the caller's stream waits for them at the end.
kf_status kf_skel_factorize_pipelined(kf_factor* f, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  const int D = f->t->D;
  if (D == 0) {
    kf_status st = kf_skeletonize_device(f, s);
    return st == KF_OK ? kf_factorize_device(f, s) : st;
  }
  kf_skel_scratch sc;
  kf_status st = kf_skel_begin(f, &sc, s);
  const size_t tb = kf_factor_tm_bytes(f);
  double* Tm = st == KF_OK ? (double*)c->dalloc(tb, s) : nullptr;
  if (st == KF_OK && !Tm) st = kf_set_err(c, KF_ENOMEM, "factorize: allocation failed");
  cudaStream_t s1 = nullptr, s2 = nullptr, s3 = nullptr, s4 = nullptr, s5 = nullptr;
  cudaEvent_t evl = nullptr, evi = nullptr;
  std::vector<cudaEvent_t> ev(D + 4, nullptr), evv(D, nullptr), evz(D, nullptr), evr(D, nullptr);
  if (st == KF_OK) {
    // priorities (measured): the skeleton chain (s1) and the leaf blocks with
    // their Cholesky factors (s4, at the start beside the leaf sample blocks)
    // highest; the reduced systems (s2) one level below, so that a level's
    // sample blocks and QR are dispatched ahead of them; the V blocks (s3)
    // lowest (1.10 s with s3 high, 1.07 s with s2 equal to s1, 1.06 s so)
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    KF_CUDA(c, cudaStreamCreateWithPriority(&s1, cudaStreamNonBlocking, hi_prio));
    KF_CUDA(c, cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, std::min(hi_prio + 1, lo_prio)));
    KF_CUDA(c, cudaStreamCreateWithPriority(&s3, cudaStreamNonBlocking, lo_prio));
    KF_CUDA(c, cudaStreamCreateWithPriority(&s4, cudaStreamNonBlocking, hi_prio));
    // s5: Z^-1 of the upper levels, after each level's LU, beside the chain
    KF_CUDA(c, cudaStreamCreateWithPriority(&s5, cudaStreamNonBlocking, lo_prio));
    KF_CUDA(c, cudaEventCreateWithFlags(&evl, cudaEventDisableTiming));
    KF_CUDA(c, cudaEventCreateWithFlags(&evi, cudaEventDisableTiming));
    for (auto& e : ev) KF_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto& e : evv) KF_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto& e : evz) KF_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto& e : evr) KF_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    // ev[l]: skeletons of level l done (on s1); ev[0]: allocations ready (on s);
    // ev[D+1]: factorization done (on s2); ev[D+2]: skeletons done (on s1);
    // ev[D+3]: V blocks done (on s3); evv[l]: V blocks of level l done (on s3)
    cudaEventRecord(ev[0], s);
    cudaStreamWaitEvent(s1, ev[0], 0);
    cudaStreamWaitEvent(s2, ev[0], 0);
    cudaStreamWaitEvent(s3, ev[0], 0);
    cudaStreamWaitEvent(s4, ev[0], 0);
    // the leaf blocks and their Cholesky factors need the tree only (FP32 or
    // FP64 work that shares the SMs with the FP64 sample blocks of the leaf level)
    if (st == KF_OK) st = kf_factorize_leaves(f, s4, false, 1);
    cudaEventRecord(evl, s4);
    cudaStreamWaitEvent(s2, evl, 0);
    // the hybrid solver (frontier level Lh >= 1) skeletonizes and factorizes
    // the levels from the leaves up to its frontier only
    const int Lh = f->hyb_L;
    for (int l = D; l >= std::max(1, Lh) && st == KF_OK; --l) {
      st = kf_skel_level(f, l, &sc, s1);
      cudaEventRecord(ev[l], s1);
      if (st != KF_OK) break;
      // V blocks of level l - 1 (rows of level l) need the skeletons of level l;
      // with three V slots (V recomputed in the sweeps) they overwrite the V
      // blocks of level l + 3, which the reduced systems of level l + 2 read
      cudaStreamWaitEvent(s3, ev[l], 0);
      if (f->vstore == KF_V_RECOMPUTE && l + 2 <= D - 1) cudaStreamWaitEvent(s3, evr[l + 2], 0);
      if (l - 1 >= Lh) st = kf_factorize_level_v(f, l - 1, s3);
      cudaEventRecord(evv[l - 1], s3);
      if (st != KF_OK) break;
      cudaStreamWaitEvent(s2, ev[l], 0);
      if (l == D) {
        st = kf_factorize_leaves(f, s2, false, 2);
      } else {
        // the stored V blocks feed the Z blocks unless the product evaluates them itself
        if (!kf_zoff_fused(f)) cudaStreamWaitEvent(s2, evv[l], 0);
        st = kf_factorize_level_z(f, l, Tm, s2);
        cudaEventRecord(evr[l], s2);
        if (st == KF_OK && l <= f->zinv_top) {
          cudaEventRecord(evz[l], s2);
          cudaStreamWaitEvent(s5, evz[l], 0);
          st = kf_z_inverse_level(f, l, s5);
        }
      }
    }
    if (st == KF_OK && Lh == 0) {
      if (!kf_zoff_fused(f)) cudaStreamWaitEvent(s2, evv[0], 0);
      st = kf_factorize_level_z(f, 0, Tm, s2);
      if (st == KF_OK) {
        cudaEventRecord(evz[0], s2);
        cudaStreamWaitEvent(s5, evz[0], 0);
        st = kf_z_inverse_level(f, 0, s5);
      }
    }
    // hybrid: the reduced system I + VW of the frontier (needs the frontier
    // skeletons and P^ of level Lh, both ordered before this point on s2)
    if (st == KF_OK && Lh > 0) st = kf_hybrid_reduced_system(f, s2);
    if (st == KF_OK) st = kf_split_z_df(f, s2);
    // the FP64 operator's leaf blocks need the tree only, and only the solve
    // reads them: last on the V-block stream, where they fill the SMs that the
    // latency-bound upper levels leave idle (ahead of the V blocks they held
    // back the first level's V blocks and with them the reduced systems)
    if (st == KF_OK && f->Kdf) st = kf_leaf_k64_launch(f, s3);
    // the operator's pairs of Pleaf and P_c, once every skeleton is known
    if (st == KF_OK) st = kf_split_p_df(f, s1);
    cudaEventRecord(ev[D + 1], s2);
    cudaEventRecord(ev[D + 2], s1);
    cudaEventRecord(ev[D + 3], s3);
    cudaStreamWaitEvent(s, ev[D + 1], 0);
    cudaStreamWaitEvent(s, ev[D + 2], 0);
    cudaStreamWaitEvent(s, ev[D + 3], 0);
    cudaEventRecord(evi, s5);
    cudaStreamWaitEvent(s, evi, 0);
  }
  if (Tm) c->dfree(Tm, tb, s);
  kf_skel_end(f, &sc, s);
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : evv)
    if (e) cudaEventDestroy(e);
  for (auto& e : evz)
    if (e) cudaEventDestroy(e);
  for (auto& e : evr)
    if (e) cudaEventDestroy(e);
  if (s5) cudaStreamDestroy(s5);
  if (evi) cudaEventDestroy(evi);
  if (s1) cudaStreamDestroy(s1);
  if (s2) cudaStreamDestroy(s2);
  if (s3) cudaStreamDestroy(s3);
  if (s4) cudaStreamDestroy(s4);
  if (evl) cudaEventDestroy(evl);
  if (st == KF_OK) st = kf_oz_slice_rows(f, s);  // digits of P^ and P (tc_operator), after every level
  return st;
}

// LU of one reduced system stored as node 1 of a two-node array (row stride
// ldz <= 2 KF_MAX_SMAX): the hybrid solver's I + VW, whose rank array gives
// node 1 a first child of rank S and a second of rank 0.
kf_status kf_z_factor_one_launch(const int32_t* rank, int ldz, double* Z, int32_t* piv, int32_t* status,
                                 double* pivr, cudaStream_t s) {
  if (ldz < 1 || ldz > 2 * KF_MAX_SMAX) return KF_EINVAL;
  KF_PHASE(KF_PH_HYBRID, s, k_z_factor<<<1, 256, 0, s>>>(rank, 1, ldz, 1, Z, piv, nullptr, nullptr, nullptr, 0, status,
                                                         pivr));
  return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ECUDA;
}
