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
#include <algorithm>
#include <vector>

#include "kf_internal.cuh"
#include "prof.cuh"

kf_status kf_tc_zoff(const int32_t* lo, const int32_t* hi, const int32_t* rank, int node0, int nn, int s_max,
                     const float* VT, const float* Ph, int ldz, double* Z, int64_t rows_per_child, int32_t* status,
                     cudaStream_t s);
kf_status kf_tc_telescope(const int32_t* lo, const int32_t* hi, const int32_t* rank, int node0, int nn, int s_max,
                          const float* Pc_hat, const double* Tm, int ldz, float* Pa_hat, int64_t rows_per_child,
                          int32_t* status, cudaStream_t s);

namespace {

template <typename T> struct Acc;
template <> struct Acc<double> { using type = double; };
template <> struct Acc<float> { using type = float; };

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
  const int tid = threadIdx.x;
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = fmax(mx, fabs((double)L[(int64_t)i * ldL + i]));
    amax_sh = mx;
  }
  __syncthreads();
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
          x[j] = acc / dg[j][j];
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
        for (int e = tid; e < TS * NB; e += blockDim.x) {
          int r = e / NB, cc = e % NB;
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
__global__ void __launch_bounds__(256) k_leaf_phat(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                   const int32_t* __restrict__ rank, int leaf0, int ldL,
                                                   const T* __restrict__ Lall, const double* __restrict__ Pleaf,
                                                   int s_max, T* __restrict__ Phat) {
  constexpr int NB = 32, TS = 64;
  __shared__ T sa[TS][NB + 1];
  __shared__ T sb[NB][TS + 1];
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
          x[i] = acc / sa[i][i];
        }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < nb) Y[(int64_t)(kb + i) * s_max + q] = x[i];
    }
    __syncthreads();
    for (int ti = kb + nb; ti < n; ti += TS)
      for (int tj = 0; tj < s; tj += TS) {
        for (int e = tid; e < TS * NB; e += blockDim.x) {
          int r = e / NB, cc = e % NB;
          sa[r][cc] = (ti + r < n && cc < nb) ? L[(int64_t)(ti + r) * ldL + kb + cc] : (T)0;
          int rr = e / TS, c2 = e % TS;
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
          x[i] = acc / sa[i][i];
        }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < nb) Y[(int64_t)(kb + i) * s_max + q] = x[i];
    }
    __syncthreads();
    // rows above: y[0:kb] -= L[kb:kb+nb, 0:kb]^T x_block
    for (int ti = 0; ti < kb; ti += TS)
      for (int tj = 0; tj < s; tj += TS) {
        for (int e = tid; e < TS * NB; e += blockDim.x) {
          int r = e % TS, cc = e / TS;   // coalesced over r (contiguous in a row of L)
          sa[r][cc] = (ti + r < kb && cc < nb) ? L[(int64_t)(kb + cc) * ldL + ti + r] : (T)0;
          int rr = e / TS, c2 = e % TS;
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
// level.  The sibling's skeleton coordinates are staged transposed in shared
// memory (yT[k][q]); one warp per row, lanes over q, coalesced stores.
template <typename T>
__global__ void __launch_bounds__(256) k_eval_vt(const double* __restrict__ X64, const float* __restrict__ X32,
                                                 const float* __restrict__ X32lo, int d,
                                                 double c_exp, const int32_t* __restrict__ lo,
                                                 const int32_t* __restrict__ hi, const int32_t* __restrict__ rank,
                                                 const int32_t* __restrict__ skel, int s_max, int node0, int rows_per_cta,
                                                 int qchunk, T* __restrict__ VT, double* __restrict__ VT64) {
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
        T kv = sizeof(T) == 8 ? (T)exp((double)(acc * c)) : (T)__expf((float)(acc * c));
        if (VT64 != nullptr) {  // FP64 operator copy: recompute the entries that matter in FP64
          const int64_t row = b + i;
          double k64 = (double)kv;
          if ((float)kv >= 5.9604645e-8f) {
            const int64_t col = sk[q0 + q];
            k64 = exp(kf_sqdist_df(X32 + row * d, X32lo + row * d, X32 + col * d, X32lo + col * d, d) * c_exp);
          }
          VT64[row * s_max + q0 + q] = k64;
          kv = (T)k64;
        }
        out[q] = kv;
      }
      __syncwarp();
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
                                              double* __restrict__ Z, int ksplit) {
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
  double* Zb = Z + (int64_t)node * ldz * ldz;
  const int roff = side == 0 ? 0 : sl, coff = side == 0 ? sl : 0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = tm * TS + ty * 4 + a, j = tn * TS + tx * 4 + b;
      if (i < M && j < Nn) atomicAdd(&Zb[(int64_t)(roff + i) * ldz + coff + j], (double)acc[a][b]);
    }
}

// Blocked LU with partial pivoting of Z (FP64) followed, for non-root nodes,
// by T = Z^-1 P_c, one CTA (256 threads) per node.
//   panel:    32 columns at a time; per column an arg-max over the rows
//             (ties: lowest row), a full-row swap, scaling, and the rank-1
//             update restricted to the panel;
//   U12:      L11^-1 A12 by the 32 x 32 unit-lower block;
//   trailing: A22 -= L21 U12, 64 x 64 register-tiled FP64 tiles;
// then X = P_c with the row swaps applied, L y = x and U t = y by 32-row
// blocks (diagonal block per column thread, off-block updates tiled).
__global__ void __launch_bounds__(256) k_z_factor(const int32_t* __restrict__ rank, int node0, int ldz, int s_max,
                                                  double* __restrict__ Z, int32_t* __restrict__ piv,
                                                  const double* __restrict__ Pc, double* __restrict__ T,
                                                  int solve_pc, int32_t* __restrict__ status, double* __restrict__ pivr) {
  constexpr int NB = 32, TS = 64;
  __shared__ double sa[TS][NB + 1];
  __shared__ double sb[NB][TS + 1];
  __shared__ double rv[8];
  __shared__ int ri[8];
  __shared__ int pk;
  __shared__ double amax_sh;
  const int nl = blockIdx.x, node = node0 + nl;
  const int z = rank[2 * node] + rank[2 * node + 1];
  double* A = Z + (int64_t)node * ldz * ldz;
  int32_t* pv = piv + (int64_t)node * ldz;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // max |Z| for the pivot test
  double mx = 0.0;
  for (int64_t e = tid; e < (int64_t)z * z; e += blockDim.x) mx = fmax(mx, fabs(A[(e / z) * ldz + e % z]));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if (lane == 0) rv[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    double m2 = 0.0;
    for (int w = 0; w < 8; ++w) m2 = fmax(m2, rv[w]);
    amax_sh = m2;
  }
  __syncthreads();
  const double amax = amax_sh;
  bool bad = false;
  double umin = INFINITY, umax = 0.0;
  for (int kb = 0; kb < z; kb += NB) {
    const int nb = min(NB, z - kb);
    for (int j = kb; j < kb + nb; ++j) {
      double bv = -1.0;
      int bi = z;
      for (int i = j + tid; i < z; i += blockDim.x) {
        double v = fabs(A[(int64_t)i * ldz + j]);
        if (v > bv) { bv = v; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, off);
        int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (lane == 0) { rv[warp] = bv; ri[warp] = bi; }
      __syncthreads();
      if (tid == 0) {
        double b2 = -1.0;
        int i2 = z;
        for (int w = 0; w < 8; ++w)
          if (rv[w] > b2 || (rv[w] == b2 && ri[w] < i2)) { b2 = rv[w]; i2 = ri[w]; }
        pk = i2;
        pv[j] = i2;
      }
      __syncthreads();
      const int p = pk;
      if (p != j)
        for (int c = tid; c < z; c += blockDim.x) {
          double t = A[(int64_t)j * ldz + c];
          A[(int64_t)j * ldz + c] = A[(int64_t)p * ldz + c];
          A[(int64_t)p * ldz + c] = t;
        }
      __syncthreads();
      const double ujj = A[(int64_t)j * ldz + j];
      umin = fmin(umin, fabs(ujj));
      umax = fmax(umax, fabs(ujj));
      if (!(fabs(ujj) > 1e-14 * amax)) bad = true;
      const double inv = ujj != 0.0 ? 1.0 / ujj : 0.0;
      for (int i = j + 1 + tid; i < z; i += blockDim.x) {
        double* Ai = A + (int64_t)i * ldz;
        const double l = Ai[j] * inv;
        Ai[j] = l;
        for (int c = j + 1; c < kb + nb; ++c) Ai[c] = fma(-l, A[(int64_t)j * ldz + c], Ai[c]);
      }
      __syncthreads();
    }
    const int c0 = kb + nb;
    if (c0 >= z) break;
    // U12 = L11^-1 A12, thread per column
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      sa[i][j] = (i < nb && j < i) ? A[(int64_t)(kb + i) * ldz + kb + j] : 0.0;
    }
    __syncthreads();
    for (int c = c0 + tid; c < z; c += blockDim.x) {
      double x[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) x[r] = r < nb ? A[(int64_t)(kb + r) * ldz + c] : 0.0;
#pragma unroll
      for (int r = 1; r < NB; ++r) {
        double acc = x[r];
#pragma unroll
        for (int t = 0; t < r; ++t) acc = fma(-sa[r][t], x[t], acc);
        x[r] = acc;
      }
#pragma unroll
      for (int r = 1; r < NB; ++r)
        if (r < nb) A[(int64_t)(kb + r) * ldz + c] = x[r];
    }
    __syncthreads();
    // A22 -= L21 U12
    const int ty = tid / 16, tx = tid % 16;
    for (int ti = c0; ti < z; ti += TS)
      for (int tj = c0; tj < z; tj += TS) {
        for (int e = tid; e < TS * NB; e += blockDim.x) {
          int r = e / NB, cc = e % NB;
          sa[r][cc] = (ti + r < z && cc < nb) ? A[(int64_t)(ti + r) * ldz + kb + cc] : 0.0;
          int rr = e / TS, c2 = e % TS;
          sb[rr][c2] = (rr < nb && tj + c2 < z) ? A[(int64_t)(kb + rr) * ldz + tj + c2] : 0.0;
        }
        __syncthreads();
        double acc[4][4] = {};
#pragma unroll 8
        for (int t = 0; t < NB; ++t) {
          double av[4], bv[4];
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
            if (i < z && j < z) A[(int64_t)i * ldz + j] -= acc[a][b];
          }
        __syncthreads();
      }
  }
  if (bad && tid == 0) atomicOr(status, KF_DEV_ILLCOND);
  if (tid == 0) pivr[node] = (z == 0 || umax == 0.0) ? 1.0 : umin / umax;
  if (!solve_pc) return;
  // ---- T = Z^-1 P_c --------------------------------------------------------------
  const int s = rank[node];
  const double* B = Pc + (int64_t)node * ldz * s_max;
  double* X = T + (int64_t)nl * ldz * s_max;
  for (int64_t e = tid; e < (int64_t)ldz * s_max; e += blockDim.x) {
    int i = (int)(e / s_max), q = (int)(e % s_max);
    X[e] = (i < z && q < s) ? B[e] : 0.0;
  }
  __syncthreads();
  if (s == 0 || z == 0) return;
  for (int k = 0; k < z; ++k) {  // row swaps in factorization order
    const int p = pv[k];
    if (p != k)
      for (int q = tid; q < s; q += blockDim.x) {
        double t = X[(int64_t)k * s_max + q];
        X[(int64_t)k * s_max + q] = X[(int64_t)p * s_max + q];
        X[(int64_t)p * s_max + q] = t;
      }
    __syncthreads();
  }
  const int ty = tid / 16, tx = tid % 16;
  // forward: L (unit lower)
  for (int kb = 0; kb < z; kb += NB) {
    const int nb = min(NB, z - kb);
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      sa[i][j] = (i < nb && j < i) ? A[(int64_t)(kb + i) * ldz + kb + j] : 0.0;
    }
    __syncthreads();
    for (int q = tid; q < s; q += blockDim.x) {
      double x[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) x[r] = r < nb ? X[(int64_t)(kb + r) * s_max + q] : 0.0;
#pragma unroll
      for (int r = 1; r < NB; ++r) {
        double acc = x[r];
#pragma unroll
        for (int t = 0; t < r; ++t) acc = fma(-sa[r][t], x[t], acc);
        x[r] = acc;
      }
#pragma unroll
      for (int r = 1; r < NB; ++r)
        if (r < nb) X[(int64_t)(kb + r) * s_max + q] = x[r];
    }
    __syncthreads();
    for (int ti = kb + nb; ti < z; ti += TS)
      for (int tj = 0; tj < s; tj += TS) {
        for (int e = tid; e < TS * NB; e += blockDim.x) {
          int r = e / NB, cc = e % NB;
          sa[r][cc] = (ti + r < z && cc < nb) ? A[(int64_t)(ti + r) * ldz + kb + cc] : 0.0;
          int rr = e / TS, c2 = e % TS;
          sb[rr][c2] = (rr < nb && tj + c2 < s) ? X[(int64_t)(kb + rr) * s_max + tj + c2] : 0.0;
        }
        __syncthreads();
        double acc[4][4] = {};
#pragma unroll 8
        for (int t = 0; t < NB; ++t) {
          double av[4], bv[4];
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
            if (i < z && j < s) X[(int64_t)i * s_max + j] -= acc[a][b];
          }
        __syncthreads();
      }
    // the diagonal-block loads of the next panel reuse sa: wait for this one
    __syncthreads();
  }
  // backward: U
  for (int kb = ((z - 1) / NB) * NB; kb >= 0; kb -= NB) {
    const int nb = min(NB, z - kb);
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      sa[i][j] = (i < nb && j < nb && j >= i) ? A[(int64_t)(kb + i) * ldz + kb + j] : 0.0;
    }
    __syncthreads();
    for (int q = tid; q < s; q += blockDim.x) {
      double x[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) x[r] = r < nb ? X[(int64_t)(kb + r) * s_max + q] : 0.0;
#pragma unroll
      for (int r = NB - 1; r >= 0; --r) {
        if (r < nb) {
          double acc = x[r];
#pragma unroll
          for (int t = r + 1; t < NB; ++t) acc = fma(-sa[r][t], x[t], acc);
          x[r] = acc / sa[r][r];
        }
      }
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < nb) X[(int64_t)(kb + r) * s_max + q] = x[r];
    }
    __syncthreads();
    // rows above: X[0:kb] -= U[0:kb, kb:kb+nb] X[kb:kb+nb]
    for (int ti = 0; ti < kb; ti += TS)
      for (int tj = 0; tj < s; tj += TS) {
        for (int e = tid; e < TS * NB; e += blockDim.x) {
          int r = e / NB, cc = e % NB;
          sa[r][cc] = (ti + r < kb && cc < nb) ? A[(int64_t)(ti + r) * ldz + kb + cc] : 0.0;
          int rr = e / TS, c2 = e % TS;
          sb[rr][c2] = (rr < nb && tj + c2 < s) ? X[(int64_t)(kb + rr) * s_max + tj + c2] : 0.0;
        }
        __syncthreads();
        double acc[4][4] = {};
#pragma unroll 8
        for (int t = 0; t < NB; ++t) {
          double av[4], bv[4];
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
            if (i < kb && j < s) X[(int64_t)i * s_max + j] -= acc[a][b];
          }
        __syncthreads();
      }
    __syncthreads();
  }
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

// FP64 copy of the leaf kernel blocks (no lambda), both triangles, for the
// FP64-accurate operator.
__global__ void k_leaf_k64(const float* __restrict__ X32lo, const float* __restrict__ X32, int d, double c_exp,
                           const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, int leaf0, int ldL,
                           double* __restrict__ K64) {
  const int lf = blockIdx.z, node = leaf0 + lf;
  const int b = lo[node], n = hi[node] - b;
  const int i = blockIdx.y;
  if (i >= n) return;
  double* Ki = K64 + ((int64_t)lf * ldL + i) * ldL;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    Ki[j] = kf_kern_hybrid(X32, X32lo, b + i, b + j, d, c_exp);
}

template <typename T>
kf_status leaves_t(kf_factor* f, cudaStream_t s) {
  kf_tree* t = f->t;
  kf_ctx* c = f->ctx;
  const int D = t->D, s_max = f->s_max;
  const int64_t N = t->N;
  const int ldL = t->leaf_max;
  T* L = (T*)f->L;
  T* Phat = (T*)f->Phat;
  const int leaf0 = 1 << D, nleaf = 1 << D;
  dim3 g((ldL + 127) / 128, ldL, nleaf);
  KF_PHASE(KF_PH_LEAF_ASM, s, k_leaf_assemble<T><<<g, 128, 0, s>>>(t->X64, t->X32, t->d, f->c_exp, f->lambda, t->d_lo, t->d_hi, leaf0, ldL, L));
  if (f->K64)
    KF_PHASE(KF_PH_LEAF_ASM, s, k_leaf_k64<<<g, 128, 0, s>>>(t->X32lo, t->X32, t->d, f->c_exp, t->d_lo, t->d_hi, leaf0, ldL, f->K64));
  KF_PHASE(KF_PH_LEAF_CHOL, s, k_leaf_cholesky<T><<<nleaf, 256, 0, s>>>(t->d_lo, t->d_hi, leaf0, ldL, L, f->status, f->pivr));
  if (D > 0)
    KF_PHASE(KF_PH_LEAF_PHAT, s, k_leaf_phat<T><<<nleaf, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, leaf0, ldL, L, f->Pleaf, s_max,
                                                                  Phat + (int64_t)(D - 1) * N * s_max));
  KF_LAUNCH_CHECK(c);
  return KF_OK;
}

template <typename T>
kf_status level_t(kf_factor* f, int l, double* Tm, cudaStream_t s) {
  kf_tree* t = f->t;
  kf_ctx* c = f->ctx;
  const int s_max = f->s_max, ldz = 2 * s_max;
  const int64_t N = t->N;
  T* Phat = (T*)f->Phat;
  T* VT = (T*)f->VT;
  auto lvl = [&](T* base, int lv) { return base + (int64_t)(lv - 1) * N * s_max; };
  const int node0 = 1 << l, nn = 1 << l;
  const int child0 = 1 << (l + 1);
  // V blocks of the children's level
  const int vt_rows = 64;
  dim3 gv((unsigned)(((N >> (l + 1)) + vt_rows) / vt_rows), 2 * nn);
  // skeleton coordinates of up to qchunk columns per pass, at most 96 KiB of shared memory
  const int qchunk = (int)std::max<int64_t>(1, std::min<int64_t>(s_max, (96 * 1024 / (int64_t)sizeof(T) - 8 * t->d) / t->d));
  const size_t vt_smem = sizeof(T) * ((size_t)t->d * qchunk + 8 * t->d);
  KF_CUDA(c, cudaFuncSetAttribute(k_eval_vt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vt_smem));
  KF_PHASE(KF_PH_EVAL_V, s, k_eval_vt<T><<<gv, 256, vt_smem, s>>>(t->X64, t->X32, t->X32lo, t->d, f->c_exp, t->d_lo, t->d_hi,
                                                                 f->rank, f->skel, s_max, child0, vt_rows, qchunk,
                                                                 lvl(VT, l + 1),
                                                                 f->VT64 ? f->VT64 + (int64_t)l * N * s_max : nullptr));
  // Z
  KF_PHASE(KF_PH_ZOFF, s, k_z_init<<<dim3(grid_for((int64_t)ldz * ldz, 256, 64), nn), 256, 0, s>>>(f->rank, node0, ldz, f->ZLU));
  const int tiles = ((s_max + 63) / 64) * ((s_max + 63) / 64);
  const int64_t rows = N >> (l + 1);
  int ksplit = (int)std::max<int64_t>(1, std::min<int64_t>(rows / 512, (152 * 8) / std::max(1, 2 * nn * tiles) + 1));
  if (sizeof(T) == 4 && f->use_tc) {
    kf_status r = kf_tc_zoff(t->d_lo, t->d_hi, f->rank, node0, nn, s_max, (const float*)lvl(VT, l + 1),
                             (const float*)lvl(Phat, l + 1), ldz, f->ZLU, rows, f->status, s);
    if (r != KF_OK) return kf_set_err(c, r, "tensor-core Z blocks failed at level %d", l);
  } else {
    KF_PHASE(KF_PH_ZOFF, s, k_zoff<T><<<dim3(tiles, ksplit, 2 * nn), 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, node0, s_max, lvl(VT, l + 1),
                                                          lvl(Phat, l + 1), ldz, f->ZLU, ksplit));
  }
  KF_PHASE(KF_PH_ZLU, s, k_z_factor<<<nn, 256, 0, s>>>(f->rank, node0, ldz, s_max, f->ZLU, f->Zpiv, f->Pc, Tm,
                                                       l >= 1 ? 1 : 0, f->status, f->pivr));
  if (l >= 1) {
    const int64_t cmax_rows = (N >> (l + 1)) + 1;
    dim3 gt((unsigned)((cmax_rows + 63) / 64), (s_max + 63) / 64, 2 * nn);
    if (sizeof(T) == 4 && f->use_tc) {
      kf_status r = kf_tc_telescope(t->d_lo, t->d_hi, f->rank, node0, nn, s_max, (const float*)lvl(Phat, l + 1), Tm,
                                    ldz, (float*)lvl(Phat, l), cmax_rows, f->status, s);
      if (r != KF_OK) return kf_set_err(c, r, "tensor-core telescoping failed at level %d", l);
    } else {
      KF_PHASE(KF_PH_TELESCOPE, s, k_telescope<T><<<gt, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, node0, s_max, lvl(Phat, l + 1), Tm, ldz,
                                        lvl(Phat, l)));
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return kf_set_err(c, KF_ECUDA, "factorize level %d: %s", l, cudaGetErrorString(e));
  return KF_OK;
}

}  // namespace

size_t kf_factor_tm_elems(const kf_factor* f) {
  const int D = f->t->D;
  return D > 0 ? (size_t)(1 << (D - 1)) * 2 * f->s_max * f->s_max : 1;
}

kf_status kf_factorize_leaves(kf_factor* f, cudaStream_t s) {
  return f->prec == KF_PREC_FP64 ? leaves_t<double>(f, s) : leaves_t<float>(f, s);
}

kf_status kf_factorize_level(kf_factor* f, int l, double* Tm, cudaStream_t s) {
  return f->prec == KF_PREC_FP64 ? level_t<double>(f, l, Tm, s) : level_t<float>(f, l, Tm, s);
}

kf_status kf_factorize_device(kf_factor* f, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  kf_status st = kf_factorize_leaves(f, s);
  if (st != KF_OK || f->t->D == 0) return st;
  const size_t tb = sizeof(double) * kf_factor_tm_elems(f);
  double* Tm = (double*)c->dalloc(tb, s);
  if (!Tm) return kf_set_err(c, KF_ENOMEM, "factorize: allocation failed");
  for (int l = f->t->D - 1; l >= 0 && st == KF_OK; --l) st = kf_factorize_level(f, l, Tm, s);
  c->dfree(Tm, tb, s);
  return st;
}

// Skeletonization and factorization interleaved on two streams: level l of
// the factorization needs the skeletons of levels l + 1 and l only, so the
// pivoted QRs of the upper levels (few nodes, one CTA each) run while the
// lower levels are factorized.  Events order the two streams; the caller's
// stream waits for both at the end.
kf_status kf_skel_factorize_pipelined(kf_factor* f, cudaStream_t s) {
  kf_ctx* c = f->ctx;
  const int D = f->t->D;
  if (D == 0) {
    kf_status st = kf_skeletonize_device(f, s);
    return st == KF_OK ? kf_factorize_device(f, s) : st;
  }
  kf_skel_scratch sc;
  kf_status st = kf_skel_begin(f, &sc, s);
  const size_t tb = sizeof(double) * kf_factor_tm_elems(f);
  double* Tm = st == KF_OK ? (double*)c->dalloc(tb, s) : nullptr;
  if (st == KF_OK && !Tm) st = kf_set_err(c, KF_ENOMEM, "factorize: allocation failed");
  cudaStream_t s1 = nullptr, s2 = nullptr;
  std::vector<cudaEvent_t> ev(D + 3, nullptr);
  if (st == KF_OK) {
    // the skeleton chain is the critical path: it runs on a high-priority stream
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    KF_CUDA(c, cudaStreamCreateWithPriority(&s1, cudaStreamNonBlocking, hi_prio));
    KF_CUDA(c, cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, lo_prio));
    for (auto& e : ev) KF_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    // ev[l]: skeletons of level l done (on s1); ev[0]: allocations ready (on s);
    // ev[D+1]: factorization done (on s2); ev[D+2]: skeletons done (on s1)
    cudaEventRecord(ev[0], s);
    cudaStreamWaitEvent(s1, ev[0], 0);
    cudaStreamWaitEvent(s2, ev[0], 0);
    for (int l = D; l >= 1 && st == KF_OK; --l) {
      st = kf_skel_level(f, l, &sc, s1);
      cudaEventRecord(ev[l], s1);
      if (st != KF_OK) break;
      cudaStreamWaitEvent(s2, ev[l], 0);
      if (l == D) st = kf_factorize_leaves(f, s2);
      else st = kf_factorize_level(f, l, Tm, s2);
    }
    if (st == KF_OK) st = kf_factorize_level(f, 0, Tm, s2);
    cudaEventRecord(ev[D + 1], s2);
    cudaEventRecord(ev[D + 2], s1);
    cudaStreamWaitEvent(s, ev[D + 1], 0);
    cudaStreamWaitEvent(s, ev[D + 2], 0);
  }
  if (Tm) c->dfree(Tm, tb, s);
  kf_skel_end(f, &sc, s);
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (s1) cudaStreamDestroy(s1);
  if (s2) cudaStreamDestroy(s2);
  return st;
}
