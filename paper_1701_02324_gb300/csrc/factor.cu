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

#include "kf_internal.cuh"
#include "prof.cuh"

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
                                                       int32_t* __restrict__ status) {
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
}

// P^ = L^-T L^-1 P for one leaf per CTA; rhs = Pleaf rows of the leaf (FP64,
// N x s_max), out = Phat level D rows (type T).  Columns are independent: a
// thread owns one column for blocks of 32 rows, the off-block update is a
// small GEMM through shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_leaf_phat(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                   const int32_t* __restrict__ rank, int leaf0, int ldL,
                                                   const T* __restrict__ Lall, const double* __restrict__ Pleaf,
                                                   int s_max, T* __restrict__ Phat) {
  constexpr int NB = 32;
  __shared__ T lb[NB][NB + 1];
  const int lf = blockIdx.x, node = leaf0 + lf;
  const int b = lo[node], n = hi[node] - b, s = rank[node];
  const T* L = Lall + (int64_t)lf * ldL * ldL;
  T* Y = Phat + (int64_t)b * s_max;
  const double* P = Pleaf + (int64_t)b * s_max;
  // copy rhs
  for (int64_t e = threadIdx.x; e < (int64_t)n * s_max; e += blockDim.x) {
    int i = (int)(e / s_max), q = (int)(e % s_max);
    Y[(int64_t)i * s_max + q] = q < s ? (T)P[(int64_t)i * s_max + q] : (T)0;
  }
  __syncthreads();
  if (s == 0) return;
  // forward: L y = p
  for (int kb = 0; kb < n; kb += NB) {
    const int nb = min(NB, n - kb);
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      lb[i][j] = (i < nb && j <= i) ? L[(int64_t)(kb + i) * ldL + kb + j] : (T)0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < s; q += blockDim.x) {
      T x[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) x[i] = i < nb ? Y[(int64_t)(kb + i) * s_max + q] : (T)0;
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        if (i < nb) {
          T acc = x[i];
          for (int t = 0; t < i; ++t) acc -= lb[i][t] * x[t];
          x[i] = acc / lb[i][i];
        }
      }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < nb) Y[(int64_t)(kb + i) * s_max + q] = x[i];
    }
    __syncthreads();
    // rows below: y_i -= L[i, kb:kb+nb] x_block
    for (int64_t e = threadIdx.x; e < (int64_t)(n - kb - nb) * s; e += blockDim.x) {
      int i = kb + nb + (int)(e / s), q = (int)(e % s);
      const T* Li = L + (int64_t)i * ldL + kb;
      T acc = (T)0;
      for (int t = 0; t < nb; ++t) acc += Li[t] * Y[(int64_t)(kb + t) * s_max + q];
      Y[(int64_t)i * s_max + q] -= acc;
    }
    __syncthreads();
  }
  // backward: L^T x = y
  for (int kb = ((n - 1) / NB) * NB; kb >= 0; kb -= NB) {
    const int nb = min(NB, n - kb);
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
      int i = e / NB, j = e % NB;
      lb[i][j] = (i < nb && j <= i) ? L[(int64_t)(kb + i) * ldL + kb + j] : (T)0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < s; q += blockDim.x) {
      T x[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) x[i] = i < nb ? Y[(int64_t)(kb + i) * s_max + q] : (T)0;
#pragma unroll
      for (int i = NB - 1; i >= 0; --i) {
        if (i < nb) {
          T acc = x[i];
          for (int t = i + 1; t < nb; ++t) acc -= lb[t][i] * x[t];
          x[i] = acc / lb[i][i];
        }
      }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < nb) Y[(int64_t)(kb + i) * s_max + q] = x[i];
    }
    __syncthreads();
    // rows above: y_i -= L[kb:kb+nb, i]^T x_block
    for (int64_t e = threadIdx.x; e < (int64_t)kb * s; e += blockDim.x) {
      int i = (int)(e / s), q = (int)(e % s);
      T acc = (T)0;
      for (int t = 0; t < nb; ++t) acc += L[(int64_t)(kb + t) * ldL + i] * Y[(int64_t)(kb + t) * s_max + q];
      Y[(int64_t)i * s_max + q] -= acc;
    }
    __syncthreads();
  }
}

// ---- V blocks: VT rows of every point of the level -------------------------------
template <typename T>
__global__ void k_eval_vt(const double* __restrict__ X64, const float* __restrict__ X32, int d, double c_exp,
                          const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                          const int32_t* __restrict__ rank, const int32_t* __restrict__ skel, int s_max, int node0,
                          T* __restrict__ VT) {
  const int nl = blockIdx.y, node = node0 + nl, sib = node ^ 1;
  const int b = lo[node], n = hi[node] - b, ss = rank[sib];
  const int32_t* sk = skel + (int64_t)sib * s_max;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * s_max;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / s_max), q = (int)(e % s_max);
    T v = (T)0;
    if (q < ss) v = kf_kern<T>::eval(X64, X32, b + i, sk[q], d, c_exp);
    VT[(int64_t)(b + i) * s_max + q] = v;
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

// LU with partial pivoting of Z (one CTA per node, FP64, in place); ties in
// |pivot| go to the lowest row; pivots below 1e-14 max|Z| raise ILLCOND.
__global__ void __launch_bounds__(512) k_z_lu(const int32_t* __restrict__ rank, int node0, int ldz,
                                              double* __restrict__ Z, int32_t* __restrict__ piv,
                                              int32_t* __restrict__ status) {
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int pk;
  const int nl = blockIdx.x, node = node0 + nl;
  const int z = rank[2 * node] + rank[2 * node + 1];
  double* A = Z + (int64_t)node * ldz * ldz;
  int32_t* pv = piv + (int64_t)node * ldz;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // max |Z|
  double mx = 0.0;
  for (int64_t e = tid; e < (int64_t)z * z; e += blockDim.x) mx = fmax(mx, fabs(A[(e / z) * ldz + e % z]));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if (lane == 0) rv[warp] = mx;
  __syncthreads();
  double amax = 0.0;
  for (int w = 0; w < nw; ++w) amax = fmax(amax, rv[w]);
  __syncthreads();
  bool bad = false;
  for (int k = 0; k < z; ++k) {
    double bv = -1.0;
    int bi = z;
    for (int i = k + tid; i < z; i += blockDim.x) {
      double v = fabs(A[(int64_t)i * ldz + k]);
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
      for (int w = 0; w < nw; ++w)
        if (rv[w] > b2 || (rv[w] == b2 && ri[w] < i2)) { b2 = rv[w]; i2 = ri[w]; }
      pk = i2;
      pv[k] = i2;
    }
    __syncthreads();
    const int p = pk;
    if (p != k)
      for (int j = tid; j < z; j += blockDim.x) {
        double t = A[(int64_t)k * ldz + j];
        A[(int64_t)k * ldz + j] = A[(int64_t)p * ldz + j];
        A[(int64_t)p * ldz + j] = t;
      }
    __syncthreads();
    double ukk = A[(int64_t)k * ldz + k];
    if (!(fabs(ukk) > 1e-14 * amax)) bad = true;
    if (ukk != 0.0) {
      for (int i = k + 1 + tid; i < z; i += blockDim.x) A[(int64_t)i * ldz + k] /= ukk;
      __syncthreads();
      const int w = z - k - 1;
      for (int64_t e = tid; e < (int64_t)w * w; e += blockDim.x) {
        int i = k + 1 + (int)(e / w), j = k + 1 + (int)(e % w);
        A[(int64_t)i * ldz + j] -= A[(int64_t)i * ldz + k] * A[(int64_t)k * ldz + j];
      }
    }
    __syncthreads();
  }
  if (bad && tid == 0) atomicOr(status, KF_DEV_ILLCOND);
}

// T = Z^-1 P_c for a non-root node; thread per column of P_c.
__global__ void k_z_solve_pc(const int32_t* __restrict__ rank, int node0, int ldz, const double* __restrict__ ZLU,
                             const int32_t* __restrict__ piv, const double* __restrict__ Pc, int s_max,
                             double* __restrict__ T) {
  const int nl = blockIdx.x, node = node0 + nl;
  const int z = rank[2 * node] + rank[2 * node + 1], s = rank[node];
  const double* A = ZLU + (int64_t)node * ldz * ldz;
  const int32_t* pv = piv + (int64_t)node * ldz;
  const double* B = Pc + (int64_t)node * ldz * s_max;
  double* X = T + (int64_t)nl * ldz * s_max;
  for (int q = threadIdx.x; q < s_max; q += blockDim.x) {
    if (q >= s) {
      for (int i = 0; i < ldz; ++i) X[(int64_t)i * s_max + q] = 0.0;
      continue;
    }
    for (int i = 0; i < z; ++i) X[(int64_t)i * s_max + q] = B[(int64_t)i * s_max + q];
    for (int i = z; i < ldz; ++i) X[(int64_t)i * s_max + q] = 0.0;
    for (int k = 0; k < z; ++k) {
      int p = pv[k];
      if (p != k) {
        double t = X[(int64_t)k * s_max + q];
        X[(int64_t)k * s_max + q] = X[(int64_t)p * s_max + q];
        X[(int64_t)p * s_max + q] = t;
      }
    }
    for (int i = 0; i < z; ++i) {
      double acc = X[(int64_t)i * s_max + q];
      for (int t = 0; t < i; ++t) acc -= A[(int64_t)i * ldz + t] * X[(int64_t)t * s_max + q];
      X[(int64_t)i * s_max + q] = acc;
    }
    for (int i = z - 1; i >= 0; --i) {
      double acc = X[(int64_t)i * s_max + q];
      for (int t = i + 1; t < z; ++t) acc -= A[(int64_t)i * ldz + t] * X[(int64_t)t * s_max + q];
      X[(int64_t)i * s_max + q] = acc / A[(int64_t)i * ldz + i];
    }
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

template <typename T>
kf_status factorize_t(kf_factor* f, cudaStream_t s) {
  kf_tree* t = f->t;
  kf_ctx* c = f->ctx;
  const int D = t->D, s_max = f->s_max, ldz = 2 * s_max;
  const int64_t N = t->N;
  const int ldL = t->leaf_max;
  T* L = (T*)f->L;
  T* Phat = (T*)f->Phat;
  T* VT = (T*)f->VT;
  auto lvl = [&](T* base, int l) { return base + (int64_t)(l - 1) * N * s_max; };
  const int leaf0 = 1 << D, nleaf = 1 << D;
  // leaves
  {
    dim3 g((ldL + 127) / 128, ldL, nleaf);
    KF_PHASE(KF_PH_LEAF_ASM, s, k_leaf_assemble<T><<<g, 128, 0, s>>>(t->X64, t->X32, t->d, f->c_exp, f->lambda, t->d_lo, t->d_hi, leaf0, ldL, L));
    KF_PHASE(KF_PH_LEAF_CHOL, s, k_leaf_cholesky<T><<<nleaf, 256, 0, s>>>(t->d_lo, t->d_hi, leaf0, ldL, L, f->status));
    if (D > 0)
      KF_PHASE(KF_PH_LEAF_PHAT, s, k_leaf_phat<T><<<nleaf, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, leaf0, ldL, L, f->Pleaf, s_max, lvl(Phat, D)));
    KF_LAUNCH_CHECK(c);
  }
  if (D == 0) return KF_OK;
  double* Tm = (double*)c->dalloc(sizeof(double) * (size_t)(1 << (D - 1)) * ldz * s_max, s);
  if (!Tm) return kf_set_err(c, KF_ENOMEM, "factorize: allocation failed");
  kf_status st = KF_OK;
  for (int l = D - 1; l >= 0 && st == KF_OK; --l) {
    const int node0 = 1 << l, nn = 1 << l;
    const int child0 = 1 << (l + 1);
    // V blocks of the children's level
    dim3 gv(grid_for((int64_t)(N >> (l + 1)) * s_max + s_max, 256, 4096), 2 * nn);
    KF_PHASE(KF_PH_EVAL_V, s, k_eval_vt<T><<<gv, 256, 0, s>>>(t->X64, t->X32, t->d, f->c_exp, t->d_lo, t->d_hi, f->rank, f->skel, s_max, child0,
                                    lvl(VT, l + 1)));
    // Z
    KF_PHASE(KF_PH_ZOFF, s, k_z_init<<<dim3(grid_for((int64_t)ldz * ldz, 256, 64), nn), 256, 0, s>>>(f->rank, node0, ldz, f->ZLU));
    const int tiles = ((s_max + 63) / 64) * ((s_max + 63) / 64);
    const int64_t rows = N >> (l + 1);
    int ksplit = (int)std::max<int64_t>(1, std::min<int64_t>(rows / 512, (152 * 8) / std::max(1, 2 * nn * tiles) + 1));
    KF_PHASE(KF_PH_ZOFF, s, k_zoff<T><<<dim3(tiles, ksplit, 2 * nn), 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, node0, s_max, lvl(VT, l + 1),
                                                          lvl(Phat, l + 1), ldz, f->ZLU, ksplit));
    KF_PHASE(KF_PH_ZLU, s, k_z_lu<<<nn, 512, 0, s>>>(f->rank, node0, ldz, f->ZLU, f->Zpiv, f->status));
    if (l >= 1) {
      KF_PHASE(KF_PH_ZSOLVE_PC, s, k_z_solve_pc<<<nn, 128, 0, s>>>(f->rank, node0, ldz, f->ZLU, f->Zpiv, f->Pc, s_max, Tm));
      const int64_t cmax_rows = (N >> (l + 1)) + 1;
      dim3 gt((unsigned)((cmax_rows + 63) / 64), (s_max + 63) / 64, 2 * nn);
      KF_PHASE(KF_PH_TELESCOPE, s, k_telescope<T><<<gt, 256, 0, s>>>(t->d_lo, t->d_hi, f->rank, node0, s_max, lvl(Phat, l + 1), Tm, ldz,
                                        lvl(Phat, l)));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = kf_set_err(c, KF_ECUDA, "factorize level %d: %s", l, cudaGetErrorString(e));
  }
  c->dfree(Tm, sizeof(double) * (size_t)(1 << (D - 1)) * ldz * s_max, s);
  return st;
}

}  // namespace

kf_status kf_factorize_device(kf_factor* f, cudaStream_t s) {
  return f->prec == KF_PREC_FP64 ? factorize_t<double>(f, s) : factorize_t<float>(f, s);
}
