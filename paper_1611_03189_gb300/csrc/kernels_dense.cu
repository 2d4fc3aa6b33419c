// Batched variable-size dense kernels of the factorization.
//
//   k_gemm       C = alpha op(A) op(B) + beta C over a list of tasks (tiles of
//                64 x 64, 16 x 16 threads, 4 x 4 outputs per thread).
//   k_sum        dst = beta dst + alpha sum_s op(src_s), sources summed in list
//                order: block gathers, merges and the deterministic Schur
//                scatter of Sec. 3.2 (several super nodes of one wave updating
//                the same neighbour block).
//   k_chol_inv   A = L L^T and L^-1, one CTA per matrix (pivot blocks A_ss and
//                the small Gram matrices of the CholQR of L^-1 U).
//   k_trunc      truncation of the well-separated block (Sec. 3.2 eq.
//                local_compression, Sec. 6 GC basis), one CTA per super node:
//                cyclic Jacobi eigen-solves of the Gram matrix A_sw A_sw^T.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cfloat>

#include "hs_internal.h"
#include "trunc_common.cuh"

namespace hs {

namespace {

template <typename T>
struct Lim;
template <>
struct Lim<double> {
  static __device__ __forceinline__ double eps() { return 2.220446049250313e-16; }
  static __device__ __forceinline__ double tiny() { return 1e-290; }
};
template <>
struct Lim<float> {
  static __device__ __forceinline__ float eps() { return 1.1920929e-07f; }
  static __device__ __forceinline__ float tiny() { return 1e-35f; }
};

__device__ __forceinline__ int find_task(const int *tile_start, int ntasks, int b) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (tile_start[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// batched GEMM
// ---------------------------------------------------------------------------
constexpr int GK = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm(const GemmTask<T> *__restrict__ tasks,
                                              const int *__restrict__ tile_start, int ntasks) {
  __shared__ T As[GK][GEMM_TM + 1];
  __shared__ T Bs[GK][GEMM_TN + 1];
  const int ti = find_task(tile_start, ntasks, blockIdx.x);
  const GemmTask<T> t = tasks[ti];
  const int local = blockIdx.x - tile_start[ti];
  const int tiles_n = (t.N + GEMM_TN - 1) / GEMM_TN;
  const int row0 = (local / tiles_n) * GEMM_TM;
  const int col0 = (local % tiles_n) * GEMM_TN;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int k0 = 0; k0 < t.K; k0 += GK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int i, k;
      if (t.ta == 0) {
        i = e / GK;
        k = e % GK;
      } else {
        k = e / GEMM_TM;
        i = e % GEMM_TM;
      }
      const int gi = row0 + i, gk = k0 + k;
      T v = T(0);
      if (gi < t.M && gk < t.K)
        v = (t.ta == 0) ? t.A[(int64_t)gi * t.lda + gk] : t.A[(int64_t)gk * t.lda + gi];
      As[k][i] = v;
      int j;
      if (t.tb == 0) {
        k = e / GEMM_TN;
        j = e % GEMM_TN;
      } else {
        j = e / GK;
        k = e % GK;
      }
      const int gj = col0 + j;
      const int gk2 = k0 + k;
      T w = T(0);
      if (gj < t.N && gk2 < t.K)
        w = (t.tb == 0) ? t.B[(int64_t)gk2 * t.ldb + gj] : t.B[(int64_t)gj * t.ldb + gk2];
      Bs[k][j] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= t.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      if (c >= t.N) continue;
      T *p = t.C + (int64_t)r * t.ldc + c;
      T v = t.alpha * acc[i][j];
      if (t.beta != T(0)) v = fma(t.beta, *p, v);
      *p = v;
    }
  }
}

// ---------------------------------------------------------------------------
// batched deterministic accumulate / copy
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_sum(const SumTask<T> *__restrict__ tasks,
                                             const SumSrc<T> *__restrict__ srcs,
                                             const int *__restrict__ tile_start, int ntasks) {
  __shared__ T sm[SUM_TILE][SUM_TILE + 1];
  const int ti = find_task(tile_start, ntasks, blockIdx.x);
  const SumTask<T> t = tasks[ti];
  const int local = blockIdx.x - tile_start[ti];
  const int tiles_c = (t.cols + SUM_TILE - 1) / SUM_TILE;
  const int i0 = (local / tiles_c) * SUM_TILE;
  const int j0 = (local % tiles_c) * SUM_TILE;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int s = 0; s < t.nsrc; ++s) {
    const SumSrc<T> src = srcs[t.first + s];
    if (!src.trans) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty + 8 * r, j = j0 + tx;
        if (i < t.rows && j < t.cols) acc[r] += src.ptr[(int64_t)i * src.ld + j];
      }
    } else {
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int jj = ty + 8 * r, ii = tx;
        T v = T(0);
        if (i0 + ii < t.rows && j0 + jj < t.cols) v = src.ptr[(int64_t)(j0 + jj) * src.ld + i0 + ii];
        sm[jj][ii] = v;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] += sm[tx][ty + 8 * r];
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 8 * r, j = j0 + tx;
    if (i < t.rows && j < t.cols) {
      T *p = t.dst + (int64_t)i * t.ld + j;
      T v = t.alpha * acc[r];
      if (t.beta != T(0)) v = fma(t.beta, *p, v);
      *p = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Cholesky and inverse of the factor, one CTA per matrix
// ---------------------------------------------------------------------------
constexpr int CHOL_THREADS = 512;

// W (ld m) holds A on entry; on exit the lower triangle holds L^-1 and the
// strict upper triangle is zero.  Returns 0 or (failing pivot + 1).  tmp holds
// 3m values.
//
// Right-looking Cholesky fused with the rows of X = L^-1 by forward
// substitution: step j forms column j of L and, in the same phase as the
// trailing update, row j of X,
//   X_jc = (delta_jc - sum_{p=c..j-1} L_jp X_pc) / L_jj   (c <= j),
// thread c owning column c of X.  Row j of L is needed only in step j, so row
// j - 1 of X (kept in tmp until then) replaces it during step j.  Two
// barriers per step.
template <typename T>
__device__ int chol_inv_inplace(T *W, int m, T *tmp, int *flag) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp0 = tid >> 5, lane0 = tid & 31, nw0 = nt >> 5;
  T *col = tmp;                  // scaled column j of L
  T *xr0 = tmp + m, *xr1 = xr0 + m;   // rows j (j even: xr0) and j - 1 of X
  (void)flag;
  for (int j = 0; j < m; ++j) {
    // every thread reads the pivot (the previous step's update is complete)
    const T d = W[(size_t)j * m + j];
    if (!(d > T(0)) || !isfinite(d)) return j + 1;
    const T djj = sqrt(d);
    for (int i = j + 1 + tid; i < m; i += nt) {
      const T l = W[(size_t)i * m + j] / djj;
      W[(size_t)i * m + j] = l;
      col[i] = l;
    }
    __syncthreads();
    // trailing update, one warp per row (lanes over columns, coalesced)
    for (int i = j + 1 + warp0; i < m; i += nw0) {
      const T li = col[i];
      T *row = W + (size_t)i * m;
      for (int c = j + 1 + lane0; c <= i; c += 32) row[c] -= li * col[c];
    }
    // row j of X; row j - 1 of X retires into row j - 1 of W
    T *xj = (j & 1) ? xr1 : xr0;
    const T *xprev = (j & 1) ? xr0 : xr1;
    const T *Lj = W + (size_t)j * m;
    for (int c = tid; c <= j; c += nt) {
      T s0 = (c == j) ? T(1) : T(0), s1 = T(0);
      int p = c;
      for (; p + 2 < j; p += 2) {
        s0 = fma(-Lj[p], W[(size_t)p * m + c], s0);
        s1 = fma(-Lj[p + 1], W[(size_t)(p + 1) * m + c], s1);
      }
      if (p + 1 < j) s0 = fma(-Lj[p], W[(size_t)p * m + c], s0);
      if (c + 1 <= j) s1 = fma(-Lj[j - 1], xprev[c], s1);
      xj[c] = (s0 + s1) / djj;
      if (c + 1 <= j) W[(size_t)(j - 1) * m + c] = xprev[c];
    }
    __syncthreads();
  }
  // the last row of X, and zeros above the diagonal
  const T *xlast = ((m - 1) & 1) ? xr1 : xr0;
  for (int c = tid; c < m; c += nt) W[(size_t)(m - 1) * m + c] = xlast[c];
  __syncthreads();
  for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
    const int i = (int)(e / m), c = (int)(e % m);
    if (c > i) W[e] = T(0);
  }
  __syncthreads();
  return 0;
}

template <typename T, bool SMEM>
__global__ void __launch_bounds__(CHOL_THREADS) k_chol_inv(const CholTask<T> *__restrict__ tasks,
                                                           int *__restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int flag;
  const CholTask<T> t = tasks[blockIdx.x];
  const int m = t.m;
  if (threadIdx.x == 0) flag = 0;
  if (m == 0) {
    if (threadIdx.x == 0) status[t.status_idx] = 0;
    return;
  }
  T *W;
  T *tmp;
  if (SMEM) {
    W = reinterpret_cast<T *>(smem_raw);
    tmp = W + (size_t)m * m;
  } else {
    W = t.Linv;  // requires ldl == m
    tmp = reinterpret_cast<T *>(smem_raw);
  }
  for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
    const int i = (int)(e / m), c = (int)(e % m);
    W[e] = (c <= i) ? t.A[(int64_t)i * t.lda + c] : T(0);
  }
  __syncthreads();
  const int st = chol_inv_inplace(W, m, tmp, &flag);
  if (SMEM && st == 0) {
    for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
      const int i = (int)(e / m), c = (int)(e % m);
      t.Linv[(int64_t)i * t.ldl + c] = W[e];
    }
  }
  if (threadIdx.x == 0) status[t.status_idx] = st;
}

// ---------------------------------------------------------------------------
// truncation: cyclic Jacobi on the Gram matrix (round-robin pair ordering)
// ---------------------------------------------------------------------------
constexpr int TRUNC_THREADS = 256;

template <typename T>
struct JacobiShared {
  int *pp, *qq;
  T *cs, *sn;
  int *flag;
};

template <typename T>
__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  s = red[32];
  __syncthreads();
  return s;
}

// Eigen-decomposition A = V diag(A') V^T of the symmetric m x m matrix A (ld
// m), in place: on exit diag(A) holds the eigenvalues.  V is filled when
// want_v.  Returns the number of sweeps.
template <typename T>
__device__ int jacobi_eig(T *A, T *V, int m, bool want_v, JacobiShared<T> sh, int max_sweeps) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (want_v)
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) V[e] = (e / m == e % m) ? T(1) : T(0);
  if (m < 2) {
    __syncthreads();
    return 0;
  }
  // scale for the absolute floor of the rotation test
  T scale = T(0);
  for (int i = 0; i < m; ++i) scale = fmax(scale, fabs(A[i * m + i]));
  // entries below eps * scale move no eigenvalue by more than the rounding of
  // the whole computation: treat them as converged (otherwise rounding noise
  // in the near-null space keeps every sweep busy)
  const T floor_abs = Lim<T>::eps() * scale + Lim<T>::tiny();
  const int mp = m + (m & 1);
  const int np = mp / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *sh.flag = 0;
    __syncthreads();
    for (int r = 0; r < mp - 1; ++r) {
      for (int i = tid; i < np; i += nt) {
        int a, b;
        if (i == 0) {
          a = r;
          b = mp - 1;
        } else {
          a = (r + i) % (mp - 1);
          b = (r - i + (mp - 1)) % (mp - 1);
        }
        if (a > b) {
          const int x = a;
          a = b;
          b = x;
        }
        T c = T(1), s = T(0);
        if (b < m) {
          const T app = A[a * m + a], aqq = A[b * m + b], apq = A[a * m + b];
          if (fabs(apq) > Lim<T>::eps() * sqrt(fabs(app * aqq)) && fabs(apq) > floor_abs) {
            const T th = (aqq - app) / (T(2) * apq);
            const T ath = fabs(th);
            const T root = (ath > T(1)) ? ath * sqrt(T(1) + (T(1) / ath) * (T(1) / ath))
                                        : sqrt(T(1) + th * th);
            T tt = T(1) / (ath + root);
            if (th < T(0)) tt = -tt;
            c = T(1) / sqrt(T(1) + tt * tt);
            s = tt * c;
            *sh.flag = 1;
          }
        }
        sh.pp[i] = a;
        sh.qq[i] = b;
        sh.cs[i] = c;
        sh.sn[i] = s;
      }
      __syncthreads();
      // A <- J^T A J, 2 x 2 blocks of (pair i rows) x (pair j cols)
      for (int w = tid; w < np * np; w += nt) {
        const int i = w / np, j = w - (w / np) * np;
        const T si = sh.sn[i], sj = sh.sn[j];
        if (si == T(0) && sj == T(0)) continue;
        const T ci = sh.cs[i], cj = sh.cs[j];
        const int a = sh.pp[i], b = sh.qq[i], c = sh.pp[j], d = sh.qq[j];
        const bool bv = b < m, dv = d < m;
        const T x00 = A[a * m + c];
        const T x01 = dv ? A[a * m + d] : T(0);
        const T x10 = bv ? A[b * m + c] : T(0);
        const T x11 = (bv && dv) ? A[b * m + d] : T(0);
        // right: columns (c, d) <- (cj col_c - sj col_d, sj col_c + cj col_d)
        const T y00 = cj * x00 - sj * x01, y01 = sj * x00 + cj * x01;
        const T y10 = cj * x10 - sj * x11, y11 = sj * x10 + cj * x11;
        // left: rows (a, b) <- (ci row_a - si row_b, si row_a + ci row_b)
        T z00 = ci * y00 - si * y10, z01 = ci * y01 - si * y11;
        T z10 = si * y00 + ci * y10, z11 = si * y01 + ci * y11;
        if (i == j && si != T(0)) {
          z01 = T(0);
          z10 = T(0);
        }
        A[a * m + c] = z00;
        if (dv) A[a * m + d] = z01;
        if (bv) A[b * m + c] = z10;
        if (bv && dv) A[b * m + d] = z11;
      }
      if (want_v) {
        for (int w = tid; w < m * np; w += nt) {
          const int row = w / np, j = w - (w / np) * np;
          const T sj = sh.sn[j];
          if (sj == T(0)) continue;
          const T cj = sh.cs[j];
          const int c = sh.pp[j], d = sh.qq[j];
          const T v0 = V[row * m + c], v1 = V[row * m + d];
          V[row * m + c] = cj * v0 - sj * v1;
          V[row * m + d] = sj * v0 + cj * v1;
        }
      }
      __syncthreads();
    }
    const int any = *sh.flag;
    __syncthreads();
    if (!any) break;
  }
  return sweep;
}

// Selects the columns of V whose eigenvalues (diag of A) exceed thr, in
// descending order, writing them to U columns col0 .. col0+k-1.  Returns k.
template <typename T>
__device__ int select_columns(const T *A, const T *V, int m, double thr, T *U, int col0,
                              double *red) {
  int cnt = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    if ((double)A[i * m + i] > thr) ++cnt;
  const int k = (int)(block_sum<T>((double)cnt, red) + 0.5);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const T di = A[i * m + i];
    if (!((double)di > thr)) continue;
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const T dj = A[j * m + j];
      if (dj > di || (dj == di && j < i)) ++rank;
    }
    if (col0 + rank >= m) continue;
    for (int r = 0; r < m; ++r) U[(int64_t)r * m + col0 + rank] = V[(int64_t)r * m + i];
  }
  __syncthreads();
  return k;
}

template <typename T, bool SMEM>
__global__ void __launch_bounds__(TRUNC_THREADS) k_trunc(const TruncTask<T> *__restrict__ tasks,
                                                        int *__restrict__ kout, int variant) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[33];
  __shared__ int flag;
  __shared__ double s_gR[kMaxK1 * 2 * kMaxPhi], s_gW[kMaxK1 * kMaxK1 + kMaxK1];
  __shared__ int s_gk;
  __shared__ T s_c[kMaxK1 * kMaxK1];
  const TruncTask<T> t = tasks[blockIdx.x];
  const double eps = t.eps;
  const int m = t.m;
  const int mp = m + (m & 1);
  const int np = mp / 2 > 0 ? mp / 2 : 1;
  unsigned char *p = smem_raw;
  T *A;
  T *V;
  if (SMEM) {
    A = reinterpret_cast<T *>(p);
    p += sizeof(T) * (size_t)m * m;
    V = reinterpret_cast<T *>(p);
    p += sizeof(T) * (size_t)m * m;
  } else {
    A = t.work;
    V = t.work + (size_t)m * m;
  }
  JacobiShared<T> sh;
  sh.cs = reinterpret_cast<T *>(p);
  p += sizeof(T) * np;
  sh.sn = reinterpret_cast<T *>(p);
  p += sizeof(T) * np;
  sh.pp = reinterpret_cast<int *>(p);
  p += sizeof(int) * np;
  sh.qq = reinterpret_cast<int *>(p);
  sh.flag = &flag;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (m == 0) {
    if (tid == 0) kout[t.k_idx] = 0;
    return;
  }
  if (variant == HS_LORASP && eps == 0.0) {
    // no truncation: complete basis U = I
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) t.U[e] = (e / m == e % m) ? T(1) : T(0);
    if (tid == 0) kout[t.k_idx] = m;
    return;
  }
  // ---- GC basis U_1 (Sec. 6: orth[phi_s, A_sw phi_w]; Appendix B: its
  // dominant left singular vectors), scratch in A and V (2 m^2 T >= m doubles)
  int k1 = 0;
  if (variant != HS_LORASP)
    k1 = gc_basis_dev<T>(t.phi, t.a, t.np, m, variant == HS_GC_PROJ, t.eps1, t.U, (double *)A, red, s_gR, s_gW,
                         &s_gk);
  // ---- ||A_sw||_2^2 = lambda_max(G)
  for (int64_t e = tid; e < (int64_t)m * m; e += nt) A[e] = t.G[e];
  __syncthreads();
  const int max_sweeps = 40;
  double thr;
  if (variant == HS_LORASP) {
    jacobi_eig<T>(A, V, m, true, sh, max_sweeps);
    double lmax = 0.0;
    for (int i = 0; i < m; ++i) lmax = fmax(lmax, (double)A[i * m + i]);
    thr = eps * eps * lmax;
    const int k = select_columns<T>(A, V, m, thr, t.U, 0, red);
    if (tid == 0) kout[t.k_idx] = min(k, t.cap);   // the columns come in descending order
    return;
  }
  if (eps == 0.0) {
    // no truncation: complete the GC basis to all of R^m (Householder QR of U_1;
    // scratch k1 m <= 2 m^2 T in A and V)
    // (nothing to complete when U_1 already spans R^m)
    if (k1 < m) {
      if (k1 <= 2)
        gc_complete<T>(t.U, m, k1, (double *)A, red);
      else
        gc_complete_n<T>(t.U, m, k1, (double *)A, s_gW, red);
    }
    if (tid == 0) kout[t.k_idx] = m;
    return;
  }
  double lmax = 0.0;
  if (eps > 0.0) {
    jacobi_eig<T>(A, V, m, false, sh, max_sweeps);
    for (int i = 0; i < m; ++i) lmax = fmax(lmax, (double)A[i * m + i]);
    __syncthreads();
  }
  // ---- matrix whose leading eigenvectors give U_2: (I - U1 U1^T) G (I - U1 U1^T),
  // or the projector I - U1 U1^T itself when eps == 0 (complete basis)
  // X = G U1 (m x k1) in V's columns 0..k1-1 (scratch, ld m), all in T
  if (eps > 0.0) {
    for (int w = tid; w < m * k1; w += nt) {
      const int i = w / k1, a = w % k1;
      T s = T(0);
      for (int j = 0; j < m; ++j) s = fma(t.G[(int64_t)i * m + j], t.U[(int64_t)j * m + a], s);
      V[i * m + a] = s;
    }
    __syncthreads();
    // c = U1^T G U1 (k1 x k1, ld kMaxK1)
    for (int a = 0; a < k1; ++a)
      for (int b = 0; b < k1; ++b) {
        double s = 0.0;
        for (int i = tid; i < m; i += nt) s += (double)(t.U[(int64_t)i * m + a] * V[i * m + b]);
        const T cab = (T)block_sum<T>(s, red);
        if (tid == 0) s_c[a * kMaxK1 + b] = cab;
      }
    __syncthreads();
    if (k1 <= 2) {
      // one or two basis vectors (one preserved vector): c in registers
      T c[2][2];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) c[a][b] = (a < k1 && b < k1) ? s_c[a * kMaxK1 + b] : T(0);
      for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
        const int i = (int)(e / m), j = (int)(e % m);
        T v = t.G[e];
        for (int a = 0; a < k1; ++a) {
          const T ui = t.U[(int64_t)i * m + a], uj = t.U[(int64_t)j * m + a];
          v = fma(-ui, V[j * m + a], fma(-V[i * m + a], uj, v));
          for (int b = 0; b < k1; ++b) v = fma(ui * c[a][b], t.U[(int64_t)j * m + b], v);
        }
        A[e] = v;
      }
    } else {
      for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
        const int i = (int)(e / m), j = (int)(e % m);
        T v = t.G[e];
        for (int a = 0; a < k1; ++a) {
          const T ui = t.U[(int64_t)i * m + a], uj = t.U[(int64_t)j * m + a];
          v = fma(-ui, V[j * m + a], fma(-V[i * m + a], uj, v));
          for (int b = 0; b < k1; ++b) v = fma(ui * s_c[a * kMaxK1 + b], t.U[(int64_t)j * m + b], v);
        }
        A[e] = v;
      }
    }
    thr = eps * eps * lmax;
  } else {
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
      const int i = (int)(e / m), j = (int)(e % m);
      double v = (i == j) ? 1.0 : 0.0;
      for (int a = 0; a < k1; ++a) v -= (double)t.U[(int64_t)i * m + a] * (double)t.U[(int64_t)j * m + a];
      A[e] = (T)v;
    }
    thr = 0.5;
  }
  __syncthreads();
  jacobi_eig<T>(A, V, m, true, sh, max_sweeps);
  const int k2 = select_columns<T>(A, V, m, thr, t.U, k1, red);
  int k = k1 + min(k2, max(t.cap - k1, 0));
  if (k > m) k = m;
  if (tid == 0) kout[t.k_idx] = k;
}

// ---------------------------------------------------------------------------
// CSR value movement
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_scatter_values(const double *__restrict__ val, const int64_t *__restrict__ dest,
                                 int64_t nnz, T *__restrict__ pool) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = dest[e];
    if (d >= 0) pool[d] = (T)val[e];
  }
}

__global__ void k_gather_values(const double *__restrict__ val, const int32_t *__restrict__ src,
                                int64_t nnz, double *__restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = val[src[e]];
}

template <typename T>
size_t trunc_small_arrays(int m) {
  const int mp = m + (m & 1);
  const int np = mp / 2 > 0 ? mp / 2 : 1;
  return 2 * sizeof(T) * np + 2 * sizeof(int) * np + 64;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
void launch_gemm(const GemmTask<T> *d_tasks, const int *d_tile_start, int ntasks, int total_tiles,
                 cudaStream_t st) {
  if (ntasks == 0 || total_tiles == 0) return;
  k_gemm<T><<<total_tiles, 256, 0, st>>>(d_tasks, d_tile_start, ntasks);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_sum(const SumTask<T> *d_tasks, const SumSrc<T> *d_srcs, const int *d_tile_start,
                int ntasks, int total_tiles, cudaStream_t st) {
  if (ntasks == 0 || total_tiles == 0) return;
  k_sum<T><<<total_tiles, 256, 0, st>>>(d_tasks, d_srcs, d_tile_start, ntasks);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

// first failing pivot over the diagonal blocks of a blocked Cholesky
static __global__ void k_status_merge(const StatusMerge *__restrict__ t, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int r = 0;
  for (int b = 0; b < t[i].nblk && !r; ++b)
    if (t[i].bs[b]) r = b * t[i].nb + t[i].bs[b];
  *t[i].out = r;
}

template <typename T>
int chol_smem_cap() {
  return sizeof(T) == 8 ? 160 : 224;
}

template <typename T>
void launch_chol_inv(const CholTask<T> *d_tasks, int ntasks, int *d_status, int max_m,
                     cudaStream_t st) {
  if (ntasks == 0) return;
  if (max_m <= chol_smem_cap<T>()) {
    const size_t sm = sizeof(T) * ((size_t)max_m * max_m + 3 * (size_t)max_m + 8);
    check_dynamic_smem(sm, allow_max_dynamic_smem<&k_chol_inv<T, true>>(), "k_chol_inv");
    k_chol_inv<T, true><<<ntasks, CHOL_THREADS, sm, st>>>(d_tasks, d_status);
  } else {
    const size_t sm = sizeof(T) * (3 * (size_t)max_m + 8);
    check_dynamic_smem(sm, allow_max_dynamic_smem<&k_chol_inv<T, false>>(), "k_chol_inv");
    k_chol_inv<T, false><<<ntasks, CHOL_THREADS, sm, st>>>(d_tasks, d_status);
  }
  count_launch();
  HS_CUDA(cudaGetLastError());
}

template <typename T>
int trunc_smem_cap() {
  return sizeof(T) == 8 ? 110 : 156;
}

template <typename T>
void launch_trunc(const TruncTask<T> *d_tasks, int ntasks, int *d_k, double eps, int variant,
                  int max_m, cudaStream_t st) {
  if (ntasks == 0) return;
  if (max_m <= trunc_smem_cap<T>()) {
    const size_t sm = 2 * sizeof(T) * (size_t)max_m * max_m + trunc_small_arrays<T>(max_m);
    check_dynamic_smem(sm, allow_max_dynamic_smem<&k_trunc<T, true>>(), "k_trunc");
    k_trunc<T, true><<<ntasks, TRUNC_THREADS, sm, st>>>(d_tasks, d_k, variant);
  } else {
    const size_t sm = trunc_small_arrays<T>(max_m);
    check_dynamic_smem(sm, allow_max_dynamic_smem<&k_trunc<T, false>>(), "k_trunc");
    k_trunc<T, false><<<ntasks, TRUNC_THREADS, sm, st>>>(d_tasks, d_k, variant);
  }
  count_launch();
  HS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_scatter_values(const double *val, const int64_t *dest, int64_t nnz, T *pool,
                           cudaStream_t st) {
  if (nnz == 0) return;
  const int grid = (int)std::min<int64_t>((nnz + 255) / 256, 152 * 16);
  k_scatter_values<T><<<grid, 256, 0, st>>>(val, dest, nnz, pool);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

void launch_gather_values(const double *val, const int32_t *src, int64_t nnz, double *out,
                          cudaStream_t st) {
  if (nnz == 0) return;
  const int grid = (int)std::min<int64_t>((nnz + 255) / 256, 152 * 16);
  k_gather_values<<<grid, 256, 0, st>>>(val, src, nnz, out);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

// D^-1/2 of each row (the reciprocal square root of its diagonal entry); a
// row whose diagonal entry is missing or not positive sets *flag
static __global__ void k_diag_scale(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                    const double *__restrict__ va, int64_t n, double *__restrict__ ds,
                                    int *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e)
      if (ci[e] == i) d += va[e];
    if (d > 0.0) {
      ds[i] = 1.0 / sqrt(d);
    } else {
      ds[i] = 1.0;
      atomicExch(flag, 1);
    }
  }
}

// out = D^-1/2 A D^-1/2 entry by entry
static __global__ void k_scale_values(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                      const double *__restrict__ va, int64_t n, const double *__restrict__ ds,
                                      double *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double di = ds[i];
    for (int e = rp[i]; e < rp[i + 1]; ++e) out[e] = va[e] * di * ds[ci[e]];
  }
}

void launch_diag_scale(const int32_t *rp, const int32_t *ci, const double *val, int64_t n, double *ds,
                       double *val_scaled, int *flag, cudaStream_t st) {
  if (n == 0) return;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_diag_scale<<<grid, 256, 0, st>>>(rp, ci, val, n, ds, flag);
  k_scale_values<<<grid, 256, 0, st>>>(rp, ci, val, n, ds, val_scaled);
  count_launch(2);
  HS_CUDA(cudaGetLastError());
}

// preserved vectors of the scaled system: out = D^1/2 raw, n x np row-major
template <typename T>
static __global__ void k_phi_scale(const T *__restrict__ raw, const double *__restrict__ ds, int64_t n, int np,
                                   T *__restrict__ out) {
  const int64_t tot = n * np;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (T)((double)raw[e] / ds[e / np]);
}

template <typename T>
void launch_phi_scale(const T *raw, const double *ds, int64_t n, int np, T *out, cudaStream_t st) {
  if (n == 0) return;
  const int grid = (int)std::min<int64_t>((n * np + 255) / 256, 152 * 16);
  k_phi_scale<T><<<grid, 256, 0, st>>>(raw, ds, n, np, out);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

// one CTA per task, a grid-stride loop over its elements
static __global__ void k_convert_list(const ConvTask *__restrict__ t, int n) {
  const ConvTask c = t[blockIdx.x];
  if (c.widen) {
    const float *s = (const float *)c.src;
    double *d = (double *)c.dst;
    for (int64_t e = threadIdx.x; e < c.n; e += blockDim.x) d[e] = (double)s[e];
  } else {
    const double *s = (const double *)c.src;
    float *d = (float *)c.dst;
    for (int64_t e = threadIdx.x; e < c.n; e += blockDim.x) d[e] = (float)s[e];
  }
}

void launch_convert_list(const ConvTask *d_tasks, int ntasks, cudaStream_t st) {
  if (ntasks == 0) return;
  k_convert_list<<<ntasks, 256, 0, st>>>(d_tasks, ntasks);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

void launch_status_merge(const StatusMerge *d_tasks, int ntasks, cudaStream_t st) {
  if (ntasks == 0) return;
  k_status_merge<<<(ntasks + 127) / 128, 128, 0, st>>>(d_tasks, ntasks);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

#define HS_INST(T)                                                                            \
  template void launch_gemm<T>(const GemmTask<T> *, const int *, int, int, cudaStream_t);     \
  template void launch_sum<T>(const SumTask<T> *, const SumSrc<T> *, const int *, int, int,   \
                              cudaStream_t);                                                  \
  template void launch_chol_inv<T>(const CholTask<T> *, int, int *, int, cudaStream_t);       \
  template int chol_smem_cap<T>();                                                            \
  template void launch_trunc<T>(const TruncTask<T> *, int, int *, double, int, int,           \
                                cudaStream_t);                                                \
  template void launch_phi_scale<T>(const T *, const double *, int64_t, int, T *, cudaStream_t); \
  template void launch_scatter_values<T>(const double *, const int64_t *, int64_t, T *,       \
                                         cudaStream_t);
HS_INST(double)
HS_INST(float)
#undef HS_INST

}  // namespace hs
