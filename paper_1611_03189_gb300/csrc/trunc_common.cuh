// Device helpers shared by the two truncation kernels (Sec. 6, GC basis).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hs {

// Block-wide sum of one double per thread (any block size up to 1024);
// red needs 33 doubles of shared memory.  Every thread gets the total.
__device__ __forceinline__ double blk_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  const double s = red[32];
  __syncthreads();
  return s;
}

// Complete the k1 <= 2 orthonormal columns U[:, 0..k1) (row-major, ld m) to an
// orthonormal basis of R^m, writing columns k1..m-1.  Q = H1 H2 from the
// Householder QR of U_1; its trailing m - k1 columns span the complement of
// span(U_1).  Used when eps = 0 (no truncation, Sec. 6 basis kept complete).
// scratch: 2 m doubles.
template <typename T>
__device__ void gc_complete(T *U, int m, int k1, double *scratch, double *red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  double *v1 = scratch, *v2 = scratch + m;
  if (k1 == 0) {
    for (int64_t q = tid; q < (int64_t)m * m; q += nt) U[q] = (T)((q / m == q % m) ? 1.0 : 0.0);
    __syncthreads();
    return;
  }
  // H1: v1 = u1 + sign(u1[0]) e1, tau1 = 2 / v1.v1  (u1 has unit norm)
  const double x0 = (double)U[0];
  const double s1 = x0 >= 0.0 ? 1.0 : -1.0;
  for (int i = tid; i < m; i += nt) v1[i] = (double)U[(int64_t)i * m] + (i == 0 ? s1 : 0.0);
  __syncthreads();
  double t = 0.0;
  for (int i = tid; i < m; i += nt) t += v1[i] * v1[i];
  const double tau1 = 2.0 / blk_sum(t, red);
  double tau2 = 0.0, c12 = 0.0;
  if (k1 == 2) {
    // y = H1 u2; v2 acts on rows 1..m-1
    double d = 0.0;
    for (int i = tid; i < m; i += nt) d += v1[i] * (double)U[(int64_t)i * m + 1];
    d = blk_sum(d, red);
    for (int i = tid; i < m; i += nt) v2[i] = (i == 0) ? 0.0 : (double)U[(int64_t)i * m + 1] - tau1 * d * v1[i];
    __syncthreads();
    double nn = 0.0;
    for (int i = 1 + tid; i < m; i += nt) nn += v2[i] * v2[i];
    const double nrm = sqrt(blk_sum(nn, red));
    const double s2 = (m > 1 && v2[1] < 0.0) ? -1.0 : 1.0;
    if (tid == 0 && m > 1) v2[1] += s2 * nrm;
    __syncthreads();
    double vv = 0.0, cv = 0.0;
    for (int i = tid; i < m; i += nt) {
      vv += v2[i] * v2[i];
      cv += v1[i] * v2[i];
    }
    vv = blk_sum(vv, red);
    c12 = blk_sum(cv, red);
    tau2 = vv > 0.0 ? 2.0 / vv : 0.0;
  } else {
    for (int i = tid; i < m; i += nt) v2[i] = 0.0;
    __syncthreads();
  }
  // Q[i][j] = d_ij - tau2 v2_i v2_j - tau1 v1_i (v1_j - tau2 v2_j c12), columns j >= k1
  for (int64_t q = tid; q < (int64_t)m * (m - k1); q += nt) {
    const int i = (int)(q / (m - k1)), j = k1 + (int)(q % (m - k1));
    const double val = (i == j ? 1.0 : 0.0) - tau2 * v2[i] * v2[j] - tau1 * v1[i] * (v1[j] - tau2 * v2[j] * c12);
    U[(int64_t)i * m + j] = (T)val;
  }
  __syncthreads();
}

}  // namespace hs
