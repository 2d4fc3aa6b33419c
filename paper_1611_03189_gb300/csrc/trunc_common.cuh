// Device helpers shared by the two truncation kernels (Sec. 6, GC basis).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hs_internal.h"

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

// U_1 of the GC family in U's columns 0 .. k1-1 (row-major, ld m); returns k1
// (<= 2 np <= kMaxK1).  The candidates are the np columns of phi_s, then the
// np columns of a = A_sw phi_w (phi, a: m x np row-major).
//   Sec. 6 (proj false): modified Gram-Schmidt with one re-orthogonalisation
//     in that order; a candidate is kept when its remainder exceeds 1e-12 of
//     its norm.
//   Appendix B, first-order one-sided projection (proj true): the same MGS
//     factors C = [phi_s, a] = Q R (R: k1 x 2 np in sR, ld 2 kMaxPhi); one
//     thread orthogonalises the columns of R by one-sided Jacobi (FP64), whose
//     norms are the singular values of C and whose normalised directions W its
//     left singular vectors in the basis Q; U_1 = Q W keeps the ones with
//     sigma_i > max(eps1, 1e-12) sigma_1, by descending sigma.
// v: m doubles of scratch (each thread uses its own rows); red: 33 doubles;
// sR: kMaxK1 * 2 kMaxPhi and sW: kMaxK1 * kMaxK1 doubles, s_k one int, all
// shared memory.
template <typename T>
__device__ __noinline__ int gc_basis_dev(const T *phi, const T *a, int np, int m, bool proj, double eps1, T *U, double *v,
                            double *red, double *sR, double *sW, int *s_k) {
  const int tid = threadIdx.x, nt = blockDim.x;
  constexpr int ldr = 2 * kMaxPhi;
  const int nc = 2 * np;
  if (proj && tid == 0)
    for (int q = 0; q < kMaxK1 * ldr; ++q) sR[q] = 0.0;
  int k1 = 0;
  for (int c = 0; c < nc; ++c) {
    const T *src = c < np ? phi + c : a + (c - np);
    double s = 0.0;
    for (int i = tid; i < m; i += nt) {
      const double x = (double)src[(size_t)i * np];
      v[i] = x;
      s += x * x;
    }
    const double ncn = sqrt(blk_sum(s, red));
    if (ncn == 0.0) continue;
    for (int pass = 0; pass < (k1 > 0 ? 2 : 0); ++pass)
      for (int l = 0; l < k1; ++l) {
        double d = 0.0;
        for (int i = tid; i < m; i += nt) d += (double)U[(int64_t)i * m + l] * v[i];
        d = blk_sum(d, red);
        for (int i = tid; i < m; i += nt) v[i] -= d * (double)U[(int64_t)i * m + l];
        if (proj && tid == 0) sR[l * ldr + c] += d;
      }
    double sv = 0.0;
    for (int i = tid; i < m; i += nt) sv += v[i] * v[i];
    const double nv = sqrt(blk_sum(sv, red));
    if (nv > 1e-12 * ncn && k1 < kMaxK1 && k1 < m) {
      for (int i = tid; i < m; i += nt) U[(int64_t)i * m + k1] = (T)(v[i] / nv);
      if (proj && tid == 0) sR[k1 * ldr + c] = nv;
      ++k1;
    }
  }
  __syncthreads();
  if (!proj || k1 == 0) return k1;
  if (tid == 0) {
    // one-sided Jacobi on the columns of R (k1 x nc)
    for (int sweep = 0; sweep < 40; ++sweep) {
      bool rot = false;
      for (int p = 0; p < nc; ++p)
        for (int q = p + 1; q < nc; ++q) {
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int r = 0; r < k1; ++r) {
            const double x = sR[r * ldr + p], y = sR[r * ldr + q];
            al += x * x;
            be += y * y;
            ga += x * y;
          }
          if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
          rot = true;
          const double zeta = (be - al) / (2.0 * ga);
          const double tt =
              fabs(zeta) > 1e100 ? 0.5 / zeta : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
          for (int r = 0; r < k1; ++r) {
            const double x = sR[r * ldr + p], y = sR[r * ldr + q];
            sR[r * ldr + p] = cs * x - sn * y;
            sR[r * ldr + q] = sn * x + cs * y;
          }
        }
      if (!rot) break;
    }
    double sig[2 * kMaxPhi];
    double smax = 0.0;
    for (int p = 0; p < nc; ++p) {
      double s = 0.0;
      for (int r = 0; r < k1; ++r) s += sR[r * ldr + p] * sR[r * ldr + p];
      sig[p] = sqrt(s);
      smax = fmax(smax, sig[p]);
    }
    const double thr = fmax(eps1, 1e-12) * smax;
    int kk = 0;
    unsigned used = 0u;
    while (kk < k1) {
      int best = -1;
      for (int p = 0; p < nc; ++p)
        if (!((used >> p) & 1u) && sig[p] > thr && (best < 0 || sig[p] > sig[best])) best = p;
      if (best < 0) break;
      used |= 1u << best;
      for (int r = 0; r < k1; ++r) sW[r * kMaxK1 + kk] = sR[r * ldr + best] / sig[best];
      ++kk;
    }
    *s_k = kk;
  }
  __syncthreads();
  const int kk = *s_k;
  // U_1 = Q W, row by row (Q in U's first k1 columns)
  for (int i = tid; i < m; i += nt) {
    double q[kMaxK1];
    for (int l = 0; l < kMaxK1; ++l) q[l] = l < k1 ? (double)U[(int64_t)i * m + l] : 0.0;
    for (int j = 0; j < kk; ++j) {
      double s = 0.0;
      for (int l = 0; l < k1; ++l) s += q[l] * sW[l * kMaxK1 + j];
      U[(int64_t)i * m + j] = (T)s;
    }
  }
  __syncthreads();
  return kk;
}

// gc_complete for any k1 <= kMaxK1: the columns k1 .. m-1 of Q = H_0 ... H_{k1-1}
// from the Householder QR of U_1 (U row-major, ld m).  H_j = I - tau_j v_j v_j^T
// zeroes column j of H_{j-1} ... H_0 U_1 below row j.  Column c of Q is
// e_c - sum_l alpha_l v_l with alpha_l = tau_l (v_l[c] - sum_{l' > l}
// alpha_l' v_l.v_l'), one thread per column.
// vh: k1 m doubles of scratch; sW: kMaxK1 * kMaxK1 + kMaxK1 shared doubles.
template <typename T>
__device__ __noinline__ void gc_complete_n(T *U, int m, int k1, double *vh, double *sW, double *red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  double *tau = sW + kMaxK1 * kMaxK1;
  for (int j = 0; j < k1; ++j) {
    double *vj = vh + (size_t)j * m;
    for (int i = tid; i < m; i += nt) vj[i] = (double)U[(int64_t)i * m + j];
    for (int l = 0; l < j; ++l) {
      const double *vl = vh + (size_t)l * m;
      double d = 0.0;
      for (int i = tid; i < m; i += nt) d += vl[i] * vj[i];
      d = blk_sum(d, red) * tau[l];
      for (int i = tid; i < m; i += nt) vj[i] -= d * vl[i];
    }
    double s = 0.0;
    for (int i = tid; i < m; i += nt)
      if (i >= j) s += vj[i] * vj[i];
    const double sig = sqrt(blk_sum(s, red));   // synchronises: vj[j] is visible
    const double alpha = vj[j];
    const double beta = alpha >= 0.0 ? sig : -sig;
    __syncthreads();
    for (int i = tid; i < m; i += nt) {
      if (i < j) vj[i] = 0.0;
      if (i == j) vj[i] = alpha + beta;
    }
    if (tid == 0) tau[j] = sig > 0.0 ? 1.0 / (sig * (sig + fabs(alpha))) : 0.0;
    __syncthreads();
  }
  for (int a = 0; a < k1; ++a)
    for (int b = a; b < k1; ++b) {
      double d = 0.0;
      for (int i = tid; i < m; i += nt) d += vh[(size_t)a * m + i] * vh[(size_t)b * m + i];
      d = blk_sum(d, red);
      if (tid == 0) {
        sW[a * kMaxK1 + b] = d;
        sW[b * kMaxK1 + a] = d;
      }
    }
  __syncthreads();
  for (int c = k1 + tid; c < m; c += nt) {
    double al[kMaxK1];
    for (int l = kMaxK1 - 1; l >= 0; --l) {
      if (l >= k1) {
        al[l] = 0.0;
        continue;
      }
      double x = vh[(size_t)l * m + c];
      for (int l2 = l + 1; l2 < k1; ++l2) x -= al[l2] * sW[l * kMaxK1 + l2];
      al[l] = tau[l] * x;
    }
    for (int i = 0; i < m; ++i) {
      double q = (i == c) ? 1.0 : 0.0;
      for (int l = 0; l < k1; ++l) q -= al[l] * vh[(size_t)l * m + i];
      U[(int64_t)i * m + c] = (T)q;
    }
  }
  __syncthreads();
}

}  // namespace hs
