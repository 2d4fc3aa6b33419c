// Truncation of large super nodes (m above the shared-memory Jacobi limit):
// symmetric eigen-decomposition of the Gram matrix by Householder
// tridiagonalisation, Sturm-sequence bisection and inverse iteration.
//
// One CTA per super node: 256 threads for m <= 128, 1024 above (a function of
// m alone, so a node gets the same arithmetic in any batch):
//   1. GC basis U_1 = orth[phi_s, A_sw phi_w] (Sec. 6; Appendix B: its dominant
//      left singular vectors), as in the Jacobi path.
//   2. ||A_sw||_2^2 = lambda_max(G).  LoRaSp: top eigenvalue of T below.  GC:
//      G = J + (rank <= 2 k1 terms in span{U_1, G U_1}), so lambda_max(G) follows
//      from the tridiagonal T of J by a warp multisection on the Haynsworth
//      inertia count of the low-rank correction (no second tridiagonalisation).
//   3. J = G (LoRaSp), (I - U1 U1^T) G (I - U1 U1^T) (GC) or I - U1 U1^T (GC,
//      eps = 0).  Tridiagonalise J = Q T Q^T; k2 = #{lambda(T) > thr} by one
//      Sturm count (FP64), thr = eps^2 lambda_max(G) (Sec. 3.2, strict).
//   4. The k2 largest eigenvalues of T by bisection (FP64), their eigenvectors
//      by inverse iteration on T (tridiagonal LU with partial pivoting, three
//      steps, modified Gram-Schmidt inside clusters of eigenvalues closer than
//      10 u ||T||), then U_2 = Q Y by the stored Householder reflectors.
// The host re-orthonormalises [U_1, U_2] afterwards (CholQR2), which keeps its
// span.  The tridiagonalisation works in global memory until the trailing
// block fits in shared memory, then finishes there.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "hs_internal.h"
#include "trunc_common.cuh"

namespace hs {

namespace {


__device__ double bsum(double v, double *red) {
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

// Block-wide sum in T (red: 33 T of shared memory); every thread gets the total.
// Reductions inside the per-step loops stay in the factor precision: on this
// GPU FP64 instructions issue at a small fraction of the FP32 rate.
template <typename T>
__device__ T bsum_t(T v, T *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    T s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : T(0);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  const T r = red[32];
  __syncthreads();
  return r;
}

// Shared scratch of the large-truncation kernel (sizes in elements).
template <typename T>
struct Big {
  double *d, *e, *pw, *red;   // tridiagonal in FP64 (rank decision), work vector
  T *dt, *et, *lam;           // tridiagonal and selected eigenvalues in T
  T *v;          // Householder vector of the current step
  T *wt;         // p, then w = p - K v of the current step
  T *redt;       // 33 T of reduction scratch
  T *tau;        // reflector coefficients
  T *tile;       // trailing block once it fits in shared memory
  int tile_cap;  // max trailing size held in shared memory
};

// Householder tridiagonalisation of the symmetric m x m matrix A (global, ld m,
// full storage; destroyed).  On exit d (diagonal) and e (sub-diagonal) hold
// T, reflector k is I - tau[k] v v^T with v[0] = 1 on rows k+1.. and v[1..]
// stored in A[k][k+2..].
template <typename T>
__device__ void tridiag(T *A, int m, Big<T> &b) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  // element (i, j) of the working matrix is W[(i - off) * ld + (j - off)]
  T *W = A;
  int off = 0, ld = m;
  bool in_smem = false;
  for (int k = 0; k + 2 < m; ++k) {
    const int n1 = m - k - 1;
    if (!in_smem && n1 + 1 <= b.tile_cap) {
      // move the trailing block rows/cols k.. into shared memory
      const int ls = m - k;
      for (int64_t q = tid; q < (int64_t)ls * ls; q += nt) {
        const int i = (int)(q / ls), j = (int)(q % ls);
        b.tile[q] = A[(int64_t)(k + i) * m + k + j];
      }
      W = b.tile;
      off = k;
      ld = ls;
      in_smem = true;
      __syncthreads();
    }
    const T *rowk = W + (int64_t)(k - off) * ld + (k - off);   // rowk[j] = A[k][k + j]
    T s2t = T(0);
    for (int i = 1 + tid; i <= n1; i += nt) s2t = fma(rowk[i], rowk[i], s2t);
    const double xn2 = (double)bsum_t<T>(s2t, b.redt);
    const double alpha = (double)rowk[1];
    const double sig = xn2 - alpha * alpha;
    double tau = 0.0, beta = alpha, scale = 0.0;
    if (sig > 0.0) {
      beta = -copysign(sqrt(xn2), alpha);
      tau = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    const T scale_t = (T)scale, tau_t = (T)tau;
    for (int i = tid; i < n1; i += nt) {
      const T vi = (i == 0) ? T(1) : rowk[1 + i] * scale_t;
      b.v[i] = vi;
      if (i >= 1) A[(int64_t)k * m + k + 1 + i] = vi;  // keep the reflector in global row k
    }
    if (tid == 0) {
      b.d[k] = (double)rowk[0];
      b.e[k] = beta;
      b.tau[k] = tau_t;
    }
    __syncthreads();
    if (tau != 0.0 && in_smem) {
      // trailing block in shared memory: by its symmetry p_i = tau sum_j
      // A22_ji v_j and the rank-2 update are column walks, thread i on column
      // i, consecutive threads on consecutive words (no per-row reductions)
      T *A22 = W + (int64_t)(k + 1 - off) * ld + (k + 1 - off);
      T pvt = T(0);
      for (int i = tid; i < n1; i += nt) {
        const T *col = A22 + i;
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        int j = 0;
        for (; j + 3 < n1; j += 4) {
          a0 = fma(col[(int64_t)j * ld], b.v[j], a0);
          a1 = fma(col[(int64_t)(j + 1) * ld], b.v[j + 1], a1);
          a2 = fma(col[(int64_t)(j + 2) * ld], b.v[j + 2], a2);
          a3 = fma(col[(int64_t)(j + 3) * ld], b.v[j + 3], a3);
        }
        for (; j < n1; ++j) a0 = fma(col[(int64_t)j * ld], b.v[j], a0);
        const T pi = tau_t * ((a0 + a1) + (a2 + a3));
        b.wt[i] = pi;
        pvt = fma(pi, b.v[i], pvt);
      }
      const T K = T(0.5) * tau_t * bsum_t<T>(pvt, b.redt);
      for (int i = tid; i < n1; i += nt) b.wt[i] = fma(-K, b.v[i], b.wt[i]);  // w
      __syncthreads();
      for (int i = tid; i < n1; i += nt) {
        T *col = A22 + i;
        const T vi = b.v[i], wi = b.wt[i];
        for (int j = 0; j < n1; ++j) {
          T &a = col[(int64_t)j * ld];
          a = fma(-b.v[j], wi, fma(-b.wt[j], vi, a));
        }
      }
      __syncthreads();
    } else if (tau != 0.0) {
      T *A22 = W + (int64_t)(k + 1 - off) * ld + (k + 1 - off);
      // p = tau * A22 v, one warp per row, four independent partial sums
      for (int i = warp; i < n1; i += nw) {
        const T *row = A22 + (int64_t)i * ld;
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        int j = lane;
        for (; j + 96 < n1; j += 128) {
          a0 = fma(row[j], b.v[j], a0);
          a1 = fma(row[j + 32], b.v[j + 32], a1);
          a2 = fma(row[j + 64], b.v[j + 64], a2);
          a3 = fma(row[j + 96], b.v[j + 96], a3);
        }
        for (; j < n1; j += 32) a0 = fma(row[j], b.v[j], a0);
        T acc = (a0 + a1) + (a2 + a3);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) b.wt[i] = tau_t * acc;
      }
      __syncthreads();
      T pvt = T(0);
      for (int i = tid; i < n1; i += nt) pvt = fma(b.wt[i], b.v[i], pvt);
      const T K = T(0.5) * tau_t * bsum_t<T>(pvt, b.redt);
      for (int i = tid; i < n1; i += nt) b.wt[i] = fma(-K, b.v[i], b.wt[i]);  // w
      __syncthreads();
      // A22 -= v w^T + w v^T, one warp per row
      for (int i = warp; i < n1; i += nw) {
        T *row = A22 + (int64_t)i * ld;
        const T vi = b.v[i], wi = b.wt[i];
#pragma unroll 4
        for (int j = lane; j < n1; j += 32) row[j] = fma(-vi, b.wt[j], fma(-wi, b.v[j], row[j]));
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    auto at = [&](int i, int j) { return (double)W[(int64_t)(i - off) * ld + (j - off)]; };
    if (m >= 2) {
      b.d[m - 2] = at(m - 2, m - 2);
      b.e[m - 2] = at(m - 1, m - 2);
      b.tau[m - 2] = T(0);
    }
    b.d[m - 1] = at(m - 1, m - 1);
    b.e[m - 1] = 0.0;
    b.tau[m - 1] = T(0);
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    b.dt[i] = (T)b.d[i];
    b.et[i] = (T)b.e[i];
  }
  __syncthreads();
}

template <typename R>
__device__ __forceinline__ R unit_round();
template <>
__device__ __forceinline__ double unit_round<double>() { return 2.220446049250313e-16; }
template <>
__device__ __forceinline__ float unit_round<float>() { return 1.1920929e-07f; }

// number of eigenvalues of the tridiagonal (d, e) below sigma (Sturm sequence)
template <typename R>
__device__ int sturm_below(const R *d, const R *e, int m, R sigma, R pivmin) {
  int c = 0;
  R q = d[0] - sigma;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < R(0)) ++c;
  for (int i = 1; i < m; ++i) {
    q = d[i] - sigma - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < R(0)) ++c;
  }
  return c;
}

template <typename R>
struct Gersh {
  R lo, hi, pivmin, tnorm;
};

// Gershgorin interval of the tridiagonal (every thread computes the same)
template <typename R>
__device__ Gersh<R> gershgorin(const R *d, const R *e, int m) {
  Gersh<R> g;
  R lo = d[0], hi = d[0], emax = R(0);
  for (int i = 0; i < m; ++i) {
    const R r = (i > 0 ? fabs(e[i - 1]) : R(0)) + (i + 1 < m ? fabs(e[i]) : R(0));
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    emax = fmax(emax, e[i] * e[i]);
  }
  g.tnorm = fmax(fabs(lo), fabs(hi));
  const R pad = unit_round<R>() * g.tnorm * R(2 * m) + R(1e-30);
  g.lo = lo - pad;
  g.hi = hi + pad;
  g.pivmin = fmax(R(1e-30) * fmax(R(1), emax), R(1e-35));
  return g;
}

// idx-th smallest eigenvalue (0-based) by bisection
template <typename R>
__device__ R bisect_eig(const R *d, const R *e, int m, int idx, const Gersh<R> &g) {
  R lo = g.lo, hi = g.hi;
  const R tol = R(4) * unit_round<R>() * g.tnorm;
  for (int it = 0; it < 200 && hi - lo > tol; ++it) {
    const R mid = R(0.5) * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_below<R>(d, e, m, mid, g.pivmin) <= idx)
      lo = mid;
    else
      hi = mid;
  }
  return R(0.5) * (lo + hi);
}

// idx-th smallest eigenvalue by multisection with one warp (33 sub-intervals per
// round; called by all 32 lanes of a warp, every lane returns the result)
template <typename R>
__device__ R multisect_eig(const R *d, const R *e, int m, int idx, const Gersh<R> &g) {
  const int lane = threadIdx.x & 31;
  R lo = g.lo, hi = g.hi;
  const R tol = R(4) * unit_round<R>() * g.tnorm;
  for (int round = 0; round < 40 && hi - lo > tol; ++round) {
    const R sig = lo + (hi - lo) * R(lane + 1) / R(33);
    const bool below = sturm_below<R>(d, e, m, sig, g.pivmin) <= idx;   // eigenvalue idx >= sig
    const unsigned mask = __ballot_sync(0xffffffffu, below);
    const int l = mask ? 31 - __clz(mask) : -1;
    const R nlo = l >= 0 ? lo + (hi - lo) * R(l + 1) / R(33) : lo;
    const R nhi = lo + (hi - lo) * R(l + 2) / R(33);
    if (!(nhi > nlo)) break;
    lo = nlo;
    hi = nhi;
  }
  return R(0.5) * (lo + hi);
}

__device__ __forceinline__ float hash_unit(uint32_t a, uint32_t b) {
  uint32_t x = a * 0x9E3779B9u ^ (b + 0x7F4A7C15u);
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return (float)(x >> 8) * (2.0f / 16777216.0f) - 1.0f;
}

// Inverse iteration for eigenvalue lam of the tridiagonal (d, e): LU of
// T - lam I with partial pivoting (rows i, i+1 interchanged when the
// sub-diagonal dominates), three solves from a fixed pseudo-random start,
// modified Gram-Schmidt against `nprev` previous vectors of the same cluster
// of close eigenvalues.  y: output (length m); lu: 4 m of scratch; flags: m
// bytes; element i of y, lu's four arrays and flags sits at index i * st (st >
// 1 interleaves the scratch of several threads, so that their accesses to
// global memory coalesce).
template <typename R>
__device__ void inverse_iteration(const R *d, const R *e, int m, R lam, R tnorm, R *y, const R *prev,
                                  int nprev, R *lu, unsigned char *flags, uint32_t seed, int st = 1) {
  const size_t sm = (size_t)m * st;
  R *u0 = lu, *u1 = lu + sm, *u2 = lu + 2 * sm, *l = lu + 3 * sm;
  auto I = [st](int i) { return (size_t)i * st; };
  const R small = unit_round<R>() * tnorm + R(1e-30);
  R a = d[0] - lam, c = (m > 1) ? e[0] : R(0);
  for (int i = 0; i + 1 < m; ++i) {
    const R bsub = e[i];
    const R an = d[i + 1] - lam;
    const R cn = (i + 2 < m) ? e[i + 1] : R(0);
    if (fabs(a) >= fabs(bsub)) {
      const R piv = (a == R(0)) ? small : a;
      const R mult = bsub / piv;
      u0[I(i)] = piv;
      u1[I(i)] = c;
      u2[I(i)] = R(0);
      l[I(i)] = mult;
      flags[I(i)] = 0;
      a = an - mult * c;
      c = cn;
    } else {
      const R mult = a / bsub;
      u0[I(i)] = bsub;
      u1[I(i)] = an;
      u2[I(i)] = cn;
      l[I(i)] = mult;
      flags[I(i)] = 1;
      a = c - mult * an;
      c = -mult * cn;
    }
  }
  u0[I(m - 1)] = a;
  for (int i = 0; i < m; ++i)
    if (fabs(u0[I(i)]) < small) u0[I(i)] = copysign(small, u0[I(i)]);
  for (int i = 0; i < m; ++i) y[I(i)] = (R)hash_unit(seed, (uint32_t)i);
  for (int it = 0; it < 3; ++it) {
    for (int i = 0; i + 1 < m; ++i) {
      if (flags[I(i)]) {
        const R t = y[I(i)];
        y[I(i)] = y[I(i + 1)];
        y[I(i + 1)] = t - l[I(i)] * y[I(i)];
      } else {
        y[I(i + 1)] -= l[I(i)] * y[I(i)];
      }
    }
    for (int i = m - 1; i >= 0; --i) {
      R s = y[I(i)];
      if (i + 1 < m) s -= u1[I(i)] * y[I(i + 1)];
      if (i + 2 < m) s -= u2[I(i)] * y[I(i + 2)];
      y[I(i)] = s / u0[I(i)];
    }
    for (int pass = 0; pass < 2; ++pass)
      for (int p = 0; p < nprev; ++p) {
        const R *q = prev + (size_t)p * m;
        R dot = R(0);
        for (int i = 0; i < m; ++i) dot += q[i] * y[I(i)];
        for (int i = 0; i < m; ++i) y[I(i)] -= dot * q[i];
      }
    // normalise, scaling by the largest entry first to keep the sum in range
    R big = R(0);
    for (int i = 0; i < m; ++i) big = fmax(big, fabs(y[I(i)]));
    const R sc = big > R(0) ? R(1) / big : R(0);
    R nrm = R(0);
    for (int i = 0; i < m; ++i) nrm += (y[I(i)] * sc) * (y[I(i)] * sc);
    nrm = sqrt(nrm);
    const R inv = nrm > R(0) ? sc / nrm : R(0);
    for (int i = 0; i < m; ++i) y[I(i)] *= inv;
  }
}


// Eigenvalues of G above sigma, for sigma > lambda_max(T), where Q^T G Q = T + Z M Z^T,
// T = tridiag(d, e) (the tridiagonal of the projected Gram J = P G P), Z = Q^T [U_1, G U_1]
// (m x 2 k1, column j at Z + j*m) and M = [[-C, I], [I, 0]], C = U_1^T G U_1 (k1 x k1,
// ld kMaxK1).  NZ >= 2 k1 bounds the small dense parts held per thread.
// Haynsworth inertia of [[T - sigma I, Z], [Z^T, -M^-1]] gives
//   #eig(G) > sigma = n_+(-M^-1 - Z^T (T - sigma I)^-1 Z) - n_+(-M^-1),  n_+(-M^-1) = k1,
// since T - sigma I is negative definite.  With T - sigma I = L D L^T (L unit
// lower bidiagonal) and W = L^-1 Z, Z^T (T - sigma I)^-1 Z = W^T D^-1 W: one
// forward sweep with register accumulators, no storage.
template <typename R, int NZ>
__device__ int count_above_lowrank(const R *d, const R *e, int m, const R *Z, int k1, const R *C, R sigma) {
  const int nz = 2 * k1;
  R w[NZ];
  R g[NZ][NZ];
  for (int a = 0; a < NZ; ++a) {
    w[a] = R(0);
    for (int b2 = 0; b2 < NZ; ++b2) g[a][b2] = R(0);
  }
  R dd = R(1), lprev = R(0);
  for (int i = 0; i < m; ++i) {
    dd = (i == 0) ? d[0] - sigma : d[i] - sigma - lprev * e[i - 1];
    const R inv = R(1) / dd;
#pragma unroll
    for (int a = 0; a < NZ; ++a)
      if (a < nz) w[a] = Z[(size_t)a * m + i] - (i == 0 ? R(0) : lprev * w[a]);
#pragma unroll
    for (int a = 0; a < NZ; ++a)
#pragma unroll
      for (int b2 = 0; b2 < NZ; ++b2)
        if (a < nz && b2 <= a) g[a][b2] = fma(w[a] * inv, w[b2], g[a][b2]);
    lprev = (i + 1 < m) ? e[i] * inv : R(0);
  }
  R S[NZ][NZ];
  for (int a = 0; a < nz; ++a)
    for (int b = 0; b < nz; ++b) {
      R v = R(0);
      if (a < k1 && b >= k1 && b - k1 == a) v = R(-1);
      if (b < k1 && a >= k1 && a - k1 == b) v = R(-1);
      if (a >= k1 && b >= k1) v = -C[(a - k1) * kMaxK1 + (b - k1)];
      S[a][b] = v - (b <= a ? g[a][b] : g[b][a]);
    }
  // symmetrise and count positive eigenvalues by cyclic Jacobi on the small matrix
  for (int a = 0; a < nz; ++a)
    for (int b = a + 1; b < nz; ++b) {
      const R v = R(0.5) * (S[a][b] + S[b][a]);
      S[a][b] = v;
      S[b][a] = v;
    }
  for (int sweep = 0; sweep < (NZ > 4 ? 16 : 12); ++sweep)
    for (int p = 0; p < nz; ++p)
      for (int q = p + 1; q < nz; ++q) {
        const R apq = S[p][q];
        if (fabs(apq) <= R(1e-30)) continue;
        const R th = (S[q][q] - S[p][p]) / (R(2) * apq);
        R tt = R(1) / (fabs(th) + sqrt(R(1) + th * th));
        if (th < R(0)) tt = -tt;
        const R c = R(1) / sqrt(R(1) + tt * tt), sn = tt * c;
        for (int k = 0; k < nz; ++k) {
          const R skp = S[k][p], skq = S[k][q];
          S[k][p] = c * skp - sn * skq;
          S[k][q] = sn * skp + c * skq;
        }
        for (int k = 0; k < nz; ++k) {
          const R spk = S[p][k], sqk = S[q][k];
          S[p][k] = c * spk - sn * sqk;
          S[q][k] = sn * spk + c * sqk;
        }
      }
  int pos = 0;
  for (int a = 0; a < nz; ++a)
    if (S[a][a] > R(0)) ++pos;
  return pos - k1;
}

// J = G - U1 X^T - X U1^T + U1 c U1^T (the Gram matrix projected off span U_1),
// X = G U1 in Y's columns (column a at Y + a m), c in shared memory (ld
// kMaxK1); one warp per row.  KB >= k1 sizes the per-row registers.
template <typename T, int KB>
__device__ void build_projected_gram(const T *G, const T *U, const T *Y, const T *s_c, T *A, int m, int k1) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < m; i += nw) {
    T ui[KB], xi[KB], cu[KB];
#pragma unroll
    for (int a = 0; a < KB; ++a) {
      ui[a] = a < k1 ? U[(int64_t)i * m + a] : T(0);
      xi[a] = a < k1 ? Y[(size_t)a * m + i] : T(0);
    }
#pragma unroll
    for (int bb = 0; bb < KB; ++bb) {
      T su = T(0);
#pragma unroll
      for (int a = 0; a < KB; ++a)
        if (a < k1) su = fma(ui[a], s_c[a * kMaxK1 + bb], su);
      cu[bb] = su;
    }
    for (int j = lane; j < m; j += 32) {
      T v = G[(int64_t)i * m + j];
#pragma unroll
      for (int a = 0; a < KB; ++a)
        if (a < k1) {
          const T uj = U[(int64_t)j * m + a];
          v = fma(-ui[a], Y[(size_t)a * m + j], fma(-xi[a], uj, v));
          v = fma(cu[a], uj, v);
        }
      A[(int64_t)i * m + j] = v;
    }
  }
}

// k1 > 2 (several preserved vectors) in a call of its own, off the register
// allocation of the one-vector path
template <typename T>
__device__ __noinline__ void build_projected_gram_wide(const T *G, const T *U, const T *Y, const T *s_c, T *A,
                                                       int m, int k1) {
  build_projected_gram<T, kMaxK1>(G, U, Y, s_c, A, m, k1);
}

// The count for k1 > 2 (several preserved vectors) in a call of its own, so
// that its 16 x 16 local arrays stay out of the kernel's register allocation.
template <typename R>
__device__ __noinline__ int count_above_lowrank_wide(const R *d, const R *e, int m, const R *Z, int k1,
                                                     const R *C, R sigma) {
  return count_above_lowrank<R, 2 * kMaxK1>(d, e, m, Z, k1, C, sigma);
}

// mode: TB_FULL does all steps in this CTA.  The multi-CTA path for very large
// nodes splits it: TB_PREP stops before the tridiagonalisation (A = J, Z saved,
// k1 and c stored in SC); the step kernels tridiagonalise; TB_POST takes d, e
// and the reflectors from global memory and stops after the eigenvectors of T
// (Y, k2 in SC) -- the reflector kernels do the two products with Q.
enum { TB_FULL = 0, TB_PREP = 1, TB_POST = 2 };

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_trunc_big(const TruncTask<T> *__restrict__ tasks, int *__restrict__ kout,
                                                 int variant, int tile_cap, int vec_smem, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[33];
  __shared__ int s_k2;
  __shared__ double s_gR[kMaxK1 * 2 * kMaxPhi], s_gW[kMaxK1 * kMaxK1 + kMaxK1];
  __shared__ int s_gk;
  __shared__ T s_c[kMaxK1 * kMaxK1];   // c = U1^T G U1, ld kMaxK1
  const TruncTask<T> t = tasks[blockIdx.x];
  const double eps = t.eps;
  const int m = t.m;
  const int tid = threadIdx.x, nt = blockDim.x;
  // global work, all T: A (m^2), Y (m^2), LU (4 m^2), LS (164 m: Z = Q^T [U1, X] in
  // 4 m, then per-thread inverse-iteration slots when the shared tile is too
  // small); then flags (m^2 bytes); then the per-node vectors when they do not
  // fit in shared memory (vec_smem == 0)
  const BigLayout<T> L = big_layout<T>(t.work, m);
  T *A = L.A;
  T *Y = L.Y;
  T *LU = L.LU;
  T *LS = L.LS;
  unsigned char *FL = L.FL;
  unsigned char *VG = L.VG;
  // vector layout (shared memory, or global at VG), then the shared tile
  Big<T> b;
  unsigned char *p = vec_smem ? smem_raw : VG;
  b.d = (double *)p;
  p += sizeof(double) * m;
  b.e = (double *)p;
  p += sizeof(double) * m;
  b.pw = (double *)p;
  p += sizeof(double) * m;
  const int me = (m + 1) & ~1;
  b.dt = (T *)p;
  p += sizeof(T) * me;
  b.et = (T *)p;
  p += sizeof(T) * me;
  b.lam = (T *)p;
  p += sizeof(T) * me;
  b.v = (T *)p;
  p += sizeof(T) * me;
  b.tau = (T *)p;
  p += sizeof(T) * me;
  b.wt = (T *)p;
  p += sizeof(T) * me;
  b.redt = (T *)p;
  p += sizeof(T) * 34;
  p = (unsigned char *)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  b.tile = (T *)(vec_smem ? p : smem_raw);
  b.tile_cap = tile_cap;
  b.red = red;
  if (m == 0) {
    if (tid == 0) kout[t.k_idx] = 0;
    return;
  }
  // ---- GC basis U_1 (same rule as the Jacobi path; scratch b.pw, m doubles)
  int k1 = 0;
  if (variant != HS_LORASP)
    k1 = gc_basis_dev<T>(t.phi, t.a, t.np, m, variant == HS_GC_PROJ, t.eps1, t.U, b.pw, red, s_gR, s_gW, &s_gk);
  const bool gc = variant != HS_LORASP;
  if (gc && eps == 0.0) {
    // no truncation: complete the GC basis to all of R^m (Householder QR of
    // U_1; scratch k1 m doubles in Y and LU, 5 m^2 T)
    // (nothing to complete when U_1 already spans R^m)
    if (k1 < m) {
      if (k1 <= 2)
        gc_complete<T>(t.U, m, k1, (double *)Y, red);
      else
        gc_complete_n<T>(t.U, m, k1, (double *)Y, s_gW, red);
    }
    if (tid == 0) kout[t.k_idx] = m;
    return;
  }
  // ---- lambda_max(G) (GC) follows from the tridiagonal of the projected Gram below
  double lmax = 0.0;
  // ---- J
  if (mode == TB_POST) {
    // J, Z and c were made by TB_PREP; Z is already Q^T [U1, X]
    for (int q = tid; q < kMaxK1 * kMaxK1; q += nt) s_c[q] = (T)L.sc_c[q];
    __syncthreads();
  } else if (!gc) {
    for (int64_t q = tid; q < (int64_t)m * m; q += nt) A[q] = t.G[q];
  } else if (eps > 0.0) {
    // X = G U1 in Y's first columns, c = U1^T X; one warp per row of G
    {
      const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
      for (int i = warp; i < m; i += nw)
        for (int a = 0; a < k1; ++a) {
          T s = T(0);
          for (int j = lane; j < m; j += 32) s = fma(t.G[(int64_t)i * m + j], t.U[(int64_t)j * m + a], s);
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (lane == 0) Y[(size_t)a * m + i] = s;
        }
    }
    __syncthreads();
    for (int q = tid; q < kMaxK1 * kMaxK1; q += nt) s_c[q] = T(0);
    __syncthreads();
    for (int a = 0; a < k1; ++a)
      for (int bb = 0; bb < k1; ++bb) {
        T s = T(0);
        for (int i = tid; i < m; i += nt) s = fma(t.U[(int64_t)i * m + a], Y[(size_t)bb * m + i], s);
        const T cab = bsum_t<T>(s, b.redt);
        if (tid == 0) s_c[a * kMaxK1 + bb] = cab;
      }
    __syncthreads();
    // J = G - U1 X^T - X U1^T + U1 c U1^T, one warp per row
    if (k1 <= 2)
      build_projected_gram<T, 2>(t.G, t.U, Y, s_c, A, m, k1);
    else
      build_projected_gram_wide<T>(t.G, t.U, Y, s_c, A, m, k1);
  } else {
    for (int64_t q = tid; q < (int64_t)m * m; q += nt) {
      const int i = (int)(q / m), j = (int)(q % m);
      double v = (i == j) ? 1.0 : 0.0;
      for (int a = 0; a < k1; ++a) v -= (double)t.U[(int64_t)i * m + a] * (double)t.U[(int64_t)j * m + a];
      A[q] = (T)v;
    }
  }
  __syncthreads();
  // X = G U1 (Y columns 0..k1-1) is needed again below: move it next to U1 first
  T *Zb = LS;  // Z = Q^T [U1, X], 2 k1 <= 2 kMaxK1 columns of m
  if (gc && eps > 0.0 && mode != TB_POST) {
    for (int64_t q = tid; q < (int64_t)m * k1; q += nt) {
      const int a = (int)(q / m), i = (int)(q % m);
      Zb[(size_t)a * m + i] = t.U[(int64_t)i * m + a];
      Zb[(size_t)(k1 + a) * m + i] = Y[(size_t)a * m + i];
    }
  }
  __syncthreads();
  if (mode == TB_PREP) {
    if (tid == 0) L.sc_int[0] = k1;
    for (int q = tid; q < kMaxK1 * kMaxK1; q += nt) L.sc_c[q] = (double)s_c[q];
    return;
  }
  if (mode == TB_POST) {
    // the step kernels left d, e, tau for k < m - 2 and the updated trailing 2 x 2 block
    if (tid == 0) {
      if (m >= 2) {
        b.d[m - 2] = (double)A[(int64_t)(m - 2) * m + m - 2];
        b.e[m - 2] = (double)A[(int64_t)(m - 1) * m + m - 2];
        b.tau[m - 2] = T(0);
      }
      b.d[m - 1] = (double)A[(int64_t)(m - 1) * m + m - 1];
      b.e[m - 1] = 0.0;
      b.tau[m - 1] = T(0);
    }
    __syncthreads();
    for (int i = tid; i < m; i += nt) {
      b.dt[i] = (T)b.d[i];
      b.et[i] = (T)b.e[i];
    }
    __syncthreads();
  } else {
    tridiag<T>(A, m, b);
  }
  const Gersh<T> g = gershgorin<T>(b.dt, b.et, m);
  double thr;
  __shared__ double s_lmax;
  if (!gc) {
    if (tid < 32) {
      const T lt = multisect_eig<T>(b.dt, b.et, m, m - 1, g);
      if (tid == 0) s_lmax = (double)lt;
    }
    __syncthreads();
    lmax = s_lmax;
    thr = eps * eps * lmax;
  } else if (eps > 0.0) {
    // Z = Q^T [U1, X]: reflectors in forward order, one warp per column
    if (mode != TB_POST) {
      const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
      for (int j = warp; j < 2 * k1; j += nw) {
        T *z = Zb + (size_t)j * m;
        for (int k = 0; k + 2 < m; ++k) {
          const T tk = b.tau[k];
          if (tk == T(0)) continue;
          const int n1 = m - k - 1;
          const T *vrow = A + (int64_t)k * m + k + 1;
          T sdot = T(0);
          for (int i = lane; i < n1; i += 32) sdot = fma(i == 0 ? T(1) : vrow[i], z[k + 1 + i], sdot);
          for (int o = 16; o > 0; o >>= 1) sdot += __shfl_xor_sync(0xffffffffu, sdot, o);
          sdot *= tk;
          for (int i = lane; i < n1; i += 32) z[k + 1 + i] -= sdot * (i == 0 ? T(1) : vrow[i]);
          __syncwarp();
        }
      }
    }
    __syncthreads();
    // lambda_max(G) by multisection on the low-rank count, one warp
    if (tid < 32) {
      const T lmaxT = multisect_eig<T>(b.dt, b.et, m, m - 1, g);
      T trace = T(0);
      for (int i = 0; i < m; ++i) trace += t.G[(int64_t)i * m + i];
      T lo = lmaxT, hi = fmax(trace, lmaxT) * T(1.0001) + T(1e-30);
      for (int round = 0; round < 40 && hi - lo > T(4) * unit_round<T>() * hi; ++round) {
        const T sig = lo + (hi - lo) * T(tid + 1) / T(33);
        const int c = k1 == 0 ? 0
                      : k1 <= 2 ? count_above_lowrank<T, 4>(b.dt, b.et, m, Zb, k1, s_c, sig)
                                : count_above_lowrank_wide<T>(b.dt, b.et, m, Zb, k1, s_c, sig);
        const unsigned above = __ballot_sync(0xffffffffu, c >= 1);
        const int l = above ? 31 - __clz(above) : -1;   // highest sigma with an eigenvalue above it
        const T nlo = l >= 0 ? lo + (hi - lo) * T(l + 1) / T(33) : lo;
        const T nhi = lo + (hi - lo) * T(l + 2) / T(33);
        lo = nlo;
        hi = nhi;
      }
      if (tid == 0) s_lmax = (double)(T(0.5) * (lo + hi));
    }
    __syncthreads();
    lmax = s_lmax;
    thr = eps * eps * lmax;
  } else {
    thr = 0.5;
  }
  // ---- rank: eigenvalues strictly above thr, one Sturm count in FP64
  if (tid == 0) {
    const Gersh<double> gd = gershgorin<double>(b.d, b.e, m);
    int k2 = m - sturm_below<double>(b.d, b.e, m, thr, gd.pivmin);
    if (k2 > m - k1) k2 = m - k1;
    if (k2 > t.cap - k1) k2 = t.cap - k1;   // max_rank_ratio: the largest eigenvalues are kept
    if (k2 < 0) k2 = 0;
    s_k2 = k2;
  }
  __syncthreads();
  const int k2 = s_k2;
  // ---- the k2 largest eigenvalues, descending (shifts for inverse iteration)
  for (int j = tid; j < k2; j += nt) b.lam[j] = bisect_eig<T>(b.dt, b.et, m, m - 1 - j, g);
  __syncthreads();
  // ---- eigenvectors of T by inverse iteration.  Only the span of the selected
  // vectors matters and the host re-orthonormalises them (CholQR2), which
  // tolerates the overlap u ||T|| / gap that inverse iteration leaves between
  // vectors of distinct eigenvalues.  Vectors are orthogonalised against each
  // other only inside clusters closer than 10 u ||T||, where they could come
  // out nearly parallel; a cluster is handled by one thread in order.
  const T ortol = T(10) * unit_round<T>() * g.tnorm;
  // cluster starts (thread 0 scans; b.pw reused as an int list)
  int *starts = (int *)b.pw;
  __shared__ int s_nc;
  if (tid == 0) {
    int nc = 0;
    for (int j = 0; j < k2; ++j)
      if (j == 0 || b.lam[j - 1] - b.lam[j] >= ortol) starts[nc++] = j;
    starts[nc] = k2;
    s_nc = nc;
  }
  __syncthreads();
  const int nc = s_nc;
  if (mode == TB_POST) {
    // the eigenvectors of T come from k_invit, spread over many CTAs
    if (tid == 0) {
      L.sc_int[2] = nc;
      *L.sc_tnorm = (double)g.tnorm;
    }
  } else {
    // each worker thread owns a slot: u0,u1,u2,l,y (5 m T) + m flags, in the
    // shared tile (see below for the global fallback)
    const size_t tile_bytes = (size_t)b.tile_cap * b.tile_cap * sizeof(T);
    const size_t slot_bytes = ((5 * (size_t)m * sizeof(T) + (size_t)m + 15) / 16) * 16;
    int nslot = (int)(tile_bytes / slot_bytes);
    // fewer than 8 slots in the tile: up to one per thread in the (otherwise unused)
    // LU and FL regions of global memory, interleaved so that the threads'
    // accesses coalesce (5 m T per slot in LU's 4 m^2, m flags in FL's m^2)
    const bool glob = nslot < 8;
    int ns_g = 0;
    if (glob) {
      ns_g = (int)((4 * (size_t)m * m) / (5 * (size_t)m));
      if (ns_g > nt) ns_g = nt;
      if (ns_g < 1) ns_g = 1;
      nslot = ns_g;
    }
    if (nslot > nt) nslot = nt;
    if (tid < nslot) {
      T *lu, *ys;
      unsigned char *fl;
      int st = 1;
      if (glob) {
        lu = LU + tid;
        ys = LU + 4 * (size_t)m * ns_g + tid;
        fl = FL + tid;
        st = ns_g;
      } else {
        unsigned char *slot = (unsigned char *)b.tile + (size_t)tid * slot_bytes;
        lu = (T *)slot;
        ys = lu + 4 * (size_t)m;
        fl = (unsigned char *)(ys + m);
      }
      for (int c = tid; c < nc; c += nslot) {
        const int j0 = starts[c], j1 = starts[c + 1];
        for (int q = j0; q < j1; ++q) {
          inverse_iteration<T>(b.dt, b.et, m, b.lam[q], g.tnorm, ys, Y + (size_t)j0 * m, q - j0, lu, fl,
                               (uint32_t)(q * 7919 + 17), st);
          for (int i = 0; i < m; ++i) Y[(size_t)q * m + i] = ys[(size_t)i * st];
        }
      }
    }
  }
  __syncthreads();
  if (mode == TB_POST) {
    // U_2 = Q Y is left to the reflector kernel
    if (tid == 0) {
      L.sc_int[0] = k1;
      L.sc_int[1] = k2;
      kout[t.k_idx] = k1 + k2;
    }
    return;
  }
  // ---- back-transformation U_2 = Q Y (reflectors in reverse order): columns
  // staged in shared memory in batches, one warp per column
  {
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    const size_t tile_elems = (size_t)b.tile_cap * b.tile_cap;
    // columns staged in the shared tile, or transformed in place in Y when
    // the tile cannot hold one column
    const bool in_place = tile_elems < (size_t)m;
    int batch = in_place ? max(k2, 1) : (int)(tile_elems / (size_t)m);
    for (int jb = 0; jb < k2; jb += batch) {
      const int nb = min(batch, k2 - jb);
      T *ysm = in_place ? Y + (size_t)jb * m : b.tile;
      if (!in_place)
        for (int64_t q = tid; q < (int64_t)nb * m; q += nt) ysm[q] = Y[(size_t)jb * m + q];
      __syncthreads();
      for (int j = warp; j < nb; j += nw) {
        T *y = ysm + (size_t)j * m;
        for (int k = m - 3; k >= 0; --k) {
          const T tk = b.tau[k];
          if (tk == T(0)) continue;
          const int n1 = m - k - 1;
          const T *vrow = A + (int64_t)k * m + k + 1;  // v[0] = 1 implicit, v[i] at vrow[i] for i >= 1
          T s = T(0);
          for (int i = lane; i < n1; i += 32) s = fma(i == 0 ? T(1) : vrow[i], y[k + 1 + i], s);
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          s *= tk;
          for (int i = lane; i < n1; i += 32) y[k + 1 + i] -= s * (i == 0 ? T(1) : vrow[i]);
          __syncwarp();
        }
      }
      __syncthreads();
      for (int64_t q = tid; q < (int64_t)m * nb; q += nt) {
        const int i = (int)(q / nb), j = (int)(q % nb);
        t.U[(int64_t)i * m + k1 + jb + j] = ysm[(size_t)j * m + i];
      }
      __syncthreads();
    }
  }
  if (tid == 0) kout[t.k_idx] = k1 + k2;
}

// ---------------------------------------------------------------------------
// Multi-CTA tridiagonalisation of very large nodes.  One CTA per node cannot
// use more than one SM, and its traffic grows as m^3: here each step is spread
// over ceil(m / kTriRows) CTAs per node, one warp per row.  Step k:
//   phase 0 (k_tri_update): rows i >= k get the rank-2 update of step k - 1,
//     A_ij -= v_i w_j + w_i v_j (w = p - K v, K = tau p.v / 2 from the CTAs'
//     partials in block order); then x_i = A_ik for i > k and d_k = A_kk, with
//     per-CTA partials of |x|^2.
//   phase 1 (k_tri_symv): every CTA forms the reflector of x from the partials
//     (same arithmetic in every CTA), v_i for its rows, p_i = tau sum_j A_ij v_j,
//     and per-CTA partials of p.v; v is also kept in row k of A for the later
//     products with Q (as the one-CTA path stores it).
// Reductions run in a fixed order, so results do not depend on scheduling.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int tri_task(const GridTri<T> *tasks, int ntasks, int b) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].blk0 <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// fixed-order sum of n partials by one warp (every lane gets it)
template <typename T>
__device__ __forceinline__ T warp_sum_parts(const T *part, int n, int lane) {
  T s = T(0);
  for (int c = lane; c < n; c += 32) s += part[c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <typename T>
__global__ void __launch_bounds__(kTriRows * 32) k_tri_update(const GridTri<T> *__restrict__ tasks, int ntasks,
                                                               int k) {
  __shared__ T sK;
  __shared__ T wpart[kTriRows];
  const GridTri<T> t = tasks[tri_task(tasks, ntasks, blockIdx.x)];
  const int m = t.m;
  if (k > m - 2) return;
  const int rb = blockIdx.x - t.blk0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = rb * kTriRows + warp;
  if (k >= 1) {
    if (warp == 0) {
      const T s = warp_sum_parts<T>(t.ppv, t.nblk, lane);
      if (lane == 0) sK = T(0.5) * t.tau[k - 1] * s;
    }
    __syncthreads();
  }
  T part = T(0);
  if (i >= k && i < m) {
    T *row = t.A + (int64_t)i * m;
    if (k >= 1) {
      const T K = sK;
      const T vi = t.V[i];
      const T wi = fma(-K, vi, t.P[i]);
      const T *V = t.V, *P = t.P;
      auto upd = [&](T a, int j) {
        const T vj = V[j];
        return fma(-vi, fma(-K, vj, P[j]), fma(-wi, vj, a));
      };
      // four independent row elements in flight per lane (the step is a
      // stream over the trailing rows)
      int j = k + lane;
      for (; j + 96 < m; j += 128) {
        const T a0 = row[j], a1 = row[j + 32], a2 = row[j + 64], a3 = row[j + 96];
        row[j] = upd(a0, j);
        row[j + 32] = upd(a1, j + 32);
        row[j + 64] = upd(a2, j + 64);
        row[j + 96] = upd(a3, j + 96);
      }
      for (; j < m; j += 32) row[j] = upd(row[j], j);
      __syncwarp();
    }
    if (k <= m - 3 && lane == 0) {
      const T x = row[k];
      if (i == k) {
        t.d[k] = (double)x;
      } else {
        t.X[i] = x;
        part = x * x;
      }
    }
  }
  if (lane == 0) wpart[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    T s = T(0);
    for (int w = 0; w < kTriRows; ++w) s += wpart[w];
    t.px[rb] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(kTriRows * 32) k_tri_symv(const GridTri<T> *__restrict__ tasks, int ntasks,
                                                             int k) {
  __shared__ double s_scale, s_tau;
  __shared__ T wpart[kTriRows];
  const GridTri<T> t = tasks[tri_task(tasks, ntasks, blockIdx.x)];
  const int m = t.m;
  if (k > m - 3) return;
  const int rb = blockIdx.x - t.blk0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    // the reflector of x = A[k+1.., k] (as in the one-CTA tridiagonalisation)
    const double xn2 = (double)warp_sum_parts<T>(t.px, t.nblk, lane);
    if (lane == 0) {
      const double alpha = (double)t.X[k + 1];
      const double sig = xn2 - alpha * alpha;
      double tau = 0.0, beta = alpha, scale = 0.0;
      if (sig > 0.0) {
        beta = -copysign(sqrt(xn2), alpha);
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      s_scale = scale;
      s_tau = tau;
      if (rb == 0) {
        t.e[k] = beta;
        t.tau[k] = (T)tau;
      }
    }
  }
  __syncthreads();
  const T scale_t = (T)s_scale, tau_t = (T)s_tau;
  const int i = rb * kTriRows + warp;
  T pv = T(0);
  if (i >= k + 1 && i < m) {
    const T vi = (i == k + 1) ? T(1) : t.X[i] * scale_t;
    T p = T(0);
    if (s_tau != 0.0) {
      const T *row = t.A + (int64_t)i * m;
      const T *X = t.X;
      auto vj = [&](int j) { return j == k + 1 ? T(1) : X[j] * scale_t; };
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      int j = k + 1 + lane;
      for (; j + 96 < m; j += 128) {
        a0 = fma(row[j], vj(j), a0);
        a1 = fma(row[j + 32], vj(j + 32), a1);
        a2 = fma(row[j + 64], vj(j + 64), a2);
        a3 = fma(row[j + 96], vj(j + 96), a3);
      }
      for (; j < m; j += 32) a0 = fma(row[j], vj(j), a0);
      T acc = (a0 + a1) + (a2 + a3);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      p = tau_t * acc;
    }
    if (lane == 0) {
      t.V[i] = vi;
      t.P[i] = p;
      pv = p * vi;
      if (i >= k + 2) t.A[(int64_t)k * m + i] = vi;   // reflector k kept in row k
    }
  }
  if (lane == 0) wpart[warp] = pv;
  __syncthreads();
  if (threadIdx.x == 0) {
    T s = T(0);
    for (int w = 0; w < kTriRows; ++w) s += wpart[w];
    t.ppv[rb] = s;
  }
}

// Inverse iteration of the multi-CTA path: one warp per CTA, `spc` of its
// threads active, each with a slot (LU of T - lam I and the vector: 5 m T and m
// flags) in shared memory, taking one cluster of close eigenvalues.  Same
// arithmetic as the one-CTA kernel; each step of the recurrence stays on chip.
template <typename T>
__device__ __forceinline__ int invit_task(const InvitTask<T> *tasks, int ntasks, int b) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].blk0 <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <typename T>
__host__ __device__ inline size_t invit_slot_bytes(int m) {
  return ((5 * (size_t)m * sizeof(T) + (size_t)m + 15) / 16) * 16;
}

template <typename T>
__global__ void __launch_bounds__(32) k_invit(const InvitTask<T> *__restrict__ tasks, int ntasks, int spc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const InvitTask<T> t = tasks[invit_task(tasks, ntasks, blockIdx.x)];
  const int m = t.m;
  const int c = (blockIdx.x - t.blk0) * spc + threadIdx.x;
  if ((int)threadIdx.x >= spc || c >= t.sc[2]) return;
  unsigned char *slot = smem_raw + (size_t)threadIdx.x * invit_slot_bytes<T>(m);
  T *lu = (T *)slot;
  T *ys = lu + 4 * (size_t)m;
  unsigned char *fl = (unsigned char *)(ys + m);
  const T tnorm = (T)*t.tnorm;
  const int j0 = t.starts[c], j1 = t.starts[c + 1];
  for (int q = j0; q < j1; ++q) {
    inverse_iteration<T>(t.dt, t.et, m, t.lam[q], tnorm, ys, t.Y + (size_t)j0 * m, q - j0, lu, fl,
                         (uint32_t)(q * 7919 + 17));
    for (int i = 0; i < m; ++i) t.Y[(size_t)q * m + i] = ys[i];
  }
}

// Products with the reflectors of a node, one CTA per batch of columns held in
// shared memory: for each reflector the block forms all the batch's dot
// products (fixed-order reduction), then updates the columns.
constexpr int RT = 256;
constexpr int RNB = 16;   // most columns per task

template <typename T>
__global__ void __launch_bounds__(RT) k_refl(const ReflTask<T> *__restrict__ tasks, int nb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[RT / 32][RNB];
  __shared__ T tot[RNB];
  const ReflTask<T> t = tasks[blockIdx.x];
  const int m = t.m;
  const int k1 = t.sc[0];
  const int ncol = t.fwd ? 2 * k1 : t.sc[1];
  if (t.j0 >= ncol) return;
  const int nc = min(nb, ncol - t.j0);
  T *Ys = (T *)smem_raw;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int64_t q = tid; q < (int64_t)nc * m; q += RT) Ys[q] = t.cols[(size_t)t.j0 * m + q];
  __syncthreads();
  for (int kk = 0; kk + 2 < m; ++kk) {
    const int k = t.fwd ? kk : m - 3 - kk;
    const T tk = t.tau[k];
    if (tk == T(0)) continue;
    const int n1 = m - k - 1;
    const T *vrow = t.A + (int64_t)k * m + k + 1;   // v[0] = 1 implicit
    T s[RNB];
#pragma unroll
    for (int c = 0; c < RNB; ++c) s[c] = T(0);
    for (int i = tid; i < n1; i += RT) {
      const T vi = i == 0 ? T(1) : vrow[i];
#pragma unroll
      for (int c = 0; c < RNB; ++c)
        if (c < nc) s[c] = fma(vi, Ys[(size_t)c * m + k + 1 + i], s[c]);
    }
#pragma unroll
    for (int c = 0; c < RNB; ++c) {
      T x = s[c];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) red[warp][c] = x;
    }
    __syncthreads();
    if (tid < nc) {
      T x = T(0);
      for (int w = 0; w < RT / 32; ++w) x += red[w][tid];
      tot[tid] = tk * x;
    }
    __syncthreads();
    for (int i = tid; i < n1; i += RT) {
      const T vi = i == 0 ? T(1) : vrow[i];
      for (int c = 0; c < nc; ++c) Ys[(size_t)c * m + k + 1 + i] -= tot[c] * vi;
    }
    __syncthreads();
  }
  if (t.fwd) {
    for (int64_t q = tid; q < (int64_t)nc * m; q += RT) t.cols[(size_t)t.j0 * m + q] = Ys[q];
  } else {
    for (int64_t q = tid; q < (int64_t)m * nc; q += RT) {
      const int i = (int)(q / nc), c = (int)(q % nc);
      t.U[(int64_t)i * m + k1 + t.j0 + c] = Ys[(size_t)c * m + i];
    }
  }
}

}  // namespace

// bytes of the per-node vectors of k_trunc_big (d, e, pw in FP64; six m-vectors
// and 34 reduction slots in T), 16-byte aligned
template <typename T>
size_t trunc_big_vec_bytes(int m) {
  return big_vec_bytes<T>(m);
}

template <typename T>
size_t trunc_big_work_elems(int m) {
  // A, Y, LU (6 m^2 T) + LS (164 m T) + flags (m^2 bytes) + the vectors (when
  // they do not fit in shared memory) + SC; Y and LU also hold k1 m doubles
  // of scratch
  const size_t bytes = sizeof(T) * (6 * (size_t)m * m + 164 * (size_t)m) + (size_t)m * m + 16 +
                       trunc_big_vec_bytes<T>(m) + 16 + kBigScBytes + 64;
  return (bytes + sizeof(T) - 1) / sizeof(T);
}

template <typename T, int NT>
void launch_trunc_big_nt(const TruncTask<T> *d_tasks, int ntasks, int *d_k, double eps, int variant, int max_m,
                         cudaStream_t st) {
  if (ntasks == 0) return;
  // the per-node vectors go to shared memory while they leave room for a
  // tile of at least 64 x 64; the rest of the budget is the tile, no larger
  // than the largest node needs
  const size_t budget = 200 * 1024;
  size_t fixed = trunc_big_vec_bytes<T>(max_m) + 32;
  const int vec_smem = fixed + 64 * 64 * sizeof(T) <= budget ? 1 : 0;
  if (!vec_smem) fixed = 32;
  int cap = 0;
  while (cap < max_m && (size_t)(cap + 1) * (cap + 1) * sizeof(T) + fixed <= budget) ++cap;
  const size_t sm = fixed + (size_t)cap * cap * sizeof(T);
  check_dynamic_smem(sm, allow_max_dynamic_smem<&k_trunc_big<T, NT>>(), "k_trunc_big");
  k_trunc_big<T, NT><<<ntasks, NT, sm, st>>>(d_tasks, d_k, variant, cap, vec_smem, TB_FULL);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_trunc_big(const TruncTask<T> *d_tasks, int ntasks, int *d_k, double eps, int variant, int max_m,
                      cudaStream_t st) {
  if (max_m <= kTruncBigMidMax)
    launch_trunc_big_nt<T, 256>(d_tasks, ntasks, d_k, eps, variant, max_m, st);
  else
    launch_trunc_big_nt<T, 1024>(d_tasks, ntasks, d_k, eps, variant, max_m, st);
}

template <typename T>
void launch_trunc_big_mode(const TruncTask<T> *d_tasks, int ntasks, int *d_k, double eps, int variant, int max_m,
                           int mode, cudaStream_t st) {
  if (ntasks == 0) return;
  // per-node vectors in global memory (the step kernels write d, e, tau there);
  // the whole budget is the tile
  const size_t budget = 200 * 1024;
  int cap = 0;
  while (cap < max_m && (size_t)(cap + 1) * (cap + 1) * sizeof(T) + 32 <= budget) ++cap;
  const size_t sm = 32 + (size_t)cap * cap * sizeof(T);
  check_dynamic_smem(sm, allow_max_dynamic_smem<&k_trunc_big<T, 1024>>(), "k_trunc_big");
  k_trunc_big<T, 1024><<<ntasks, 1024, sm, st>>>(d_tasks, d_k, variant, cap, 0, mode);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_tri_step(const GridTri<T> *d_tasks, int ntasks, int total_blocks, int k, int phase, cudaStream_t st) {
  if (ntasks == 0 || total_blocks == 0) return;
  if (phase == 0)
    k_tri_update<T><<<total_blocks, kTriRows * 32, 0, st>>>(d_tasks, ntasks, k);
  else
    k_tri_symv<T><<<total_blocks, kTriRows * 32, 0, st>>>(d_tasks, ntasks, k);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

template <typename T>
int refl_batch(int m) {
  const size_t budget = 200 * 1024;
  const int nb = (int)(budget / (sizeof(T) * (size_t)std::max(m, 1)));
  return std::max(1, std::min(nb, RNB));
}

template <typename T>
void launch_refl(const ReflTask<T> *d_tasks, int ntasks, int nb, int m_max, cudaStream_t st) {
  if (ntasks == 0) return;
  const size_t sm = sizeof(T) * (size_t)nb * m_max;
  check_dynamic_smem(sm, allow_max_dynamic_smem<&k_refl<T>>(), "k_refl");
  k_refl<T><<<ntasks, RT, sm, st>>>(d_tasks, nb);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

template <typename T>
int invit_slots(int m) {
  const size_t budget = 200 * 1024;
  const int spc = (int)(budget / invit_slot_bytes<T>(std::max(m, 1)));
  return std::max(1, std::min(spc, 32));
}

template <typename T>
void launch_invit(const InvitTask<T> *d_tasks, int ntasks, int total_blocks, int spc, int m_max, cudaStream_t st) {
  if (ntasks == 0 || total_blocks == 0) return;
  const size_t sm = (size_t)spc * invit_slot_bytes<T>(m_max);
  check_dynamic_smem(sm, allow_max_dynamic_smem<&k_invit<T>>(), "k_invit");
  k_invit<T><<<total_blocks, 32, sm, st>>>(d_tasks, ntasks, spc);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

template int invit_slots<double>(int);
template int invit_slots<float>(int);
template void launch_invit<double>(const InvitTask<double> *, int, int, int, int, cudaStream_t);
template void launch_invit<float>(const InvitTask<float> *, int, int, int, int, cudaStream_t);
template void launch_trunc_big_mode<double>(const TruncTask<double> *, int, int *, double, int, int, int,
                                            cudaStream_t);
template void launch_trunc_big_mode<float>(const TruncTask<float> *, int, int *, double, int, int, int,
                                           cudaStream_t);
template void launch_tri_step<double>(const GridTri<double> *, int, int, int, int, cudaStream_t);
template void launch_tri_step<float>(const GridTri<float> *, int, int, int, int, cudaStream_t);
template int refl_batch<double>(int);
template int refl_batch<float>(int);
template void launch_refl<double>(const ReflTask<double> *, int, int, int, cudaStream_t);
template void launch_refl<float>(const ReflTask<float> *, int, int, int, cudaStream_t);
template size_t trunc_big_work_elems<double>(int);
template size_t trunc_big_work_elems<float>(int);
template void launch_trunc_big<double>(const TruncTask<double> *, int, int *, double, int, int, cudaStream_t);
template void launch_trunc_big<float>(const TruncTask<float> *, int, int *, double, int, int, cudaStream_t);

}  // namespace hs
