// Householder tridiagonalisation of a large super node's Gram matrix J by one
// thread-block cluster (Sec. 3.2: the eigen-solve behind the rank decision
// sigma_i > eps ||A_sw|| and the basis U_2; Sec. 6 for the projected J of GC).
//
// The multi-CTA path needs two kernel launches per Householder step (the
// reflector needs a reduction over the whole column, the rank-2 update the
// whole vector p), and at a few microseconds per launch the m - 2 steps of a
// node of a few hundred unknowns are launch-bound.  Here the whole m x m
// matrix stays in shared memory for all steps: the C CTAs of a cluster each
// hold a slab of ceil(m / C) columns (all rows), and the steps synchronise
// with cluster barriers instead of kernel boundaries (a node that fits one
// CTA's shared memory runs alone in one CTA, tri_cta below).  J is symmetric,
// so every product is a column walk: thread i owns column i (with up to four
// threads splitting its rows), consecutive threads on consecutive words.
// Step k:
//   1. every CTA copies column k (= row k) from its owner's slab through
//      distributed shared memory, and forms the reflector I - tau v v^T of
//      x = J[k+1.., k] (the same FP64 scalars in every CTA);
//   2. p_i = tau sum_j J_ji v_j for its own columns, and its share of p.v;
//   3. cluster barrier; K = tau (p.v) / 2 from the CTAs' shares in rank order,
//      w_j = p_j - K v_j with p_j read from the owner of column j;
//   4. J_ji -= v_j w_i + w_j v_i on its own columns.
// Step 4 is deferred into steps 1 and 2 of the next step (the column read in
// step 1 gets it on the fly, the rest in the same walk as step 2), which
// leaves one walk of the slab and one cluster barrier per step.
// Outputs are those of the step kernels: d, e (FP64) and tau, reflector k in
// global row k of A (v[0] = 1 implicit, v[1..] at A[k][k+2..]), the trailing
// 2 x 2 block in A, so the eigenvalue and eigenvector kernels that follow are
// unchanged.  Cluster size C (1, 2, 4 or 8) is the smallest that fits the slab
// in shared memory; it depends on m alone, as does every reduction order, so a
// node gets the same bits in any batch.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "hs_internal.h"

namespace cg = cooperative_groups;

namespace hs {

namespace {

constexpr int kClThreads = 256;

// fixed-order block sum (every thread gets the total); red: 33 T
template <typename T>
__device__ T cl_bsum(T v, T *red) {
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

// threads per owned column in the cluster kernel (1 .. 4)
__host__ __device__ inline int cl_tpc(int R, int nt) {
  const int q = R > 0 ? nt / R : 1;
  return q < 1 ? 1 : q > 4 ? 4 : q;
}

template <typename T>
__host__ __device__ inline size_t cl_smem_bytes(int m, int C) {
  if (C == 1) return sizeof(T) * ((size_t)m * (m | 1) + 4 * (size_t)m + 64);
  const int R = (m + C - 1) / C;
  return sizeof(T) * ((size_t)R * m + 5 * (size_t)m + (size_t)R * (2 + cl_tpc(R, kClThreads)) + 72);
}

// Block sum with one barrier: each warp's partial goes to red[warp], and every
// thread adds the partials in warp order (the same total in every thread).
// Calls must alternate between two red buffers, so that a buffer is written
// again only after a barrier that follows every read of it.
template <typename T>
__device__ __forceinline__ T cta_sum(T v, T *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = red[0];
  for (int q = 1; q < (int)(blockDim.x >> 5); ++q) s += red[q];
  return s;
}

// One CTA holds the whole m x m matrix (ld = m | 1, odd, so that the column
// walks below are free of bank conflicts) and runs every step alone.  By
// symmetry of the trailing block, p_i = tau sum_j J_ji v_j and the rank-2
// update are column walks: thread i owns column i and loops over the rows,
// consecutive threads on consecutive words (no per-row warp reductions).
// The rank-2 update of step k is applied lazily: row k + 1 first (it gives
// the next reflector), then the rest of the trailing block in the same pass
// that forms the next p, so each step walks the trailing block once.  The
// updated values are those of applying it at once (same expression).
template <typename T>
__device__ void tri_cta(const GridTri<T> &t, unsigned char *smem_raw) {
  const int m = t.m;
  const int ld = m | 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  T *W = reinterpret_cast<T *>(smem_raw);   // m x ld
  T *vp = W + (size_t)m * ld;                // pending update (v, w) of the previous step
  T *wp = vp + m;
  T *v = wp + m;                             // this step's reflector and w
  T *w = v + m;
  T *red0 = w + m;                           // two reduction buffers of 32 T
  T *red1 = red0 + 32;
  for (int64_t q = tid; q < (int64_t)m * m; q += nt) {
    const int i = (int)(q / m), j = (int)(q % m);
    W[(size_t)i * ld + j] = t.A[q];
  }
  for (int j = tid; j < m; j += nt) vp[j] = wp[j] = T(0);
  __syncthreads();
  for (int k = 0; k + 2 < m; ++k) {
    T *rowk = W + (size_t)k * ld;              // row k = column k
    // the pending update on row k (columns >= k), and the norm of its tail
    const T vk = vp[k], wk = wp[k];
    if (tid == 0) rowk[k] = fma(-vk, wp[k], fma(-wk, vp[k], rowk[k]));
    T s2t = T(0);
    for (int j = k + 1 + tid; j < m; j += nt) {
      const T a = fma(-vk, wp[j], fma(-wk, vp[j], rowk[j]));
      rowk[j] = a;
      s2t = fma(a, a, s2t);
    }
    const double xn2 = (double)cta_sum<T>(s2t, red0);   // barrier: row k complete
    const double alpha = (double)rowk[k + 1];
    const double sig = xn2 - alpha * alpha;
    double tau = 0.0, beta = alpha, scale = 0.0;
    if (sig > 0.0) {
      beta = -copysign(sqrt(xn2), alpha);
      tau = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    const T scale_t = (T)scale, tau_t = (T)tau;
    for (int j = k + 1 + tid; j < m; j += nt) {
      const T vj = (j == k + 1) ? T(1) : rowk[j] * scale_t;
      v[j] = vj;
      if (j >= k + 2) t.A[(int64_t)k * m + j] = vj;   // reflector k in global row k
    }
    if (tid == 0) {
      t.d[k] = (double)rowk[k];
      t.e[k] = beta;
      t.tau[k] = tau_t;
    }
    __syncthreads();
    // one walk of each trailing column i > k: the pending update of rows
    // j > k, then p_i = tau sum_j J_ji v_j (tau = 0 gives p = w = 0, an
    // update that changes nothing)
    T pvt = T(0);
    for (int i = k + 1 + tid; i < m; i += nt) {
      T *col = W + i;
      const T vi = vp[i], wi = wp[i];
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      int j = k + 1;
      for (; j + 3 < m; j += 4) {
        const T x0 = fma(-vp[j], wi, fma(-wp[j], vi, col[(size_t)j * ld]));
        const T x1 = fma(-vp[j + 1], wi, fma(-wp[j + 1], vi, col[(size_t)(j + 1) * ld]));
        const T x2 = fma(-vp[j + 2], wi, fma(-wp[j + 2], vi, col[(size_t)(j + 2) * ld]));
        const T x3 = fma(-vp[j + 3], wi, fma(-wp[j + 3], vi, col[(size_t)(j + 3) * ld]));
        col[(size_t)j * ld] = x0;
        col[(size_t)(j + 1) * ld] = x1;
        col[(size_t)(j + 2) * ld] = x2;
        col[(size_t)(j + 3) * ld] = x3;
        a0 = fma(x0, v[j], a0);
        a1 = fma(x1, v[j + 1], a1);
        a2 = fma(x2, v[j + 2], a2);
        a3 = fma(x3, v[j + 3], a3);
      }
      for (; j < m; ++j) {
        const T x0 = fma(-vp[j], wi, fma(-wp[j], vi, col[(size_t)j * ld]));
        col[(size_t)j * ld] = x0;
        a0 = fma(x0, v[j], a0);
      }
      const T p = tau_t * ((a0 + a1) + (a2 + a3));
      w[i] = p;
      pvt = fma(p, v[i], pvt);
    }
    const T K = T(0.5) * tau_t * cta_sum<T>(pvt, red1);
    for (int i = k + 1 + tid; i < m; i += nt) w[i] = fma(-K, v[i], w[i]);
    __syncthreads();
    T *x = vp;   // this step's (v, w) become the pending update
    vp = v;
    v = x;
    x = wp;
    wp = w;
    w = x;
  }
  // the last pending update on the trailing 2 x 2 block, which is written out
  for (int i = max(m - 2, 0) + tid; i < m; i += nt)
    for (int j = m - 2; j <= i; ++j) {
      const T a = fma(-vp[i], wp[j], fma(-wp[i], vp[j], W[(size_t)i * ld + j]));
      t.A[(int64_t)i * m + j] = a;
    }
}

template <typename T, int C>
__global__ void __launch_bounds__(kClThreads) k_tri_cluster(const GridTri<T> *__restrict__ tasks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if constexpr (C == 1) {
    tri_cta<T>(tasks[blockIdx.x], smem_raw);
    return;
  }
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const GridTri<T> t = tasks[blockIdx.x / C];
  const int m = t.m;
  const int R = (m + C - 1) / C;
  const int c0 = crank * R, c1 = min(m, c0 + R);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tpc = cl_tpc(R, nt);               // threads per column
  const int ci = tid % R, part = tid / R;      // own column c0 + ci, rows j = part (mod tpc)
  T *slab = reinterpret_cast<T *>(smem_raw);   // columns c0 .. c1-1 of J, all rows: slab[j R + (i - c0)]
  T *x = slab + (size_t)m * R;                 // column k of J, rows k..
  T *vp = x + m;                               // pending update (v, w) of the previous step
  T *wp = vp + m;
  T *v = wp + m;                               // this step's reflector and w
  T *w = v + m;
  T *pseg = w + m;                             // p on the own columns, two buffers (step parity)
  T *psum = pseg + 2 * (size_t)R;              // tpc partial sums per own column
  T *red0 = psum + (size_t)R * tpc;            // two reduction buffers of 32 T
  T *red1 = red0 + 32;
  T *pvpart = red1 + 32;                       // this CTA's share of p.v, two buffers

  for (int64_t q = tid; q < (int64_t)m * R; q += nt) {
    const int j = (int)(q / R), i = c0 + (int)(q % R);
    slab[q] = i < c1 ? t.A[(int64_t)j * m + i] : T(0);
  }
  for (int j = tid; j < m; j += nt) vp[j] = wp[j] = T(0);
  cluster.sync();

  // The rank-2 update of step k is applied lazily, as in tri_cta: to column
  // k + 1 as it is read from its owner, and to the rest of the own columns in
  // the pass that forms the next p.  One cluster barrier per step: p and the
  // share of p.v are double-buffered, so a CTA that runs ahead never
  // overwrites what a slower one still reads, and the column a step reads is
  // not written in that step.
  for (int k = 0; k + 2 < m; ++k) {
    const int owner = k / R;
    const T *ocol = cluster.map_shared_rank(slab, owner) + (k - owner * R);
    const T vk = vp[k], wk = wp[k];
    T s2t = T(0);
    for (int j = k + tid; j < m; j += nt) {
      const T a = fma(-vp[j], wk, fma(-wp[j], vk, ocol[(size_t)j * R]));
      x[j] = a;
      if (j > k) s2t = fma(a, a, s2t);
    }
    const double xn2 = (double)cta_sum<T>(s2t, red0);   // barrier: x complete
    const double alpha = (double)x[k + 1];
    const double sig = xn2 - alpha * alpha;
    double tau = 0.0, beta = alpha, scale = 0.0;
    if (sig > 0.0) {
      beta = -copysign(sqrt(xn2), alpha);
      tau = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    const T scale_t = (T)scale, tau_t = (T)tau;
    for (int j = k + 1 + tid; j < m; j += nt) {
      const T vj = (j == k + 1) ? T(1) : x[j] * scale_t;
      v[j] = vj;
      if (crank == owner && j >= k + 2) t.A[(int64_t)k * m + j] = vj;   // reflector k in global row k
    }
    if (crank == owner && tid == 0) {
      t.d[k] = (double)x[k];
      t.e[k] = beta;
      t.tau[k] = tau_t;
    }
    __syncthreads();
    // the own columns i > k: pending update of rows j > k, then
    // p_i = tau sum_j J_ji v_j (rows split over tpc threads per column)
    T *pk = pseg + (k & 1) * R;
    const int i = c0 + ci;
    const bool mine = part < tpc && i < c1 && i > k;
    if (mine) {
      const T vi = vp[i], wi = wp[i];
      T a0 = T(0), a1 = T(0);
      int j = k + 1 + part;
      for (; j + tpc < m; j += 2 * tpc) {
        T *s0 = slab + (size_t)j * R + ci;
        T *s1 = slab + (size_t)(j + tpc) * R + ci;
        const T x0 = fma(-vp[j], wi, fma(-wp[j], vi, *s0));
        const T x1 = fma(-vp[j + tpc], wi, fma(-wp[j + tpc], vi, *s1));
        *s0 = x0;
        *s1 = x1;
        a0 = fma(x0, v[j], a0);
        a1 = fma(x1, v[j + tpc], a1);
      }
      if (j < m) {
        T *s0 = slab + (size_t)j * R + ci;
        const T x0 = fma(-vp[j], wi, fma(-wp[j], vi, *s0));
        *s0 = x0;
        a0 = fma(x0, v[j], a0);
      }
      psum[part * R + ci] = a0 + a1;
    }
    __syncthreads();
    T pvt = T(0);
    if (part == 0 && i < c1 && i > k) {
      T acc = T(0);
      for (int q = 0; q < tpc; ++q) acc += psum[q * R + ci];
      const T p = tau_t * acc;
      pk[ci] = p;
      pvt = p * v[i];
    }
    const T pv_own = cta_sum<T>(pvt, red1);
    if (tid == 0) pvpart[k & 1] = pv_own;
    cluster.sync();   // every CTA's p and share of p.v are visible; every pass of step k is done
    T pv = T(0);
    for (int c = 0; c < C; ++c) pv += cluster.map_shared_rank(pvpart, c)[k & 1];
    const T K = T(0.5) * tau_t * pv;
    for (int j = k + 1 + tid; j < m; j += nt) {
      const int oj = j / R;
      const T pj = cluster.map_shared_rank(pseg, oj)[(k & 1) * R + j - oj * R];
      w[j] = fma(-K, v[j], pj);
    }
    __syncthreads();
    T *y = vp;   // this step's (v, w) become the pending update
    vp = v;
    v = y;
    y = wp;
    wp = w;
    w = y;
  }
  // the last pending update on the trailing 2 x 2 block, lower triangle,
  // written out by the owners of its columns
  for (int j = max(c0, m - 2) + tid; j < c1; j += nt)
    for (int i = j; i < m; ++i)
      t.A[(int64_t)i * m + j] = fma(-vp[i], wp[j], fma(-wp[i], vp[j], slab[(size_t)i * R + (j - c0)]));
  // no CTA may leave while others still read its shared memory
  cluster.sync();
}

template <typename T, int C>
void launch_cluster_c(const GridTri<T> *d_tasks, int ntasks, int m_max, cudaStream_t st) {
  const size_t sm = cl_smem_bytes<T>(m_max, C);
  check_dynamic_smem(sm, allow_max_dynamic_smem<&k_tri_cluster<T, C>>(), "k_tri_cluster");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ntasks * C), 1, 1);
  cfg.blockDim = dim3(kClThreads, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  HS_CUDA(cudaLaunchKernelEx(&cfg, k_tri_cluster<T, C>, d_tasks));
  count_launch();
}

// whether a cluster of C CTAs with `sm` bytes each can be resident at all
template <typename T, int C>
bool cluster_fits(size_t sm) {
  if (sm > (size_t)allow_max_dynamic_smem<&k_tri_cluster<T, C>>()) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kClThreads, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, k_tri_cluster<T, C>, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

// Largest m a cluster of C CTAs takes (0 if such a cluster with the kernel's
// largest shared-memory size cannot be resident), once per device.
template <typename T>
int tri_cluster_max_m(int C) {
  static std::mutex mu;
  static int table[64][4];
  static bool ready[64] = {false};
  int dev = 0;
  HS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) fail(HS_ERR_CUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (!ready[dev]) {
    const int cs[4] = {1, 2, 4, 8};
    for (int q = 0; q < 4; ++q) {
      const int c = cs[q];
      int lim = 0;
      bool ok = false;
      if (c == 1) lim = allow_max_dynamic_smem<&k_tri_cluster<T, 1>>(), ok = cluster_fits<T, 1>(lim);
      if (c == 2) lim = allow_max_dynamic_smem<&k_tri_cluster<T, 2>>(), ok = cluster_fits<T, 2>(lim);
      if (c == 4) lim = allow_max_dynamic_smem<&k_tri_cluster<T, 4>>(), ok = cluster_fits<T, 4>(lim);
      if (c == 8) lim = allow_max_dynamic_smem<&k_tri_cluster<T, 8>>(), ok = cluster_fits<T, 8>(lim);
      int mm = 0;
      if (ok)
        // (several CTAs: at most one owned column per thread)
        while (cl_smem_bytes<T>(mm + 1, c) <= (size_t)lim && (c == 1 || (mm + c) / c <= kClThreads)) ++mm;
      table[dev][q] = mm;
    }
    ready[dev] = true;
  }
  const int q = C == 1 ? 0 : C == 2 ? 1 : C == 4 ? 2 : 3;
  return table[dev][q];
}

}  // namespace

// The smallest cluster (1, 2, 4 or 8 CTAs) whose slabs fit; larger nodes take
// the step kernels.  HS_TRI_CLUSTER=1 (environment) keeps clusters to one CTA.
template <typename T>
int tri_cluster_size(int m) {
  static const int cmax = [] {
    const char *e = std::getenv("HS_TRI_CLUSTER");
    return (e && e[0] == '1') ? 1 : 8;
  }();
  for (int c : {1, 2, 4, 8})
    if (c <= cmax && m <= tri_cluster_max_m<T>(c)) return c;
  return 0;
}

template <typename T>
void launch_tri_cluster(const GridTri<T> *d_tasks, int ntasks, int C, int m_max, cudaStream_t st) {
  if (ntasks == 0) return;
  switch (C) {
    case 1: launch_cluster_c<T, 1>(d_tasks, ntasks, m_max, st); break;
    case 2: launch_cluster_c<T, 2>(d_tasks, ntasks, m_max, st); break;
    case 4: launch_cluster_c<T, 4>(d_tasks, ntasks, m_max, st); break;
    case 8: launch_cluster_c<T, 8>(d_tasks, ntasks, m_max, st); break;
    default: fail(HS_ERR_INVALID, "internal: cluster size of the tridiagonalisation");
  }
  HS_CUDA(cudaGetLastError());
}

template int tri_cluster_size<double>(int);
template int tri_cluster_size<float>(int);
template void launch_tri_cluster<double>(const GridTri<double> *, int, int, int, cudaStream_t);
template void launch_tri_cluster<float>(const GridTri<float> *, int, int, int, cudaStream_t);

}  // namespace hs
