// Householder tridiagonalisation of a large super node's Gram matrix J by one
// thread-block cluster (Sec. 3.2: the eigen-solve behind the rank decision
// sigma_i > eps ||A_sw|| and the basis U_2; Sec. 6 for the projected J of GC).
//
// The multi-CTA path needs two kernel launches per Householder step (the
// reflector needs a reduction over the whole column, the rank-2 update the
// whole vector p), and at a few microseconds per launch the m - 2 steps of a
// node of a few hundred unknowns are launch-bound.  Here the whole m x m
// matrix stays in shared memory for all steps: the C CTAs of a cluster each
// hold a slab of ceil(m / C) rows, and the steps synchronise with cluster
// barriers instead of kernel boundaries (a node that fits one CTA's shared
// memory runs alone in one CTA, tri_cta below).  Step k:
//   1. every CTA copies row k (= column k, J symmetric) from its owner's slab
//      through distributed shared memory, and forms the reflector
//      I - tau v v^T of x = J[k+1.., k] (the same FP64 scalars in every CTA);
//   2. p_i = tau sum_j J_ij v_j for its own rows, and its share of p.v;
//   3. cluster barrier; K = tau (p.v) / 2 from the CTAs' shares in rank order,
//      w_j = p_j - K v_j with p_j read from the owner of row j;
//   4. J_ij -= v_i w_j + w_i v_j on its own rows; cluster barrier.
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

template <typename T>
__host__ __device__ inline size_t cl_smem_bytes(int m, int C) {
  if (C == 1) return sizeof(T) * ((size_t)m * (m | 1) + 2 * (size_t)m + 40);
  const int R = (m + C - 1) / C;
  return sizeof(T) * ((size_t)R * m + 3 * (size_t)m + R + 48);
}

// One CTA holds the whole m x m matrix (ld = m | 1, odd, so that the column
// walks below are free of bank conflicts) and runs every step alone.  By
// symmetry of the trailing block, p_i = tau sum_j J_ji v_j and the rank-2
// update are column walks: thread i owns column i and loops over the rows,
// consecutive threads on consecutive words (no per-row warp reductions).
template <typename T>
__device__ void tri_cta(const GridTri<T> &t, unsigned char *smem_raw) {
  const int m = t.m;
  const int ld = m | 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  T *W = reinterpret_cast<T *>(smem_raw);   // m x ld
  T *v = W + (size_t)m * ld;
  T *w = v + m;
  T *red = w + m;                            // 33 T
  for (int64_t q = tid; q < (int64_t)m * m; q += nt) {
    const int i = (int)(q / m), j = (int)(q % m);
    W[(size_t)i * ld + j] = t.A[q];
  }
  __syncthreads();
  for (int k = 0; k + 2 < m; ++k) {
    const T *rowk = W + (size_t)k * ld;        // row k = column k
    T s2t = T(0);
    for (int j = k + 1 + tid; j < m; j += nt) s2t = fma(rowk[j], rowk[j], s2t);
    const double xn2 = (double)cl_bsum<T>(s2t, red);
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
    if (tau == 0.0) continue;
    // p_i = tau sum_j J_ji v_j, thread per column, four partial sums
    T pvt = T(0);
    for (int i = k + 1 + tid; i < m; i += nt) {
      const T *col = W + i;
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      int j = k + 1;
      for (; j + 3 < m; j += 4) {
        a0 = fma(col[(size_t)j * ld], v[j], a0);
        a1 = fma(col[(size_t)(j + 1) * ld], v[j + 1], a1);
        a2 = fma(col[(size_t)(j + 2) * ld], v[j + 2], a2);
        a3 = fma(col[(size_t)(j + 3) * ld], v[j + 3], a3);
      }
      for (; j < m; ++j) a0 = fma(col[(size_t)j * ld], v[j], a0);
      const T p = tau_t * ((a0 + a1) + (a2 + a3));
      w[i] = p;
      pvt = fma(p, v[i], pvt);
    }
    const T K = T(0.5) * tau_t * cl_bsum<T>(pvt, red);
    for (int i = k + 1 + tid; i < m; i += nt) w[i] = fma(-K, v[i], w[i]);
    __syncthreads();
    // J_ji -= v_j w_i + w_j v_i, thread per column
    for (int i = k + 1 + tid; i < m; i += nt) {
      T *col = W + i;
      const T vi = v[i], wi = w[i];
      for (int j = k + 1; j < m; ++j) {
        T &a = col[(size_t)j * ld];
        a = fma(-v[j], wi, fma(-w[j], vi, a));
      }
    }
    __syncthreads();
  }
  for (int i = max(m - 2, 0) + tid; i < m; i += nt)
    for (int j = m - 2; j <= i; ++j) t.A[(int64_t)i * m + j] = W[(size_t)i * ld + j];
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
  const int r0 = crank * R, r1 = min(m, r0 + R);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  T *slab = reinterpret_cast<T *>(smem_raw);   // rows r0 .. r1-1, ld m
  T *xrow = slab + (size_t)R * m;              // row k of J, columns k..
  T *v = xrow + m;                             // reflector
  T *w = v + m;                                // w = p - K v
  T *pseg = w + m;                             // p on the own rows
  T *red = pseg + R;                           // 33 T of reduction scratch, then the share of p.v
  T *pvpart = red + 40;

  for (int64_t q = tid; q < (int64_t)(r1 - r0) * m; q += nt) slab[q] = t.A[(int64_t)r0 * m + q];
  cluster.sync();

  for (int k = 0; k + 2 < m; ++k) {
    const int owner = k / R;
    const T *srow = cluster.map_shared_rank(slab, owner) + (size_t)(k - owner * R) * m;
    for (int j = k + tid; j < m; j += nt) xrow[j] = srow[j];
    __syncthreads();
    T s2t = T(0);
    for (int j = k + 1 + tid; j < m; j += nt) s2t = fma(xrow[j], xrow[j], s2t);
    const double xn2 = (double)cl_bsum<T>(s2t, red);
    const double alpha = (double)xrow[k + 1];
    const double sig = xn2 - alpha * alpha;
    double tau = 0.0, beta = alpha, scale = 0.0;
    if (sig > 0.0) {
      beta = -copysign(sqrt(xn2), alpha);
      tau = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    const T scale_t = (T)scale, tau_t = (T)tau;
    for (int j = k + 1 + tid; j < m; j += nt) {
      const T vj = (j == k + 1) ? T(1) : xrow[j] * scale_t;
      v[j] = vj;
      if (crank == owner && j >= k + 2) t.A[(int64_t)k * m + j] = vj;   // reflector k in global row k
    }
    if (crank == owner && tid == 0) {
      t.d[k] = (double)xrow[k];
      t.e[k] = beta;
      t.tau[k] = tau_t;
    }
    __syncthreads();
    if (tau == 0.0) continue;   // the same decision in every CTA: no update, no barrier
    // p_i = tau J_i v on the own rows i > k, one warp per row
    const int i0 = max(r0, k + 1);
    for (int i = i0 + warp; i < r1; i += nw) {
      const T *row = slab + (size_t)(i - r0) * m;
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      int j = k + 1 + lane;
      for (; j + 96 < m; j += 128) {
        a0 = fma(row[j], v[j], a0);
        a1 = fma(row[j + 32], v[j + 32], a1);
        a2 = fma(row[j + 64], v[j + 64], a2);
        a3 = fma(row[j + 96], v[j + 96], a3);
      }
      for (; j < m; j += 32) a0 = fma(row[j], v[j], a0);
      T acc = (a0 + a1) + (a2 + a3);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) pseg[i - r0] = tau_t * acc;
    }
    __syncthreads();
    T pvt = T(0);
    for (int i = i0 + tid; i < r1; i += nt) pvt = fma(pseg[i - r0], v[i], pvt);
    const T pv_own = cl_bsum<T>(pvt, red);
    if (tid == 0) *pvpart = pv_own;
    cluster.sync();   // every CTA's p and share of p.v are visible
    T pv = T(0);
    for (int c = 0; c < C; ++c) pv += *cluster.map_shared_rank(pvpart, c);
    const T K = T(0.5) * tau_t * pv;
    for (int j = k + 1 + tid; j < m; j += nt) {
      const int oj = j / R;
      const T pj = cluster.map_shared_rank(pseg, oj)[j - oj * R];
      w[j] = fma(-K, v[j], pj);
    }
    __syncthreads();
    // J_ij -= v_i w_j + w_i v_j on the own rows i > k, one warp per row
    for (int i = i0 + warp; i < r1; i += nw) {
      T *row = slab + (size_t)(i - r0) * m;
      const T vi = v[i], wi = w[i];
      for (int j = k + 1 + lane; j < m; j += 32) row[j] = fma(-vi, w[j], fma(-wi, v[j], row[j]));
    }
    cluster.sync();   // the update is complete before the next row is read
  }
  // the trailing 2 x 2 block (read back by the eigenvalue kernel)
  for (int i = max(r0, m - 2) + tid; i < r1; i += nt)
    for (int j = m - 2; j <= i; ++j) t.A[(int64_t)i * m + j] = slab[(size_t)(i - r0) * m + j];
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
        while (cl_smem_bytes<T>(mm + 1, c) <= (size_t)lim) ++mm;
      table[dev][q] = mm;
    }
    ready[dev] = true;
  }
  const int q = C == 1 ? 0 : C == 2 ? 1 : C == 4 ? 2 : 3;
  return table[dev][q];
}

}  // namespace

// Clusters of several CTAs pay two cluster barriers and three rounds of
// distributed-shared-memory reads per step; on the 2D workloads they were
// slower than the step kernels, so only one-CTA nodes take this path unless
// HS_TRI_CLUSTER=2 (environment) allows up to eight CTAs.
template <typename T>
int tri_cluster_size(int m) {
  static const int cmax = [] {
    const char *e = std::getenv("HS_TRI_CLUSTER");
    return (e && e[0] == '2') ? 8 : 1;
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
