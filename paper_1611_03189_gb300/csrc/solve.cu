// Solve phase: the apply z = A_H^-1 r (Appendix A, Algorithm 2) and FP64
// preconditioned conjugate gradients around it.
//
// Workspace layout: one vector per level, level L first (the unknowns in
// cluster order), then the red nodes made at level L, ..., then the root; each
// unknown holds nrhs consecutive doubles.  A super node's unknowns at a level
// are the concatenation of its two children's, so super node and red nodes of
// a level share the same memory.
//
// Per wave (in elimination order) the forward pass runs
//   k_f1:  t_s = M_ss phi_s, phi_r += P_ss phi_s       (restriction)
//   k_f2:  phi_n -= sum_s A_ns t_s                     (forward substitution)
// then the root solve (k_copy, k_root), then per wave in reverse order
//   k_b1:  v_s = phi_s - sum_n A_sn x_n, y_s = P_ss^T x_r
//   k_b2:  x_s = M_ss v_s + y_s           (backward substitution and prolongation).
// Contributions to one phi_n are summed in a fixed order, so results do not
// depend on scheduling.
#include <algorithm>
#include <cmath>
#include <vector>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

#include "handle.h"

namespace hs {

namespace {

constexpr int AW = 8;         // warps per CTA in the apply kernels
constexpr int AT = AW * 32;

// last node i in nodes[first, first+count) with key(i) <= w (keys are prefix sums)
template <typename F>
__device__ __forceinline__ int find_last(int first, int count, int w, F key) {
  int lo = first, hi = first + count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (key(mid) <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// The same index, from a start known not to be past it (hint >= 0: the
// answer for the CTA's first warp): a forward scan over the few node
// boundaries inside the CTA's rows instead of a search of the whole wave.
template <typename F>
__device__ __forceinline__ int find_from(int first, int count, int w, int hint, F key) {
  if (hint < 0) return find_last(first, count, w, key);
  int i = hint;
  const int last = first + count - 1;
  while (i < last && key(i + 1) <= w) ++i;
  return i;
}

template <typename T, int NR>
__device__ __forceinline__ void warp_reduce(T (&acc)[NR]) {
#pragma unroll
  for (int j = 0; j < NR; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
}


// acc[j] += sum_c A[c] x[c*stride + j] for c = lane, lane+32, ... < len, four
// independent loads in flight per lane
template <typename T, int NR>
__device__ __forceinline__ void row_dot(const T *__restrict__ A, const T *__restrict__ x, int len,
                                        int64_t stride, int nr, int lane, T (&acc)[NR]) {
  int c = lane;
  for (; c + 96 < len; c += 128) {
    const T a0 = A[c], a1 = A[c + 32], a2 = A[c + 64], a3 = A[c + 96];
    const T *x0 = x + (int64_t)c * stride, *x1 = x0 + 32 * stride, *x2 = x0 + 64 * stride,
            *x3 = x0 + 96 * stride;
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (j < nr) acc[j] = fma(a3, x3[j], fma(a2, x2[j], fma(a1, x1[j], fma(a0, x0[j], acc[j]))));
  }
  for (; c < len; c += 32) {
    const T a = A[c];
    const T *xc = x + (int64_t)c * stride;
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (j < nr) acc[j] = fma(a, xc[j], acc[j]);
  }
}

// acc[j] += sum_q A[q*ld] t[q*stride + j] for q < len (column walk, unrolled by 4)
template <typename T, int NR>
__device__ __forceinline__ void col_dot(const T *__restrict__ A, int64_t ld, const T *__restrict__ t, int len,
                                        int64_t stride, int nr, T (&acc)[NR]) {
  int q = 0;
  for (; q + 3 < len; q += 4) {
    const T a0 = A[q * ld], a1 = A[(q + 1) * ld], a2 = A[(q + 2) * ld], a3 = A[(q + 3) * ld];
    const T *t0 = t + (int64_t)q * stride;
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (j < nr)
        acc[j] = fma(a3, t0[3 * stride + j], fma(a2, t0[2 * stride + j], fma(a1, t0[stride + j], fma(a0, t0[j], acc[j]))));
  }
  for (; q < len; ++q) {
    const T a = A[q * ld];
    const T *tq = t + (int64_t)q * stride;
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (j < nr) acc[j] = fma(a, tq[j], acc[j]);
  }
}

// Each step of Algorithm 2 below is a __device__ function of one warp's share
// (virtual warp w of the step); the per-step kernels give warp w = global warp
// index, the persistent kernel walks w over all warps of the grid.

// F1: one warp per row of [M_ss; P_ss]: t_s = M_ss phi_s, phi_r += P_ss phi_s
template <typename T, int NR>
__device__ __forceinline__ void f1_warp(const ApplyNode *__restrict__ nodes, int first, int count, int w, int lane,
                                        T *__restrict__ ws, T *__restrict__ tb, int nrhs, int j0, int hint = -1) {
  const int ni = find_from(first, count, w, hint, [&](int i) { return nodes[i].row0; });
  const ApplyNode nd = nodes[ni];
  const int r = w - nd.row0;
  const T *Ar = r < nd.m ? (const T *)nd.M + (int64_t)r * nd.m : (const T *)nd.P + (int64_t)(r - nd.m) * nd.m;
  const T *x = ws + nd.xs * nrhs + j0;
  const int nr = min(NR, nrhs - j0);
  T acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = T(0);
  row_dot<T, NR>(Ar, x, nd.m, nrhs, nr, lane, acc);
  warp_reduce<T, NR>(acc);
  if (lane == 0) {
    T *o = r < nd.m ? tb + (nd.toff + r) * nrhs + j0 : ws + (nd.xr + r - nd.m) * nrhs + j0;
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (j < nr) {
        if (r < nd.m)
          o[j] = acc[j];
        else
          o[j] += acc[j];
      }
  }
}

template <typename T, int NR>
__global__ void __launch_bounds__(AT) k_f1(const ApplyNode *__restrict__ nodes, int first, int count, int rows,
                                           T *__restrict__ ws, T *__restrict__ tb, int nrhs, int j0,
                                           const int *__restrict__ hint) {
  const int w = blockIdx.x * AW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w < rows) f1_warp<T, NR>(nodes, first, count, w, lane, ws, tb, nrhs, j0, hint ? hint[blockIdx.x] : -1);
}

// F2: phi_n -= sum_s A_ns t_s; one warp per 32 rows of a target, contributions in order
template <typename T, int NR>
__device__ __forceinline__ void f2_warp(const ApplyTarget *__restrict__ tg, int first, int count, int w, int lane,
                                        const ApplyContrib *__restrict__ cb, T *__restrict__ ws,
                                        const T *__restrict__ tb, int nrhs, int j0, int hint = -1) {
  const int ti = find_from(first, count, w, hint, [&](int i) { return tg[i].ch0; });
  const ApplyTarget t = tg[ti];
  const int i = (w - t.ch0) * 32 + lane;
  if (i >= t.size) return;
  const int nr = min(NR, nrhs - j0);
  T acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = T(0);
  for (int c = 0; c < t.count; ++c) {
    const ApplyContrib ac = cb[t.first + c];
    const T *A = (const T *)ac.A + i;
    const T *tv = tb + ac.toff * nrhs + j0;
    col_dot<T, NR>(A, ac.ld, tv, ac.m, nrhs, nr, acc);
  }
  T *o = ws + (t.x + i) * nrhs + j0;
#pragma unroll
  for (int j = 0; j < NR; ++j)
    if (j < nr) o[j] -= acc[j];
}

template <typename T, int NR>
__global__ void __launch_bounds__(AT) k_f2(const ApplyTarget *__restrict__ tg, int first, int count, int chunks,
                                           const ApplyContrib *__restrict__ cb, T *__restrict__ ws,
                                           const T *__restrict__ tb, int nrhs, int j0, const int *__restrict__ hint) {
  const int w = blockIdx.x * AW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w < chunks) f2_warp<T, NR>(tg, first, count, w, lane, cb, ws, tb, nrhs, j0, hint ? hint[blockIdx.x] : -1);
}

// B1 (warps < rows_b): v_s = phi_s - sum_n A_sn x_n, one warp per row of s.
// B2a (warps >= rows_b): y_s = P_ss^T x_r, one warp per 32 columns of P_ss.
template <typename T, int NR>
__device__ __forceinline__ void b1_warp(const ApplyNode *__restrict__ nodes, int first, int count, int rows_b,
                                        int w, int lane, const ApplyNbr *__restrict__ nb, const T *__restrict__ ws,
                                        T *__restrict__ tb, T *__restrict__ tb2, int nrhs, int j0, int hint_b = -1,
                                        int hint_p = -1) {
  const int nr = min(NR, nrhs - j0);
  T acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = T(0);
  if (w < rows_b) {
    const int ni = find_from(first, count, w, hint_b, [&](int i) { return nodes[i].brow0; });
    const ApplyNode nd = nodes[ni];
    const int r = w - nd.brow0;
    for (int b = 0; b < nd.nb_count; ++b) {
      const ApplyNbr n = nb[nd.nb_first + b];
      const T *Ar = (const T *)nd.AsN + (int64_t)r * nd.dN + n.col;
      const T *xn = ws + n.x * nrhs + j0;
      row_dot<T, NR>(Ar, xn, n.size, nrhs, nr, lane, acc);
    }
    warp_reduce<T, NR>(acc);
    if (lane == 0) {
      const T *ph = ws + (nd.xs + r) * nrhs + j0;
      T *o = tb + (nd.toff + r) * nrhs + j0;
#pragma unroll
      for (int j = 0; j < NR; ++j)
        if (j < nr) o[j] = ph[j] - acc[j];
    }
  } else {
    const int w2 = w - rows_b;
    const int ni = find_from(first, count, w2, hint_p, [&](int i) { return nodes[i].pch0; });
    const ApplyNode nd = nodes[ni];
    const int i = (w2 - nd.pch0) * 32 + lane;
    if (i >= nd.m || nd.k == 0) return;
    const T *P = (const T *)nd.P + i;
    const T *xr = ws + nd.xr * nrhs + j0;
    col_dot<T, NR>(P, nd.m, xr, nd.k, nrhs, nr, acc);
    T *o = tb2 + (nd.toff + i) * nrhs + j0;
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (j < nr) o[j] = acc[j];
  }
}

template <typename T, int NR>
__global__ void __launch_bounds__(AT) k_b1(const ApplyNode *__restrict__ nodes, int first, int count, int rows_b,
                                           int pch, const ApplyNbr *__restrict__ nb, const T *__restrict__ ws,
                                           T *__restrict__ tb, T *__restrict__ tb2, int nrhs, int j0,
                                           const int *__restrict__ hint_b, const int *__restrict__ hint_p) {
  const int w = blockIdx.x * AW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w < rows_b + pch)
    b1_warp<T, NR>(nodes, first, count, rows_b, w, lane, nb, ws, tb, tb2, nrhs, j0,
                   hint_b ? hint_b[blockIdx.x] : -1, hint_p ? hint_p[blockIdx.x] : -1);
}

// B2b: x_s = M_ss v_s + y_s, one warp per row of s
template <typename T, int NR>
__device__ __forceinline__ void b2_warp(const ApplyNode *__restrict__ nodes, int first, int count, int w, int lane,
                                        T *__restrict__ ws, const T *__restrict__ tb, const T *__restrict__ tb2,
                                        int nrhs, int j0, int hint = -1) {
  const int ni = find_from(first, count, w, hint, [&](int i) { return nodes[i].brow0; });
  const ApplyNode nd = nodes[ni];
  const int r = w - nd.brow0;
  const T *Mr = (const T *)nd.M + (int64_t)r * nd.m;
  const T *v = tb + nd.toff * nrhs + j0;
  const int nr = min(NR, nrhs - j0);
  T acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = T(0);
  row_dot<T, NR>(Mr, v, nd.m, nrhs, nr, lane, acc);
  warp_reduce<T, NR>(acc);
  if (lane == 0) {
    const T *y = tb2 + (nd.toff + r) * nrhs + j0;
    T *o = ws + (nd.xs + r) * nrhs + j0;
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (j < nr) o[j] = acc[j] + (nd.k > 0 ? y[j] : T(0));
  }
}

template <typename T, int NR>
__global__ void __launch_bounds__(AT) k_b2(const ApplyNode *__restrict__ nodes, int first, int count, int rows_b,
                                           T *__restrict__ ws, const T *__restrict__ tb,
                                           const T *__restrict__ tb2, int nrhs, int j0, const int *__restrict__ hint) {
  const int w = blockIdx.x * AW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w < rows_b) b2_warp<T, NR>(nodes, first, count, w, lane, ws, tb, tb2, nrhs, j0, hint ? hint[blockIdx.x] : -1);
}

template <typename T>
__global__ void k_copy(const T *__restrict__ src, T *__restrict__ dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

// root: x = A_root^-1 phi (phi copied to tb first), one warp per row
template <typename T, int NR>
__device__ __forceinline__ void root_warp(const T *__restrict__ Ainv, int m, int64_t off, int w, int lane,
                                          T *__restrict__ ws, const T *__restrict__ tb, int nrhs, int j0) {
  const T *Ar = Ainv + (int64_t)w * m;
  const int nr = min(NR, nrhs - j0);
  T acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = T(0);
  row_dot<T, NR>(Ar, tb + j0, m, nrhs, nr, lane, acc);
  warp_reduce<T, NR>(acc);
  if (lane == 0) {
    T *o = ws + (off + w) * nrhs + j0;
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (j < nr) o[j] = acc[j];
  }
}

template <typename T, int NR>
__global__ void __launch_bounds__(AT) k_root(const T *__restrict__ Ainv, int m, int64_t off,
                                             T *__restrict__ ws, const T *__restrict__ tb, int nrhs,
                                             int j0) {
  const int w = blockIdx.x * AW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w < m) root_warp<T, NR>(Ainv, m, off, w, lane, ws, tb, nrhs, j0);
}

// ---------------------------------------------------------------------------
// Persistent apply: the whole of Algorithm 2 for one chunk of right-hand sides
// in ONE cooperative launch.  The per-step launches above cost a launch
// latency per dependent step (about four per wave, some 240 at the 512 x 512
// workload); here every CTA of a grid sized to be resident walks the step
// list (forward f1, f2 per wave; root copy and solve; backward b1, b2 per
// wave in reverse), the warps of the grid sharing each step's virtual warps,
// with a grid-wide barrier between dependent steps.  The barrier is one
// arrival counter; its wait is bounded (clock cycles) and a wait that runs
// out sets *err and ends the kernel (the host reports HS_ERR_TIMEOUT).
// The steps and their arithmetic are those of the per-step kernels, so the
// result is the same bit for bit.
// ---------------------------------------------------------------------------
enum { AS_F1 = 0, AS_F2 = 1, AS_COPY = 2, AS_ROOT = 3, AS_B1 = 4, AS_B2 = 5 };

struct ApplyStepDev {
  int kind;
  int wave;          // index into the waves (f1, f2, b1, b2)
};

// Grid barrier number `round` (0, 1, ...): one counter that only grows; CTA
// thread 0 adds 1 with release semantics and waits, with acquire loads, until
// all CTAs of this and every earlier round have arrived.  The counter is
// cleared on the stream before each launch.
__device__ __forceinline__ unsigned atom_add_release_gpu(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// hs_test_wait_probe's switch for the persistent apply, per device
__device__ int g_apply_probe = 0;

__device__ bool grid_barrier(unsigned *bar, unsigned round, int *err, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = (round + 1u) * gridDim.x;
    atom_add_release_gpu(bar, 1u);
    const long long t0 = clock64();
    while (ld_acquire_gpu(bar) < target) {
      if (clock64() - t0 > limit) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T, int NR>
__global__ void __launch_bounds__(AT) k_apply_persistent(
    const ApplyStepDev *__restrict__ steps, int nsteps, const WaveApply *__restrict__ waves,
    const ApplyNode *__restrict__ nodes, const ApplyNbr *__restrict__ nbrs, const ApplyTarget *__restrict__ tg,
    const ApplyContrib *__restrict__ cb, const T *__restrict__ root_inv, int root_m, int64_t root_off,
    T *__restrict__ ws, T *__restrict__ tb, T *__restrict__ tb2, int nrhs, int j0, unsigned *bar, int *err,
    long long limit) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * AW + (threadIdx.x >> 5), nwarps = gridDim.x * AW;
  // test of the time-out path: a barrier round no launch can complete (the
  // switch is read at run time, so recorded graphs follow it too)
  if (g_apply_probe && !grid_barrier(bar, 1u << 20, err, limit)) return;
  for (int si = 0; si < nsteps; ++si) {
    const ApplyStepDev st = steps[si];
    if (st.kind == AS_COPY) {
      const int64_t n = (int64_t)root_m * nrhs;
      for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        tb[e] = ws[root_off * nrhs + e];
    } else if (st.kind == AS_ROOT) {
      for (int w = gw; w < root_m; w += nwarps) root_warp<T, NR>(root_inv, root_m, root_off, w, lane, ws, tb, nrhs, j0);
    } else {
      const WaveApply wa = waves[st.wave];
      if (st.kind == AS_F1) {
        for (int w = gw; w < wa.rows_f; w += nwarps)
          f1_warp<T, NR>(nodes, wa.node_first, wa.node_count, w, lane, ws, tb, nrhs, j0);
      } else if (st.kind == AS_F2) {
        for (int w = gw; w < wa.tch; w += nwarps)
          f2_warp<T, NR>(tg, wa.tgt_first, wa.tgt_count, w, lane, cb, ws, tb, nrhs, j0);
      } else if (st.kind == AS_B1) {
        for (int w = gw; w < wa.rows_b + wa.pch; w += nwarps)
          b1_warp<T, NR>(nodes, wa.node_first, wa.node_count, wa.rows_b, w, lane, nbrs, ws, tb, tb2, nrhs, j0);
      } else {
        for (int w = gw; w < wa.rows_b; w += nwarps)
          b2_warp<T, NR>(nodes, wa.node_first, wa.node_count, w, lane, ws, tb, tb2, nrhs, j0);
      }
    }
    if (si + 1 < nsteps && !grid_barrier(bar, (unsigned)si, err, limit)) return;
  }
}

// user layout (column-major, ld, FP64) <-> workspace layout (unknown-major, cluster order, T)
// ds (optional): D^-1/2 per cluster-order unknown of a scaled factorization
// (A_H^-1 = D^-1/2 A'_H^-1 D^-1/2), applied on the way in and on the way out
template <typename T>
__global__ void k_gather_in(const double *__restrict__ r, int64_t ld, const int32_t *__restrict__ perm,
                            int64_t n, int nrhs, int nrhs_p, T *__restrict__ out, const double *__restrict__ ds) {
  const int64_t total = n * nrhs_p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / nrhs_p;
    const int j = (int)(e - p * nrhs_p);
    const double v = j < nrhs ? r[(int64_t)perm[p] + j * ld] : 0.0;
    out[e] = (T)(ds ? v * ds[p] : v);
  }
}

template <typename T>
__global__ void k_scatter_out(const T *__restrict__ in, const int32_t *__restrict__ perm, int64_t n, int nrhs,
                              int nrhs_p, double *__restrict__ z, int64_t ld, const double *__restrict__ ds) {
  const int64_t total = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / nrhs;
    const int j = (int)(e - p * nrhs);
    const double v = (double)in[p * nrhs_p + j];
    z[(int64_t)perm[p] + j * ld] = ds ? v * ds[p] : v;
  }
}

// element-wise precision change between the FP64 PCG vectors (n x np,
// unknown-major) and the workspace, times ds[unknown] when scaling
template <typename A, typename B>
__global__ void k_convert(const A *__restrict__ a, B *__restrict__ b, int64_t n, int np,
                          const double *__restrict__ ds) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = ds ? (B)((double)a[e] * ds[e / np]) : (B)a[e];
}

// ---------------------------------------------------------------------------
// PCG kernels.  Vectors are n x NP (row-major, NP = right-hand sides rounded up
// to a power of two <= 32).  Every reduction visits the rows of one right-hand
// side in an order that depends on n alone: thread t of block b takes rows
// b*PT + t + k*gridDim*PT in turn, blocks reduce in a fixed tree, and the last
// block to finish adds the block partials in block order.  So a right-hand
// side gets the same bits whether it is solved alone or batched with others
// (the apply and the SpMV are column-wise already).
// ---------------------------------------------------------------------------
constexpr int PT = 256;

struct PcgScal {       // per-rhs scalars, each an array of NP doubles
  double *bnorm2, *rz, *alpha, *beta, *pq, *rr;
};
struct PcgFlags {
  int *active, *iters, *counter, *done;
};

// block sums of v[j] -> part[block*NP + j], in a fixed order
template <int NP>
__device__ void block_partial(const double (&v)[NP], double *part) {
  __shared__ double wsum[PT / 32][NP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    double s = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) wsum[warp][j] = s;
  }
  __syncthreads();
  if (threadIdx.x < NP) {
    double s = 0.0;
    for (int w = 0; w < PT / 32; ++w) s += wsum[w][threadIdx.x];
    part[blockIdx.x * NP + threadIdx.x] = s;
  }
}

// returns true in the last block to finish; sums[j] = ordered total
template <int NP>
__device__ bool finish_sum(const double *part, int *counter, double *sums) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  if (threadIdx.x < NP) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += ((volatile const double *)part)[b * NP + threadIdx.x];
    sums[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0;
  return true;
}

enum { DOT_BNORM = 0, DOT_RZ_FIRST = 1, DOT_RZ = 2, DOT_PLAIN = 3 };

template <int NP>
__global__ void __launch_bounds__(PT) k_dot(const double *__restrict__ u, const double *__restrict__ w, int64_t n,
                                            double *part, PcgScal sc, PcgFlags fl, int mode, double *plain_out) {
  __shared__ double sums[NP];
  double v[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) v[j] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)PT + threadIdx.x; i < n; i += (int64_t)gridDim.x * PT)
#pragma unroll
    for (int j = 0; j < NP; ++j) v[j] = fma(u[i * NP + j], w[i * NP + j], v[j]);
  block_partial<NP>(v, part);
  if (!finish_sum<NP>(part, fl.counter, sums)) return;
  const int j = threadIdx.x;
  if (j < NP) {
    const double s = sums[j];
    if (mode == DOT_BNORM) {
      sc.bnorm2[j] = s;
      fl.active[j] = s > 0.0 ? 1 : 0;
      fl.iters[j] = 0;
    } else if (mode == DOT_RZ_FIRST) {
      sc.beta[j] = 0.0;
      sc.rz[j] = s;
    } else if (mode == DOT_RZ) {
      sc.beta[j] = (fl.active[j] && sc.rz[j] != 0.0) ? s / sc.rz[j] : 0.0;
      sc.rz[j] = s;
    } else {
      plain_out[j] = s;
    }
  }
}

// p_new = z + beta p_old ; q = A p_new ; partial p_new . q ; alpha = rz / (p.q)
template <int NP>
__global__ void __launch_bounds__(PT) k_spmv_p(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                               const double *__restrict__ va, int64_t n,
                                               const double *__restrict__ z, const double *__restrict__ pold,
                                               double *__restrict__ pnew, double *__restrict__ q,
                                               double *part, PcgScal sc, PcgFlags fl) {
  __shared__ double sums[NP];
  double beta[NP], v[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    beta[j] = sc.beta[j];
    v[j] = 0.0;
  }
  for (int64_t i = blockIdx.x * (int64_t)PT + threadIdx.x; i < n; i += (int64_t)gridDim.x * PT) {
    double acc[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) acc[j] = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const double a = va[k];
      const int64_t c = (int64_t)ci[k] * NP;
#pragma unroll
      for (int j = 0; j < NP; ++j) acc[j] = fma(a, fma(beta[j], pold[c + j], z[c + j]), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const double pn = fma(beta[j], pold[i * NP + j], z[i * NP + j]);
      pnew[i * NP + j] = pn;
      q[i * NP + j] = acc[j];
      v[j] = fma(pn, acc[j], v[j]);
    }
  }
  block_partial<NP>(v, part);
  if (!finish_sum<NP>(part, fl.counter, sums)) return;
  const int j = threadIdx.x;
  if (j < NP) {
    sc.pq[j] = sums[j];
    sc.alpha[j] = (fl.active[j] && sums[j] != 0.0) ? sc.rz[j] / sums[j] : 0.0;
  }
}

// x += alpha p ; r -= alpha q ; partial ||r||^2 ; convergence per rhs
template <int NP>
__global__ void __launch_bounds__(PT) k_update(double *__restrict__ x, double *__restrict__ r,
                                               const double *__restrict__ p, const double *__restrict__ q, int64_t n,
                                               double *part, PcgScal sc, PcgFlags fl, double rtol2) {
  __shared__ double sums[NP];
  double alpha[NP], v[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    alpha[j] = sc.alpha[j];
    v[j] = 0.0;
  }
  for (int64_t i = blockIdx.x * (int64_t)PT + threadIdx.x; i < n; i += (int64_t)gridDim.x * PT)
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const int64_t e = i * NP + j;
      const double xv = fma(alpha[j], p[e], x[e]);
      const double rv = fma(-alpha[j], q[e], r[e]);
      x[e] = xv;
      r[e] = rv;
      v[j] = fma(rv, rv, v[j]);
    }
  block_partial<NP>(v, part);
  if (!finish_sum<NP>(part, fl.counter, sums)) return;
  const int j = threadIdx.x;
  if (j < NP) {
    sc.rr[j] = sums[j];
    if (fl.active[j]) {
      fl.iters[j] += 1;
      if (sums[j] <= rtol2 * sc.bnorm2[j]) fl.active[j] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0;
    for (int i = 0; i < NP; ++i) any |= fl.active[i];
    *fl.done = any ? 0 : 1;
  }
}

// calls f(std::integral_constant<int, NP>{}) for the power of two np <= 32
template <typename F>
void with_np(int np, F &&f) {
  switch (np) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 16: f(std::integral_constant<int, 16>{}); break;
    case 32: f(std::integral_constant<int, 32>{}); break;
    default: fail(HS_ERR_INVALID, "right-hand-side block must be a power of two <= 32");
  }
}

// q = b - A x
__global__ void k_residual(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ va, int64_t n, int nrhs_p,
                           const double *__restrict__ x, const double *__restrict__ b,
                           double *__restrict__ q) {
  const int64_t total = n * nrhs_p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nrhs_p;
    const int j = (int)(e - i * nrhs_p);
    double acc = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) acc = fma(va[k], x[(int64_t)ci[k] * nrhs_p + j], acc);
    q[e] = b[e] - acc;
  }
}

int grid_for(int64_t total) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
}

// grid of the PCG reduction kernels: a function of n only (see above)
int rgrid_for(int64_t n) { return grid_for(n); }

// a wave's per-CTA search starts (nullptr: the kernels search the whole wave)
inline const int *hint_at(const FactorHandle &h, int off) { return (h.d_hints && off >= 0) ? h.d_hints + off : nullptr; }

// One pass of Algorithm 2 over right-hand sides [j0, j0 + NR) of the
// workspace ws (layout [unknown][nrhs]); tb and tb2 are the per-wave scratch.
template <typename T, int NR>
void apply_waves_nr(const FactorHandle &h, T *ws, T *tb, T *tb2, int nrhs, int j0, cudaStream_t st) {
  auto blocks = [](int warps) { return (warps + AW - 1) / AW; };
  for (const LevelApply &la : h.levels)
    for (int w = la.wave_first; w < la.wave_first + la.wave_count; ++w) {
      const WaveApply &wa = h.waves[w];
      if (wa.rows_f) {
        k_f1<T, NR><<<blocks(wa.rows_f), AT, 0, st>>>(h.d_nodes, wa.node_first, wa.node_count, wa.rows_f, ws, tb,
                                                      nrhs, j0, hint_at(h, wa.hf1));
        count_launch();
      }
      if (wa.tch) {
        k_f2<T, NR><<<blocks(wa.tch), AT, 0, st>>>(h.d_targets, wa.tgt_first, wa.tgt_count, wa.tch, h.d_contribs,
                                                   ws, tb, nrhs, j0, hint_at(h, wa.hf2));
        count_launch();
      }
    }
  if (h.root_m > 0) {
    const int64_t cnt = (int64_t)h.root_m * nrhs;
    k_copy<T><<<(int)std::min<int64_t>((cnt + 255) / 256, 1024), 256, 0, st>>>(ws + h.root_off * nrhs, tb, cnt);
    k_root<T, NR><<<blocks(h.root_m), AT, 0, st>>>((const T *)h.root_inv, h.root_m, h.root_off, ws, tb, nrhs, j0);
    count_launch(2);
  }
  for (int li = (int)h.levels.size() - 1; li >= 0; --li) {
    const LevelApply &la = h.levels[li];
    for (int w = la.wave_first + la.wave_count - 1; w >= la.wave_first; --w) {
      const WaveApply &wa = h.waves[w];
      if (!wa.rows_b) continue;
      k_b1<T, NR><<<blocks(wa.rows_b + wa.pch), AT, 0, st>>>(h.d_nodes, wa.node_first, wa.node_count, wa.rows_b,
                                                             wa.pch, h.d_nbrs, ws, tb, tb2, nrhs, j0,
                                                             hint_at(h, wa.hb), hint_at(h, wa.hp));
      k_b2<T, NR><<<blocks(wa.rows_b), AT, 0, st>>>(h.d_nodes, wa.node_first, wa.node_count, wa.rows_b, ws, tb,
                                                    tb2, nrhs, j0, hint_at(h, wa.hb));
      count_launch(2);
    }
  }
  HS_CUDA(cudaGetLastError());
}

// The persistent apply is opt-in (HS_APPLY_PERSISTENT=1): on the 512 x 512
// workload its grid barriers cost more than the graph's launch gaps.
// HS_APPLY_PERSISTENT_BPS (1..4) sets the CTAs per SM.
bool persistent_apply_enabled() {
  static const bool on = [] {
    const char *e = std::getenv("HS_APPLY_PERSISTENT");
    return e && e[0] == '1';
  }();
  return on;
}
int persistent_apply_bps() {
  static const int v = [] {
    const char *e = std::getenv("HS_APPLY_PERSISTENT_BPS");
    const int b = e ? std::atoi(e) : 0;
    return b >= 1 && b <= 4 ? b : 0;
  }();
  return v;
}

// One chunk of right-hand sides [j0, j0 + NR) through the persistent kernel.
// The grid is the number of CTAs that can be resident at once (at most four
// per SM), launched cooperatively so that they are; the barrier words are
// cleared on the stream first.
template <typename T, int NR>
void apply_persistent_nr(const FactorHandle &h, T *ws, T *tb, T *tb2, int nrhs, int j0, cudaStream_t st) {
  static int blocks_per_sm[64] = {0};
  static std::mutex mu;
  int dev = 0;
  HS_CUDA(cudaGetDevice(&dev));
  int bps = 0, nsm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) fail(HS_ERR_CUDA, "device ordinal out of range");
    if (!blocks_per_sm[dev]) {
      int b = 0;
      HS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_apply_persistent<T, NR>, AT, 0));
      blocks_per_sm[dev] = std::max(1, std::min(b, persistent_apply_bps() ? persistent_apply_bps() : 4));
    }
    bps = blocks_per_sm[dev];
  }
  HS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  HS_CUDA(cudaMemsetAsync(h.d_apply_bar, 0, sizeof(unsigned), st));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nsm * bps), 1, 1);
  cfg.blockDim = dim3(AT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // about one second of SM clocks per barrier unless hs_opts.timeout_cycles says otherwise
  const long long limit = h.timeout_cycles > 0 ? (long long)h.timeout_cycles : 2000000000LL;
  HS_CUDA(cudaLaunchKernelEx(&cfg, k_apply_persistent<T, NR>, (const ApplyStepDev *)h.d_apply_steps,
                             h.apply_nsteps, (const WaveApply *)h.d_waves, (const ApplyNode *)h.d_nodes,
                             (const ApplyNbr *)h.d_nbrs, (const ApplyTarget *)h.d_targets,
                             (const ApplyContrib *)h.d_contribs, (const T *)h.root_inv, h.root_m, h.root_off, ws, tb,
                             tb2, nrhs, j0, h.d_apply_bar, h.d_apply_err, limit));
  count_launch();
}

template <typename T, int NR>
void apply_chunk_nr(const FactorHandle &h, T *ws, T *tb, T *tb2, int nrhs, int j0, cudaStream_t st) {
  if (persistent_apply_enabled() && h.d_apply_steps && h.apply_nsteps > 0)
    apply_persistent_nr<T, NR>(h, ws, tb, tb2, nrhs, j0, st);
  else
    apply_waves_nr<T, NR>(h, ws, tb, tb2, nrhs, j0, st);
}

// The whole apply on a workspace whose level-L part holds the right-hand
// sides: red-node parts cleared (Algorithm 2 starts them at zero), then the
// right-hand sides in chunks of at most 16 (register accumulators).
template <typename T>
void apply_chunks(const FactorHandle &h, T *ws, T *tb, T *tb2, int nrhs, cudaStream_t st) {
  const int64_t n = h.plan.n;
  if (h.ws_size > n) HS_CUDA(cudaMemsetAsync(ws + n * nrhs, 0, sizeof(T) * (h.ws_size - n) * nrhs, st));
  for (int j0 = 0; j0 < nrhs;) {
    const int rem = nrhs - j0;
    if (rem > 8) {
      apply_chunk_nr<T, 16>(h, ws, tb, tb2, nrhs, j0, st);
      j0 += 16;
    } else if (rem > 4) {
      apply_chunk_nr<T, 8>(h, ws, tb, tb2, nrhs, j0, st);
      j0 += 8;
    } else if (rem > 2) {
      apply_chunk_nr<T, 4>(h, ws, tb, tb2, nrhs, j0, st);
      j0 += 4;
    } else if (rem == 2) {
      apply_chunk_nr<T, 2>(h, ws, tb, tb2, nrhs, j0, st);
      j0 += 2;
    } else {
      apply_chunk_nr<T, 1>(h, ws, tb, tb2, nrhs, j0, st);
      j0 += 1;
    }
  }
}

// apply on the handle's workspace d_ws, launched directly
void apply_ws_direct(const FactorHandle &h, int nrhs, cudaStream_t st) {
  if (h.prec == HS_PREC_F64) {
    double *tb = (double *)h.d_t;
    apply_chunks<double>(h, (double *)h.d_ws, tb, tb + h.t_cap * h.nrhs_cap, nrhs, st);
  } else {
    float *tb = (float *)h.d_t;
    apply_chunks<float>(h, (float *)h.d_ws, tb, tb + h.t_cap * h.nrhs_cap, nrhs, st);
  }
}

// ---------------------------------------------------------------------------
// CUDA graphs.  One apply is about four dependent launches per wave (some 240
// at the 512 x 512 workload), each too short to hide its launch latency, so
// the launch sequence is recorded once per factorization and right-hand-side
// count and replayed with one cudaGraphLaunch.  Recording happens on a private
// stream of the handle in thread-local capture mode (other threads keep
// working); the graph is then launched on the caller's stream.  Graphs hold
// the handle's device pointers, so they are dropped whenever the schedule or
// the solve buffers change.  HS_APPLY_GRAPH=0 in the environment selects
// direct launches instead.
// ---------------------------------------------------------------------------
bool graphs_enabled() {
  static const bool on = [] {
    const char *e = std::getenv("HS_APPLY_GRAPH");
    return !(e && e[0] == '0');
  }();
  return on;
}

template <typename F>
const GraphEntry &graph_for(FactorHandle &h, int key, F &&record) {
  for (const GraphEntry &g : h.graphs)
    if (g.key == key) return g;
  if (!h.cap_stream) HS_CUDA(cudaStreamCreateWithFlags(&h.cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  HS_CUDA(cudaStreamBeginCapture(h.cap_stream, cudaStreamCaptureModeThreadLocal));
  try {
    CountPause pause;   // launches are counted when the graph runs
    record(h.cap_stream);
  } catch (...) {
    cudaStreamEndCapture(h.cap_stream, &graph);
    if (graph) cudaGraphDestroy(graph);
    throw;
  }
  HS_CUDA(cudaStreamEndCapture(h.cap_stream, &graph));
  size_t nn = 0;
  cudaError_t e = cudaGraphGetNodes(graph, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (e == cudaSuccess && nn) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
  int kernels = 0;
  for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
    cudaGraphNodeType t;
    e = cudaGraphNodeGetType(nodes[i], &t);
    kernels += (e == cudaSuccess && t == cudaGraphNodeTypeKernel) ? 1 : 0;
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  HS_CUDA(e);
  h.graphs.push_back(GraphEntry{key, exec, kernels});
  return h.graphs.back();
}

void run_graph(const GraphEntry &g, cudaStream_t st) {
  HS_CUDA(cudaGraphLaunch(g.exec, st));
  count_launch(g.kernels);
}

void apply_ws(FactorHandle &h, int nrhs, cudaStream_t st) {
  if (!graphs_enabled()) {
    apply_ws_direct(h, nrhs, st);
    return;
  }
  run_graph(graph_for(h, nrhs, [&](cudaStream_t cs) { apply_ws_direct(h, nrhs, cs); }), st);
}

void ensure_buffers(FactorHandle &h, int nrhs_cap, cudaStream_t st) {
  const int64_t tneed0 = std::max<int64_t>(std::max<int64_t>(h.tmax, h.root_m), 1);
  if (h.nrhs_cap >= nrhs_cap && h.d_ws && h.ws_cap >= h.ws_size && h.t_cap >= tneed0) return;
  nrhs_cap = std::max(nrhs_cap, h.nrhs_cap);
  h.drop_graphs();   // they hold the old buffers
  h.alloc.put(h.d_ws, st);
  h.alloc.put(h.d_t, st);
  h.alloc.put(h.d_pcg, st);
  h.alloc.put(h.d_part, st);
  h.alloc.put(h.d_scal, st);
  h.alloc.put(h.d_iflags, st);
  h.d_ws = h.d_t = h.d_pcg = h.d_part = h.d_scal = nullptr;
  h.d_iflags = nullptr;
  h.nrhs_cap = 0;   // until every buffer below exists (an allocation may fail)
  const int64_t n = h.plan.n;
  const size_t es = h.prec == HS_PREC_F64 ? sizeof(double) : sizeof(float);
  h.alloc.get(&h.d_ws, es * std::max<int64_t>(h.ws_size, 1) * nrhs_cap, st);
  const int64_t tneed = tneed0;
  h.alloc.get(&h.d_t, es * 2 * tneed * nrhs_cap, st);
  h.ws_cap = std::max<int64_t>(h.ws_size, 1);
  h.t_cap = tneed;
  h.alloc.get(&h.d_pcg, sizeof(double) * 7 * n * nrhs_cap, st);
  h.part_blocks = 152 * 8;
  h.alloc.get(&h.d_part, sizeof(double) * h.part_blocks * 32, st);
  h.alloc.get(&h.d_scal, sizeof(double) * 6 * 32, st);
  h.alloc.get(&h.d_iflags, sizeof(int) * (2 * 32 + 2), st);
  HS_CUDA(cudaMemset(h.d_iflags, 0, sizeof(int) * (2 * 32 + 2)));
  if (!h.h_done) HS_CUDA(cudaMallocHost(&h.h_done, sizeof(int)));
  h.nrhs_cap = nrhs_cap;
}

}  // namespace

void apply_prepare(FactorHandle &h, cudaStream_t st) {
  // the step list of Algorithm 2, in the order of the per-step launches
  std::vector<ApplyStepDev> steps;
  for (const LevelApply &la : h.levels)
    for (int w = la.wave_first; w < la.wave_first + la.wave_count; ++w) {
      if (h.waves[w].rows_f) steps.push_back(ApplyStepDev{AS_F1, w});
      if (h.waves[w].tch) steps.push_back(ApplyStepDev{AS_F2, w});
    }
  if (h.root_m > 0) {
    steps.push_back(ApplyStepDev{AS_COPY, 0});
    steps.push_back(ApplyStepDev{AS_ROOT, 0});
  }
  for (int li = (int)h.levels.size() - 1; li >= 0; --li) {
    const LevelApply &la = h.levels[li];
    for (int w = la.wave_first + la.wave_count - 1; w >= la.wave_first; --w) {
      if (!h.waves[w].rows_b) continue;
      steps.push_back(ApplyStepDev{AS_B1, w});
      steps.push_back(ApplyStepDev{AS_B2, w});
    }
  }
  // per-CTA search starts of the per-step kernels: for CTA b, the last node
  // (target) whose first row (chunk) is <= b AW, found by one sweep per key
  std::vector<int> hints;
  auto sweep = [&](int nrows, int first, int count, auto key) -> int {
    if (nrows <= 0 || count <= 0) return -1;
    const int off = (int)hints.size();
    const int nb = (nrows + AW - 1) / AW;
    int i = first;
    for (int b = 0; b < nb; ++b) {
      const int w0 = b * AW;
      while (i + 1 < first + count && key(i + 1) <= w0) ++i;
      hints.push_back(i);
    }
    return off;
  };
  for (WaveApply &wa : h.waves) {
    const ApplyNode *nd = h.nodes.data();
    const ApplyTarget *tg = h.targets.data();
    wa.hf1 = sweep(wa.rows_f, wa.node_first, wa.node_count, [&](int i) { return nd[i].row0; });
    wa.hf2 = sweep(wa.tch, wa.tgt_first, wa.tgt_count, [&](int i) { return tg[i].ch0; });
    // b1 runs blocks(rows_b + pch) CTAs: by brow0 for its first rows_b warps,
    // by pch0 for the rest (CTA b's first warp there: max(b AW - rows_b, 0))
    const int nb1 = (wa.rows_b + wa.pch + AW - 1) / AW;
    wa.hb = sweep(nb1 * AW, wa.node_first, wa.node_count, [&](int i) { return nd[i].brow0; });
    if (wa.pch > 0 && wa.node_count > 0) {
      wa.hp = (int)hints.size();
      int i = wa.node_first;
      for (int b = 0; b < nb1; ++b) {
        const int w2 = std::max(b * AW - wa.rows_b, 0);
        while (i + 1 < wa.node_first + wa.node_count && nd[i + 1].pch0 <= w2) ++i;
        hints.push_back(i);
      }
    } else {
      wa.hp = -1;
    }
  }
  if (hints.size() > h.hints_cap) {
    h.alloc.put(h.d_hints, st);
    h.d_hints = nullptr;
    h.alloc.get(&h.d_hints, sizeof(int) * hints.size(), st);
    h.hints_cap = hints.size();
  }
  if (!hints.empty())
    HS_CUDA(cudaMemcpyAsync(h.d_hints, hints.data(), sizeof(int) * hints.size(), cudaMemcpyHostToDevice, st));
  h.alloc.put(h.d_apply_steps, st);
  h.alloc.put(h.d_waves, st);
  h.d_apply_steps = nullptr;
  h.d_waves = nullptr;
  h.apply_nsteps = (int)steps.size();
  if (steps.empty()) return;
  h.alloc.get(&h.d_apply_steps, sizeof(ApplyStepDev) * steps.size(), st);
  HS_CUDA(cudaMemcpyAsync(h.d_apply_steps, steps.data(), sizeof(ApplyStepDev) * steps.size(), cudaMemcpyHostToDevice,
                          st));
  h.alloc.get(&h.d_waves, sizeof(WaveApply) * std::max<size_t>(h.waves.size(), 1), st);
  if (!h.waves.empty())
    HS_CUDA(cudaMemcpyAsync(h.d_waves, h.waves.data(), sizeof(WaveApply) * h.waves.size(), cudaMemcpyHostToDevice,
                            st));
  if (!h.d_apply_bar) {
    h.alloc.get(&h.d_apply_bar, 2 * sizeof(unsigned) + sizeof(int), st);
    HS_CUDA(cudaMemsetAsync(h.d_apply_bar, 0, 2 * sizeof(unsigned) + sizeof(int), st));
    h.d_apply_err = (int *)(h.d_apply_bar + 2);
  }
}

void set_apply_probe(bool on) {
  const int v = on ? 1 : 0;
  HS_CUDA(cudaMemcpyToSymbol(g_apply_probe, &v, sizeof(int)));
}

int apply_error(FactorHandle &h) {
  if (!h.d_apply_err) return 0;
  int e = 0;
  HS_CUDA(cudaMemcpy(&e, h.d_apply_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) HS_CUDA(cudaMemset(h.d_apply_err, 0, sizeof(int)));   // reported once
  return e;
}

void apply_solve(FactorHandle &h, const double *r, double *z, int nrhs, int64_t ld, cudaStream_t st) {
  ensure_buffers(h, std::max(nrhs, h.nrhs_cap), st);
  const int64_t n = h.plan.n;
  if (h.prec == HS_PREC_F64) {
    k_gather_in<double><<<grid_for(n * nrhs), 256, 0, st>>>(r, ld, h.d_perm, n, nrhs, nrhs, (double *)h.d_ws,
                                                            h.d_dscale);
    apply_ws(h, nrhs, st);
    k_scatter_out<double><<<grid_for(n * nrhs), 256, 0, st>>>((const double *)h.d_ws, h.d_perm, n, nrhs, nrhs, z, ld,
                                                              h.d_dscale);
  } else {
    k_gather_in<float><<<grid_for(n * nrhs), 256, 0, st>>>(r, ld, h.d_perm, n, nrhs, nrhs, (float *)h.d_ws,
                                                           h.d_dscale);
    apply_ws(h, nrhs, st);
    k_scatter_out<float><<<grid_for(n * nrhs), 256, 0, st>>>((const float *)h.d_ws, h.d_perm, n, nrhs, nrhs, z, ld,
                                                             h.d_dscale);
  }
  count_launch(2);
  HS_CUDA(cudaGetLastError());
}

namespace {

// z = A_H^-1 r on the FP64 PCG vectors (layout n x np): through the workspace
// in the factor precision
void apply_pcg(FactorHandle &h, const double *R, double *Z, int np, cudaStream_t st, bool direct) {
  const int64_t tot = h.plan.n * np;
  if (h.prec == HS_PREC_F64 && !h.scale) {
    HS_CUDA(cudaMemcpyAsync(h.d_ws, R, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
  } else if (h.prec == HS_PREC_F64) {
    k_convert<double, double><<<grid_for(tot), 256, 0, st>>>(R, (double *)h.d_ws, tot, np, h.d_dscale);
    count_launch();
  } else {
    k_convert<double, float><<<grid_for(tot), 256, 0, st>>>(R, (float *)h.d_ws, tot, np, h.d_dscale);
    count_launch();
  }
  if (direct)
    apply_ws_direct(h, np, st);
  else
    apply_ws(h, np, st);
  if (h.prec == HS_PREC_F64 && !h.scale) {
    HS_CUDA(cudaMemcpyAsync(Z, h.d_ws, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
  } else if (h.prec == HS_PREC_F64) {
    k_convert<double, double><<<grid_for(tot), 256, 0, st>>>((const double *)h.d_ws, Z, tot, np, h.d_dscale);
    count_launch();
  } else {
    k_convert<float, double><<<grid_for(tot), 256, 0, st>>>((const float *)h.d_ws, Z, tot, np, h.d_dscale);
    count_launch();
  }
}

}  // namespace

int pcg_solve(FactorHandle &h, const double *b, double *x, int nrhs, int64_t ld, double rtol,
              int maxit, int *iters, double *relres, cudaStream_t st) {
  int np = 1;
  while (np < nrhs) np <<= 1;
  ensure_buffers(h, std::max(np, h.nrhs_cap), st);
  const int64_t n = h.plan.n;
  const int64_t tot = n * np;
  double *X = h.d_pcg, *R = X + tot, *P0 = R + tot, *P1 = P0 + tot, *Q = P1 + tot, *B = Q + tot, *Z = B + tot;
  PcgScal sc{h.d_scal, h.d_scal + 32, h.d_scal + 64, h.d_scal + 96, h.d_scal + 128, h.d_scal + 160};
  PcgFlags fl{h.d_iflags, h.d_iflags + 32, h.d_iflags + 64, h.d_iflags + 65};
  const int g = rgrid_for(n);
  const double rtol2 = rtol * rtol;
  k_gather_in<double><<<grid_for(tot), 256, 0, st>>>(b, ld, h.d_perm, n, nrhs, np, B, nullptr);
  count_launch();
  HS_CUDA(cudaMemcpyAsync(R, B, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
  HS_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * tot, st));
  HS_CUDA(cudaMemsetAsync(P0, 0, sizeof(double) * tot, st));
  with_np(np, [&](auto c) {
    constexpr int NP = decltype(c)::value;
    k_dot<NP><<<g, PT, 0, st>>>(B, B, n, h.d_part, sc, fl, DOT_BNORM, nullptr);
  });
  count_launch();
  // z = A_H^-1 r ; first direction p = z (beta = 0)
  apply_pcg(h, R, Z, np, st, !graphs_enabled());
  with_np(np, [&](auto c) {
    constexpr int NP = decltype(c)::value;
    k_dot<NP><<<g, PT, 0, st>>>(R, Z, n, h.d_part, sc, fl, DOT_RZ_FIRST, nullptr);
    k_spmv_p<NP><<<g, PT, 0, st>>>(h.d_rowptr, h.d_col, h.d_val, n, Z, P0, P1, Q, h.d_part, sc, fl);
    k_update<NP><<<g, PT, 0, st>>>(X, R, P1, Q, n, h.d_part, sc, fl, rtol2);
  });
  count_launch(3);
  HS_CUDA(cudaGetLastError());
  // One iteration after the first: z = A_H^-1 r, beta, p_new = z + beta p_old,
  // q = A p_new, alpha, x and r updates.  Right-hand sides that have converged
  // get alpha = beta = 0 and stay as they are.  Recorded as a graph per
  // direction buffer pair.
  auto body = [&, np](cudaStream_t cs, double *pold, double *pnew) {
    apply_pcg(h, R, Z, np, cs, true);
    with_np(np, [&](auto c) {
      constexpr int NP = decltype(c)::value;
      k_dot<NP><<<g, PT, 0, cs>>>(R, Z, n, h.d_part, sc, fl, DOT_RZ, nullptr);
      k_spmv_p<NP><<<g, PT, 0, cs>>>(h.d_rowptr, h.d_col, h.d_val, n, Z, pold, pnew, Q, h.d_part, sc, fl);
      k_update<NP><<<g, PT, 0, cs>>>(X, R, pnew, Q, n, h.d_part, sc, fl, rtol2);
    });
    count_launch(3);
    HS_CUDA(cudaGetLastError());
  };
  int it = 1;
  while (true) {
    HS_CUDA(cudaMemcpyAsync(h.h_done, fl.done, sizeof(int), cudaMemcpyDeviceToHost, st));
    HS_CUDA(cudaStreamSynchronize(st));
    if (*h.h_done || it >= maxit) break;
    // after an odd number of iterations the latest direction is in P1
    double *pold = (it & 1) ? P1 : P0, *pnew = (it & 1) ? P0 : P1;
    if (graphs_enabled()) {
      const int key = kPcgGraphKey + 2 * np + (it & 1);
      run_graph(graph_for(h, key, [&](cudaStream_t cs) { body(cs, pold, pnew); }), st);
    } else {
      body(st, pold, pnew);
    }
    ++it;
  }
  // true relative residual
  k_residual<<<grid_for(tot), 256, 0, st>>>(h.d_rowptr, h.d_col, h.d_val, n, np, X, B, Q);
  count_launch();
  double *rr_d = h.d_scal + 5 * 32;
  with_np(np, [&](auto c) {
    constexpr int NP = decltype(c)::value;
    k_dot<NP><<<g, PT, 0, st>>>(Q, Q, n, h.d_part, sc, fl, DOT_PLAIN, rr_d);
  });
  count_launch();
  k_scatter_out<double><<<grid_for(n * nrhs), 256, 0, st>>>(X, h.d_perm, n, nrhs, np, x, ld, nullptr);
  count_launch();
  HS_CUDA(cudaGetLastError());
  std::vector<double> hs(6 * 32);
  std::vector<int> hi(2 * 32 + 2);
  HS_CUDA(cudaMemcpyAsync(hs.data(), h.d_scal, sizeof(double) * 6 * 32, cudaMemcpyDeviceToHost, st));
  HS_CUDA(cudaMemcpyAsync(hi.data(), h.d_iflags, sizeof(int) * (2 * 32 + 2), cudaMemcpyDeviceToHost, st));
  HS_CUDA(cudaStreamSynchronize(st));
  if (apply_error(h)) fail(HS_ERR_TIMEOUT, "a grid barrier of the persistent apply ran out");
  bool all = true;
  for (int j = 0; j < nrhs; ++j) {
    iters[j] = hi[32 + j];
    const double bn = hs[j];
    relres[j] = bn > 0 ? std::sqrt(hs[160 + j] / bn) : 0.0;
    all = all && hi[j] == 0;
  }
  return all ? HS_OK : HS_ERR_NO_CONVERGENCE;
}

// ---------------------------------------------------------------------------
// GMRES (hs_gmres): the outer solver of the paper's experiments (Sec. 7,
// Tables 2-5), right-preconditioned by A_H^-1, x_0 = 0, FP64.  Arnoldi on
// A A_H^-1 with classical Gram-Schmidt applied twice (two fused passes instead
// of the j + 1 dependent reductions of modified Gram-Schmidt); the Hessenberg
// least-squares problem by Givens rotations on the host, which reads one
// column of dot products per step.  Flexible form: the preconditioned vectors
// z_j = A_H^-1 v_j are kept and a cycle ends with x += Z y.  With an FP32
// factor each application of A_H^-1 rounds differently; x = A_H^-1 (V y)
// would then miss the Arnoldi relation A Z = V H by that rounding (a true
// residual near 1e-6 where the estimate says 1e-10), while A Z y stays exact.
// Reductions run in an order fixed by n alone.
// ---------------------------------------------------------------------------
namespace {

constexpr int GT = 256;

int gm_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 4095) / 4096, 128)); }

// part[i * gridDim.x + b] = block b's share of V_i . w, i = blockIdx.y < nv
__global__ void __launch_bounds__(GT) k_gm_dots(const double *__restrict__ V, int64_t n,
                                                const double *__restrict__ w, double *__restrict__ part) {
  __shared__ double ws[GT / 32];
  const double *v = V + (int64_t)blockIdx.y * n;
  double s = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)GT + threadIdx.x; k < n; k += (int64_t)gridDim.x * GT)
    s = fma(v[k], w[k], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < GT / 32; ++q) t += ws[q];
    part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// h[i] = sum over b of part[i * nb + b], one warp per i
__global__ void k_gm_sum(const double *__restrict__ part, int nb, int nv, double *__restrict__ h) {
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= nv) return;
  double s = 0.0;
  for (int b = lane; b < nb; b += 32) s += part[(int64_t)i * nb + b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) h[i] = s;
}

// w -= sum_{i < nv} h_i V_i
__global__ void k_gm_sub(const double *__restrict__ V, int64_t n, int nv, const double *__restrict__ h,
                         double *__restrict__ w) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double s = w[k];
    for (int i = 0; i < nv; ++i) s = fma(-h[i], V[(int64_t)i * n + k], s);
    w[k] = s;
  }
}

// u = sum_{i < nv} y_i V_i
__global__ void k_gm_comb(const double *__restrict__ V, int64_t n, int nv, const double *__restrict__ y,
                          double *__restrict__ u) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < nv; ++i) s = fma(y[i], V[(int64_t)i * n + k], s);
    u[k] = s;
  }
}

// v = a w ; x += z
__global__ void k_gm_scale(const double *__restrict__ w, int64_t n, double a, double *__restrict__ v) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    v[k] = a * w[k];
}
__global__ void k_gm_add(double *__restrict__ x, const double *__restrict__ z, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    x[k] += z[k];
}

// y = A x (permuted CSR)
__global__ void k_spmv(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ va,
                       int64_t n, const double *__restrict__ x, double *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) acc = fma(va[k], x[ci[k]], acc);
    y[i] = acc;
  }
}

// out[0 .. nv) = V_i . w for i < nv (device), through part
void gm_dots(const double *V, int64_t n, int nv, const double *w, double *part, double *out, cudaStream_t st) {
  const int nb = gm_blocks(n);
  k_gm_dots<<<dim3(nb, nv), GT, 0, st>>>(V, n, w, part);
  k_gm_sum<<<(nv * 32 + 255) / 256, 256, 0, st>>>(part, nb, nv, out);
  count_launch(2);
}

}  // namespace

int gmres_solve(FactorHandle &h, const double *b, double *x, double rtol, int maxit, int restart, int *iters,
                double *relres, cudaStream_t st) {
  ensure_buffers(h, std::max(1, h.nrhs_cap), st);
  const int64_t n = h.plan.n;
  const int mr = std::max(1, (restart > 0 && restart < maxit) ? restart : maxit);
  // V (mr + 1 vectors), Z (mr), w, u, X, B, R; part (mr + 1) x blocks; h1, h2,
  // |w|^2; y
  const int nb = gm_blocks(n);
  const size_t need = (size_t)(2 * mr + 6) * n + (size_t)(mr + 1) * nb + 2 * (size_t)(mr + 1) + 2 + (size_t)(mr + 1);
  if (h.gm_cap < need) {
    h.alloc.put(h.d_gm, st);
    h.d_gm = nullptr;
    h.gm_cap = 0;
    h.alloc.get(&h.d_gm, sizeof(double) * need, st);
    h.gm_cap = need;
  }
  double *V = h.d_gm, *Zm = V + (size_t)(mr + 1) * n, *W = Zm + (size_t)mr * n, *U = W + n, *X = U + n, *B = X + n,
         *R = B + n;
  double *part = R + n, *hd = part + (size_t)(mr + 1) * nb, *yd = hd + 2 * (size_t)(mr + 1) + 2;
  const int g = grid_for(n);
  k_gather_in<double><<<g, 256, 0, st>>>(b, n, h.d_perm, n, 1, 1, B, nullptr);
  count_launch();
  HS_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * n, st));
  std::vector<double> hh(2 * (size_t)(mr + 1) + 2);
  auto read = [&](int cnt) {
    HS_CUDA(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    HS_CUDA(cudaStreamSynchronize(st));
  };
  gm_dots(B, n, 1, B, part, hd, st);
  read(1);
  const double bnorm = std::sqrt(hh[0]);
  int total = 0;
  bool converged = bnorm == 0.0;
  // Hessenberg (column-major, ld mr + 1), Givens rotations, rotated rhs
  std::vector<double> H((size_t)(mr + 1) * mr), cs(mr), sn(mr), gv(mr + 1), y(mr);
  while (!converged && total < maxit) {
    // r = b - A x; v_0 = r / |r|
    if (total == 0) {
      HS_CUDA(cudaMemcpyAsync(R, B, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    } else {
      k_residual<<<g, 256, 0, st>>>(h.d_rowptr, h.d_col, h.d_val, n, 1, X, B, R);
      count_launch();
    }
    gm_dots(R, n, 1, R, part, hd, st);
    read(1);
    const double beta = std::sqrt(hh[0]);
    if (beta < rtol * bnorm) {
      converged = true;
      break;
    }
    k_gm_scale<<<g, 256, 0, st>>>(R, n, 1.0 / beta, V);
    count_launch();
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int j = 0;
    for (; j < mr && total < maxit; ++j) {
      // z_j = A_H^-1 v_j ; w = A z_j
      double *zj = Zm + (size_t)j * n;
      apply_pcg(h, V + (size_t)j * n, zj, 1, st, !graphs_enabled());
      k_spmv<<<g, 256, 0, st>>>(h.d_rowptr, h.d_col, h.d_val, n, zj, W);
      count_launch();
      // two passes of classical Gram-Schmidt, then |w|^2
      double *h1 = hd, *h2 = hd + (mr + 1);
      gm_dots(V, n, j + 1, W, part, h1, st);
      k_gm_sub<<<g, 256, 0, st>>>(V, n, j + 1, h1, W);
      gm_dots(V, n, j + 1, W, part, h2, st);
      k_gm_sub<<<g, 256, 0, st>>>(V, n, j + 1, h2, W);
      gm_dots(W, n, 1, W, part, hd + 2 * (mr + 1), st);
      count_launch(2);
      HS_CUDA(cudaGetLastError());
      HS_CUDA(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * (2 * (mr + 1) + 1), cudaMemcpyDeviceToHost, st));
      HS_CUDA(cudaStreamSynchronize(st));
      double *col = &H[(size_t)j * (mr + 1)];
      for (int i = 0; i <= j; ++i) col[i] = hh[i] + hh[(mr + 1) + i];
      const double hn = std::sqrt(hh[2 * (mr + 1)]);
      col[j + 1] = hn;
      ++total;
      // previous rotations, then the one that zeroes col[j + 1]
      for (int i = 0; i < j; ++i) {
        const double a = col[i], c = col[i + 1];
        col[i] = cs[i] * a + sn[i] * c;
        col[i + 1] = -sn[i] * a + cs[i] * c;
      }
      const double den = std::hypot(col[j], col[j + 1]);
      cs[j] = den > 0.0 ? col[j] / den : 1.0;
      sn[j] = den > 0.0 ? col[j + 1] / den : 0.0;
      col[j] = den;
      col[j + 1] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      if (std::fabs(gv[j + 1]) < rtol * bnorm || hn == 0.0) {
        converged = true;
        ++j;
        break;
      }
      if (j + 1 < mr && total < maxit) {
        k_gm_scale<<<g, 256, 0, st>>>(W, n, 1.0 / hn, V + (size_t)(j + 1) * n);
        count_launch();
      }
    }
    // y = R^-1 g (upper triangular, j columns); x += Z y
    const int k = j;
    for (int i = k - 1; i >= 0; --i) {
      double s = gv[i];
      for (int c = i + 1; c < k; ++c) s -= H[(size_t)c * (mr + 1) + i] * y[c];
      const double d = H[(size_t)i * (mr + 1) + i];
      y[i] = d != 0.0 ? s / d : 0.0;
    }
    HS_CUDA(cudaMemcpyAsync(yd, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
    k_gm_comb<<<g, 256, 0, st>>>(Zm, n, k, yd, U);
    count_launch();
    k_gm_add<<<g, 256, 0, st>>>(X, U, n);
    count_launch();
    HS_CUDA(cudaGetLastError());
  }
  // true relative residual, x back to the original order
  k_residual<<<g, 256, 0, st>>>(h.d_rowptr, h.d_col, h.d_val, n, 1, X, B, R);
  count_launch();
  gm_dots(R, n, 1, R, part, hd, st);
  read(1);
  k_scatter_out<double><<<g, 256, 0, st>>>(X, h.d_perm, n, 1, 1, x, n, nullptr);
  count_launch();
  HS_CUDA(cudaGetLastError());
  HS_CUDA(cudaStreamSynchronize(st));
  if (apply_error(h)) fail(HS_ERR_TIMEOUT, "a grid barrier of the persistent apply ran out");
  *iters = total;
  *relres = bnorm > 0.0 ? std::sqrt(hh[0]) / bnorm : 0.0;
  return converged ? HS_OK : HS_ERR_NO_CONVERGENCE;
}

// ---------------------------------------------------------------------------
// Allocation-free apply (hs_apply_static).  Some callers cannot allocate device
// memory when they solve: a service that fixes its device-memory footprint at
// start-up, or code running where a cudaMalloc could block behind other work
// or is not permitted.  For them
// the apply workspace comes from one file-scope device array instead of the
// handle's lazily grown buffers.  The array is shared by every call on a
// device and keeps the previous call's contents; calls that overlap on the
// GPU race on it.
// ---------------------------------------------------------------------------
constexpr size_t kStaticApplyBytes = size_t(16) << 20;   // 16 MiB per device
static __device__ __align__(256) unsigned char g_static_apply_ws[kStaticApplyBytes];

namespace {

std::mutex g_static_mu;
void *g_static_ptr[64] = {nullptr};

// Device address of the array for the current device.  Outside a stream
// capture it is looked up on every call (with the device current), so a
// device reset or a new primary context never leaves a stale address behind;
// while `st` is capturing, the address cached by the last call outside a
// capture is used, and a device that has none yet is an error.
void *static_ws_for_current_device(cudaStream_t st) {
  int dev = 0;
  HS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) fail(HS_ERR_CUDA, "device ordinal out of range for the static apply buffer");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t ce = cudaStreamIsCapturing(st, &cs);
  const bool capturing = ce != cudaSuccess || cs != cudaStreamCaptureStatusNone;
  if (ce != cudaSuccess) cudaGetLastError();   // a query error is not sticky; clear it
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!capturing) {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_apply_ws);
    if (e != cudaSuccess || !ptr)
      fail(HS_ERR_CUDA, std::string("cudaGetSymbolAddress of the static apply buffer: ") + cudaGetErrorString(e));
    g_static_ptr[dev] = ptr;
  } else if (!g_static_ptr[dev]) {
    fail(HS_ERR_INVALID, "hs_apply_static: the first call on a device must come before any stream capture");
  }
  return g_static_ptr[dev];
}

template <typename T>
void apply_static_t(FactorHandle &h, const double *r, double *z, int nrhs, int64_t ld, cudaStream_t st) {
  const int64_t n = h.plan.n;
  const int64_t tcap = std::max<int64_t>(std::max<int64_t>(h.tmax, h.root_m), 1);
  // layout: workspace (ws_size x nrhs), t (tcap x nrhs), second t (tcap x nrhs), 256-byte aligned parts
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t ws_b = up(sizeof(T) * (size_t)h.ws_size * nrhs);
  const size_t t_b = up(sizeof(T) * (size_t)tcap * nrhs);
  const size_t need = ws_b + 2 * t_b;
  if (need > kStaticApplyBytes)
    fail(HS_ERR_CAPACITY, "hs_apply_static needs " + std::to_string(need) + " bytes of workspace for this factor and " +
                              std::to_string(nrhs) + " right-hand sides; the static buffer holds " +
                              std::to_string(kStaticApplyBytes) + " bytes");
  unsigned char *base = (unsigned char *)static_ws_for_current_device(st);
  T *ws = (T *)base, *tb = (T *)(base + ws_b), *tb2 = (T *)(base + ws_b + t_b);
  k_gather_in<T><<<grid_for(n * nrhs), 256, 0, st>>>(r, ld, h.d_perm, n, nrhs, nrhs, ws, h.d_dscale);
  count_launch();
  apply_chunks<T>(h, ws, tb, tb2, nrhs, st);
  k_scatter_out<T><<<grid_for(n * nrhs), 256, 0, st>>>(ws, h.d_perm, n, nrhs, nrhs, z, ld, h.d_dscale);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

}  // namespace

void apply_static(FactorHandle &h, const double *r, double *z, int nrhs, int64_t ld, cudaStream_t st) {
  if (h.prec == HS_PREC_F64)
    apply_static_t<double>(h, r, z, nrhs, ld, st);
  else
    apply_static_t<float>(h, r, z, nrhs, ld, st);
}

FactorHandle::~FactorHandle() {
  drop_graphs();
  if (cap_stream) cudaStreamDestroy(cap_stream);
  if (h_done) cudaFreeHost(h_done);
  alloc.put(d_src, stream);
  alloc.put(d_leaf_dest, stream);
  alloc.put(d_phi0, stream);
  alloc.put(d_phi_raw, stream);
  alloc.put(d_apply_steps, stream);
  alloc.put(d_waves, stream);
  alloc.put(d_apply_bar, stream);
  alloc.put(d_hints, stream);
  alloc.put(d_dscale, stream);
  alloc.put(d_val_f, stream);
  alloc.put(d_flag, stream);
  alloc.put(d_rowptr, stream);
  alloc.put(d_col, stream);
  alloc.put(d_val, stream);
  alloc.put(d_perm, stream);
  alloc.put(d_nodes, stream);
  alloc.put(d_nbrs, stream);
  alloc.put(d_targets, stream);
  alloc.put(d_contribs, stream);
  alloc.put(d_ws, stream);
  alloc.put(d_t, stream);
  alloc.put(d_pcg, stream);
  alloc.put(d_gm, stream);
  alloc.put(d_part, stream);
  alloc.put(d_scal, stream);
  alloc.put(d_iflags, stream);
}

}  // namespace hs
