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
//   k_fwd_node:   t_s = M_ss phi_s, phi_r += P_ss phi_s      (restriction)
//   k_fwd_target: phi_n -= sum_s A_ns t_s                    (forward substitution)
// then the root solve, then per wave in reverse order
//   k_bwd_node:   x_s = M_ss (phi_s - sum_n A_sn x_n) + P_ss^T x_r
//                                        (backward substitution and prolongation).
// Contributions to one phi_n are summed in a fixed order, so results do not
// depend on scheduling.
#include <algorithm>
#include <cstring>

#include "handle.h"

namespace hs {

namespace {

constexpr int AT = 256;     // threads of the apply kernels
constexpr int MAXR = 16;    // right-hand sides per register pass

template <typename T>
__global__ void __launch_bounds__(AT) k_fwd_node(const ApplyNode *__restrict__ nodes, int first,
                                                 double *__restrict__ ws, double *__restrict__ tb,
                                                 int nrhs) {
  const ApplyNode nd = nodes[first + blockIdx.x];
  const T *M = (const T *)nd.M;
  const T *P = (const T *)nd.P;
  const double *phs = ws + nd.xs * nrhs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int rows = nd.m + nd.k;
  for (int row = warp; row < rows; row += nw) {
    const T *Ar = row < nd.m ? M + (int64_t)row * nd.m : P + (int64_t)(row - nd.m) * nd.m;
    for (int j0 = 0; j0 < nrhs; j0 += MAXR) {
      const int nr = min(MAXR, nrhs - j0);
      double acc[MAXR];
#pragma unroll
      for (int j = 0; j < MAXR; ++j) acc[j] = 0.0;
      for (int c = lane; c < nd.m; c += 32) {
        const double a = (double)Ar[c];
        const double *x = phs + (int64_t)c * nrhs + j0;
#pragma unroll
        for (int j = 0; j < MAXR; ++j)
          if (j < nr) acc[j] = fma(a, x[j], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < MAXR; ++j)
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
      if (lane == 0) {
        if (row < nd.m) {
          double *o = tb + (nd.toff + row) * nrhs + j0;
          for (int j = 0; j < nr; ++j) o[j] = acc[j];
        } else {
          double *o = ws + (nd.xr + row - nd.m) * nrhs + j0;
          for (int j = 0; j < nr; ++j) o[j] += acc[j];
        }
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(AT) k_fwd_target(const ApplyTarget *__restrict__ tg, int first,
                                                   const ApplyContrib *__restrict__ cb,
                                                   double *__restrict__ ws,
                                                   const double *__restrict__ tb, int nrhs) {
  const ApplyTarget t = tg[first + blockIdx.x];
  const int total = t.size * nrhs;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int i = e / nrhs, j = e - (e / nrhs) * nrhs;
    double acc = 0.0;
    for (int c = 0; c < t.count; ++c) {
      const ApplyContrib ac = cb[t.first + c];
      const T *A = (const T *)ac.A;
      const double *tv = tb + ac.toff * nrhs + j;
      for (int q = 0; q < ac.m; ++q) acc = fma((double)A[(int64_t)q * ac.ld + i], tv[(int64_t)q * nrhs], acc);
    }
    ws[(t.x + i) * nrhs + j] -= acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(AT) k_bwd_node(const ApplyNode *__restrict__ nodes, int first,
                                                 const ApplyNbr *__restrict__ nb,
                                                 double *__restrict__ ws, double *__restrict__ tb,
                                                 int nrhs) {
  const ApplyNode nd = nodes[first + blockIdx.x];
  const T *M = (const T *)nd.M;
  const T *P = (const T *)nd.P;
  const T *AsN = (const T *)nd.AsN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double *v = tb + nd.toff * nrhs;
  // v = phi_s - sum_n A_sn x_n
  for (int row = warp; row < nd.m; row += nw) {
    for (int j0 = 0; j0 < nrhs; j0 += MAXR) {
      const int nr = min(MAXR, nrhs - j0);
      double acc[MAXR];
#pragma unroll
      for (int j = 0; j < MAXR; ++j) acc[j] = 0.0;
      for (int b = 0; b < nd.nb_count; ++b) {
        const ApplyNbr n = nb[nd.nb_first + b];
        const T *Ar = AsN + (int64_t)row * nd.dN + n.col;
        const double *xn = ws + n.x * nrhs + j0;
        for (int q = lane; q < n.size; q += 32) {
          const double a = (double)Ar[q];
#pragma unroll
          for (int j = 0; j < MAXR; ++j)
            if (j < nr) acc[j] = fma(a, xn[(int64_t)q * nrhs + j], acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < MAXR; ++j)
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
      if (lane == 0) {
        const double *ph = ws + (nd.xs + row) * nrhs + j0;
        for (int j = 0; j < nr; ++j) v[(int64_t)row * nrhs + j0 + j] = ph[j] - acc[j];
      }
    }
  }
  __syncthreads();
  // x_s = M_ss v + P_ss^T x_r
  for (int row = warp; row < nd.m; row += nw) {
    for (int j0 = 0; j0 < nrhs; j0 += MAXR) {
      const int nr = min(MAXR, nrhs - j0);
      double acc[MAXR];
#pragma unroll
      for (int j = 0; j < MAXR; ++j) acc[j] = 0.0;
      const T *Mr = M + (int64_t)row * nd.m;
      for (int c = lane; c < nd.m; c += 32) {
        const double a = (double)Mr[c];
        const double *x = v + (int64_t)c * nrhs + j0;
#pragma unroll
        for (int j = 0; j < MAXR; ++j)
          if (j < nr) acc[j] = fma(a, x[j], acc[j]);
      }
      if (nd.k > 0) {
        const double *xr = ws + nd.xr * nrhs + j0;
        for (int q = lane; q < nd.k; q += 32) {
          const double a = (double)P[(int64_t)q * nd.m + row];
#pragma unroll
          for (int j = 0; j < MAXR; ++j)
            if (j < nr) acc[j] = fma(a, xr[(int64_t)q * nrhs + j], acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < MAXR; ++j)
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
      if (lane == 0) {
        double *o = ws + (nd.xs + row) * nrhs + j0;
        for (int j = 0; j < nr; ++j) o[j] = acc[j];
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(AT) k_root(const T *__restrict__ Ainv, int m, int64_t off,
                                             double *__restrict__ ws, double *__restrict__ tb,
                                             int nrhs) {
  for (int64_t e = threadIdx.x; e < (int64_t)m * nrhs; e += blockDim.x) tb[e] = ws[off * nrhs + e];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = warp; row < m; row += nw) {
    for (int j0 = 0; j0 < nrhs; j0 += MAXR) {
      const int nr = min(MAXR, nrhs - j0);
      double acc[MAXR];
#pragma unroll
      for (int j = 0; j < MAXR; ++j) acc[j] = 0.0;
      const T *Ar = Ainv + (int64_t)row * m;
      for (int c = lane; c < m; c += 32) {
        const double a = (double)Ar[c];
#pragma unroll
        for (int j = 0; j < MAXR; ++j)
          if (j < nr) acc[j] = fma(a, tb[(int64_t)c * nrhs + j0 + j], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < MAXR; ++j)
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
      if (lane == 0)
        for (int j = 0; j < nr; ++j) ws[(off + row) * nrhs + j0 + j] = acc[j];
    }
  }
}

// user layout (column-major, ld) <-> workspace layout (unknown-major, cluster order)
__global__ void k_gather_in(const double *__restrict__ r, int64_t ld, const int32_t *__restrict__ perm,
                            int64_t n, int nrhs, int nrhs_p, double *__restrict__ out) {
  const int64_t total = n * nrhs_p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / nrhs_p;
    const int j = (int)(e - p * nrhs_p);
    out[e] = j < nrhs ? r[(int64_t)perm[p] + j * ld] : 0.0;
  }
}

__global__ void k_scatter_out(const double *__restrict__ in, const int32_t *__restrict__ perm,
                              int64_t n, int nrhs, int nrhs_p, double *__restrict__ z, int64_t ld) {
  const int64_t total = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / nrhs;
    const int j = (int)(e - p * nrhs);
    z[(int64_t)perm[p] + j * ld] = in[p * nrhs_p + j];
  }
}

// ---------------------------------------------------------------------------
// PCG kernels.  nrhs_p is a power of two <= 32; element e = (row, rhs) with the
// rhs fastest.  Block partial sums are reduced by the last block to finish, in
// block order, so every reduction is deterministic.
// ---------------------------------------------------------------------------
constexpr int PT = 256;

struct PcgScal {       // per-rhs scalars, each an array of nrhs_p doubles
  double *bnorm2, *rz, *alpha, *beta, *pq, *rr;
};
struct PcgFlags {
  int *active, *iters, *counter, *done;
};

// block partial of v (one value per thread, rhs = e % nrhs_p) -> part[block*nrhs_p + j]
__device__ void block_partial(double v, int nrhs_p, double *part) {
  __shared__ double wsum[PT / 32][32];
  for (int o = 16; o >= nrhs_p; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane < nrhs_p) wsum[warp][lane] = v;
  __syncthreads();
  if (threadIdx.x < nrhs_p) {
    // warps cover consecutive element ranges, lane j of each warp holds rhs j
    double s = 0.0;
    for (int w = 0; w < PT / 32; ++w) s += wsum[w][threadIdx.x];
    part[blockIdx.x * nrhs_p + threadIdx.x] = s;
  }
}

// returns true in the last block to finish; sums[j] = ordered total
__device__ bool finish_sum(const double *part, int nrhs_p, int *counter, double *sums) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  if (threadIdx.x < nrhs_p) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += ((volatile const double *)part)[b * nrhs_p + threadIdx.x];
    sums[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0;
  return true;
}

enum { DOT_BNORM = 0, DOT_RZ_FIRST = 1, DOT_RZ = 2, DOT_PLAIN = 3 };

__global__ void __launch_bounds__(PT) k_dot(const double *__restrict__ u, const double *__restrict__ w,
                                            int64_t n, int nrhs_p, double *part, PcgScal sc,
                                            PcgFlags fl, int mode, double *plain_out) {
  __shared__ double sums[32];
  double v = 0.0;
  const int64_t total = n * nrhs_p;
  // each thread walks e = base + k * stride with stride a multiple of nrhs_p, so its rhs is fixed
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    v = fma(u[e], w[e], v);
  block_partial(v, nrhs_p, part);
  if (!finish_sum(part, nrhs_p, fl.counter, sums)) return;
  const int j = threadIdx.x;
  if (j < nrhs_p) {
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
__global__ void __launch_bounds__(PT) k_spmv_p(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                               const double *__restrict__ va, int64_t n, int nrhs_p,
                                               const double *__restrict__ z, const double *__restrict__ pold,
                                               double *__restrict__ pnew, double *__restrict__ q,
                                               double *part, PcgScal sc, PcgFlags fl) {
  __shared__ double sums[32];
  double v = 0.0;
  const int64_t total = n * nrhs_p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nrhs_p;
    const int j = (int)(e - i * nrhs_p);
    const double b = sc.beta[j];
    double acc = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t c = (int64_t)ci[k] * nrhs_p + j;
      acc = fma(va[k], fma(b, pold[c], z[c]), acc);
    }
    const double pn = fma(b, pold[e], z[e]);
    pnew[e] = pn;
    q[e] = acc;
    v = fma(pn, acc, v);
  }
  block_partial(v, nrhs_p, part);
  if (!finish_sum(part, nrhs_p, fl.counter, sums)) return;
  const int j = threadIdx.x;
  if (j < nrhs_p) {
    sc.pq[j] = sums[j];
    sc.alpha[j] = (fl.active[j] && sums[j] != 0.0) ? sc.rz[j] / sums[j] : 0.0;
  }
}

// x += alpha p ; r -= alpha q ; partial ||r||^2 ; convergence per rhs
__global__ void __launch_bounds__(PT) k_update(double *__restrict__ x, double *__restrict__ r,
                                               const double *__restrict__ p, const double *__restrict__ q,
                                               int64_t n, int nrhs_p, double *part, PcgScal sc,
                                               PcgFlags fl, double rtol2) {
  __shared__ double sums[32];
  double v = 0.0;
  const int64_t total = n * nrhs_p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % nrhs_p);
    const double a = sc.alpha[j];
    const double xv = fma(a, p[e], x[e]);
    const double rv = fma(-a, q[e], r[e]);
    x[e] = xv;
    r[e] = rv;
    v = fma(rv, rv, v);
  }
  block_partial(v, nrhs_p, part);
  if (!finish_sum(part, nrhs_p, fl.counter, sums)) return;
  const int j = threadIdx.x;
  if (j < nrhs_p) {
    sc.rr[j] = sums[j];
    if (fl.active[j]) {
      fl.iters[j] += 1;
      if (sums[j] <= rtol2 * sc.bnorm2[j]) fl.active[j] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0;
    for (int i = 0; i < nrhs_p; ++i) any |= fl.active[i];
    *fl.done = any ? 0 : 1;
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

// grid for the reduction kernels: stride (grid * PT) must be a multiple of nrhs_p
int rgrid_for(int64_t total) { return grid_for(total); }

template <typename T>
void apply_ws_t(FactorHandle &h, int nrhs, cudaStream_t st) {
  double *ws = h.d_ws;
  const int64_t n = h.plan.n;
  if (h.ws_size > n)
    HS_CUDA(cudaMemsetAsync(ws + n * nrhs, 0, sizeof(double) * (h.ws_size - n) * nrhs, st));
  for (const LevelApply &la : h.levels)
    for (int w = la.wave_first; w < la.wave_first + la.wave_count; ++w) {
      const WaveApply &wa = h.waves[w];
      if (wa.node_count) k_fwd_node<T><<<wa.node_count, AT, 0, st>>>(h.d_nodes, wa.node_first, ws, h.d_t, nrhs);
      if (wa.tgt_count)
        k_fwd_target<T><<<wa.tgt_count, AT, 0, st>>>(h.d_targets, wa.tgt_first, h.d_contribs, ws, h.d_t, nrhs);
    }
  if (h.root_m > 0)
    k_root<T><<<1, AT, 0, st>>>((const T *)h.root_inv, h.root_m, h.root_off, ws, h.d_t, nrhs);
  for (int li = (int)h.levels.size() - 1; li >= 0; --li) {
    const LevelApply &la = h.levels[li];
    for (int w = la.wave_first + la.wave_count - 1; w >= la.wave_first; --w) {
      const WaveApply &wa = h.waves[w];
      if (wa.node_count)
        k_bwd_node<T><<<wa.node_count, AT, 0, st>>>(h.d_nodes, wa.node_first, h.d_nbrs, ws, h.d_t, nrhs);
    }
  }
  HS_CUDA(cudaGetLastError());
}

void apply_ws(FactorHandle &h, int nrhs, cudaStream_t st) {
  if (h.prec == HS_PREC_F64)
    apply_ws_t<double>(h, nrhs, st);
  else
    apply_ws_t<float>(h, nrhs, st);
}

void ensure_buffers(FactorHandle &h, int nrhs_cap) {
  if (h.nrhs_cap >= nrhs_cap && h.d_ws) return;
  cudaFree(h.d_ws);
  cudaFree(h.d_t);
  cudaFree(h.d_pcg);
  cudaFree(h.d_part);
  cudaFree(h.d_scal);
  cudaFree(h.d_iflags);
  h.d_ws = h.d_t = h.d_pcg = h.d_part = h.d_scal = nullptr;
  h.d_iflags = nullptr;
  const int64_t n = h.plan.n;
  HS_CUDA(cudaMalloc(&h.d_ws, sizeof(double) * std::max<int64_t>(h.ws_size, 1) * nrhs_cap));
  const int64_t tneed = std::max<int64_t>(std::max<int64_t>(h.tmax, h.root_m), 1);
  HS_CUDA(cudaMalloc(&h.d_t, sizeof(double) * tneed * nrhs_cap));
  HS_CUDA(cudaMalloc(&h.d_pcg, sizeof(double) * 6 * n * nrhs_cap));
  h.part_blocks = 152 * 8;
  HS_CUDA(cudaMalloc(&h.d_part, sizeof(double) * h.part_blocks * 32));
  HS_CUDA(cudaMalloc(&h.d_scal, sizeof(double) * 6 * 32));
  HS_CUDA(cudaMalloc(&h.d_iflags, sizeof(int) * (2 * 32 + 2)));
  HS_CUDA(cudaMemset(h.d_iflags, 0, sizeof(int) * (2 * 32 + 2)));
  h.nrhs_cap = nrhs_cap;
}

}  // namespace

void apply_solve(FactorHandle &h, const double *r, double *z, int nrhs, int64_t ld, cudaStream_t st) {
  ensure_buffers(h, std::max(nrhs, h.nrhs_cap));
  const int64_t n = h.plan.n;
  k_gather_in<<<grid_for(n * nrhs), 256, 0, st>>>(r, ld, h.d_perm, n, nrhs, nrhs, h.d_ws);
  apply_ws(h, nrhs, st);
  k_scatter_out<<<grid_for(n * nrhs), 256, 0, st>>>(h.d_ws, h.d_perm, n, nrhs, nrhs, z, ld);
  HS_CUDA(cudaGetLastError());
}

int pcg_solve(FactorHandle &h, const double *b, double *x, int nrhs, int64_t ld, double rtol,
              int maxit, int *iters, double *relres, cudaStream_t st) {
  int np = 1;
  while (np < nrhs) np <<= 1;
  ensure_buffers(h, std::max(np, h.nrhs_cap));
  const int64_t n = h.plan.n;
  const int64_t tot = n * np;
  double *X = h.d_pcg, *R = X + tot, *P0 = R + tot, *P1 = P0 + tot, *Q = P1 + tot, *B = Q + tot;
  PcgScal sc{h.d_scal, h.d_scal + 32, h.d_scal + 64, h.d_scal + 96, h.d_scal + 128, h.d_scal + 160};
  PcgFlags fl{h.d_iflags, h.d_iflags + 32, h.d_iflags + 64, h.d_iflags + 65};
  const int g = rgrid_for(tot);
  // grid * PT is a multiple of 256, hence of np (np <= 32): each thread keeps one rhs
  k_gather_in<<<grid_for(tot), 256, 0, st>>>(b, ld, h.d_perm, n, nrhs, np, B);
  HS_CUDA(cudaMemcpyAsync(R, B, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
  HS_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * tot, st));
  HS_CUDA(cudaMemsetAsync(P0, 0, sizeof(double) * tot, st));
  k_dot<<<g, PT, 0, st>>>(B, B, n, np, h.d_part, sc, fl, DOT_BNORM, nullptr);
  // z = A_H^-1 r in the level-L segment of the workspace
  double *Z = h.d_ws;
  HS_CUDA(cudaMemcpyAsync(Z, R, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
  apply_ws(h, np, st);
  k_dot<<<g, PT, 0, st>>>(R, Z, n, np, h.d_part, sc, fl, DOT_RZ_FIRST, nullptr);
  int *done_h = nullptr;
  HS_CUDA(cudaMallocHost(&done_h, sizeof(int)));
  double *pold = P0, *pnew = P1;
  int it = 0;
  const double rtol2 = rtol * rtol;
  bool converged = false;
  while (it < maxit) {
    k_spmv_p<<<g, PT, 0, st>>>(h.d_rowptr, h.d_col, h.d_val, n, np, Z, pold, pnew, Q, h.d_part, sc, fl);
    k_update<<<g, PT, 0, st>>>(X, R, pnew, Q, n, np, h.d_part, sc, fl, rtol2);
    HS_CUDA(cudaGetLastError());
    ++it;
    HS_CUDA(cudaMemcpyAsync(done_h, fl.done, sizeof(int), cudaMemcpyDeviceToHost, st));
    HS_CUDA(cudaStreamSynchronize(st));
    if (*done_h) {
      converged = true;
      break;
    }
    std::swap(pold, pnew);
    HS_CUDA(cudaMemcpyAsync(Z, R, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
    apply_ws(h, np, st);
    k_dot<<<g, PT, 0, st>>>(R, Z, n, np, h.d_part, sc, fl, DOT_RZ, nullptr);
  }
  cudaFreeHost(done_h);
  // true relative residual
  k_residual<<<grid_for(tot), 256, 0, st>>>(h.d_rowptr, h.d_col, h.d_val, n, np, X, B, Q);
  double *rr_d = h.d_scal + 5 * 32;
  k_dot<<<g, PT, 0, st>>>(Q, Q, n, np, h.d_part, sc, fl, DOT_PLAIN, rr_d);
  k_scatter_out<<<grid_for(n * nrhs), 256, 0, st>>>(X, h.d_perm, n, nrhs, np, x, ld);
  HS_CUDA(cudaGetLastError());
  std::vector<double> hs(6 * 32);
  std::vector<int> hi(2 * 32 + 2);
  HS_CUDA(cudaMemcpyAsync(hs.data(), h.d_scal, sizeof(double) * 6 * 32, cudaMemcpyDeviceToHost, st));
  HS_CUDA(cudaMemcpyAsync(hi.data(), h.d_iflags, sizeof(int) * (2 * 32 + 2), cudaMemcpyDeviceToHost, st));
  HS_CUDA(cudaStreamSynchronize(st));
  bool all = true;
  for (int j = 0; j < nrhs; ++j) {
    iters[j] = hi[32 + j];
    const double bn = hs[j];
    relres[j] = bn > 0 ? std::sqrt(hs[160 + j] / bn) : 0.0;
    all = all && hi[j] == 0;
  }
  (void)converged;
  return all ? HS_OK : HS_ERR_NO_CONVERGENCE;
}

FactorHandle::~FactorHandle() {
  cudaFree(d_rowptr);
  cudaFree(d_col);
  cudaFree(d_val);
  cudaFree(d_perm);
  cudaFree(d_nodes);
  cudaFree(d_nbrs);
  cudaFree(d_targets);
  cudaFree(d_contribs);
  cudaFree(d_ws);
  cudaFree(d_t);
  cudaFree(d_pcg);
  cudaFree(d_part);
  cudaFree(d_scal);
  cudaFree(d_iflags);
}

}  // namespace hs
