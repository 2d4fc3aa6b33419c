// The factorization handle: device memory, the records the solve reads, and
// the host-side description of the apply schedule.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "hs_internal.h"
#include "plan.h"

namespace hs {

// Where a handle's device memory comes from: the CUDA runtime, or the
// caller's hook (hs_opts.allocator).  get() fails with HS_ERR_OOM when the
// hook has no memory and HS_ERR_INVALID when it returns a pointer that is
// not 256-byte aligned; put() waits for the work enqueued on the freeing
// call's stream before it hands a block back to the hook.
struct DevAlloc {
  hs_alloc_fn fa = nullptr;
  hs_free_fn ff = nullptr;
  void *ctx = nullptr;
  int device = 0;
  bool hooked() const { return fa != nullptr; }
  void *get(size_t bytes, cudaStream_t st) const;
  void put(void *p, cudaStream_t st) const noexcept;
  template <typename X>
  void get(X **p, size_t bytes, cudaStream_t st) const {
    *p = (X *)get(bytes, st);
  }
};

// Chunked bump allocator over device chunks (256-byte aligned) taken from a
// DevAlloc.
class DevArena {
 public:
  explicit DevArena(size_t min_chunk) : min_chunk_(min_chunk) {}
  DevArena(size_t min_chunk, const DevAlloc &al) : min_chunk_(min_chunk), al_(al) {}
  ~DevArena();
  void *alloc(size_t bytes);
  void reset();  // keeps the chunks for reuse
  size_t used() const { return used_; }
  size_t reserved() const { return reserved_; }
  void set_alloc(const DevAlloc &al, cudaStream_t st) {
    al_ = al;
    st_ = st;
  }

 private:
  std::vector<std::pair<char *, size_t>> chunks_;
  DevAlloc al_;
  cudaStream_t st_ = nullptr;
  size_t min_chunk_;
  int cur_ = -1;
  size_t off_ = 0;
  size_t used_ = 0, reserved_ = 0;
};

// Apply schedule, one entry per super node of a wave (Algorithm 2).
// Vectors live in one workspace: level L (n unknowns in cluster order), then
// level L-1 (the red nodes made at level L), ..., then the root.  Every value
// is stored as [unknown][rhs] (nrhs consecutive doubles per unknown).
struct ApplyNode {
  const void *M;     // M_ss, m x m
  const void *P;     // P_ss, k x m
  const void *AsN;   // [A_{s n}]_n, m x dN (ld dN)
  int64_t xs;        // unknown offset of s in the workspace
  int64_t xr;        // unknown offset of the red node r (or -1)
  int64_t toff;      // unknown offset of t_s in the per-wave scratch
  int m, k, dN;
  int nb_first, nb_count;
  int row0;          // prefix of (m + k) rows inside the wave (forward GEMV rows)
  int brow0;         // prefix of m rows inside the wave (backward rows)
  int pch0;          // prefix of 32-column chunks of P_ss inside the wave (k > 0 nodes)
};
struct ApplyNbr {
  int64_t x;         // unknown offset of neighbour n
  int size;
  int col;           // column offset of A_{s n} inside AsN
};
struct ApplyTarget {  // forward substitution, gathered by neighbour
  int64_t x;
  int size;
  int first, count;
  int ch0;           // prefix of 32-row chunks inside the wave
};
struct ApplyContrib {
  const void *A;     // AsN + col, element (i in s, q in n) at A[i*ld + q]
  int ld;
  int m;
  int64_t toff;
};

struct WaveApply {
  int node_first, node_count;
  int tgt_first, tgt_count;
  int max_m;
  int64_t tsize;     // unknowns of t scratch used
  int rows_f;        // sum of (m + k): forward GEMV rows
  int rows_b;        // sum of m: backward rows
  int pch;           // sum of 32-column chunks of P_ss
  int tch;           // sum of 32-row chunks of the targets
  // offsets into FactorHandle::d_hints of the per-CTA search starts of the
  // per-step kernels (-1: none): f1 by row0, f2 by ch0, b1/b2 by brow0, b1's
  // P_ss^T part by pch0
  int hf1 = -1, hf2 = -1, hb = -1, hp = -1;
};
struct LevelApply {
  int level;
  int wave_first, wave_count;
};

// A recorded launch sequence (CUDA graph) of the solve.  key: the
// right-hand-side count of an apply, or kPcgGraphKey + 2 * nrhs_p + parity
// for one PCG iteration.
struct GraphEntry {
  int key;
  cudaGraphExec_t exec;
  int kernels;       // kernel nodes, counted by hs_launch_count per replay
};
constexpr int kPcgGraphKey = 1 << 16;

struct FactorHandle {
  Plan plan;
  int prec = HS_PREC_F64;
  int variant = HS_GC_CONSTANT;
  double eps = 0.0;
  std::vector<double> eps_level;       // per level above the leaves (empty: eps everywhere)
  int nphi = 1;                        // preserved vectors per node (GC family)
  double eps1 = 0.0;                   // first tolerance of HS_GC_PROJ (Appendix B)
  int64_t timeout_cycles = 0;          // bound of the kernels' waits (0: default)
  double max_rank_ratio = 0.0;         // rank cap k <= floor(ratio m) (0: none)
  bool rank_f64 = false;               // FP32 factors: truncation (Gram, eigen-solve, rank) in FP64
  cudaStream_t stream = nullptr;
  int device = 0;
  bool valid = false;                  // holds a usable factorization
  DevAlloc alloc;                      // source of every device block the handle holds

  // permuted CSR (cluster order), FP64, for the SpMV of PCG
  int32_t *d_rowptr = nullptr, *d_col = nullptr;
  double *d_val = nullptr;
  int32_t *d_perm = nullptr;
  // symmetric diagonal scaling (hs_opts.scale): D^-1/2 per cluster-order
  // unknown, and the scaled values D^-1/2 A D^-1/2 the factorization reads
  bool scale = false;
  double *d_dscale = nullptr;
  double *d_val_f = nullptr;
  int *d_flag = nullptr;               // set when a diagonal entry is not positive
  const double *factor_values() const { return scale ? d_val_f : d_val; }

  std::unique_ptr<DevArena> pers;      // factor records and live blocks
  std::unique_ptr<DevArena> scratch;   // per-wave scratch of the factorization

  // apply schedule (host copies and device copies)
  std::vector<ApplyNode> nodes;
  std::vector<ApplyNbr> nbrs;
  std::vector<ApplyTarget> targets;
  std::vector<ApplyContrib> contribs;
  std::vector<WaveApply> waves;        // in elimination order, levels L..2
  std::vector<LevelApply> levels;      // levels L..2
  ApplyNode *d_nodes = nullptr;
  ApplyNbr *d_nbrs = nullptr;
  ApplyTarget *d_targets = nullptr;
  ApplyContrib *d_contribs = nullptr;
  // the persistent apply: step list (kind, wave) and the waves on the device,
  // the grid barrier's counter and generation, and its time-out flag
  void *d_apply_steps = nullptr;
  int apply_nsteps = 0;
  WaveApply *d_waves = nullptr;
  unsigned *d_apply_bar = nullptr;
  int *d_apply_err = nullptr;
  // per-CTA first node (or target) of each per-step apply kernel, for a
  // CTA's first warp; each warp scans forward from it (WaveApply::hf1 ...)
  int *d_hints = nullptr;
  size_t hints_cap = 0;
  int64_t ws_size = 0;                 // unknowns in the apply workspace
  int64_t tmax = 0;                    // max unknowns of t scratch per wave
  int64_t root_off = 0;
  int root_m = 0;
  const void *root_inv = nullptr;      // A_root^-1 (m x m)

  // cached maps of the pattern (reused by hs_factor_refactor)
  int32_t *d_src = nullptr;            // permuted entry -> original CSR entry
  int64_t *d_leaf_dest = nullptr;      // permuted entry -> offset in the leaf blocks (or -1)
  std::vector<std::pair<int, int>> leaf_blocks;   // leaf block list, in storage order
  std::vector<int64_t> leaf_block_off;
  int64_t leaf_total = 0;
  void *d_phi0 = nullptr;              // leaf preserved vectors (GC): n x nphi row-major, factor precision
  void *d_phi_raw = nullptr;           // the caller's vectors before the scaling D^1/2 phi (scaling on)
  int64_t nnz = 0;

  // solve buffers (grown on demand)
  int nrhs_cap = 0;
  int64_t ws_cap = 0, t_cap = 0;
  void *d_ws = nullptr, *d_t = nullptr;  // apply workspace and scratch, factor precision
  double *d_pcg = nullptr;             // x, r, p, p2, q, b, z (7 n nrhs), FP64
  double *d_gm = nullptr;              // GMRES: Krylov basis and vectors, FP64
  size_t gm_cap = 0;                   // doubles in d_gm
  double *d_part = nullptr;            // per-block partial sums
  double *d_scal = nullptr;            // per-rhs scalars
  int *d_iflags = nullptr;             // per-rhs ints + block counter
  int part_blocks = 0;
  int *h_done = nullptr;               // pinned: PCG "all converged" flag

  // recorded solve graphs and the private stream they are recorded on
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;
  void drop_graphs() {
    for (GraphEntry &g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }

  // per-level ranks: ranks[li][s] = k or -1
  std::vector<std::vector<int>> ranks;
  hs_info info{};

  ~FactorHandle();
};

// factor.cu
void factorize(FactorHandle &h, const hs_csr &A, const hs_opts &o, const double *phi_host);
// device time per factor phase into hs_info.phase_ms (event pairs; small cost)
void set_phase_profiling(bool on);
// Independent problems factored in lock step, their steps batched into shared
// launches.  With more than one problem, a failed pivot (not SPD) takes only
// that problem out: status[p] = HS_ERR_NOT_SPD and msg[p] say so.
void factorize_batch(const std::vector<FactorHandle *> &hs, const std::vector<const double *> &phis,
                     cudaStream_t st, std::vector<int> *status, std::vector<std::string> *msg);

// solve.cu
void apply_solve(FactorHandle &h, const double *r, double *z, int nrhs, int64_t ld,
                 cudaStream_t st);
int pcg_solve(FactorHandle &h, const double *b, double *x, int nrhs, int64_t ld, double rtol,
              int maxit, int *iters, double *relres, cudaStream_t st);
// right-preconditioned restarted GMRES, one right-hand side (hs_gmres)
int gmres_solve(FactorHandle &h, const double *b, double *x, double rtol, int maxit, int restart, int *iters,
                double *relres, cudaStream_t st);
void apply_static(FactorHandle &h, const double *r, double *z, int nrhs, int64_t ld, cudaStream_t st);
// after a factorization: the persistent apply's step list and waves to the device
void apply_prepare(FactorHandle &h, cudaStream_t st);
// 1 if a grid barrier of the persistent apply ran out (synchronous read; the
// flag is cleared, so a time-out is reported once)
int apply_error(FactorHandle &h);
// the persistent apply's time-out probe on the current device (hs_test_wait_probe)
void set_apply_probe(bool on);

}  // namespace hs
