// Internal declarations of the GB300 hierarchical solver library.
//
// Everything here sits below the C ABI of include/hs.h.  Dense blocks are
// row-major with an explicit leading dimension.  Batched kernels take arrays of
// task descriptors built on the host, one descriptor per (super node, operation).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/hs.h"

namespace hs {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
struct Error {
  int code;
  std::string msg;
};

void set_error(const std::string &msg);
[[noreturn]] void fail(int code, const std::string &msg);

// kernel launches of this library in the process (hs_launch_count)
void count_launch(int n = 1);
// While one is alive, count_launch on this thread counts nothing (launches
// recorded into a CUDA graph are counted when the graph runs).
struct CountPause {
  CountPause();
  ~CountPause();
};

#define HS_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      ::hs::fail(e_ == cudaErrorMemoryAllocation ? HS_ERR_OOM : HS_ERR_CUDA,            \
                 std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

// The largest dynamic shared memory a kernel may request is a process-wide
// attribute of the function.  It is raised once per kernel and device to the
// device's opt-in limit and never lowered, so launches from several host
// threads cannot undo each other's setting between set and launch.  Returns
// the usable dynamic bytes.
template <auto Kernel>
int allow_max_dynamic_smem() {
  static std::mutex mu;
  static int limit[64] = {0};
  int dev = 0;
  HS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) fail(HS_ERR_CUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (!limit[dev]) {
    int optin = 0;
    HS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    HS_CUDA(cudaFuncGetAttributes(&fa, Kernel));
    const int dyn = optin - (int)fa.sharedSizeBytes;
    HS_CUDA(cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    limit[dev] = dyn;
  }
  return limit[dev];
}

// fails with HS_ERR_CAPACITY when `bytes` exceed what the kernel may request
inline void check_dynamic_smem(size_t bytes, int limit, const char *what) {
  if (bytes > (size_t)limit)
    fail(HS_ERR_CAPACITY, std::string(what) + " needs " + std::to_string(bytes) +
                              " bytes of shared memory; the device allows " + std::to_string(limit));
}

// ---------------------------------------------------------------------------
// task descriptors (shared by host and device)
// ---------------------------------------------------------------------------

// C = alpha * op(A) * op(B) + beta * C, all row-major.
// op(A) is M x K: A[i*lda + k] (ta = 0) or A[k*lda + i] (ta = 1).
// op(B) is K x N: B[k*ldb + j] (tb = 0) or B[j*ldb + k] (tb = 1).
template <typename T>
struct GemmTask {
  const T *A;
  const T *B;
  T *C;
  int M, N, K;
  int lda, ldb, ldc;
  int ta, tb;
  T alpha, beta;
};

// dst = beta * dst + alpha * sum_s op(src_s), rows x cols; sources listed in
// `srcs[first .. first + nsrc)` and summed in that order (deterministic).
template <typename T>
struct SumSrc {
  const T *ptr;
  int ld;
  int trans;  // 1: element (i, j) is ptr[j*ld + i]
};

template <typename T>
struct SumTask {
  T *dst;
  int ld;
  int rows, cols;
  int first, nsrc;
  T alpha, beta;
};

// Cholesky factor and its inverse: A = L L^T, writes Linv = L^-1 (lower, zero
// above the diagonal).  status[idx] = 0 ok, j+1 if the j-th pivot failed.
template <typename T>
struct CholTask {
  const T *A;
  T *Linv;
  int m;
  int lda, ldl;
  int status_idx;
};

// Preserved vectors per node (GC family, HS_MAX_PHI) and the size of the GC
// basis U_1 they give: the columns of phi_s and of A_sw phi_w.
constexpr int kMaxPhi = 4;
constexpr int kMaxK1 = 2 * kMaxPhi;
static_assert(kMaxPhi == HS_MAX_PHI, "the kernels' vector limit must match the ABI's");

// Truncation of one super node (Sec. 3.2 compression, Sec. 6 GC basis,
// Appendix B projection).  G = A_sw A_sw^T (m x m, ld m); a = A_sw phi_w and
// phi = phi_s, both m x np row-major (np = 0 for LoRaSp).
// Outputs U (m x k, row-major, ld m) and k.  Work: 2 m^2 T.
template <typename T>
struct TruncTask {
  const T *G;
  const T *a;
  const T *phi;
  T *U;
  T *work;
  double eps;   // truncation tolerance of this node's level
  double eps1;  // HS_GC_PROJ: tolerance of the SVD of [phi_s, A_sw phi_w]
  int m;
  int np;       // preserved vectors (columns of phi and a)
  int k_idx;    // index into the rank array
  int cap;      // largest rank k kept (hs_opts.max_rank_ratio; m: no cap); the
                // GC basis U_1 is always kept whole
};

// ---------------------------------------------------------------------------
// kernel launchers (kernels_dense.cu)
// ---------------------------------------------------------------------------
template <typename T>
void launch_gemm(const GemmTask<T> *d_tasks, const int *d_tile_start, int ntasks, int total_tiles,
                 cudaStream_t st);
template <typename T>
void launch_sum(const SumTask<T> *d_tasks, const SumSrc<T> *d_srcs, const int *d_tile_start,
                int ntasks, int total_tiles, cudaStream_t st);
// largest m the Cholesky kernel keeps in shared memory (larger ones are
// factored blockwise by the host-driven multi-CTA path)
template <typename T>
int chol_smem_cap();
// per large task of a blocked Cholesky: its diagonal-block statuses (bs,
// nblk blocks of nb) merged into *out = first failing pivot + 1, else 0
struct StatusMerge {
  const int *bs;
  int nblk, nb;
  int *out;
};
void launch_status_merge(const StatusMerge *d_tasks, int ntasks, cudaStream_t st);
// element-wise FP32 -> FP64 (widen = 1) or FP64 -> FP32 copies of a task list
// (one CTA per task): the FP64 truncation of the mixed factors
// (hs_opts.rank_f64) reads FP64 copies of the FP32 blocks and writes its
// basis back in FP32
struct ConvTask {
  const void *src;
  void *dst;
  int64_t n;
  int widen;
};
void launch_convert_list(const ConvTask *d_tasks, int ntasks, cudaStream_t st);
template <typename T>
void launch_chol_inv(const CholTask<T> *d_tasks, int ntasks, int *d_status, int max_m,
                     cudaStream_t st);
template <typename T>
void launch_trunc(const TruncTask<T> *d_tasks, int ntasks, int *d_k, double eps, int variant,
                  int max_m, cudaStream_t st);
// large super nodes (kernels_eig.cu): tridiagonalisation / bisection / inverse iteration
// Global work area of one large-truncation node (offsets from TruncTask::work;
// the host computes the same addresses for the multi-CTA kernels):
//   A (m^2 T)   Gram / J, then the Householder reflectors in its rows
//   Y (m^2 T)   eigenvectors of T; before that the multi-CTA tridiagonalisation
//               keeps its step vectors here
//   LU (4 m^2 T), LS (164 m T), FL (m^2 bytes): inverse iteration and Z
//   VG          the per-node vectors (d, e, pw in FP64; dt, et, lam, v, tau, wt,
//               redt in T) when they are not in shared memory
//   SC          persistent scalars between the kernels of the multi-CTA path:
//               k1, k2, cluster count (ints), the norm bound of T, then
//               c = U1^T G U1 (kMaxK1 x kMaxK1 doubles)
template <typename T>
struct BigLayout {
  T *A, *Y, *LU, *LS;
  unsigned char *FL, *VG;
  double *d, *e, *pw;
  T *dt, *et, *lam, *v, *tau, *wt, *redt;
  int *sc_int;        // k1, k2, number of eigenvalue clusters
  double *sc_c;       // c = U1^T G U1 (kMaxK1 x kMaxK1 doubles, ld kMaxK1)
  double *sc_tnorm;   // norm bound of T (inverse-iteration tolerance)
};

template <typename T>
__host__ __device__ inline size_t big_vec_bytes(int m) {
  return 3 * sizeof(double) * (size_t)m + 6 * sizeof(T) * (size_t)((m + 1) & ~1) + 34 * sizeof(T) + 16;
}

// bytes of the SC area (after its 16-byte alignment)
constexpr size_t kBigScBytes = 24 + sizeof(double) * kMaxK1 * kMaxK1;

template <typename T>
__host__ __device__ inline BigLayout<T> big_layout(T *work, int m) {
  BigLayout<T> L;
  L.A = work;
  L.Y = work + (size_t)m * m;
  L.LU = L.Y + (size_t)m * m;
  L.LS = L.LU + 4 * (size_t)m * m;
  L.FL = (unsigned char *)(L.LS + 164 * (size_t)m);
  L.VG = (unsigned char *)(((uintptr_t)(L.FL + (size_t)m * m) + 15) & ~(uintptr_t)15);
  const size_t me = (size_t)((m + 1) & ~1);
  unsigned char *p = L.VG;
  L.d = (double *)p;
  p += sizeof(double) * m;
  L.e = (double *)p;
  p += sizeof(double) * m;
  L.pw = (double *)p;
  p += sizeof(double) * m;
  L.dt = (T *)p;
  p += sizeof(T) * me;
  L.et = (T *)p;
  p += sizeof(T) * me;
  L.lam = (T *)p;
  p += sizeof(T) * me;
  L.v = (T *)p;
  p += sizeof(T) * me;
  L.tau = (T *)p;
  p += sizeof(T) * me;
  L.wt = (T *)p;
  p += sizeof(T) * me;
  L.redt = (T *)p;
  unsigned char *sc = (unsigned char *)(((uintptr_t)(L.VG + big_vec_bytes<T>(m)) + 15) & ~(uintptr_t)15);
  L.sc_int = (int *)sc;
  L.sc_tnorm = (double *)(sc + 16);
  L.sc_c = (double *)(sc + 24);
  return L;
}

// One node of the multi-CTA tridiagonalisation (very large super nodes): its
// matrix A (m x m, ld m) and step vectors in the node's work area, the
// tridiagonal d, e and the reflector coefficients tau.  The node owns nblk =
// ceil(m / kTriRows) consecutive CTAs starting at blk0.
constexpr int kTriRows = 8;   // rows per CTA, one warp each
template <typename T>
struct GridTri {
  T *A;
  T *X, *P, *V;      // column k, p, v of the current step
  T *px, *ppv;       // per-CTA partial sums (|x|^2, p.v)
  double *d, *e;
  T *tau;
  int m, nblk, blk0;
};

// Inverse iteration of a node's selected eigenvalues (multi-CTA path): the
// clusters of close eigenvalues (starts, count in sc[2]) are spread one per
// thread over many CTAs, each thread's LU and vector in shared memory.
template <typename T>
struct InvitTask {
  const T *dt, *et, *lam;
  const int *starts;
  const int *sc;
  const double *tnorm;
  T *Y;              // eigenvectors of T, column q at Y + q m
  int m, blk0;
};

// Products with Q = H_0 ... H_{m-3} of a node's reflectors: forward (Q^T, the
// 2 k1 columns of Z, in place) or backward (Q Y into U columns k1..).  A task is
// one batch of columns [j0, j0 + nb) of one node; k1, k2 come from the node's
// scalar area (sc).
template <typename T>
struct ReflTask {
  const T *A;
  const T *tau;
  T *cols;           // column-major, ld m
  T *U;              // backward: output, row-major m x m
  const int *sc;
  int m, j0, fwd;
};

// Large-node truncations of m <= kTruncBigMidMax run 256 threads per node,
// larger ones 1024; launch_trunc_big takes tasks of one class at a time.
constexpr int kTruncBigMidMax = 128;

template <typename T>
size_t trunc_big_work_elems(int m);
template <typename T>
void launch_trunc_big(const TruncTask<T> *d_tasks, int ntasks, int *d_k, double eps, int variant,
                      int max_m, cudaStream_t st);
// the multi-CTA path: k_trunc_big in one of its modes (TB_PREP = 1, TB_POST = 2)
template <typename T>
void launch_trunc_big_mode(const TruncTask<T> *d_tasks, int ntasks, int *d_k, double eps, int variant, int max_m,
                           int mode, cudaStream_t st);
// one step k of the multi-CTA tridiagonalisation over `total_blocks` CTAs
// (phase 0: apply step k-1's update and take column k; phase 1: reflector
// and p = tau A v)
template <typename T>
void launch_tri_step(const GridTri<T> *d_tasks, int ntasks, int total_blocks, int k, int phase, cudaStream_t st);
// the whole tridiagonalisation of each node by one thread-block cluster
// (kernels_cluster.cu): the cluster size (1, 2, 4 or 8 CTAs) that holds a node
// of size m in shared memory, 0 when none does; all tasks of a launch use
// cluster size C
template <typename T>
int tri_cluster_size(int m);
template <typename T>
void launch_tri_cluster(const GridTri<T> *d_tasks, int ntasks, int C, int m_max, cudaStream_t st);
// inverse iteration over total_blocks CTAs of `spc` slots each
template <typename T>
void launch_invit(const InvitTask<T> *d_tasks, int ntasks, int total_blocks, int spc, int m_max, cudaStream_t st);
// slots per CTA of launch_invit for nodes of size up to m
template <typename T>
int invit_slots(int m);
// reflector products (one CTA per task); nb columns per task
template <typename T>
void launch_refl(const ReflTask<T> *d_tasks, int ntasks, int nb, int m_max, cudaStream_t st);
// columns per reflector task that fit the shared-memory budget for nodes of size m
template <typename T>
int refl_batch(int m);
// largest m handled by the shared-memory Jacobi truncation
template <typename T>
constexpr int jacobi_cap() {
  return sizeof(T) == 8 ? 110 : 156;
}
template <typename T>
void launch_scatter_values(const double *val, const int64_t *dest, int64_t nnz, T *pool,
                           cudaStream_t st);
void launch_gather_values(const double *val, const int32_t *src, int64_t nnz, double *out,
                          cudaStream_t st);
// symmetric diagonal scaling of a CSR matrix (rows rp, columns ci, values val,
// n rows): ds = D^-1/2, val_scaled = D^-1/2 A D^-1/2; *flag = 1 if a diagonal
// entry is missing or not positive
void launch_diag_scale(const int32_t *rp, const int32_t *ci, const double *val, int64_t n, double *ds,
                       double *val_scaled, int *flag, cudaStream_t st);
// out = D^1/2 raw for n x np vectors (row-major, row p scaled by 1 / ds[p])
template <typename T>
void launch_phi_scale(const T *raw, const double *ds, int64_t n, int np, T *out, cudaStream_t st);

// tile bookkeeping for the batched GEMM / sum kernels
constexpr int GEMM_TM = 64;
constexpr int GEMM_TN = 64;
constexpr int SUM_TILE = 32;

// Tensor-core GEMM (kernels_tc.cu): operand precision of the tcgen05 path.
// C = alpha op(A) op(B) + beta C on FP32 data with the operands rounded to
// TF32 or BF16 and FP32 accumulation; tiles of TC_TILE_M x bn (bn = 64 or
// 128), tile_start counted in those tiles.  *d_err becomes 1 if a bounded
// wait of the kernel ran out (the tile is then not written).
// HS_TC_TF32X3: each FP32 operand is split into TF32 high and low parts
// (a = a_hi + a_lo) and a b is taken as a_hi b_hi + a_hi b_lo + a_lo b_hi,
// three tensor-core MMAs with near-FP32 accuracy.
enum { HS_TC_NONE = 0, HS_TC_TF32 = 1, HS_TC_BF16 = 2, HS_TC_TF32X3 = 3 };
constexpr int TC_TILE_M = 128;
// tensor-core operand precision of a factor precision (HS_TC_NONE for the
// FP64 and FP32 factors)
inline int tc_kind_of(int prec) {
  return prec == HS_PREC_TF32 ? HS_TC_TF32 : prec == HS_PREC_BF16 ? HS_TC_BF16
                                              : prec == HS_PREC_TF32X3 ? HS_TC_TF32X3 : HS_TC_NONE;
}
// wait_cycles: bound of each mbarrier wait in SM clock cycles (0: the
// default, about one second)
void launch_gemm_tc(int kind, int bn, const GemmTask<float> *d_tasks, const int *d_tile_start, int ntasks,
                    int total_tiles, int *d_err, cudaStream_t st, long long wait_cycles = 0);
// GEMM autotuner (kernels_tc.cu): the variant for a task of this shape in
// precision `kind` -- 0 for the CUDA-core kernel, 64 or 128 for the
// tensor-core kernel of that tile width.  gemm_tune builds the device's table
// (synchronising the device) if it does not exist yet; gemm_tune_report
// copies it out: per shape class, the times (ms) of the three variants and
// the choice.
void gemm_tune(int kind);
// hs_test_wait_probe: tensor-core GEMM launches first wait on a barrier that
// nothing arrives at, so that their bounded wait runs out
void set_wait_probe(bool on);
int gemm_route(int kind, int M, int N, int K);
int gemm_tune_report(int kind, float *ms, int *route, int cap);

}  // namespace hs
