// C ABI of include/hs.h.  Every entry point catches hs::Error (and any other
// C++ exception) and turns it into a status code plus a thread-local message.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "handle.h"

namespace hs {

namespace {
thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};
thread_local int g_count_paused = 0;
}

void count_launch(int n) {
  if (!g_count_paused) g_launches.fetch_add(n, std::memory_order_relaxed);
}
CountPause::CountPause() { ++g_count_paused; }
CountPause::~CountPause() { --g_count_paused; }

void set_error(const std::string &msg) { g_err = msg; }

[[noreturn]] void fail(int code, const std::string &msg) { throw Error{code, msg}; }

template <typename F>
int guarded(F &&f) {
  try {
    g_err.clear();
    return f();
  } catch (const Error &e) {
    g_err = e.msg;
    return e.code;
  } catch (const std::bad_alloc &) {
    g_err = "host allocation failed";
    return HS_ERR_OOM;
  } catch (const std::exception &e) {
    g_err = e.what();
    return HS_ERR_INVALID;
  } catch (...) {
    g_err = "unknown error";
    return HS_ERR_INVALID;
  }
}

namespace {

void require_device() {
  int n = 0;
  const cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0)
    fail(HS_ERR_CUDA, std::string("no CUDA device: ") + (e == cudaSuccess ? "count is 0" : cudaGetErrorString(e)));
}

// The factor's buffers live on the device that was current when it was
// created; every later call on the handle must run with that device current.
void require_factor_device(const FactorHandle &h) {
  require_device();
  int dev = -1;
  HS_CUDA(cudaGetDevice(&dev));
  if (dev != h.device)
    fail(HS_ERR_INVALID, "the current device is " + std::to_string(dev) + " but the factorization lives on device " +
                             std::to_string(h.device));
}

template <typename X>
X *upload_vec(const FactorHandle &h, const std::vector<X> &v, cudaStream_t st) {
  X *d = nullptr;
  h.alloc.get(&d, sizeof(X) * std::max<size_t>(v.size(), 1), st);
  if (!v.empty()) HS_CUDA(cudaMemcpyAsync(d, v.data(), sizeof(X) * v.size(), cudaMemcpyHostToDevice, st));
  return d;
}

// Values -> permuted CSR, numeric factorization, apply schedule to the device,
// counters.  Used by hs_factor_create and hs_factor_refactor (one handle) and
// their batched forms (several handles factored in lock step).
void numeric_pre(FactorHandle &h, const double *val, cudaStream_t st) {
  h.stream = st;
  h.drop_graphs();   // the schedule and the record pointers change
  launch_gather_values(val, h.d_src, h.nnz, h.d_val, st);
  if (h.scale) {
    HS_CUDA(cudaMemsetAsync(h.d_flag, 0, sizeof(int), st));
    launch_diag_scale(h.d_rowptr, h.d_col, h.d_val, h.plan.n, h.d_dscale, h.d_val_f, h.d_flag, st);
    int bad = 0;
    HS_CUDA(cudaMemcpyAsync(&bad, h.d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    HS_CUDA(cudaStreamSynchronize(st));
    if (bad) fail(HS_ERR_NOT_SPD, "diagonal scaling: a diagonal entry is missing or not positive");
  }
  h.alloc.put(h.d_nodes, st);
  h.alloc.put(h.d_nbrs, st);
  h.alloc.put(h.d_targets, st);
  h.alloc.put(h.d_contribs, st);
  h.d_nodes = nullptr;
  h.d_nbrs = nullptr;
  h.d_targets = nullptr;
  h.d_contribs = nullptr;
}

void numeric_failed(FactorHandle &h) {
  h.nodes.clear();
  h.waves.clear();
  h.levels.clear();
  h.root_m = 0;
}

void numeric_post(FactorHandle &h, float ms, cudaStream_t st) {
  h.d_nodes = upload_vec(h, h.nodes, st);
  h.d_nbrs = upload_vec(h, h.nbrs, st);
  h.d_targets = upload_vec(h, h.targets, st);
  h.d_contribs = upload_vec(h, h.contribs, st);
  apply_prepare(h, st);
  hs_info &in = h.info;
  in.n = h.plan.n;
  in.levels = h.plan.L;
  in.waves = h.plan.total_waves;
  in.factor_ms = ms;
  const double tb = h.prec == HS_PREC_F64 ? 8.0 : 4.0;
  double fb = 0.0;
  for (const auto &nd : h.nodes) fb += 2.0 * ((double)nd.m * nd.m + (double)nd.k * nd.m + (double)nd.m * nd.dN);
  fb += (double)h.root_m * h.root_m;
  in.factor_bytes = (int64_t)(fb * tb);
  in.device_bytes = (int64_t)(h.pers->reserved() + h.scratch->reserved());
}

// Numeric factorization of one or more handles on stream st (lock step when
// more than one); factor_ms is the device time of the whole call.  status
// (optional): per-problem result of a batch (HS_OK or HS_ERR_NOT_SPD, message
// in msg); failed problems hold no valid factorization.
void numeric_factor_all(const std::vector<FactorHandle *> &hs, const std::vector<const double *> &vals,
                        const std::vector<const double *> &phis, cudaStream_t st,
                        std::vector<int> *status = nullptr, std::vector<std::string> *msg = nullptr) {
  for (size_t p = 0; p < hs.size(); ++p) numeric_pre(*hs[p], vals[p], st);
  cudaEvent_t e0, e1;
  HS_CUDA(cudaEventCreate(&e0));
  HS_CUDA(cudaEventCreate(&e1));
  HS_CUDA(cudaEventRecord(e0, st));
  std::vector<int> stat;
  std::vector<std::string> msgs;
  try {
    factorize_batch(hs, phis, st, &stat, &msgs);
  } catch (...) {
    cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (FactorHandle *h : hs) numeric_failed(*h);
    throw;
  }
  HS_CUDA(cudaEventRecord(e1, st));
  HS_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  HS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (size_t p = 0; p < hs.size(); ++p) {
    if (stat[p] == HS_OK)
      numeric_post(*hs[p], ms, st);
    else
      numeric_failed(*hs[p]);
  }
  HS_CUDA(cudaStreamSynchronize(st));
  if (status) *status = stat;
  if (msg) *msg = msgs;
}

void numeric_factor(FactorHandle &h, const double *val, const double *phi_host, cudaStream_t st) {
  numeric_factor_all({&h}, {val}, {phi_host}, st);
}

// neighbour rule of a clustering (0 reads as 1)
int nbr_rule(int32_t d) {
  if (d < 0 || d > 2) fail(HS_ERR_INVALID, "nbr_dist must be 0, 1 or 2");
  return d == 0 ? 1 : d;
}

// checks and planning of hs_factor_create; the handle is left ready for numeric_factor
void setup_handle(FactorHandle &h, const hs_csr *A, const hs_clustering *cl, const hs_opts *o, cudaStream_t st) {
  if (!A || !cl) fail(HS_ERR_INVALID, "null argument");
  if (A->n <= 0 || A->nnz <= 0 || !A->rowptr || !A->col || !A->val) fail(HS_ERR_INVALID, "bad CSR");
  if (!cl->perm || !cl->leaf_ptr) fail(HS_ERR_INVALID, "bad clustering");
  HS_CUDA(cudaGetDevice(&h.device));
  h.stream = st;
  if (o->allocator) {
    h.alloc.fa = o->allocator->alloc;
    h.alloc.ff = o->allocator->free;
    h.alloc.ctx = o->allocator->ctx;
  }
  h.alloc.device = h.device;
  h.prec = o->factor_prec;
  h.variant = o->variant;
  h.eps = o->eps;
  h.nphi = (o->variant == HS_GC_USER || o->variant == HS_GC_PROJ) ? std::max(o->n_phi, 1) : 1;
  h.eps1 = o->variant == HS_GC_PROJ ? o->eps1 : 0.0;
  h.timeout_cycles = o->timeout_cycles;
  h.max_rank_ratio = o->max_rank_ratio;
  h.rank_f64 = o->rank_f64 != 0 && o->factor_prec != HS_PREC_F64;
  h.eps_level.clear();
  // pattern to the host for the planner
  std::vector<int32_t> rp(A->n + 1), ci(A->nnz);
  HS_CUDA(cudaMemcpyAsync(rp.data(), A->rowptr, sizeof(int32_t) * (A->n + 1), cudaMemcpyDeviceToHost, st));
  HS_CUDA(cudaMemcpyAsync(ci.data(), A->col, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToHost, st));
  HS_CUDA(cudaStreamSynchronize(st));
  if (rp[A->n] != A->nnz) fail(HS_ERR_INVALID, "rowptr[n] != nnz");
  build_plan(A->n, rp.data(), ci.data(), cl->perm, cl->leaf_ptr, cl->nleaf, h.plan, nbr_rule(cl->nbr_dist),
             o->order_mode);
  if (o->eps_level) {
    const int need = std::max(h.plan.L - 1, 0);
    if (o->n_eps_level < need)
      fail(HS_ERR_INVALID, "eps_level has " + std::to_string(o->n_eps_level) + " entries; this clustering needs " +
                               std::to_string(need));
    h.eps_level.assign(o->eps_level, o->eps_level + need);
  }
  // permuted CSR on the device; values gathered there
  h.d_rowptr = upload_vec(h, h.plan.prow, st);
  h.d_col = upload_vec(h, h.plan.pcol, st);
  h.d_perm = upload_vec(h, h.plan.perm, st);
  h.d_src = upload_vec(h, h.plan.psrc, st);
  h.nnz = A->nnz;
  h.alloc.get(&h.d_val, sizeof(double) * A->nnz, st);
  h.scale = o->scale != 0;
  if (h.scale) {
    h.alloc.get(&h.d_val_f, sizeof(double) * A->nnz, st);
    h.alloc.get(&h.d_dscale, sizeof(double) * A->n, st);
    h.alloc.get(&h.d_flag, sizeof(int), st);
  }
}

void check_opts(const hs_opts *o) {
  if (!o) fail(HS_ERR_INVALID, "null argument");
  if (!(o->eps >= 0.0) || !std::isfinite(o->eps)) fail(HS_ERR_INVALID, "eps must be finite and >= 0");
  if (o->eps > 0.0 && o->eps < 1e-6) fail(HS_ERR_INVALID, "0 < eps < 1e-6 is not supported");
  if (o->variant < HS_LORASP || o->variant > HS_GC_PROJ) fail(HS_ERR_INVALID, "unknown variant");
  const bool user = o->variant == HS_GC_USER || o->variant == HS_GC_PROJ;
  if (o->n_phi < 0 || o->n_phi > (user ? HS_MAX_PHI : 1))
    fail(HS_ERR_INVALID, user ? "n_phi must be 0 .. HS_MAX_PHI" : "n_phi > 1 needs HS_GC_USER or HS_GC_PROJ");
  if (o->variant == HS_GC_PROJ && (!(o->eps1 >= 0.0) || !std::isfinite(o->eps1)))
    fail(HS_ERR_INVALID, "eps1 must be finite and >= 0");
  if (o->scale != 0 && o->scale != 1) fail(HS_ERR_INVALID, "scale must be 0 or 1");
  if (o->timeout_cycles < 0) fail(HS_ERR_INVALID, "timeout_cycles must be >= 0");
  if (!(o->max_rank_ratio >= 0.0 && o->max_rank_ratio <= 1.0))
    fail(HS_ERR_INVALID, "max_rank_ratio must be in [0, 1]");
  if (o->rank_f64 != 0 && o->rank_f64 != 1) fail(HS_ERR_INVALID, "rank_f64 must be 0 or 1");
  if (o->allocator && (!o->allocator->alloc || !o->allocator->free))
    fail(HS_ERR_INVALID, "an allocator hook needs both alloc and free");
  if (o->order_mode != HS_ORDER_WAVES && o->order_mode != HS_ORDER_SEQUENTIAL)
    fail(HS_ERR_INVALID, "order_mode must be HS_ORDER_WAVES or HS_ORDER_SEQUENTIAL");
  if (o->factor_prec != HS_PREC_F64 && o->factor_prec != HS_PREC_F32 && o->factor_prec != HS_PREC_TF32 &&
      o->factor_prec != HS_PREC_BF16 && o->factor_prec != HS_PREC_TF32X3)
    fail(HS_ERR_INVALID, "unknown factor_prec");
  if (o->eps_level) {
    if (o->n_eps_level < 0) fail(HS_ERR_INVALID, "n_eps_level < 0");
    for (int j = 0; j < o->n_eps_level; ++j) {
      const double e = o->eps_level[j];
      if (!(e >= 0.0) || !std::isfinite(e)) fail(HS_ERR_INVALID, "eps_level entries must be finite and >= 0");
      if (e > 0.0 && e < 1e-6) fail(HS_ERR_INVALID, "0 < eps_level[j] < 1e-6 is not supported");
    }
  }
}

}  // namespace

}  // namespace hs

using hs::fail;

struct hs_factor_s {
  hs::FactorHandle h;
};
struct hs_plan_s {
  hs::Plan p;
};

extern "C" {

const char *hs_last_error(void) { return hs::g_err.c_str(); }

int hs_factor_create(const hs_csr *A, const hs_clustering *cl, const hs_opts *o, void *stream,
                     hs_factor *out) {
  return hs::guarded([&]() -> int {
    if (!A || !cl || !o || !out) fail(HS_ERR_INVALID, "null argument");
    *out = nullptr;
    hs::check_opts(o);
    if ((o->variant == HS_GC_USER || o->variant == HS_GC_PROJ) && !o->phi)
      fail(HS_ERR_INVALID, "HS_GC_USER and HS_GC_PROJ need phi");
    hs::require_device();
    cudaStream_t st = (cudaStream_t)stream;
    std::unique_ptr<hs_factor_s> f(new hs_factor_s());
    hs::setup_handle(f->h, A, cl, o, st);
    hs::numeric_factor(f->h, A->val, o->phi, st);
    f->h.valid = true;
    *out = f.release();
    return HS_OK;
  });
}

int hs_factor_create_batch(int32_t count, const hs_csr *A, const hs_clustering *cl, const hs_opts *o,
                           const double *const *phi, void *stream, hs_factor *out, int32_t *status) {
  return hs::guarded([&]() -> int {
    if (count < 1 || !A || !cl || !o || !out) fail(HS_ERR_INVALID, "null argument or count < 1");
    for (int32_t p = 0; p < count; ++p) out[p] = nullptr;
    hs::check_opts(o);
    const bool user = o->variant == HS_GC_USER || o->variant == HS_GC_PROJ;
    if (user && !phi) fail(HS_ERR_INVALID, "HS_GC_USER and HS_GC_PROJ need phi");
    hs::require_device();
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<std::unique_ptr<hs_factor_s>> fs;
    std::vector<hs::FactorHandle *> hs_;
    std::vector<const double *> vals, phis;
    for (int32_t p = 0; p < count; ++p) {
      if (user && !phi[p]) fail(HS_ERR_INVALID, "HS_GC_USER and HS_GC_PROJ need phi for every problem");
      fs.emplace_back(new hs_factor_s());
      try {
        hs::setup_handle(fs.back()->h, &A[p], &cl[p], o, st);
      } catch (hs::Error &e) {
        throw hs::Error{e.code, "problem " + std::to_string(p) + ": " + e.msg};
      }
      hs_.push_back(&fs.back()->h);
      vals.push_back(A[p].val);
      phis.push_back(user ? phi[p] : nullptr);
    }
    std::vector<int> stat;
    std::vector<std::string> msgs;
    hs::numeric_factor_all(hs_, vals, phis, st, &stat, &msgs);
    int first = -1;
    for (int32_t p = 0; p < count; ++p) {
      if (status) status[p] = stat[p];
      if (stat[p] == HS_OK) {
        fs[p]->h.valid = true;
        out[p] = fs[p].release();
      } else if (first < 0) {
        first = p;
      }
    }
    if (first >= 0) fail(stat[first], msgs[first]);   // the others are returned
    return HS_OK;
  });
}

int hs_factor_refactor(hs_factor f, const double *val, void *stream) {
  return hs::guarded([&]() -> int {
    if (!f || !val) fail(HS_ERR_INVALID, "null argument");
    hs::require_factor_device(f->h);
    f->h.valid = false;
    hs::numeric_factor(f->h, val, nullptr, (cudaStream_t)stream);
    f->h.valid = true;
    return HS_OK;
  });
}

int hs_factor_refactor_batch(int32_t count, hs_factor *f, const double *const *val, void *stream,
                             int32_t *status) {
  return hs::guarded([&]() -> int {
    if (count < 1 || !f || !val) fail(HS_ERR_INVALID, "null argument or count < 1");
    std::vector<hs::FactorHandle *> hs_;
    std::vector<const double *> vals, phis;
    for (int32_t p = 0; p < count; ++p) {
      if (!f[p] || !val[p]) fail(HS_ERR_INVALID, "null handle or values");
      for (int32_t q = 0; q < p; ++q)
        if (f[q] == f[p]) fail(HS_ERR_INVALID, "a handle appears twice in the batch");
      hs_.push_back(&f[p]->h);
      vals.push_back(val[p]);
      phis.push_back(nullptr);
    }
    for (auto *h : hs_) hs::require_factor_device(*h);
    for (auto *h : hs_) h->valid = false;
    std::vector<int> stat;
    std::vector<std::string> msgs;
    hs::numeric_factor_all(hs_, vals, phis, (cudaStream_t)stream, &stat, &msgs);
    int first = -1;
    for (int32_t p = 0; p < count; ++p) {
      if (status) status[p] = stat[p];
      hs_[p]->valid = stat[p] == HS_OK;
      if (stat[p] != HS_OK && first < 0) first = p;
    }
    if (first >= 0) fail(stat[first], msgs[first]);
    return HS_OK;
  });
}

int hs_gemm_tc(int32_t prec, int32_t M, int32_t N, int32_t K, float alpha, const float *A, int64_t lda,
               int32_t ta, const float *B, int64_t ldb, int32_t tb, float beta, float *C, int64_t ldc,
               int32_t bn, void *stream) {
  return hs::guarded([&]() -> int {
    if (prec != HS_PREC_TF32 && prec != HS_PREC_BF16 && prec != HS_PREC_TF32X3)
      fail(HS_ERR_INVALID, "prec must be HS_PREC_TF32, HS_PREC_BF16 or HS_PREC_TF32X3");
    if (M < 1 || N < 1 || K < 0) fail(HS_ERR_INVALID, "need M, N >= 1 and K >= 0");
    if (!A || !B || !C) fail(HS_ERR_INVALID, "null argument");
    if (bn != 0 && bn != 64 && bn != 128) fail(HS_ERR_INVALID, "bn must be 0, 64 or 128");
    const int64_t need_a = ta ? M : K, need_b = tb ? K : N;
    if (lda < std::max<int64_t>(need_a, 1) || ldb < std::max<int64_t>(need_b, 1) || ldc < N)
      fail(HS_ERR_INVALID, "leading dimension too small");
    if (lda > INT32_MAX || ldb > INT32_MAX || ldc > INT32_MAX) fail(HS_ERR_INVALID, "leading dimension too large");
    hs::require_device();
    cudaStream_t st = (cudaStream_t)stream;
    const int w = bn ? bn : (N <= 64 ? 64 : 128);
    hs::GemmTask<float> t;
    t.A = A;
    t.B = B;
    t.C = C;
    t.M = M;
    t.N = N;
    t.K = K;
    t.lda = (int)lda;
    t.ldb = (int)ldb;
    t.ldc = (int)ldc;
    t.ta = ta ? 1 : 0;
    t.tb = tb ? 1 : 0;
    t.alpha = alpha;
    t.beta = beta;
    const int tiles = ((M + hs::TC_TILE_M - 1) / hs::TC_TILE_M) * ((N + w - 1) / w);
    char *d = nullptr;
    HS_CUDA(cudaMalloc(&d, 256 + sizeof(t)));
    struct Free {
      char *p;
      ~Free() { cudaFree(p); }
    } fr{d};
    int *d_err = (int *)d, *d_ts = (int *)(d + 16);
    hs::GemmTask<float> *d_t = (hs::GemmTask<float> *)(d + 256);
    HS_CUDA(cudaMemsetAsync(d, 0, 256, st));
    HS_CUDA(cudaMemcpyAsync(d_t, &t, sizeof(t), cudaMemcpyHostToDevice, st));
    hs::launch_gemm_tc(hs::tc_kind_of(prec), w, d_t, d_ts, 1, tiles, d_err, st);
    int herr = 0;
    HS_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    HS_CUDA(cudaStreamSynchronize(st));
    if (herr) fail(HS_ERR_TIMEOUT, "hs_gemm_tc: a bounded wait of the tensor-core GEMM ran out");
    return HS_OK;
  });
}

int hs_gemm_tune_report(int32_t prec, float *ms, int32_t *route, int32_t cap) {
  int n = 0;
  const int rc = hs::guarded([&]() -> int {
    if (prec != HS_PREC_TF32 && prec != HS_PREC_BF16 && prec != HS_PREC_TF32X3)
      fail(HS_ERR_INVALID, "prec must be HS_PREC_TF32, HS_PREC_BF16 or HS_PREC_TF32X3");
    if (cap < 0 || (cap > 0 && (!ms || !route))) fail(HS_ERR_INVALID, "null argument");
    hs::require_device();
    std::vector<int> r(std::max(cap, 0));
    n = hs::gemm_tune_report(hs::tc_kind_of(prec), ms, r.data(), cap);
    for (int i = 0; i < cap && i < n; ++i) route[i] = r[i];
    return HS_OK;
  });
  return rc == HS_OK ? n : -rc;
}

int64_t hs_launch_count(void) { return hs::g_launches.load(); }

int hs_abi_sizes(int64_t *sizes, int32_t cap) {
  const int64_t v[5] = {(int64_t)sizeof(hs_csr), (int64_t)sizeof(hs_clustering), (int64_t)sizeof(hs_opts),
                        (int64_t)sizeof(hs_info), (int64_t)sizeof(hs_allocator)};
  for (int32_t i = 0; i < cap && i < 5 && sizes; ++i) sizes[i] = v[i];
  return 5;
}

int hs_test_wait_probe(int32_t on) {
  return hs::guarded([&]() -> int {
    hs::set_wait_probe(on != 0);
    hs::require_device();
    hs::set_apply_probe(on != 0);
    return HS_OK;
  });
}

int hs_profile_phases(int32_t on) {
  hs::set_phase_profiling(on != 0);
  return HS_OK;
}

int hs_apply(hs_factor f, const double *r, double *z, int32_t nrhs, int64_t ld, void *stream) {
  return hs::guarded([&]() -> int {
    if (!f || !r || !z) fail(HS_ERR_INVALID, "null argument");
    if (nrhs < 1 || nrhs > 64) fail(HS_ERR_INVALID, "nrhs must be in [1, 64]");
    if (ld < f->h.plan.n) fail(HS_ERR_INVALID, "ld < n");
    hs::require_factor_device(f->h);
    cudaStream_t st = (cudaStream_t)stream;
    // r and z may alias: r is gathered into the workspace before z is written
    if (!f->h.valid) fail(HS_ERR_INVALID, "the handle holds no valid factorization");
    hs::apply_solve(f->h, r, z, nrhs, ld, st);
    return HS_OK;
  });
}

int hs_apply_static(hs_factor f, const double *r, double *z, int32_t nrhs, int64_t ld, void *stream) {
  return hs::guarded([&]() -> int {
    if (!f || !r || !z) fail(HS_ERR_INVALID, "null argument");
    if (nrhs < 1 || nrhs > 64) fail(HS_ERR_INVALID, "nrhs must be in [1, 64]");
    if (ld < f->h.plan.n) fail(HS_ERR_INVALID, "ld < n");
    hs::require_factor_device(f->h);
    if (!f->h.valid) fail(HS_ERR_INVALID, "the handle holds no valid factorization");
    hs::apply_static(f->h, r, z, nrhs, ld, (cudaStream_t)stream);
    return HS_OK;
  });
}

int hs_pcg(hs_factor f, const double *b, double *x, int32_t nrhs, int64_t ld, double rtol, int32_t maxit,
           int32_t *iters, double *relres, void *stream) {
  return hs::guarded([&]() -> int {
    if (!f || !b || !x || !iters || !relres) fail(HS_ERR_INVALID, "null argument");
    if (nrhs < 1 || nrhs > 32) fail(HS_ERR_INVALID, "nrhs must be in [1, 32]");
    if (ld < f->h.plan.n) fail(HS_ERR_INVALID, "ld < n");
    if (!(rtol > 0.0) || maxit < 1) fail(HS_ERR_INVALID, "rtol must be > 0 and maxit >= 1");
    hs::require_factor_device(f->h);
    if (!f->h.valid) fail(HS_ERR_INVALID, "the handle holds no valid factorization");
    return hs::pcg_solve(f->h, b, x, nrhs, ld, rtol, maxit, iters, relres, (cudaStream_t)stream);
  });
}

int hs_gmres(hs_factor f, const double *b, double *x, double rtol, int32_t maxit, int32_t restart,
             int32_t *iters, double *relres, void *stream) {
  return hs::guarded([&]() -> int {
    if (!f || !b || !x || !iters || !relres) fail(HS_ERR_INVALID, "null argument");
    if (!(rtol > 0.0) || maxit < 1 || restart < 0) fail(HS_ERR_INVALID, "rtol must be > 0, maxit >= 1, restart >= 0");
    if ((restart > 0 ? std::min(restart, maxit) : maxit) > 1000)
      fail(HS_ERR_INVALID, "the Krylov basis is limited to 1000 vectors (restart, or maxit without restart)");
    hs::require_factor_device(f->h);
    if (!f->h.valid) fail(HS_ERR_INVALID, "the handle holds no valid factorization");
    int it = 0;
    const int r = hs::gmres_solve(f->h, b, x, rtol, maxit, restart, &it, relres, (cudaStream_t)stream);
    *iters = it;
    return r;
  });
}

int hs_factor_info(hs_factor f, hs_info *info) {
  return hs::guarded([&]() -> int {
    if (!f || !info) fail(HS_ERR_INVALID, "null argument");
    *info = f->h.info;
    return HS_OK;
  });
}

int hs_factor_ranks(hs_factor f, int32_t level, int32_t *ranks, int32_t cap, int32_t *count) {
  return hs::guarded([&]() -> int {
    if (!f || !count) fail(HS_ERR_INVALID, "null argument");
    const hs::Plan &p = f->h.plan;
    if (level < 2 || level > p.L) fail(HS_ERR_INVALID, "level out of range");
    const auto &rk = f->h.ranks[p.L - level];
    *count = (int32_t)rk.size();
    for (int32_t i = 0; i < (int32_t)rk.size() && i < cap && ranks; ++i) ranks[i] = rk[i];
    return HS_OK;
  });
}

int hs_factor_destroy(hs_factor f) {
  return hs::guarded([&]() -> int {
    delete f;
    return HS_OK;
  });
}

int hs_plan_create(int64_t n, const int32_t *rowptr, const int32_t *col, const hs_clustering *cl,
                   hs_plan *out) {
  return hs::guarded([&]() -> int {
    if (!rowptr || !col || !cl || !cl->perm || !cl->leaf_ptr || !out) fail(HS_ERR_INVALID, "null argument");
    *out = nullptr;
    std::unique_ptr<hs_plan_s> p(new hs_plan_s());
    hs::build_plan(n, rowptr, col, cl->perm, cl->leaf_ptr, cl->nleaf, p->p, hs::nbr_rule(cl->nbr_dist));
    *out = p.release();
    return HS_OK;
  });
}

int hs_plan_level_waves(hs_plan p, int32_t level, int32_t *wave_of, int32_t cap, int32_t *nwaves) {
  return hs::guarded([&]() -> int {
    if (!p || !nwaves) fail(HS_ERR_INVALID, "null argument");
    const hs::Plan &P = p->p;
    if (level < 2 || level > P.L) fail(HS_ERR_INVALID, "level out of range");
    const hs::PlanLevel &lv = P.levels[P.L - level];
    *nwaves = (int32_t)lv.waves.size();
    for (int i = 0; i < lv.nsup && i < cap && wave_of; ++i) wave_of[i] = lv.sup[i].wave;
    return HS_OK;
  });
}

int hs_plan_super_lists(hs_plan p, int32_t level, int32_t s, int32_t *nbrs, int32_t *wsep, int32_t cap,
                        int32_t *nn, int32_t *nw) {
  return hs::guarded([&]() -> int {
    if (!p || !nn || !nw) fail(HS_ERR_INVALID, "null argument");
    const hs::Plan &P = p->p;
    if (level < 2 || level > P.L) fail(HS_ERR_INVALID, "level out of range");
    const hs::PlanLevel &lv = P.levels[P.L - level];
    if (s < 0 || s >= lv.nsup) fail(HS_ERR_INVALID, "super node out of range");
    const hs::PlanSuper &ps = lv.sup[s];
    *nn = (int32_t)ps.N.size();
    *nw = (int32_t)ps.W.size();
    for (int i = 0; i < (int)ps.N.size() && i < cap && nbrs; ++i) nbrs[i] = ps.N[i];
    for (int i = 0; i < (int)ps.W.size() && i < cap && wsep; ++i) wsep[i] = ps.W[i];
    return HS_OK;
  });
}

int hs_plan_destroy(hs_plan p) {
  return hs::guarded([&]() -> int {
    delete p;
    return HS_OK;
  });
}

}  // extern "C"
