// Numeric factorization (Algorithm 1; Sec. 3.2 compression / extension /
// elimination; Sec. 6 GC basis), level by level and wave by wave.
//
// Per wave every super node s of the wave is processed by batched kernels:
//   A. gather [A_sn]_n (kept as a factor record) and [A_sw]_w; L^-1 of
//      A_ss = L L^T; Gram G = A_sw A_sw^T and a = A_sw phi_w; truncation -> U, k.
//      One device->host read of the ranks k (sizes of the new red nodes).
//   B. L^-1 U = Q R by CholQR2 (twice: Q1 = L^-1 U R1^-1, Q = Q1 R2^-1), then
//        P_ss = R^-1 Q^T L^-1            M_ss = L^-T L^-1 - (L^-T Q)(L^-T Q)^T
//        A_rr = S^-1 = R^-1 R^-T          A_nr = (L^-1 A_sn)^T Q R^-T
//        A_rw = U^T A_sw (= R_w^T)        phi_r = U^T phi_s
//        Z_s  = (L^-1 A_sN)^T (L^-1 A_sN) - (Q^T L^-1 A_sN)^T (Q^T L^-1 A_sN)
//      and the Schur update A_nn' -= Z_s[n, n'] gathered per target block with
//      the contributions of the wave summed in ascending super-node order.
// Identities: S = U^T A_ss^-1 U = R^T R, P_ss = S^-1 U^T A_ss^-1,
// M_ss = A_ss^-1 - P_ss^T S P_ss = L^-T (I - Q Q^T) L^-1, and
// A_ns M_ss A_sn' is the Schur term of ~~A_nn' (eq. eliminated).
//
// One executor (execute) drives one problem or many independent ones in lock
// step: at every step (level from the leaves, wave) all problems that have it
// share the launches.  Truncations of nodes with m >= 128 spread their
// tridiagonalisation over the GPU (trunc_grid); Cholesky factors above the
// shared-memory limit are blocked (Exec::chol_inv_blocked).
#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <type_traits>

#include "flat_map.h"
#include "handle.h"

namespace hs {

// ---------------------------------------------------------------------------
// DevArena
// ---------------------------------------------------------------------------
void *DevAlloc::get(size_t bytes, cudaStream_t st) const {
  if (!fa) {
    void *p = nullptr;
    HS_CUDA(cudaMalloc(&p, bytes));
    return p;
  }
  void *p = fa((uint64_t)bytes, device, (void *)st, ctx);
  if (!p) fail(HS_ERR_OOM, "the allocator hook returned no memory for " + std::to_string(bytes) + " bytes");
  if ((uintptr_t)p & 255) {
    put(p, st);
    fail(HS_ERR_INVALID, "the allocator hook returned a pointer that is not 256-byte aligned");
  }
  return p;
}

void DevAlloc::put(void *p, cudaStream_t st) const noexcept {
  if (!p) return;
  if (!ff) {
    cudaFree(p);
    return;
  }
  // the library's work that used the block is on `st` (a handle's calls are
  // ordered); a device-wide synchronisation here would also invalidate
  // graph captures other threads have under way on this device
  if (cudaStreamSynchronize(st) != cudaSuccess) cudaGetLastError();   // not left for a later check
  ff(p, device, (void *)st, ctx);
}

DevArena::~DevArena() {
  for (auto &c : chunks_) al_.put(c.first, st_);
}

void *DevArena::alloc(size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  while (cur_ >= 0 && cur_ < (int)chunks_.size() && off_ + bytes > chunks_[cur_].second) {
    ++cur_;
    off_ = 0;
  }
  if (cur_ < 0 || cur_ >= (int)chunks_.size()) {
    const size_t sz = std::max(min_chunk_, bytes);
    char *p = (char *)al_.get(sz, st_);
    chunks_.push_back({p, sz});
    cur_ = (int)chunks_.size() - 1;
    off_ = 0;
    reserved_ += sz;
  }
  void *r = chunks_[cur_].first + off_;
  off_ += bytes;
  used_ += bytes;
  return r;
}

void DevArena::reset() {
  cur_ = chunks_.empty() ? -1 : 0;
  off_ = 0;
  used_ = 0;
}

namespace {

inline uint64_t bkey(int a, int b) {
  if (a > b) std::swap(a, b);
  return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
}

template <typename T>
struct BlockRef {
  T *ptr;
  int ld;
  int rowkey;  // key whose unknowns index the rows of the stored matrix
};

// Pinned host staging for descriptor uploads, two buffers used in alternate
// waves: a wave's host->device copies have completed by the next wave's
// synchronisation, so a buffer is rewritten only two waves later.  Callers
// flip (next_wave) once per synchronised step and never twice between two
// synchronisations.
struct Staging {
  char *buf[2] = {nullptr, nullptr};
  size_t cap[2] = {0, 0};
  size_t off = 0;
  int cur = 0;
  std::vector<char *> retired;  // outgrown buffers, freed after the final synchronisation
  ~Staging() {
    for (int i = 0; i < 2; ++i) cudaFreeHost(buf[i]);
    for (char *p : retired) cudaFreeHost(p);
  }
  void next_wave() {
    cur ^= 1;
    off = 0;
  }
  char *put(const char *src, size_t n) {
    size_t o = (off + 255) & ~(size_t)255;
    if (o + n > cap[cur]) {
      if (buf[cur]) retired.push_back(buf[cur]);
      cap[cur] = std::max<size_t>(std::max<size_t>(2 * cap[cur], n + 256), (size_t)4 << 20);
      HS_CUDA(cudaMallocHost(&buf[cur], cap[cur]));
      o = 0;
    }
    std::memcpy(buf[cur] + o, src, n);
    off = o + n;
    return buf[cur] + o;
  }
};

struct Uploader {
  std::vector<char> buf;
  template <typename X>
  size_t add(const std::vector<X> &v) {
    const size_t off = (buf.size() + 15) & ~(size_t)15;
    buf.resize(off + v.size() * sizeof(X));
    if (!v.empty()) std::memcpy(buf.data() + off, v.data(), v.size() * sizeof(X));
    return off;
  }
  char *upload(DevArena &a, Staging &sg, cudaStream_t st) {
    if (buf.empty()) return nullptr;
    char *d = (char *)a.alloc(buf.size());
    const char *h = sg.put(buf.data(), buf.size());
    HS_CUDA(cudaMemcpyAsync(d, h, buf.size(), cudaMemcpyHostToDevice, st));
    return d;
  }
};

// Receives an event before and after each tensor-core launch of a GEMM batch
// (with the flops of the tasks launched), for the kernel's device time.
struct TcTimer {
  virtual void before(cudaStream_t st) = 0;
  virtual void after(cudaStream_t st, double flops) = 0;
  virtual ~TcTimer() = default;
};

template <typename T>
struct GemmBatch {
  std::vector<GemmTask<T>> tasks;
  double flops = 0.0;
  int tc = HS_TC_NONE;   // float batches: run on the tensor cores in this precision
  void add(const T *A, int lda, int ta, const T *B, int ldb, int tb, T *C, int ldc, int M, int N,
           int K, T alpha, T beta) {
    if (M <= 0 || N <= 0) return;
    if (K <= 0 && beta == T(1)) return;
    GemmTask<T> t;
    t.A = A;
    t.B = B;
    t.C = C;
    t.M = M;
    t.N = N;
    t.K = K;
    t.lda = lda;
    t.ldb = ldb;
    t.ldc = ldc;
    t.ta = ta;
    t.tb = tb;
    t.alpha = alpha;
    t.beta = beta;
    tasks.push_back(t);
    flops += 2.0 * M * N * (double)std::max(K, 0);
  }
  // d_err: error word of the tensor-core kernel (bounded waits).  With `tc`
  // set, each task goes to the variant the autotuner picked for its shape
  // (CUDA-core kernel, or tensor-core kernel with 64- or 128-wide tiles): up
  // to three launches, whose tasks are independent of each other.
  void launch(DevArena &scr, Staging &sg, cudaStream_t st, int *d_err = nullptr, TcTimer *timer = nullptr,
              long long wait_cycles = 0) {
    if (tasks.empty()) return;
    const bool on_tc = std::is_same<T, float>::value && tc != HS_TC_NONE;
    std::vector<GemmTask<T>> part[3];
    if (on_tc) {
      for (const GemmTask<T> &t : tasks) {
        const int r = gemm_route(tc, t.M, t.N, t.K);
        part[r == 0 ? 0 : r == 64 ? 1 : 2].push_back(t);
      }
    } else {
      part[0].swap(tasks);
    }
    tasks.clear();
    const int tms[3] = {GEMM_TM, TC_TILE_M, TC_TILE_M}, tns[3] = {GEMM_TN, 64, 128};
    for (int v = 0; v < 3; ++v) {
      if (part[v].empty()) continue;
      std::vector<int> tile_start;
      int tiles = 0;
      for (const GemmTask<T> &t : part[v]) {
        tile_start.push_back(tiles);
        tiles += ((t.M + tms[v] - 1) / tms[v]) * ((t.N + tns[v] - 1) / tns[v]);
      }
      Uploader u;
      const size_t ot = u.add(part[v]);
      const size_t os = u.add(tile_start);
      char *d = u.upload(scr, sg, st);
      if (v == 0) {
        launch_gemm<T>((const GemmTask<T> *)(d + ot), (const int *)(d + os), (int)part[v].size(), tiles, st);
        continue;
      }
      if constexpr (std::is_same<T, float>::value) {
        if (!d_err) fail(HS_ERR_INVALID, "internal: tensor-core GEMM launched without an error word");
        double f = 0.0;
        for (const GemmTask<T> &t : part[v]) f += 2.0 * t.M * t.N * (double)std::max(t.K, 0);
        if (timer) timer->before(st);
        launch_gemm_tc(tc, tns[v], (const GemmTask<float> *)(d + ot), (const int *)(d + os), (int)part[v].size(),
                       tiles, d_err, st, wait_cycles);
        if (timer) timer->after(st, f);
      }
    }
  }
};

template <typename T>
struct SumBatch {
  std::vector<SumTask<T>> tasks;
  std::vector<SumSrc<T>> srcs;
  std::vector<int> tile_start;
  int tiles = 0;
  // begins a task; sources are appended with src() afterwards
  void begin(T *dst, int ld, int rows, int cols, T alpha, T beta) {
    SumTask<T> t;
    t.dst = dst;
    t.ld = ld;
    t.rows = rows;
    t.cols = cols;
    t.first = (int)srcs.size();
    t.nsrc = 0;
    t.alpha = alpha;
    t.beta = beta;
    tasks.push_back(t);
  }
  void src(const T *p, int ld, int trans) {
    SumSrc<T> s;
    s.ptr = p;
    s.ld = ld;
    s.trans = trans;
    srcs.push_back(s);
    tasks.back().nsrc++;
  }
  void end() {
    SumTask<T> &t = tasks.back();
    if (t.rows <= 0 || t.cols <= 0 || (t.nsrc == 0 && t.beta == T(1))) {
      srcs.resize(t.first);
      tasks.pop_back();
      return;
    }
    tile_start.push_back(tiles);
    tiles += ((t.rows + SUM_TILE - 1) / SUM_TILE) * ((t.cols + SUM_TILE - 1) / SUM_TILE);
  }
  void copy(T *dst, int ld, int rows, int cols, const T *s, int sld, int trans) {
    begin(dst, ld, rows, cols, T(1), T(0));
    src(s, sld, trans);
    end();
  }
  void launch(DevArena &scr, Staging &sg, cudaStream_t st) {
    if (tasks.empty()) return;
    Uploader u;
    const size_t ot = u.add(tasks);
    const size_t os = u.add(srcs);
    const size_t ol = u.add(tile_start);
    char *d = u.upload(scr, sg, st);
    launch_sum<T>((const SumTask<T> *)(d + ot), (const SumSrc<T> *)(d + os), (const int *)(d + ol),
                  (int)tasks.size(), tiles, st);
    tasks.clear();
    srcs.clear();
    tile_start.clear();
    tiles = 0;
  }
};

// What a Cholesky status word refers to; formatted only when it reports a failure.
struct Tag {
  int kind;   // 0 A_ss, 1 S (first CholQR pass), 2 S (second pass), 3 U^T U, 4 root block
  int level;
  int s;
  int prob;   // problem of a batched factorization (-1: a single one)
};

inline std::string describe(const Tag &t) {
  static const char *names[] = {"A_ss", "S (first CholQR pass)", "S (second CholQR pass)", "U^T U", "root block"};
  const std::string pre = t.prob >= 0 ? "problem " + std::to_string(t.prob) + ": " : std::string();
  if (t.kind == 4) return pre + "root block";
  return pre + "level " + std::to_string(t.level) + " super node " + std::to_string(t.s) + ": " + names[t.kind];
}

template <typename T>
struct CholBatch {
  std::vector<CholTask<T>> tasks;
  std::vector<Tag> what;
  int max_m = 0;
  double flops = 0.0;
  void add(const T *A, int lda, T *Linv, int m, const Tag &w) {
    if (m <= 0) return;
    CholTask<T> t;
    t.A = A;
    t.Linv = Linv;
    t.m = m;
    t.lda = lda;
    t.ldl = m;
    t.status_idx = (int)tasks.size();
    tasks.push_back(t);
    what.push_back(w);
    max_m = std::max(max_m, m);
    flops += 2.0 * (double)m * m * m / 3.0;
  }
};

// Largest super node whose truncation uses the shared-memory Jacobi kernel
// (default 32: above that the tridiagonal path needs fewer operations than
// the ~10 Jacobi sweeps, and on the 512 x 512 workload it took less time);
// larger ones use the tridiagonal path.
// HS_EIG_SMALL_MAX (environment) lowers the limit, which lets small test
// problems exercise the tridiagonal path.
template <typename T>
int eig_small_max() {
  static const int v = [] {
    const char *e = std::getenv("HS_EIG_SMALL_MAX");
    const int cap = std::min(32, jacobi_cap<T>());
    if (!e) return cap;
    const int x = std::atoi(e);
    return x < 0 ? cap : std::min(x, cap);
  }();
  return v;
}

std::atomic<int> g_phase_prof{0};
bool phase_profiling() { return g_phase_prof.load() != 0; }

// The cluster tridiagonalisation of the multi-CTA path (HS_TRI_CLUSTER=0 in
// the environment turns it off: every node then takes the step kernels).
inline bool tri_cluster_enabled() {
  static const bool v = [] {
    const char *e = std::getenv("HS_TRI_CLUSTER");
    return !(e && e[0] == '0');
  }();
  return v;
}

// Smallest super node whose truncation takes the multi-CTA path (cluster or
// step-kernel tridiagonalisation, eigenvectors of T for the whole wave,
// reflector products by batches of columns); below it one CTA per node does
// everything (default 64).  HS_GRID_TRIDIAG_MIN (environment) moves the
// limit, which lets small test problems exercise the path.
inline int grid_tridiag_min() {
  static const int v = [] {
    const char *e = std::getenv("HS_GRID_TRIDIAG_MIN");
    const int x = e ? std::atoi(e) : 0;
    return x > 3 ? x : 64;
  }();
  return v;
}

template <typename T>
T *talloc(DevArena &a, size_t n) {
  return (T *)a.alloc(sizeof(T) * std::max<size_t>(n, 1));
}

// Pending device status words checked at the next synchronisation point.
struct PendingStatus {
  int *d = nullptr;
  std::vector<Tag> what;
};

// What the launches of one factorization step share: the stream, an arena for
// task descriptors, the pinned staging buffers, the status words to check and
// the host buffer of the per-wave rank read.  One Exec drives one problem, or
// many independent problems whose steps are batched into the same launches.
struct Exec : TcTimer {
  cudaStream_t st = nullptr;
  DevArena scr{16ull << 20};
  Staging sg;
  std::vector<PendingStatus> pending;
  DevArena stat{1ull << 20};   // status words: kept until the sync_check that reads them
  int *hbuf = nullptr;
  size_t hbuf_cap = 0;
  cudaEvent_t ev_big[2] = {nullptr, nullptr};
  // batched: a problem whose pivot fails is marked here and leaves the lock
  // step; the others go on (single: the failure is an error of the call)
  std::vector<int> prob_status;
  std::vector<std::string> prob_msg;
  // host time spent waiting for the device (sync_check), in ms
  double wait_ms = 0.0;
  // tensor-core precision of the elimination's contractions (HS_TC_NONE for
  // the FP64 and FP32 factors) and the error word of that kernel's bounded
  // waits, read at every sync_check after a tensor-core launch
  int tc = HS_TC_NONE;
  int *d_err = nullptr;
  bool tc_pending = false;
  long long wait_cycles = 0;   // bound of the kernels' waits (hs_opts.timeout_cycles; 0 = default)
  // device time of the tensor-core launches: an event pair around each,
  // read and summed at the next sync_check (the pairs are then reused)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tc_ev;
  size_t tc_ev_used = 0;
  double tc_ms = 0.0, tc_flops = 0.0;
  int64_t tc_launches = 0;
  // optional device time per phase (hs_profile_phases): event pairs around
  // each launch group, read after the final synchronisation
  bool prof = false;
  struct Span {
    int phase;
    cudaEvent_t e0, e1;
  };
  std::vector<Span> spans;
  std::vector<size_t> open;     // spans begun and not yet ended (nesting)
  void begin(int phase) {
    if (!prof) return;
    Span sp{phase, nullptr, nullptr};
    HS_CUDA(cudaEventCreate(&sp.e0));
    HS_CUDA(cudaEventCreate(&sp.e1));
    HS_CUDA(cudaEventRecord(sp.e0, st));
    open.push_back(spans.size());
    spans.push_back(sp);
  }
  void end() {
    if (!prof || open.empty()) return;
    HS_CUDA(cudaEventRecord(spans[open.back()].e1, st));
    open.pop_back();
  }
  void phase_times(double *ms, int nphase) {
    for (Span &sp : spans) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, sp.e0, sp.e1) == cudaSuccess && sp.phase < nphase) ms[sp.phase] += t;
    }
  }
  // a second stream for work that runs beside the factor stream (joined
  // back by an event before anything depends on it)
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaStream_t side_stream() {
    if (!side) {
      HS_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
      HS_CUDA(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
      HS_CUDA(cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming));
    }
    return side;
  }
  explicit Exec(cudaStream_t s) : st(s) {
    HS_CUDA(cudaEventCreate(&ev_big[0]));
    HS_CUDA(cudaEventCreate(&ev_big[1]));
  }
  // the device memory of this factorization's descriptors and status words
  // comes from the (first) handle's source; set before the first allocation
  DevAlloc al;
  void use_alloc(const DevAlloc &a) {
    al = a;
    scr.set_alloc(a, st);
    stat.set_alloc(a, st);
  }
  ~Exec() {
    // copies from the pinned staging buffers may still be in flight after an error
    cudaStreamSynchronize(st);
    if (side) {
      cudaStreamSynchronize(side);
      cudaStreamDestroy(side);
      cudaEventDestroy(fork_ev);
      cudaEventDestroy(join_ev);
    }
    al.put(d_err, st);
    for (auto &e : tc_ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    for (Span &sp : spans) {
      cudaEventDestroy(sp.e0);
      cudaEventDestroy(sp.e1);
    }
    cudaFreeHost(hbuf);
    cudaEventDestroy(ev_big[0]);
    cudaEventDestroy(ev_big[1]);
  }
  int *host_ints(size_t n) {
    if (n > hbuf_cap) {
      cudaFreeHost(hbuf);
      hbuf = nullptr;
      hbuf_cap = std::max(n, (size_t)1 << 16);
      HS_CUDA(cudaMallocHost(&hbuf, hbuf_cap * sizeof(int)));
    }
    return hbuf;
  }
  bool mark_failed(const Tag &t, int pivot) {
    const std::string msg = describe(t) + " is not positive definite (pivot " + std::to_string(pivot) + ")";
    if (t.prob < 0 || t.prob >= (int)prob_status.size()) fail(HS_ERR_NOT_SPD, msg);
    if (prob_status[t.prob] == HS_OK) {
      prob_status[t.prob] = HS_ERR_NOT_SPD;
      prob_msg[t.prob] = msg;
    }
    return true;
  }
  bool ok(int prob) const { return prob < 0 || prob >= (int)prob_status.size() || prob_status[prob] == HS_OK; }
  // a GEMM batch: on the tensor cores in precision `tc` when that is set and
  // the batch is FP32, else on the CUDA cores
  template <typename T>
  void gemm(GemmBatch<T> &g, bool tensor_cores = true) {
    if (g.tasks.empty()) return;
    g.tc = (tensor_cores && std::is_same<T, float>::value) ? tc : HS_TC_NONE;
    if (g.tc != HS_TC_NONE) {
      if (!d_err) {
        al.get(&d_err, 256, st);
        HS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
      }
      tc_pending = true;
      g.launch(scr, sg, st, d_err, this, wait_cycles);
      return;
    }
    g.launch(scr, sg, st, d_err);
  }
  void before(cudaStream_t s) override {
    if (tc_ev_used == tc_ev.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
      HS_CUDA(cudaEventCreate(&e.first));
      HS_CUDA(cudaEventCreate(&e.second));
      tc_ev.push_back(e);
    }
    HS_CUDA(cudaEventRecord(tc_ev[tc_ev_used].first, s));
  }
  void after(cudaStream_t s, double flops) override {
    HS_CUDA(cudaEventRecord(tc_ev[tc_ev_used].second, s));
    ++tc_ev_used;
    tc_flops += flops;
  }
  // waits for the stream, then checks the pending status words
  void sync_check() {
    const auto t0 = std::chrono::steady_clock::now();
    HS_CUDA(cudaStreamSynchronize(st));
    wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (tc_pending) {
      int e = 0;
      HS_CUDA(cudaMemcpy(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (e) fail(HS_ERR_TIMEOUT, "a bounded wait of the tensor-core GEMM ran out");
      tc_pending = false;
      for (size_t i = 0; i < tc_ev_used; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, tc_ev[i].first, tc_ev[i].second) == cudaSuccess) tc_ms += t;
      }
      tc_launches += (int64_t)tc_ev_used;
      tc_ev_used = 0;
    }
    for (auto &ps : pending) {
      std::vector<int> hv(ps.what.size());
      HS_CUDA(cudaMemcpy(hv.data(), ps.d, ps.what.size() * sizeof(int), cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < ps.what.size(); ++i)
        if (hv[i] != 0) mark_failed(ps.what[i], hv[i] - 1);
    }
    pending.clear();
    stat.reset();
  }
  // Cholesky-inverse batch whose statuses are checked at the next sync_check
  template <typename T>
  void chol_checked(CholBatch<T> &cb) {
    if (cb.tasks.empty()) return;
    PendingStatus ps;
    ps.d = (int *)stat.alloc(sizeof(int) * cb.tasks.size());
    ps.what = cb.what;
    chol_inv_any<T>(cb.tasks, ps.d);
    pending.push_back(ps);
  }

  // L^-1 of A = L L^T for every task; status[t.status_idx] = 0 or failing
  // pivot + 1.  Matrices that fit in shared memory take one CTA each; larger
  // ones the blocked path below.
  template <typename T>
  void chol_inv_any(const std::vector<CholTask<T>> &tasks, int *status) {
    std::vector<CholTask<T>> small, large;
    int small_max = 0;
    for (const CholTask<T> &t : tasks) {
      if (t.m <= chol_smem_cap<T>()) {
        small.push_back(t);
        small_max = std::max(small_max, t.m);
      } else {
        large.push_back(t);
      }
    }
    if (!small.empty()) {
      Uploader u;
      const size_t o = u.add(small);
      char *d = u.upload(scr, sg, st);
      launch_chol_inv<T>((const CholTask<T> *)(d + o), (int)small.size(), status, small_max, st);
    }
    if (!large.empty()) chol_inv_blocked<T>(large, status);
  }

  // Blocked right-looking Cholesky with the block-triangular inverse, for
  // matrices too large for one CTA (at the top levels of 3D problems the
  // pivot blocks reach thousands of unknowns).  Block columns of kCholNb:
  //   D_b = L_bb^-1 (one CTA, shared memory), panel L_ib = W_ib D_b^T,
  //   trailing update W_ik -= L_ib L_kb^T (batched GEMMs over the GPU);
  // then block rows of X = L^-1: X_ii = D_i, X_i,0:i = -D_i (L_i,0:i X_0:i,0:i).
  // All large tasks of the batch advance together, one launch per kind and
  // block step.
  template <typename T>
  void chol_inv_blocked(const std::vector<CholTask<T>> &tasks, int *status) {
    constexpr int nb = 128;
    struct Work {
      CholTask<T> t;
      T *W, *Lf, *D, *Tb;
      int nblk;
      int *bs;
    };
    std::vector<Work> w;
    int maxblk = 0, nbs = 0;
    for (const CholTask<T> &t : tasks) {
      Work x;
      x.t = t;
      const size_t m = (size_t)t.m;
      x.W = (T *)scr.alloc(sizeof(T) * m * m);
      x.Lf = (T *)scr.alloc(sizeof(T) * m * m);
      x.nblk = (t.m + nb - 1) / nb;
      x.D = (T *)scr.alloc(sizeof(T) * (size_t)x.nblk * nb * nb);
      x.Tb = (T *)scr.alloc(sizeof(T) * (size_t)nb * m);
      x.bs = nullptr;
      nbs += x.nblk;
      maxblk = std::max(maxblk, x.nblk);
      w.push_back(x);
    }
    int *bs = (int *)stat.alloc(sizeof(int) * nbs);
    {
      int off = 0;
      SumBatch<T> cp;
      for (Work &x : w) {
        x.bs = bs + off;
        off += x.nblk;
        cp.copy(x.W, x.t.m, x.t.m, x.t.m, x.t.A, x.t.lda, 0);
        // the inverse is lower triangular with a zero strict upper part
        HS_CUDA(cudaMemsetAsync(x.t.Linv, 0, sizeof(T) * (size_t)x.t.m * x.t.m, st));
      }
      cp.launch(scr, sg, st);
    }
    for (int b = 0; b < maxblk; ++b) {
      std::vector<CholTask<T>> dc;
      GemmBatch<T> pan, trl;
      for (Work &x : w) {
        if (b >= x.nblk) continue;
        const int m = x.t.m, j0 = b * nb, jb = std::min(nb, m - j0), rest = m - j0 - jb;
        T *Db = x.D + (size_t)b * nb * nb;
        CholTask<T> c;
        c.A = x.W + (size_t)j0 * m + j0;
        c.lda = m;
        c.Linv = Db;
        c.ldl = jb;
        c.m = jb;
        c.status_idx = (int)(x.bs - bs) + b;
        dc.push_back(c);
        if (rest > 0) {
          T *Lp = x.Lf + (size_t)(j0 + jb) * m + j0;
          pan.add(x.W + (size_t)(j0 + jb) * m + j0, m, 0, Db, jb, 1, Lp, m, rest, jb, jb, T(1), T(0));
          trl.add(Lp, m, 0, Lp, m, 1, x.W + (size_t)(j0 + jb) * m + j0 + jb, m, rest, rest, jb, T(-1), T(1));
        }
      }
      Uploader u;
      const size_t o = u.add(dc);
      char *d = u.upload(scr, sg, st);
      launch_chol_inv<T>((const CholTask<T> *)(d + o), (int)dc.size(), bs, nb, st);
      gemm(pan, false);   // the Cholesky of A_ss stays in FP32 on every path
      gemm(trl, false);
    }
    for (int b = 0; b < maxblk; ++b) {
      GemmBatch<T> g1, g2;
      SumBatch<T> dg;
      for (Work &x : w) {
        if (b >= x.nblk) continue;
        const int m = x.t.m, i0 = b * nb, jb = std::min(nb, m - i0);
        const T *Db = x.D + (size_t)b * nb * nb;
        if (b > 0) {
          g1.add(x.Lf + (size_t)i0 * m, m, 0, x.t.Linv, m, 0, x.Tb, m, jb, i0, i0, T(1), T(0));
          g2.add(Db, jb, 0, x.Tb, m, 0, x.t.Linv + (size_t)i0 * m, m, jb, i0, jb, T(-1), T(0));
        }
        dg.copy(x.t.Linv + (size_t)i0 * m + i0, m, jb, jb, Db, jb, 0);
      }
      gemm(g1, false);
      gemm(g2, false);
      dg.launch(scr, sg, st);
    }
    std::vector<StatusMerge> sm;
    for (Work &x : w) sm.push_back(StatusMerge{x.bs, x.nblk, nb, status + x.t.status_idx});
    Uploader u;
    const size_t o = u.add(sm);
    char *d = u.upload(scr, sg, st);
    launch_status_merge((const StatusMerge *)(d + o), (int)sm.size(), st);
  }
};

// The batched launches of one wave step, shared by the problems taking part.
template <typename T>
struct WaveBatches {
  // phase A: gather, Cholesky of A_ss, Gram, truncation (statuses and ranks read back)
  SumBatch<T> gather;
  GemmBatch<T> gram;
  CholBatch<T> chol;
  std::vector<TruncTask<T>> trunc, trunc_big;
  int max_trunc_m = 0, max_big_m = 0;
  // the FP64 truncation of the mixed factors (hs_opts.rank_f64): FP64 copies
  // of A_sW, phi_W and phi_s, their Gram, FP64 truncation tasks (ranks in the
  // slots after the T tasks', from k_off64 on), the basis narrowed to T
  std::vector<ConvTask> widen, narrow;
  GemmBatch<double> gram64;
  std::vector<TruncTask<double>> trunc64, trunc_big64;
  int max_trunc64_m = 0, max_big64_m = 0;
  size_t k_off64 = 0;
  // large-path re-orthonormalisation of U (CholQR2)
  GemmBatch<T> o1, o2, o3, o4;
  CholBatch<T> oc1, oc2;
  // phase B and the Schur update
  GemmBatch<T> g1, g2, g3, g4, g5, g6, g7, g8;
  CholBatch<T> c1, c2;
  SumBatch<T> schur;
};

template <typename T>
class Run {
 public:
  Run(FactorHandle &h, const double *phi_host, Exec &ex, int prob)
      : h_(h), P_(h.plan), ex_(ex), st_(ex.st), prob_(prob) {
    use_phi_ = h.variant != HS_LORASP;
    phi_host_ = phi_host;
    h.stream = ex.st;
  }

  bool ok() const { return ex_.ok(prob_); }
  int levels() const { return (int)P_.levels.size(); }
  int waves(int li) const { return li < levels() ? (int)P_.levels[li].waves.size() : 0; }
  FactorHandle &handle() { return h_; }

  void begin();                                  // outputs cleared, leaf blocks
  void level_begin(int li, SumBatch<T> &sb);     // merge into the level's super nodes
  void wave_a(int li, int widx, WaveBatches<T> &B);
  void wave_b(const int *hb, size_t nchol, size_t ntrunc, double big_ms, WaveBatches<T> &B);
  // the elimination's GEMM tasks of super nodes [c_next_, c_next_ + count)
  // of the wave; returns whether nodes remain
  bool wave_c(WaveBatches<T> &B, size_t count);
  void wave_d(WaveBatches<T> &B);               // Schur targets, red-node blocks, apply records
  void level_end(int li);
  void root_a(SumBatch<T> &sb);                  // merge of the last red nodes
  void root_b(CholBatch<T> &cb, GemmBatch<T> &g);
  void finish();

 private:
  struct Sup {
    int s = 0, m = 0, k = 0, dN = 0, dW = 0;
    std::vector<int> Noff, Woff;
    T *AsN = nullptr, *AsW = nullptr, *phiW = nullptr, *Linv = nullptr, *G = nullptr, *a = nullptr;
    T *U = nullptr, *work = nullptr;
    T *Ut = nullptr, *S1 = nullptr, *L1 = nullptr, *Q1 = nullptr, *S2 = nullptr, *L2 = nullptr;
    T *Q = nullptr, *Rinv = nullptr, *Wt = nullptr, *Gt = nullptr, *Tm = nullptr, *Z = nullptr;
    T *M = nullptr, *Pm = nullptr, *ANr = nullptr, *Arr = nullptr, *ArW = nullptr, *phir = nullptr;
    bool red = false;
  };

  void leaf_setup();
  void merge(int nred, int key_base, SumBatch<T> &sb);
  void end_level(const PlanLevel &lv, int li);
  Tag tag(int kind, int level, int s) const { return Tag{kind, level, s, prob_}; }
  // the truncation (Gram, eigen-solve, rank) in FP64 on an FP32 factor
  bool rank64() const { return std::is_same<T, float>::value && h_.rank_f64; }
  // tolerance of the super nodes of a level (adaptive list indexed from the leaves)
  double level_eps(int level) const {
    const int j = P_.L - level;
    return (j >= 0 && j < (int)h_.eps_level.size()) ? h_.eps_level[j] : h_.eps;
  }

  FactorHandle &h_;
  const Plan &P_;
  Exec &ex_;
  cudaStream_t st_;
  int prob_;
  bool use_phi_ = false;
  const double *phi_host_ = nullptr;

  FlatMap<BlockRef<T>> blocks_;
  std::vector<int> size_;      // by key of the current level
  std::vector<T *> phi_;       // by key
  int nsup_ = 0;
  int nred_ = 0;               // red nodes entering the current level
  // vector layout of the apply workspace
  int64_t seg_off_ = 0;             // segment of the current level's red/super nodes
  std::vector<int64_t> red_off_;    // red node offsets inside that segment (by red index)
  int64_t seg_size_ = 0;
  std::vector<int64_t> sup_off_;    // super node offsets inside the segment
  // records of the current level, resolved at the level end
  struct Rec {
    int node;       // index into h_.nodes
    int s;
    std::vector<int> N;
  };
  std::vector<Rec> recs_;
  // the wave in progress: its super nodes and its slices of the shared batches
  const PlanLevel *lv_ = nullptr;
  std::vector<Sup> cur_;
  std::vector<int> trunc_sup_, big_sup_;      // super nodes of this run's truncation tasks
  std::vector<int> trunc64_sup_, big64_sup_;  // the same for the FP64 truncation tasks
  size_t chol_first_ = 0, chol_count_ = 0, trunc_first_ = 0, big_first_ = 0;
  size_t trunc64_first_ = 0, big64_first_ = 0;
  size_t c_next_ = 0;   // next super node of the wave whose phase-B tasks are built
  double flops_ = 0.0;
  // device time (of the launches taken part in) and nominal eigen-solve flops
  // of the large-node truncations
  double big_ms_ = 0.0, big_flops_ = 0.0, eig_flops_ = 0.0, alg_flops_ = 0.0;
  int big_launches_ = 0;
  // root records waiting for root_b
  T *root_linv_ = nullptr, *root_ainv_ = nullptr;
};

// Leaf red nodes and their blocks from the permuted CSR (Sec. 2.1: blocks
// A_{I_i I_j} of the leaf partition).  Entries below the block diagonal are
// taken from their symmetric counterpart.
template <typename T>
void Run<T>::leaf_setup() {
  const int nleaf = P_.nleaf;
  const auto &lp = P_.leaf_ptr;
  size_.assign(nleaf, 0);
  for (int i = 0; i < nleaf; ++i) size_[i] = lp[i + 1] - lp[i];
  if (!h_.d_leaf_dest) {
    // block list, storage offsets and the entry -> block position map (once per pattern)
    std::vector<int> leaf_of(P_.n);
    for (int i = 0; i < nleaf; ++i)
      for (int p = lp[i]; p < lp[i + 1]; ++p) leaf_of[p] = i;
    FlatMap<int64_t> off;
    h_.leaf_blocks.clear();
    h_.leaf_block_off.clear();
    int64_t total = 0;
    for (int64_t p = 0; p < P_.n; ++p)
      for (int e = P_.prow[p]; e < P_.prow[p + 1]; ++e) {
        const int a = leaf_of[p], b = leaf_of[P_.pcol[e]];
        if (a > b) continue;
        const uint64_t key = bkey(a, b);
        if (!off.count(key)) {
          off[key] = total;
          h_.leaf_blocks.emplace_back(a, b);
          h_.leaf_block_off.push_back(total);
          total += ((int64_t)size_[a] * size_[b] + 3) & ~(int64_t)3;
        }
      }
    std::vector<int64_t> dest(P_.nnz, -1);
    for (int64_t p = 0; p < P_.n; ++p)
      for (int e = P_.prow[p]; e < P_.prow[p + 1]; ++e) {
        const int c = P_.pcol[e];
        const int a = leaf_of[p], b = leaf_of[c];
        if (a > b) continue;
        dest[e] = off[bkey(a, b)] + (int64_t)(p - lp[a]) * size_[b] + (c - lp[b]);
      }
    h_.alloc.get(&h_.d_leaf_dest, sizeof(int64_t) * std::max<int64_t>(P_.nnz, 1), st_);
    HS_CUDA(cudaMemcpyAsync(h_.d_leaf_dest, dest.data(), sizeof(int64_t) * P_.nnz, cudaMemcpyHostToDevice, st_));
    h_.leaf_total = total;
    if (use_phi_) {
      // preserved vectors of the leaves (GC): ones, or the caller's vectors
      // permuted; n x nphi row-major (a node's rows are contiguous)
      const int np = h_.nphi;
      const bool user = h_.variant == HS_GC_USER || h_.variant == HS_GC_PROJ;
      std::vector<T> ph((size_t)P_.n * np);
      for (int64_t p = 0; p < P_.n; ++p)
        for (int j = 0; j < np; ++j)
          ph[(size_t)p * np + j] = user ? (T)phi_host_[(size_t)j * P_.n + P_.perm[p]] : T(1);
      h_.alloc.get(&h_.d_phi0, sizeof(T) * ph.size(), st_);
      if (h_.scale && user) {
        // the caller's vectors are kept; each factorization maps them to D^1/2 phi
        h_.alloc.get(&h_.d_phi_raw, sizeof(T) * ph.size(), st_);
        HS_CUDA(cudaMemcpyAsync(h_.d_phi_raw, ph.data(), sizeof(T) * ph.size(), cudaMemcpyHostToDevice, st_));
      } else {
        HS_CUDA(cudaMemcpyAsync(h_.d_phi0, ph.data(), sizeof(T) * ph.size(), cudaMemcpyHostToDevice, st_));
      }
    }
  }
  if (h_.d_phi_raw)
    launch_phi_scale<T>((const T *)h_.d_phi_raw, h_.d_dscale, P_.n, h_.nphi, (T *)h_.d_phi0, st_);
  const int64_t total = h_.leaf_total;
  T *base = talloc<T>(*h_.pers, total);
  HS_CUDA(cudaMemsetAsync(base, 0, sizeof(T) * std::max<int64_t>(total, 1), st_));
  launch_scatter_values<T>(h_.factor_values(), h_.d_leaf_dest, P_.nnz, base, st_);
  blocks_.clear();
  blocks_.reserve(h_.leaf_blocks.size());
  for (size_t i = 0; i < h_.leaf_blocks.size(); ++i) {
    const auto &ab = h_.leaf_blocks[i];
    BlockRef<T> br;
    br.ptr = base + h_.leaf_block_off[i];
    br.ld = size_[ab.second];
    br.rowkey = ab.first;
    blocks_[bkey(ab.first, ab.second)] = br;
  }
  phi_.assign(nleaf, nullptr);
  if (use_phi_)
    for (int i = 0; i < nleaf; ++i) phi_[i] = (T *)h_.d_phi0 + (size_t)lp[i] * h_.nphi;
  // vector layout: level L segment = the permuted unknowns
  seg_off_ = 0;
  red_off_.assign(nleaf, 0);
  for (int i = 0; i < nleaf; ++i) red_off_[i] = lp[i];
  seg_size_ = P_.n;
}

// Merge the red nodes (keys key_base + i, i < nred) pairwise into super nodes
// (Sec. 3: I^s_i = I^r_{2i-1} u I^r_{2i}); blocks are assembled 2 x 2.
template <typename T>
void Run<T>::merge(int nred, int key_base, SumBatch<T> &sb) {
  const int nsup = std::max(1, nred / 2);
  std::vector<int> rsize(2 * nsup, -1);
  for (int i = 0; i < nred; ++i) rsize[i] = size_[key_base + i];
  std::vector<int> ssize(nsup, -1), coff(2 * nsup, 0);
  for (int j = 0; j < nsup; ++j) {
    int m = 0;
    bool any = false;
    for (int c = 2 * j; c <= 2 * j + 1; ++c)
      if (rsize[c] >= 0) {
        coff[c] = m;
        m += rsize[c];
        any = true;
      }
    ssize[j] = any ? m : -1;
  }
  // super-block list
  FlatMap<int64_t> off;
  off.reserve(blocks_.size());
  std::vector<std::pair<int, int>> order;
  std::vector<int64_t> order_off;
  int64_t total = 0;
  for (auto &kv : blocks_) {
    const int a = (int)(kv.first >> 32) - key_base, b = (int)(kv.first & 0xffffffffu) - key_base;
    if (a < 0 || b < 0 || a >= nred || b >= nred) fail(HS_ERR_INVALID, "internal: stray block at merge");
    const int I = a / 2, J = b / 2;
    auto ins = off.try_emplace(bkey(I, J));
    if (ins.second) {
      *ins.first = total;
      order.emplace_back(std::min(I, J), std::max(I, J));
      order_off.push_back(total);
      total += ((int64_t)ssize[I] * ssize[J] + 3) & ~(int64_t)3;
    }
  }
  T *base = talloc<T>(*h_.pers, total);
  HS_CUDA(cudaMemsetAsync(base, 0, sizeof(T) * std::max<int64_t>(total, 1), st_));
  FlatMap<BlockRef<T>> nb;
  nb.reserve(order.size());
  for (size_t q = 0; q < order.size(); ++q) {
    const auto &IJ = order[q];
    BlockRef<T> br;
    br.ptr = base + order_off[q];
    br.ld = ssize[IJ.second];
    br.rowkey = IJ.first;
    nb[bkey(IJ.first, IJ.second)] = br;
  }
  for (auto &kv : blocks_) {
    const int a = std::min((int)(kv.first >> 32), (int)(kv.first & 0xffffffffu)) - key_base;
    const int b = std::max((int)(kv.first >> 32), (int)(kv.first & 0xffffffffu)) - key_base;
    const BlockRef<T> &rb = kv.second;
    const int I = a / 2, J = b / 2;
    auto sit = nb.find(bkey(I, J));
    if (sit == nb.end()) fail(HS_ERR_INVALID, "internal: missing super block at merge");
    const BlockRef<T> sbk = sit->second;
    // rows a, cols b
    const int ta = (rb.rowkey - key_base == a) ? 0 : 1;
    sb.copy(sbk.ptr + (int64_t)coff[a] * sbk.ld + coff[b], sbk.ld, rsize[a], rsize[b], rb.ptr, rb.ld, ta);
    if (I == J && a != b)  // mirrored sub-block of a diagonal super block
      sb.copy(sbk.ptr + (int64_t)coff[b] * sbk.ld + coff[a], sbk.ld, rsize[b], rsize[a], rb.ptr, rb.ld,
              1 - ta);
  }
  // preserved vectors (m x nphi row-major per node): contiguous per level
  std::vector<T *> nphi(2 * nsup, nullptr);
  if (use_phi_) {
    const int np = h_.nphi;
    int64_t tot = 0;
    for (int j = 0; j < nsup; ++j) tot += std::max(ssize[j], 0);
    T *v = talloc<T>(*h_.pers, tot * np);
    int64_t o = 0;
    for (int j = 0; j < nsup; ++j) {
      if (ssize[j] < 0) continue;
      nphi[j] = v + o * np;
      for (int c = 2 * j; c <= 2 * j + 1; ++c)
        if (rsize[c] > 0) sb.copy(v + (o + coff[c]) * np, np, rsize[c], np, phi_[key_base + c], np, 0);
      o += ssize[j];
    }
  }
  blocks_.swap(nb);
  phi_.swap(nphi);
  size_.assign(2 * nsup, -1);
  for (int j = 0; j < nsup; ++j) size_[j] = ssize[j];
  // super offsets in the vector segment = offset of the first existing child
  sup_off_.assign(nsup, 0);
  for (int j = 0; j < nsup; ++j) {
    int64_t o = -1;
    for (int c = 2 * j; c <= 2 * j + 1 && o < 0; ++c)
      if (rsize[c] >= 0) o = red_off_[c];
    sup_off_[j] = o;
  }
  nsup_ = nsup;
}

template <typename T>
void Run<T>::wave_a(int li, int widx, WaveBatches<T> &B) {
  const PlanLevel &lv = P_.levels[li];
  lv_ = &lv;
  DevArena &scr = *h_.scratch;
  DevArena &per = *h_.pers;
  const std::vector<int> &wl = lv.waves[widx];
  cur_.assign(wl.size(), Sup());
  c_next_ = 0;
  trunc_sup_.clear();
  big_sup_.clear();
  trunc64_sup_.clear();
  big64_sup_.clear();
  chol_first_ = B.chol.tasks.size();
  trunc_first_ = B.trunc.size();
  big_first_ = B.trunc_big.size();
  trunc64_first_ = B.trunc64.size();
  big64_first_ = B.trunc_big64.size();
  const double f0 = B.chol.flops + B.gram.flops + B.gram64.flops;
  for (size_t q = 0; q < wl.size(); ++q) {
    Sup &x = cur_[q];
    const int s = wl[q];
    const PlanSuper &ps = lv.sup[s];
    x.s = s;
    x.m = size_[s];
    x.red = !ps.W.empty();
    for (int n : ps.N) {
      if (size_[n] < 0) fail(HS_ERR_INVALID, "internal: neighbour does not exist");
      x.Noff.push_back(x.dN);
      x.dN += size_[n];
    }
    for (int w : ps.W) {
      if (size_[w] < 0) fail(HS_ERR_INVALID, "internal: well-separated node does not exist");
      x.Woff.push_back(x.dW);
      x.dW += size_[w];
    }
    const int m = x.m;
    x.AsN = talloc<T>(per, (size_t)m * x.dN);
    x.Linv = talloc<T>(scr, (size_t)m * m);
    auto oriented = [&](int row, int other, T *dst, int ld, int cols) {
      auto it = blocks_.find(bkey(row, other));
      if (it == blocks_.end()) fail(HS_ERR_INVALID, "internal: missing block");
      const BlockRef<T> &b = it->second;
      B.gather.copy(dst, ld, size_[row], cols, b.ptr, b.ld, b.rowkey == row ? 0 : 1);
    };
    for (size_t j = 0; j < ps.N.size(); ++j) oriented(s, ps.N[j], x.AsN + x.Noff[j], x.dN, size_[ps.N[j]]);
    if (x.red) {
      x.AsW = talloc<T>(scr, (size_t)m * x.dW);
      for (size_t j = 0; j < ps.W.size(); ++j) oriented(s, ps.W[j], x.AsW + x.Woff[j], x.dW, size_[ps.W[j]]);
      x.G = rank64() ? nullptr : talloc<T>(scr, (size_t)m * m);
      x.U = talloc<T>(scr, (size_t)m * m);
      if (use_phi_) {
        const int np = h_.nphi;
        x.phiW = talloc<T>(scr, (size_t)x.dW * np);
        x.a = talloc<T>(scr, (size_t)m * np);
        for (size_t j = 0; j < ps.W.size(); ++j)
          if (size_[ps.W[j]] > 0)
            B.gather.copy(x.phiW + (size_t)x.Woff[j] * np, np, size_[ps.W[j]], np, phi_[ps.W[j]], np, 0);
      }
    }
    auto dit = blocks_.find(bkey(s, s));
    if (dit == blocks_.end()) fail(HS_ERR_INVALID, "internal: missing diagonal block");
    B.chol.add(dit->second.ptr, dit->second.ld, x.Linv, m, tag(0, lv.level, s));
    if (x.red && m > 0 && rank64()) {
      // FP64 copies of the FP32 operands; Gram, eigen-solve and rank in FP64
      const int np = use_phi_ ? h_.nphi : 0;
      double *AsW64 = talloc<double>(scr, (size_t)m * x.dW);
      B.widen.push_back(ConvTask{x.AsW, AsW64, (int64_t)m * x.dW, 1});
      TruncTask<double> tt;
      tt.G = talloc<double>(scr, (size_t)m * m);
      tt.a = nullptr;
      tt.phi = nullptr;
      if (use_phi_) {
        double *phiW64 = talloc<double>(scr, (size_t)x.dW * np);
        B.widen.push_back(ConvTask{x.phiW, phiW64, (int64_t)x.dW * np, 1});
        double *phi64 = talloc<double>(scr, (size_t)m * np);
        B.widen.push_back(ConvTask{phi_[s], phi64, (int64_t)m * np, 1});
        double *a64 = talloc<double>(scr, (size_t)m * np);
        B.gram64.add(AsW64, x.dW, 0, phiW64, np, 0, a64, np, m, np, x.dW, 1.0, 0.0);
        tt.a = a64;
        tt.phi = phi64;
      }
      B.gram64.add(AsW64, x.dW, 0, AsW64, x.dW, 1, const_cast<double *>(tt.G), m, m, m, x.dW, 1.0, 0.0);
      tt.np = np;
      tt.eps1 = h_.eps1;
      double *U64 = talloc<double>(scr, (size_t)m * m);
      tt.U = U64;
      tt.work = nullptr;
      tt.eps = level_eps(lv.level);
      tt.m = m;
      tt.k_idx = 0;
      tt.cap = (h_.max_rank_ratio > 0.0 && tt.eps > 0.0)
                   ? std::max(1, (int)std::floor(h_.max_rank_ratio * (double)m))
                   : m;
      if (m <= eig_small_max<double>()) {
        B.trunc64.push_back(tt);
        trunc64_sup_.push_back((int)q);
        B.max_trunc64_m = std::max(B.max_trunc64_m, m);
      } else {
        tt.work = talloc<double>(scr, trunc_big_work_elems<double>(m));
        big64_sup_.push_back((int)q);
        B.max_big64_m = std::max(B.max_big64_m, m);
        B.trunc_big64.push_back(tt);
      }
      B.narrow.push_back(ConvTask{U64, x.U, (int64_t)m * m, 0});
    } else if (x.red && m > 0) {
      B.gram.add(x.AsW, x.dW, 0, x.AsW, x.dW, 1, x.G, m, m, m, x.dW, T(1), T(0));
      if (use_phi_) B.gram.add(x.AsW, x.dW, 0, x.phiW, h_.nphi, 0, x.a, h_.nphi, m, h_.nphi, x.dW, T(1), T(0));
      TruncTask<T> tt;
      tt.G = x.G;
      tt.a = x.a;
      tt.phi = phi_[s];
      tt.np = use_phi_ ? h_.nphi : 0;
      tt.eps1 = h_.eps1;
      tt.U = x.U;
      tt.work = nullptr;
      tt.eps = level_eps(lv.level);
      tt.m = m;
      // the rank cap (hs_opts.max_rank_ratio): floor(ratio m), at least 1
      tt.cap = (h_.max_rank_ratio > 0.0 && tt.eps > 0.0)
                   ? std::max(1, (int)std::floor(h_.max_rank_ratio * (double)m))
                   : m;
      if (m <= eig_small_max<T>()) {
        B.trunc.push_back(tt);
        trunc_sup_.push_back((int)q);
        B.max_trunc_m = std::max(B.max_trunc_m, m);
      } else {
        tt.work = talloc<T>(scr, trunc_big_work_elems<T>(m));
        big_sup_.push_back((int)q);
        B.max_big_m = std::max(B.max_big_m, m);
        B.trunc_big.push_back(tt);
      }
    }
  }
  flops_ += B.chol.flops + B.gram.flops + B.gram64.flops - f0;
  chol_count_ = B.chol.tasks.size() - chol_first_;
}

template <typename T>
void Run<T>::wave_b(const int *hb, size_t nchol, size_t ntrunc, double big_ms, WaveBatches<T> &B) {
  DevArena &scr = *h_.scratch;
  // this run's slices of the statuses and ranks read after phase A
  std::vector<Sup> &S = cur_;
  bool bad = false;
  for (size_t i = chol_first_; i < chol_first_ + chol_count_; ++i)
    if (hb[i] != 0) bad = ex_.mark_failed(B.chol.what[i], hb[i] - 1);
  if (bad) return;   // this problem leaves the lock step
  for (size_t i = 0; i < trunc_sup_.size(); ++i) S[trunc_sup_[i]].k = hb[nchol + trunc_first_ + i];
  for (size_t i = 0; i < big_sup_.size(); ++i) S[big_sup_[i]].k = hb[nchol + ntrunc + big_first_ + i];
  for (size_t i = 0; i < trunc64_sup_.size(); ++i) S[trunc64_sup_[i]].k = hb[nchol + B.k_off64 + trunc64_first_ + i];
  for (size_t i = 0; i < big64_sup_.size(); ++i)
    S[big64_sup_[i]].k = hb[nchol + B.k_off64 + B.trunc64.size() + big64_first_ + i];
  for (size_t i = 0; i < trunc64_sup_.size(); ++i) trunc_sup_.push_back(trunc64_sup_[i]);
  for (size_t i = 0; i < big64_sup_.size(); ++i) big_sup_.push_back(big64_sup_[i]);
  // nominal eigen-solve work of a node: Householder tridiagonalisation
  // (4/3 m^3) and back-transformation of the k kept vectors (2 m^2 k)
  auto eig_work = [](double m, double k) { return 4.0 / 3.0 * m * m * m + 2.0 * m * m * k; };
  for (size_t i = 0; i < trunc_sup_.size(); ++i) eig_flops_ += eig_work(S[trunc_sup_[i]].m, S[trunc_sup_[i]].k);
  if (!big_sup_.empty()) {
    big_ms_ += big_ms;
    ++big_launches_;
    for (int q : big_sup_) {
      const double w = eig_work(S[q].m, S[q].k);
      big_flops_ += w;
      eig_flops_ += w;
    }
  }
  if (!big_sup_.empty()) {
    // U of the large path: re-orthonormalise by CholQR2 (same span)
    std::vector<T *> U1s(S.size(), nullptr), U2s(S.size(), nullptr);
    for (int q : big_sup_) {
      Sup &x = S[q];
      const int m = x.m, k = x.k;
      if (k <= 0) continue;
      T *Sg = talloc<T>(scr, (size_t)k * k), *Lg = talloc<T>(scr, (size_t)k * k);
      T *Sg2 = talloc<T>(scr, (size_t)k * k), *Lg2 = talloc<T>(scr, (size_t)k * k);
      U1s[q] = talloc<T>(scr, (size_t)m * m);
      U2s[q] = talloc<T>(scr, (size_t)m * m);
      B.o1.add(x.U, m, 1, x.U, m, 0, Sg, k, k, k, m, T(1), T(0));
      B.oc1.add(Sg, k, Lg, k, tag(3, lv_->level, x.s));
      B.o2.add(x.U, m, 0, Lg, k, 1, U1s[q], m, m, k, k, T(1), T(0));
      B.o3.add(U1s[q], m, 1, U1s[q], m, 0, Sg2, k, k, k, m, T(1), T(0));
      B.oc2.add(Sg2, k, Lg2, k, tag(3, lv_->level, x.s));
      B.o4.add(U1s[q], m, 0, Lg2, k, 1, U2s[q], m, m, k, k, T(1), T(0));
    }
    for (int q : big_sup_)
      if (U2s[q]) S[q].U = U2s[q];
  }

}

template <typename T>
bool Run<T>::wave_c(WaveBatches<T> &B, size_t count) {
  DevArena &scr = *h_.scratch;
  DevArena &per = *h_.pers;
  // phase B
  std::vector<Sup> &S = cur_;
  const double f0 = B.c1.flops + B.c2.flops + B.g1.flops + B.g2.flops + B.g3.flops + B.g4.flops + B.g5.flops +
                    B.g6.flops + B.g7.flops + B.g8.flops;
  const size_t q0 = c_next_, q1 = std::min(S.size(), c_next_ + count);
  c_next_ = q1;
  for (size_t q = q0; q < q1; ++q) {
    Sup &x = S[q];
    const int m = x.m, k = x.k, dN = x.dN;
    if (k > m || k < 0) fail(HS_ERR_INVALID, "internal: rank out of range");
    if (k > 0) {
      x.Ut = talloc<T>(scr, (size_t)m * k);
      x.S1 = talloc<T>(scr, (size_t)k * k);
      x.L1 = talloc<T>(scr, (size_t)k * k);
      x.Q1 = talloc<T>(scr, (size_t)m * k);
      x.S2 = talloc<T>(scr, (size_t)k * k);
      x.L2 = talloc<T>(scr, (size_t)k * k);
      x.Q = talloc<T>(scr, (size_t)m * k);
      x.Rinv = talloc<T>(scr, (size_t)k * k);
      x.Wt = talloc<T>(scr, (size_t)m * k);
      x.Tm = talloc<T>(scr, (size_t)k * dN);
    }
    x.Gt = talloc<T>(scr, (size_t)m * dN);
    x.Z = talloc<T>(scr, (size_t)dN * dN);
    x.M = talloc<T>(per, (size_t)m * m);
    x.Pm = talloc<T>(per, (size_t)k * m);
    if (x.red) {
      x.ANr = talloc<T>(per, (size_t)dN * k);
      x.Arr = talloc<T>(per, (size_t)k * k);
      x.ArW = talloc<T>(per, (size_t)k * x.dW);
      x.phir = use_phi_ ? talloc<T>(per, (size_t)k * h_.nphi) : nullptr;
    }
    // L^-1 U and its CholQR2
    B.g1.add(x.Linv, m, 0, x.U, m, 0, x.Ut, k, m, k, m, T(1), T(0));
    B.g2.add(x.Ut, k, 1, x.Ut, k, 0, x.S1, k, k, k, m, T(1), T(0));
    B.c1.add(x.S1, k, x.L1, k, tag(1, lv_->level, x.s));
    B.g3.add(x.Ut, k, 0, x.L1, k, 1, x.Q1, k, m, k, k, T(1), T(0));
    B.g4.add(x.Q1, k, 1, x.Q1, k, 0, x.S2, k, k, k, m, T(1), T(0));
    B.c2.add(x.S2, k, x.L2, k, tag(2, lv_->level, x.s));
    B.g5.add(x.Q1, k, 0, x.L2, k, 1, x.Q, k, m, k, k, T(1), T(0));
    B.g5.add(x.L1, k, 1, x.L2, k, 1, x.Rinv, k, k, k, k, T(1), T(0));
    // quantities needing Q / L^-1
    B.g6.add(x.Linv, m, 1, x.Q, k, 0, x.Wt, k, m, k, m, T(1), T(0));          // L^-T Q
    B.g6.add(x.Linv, m, 0, x.AsN, dN, 0, x.Gt, dN, m, dN, m, T(1), T(0));       // L^-1 A_sN
    B.g6.add(x.Linv, m, 1, x.Linv, m, 0, x.M, m, m, m, m, T(1), T(0));          // L^-T L^-1
    if (x.red) {
      B.g6.add(x.U, m, 1, x.AsW, x.dW, 0, x.ArW, x.dW, k, x.dW, m, T(1), T(0));  // U^T A_sW
      if (use_phi_) B.g6.add(x.U, m, 1, phi_[x.s], h_.nphi, 0, x.phir, h_.nphi, k, h_.nphi, m, T(1), T(0));
    }
    B.g7.add(x.Rinv, k, 0, x.Wt, k, 1, x.Pm, m, k, m, k, T(1), T(0));           // P_ss = R^-1 (L^-T Q)^T
    B.g7.add(x.Wt, k, 0, x.Wt, k, 1, x.M, m, m, m, k, T(-1), T(1));             // M_ss -= W W^T
    B.g7.add(x.Q, k, 1, x.Gt, dN, 0, x.Tm, dN, k, dN, m, T(1), T(0));           // Q^T L^-1 A_sN
    B.g7.add(x.Gt, dN, 1, x.Gt, dN, 0, x.Z, dN, dN, dN, m, T(1), T(0));         // (L^-1 A_sN)^T (L^-1 A_sN)
    B.g8.add(x.Tm, dN, 1, x.Tm, dN, 0, x.Z, dN, dN, dN, k, T(-1), T(1));        // - T^T T
    if (x.red) {
      B.g8.add(x.Tm, dN, 1, x.Rinv, k, 1, x.ANr, k, dN, k, k, T(1), T(0));      // A_Nr = T^T R^-T
      B.g8.add(x.Rinv, k, 0, x.Rinv, k, 1, x.Arr, k, k, k, k, T(1), T(0));      // A_rr = R^-1 R^-T
    }
  }
  flops_ += B.c1.flops + B.c2.flops + B.g1.flops + B.g2.flops + B.g3.flops + B.g4.flops + B.g5.flops +
            B.g6.flops + B.g7.flops + B.g8.flops - f0;
  // algorithmic work of the elimination, counted from the actual sizes: Gram
  // 2 m^2 w and R^T 2 m k w of the truncation (Sec. 3.2), Cholesky m^3/3,
  // Y 2 m^2 k, S 2 m k^2 + k^3/3, G_n 2 m^2 d_N, H_n 2 m k d_N, the Schur
  // update 2 (m + k) d_N^2 over all neighbour pairs, and M_ss, P_ss 2 m^2 k
  // (w = sum of the well-separated widths, d_N = sum of the neighbour sizes)
  for (size_t q = q0; q < q1; ++q) {
    const Sup &x = S[q];
    const double m = x.m, k = x.k, dN = x.dN, w = x.red ? x.dW : 0;
    alg_flops_ += 2 * m * m * w + 2 * m * k * w + m * m * m / 3 + 2 * m * m * k + 2 * m * k * k + k * k * k / 3 +
                  2 * m * m * dN + 2 * m * k * dN + 2 * (m + k) * dN * dN + 2 * m * m * k;
  }
  return c_next_ < S.size();
}

// Runs on the host while the GPU executes the wave's GEMMs (wave_c's tasks
// are launched before this is called).
template <typename T>
void Run<T>::wave_d(WaveBatches<T> &B) {
  DevArena &per = *h_.pers;
  std::vector<Sup> &S = cur_;
  // register the red nodes' blocks and gather the Schur update by target:
  // targets in order of first appearance, each target's contributions in
  // ascending super-node order (a stable counting sort of the contributions)
  FlatMap<int> tgt_idx;
  std::vector<uint64_t> tgt_order;
  std::vector<int> c_tgt, c_sup;
  for (size_t q = 0; q < S.size(); ++q) {
    const Sup &x = S[q];
    const PlanSuper &ps = lv_->sup[x.s];
    for (size_t i = 0; i < ps.N.size(); ++i)
      for (size_t j = i; j < ps.N.size(); ++j) {
        const uint64_t key = bkey(ps.N[i], ps.N[j]);
        auto ins = tgt_idx.try_emplace(key);
        if (ins.second) {
          *ins.first = (int)tgt_order.size();
          tgt_order.push_back(key);
        }
        c_tgt.push_back(*ins.first);
        c_sup.push_back((int)q);
      }
  }
  std::vector<int> c_start(tgt_order.size() + 1, 0), c_list(c_tgt.size());
  for (int t : c_tgt) ++c_start[t + 1];
  for (size_t t = 0; t < tgt_order.size(); ++t) c_start[t + 1] += c_start[t];
  {
    std::vector<int> cur(c_start.begin(), c_start.end() - 1);
    for (size_t c = 0; c < c_tgt.size(); ++c) c_list[cur[c_tgt[c]]++] = c_sup[c];
  }
  // new fill blocks (zero) in one allocation
  {
    int64_t total = 0;
    std::vector<std::pair<uint64_t, int64_t>> fresh;
    for (uint64_t key : tgt_order)
      if (!blocks_.count(key)) {
        const int a = (int)(key >> 32), b = (int)(key & 0xffffffffu);
        fresh.emplace_back(key, total);
        total += ((int64_t)size_[a] * size_[b] + 3) & ~(int64_t)3;
      }
    if (!fresh.empty()) {
      T *base = talloc<T>(per, total);
      HS_CUDA(cudaMemsetAsync(base, 0, sizeof(T) * total, st_));
      for (auto &f : fresh) {
        const int a = (int)(f.first >> 32), b = (int)(f.first & 0xffffffffu);
        BlockRef<T> br;
        br.ptr = base + f.second;
        br.ld = size_[b];
        br.rowkey = a;
        blocks_[f.first] = br;
      }
    }
  }
  for (size_t ti = 0; ti < tgt_order.size(); ++ti) {
    const uint64_t key = tgt_order[ti];
    auto dit = blocks_.find(key);
    if (dit == blocks_.end()) fail(HS_ERR_INVALID, "internal: missing Schur target");
    const BlockRef<T> dst = dit->second;
    const int a = (int)(key >> 32), b = (int)(key & 0xffffffffu);
    const int rk = dst.rowkey, ck = (rk == a) ? b : a;
    B.schur.begin(dst.ptr, dst.ld, size_[rk], size_[ck], T(-1), T(1));
    for (int c = c_start[ti]; c < c_start[ti + 1]; ++c) {
      const Sup &x = S[c_list[c]];
      const PlanSuper &ps = lv_->sup[x.s];
      // offsets of the row key and column key inside s's neighbour list
      int orow = -1, ocol = -1;
      for (size_t i = 0; i < ps.N.size(); ++i) {
        if (ps.N[i] == rk) orow = x.Noff[i];
        if (ps.N[i] == ck) ocol = x.Noff[i];
      }
      B.schur.src(x.Z + (int64_t)orow * x.dN + ocol, x.dN, 0);
    }
    B.schur.end();
  }

  // new red nodes, removal of the eliminated super nodes, apply records
  for (auto &x : S) {
    const PlanSuper &ps = lv_->sup[x.s];
    if (x.red) {
      const int r = nsup_ + x.s;
      size_[r] = x.k;
      phi_[r] = x.phir;
      BlockRef<T> rr;
      rr.ptr = x.Arr;
      rr.ld = x.k;
      rr.rowkey = r;
      blocks_[bkey(r, r)] = rr;
      for (size_t i = 0; i < ps.N.size(); ++i) {
        BlockRef<T> b;
        b.ptr = x.ANr + (int64_t)x.Noff[i] * x.k;
        b.ld = x.k;
        b.rowkey = ps.N[i];
        blocks_[bkey(ps.N[i], r)] = b;
      }
      for (size_t i = 0; i < ps.W.size(); ++i) {
        BlockRef<T> b;
        b.ptr = x.ArW + x.Woff[i];
        b.ld = x.dW;
        b.rowkey = r;
        blocks_[bkey(ps.W[i], r)] = b;
      }
    }
    blocks_.erase(bkey(x.s, x.s));
    for (int n : ps.N) blocks_.erase(bkey(x.s, n));
    for (int w : ps.W) blocks_.erase(bkey(x.s, w));
    ApplyNode an{};
    an.M = x.M;
    an.P = x.Pm;
    an.AsN = x.AsN;
    an.m = x.m;
    an.k = x.red ? x.k : 0;
    an.dN = x.dN;
    an.xr = -1;
    Rec rc;
    rc.node = (int)h_.nodes.size();
    rc.s = x.s;
    rc.N = ps.N;
    h_.nodes.push_back(an);
    recs_.push_back(rc);
    h_.ranks.back()[x.s] = x.red ? x.k : -1;
    h_.info.max_rank = std::max(h_.info.max_rank, x.red ? x.k : 0);
    h_.info.max_super = std::max(h_.info.max_super, x.m);
  }
  h_.info.super_nodes += (int)S.size();
  WaveApply wa{};
  wa.node_first = (int)h_.nodes.size() - (int)S.size();
  wa.node_count = (int)S.size();
  h_.waves.push_back(wa);
}

template <typename T>
void Run<T>::end_level(const PlanLevel &lv, int li) {
  (void)li;
  const int nsup = nsup_;
  // red nodes of the parent level: layout of the next segment
  const int64_t next_seg = seg_off_ + seg_size_;
  std::vector<int64_t> roff(nsup, -1);
  int64_t o = 0;
  for (int i = 0; i < nsup; ++i)
    if (lv.red_made[i]) {
      roff[i] = o;
      o += size_[nsup + i];
    }
  auto xoff = [&](int key) -> int64_t {
    if (key < nsup) return seg_off_ + sup_off_[key];
    return next_seg + roff[key - nsup];
  };
  // resolve the apply records of the level, wave by wave
  const int wfirst = (int)h_.waves.size() - (int)lv.waves.size();
  size_t rp = 0;
  for (int w = wfirst; w < (int)h_.waves.size(); ++w) {
    WaveApply &wa = h_.waves[w];
    // contributions (node, column) by target key, in node order; the targets
    // in ascending key order
    FlatMap<int> tix;
    std::vector<int> torder, c_t, c_node, c_col;
    int64_t t = 0;
    wa.max_m = 0;
    wa.rows_f = wa.rows_b = wa.pch = wa.tch = 0;
    for (int q = 0; q < wa.node_count; ++q, ++rp) {
      const Rec &rc = recs_[rp];
      ApplyNode &an = h_.nodes[rc.node];
      an.xs = xoff(rc.s);
      an.xr = lv.red_made[rc.s] ? xoff(nsup + rc.s) : -1;
      an.toff = t;
      t += an.m;
      an.row0 = wa.rows_f;
      wa.rows_f += an.m + an.k;
      an.brow0 = wa.rows_b;
      wa.rows_b += an.m;
      an.pch0 = wa.pch;
      if (an.k > 0) wa.pch += (an.m + 31) / 32;
      wa.max_m = std::max(wa.max_m, an.m);
      an.nb_first = (int)h_.nbrs.size();
      an.nb_count = (int)rc.N.size();
      int col = 0;
      for (int n : rc.N) {
        ApplyNbr nb;
        nb.x = xoff(n);
        nb.size = size_[n];
        nb.col = col;
        col += size_[n];
        h_.nbrs.push_back(nb);
        auto ins = tix.try_emplace((uint64_t)n);
        if (ins.second) {
          *ins.first = (int)torder.size();
          torder.push_back(n);
        }
        c_t.push_back(*ins.first);
        c_node.push_back(rc.node);
        c_col.push_back(nb.col);
      }
    }
    // group the contributions by target (stable counting sort)
    std::vector<int> c_start(torder.size() + 1, 0), c_list(c_t.size());
    for (int x : c_t) ++c_start[x + 1];
    for (size_t x = 0; x < torder.size(); ++x) c_start[x + 1] += c_start[x];
    {
      std::vector<int> cur(c_start.begin(), c_start.end() - 1);
      for (size_t c = 0; c < c_t.size(); ++c) c_list[cur[c_t[c]]++] = (int)c;
    }
    wa.tsize = t;
    h_.tmax = std::max(h_.tmax, t);
    std::vector<int> tsorted(torder.size());
    for (size_t x = 0; x < torder.size(); ++x) tsorted[x] = (int)x;
    std::sort(tsorted.begin(), tsorted.end(), [&](int p, int q) { return torder[p] < torder[q]; });
    wa.tgt_first = (int)h_.targets.size();
    wa.tgt_count = (int)torder.size();
    for (int ti : tsorted) {
      const int n = torder[ti];
      ApplyTarget tg;
      tg.x = xoff(n);
      tg.size = size_[n];
      tg.ch0 = wa.tch;
      wa.tch += (tg.size + 31) / 32;
      tg.first = (int)h_.contribs.size();
      tg.count = c_start[ti + 1] - c_start[ti];
      for (int cc = c_start[ti]; cc < c_start[ti + 1]; ++cc) {
        const int c = c_list[cc];
        const ApplyNode &an = h_.nodes[c_node[c]];
        ApplyContrib ac;
        ac.A = (const char *)an.AsN + sizeof(T) * (size_t)c_col[c];
        ac.ld = an.dN;
        ac.m = an.m;
        ac.toff = an.toff;
        h_.contribs.push_back(ac);
      }
      h_.targets.push_back(tg);
    }
  }
  recs_.clear();
  LevelApply la;
  la.level = lv.level;
  la.wave_first = wfirst;
  la.wave_count = (int)lv.waves.size();
  h_.levels.push_back(la);
  // parent level: red node nsup+i becomes red i
  FlatMap<BlockRef<T>> nb;
  nb.reserve(blocks_.size());
  for (auto &kv : blocks_) {
    const int a = (int)(kv.first >> 32), b = (int)(kv.first & 0xffffffffu);
    if (a < nsup || b < nsup) fail(HS_ERR_INVALID, "internal: super node block left at level end");
    BlockRef<T> br = kv.second;
    br.rowkey -= nsup;
    nb[bkey(a - nsup, b - nsup)] = br;
  }
  blocks_.swap(nb);
  std::vector<int> ns(nsup, -1);
  std::vector<T *> nphi(nsup, nullptr);
  for (int i = 0; i < nsup; ++i)
    if (lv.red_made[i]) {
      ns[i] = size_[nsup + i];
      nphi[i] = phi_[nsup + i];
    }
  size_.swap(ns);
  phi_.swap(nphi);
  red_off_ = roff;
  seg_off_ = next_seg;
  seg_size_ = o;
}

template <typename T>
void Run<T>::begin() {
  h_.nodes.clear();
  h_.nbrs.clear();
  h_.targets.clear();
  h_.contribs.clear();
  h_.waves.clear();
  h_.levels.clear();
  h_.ranks.clear();
  h_.tmax = 0;
  leaf_setup();
  nred_ = P_.nleaf;
}

template <typename T>
void Run<T>::level_begin(int li, SumBatch<T> &sb) {
  const PlanLevel &lv = P_.levels[li];
  merge(nred_, 0, sb);
  for (int j = 0; j < lv.nsup; ++j)
    if ((size_[j] >= 0) != (bool)lv.exists[j]) fail(HS_ERR_INVALID, "internal: plan/executor mismatch");
  h_.ranks.emplace_back(lv.nsup, -1);
}

template <typename T>
void Run<T>::level_end(int li) {
  end_level(P_.levels[li], li);
  nred_ = P_.levels[li].nsup;
}

// the remaining red nodes (level 1, or the single leaf) form the root
template <typename T>
void Run<T>::root_a(SumBatch<T> &sb) {
  const int nred = (int)size_.size();
  bool any = false;
  for (int s : size_) any = any || s > 0;
  h_.root_m = 0;
  root_linv_ = root_ainv_ = nullptr;
  if (!any) {
    h_.ws_size = seg_off_ + seg_size_;
    return;
  }
  merge(nred, 0, sb);
  const int m = size_[0];
  h_.root_m = m;
  h_.root_off = seg_off_ + sup_off_[0];
  h_.ws_size = seg_off_ + seg_size_;
  root_linv_ = talloc<T>(*h_.scratch, (size_t)m * m);
  root_ainv_ = talloc<T>(*h_.pers, (size_t)m * m);
}

template <typename T>
void Run<T>::root_b(CholBatch<T> &cb, GemmBatch<T> &g) {
  if (!root_ainv_) return;
  const int m = h_.root_m;
  auto bit = blocks_.find(bkey(0, 0));
  if (bit == blocks_.end()) fail(HS_ERR_INVALID, "internal: missing root block");
  const BlockRef<T> b = bit->second;
  const double f0 = cb.flops + g.flops;
  cb.add(b.ptr, b.ld, root_linv_, m, tag(4, 0, 0));
  alg_flops_ += (double)m * m * m / 3;
  g.add(root_linv_, m, 1, root_linv_, m, 0, root_ainv_, m, m, m, m, T(1), T(0));
  flops_ += cb.flops + g.flops - f0;
  h_.root_inv = root_ainv_;
  h_.info.root_size = m;
}

template <typename T>
void Run<T>::finish() {
  h_.info.factor_flops = flops_;
  h_.info.eig_flops = eig_flops_;
  h_.info.trunc_big_ms = big_ms_;
  h_.info.trunc_big_flops = big_flops_;
  h_.info.trunc_big_launches = big_launches_;
  h_.info.alg_flops = alg_flops_;
}

// Truncation of very large nodes across the whole GPU: k_trunc_big up to J
// (TB_PREP), the tridiagonal steps (two launches per step over all the nodes'
// CTAs), Z = Q^T [U1, X] (GC), k_trunc_big from T to its eigenvectors
// (TB_POST), then U_2 = Q Y by batches of columns.
template <typename T>
void trunc_grid(Exec &ex, const std::vector<TruncTask<T>> &tasks, const TruncTask<T> *d_tasks, int *d_k,
                double eps, int variant, int max_m) {
  const int n = (int)tasks.size();
  // nested spans (phases 10-14) inside the large-truncation span (5)
  ex.begin(10);
  launch_trunc_big_mode<T>(d_tasks, n, d_k, eps, variant, max_m, 1 /* TB_PREP */, ex.st);
  ex.end();
  std::vector<GridTri<T>> gt(n);
  int blocks = 0;
  for (int q = 0; q < n; ++q) {
    const TruncTask<T> &t = tasks[q];
    const BigLayout<T> L = big_layout<T>(t.work, t.m);
    GridTri<T> &g = gt[q];
    g.A = L.A;
    g.X = L.Y;                 // the step vectors live in Y until TB_POST
    g.P = L.Y + t.m;
    g.V = L.Y + 2 * (size_t)t.m;
    g.px = L.Y + 3 * (size_t)t.m;
    g.ppv = L.Y + 4 * (size_t)t.m;
    g.d = L.d;
    g.e = L.e;
    g.tau = L.tau;
    g.m = t.m;
    g.nblk = (t.m + kTriRows - 1) / kTriRows;
    g.blk0 = blocks;
    blocks += g.nblk;
  }
  // nodes that fit a thread-block cluster's shared memory are tridiagonalised
  // there in one launch per cluster size; the others by the step kernels
  std::vector<GridTri<T>> by_c[4], steps;
  int cmax[4] = {0, 0, 0, 0}, smax = 0;
  for (const GridTri<T> &g : gt) {
    const int c = tri_cluster_enabled() ? tri_cluster_size<T>(g.m) : 0;
    if (c > 0) {
      const int q = c == 1 ? 0 : c == 2 ? 1 : c == 4 ? 2 : 3;
      by_c[q].push_back(g);
      cmax[q] = std::max(cmax[q], g.m);
    } else {
      GridTri<T> h = g;
      h.blk0 = 0;
      steps.push_back(h);
      smax = std::max(smax, g.m);
    }
  }
  int sblocks = 0;
  for (GridTri<T> &g : steps) {
    g.blk0 = sblocks;
    sblocks += g.nblk;
  }
  Uploader u;
  const size_t og = u.add(steps);
  size_t oc[4];
  for (int q = 0; q < 4; ++q) oc[q] = u.add(by_c[q]);
  char *dg = u.upload(ex.scr, ex.sg, ex.st);
  const GridTri<T> *d_gt = (const GridTri<T> *)(dg + og);
  ex.begin(11);
  // the cluster launches run on a side stream, beside the step kernels
  const bool fork = !steps.empty() && (by_c[0].size() + by_c[1].size() + by_c[2].size() + by_c[3].size()) > 0;
  cudaStream_t cs = fork ? ex.side_stream() : ex.st;
  if (fork) {
    HS_CUDA(cudaEventRecord(ex.fork_ev, ex.st));
    HS_CUDA(cudaStreamWaitEvent(cs, ex.fork_ev, 0));
  }
  for (int q = 0; q < 4; ++q)
    launch_tri_cluster<T>((const GridTri<T> *)(dg + oc[q]), (int)by_c[q].size(), 1 << q, cmax[q], cs);
  for (int k = 0; k + 2 <= smax; ++k) {
    launch_tri_step<T>(d_gt, (int)steps.size(), sblocks, k, 0, ex.st);
    if (k + 3 <= smax) launch_tri_step<T>(d_gt, (int)steps.size(), sblocks, k, 1, ex.st);
  }
  if (fork) {
    HS_CUDA(cudaEventRecord(ex.join_ev, cs));
    HS_CUDA(cudaStreamWaitEvent(ex.st, ex.join_ev, 0));
  }
  ex.end();
  (void)blocks;
  const int nb = refl_batch<T>(max_m);
  if (variant != HS_LORASP) {
    // Z = Q^T [U_1, G U_1] has 2 k1 <= 4 np columns, in batches of up to 4
    const int nbz = std::min(nb, 4);
    std::vector<ReflTask<T>> zf;
    for (const TruncTask<T> &t : tasks) {
      const BigLayout<T> L = big_layout<T>(t.work, t.m);
      for (int j0 = 0; j0 < 4 * std::max(t.np, 1); j0 += nbz)
        zf.push_back(ReflTask<T>{L.A, L.tau, L.LS, t.U, L.sc_int, t.m, j0, 1});
    }
    Uploader uz;
    const size_t oz = uz.add(zf);
    char *dz = uz.upload(ex.scr, ex.sg, ex.st);
    ex.begin(12);
    launch_refl<T>((const ReflTask<T> *)(dz + oz), (int)zf.size(), nbz, max_m, ex.st);
    ex.end();
  }
  ex.begin(13);
  launch_trunc_big_mode<T>(d_tasks, n, d_k, eps, variant, max_m, 2 /* TB_POST */, ex.st);
  {
    // eigenvectors of T: clusters spread over many CTAs (at most m per node)
    const int spc = invit_slots<T>(max_m);
    std::vector<InvitTask<T>> it;
    int iblocks = 0;
    for (const TruncTask<T> &t : tasks) {
      const BigLayout<T> L = big_layout<T>(t.work, t.m);
      InvitTask<T> x;
      x.dt = L.dt;
      x.et = L.et;
      x.lam = L.lam;
      x.starts = (const int *)L.pw;
      x.sc = L.sc_int;
      x.tnorm = L.sc_tnorm;
      x.Y = L.Y;
      x.m = t.m;
      x.blk0 = iblocks;
      iblocks += (t.m + spc - 1) / spc;
      it.push_back(x);
    }
    Uploader ui;
    const size_t oi = ui.add(it);
    char *di = ui.upload(ex.scr, ex.sg, ex.st);
    launch_invit<T>((const InvitTask<T> *)(di + oi), (int)it.size(), iblocks, spc, max_m, ex.st);
  }
  ex.end();
  std::vector<ReflTask<T>> yb;
  for (const TruncTask<T> &t : tasks) {
    const BigLayout<T> L = big_layout<T>(t.work, t.m);
    for (int j0 = 0; j0 < t.m; j0 += nb) yb.push_back(ReflTask<T>{L.A, L.tau, L.Y, t.U, L.sc_int, t.m, j0, 0});
  }
  Uploader uy;
  const size_t oy = uy.add(yb);
  char *dy = uy.upload(ex.scr, ex.sg, ex.st);
  ex.begin(14);
  launch_refl<T>((const ReflTask<T> *)(dy + oy), (int)yb.size(), nb, max_m, ex.st);
  ex.end();
}

// Host time per part of the factorization loop, printed to stderr after each
// factorization when HS_HOST_PROFILE=1 (environment): the time since the
// previous tick goes to the named part.
struct HostClock {
  static constexpr int kParts = 12;
  bool on = false;
  double ms[kParts] = {};
  std::chrono::steady_clock::time_point t;
  HostClock() {
    const char *e = std::getenv("HS_HOST_PROFILE");
    on = e && e[0] == '1';
    t = std::chrono::steady_clock::now();
  }
  void tick(int part) {
    if (!on) return;
    const auto n = std::chrono::steady_clock::now();
    ms[part] += std::chrono::duration<double, std::milli>(n - t).count();
    t = n;
  }
  void report() const {
    if (!on) return;
    static const char *names[kParts] = {"level_begin", "wave_a",  "launch_a", "sync_wait", "wave_b",    "launch_qr",
                                        "wave_c",      "launch_c", "wave_d",   "launch_schur", "level_end", "root"};
    std::fprintf(stderr, "hs host ms:");
    for (int i = 0; i < kParts; ++i) std::fprintf(stderr, " %s=%.2f", names[i], ms[i]);
    std::fprintf(stderr, "\n");
  }
};

// Runs the factorizations of `runs` in lock step: at every step (level counted
// from the leaves, wave index) the work of all problems that have that step
// goes into one launch per kernel kind, with one read of the new ranks.
// The large-node truncation tasks of a wave split by class (256 or 1024
// threads per node, or the multi-CTA path), uploaded, then launched.
template <typename U>
struct BigClasses {
  std::vector<TruncTask<U>> cls[3];
  int cmax[3] = {0, 0, 0};
  size_t o[3] = {0, 0, 0};
  char *d = nullptr;
  void prepare(Exec &ex, const std::vector<TruncTask<U>> &tasks) {
    for (const TruncTask<U> &t : tasks) {
      const int c = (t.eps > 0.0 && t.m >= grid_tridiag_min()) ? 2 : t.m <= kTruncBigMidMax ? 0 : 1;
      cls[c].push_back(t);
      cmax[c] = std::max(cmax[c], t.m);
    }
    Uploader u;
    o[0] = u.add(cls[0]);
    o[1] = u.add(cls[1]);
    o[2] = u.add(cls[2]);
    d = u.upload(ex.scr, ex.sg, ex.st);
  }
  void launch(Exec &ex, int *d_k, double eps, int variant) {
    launch_trunc_big<U>((const TruncTask<U> *)(d + o[0]), (int)cls[0].size(), d_k, eps, variant, cmax[0], ex.st);
    launch_trunc_big<U>((const TruncTask<U> *)(d + o[1]), (int)cls[1].size(), d_k, eps, variant, cmax[1], ex.st);
    if (!cls[2].empty()) trunc_grid<U>(ex, cls[2], (const TruncTask<U> *)(d + o[2]), d_k, eps, variant, cmax[2]);
  }
};

template <typename T>
void execute(Exec &ex, std::vector<std::unique_ptr<Run<T>>> &runs) {
  const auto t_start = std::chrono::steady_clock::now();
  HostClock hc;
  for (auto &r : runs) {
    r->handle().scratch->reset();
    r->begin();
  }
  int maxL = 0;
  for (auto &r : runs) maxL = std::max(maxL, r->levels());
  for (int li = 0; li < maxL; ++li) {
    std::vector<Run<T> *> part;
    for (auto &r : runs)
      if (li < r->levels() && r->ok()) part.push_back(r.get());
    {
      // the merge's descriptors go into the staging buffer in use: flipping
      // to the other one here would make the next wave step flip back to a
      // buffer whose copies may still be pending (no synchronisation between)
      ex.scr.reset();
      SumBatch<T> sb;
      for (Run<T> *r : part) {
        r->handle().scratch->reset();
        r->level_begin(li, sb);
      }
      ex.begin(0);
      sb.launch(ex.scr, ex.sg, ex.st);
      ex.end();
      hc.tick(0);
    }
    int nw = 0;
    for (Run<T> *r : part) nw = std::max(nw, r->waves(li));
    for (int w = 0; w < nw; ++w) {
      std::vector<Run<T> *> wp;
      for (Run<T> *r : part)
        if (w < r->waves(li) && r->ok()) wp.push_back(r);
      if (wp.empty()) continue;
      // one flip of the staging buffers per wave step: the other buffer's
      // copies were enqueued before the previous step's synchronisation
      ex.scr.reset();
      ex.sg.next_wave();
      for (Run<T> *r : wp) r->handle().scratch->reset();
      WaveBatches<T> B;
      // phase A
      for (Run<T> *r : wp) r->wave_a(li, w, B);
      hc.tick(1);
      const size_t nchol = B.chol.tasks.size(), ntrunc = B.trunc.size(), nbig = B.trunc_big.size();
      const size_t nt64 = B.trunc64.size(), nb64 = B.trunc_big64.size();
      for (size_t i = 0; i < ntrunc; ++i) B.trunc[i].k_idx = (int)i;
      for (size_t i = 0; i < nbig; ++i) B.trunc_big[i].k_idx = (int)(ntrunc + i);
      B.k_off64 = ntrunc + nbig;
      for (size_t i = 0; i < nt64; ++i) B.trunc64[i].k_idx = (int)(B.k_off64 + i);
      for (size_t i = 0; i < nb64; ++i) B.trunc_big64[i].k_idx = (int)(B.k_off64 + nt64 + i);
      ex.begin(1);
      B.gather.launch(ex.scr, ex.sg, ex.st);
      ex.end();
      int *d_stat = (int *)ex.scr.alloc(sizeof(int) * (nchol + ntrunc + nbig + nt64 + nb64 + 1));
      int *d_k = d_stat + nchol;
      if (nchol) {
        ex.begin(2);
        ex.chol_inv_any<T>(B.chol.tasks, d_stat);
        ex.end();
      }
      ex.begin(3);
      ex.gemm(B.gram, false);   // the Gram feeds the rank decision
      if (!B.widen.empty()) {
        // FP64 truncation of an FP32 factor: FP64 copies, then their Gram
        Uploader u;
        const size_t o = u.add(B.widen);
        char *d = u.upload(ex.scr, ex.sg, ex.st);
        launch_convert_list((const ConvTask *)(d + o), (int)B.widen.size(), ex.st);
        ex.gemm(B.gram64, false);
      }
      ex.end();
      const double eps = wp[0]->handle().eps;
      const int variant = wp[0]->handle().variant;
      if (ntrunc) {
        Uploader u;
        const size_t o = u.add(B.trunc);
        char *d = u.upload(ex.scr, ex.sg, ex.st);
        ex.begin(4);
        launch_trunc<T>((const TruncTask<T> *)(d + o), (int)ntrunc, d_k, eps, variant, B.max_trunc_m, ex.st);
        ex.end();
      }
      if (nt64) {
        Uploader u;
        const size_t o = u.add(B.trunc64);
        char *d = u.upload(ex.scr, ex.sg, ex.st);
        ex.begin(4);
        launch_trunc<double>((const TruncTask<double> *)(d + o), (int)nt64, d_k, eps, variant, B.max_trunc64_m,
                             ex.st);
        ex.end();
      }
      if (nbig || nb64) {
        // one launch per class (k_idx keeps each rank's slot): 256 or 1024
        // threads per node, or the multi-CTA path for very large nodes
        BigClasses<T> bc;
        BigClasses<double> bc64;
        if (nbig) bc.prepare(ex, B.trunc_big);
        if (nb64) bc64.prepare(ex, B.trunc_big64);
        ex.begin(5);
        HS_CUDA(cudaEventRecord(ex.ev_big[0], ex.st));
        if (nbig) bc.launch(ex, d_k, eps, variant);
        if (nb64) bc64.launch(ex, d_k, eps, variant);
        HS_CUDA(cudaEventRecord(ex.ev_big[1], ex.st));
        ex.end();
      }
      if (!B.narrow.empty()) {
        // the FP64 bases back to the factor precision
        Uploader u;
        const size_t o = u.add(B.narrow);
        char *d = u.upload(ex.scr, ex.sg, ex.st);
        launch_convert_list((const ConvTask *)(d + o), (int)B.narrow.size(), ex.st);
      }
      // one read of the statuses and ranks
      const size_t nread = nchol + ntrunc + nbig + nt64 + nb64;
      int *hb = ex.host_ints(nread + 1);
      if (nread) HS_CUDA(cudaMemcpyAsync(hb, d_stat, sizeof(int) * nread, cudaMemcpyDeviceToHost, ex.st));
      hc.tick(2);
      ex.sync_check();
      hc.tick(3);
      float big_ms = 0.f;
      if (nbig || nb64) HS_CUDA(cudaEventElapsedTime(&big_ms, ex.ev_big[0], ex.ev_big[1]));
      for (Run<T> *r : wp)
        if (r->ok()) r->wave_b(hb, nchol, ntrunc, big_ms, B);
      hc.tick(4);
      // U of the large path: CholQR2
      ex.begin(6);
      ex.gemm(B.o1);
      ex.chol_checked(B.oc1);
      ex.gemm(B.o2);
      ex.gemm(B.o3);
      ex.chol_checked(B.oc2);
      ex.gemm(B.o4);
      ex.end();
      hc.tick(5);
      // phase B and the Schur update.  The GEMM tasks are built and launched
      // in chunks of super nodes, so that the GPU starts on the first chunk
      // while the host builds the next (large waves at the lower levels hold
      // thousands of nodes); the host then builds the Schur targets and the
      // new blocks (wave_d) while the GPU runs the last chunk.  Tasks of
      // different nodes are independent, and a task's arithmetic does not
      // depend on its chunk.  The first chunk is small: the GPU is idle from
      // the rank read until its launches arrive.
      size_t chunk = 64;
      bool more = true;
      while (more) {
        more = false;
        for (Run<T> *r : wp)
          if (r->ok() && r->wave_c(B, chunk)) more = true;
        chunk = 512;
        hc.tick(6);
        ex.begin(7);
        ex.gemm(B.g1);
        ex.gemm(B.g2);
        ex.chol_checked(B.c1);
        ex.gemm(B.g3);
        ex.gemm(B.g4);
        ex.chol_checked(B.c2);
        ex.gemm(B.g5);
        ex.gemm(B.g6);
        ex.gemm(B.g7);
        ex.gemm(B.g8);
        ex.end();
        B.c1.tasks.clear();
        B.c1.what.clear();
        B.c2.tasks.clear();
        B.c2.what.clear();
        hc.tick(7);
      }
      for (Run<T> *r : wp)
        if (r->ok()) r->wave_d(B);
      hc.tick(8);
      ex.begin(8);
      B.schur.launch(ex.scr, ex.sg, ex.st);
      ex.end();
      hc.tick(9);
    }
    for (Run<T> *r : part)
      if (r->ok()) r->level_end(li);
    hc.tick(10);
  }
  // the roots (one flip: the last wave step synchronised after the other
  // buffer's copies)
  ex.scr.reset();
  ex.sg.next_wave();
  {
    SumBatch<T> sb;
    for (auto &r : runs)
      if (r->ok()) {
        r->handle().scratch->reset();
        r->root_a(sb);
      }
    ex.begin(9);
    sb.launch(ex.scr, ex.sg, ex.st);
    CholBatch<T> cb;
    GemmBatch<T> g;
    for (auto &r : runs)
      if (r->ok()) r->root_b(cb, g);
    ex.chol_checked(cb);
    ex.gemm(g);
    ex.end();
  }
  ex.sync_check();
  hc.tick(11);
  hc.report();
  const double total =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  for (auto &r : runs)
    if (r->ok()) {
      r->finish();
      r->handle().info.host_ms = total;
      r->handle().info.wait_ms = ex.wait_ms;
      r->handle().info.tc_flops = ex.tc_flops;
      r->handle().info.tc_ms = ex.tc_ms;
      r->handle().info.tc_launches = ex.tc_launches;
      ex.phase_times(r->handle().info.phase_ms, 16);
    }
}

}  // namespace

namespace {

template <typename T>
void factorize_t(const std::vector<FactorHandle *> &hs, const std::vector<const double *> &phis,
                 cudaStream_t st, std::vector<int> *status, std::vector<std::string> *msg) {
  Exec ex(st);
  ex.use_alloc(hs[0]->alloc);
  ex.prof = phase_profiling();
  const int prec = hs[0]->prec;
  ex.tc = tc_kind_of(prec);
  gemm_tune(ex.tc);   // the GEMM autotuner's table, built once per device and precision
  ex.wait_cycles = hs[0]->timeout_cycles;
  if (hs.size() > 1) {
    ex.prob_status.assign(hs.size(), HS_OK);
    ex.prob_msg.assign(hs.size(), std::string());
  }
  std::vector<std::unique_ptr<Run<T>>> runs;
  for (size_t p = 0; p < hs.size(); ++p) {
    FactorHandle &h = *hs[p];
    if (!h.pers) h.pers.reset(new DevArena(256ull << 20, h.alloc));
    if (!h.scratch) h.scratch.reset(new DevArena(64ull << 20, h.alloc));
    h.pers->set_alloc(h.alloc, st);
    h.scratch->set_alloc(h.alloc, st);
    h.pers->reset();     // a refactorization reuses the previous factor's memory
    h.scratch->reset();
    h.info = hs_info{};
    runs.emplace_back(new Run<T>(h, phis[p], ex, hs.size() > 1 ? (int)p : -1));
  }
  execute<T>(ex, runs);
  if (status) *status = ex.prob_status.empty() ? std::vector<int>(hs.size(), HS_OK) : ex.prob_status;
  if (msg) *msg = ex.prob_msg.empty() ? std::vector<std::string>(hs.size()) : ex.prob_msg;
}

}  // namespace

void set_phase_profiling(bool on) { g_phase_prof.store(on ? 1 : 0); }

void factorize(FactorHandle &h, const hs_csr &A, const hs_opts &o, const double *phi_host) {
  (void)A;
  (void)o;
  factorize_batch({&h}, {phi_host}, h.stream, nullptr, nullptr);
}

void factorize_batch(const std::vector<FactorHandle *> &hs, const std::vector<const double *> &phis,
                     cudaStream_t st, std::vector<int> *status, std::vector<std::string> *msg) {
  if (hs.empty()) return;
  const int prec = hs[0]->prec;
  for (FactorHandle *h : hs)
    if (h->prec != prec || h->eps != hs[0]->eps || h->variant != hs[0]->variant)
      fail(HS_ERR_INVALID, "a batched factorization needs one precision, tolerance and variant");
  if (prec == HS_PREC_F64)
    factorize_t<double>(hs, phis, st, status, msg);
  else
    factorize_t<float>(hs, phis, st, status, msg);
}

}  // namespace hs
