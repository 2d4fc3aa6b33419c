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
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>

#include "handle.h"

namespace hs {

// ---------------------------------------------------------------------------
// DevArena
// ---------------------------------------------------------------------------
DevArena::~DevArena() {
  for (auto &c : chunks_) cudaFree(c.first);
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
    char *p = nullptr;
    HS_CUDA(cudaMalloc(&p, sz));
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
// synchronisation, so a buffer is rewritten only two waves later.
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

template <typename T>
struct GemmBatch {
  std::vector<GemmTask<T>> tasks;
  std::vector<int> tile_start;
  int tiles = 0;
  double flops = 0.0;
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
    tile_start.push_back(tiles);
    tiles += ((M + GEMM_TM - 1) / GEMM_TM) * ((N + GEMM_TN - 1) / GEMM_TN);
    flops += 2.0 * M * N * (double)std::max(K, 0);
  }
  void launch(DevArena &scr, Staging &sg, cudaStream_t st) {
    if (tasks.empty()) return;
    Uploader u;
    const size_t ot = u.add(tasks);
    const size_t os = u.add(tile_start);
    char *d = u.upload(scr, sg, st);
    launch_gemm<T>((const GemmTask<T> *)(d + ot), (const int *)(d + os), (int)tasks.size(), tiles, st);
    tasks.clear();
    tile_start.clear();
    tiles = 0;
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
};

inline std::string describe(const Tag &t) {
  static const char *names[] = {"A_ss", "S (first CholQR pass)", "S (second CholQR pass)", "U^T U", "root block"};
  if (t.kind == 4) return "root block";
  return "level " + std::to_string(t.level) + " super node " + std::to_string(t.s) + ": " + names[t.kind];
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
// (default 64: above that the tridiagonal path needs far fewer operations than
// the ~10 Jacobi sweeps); larger ones use the tridiagonal path.
// HS_EIG_SMALL_MAX (environment) lowers the limit, which lets small test
// problems exercise the tridiagonal path.
template <typename T>
int eig_small_max() {
  static const int v = [] {
    const char *e = std::getenv("HS_EIG_SMALL_MAX");
    const int cap = std::min(64, jacobi_cap<T>());
    if (!e) return cap;
    const int x = std::atoi(e);
    return x < 0 ? cap : std::min(x, cap);
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

template <typename T>
class Run {
 public:
  Run(FactorHandle &h, const double *phi_host) : h_(h), P_(h.plan), st_(h.stream) {
    use_phi_ = h.variant != HS_LORASP;
    phi_host_ = phi_host;
    HS_CUDA(cudaMallocHost(&hbuf_, hbuf_cap_ * sizeof(int)));
  }
  ~Run() {
    // copies from the pinned staging buffers may still be in flight after an error
    cudaStreamSynchronize(st_);
    cudaFreeHost(hbuf_);
  }

  void run();

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
  void merge(int nred, int key_base);
  void wave(const PlanLevel &lv, int li, int widx);
  void end_level(const PlanLevel &lv, int li);
  void root();
  void sync_check();
  int *host_ints(size_t n);

  FactorHandle &h_;
  const Plan &P_;
  cudaStream_t st_;
  bool use_phi_ = false;
  const double *phi_host_ = nullptr;

  std::unordered_map<uint64_t, BlockRef<T>> blocks_;
  std::vector<int> size_;      // by key of the current level
  std::vector<T *> phi_;       // by key
  int nsup_ = 0;
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
  std::vector<PendingStatus> pending_;
  Staging sg_;
  int *hbuf_ = nullptr;
  size_t hbuf_cap_ = 1 << 16;
  double flops_ = 0.0;
  int lv_level_hint_ = 0;
};

template <typename T>
int *Run<T>::host_ints(size_t n) {
  if (n > hbuf_cap_) {
    cudaFreeHost(hbuf_);
    hbuf_cap_ = std::max(n, 2 * hbuf_cap_);
    HS_CUDA(cudaMallocHost(&hbuf_, hbuf_cap_ * sizeof(int)));
  }
  return hbuf_;
}

template <typename T>
void Run<T>::sync_check() {
  HS_CUDA(cudaStreamSynchronize(st_));
  for (auto &ps : pending_) {
    std::vector<int> hv(ps.what.size());
    int *hb = hv.data();
    HS_CUDA(cudaMemcpy(hb, ps.d, ps.what.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < ps.what.size(); ++i)
      if (hb[i] != 0)
        fail(HS_ERR_NOT_SPD, describe(ps.what[i]) + " is not positive definite (pivot " +
                                 std::to_string(hb[i] - 1) + ")");
  }
  pending_.clear();
}

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
    std::unordered_map<uint64_t, int64_t> off;
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
    HS_CUDA(cudaMalloc(&h_.d_leaf_dest, sizeof(int64_t) * std::max<int64_t>(P_.nnz, 1)));
    HS_CUDA(cudaMemcpyAsync(h_.d_leaf_dest, dest.data(), sizeof(int64_t) * P_.nnz, cudaMemcpyHostToDevice, st_));
    h_.leaf_total = total;
    if (use_phi_) {
      // preserved vector of the leaves (GC): ones, or the caller's phi permuted
      std::vector<T> ph(P_.n);
      for (int64_t p = 0; p < P_.n; ++p)
        ph[p] = (h_.variant == HS_GC_USER) ? (T)phi_host_[P_.perm[p]] : T(1);
      HS_CUDA(cudaMalloc(&h_.d_phi0, sizeof(T) * P_.n));
      HS_CUDA(cudaMemcpyAsync(h_.d_phi0, ph.data(), sizeof(T) * P_.n, cudaMemcpyHostToDevice, st_));
    }
  }
  const int64_t total = h_.leaf_total;
  T *base = talloc<T>(*h_.pers, total);
  HS_CUDA(cudaMemsetAsync(base, 0, sizeof(T) * std::max<int64_t>(total, 1), st_));
  launch_scatter_values<T>(h_.d_val, h_.d_leaf_dest, P_.nnz, base, st_);
  blocks_.clear();
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
    for (int i = 0; i < nleaf; ++i) phi_[i] = (T *)h_.d_phi0 + lp[i];
  // vector layout: level L segment = the permuted unknowns
  seg_off_ = 0;
  red_off_.assign(nleaf, 0);
  for (int i = 0; i < nleaf; ++i) red_off_[i] = lp[i];
  seg_size_ = P_.n;
}

// Merge the red nodes (keys key_base + i, i < nred) pairwise into super nodes
// (Sec. 3: I^s_i = I^r_{2i-1} u I^r_{2i}); blocks are assembled 2 x 2.
template <typename T>
void Run<T>::merge(int nred, int key_base) {
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
  std::unordered_map<uint64_t, int64_t> off;
  std::vector<std::pair<int, int>> order;
  int64_t total = 0;
  for (auto &kv : blocks_) {
    const int a = (int)(kv.first >> 32) - key_base, b = (int)(kv.first & 0xffffffffu) - key_base;
    if (a < 0 || b < 0 || a >= nred || b >= nred) fail(HS_ERR_INVALID, "internal: stray block at merge");
    const int I = a / 2, J = b / 2;
    const uint64_t key = bkey(I, J);
    if (!off.count(key)) {
      off[key] = total;
      order.emplace_back(std::min(I, J), std::max(I, J));
      total += ((int64_t)ssize[I] * ssize[J] + 3) & ~(int64_t)3;
    }
  }
  T *base = talloc<T>(*h_.pers, total);
  HS_CUDA(cudaMemsetAsync(base, 0, sizeof(T) * std::max<int64_t>(total, 1), st_));
  std::unordered_map<uint64_t, BlockRef<T>> nb;
  for (auto &IJ : order) {
    BlockRef<T> br;
    br.ptr = base + off[bkey(IJ.first, IJ.second)];
    br.ld = ssize[IJ.second];
    br.rowkey = IJ.first;
    nb[bkey(IJ.first, IJ.second)] = br;
  }
  SumBatch<T> sb;
  for (auto &kv : blocks_) {
    const int a = std::min((int)(kv.first >> 32), (int)(kv.first & 0xffffffffu)) - key_base;
    const int b = std::max((int)(kv.first >> 32), (int)(kv.first & 0xffffffffu)) - key_base;
    const BlockRef<T> &rb = kv.second;
    const int I = a / 2, J = b / 2;
    const BlockRef<T> &sbk = nb[bkey(I, J)];
    // rows a, cols b
    const int ta = (rb.rowkey - key_base == a) ? 0 : 1;
    sb.copy(sbk.ptr + (int64_t)coff[a] * sbk.ld + coff[b], sbk.ld, rsize[a], rsize[b], rb.ptr, rb.ld, ta);
    if (I == J && a != b)  // mirrored sub-block of a diagonal super block
      sb.copy(sbk.ptr + (int64_t)coff[b] * sbk.ld + coff[a], sbk.ld, rsize[b], rsize[a], rb.ptr, rb.ld,
              1 - ta);
  }
  // preserved vectors: contiguous per level
  std::vector<T *> nphi(2 * nsup, nullptr);
  if (use_phi_) {
    int64_t tot = 0;
    for (int j = 0; j < nsup; ++j) tot += std::max(ssize[j], 0);
    T *v = talloc<T>(*h_.pers, tot);
    int64_t o = 0;
    for (int j = 0; j < nsup; ++j) {
      if (ssize[j] < 0) continue;
      nphi[j] = v + o;
      for (int c = 2 * j; c <= 2 * j + 1; ++c)
        if (rsize[c] > 0) sb.copy(v + o + coff[c], 1, rsize[c], 1, phi_[key_base + c], 1, 0);
      o += ssize[j];
    }
  }
  sb.launch(*h_.scratch, sg_, st_);
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
void Run<T>::wave(const PlanLevel &lv, int li, int widx) {
  (void)li;
  DevArena &scr = *h_.scratch;
  DevArena &per = *h_.pers;
  const std::vector<int> &wl = lv.waves[widx];
  std::vector<Sup> S(wl.size());
  SumBatch<T> gather;
  GemmBatch<T> gram;
  CholBatch<T> chol;
  std::vector<TruncTask<T>> trunc, trunc_big;
  int max_trunc_m = 0, max_big_m = 0;
  std::vector<int> trunc_sup, big_sup;
  for (size_t q = 0; q < wl.size(); ++q) {
    Sup &x = S[q];
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
      gather.copy(dst, ld, size_[row], cols, b.ptr, b.ld, b.rowkey == row ? 0 : 1);
    };
    for (size_t j = 0; j < ps.N.size(); ++j) oriented(s, ps.N[j], x.AsN + x.Noff[j], x.dN, size_[ps.N[j]]);
    if (x.red) {
      x.AsW = talloc<T>(scr, (size_t)m * x.dW);
      for (size_t j = 0; j < ps.W.size(); ++j) oriented(s, ps.W[j], x.AsW + x.Woff[j], x.dW, size_[ps.W[j]]);
      x.G = talloc<T>(scr, (size_t)m * m);
      x.U = talloc<T>(scr, (size_t)m * m);
      if (use_phi_) {
        x.phiW = talloc<T>(scr, x.dW);
        x.a = talloc<T>(scr, m);
        for (size_t j = 0; j < ps.W.size(); ++j)
          if (size_[ps.W[j]] > 0) gather.copy(x.phiW + x.Woff[j], 1, size_[ps.W[j]], 1, phi_[ps.W[j]], 1, 0);
      }
    }
    auto dit = blocks_.find(bkey(s, s));
    if (dit == blocks_.end()) fail(HS_ERR_INVALID, "internal: missing diagonal block");
    chol.add(dit->second.ptr, dit->second.ld, x.Linv, m, Tag{0, lv.level, s});
    if (x.red && m > 0) {
      gram.add(x.AsW, x.dW, 0, x.AsW, x.dW, 1, x.G, m, m, m, x.dW, T(1), T(0));
      if (use_phi_) gram.add(x.AsW, x.dW, 0, x.phiW, 1, 0, x.a, 1, m, 1, x.dW, T(1), T(0));
      TruncTask<T> tt;
      tt.G = x.G;
      tt.a = x.a;
      tt.phi = phi_[s];
      tt.U = x.U;
      tt.work = nullptr;
      tt.m = m;
      if (m <= eig_small_max<T>()) {
        tt.k_idx = (int)trunc.size();
        trunc.push_back(tt);
        trunc_sup.push_back((int)q);
        max_trunc_m = std::max(max_trunc_m, m);
      } else {
        tt.work = talloc<T>(scr, trunc_big_work_elems<T>(m));
        big_sup.push_back((int)q);
        max_big_m = std::max(max_big_m, m);
        trunc_big.push_back(tt);
      }
    }
  }
  for (size_t i = 0; i < trunc_big.size(); ++i) trunc_big[i].k_idx = (int)(trunc.size() + i);
  gather.launch(scr, sg_, st_);
  // phase A kernels
  int *d_stat = (int *)scr.alloc(sizeof(int) * (chol.tasks.size() + trunc.size() + trunc_big.size() + 1));
  int *d_k = d_stat + chol.tasks.size();
  if (!chol.tasks.empty()) {
    Uploader u;
    const size_t o = u.add(chol.tasks);
    char *d = u.upload(scr, sg_, st_);
    launch_chol_inv<T>((const CholTask<T> *)(d + o), (int)chol.tasks.size(), d_stat, chol.max_m, st_);
  }
  flops_ += chol.flops + gram.flops;
  gram.launch(scr, sg_, st_);
  if (!trunc.empty()) {
    Uploader u;
    const size_t o = u.add(trunc);
    char *d = u.upload(scr, sg_, st_);
    launch_trunc<T>((const TruncTask<T> *)(d + o), (int)trunc.size(), d_k, h_.eps, h_.variant,
                    max_trunc_m, st_);
  }
  if (!trunc_big.empty()) {
    Uploader u;
    const size_t o = u.add(trunc_big);
    char *d = u.upload(scr, sg_, st_);
    launch_trunc_big<T>((const TruncTask<T> *)(d + o), (int)trunc_big.size(), d_k, h_.eps, h_.variant,
                        max_big_m, st_);
  }
  // one read of the statuses and ranks
  const size_t nread = chol.tasks.size() + trunc.size() + trunc_big.size();
  int *hb = host_ints(nread + 1);
  if (nread) HS_CUDA(cudaMemcpyAsync(hb, d_stat, sizeof(int) * nread, cudaMemcpyDeviceToHost, st_));
  sync_check();
  for (size_t i = 0; i < chol.tasks.size(); ++i)
    if (hb[i] != 0)
      fail(HS_ERR_NOT_SPD, describe(chol.what[i]) + " is not positive definite (pivot " + std::to_string(hb[i] - 1) + ")");
  for (size_t i = 0; i < trunc.size(); ++i) S[trunc_sup[i]].k = hb[chol.tasks.size() + i];
  for (size_t i = 0; i < trunc_big.size(); ++i) S[big_sup[i]].k = hb[chol.tasks.size() + trunc.size() + i];
  if (!big_sup.empty()) {
    // U of the large path: re-orthonormalise by CholQR2 (same span)
    GemmBatch<T> o1, o2, o3, o4;
    CholBatch<T> oc1, oc2;
    std::vector<T *> U1s(S.size(), nullptr), U2s(S.size(), nullptr);
    for (int q : big_sup) {
      Sup &x = S[q];
      const int m = x.m, k = x.k;
      if (k <= 0) continue;
      T *Sg = talloc<T>(scr, (size_t)k * k), *Lg = talloc<T>(scr, (size_t)k * k);
      T *Sg2 = talloc<T>(scr, (size_t)k * k), *Lg2 = talloc<T>(scr, (size_t)k * k);
      U1s[q] = talloc<T>(scr, (size_t)m * m);
      U2s[q] = talloc<T>(scr, (size_t)m * m);
      o1.add(x.U, m, 1, x.U, m, 0, Sg, k, k, k, m, T(1), T(0));
      oc1.add(Sg, k, Lg, k, Tag{3, lv.level, x.s});
      o2.add(x.U, m, 0, Lg, k, 1, U1s[q], m, m, k, k, T(1), T(0));
      o3.add(U1s[q], m, 1, U1s[q], m, 0, Sg2, k, k, k, m, T(1), T(0));
      oc2.add(Sg2, k, Lg2, k, Tag{3, lv.level, x.s});
      o4.add(U1s[q], m, 0, Lg2, k, 1, U2s[q], m, m, k, k, T(1), T(0));
    }
    auto chol_now = [&](CholBatch<T> &cb) {
      if (cb.tasks.empty()) return;
      PendingStatus ps;
      ps.d = (int *)per.alloc(sizeof(int) * cb.tasks.size());
      ps.what = cb.what;
      Uploader u;
      const size_t o = u.add(cb.tasks);
      char *d = u.upload(scr, sg_, st_);
      launch_chol_inv<T>((const CholTask<T> *)(d + o), (int)cb.tasks.size(), ps.d, cb.max_m, st_);
      pending_.push_back(ps);
    };
    o1.launch(scr, sg_, st_);
    chol_now(oc1);
    o2.launch(scr, sg_, st_);
    o3.launch(scr, sg_, st_);
    chol_now(oc2);
    o4.launch(scr, sg_, st_);
    for (int q : big_sup)
      if (U2s[q]) S[q].U = U2s[q];
  }

  // phase B
  GemmBatch<T> g1, g2, g3, g4, g5, g6, g7, g8;
  CholBatch<T> c1, c2;
  for (auto &x : S) {
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
      x.phir = use_phi_ ? talloc<T>(per, k) : nullptr;
    }
    // L^-1 U and its CholQR2
    g1.add(x.Linv, m, 0, x.U, m, 0, x.Ut, k, m, k, m, T(1), T(0));
    g2.add(x.Ut, k, 1, x.Ut, k, 0, x.S1, k, k, k, m, T(1), T(0));
    c1.add(x.S1, k, x.L1, k, Tag{1, lv.level, x.s});
    g3.add(x.Ut, k, 0, x.L1, k, 1, x.Q1, k, m, k, k, T(1), T(0));
    g4.add(x.Q1, k, 1, x.Q1, k, 0, x.S2, k, k, k, m, T(1), T(0));
    c2.add(x.S2, k, x.L2, k, Tag{2, lv.level, x.s});
    g5.add(x.Q1, k, 0, x.L2, k, 1, x.Q, k, m, k, k, T(1), T(0));
    g5.add(x.L1, k, 1, x.L2, k, 1, x.Rinv, k, k, k, k, T(1), T(0));
    // quantities needing Q / L^-1
    g6.add(x.Linv, m, 1, x.Q, k, 0, x.Wt, k, m, k, m, T(1), T(0));          // L^-T Q
    g6.add(x.Linv, m, 0, x.AsN, dN, 0, x.Gt, dN, m, dN, m, T(1), T(0));       // L^-1 A_sN
    g6.add(x.Linv, m, 1, x.Linv, m, 0, x.M, m, m, m, m, T(1), T(0));          // L^-T L^-1
    if (x.red) {
      g6.add(x.U, m, 1, x.AsW, x.dW, 0, x.ArW, x.dW, k, x.dW, m, T(1), T(0));  // U^T A_sW
      if (use_phi_) g6.add(x.U, m, 1, phi_[x.s], 1, 0, x.phir, 1, k, 1, m, T(1), T(0));
    }
    g7.add(x.Rinv, k, 0, x.Wt, k, 1, x.Pm, m, k, m, k, T(1), T(0));           // P_ss = R^-1 (L^-T Q)^T
    g7.add(x.Wt, k, 0, x.Wt, k, 1, x.M, m, m, m, k, T(-1), T(1));             // M_ss -= W W^T
    g7.add(x.Q, k, 1, x.Gt, dN, 0, x.Tm, dN, k, dN, m, T(1), T(0));           // Q^T L^-1 A_sN
    g7.add(x.Gt, dN, 1, x.Gt, dN, 0, x.Z, dN, dN, dN, m, T(1), T(0));         // (L^-1 A_sN)^T (L^-1 A_sN)
    g8.add(x.Tm, dN, 1, x.Tm, dN, 0, x.Z, dN, dN, dN, k, T(-1), T(1));        // - T^T T
    if (x.red) {
      g8.add(x.Tm, dN, 1, x.Rinv, k, 1, x.ANr, k, dN, k, k, T(1), T(0));      // A_Nr = T^T R^-T
      g8.add(x.Rinv, k, 0, x.Rinv, k, 1, x.Arr, k, k, k, k, T(1), T(0));      // A_rr = R^-1 R^-T
    }
  }
  auto run_chol = [&](CholBatch<T> &cb) {
    if (cb.tasks.empty()) return;
    PendingStatus ps;
    // read at the next synchronisation, after the scratch arena was reset
    ps.d = (int *)per.alloc(sizeof(int) * cb.tasks.size());
    ps.what = cb.what;
    Uploader u;
    const size_t o = u.add(cb.tasks);
    char *d = u.upload(scr, sg_, st_);
    launch_chol_inv<T>((const CholTask<T> *)(d + o), (int)cb.tasks.size(), ps.d, cb.max_m, st_);
    pending_.push_back(ps);
    flops_ += cb.flops;
  };
  for (GemmBatch<T> *g : {&g1, &g2, &g3, &g4, &g5, &g6, &g7, &g8}) flops_ += g->flops;
  g1.launch(scr, sg_, st_);
  g2.launch(scr, sg_, st_);
  run_chol(c1);
  g3.launch(scr, sg_, st_);
  g4.launch(scr, sg_, st_);
  run_chol(c2);
  g5.launch(scr, sg_, st_);
  g6.launch(scr, sg_, st_);
  g7.launch(scr, sg_, st_);
  g8.launch(scr, sg_, st_);

  // register the red nodes' blocks and gather the Schur update by target
  std::unordered_map<uint64_t, std::vector<std::pair<int, int>>> tgt;  // target -> (sup idx, pair)
  std::vector<uint64_t> tgt_order;
  for (size_t q = 0; q < S.size(); ++q) {
    const Sup &x = S[q];
    const PlanSuper &ps = lv.sup[x.s];
    for (size_t i = 0; i < ps.N.size(); ++i)
      for (size_t j = i; j < ps.N.size(); ++j) {
        const uint64_t key = bkey(ps.N[i], ps.N[j]);
        auto it = tgt.find(key);
        if (it == tgt.end()) {
          tgt_order.push_back(key);
          it = tgt.emplace(key, std::vector<std::pair<int, int>>()).first;
        }
        it->second.emplace_back((int)q, (int)(i * ps.N.size() + j));
      }
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
  SumBatch<T> schur;
  for (uint64_t key : tgt_order) {
    const BlockRef<T> &dst = blocks_[key];
    const int a = (int)(key >> 32), b = (int)(key & 0xffffffffu);
    const int rk = dst.rowkey, ck = (rk == a) ? b : a;
    schur.begin(dst.ptr, dst.ld, size_[rk], size_[ck], T(-1), T(1));
    for (auto &c : tgt[key]) {
      const Sup &x = S[c.first];
      const PlanSuper &ps = lv.sup[x.s];
      // offsets of the row key and column key inside s's neighbour list
      int orow = -1, ocol = -1;
      for (size_t i = 0; i < ps.N.size(); ++i) {
        if (ps.N[i] == rk) orow = x.Noff[i];
        if (ps.N[i] == ck) ocol = x.Noff[i];
      }
      schur.src(x.Z + (int64_t)orow * x.dN + ocol, x.dN, 0);
    }
    schur.end();
  }
  schur.launch(scr, sg_, st_);

  // new red nodes, removal of the eliminated super nodes, apply records
  for (auto &x : S) {
    const PlanSuper &ps = lv.sup[x.s];
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
    std::unordered_map<int, std::vector<std::pair<int, int>>> by_target;  // key -> (node, col)
    std::vector<int> torder;
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
        if (!by_target.count(n)) torder.push_back(n);
        by_target[n].emplace_back(rc.node, nb.col);
      }
    }
    wa.tsize = t;
    h_.tmax = std::max(h_.tmax, t);
    std::sort(torder.begin(), torder.end());
    wa.tgt_first = (int)h_.targets.size();
    wa.tgt_count = (int)torder.size();
    for (int n : torder) {
      ApplyTarget tg;
      tg.x = xoff(n);
      tg.size = size_[n];
      tg.ch0 = wa.tch;
      wa.tch += (tg.size + 31) / 32;
      tg.first = (int)h_.contribs.size();
      tg.count = (int)by_target[n].size();
      for (auto &c : by_target[n]) {
        const ApplyNode &an = h_.nodes[c.first];
        ApplyContrib ac;
        ac.A = (const char *)an.AsN + sizeof(T) * (size_t)c.second;
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
  std::unordered_map<uint64_t, BlockRef<T>> nb;
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
void Run<T>::root() {
  // the remaining red nodes (level 1, or the single leaf) form the root
  const int nred = (int)size_.size();
  bool any = false;
  for (int s : size_) any = any || s > 0;
  h_.root_m = 0;
  if (!any) {
    h_.ws_size = seg_off_ + seg_size_;
    return;
  }
  merge(nred, 0);
  const int m = size_[0];
  h_.root_m = m;
  h_.root_off = seg_off_ + sup_off_[0];
  h_.ws_size = seg_off_ + seg_size_;
  const BlockRef<T> &b = blocks_.at(bkey(0, 0));
  T *Linv = talloc<T>(*h_.scratch, (size_t)m * m);
  T *Ainv = talloc<T>(*h_.pers, (size_t)m * m);
  CholBatch<T> cb;
  cb.add(b.ptr, b.ld, Linv, m, Tag{4, 0, 0});
  PendingStatus ps;
  ps.d = (int *)h_.pers->alloc(sizeof(int));
  ps.what = cb.what;
  Uploader u;
  const size_t o = u.add(cb.tasks);
  char *d = u.upload(*h_.scratch, sg_, st_);
  launch_chol_inv<T>((const CholTask<T> *)(d + o), 1, ps.d, m, st_);
  pending_.push_back(ps);
  GemmBatch<T> g;
  g.add(Linv, m, 1, Linv, m, 0, Ainv, m, m, m, m, T(1), T(0));
  flops_ += cb.flops + g.flops;
  g.launch(*h_.scratch, sg_, st_);
  h_.root_inv = Ainv;
  h_.info.root_size = m;
}

template <typename T>
void Run<T>::run() {
  h_.nodes.clear();
  h_.nbrs.clear();
  h_.targets.clear();
  h_.contribs.clear();
  h_.waves.clear();
  h_.levels.clear();
  h_.ranks.clear();
  h_.tmax = 0;
  leaf_setup();
  int nred = P_.nleaf;
  for (size_t li = 0; li < P_.levels.size(); ++li) {
    const PlanLevel &lv = P_.levels[li];
    lv_level_hint_ = lv.level;
    merge(nred, 0);
    for (int j = 0; j < lv.nsup; ++j)
      if ((size_[j] >= 0) != (bool)lv.exists[j]) fail(HS_ERR_INVALID, "internal: plan/executor mismatch");
    h_.ranks.emplace_back(lv.nsup, -1);
    for (int w = 0; w < (int)lv.waves.size(); ++w) {
      h_.scratch->reset();
      sg_.next_wave();
      wave(lv, (int)li, w);
    }
    end_level(lv, (int)li);
    nred = lv.nsup;
  }
  h_.scratch->reset();
  sg_.next_wave();
  root();
  sync_check();
  h_.info.factor_flops = flops_;
}

}  // namespace

void factorize(FactorHandle &h, const hs_csr &A, const hs_opts &o, const double *phi_host) {
  (void)A;
  (void)o;
  if (!h.pers) h.pers.reset(new DevArena(256ull << 20));
  if (!h.scratch) h.scratch.reset(new DevArena(64ull << 20));
  h.pers->reset();     // a refactorization reuses the previous factor's memory
  h.scratch->reset();
  h.info = hs_info{};
  if (h.prec == HS_PREC_F64) {
    Run<double> r(h, phi_host);
    r.run();
  } else {
    Run<float> r(h, phi_host);
    r.run();
  }
}

}  // namespace hs
