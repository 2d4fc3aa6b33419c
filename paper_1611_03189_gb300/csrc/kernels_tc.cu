// Batched variable-size GEMM on the fifth-generation tensor cores (tcgen05)
// for the dense contractions of the factorization (Sec. 3.2: the products
// that form L^-1 U, its CholQR, L^-1 A_sN, M_ss, P_ss, A_Nr, A_rr and the
// Schur update of the neighbour blocks; Appendix A: the records P_ss, M_ss):
//
//     C = alpha op(A) op(B) + beta C,   A, B, C FP32 in global memory,
//
// with the operands rounded to TF32 (round to nearest, ties away) or BF16
// (round to nearest even) on their way into shared memory and the products
// accumulated in FP32 in tensor memory (TMEM).  In the TF32X3 form each
// operand is split into TF32 high and low parts and every product is taken
// as a_hi b_hi + a_hi b_lo + a_lo b_hi (three MMAs), which keeps about the
// accuracy of FP32 operands.
//
// One CTA of 256 threads computes one 128 x BN tile of one task (tasks of any
// size, leading dimension and transpose; a tile list is walked by a binary
// search of tile_start as in the SIMT kernel):
//   - every thread stages its share of the next K slice (128 bytes of K per
//     row) of op(A) and of op(B)^T into shared memory in the canonical
//     K-major layout without swizzle: core matrices of 8 rows x 16 bytes,
//     the 8 core matrices of a row group contiguous (K stride 128 bytes), row
//     groups 1024 bytes apart.  The blocks have arbitrary leading dimensions
//     (node sizes), which a bulk tensor copy cannot take (it needs 16-byte
//     strides), and the copy also converts the precision, so it is a plain
//     load / convert / 16-byte shared store;
//   - one thread issues the slice's four tcgen05.mma (K = 8 TF32 or 16 BF16
//     each) and commits them to the slice's mbarrier: a stage is refilled only
//     after the tensor core has read it, and the loads of slice s + 1 overlap
//     the MMAs of slice s (STAGES slices in flight);
//   - the epilogue reads the 128 x BN FP32 accumulator from TMEM (tcgen05.ld;
//     warp w reads TMEM lanes, i.e. tile rows, 32 (w % 4) .. + 31 and half
//     w / 4 of the columns), stages it in shared memory and writes C row by
//     row (coalesced) with alpha and beta.
// Every wait on an mbarrier is bounded (wait_cycles SM clocks, by default
// about one second).  On time-out the CTA stores 1 in *err, waits once more
// (with the default bound) for its tensor-core work, frees its TMEM and
// returns without writing C.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "hs_internal.h"

namespace hs {

namespace {

constexpr int TC_THREADS = 256;     // 8 warps: more loads in flight per CTA
// hs_test_wait_probe: when set, every launch first waits on a barrier that
// nothing arrives at (a test of the bounded wait's time-out path)
std::atomic<int> g_wait_probe{0};
constexpr int TC_BM = 128;           // tile rows = TMEM lanes (M of the MMA)
constexpr int TC_KBYTES = 128;       // bytes of K per stage and row
constexpr long long kTcWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// true when the phase of `parity` completed within `limit` SM clock cycles.
// The non-blocking test comes first, so that a short limit is honoured (a
// blocking try_wait may itself suspend for longer than the limit); long limits
// also use the blocking form, which frees the issue slots while it waits.
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (true) {
    if (mbar_test_wait(bar, parity)) return true;
    if (clock64() - t0 > limit) return false;
    if (limit >= 1000000 && mbar_try_wait(bar, parity)) return true;
  }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor of tcgen05: start address, leading-dimension
// byte offset (between core matrices adjacent in K), stride-dimension byte
// offset (between 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Precision of the operands: TF32 (kind::tf32, 4-byte elements, K = 8 per
// MMA) or BF16 (kind::f16 with BF16 inputs, 2-byte elements, K = 16 per MMA).
template <int KIND>
struct TcPrec;
template <>
struct TcPrec<HS_TC_TF32> {
  static constexpr int epc = 4;          // elements per 16-byte chunk
  static constexpr uint32_t fmt = 2;     // TF32 in the instruction descriptor
};
template <>
struct TcPrec<HS_TC_BF16> {
  static constexpr int epc = 8;
  static constexpr uint32_t fmt = 1;     // BF16
};
template <>
struct TcPrec<HS_TC_TF32X3> {
  static constexpr int epc = 4;
  static constexpr uint32_t fmt = 2;     // TF32 high and low parts
};

// Instruction descriptor: FP32 accumulator, A and B of the given format, both
// K-major, N = BN, M = 128.
template <int KIND, int BN>
__device__ __forceinline__ uint32_t instr_desc() {
  return (1u << 4) | (TcPrec<KIND>::fmt << 7) | (TcPrec<KIND>::fmt << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma_issue(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (KIND == HS_TC_TF32 || KIND == HS_TC_TF32X3)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// two floats -> one word of two BF16 (lo = first element, at the lower address)
__device__ __forceinline__ uint32_t to_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ int find_tile_task(const int *tile_start, int ntasks, int b) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_start[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// One operand's share of a K slice in registers: NR rows x 8 EPC-element
// chunks (16 bytes of the converted operand each) per stage, PER chunks per
// thread.
template <int KIND, int NR>
struct Slice {
  static constexpr int EPC = TcPrec<KIND>::epc;
  static constexpr int PER = NR * 8 / TC_THREADS;                 // K-contiguous: chunks per thread
  static constexpr int NQT = (2 * NR + TC_THREADS - 1) / TC_THREADS;   // rows contiguous: quads per thread
  static constexpr int SIZE = PER * EPC > NQT * 4 * EPC ? PER * EPC : NQT * 4 * EPC;
  float v[SIZE];
};

// Load rows [r0, r0 + NR) x K elements [k0, k0 + 8 EPC) of an operand X(row, k)
// into registers.  kcontig: X(row, k) = X[row * ld + k], else X[k * ld + row].
// Rows >= R and k >= K read as zero.
//  - K contiguous: item q of a thread is chunk c = tid + 128 q (row group
//    c / 64, row c % 8 of the group, K chunk (c / 8) % 8), one or two 16-byte
//    loads when aligned;
//  - rows contiguous: item qq is a quad of 4 consecutive rows x one K chunk
//    (quad d = tid + 128 qq: row quad d % (NR/4), K chunk d / (NR/4)); each of
//    its EPC k values is one 16-byte load along the rows when aligned, and the
//    quad is transposed in registers into 4 chunks (v[4 EPC qq + EPC r + kk]
//    holds row 4 quad + r, k chunk element kk).
template <int KIND, int NR>
__device__ __forceinline__ void load_slice(Slice<KIND, NR> &sl, const float *__restrict__ X, int ld, bool kcontig,
                                           bool vec, int R, int r0, int K, int k0) {
  constexpr int EPC = Slice<KIND, NR>::EPC, PER = Slice<KIND, NR>::PER;
  if (kcontig) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int c = threadIdx.x + TC_THREADS * q;
      const int grp = c >> 6, rr = c & 7, kc = (c >> 3) & 7;
      const int row = r0 + grp * 8 + rr;
      const int kb = k0 + kc * EPC;
      float *v = sl.v + q * EPC;
      if (row < R && vec && kb + EPC <= K) {
        const float4 *p = reinterpret_cast<const float4 *>(X + (int64_t)row * ld + kb);
#pragma unroll
        for (int j = 0; j < EPC / 4; ++j) {
          const float4 w = __ldg(p + j);
          v[4 * j] = w.x;
          v[4 * j + 1] = w.y;
          v[4 * j + 2] = w.z;
          v[4 * j + 3] = w.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < EPC; ++j) {
          const int k = kb + j;
          v[j] = (row < R && k < K) ? __ldg(X + (int64_t)row * ld + k) : 0.f;
        }
      }
    }
  } else {
    constexpr int NQ = NR / 4, NQT = Slice<KIND, NR>::NQT;
#pragma unroll
    for (int qq = 0; qq < NQT; ++qq) {
      const int d = threadIdx.x + TC_THREADS * qq;
      if (d >= NQ * 8) break;   // fewer quads than threads (narrow tiles)
      const int rq = d % NQ, kc = d / NQ;
      const int row = r0 + 4 * rq;
      float *v = sl.v + qq * 4 * EPC;
#pragma unroll
      for (int kk = 0; kk < EPC; ++kk) {
        const int k = k0 + kc * EPC + kk;
        if (vec && row + 3 < R && k < K) {
          const float4 w = __ldg(reinterpret_cast<const float4 *>(X + (int64_t)k * ld + row));
          v[kk] = w.x;
          v[EPC + kk] = w.y;
          v[2 * EPC + kk] = w.z;
          v[3 * EPC + kk] = w.w;
        } else {
#pragma unroll
          for (int r = 0; r < 4; ++r)
            v[r * EPC + kk] = (row + r < R && k < K) ? __ldg(X + (int64_t)k * ld + row + r) : 0.f;
        }
      }
    }
  }
}

// EPC floats -> one 16-byte chunk of the operand (and, for TF32X3, of its low part)
template <int KIND>
__device__ __forceinline__ void make_chunk(const float *v, uint4 &w, uint4 &lo) {
  if (KIND == HS_TC_TF32X3) {
    // a = a_hi + a_lo, both TF32: a_lo carries the next 11 bits of a
    w.x = to_tf32(v[0]);
    w.y = to_tf32(v[1]);
    w.z = to_tf32(v[2]);
    w.w = to_tf32(v[3]);
    lo.x = to_tf32(v[0] - __uint_as_float(w.x));
    lo.y = to_tf32(v[1] - __uint_as_float(w.y));
    lo.z = to_tf32(v[2] - __uint_as_float(w.z));
    lo.w = to_tf32(v[3] - __uint_as_float(w.w));
  } else if (KIND == HS_TC_TF32) {
    w.x = to_tf32(v[0]);
    w.y = to_tf32(v[1]);
    w.z = to_tf32(v[2]);
    w.w = to_tf32(v[3]);
  } else {
    constexpr int EPC = TcPrec<KIND>::epc;
    w.x = to_bf16x2(v[0], v[1]);
    w.y = to_bf16x2(v[2], v[3]);
    w.z = to_bf16x2(v[4 % EPC], v[5 % EPC]);
    w.w = to_bf16x2(v[6 % EPC], v[7 % EPC]);
  }
}

// Convert a slice in registers and store it into one stage buffer (dst; for
// TF32X3 the low parts into dst_lo) in the canonical K-major layout: chunk of
// row g * 8 + rr and K chunk kc at byte g * 1024 + kc * 128 + rr * 16.
template <int KIND, int NR>
__device__ __forceinline__ void store_slice(unsigned char *dst, unsigned char *dst_lo, const Slice<KIND, NR> &sl,
                                            bool kcontig) {
  constexpr int EPC = Slice<KIND, NR>::EPC, PER = Slice<KIND, NR>::PER;
  if (kcontig) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int c = threadIdx.x + TC_THREADS * q;
      const int grp = c >> 6, rr = c & 7, kc = (c >> 3) & 7;
      uint4 w, lo;
      make_chunk<KIND>(sl.v + q * EPC, w, lo);
      const int off = grp * 1024 + kc * 128 + rr * 16;
      *reinterpret_cast<uint4 *>(dst + off) = w;
      if (KIND == HS_TC_TF32X3) *reinterpret_cast<uint4 *>(dst_lo + off) = lo;
    }
  } else {
    constexpr int NQ = NR / 4, NQT = Slice<KIND, NR>::NQT;
#pragma unroll
    for (int qq = 0; qq < NQT; ++qq) {
      const int d = threadIdx.x + TC_THREADS * qq;
      if (d >= NQ * 8) break;
      const int rq = d % NQ, kc = d / NQ;
      uint4 w[4], lo[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) make_chunk<KIND>(sl.v + qq * 4 * EPC + r * EPC, w[r], lo[r]);
      // the quad's rows in an order rotated by rq / 2, so that the eight
      // lanes of a store phase write eight different 16-byte bank groups
      // (chunks picked by selects: a run-time register index would put the
      // slice in local memory)
      const int rot = (rq >> 1) & 3;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = (j + rot) & 3;
        uint4 x = w[0], y = lo[0];
#pragma unroll
        for (int i = 1; i < 4; ++i)
          if (r == i) {
            x = w[i];
            y = lo[i];
          }
        const int row = 4 * rq + r;
        const int off = (row >> 3) * 1024 + kc * 128 + (row & 7) * 16;
        *reinterpret_cast<uint4 *>(dst + off) = x;
        if (KIND == HS_TC_TF32X3) *reinterpret_cast<uint4 *>(dst_lo + off) = y;
      }
    }
  }
}

template <int KIND, int BN, int STAGES>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(const GemmTask<float> *__restrict__ tasks,
                                                         const int *__restrict__ tile_start, int ntasks, int *err,
                                                         long long wait_cycles, int probe) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int A_BYTES = TC_BM * TC_KBYTES;
  constexpr int B_BYTES = BN * TC_KBYTES;
  constexpr int PARTS = KIND == HS_TC_TF32X3 ? 2 : 1;   // high (and low) parts of each operand
  constexpr int STAGE_BYTES = PARTS * (A_BYTES + B_BYTES);
  constexpr int EPC = TcPrec<KIND>::epc;
  constexpr int KS = 8 * EPC;              // K elements per stage
  constexpr uint32_t NCOLS = BN < 32 ? 32 : BN;
  static_assert(TC_BM * (BN + 1) * 4 <= STAGES * STAGE_BYTES, "epilogue staging must fit the stage buffers");
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);   // STAGES + 1 (the probe's)
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + STAGES + 1);
  int *flag = reinterpret_cast<int *>(tslot + 1);

  const int ti = find_tile_task(tile_start, ntasks, blockIdx.x);
  const GemmTask<float> t = tasks[ti];
  const int local = blockIdx.x - tile_start[ti];
  const int tiles_n = (t.N + BN - 1) / BN;
  const int row0 = (local / tiles_n) * TC_BM;
  const int col0 = (local % tiles_n) * BN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s <= STAGES; ++s) mbar_init(smem_u32(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *flag = 0;
    // test of the time-out path: a wait on a barrier nothing arrives at
    if (probe && !mbar_wait_bounded(smem_u32(&bars[STAGES]), 0u, wait_cycles)) *flag = 1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const bool a_kc = t.ta == 0, b_kc = t.tb != 0;   // op(B)^T(j, k) = B[j ldb + k] when tb
  // 16-byte loads need a 16-byte aligned base and a leading dimension that is
  // a multiple of 4 floats (along K for K-contiguous operands, along the rows
  // for the others)
  const bool a_vec = (t.lda & 3) == 0 && ((uintptr_t)t.A & 15) == 0;
  const bool b_vec = (t.ldb & 3) == 0 && ((uintptr_t)t.B & 15) == 0;
  const int nk = (t.K > 0 && !*flag) ? (t.K + KS - 1) / KS : 0;
  const uint32_t idesc = instr_desc<KIND, BN>();
  const uint32_t sbase = smem_u32(smem);

  // Register double buffer (4-byte operand elements): slice kt + 1 is loaded
  // before slice kt is converted and stored, so its loads are in flight
  // across the store, the barrier and the MMA issue.  BF16 chunks take twice
  // the registers; there one buffer is loaded after the MMA issue.
  constexpr bool DB = EPC == 4;
  Slice<KIND, TC_BM> ra0, ra1;
  Slice<KIND, BN> rb0, rb1;
  if (nk > 0) {
    load_slice<KIND, TC_BM>(ra0, t.A, t.lda, a_kc, a_vec, t.M, row0, t.K, 0);
    load_slice<KIND, BN>(rb0, t.B, t.ldb, b_kc, b_vec, t.N, col0, t.K, 0);
  }
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt % STAGES;
    const bool odd = DB && (kt & 1);
    if (DB && kt + 1 < nk) {
      if (odd) {
        load_slice<KIND, TC_BM>(ra0, t.A, t.lda, a_kc, a_vec, t.M, row0, t.K, (kt + 1) * KS);
        load_slice<KIND, BN>(rb0, t.B, t.ldb, b_kc, b_vec, t.N, col0, t.K, (kt + 1) * KS);
      } else {
        load_slice<KIND, TC_BM>(ra1, t.A, t.lda, a_kc, a_vec, t.M, row0, t.K, (kt + 1) * KS);
        load_slice<KIND, BN>(rb1, t.B, t.ldb, b_kc, b_vec, t.N, col0, t.K, (kt + 1) * KS);
      }
    }
    if (kt >= STAGES) {
      // the MMAs of slice kt - STAGES read this stage: wait for their commit
      if (tid == 0 && !mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((kt / STAGES - 1) & 1), wait_cycles))
        *flag = 1;
      __syncthreads();
      if (*flag) break;
    }
    // stage layout: A high, B high, then (TF32X3) A low, B low
    unsigned char *sa = smem + s * STAGE_BYTES;
    unsigned char *slo = sa + A_BYTES + B_BYTES;
    if (odd) {
      store_slice<KIND, TC_BM>(sa, slo, ra1, a_kc);
      store_slice<KIND, BN>(sa + A_BYTES, slo + A_BYTES, rb1, b_kc);
    } else {
      store_slice<KIND, TC_BM>(sa, slo, ra0, a_kc);
      store_slice<KIND, BN>(sa + A_BYTES, slo + A_BYTES, rb0, b_kc);
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = sbase + s * STAGE_BYTES, b0 = a0 + A_BYTES;
      const uint32_t al = b0 + B_BYTES, bl = al + A_BYTES;
#pragma unroll
      for (int j = 0; j < 4; ++j) {   // 32 bytes of K per MMA: core matrices 2j, 2j + 1
        const uint64_t ah = smem_desc(a0 + 256 * j, 128, 1024), bh = smem_desc(b0 + 256 * j, 128, 1024);
        if (KIND == HS_TC_TF32X3) {
          // the two small cross terms first, then the leading one
          mma_issue<KIND>(tmem, smem_desc(al + 256 * j, 128, 1024), bh, idesc, (kt > 0 || j > 0) ? 1u : 0u);
          mma_issue<KIND>(tmem, ah, smem_desc(bl + 256 * j, 128, 1024), idesc, 1u);
          mma_issue<KIND>(tmem, ah, bh, idesc, 1u);
        } else {
          mma_issue<KIND>(tmem, ah, bh, idesc, (kt > 0 || j > 0) ? 1u : 0u);
        }
      }
      mma_commit(smem_u32(&bars[s]));
    }
    if (!DB && kt + 1 < nk) {
      load_slice<KIND, TC_BM>(ra0, t.A, t.lda, a_kc, a_vec, t.M, row0, t.K, (kt + 1) * KS);
      load_slice<KIND, BN>(rb0, t.B, t.ldb, b_kc, b_vec, t.N, col0, t.K, (kt + 1) * KS);
    }
  }
  // all MMAs of the tile are complete when the last commit's phase is
  if (nk > 0 && tid == 0 && !*flag) {
    const int last = nk - 1;
    if (!mbar_wait_bounded(smem_u32(&bars[last % STAGES]), (uint32_t)((last / STAGES) & 1), wait_cycles))
      *flag = 1;
  }
  __syncthreads();
  tc_fence_after();
  const bool ok = *flag == 0;
  if (ok) {
    float *cs = reinterpret_cast<float *>(smem);   // 128 x (BN + 1), over the stage buffers
    // warp w reads TMEM lanes (rows) 32 (w % 4) .. + 31, columns of half w / 4
    const int q4 = warp & 3, half = warp >> 2;
    const int r = q4 * 32 + lane;
#pragma unroll 1
    for (int c = half * (BN / 2); c < (half + 1) * (BN / 2); c += 16) {
      uint32_t v[16];
      if (nk > 0) {
        tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)c, v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0u;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) cs[r * (BN + 1) + c + j] = __uint_as_float(v[j]);
    }
    __syncthreads();
    constexpr int RPI = TC_THREADS / BN;   // rows written per pass
    const int cc = tid % BN, rsub = tid / BN;
    const int gc = col0 + cc;
    if (gc < t.N) {
#pragma unroll 4
      for (int i = rsub; i < TC_BM; i += RPI) {
        const int gr = row0 + i;
        if (gr >= t.M) break;
        float *p = t.C + (int64_t)gr * t.ldc + gc;
        float x = t.alpha * cs[i * (BN + 1) + cc];
        if (t.beta != 0.f) x = fmaf(t.beta, *p, x);
        *p = x;
      }
    }
  } else {
    if (tid == 0) {
      atomicExch(err, 1);
      // the tensor core's outstanding work gets one more wait, with the
      // default bound (not the caller's, which may be very short), before
      // its tensor memory is released
      for (int s = 0; s < STAGES; ++s) {
        const int uses = nk > s ? (nk - 1 - s) / STAGES : -1;
        if (uses >= 0) (void)mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)(uses & 1), kTcWaitCycles);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
  }
}

template <int KIND, int BN>
void launch_tc_bn(const GemmTask<float> *d_tasks, const int *d_tile_start, int ntasks, int total_tiles, int *d_err,
                  long long wait_cycles, cudaStream_t st) {
  // 128-wide tiles keep three K slices in flight (96 KB, two CTAs per SM);
  // 64-wide tiles two (48 KB, four CTAs per SM), for the many small tasks
  constexpr int PARTS = KIND == HS_TC_TF32X3 ? 2 : 1;
  constexpr int STAGES = (BN == 128 && PARTS == 1) ? 3 : 2;
  constexpr size_t smem = (size_t)STAGES * PARTS * (TC_BM + BN) * TC_KBYTES + 8 * (STAGES + 1) + 16;
  const int lim = allow_max_dynamic_smem<k_gemm_tc<KIND, BN, STAGES>>();
  check_dynamic_smem(smem, lim, "the tensor-core GEMM");
  k_gemm_tc<KIND, BN, STAGES><<<total_tiles, TC_THREADS, smem, st>>>(
      d_tasks, d_tile_start, ntasks, d_err, wait_cycles > 0 ? wait_cycles : kTcWaitCycles,
      g_wait_probe.load() ? 1 : 0);
  count_launch();
  HS_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Autotuner of the batched GEMM.  For each class of task shapes (the larger of
// M and N, and K, each bucketed by powers of four) it times three variants on
// a synthetic batch of that class -- the CUDA-core kernel with 64 x 64 tiles
// and the tensor-core kernel with 128 x 64 and 128 x 128 tiles -- and keeps
// the fastest (a tensor-core variant must win by 15%).  Small tasks favour the
// CUDA-core kernel (more CTAs per SM, no TMEM set-up); large ones the tensor
// cores.  The table is built once per
// device and operand precision, on a private stream after a device-wide
// synchronisation, the first time a factorization needs it; afterwards a
// task's variant depends on its shape alone, so a problem computes the same
// bits alone and in a batch.  HS_GEMM_ROUTE (environment) = simt, tc64 or
// tc128 fixes the variant for every task.
// ---------------------------------------------------------------------------
constexpr int kTuneMN = 5;   // max(M, N) <= 32, 64, 128, 256, more
constexpr int kTuneK = 4;    // K <= 32, 128, 512, more
const int kTuneMNRep[kTuneMN] = {32, 64, 128, 256, 512};
const int kTuneKRep[kTuneK] = {32, 128, 512, 1024};

int tune_mn_class(int v) {
  int c = 0;
  while (c < kTuneMN - 1 && v > kTuneMNRep[c]) ++c;
  return c;
}
int tune_k_class(int v) {
  int c = 0;
  while (c < kTuneK - 1 && v > kTuneKRep[c]) ++c;
  return c;
}

int forced_route() {
  static const int v = [] {
    const char *e = std::getenv("HS_GEMM_ROUTE");
    if (!e) return -1;
    const std::string s(e);
    return s == "simt" ? 0 : s == "tc64" ? 64 : s == "tc128" ? 128 : -1;
  }();
  return v;
}

struct TuneTable {
  bool ready = false;
  int route[kTuneMN][kTuneK];
  float ms[kTuneMN][kTuneK][3];
};

std::mutex g_tune_mu;
TuneTable g_tune[64][4];   // [device][kind]

void tune_device(int kind, TuneTable &tt) {
  HS_CUDA(cudaDeviceSynchronize());
  cudaStream_t st = nullptr;
  HS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  struct Cleanup {
    cudaStream_t st;
    std::vector<void *> mem;
    std::vector<cudaEvent_t> ev;
    ~Cleanup() {
      if (st) cudaStreamSynchronize(st);
      for (void *p : mem) cudaFree(p);
      for (cudaEvent_t e : ev) cudaEventDestroy(e);
      if (st) cudaStreamDestroy(st);
    }
  } cl{st, {}, {}};
  const size_t ab = (size_t)512 * 1024;                   // largest A and B
  const size_t cbytes = (size_t)40 << 20;                 // C of all tasks of a batch
  float *A = nullptr, *B = nullptr, *Cb = nullptr;
  int *d_err = nullptr;
  HS_CUDA(cudaMalloc(&A, ab * sizeof(float)));
  cl.mem.push_back(A);
  HS_CUDA(cudaMalloc(&B, ab * sizeof(float)));
  cl.mem.push_back(B);
  HS_CUDA(cudaMalloc(&Cb, cbytes));
  cl.mem.push_back(Cb);
  HS_CUDA(cudaMalloc(&d_err, sizeof(int)));
  cl.mem.push_back(d_err);
  HS_CUDA(cudaMemsetAsync(A, 0, ab * sizeof(float), st));
  HS_CUDA(cudaMemsetAsync(B, 0, ab * sizeof(float), st));
  HS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
  cudaEvent_t e0, e1;
  HS_CUDA(cudaEventCreate(&e0));
  cl.ev.push_back(e0);
  HS_CUDA(cudaEventCreate(&e1));
  cl.ev.push_back(e1);
  // descriptors: tasks, then the tile starts of the three variants
  const int max_tasks = 2048;
  char *d_desc = nullptr;
  const size_t desc_bytes = sizeof(GemmTask<float>) * max_tasks + 3 * sizeof(int) * (max_tasks + 16);
  HS_CUDA(cudaMalloc(&d_desc, desc_bytes));
  cl.mem.push_back(d_desc);
  for (int cm = 0; cm < kTuneMN; ++cm)
    for (int ck = 0; ck < kTuneK; ++ck) {
      const int M = kTuneMNRep[cm], N = M, K = kTuneKRep[ck];
      const double per = 2.0 * M * N * K;
      // at least 8 tasks, so that even the largest class fills a good part
      // of the GPU, as the factor's batches of that class do
      int T = (int)std::max(8.0, std::min((double)max_tasks, 64e6 / per));
      T = (int)std::min<size_t>((size_t)T, cbytes / (sizeof(float) * (size_t)M * N));
      std::vector<GemmTask<float>> tasks(T);
      for (int i = 0; i < T; ++i) {
        GemmTask<float> &t = tasks[i];
        t.A = A;
        t.B = B;
        t.C = Cb + (size_t)i * M * N;
        t.M = M;
        t.N = N;
        t.K = K;
        t.lda = K;
        t.ldb = N;
        t.ldc = N;
        t.ta = 0;
        t.tb = 0;
        t.alpha = 1.f;
        t.beta = 0.f;
      }
      const int tms[3] = {GEMM_TM, TC_TILE_M, TC_TILE_M}, tns[3] = {GEMM_TN, 64, 128};
      std::vector<int> starts(3 * (T + 1));
      int tiles[3];
      for (int v = 0; v < 3; ++v) {
        int acc = 0;
        for (int i = 0; i < T; ++i) {
          starts[v * (T + 1) + i] = acc;
          acc += ((M + tms[v] - 1) / tms[v]) * ((N + tns[v] - 1) / tns[v]);
        }
        tiles[v] = acc;
      }
      GemmTask<float> *d_t = (GemmTask<float> *)d_desc;
      int *d_s = (int *)(d_desc + sizeof(GemmTask<float>) * max_tasks);
      HS_CUDA(cudaMemcpyAsync(d_t, tasks.data(), sizeof(GemmTask<float>) * T, cudaMemcpyHostToDevice, st));
      HS_CUDA(cudaMemcpyAsync(d_s, starts.data(), sizeof(int) * starts.size(), cudaMemcpyHostToDevice, st));
      float best = 1e30f;
      int choice = 0;
      for (int v = 0; v < 3; ++v) {
        float tmin = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
          HS_CUDA(cudaEventRecord(e0, st));
          if (v == 0)
            launch_gemm<float>(d_t, d_s, T, tiles[0], st);
          else if (v == 1)
            launch_gemm_tc(kind, 64, d_t, d_s + (T + 1), T, tiles[1], d_err, st);
          else
            launch_gemm_tc(kind, 128, d_t, d_s + 2 * (T + 1), T, tiles[2], d_err, st);
          HS_CUDA(cudaEventRecord(e1, st));
          HS_CUDA(cudaEventSynchronize(e1));
          float t = 0.f;
          HS_CUDA(cudaEventElapsedTime(&t, e0, e1));
          if (rep > 0) tmin = std::min(tmin, t);   // the first run warms up
        }
        tt.ms[cm][ck][v] = tmin;
        // a tensor-core variant must beat the CUDA-core kernel by 15%: the
        // synthetic batch has one shape, the factor's batches mix shapes, and
        // near a tie the CUDA-core kernel also keeps FP32 operands
        const float t_eff = v == 0 ? tmin : tmin * 1.15f;
        if (t_eff < best) {
          best = t_eff;
          choice = v == 0 ? 0 : v == 1 ? 64 : 128;
        }
      }
      tt.route[cm][ck] = choice;
    }
  int herr = 0;
  HS_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  HS_CUDA(cudaStreamSynchronize(st));
  if (herr) fail(HS_ERR_TIMEOUT, "a bounded wait of the tensor-core GEMM ran out while tuning");
  tt.ready = true;
}

const TuneTable &tune_table(int kind) {
  int dev = 0;
  HS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || kind < 1 || kind > 3) fail(HS_ERR_INVALID, "internal: GEMM tuner device or kind");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  TuneTable &tt = g_tune[dev][kind];
  if (!tt.ready) tune_device(kind, tt);
  return tt;
}

}  // namespace

void launch_gemm_tc(int kind, int bn, const GemmTask<float> *d_tasks, const int *d_tile_start, int ntasks,
                    int total_tiles, int *d_err, cudaStream_t st, long long wait_cycles) {
  if (ntasks == 0 || total_tiles == 0) return;
  if (kind == HS_TC_TF32 && bn == 128)
    launch_tc_bn<HS_TC_TF32, 128>(d_tasks, d_tile_start, ntasks, total_tiles, d_err, wait_cycles, st);
  else if (kind == HS_TC_TF32 && bn == 64)
    launch_tc_bn<HS_TC_TF32, 64>(d_tasks, d_tile_start, ntasks, total_tiles, d_err, wait_cycles, st);
  else if (kind == HS_TC_BF16 && bn == 128)
    launch_tc_bn<HS_TC_BF16, 128>(d_tasks, d_tile_start, ntasks, total_tiles, d_err, wait_cycles, st);
  else if (kind == HS_TC_BF16 && bn == 64)
    launch_tc_bn<HS_TC_BF16, 64>(d_tasks, d_tile_start, ntasks, total_tiles, d_err, wait_cycles, st);
  else if (kind == HS_TC_TF32X3 && bn == 128)
    launch_tc_bn<HS_TC_TF32X3, 128>(d_tasks, d_tile_start, ntasks, total_tiles, d_err, wait_cycles, st);
  else if (kind == HS_TC_TF32X3 && bn == 64)
    launch_tc_bn<HS_TC_TF32X3, 64>(d_tasks, d_tile_start, ntasks, total_tiles, d_err, wait_cycles, st);
  else
    fail(HS_ERR_INVALID, "tensor-core GEMM: unknown precision or tile width");
}

void set_wait_probe(bool on) { g_wait_probe.store(on ? 1 : 0); }

void gemm_tune(int kind) {
  if (kind != HS_TC_NONE && forced_route() < 0) (void)tune_table(kind);
}

int gemm_route(int kind, int M, int N, int K) {
  if (kind == HS_TC_NONE) return 0;
  const int f = forced_route();
  if (f >= 0) return f;
  const TuneTable &tt = tune_table(kind);
  return tt.route[tune_mn_class(std::max(M, N))][tune_k_class(K)];
}

int gemm_tune_report(int kind, float *ms, int *route, int cap) {
  const TuneTable &tt = tune_table(kind);
  int n = 0;
  for (int cm = 0; cm < kTuneMN; ++cm)
    for (int ck = 0; ck < kTuneK; ++ck, ++n)
      if (n < cap) {
        for (int v = 0; v < 3; ++v) ms[3 * n + v] = tt.ms[cm][ck][v];
        route[n] = tt.route[cm][ck];
      }
  return kTuneMN * kTuneK;
}

}  // namespace hs
