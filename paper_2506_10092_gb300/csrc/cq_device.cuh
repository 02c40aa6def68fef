// cq_device.cuh -- device helpers of the cq library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cq_desc.h"

namespace cq {

constexpr int kThreads = 512;              // fused kernel block size (16 warps)
constexpr int kWarps = kThreads / 32;
constexpr int kMaxGroupsPerWarp = 16;      // tile_rows <= kThreads * 16
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Retire an mbarrier whose phases are all complete, before its words are
// reused as ordinary shared memory.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Order this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses to the same words.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait that may suspend the thread in hardware for up to `hint_ns`
// nanoseconds while the phase is incomplete (no issue slots are spent).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: gives up after ~2 s of wall time, records CQ_ERR_TIMEOUT and
// returns false; the caller carries on (results are then flagged invalid).
// Waiting threads sleep inside try_wait instead of spinning.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err,
                                                  uint64_t limit_ns = 2000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (;;) {
    if (mbar_try_wait_sleep(bar, parity, 100000u)) return true;
    if (global_timer_ns() - t0 > limit_ns) {
      atomicCAS(err, 0, (int)CQ_ERR_TIMEOUT);
      return false;
    }
  }
}

// 1-D bulk copy global -> shared, completing on an mbarrier (TMA engine).
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ---------------------------------------------------------------- integer helpers
__device__ __forceinline__ long long ldg_val(const void* p, uint64_t i, bool v64) {
  return v64 ? __ldg(reinterpret_cast<const long long*>(p) + i)
             : (long long)__ldg(reinterpret_cast<const int*>(p) + i);
}

// Field `o` of an LSB-first bit stream held in shared memory (words may be
// read one or two past the field; the stage carries 16 bytes of slack).
__device__ __forceinline__ uint64_t extract_field(const uint32_t* w, uint32_t o, uint32_t bw) {
  const uint64_t bit = (uint64_t)o * bw;
  const uint32_t q = (uint32_t)(bit >> 5);
  const uint32_t sh = (uint32_t)(bit & 31);
  const uint32_t lo = __funnelshift_r(w[q], w[q + 1], sh);
  if (bw <= 32) return bw == 32 ? lo : (lo & ((1u << bw) - 1u));
  const uint32_t hi = __funnelshift_r(w[q + 1], w[q + 2], sh);
  const uint64_t v = ((uint64_t)hi << 32) | lo;
  return bw == 64 ? v : (v & ((1ull << bw) - 1ull));
}

// number of set bits at positions <= o (o < tile_rows)
__device__ __forceinline__ uint32_t rank_incl(const uint32_t* B, const uint32_t* P, uint32_t o) {
  const uint32_t b = o & 31;
  const uint32_t m = b == 31 ? 0xFFFFFFFFu : ((2u << b) - 1u);
  return P[o >> 5] + __popc(B[o >> 5] & m);
}

// number of set bits at positions < o
__device__ __forceinline__ uint32_t rank_excl(const uint32_t* B, const uint32_t* P, uint32_t o) {
  return P[o >> 5] + __popc(B[o >> 5] & ((1u << (o & 31)) - 1u));
}

// 128-bit helpers (two's complement in a pair of 64-bit words)
struct I128 {
  unsigned long long lo;
  long long hi;
};

__device__ __forceinline__ I128 mul_s64(long long a, long long b) {
  I128 r;
  r.lo = (unsigned long long)a * (unsigned long long)b;
  r.hi = __mul64hi(a, b);
  return r;
}

__device__ __forceinline__ I128 sext(long long a) {
  I128 r;
  r.lo = (unsigned long long)a;
  r.hi = a < 0 ? -1 : 0;
  return r;
}

// Exact 128-bit add into two shared/global words: the returned old low word
// tells whether this addition carried, so the high word receives exactly the
// carry of this addend (order independent).
__device__ __forceinline__ void atomic_add_i128(unsigned long long* lo_w, unsigned long long* hi_w, I128 x) {
  const unsigned long long old = atomicAdd(lo_w, x.lo);
  const unsigned long long carry = (old + x.lo) < old ? 1ull : 0ull;
  const unsigned long long h = (unsigned long long)x.hi + carry;
  if (h) atomicAdd(hi_w, h);
}

// Global SUM accumulator: three words, value = w0 + w1 * 2^32 + w2 * 2^64 with
// w0, w1 receiving 32-bit limbs (unsigned) and w2 the signed top.  Every
// update is a fire-and-forget atomic add; exact for < 2^32 updates per word,
// which the host guarantees: one launch covers at most 2^31 rows (each row or
// flushed group adds at most one limb per word), and the limbs are folded
// into the next word between launches (fold_sums_kernel).
__device__ __forceinline__ void global_add_limbs(unsigned long long* w0, unsigned long long* w1, unsigned long long* w2,
                                                 I128 x) {
  const unsigned long long l0 = x.lo & 0xFFFFFFFFull;
  const unsigned long long l1 = x.lo >> 32;
  if (l0) atomicAdd(w0, l0);
  if (l1) atomicAdd(w1, l1);
  if (x.hi) atomicAdd(w2, (unsigned long long)x.hi);
}

// Correctly rounded (nearest even) conversion of a 128-bit integer to double:
// the top 64 significant bits with a sticky bit for everything below are
// rounded once by the hardware 64-bit conversion, then scaled exactly.
__device__ __forceinline__ double i128_to_double(I128 x) {
  const bool neg = x.hi < 0;
  unsigned long long lo = x.lo, hi = (unsigned long long)x.hi;
  if (neg) {  // negate
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0 ? 1ull : 0ull);
  }
  double d;
  if (hi == 0) {
    d = __ull2double_rn(lo);
  } else {
    const int sh = 64 - __clzll((long long)hi);  // 1..64 bits above the low word
    unsigned long long top = sh == 64 ? hi : ((hi << (64 - sh)) | (lo >> sh));
    const unsigned long long rest = sh == 64 ? lo : (lo & ((1ull << sh) - 1ull));
    if (rest) top |= 1ull;
    d = __ull2double_rn(top) * __longlong_as_double((long long)(1023 + sh) << 52);
  }
  return neg ? -d : d;
}

// ------------------------------------------------------------------ warp search
// Number of elements x of sorted array a[0..n) with x < key (strict) or
// x <= key, by a 32-ary search (one coalesced probe per step).
__device__ __forceinline__ unsigned long long warp_count_below(const void* a, bool e64, unsigned long long n, long long key,
                                               bool strict) {
  const int lane = threadIdx.x & 31;
  unsigned long long lo = 0, hi = n;
  while (hi - lo > 32) {
    const unsigned long long step = (hi - lo + 31) / 32;
    const unsigned long long p = lo + (unsigned long long)(lane + 1) * step - 1;
    bool t = false;
    if (p < hi) {
      const long long x = ldg_val(a, p, e64);
      t = strict ? (x < key) : (x <= key);
    }
    const uint32_t c = __popc(__ballot_sync(0xFFFFFFFFu, t));
    const unsigned long long nlo = lo + (unsigned long long)c * step;
    const unsigned long long nhi = lo + (unsigned long long)(c + 1) * step - 1;
    lo = nlo;
    hi = nhi < hi ? nhi : hi;
  }
  bool t = false;
  if (lo + lane < hi) {
    const long long x = ldg_val(a, lo + lane, e64);
    t = strict ? (x < key) : (x <= key);
  }
  return lo + __popc(__ballot_sync(0xFFFFFFFFu, t));
}

}  // namespace cq
