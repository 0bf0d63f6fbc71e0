// tcgen05 building blocks shared by the tensor-core kernels (hand-written
// PTX for sm_103a): tensor-memory allocation, 16-bit MMAs with FP32
// accumulators in tensor memory, commit to an mbarrier, bounded waits, TMEM
// loads, bulk copies, shared-memory matrix descriptors (no swizzle) and the
// core-matrix tile layout (8 rows x 16 bytes).
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace fv {
namespace tc {

// every mbarrier wait gives up after 4e9 SM cycles (2 s at the 2032 MHz maximum
// clock, longer at lower clocks); the bound is kept in SM cycles because the
// cycle counter is cheap to read, while a read of the global nanosecond timer
// costs hundreds of cycles
constexpr long long kTcWaitCycles = 4000000000ll;

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }


__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

// One test of the phase; a thread whose phase is not complete is suspended
// until it completes or for at most about 1 ms (the suspend-time hint), so
// waiting threads leave the issue slots to the threads they wait for (the MMA
// issuers share the SM sub-partitions with them).
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity), "n"(1000000)
      : "memory");
  return ok != 0;
}

// Wait for the phase with parity `parity` to complete; false after the bound.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > kTcWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

// Bulk copies (cp.async.bulk) from global to shared memory: addresses 16-byte
// aligned, sizes multiples of 16; they complete on an mbarrier armed with the
// bytes to expect.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
// L2 policy for data streamed through once (first to be evicted).
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
               ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(bar)), "l"(pol)
               : "memory");
}

// Bulk copies from shared to global memory, tracked per thread in bulk groups:
// wait_read<N> returns once at most N of the issuing thread's groups still
// read their shared-memory source; bulk_wait_all once all have completed.
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(su32(src)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
template <int N> __device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle: start, LBO (K-direction core
// matrix stride), SBO (M/N-direction 8-row group stride), version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: D F32, A/B format fmt (0 F16, 1 BF16), majors, N, M.
__device__ __forceinline__ uint32_t idesc_f16(uint32_t fmt, int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// 16-bit operand formats for kind::f16: BF16 (8-bit significand, FP32 range)
// or FP16 (11-bit significand; the reverse sweep scales its adjoints by a
// power of two to stay inside FP16's range).
struct OpBF16 {
  static constexpr uint32_t fmt = 1;
  static constexpr uint32_t one = 0x3F80u;   // 1.0

  __device__ static __forceinline__ uint32_t pack(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
  }
  __device__ static __forceinline__ float lo(uint32_t u) { return __uint_as_float(u << 16); }
  __device__ static __forceinline__ float hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }
};
struct OpF16 {
  static constexpr uint32_t fmt = 0;
  static constexpr uint32_t one = 0x3C00u;   // 1.0

  __device__ static __forceinline__ uint32_t pack(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
  }
  __device__ static __forceinline__ float lo(uint32_t u) { return __half2float(__ushort_as_half((unsigned short)(u & 0xFFFFu))); }
  __device__ static __forceinline__ float hi(uint32_t u) { return __half2float(__ushort_as_half((unsigned short)(u >> 16))); }
};

__device__ __forceinline__ __half2 u32_h2(uint32_t u) {
  __half2 h;
  *reinterpret_cast<uint32_t*>(&h) = u;
  return h;
}
__device__ __forceinline__ uint32_t h2_u32(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The bias column of an activation tile holds (1, 0, 0) in the value and
// tangent streams.  Of eight packed columns [cc, cc + 8) (four words per
// stream), set column k to that: value 1, tangents 0.  Called only by the
// warps whose column range holds the bias column (a warp-uniform branch).
template <class OP>
__device__ __forceinline__ void set_bias_col(int k, uint32_t pv[4], uint32_t px[4], uint32_t py[4]) {
  const int sel = k >> 1;
  const uint32_t keep = (k & 1) ? 0x0000FFFFu : 0xFFFF0000u;
  const uint32_t one = (k & 1) ? (OP::one << 16) : OP::one;
#pragma unroll
  for (int w = 0; w < 4; ++w) {           // constant indices: the words stay in registers
    pv[w] = sel == w ? ((pv[w] & keep) | one) : pv[w];
    px[w] = sel == w ? (px[w] & keep) : px[w];
    py[w] = sel == w ? (py[w] & keep) : py[w];
  }
}

// Activation tile layout (one stream): row p, column k of a [128 x Kb] BF16
// tile: (p/8)*Kb*16 + (k/8)*128 + (p%8)*16 + (k%8)*2 bytes.  A stream spans
// 256*Kb bytes.
__device__ __forceinline__ uint32_t row_off(int p, int Kb) { return (p >> 3) * (Kb * 16) + (p & 7) * 16; }

// 8 columns [c, c+8) of row p (one 16-byte core-matrix row segment).
__device__ __forceinline__ void st8(uint8_t* stream, int Kb, int p, int c, const uint32_t pk[4]) {
  *reinterpret_cast<uint4*>(stream + row_off(p, Kb) + (c >> 3) * 128) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
}
template <class OP>
__device__ __forceinline__ void ld8(const uint8_t* stream, int Kb, int p, int c, float v[8]) {
  const uint4 x = *reinterpret_cast<const uint4*>(stream + row_off(p, Kb) + (c >> 3) * 128);
  const uint32_t u[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) { v[2 * i] = OP::lo(u[i]); v[2 * i + 1] = OP::hi(u[i]); }
}

}  // namespace tc
}  // namespace fv
