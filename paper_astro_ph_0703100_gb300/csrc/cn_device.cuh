// Device-side primitives shared by the sm_103a kernels of libcunbody.
//
// Inline PTX only for what the CUDA C++ front end does not expose directly:
// mbarrier phase tracking, the non-multicast bulk copy global -> shared
// (the j-tile staging step, the J-PACKING of Section 2.2), the
// asynchronous copies of the list gather, the MUFU inverse
// square root and the global nanosecond timer used to bound every wait.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cn {

// Device status word bits (read back by cn_get_device_status).
enum : int {
  kStatusTimeoutFull = 1,     // a consumer gave up waiting for a j-tile
  kStatusTimeoutEmpty = 2,    // the producer gave up waiting for a free stage
  kStatusTimeoutDrain = 4,    // copies still in flight when a CTA had to leave
  kStatusBadSchedule = 8,     // a work item fell outside the planned tables
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the asynchronous (bulk copy) proxy.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test_parity(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for the phase with the given parity to complete, for at most
// `limit_ns` nanoseconds of global time. Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_test_parity(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1; it < (1u << 28); ++it) {
    if (mbar_test_parity(bar, parity)) return true;
    if ((it & 63u) == 0 && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global memory into this CTA's shared memory; completion is signalled on
// `bar` as transaction bytes. Non-multicast.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// MUFU inverse square root (approximate, flush-to-zero): one instruction.
__device__ __forceinline__ float rsqrt_mufu(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no overflow).
// Uses the _rn intrinsics so that no step is contracted or reassociated.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fadd_rn(s, -a);
  const float ap = __fadd_rn(s, -bp);
  e = __fadd_rn(__fadd_rn(a, -ap), __fadd_rn(b, -bp));
}

// Adds the FP32 value x into the double-single pair (hi, lo).
__device__ __forceinline__ void ds_accumulate(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  hi = s;
  lo = __fadd_rn(lo, e);
}

// Programmatic dependent launch (PTX griddepcontrol, sm_90 and later).
// grid_dependency_wait: returns once the grids this one depends on in its
// stream have completed and their memory writes are visible (immediately
// when the kernel was launched without programmatic serialization).
// grid_launch_dependents: lets the stream's next grid, if it was launched
// with programmatic serialization, be scheduled before this one ends.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Asynchronous copies global -> shared of the gathering list kernel, issued
// without waiting: 4 bytes (a list index), 16 bytes (a record) or 16 zero
// bytes (src-size 0: nothing is read). cp_async_wait_all waits for every
// committed group of this thread, cp_async_wait_prior for all but the
// latest; cp_async_arrive_noinc makes the mbarrier count one arrival of
// this thread once all its earlier copies have landed.
__device__ __forceinline__ void cp_async_4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_zero_16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, 0;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void set_status(int* status, int bits) {
  if (status) atomicOr(status, bits);
}

}  // namespace cn
