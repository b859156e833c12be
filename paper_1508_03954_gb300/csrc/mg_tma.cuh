// mg_tma.cuh -- tensor-memory-accelerator plane loads with mbarrier completion
// (sm_103a, inline PTX).
//
// A level array of (n+1)^3 complex values is described to the TMA unit as a
// 3D tensor of 2(n+1) x (n+1) x (n+1) reals (x fastest); one load copies a
// box of (2 w) x 32 x 1 reals -- w complex columns, 32 rows, one z plane --
// into shared memory.  Coordinates outside the tensor (the halo beyond the
// Dirichlet ring, planes below 0 or above n) are filled with zeros by the
// hardware, so the kernels need no bounds tests for their plane loads.  The
// copy signals an mbarrier (arrival count 1: the issuing thread's
// arrive.expect_tx) with the box's byte count.  Waits are bounded: after
// `limit` unsuccessful polls the wait sets bit 2 of the context's sticky
// error flag and returns false (the host reports MG_ERR_TIMEOUT).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace mg {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes the initialised barriers visible to the async proxy
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// orders this thread's earlier shared-memory accesses before later async-proxy writes
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// box load of one plane: x in reals (x * element size a multiple of 16 bytes), y, z
__device__ __forceinline__ void tma_load_plane(void* dst, const CUtensorMap* map, unsigned long long* bar, int x,
                                               int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the completion of the barrier phase of the given parity
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned limit,
                                                  unsigned* err) {
  unsigned spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++spins > limit) {
      if (err != nullptr) atomicOr(err, 2u);
      return false;
    }
  }
  return true;
}

}  // namespace mg
