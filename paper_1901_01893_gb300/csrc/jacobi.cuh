// Pieces shared by the Jacobi eigensolvers: the round-robin pair schedule and the
// thread-block-cluster primitives (distributed shared memory, cluster mbarriers and
// barriers) in inline PTX.
#pragma once

#include <stdint.h>

#include "common.cuh"

// Round `round` of the cyclic round-robin ("circle") ordering of n (even) indices:
// pair k < n/2 is (p, q), p < q.  Index 0 stays put and the others rotate by one per
// round, so n - 1 rounds of n/2 disjoint pairs meet every pair exactly once.
__device__ __forceinline__ void jpair(int round, int k, int n, int& p, int& q) {
  const int m = n - 1;
  int a, b;
  if (k == 0) {
    a = 0;
    b = 1 + (round % m);
  } else {
    a = 1 + ((k + round) % m);
    b = 1 + ((m - k + round) % m);
  }
  p = min(a, b);
  q = max(a, b);
}

// iteration limit of every mbarrier wait (then the waiting side reports SMSM_ERR_TIMEOUT)
#define JAC_MAXWAIT (1L << 22)

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_st_v4(uint32_t a, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void cl_st_s32(uint32_t a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_arrive(uint32_t remote_mbar, uint32_t count) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(remote_mbar), "r"(count)
               : "memory");
}
// bounded wait on a local mbarrier phase, acquiring what the other CTA released
__device__ __forceinline__ bool cl_wait(uint64_t* mbar, uint32_t parity) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(mbar);
  for (long it = 0; it < JAC_MAXWAIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        "selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// 16-byte load from a shared::cluster address (another CTA's shared memory via cl_map)
__device__ __forceinline__ float4 cl_ld_v4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a)
               : "memory");
  return v;
}
