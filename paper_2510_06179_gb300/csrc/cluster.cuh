// Thread-block-cluster primitives for the distributed PCG (inline PTX, sm_90+ cluster model):
// CTA rank and cluster ids, distributed shared memory (DSMEM) loads and stores through
// mapa-translated addresses, and mbarrier-based waits that give up after a time limit
// instead of blocking forever.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmpc {
namespace cl {

__device__ __forceinline__ uint32_t rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t ncta() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t nclusters() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// shared::cta address of a pointer into this CTA's shared memory
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// the same shared-memory offset in CTA `r` of the cluster (shared::cluster window)
__device__ __forceinline__ uint32_t map(uint32_t a, uint32_t r) {
  uint32_t o;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(o) : "r"(a), "r"(r));
  return o;
}

__device__ __forceinline__ float ld_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ double ld_f64(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ int ld_s32(uint32_t a) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_f32(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void st_f64(uint32_t a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

// Asynchronous store into another CTA's shared memory that signals the mbarrier `bar` of that
// CTA (both shared::cluster addresses) with its 4 or 8 bytes when it lands.
__device__ __forceinline__ void st_async_f32(uint32_t a, float v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(a), "f"(v), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void st_async_f64(uint32_t a, double v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(a), "d"(v), "r"(bar)
               : "memory");
}
// arrive on this CTA's mbarrier at `a`, announcing `bytes` of asynchronous stores for its phase
__device__ __forceinline__ void arrive_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(a), "r"(bytes)
               : "memory");
}

// mbarrier in this CTA's shared memory, expecting `count` arrivals per phase
__device__ __forceinline__ void bar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
// make the initialised barriers visible to the other CTAs of the cluster
__device__ __forceinline__ void fence_bar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// arrive on the mbarrier at shared::cluster address `a` (possibly another CTA's), releasing
// this thread's earlier writes at cluster scope
__device__ __forceinline__ void arrive_remote(uint32_t a) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(a) : "memory");
}
// one bounded wait for the phase with parity `par` of this CTA's mbarrier at `a`; acquire at
// cluster scope.  Returns false when `limit_ns` passed first.
__device__ __forceinline__ bool wait(uint32_t a, uint32_t par, unsigned long long limit_ns) {
  const unsigned long long t0 = now_ns();
  for (uint32_t n = 0; n < (1u << 30); ++n) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(par)
        : "memory");
    if (ok) return true;
    if ((n & 15) == 15 && now_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// hardware cluster barrier (all threads of all CTAs); used only at kernel entry and exit,
// which every thread of every CTA reaches on the same straight-line path
__device__ __forceinline__ void sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

}  // namespace cl
}  // namespace dmpc
