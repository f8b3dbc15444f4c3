// Device-side building blocks shared by the kernels of libhmc (sm_103a):
// mbarrier waits with an iteration bound, bulk asynchronous copies, cluster
// (DSMEM) addressing and signalling, and the Philox4x64-10 generator.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_fp16.h>

namespace hmc {

// Error bits written to the handle's device error word.
enum : int {
  ERR_TIMEOUT_STAGE = 1,     // wait for an X tile in shared memory ran out
  ERR_TIMEOUT_EXCHANGE = 2,  // wait for peers' partial logits ran out
  ERR_TIMEOUT_SLOT = 4,      // wait for an exchange slot to be released ran out
  ERR_TIMEOUT_MMA = 8,       // wait for a tensor-core commit ran out
  ERR_BAD_LABEL = 16,        // label outside [0, K)
  ERR_NONFINITE_X = 32,      // non-finite predictor value
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init_cluster() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_local(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One probe of the phase with the given parity (CTA-scope acquire).
__device__ __forceinline__ bool mbar_test_cta(uint32_t bar, uint32_t parity) {
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

// One probe with cluster-scope acquire (data written by peer CTAs).
__device__ __forceinline__ bool mbar_test_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded waits: return false when `limit` probes did not see the phase.
__device__ __forceinline__ bool mbar_wait_cta(uint64_t* bar, uint32_t parity, long long limit) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < limit; ++i)
    if (mbar_test_cta(a, parity)) return true;
  return false;
}

__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, long long limit) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < limit; ++i)
    if (mbar_test_cluster(a, parity)) return true;
  return false;
}

// ------------------------------------------------------------ bulk copies
// Contiguous global -> shared copy completing on a local mbarrier
// (both addresses 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Order this thread's generic-proxy shared-memory writes before later async-proxy reads.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Four E4M3 values (bytes of w, byte 0 first) -> four BF16 values as two
// bf16x2 words (element 0 in the low half of lo).  Exact: E4M3 -> FP16 by the
// hardware conversion, then FP16 -> BF16 by moving the fields (every E4M3
// value is a normal FP16 number whose significand fits BF16's 7 bits; the
// exponent bias grows from 15 to 127).  Zero stays zero; X is finite.
__device__ __forceinline__ uint32_t f16x2_to_bf16x2_exact(uint32_t h) {
  const uint32_t sign = h & 0x80008000u;
  const uint32_t mag = h & 0x7fff7fffu;
  const uint32_t t = ((mag >> 3) & 0x0fff0fffu) + 0x38003800u;
  const uint32_t nz = __vcmpne2(mag, 0u);
  return (t & nz) | sign;
}
__device__ __forceinline__ void fp8x4_to_bf16x4(uint32_t w, uint32_t& lo, uint32_t& hi) {
  const __half2_raw a = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(w & 0xffffu), __NV_E4M3);
  const __half2_raw b = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(w >> 16), __NV_E4M3);
  lo = f16x2_to_bf16x2_exact(uint32_t(a.x) | (uint32_t(a.y) << 16));
  hi = f16x2_to_bf16x2_exact(uint32_t(b.x) | (uint32_t(b.y) << 16));
}

// Bulk prefetch of a contiguous global range into L2 (16-byte aligned address,
// bytes a multiple of 16); no shared memory and no completion to wait for.
__device__ __forceinline__ void bulk_prefetch_l2(const void* gsrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gsrc), "r"(bytes) : "memory");
}

// ----------------------------------------------------------------- cluster
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_peer(uint32_t local_addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
  return r;
}

// Asynchronous remote stores that complete transaction bytes on the remote
// CTA's mbarrier (both addresses already mapped to the peer).
__device__ __forceinline__ void st_async_v4f(uint32_t raddr, float a, float b, float c, float d, uint32_t rbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(raddr),
      "f"(a), "f"(b), "f"(c), "f"(d), "r"(rbar)
      : "memory");
}

__device__ __forceinline__ void st_async_v2d(uint32_t raddr, double a, double b, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(raddr),
               "d"(a), "d"(b), "r"(rbar)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_remote(uint32_t rbar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(rbar) : "memory");
}

// --------------------------------------------------------- Philox4x64-10
// Counter-based generator of Salmon, Moraes, Dror & Shaw (SC'11): ten rounds
// of two 64x64->128 multiplies, key bumped by the Weyl constants.
struct u64x4 {
  uint64_t x, y, z, w;
};

__device__ __forceinline__ u64x4 philox4x64_10(u64x4 c, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, c.x), lo0 = M0 * c.x;
    const uint64_t hi1 = __umul64hi(M1, c.z), lo1 = M1 * c.z;
    c = u64x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// 64-bit word -> double in (0, 1): ((w >> 11) + 0.5) * 2^-53.
__device__ __forceinline__ double word_to_uniform(uint64_t w) {
  return (static_cast<double>(w >> 11) + 0.5) * 1.1102230246251565404e-16;
}

enum : uint64_t { TAG_MOMENTUM = 0, TAG_ACCEPT = 1 };

// Normals q = 4*blk .. 4*blk+3 of the momentum draw of (chain, iteration):
// Box-Muller on the word pairs (w0, w1) and (w2, w3), cosine then sine.
__device__ __forceinline__ void momentum_block(uint64_t seed, uint64_t iteration, uint64_t chain, uint64_t blk,
                                               double out[4]) {
  const u64x4 w = philox4x64_10(u64x4{blk, iteration, chain, TAG_MOMENTUM}, seed, 0ull);
  const double two_pi = 2.0 * 3.14159265358979323846;
  {
    const double r = sqrt(-2.0 * log(word_to_uniform(w.x)));
    const double t = two_pi * word_to_uniform(w.y);
    out[0] = r * cos(t);
    out[1] = r * sin(t);
  }
  {
    const double r = sqrt(-2.0 * log(word_to_uniform(w.z)));
    const double t = two_pi * word_to_uniform(w.w);
    out[2] = r * cos(t);
    out[3] = r * sin(t);
  }
}

__device__ __forceinline__ double accept_uniform(uint64_t seed, uint64_t iteration, uint64_t chain) {
  const u64x4 w = philox4x64_10(u64x4{0ull, iteration, chain, TAG_ACCEPT}, seed, 0ull);
  return word_to_uniform(w.x);
}

}  // namespace hmc
