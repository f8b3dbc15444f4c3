// Fused log-posterior + gradient pass on the 5th-generation tensor cores
// (tcgen05) for X stored in BF16, many chains at once (Eqs. softmax, loglike,
// logkernel and gradient of Sec. 2.1, evaluated for C = chains*(K-1)
// coefficient columns).
//
// Decomposition: a cluster of S CTAs walks row tiles of 128 rows; CTA `rank`
// owns the column slice [rank*PC, (rank+1)*PC) (PC a multiple of 128) of X and
// of the coefficients, and accumulates the gradient rows of that slice in
// TMEM across all of the cluster's tiles.  Per tile:
//   sweep 1  TMA brings 128 x 64 boxes of X (128-byte swizzle) together with
//            the matching 64-column box of the BF16 coefficients; MMA
//            D_z[128 x N] += X_box . B_box^T (both operands K-major).
//   exchange the epilogue warps read D_z (one row per thread), publish the
//            CTA's partial logits to global memory (L2), and signal every
//            peer (remote mbarrier arrive); each CTA then owns 128/S rows:
//            it sums the S partials in rank order, forms the softmax with the
//            zero logit of class K, the residual R = Y - P (BF16) and the row
//            log-likelihood, publishes its R rows and signals again.
//   sweep 2  TMA loads the tile's full R (128 x N, MN-major) and re-reads X
//            in 128-column blocks (an L2 hit: the tile was streamed one
//            sweep earlier); MMA D_g[mb] (128 columns x N) += X_blk^T . R with
//            X_blk read MN-major from the same swizzled boxes.
// Sweeps are interleaved S1(0), S1(1), S2(0), S1(2), S2(1), ... so the
// exchange of one tile overlaps the next tile's first sweep.
// Warp roles: warp 0 TMA producer, warp 1 TMEM owner + MMA issuer, warps 2-5
// epilogue (TMEM lanes 0-127).  All waits are bounded.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "internal.h"
#include "tc_common.cuh"

namespace hmc {
namespace tc {

constexpr int kThreads = 192;
constexpr int kRows = 128;
constexpr int kBox = 64;          // BF16 elements per 128-byte box row
constexpr int kBoxBytes = kRows * 128;

struct TcArgs {
  int64_t n;
  int32_t p_pad, PC, S, N, NP, C, Km1, chains, MB, NST, nclusters;
  int64_t ntiles;
  uint32_t tmem_cols, stage_bytes;
  float* gpart;             // [cluster][C][p_pad] partial gradient (this launch's columns)
  int64_t gpart_cstride;
  double* lpart;            // [cluster*S + rank][lpart_cstride] partial log-likelihood per chain
  int32_t lpart_cstride;
  float* zg;                // [nclu][2][S][128][N]
  __nv_bfloat16* rg;        // [nclu][2][128][NP]
  const int32_t* y;
  int* err;
  long long spin_limit;
  int32_t inject_timeout;
};

struct Smem {
  size_t ring, rbuf, lacc, bars, total;
};

__host__ __device__ inline size_t al(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline Smem smem_layout(int NST, uint32_t stage_bytes, int NP, int items) {
  Smem L;
  size_t off = 0;
  L.ring = off;  off = al(off + size_t(NST) * stage_bytes, 1024);
  L.rbuf = off;  off = al(off + size_t(NP / kBox) * kBoxBytes, 1024);
  L.lacc = off;  off = al(off + size_t(items) * 8, 16);
  L.bars = off;  off = al(off + size_t(2 * NST + 16) * 8 + 16, 16);
  L.total = off + 1024;  // slack for aligning the dynamic base to 1024
  return L;
}

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, long long limit, volatile int* abort,
                                             bool cluster_scope) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < limit; ++i) {
    if (cluster_scope ? mbar_test_cluster(a, parity) : mbar_test_cta(a, parity)) return true;
    if ((i & 63) == 63 && *abort) return false;
  }
  return false;
}

__device__ __forceinline__ void named_bar_epi() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__global__ void __launch_bounds__(kThreads, 1)
    lpg_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB,
                  const __grid_constant__ CUtensorMap tmR, const TcArgs A) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int S = A.S, N = A.N, NST = A.NST;
  const uint32_t rank = (S > 1) ? cluster_rank() : 0u;
  const int cl = blockIdx.x / S;
  const int RS = kRows / S;                        // rows this CTA owns in the exchange
  const int items = RS * A.chains;
  const Smem Lo = smem_layout(NST, A.stage_bytes, A.NP, items);
  unsigned char* ring = smem + Lo.ring;
  unsigned char* rbuf = smem + Lo.rbuf;
  double* lacc = reinterpret_cast<double*>(smem + Lo.lacc);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lo.bars);
  uint64_t* full = bars;
  uint64_t* empty = bars + NST;
  uint64_t* zdone = bars + 2 * NST;
  uint64_t* zfree = zdone + 1;
  uint64_t* zrdy = zdone + 2;    // [2]
  uint64_t* rrdy = zdone + 4;    // [2]
  uint64_t* rfull = zdone + 6;
  uint64_t* rfree = zdone + 7;
  uint64_t* gdone = zdone + 8;
  uint64_t* drain = zdone + 9;
  uint64_t* never = zdone + 10;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(zdone + 11);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(zdone + 12);

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(zdone, 1);
    mbar_init(zfree, 4);
    mbar_init(&zrdy[0], S);
    mbar_init(&zrdy[1], S);
    mbar_init(&rrdy[0], S);
    mbar_init(&rrdy[1], S);
    mbar_init(rfull, 1);
    mbar_init(rfree, 1);
    mbar_init(gdone, 1);
    mbar_init(drain, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    fence_mbar_init_cluster();
    prefetch_tmap(&tmX);
    prefetch_tmap(&tmB);
    prefetch_tmap(&tmR);
  }
  for (int i = tid; i < items; i += kThreads) lacc[i] = 0.0;
  if (warp == 1) tmem_alloc(tmem_slot, A.tmem_cols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  if (A.inject_timeout && tid == 0) {
    if (!wait_bounded(never, 0u, A.spin_limit, abort_flag, false)) {
      *abort_flag = 1;
      atomicOr(A.err, ERR_TIMEOUT_STAGE);
    }
  }
  if (S > 1)
    cluster_sync_all();
  else
    __syncthreads();

  const int64_t nclu = A.nclusters;
  const int64_t T = (*abort_flag || cl >= A.ntiles) ? 0 : (A.ntiles - 1 - cl) / nclu + 1;
  const int64_t nphase = 2 * T;
  const int NKB = A.PC / kBox;
  auto phase = [&](int64_t k, bool* s2) -> int64_t {
    if (k == 0) { *s2 = false; return 0; }
    if (k == nphase - 1) { *s2 = true; return T - 1; }
    const int64_t v = (k + 1) / 2;
    *s2 = (k % 2) == 0;
    return *s2 ? v - 1 : v;
  };
  auto fail = [&](int bit) {
    *abort_flag = 1;
    atomicOr(A.err, bit);
  };

  int64_t issued = 0;  // producer: ring uses issued
  int64_t r_loads = 0;
  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int64_t j = 0;
      for (int64_t k = 0; k < nphase && !*abort_flag; ++k) {
        bool s2;
        const int64_t u = phase(k, &s2);
        const int row0 = int((cl + u * nclu) * kRows);
        if (!s2) {
          for (int kb = 0; kb < NKB; ++kb, ++j) {
            const int st = int(j % NST);
            if (!wait_bounded(&empty[st], uint32_t(((j / NST) & 1) ^ 1), A.spin_limit, abort_flag, false)) {
              fail(ERR_TIMEOUT_STAGE);
              break;
            }
            unsigned char* sp = ring + size_t(st) * A.stage_bytes;
            mbar_arrive_expect_tx(&full[st], uint32_t(kBoxBytes + N * 128));
            const int c0 = int(rank) * A.PC + kb * kBox;
            tma_load_2d(sp, &tmX, c0, row0, &full[st]);
            tma_load_2d(sp + kBoxBytes, &tmB, c0, 0, &full[st]);
            issued = j + 1;
          }
        } else {
          if (u >= 1 && !wait_bounded(rfree, uint32_t((u - 1) & 1), A.spin_limit, abort_flag, false)) {
            fail(ERR_TIMEOUT_MMA);
            break;
          }
          if (!wait_bounded(&rrdy[u & 1], uint32_t((u >> 1) & 1), A.spin_limit, abort_flag, true)) {
            fail(ERR_TIMEOUT_EXCHANGE);
            break;
          }
          fence_proxy_async_global();
          const int nrb = A.NP / kBox;
          mbar_arrive_expect_tx(rfull, uint32_t(nrb * kBoxBytes));
          for (int h = 0; h < nrb; ++h)
            tma_load_2d(rbuf + size_t(h) * kBoxBytes, &tmR, h * kBox, int((cl * 2 + (u & 1)) * kRows), rfull);
          r_loads = u + 1;
          for (int mb = 0; mb < A.MB; ++mb, ++j) {
            const int st = int(j % NST);
            if (!wait_bounded(&empty[st], uint32_t(((j / NST) & 1) ^ 1), A.spin_limit, abort_flag, false)) {
              fail(ERR_TIMEOUT_STAGE);
              break;
            }
            unsigned char* sp = ring + size_t(st) * A.stage_bytes;
            mbar_arrive_expect_tx(&full[st], uint32_t(2 * kBoxBytes));
            const int c0 = int(rank) * A.PC + mb * 128;
            tma_load_2d(sp, &tmX, c0, row0, &full[st]);
            tma_load_2d(sp + kBoxBytes, &tmX, c0 + kBox, row0, &full[st]);
            issued = j + 1;
          }
        }
      }
      // Every copy issued must land before shared memory is released.
      for (int64_t jj = (issued > NST ? issued - NST : 0); jj < issued; ++jj)
        (void)wait_bounded(&full[jj % NST], uint32_t((jj / NST) & 1), A.spin_limit, abort_flag, false);
      if (r_loads > 0) (void)wait_bounded(rfull, uint32_t((r_loads - 1) & 1), A.spin_limit, abort_flag, false);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t id_s1 = idesc_bf16(kRows, N, false, false);
      const uint32_t id_s2 = idesc_bf16(kRows, N, true, true);
      const uint32_t rb = smem_u32(rbuf);
      int64_t j = 0;
      for (int64_t k = 0; k < nphase && !*abort_flag; ++k) {
        bool s2;
        const int64_t u = phase(k, &s2);
        if (!s2) {
          if (u >= 1 && !wait_bounded(zfree, uint32_t((u - 1) & 1), A.spin_limit, abort_flag, false)) {
            fail(ERR_TIMEOUT_MMA);
            break;
          }
          fence_after_sync();
          for (int kb = 0; kb < NKB; ++kb, ++j) {
            const int st = int(j % NST);
            if (!wait_bounded(&full[st], uint32_t((j / NST) & 1), A.spin_limit, abort_flag, false)) {
              fail(ERR_TIMEOUT_STAGE);
              break;
            }
            fence_after_sync();
            const uint32_t xa = smem_u32(ring + size_t(st) * A.stage_bytes);
            const uint32_t ba = xa + kBoxBytes;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
              const uint64_t ad = smem_desc(xa + 32u * s, 16u, 1024u, 2u);
              const uint64_t bd = smem_desc(ba + 32u * s, 16u, 1024u, 2u);
              mma_bf16(tmem, ad, bd, id_s1, (kb > 0 || s > 0) ? 1u : 0u);
            }
            mma_commit(&empty[st]);
          }
          if (*abort_flag) break;
          mma_commit(zdone);
        } else {
          if (!wait_bounded(rfull, uint32_t(u & 1), A.spin_limit, abort_flag, false)) {
            fail(ERR_TIMEOUT_STAGE);
            break;
          }
          fence_after_sync();
          for (int mb = 0; mb < A.MB; ++mb, ++j) {
            const int st = int(j % NST);
            if (!wait_bounded(&full[st], uint32_t((j / NST) & 1), A.spin_limit, abort_flag, false)) {
              fail(ERR_TIMEOUT_STAGE);
              break;
            }
            fence_after_sync();
            const uint32_t xa = smem_u32(ring + size_t(st) * A.stage_bytes);
            const uint32_t dcol = tmem + uint32_t(N + mb * N);
#pragma unroll
            for (int s = 0; s < 8; ++s) {
              const uint64_t ad = smem_desc(xa + 2048u * s, uint32_t(kBoxBytes), 1024u, 2u);
              const uint64_t bd = smem_desc(rb + 2048u * s, uint32_t(kBoxBytes), 1024u, 2u);
              mma_bf16(dcol, ad, bd, id_s2, (u > 0 || s > 0) ? 1u : 0u);
            }
            mma_commit(&empty[st]);
          }
          if (*abort_flag) break;
          mma_commit(rfree);
        }
      }
      mma_commit(gdone);
      mma_commit(drain);
      (void)wait_bounded(drain, 0u, A.spin_limit, abort_flag, false);
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 2-5)
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int row = 32 * q + lane;          // tile row (sweep-1 accumulator lane)
    const uint32_t tq = tmem + (uint32_t(32 * q) << 16);
    const int ew = warp - 2;
    const int Km1 = A.Km1, chains = A.chains;
    for (int64_t u = 0; u < T && !*abort_flag; ++u) {
      const int slot = int(u & 1);
      const int64_t row0 = (cl + u * nclu) * kRows;
      bool ok = wait_bounded(zdone, uint32_t(u & 1), A.spin_limit, abort_flag, false);
      if (!ok) {
        fail(ERR_TIMEOUT_MMA);
        break;
      }
      fence_after_sync();
      float* zrow = A.zg + ((size_t(cl) * 2 + slot) * S + rank) * kRows * size_t(N) + size_t(row) * N;
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tmem_ld16(tq + uint32_t(c0), v);
#pragma unroll
        for (int e = 0; e < 16; e += 4) *reinterpret_cast<float4*>(zrow + c0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive_local(zfree);
      __threadfence();
      named_bar_epi();
      if (ew == 0 && lane < S) mbar_arrive_remote(map_peer(smem_u32(&zrdy[slot]), uint32_t(lane)));
      ok = wait_bounded(&zrdy[slot], uint32_t((u >> 1) & 1), A.spin_limit, abort_flag, true);
      if (!ok) {
        fail(ERR_TIMEOUT_EXCHANGE);
        break;
      }
      // Owned rows: sum the S partials in rank order, softmax, residual, log-lik.
      const float* zs = A.zg + (size_t(cl) * 2 + slot) * S * kRows * size_t(N);
      __nv_bfloat16* rs = A.rg + (size_t(cl) * 2 + slot) * kRows * size_t(A.NP);
      for (int it = ew; it < items; it += 4) {
        const int il = it / chains, c = it - il * chains;
        const int r = int(rank) * RS + il;
        const int64_t grow = row0 + r;
        const bool valid = grow < A.n;
        const int cb = c * Km1;
        float z = 0.f;
        if (lane < Km1)
          for (int pr = 0; pr < S; ++pr) z += __ldcg(zs + (size_t(pr) * kRows + r) * N + cb + lane);
        float mx = (lane < Km1) ? fmaxf(z, 0.f) : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float e = (lane < Km1) ? expf(z - mx) : 0.f;
        float se = e;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
        se += expf(-mx);
        const int yi = valid ? __ldg(A.y + grow) : 0;
        const float zy = __shfl_sync(0xffffffffu, z, yi < Km1 ? yi : 0);
        if (lane < Km1)
          rs[size_t(r) * A.NP + cb + lane] = __float2bfloat16_rn(valid ? ((lane == yi ? 1.f : 0.f) - e / se) : 0.f);
        if (lane == 0 && valid) lacc[it] += double((yi < Km1 ? zy : 0.f) - mx - logf(se));
      }
      __threadfence();
      fence_proxy_async_global();
      named_bar_epi();
      if (ew == 0 && lane < S) mbar_arrive_remote(map_peer(smem_u32(&rrdy[slot]), uint32_t(lane)));
    }
    // Drain the gradient accumulators of this CTA's column slice.
    bool gok = false;
    if (T > 0 && !*abort_flag) {
      gok = wait_bounded(gdone, 0u, A.spin_limit, abort_flag, false);
      if (!gok) fail(ERR_TIMEOUT_MMA);
    }
    if (gok && !*abort_flag) {
      fence_after_sync();
      float* gp = A.gpart + size_t(cl) * A.gpart_cstride;
      for (int mb = 0; mb < A.MB; ++mb) {
        const int col = int(rank) * A.PC + mb * 128 + row;
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tmem_ld16(tq + uint32_t(N + mb * N + c0), v);
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (c0 + e < A.C) gp[size_t(c0 + e) * A.p_pad + col] = v[e];
        }
      }
    } else {
      float* gp = A.gpart + size_t(cl) * A.gpart_cstride;
      for (int mb = 0; mb < A.MB; ++mb) {
        const int col = int(rank) * A.PC + mb * 128 + row;
        for (int c = 0; c < A.C; ++c) gp[size_t(c) * A.p_pad + col] = 0.f;
      }
    }
    fence_before_sync();
    named_bar_epi();
    if (ew == 0)
      for (int c = lane; c < chains; c += 32) {
        double s = 0.0;
        for (int il = 0; il < RS; ++il) s += lacc[il * chains + c];
        A.lpart[(size_t(cl) * S + rank) * A.lpart_cstride + c] = s;
      }
  }
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    tmem_dealloc(tmem, A.tmem_cols);
  }
  if (S > 1) cluster_sync_all();
}

// FP32 coefficients [C][p_pad] -> BF16 B operand [N][p_pad] (rows >= C stay zero).
__global__ void beta_to_bf16_kernel(const float* beta, __nv_bfloat16* out, int C, int p_pad) {
  const int64_t total = int64_t(C) * p_pad;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = __float2bfloat16_rn(beta[i]);
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map_bf16(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                   uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc

// Plan: N = C rounded to 16, MB = PC / 128, TMEM = N * (1 + MB) <= 512.
bool tc_plan(int64_t p, int C, int S, TcPlan* out) {
  const int N = std::max(16, (C + 15) / 16 * 16);
  if (N > 256) return false;
  const int PC = int((p + int64_t(128) * S - 1) / (int64_t(128) * S) * 128);
  const int MB = PC / 128;
  const int cols = N * (1 + MB);
  if (cols > 512) return false;
  uint32_t tcols = 32;
  while (tcols < uint32_t(cols)) tcols <<= 1;
  out->N = N;
  out->NP = (N + 63) / 64 * 64;
  out->PC = PC;
  out->MB = MB;
  out->S = S;
  out->tmem_cols = tcols;
  out->stage_bytes = uint32_t(tc::al(size_t(tc::kBoxBytes) + std::max<size_t>(tc::kBoxBytes, size_t(N) * 128), 1024));
  return true;
}

size_t tc_smem_bytes(const TcPlan& pl, int NST, int chains) {
  return tc::smem_layout(NST, pl.stage_bytes, pl.NP, (128 / pl.S) * chains).total;
}

cudaError_t tc_prepare(size_t smem, int S) {
  cudaError_t e = cudaFuncSetAttribute(tc::lpg_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  if (S > 8) e = cudaFuncSetAttribute(tc::lpg_tc_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t tc_max_active_clusters(size_t smem, int S, int* out) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(S, 1, 1);
  cfg.blockDim = dim3(tc::kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(out, tc::lpg_tc_kernel, &cfg);
}

bool tc_make_maps(const TcPlan& pl, const void* X, int64_t n, int32_t p_pad, const void* bbf, const void* rg,
                  int nclusters, TcMaps* maps) {
  static_assert(sizeof(TcMaps) >= 3 * sizeof(CUtensorMap), "map storage");
  CUtensorMap* m = reinterpret_cast<CUtensorMap*>(maps->bytes);
  if (!tc::make_map_bf16(&m[0], X, uint64_t(p_pad), uint64_t(std::max<int64_t>(n, 1)), tc::kBox, tc::kRows)) return false;
  if (!tc::make_map_bf16(&m[1], bbf, uint64_t(p_pad), uint64_t(pl.N), tc::kBox, uint32_t(pl.N))) return false;
  if (!tc::make_map_bf16(&m[2], rg, uint64_t(pl.NP), uint64_t(nclusters) * 2 * tc::kRows, tc::kBox, tc::kRows))
    return false;
  return true;
}

cudaError_t tc_beta_to_bf16(const float* beta, void* out, int C, int p_pad, cudaStream_t s) {
  const int64_t total = int64_t(C) * p_pad;
  int g = int(std::min<int64_t>(4096, (total + 255) / 256));
  if (g < 1) g = 1;
  tc::beta_to_bf16_kernel<<<g, 256, 0, s>>>(beta, static_cast<__nv_bfloat16*>(out), C, p_pad);
  return cudaGetLastError();
}

cudaError_t tc_launch(const TcPlan& pl, const TcMaps& maps, const TcLaunch& L, size_t smem, cudaStream_t stream) {
  const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(maps.bytes);
  tc::TcArgs a{};
  a.n = L.n;
  a.p_pad = L.p_pad;
  a.PC = pl.PC;
  a.S = pl.S;
  a.N = pl.N;
  a.NP = pl.NP;
  a.C = L.C;
  a.Km1 = L.Km1;
  a.chains = L.chains;
  a.MB = pl.MB;
  a.NST = L.NST;
  a.nclusters = L.nclusters;
  a.ntiles = (L.n + tc::kRows - 1) / tc::kRows;
  a.tmem_cols = pl.tmem_cols;
  a.stage_bytes = pl.stage_bytes;
  a.gpart = static_cast<float*>(L.gpart);
  a.gpart_cstride = L.gpart_cstride;
  a.lpart = L.lpart;
  a.lpart_cstride = L.lpart_cstride;
  a.zg = static_cast<float*>(L.zg);
  a.rg = static_cast<__nv_bfloat16*>(L.rg);
  a.y = L.y;
  a.err = L.err;
  a.spin_limit = L.spin_limit;
  a.inject_timeout = L.inject_timeout;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(L.nclusters * pl.S, 1, 1);
  cfg.blockDim = dim3(tc::kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pl.S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc::lpg_tc_kernel, m[0], m[1], m[2], a);
}

}  // namespace hmc
