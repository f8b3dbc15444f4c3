// Fused log-posterior + gradient pass on CUDA cores (Eqs. softmax, loglike,
// logkernel and gradient of Sec. 2.1).  One launch evaluates, for `chains`
// coefficient states at once (C = chains*(K-1) columns),
//   * the per-cluster partial log-likelihood  sum_i log psi_{i,y_i}, and
//   * the per-cluster partial gradient        X^T (Y - psi(XB))
// reading every element of X from HBM once.
//
// Work decomposition (GB300): a thread-block cluster of S CTAs owns a row
// tile of BM rows; CTA `rank` holds the column slice [rank*PC, (rank+1)*PC)
// of those rows in shared memory (bulk-async copies, NSTAGE-deep pipeline)
// and the matching slice of the coefficients.  Per tile:
//   1. logit phase: lane <-> row, warps split the slice's columns; each lane
//      accumulates the C partial logits of its row (coefficients broadcast
//      from shared memory); a fixed-order cross-warp sum gives the CTA's
//      partial logits.
//   2. exchange: every CTA pushes its partial logits into every peer's
//      shared memory (st.async completing on the peer's mbarrier); every CTA
//      then sums the S partials in rank order, so all CTAs hold identical
//      logits.
//   3. softmax with the fixed zero logit of class K (max-shifted), residual
//      R = Y - P and the row log-likelihood z_{y_i} - logsumexp_i.
//   4. gradient phase: thread <-> 4 columns, partial X^T R accumulated in
//      registers across all tiles of the cluster (no atomics).
// At the end each CTA writes its slice of the cluster's partial gradient.
#pragma once
#include "device_common.cuh"
#include "internal.h"

namespace hmc {
namespace simt {

constexpr int kMaxThreads = kSimtMaxThreads;

template <typename XT>
struct Vec;
template <>
struct Vec<double> {
  static constexpr int N = 2;
};
template <>
struct Vec<float> {
  static constexpr int N = 4;
};
template <>
struct Vec<__nv_bfloat16> {
  static constexpr int N = 8;
};
template <>
struct Vec<__nv_fp8_e4m3> {
  static constexpr int N = 16;
};

__device__ __forceinline__ float bf16lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

__device__ __forceinline__ void fp8x2(uint32_t two, float& a, float& b) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(two & 0xffffu), __NV_E4M3);
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&h));
  a = f.x;
  b = f.y;
}

// 16 bytes of X (shared memory, 16-byte aligned) -> Vec<XT>::N values.
template <typename XT, typename AT>
__device__ __forceinline__ void load16(const unsigned char* p, AT* o);

template <>
__device__ __forceinline__ void load16<double, double>(const unsigned char* p, double* o) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  o[0] = v.x;
  o[1] = v.y;
}
template <>
__device__ __forceinline__ void load16<float, float>(const unsigned char* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
template <>
__device__ __forceinline__ void load16<__nv_bfloat16, float>(const unsigned char* p, float* o) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  o[0] = bf16lo(v.x); o[1] = bf16hi(v.x);
  o[2] = bf16lo(v.y); o[3] = bf16hi(v.y);
  o[4] = bf16lo(v.z); o[5] = bf16hi(v.z);
  o[6] = bf16lo(v.w); o[7] = bf16hi(v.w);
}
template <>
__device__ __forceinline__ void load16<__nv_fp8_e4m3, float>(const unsigned char* p, float* o) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    fp8x2(w[q], o[4 * q + 0], o[4 * q + 1]);
    fp8x2(w[q] >> 16, o[4 * q + 2], o[4 * q + 3]);
  }
}

// 4 consecutive elements of X (aligned to 4 elements).
template <typename XT, typename AT>
__device__ __forceinline__ void load4(const unsigned char* p, AT* o);

template <>
__device__ __forceinline__ void load4<double, double>(const unsigned char* p, double* o) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 16);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
template <>
__device__ __forceinline__ void load4<float, float>(const unsigned char* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void load4<__nv_bfloat16, float>(const unsigned char* p, float* o) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  o[0] = bf16lo(v.x); o[1] = bf16hi(v.x); o[2] = bf16lo(v.y); o[3] = bf16hi(v.y);
}
template <>
__device__ __forceinline__ void load4<__nv_fp8_e4m3, float>(const unsigned char* p, float* o) {
  const uint32_t v = *reinterpret_cast<const uint32_t*>(p);
  fp8x2(v, o[0], o[1]);
  fp8x2(v >> 16, o[2], o[3]);
}

// N consecutive coefficient values from shared memory (16-byte aligned).
template <typename AT, int N>
__device__ __forceinline__ void load_coef(const AT* p, AT* o) {
  if constexpr (sizeof(AT) == 4) {
#pragma unroll
    for (int q = 0; q < N; q += 4) {
      const float4 v = *reinterpret_cast<const float4*>(p + q);
      o[q] = v.x; o[q + 1] = v.y; o[q + 2] = v.z; o[q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < N; q += 2) {
      const double2 v = *reinterpret_cast<const double2*>(p + q);
      o[q] = v.x; o[q + 1] = v.y;
    }
  }
}

template <typename AT>
__device__ __forceinline__ AT ex(AT x);
template <>
__device__ __forceinline__ float ex<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double ex<double>(double x) { return exp(x); }
template <typename AT>
__device__ __forceinline__ AT lg(AT x);
template <>
__device__ __forceinline__ float lg<float>(float x) { return logf(x); }
template <>
__device__ __forceinline__ double lg<double>(double x) { return log(x); }

// Width of one exchanged logit row: a whole number of 16-byte vectors.
template <typename AT, int CT>
struct Ex {
  static constexpr int PV = 16 / sizeof(AT);
  static constexpr int CTP = ((CT + PV - 1) / PV) * PV;
};

// Shared-memory layout; the host computes the same size with smem_bytes().
struct Layout {
  size_t xs, bs, red, zx, rs, lrow, bars, total;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline Layout layout(int xbytes, int abytes, int CT, int CTP, int PC, int BM, int S, int NT,
                                         int NSTAGE) {
  Layout L;
  const size_t xpitch = size_t(PC) * xbytes + 16;
  size_t off = 0;
  L.xs = off;   off = align16(off + size_t(NSTAGE) * BM * xpitch);
  L.bs = off;   off = align16(off + size_t(CT) * PC * abytes);
  L.red = off;  off = align16(off + size_t(NT / 32) * BM * CT * abytes);
  L.zx = off;   off = align16(off + size_t(2) * S * BM * CTP * abytes);
  L.rs = off;   off = align16(off + size_t(BM) * CTP * abytes);
  L.lrow = off; off = align16(off + size_t(BM) * CT * 8);
  L.bars = off; off = align16(off + size_t(NSTAGE + 5) * 8);
  L.total = off;
  return L;
}

template <typename XT, typename AT, int CT>
__global__ void __launch_bounds__(kMaxThreads, 1) lpg_kernel(const LpgArgs A) {
  constexpr int VEC = Vec<XT>::N;
  constexpr int PV = Ex<AT, CT>::PV;
  constexpr int CTP = Ex<AT, CT>::CTP;
  extern __shared__ __align__(128) unsigned char smem[];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NT = A.NT, NW = NT >> 5;
  const int S = A.S, BM = A.BM, PC = A.PC, NSTAGE = A.NSTAGE;
  const uint32_t rank = (S > 1) ? cluster_rank() : 0u;
  const int cl = blockIdx.x / S;
  const size_t xpitch = size_t(PC) * sizeof(XT) + 16;
  const Layout Lo = layout(sizeof(XT), sizeof(AT), CT, CTP, PC, BM, S, NT, NSTAGE);
  unsigned char* xs = smem + Lo.xs;
  AT* bs = reinterpret_cast<AT*>(smem + Lo.bs);
  AT* red = reinterpret_cast<AT*>(smem + Lo.red);
  AT* zx = reinterpret_cast<AT*>(smem + Lo.zx);
  AT* rs = reinterpret_cast<AT*>(smem + Lo.rs);
  double* lrow = reinterpret_cast<double*>(smem + Lo.lrow);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lo.bars);
  uint64_t* zfull = full + NSTAGE;
  uint64_t* zempty = zfull + 2;
  uint64_t* never = zempty + 2;  // fault injection: a barrier no thread arrives at

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(&full[s], 1);
    mbar_init(&zfull[0], 1);
    mbar_init(&zfull[1], 1);
    mbar_init(&zempty[0], S);
    mbar_init(&zempty[1], S);
    mbar_init(never, 1);
    fence_mbar_init_cluster();
  }
  // Coefficient slice, FP8 column scales folded in: X B = X_q diag(s) B.
  {
    const AT* beta = static_cast<const AT*>(A.beta);
    for (int idx = tid; idx < CT * PC; idx += NT) {
      const int k = idx / PC, j = idx - k * PC;
      const int col = int(rank) * PC + j;
      AT v = AT(0);
      if (k < A.C) {
        v = beta[size_t(k) * A.p_pad + col];
        if (A.xscale) v *= AT(A.xscale[col]);
      }
      bs[idx] = v;
    }
    for (int idx = tid; idx < BM * CTP; idx += NT) rs[idx] = AT(0);
  }
  if (S > 1)
    cluster_sync_all();
  else
    __syncthreads();

  const int64_t nclu = A.nclusters;
  const int64_t my_tiles = (cl < A.ntiles) ? (A.ntiles - 1 - cl) / nclu + 1 : 0;
  const uint32_t row_bytes = uint32_t(PC) * sizeof(XT);

  auto issue = [&](int64_t t) {  // warp 0 only
    const int s = int(t % NSTAGE);
    const int64_t row0 = (cl + t * nclu) * BM;
    const int rv = int(min(int64_t(BM), A.n - row0));
    if (lane == 0) mbar_arrive_expect_tx(&full[s], row_bytes * uint32_t(rv));
    __syncwarp();
    const XT* src = static_cast<const XT*>(A.X) + size_t(row0) * A.p_pad + size_t(rank) * PC;
    for (int i = lane; i < rv; i += 32)
      bulk_g2s(xs + (size_t(s) * BM + i) * xpitch, src + size_t(i) * A.p_pad, row_bytes, &full[s]);
  };

  AT G[4][CT];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < CT; ++k) G[q][k] = AT(0);
  double lacc = 0.0;
  int err = 0;
  int64_t issued = 0;

  if (A.inject_timeout) {
    const bool ok = mbar_wait_cta(never, 0u, A.spin_limit);
    if (__syncthreads_or(!ok)) err |= ERR_TIMEOUT_STAGE;
  }
  const int64_t run_tiles = err ? 0 : my_tiles;

  if (warp == 0) {
    for (int64_t t = 0; t < min(int64_t(NSTAGE - 1), run_tiles); ++t) issue(t);
  }
  issued = min(int64_t(NSTAGE - 1), run_tiles);

  int64_t t = 0;
  for (; t < run_tiles; ++t) {
    if (t + NSTAGE - 1 < run_tiles) {
      if (warp == 0) issue(t + NSTAGE - 1);
      issued = t + NSTAGE;
    }
    const int s = int(t % NSTAGE);
    const int64_t row0 = (cl + t * nclu) * BM;
    const int rv = int(min(int64_t(BM), A.n - row0));
    {
      const bool ok = mbar_wait_cta(&full[s], uint32_t((t / NSTAGE) & 1), A.spin_limit);
      if (__syncthreads_or(!ok)) {
        err |= ERR_TIMEOUT_STAGE;
        break;
      }
    }
    const unsigned char* xst = xs + size_t(s) * BM * xpitch;

    // 1. partial logits of this CTA's column slice.
    {
      const int LPR = 32 / BM;
      const int i = lane % BM, sub = lane / BM;
      const int G16 = PC / VEC;
      const int gpw = (G16 + NW - 1) / NW;
      const int gbeg = warp * gpw, gend = min(G16, gbeg + gpw);
      AT z[CT];
#pragma unroll
      for (int k = 0; k < CT; ++k) z[k] = AT(0);
      const unsigned char* xrow = xst + size_t(i) * xpitch;
      for (int g = gbeg + sub; g < gend; g += LPR) {
        AT xv[VEC];
        load16<XT, AT>(xrow + size_t(g) * 16, xv);
#pragma unroll
        for (int k = 0; k < CT; ++k) {
          AT bv[VEC];
          load_coef<AT, VEC>(bs + size_t(k) * PC + size_t(g) * VEC, bv);
          AT acc = z[k];
#pragma unroll
          for (int q = 0; q < VEC; ++q) acc = fma(xv[q], bv[q], acc);
          z[k] = acc;
        }
      }
      for (int o = BM; o < 32; o <<= 1)
#pragma unroll
        for (int k = 0; k < CT; ++k) z[k] += __shfl_xor_sync(0xffffffffu, z[k], o);
      if (sub == 0)
#pragma unroll
        for (int k = 0; k < CT; ++k) red[(size_t(warp) * BM + i) * CT + k] = z[k];
    }
    __syncthreads();

    // 2. exchange the partial logits across the cluster.
    const int xsl = int(t & 1);
    const uint32_t use = uint32_t(t >> 1);
    AT* zslot = zx + size_t(xsl) * S * BM * CTP;
    if (S > 1) {
      if (tid == 0) mbar_arrive_expect_tx(&zfull[xsl], uint32_t(S * BM * CTP * sizeof(AT)));
      const bool ok = mbar_wait_cluster(&zempty[xsl], (use & 1u) ^ 1u, A.spin_limit);
      if (__syncthreads_or(!ok)) {
        err |= ERR_TIMEOUT_SLOT;
        break;
      }
    }
    {
      const int nv = CTP / PV;
      for (int it = tid; it < BM * nv; it += NT) {
        const int i = it / nv, kv = (it - i * nv) * PV;
        AT v[PV];
#pragma unroll
        for (int q = 0; q < PV; ++q) {
          const int k = kv + q;
          AT sum = AT(0);
          if (k < CT)
            for (int w = 0; w < NW; ++w) sum += red[(size_t(w) * BM + i) * CT + k];
          v[q] = sum;
        }
        AT* dst = zslot + (size_t(rank) * BM + i) * CTP + kv;
        if (S == 1) {
#pragma unroll
          for (int q = 0; q < PV; ++q) dst[q] = v[q];
        } else {
          const uint32_t laddr = smem_u32(dst), lbar = smem_u32(&zfull[xsl]);
          for (int r = 0; r < S; ++r) {
            const uint32_t ra = map_peer(laddr, uint32_t(r)), rb = map_peer(lbar, uint32_t(r));
            if constexpr (sizeof(AT) == 4)
              st_async_v4f(ra, float(v[0]), float(v[1]), float(v[2]), float(v[3]), rb);
            else
              st_async_v2d(ra, double(v[0]), double(v[1]), rb);
          }
        }
      }
    }
    if (S > 1) {
      const bool ok = mbar_wait_cluster(&zfull[xsl], use & 1u, A.spin_limit);
      if (__syncthreads_or(!ok)) {
        err |= ERR_TIMEOUT_EXCHANGE;
        break;
      }
    } else {
      __syncthreads();
    }

    // 3. softmax with the zero logit of class K, residual, log-likelihood.
    {
      const int Km1 = A.Km1, chains = A.chains;
      for (int it = tid; it < BM * chains; it += NT) {
        const int i = it / chains, c = it - i * chains;
        const int cb = c * Km1;
        if (i >= rv) {
          lrow[size_t(i) * CT + c] = 0.0;
#pragma unroll
          for (int k = 0; k < CT; ++k)
            if (k < Km1) rs[size_t(i) * CTP + cb + k] = AT(0);
          continue;
        }
        const int yi = __ldg(A.y + row0 + i);
        AT z[CT];
        AT m = AT(0);
        AT zy = AT(0);
#pragma unroll
        for (int k = 0; k < CT; ++k) {
          if (k < Km1) {
            AT sum = AT(0);
            for (int r = 0; r < S; ++r) sum += zslot[(size_t(r) * BM + i) * CTP + cb + k];
            z[k] = sum;
            m = max(m, sum);
            if (k == yi) zy = sum;
          }
        }
        AT se = ex<AT>(-m);
#pragma unroll
        for (int k = 0; k < CT; ++k)
          if (k < Km1) {
            z[k] = ex<AT>(z[k] - m);
            se += z[k];
          }
        const AT inv = AT(1) / se;
#pragma unroll
        for (int k = 0; k < CT; ++k)
          if (k < Km1) rs[size_t(i) * CTP + cb + k] = (k == yi ? AT(1) : AT(0)) - z[k] * inv;
        lrow[size_t(i) * CT + c] = double(zy - m - lg<AT>(se));
      }
    }
    __syncthreads();
    if (S > 1 && tid < S) mbar_arrive_remote(map_peer(smem_u32(&zempty[xsl]), uint32_t(tid)));
    if (rank == 0 && tid < A.chains) {
      double sl = 0.0;
      for (int i = 0; i < rv; ++i) sl += lrow[size_t(i) * CT + tid];
      lacc += sl;
    }

    // 4. partial X^T R for this thread's 4 columns.
    if (4 * tid < PC) {
      const unsigned char* xcol = xst + size_t(4) * tid * sizeof(XT);
      for (int i = 0; i < rv; ++i) {
        AT r[CTP];
        load_coef<AT, CTP>(rs + size_t(i) * CTP, r);
        AT xv[4];
        load4<XT, AT>(xcol + size_t(i) * xpitch, xv);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int k = 0; k < CT; ++k) G[q][k] = fma(xv[q], r[k], G[q][k]);
      }
    }
    __syncthreads();
  }

  if (err) {
    // Let every copy this CTA issued land before its shared memory goes away.
    if (tid == 0) {
      for (int64_t tt = t; tt < issued; ++tt)
        (void)mbar_wait_cta(&full[tt % NSTAGE], uint32_t((tt / NSTAGE) & 1), A.spin_limit);
      atomicOr(A.err, err);
    }
  }
  if (4 * tid < PC) {
    AT* gp = static_cast<AT*>(A.gpart) + size_t(cl) * A.gpart_cstride;
    const int col = int(rank) * PC + 4 * tid;
    AT sc[4] = {AT(1), AT(1), AT(1), AT(1)};
    if (A.xscale)
#pragma unroll
      for (int q = 0; q < 4; ++q) sc[q] = AT(A.xscale[col + q]);
#pragma unroll
    for (int k = 0; k < CT; ++k) {
      if (k < A.C) {
        AT* d = gp + size_t(k) * A.p_pad + col;
        if constexpr (sizeof(AT) == 4) {
          *reinterpret_cast<float4*>(d) =
              make_float4(float(G[0][k] * sc[0]), float(G[1][k] * sc[1]), float(G[2][k] * sc[2]), float(G[3][k] * sc[3]));
        } else {
          reinterpret_cast<double2*>(d)[0] = make_double2(double(G[0][k] * sc[0]), double(G[1][k] * sc[1]));
          reinterpret_cast<double2*>(d)[1] = make_double2(double(G[2][k] * sc[2]), double(G[3][k] * sc[3]));
        }
      }
    }
  }
  if (rank == 0 && tid < A.chains) A.lpart[size_t(cl) * A.lpart_cstride + tid] = lacc;
  if (S > 1) cluster_sync_all();
}

}  // namespace simt
}  // namespace hmc
