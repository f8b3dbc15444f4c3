// Fused log-posterior + gradient pass on CUDA cores (Eqs. softmax, loglike,
// logkernel and gradient of Sec. 2.1).  One launch evaluates, for `chains`
// coefficient states at once (C = chains*(K-1) columns),
//   * the per-cluster partial log-likelihood  sum_i log psi_{i,y_i}, and
//   * the per-cluster partial gradient        X^T (Y - psi(XB))
// reading every element of X from HBM once.
//
// Work decomposition (GB300): a thread-block cluster of S CTAs walks
// super-tiles of BM rows; CTA `rank` owns the column slice
// [rank*PC, (rank+1)*PC) of X and of the coefficients.  X reaches shared
// memory through a ring of NSTAGE chunk buffers (CR rows x PC columns each,
// bulk-async copies completing on mbarriers).  Each super-tile is swept twice:
//   sweep 1 (logits): lane <-> row of the chunk, warps split the slice's
//      columns, coefficients broadcast from shared memory; after the last
//      chunk a fixed-order cross-warp sum gives the CTA's partial logits,
//      which are pushed into every peer's exchange slot (st.async completing
//      on the peer's mbarrier);
//   sweep 2 (gradient): every CTA sums the S partials in rank order (so all
//      CTAs hold identical logits), forms the softmax with the fixed zero
//      logit of class K, the residual R = Y - P and the row log-likelihood,
//      then re-reads the super-tile's chunks (an L2 hit: they were streamed a
//      moment earlier) and accumulates X^T R in registers (thread <-> 4
//      columns), across all super-tiles of the cluster, without atomics.
// Sweeps are interleaved S1(0), S1(1), S2(0), S1(2), S2(1), ... so the
// exchange of one super-tile completes while the next one's logits are formed.
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

// (a0, a1) += x * (r0, r1) with one packed FP32x2 FMA (each lane rounded once,
// exactly as two scalar FMAs).
__device__ __forceinline__ void fma2(float& a0, float& a1, float x, float r0, float r1) {
  unsigned long long acc, xx, rr;
  asm("mov.b64 %0, {%1, %2};" : "=l"(acc) : "f"(a0), "f"(a1));
  asm("mov.b64 %0, {%1, %1};" : "=l"(xx) : "f"(x));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rr) : "f"(r0), "f"(r1));
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(xx), "l"(rr));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(acc));
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

// Coefficients in shared memory, group-major: for column group g (VEC
// columns) the CT x VEC values are contiguous, padded to an odd number of
// 16-byte units so that the groups read together by one warp fall in
// different banks.
template <typename AT, int CT, int VEC>
struct Coef {
  static constexpr int RAW = CT * VEC;                         // values per group
  static constexpr int UNITS = (RAW * int(sizeof(AT)) + 15) / 16;
  static constexpr int STRIDE = ((UNITS % 2) ? UNITS : UNITS + 1) * 16 / int(sizeof(AT));
};

// Width of one exchanged logit row: a whole number of 16-byte vectors.
template <typename AT, int CT>
struct Ex {
  static constexpr int PV = 16 / sizeof(AT);
  static constexpr int CTP = ((CT + PV - 1) / PV) * PV;
};

// Shared-memory layout; the host computes the same size with smem_bytes().
struct Layout {
  size_t xs, bs, red, zx, rs, lrow, ylab, bars, total;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline Layout layout(int xbytes, int abytes, int CT, int CTP, int PC, int BM, int S, int NT,
                                         int NSTAGE, int CR, int coef_stride) {
  Layout L;
  const size_t xpitch = size_t(PC) * xbytes + 16;
  size_t off = 0;
  L.xs = off;   off = align16(off + size_t(NSTAGE) * CR * xpitch);
  L.bs = off;   off = align16(off + size_t(PC / (16 / xbytes)) * coef_stride * abytes);
  L.red = off;  off = align16(off + size_t(NT / 32) * BM * CT * abytes);
  L.zx = off;   off = align16(off + size_t(2) * S * BM * CTP * abytes);
  L.rs = off;   off = align16(off + size_t(BM) * CTP * abytes);
  L.lrow = off; off = align16(off + size_t(BM) * CT * 8);
  L.ylab = off; off = align16(off + size_t(BM) * 4);
  L.bars = off; off = align16(off + size_t(NSTAGE + 5) * 8);
  L.total = off;
  return L;
}

template <typename XT, typename AT, int CT>
__device__ __forceinline__ void lpg_body(const LpgArgs& A, const int cl) {
  constexpr int VEC = Vec<XT>::N;
  constexpr int PV = Ex<AT, CT>::PV;
  constexpr int CTP = Ex<AT, CT>::CTP;
  extern __shared__ __align__(128) unsigned char smem[];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NT = A.NT, NW = NT >> 5;
  const int S = A.S, BM = A.BM, PC = A.PC, NSTAGE = A.NSTAGE, CR = A.CR;
  const uint32_t rank = (S > 1) ? cluster_rank() : 0u;
  const size_t xpitch = size_t(PC) * sizeof(XT) + 16;
  constexpr int CSTR = Coef<AT, CT, VEC>::STRIDE;
  const Layout Lo = layout(sizeof(XT), sizeof(AT), CT, CTP, PC, BM, S, NT, NSTAGE, CR, CSTR);
  unsigned char* xs = smem + Lo.xs;
  AT* bs = reinterpret_cast<AT*>(smem + Lo.bs);
  AT* red = reinterpret_cast<AT*>(smem + Lo.red);
  AT* zx = reinterpret_cast<AT*>(smem + Lo.zx);
  AT* rs = reinterpret_cast<AT*>(smem + Lo.rs);
  double* lrow = reinterpret_cast<double*>(smem + Lo.lrow);
  int* ylab = reinterpret_cast<int*>(smem + Lo.ylab);
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
      bs[size_t(j / VEC) * CSTR + k * VEC + (j % VEC)] = v;
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
  auto row0_of = [&](int64_t u) { return (cl + u * nclu) * BM; };
  auto rows_of = [&](int64_t u) { return int(min(int64_t(BM), A.n - row0_of(u))); };
  auto nch_of = [&](int64_t u) { return (rows_of(u) + CR - 1) / CR; };

  AT G[4][CT];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < CT; ++k) G[q][k] = AT(0);
  double lacc = 0.0;
  int err = 0;

  if (A.inject_timeout) {
    const bool ok = mbar_wait_cta(never, 0u, A.spin_limit);
    if (__syncthreads_or(!ok)) err |= ERR_TIMEOUT_STAGE;
  }
  const int64_t T = err ? 0 : my_tiles;
  const int64_t nphase = 2 * T;
  // Phase k of the sweep order S1(0), S1(1), S2(0), S1(2), S2(1), ..., S2(T-1):
  // returns the super-tile, sets *s2 for a gradient sweep.
  auto phase = [&](int64_t k, bool* s2) -> int64_t {
    if (k == 0) { *s2 = false; return 0; }
    if (k == nphase - 1) { *s2 = true; return T - 1; }
    const int64_t v = (k + 1) / 2;
    *s2 = (k % 2) == 0;
    return *s2 ? v - 1 : v;
  };

  // Producer cursor (identical in every thread; warp 0 issues).
  int64_t pk = 0, issued = 0, xwaited = 0;
  int pc = 0;
  auto issue_next = [&]() {
    if (pk >= nphase) return;
    bool s2;
    const int64_t u = phase(pk, &s2);
    const int64_t row0 = row0_of(u) + int64_t(pc) * CR;
    const int rv = min(CR, rows_of(u) - pc * CR);
    const int slot = int(issued % NSTAGE);
    if (warp == 0) {
      if (lane == 0) mbar_arrive_expect_tx(&full[slot], row_bytes * uint32_t(rv));
      __syncwarp();
      const XT* src = static_cast<const XT*>(A.X) + size_t(row0) * A.p_pad + size_t(rank) * PC;
      for (int i = lane; i < rv; i += 32)
        bulk_g2s(xs + (size_t(slot) * CR + i) * xpitch, src + size_t(i) * A.p_pad, row_bytes, &full[slot]);
    }
    issued += 1;
    if (++pc == nch_of(u)) {
      pc = 0;
      ++pk;
    }
  };
  for (int i = 0; i < NSTAGE; ++i) issue_next();

  int64_t m = 0;        // chunks consumed
  int lab0 = 0, lab1 = 0;  // labels of rows tid and tid + NT of super-tile lab_tile
  int64_t lab_tile = -1;
  auto load_labels = [&](int64_t u) {
    const int r = rows_of(u);
    const int32_t* yp = A.y + row0_of(u);
    lab0 = (tid < r) ? __ldg(yp + tid) : 0;
    lab1 = (tid + NT < r) ? __ldg(yp + tid + NT) : 0;
    lab_tile = u;
  };
  for (int64_t k = 0; k < nphase && !err; ++k) {
    bool s2;
    const int64_t u = phase(k, &s2);
    const int rv = rows_of(u);
    const int nch = (rv + CR - 1) / CR;
    const int xsl = int(u & 1);
    const uint32_t use = uint32_t(u >> 1);
    if (!s2) {
      if (u >= 1) load_labels(u - 1);  // the super-tile whose gradient sweep comes next
    } else {
      if (lab_tile != u) load_labels(u);
      if (tid < BM) ylab[tid] = lab0;
      if (tid + NT < BM) ylab[tid + NT] = lab1;
      const AT* zslot = zx + size_t(xsl) * S * BM * CTP;
      if (S > 1) {
        const bool ok = mbar_wait_cluster(&zfull[xsl], use & 1u, A.spin_limit);
        if (__syncthreads_or(!ok)) {
          err |= ERR_TIMEOUT_EXCHANGE;
          break;
        }
      } else {
        __syncthreads();
      }
      // Softmax with the zero logit of class K, residual and row
      // log-likelihood: one warp per (row, chain), lane <-> class.
      const int Km1 = A.Km1, chains = A.chains;
      for (int it = warp; it < BM * chains; it += NW) {
        const int i = it / chains, c = it - i * chains;
        const int cb = c * Km1;
        AT z = AT(0);
        if (lane < Km1)
          for (int r = 0; r < S; ++r) z += zslot[(size_t(r) * BM + i) * CTP + cb + lane];
        AT mx = (lane < Km1) ? max(z, AT(0)) : AT(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const AT e = (lane < Km1) ? ex<AT>(z - mx) : AT(0);
        AT se = e;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
        se += ex<AT>(-mx);
        const int yi = ylab[i];
        const AT zy = __shfl_sync(0xffffffffu, z, yi < Km1 ? yi : 0);
        const bool valid = i < rv;
        if (lane < Km1) rs[size_t(i) * CTP + cb + lane] = valid ? (lane == yi ? AT(1) : AT(0)) - e / se : AT(0);
        if (lane == 0) lrow[size_t(i) * CT + c] = valid ? double((yi < Km1 ? zy : AT(0)) - mx - lg<AT>(se)) : 0.0;
      }
      __syncthreads();
      if (S > 1 && tid < S) mbar_arrive_remote(map_peer(smem_u32(&zempty[xsl]), uint32_t(tid)));
      if (rank == 0 && tid < A.chains) {
        double sl = 0.0;
        for (int i = 0; i < rv; ++i) sl += lrow[size_t(i) * CT + tid];
        lacc += sl;
      }
    }

    for (int c = 0; c < nch; ++c, ++m) {
      const int slot = int(m % NSTAGE);
      {
        const bool ok = mbar_wait_cta(&full[slot], uint32_t((m / NSTAGE) & 1), A.spin_limit);
        if (__syncthreads_or(!ok)) {
          err |= ERR_TIMEOUT_STAGE;
          break;
        }
      }
      xwaited = m + 1;
      const unsigned char* xst = xs + size_t(slot) * CR * xpitch;
      const int crv = min(CR, rv - c * CR);
      if (!s2) {
        // Sweep 1: partial logits of this chunk's rows.
        const int LPR = 32 / CR;
        const int i = lane % CR, sub = lane / CR;
        const int G16 = PC / VEC;
        const int gpw = (G16 + NW - 1) / NW;
        const int gbeg = warp * gpw, gend = min(G16, gbeg + gpw);
        AT z[CT];
#pragma unroll
        for (int kk = 0; kk < CT; ++kk) z[kk] = AT(0);
        const unsigned char* xrow = xst + size_t(i) * xpitch;
        for (int g = gbeg + sub; g < gend; g += LPR) {
          AT xv[VEC];
          load16<XT, AT>(xrow + size_t(g) * 16, xv);
          const AT* bg = bs + size_t(g) * CSTR;
#pragma unroll
          for (int kk = 0; kk < CT; ++kk) {
            AT bv[VEC];
            load_coef<AT, VEC>(bg + kk * VEC, bv);
            AT acc = z[kk];
#pragma unroll
            for (int q = 0; q < VEC; ++q) acc = fma(xv[q], bv[q], acc);
            z[kk] = acc;
          }
        }
        for (int o = CR; o < 32; o <<= 1)
#pragma unroll
          for (int kk = 0; kk < CT; ++kk) z[kk] += __shfl_xor_sync(0xffffffffu, z[kk], o);
        if (sub == 0)
#pragma unroll
          for (int kk = 0; kk < CT; ++kk) red[(size_t(warp) * BM + c * CR + i) * CT + kk] = z[kk];
      } else if (4 * tid < PC) {
        // Sweep 2: partial X^T R for this thread's 4 columns.
        const unsigned char* xcol = xst + size_t(4) * tid * sizeof(XT);
        const AT* rrow = rs + size_t(c) * CR * CTP;
        for (int i = 0; i < crv; ++i) {
          AT r[CTP];
          load_coef<AT, CTP>(rrow + size_t(i) * CTP, r);
          AT xv[4];
          load4<XT, AT>(xcol + size_t(i) * xpitch, xv);
          if constexpr (sizeof(AT) == 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
#pragma unroll
              for (int kk = 0; kk + 1 < CT; kk += 2) fma2(G[q][kk], G[q][kk + 1], xv[q], r[kk], r[kk + 1]);
              if (CT % 2) G[q][CT - 1] = fma(xv[q], r[CT - 1], G[q][CT - 1]);
            }
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
              for (int kk = 0; kk < CT; ++kk) G[q][kk] = fma(xv[q], r[kk], G[q][kk]);
          }
        }
      }
      __syncthreads();   // ring slot free
      issue_next();
    }
    if (err) break;

    if (!s2) {
      // Partial logits of super-tile u: fixed-order sum over warps, pushed to
      // every peer's slot u&1.
      if (S > 1) {
        if (tid == 0) mbar_arrive_expect_tx(&zfull[xsl], uint32_t(S * BM * CTP * sizeof(AT)));
        const bool ok = mbar_wait_cluster(&zempty[xsl], (use & 1u) ^ 1u, A.spin_limit);
        if (__syncthreads_or(!ok)) {
          err |= ERR_TIMEOUT_SLOT;
          break;
        }
      }
      AT* zslot = zx + size_t(xsl) * S * BM * CTP;
      const int nv = CTP / PV;
      for (int it = tid; it < BM * nv; it += NT) {
        const int i = it / nv, kv = (it - i * nv) * PV;
        AT v[PV];
#pragma unroll
        for (int q = 0; q < PV; ++q) {
          const int kk = kv + q;
          AT sum = AT(0);
          if (kk < CT && i < rv)
            for (int w = 0; w < NW; ++w) sum += red[(size_t(w) * BM + i) * CT + kk];
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
      if (S == 1) __syncthreads();
    }
  }

  if (err) {
    // Let every copy this CTA issued land before its shared memory goes away.
    if (tid == 0) {
      for (int64_t tt = xwaited; tt < issued; ++tt)
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
    for (int kk = 0; kk < CT; ++kk) {
      if (kk < A.C) {
        AT* d = gp + size_t(kk) * A.p_pad + col;
        if constexpr (sizeof(AT) == 4) {
          *reinterpret_cast<float4*>(d) = make_float4(float(G[0][kk] * sc[0]), float(G[1][kk] * sc[1]),
                                                      float(G[2][kk] * sc[2]), float(G[3][kk] * sc[3]));
        } else {
          reinterpret_cast<double2*>(d)[0] = make_double2(double(G[0][kk] * sc[0]), double(G[1][kk] * sc[1]));
          reinterpret_cast<double2*>(d)[1] = make_double2(double(G[2][kk] * sc[2]), double(G[3][kk] * sc[3]));
        }
      }
    }
  }
  if (rank == 0 && tid < A.chains) A.lpart[size_t(cl) * A.lpart_cstride + tid] = lacc;
  if (S > 1) cluster_sync_all();
}

template <typename XT, typename AT, int CT>
__global__ void __launch_bounds__(kMaxThreads, 1) lpg_kernel(const LpgArgs A) {
  lpg_body<XT, AT, CT>(A, int(blockIdx.x) / A.S);
}

// Several independent problems in one launch: clusters [first[b], first[b+1])
// of the grid work on problem b (its own X, labels, coefficients, tiles and
// partial slots); every problem shares the cluster size and block size.
template <typename XT, typename AT, int CT>
__global__ void __launch_bounds__(kMaxThreads, 1)
    lpg_kernel_batched(const LpgArgs* __restrict__ table, const int* __restrict__ first, int nprob, int chains) {
  __shared__ LpgArgs args;
  __shared__ int cl_local;
  if (threadIdx.x == 0) {
    const int S = table[0].S;
    const int gcl = int(blockIdx.x) / S;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {  // last b with first[b] <= gcl
      const int mid = (lo + hi + 1) / 2;
      if (first[mid] <= gcl) lo = mid; else hi = mid - 1;
    }
    args = table[lo];
    args.chains = chains;
    args.C = chains * args.Km1;
    cl_local = gcl - first[lo];
  }
  __syncthreads();
  lpg_body<XT, AT, CT>(args, cl_local);
}

}  // namespace simt
}  // namespace hmc
