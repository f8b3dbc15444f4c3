// Fused log-posterior + gradient pass on CUDA cores (Eqs. softmax, loglike,
// logkernel and gradient of Sec. 2.1).  One launch evaluates, for `chains`
// coefficient states at once (C = chains*(K-1) columns),
//   * the per-cluster partial log-likelihood  sum_i log psi_{i,y_i}, and
//   * the per-cluster partial gradient        X^T (Y - psi(XB))
// reading every element of X from HBM once.
//
// Work decomposition (GB300): a thread-block cluster of S CTAs walks
// super-tiles of BM = kSimtRows rows; CTA `rank` owns the column slice
// [rank*PC, (rank+1)*PC) of X and of the coefficients.  Inside a CTA three
// warp roles run their own loops over the cluster's tiles, handing tiles
// over through mbarriers:
//   producer (1 warp): bulk-async copies of each tile's slice into a ring
//      of NSTAGE shared-memory slots, with bulk L2 prefetches further ahead;
//   logit group (NWL warps): sweep 1 -- lane = (row group a, phase c) holds
//      R rows and visits the quads (4 columns) c, c+P, ... of the 32-quad
//      spans of its warp, so each coefficient vector loaded from shared memory
//      feeds R rows; the ring slot is released as soon as these loads are
//      done; a shuffle reduce-scatter over the P phases and a fixed-order sum
//      over warps give the CTA's partial logits, pushed into every peer's
//      exchange slot (st.async completing on the peer's mbarrier);
//   gradient group (NWC warps, one per span): once every CTA's partials of a
//      tile have arrived, sums the S partials in rank order (so all CTAs hold
//      identical logits), forms the softmax with the fixed zero logit of
//      class K, the residual R = Y - P and the row log-likelihood, then
//      thread <-> quad accumulates X^T R in registers across all tiles of the
//      cluster, without atomics.  Its X quads are read again from global
//      memory: the tile was streamed through L2 at most a few tiles earlier,
//      so this is an L2 hit and HBM still sees X once.
// The ring therefore only covers the HBM latency and sweep 1; the exchange,
// softmax and sweep 2 of up to kNZ earlier tiles run behind it, so the
// latency of the cluster exchange no longer holds ring slots.
//
// Every wait is bounded.  A wait that runs out records an error bit and the
// role carries on (later waits are skipped), so all barriers stay matched,
// every copy in flight lands, and the kernel returns.
#pragma once
#include "device_common.cuh"
#include "internal.h"

namespace hmc {
namespace simt {

constexpr int kMaxThreads = kSimtMaxThreads;   // 2 x 7 consumer warps + producer
constexpr int kBM = kSimtRows;   // rows per super-tile
constexpr int kNZ = 2;   // exchange slots: tiles the logit group may run ahead of the gradient group

__device__ __forceinline__ float bf16lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

__device__ __forceinline__ void fp8x2(uint32_t two, float& a, float& b) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(two & 0xffffu), __NV_E4M3);
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&h));
  a = f.x;
  b = f.y;
}

// 4 consecutive elements of X in shared memory (aligned to 4 elements).
template <typename XT, typename AT>
__device__ __forceinline__ void load_quad(const unsigned char* p, AT* o);

template <>
__device__ __forceinline__ void load_quad<double, double>(const unsigned char* p, double* o) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 16);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
template <>
__device__ __forceinline__ void load_quad<float, float>(const unsigned char* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void load_quad<__nv_bfloat16, float>(const unsigned char* p, float* o) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  o[0] = bf16lo(v.x); o[1] = bf16hi(v.x); o[2] = bf16lo(v.y); o[3] = bf16hi(v.y);
}
template <>
__device__ __forceinline__ void load_quad<__nv_fp8_e4m3, float>(const unsigned char* p, float* o) {
  const uint32_t v = *reinterpret_cast<const uint32_t*>(p);
  fp8x2(v, o[0], o[1]);
  fp8x2(v >> 16, o[2], o[3]);
}

// 4 consecutive elements of X from global memory as raw 32-bit words
// (read-only path, no L1 allocation: each word is used by one thread once).
template <typename XT>
__device__ __forceinline__ void ldg_quad(const XT* p, uint32_t* w);
template <>
__device__ __forceinline__ void ldg_quad<float>(const float* p, uint32_t* w) {
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
}
template <>
__device__ __forceinline__ void ldg_quad<double>(const double* p, uint32_t* w) {
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]) : "l"(p + 2));
}
template <>
__device__ __forceinline__ void ldg_quad<__nv_bfloat16>(const __nv_bfloat16* p, uint32_t* w) {
  asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "l"(p));
}
template <>
__device__ __forceinline__ void ldg_quad<__nv_fp8_e4m3>(const __nv_fp8_e4m3* p, uint32_t* w) {
  asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(w[0]) : "l"(p));
}

template <typename XT, typename AT>
__device__ __forceinline__ void quad_of_words(const uint32_t* w, AT* o);
template <>
__device__ __forceinline__ void quad_of_words<float, float>(const uint32_t* w, float* o) {
#pragma unroll
  for (int j = 0; j < 4; ++j) o[j] = __uint_as_float(w[j]);
}
template <>
__device__ __forceinline__ void quad_of_words<double, double>(const uint32_t* w, double* o) {
#pragma unroll
  for (int j = 0; j < 4; ++j) o[j] = __hiloint2double(int(w[2 * j + 1]), int(w[2 * j]));
}
template <>
__device__ __forceinline__ void quad_of_words<__nv_bfloat16, float>(const uint32_t* w, float* o) {
  o[0] = bf16lo(w[0]); o[1] = bf16hi(w[0]); o[2] = bf16lo(w[1]); o[3] = bf16hi(w[1]);
}
template <>
__device__ __forceinline__ void quad_of_words<__nv_fp8_e4m3, float>(const uint32_t* w, float* o) {
  fp8x2(w[0], o[0], o[1]);
  fp8x2(w[0] >> 16, o[2], o[3]);
}

// Packed FP32 pairs (f32x2): one instruction issues two IEEE fused
// multiply-adds, so the FP32 sweeps need half the FMA issue slots.  The low
// half of the 64-bit register is the first element.
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ float2 unpack2(uint64_t v) {
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(v));
  return f;
}

// 4 consecutive elements of X in shared memory as two FP32 pairs (x0,x1), (x2,x3).
template <typename XT>
__device__ __forceinline__ void load_quad2(const unsigned char* p, uint64_t* o) {
  if constexpr (sizeof(XT) == 4) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
    o[0] = v.x;
    o[1] = v.y;
  } else {
    float f[4];
    load_quad<XT, float>(p, f);
    o[0] = pack2(f[0], f[1]);
    o[1] = pack2(f[2], f[3]);
  }
}

// N consecutive values of the state type from shared memory (16-byte aligned).
template <typename AT, int N>
__device__ __forceinline__ void load_vec(const AT* p, AT* o) {
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

// Named barrier of one consumer group (ids 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Shape of one instantiation (class bound CT, state type of `abytes` bytes).
struct ShapeRT {
  int R;     // rows per lane in sweep 1
  int A;     // row groups per warp
  int P;     // phases per row group
  int QPL;   // quads per lane per 32-quad span
  int PV;    // values per 16-byte vector
  int CTP;   // exchanged / residual row width (whole 16-byte vectors)
  int CTQ;   // classes padded so that R*CTQ splits evenly over the P phases
  int V;     // values per lane entering the reduce-scatter
  int VP;    // values per lane leaving it
};

__host__ __device__ constexpr ShapeRT shape_rt(int abytes, int CT) {
  ShapeRT s{};
  s.R = 2;
  s.A = kBM / s.R;
  s.P = 32 / s.A;
  s.QPL = 32 / s.P;
  s.PV = 16 / abytes;
  s.CTP = ((CT + s.PV - 1) / s.PV) * s.PV;
  int c = s.CTP;
  while ((s.R * c) % s.P) ++c;
  s.CTQ = c;
  s.V = s.R * s.CTQ;
  s.VP = s.V / s.P;
  return s;
}

// Warps an instantiation supports (register budget of its launch bound):
// gradient warps (one per 32 column quads) and logit warps (half as many,
// each sweeping several spans).
__host__ __device__ constexpr int max_grad_warps(int abytes, int CT) { return (abytes == 4 && CT <= 12) ? 10 : 5; }
__host__ __device__ constexpr int logit_warps(int nwc) { return (nwc + 1) / 2; }
__host__ __device__ constexpr int max_threads(int abytes, int CT) {
  return 32 * (max_grad_warps(abytes, CT) + logit_warps(max_grad_warps(abytes, CT)) + 1);
}

template <typename AT, int CT>
struct Shape {
  static constexpr ShapeRT s = shape_rt(int(sizeof(AT)), CT);
  static constexpr int R = s.R, A = s.A, P = s.P, QPL = s.QPL, PV = s.PV, CTP = s.CTP, CTQ = s.CTQ, V = s.V,
                       VP = s.VP;
  static_assert(CTQ >= CTP, "reduce-scatter rows cover the exchanged width");
  static_assert(V % P == 0, "whole values per lane after the reduce-scatter");
};

// Shared-memory layout; the host computes the same size with simt_smem_bytes().
struct Layout {
  size_t xs, bs, red, zx, rs, lrow, ylab, bars, total;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// NWL: logit warps.
__host__ __device__ inline Layout layout(int xbytes, int abytes, int CT, int CTP, int V, int A, int PC, int S, int NWL,
                                         int NSTAGE) {
  Layout L;
  const size_t xpitch = size_t(PC) * xbytes + 16;
  size_t off = 0;
  L.xs = off;   off = align16(off + size_t(NSTAGE) * kBM * xpitch);
  L.bs = off;   off = align16(off + size_t(CT) * PC * abytes);
  L.red = off;  off = align16(off + size_t(2) * NWL * A * V * abytes);
  L.zx = off;   off = align16(off + size_t(kNZ) * S * kBM * CTP * abytes);
  L.rs = off;   off = align16(off + size_t(kNZ) * kBM * CTP * abytes);
  L.lrow = off; off = align16(off + size_t(kNZ) * kBM * CT * 8);
  L.ylab = off; off = align16(off + size_t(kNZ) * kBM * 4);
  L.bars = off; off = align16(off + size_t(2 * NSTAGE + 2 * kNZ + 2) * 8);
  L.total = off;
  return L;
}

template <typename XT, typename AT, int CT>
__device__ __forceinline__ void lpg_body(const LpgArgs& A, const int cl) {
  using Sh = Shape<AT, CT>;
  constexpr int R = Sh::R, NA = Sh::A, P = Sh::P, QPL = Sh::QPL, PV = Sh::PV, CTP = Sh::CTP, CTQ = Sh::CTQ,
                V = Sh::V, VP = Sh::VP;
  constexpr int BM = kBM;
  constexpr int QW = int(sizeof(XT));     // 32-bit words of one quad of X
  constexpr int XB = BM < (QW > 4 ? 4 : 8) ? BM : (QW > 4 ? 4 : 8);   // rows of X a gradient thread holds in registers
  constexpr int MAXW = logit_warps(max_grad_warps(int(sizeof(AT)), CT));
  extern __shared__ __align__(128) unsigned char smem[];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NTB = int(blockDim.x);
  const int NWL = A.NWL, NTL = NWL * 32;                 // logit warps / threads
  const int NWC = NTB / 32 - 1 - NWL, NTG = NWC * 32;    // gradient warps / threads
  const bool logit = warp < NWL, producer = warp == NWL + NWC;
  const int S = A.S, PC = A.PC, NSTAGE = A.NSTAGE;
  const int nq = PC >> 2;                                  // column quads of the slice
  const uint32_t rank = (S > 1) ? cluster_rank() : 0u;
  const size_t xpitch = size_t(PC) * sizeof(XT) + 16;
  int err0 = 0;

  const Layout Lo = layout(sizeof(XT), sizeof(AT), CT, CTP, V, NA, PC, S, NWL, NSTAGE);
  unsigned char* xs = smem + Lo.xs;
  AT* bs = reinterpret_cast<AT*>(smem + Lo.bs);
  AT* red = reinterpret_cast<AT*>(smem + Lo.red);
  AT* zx = reinterpret_cast<AT*>(smem + Lo.zx);
  AT* rs = reinterpret_cast<AT*>(smem + Lo.rs);            // [kNZ][BM][CTP] residual rows
  double* lrow = reinterpret_cast<double*>(smem + Lo.lrow);  // [kNZ][BM][CT] row log-likelihoods
  int* ylab = reinterpret_cast<int*>(smem + Lo.ylab);       // [kNZ][BM] labels
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lo.bars);
  uint64_t* empty = full + NSTAGE;
  uint64_t* zfull = empty + NSTAGE;
  uint64_t* zempty = zfull + kNZ;
  uint64_t* never = zempty + kNZ;  // fault injection: a barrier no thread arrives at
  uint64_t* bbar = never + 1;    // coefficient slice landed

  if (tid == 0) {
    // A ring slot is empty once every logit warp has finished sweep 1 on it
    // (the gradient sweep reads the tile again from L2, not from the ring).
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NWL);
    }
    // Exchange slot b of tile t is full once every logit thread of this CTA
    // has arrived (labels and, for S = 1, the logits written) and, for S > 1,
    // the partials of all S CTAs have landed; it is empty once the gradient
    // group of every CTA has read it.
    for (int b = 0; b < kNZ; ++b) {
      mbar_init(&zfull[b], NTL);
      mbar_init(&zempty[b], S);
    }
    mbar_init(never, 1);
    mbar_init(bbar, 1);
    fence_mbar_init_cluster();
  }
  __syncthreads();
  // Coefficient slice, class-major (one bulk copy per class row), FP8
  // column scales folded in: X B = X_q diag(s) B.  Rows past C start at zero.
  {
    if (producer) {
      const uint32_t rb = uint32_t(PC) * sizeof(AT);
      if (lane == 0) mbar_arrive_expect_tx(bbar, rb * uint32_t(A.C));
      __syncwarp();
      const AT* beta = static_cast<const AT*>(A.beta) + size_t(rank) * PC;
      for (int k = lane; k < A.C; k += 32) bulk_g2s(bs + size_t(k) * PC, beta + size_t(k) * A.p_pad, rb, bbar);
    }
    for (int idx = A.C * PC + tid; idx < CT * PC; idx += NTB) bs[idx] = AT(0);
    for (int idx = tid; idx < kNZ * BM * CTP; idx += NTB) rs[idx] = AT(0);
    if (!mbar_wait_cta(bbar, 0u, A.spin_limit)) err0 |= ERR_TIMEOUT_STAGE;
    if (A.xscale) {
      for (int idx = tid; idx < A.C * PC; idx += NTB) {
        const int j = idx % PC;
        bs[idx] *= AT(A.xscale[int(rank) * PC + j]);
      }
    }
  }
  if (S > 1)
    cluster_sync_all();
  else
    __syncthreads();

  const int64_t nclu = A.nclusters;
  const int64_t T = (cl < A.ntiles) ? (A.ntiles - 1 - cl) / nclu + 1 : 0;   // super-tiles of this cluster
  auto row0_of = [&](int64_t t) { return (cl + t * nclu) * BM; };
  auto rows_of = [&](int64_t t) { return int(min(int64_t(BM), A.n - row0_of(t))); };
  const uint32_t row_bytes = uint32_t(PC) * sizeof(XT);
  int err = err0;
  long long lim = err0 ? 0 : A.spin_limit;
  if (A.inject_timeout && !producer) {
    if (!mbar_wait_cta(never, 0u, lim)) {
      err |= ERR_TIMEOUT_STAGE;
      lim = 0;
    }
  }

  if (producer) {
    // ---------------------------------------------------------------- producer
    const XT* Xs = static_cast<const XT*>(A.X) + size_t(rank) * PC;
    // Tiles ahead of the ring are pulled into L2 with bulk prefetches, up to
    // about 64 KB per CTA beyond the ring (small ring slots).  More is slower:
    // prefetched tiles then evict tiles the gradient sweep has yet to re-read
    // from L2 (measured on the n=10^4 p=5000 FP32 problem).
    const int64_t tile_bytes = int64_t(BM) * row_bytes;
    const int64_t PF = max(int64_t(NSTAGE), min(int64_t(24), (int64_t(64) * 1024 + tile_bytes - 1) / tile_bytes));
    auto prefetch = [&](int64_t t) {
      const int rv = rows_of(t);
      const XT* src = Xs + size_t(row0_of(t)) * A.p_pad;
      if (lane < rv) bulk_prefetch_l2(src + size_t(lane) * A.p_pad, row_bytes);
    };
    for (int64_t t = NSTAGE; t < min(PF, T); ++t) prefetch(t);
    for (int64_t t = 0; t < T; ++t) {
      if (t + PF < T) prefetch(t + PF);
      const int slot = int(t % NSTAGE);
      if (t >= NSTAGE) {
        if (!mbar_wait_cta(&empty[slot], uint32_t(((t / NSTAGE) - 1) & 1), lim)) {
          err |= ERR_TIMEOUT_SLOT;
          lim = 0;
        }
      }
      const int rv = rows_of(t);
      if (lane == 0) mbar_arrive_expect_tx(&full[slot], row_bytes * uint32_t(rv));
      __syncwarp();
      const XT* src = Xs + size_t(row0_of(t)) * A.p_pad;
      if (lane < rv) bulk_g2s(xs + (size_t(slot) * BM + lane) * xpitch, src + size_t(lane) * A.p_pad, row_bytes, &full[slot]);
    }
    // Every copy must land before shared memory is released.
    for (int64_t t = max(int64_t(0), T - NSTAGE); t < T; ++t)
      (void)mbar_wait_cta(&full[t % NSTAGE], uint32_t((t / NSTAGE) & 1), A.spin_limit);
  } else if (logit) {
    // ---------------------------------------------------------------- logit group
    const int ga = lane / P, gc = lane % P;        // row group, phase
    for (int64_t t = 0; t < T; ++t) {
      const int slot = int(t % NSTAGE);
      const int buf = int(t % kNZ);
      const int rb2 = int(t & 1);          // reduction buffer
      const int rv = rows_of(t);
      // Labels of this tile: loaded now, stored with the exchange (the load's
      // latency overlaps the sweep).
      int ylv = 0;
      if (tid < BM && tid < rv) {
        ylv = __ldg(A.y + row0_of(t) + tid);
        // A label outside the classes is reported, not used as a lane index.
        if (ylv < 0 || ylv >= A.Km1 + A.zlogit) {
          err |= ERR_BAD_LABEL;
          ylv = 0;
        }
      }
      if (!mbar_wait_cta(&full[slot], uint32_t((t / NSTAGE) & 1), lim)) {
        err |= ERR_TIMEOUT_STAGE;
        lim = 0;
      }
      const unsigned char* xst = xs + size_t(slot) * BM * xpitch;
      AT acc[R][CT];
      if constexpr (sizeof(AT) == 4) {
        // FP32 state: even and odd columns accumulate in the two halves of
        // an f32x2 pair, added at the end.
        uint64_t acc2[R][CT];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < CT; ++c) acc2[r][c] = 0ull;
        for (int q0 = warp * 32; q0 < nq; q0 += NWL * 32) {
#pragma unroll
          for (int m = 0; m < QPL; ++m) {
            const int q = q0 + gc + m * P;
            if (q < nq) {
              uint64_t xv[R][2];
#pragma unroll
              for (int r = 0; r < R; ++r)
                load_quad2<XT>(xst + size_t(ga * R + r) * xpitch + size_t(q) * 4 * sizeof(XT), xv[r]);
#pragma unroll
              for (int c = 0; c < CT; ++c) {
                const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(bs + size_t(c) * PC + 4 * q);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                  acc2[r][c] = ffma2(xv[r][0], b.x, acc2[r][c]);
                  acc2[r][c] = ffma2(xv[r][1], b.y, acc2[r][c]);
                }
              }
            }
          }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < CT; ++c) {
            const float2 f = unpack2(acc2[r][c]);
            acc[r][c] = AT(f.x + f.y);
          }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < CT; ++c) acc[r][c] = AT(0);
        for (int q0 = warp * 32; q0 < nq; q0 += NWL * 32) {
#pragma unroll
          for (int m = 0; m < QPL; ++m) {
            const int q = q0 + gc + m * P;
            if (q < nq) {
              AT xv[R][4];
#pragma unroll
              for (int r = 0; r < R; ++r)
                load_quad<XT, AT>(xst + size_t(ga * R + r) * xpitch + size_t(q) * 4 * sizeof(XT), xv[r]);
#pragma unroll
              for (int c = 0; c < CT; ++c) {
                AT b[4];
                load_vec<AT, 4>(bs + size_t(c) * PC + 4 * q, b);
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                  for (int j = 0; j < 4; ++j) acc[r][c] = fma(xv[r][j], b[j], acc[r][c]);
              }
            }
          }
        }
      }
      // Sweep 1 is done with this ring slot.
      __syncwarp();
      if (lane == 0) mbar_arrive_local(&empty[slot]);
      AT val[V];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < CTQ; ++c) val[r * CTQ + c] = (c < CT) ? acc[r][c] : AT(0);
      // Reduce-scatter over the P phases of the row group: after the step
      // with mask m a lane keeps the half of its values selected by bit m,
      // so phase gc ends with the sums of values [gc*VP, (gc+1)*VP).
#pragma unroll
      for (int m = P / 2, h = V / 2; m >= 1; m >>= 1, h >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
          const AT send = up ? val[i] : val[i + h];
          const AT keep = up ? val[i + h] : val[i];
          val[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
      }
      {
        AT* rw = red + ((size_t(rb2) * NWL + warp) * NA + ga) * V + gc * VP;
#pragma unroll
        for (int i = 0; i < VP; ++i) rw[i] = val[i];
      }
      group_sync(1, NTL);

      // Exchange slot `buf` must have been read by every CTA (tile t - kNZ).
      const uint32_t zpar = uint32_t((t / kNZ) & 1);
      if (!(S > 1 ? mbar_wait_cluster(&zempty[buf], zpar ^ 1u, lim)
                  : mbar_wait_cta(&zempty[buf], zpar ^ 1u, lim))) {
        err |= ERR_TIMEOUT_SLOT;
        lim = 0;
      }
      if (tid < BM) ylab[buf * BM + tid] = ylv;
      if (S > 1 && tid == 0) mbar_arrive_expect_tx(&zfull[buf], uint32_t(S * BM * CTP * sizeof(AT)));
      // One (row, class) value per thread: the NWL warp partials are loaded
      // together and added in warp order; PV neighbouring classes are then
      // gathered into one lane, which pushes them as a 16-byte vector.
      constexpr int NV = BM * CTP;
      for (int base = 0; base < NV; base += NTL) {
        const int idx = base + tid;
        const bool act = idx < NV;
        const int i = act ? idx / CTP : 0, kc = act ? idx - (idx / CTP) * CTP : 0;
        const int a = i / R, r = i % R;
        AT sum = AT(0);
        if (act && kc < CT) {
          AT wv[MAXW];
#pragma unroll
          for (int w = 0; w < MAXW; ++w)
            wv[w] = (w < NWL) ? red[((size_t(rb2) * NWL + w) * NA + a) * V + r * CTQ + kc] : AT(0);
#pragma unroll
          for (int w = 0; w < MAXW; ++w)
            if (w < NWL) sum += wv[w];
        }
        AT v[PV];
#pragma unroll
        for (int q = 0; q < PV; ++q) v[q] = __shfl_sync(0xffffffffu, sum, (lane + q) & 31);
        if (act && kc % PV == 0) {
          AT* dst = zx + (size_t(buf) * S + rank) * BM * CTP + size_t(i) * CTP + kc;
          if (S == 1) {
#pragma unroll
            for (int q = 0; q < PV; ++q) dst[q] = v[q];
          } else {
            const uint32_t laddr = smem_u32(dst), lbar = smem_u32(&zfull[buf]);
            for (int r2 = 0; r2 < S; ++r2) {
              const uint32_t ra = map_peer(laddr, uint32_t(r2)), rb = map_peer(lbar, uint32_t(r2));
              if constexpr (sizeof(AT) == 4)
                st_async_v4f(ra, float(v[0]), float(v[1]), float(v[2]), float(v[3]), rb);
              else
                st_async_v2d(ra, double(v[0]), double(v[1]), rb);
            }
          }
        }
      }
      // Release: labels (and the local logits when S = 1) are visible to the
      // gradient group once its wait on zfull completes.
      if (!(S > 1 && tid == 0)) mbar_arrive_local(&zfull[buf]);
    }
  } else {
    // ---------------------------------------------------------------- gradient group
    const int gw = warp - NWL, gt = tid - NTL;     // warp / thread within the group
    const int qq = gw * 32 + lane;                 // this thread's quad
    // FP32 state: class pairs (c, c+1) of a column accumulate in one f32x2
    // register (CTH pairs per column); FP64 state: one register per class.
    constexpr int CTH = (CT + 1) / 2;
    constexpr bool kPair = sizeof(AT) == 4;
    uint64_t G2[4][kPair ? CTH : 1];
    AT G[4][kPair ? 1 : CT];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
      for (int k = 0; k < (kPair ? CTH : 1); ++k) G2[q][k] = 0ull;
#pragma unroll
      for (int k = 0; k < (kPair ? 1 : CT); ++k) G[q][k] = AT(0);
    }
    double lacc = 0.0;
    const int Km1 = A.Km1, chains = A.chains;
    const bool zl = A.zlogit != 0;
    int W = 1;
    while (W < Km1) W <<= 1;
    const int RPW = 32 / W, sl = lane % W;
    const int ntask = BM * chains;

    const XT* Xq = static_cast<const XT*>(A.X) + size_t(rank) * PC + size_t(qq) * 4;
    for (int64_t t = 0; t < T; ++t) {
      const int buf = int(t % kNZ);
      const int rv = rows_of(t);
      // This thread's column quad of the tile's rows, read again from L2
      // (the producer streamed the tile at most a few tiles earlier); the
      // loads are issued before the exchange wait so their latency overlaps it.
      // Up to XB rows are in flight; row i + XB is loaded once row i is used.
      uint32_t xw[XB][QW];
      const XT* src = Xq + size_t(row0_of(t)) * A.p_pad;
      if (qq < nq) {
#pragma unroll
        for (int i = 0; i < XB; ++i)
          if (i < rv) ldg_quad<XT>(src + size_t(i) * A.p_pad, xw[i]);
      }
      if (!(S > 1 ? mbar_wait_cluster(&zfull[buf], uint32_t((t / kNZ) & 1), lim)
                  : mbar_wait_cta(&zfull[buf], uint32_t((t / kNZ) & 1), lim))) {
        err |= ERR_TIMEOUT_EXCHANGE;
        lim = 0;
      }
      // Softmax with the zero logit of class K, residual and row
      // log-likelihood: a warp takes 32/W (row, chain) tasks at once, W
      // lanes per task (W = K-1 rounded up to a power of two), lane <-> class.
      const AT* zs = zx + size_t(buf) * S * BM * CTP;
      AT* rsb = rs + size_t(buf) * BM * CTP;
      double* lrb = lrow + size_t(buf) * BM * CT;
      for (int base = gw * RPW; base < ntask; base += NWC * RPW) {
        const int it = base + lane / W;
        const bool task = it < ntask;
        const int i = task ? it / chains : 0, c = task ? it - (it / chains) * chains : 0;
        const int cb = c * Km1;
        const bool valid = task && i < rv;
        const bool cls = task && sl < Km1;
        AT z = AT(0);
        if (cls) {
          AT zr[16];
#pragma unroll
          for (int r = 0; r < 16; ++r) zr[r] = (r < S) ? zs[(size_t(r) * BM + i) * CTP + cb + sl] : AT(0);
#pragma unroll
          for (int r = 0; r < 16; ++r)
            if (r < S) z += zr[r];
        }
        // With the zero logit of class K the row maximum includes 0 and the sum
        // e^{-m}; without it (unconstrained layout) only the Km1 free logits count.
        AT mx = cls ? (zl ? max(z, AT(0)) : z) : (zl ? AT(0) : AT(-INFINITY));
        for (int o = W / 2; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o, W));
        const AT e = cls ? ex<AT>(z - mx) : AT(0);
        AT se = e;
        for (int o = W / 2; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o, W);
        if (zl) se += ex<AT>(-mx);
        const int yi = valid ? ylab[buf * BM + i] : 0;
        const AT zy = __shfl_sync(0xffffffffu, z, yi < Km1 ? yi : 0, W);
        if (cls) rsb[size_t(i) * CTP + cb + sl] = valid ? (sl == yi ? AT(1) : AT(0)) - e / se : AT(0);
        if (task && sl == 0) lrb[size_t(i) * CT + c] = valid ? double((yi < Km1 ? zy : AT(0)) - mx - lg<AT>(se)) : 0.0;
      }
      group_sync(2, NTG);
      // Exchange slot `buf` read: release it in every CTA of the cluster.
      if (gt < S) {
        if (S > 1)
          mbar_arrive_remote(map_peer(smem_u32(&zempty[buf]), uint32_t(gt)));
        else
          mbar_arrive_local(&zempty[buf]);
      }
      // Sweep 2: G += X_tile^T R over the tile's rows (fixed row order;
      // rows past the end of X contribute zero).
      if (qq < nq) {
#pragma unroll
        for (int i = 0; i < BM; ++i) {
          AT xv[4];
          quad_of_words<XT, AT>(xw[i % XB], xv);
          if (i + XB < BM && i + XB < rv) ldg_quad<XT>(src + size_t(i + XB) * A.p_pad, xw[i % XB]);
          if (i >= rv)
#pragma unroll
            for (int q = 0; q < 4; ++q) xv[q] = AT(0);
          if constexpr (kPair) {
            uint64_t r2[CTP / 2];
#pragma unroll
            for (int k = 0; k < CTP / 4; ++k) {
              const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(rsb + size_t(i) * CTP + 4 * k);
              r2[2 * k] = v.x;
              r2[2 * k + 1] = v.y;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const uint64_t xd = pack2(float(xv[q]), float(xv[q]));
#pragma unroll
              for (int k = 0; k < CTH; ++k) G2[q][k] = ffma2(xd, r2[k], G2[q][k]);
            }
          } else {
            AT r[CTP];
            load_vec<AT, CTP>(rsb + size_t(i) * CTP, r);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
              for (int c = 0; c < CT; ++c) G[q][c] = fma(xv[q], r[c], G[q][c]);
          }
        }
      }
      if (rank == 0 && gt < chains) {
        double sl2 = 0.0;
        for (int i = 0; i < rv; ++i) sl2 += lrb[size_t(i) * CT + gt];
        lacc += sl2;
      }
    }

    if (qq < nq) {
      AT* gp = static_cast<AT*>(A.gpart) + size_t(cl) * A.gpart_cstride;
      const int col = int(rank) * PC + 4 * qq;
      AT sc[4] = {AT(1), AT(1), AT(1), AT(1)};
      if (A.xscale)
#pragma unroll
        for (int q = 0; q < 4; ++q) sc[q] = AT(A.xscale[col + q]);
#pragma unroll
      for (int kk = 0; kk < CT; ++kk) {
        if (kk < A.C) {
          AT* d = gp + size_t(kk) * A.p_pad + col;
          if constexpr (kPair) {
            float g[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float2 f = unpack2(G2[q][kk / 2]);
              g[q] = (kk & 1) ? f.y : f.x;
            }
            *reinterpret_cast<float4*>(d) = make_float4(g[0] * float(sc[0]), g[1] * float(sc[1]),
                                                        g[2] * float(sc[2]), g[3] * float(sc[3]));
          } else {
            reinterpret_cast<double2*>(d)[0] = make_double2(double(G[0][kk] * sc[0]), double(G[1][kk] * sc[1]));
            reinterpret_cast<double2*>(d)[1] = make_double2(double(G[2][kk] * sc[2]), double(G[3][kk] * sc[3]));
          }
        }
      }
    }
    if (rank == 0 && gt < A.chains) A.lpart[size_t(cl) * A.lpart_cstride + gt] = lacc;
  }
  if (err) atomicOr(A.err, err);
  if (S > 1)
    cluster_sync_all();   // no peer may still write into this CTA's shared memory
  else
    __syncthreads();
}

template <typename XT, typename AT, int CT>
__global__ void __launch_bounds__(max_threads(int(sizeof(AT)), CT), 1) lpg_kernel(const LpgArgs A) {
  lpg_body<XT, AT, CT>(A, int(blockIdx.x) / A.S);
}

// Several independent problems in one launch: clusters [first[b], first[b+1])
// of the grid work on problem b (its own X, labels, coefficients, tiles and
// partial slots); every problem shares the cluster size and block size.
template <typename XT, typename AT, int CT>
__global__ void __launch_bounds__(max_threads(int(sizeof(AT)), CT), 1)
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
