// Fused log-posterior + gradient pass on the 5th-generation tensor cores
// (tcgen05) for X stored in BF16 or per-column-scaled FP8 (widened to BF16 in
// shared memory), many chains at once (Eqs. softmax, loglike,
// logkernel and gradient of Sec. 2.1, evaluated for C = chains*(K-1)
// coefficient columns).
//
// Decomposition: a cluster of S CTAs walks row tiles of 128 rows; CTA `rank`
// owns the column slice [rank*PC, (rank+1)*PC) (PC a multiple of 128) of X and
// of the coefficients, and accumulates the gradient rows of that slice in
// TMEM across all of the cluster's tiles.  Per tile:
//   sweep 1  bulk-async copies bring 128 x 64 boxes of X together with the
//            matching 64-column box of the coefficients as two BF16 terms
//            (B = B_hi + B_lo); MMAs D_z[128 x N] += X_box . B_hi^T and
//            += X_box . B_lo^T (both operands K-major), so the logits carry
//            the coefficients to ~16 bits.
//            X and the coefficient operand are stored in device memory as
//            the shared-memory image of these boxes (128-byte swizzle already
//            applied, each box 16 KB contiguous), so every copy is a long
//            contiguous read.
//   exchange (distributed shared memory only) the drain warps read D_z, one
//            row per thread, and push each row with st.async into the shared
//            memory of the CTA that owns it (rows are split 128/S per CTA);
//            the owner sums the S partials in rank order, forms the softmax
//            with the zero logit of class K, the residual R = Y - P (BF16) and
//            the row log-likelihood, and pushes its R rows with st.async
//            straight into every peer's MMA operand buffer (swizzled layout).
//            Completion is counted in mbarrier transaction bytes.
//   sweep 2  X is re-read in 128-column blocks (an L2 hit: the tile was
//            streamed one sweep earlier); MMA D_g[mb] (128 columns x N) +=
//            X_blk^T . R with X_blk read MN-major from the same swizzled boxes
//            and R MN-major from the operand buffer.  The commit of these MMAs
//            is multicast to every CTA of the cluster, telling the owners
//            that the R buffer may take the rows of a later tile.
// Sweeps are interleaved S1(0), S1(1), S2(0), S1(2), S2(1), ... so the
// exchange of one tile overlaps the next tile's first sweep.
// Warp roles: warp 0 TMA producer (lane 0 alone: no other role shares its
// warp, so nothing suspends the copy issue), warp 1 TMEM owner + MMA issuer,
// warps 2-5 drain group (TMEM lanes 0-127; the gradient slice at the end),
// warps 6-13 softmax group, warps 14-21 FP8 converters (FP8 X only).  All
// waits are bounded.
#include <algorithm>
#include <vector>
#include <cstring>

#include "internal.h"
#include "tc_common.cuh"

namespace hmc {
namespace tc {

constexpr int kThreadsBf16 = 448;   // warps 0-13
constexpr int kThreadsFp8 = 704;    // + warps 14-21 (FP8 converters)
constexpr int kSoftThreads = 256;   // warps 6-13
constexpr int kConvWarps = 8;       // warps 14-21: FP8 -> BF16 converters (FP8 X only)
constexpr int kConvThreads = 32 * kConvWarps;
constexpr int kFp8BoxBytes = 128 * 64;   // one FP8 box: 128 rows x 64 bytes, row-major
constexpr int kMaxDepth = kTcMaxDepth;   // largest number of logit accumulators / exchange slots / R buffers
constexpr int kRows = 128;
constexpr int kBox = 64;          // BF16 elements per 128-byte box row
constexpr int kBoxBytes = kRows * 128;

struct TcArgs {
  const void* xs;           // X boxes, [row tile][p_pad / 64][box]: BF16 in its swizzled shared-memory
                            // image (16 KB), or FP8 E4M3 row-major (8 KB) when fp8
  const float* xscale;      // FP8: per-column scales s_j (X = X_q diag(s)); nullptr for BF16
  const __nv_bfloat16* bs;  // coefficient operand boxes: [p_pad / 64][N rows x 128 B]
  int64_t n;
  int32_t p_pad, PC, S, N, NP, C, Km1, chains, MB, NST, nclusters;
  int64_t ntiles;
  uint32_t tmem_cols, stage_bytes;
  float* gpart;             // [cluster][C][p_pad] partial gradient (this launch's columns)
  int64_t gpart_cstride;
  double* lpart;            // [cluster*S + rank][lpart_cstride] partial log-likelihood per chain
  int32_t lpart_cstride;
  const int32_t* y;
  int* err;
  long long spin_limit;
  int32_t inject_timeout;
  int32_t fp8;
  int32_t zlogit;           // 1: class K is the implied zero logit; 0: all Km1 classes free
  // Pipeline depths (host-chosen from the TMEM and shared-memory budgets):
  int32_t nz;      // logit accumulators in TMEM (sweep 1 of the next tiles runs while one drains)
  int32_t slots;   // partial-logit receive slots (reuse gated by a cluster 'consumed' barrier)
  int32_t rbufs;   // R operand buffers (reuse gated by a cluster 'free' barrier)
  int32_t la;      // tiles of lookahead between the two sweeps of a tile
};

struct Smem {
  size_t ring, stage, rbuf, zx, rloc, lacc, ylab, bars, total;
};

__host__ __device__ inline size_t al(size_t v, size_t a) { return (v + a - 1) / a * a; }

// zx: [slots][S][RS][N] fp32 partial logits received for the owned rows;
// rloc: [RS][NP] bf16 residual rows of the owned rows before they are pushed.
__host__ __device__ inline Smem smem_layout(int NST, uint32_t stage_bytes, int NP, int N, int S, int chains, bool fp8,
                                            int slots, int rbufs) {
  Smem L;
  const int RS = kRows / S;
  size_t off = 0;
  L.ring = off;  off = al(off + size_t(NST) * stage_bytes, 1024);
  // FP8 boxes land in the upper half of their slot's X area and are widened in place.
  L.stage = off;
  L.rbuf = off;  off = al(off + size_t(rbufs) * (NP / kBox) * kBoxBytes, 1024);
  L.zx = off;    off = al(off + size_t(slots) * kRows * N * 4, 16);
  L.rloc = off;  off = al(off + size_t(RS) * NP * 2, 16);
  L.lacc = off;  off = al(off + size_t(RS) * chains * 8, 16);
  L.ylab = off;  off = al(off + size_t(RS) * 4, 16);
  L.bars = off;  off = al(off + size_t(3 * NST + 6 * kMaxDepth + 6) * 8 + 16, 16);
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

__device__ __forceinline__ void named_bar_drain() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ void named_bar_soft() { asm volatile("bar.sync 2, 256;" ::: "memory"); }
// Barrier of the FP8 converter group (named barrier 3), and the same barrier
// ANDing a flag across the group (so every converter leaves its loop together).
__device__ __forceinline__ void conv_bar() { asm volatile("bar.sync 3, %0;" ::"n"(kConvThreads) : "memory"); }
__device__ __forceinline__ bool conv_bar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.and.pred po, 3, %2, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"(v ? 1u : 0u), "n"(kConvThreads)
      : "memory");
  return r != 0;
}
// Named barrier of the softmax group that also ANDs a flag across its threads.
__device__ __forceinline__ bool named_bar_soft_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.and.pred po, 2, 256, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"(v ? 1u : 0u)
      : "memory");
  return r != 0;
}

// One cluster's share of the fused pass for problem A; cl = the cluster's
// index among the clusters working on this problem.
template <bool kFP8>
__device__ __forceinline__ void tc_body(const TcArgs& A, const int cl) {
  constexpr int kThreads = kFP8 ? kThreadsFp8 : kThreadsBf16;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int S = A.S, N = A.N, NST = A.NST, NP = A.NP;
  const uint32_t rank = (S > 1) ? cluster_rank() : 0u;
  const int RS = kRows / S;                        // rows this CTA owns in the exchange
  const int chains = A.chains, C = A.C, Km1 = A.Km1;
  const bool zl = A.zlogit != 0;
  const int C8 = (C + 7) / 8;                      // 16-byte chunks of one R row
  constexpr bool fp8 = kFP8;
  const int NZ = A.nz, SLOTS = A.slots, RBUFS = A.rbufs, LA = A.la;
  const Smem Lo = smem_layout(NST, A.stage_bytes, NP, N, S, chains, fp8, SLOTS, RBUFS);
  unsigned char* ring = smem + Lo.ring;
  unsigned char* rbuf = smem + Lo.rbuf;
  float* zx = reinterpret_cast<float*>(smem + Lo.zx);
  __nv_bfloat16* rloc = reinterpret_cast<__nv_bfloat16*>(smem + Lo.rloc);
  double* lacc = reinterpret_cast<double*>(smem + Lo.lacc);
  int* ylab = reinterpret_cast<int*>(smem + Lo.ylab);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lo.bars);
  uint64_t* full = bars;
  uint64_t* empty = bars + NST;
  uint64_t* conv = bars + 2 * NST;      // FP8: ring slot converted to BF16 (kConvWarps arrivals)
  uint64_t* zdone = bars + 3 * NST;        // [nz] sweep 1 of a tile finished in accumulator z
  uint64_t* zfree = zdone + kMaxDepth;      // [nz] accumulator z drained
  uint64_t* zrdy = zfree + kMaxDepth;       // [slots] partial logits of the owned rows received
  uint64_t* zxfree = zrdy + kMaxDepth;      // [slots] every owner has consumed the slot's partials
  uint64_t* rfull = zxfree + kMaxDepth;     // [rbufs] every owner's R rows received (R buffer b)
  uint64_t* rfreec = rfull + kMaxDepth;     // [rbufs] every CTA's gradient sweep finished reading R buffer b
  uint64_t* gdone = rfreec + kMaxDepth;
  uint64_t* drain = gdone + 1;
  uint64_t* never = gdone + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gdone + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gdone + 4);
  const size_t rbuf_bytes = size_t(NP / kBox) * kBoxBytes;

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&conv[s], kConvWarps);
    }
    for (int b = 0; b < kMaxDepth; ++b) {
      mbar_init(&zdone[b], 1);
      mbar_init(&zfree[b], 4);
      mbar_init(&zrdy[b], 1);
      mbar_init(&zxfree[b], S);
      mbar_init(&rfull[b], 1);
      mbar_init(&rfreec[b], S);
    }
    mbar_init(gdone, 1);
    mbar_init(drain, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    fence_mbar_init_cluster();
  }
  // R operand buffer and the local R rows start (and stay, past column C) zero.
  for (size_t i = tid; i < RBUFS * rbuf_bytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(rbuf)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < RS * NP / 8; i += kThreads) reinterpret_cast<uint4*>(rloc)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < RS * chains; i += kThreads) lacc[i] = 0.0;
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
  const int64_t nkb_all = A.p_pad / kBox;
  // Phase k of the sweep order: S1(0..first-1), then pairs S1(v), S2(v-la),
  // then the remaining S2 phases.  Returns the tile; *s2 marks a gradient sweep.
  const int64_t first = T < LA ? T : LA;
  auto phase = [&](int64_t k, bool* s2) -> int64_t {
    if (k < first) { *s2 = false; return k; }
    const int64_t k1 = k - first;
    if (k1 < 2 * (T - first)) {
      *s2 = (k1 & 1) != 0;
      return *s2 ? (k1 >> 1) : first + (k1 >> 1);
    }
    *s2 = true;
    return T - first + (k1 - 2 * (T - first));
  };
  auto fail = [&](int bit) {
    *abort_flag = 1;
    atomicOr(A.err, bit);
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int64_t j = 0, issued = 0;
      for (int64_t k = 0; k < nphase && !*abort_flag; ++k) {
        bool s2;
        const int64_t u = phase(k, &s2);
        const int nb = s2 ? A.MB : NKB;
        for (int b = 0; b < nb; ++b, ++j) {
          const int st = int(j % NST);
          if (!wait_bounded(&empty[st], uint32_t(((j / NST) & 1) ^ 1), A.spin_limit, abort_flag, false)) {
            fail(ERR_TIMEOUT_STAGE);
            break;
          }
          unsigned char* sp = ring + size_t(st) * A.stage_bytes;
          const int64_t t = cl + u * nclu;  // row tile
          const uint32_t xbox = fp8 ? uint32_t(kFp8BoxBytes) : uint32_t(kBoxBytes);
          const unsigned char* xt = reinterpret_cast<const unsigned char*>(A.xs) + size_t(t) * nkb_all * xbox;
          // BF16 X lands in the slot itself; FP8 X lands in the upper half of the
          // slot's X area and the converter warps widen it in place.
          unsigned char* xdst = fp8 ? sp + size_t(s2 ? 2 : 1) * (kBoxBytes - kFp8BoxBytes) : sp;
          if (!s2) {
            const int kb = int(rank) * NKB + b;
            mbar_arrive_expect_tx(&full[st], xbox + uint32_t(2 * N * 128));
            bulk_g2s(xdst, xt + size_t(kb) * xbox, xbox, &full[st]);
            bulk_g2s(sp + kBoxBytes, reinterpret_cast<const unsigned char*>(A.bs) + size_t(kb) * 2 * N * 128,
                     uint32_t(2 * N * 128), &full[st]);
          } else {
            const int kb = int(rank) * NKB + 2 * b;
            mbar_arrive_expect_tx(&full[st], 2 * xbox);
            bulk_g2s(xdst, xt + size_t(kb) * xbox, 2 * xbox, &full[st]);
          }
          issued = j + 1;
        }
      }
      // Every copy issued must land before shared memory is released.
      for (int64_t jj = (issued > NST ? issued - NST : 0); jj < issued; ++jj)
        (void)wait_bounded(&full[jj % NST], uint32_t((jj / NST) & 1), A.spin_limit, abort_flag, false);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t id_s1 = idesc_bf16(kRows, N, false, false);
      const uint32_t id_s2 = idesc_bf16(kRows, N, true, true);
      const uint32_t rb = smem_u32(rbuf);
      const uint32_t rbytes = uint32_t(kRows) * C8 * 16;
      int64_t j = 0;
      for (int64_t k = 0; k < nphase && !*abort_flag; ++k) {
        bool s2;
        const int64_t u = phase(k, &s2);
        if (!s2) {
          // Accumulator z = u % nz was last used by tile u - nz: it must be drained.
          const int z = int(u % NZ);
          if (u >= NZ && !wait_bounded(&zfree[z], uint32_t(((u / NZ) - 1) & 1), A.spin_limit, abort_flag, false)) {
            fail(ERR_TIMEOUT_MMA);
            break;
          }
          const uint32_t dz = tmem + uint32_t(z * N);
          fence_after_sync();
          for (int kb = 0; kb < NKB; ++kb, ++j) {
            const int st = int(j % NST);
            if (!wait_bounded(fp8 ? &conv[st] : &full[st], uint32_t((j / NST) & 1), A.spin_limit, abort_flag, false)) {
              fail(ERR_TIMEOUT_STAGE);
              break;
            }
            fence_after_sync();
            const uint32_t xa = smem_u32(ring + size_t(st) * A.stage_bytes);
            const uint32_t ba = xa + kBoxBytes;             // hi rows; lo rows N * 128 bytes further
#pragma unroll
            for (int s = 0; s < 4; ++s) {
              const uint64_t ad = smem_desc(xa + 32u * s, 16u, 1024u, 2u);
              const uint64_t bd = smem_desc(ba + 32u * s, 16u, 1024u, 2u);
              const uint64_t bl = smem_desc(ba + uint32_t(N) * 128u + 32u * s, 16u, 1024u, 2u);
              mma_bf16(dz, ad, bd, id_s1, (kb > 0 || s > 0) ? 1u : 0u);
              mma_bf16(dz, ad, bl, id_s1, 1u);
            }
            mma_commit(&empty[st]);
          }
          if (*abort_flag) break;
          mma_commit(&zdone[z]);
        } else {
          const int rbi = int(u % RBUFS);
          mbar_arrive_expect_tx(&rfull[rbi], rbytes);
          if (!wait_bounded(&rfull[rbi], uint32_t((u / RBUFS) & 1), A.spin_limit, abort_flag, true)) {
            fail(ERR_TIMEOUT_EXCHANGE);
            break;
          }
          fence_after_sync();
          for (int mb = 0; mb < A.MB; ++mb, ++j) {
            const int st = int(j % NST);
            if (!wait_bounded(fp8 ? &conv[st] : &full[st], uint32_t((j / NST) & 1), A.spin_limit, abort_flag, false)) {
              fail(ERR_TIMEOUT_STAGE);
              break;
            }
            fence_after_sync();
            const uint32_t xa = smem_u32(ring + size_t(st) * A.stage_bytes);
            const uint32_t dcol = tmem + uint32_t((NZ + mb) * N);
#pragma unroll
            for (int s = 0; s < 8; ++s) {
              const uint64_t ad = smem_desc(xa + 2048u * s, uint32_t(kBoxBytes), 1024u, 2u);
              const uint64_t bd = smem_desc(rb + uint32_t(rbi * rbuf_bytes) + 2048u * s, uint32_t(kBoxBytes), 1024u, 2u);
              mma_bf16(dcol, ad, bd, id_s2, (u > 0 || s > 0) ? 1u : 0u);
            }
            mma_commit(&empty[st]);
          }
          if (*abort_flag) break;
          // R buffer rbi is free once these MMAs complete: the commit arrives on
          // that buffer's barrier in every CTA of the cluster, so each owner may
          // push the R rows of tile u + rbufs.  Only tiles whose buffer is used
          // again signal, so every remote arrival has a waiter in its CTA (and
          // lands before that CTA can leave the kernel).
          if (u + RBUFS < T) {
            if (S > 1)
              mma_commit_multicast(&rfreec[rbi], uint16_t((1u << S) - 1u));
            else
              mma_commit(&rfreec[rbi]);
          }
        }
      }
      mma_commit(gdone);
      mma_commit(drain);
      (void)wait_bounded(drain, 0u, A.spin_limit, abort_flag, false);
    }
  } else if (kFP8 && warp >= 14) {
    // --------------------------------------- FP8 converters (warps 14-21)
    // Each FP8 box (128 rows x 64 bytes, landed in the upper half of its
    // slot's X area) is widened to BF16 (exact: every E4M3 value is a BF16
    // value) and written over the slot in the 128-byte-swizzled layout the
    // MMAs read; sweep-2 slots hold two boxes.  Every converter thread reads
    // all its input chunks before a converter-group barrier and only then
    // writes, so the in-place widening never overwrites unread input.
    {
      const int ct = tid - kThreadsBf16;   // 0 .. kConvThreads - 1
      int64_t j = 0;
      bool ok = true;
      for (int64_t k = 0; k < nphase && ok; ++k) {
        bool s2;
        (void)phase(k, &s2);
        const int nb = s2 ? A.MB : NKB;
        const int nbox = s2 ? 2 : 1;
        for (int b = 0; b < nb; ++b, ++j) {
          const int st = int(j % NST);
          const bool got = wait_bounded(&full[st], uint32_t((j / NST) & 1), A.spin_limit, abort_flag, false);
          // Every converter agrees before the group barriers below.
          if (!conv_bar_and(got && !*abort_flag)) {
            if (!got) fail(ERR_TIMEOUT_STAGE);
            ok = false;
            break;
          }
          unsigned char* dst = ring + size_t(st) * A.stage_bytes;
          const unsigned char* src = dst + size_t(nbox) * (kBoxBytes - kFp8BoxBytes);
          // Input chunk ci (16 bytes) of box bx: row ci / 4, elements 16 (ci % 4) ...
          constexpr int kPer = (2 * kFp8BoxBytes / 16) / kConvThreads;   // chunks per thread, two boxes
          uint4 w[kPer];
#pragma unroll
          for (int i = 0; i < kPer; ++i)
            if (i < nbox * kPer / 2) w[i] = *reinterpret_cast<const uint4*>(src + size_t(ct + kConvThreads * i) * 16);
          conv_bar();
#pragma unroll
          for (int i = 0; i < kPer; ++i) {
            if (i >= nbox * kPer / 2) break;
            const int g = ct + kConvThreads * i;               // chunk over both boxes
            const int bx = g / (kFp8BoxBytes / 16), ci = g % (kFp8BoxBytes / 16);
            const int r = ci >> 2, qq = ci & 3;
            uint32_t o[8];
            fp8x4_to_bf16x4(w[i].x, o[0], o[1]);
            fp8x4_to_bf16x4(w[i].y, o[2], o[3]);
            fp8x4_to_bf16x4(w[i].z, o[4], o[5]);
            fp8x4_to_bf16x4(w[i].w, o[6], o[7]);
            unsigned char* rowp = dst + size_t(bx) * kBoxBytes + size_t(r) * 128;
            *reinterpret_cast<uint4*>(rowp + ((((2 * qq) ^ (r & 7))) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
            *reinterpret_cast<uint4*>(rowp + ((((2 * qq + 1) ^ (r & 7))) << 4)) = make_uint4(o[4], o[5], o[6], o[7]);
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive_local(&conv[st]);
        }
      }
    }
  } else if (warp < 6) {
    // ------------------------------------------------ drain group (warps 2-5)
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int row = 32 * q + lane;          // tile row (sweep-1 accumulator lane)
    const uint32_t tq = tmem + (uint32_t(32 * q) << 16);
    const uint32_t owner = uint32_t(row / RS), rl = uint32_t(row % RS);
    for (int64_t u = 0; u < T && !*abort_flag; ++u) {
      const int slot = int(u % SLOTS);
      const int z = int(u % NZ);
      // Lane 0 waits for each barrier and the warp follows it (one waiter per
      // warp keeps the barrier probes off the shared-memory pipe).
      bool ok = (lane == 0) ? wait_bounded(&zdone[z], uint32_t((u / NZ) & 1), A.spin_limit, abort_flag, false) : true;
      if (!__shfl_sync(0xffffffffu, ok, 0)) {
        if (lane == 0) fail(ERR_TIMEOUT_MMA);
        break;
      }
      fence_after_sync();
      // The owners' slot was last filled with tile u - slots: they must have consumed it.
      ok = (lane == 0 && u >= SLOTS)
               ? wait_bounded(&zxfree[slot], uint32_t(((u / SLOTS) - 1) & 1), A.spin_limit, abort_flag, true)
               : true;
      if (!__shfl_sync(0xffffffffu, ok, 0)) {
        if (lane == 0) fail(ERR_TIMEOUT_SLOT);
        break;
      }
      // This row's partial logits go to the owner's slot [slot][rank][rl].
      const uint32_t laddr = smem_u32(zx + ((size_t(slot) * S + rank) * RS + rl) * N);
      const uint32_t raddr = (S > 1) ? map_peer(laddr, owner) : laddr;
      const uint32_t rbar = (S > 1) ? map_peer(smem_u32(&zrdy[slot]), owner) : smem_u32(&zrdy[slot]);
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tmem_ld16(tq + uint32_t(z * N + c0), v);
#pragma unroll
        for (int e = 0; e < 16; e += 4) st_async_v4f(raddr + uint32_t(c0 + e) * 4u, v[e], v[e + 1], v[e + 2], v[e + 3], rbar);
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive_local(&zfree[z]);
    }
    // Drain the gradient accumulators of this CTA's column slice.
    bool gok = false;
    if (T > 0 && !*abort_flag) {
      gok = wait_bounded(gdone, 0u, A.spin_limit, abort_flag, false);
      if (!gok) fail(ERR_TIMEOUT_MMA);
    }
    float* gp = A.gpart + size_t(cl) * A.gpart_cstride;
    if (gok && !*abort_flag) {
      fence_after_sync();
      for (int mb = 0; mb < A.MB; ++mb) {
        const int col = int(rank) * A.PC + mb * 128 + row;
        const float sc = A.xscale ? A.xscale[col] : 1.0f;   // g = diag(s) X_q^T R
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tmem_ld16(tq + uint32_t((NZ + mb) * N + c0), v);
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (c0 + e < C) gp[size_t(c0 + e) * A.p_pad + col] = v[e] * sc;
        }
      }
    } else {
      for (int mb = 0; mb < A.MB; ++mb) {
        const int col = int(rank) * A.PC + mb * 128 + row;
        for (int c = 0; c < C; ++c) gp[size_t(c) * A.p_pad + col] = 0.f;
      }
    }
    fence_before_sync();
  } else {
    // --------------------------------------------- softmax group (warps 6-13)
    const int st = tid - 192;               // 0..255
    const int sw = warp - 6;                // 0..7
    const uint32_t rb_local = smem_u32(rbuf);
    for (int64_t u = 0; u < T && !*abort_flag; ++u) {
      const int slot = int(u % SLOTS);
      const uint32_t use_par = uint32_t((u / SLOTS) & 1);
      const int64_t row0 = (cl + u * nclu) * kRows;
      if (st == 0) mbar_arrive_expect_tx(&zrdy[slot], uint32_t(kRows) * N * 4);
      if (st < RS) {
        const int64_t grow = row0 + int(rank) * RS + st;
        ylab[st] = grow < A.n ? __ldg(A.y + grow) : -1;
      }
      // One thread waits for the partials; after the group barrier every thread
      // takes its own cluster-scope acquire of the completed phase.
      const bool zok = (st == 0) ? wait_bounded(&zrdy[slot], use_par, A.spin_limit, abort_flag, true) : true;
      if (!named_bar_soft_and(zok)) {
        if (!zok) fail(ERR_TIMEOUT_EXCHANGE);
        break;
      }
      (void)mbar_test_cluster(smem_u32(&zrdy[slot]), use_par);
      // Softmax with the zero logit of class K, residual and row log-likelihood:
      // one warp per (owned row, chain), lane <-> class; the S partials are
      // summed in rank order.
      const float* zsl = zx + size_t(slot) * S * RS * N;
      const uint32_t zsl_s = smem_u32(zsl);
      // Four (row, chain) tasks per warp in flight at once, so their load,
      // shuffle and exp latencies overlap.
      constexpr int kG = 4;
      for (int it0 = sw; it0 < RS * chains; it0 += 8 * kG) {
        float z[kG], mx[kG], se[kG], e[kG], zy[kG];
        int yi[kG], cb[kG], il[kG];
        bool act[kG];
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          const int it = it0 + 8 * g;
          act[g] = it < RS * chains;
          il[g] = act[g] ? it / chains : 0;
          const int c = act[g] ? it - il[g] * chains : 0;
          cb[g] = c * Km1;
          yi[g] = act[g] ? ylab[il[g]] : -1;
        }
        // The S partials of each logit, summed in rank order.
#pragma unroll
        for (int g = 0; g < kG; ++g) z[g] = 0.f;
#pragma unroll
        for (int pr = 0; pr < 16; ++pr)
          if (pr < S)
#pragma unroll
            for (int g = 0; g < kG; ++g)
              if (act[g] && lane < Km1) {
                float t;
                asm volatile("ld.shared.f32 %0, [%1];" : "=f"(t) : "r"(zsl_s + uint32_t(((pr * RS + il[g]) * N + cb[g] + lane) * 4)));
                z[g] += t;
              }
        // With the zero logit of class K the row maximum includes 0 and the sum
        // e^{-m}; without it (unconstrained layout) only the Km1 free logits count.
#pragma unroll
        for (int g = 0; g < kG; ++g) mx[g] = (lane < Km1) ? (zl ? fmaxf(z[g], 0.f) : z[g]) : (zl ? 0.f : -INFINITY);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int g = 0; g < kG; ++g) mx[g] = fmaxf(mx[g], __shfl_xor_sync(0xffffffffu, mx[g], o));
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          e[g] = (lane < Km1) ? expf(z[g] - mx[g]) : 0.f;
          se[g] = e[g];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int g = 0; g < kG; ++g) se[g] += __shfl_xor_sync(0xffffffffu, se[g], o);
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          if (zl) se[g] += expf(-mx[g]);
          const bool valid = yi[g] >= 0;
          zy[g] = __shfl_sync(0xffffffffu, z[g], (valid && yi[g] < Km1) ? yi[g] : 0);
          if (act[g] && lane < Km1)
            rloc[il[g] * NP + cb[g] + lane] =
                __float2bfloat16_rn(valid ? ((lane == yi[g] ? 1.f : 0.f) - e[g] / se[g]) : 0.f);
          if (act[g] && lane == 0 && valid)
            lacc[il[g] * chains + (cb[g] / Km1)] += double((yi[g] < Km1 ? zy[g] : 0.f) - mx[g] - logf(se[g]));
        }
      }
      // The partials of tile u are consumed: peers may push tile u + 1.
      named_bar_soft();
      if (sw == 1 && lane < S)
        mbar_arrive_remote(S > 1 ? map_peer(smem_u32(&zxfree[slot]), uint32_t(lane)) : smem_u32(&zxfree[slot]));
      // R buffer b = u % rbufs: every CTA's gradient sweep of tile u - rbufs
      // must be done reading it.
      const int rbi = int(u % RBUFS);
      bool fok = true;
      if (u >= RBUFS && st == 0) {
        fok = wait_bounded(&rfreec[rbi], uint32_t(((u - RBUFS) / RBUFS) & 1), A.spin_limit, abort_flag, true);
        if (!fok) fail(ERR_TIMEOUT_EXCHANGE);
      }
      if (!named_bar_soft_and(fok && !*abort_flag)) break;
      // Push the owned R rows into every peer's operand buffer (MN-major,
      // 128-byte swizzle: 16-byte chunk j of row r sits at chunk j ^ (r % 8)).
      for (int it = st; it < RS * C8 * S; it += kSoftThreads) {
        const int peer = it % S, rest = it / S;
        const int c8 = rest % C8, il = rest / C8;
        const int r = int(rank) * RS + il;
        uint4 v;
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "r"(smem_u32(rloc + il * NP + c8 * 8)));
        const uint32_t off = uint32_t((c8 >> 3) * kBoxBytes + r * 128 + (((c8 & 7) ^ (r & 7)) << 4));
        const uint32_t la = rb_local + uint32_t(rbi * rbuf_bytes) + off;
        const uint32_t ra = (S > 1) ? map_peer(la, uint32_t(peer)) : la;
        const uint32_t rbar = (S > 1) ? map_peer(smem_u32(&rfull[rbi]), uint32_t(peer)) : smem_u32(&rfull[rbi]);
        st_async_v4f(ra, __uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z), __uint_as_float(v.w), rbar);
      }
    }
    named_bar_soft();
    if (sw == 0)
      for (int c = lane; c < chains; c += 32) {
        double sum = 0.0;
        for (int il = 0; il < RS; ++il) sum += lacc[il * chains + c];
        A.lpart[(size_t(cl) * S + rank) * A.lpart_cstride + c] = sum;
      }
  }
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    tmem_dealloc(tmem, A.tmem_cols);
  }
  if (S > 1) cluster_sync_all();
}

template <bool kFP8>
__global__ void __launch_bounds__(kFP8 ? kThreadsFp8 : kThreadsBf16, 1) lpg_tc_kernel(const TcArgs A) {
  tc_body<kFP8>(A, int(blockIdx.x) / A.S);
}

// Several independent problems in one launch: clusters [first[b], first[b+1])
// of the grid work on problem b with its own arguments (X, labels, operand
// boxes, tile plan, partial slots); every problem shares the cluster size and
// the storage type.  `chains` is the call's chain count.
template <bool kFP8>
__global__ void __launch_bounds__(kFP8 ? kThreadsFp8 : kThreadsBf16, 1)
    lpg_tc_kernel_batched(const TcArgs* __restrict__ table, const int* __restrict__ first, int nprob, int chains) {
  __shared__ TcArgs args;
  __shared__ int cl_local;
  if (threadIdx.x == 0) {
    const int gcl = int(blockIdx.x) / table[0].S;
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
  tc_body<kFP8>(args, cl_local);
}

// Coefficients of every problem of a batch into their operand boxes: block
// row b (blockIdx.y) converts problem b.
struct BetaTiles {
  const float* beta;
  const float* scales;
  __nv_bfloat16* out;
  int32_t Km1, N, p_pad;
};

// Byte offset of element (row r, column c) of a 128-byte-swizzled box whose
// rows hold 64 BF16 values: 16-byte chunk (c / 8) is stored at chunk
// (c / 8) ^ (r % 8).
__host__ __device__ inline uint32_t sw128_offset(int r, int c) {
  return uint32_t(r) * 128u + uint32_t(((c >> 3) ^ (r & 7)) << 4) + uint32_t((c & 7) * 2);
}

// X (row-major n x p, float or double) -> BF16 boxes of 128 rows x 64 columns
// in their shared-memory image, [n_pad / 128][p_pad / 64][16 KB]; padding zero.
template <typename IT>
__global__ void x_to_tiles_kernel(const IT* X, __nv_bfloat16* out, int64_t n, int32_t p, int32_t p_pad, int64_t n_pad,
                                  int* err) {
  const int64_t total = n_pad * p_pad;
  const int64_t nkb = p_pad / kBox;
  int bad = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = i / p_pad, col = i - row * p_pad;
    float v = 0.f;
    if (row < n && col < p) {
      const IT x = X[row * p + col];
      if (!isfinite(double(x))) bad = 1;
      v = float(x);
    }
    const int64_t t = row / kRows, kb = col / kBox;
    const size_t off = size_t(t * nkb + kb) * kBoxBytes + sw128_offset(int(row % kRows), int(col % kBox));
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(out) + off) = __float2bfloat16_rn(v);
  }
  if (bad) atomicOr(err, ERR_NONFINITE_X);
}

// X (row-major n x p, float or double) -> FP8 E4M3 boxes of 128 rows x 64
// columns, row-major inside a box, [n_pad / 128][p_pad / 64][8 KB]: x_q =
// RNE-satfinite(x / s_j), the per-column scale s_j computed beforehand.
template <typename IT>
__global__ void x_to_tiles_fp8_kernel(const IT* X, const float* scales, unsigned char* out, int64_t n, int32_t p,
                                      int32_t p_pad, int64_t n_pad, int* err) {
  const int64_t total = n_pad * p_pad;
  const int64_t nkb = p_pad / kBox;
  int bad = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = i / p_pad, col = i - row * p_pad;
    unsigned char q = 0;
    if (row < n && col < p) {
      const IT x = X[row * p + col];
      if (!isfinite(double(x))) bad = 1;
      q = static_cast<unsigned char>(__nv_cvt_float_to_fp8(float(x) / scales[col], __NV_SATFINITE, __NV_E4M3));
    }
    const int64_t t = row / kRows, kb = col / kBox;
    out[size_t(t * nkb + kb) * kFp8BoxBytes + size_t(row % kRows) * 64 + size_t(col % kBox)] = q;
  }
  if (bad) atomicOr(err, ERR_NONFINITE_X);
}

__global__ void fp8_tiles_to_rows_kernel(const unsigned char* tiles, unsigned char* out, int64_t n, int32_t p,
                                         int32_t p_pad) {
  const int64_t total = n * p;
  const int64_t nkb = p_pad / kBox;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = i / p, col = i - row * p;
    const int64_t t = row / kRows, kb = col / kBox;
    out[i] = tiles[size_t(t * nkb + kb) * kFp8BoxBytes + size_t(row % kRows) * 64 + size_t(col % kBox)];
  }
}

// Inverse of x_to_tiles for the stored values (BF16 bits, row-major n x p).
__global__ void tiles_to_rows_kernel(const __nv_bfloat16* tiles, uint16_t* out, int64_t n, int32_t p, int32_t p_pad) {
  const int64_t total = n * p;
  const int64_t nkb = p_pad / kBox;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = i / p, col = i - row * p;
    const int64_t t = row / kRows, kb = col / kBox;
    const size_t off = size_t(t * nkb + kb) * kBoxBytes + sw128_offset(int(row % kRows), int(col % kBox));
    out[i] = *reinterpret_cast<const uint16_t*>(reinterpret_cast<const unsigned char*>(tiles) + off);
  }
}

// Coefficient value v of class row k, column col -> its two BF16 terms in the
// operand box of column block col / 64: rows [0, N) hold hi = bf16(v), rows
// [N, 2N) hold lo = bf16(v - hi), so hi + lo carries v to about 16 bits and the
// logits X (hi + lo)^T lose nothing to the rounding of the coefficients.
__device__ __forceinline__ void put_coef(unsigned char* out, int N, int k, int64_t col, float v) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
  const size_t box = size_t(col / kBox) * 2 * N * 128;
  *reinterpret_cast<__nv_bfloat16*>(out + box + sw128_offset(k, int(col % kBox))) = hi;
  *reinterpret_cast<__nv_bfloat16*>(out + box + sw128_offset(N + k, int(col % kBox))) = lo;
}

// FP32 coefficients [C][p_pad] -> BF16 operand boxes [p_pad / 64][2N rows x 128 B]
// (hi rows then lo rows; rows C..N-1 of each zero), K-major with the 128-byte
// swizzle.  With FP8 X the column scales are folded in: X B = X_q (diag(s) B).
__global__ void beta_to_tiles_kernel(const float* beta, const float* scales, __nv_bfloat16* out, int C, int N,
                                     int p_pad) {
  const int64_t total = int64_t(N) * p_pad;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int k = int(i / p_pad);
    const int64_t col = i - int64_t(k) * p_pad;
    const float v = (k < C) ? beta[size_t(k) * p_pad + col] * (scales ? scales[col] : 1.0f) : 0.f;
    put_coef(reinterpret_cast<unsigned char*>(out), N, k, col, v);
  }
}

__global__ void beta_to_tiles_batched_kernel(const BetaTiles* __restrict__ table, int chains) {
  const BetaTiles b = table[blockIdx.y];
  const int C = chains * b.Km1;
  const int64_t total = int64_t(b.N) * b.p_pad;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int k = int(i / b.p_pad);
    const int64_t col = i - int64_t(k) * b.p_pad;
    const float v = (k < C) ? b.beta[size_t(k) * b.p_pad + col] * (b.scales ? b.scales[col] : 1.0f) : 0.f;
    put_coef(reinterpret_cast<unsigned char*>(b.out), b.N, k, col, v);
  }
}

}  // namespace tc

// Plan: N = C rounded to 16, MB = PC / 128, TMEM = N * (1 + MB) <= 512.
bool tc_plan(int64_t p, int C, int S, TcPlan* out) {
  const int N = std::max(16, (C + 15) / 16 * 16);
  if (N > 256) return false;
  const int PC = int((p + int64_t(128) * S - 1) / (int64_t(128) * S) * 128);
  const int MB = PC / 128;
  if (N * (1 + MB) > 512) return false;
  // As many logit accumulators as TMEM holds next to the gradient slice.
  const int nz = std::max(1, std::min(kTcMaxDepth, (512 - N * MB) / N));
  const int cols = N * (nz + MB);
  uint32_t tcols = 32;
  while (tcols < uint32_t(cols)) tcols <<= 1;
  out->nz = nz;
  out->slots = out->rbufs = out->la = 1;
  out->N = N;
  out->NP = (N + 63) / 64 * 64;
  out->PC = PC;
  out->MB = MB;
  out->S = S;
  out->tmem_cols = tcols;
  out->stage_bytes = uint32_t(tc::al(size_t(tc::kBoxBytes) + std::max<size_t>(tc::kBoxBytes, size_t(2 * N) * 128), 1024));
  return true;
}

size_t tc_smem_bytes(const TcPlan& pl, int NST, int chains, bool fp8) {
  return tc::smem_layout(NST, pl.stage_bytes, pl.NP, pl.N, pl.S, chains, fp8, pl.slots, pl.rbufs).total;
}

static void (*tc_kernel(bool fp8))(const tc::TcArgs) { return fp8 ? tc::lpg_tc_kernel<true> : tc::lpg_tc_kernel<false>; }
using TcBatchedFn = void (*)(const tc::TcArgs*, const int*, int, int);
static TcBatchedFn tc_kernel_batched(bool fp8) {
  return fp8 ? tc::lpg_tc_kernel_batched<true> : tc::lpg_tc_kernel_batched<false>;
}

int tc_threads(bool fp8) { return fp8 ? tc::kThreadsFp8 : tc::kThreadsBf16; }

cudaError_t tc_prepare(size_t smem, int S, bool fp8) {
  cudaError_t e = cudaFuncSetAttribute(tc_kernel(fp8), cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  if (S > 8) e = cudaFuncSetAttribute(tc_kernel(fp8), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t tc_max_active_clusters(size_t smem, int S, bool fp8, int* out) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(S, 1, 1);
  cfg.blockDim = dim3(tc_threads(fp8), 1, 1);
  cfg.dynamicSmemBytes = smem;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(out, tc_kernel(fp8), &cfg);
}

cudaError_t tc_x_to_tiles(int in_dtype, const void* X, void* out, int64_t n, int32_t p, int32_t p_pad, int* err,
                          cudaStream_t s) {
  const int64_t n_pad = (n + tc::kRows - 1) / tc::kRows * tc::kRows;
  const int g = std::max(1, int(std::min<int64_t>(8192, (n_pad * p_pad + 255) / 256)));
  if (in_dtype == HMC_F64)
    tc::x_to_tiles_kernel<double><<<g, 256, 0, s>>>(static_cast<const double*>(X), static_cast<__nv_bfloat16*>(out), n,
                                                    p, p_pad, n_pad, err);
  else
    tc::x_to_tiles_kernel<float><<<g, 256, 0, s>>>(static_cast<const float*>(X), static_cast<__nv_bfloat16*>(out), n,
                                                   p, p_pad, n_pad, err);
  return cudaGetLastError();
}

cudaError_t tc_x_to_tiles_fp8(int in_dtype, const void* X, const float* scales, void* out, int64_t n, int32_t p,
                              int32_t p_pad, int* err, cudaStream_t s) {
  const int64_t n_pad = (n + tc::kRows - 1) / tc::kRows * tc::kRows;
  const int g = std::max(1, int(std::min<int64_t>(8192, (n_pad * p_pad + 255) / 256)));
  if (in_dtype == HMC_F64)
    tc::x_to_tiles_fp8_kernel<double><<<g, 256, 0, s>>>(static_cast<const double*>(X), scales,
                                                        static_cast<unsigned char*>(out), n, p, p_pad, n_pad, err);
  else
    tc::x_to_tiles_fp8_kernel<float><<<g, 256, 0, s>>>(static_cast<const float*>(X), scales,
                                                       static_cast<unsigned char*>(out), n, p, p_pad, n_pad, err);
  return cudaGetLastError();
}

cudaError_t tc_tiles_to_rows(const void* tiles, void* out_bits, int64_t n, int32_t p, int32_t p_pad, bool fp8,
                             cudaStream_t s) {
  const int g = std::max(1, int(std::min<int64_t>(8192, (n * p + 255) / 256)));
  if (fp8)
    tc::fp8_tiles_to_rows_kernel<<<g, 256, 0, s>>>(static_cast<const unsigned char*>(tiles),
                                                   static_cast<unsigned char*>(out_bits), n, p, p_pad);
  else
    tc::tiles_to_rows_kernel<<<g, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(tiles),
                                              static_cast<uint16_t*>(out_bits), n, p, p_pad);
  return cudaGetLastError();
}

cudaError_t tc_beta_to_tiles(const float* beta, const float* scales, void* out, int C, int N, int p_pad,
                             cudaStream_t s) {
  const int64_t total = int64_t(N) * p_pad;
  const int g = std::max(1, int(std::min<int64_t>(4096, (total + 255) / 256)));
  tc::beta_to_tiles_kernel<<<g, 256, 0, s>>>(beta, scales, static_cast<__nv_bfloat16*>(out), C, N, p_pad);
  return cudaGetLastError();
}

static tc::TcArgs make_args(const TcPlan& pl, const TcLaunch& L) {
  tc::TcArgs a{};
  a.xs = L.xs;
  a.xscale = L.xscale;
  a.fp8 = L.fp8;
  a.bs = static_cast<const __nv_bfloat16*>(L.bs);
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
  a.y = L.y;
  a.err = L.err;
  a.spin_limit = L.spin_limit;
  a.inject_timeout = L.inject_timeout;
  a.zlogit = L.zlogit;
  a.nz = pl.nz;
  a.slots = pl.slots;
  a.rbufs = pl.rbufs;
  a.la = pl.la;
  return a;
}

static void tc_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int clusters, int S, bool fp8, size_t smem,
                      cudaStream_t stream) {
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3(clusters * S, 1, 1);
  cfg.blockDim = dim3(tc_threads(fp8), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

cudaError_t tc_launch(const TcPlan& pl, const TcLaunch& L, size_t smem, cudaStream_t stream) {
  const tc::TcArgs a = make_args(pl, L);
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  tc_config(cfg, attr, L.nclusters, pl.S, L.fp8 != 0, smem, stream);
  return cudaLaunchKernelEx(&cfg, tc_kernel(L.fp8 != 0), a);
}

// ---- one launch for several problems
cudaError_t tc_prepare_batched(size_t smem, int S, bool fp8) {
  cudaError_t e = cudaFuncSetAttribute(tc_kernel_batched(fp8), cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  if (S > 8) e = cudaFuncSetAttribute(tc_kernel_batched(fp8), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t tc_max_active_clusters_batched(size_t smem, int S, bool fp8, int* out) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  tc_config(cfg, attr, 1, S, fp8, smem, nullptr);
  return cudaOccupancyMaxActiveClusters(out, tc_kernel_batched(fp8), &cfg);
}

cudaError_t tc_upload_batch(const TcPlan* plans, const TcLaunch* launches, int m, void** d_table) {
  std::vector<tc::TcArgs> t(m);
  for (int b = 0; b < m; ++b) t[b] = make_args(plans[b], launches[b]);
  cudaError_t e = cudaMalloc(d_table, size_t(m) * sizeof(tc::TcArgs));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*d_table, t.data(), size_t(m) * sizeof(tc::TcArgs), cudaMemcpyHostToDevice);
}

cudaError_t tc_upload_beta_table(const TcBetaBox* boxes, int m, void** d_table) {
  std::vector<tc::BetaTiles> t(m);
  for (int b = 0; b < m; ++b)
    t[b] = tc::BetaTiles{boxes[b].beta, boxes[b].scales, static_cast<__nv_bfloat16*>(boxes[b].out), boxes[b].Km1,
                         boxes[b].N, boxes[b].p_pad};
  cudaError_t e = cudaMalloc(d_table, size_t(m) * sizeof(tc::BetaTiles));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*d_table, t.data(), size_t(m) * sizeof(tc::BetaTiles), cudaMemcpyHostToDevice);
}

int tc_beta_job_bytes() { return int(sizeof(tc::BetaTiles)); }

cudaError_t tc_beta_to_tiles_batched(const void* d_table, int m, int chains, int64_t max_elems, cudaStream_t s) {
  const int gx = std::max(1, int(std::min<int64_t>(512, (max_elems + 255) / 256)));
  tc::beta_to_tiles_batched_kernel<<<dim3(gx, m), 256, 0, s>>>(static_cast<const tc::BetaTiles*>(d_table), chains);
  return cudaGetLastError();
}

cudaError_t tc_launch_batched(const void* d_table, const int* d_first, int m, int chains, int total_clusters, int S,
                              bool fp8, size_t smem, cudaStream_t stream) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  tc_config(cfg, attr, total_clusters, S, fp8, smem, stream);
  return cudaLaunchKernelEx(&cfg, tc_kernel_batched(fp8), static_cast<const tc::TcArgs*>(d_table), d_first, m, chains);
}

}  // namespace hmc
