// Two-pass evaluation of the log-posterior and its gradient on the tensor
// cores (tcgen05), X stored in BF16 (Eqs. softmax, loglike, logkernel and
// gradient of Sec. 2.1, for C = chains*(K-1) coefficient columns at once).
//
// The fused engine (lpg_tc.cu) keeps each CTA's gradient slice in TMEM for the
// whole pass, which caps the chains of one launch (TMEM holds p/16 x N FP32
// values per SM) and ties the CTAs of a cluster together through a logit
// exchange every row tile.  Here the two contractions run as two streaming
// passes with nothing held across tiles but the accumulators of one unit:
//
//  pass A  (logits, softmax, residual)  units (U consecutive row tiles of 128
//          rows, chain group g): D_i[128 x N] = X_{t_i} B_g^T over all p
//          features for the U tiles, B as two BF16 terms (hi + lo, ~16 bits)
//          that every tile of the unit takes from the same ring slot (U X
//          boxes + one coefficient box per 64 features: the coefficient bytes
//          per X byte fall as U grows), accumulated in TMEM (two sets of U
//          accumulators, so the epilogue of one unit overlaps the MMAs of the
//          next).  The units' feature boxes are split evenly over the CTAs
//          (each CTA takes the same number of (unit, 64-feature box) steps,
//          so a unit may start on one CTA and end on the next): the CTA that
//          holds a unit's first boxes finishes it, adding in the partial
//          logits its neighbour stored for the unit's last boxes (a fixed sum
//          order, a release/acquire flag per CTA).  The
//          epilogue (one thread per row) forms the softmax of every chain with
//          the zero logit of class K, the row log-likelihood and the residual
//          R = Y - P, which it writes in BF16 as the MN-major, 128-byte-swizzled
//          boxes pass B reads.  Every CTA adds its units' log-likelihoods per
//          chain in unit order: one FP64 partial per CTA and chain.
//  pass B  (gradient X^T R)  units (feature group f of MB blocks of 128
//          features, chain group g, row range q): D[mb][128 features x N] +=
//          X_blk^T R over the tiles of the range, one TMEM accumulator per
//          feature block; written once at the end as the range's partial slice
//          (fixed-order reduction afterwards, no atomics).
//
// X crosses HBM twice per gradient when it is larger than L2 (once when the
// second pass finds it in L2); in exchange every SM streams (no cluster
// exchange, no TMEM limit on the chains of one call) and both passes are
// balanced over the SM count.
//
// Warp roles in both kernels: warp 0 bulk-copy producer (lane 0), warp 1 TMEM
// owner and MMA issuer (lane 0), then the epilogue warps: pass A two per TMEM
// lane quarter for BF16 X (warps 2-9, quarter warp % 4, half (warp - 2) / 4:
// the softmax of one row is a serial chain, so a second warp per scheduler
// hides its latency), one for FP8 X (warps 2-5); pass B one per quarter (warps
// 2-5); with FP8 X, eight converter warps follow in both kernels.  Every wait
// is bounded; a wait that runs out sets an error bit and an abort flag, and
// every role then leaves its loop.
#include <algorithm>
#include <vector>

#include "internal.h"
#include "tc_common.cuh"

namespace hmc {
namespace tc2 {

using tc::fence_after_sync;
using tc::fence_before_sync;
using tc::idesc_bf16;
using tc::mma_bf16;
using tc::mma_commit;
using tc::smem_desc;
using tc::tmem_alloc;
using tc::tmem_dealloc;
using tc::tmem_ld16;

constexpr int kRows = 128;
constexpr int kBox = 64;                 // BF16 values per 128-byte row of a box
constexpr int kBoxBytes = kRows * 128;   // one 128 x 64 BF16 box
constexpr int kMaxCols = 256;            // accumulator columns of one row tile (chains x classes of a group), at most
// Pass A: epilogue warps per TMEM lane quarter, two for BF16 X, one for FP8 X
// (whose eight converter warps need the registers).
__host__ __device__ constexpr int epi_halves(bool fp8) { return fp8 ? 1 : 2; }
constexpr int kConvWarps = 8;                      // FP8 X: converter warps (both passes)
constexpr int kConvThreads = 32 * kConvWarps;
// Converter groups taking alternate ring steps: one in pass A (its steps carry
// U boxes), two in pass B (two boxes a step) -- measured on n=5e4 p=1e4 K=20:
// pass A 383 us with one group against 402-445 with two, pass B 250-259 with
// two against 296 with one.
constexpr int kConvGroupsA = 1, kConvGroupsB = 2;
constexpr int kFp8BoxBytes = kRows * 64;           // FP8 box: 128 rows x 64 E4M3 codes, row-major
// Blocks: pass A producer, MMA issuer, epilogue warps [, converters]; pass B
// producer, MMA issuer, four drain warps [, converters].
__host__ __device__ constexpr int threads_a(bool fp8) { return 64 + 128 * epi_halves(fp8) + (fp8 ? kConvThreads : 0); }
__host__ __device__ constexpr int threads_b(bool fp8) { return 192 + (fp8 ? kConvThreads : 0); }

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, long long limit, volatile int* abort) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < limit; ++i) {
    if (mbar_test_cta(a, parity)) return true;
    if ((i & 63) == 63 && *abort) return false;
  }
  return false;
}

// Bounded wait that does not give up on the abort flag: used where a role must
// see its own bulk copies or MMAs complete before shared memory or TMEM is
// released, also on the error path.
__device__ __forceinline__ void wait_drain(uint64_t* bar, uint32_t parity, long long limit) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < limit; ++i)
    if (mbar_test_cta(a, parity)) return;
}

// Pass A's epilogue barrier over its T threads.
template <int T>
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(T) : "memory"); }
// The same barrier, ANDing a flag over the epilogue threads (so every
// epilogue warp leaves its loop at the same unit).
template <int T>
__device__ __forceinline__ bool epi_bar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.and.pred po, 1, %2, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"(v ? 1u : 0u), "n"(T)
      : "memory");
  return r != 0;
}

// Whole warp: store 16 consecutive 32-bit columns of this warp's 32 TMEM lanes
// (one lane per thread); tmem_st_wait() waits for this thread's stores.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Predicated shared-memory store and load (PTX predicates, so a sweep over a
// row's columns has no branch at a chain's last column).
__device__ __forceinline__ void st_shared_if(float* p, float v, bool pred) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.f32 [%0], %1;\n\t}" ::"r"(smem_u32(p)),
               "f"(v), "r"(uint32_t(pred))
               : "memory");
}
__device__ __forceinline__ float ld_shared_if(const float* p, float old, bool pred) {
  float v = old;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.shared.f32 %0, [%1];\n\t}"
               : "+f"(v)
               : "r"(smem_u32(p)), "r"(uint32_t(pred))
               : "memory");
  return v;
}

// Bits e of a 16-column block whose column offset lies in [lo, hi).
__device__ __forceinline__ uint32_t col_bits(int lo, int hi) {
  lo = max(lo, 0);
  hi = min(hi, 16);
  return hi > lo ? ((1u << hi) - 1u) & ~((1u << lo) - 1u) : 0u;
}

// (hi, lo) += (bh, bl) for unevaluated float pairs (value hi + lo, |lo| below
// half an ulp of hi): Knuth's TwoSum of the leading parts, the trailing parts
// and the rounding error added, and a Dekker FastTwoSum renormalisation.  Row
// log-likelihood sums carried this way keep about twice FP32's precision
// without FP64 arithmetic, which this part runs at a small fraction of FP32's rate.
__device__ __forceinline__ void add_pair(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float bv = s - hi;
  const float e = (hi - (s - bv)) + (bh - bv);
  const float t = e + (lo + bl);
  hi = s + t;
  lo = t - (hi - s);
}

// The barrier of FP8 converter group cg of T threads (named barrier 2 + cg),
// and the same barrier ANDing a flag over the group (so all its warps leave
// their loop together).
template <int T>
__device__ __forceinline__ void conv_bar(int cg) {
  asm volatile("bar.sync %0, %1;" ::"r"(2 + cg), "n"(T) : "memory");
}
template <int T>
__device__ __forceinline__ bool conv_bar_and(int cg, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.and.pred po, %2, %3, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"(v ? 1u : 0u), "r"(2 + cg), "n"(T)
      : "memory");
  return r != 0;
}

// Widen nbox FP8 boxes (128 x 64 E4M3 codes, row-major) that landed in the
// upper halves of `slot`'s BF16 box areas (box i's codes at i * in_stride +
// in_off) into the 128-byte-swizzled BF16 boxes the MMAs read (box i at
// i * kBoxBytes of `slot`), exactly (every E4M3 value is a BF16 value).  Every
// converter thread reads all its input chunks before the group barrier and
// writes only after it, so the in-place widening never overwrites unread
// input.  cg: converter group of T threads, ct: thread index within it.
template <int kMaxBoxes, int T>
__device__ __forceinline__ void widen_fp8_boxes(unsigned char* slot, int nbox, uint32_t in_stride, uint32_t in_off,
                                                int cg, int ct) {
  constexpr int kGroupThreads = T;
  constexpr int kChunks = kFp8BoxBytes / 16;                  // 16-byte input chunks per box
  constexpr int kPer = kMaxBoxes * kChunks / kGroupThreads;   // chunks per thread at most
  uint4 w[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int g = ct + kGroupThreads * i;
    if (g < nbox * kChunks)
      w[i] = *reinterpret_cast<const uint4*>(slot + size_t(g / kChunks) * in_stride + in_off + size_t(g % kChunks) * 16);
  }
  conv_bar<T>(cg);
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int g = ct + kGroupThreads * i;
    if (g >= nbox * kChunks) break;
    const int bx = g / kChunks, ci = g % kChunks;
    const int r = ci >> 2, qq = ci & 3;                      // row, 16-code quarter of the row
    uint32_t o[8];
    fp8x4_to_bf16x4(w[i].x, o[0], o[1]);
    fp8x4_to_bf16x4(w[i].y, o[2], o[3]);
    fp8x4_to_bf16x4(w[i].z, o[4], o[5]);
    fp8x4_to_bf16x4(w[i].w, o[6], o[7]);
    unsigned char* rowp = slot + size_t(bx) * kBoxBytes + size_t(r) * 128;
    *reinterpret_cast<uint4*>(rowp + (((2 * qq) ^ (r & 7)) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<uint4*>(rowp + (((2 * qq + 1) ^ (r & 7)) << 4)) = make_uint4(o[4], o[5], o[6], o[7]);
  }
  fence_proxy_async_smem();
}

__host__ __device__ inline size_t al(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ------------------------------------------------------------------ pass A
struct LogitArgs {
  const unsigned char* xs;   // X boxes [ntiles][nkb][16 KB BF16 | 8 KB FP8 codes]
  const unsigned char* bs;   // coefficient operand [ngroups][nkb][2N rows x 128 B] (hi rows, then lo rows)
  const int32_t* y;
  unsigned char* rout;       // R boxes [ntiles][ngroups][NB][16 KB]
  double* lpart;             // [gridDim.x][lpart_cstride]: this CTA's log-likelihood per chain
  int32_t lpart_cstride;
  int* err;
  int64_t n, ntiles;
  int32_t nkb, N, NB, Km1, zlogit, gc, ngroups, chains, NST;
  int32_t U;                 // row tiles per unit
  uint32_t stage_bytes, tmem_cols;
  long long spin_limit;
  float* spart;              // [gridDim.x][U][N][128]: partial logits of a unit's last boxes (split units)
  int* sflag;                // [gridDim.x]: 1 while the CTA's stored partial waits to be added
};

// One stretch of a CTA's feature-box steps: unit u, boxes [k0, k1).
struct Seg {
  int64_t u;
  int k0, k1;
};
__device__ __forceinline__ bool next_seg(int64_t& pos, int64_t end, int nkb, Seg& sg) {
  if (pos >= end) return false;
  sg.u = pos / nkb;
  sg.k0 = int(pos - sg.u * nkb);
  sg.k1 = int(min(int64_t(nkb), int64_t(sg.k0) + (end - pos)));
  pos += sg.k1 - sg.k0;
  return true;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct LogitSmem {
  size_t ring, mx, sm, zy, llr, llc, tab, bars, total;
};

__host__ __device__ inline LogitSmem logit_smem(int NST, uint32_t stage_bytes, int gc, int chains) {
  LogitSmem L;
  size_t off = 0;
  L.ring = off;  off = al(off + size_t(NST) * stage_bytes, 1024);
  L.mx = off;    off = al(off + size_t(gc) * kRows * 4, 16);
  L.sm = off;    off = al(off + size_t(gc) * kRows * 4, 16);
  L.zy = off;    off = al(off + size_t(gc) * kRows * 4, 16);
  L.llr = off;   off = al(off + size_t(gc) * 4 * 8, 16);
  L.llc = off;   off = al(off + size_t(chains) * 8, 16);
  L.tab = off;   off = al(off + size_t(kMaxCols + kMaxCols / 16) * 4, 16);
  // full, empty [NST]; zdone, zfree [2]; mdrain; TMEM slot; abort flag; (pad); conv [NST]
  L.bars = off;  off = al(off + size_t(3 * NST + 8) * 8 + 16, 16);
  L.total = off + 1024;   // slack for aligning the dynamic base to 1024
  return L;
}

template <bool kFP8>
__global__ void __launch_bounds__(threads_a(kFP8), 1) logits_kernel(const LogitArgs A) {
  constexpr int kEpiHalves = epi_halves(kFP8);
  constexpr int kEpiThreads = 128 * kEpiHalves;
  constexpr int kFold = kFP8 ? 1 : 3;           // partial-logit blocks in flight when folding (no spills)
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = A.N, NST = A.NST, Km1 = A.Km1, gc = A.gc;
  const bool zl = A.zlogit != 0;
  const LogitSmem Lo = logit_smem(NST, A.stage_bytes, gc, A.chains);
  unsigned char* ring = smem + Lo.ring;
  float* s_m = reinterpret_cast<float*>(smem + Lo.mx);     // [gc][128] maximum logit of each chain, then its log-normaliser
  float* s_s = reinterpret_cast<float*>(smem + Lo.sm);     // [gc][128] sum of shifted exponentials
  float* s_zy = reinterpret_cast<float*>(smem + Lo.zy);    // [gc][128] logit of the observed class
  float2* s_wsum = reinterpret_cast<float2*>(smem + Lo.llr);  // [gc][4] log-likelihood sums of each warp's rows (pairs)
  float2* s_llc = reinterpret_cast<float2*>(smem + Lo.llc);   // [chains] this CTA's sums (pairs)
  int* s_cm = reinterpret_cast<int*>(smem + Lo.tab);          // [N] column j: chain c * 128 | class k << 16
  uint32_t* s_cend = reinterpret_cast<uint32_t*>(s_cm + kMaxCols);  // [N / 16] bit e: column 16b + e ends a chain
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lo.bars);
  uint64_t* full = bars;
  uint64_t* empty = bars + NST;
  uint64_t* zdone = bars + 2 * NST;      // [2] accumulator a holds a finished unit
  uint64_t* zfree = zdone + 2;           // [2] accumulator a drained
  uint64_t* mdrain = zfree + 2;          // every MMA of this CTA complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdrain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(mdrain + 2);
  uint64_t* conv = mdrain + 4;           // FP8: [NST] ring slot widened to BF16 (one group's warps arrive)

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&zdone[a], 1);
      mbar_init(&zfree[a], kEpiThreads / 32);
    }
    mbar_init(mdrain, 1);
    if (kFP8)
      for (int s = 0; s < NST; ++s) mbar_init(&conv[s], kConvWarps / kConvGroupsA);
    *abort_flag = 0;
    fence_mbar_init_cluster();
  }
  for (int c = tid; c < A.chains; c += int(blockDim.x)) s_llc[c] = make_float2(0.f, 0.f);
  for (int j = tid; j < N; j += int(blockDim.x)) {
    const int c = j / Km1;   // columns past the group's last chain point at chain gc - 1 (masked where read)
    s_cm[j] = min(c, gc - 1) * kRows | (j - c * Km1) << 16;
  }
  for (int b = tid; b < N / 16; b += int(blockDim.x)) {
    uint32_t m = 0;
    for (int e = 0; e < 16; ++e) m |= ((16 * b + e + 1) % Km1 == 0 ? 1u : 0u) << e;
    s_cend[b] = m;
  }
  if (warp == 1) tmem_alloc(tmem_slot, A.tmem_cols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int U = A.U;
  const int64_t ntg = (A.ntiles + U - 1) / U;       // tile groups
  const int64_t units = ntg * A.ngroups;
  const int64_t G = gridDim.x;
  // This CTA's (unit, feature box) steps: an even share of all of them.  The
  // host launches G <= units CTAs, so a share spans at least one unit's boxes and
  // a unit is split over at most two CTAs.
  const int64_t W = units * A.nkb;
  const int64_t s_begin = int64_t(blockIdx.x) * W / G, s_end = (int64_t(blockIdx.x) + 1) * W / G;
  auto fail = [&](int bit) {
    *abort_flag = 1;
    atomicOr(A.err, bit);
  };
  const uint32_t coef_bytes = uint32_t(2 * N * 128);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int64_t s = 0, issued = 0, pos = s_begin;
      Seg sg;
      while (!*abort_flag && next_seg(pos, s_end, A.nkb, sg)) {
        const int64_t u = sg.u;
        const int64_t t0 = (u / A.ngroups) * U;
        const int nt = int(min(int64_t(U), A.ntiles - t0));   // tiles of this unit
        const int g = int(u % A.ngroups);
        const unsigned char* bt = A.bs + size_t(g) * A.nkb * coef_bytes;
        for (int kb = sg.k0; kb < sg.k1; ++kb, ++s) {
          const int st = int(s % NST);
          if (!wait_bounded(&empty[st], uint32_t(((s / NST) & 1) ^ 1), A.spin_limit, abort_flag)) {
            fail(ERR_TIMEOUT_STAGE);
            break;
          }
          unsigned char* sp = ring + size_t(st) * A.stage_bytes;
          // BF16 boxes land in place; FP8 boxes in the upper half of each box area
          // (the converter warps widen them in place).
          constexpr uint32_t xbox = kFP8 ? uint32_t(kFp8BoxBytes) : uint32_t(kBoxBytes);
          constexpr uint32_t xoff = kFP8 ? uint32_t(kBoxBytes - kFp8BoxBytes) : 0u;
          mbar_arrive_expect_tx(&full[st], uint32_t(nt) * xbox + coef_bytes);
          for (int i = 0; i < nt; ++i)
            bulk_g2s(sp + size_t(i) * kBoxBytes + xoff, A.xs + (size_t(t0 + i) * A.nkb + kb) * xbox, xbox, &full[st]);
          bulk_g2s(sp + size_t(U) * kBoxBytes, bt + size_t(kb) * coef_bytes, coef_bytes, &full[st]);
          issued = s + 1;
        }
      }
      // Every copy issued must land before shared memory is released.
      for (int64_t q = (issued > NST ? issued - NST : 0); q < issued; ++q)
        wait_drain(&full[q % NST], uint32_t((q / NST) & 1), A.spin_limit);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kRows, N, false, false);
      int64_t s = 0, pos = s_begin;
      Seg sg;
      for (int64_t j = 0; !*abort_flag && next_seg(pos, s_end, A.nkb, sg); ++j) {
        const int a = int(j & 1);
        if (j >= 2 && !wait_bounded(&zfree[a], uint32_t(((j >> 1) - 1) & 1), A.spin_limit, abort_flag)) {
          fail(ERR_TIMEOUT_MMA);
          break;
        }
        fence_after_sync();
        const int64_t u = sg.u;
        const int nt = int(min(int64_t(U), A.ntiles - (u / A.ngroups) * U));
        for (int kb = sg.k0; kb < sg.k1; ++kb, ++s) {
          const int st = int(s % NST);
          if (!wait_bounded(kFP8 ? &conv[st] : &full[st], uint32_t((s / NST) & 1), A.spin_limit, abort_flag)) {
            fail(ERR_TIMEOUT_STAGE);
            break;
          }
          fence_after_sync();
          const uint32_t sa = smem_u32(ring + size_t(st) * A.stage_bytes);
          const uint32_t ba = sa + uint32_t(U * kBoxBytes);
          for (int i = 0; i < nt; ++i) {
            const uint32_t d = tmem + uint32_t((a * U + i) * N);
            const uint32_t xa = sa + uint32_t(i * kBoxBytes);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint64_t ad = smem_desc(xa + 32u * k, 16u, 1024u, 2u);
              const uint64_t bh = smem_desc(ba + 32u * k, 16u, 1024u, 2u);
              const uint64_t bl = smem_desc(ba + uint32_t(N) * 128u + 32u * k, 16u, 1024u, 2u);
              mma_bf16(d, ad, bh, idesc, (kb > sg.k0 || k > 0) ? 1u : 0u);
              mma_bf16(d, ad, bl, idesc, 1u);
            }
          }
          mma_commit(&empty[st]);
        }
        if (*abort_flag) break;
        mma_commit(&zdone[a]);
      }
      // TMEM and shared memory stay allocated until every MMA has completed.
      mma_commit(mdrain);
      wait_drain(mdrain, 0u, A.spin_limit);
    }
  } else if (kFP8 && warp >= 2 + kEpiThreads / 32) {
    // ------------------------------------------------------------ FP8 converters
    // Group cg widens the ring steps s with s % kConvGroups == cg.
    constexpr int kConvGroups = kConvGroupsA, kGroupThreads = kConvThreads / kConvGroupsA;
    const int cv = tid - (64 + kEpiThreads);
    const int cg = cv / kGroupThreads, ct = cv % kGroupThreads;
    int64_t s = 0, pos = s_begin;
    Seg sg;
    bool ok = true;
    while (ok && next_seg(pos, s_end, A.nkb, sg)) {
      const int nt = int(min(int64_t(U), A.ntiles - (sg.u / A.ngroups) * U));
      for (int kb = sg.k0; kb < sg.k1; ++kb, ++s) {
        if (int(s % kConvGroups) != cg) continue;
        const int st = int(s % NST);
        // One thread per group polls the copies' barrier; the group barrier
        // passes the result (and orders the landed bytes) to the others.
        const bool got = ct == 0 ? wait_bounded(&full[st], uint32_t((s / NST) & 1), A.spin_limit, abort_flag) : true;
        if (!conv_bar_and<kGroupThreads>(cg, got && !*abort_flag)) {   // the group agrees before its barrier below
          if (!got) fail(ERR_TIMEOUT_STAGE);
          ok = false;
          break;
        }
        widen_fp8_boxes<4, kGroupThreads>(ring + size_t(st) * A.stage_bytes, nt, uint32_t(kBoxBytes),
                                          uint32_t(kBoxBytes - kFp8BoxBytes), cg, ct);
        __syncwarp();
        if (lane == 0) mbar_arrive_local(&conv[st]);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2-9)
    const int q = warp & 3;
    const int hf = (warp - 2) >> 2;                // which half of the quarter's work
    const int r = 32 * q + lane;                   // tile row = TMEM lane
    const uint32_t tq = tmem + (uint32_t(32 * q) << 16);
    int64_t pos = s_begin;
    Seg sg;
    for (int64_t j = 0; next_seg(pos, s_end, A.nkb, sg); ++j) {
      const int a = int(j & 1);
      bool ok = (lane == 0) ? wait_bounded(&zdone[a], uint32_t((j >> 1) & 1), A.spin_limit, abort_flag) : true;
      if (!ok) fail(ERR_TIMEOUT_MMA);
      if (!epi_bar_and<kEpiThreads>(ok)) break;
      fence_after_sync();
      const int64_t u = sg.u;
      const int64_t t0 = (u / A.ngroups) * U;
      const int nt = int(min(int64_t(U), A.ntiles - t0));
      const int g = int(u % A.ngroups);
      const int nch = min(gc, A.chains - g * gc);   // chains of this group
      const int Cg = nch * Km1;
      // Sweeps 1-2 of half hf take chains [ch0, ch1); sweep 3 takes the 16-column
      // blocks b with b % kEpiHalves == hf.
      const int chm = (nch + kEpiHalves - 1) / kEpiHalves;
      const int ch0 = min(nch, hf * chm), ch1 = min(nch, ch0 + chm);
      const int cb = ch0 * Km1, ce = ch1 * Km1;
      if (sg.k0 > 0) {
        // The last boxes of a unit the previous CTA started: store the partial
        // logits for it and raise this CTA's flag.
        float* pp = A.spart + size_t(blockIdx.x) * U * N * kRows;
        for (int i = 0; i < nt; ++i) {
          const uint32_t acc = tq + uint32_t((a * U + i) * N);
          for (int c0 = 16 * hf; c0 < Cg; c0 += 16 * kEpiHalves) {
            float v[16];
            tmem_ld16(acc + uint32_t(c0), v);
#pragma unroll
            for (int e = 0; e < 16; ++e) pp[(size_t(i) * N + c0 + e) * kRows + r] = v[e];
          }
        }
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive_local(&zfree[a]);
        __threadfence();
        epi_bar<kEpiThreads>();
        if (warp == 2 && lane == 0) st_release(A.sflag + blockIdx.x, 1);
        continue;
      }
      // A unit whose last boxes the next CTA holds: wait for its stored partial.
      const bool head = sg.k1 < A.nkb;
      const float* hp = A.spart + size_t(blockIdx.x + 1) * U * N * kRows;
      if (head) {
        bool got = true;
        if (warp == 2 && lane == 0) {
          got = false;
          for (long long it = 0; it < A.spin_limit && !got; ++it) {
            got = ld_acquire(A.sflag + blockIdx.x + 1) != 0;
            if (!got && (it & 63) == 63 && *abort_flag) break;
          }
          if (!got) fail(ERR_TIMEOUT_EXCHANGE);
        }
        if (!epi_bar_and<kEpiThreads>(got)) break;
        (void)ld_acquire(A.sflag + blockIdx.x + 1);   // every thread's own acquire of the stored partial
      }
      for (int i = 0; i < nt; ++i) {
        const int64_t t = t0 + i;
        const int64_t grow = t * kRows + r;
        const bool valid = grow < A.n;
        const int yv = valid ? __ldg(A.y + grow) : -1;
        const uint32_t acc = tq + uint32_t((a * U + i) * N);
        if (head) {
          // Add the next CTA's partial logits to the accumulator in place (16-column
          // blocks interleaved over the quarter's warps, kFold blocks in flight), so
          // the sweeps below read TMEM only.
          const float* hpi = hp + size_t(i) * N * kRows + r;   // partial of column col: hpi[col * kRows]
          for (int c0 = 16 * hf; c0 < Cg; c0 += 16 * kFold * kEpiHalves) {
            float h[kFold][16], v[16];
#pragma unroll
            for (int j = 0; j < kFold; ++j)
              if (c0 + 16 * kEpiHalves * j < Cg)
#pragma unroll
                for (int e = 0; e < 16; ++e) h[j][e] = hpi[size_t(c0 + 16 * kEpiHalves * j + e) * kRows];
#pragma unroll
            for (int j = 0; j < kFold; ++j)
              if (c0 + 16 * kEpiHalves * j < Cg) {
                const uint32_t ta = acc + uint32_t(c0 + 16 * kEpiHalves * j);
                tmem_ld16(ta, v);
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] += h[j][e];
                tmem_st16(ta, v);
              }
          }
          tmem_st_wait();
          fence_before_sync();
          epi_bar<kEpiThreads>();   // every column of the tile holds the whole unit's logits
          fence_after_sync();
        }
        // Sweeps 1-2 over the half's columns [cb, ce) in order, branch-free: bit e
        // of s_cend marks a chain's last column, where the chain's result is stored
        // (predicated) and the running value restarts.
        // Sweep 1: the maximum of every chain's logits (the zero logit of class K
        // included) and the logit of the observed class (at column d of the chain).
        if (cb < ce) {
          const float m0 = zl ? 0.f : -INFINITY;
          float m = m0, zy = 0.f;
          int ix = ch0 * kRows + r;
          int d = ch0 * Km1 + (yv >= 0 && yv < Km1 ? yv : -32);   // -32: no column of any chain
          for (int c0 = cb & ~15; c0 < ce; c0 += 16) {
            float v[16];
            tmem_ld16(acc + uint32_t(c0), v);
            const uint32_t in = col_bits(cb - c0, ce - c0), ends = s_cend[c0 >> 4] & in;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const bool last = (ends >> e) & 1u;
              m = fmaxf(m, (in >> e) & 1u ? v[e] : -INFINITY);
              zy = c0 + e == d ? v[e] : zy;
              st_shared_if(s_m + ix, m, last);
              st_shared_if(s_zy + ix, zy, last);
              ix += last ? kRows : 0;
              d += last ? Km1 : 0;
              m = last ? m0 : m;
            }
          }
        }
        // Sweep 2: every chain's sum of exponentials shifted by its maximum (the
        // next chain's maximum is loaded one chain ahead).
        if (cb < ce) {
          int ix = ch0 * kRows + r, cn = ch0 + 2;
          float mc = s_m[ix], mn = ch0 + 1 < ch1 ? s_m[ix + kRows] : 0.f, ss = 0.f;
          for (int c0 = cb & ~15; c0 < ce; c0 += 16) {
            float v[16];
            tmem_ld16(acc + uint32_t(c0), v);
            const uint32_t in = col_bits(cb - c0, ce - c0), ends = s_cend[c0 >> 4] & in;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const bool last = (ends >> e) & 1u;
              const float x = expf(v[e] - mc);
              ss += (in >> e) & 1u ? x : 0.f;
              st_shared_if(s_s + ix, ss, last);
              ix += last ? kRows : 0;
              mc = last ? mn : mc;
              mn = ld_shared_if(s_m + cn * kRows + r, mn, last && cn < ch1);
              cn += last ? 1 : 0;
              ss = last ? 0.f : ss;
            }
          }
        }
        // Per chain: the log-normaliser lse = m + log(sum) (the zero logit's term
        // added to the sum last) replaces the maximum, the row's log-likelihood
        // zy - lse replaces the observed logit, and the log-likelihoods are summed
        // over the warp's 32 rows as float pairs, two chains at a time.
        for (int c = ch0; c < ch1; c += 2) {
          const bool two = c + 1 < ch1;
          float ll[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};
#pragma unroll
          for (int j = 0; j < 2; ++j)
            if (j == 0 || two) {
              const int ix = (c + j) * kRows + r;
              const float mx = s_m[ix], ssum = s_s[ix] + (zl ? expf(-mx) : 0.f);
              const float lse = mx + logf(ssum);
              s_m[ix] = lse;
              ll[j] = valid ? s_zy[ix] - lse : 0.f;
            }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float a0 = __shfl_down_sync(0xffffffffu, ll[0], o), b0 = __shfl_down_sync(0xffffffffu, lo[0], o);
            const float a1 = __shfl_down_sync(0xffffffffu, ll[1], o), b1 = __shfl_down_sync(0xffffffffu, lo[1], o);
            add_pair(ll[0], lo[0], a0, b0);
            add_pair(ll[1], lo[1], a1, b1);
          }
          if (lane == 0) {
            s_wsum[c * 4 + q] = make_float2(ll[0], lo[0]);
            if (two) s_wsum[(c + 1) * 4 + q] = make_float2(ll[1], lo[1]);
          }
        }
        epi_bar<kEpiThreads>();   // every chain's log-normaliser of this tile is in shared memory
        // Sweep 3: R = Y - P, P = exp(z - lse), for the group's columns (zero past Cg
        // and on rows past n), written as BF16 in the MN-major 128-byte-swizzled
        // boxes of pass B: 16-byte chunk j (8 columns) of row r of box b at chunk
        // j ^ (r % 8).  Each column's chain and class come from s_cm, so the 16
        // columns of a block are independent.  R is rounded to BF16, whose
        // precision (2^-9) the fast exponential's error (a few ulp of FP32) is far below.
        unsigned char* rb = A.rout + (size_t(t) * A.ngroups + g) * A.NB * kBoxBytes;
        for (int c0 = 16 * hf; c0 < A.NB * kBox; c0 += 16 * kEpiHalves) {
          uint32_t w[8];
          if (c0 < Cg) {
            float v[16];
            tmem_ld16(acc + uint32_t(c0), v);
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
              float rv[2];
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                const int ck = s_cm[c0 + e + hh];
                const float x = ((ck >> 16) == yv ? 1.f : 0.f) - __expf(v[e + hh] - s_m[(ck & 0xffff) + r]);
                rv[hh] = valid && c0 + e + hh < Cg ? x : 0.f;
              }
              const __nv_bfloat162 b2 = __floats2bfloat162_rn(rv[0], rv[1]);
              w[e / 2] = *reinterpret_cast<const uint32_t*>(&b2);
            }
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) w[e] = 0u;
          }
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int cc = c0 + 8 * hh;                // first column of this 16-byte chunk
            const int box = cc / kBox, chunk = (cc % kBox) / 8;
            unsigned char* dst = rb + size_t(box) * kBoxBytes + size_t(r) * 128 + size_t((chunk ^ (r & 7)) << 4);
            *reinterpret_cast<uint4*>(dst) = make_uint4(w[4 * hh], w[4 * hh + 1], w[4 * hh + 2], w[4 * hh + 3]);
          }
        }
        // This CTA's per-chain sums, in tile order: the four quarters' 32-row sums
        // in lane-quarter order.
        if (hf == 0 && r < nch) {
          float hi = s_wsum[r * 4].x, lo = s_wsum[r * 4].y;
#pragma unroll
          for (int k = 1; k < 4; ++k) add_pair(hi, lo, s_wsum[r * 4 + k].x, s_wsum[r * 4 + k].y);
          float2 cs = s_llc[g * gc + r];
          add_pair(cs.x, cs.y, hi, lo);
          s_llc[g * gc + r] = cs;
        }
        epi_bar<kEpiThreads>();   // shared state free for the next tile
      }
      // The unit's accumulators are read: the MMA issuer may start unit j + 2 in them.
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive_local(&zfree[a]);
      // The neighbour's partial is consumed (every read happened before the last
      // barrier of the tile loop): lower its flag for the next launch.
      if (head && warp == 2 && lane == 0) A.sflag[blockIdx.x + 1] = 0;
    }
  }
  __syncthreads();
  for (int c = tid; c < A.chains; c += int(blockDim.x))
    A.lpart[size_t(blockIdx.x) * A.lpart_cstride + c] = double(s_llc[c].x) + double(s_llc[c].y);
  if (warp == 1) {
    fence_after_sync();
    tmem_dealloc(tmem, A.tmem_cols);
  }
}

// ------------------------------------------------------------------ pass B
struct GradArgs {
  const unsigned char* xs;   // X boxes [ntiles][nkb][16 KB BF16 | 8 KB FP8 codes]
  const float* xscale;       // FP8: per-column scales s_j (G = diag(s) X_q^T R); nullptr for BF16
  const unsigned char* rs;   // R boxes [ntiles][ngroups][NB][16 KB]
  float* gpart;              // [Q][C][p_pad] partial gradient slices
  int64_t gpart_cstride;
  int* err;
  int64_t ntiles;
  int32_t nkb, p_pad, N, NB, Km1, gc, ngroups, chains;
  int32_t MB, nfg, Q, NST, NRS;
  uint32_t tmem_cols;
  long long spin_limit;
};

struct GradSmem {
  size_t ring, rring, bars, total;
};

__host__ __device__ inline GradSmem grad_smem(int NST, int NRS, int NB) {
  GradSmem L;
  size_t off = 0;
  L.ring = off;   off = al(off + size_t(NST) * 2 * kBoxBytes, 1024);
  L.rring = off;  off = al(off + size_t(NRS) * NB * kBoxBytes, 1024);
  // full, empty [NST]; rfull, rempty [NRS]; gdone; TMEM slot; abort flag; (pad); conv [NST]
  L.bars = off;   off = al(off + size_t(3 * NST + 2 * NRS + 4) * 8 + 16, 16);
  L.total = off + 1024;
  return L;
}

template <bool kFP8>
__global__ void __launch_bounds__(threads_b(kFP8), 1) grad_kernel(const GradArgs A) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = A.N, NST = A.NST, NRS = A.NRS;
  const GradSmem Lo = grad_smem(NST, NRS, A.NB);
  unsigned char* ring = smem + Lo.ring;
  unsigned char* rring = smem + Lo.rring;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lo.bars);
  uint64_t* full = bars;
  uint64_t* empty = bars + NST;
  uint64_t* rfull = bars + 2 * NST;
  uint64_t* rempty = rfull + NRS;
  uint64_t* gdone = rempty + NRS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gdone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gdone + 2);
  uint64_t* conv = gdone + 4;            // FP8: [NST] ring slot widened to BF16 (one group's warps arrive)

  // This CTA's unit: feature group f, chain group g, row range q.
  const int b = blockIdx.x;
  const int f = b % A.nfg, g = (b / A.nfg) % A.ngroups, q = b / (A.nfg * A.ngroups);
  const int nblk = A.p_pad / 128;
  const int mb0 = f * A.MB, mbn = max(0, min(A.MB, nblk - mb0));
  const int64_t t0 = int64_t(q) * A.ntiles / A.Q, t1 = int64_t(q + 1) * A.ntiles / A.Q;
  const int64_t T = t1 - t0;
  const int nch = min(A.gc, A.chains - g * A.gc);
  const int Cg = nch * A.Km1;

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < NRS; ++s) {
      mbar_init(&rfull[s], 1);
      mbar_init(&rempty[s], 1);
    }
    mbar_init(gdone, 1);
    if (kFP8)
      for (int s = 0; s < NST; ++s) mbar_init(&conv[s], kConvWarps / kConvGroupsB);
    *abort_flag = 0;
    fence_mbar_init_cluster();
  }
  if (warp == 1) tmem_alloc(tmem_slot, A.tmem_cols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  auto fail = [&](int bit) {
    *abort_flag = 1;
    atomicOr(A.err, bit);
  };
  const uint32_t rbytes = uint32_t(A.NB) * kBoxBytes;

  if (warp == 0) {
    if (lane == 0) {
      int64_t s = 0, issued = 0, rissued = 0;
      for (int64_t i = 0; i < T && !*abort_flag && mbn > 0; ++i) {
        const int64_t t = t0 + i;
        const int rsl = int(i % NRS);
        if (!wait_bounded(&rempty[rsl], uint32_t(((i / NRS) & 1) ^ 1), A.spin_limit, abort_flag)) {
          fail(ERR_TIMEOUT_STAGE);
          break;
        }
        mbar_arrive_expect_tx(&rfull[rsl], rbytes);
        bulk_g2s(rring + size_t(rsl) * rbytes, A.rs + (size_t(t) * A.ngroups + g) * rbytes, rbytes, &rfull[rsl]);
        rissued = i + 1;
        // Two X boxes per step: BF16 in place, FP8 (two consecutive 8 KB boxes) in
        // the upper half of the slot, widened in place by the converter warps.
        constexpr uint32_t xbox = kFP8 ? uint32_t(kFp8BoxBytes) : uint32_t(kBoxBytes);
        constexpr uint32_t xoff = kFP8 ? uint32_t(2 * (kBoxBytes - kFp8BoxBytes)) : 0u;
        const unsigned char* xt = A.xs + size_t(t) * A.nkb * xbox;
        for (int mb = 0; mb < mbn; ++mb, ++s) {
          const int st = int(s % NST);
          if (!wait_bounded(&empty[st], uint32_t(((s / NST) & 1) ^ 1), A.spin_limit, abort_flag)) {
            fail(ERR_TIMEOUT_STAGE);
            break;
          }
          mbar_arrive_expect_tx(&full[st], 2 * xbox);
          bulk_g2s(ring + size_t(st) * 2 * kBoxBytes + xoff, xt + size_t(2 * (mb0 + mb)) * xbox, 2 * xbox, &full[st]);
          issued = s + 1;
        }
      }
      for (int64_t qq = (issued > NST ? issued - NST : 0); qq < issued; ++qq)
        wait_drain(&full[qq % NST], uint32_t((qq / NST) & 1), A.spin_limit);
      for (int64_t qq = (rissued > NRS ? rissued - NRS : 0); qq < rissued; ++qq)
        wait_drain(&rfull[qq % NRS], uint32_t((qq / NRS) & 1), A.spin_limit);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kRows, N, true, true);
      int64_t s = 0;
      for (int64_t i = 0; i < T && !*abort_flag && mbn > 0; ++i) {
        const int rsl = int(i % NRS);
        if (!wait_bounded(&rfull[rsl], uint32_t((i / NRS) & 1), A.spin_limit, abort_flag)) {
          fail(ERR_TIMEOUT_STAGE);
          break;
        }
        fence_after_sync();
        const uint32_t rb = smem_u32(rring + size_t(rsl) * rbytes);
        for (int mb = 0; mb < mbn; ++mb, ++s) {
          const int st = int(s % NST);
          if (!wait_bounded(kFP8 ? &conv[st] : &full[st], uint32_t((s / NST) & 1), A.spin_limit, abort_flag)) {
            fail(ERR_TIMEOUT_STAGE);
            break;
          }
          fence_after_sync();
          const uint32_t xa = smem_u32(ring + size_t(st) * 2 * kBoxBytes);
          const uint32_t d = tmem + uint32_t(mb * N);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint64_t ad = smem_desc(xa + 2048u * k, uint32_t(kBoxBytes), 1024u, 2u);
            const uint64_t bd = smem_desc(rb + 2048u * k, uint32_t(kBoxBytes), 1024u, 2u);
            mma_bf16(d, ad, bd, idesc, (i > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(&empty[st]);
        }
        if (*abort_flag) break;
        mma_commit(&rempty[rsl]);
      }
      mma_commit(gdone);
      wait_drain(gdone, 0u, A.spin_limit);   // every MMA complete before TMEM is released
    }
  } else if (kFP8 && warp >= 6) {
    // ------------------------------------------------------------ FP8 converters (warps 6-9)
    // Group cg widens the ring steps s with s % kConvGroups == cg.
    constexpr int kConvGroups = kConvGroupsB, kGroupThreads = kConvThreads / kConvGroupsB;
    const int cv = tid - 192;
    const int cg = cv / kGroupThreads, ct = cv % kGroupThreads;
    int64_t s = 0;
    bool ok = true;
    for (int64_t i = 0; i < T && ok && mbn > 0; ++i) {
      for (int mb = 0; mb < mbn; ++mb, ++s) {
        if (int(s % kConvGroups) != cg) continue;
        const int st = int(s % NST);
        // One thread per group polls the copies' barrier; the group barrier
        // passes the result (and orders the landed bytes) to the others.
        const bool got = ct == 0 ? wait_bounded(&full[st], uint32_t((s / NST) & 1), A.spin_limit, abort_flag) : true;
        if (!conv_bar_and<kGroupThreads>(cg, got && !*abort_flag)) {   // the group agrees before its barrier below
          if (!got) fail(ERR_TIMEOUT_STAGE);
          ok = false;
          break;
        }
        // The two 8 KB boxes sit back to back in the slot's upper 16 KB.
        widen_fp8_boxes<2, kGroupThreads>(ring + size_t(st) * 2 * kBoxBytes, 2, uint32_t(kFp8BoxBytes),
                                          uint32_t(2 * (kBoxBytes - kFp8BoxBytes)), cg, ct);
        __syncwarp();
        if (lane == 0) mbar_arrive_local(&conv[st]);
      }
    }
  } else {
    // ------------------------------------------------------------ drain (warps 2-5)
    const int qd = warp & 3;
    const int row = 32 * qd + lane;               // feature within a block = TMEM lane
    const uint32_t tq = tmem + (uint32_t(32 * qd) << 16);
    bool ok = (lane == 0) ? wait_bounded(gdone, 0u, A.spin_limit, abort_flag) : true;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok && lane == 0) fail(ERR_TIMEOUT_MMA);
    fence_after_sync();
    float* gp = A.gpart + size_t(q) * A.gpart_cstride + size_t(g) * A.gc * A.Km1 * A.p_pad;
    for (int mb = 0; mb < mbn; ++mb) {
      const int col = (mb0 + mb) * 128 + row;
      for (int c0 = 0; c0 < Cg; c0 += 16) {
        float v[16];
        if (ok && T > 0) tmem_ld16(tq + uint32_t(mb * N + c0), v);
        const float sc = A.xscale ? A.xscale[col] : 1.f;
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if (c0 + e < Cg) gp[size_t(c0 + e) * A.p_pad + col] = (ok && T > 0) ? v[e] * sc : 0.f;
      }
    }
    fence_before_sync();
  }
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    tmem_dealloc(tmem, A.tmem_cols);
  }
}

// Coefficients [chains][Km1][p_pad] (FP32) -> operand boxes of every chain group,
// [group][p_pad / 64][2N rows x 128 B]: rows [0, N) the hi term bf16(v), rows
// [N, 2N) the lo term bf16(v - hi); columns past the group's C are zero.  With
// FP8 X the column scales are folded in: X B = X_q (diag(s) B).
// One thread per (row k, 8 consecutive columns): two 16-byte loads, one
// 16-byte chunk of each term stored (8 columns of a 128-byte box row are one
// swizzled chunk).
__global__ void beta_boxes_kernel(const float* beta, const float* scales, unsigned char* out, int32_t Km1, int32_t gc,
                                  int32_t chains, int32_t N, int32_t p_pad) {
  const int g = blockIdx.y;
  const int nch = min(gc, chains - g * gc);
  const int Cg = nch * Km1;
  const float* bg = beta + size_t(g) * gc * Km1 * p_pad;
  unsigned char* og = out + size_t(g) * (p_pad / kBox) * 2 * N * 128;
  const int p8 = p_pad / 8;
  const int64_t total = int64_t(N) * p8;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int k = int(i / p8);
    const int col = 8 * int(i - int64_t(k) * p8);
    float v[8];
    if (k < Cg) {
      const float4 a = *reinterpret_cast<const float4*>(bg + size_t(k) * p_pad + col);
      const float4 c = *reinterpret_cast<const float4*>(bg + size_t(k) * p_pad + col + 4);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = c.x; v[5] = c.y; v[6] = c.z; v[7] = c.w;
      if (scales) {
        const float4 s0 = *reinterpret_cast<const float4*>(scales + col);
        const float4 s1 = *reinterpret_cast<const float4*>(scales + col + 4);
        v[0] *= s0.x; v[1] *= s0.y; v[2] *= s0.z; v[3] *= s0.w; v[4] *= s1.x; v[5] *= s1.y; v[6] *= s1.z; v[7] *= s1.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = 0.f;
    }
    uint32_t wh[4], wl[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * j] - __low2float(h2), v[2 * j + 1] - __high2float(h2));
      wh[j] = *reinterpret_cast<const uint32_t*>(&h2);
      wl[j] = *reinterpret_cast<const uint32_t*>(&l2);
    }
    unsigned char* box = og + size_t(col / kBox) * 2 * N * 128;
    const int chunk = (col % kBox) >> 3;
    *reinterpret_cast<uint4*>(box + size_t(k) * 128 + ((chunk ^ (k & 7)) << 4)) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    *reinterpret_cast<uint4*>(box + size_t(N + k) * 128 + ((chunk ^ ((N + k) & 7)) << 4)) =
        make_uint4(wl[0], wl[1], wl[2], wl[3]);
  }
}

}  // namespace tc2

// ------------------------------------------------------------------ host side
int tc2_threads(bool fp8) { return tc2::threads_a(fp8); }

static uint32_t logit_stage(int U, int N) {
  return uint32_t(tc2::al(size_t(U) * tc2::kBoxBytes + size_t(2 * N) * 128, 1024));
}

size_t tc2_logit_smem(int NST, int U, int N, int gc, int chains) {
  return tc2::logit_smem(NST, logit_stage(U, N), gc, chains).total;
}

size_t tc2_grad_smem(int NST, int NRS, int NB) { return tc2::grad_smem(NST, NRS, NB).total; }

cudaError_t tc2_prepare() {
  int dev = 0, smem_max = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (auto fn : {tc2::logits_kernel<false>, tc2::logits_kernel<true>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  for (auto fn : {tc2::grad_kernel<false>, tc2::grad_kernel<true>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  return e;
}

cudaError_t tc2_beta_boxes(const float* beta, const float* scales, void* out, int Km1, int gc, int chains, int N,
                           int p_pad, int ngroups, cudaStream_t s) {
  const int64_t total = int64_t(N) * (p_pad / 8);
  const int gx = std::max(1, int(std::min<int64_t>(1024, (total + 255) / 256)));
  tc2::beta_boxes_kernel<<<dim3(gx, ngroups), 256, 0, s>>>(beta, scales, static_cast<unsigned char*>(out), Km1, gc,
                                                            chains, N, p_pad);
  return cudaGetLastError();
}

static uint32_t pow2_cols(int cols) {
  uint32_t t = 32;
  while (t < uint32_t(cols)) t <<= 1;
  return t;
}

cudaError_t tc2_launch(const Tc2Plan& P, const Tc2Launch& L, cudaStream_t stream, cudaEvent_t between, bool capturing) {
  {
    tc2::LogitArgs a{};
    a.xs = static_cast<const unsigned char*>(L.xs);
    a.bs = static_cast<const unsigned char*>(L.bs);
    a.y = L.y;
    a.rout = static_cast<unsigned char*>(L.rbuf);
    a.lpart = L.lpart;
    a.lpart_cstride = L.lpart_cstride;
    a.err = L.err;
    a.n = L.n;
    a.ntiles = (L.n + tc2::kRows - 1) / tc2::kRows;
    a.nkb = P.p_pad / tc2::kBox;
    a.N = P.N;
    a.NB = P.NB;
    a.Km1 = L.Km1;
    a.zlogit = L.zlogit;
    a.gc = P.gc;
    a.ngroups = (L.chains + P.gc - 1) / P.gc;
    a.chains = L.chains;
    a.NST = P.nstA;
    a.U = P.U;
    a.spart = static_cast<float*>(L.spart);
    a.sflag = L.sflag;
    a.stage_bytes = logit_stage(P.U, P.N);
    a.tmem_cols = pow2_cols(2 * P.U * P.N);
    a.spin_limit = L.spin_limit;
    if (L.fp8)
      tc2::logits_kernel<true><<<P.gridA, tc2::threads_a(true), P.smemA, stream>>>(a);
    else
      tc2::logits_kernel<false><<<P.gridA, tc2::threads_a(false), P.smemA, stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (between) {
      e = capturing ? cudaEventRecordWithFlags(between, stream, cudaEventRecordExternal) : cudaEventRecord(between, stream);
      if (e != cudaSuccess) return e;
    }
  }
  tc2::GradArgs b{};
  b.xs = static_cast<const unsigned char*>(L.xs);
  b.xscale = L.fp8 ? L.xscale : nullptr;
  b.rs = static_cast<const unsigned char*>(L.rbuf);
  b.gpart = static_cast<float*>(L.gpart);
  b.gpart_cstride = L.gpart_cstride;
  b.err = L.err;
  b.ntiles = (L.n + tc2::kRows - 1) / tc2::kRows;
  b.nkb = P.p_pad / tc2::kBox;
  b.p_pad = P.p_pad;
  b.N = P.N;
  b.NB = P.NB;
  b.Km1 = L.Km1;
  b.gc = P.gc;
  b.ngroups = (L.chains + P.gc - 1) / P.gc;
  b.chains = L.chains;
  b.MB = P.MB;
  b.nfg = P.nfg;
  b.Q = P.Q;
  b.NST = P.nstB;
  b.NRS = P.nrsB;
  b.tmem_cols = pow2_cols(P.MB * P.N);
  b.spin_limit = L.spin_limit;
  if (L.fp8)
    tc2::grad_kernel<true><<<P.nfg * b.ngroups * P.Q, tc2::threads_b(true), P.smemB, stream>>>(b);
  else
    tc2::grad_kernel<false><<<P.nfg * b.ngroups * P.Q, tc2::threads_b(false), P.smemB, stream>>>(b);
  return cudaGetLastError();
}

// Plan for `chains` chains of a problem (n, p, Km1) on nsm SMs with smem_max
// bytes of shared memory per block: the chain group (largest whose MMA N <= 256
// fits pass A's shared memory with >= 3 ring slots), pass A's tiles per unit and
// grid, and pass B's split (feature blocks per CTA, row ranges); both passes'
// choices minimise the bytes the busiest CTA streams.
bool tc2_plan(int64_t n, int64_t p, int Km1, int chains, int nsm, int smem_max, int force_U, Tc2Plan* out) {
  Tc2Plan P{};
  P.p_pad = int((p + 127) / 128 * 128);
  const int64_t ntiles = (n + 127) / 128;
  if (ntiles < 1 || Km1 < 1) return false;
  int gc = 0;
  for (int g = chains; g >= 1; --g) {
    const int N = std::max(16, (g * Km1 + 15) / 16 * 16);
    if (N > 256) continue;
    const int ngroups = (chains + g - 1) / g;
    const int gb = (chains + ngroups - 1) / ngroups;   // even groups
    const int Nb = std::max(16, (gb * Km1 + 15) / 16 * 16);
    if (tc2_logit_smem(3, 1, Nb, gb, chains) > size_t(smem_max)) continue;
    gc = gb;
    break;
  }
  if (!gc) return false;
  P.gc = gc;
  P.N = std::max(16, (gc * Km1 + 15) / 16 * 16);
  P.NB = (P.N + 63) / 64;
  const int ngroups = (chains + gc - 1) / gc;
  // Tiles per unit: U tiles share each coefficient box, so a unit streams
  // U * 16 KB of X and 2N * 128 B of coefficients per 64 features, and its
  // softmax epilogue overlaps the next unit's streaming.  The largest U that
  // fits (TMEM, shared memory) while still giving at least 0.8 units per SM is
  // taken (measured: n=5e4 p=1e4 K=20 4 chains, U = 1, 2 split, 3 -> 310, 295,
  // 266 us); when even U = 1 gives fewer, U = 1.
  P.U = 1;
  for (int U = 1; U <= 4; ++U) {
    if (2 * U * P.N > 512 || tc2_logit_smem(3, U, P.N, gc, chains) > size_t(smem_max)) break;
    if (force_U) {
      if (U == force_U) P.U = U;
      continue;
    }
    const int64_t units = (ntiles + U - 1) / U * ngroups;
    if (U == 1 || 5 * units >= 4 * int64_t(nsm)) P.U = U;
  }
  if (force_U && P.U != force_U) return false;
  P.nstA = 3;
  for (int s = 8; s > 3; --s)
    if (tc2_logit_smem(s, P.U, P.N, gc, chains) <= size_t(smem_max)) {
      P.nstA = s;
      break;
    }
  P.smemA = std::max(tc2_logit_smem(P.nstA, P.U, P.N, gc, chains), size_t(116 * 1024));
  P.gridA = int(std::min<int64_t>(nsm, (ntiles + P.U - 1) / P.U * ngroups));
  // Pass B.
  const int nblk = P.p_pad / 128;
  const int mbmax = std::min(nblk, std::max(1, 512 / P.N));
  double best = -1.0;
  for (int MB = 1; MB <= mbmax; ++MB) {
    const int nfg = (nblk + MB - 1) / MB;
    const int64_t base = int64_t(nfg) * ngroups;
    const int Q = int(std::max<int64_t>(1, std::min<int64_t>(ntiles, nsm / std::max<int64_t>(1, base))));
    const int64_t ctas = base * Q;
    const double waves = double((ctas + nsm - 1) / nsm);
    const double per_cta = double((ntiles + Q - 1) / Q) * (2.0 * MB + P.NB);   // boxes streamed by the busiest CTA
    const double cost = per_cta * waves;
    if (best < 0 || cost < best) {
      best = cost;
      P.MB = MB;
      P.nfg = nfg;
      P.Q = Q;
    }
  }
  // Two R slots (the next tile's residual lands while this one is used) with at
  // least three X slots, else one R slot.
  P.nrsB = 2;
  P.nstB = 0;
  for (int r = 2; r >= 1 && !P.nstB; --r)
    for (int s = 8; s >= (r == 2 ? 3 : 2) && !P.nstB; --s)
      if (tc2_grad_smem(s, r, P.NB) <= size_t(smem_max)) {
        P.nstB = s;
        P.nrsB = r;
      }
  if (!P.nstB) return false;
  P.smemB = std::max(tc2_grad_smem(P.nstB, P.nrsB, P.NB), size_t(116 * 1024));
  *out = P;
  return true;
}

}  // namespace hmc
