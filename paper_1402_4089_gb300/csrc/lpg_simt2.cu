// Two-pass evaluation of the log-posterior and its gradient on CUDA cores
// (Eqs. softmax, loglike, logkernel and gradient of Sec. 2.1) for FP64 or FP32
// X, used where the fused CUDA-core pass has no tile: its cluster holds every
// coefficient column of its feature slice next to a ring of row tiles in
// shared memory, which does not fit for wide problems with many classes (FP32
// X, K - 1 > 12 and p > 10240, i.e. the K = 15, 20 columns of Table 1 at
// p = 20000), nor for more classes per chain than that pass handles.
//
//  pass 1a (logits_kernel): Z = X B^T for a block of 8 warps x RW rows over one
//          feature split.  Coefficient chunks of 128 features x C columns are
//          staged in shared memory by cp.async together with the block's rows
//          of X for the same features, in a ring of 2 or 4 stages (the copies
//          of the next chunks overlap the arithmetic of chunk k).  A warp's lanes are 8
//          feature lanes x 4 class groups: lane (f, g) takes features 4f .. 4f+3
//          of every 32-feature slice and the classes c = g, g + 4, ..., so one
//          shared-memory vector load of coefficients feeds 4 RW FMAs and the
//          four class groups read X as broadcasts; a butterfly over the feature
//          lanes gives the rows' logits, written as one partial per feature
//          split.
//          Feature splits give small N enough blocks.  Launches of at most 16
//          columns use logits_lanes_kernel instead (lane = 4 features, all
//          classes, X straight from global memory), which measures faster there.
//  pass 1b (softmax_kernel): one warp per row sums the splits in a fixed
//          order, forms the softmax with the zero logit of class K (or
//          without it, unconstrained layout), the residual R[i][C] and the row
//          log-likelihoods (FP64), summed over the block's 8 rows in row order
//          (the reduction sums the blocks in order).
//  pass 2  (grad_kernel): G_q[c][j] = sum over row range q of X[i][j] R[i][c];
//          a thread takes FT consecutive features, 64 residual rows at a time
//          are staged in shared memory, X loads are issued 8 rows at a time and
//          the next 8 rows are loaded while the current ones are used; one
//          partial slice per row range, summed in range order.
//
// X is read from HBM twice (once per pass).
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace hmc {
namespace simt2 {

constexpr int kMaxC = 64;       // coefficient columns of one launch
constexpr int kWarps = 8;       // warps per block (both passes: 256 threads)
constexpr int kChunk = 128;     // pass 1a: features per staged coefficient chunk
constexpr int kStage = 64;      // pass 2: residual rows staged per step
constexpr int kUnroll = 8;      // pass 2: X rows loaded together
constexpr int kRowsMax = 32;    // pass 1a: rows of a block at most (feature-split sizing)
constexpr size_t kRing4Bytes = 110 * 1024;   // pass 1a: largest four-stage ring (two blocks per SM)

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

// Four consecutive values (16-byte aligned for float, 32-byte for double) in
// the state type.
template <typename XT, typename AT>
__device__ __forceinline__ void load4(const XT* p, AT* o) {
  if constexpr (sizeof(XT) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = AT(v.x); o[1] = AT(v.y); o[2] = AT(v.z); o[3] = AT(v.w);
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    o[0] = AT(a.x); o[1] = AT(a.y); o[2] = AT(b.x); o[3] = AT(b.y);
  }
}

// FT consecutive values (FT in {1, 2, 4}, aligned to FT elements).
template <typename XT, typename AT, int FT>
__device__ __forceinline__ void loadft(const XT* p, AT* o) {
  if constexpr (FT == 4) {
    load4<XT, AT>(p, o);
  } else if constexpr (FT == 2) {
    if constexpr (sizeof(XT) == 4) {
      const float2 v = *reinterpret_cast<const float2*>(p);
      o[0] = AT(v.x); o[1] = AT(v.y);
    } else {
      const double2 v = *reinterpret_cast<const double2*>(p);
      o[0] = AT(v.x); o[1] = AT(v.y);
    }
  } else {
    o[0] = AT(*p);
  }
}

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Rows one warp takes in pass 1a: every staged coefficient value serves RW
// rows; a lane holds RW x CB / 4 logit accumulators (at most 64 words).
template <typename AT, int CB>
__host__ __device__ constexpr int rows_per_warp() {
  return sizeof(AT) == 8 ? 2 : 4;
}

// Rows one warp takes in the narrow pass-1a kernel: RW x CB logit accumulators
// per lane, at most 32 words.
template <typename AT, int CB>
__host__ __device__ constexpr int lane_rows() {
  return sizeof(AT) == 8 ? (CB <= 8 ? 2 : 1) : (CB <= 8 ? 4 : 2);
}

// Features one thread takes in pass 2: FT x CB <= 32 accumulator words (64 at
// CB = 64), next to two batches of 8 rows x FT X values.
template <typename AT, int CB>
__host__ __device__ constexpr int features_per_thread() {
  return sizeof(AT) == 8 ? (CB <= 8 ? 2 : 1) : (CB <= 16 ? 2 : 1);
}

// Blocks per SM the register budget is sized for: two, except FP64 at 64 columns.
template <typename AT, int CB>
__host__ __device__ constexpr int min_blocks() {
  return sizeof(AT) == 8 && CB == 64 ? 1 : 2;
}

// Stage coefficient chunk k (columns c < C, features [128 k, 128 k + 128) that
// lie below p_pad) into `dst` [C][kChunk].
template <typename AT>
__device__ __forceinline__ void stage_chunk(AT* dst, const AT* __restrict__ beta, int k, int32_t p_pad, int32_t C) {
  constexpr int kVec = 16 / sizeof(AT);             // values per 16-byte copy
  constexpr int kPerRow = kChunk / kVec;
  const int j0 = k * kChunk;
  const int valid = min(kChunk, p_pad - j0);       // multiple of 4 (p_pad is)
  for (int e = threadIdx.x; e < C * kPerRow; e += blockDim.x) {
    const int c = e / kPerRow, v = e - c * kPerRow;
    if (v * kVec < valid)
      cp_async16(dst + c * kChunk + v * kVec, beta + size_t(c) * p_pad + j0 + v * kVec);
    else   // past p_pad: zeros (X is zero there too, and 0 x a stale NaN would not be)
      *reinterpret_cast<uint4*>(dst + c * kChunk + v * kVec) = make_uint4(0u, 0u, 0u, 0u);
  }
}

// Stage X rows [i0, i0 + rows) of chunk k into `dst` [rows][kChunk] (rows past
// n read row n - 1, features past p_pad are zero).
template <typename XT>
__device__ __forceinline__ void stage_x(XT* dst, const XT* __restrict__ X, int64_t i0, int rows, int64_t n, int k,
                                        int32_t p_pad) {
  constexpr int kVec = 16 / sizeof(XT);
  constexpr int kPerRow = kChunk / kVec;
  const int j0 = k * kChunk;
  const int valid = min(kChunk, p_pad - j0);
  for (int e = threadIdx.x; e < rows * kPerRow; e += blockDim.x) {
    const int r = e / kPerRow, v = e - r * kPerRow;
    if (v * kVec < valid)
      cp_async16(dst + r * kChunk + v * kVec, X + size_t(min(i0 + r, n - 1)) * p_pad + j0 + v * kVec);
    else
      *reinterpret_cast<uint4*>(dst + r * kChunk + v * kVec) = make_uint4(0u, 0u, 0u, 0u);
  }
}

// Pass 1a for narrow launches (CB <= 16), where it measures faster than the
// class-split kernel below: lane l takes features 4l .. 4l + 3 of each chunk
// and every class, X is loaded from global memory one chunk ahead into
// registers, a butterfly over all 32 lanes gives the rows' logits.  Grid and
// zpart as for logits_kernel; dynamic shared memory 2 x C x kChunk state
// values.
template <typename XT, typename AT, int CB>
__global__ void __launch_bounds__(32 * kWarps, min_blocks<AT, CB>()) logits_lanes_kernel(const XT* __restrict__ X, const AT* __restrict__ beta,
                                                             AT* __restrict__ zpart, int64_t n, int32_t p_pad,
                                                             int32_t C, int32_t cps) {
  constexpr int RW = lane_rows<AT, CB>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AT* bs = reinterpret_cast<AT*>(smem_raw);        // [2][C][kChunk]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nchunks = (p_pad + kChunk - 1) / kChunk;
  const int k0 = blockIdx.y * cps, k1 = min(nchunks, k0 + cps);
  const int64_t i0 = (int64_t(blockIdx.x) * kWarps + warp) * RW;
  const XT* xr[RW];
#pragma unroll
  for (int r = 0; r < RW; ++r) xr[r] = X + size_t(min(i0 + r, n - 1)) * p_pad;   // rows past n: read, not written
  AT z[RW][CB];
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int c = 0; c < CB; ++c) z[r][c] = AT(0);
  if (k0 < k1) {
    stage_chunk<AT>(bs, beta, k0, p_pad, C);
    cp_async_commit();
    AT xn[RW][4];
    {
      const int j = k0 * kChunk + 4 * lane;
#pragma unroll
      for (int r = 0; r < RW; ++r) {
        if (j < p_pad) load4<XT, AT>(xr[r] + j, xn[r]);
        else xn[r][0] = xn[r][1] = xn[r][2] = xn[r][3] = AT(0);
      }
    }
    for (int k = k0; k < k1; ++k) {
      const int buf = (k - k0) & 1;
      if (k + 1 < k1) stage_chunk<AT>(bs + (buf ^ 1) * C * kChunk, beta, k + 1, p_pad, C);
      cp_async_commit();                           // (possibly empty) group of chunk k + 1
      AT xv[RW][4];
#pragma unroll
      for (int r = 0; r < RW; ++r)
#pragma unroll
        for (int f = 0; f < 4; ++f) xv[r][f] = xn[r][f];
      const int jn = (k + 1) * kChunk + 4 * lane;
      if (k + 1 < k1) {
#pragma unroll
        for (int r = 0; r < RW; ++r) {
          if (jn < p_pad) load4<XT, AT>(xr[r] + jn, xn[r]);
          else xn[r][0] = xn[r][1] = xn[r][2] = xn[r][3] = AT(0);
        }
      }
      cp_async_wait<1>();                          // chunk k has landed (this thread's copies)
      __syncthreads();                             // ... and every thread's
      const AT* b = bs + buf * C * kChunk + 4 * lane;
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        if (c < C) {
          AT bv[4];
          load4<AT, AT>(b + c * kChunk, bv);       // features past p_pad: X is 0 there
#pragma unroll
          for (int r = 0; r < RW; ++r)
            z[r][c] = fma(xv[r][0], bv[0], fma(xv[r][1], bv[1], fma(xv[r][2], bv[2], fma(xv[r][3], bv[3], z[r][c]))));
        }
      }
      __syncthreads();                             // buffer buf is refilled two chunks on
    }
    cp_async_wait<0>();
  }
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int c = 0; c < CB; ++c)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) z[r][c] += __shfl_xor_sync(0xffffffffu, z[r][c], o);
  AT* zp = zpart + size_t(blockIdx.y) * n * C;
#pragma unroll
  for (int r = 0; r < RW; ++r) {
    if (i0 + r >= n) break;
#pragma unroll
    for (int c = 0; c < CB; ++c)
      if ((c & 31) == lane && c < C) zp[size_t(i0 + r) * C + c] = z[r][c];
  }
}

// CB: class bound of the instantiation (>= C, a multiple of 4); NSTG: ring
// stages.  Grid: (row blocks, feature splits); split s covers chunks
// [s * cps, min((s + 1) * cps, nchunks)).  zpart: [FS][n][C].  Dynamic shared
// memory: NSTG x (C coefficient rows x kChunk state values + 8 RW X rows x
// kChunk X values).
template <typename XT, typename AT, int CB, int NSTG>
__global__ void __launch_bounds__(32 * kWarps, min_blocks<AT, CB>()) logits_kernel(const XT* __restrict__ X, const AT* __restrict__ beta,
                                                             AT* __restrict__ zpart, int64_t n, int32_t p_pad,
                                                             int32_t C, int32_t cps) {
  constexpr int RW = rows_per_warp<AT, CB>();
  constexpr int BR = kWarps * RW;                  // rows of the block
  constexpr int TPL = CB / 4;                      // classes per lane
  constexpr int kSlices = kChunk / 32;             // 32-feature slices per chunk
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AT* bs = reinterpret_cast<AT*>(smem_raw);        // [NSTG][C][kChunk]
  XT* xs = reinterpret_cast<XT*>(bs + NSTG * C * kChunk);   // [NSTG][BR][kChunk]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int fl = lane & 7, cg = lane >> 3;          // feature lane, class group
  const int nchunks = (p_pad + kChunk - 1) / kChunk;
  const int k0 = blockIdx.y * cps, k1 = min(nchunks, k0 + cps);
  const int64_t ib = int64_t(blockIdx.x) * BR;      // first row of the block
  const int64_t i0 = ib + warp * RW;                // first row of the warp
  AT z[RW][TPL];
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int t = 0; t < TPL; ++t) z[r][t] = AT(0);
  if (k0 < k1) {
    // Chunks k0 .. k0 + NSTG - 2 in flight, one commit group each (possibly empty).
#pragma unroll
    for (int q = 0; q < NSTG - 1; ++q) {
      if (k0 + q < k1) {
        stage_chunk<AT>(bs + q * C * kChunk, beta, k0 + q, p_pad, C);
        stage_x<XT>(xs + q * BR * kChunk, X, ib, BR, n, k0 + q, p_pad);
      }
      cp_async_commit();
    }
    for (int k = k0; k < k1; ++k) {
      const int buf = (k - k0) % NSTG;
      const int kn = k + NSTG - 1;                 // the chunk refilling the slot freed by chunk k - 1
      if (kn < k1) {
        const int nb = (kn - k0) % NSTG;
        stage_chunk<AT>(bs + nb * C * kChunk, beta, kn, p_pad, C);
        stage_x<XT>(xs + nb * BR * kChunk, X, ib, BR, n, kn, p_pad);
      }
      cp_async_commit();
      cp_async_wait<NSTG - 1>();                   // chunk k has landed (this thread's copies)
      __syncthreads();                             // ... and every thread's
      const AT* b = bs + buf * C * kChunk + 4 * fl;
      const XT* xw = xs + (buf * BR + warp * RW) * kChunk + 4 * fl;
#pragma unroll
      for (int sl = 0; sl < kSlices; ++sl) {
        AT xv[RW][4];
#pragma unroll
        for (int r = 0; r < RW; ++r) load4<XT, AT>(xw + r * kChunk + 32 * sl, xv[r]);   // broadcast over class groups
#pragma unroll
        for (int t = 0; t < TPL; ++t) {
          const int c = cg + 4 * t;
          if (c < C) {
            AT bv[4];
            load4<AT, AT>(b + c * kChunk + 32 * sl, bv);   // features past p_pad: X is 0 there
#pragma unroll
            for (int r = 0; r < RW; ++r)
              z[r][t] = fma(xv[r][0], bv[0], fma(xv[r][1], bv[1], fma(xv[r][2], bv[2], fma(xv[r][3], bv[3], z[r][t]))));
          }
        }
      }
      __syncthreads();                             // slot buf is refilled in the next iteration
    }
    cp_async_wait<0>();
  }
  // Sum over the 8 feature lanes of each class group (lane bits 0-2).
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int t = 0; t < TPL; ++t)
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) z[r][t] += __shfl_xor_sync(0xffffffffu, z[r][t], o);
  if (fl != 0) return;
  AT* zp = zpart + size_t(blockIdx.y) * n * C;
#pragma unroll
  for (int r = 0; r < RW; ++r) {
    if (i0 + r >= n) break;
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
      const int c = cg + 4 * t;
      if (c < C) zp[size_t(i0 + r) * C + c] = z[r][t];
    }
  }
}

// One warp per row: the lanes sum the row's logits over the FS splits in split
// order (columns across lanes, 8 split loads in flight), lane ch < chains forms
// chain ch's maximum, normaliser and row log-likelihood, and the lanes write
// the residual row R[i][0 .. C) column by column.  The block's 8 row
// log-likelihoods of each chain are summed in row order into lblk[block].
template <typename AT>
__global__ void __launch_bounds__(32 * kWarps) softmax_kernel(const AT* __restrict__ zpart, const int32_t* __restrict__ y,
                                                             AT* __restrict__ R, double* __restrict__ lblk,
                                                             int32_t lstride, int64_t n, int32_t C, int32_t Km1,
                                                             int32_t chains, int32_t FS, int32_t zlogit, int* err) {
  __shared__ AT zs[kWarps][kMaxC];
  __shared__ AT ms[kWarps][kMaxC], is[kWarps][kMaxC];   // per chain: maximum, 1 / normaliser
  __shared__ double ls[kWarps][kMaxC];                  // per chain: row log-likelihood
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = int64_t(blockIdx.x) * kWarps + w;
  if (i < n) {                                          // warp-uniform
    const size_t sstride = size_t(n) * C;
    for (int c = lane; c < C; c += 32) {
      const AT* zc = zpart + size_t(i) * C + c;
      AT v = zc[0];
      int sp = 1;
      for (; sp + 8 <= FS; sp += 8) {
        AT t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = zc[size_t(sp + u) * sstride];
#pragma unroll
        for (int u = 0; u < 8; ++u) v += t[u];
      }
      for (; sp < FS; ++sp) v += zc[size_t(sp) * sstride];
      zs[w][c] = v;
    }
    __syncwarp();
    int yi = y[i];
    if (yi < 0 || yi >= Km1 + zlogit) {
      if (lane == 0) atomicOr(err, ERR_BAD_LABEL);
      yi = 0;
    }
    for (int ch = lane; ch < chains; ch += 32) {
      const AT* z = zs[w] + ch * Km1;
      AT m = zlogit ? AT(0) : AT(-INFINITY);
      for (int k = 0; k < Km1; ++k) m = max(m, z[k]);
      AT sum = zlogit ? ex<AT>(-m) : AT(0);
      for (int k = 0; k < Km1; ++k) sum += ex<AT>(z[k] - m);
      ms[w][ch] = m;
      is[w][ch] = AT(1) / sum;
      const AT zy = yi < Km1 ? z[yi] : AT(0);     // yi == Km1: class K, logit 0
      ls[w][ch] = double(zy - m - lg<AT>(sum));
    }
    __syncwarp();
    AT* ri = R + size_t(i) * C;
    for (int c = lane; c < C; c += 32) {
      const int ch = c / Km1, k = c - ch * Km1;
      ri[c] = (k == yi ? AT(1) : AT(0)) - ex<AT>(zs[w][c] - ms[w][ch]) * is[w][ch];
    }
  }
  __syncthreads();
  if (threadIdx.x < chains) {
    const int rows = int(min(int64_t(kWarps), n - int64_t(blockIdx.x) * kWarps));
    double acc = 0.0;
    for (int r = 0; r < rows; ++r) acc += ls[r][threadIdx.x];
    lblk[size_t(blockIdx.x) * lstride + threadIdx.x] = acc;
  }
}

// Thread: FT consecutive features of the block's 256 FT-feature slice, rows of
// range q = [q n / Q, (q + 1) n / Q).
template <typename XT, typename AT, int CB>
__global__ void __launch_bounds__(32 * kWarps, min_blocks<AT, CB>()) grad_kernel(const XT* __restrict__ X, const AT* __restrict__ R,
                                                           AT* __restrict__ gpart, int64_t gpart_cstride, int64_t n,
                                                           int32_t p_pad, int32_t C, int32_t Q, const float* xscale) {
  constexpr int FT = features_per_thread<AT, CB>();
  __shared__ __align__(16) AT rs[kStage][CB];
  const int span = 32 * kWarps * FT;
  const int nfb = (p_pad + span - 1) / span;
  const int fb = blockIdx.x % nfb, q = blockIdx.x / nfb;
  const int64_t j = int64_t(fb) * span + int64_t(threadIdx.x) * FT;
  const bool active = j < p_pad;                    // p_pad % 4 == 0: all FT features valid
  const int64_t r0 = int64_t(q) * n / Q, r1 = int64_t(q + 1) * n / Q;
  AT g[FT][CB];
#pragma unroll
  for (int f = 0; f < FT; ++f)
#pragma unroll
    for (int c = 0; c < CB; ++c) g[f][c] = AT(0);
  for (int64_t i0 = r0; i0 < r1; i0 += kStage) {
    const int rows = int(min(int64_t(kStage), r1 - i0));
    __syncthreads();
    for (int e = threadIdx.x; e < kStage * CB; e += blockDim.x) {
      const int rr = e / CB, c = e - rr * CB;
      rs[rr][c] = (rr < rows && c < C) ? R[size_t(i0 + rr) * C + c] : AT(0);
    }
    __syncthreads();
    if (!active) continue;
    AT xv[kUnroll][FT];
    auto load_batch = [&](int rr, AT (*o)[FT]) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (rr + u < rows) {
          loadft<XT, AT, FT>(X + size_t(i0 + rr + u) * p_pad + j, o[u]);
        } else {
#pragma unroll
          for (int f = 0; f < FT; ++f) o[u][f] = AT(0);
        }
      }
    };
    load_batch(0, xv);
    for (int rr = 0; rr < rows; rr += kUnroll) {
      AT xn[kUnroll][FT];
      if (rr + kUnroll < rows) load_batch(rr + kUnroll, xn);   // the next 8 rows while these are used
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          const AT rv = rs[rr + u][c];             // rows past `rows` are zero
#pragma unroll
          for (int f = 0; f < FT; ++f) g[f][c] = fma(xv[u][f], rv, g[f][c]);
        }
      if (rr + kUnroll < rows) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
          for (int f = 0; f < FT; ++f) xv[u][f] = xn[u][f];
      }
    }
  }
  if (!active) return;
  AT* gp = gpart + size_t(q) * gpart_cstride;
#pragma unroll
  for (int f = 0; f < FT; ++f) {
    const AT sc = xscale ? AT(xscale[j + f]) : AT(1);
#pragma unroll
    for (int c = 0; c < CB; ++c)
      if (c < C) gp[size_t(c) * p_pad + j + f] = g[f][c] * sc;
  }
}

template <typename XT, typename AT, int CB>
cudaError_t launch_cb(const Simt2Launch& L, cudaStream_t s, cudaEvent_t between, bool capturing) {
  const XT* X = static_cast<const XT*>(L.X);
  const AT* beta = static_cast<const AT*>(L.beta);
  AT* R = static_cast<AT*>(L.rbuf);
  AT* zp = static_cast<AT*>(L.zpart);
  constexpr bool narrow = CB <= 16;
  constexpr int rows = kWarps * (narrow ? lane_rows<AT, CB>() : rows_per_warp<AT, CB>());
  const int nchunks = (L.p_pad + kChunk - 1) / kChunk;
  const int fs = std::max(1, std::min(L.FS, nchunks));
  const int cps = (nchunks + fs - 1) / fs;
  const int fs_used = (nchunks + cps - 1) / cps;
  const dim3 g1(unsigned((L.n + rows - 1) / rows), unsigned(fs_used));
  if constexpr (narrow) {
    const size_t smem = size_t(2) * L.C * kChunk * sizeof(AT);
    logits_lanes_kernel<XT, AT, CB><<<g1, 32 * kWarps, smem, s>>>(X, beta, zp, L.n, L.p_pad, L.C, cps);
  } else {
    const size_t stage = size_t(kChunk) * (L.C * sizeof(AT) + kWarps * rows_per_warp<AT, CB>() * sizeof(XT));
    if (4 * stage <= kRing4Bytes)   // four stages where two blocks still fit an SM (within what simt2_prepare allowed)
      logits_kernel<XT, AT, CB, 4><<<g1, 32 * kWarps, 4 * stage, s>>>(X, beta, zp, L.n, L.p_pad, L.C, cps);
    else
      logits_kernel<XT, AT, CB, 2><<<g1, 32 * kWarps, 2 * stage, s>>>(X, beta, zp, L.n, L.p_pad, L.C, cps);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  softmax_kernel<AT><<<unsigned((L.n + kWarps - 1) / kWarps), 32 * kWarps, 0, s>>>(
      zp, L.y, R, L.lrow, L.lrow_stride, L.n, L.C, L.Km1, L.chains, fs_used, L.zlogit, L.err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (between) {
    e = capturing ? cudaEventRecordWithFlags(between, s, cudaEventRecordExternal) : cudaEventRecord(between, s);
    if (e != cudaSuccess) return e;
  }
  constexpr int span = 32 * kWarps * features_per_thread<AT, CB>();
  const int nfb = (L.p_pad + span - 1) / span;
  grad_kernel<XT, AT, CB><<<dim3(unsigned(nfb * L.Q)), 32 * kWarps, 0, s>>>(X, R, static_cast<AT*>(L.gpart),
                                                                           L.gpart_cstride, L.n, L.p_pad, L.C, L.Q,
                                                                           L.xscale);
  return cudaGetLastError();
}

template <typename XT, typename AT>
cudaError_t launch_t(const Simt2Launch& L, cudaStream_t s, cudaEvent_t between, bool capturing) {
  if (L.C <= 8) return launch_cb<XT, AT, 8>(L, s, between, capturing);
  if (L.C <= 16) return launch_cb<XT, AT, 16>(L, s, between, capturing);
  if (L.C <= 32) return launch_cb<XT, AT, 32>(L, s, between, capturing);
  return launch_cb<XT, AT, kMaxC>(L, s, between, capturing);
}

template <typename XT, typename AT, int CB>
cudaError_t prepare_cb() {
  if constexpr (CB <= 16) {
    return cudaFuncSetAttribute(logits_lanes_kernel<XT, AT, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(2 * CB * kChunk * sizeof(AT)));
  } else {
    const int two = int(2 * kChunk * (CB * sizeof(AT) + kWarps * rows_per_warp<AT, CB>() * sizeof(XT)));
    cudaError_t e = cudaFuncSetAttribute(logits_kernel<XT, AT, CB, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, two);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(logits_kernel<XT, AT, CB, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(kRing4Bytes));
  }
}

}  // namespace simt2

int simt2_max_c() { return simt2::kMaxC; }

int64_t simt2_ll_blocks(int64_t n) { return (n + simt2::kWarps - 1) / simt2::kWarps; }

cudaError_t simt2_prepare(int xt) {
  using namespace simt2;
  cudaError_t e = cudaSuccess;
  if (xt == HMC_F64) {
    for (cudaError_t r : {prepare_cb<double, double, 8>(), prepare_cb<double, double, 16>(),
                          prepare_cb<double, double, 32>(), prepare_cb<double, double, kMaxC>()})
      if (r != cudaSuccess) e = r;
  } else {
    for (cudaError_t r : {prepare_cb<float, float, 8>(), prepare_cb<float, float, 16>(), prepare_cb<float, float, 32>(),
                          prepare_cb<float, float, kMaxC>()})
      if (r != cudaSuccess) e = r;
  }
  return e;
}

// Row ranges of pass 2 (partial gradient slices): about four blocks per SM,
// with the slices' bytes (Q C p_pad) kept to a quarter of X's (n p_pad).
int simt2_row_ranges(int64_t n, int32_t p_pad, int32_t C, int nsm) {
  const int64_t span = 4 * 256;                    // features of a block at FT = 4 (the fewest blocks)
  const int64_t nfb = std::max<int64_t>(1, (p_pad + span - 1) / span);
  const int64_t want = (4 * int64_t(nsm) + nfb - 1) / nfb;
  const int64_t cap = std::max<int64_t>(1, n / (4 * int64_t(std::max(C, 1))));
  return int(std::max<int64_t>(1, std::min<int64_t>({want, cap, 64})));
}

// Feature splits of pass 1a: enough blocks for two per SM at the largest row
// block (32 rows).
int simt2_feature_splits(int64_t n, int32_t p_pad, int nsm) {
  const int64_t nchunks = (p_pad + simt2::kChunk - 1) / simt2::kChunk;
  const int64_t rowblocks = std::max<int64_t>(1, (n + simt2::kRowsMax - 1) / simt2::kRowsMax);
  const int64_t want = (2 * int64_t(nsm) + rowblocks - 1) / rowblocks;
  return int(std::max<int64_t>(1, std::min<int64_t>(want, nchunks)));
}

cudaError_t simt2_launch(int xt, const Simt2Launch& L, cudaStream_t s, cudaEvent_t between, bool capturing) {
  if (L.n == 0) return cudaSuccess;
  if (L.C < 1 || L.C > simt2::kMaxC || L.p_pad % 4 || L.FS < 1 || L.Q < 1) return cudaErrorInvalidValue;
  if (xt == HMC_F64) return simt2::launch_t<double, double>(L, s, between, capturing);
  return simt2::launch_t<float, float>(L, s, between, capturing);
}

}  // namespace hmc
