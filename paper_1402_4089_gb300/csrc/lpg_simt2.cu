// Two-pass evaluation of the log-posterior and its gradient on CUDA cores
// (Eqs. softmax, loglike, logkernel and gradient of Sec. 2.1) for FP64 or FP32
// X, used where the fused CUDA-core pass has no tile: its cluster holds every
// coefficient column of its feature slice next to a ring of row tiles in
// shared memory, which does not fit for wide problems with many classes (FP32
// X, K - 1 > 12 and p > 10240, i.e. the K = 15, 20 columns of Table 1 at
// p = 20000).  Nothing here is held across rows but one row's logits:
//
//  pass 1 (one warp per 1 to 4 rows): lane l accumulates the dot products of
//         the rows with every coefficient column over features 4l, 4l + 128,
//         ... (float4 / double2 loads, each coefficient load from L2 serving
//         every row of the warp), a butterfly reduction gives every lane the
//         rows' logits; the softmax with the
//         zero logit of class K (or without it, unconstrained layout), the
//         residual R[i][C] and the row log-likelihood of every chain are
//         written to global memory (FP64 log-likelihoods, summed later in row
//         order by the reduction).
//  pass 2 (one thread per feature j and row range q): G_q[c][j] = sum over the
//         range's rows of X[i][j] R[i][c], the rows' residuals staged in shared
//         memory; one partial slice per row range, summed in range order.
//
// X is read from HBM twice (once per pass).
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace hmc {
namespace simt2 {

constexpr int kMaxC = 64;          // coefficient columns of one launch
constexpr int kRowsPerBlock = 8;   // pass 1: warps (rows) per block
constexpr int kStage = 32;         // pass 2: residual rows staged per step

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

// Four consecutive values of X (aligned) in the state type.
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

// Rows one warp takes in pass 1: every coefficient load (from L2) serves RW
// rows, with the logit registers (RW x CB per lane) kept at about 64 words.
template <typename AT, int CB>
__host__ __device__ constexpr int rows_per_warp() {
  return sizeof(AT) == 4 ? (CB <= 16 ? 4 : CB <= 32 ? 2 : 1) : (CB <= 8 ? 4 : CB <= 16 ? 2 : 1);
}

// CB: class bound of the instantiation (>= C).
template <typename XT, typename AT, int CB>
__global__ void __launch_bounds__(32 * kRowsPerBlock) logits_kernel(const XT* __restrict__ X, const int32_t* __restrict__ y,
                                                                     const AT* __restrict__ beta, AT* __restrict__ R,
                                                                     double* __restrict__ lrow, int32_t lstride, int64_t n,
                                                                     int32_t p_pad, int32_t C, int32_t Km1, int32_t chains,
                                                                     int32_t zlogit, int* err) {
  constexpr int RW = rows_per_warp<AT, CB>();
  const int lane = threadIdx.x & 31;
  const int64_t i0 = (int64_t(blockIdx.x) * kRowsPerBlock + (threadIdx.x >> 5)) * RW;
  if (i0 >= n) return;
  const XT* xr[RW];
#pragma unroll
  for (int r = 0; r < RW; ++r) xr[r] = X + size_t(min(i0 + r, n - 1)) * p_pad;   // rows past n: read, not written
  AT z[RW][CB];
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int c = 0; c < CB; ++c) z[r][c] = AT(0);
  for (int j = 4 * lane; j < p_pad; j += 128) {
    AT xv[RW][4];
#pragma unroll
    for (int r = 0; r < RW; ++r) load4<XT, AT>(xr[r] + j, xv[r]);
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      if (c < C) {
        AT b[4];
        load4<AT, AT>(beta + size_t(c) * p_pad + j, b);
#pragma unroll
        for (int r = 0; r < RW; ++r)
          z[r][c] = fma(xv[r][0], b[0], fma(xv[r][1], b[1], fma(xv[r][2], b[2], fma(xv[r][3], b[3], z[r][c]))));
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int c = 0; c < CB; ++c)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) z[r][c] += __shfl_xor_sync(0xffffffffu, z[r][c], o);
#pragma unroll
  for (int r = 0; r < RW; ++r) {
    const int64_t i = i0 + r;
    if (i >= n) break;
    int yi = y[i];
    if (yi < 0 || yi >= Km1 + zlogit) {
      if (lane == 0) atomicOr(err, ERR_BAD_LABEL);
      yi = 0;
    }
    // Lane ch < chains takes chain ch: softmax over its Km1 logits (plus the
    // zero logit of class K in the identifiable layouts), residual and
    // log-likelihood.
    for (int ch = lane; ch < chains; ch += 32) {
      AT m = zlogit ? AT(0) : AT(-INFINITY), zy = AT(0);
#pragma unroll
      for (int c = 0; c < CB; ++c)
        if (c >= ch * Km1 && c < (ch + 1) * Km1) {
          m = max(m, z[r][c]);
          if (c - ch * Km1 == yi) zy = z[r][c];
        }
      AT s = zlogit ? ex<AT>(-m) : AT(0);
#pragma unroll
      for (int c = 0; c < CB; ++c)
        if (c >= ch * Km1 && c < (ch + 1) * Km1) s += ex<AT>(z[r][c] - m);
      const AT inv = AT(1) / s;
#pragma unroll
      for (int c = 0; c < CB; ++c)
        if (c >= ch * Km1 && c < (ch + 1) * Km1)
          R[size_t(i) * C + c] = (c - ch * Km1 == yi ? AT(1) : AT(0)) - ex<AT>(z[r][c] - m) * inv;
      lrow[size_t(i) * lstride + ch] = double(zy - m - lg<AT>(s));
    }
  }
}

// One thread per feature j of the block's 256-feature slice, rows [r0, r1).
template <typename XT, typename AT, int CB>
__global__ void __launch_bounds__(256) grad_kernel(const XT* __restrict__ X, const AT* __restrict__ R, AT* __restrict__ gpart,
                                                   int64_t gpart_cstride, int64_t n, int32_t p_pad, int32_t C, int32_t Q,
                                                   const float* xscale) {
  __shared__ AT rs[kStage][CB];
  const int nfb = (p_pad + 255) / 256;
  const int fb = blockIdx.x % nfb, q = blockIdx.x / nfb;
  const int64_t j = int64_t(fb) * 256 + threadIdx.x;
  const int64_t r0 = int64_t(q) * n / Q, r1 = int64_t(q + 1) * n / Q;
  AT g[CB];
#pragma unroll
  for (int c = 0; c < CB; ++c) g[c] = AT(0);
  for (int64_t i0 = r0; i0 < r1; i0 += kStage) {
    const int rows = int(min(int64_t(kStage), r1 - i0));
    __syncthreads();
    for (int e = threadIdx.x; e < rows * CB; e += blockDim.x) {
      const int rr = e / CB, c = e - rr * CB;
      rs[rr][c] = (c < C) ? R[size_t(i0 + rr) * C + c] : AT(0);
    }
    __syncthreads();
    if (j < p_pad)
      for (int rr = 0; rr < rows; ++rr) {
        const AT xv = AT(X[size_t(i0 + rr) * p_pad + j]);
#pragma unroll
        for (int c = 0; c < CB; ++c) g[c] = fma(xv, rs[rr][c], g[c]);
      }
  }
  if (j < p_pad) {
    const AT sc = xscale ? AT(xscale[j]) : AT(1);
    AT* gp = gpart + size_t(q) * gpart_cstride;
#pragma unroll
    for (int c = 0; c < CB; ++c)
      if (c < C) gp[size_t(c) * p_pad + j] = g[c] * sc;
  }
}

template <typename XT, typename AT, int CB>
cudaError_t launch_cb(const Simt2Launch& L, cudaStream_t s) {
  const XT* X = static_cast<const XT*>(L.X);
  const AT* beta = static_cast<const AT*>(L.beta);
  AT* R = static_cast<AT*>(L.rbuf);
  constexpr int rows = kRowsPerBlock * rows_per_warp<AT, CB>();
  const int64_t b1 = (L.n + rows - 1) / rows;
  logits_kernel<XT, AT, CB><<<dim3(unsigned(b1)), 32 * kRowsPerBlock, 0, s>>>(X, L.y, beta, R, L.lrow, L.lrow_stride, L.n,
                                                                              L.p_pad, L.C, L.Km1, L.chains, L.zlogit, L.err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nfb = (L.p_pad + 255) / 256;
  grad_kernel<XT, AT, CB><<<dim3(unsigned(nfb * L.Q)), 256, 0, s>>>(X, R, static_cast<AT*>(L.gpart), L.gpart_cstride, L.n,
                                                                     L.p_pad, L.C, L.Q, L.xscale);
  return cudaGetLastError();
}

template <typename XT, typename AT>
cudaError_t launch_t(const Simt2Launch& L, cudaStream_t s) {
  if (L.C <= 8) return launch_cb<XT, AT, 8>(L, s);
  if (L.C <= 16) return launch_cb<XT, AT, 16>(L, s);
  if (L.C <= 32) return launch_cb<XT, AT, 32>(L, s);
  return launch_cb<XT, AT, kMaxC>(L, s);
}

}  // namespace simt2

int simt2_max_c() { return simt2::kMaxC; }

// Row ranges of pass 2: enough blocks for about two per SM.
int simt2_row_ranges(int64_t n, int32_t p_pad, int nsm) {
  const int nfb = (p_pad + 255) / 256;
  const int64_t want = std::max<int64_t>(1, (2 * int64_t(nsm) + nfb - 1) / nfb);
  return int(std::max<int64_t>(1, std::min<int64_t>({want, (n + 63) / 64, 64})));
}

cudaError_t simt2_launch(int xt, const Simt2Launch& L, cudaStream_t s) {
  if (L.n == 0) return cudaSuccess;
  if (L.C > simt2::kMaxC || L.p_pad % 4) return cudaErrorInvalidValue;
  if (xt == HMC_F64) return simt2::launch_t<double, double>(L, s);
  return simt2::launch_t<float, float>(L, s);
}

}  // namespace hmc
