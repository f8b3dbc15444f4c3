// Per-coefficient kernels of the sampler: fixed-order reduction of the fused
// pass's partial gradients plus the prior term (Eq. gradient), the leapfrog
// momentum / coefficient updates (Eqs. hmc1-hmc3), the momentum draw, the
// Metropolis test with momentum (Eq. accept, kinetic energy eta.eta/2), the
// keep-or-restore select, and the upload / layout conversions.
//
// Scalars (log K, kinetic energy) are summed in FP64: per-block partials in
// fixed slots, combined by the last block of each chain (ticket counter) in a
// fixed tree, so results are bitwise repeatable.
#include <cmath>

#include "device_common.cuh"
#include "internal.h"

namespace hmc {
namespace {

constexpr int kThreads = 256;

// Log-prior term of one coefficient, formed in the state's precision (FP64
// arithmetic is scarce on this GPU) and returned for FP64 accumulation.
template <typename ST>
__device__ __forceinline__ double prior_term(ST b, int kind, double s) {
  if constexpr (sizeof(ST) == 4) {
    const float x = float(b) / float(s);
    if (kind == HMC_PRIOR_CAUCHY) return double(-log1pf(x * x));
    return double(-0.5f * x * x);
  } else {
    const double x = double(b);
    if (kind == HMC_PRIOR_CAUCHY) return -log1p((x / s) * (x / s));
    return -(x * x) / (2.0 * s * s);
  }
}

template <typename ST>
__device__ __forceinline__ ST prior_deriv(ST b, int kind, double s) {
  if (kind == HMC_PRIOR_CAUCHY) return ST(-2.0) * b / (ST(s * s) + b * b);
  return -b / ST(s * s);
}

// Fixed-order block sums of N doubles: a butterfly within each warp (every
// lane ends with the same bits), then the warps' sums in a butterfly of warp 0;
// the results are valid in thread 0.  Plain FP64 additions in a fixed tree:
// the trees here meet at most a few thousand partials, whose rounding stays far
// below what the accept test or the oracle comparisons can see, and every
// dependent FP64 step is slow on this GPU (its FP64 units are few), so the
// chains are kept short and the N sums interleave.
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N]) {
  constexpr int kWarps = kThreads / 32;
  __shared__ double ws[N][kWarps];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();   // ws may still be read by a previous call
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) ws[k][w] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = lane < kWarps ? ws[k][lane] : 0.0;
#pragma unroll
    for (int o = kWarps / 2; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < N; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
}

// Thread t's in-order share of v[i * stride], i = t, t + blockDim, ...: four
// interleaved accumulators (fixed assignment, combined in order) keep the
// dependent FP64 chain a quarter as long.
__device__ __forceinline__ double thread_share(const double* v, int n, size_t stride) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int i = threadIdx.x;
  for (; i + 3 * int(blockDim.x) < n; i += 4 * int(blockDim.x)) {
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] += v[size_t(i + u * int(blockDim.x)) * stride];
  }
  for (; i < n; i += blockDim.x) acc[0] += v[size_t(i) * stride];
  return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// Ticket: true in exactly one block (the last to finish) of chain c.
__device__ __forceinline__ bool last_block(unsigned int* ticket, unsigned int nblk) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == nblk - 1u);
  __syncthreads();
  if (is_last) __threadfence();
  return is_last != 0;
}

// Split-K sum of coefficient `idx` over the partials [b0, b1), in order, four
// loads in flight.
template <typename ST>
__device__ __forceinline__ ST partial_range_sum(const ST* gpi, int64_t cstride, int b0, int b1) {
  ST g = ST(0);
  for (int b = b0; b < b1; b += 4) {
    ST v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (b + k < b1) ? gpi[size_t(b + k) * cstride] : ST(0);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (b + k < b1) g += v[k];
  }
  return g;
}

// The update of coefficient idx (column j of row k = e / p_pad of chain c) from
// its split-K gradient sum g: prior derivative, gradient (also in the user
// layout when asked), momentum and coefficient steps, and the FP64 scalar terms.
template <typename ST>
__device__ __forceinline__ void update_one(const UpdateArgs& A, int mode, int c, int64_t e, int j, size_t idx, ST g,
                                           ST ce, ST eb, double& prior_s, double& kin_s) {
  ST* beta = static_cast<ST*>(A.beta);
  ST* eta = static_cast<ST*>(A.eta);
  ST* grad = static_cast<ST*>(A.grad);
  const ST bv = beta[idx];
  g += prior_deriv(bv, A.prior_kind, A.prior_scale);
  grad[idx] = g;
  if (A.ugrad) {
    ST* ug = static_cast<ST*>(A.ugrad) + size_t(c) * A.ku * A.p;
    const int k = int(e / A.p_pad);
    ug[size_t(k) * A.p + j] = g;
    if (k == 0 && A.ku > A.Km1) ug[size_t(A.Km1) * A.p + j] = ST(0);   // masked row K
  }
  ST ev = ST(0);
  if (mode & (UPD_ETA_HALF | UPD_ETA_FULL)) {
    ev = eta[idx] + ce * g;
    eta[idx] = ev;
  }
  if (mode & UPD_SCALARS) {
    prior_s += prior_term(bv, A.prior_kind, A.prior_scale);
    if (mode & UPD_ACCEPT) kin_s += double(ev) * double(ev);
  }
  if (mode & UPD_BETA) beta[idx] = bv + eb * ev;
}

// GRP: a group of G lanes (A.glanes, a power of two <= 32) shares each coefficient:
// lane l of the group sums the partials [l nparts / G, (l + 1) nparts / G) in
// order and the G range sums meet in a butterfly (every lane of the group ends
// with the same bits: each step adds the same two values); lane 0 of the group
// applies the update.  G = 1 is the plain in-order sum.  V4 (FP32, G = 1, p_pad,
// the slice stride and the state buffers 16-byte aligned): each thread takes four
// consecutive coefficients of one row with 16-byte loads and stores, the same
// arithmetic per coefficient (the gradient sums identical bit for bit); a row's
// last four columns holding padding go through the per-coefficient path.
template <typename ST, bool GRP, bool V4>
__global__ void __launch_bounds__(kThreads) reduce_update_kernel(const UpdateArgs A, int mode) {
  const int c = blockIdx.y;
  const int64_t per_chain = int64_t(A.Km1) * A.p_pad;
  const size_t base = size_t(c) * per_chain;
  const ST* gp = static_cast<const ST*>(A.gpart);
  ST* beta = static_cast<ST*>(A.beta);
  ST* eta = static_cast<ST*>(A.eta);
  ST* grad = static_cast<ST*>(A.grad);
  const ST ce = (mode & UPD_ETA_HALF) ? ST(0.5 * A.eps) : ST(A.eps);
  const ST eb = ST(A.eps);
  const int G = GRP ? A.glanes : 1;                 // a power of two
  const int gsh = GRP ? __ffs(G) - 1 : 0;
  const int lane = threadIdx.x & 31, gl = lane & (G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int b0 = (gl * A.nparts) >> gsh, b1 = ((gl + 1) * A.nparts) >> gsh;
  const int64_t stride = (int64_t(gridDim.x) * blockDim.x) >> gsh;
  double prior_s = 0.0, kin_s = 0.0;
  if constexpr (V4) {
    const int64_t n4 = per_chain / 4;
    for (int64_t e4 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e4 < n4; e4 += int64_t(gridDim.x) * blockDim.x) {
      const int64_t e = 4 * e4;
      const int j = int(e % A.p_pad);
      if (j >= A.p) continue;  // padding columns stay zero
      const size_t idx = base + size_t(e);
      if (j + 4 > A.p) {
        for (int i = 0; j + i < A.p; ++i)
          update_one<ST>(A, mode, c, e + i, j + i, idx + i, partial_range_sum(gp + idx + i, A.gpart_cstride, 0, A.nparts),
                         ce, eb, prior_s, kin_s);
        continue;
      }
      // Split-K sums of the four coefficients, slices in order, four slices in flight.
      float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int b = 0; b < A.nparts; b += 4) {
        float4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          v[k] = (b + k < A.nparts) ? *reinterpret_cast<const float4*>(gp + idx + size_t(b + k) * A.gpart_cstride)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (b + k < A.nparts) {
            g.x += v[k].x;
            g.y += v[k].y;
            g.z += v[k].z;
            g.w += v[k].w;
          }
      }
      const float4 bv = *reinterpret_cast<const float4*>(beta + idx);
      float4 gg;
      gg.x = g.x + prior_deriv(bv.x, A.prior_kind, A.prior_scale);
      gg.y = g.y + prior_deriv(bv.y, A.prior_kind, A.prior_scale);
      gg.z = g.z + prior_deriv(bv.z, A.prior_kind, A.prior_scale);
      gg.w = g.w + prior_deriv(bv.w, A.prior_kind, A.prior_scale);
      *reinterpret_cast<float4*>(grad + idx) = gg;
      if (A.ugrad) {
        ST* ug = static_cast<ST*>(A.ugrad) + size_t(c) * A.ku * A.p;
        const int k = int(e / A.p_pad);
        ST* row = ug + size_t(k) * A.p + j;
        row[0] = gg.x;
        row[1] = gg.y;
        row[2] = gg.z;
        row[3] = gg.w;
        if (k == 0 && A.ku > A.Km1)   // masked row K
          for (int i = 0; i < 4; ++i) ug[size_t(A.Km1) * A.p + j + i] = ST(0);
      }
      float4 ev = make_float4(0.f, 0.f, 0.f, 0.f);
      if (mode & (UPD_ETA_HALF | UPD_ETA_FULL)) {
        const float4 e0 = *reinterpret_cast<const float4*>(eta + idx);
        ev = make_float4(e0.x + ce * gg.x, e0.y + ce * gg.y, e0.z + ce * gg.z, e0.w + ce * gg.w);
        *reinterpret_cast<float4*>(eta + idx) = ev;
      }
      if (mode & UPD_SCALARS) {
        prior_s += prior_term(bv.x, A.prior_kind, A.prior_scale);
        prior_s += prior_term(bv.y, A.prior_kind, A.prior_scale);
        prior_s += prior_term(bv.z, A.prior_kind, A.prior_scale);
        prior_s += prior_term(bv.w, A.prior_kind, A.prior_scale);
        if (mode & UPD_ACCEPT)
          kin_s += ((double(ev.x) * double(ev.x) + double(ev.y) * double(ev.y)) + double(ev.z) * double(ev.z)) +
                   double(ev.w) * double(ev.w);
      }
      if (mode & UPD_BETA)
        *reinterpret_cast<float4*>(beta + idx) =
            make_float4(bv.x + eb * ev.x, bv.y + eb * ev.y, bv.z + eb * ev.z, bv.w + eb * ev.w);
    }
  } else {
    for (int64_t e = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> gsh; e < per_chain; e += stride) {
      const int j = int(e % A.p_pad);
      if (j >= A.p) continue;  // padding columns stay zero (the whole group skips)
      const size_t idx = base + size_t(e);
      ST g = partial_range_sum(gp + idx, A.gpart_cstride, b0, b1);
      if (GRP) {
        for (int o = 1; o < G; o <<= 1) g += __shfl_xor_sync(gmask, g, o);
        if (gl != 0) continue;
      }
      update_one<ST>(A, mode, c, e, j, idx, g, ce, eb, prior_s, kin_s);
    }
  }
  if (!(mode & UPD_SCALARS)) return;
  double bs[2] = {prior_s, kin_s};
  block_sum<2>(bs);
  if (threadIdx.x == 0) {
    double* sl = A.scal + (size_t(c) * A.nblk + blockIdx.x) * 2;
    sl[0] = bs[0];
    sl[1] = bs[1];
  }
  if (!last_block(A.tickets + c, gridDim.x)) return;
  // The whole last block sums the block partials and the log-likelihood
  // partials of the gradient pass, each in a fixed order, in one tree.
  const double* sl = A.scal + size_t(c) * A.nblk * 2;
  double tot[3] = {thread_share(sl, int(gridDim.x), 2), thread_share(sl + 1, int(gridDim.x), 2),
                   thread_share(A.lpart + c, A.nlparts, size_t(A.lpart_cstride))};
  block_sum<3>(tot);
  const double prv = tot[0], kiv = tot[1], liv = tot[2];
  if (threadIdx.x != 0) return;
  const double logk = liv + prv;
  A.tickets[c] = 0u;
  if (!(mode & UPD_ACCEPT)) {
    A.logk[c] = logk;
    if (A.ulogk) A.ulogk[c] = logk;
    return;
  }
  const int64_t it = *A.iter;
  const double T = A.temps ? A.temps[*A.local_iter] : 1.0;
  const double h0 = A.h0[c];
  const double h1 = -logk + 0.5 * kiv;
  const bool finite = isfinite(h1);
  const double u = accept_uniform(*A.seed, uint64_t(it), uint64_t(c) | (uint64_t(A.chains_word_hi) << 32));
  const bool acc = finite && (log(u) < (h0 - h1) / T);
  A.accept[c] = acc ? 1 : 0;
  hmc_chain_stats* st = static_cast<hmc_chain_stats*>(A.stats) + c;
  st->iterations += 1;
  st->accepted += acc ? 1 : 0;
  st->diverged += finite ? 0 : 1;
  if (finite) st->sum_abs_dH += fabs(h1 - h0);
  const double kept = acc ? logk : A.logk0[c];
  A.logk[c] = kept;
  st->logpost = kept;
}

// Start of a trajectory: eta ~ N(0, I), save (beta, grad, log K), H0, then
// the first momentum half step and the first coefficient step.
template <typename ST>
__global__ void __launch_bounds__(kThreads) traj_start_kernel(const UpdateArgs A) {
  const int c = blockIdx.y;
  const int64_t per_chain_q = int64_t(A.Km1) * A.p;
  const int64_t nqb = (per_chain_q + 3) / 4;
  const size_t base = size_t(c) * A.Km1 * A.p_pad;
  ST* beta = static_cast<ST*>(A.beta);
  ST* eta = static_cast<ST*>(A.eta);
  const ST* grad = static_cast<const ST*>(A.grad);
  ST* beta0 = static_cast<ST*>(A.beta0);
  ST* grad0 = static_cast<ST*>(A.grad0);
  const uint64_t it = uint64_t(*A.iter);
  const uint64_t seed = *A.seed;
  const uint64_t chain_word = uint64_t(c) | (uint64_t(A.chains_word_hi) << 32);
  const ST half = ST(0.5 * A.eps), full = ST(A.eps);
  double kin = 0.0;
  for (int64_t qb = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; qb < nqb; qb += int64_t(gridDim.x) * blockDim.x) {
    double z[4];
    momentum_block(seed, it, chain_word, uint64_t(qb), z);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t q = qb * 4 + r;
      if (q >= per_chain_q) break;
      const int64_t k = q / A.p, j = q - k * A.p;
      const size_t idx = base + size_t(k) * A.p_pad + size_t(j);
      const ST e = ST(z[r]);
      kin += double(e) * double(e);
      const ST b = beta[idx], g = grad[idx];
      beta0[idx] = b;
      grad0[idx] = g;
      const ST eh = e + half * g;
      eta[idx] = eh;
      beta[idx] = b + full * eh;
    }
  }
  double kb[1] = {kin};
  block_sum<1>(kb);
  if (threadIdx.x == 0) A.scal[(size_t(c) * A.nblk + blockIdx.x) * 2 + 1] = kb[0];
  if (!last_block(A.tickets + c, gridDim.x)) return;
  double kt[1] = {thread_share(A.scal + size_t(c) * A.nblk * 2 + 1, int(gridDim.x), 2)};
  block_sum<1>(kt);
  const double kiv = kt[0];
  if (threadIdx.x != 0) return;
  A.tickets[c] = 0u;
  A.logk0[c] = A.logk[c];
  A.h0[c] = -A.logk[c] + 0.5 * kiv;
}

// Keep the proposal or restore the trajectory start; write the sample; the
// last block advances the iteration counters.
template <typename ST>
__global__ void __launch_bounds__(kThreads) select_kernel(const UpdateArgs A, unsigned int* ticket_all) {
  const int c = blockIdx.y;
  const int64_t per_chain = int64_t(A.Km1) * A.p_pad;
  const size_t base = size_t(c) * per_chain;
  ST* beta = static_cast<ST*>(A.beta);
  ST* grad = static_cast<ST*>(A.grad);
  const ST* beta0 = static_cast<const ST*>(A.beta0);
  const ST* grad0 = static_cast<const ST*>(A.grad0);
  const bool acc = A.accept[c] != 0;
  const int64_t li = *A.local_iter;
  ST* out = nullptr;
  if (A.samples && ((li + 1) % A.thin) == 0) {
    const int64_t slot = (li + 1) / A.thin - 1;
    out = static_cast<ST*>(A.samples) + size_t(slot) * A.sample_slot_stride + size_t(c) * A.ku * A.p;
    // Rows past the free ones (the masked row K) are zero in every sample.
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < int64_t(A.ku - A.Km1) * A.p;
         e += int64_t(gridDim.x) * blockDim.x)
      out[size_t(A.Km1) * A.p + size_t(e)] = ST(0);
  }
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < per_chain;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = e / A.p_pad, j = e - k * A.p_pad;
    if (j >= A.p) continue;
    const size_t idx = base + size_t(e);
    ST b = beta[idx];
    if (!acc) {
      b = beta0[idx];
      beta[idx] = b;
      grad[idx] = grad0[idx];
    }
    if (out) out[size_t(k) * A.p + size_t(j)] = b;
  }
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(ticket_all, 1u) == gridDim.x * gridDim.y - 1u);
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    *ticket_all = 0u;
    *A.iter += 1;
    *A.local_iter += 1;
  }
}

// hmc_leapfrog start: first half step of the momentum and first coefficient step.
template <typename ST>
__global__ void leap_start_kernel(const UpdateArgs A, int64_t total) {
  ST* beta = static_cast<ST*>(A.beta);
  ST* eta = static_cast<ST*>(A.eta);
  const ST* grad = static_cast<const ST*>(A.grad);
  const ST half = ST(0.5 * A.eps), full = ST(A.eps);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const ST e = eta[i] + half * grad[i];
    eta[i] = e;
    beta[i] = beta[i] + full * e;
  }
}

// [chains][ku][p] -> [chains][km1][p_pad]: rows past km1 of a chain are dropped,
// padding columns are zero.
template <typename T>
__global__ void pack_kernel(const T* src, T* dst, int64_t chains, int32_t ku, int32_t km1, int32_t p, int32_t p_pad) {
  const int64_t total = chains * km1 * p_pad;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / p_pad, j = i - r * p_pad;
    const int64_t c = r / km1, k = r - c * km1;
    dst[i] = (j < p) ? src[(c * ku + k) * p + j] : T(0);
  }
}

// [chains][km1][p_pad] -> [chains][ku][p]: rows past km1 of a chain are zero.
template <typename T>
__global__ void unpack_kernel(const T* src, T* dst, int64_t chains, int32_t ku, int32_t km1, int32_t p,
                              int32_t p_pad) {
  const int64_t total = chains * ku * p;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / p, j = i - r * p;
    const int64_t c = r / ku, k = r - c * ku;
    dst[i] = (k < km1) ? src[(c * km1 + k) * p_pad + j] : T(0);
  }
}

template <typename IT>
__device__ __forceinline__ float to_f32(IT v) {
  return float(v);
}

template <typename IT, typename XT>
__global__ void convert_x_kernel(const IT* src, XT* dst, const float* scales, int64_t n, int32_t p, int32_t p_pad,
                                 int* err) {
  const int64_t total = n * p_pad;
  int bad = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / p_pad, j = i - r * p_pad;
    if (j >= p) {
      dst[i] = XT(0.0f);
      continue;
    }
    const IT v = src[r * p + j];
    if (!isfinite(double(v))) bad = 1;
    if constexpr (std::is_same<XT, double>::value) {
      dst[i] = double(v);
    } else if constexpr (std::is_same<XT, float>::value) {
      dst[i] = float(v);
    } else if constexpr (std::is_same<XT, __nv_bfloat16>::value) {
      dst[i] = __float2bfloat16_rn(float(v));
    } else {
      const float q = float(v) / scales[j];
      __nv_fp8_e4m3 o;
      o.__x = __nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
      dst[i] = o;
    }
  }
  if (bad) atomicOr(err, ERR_NONFINITE_X);
}

template <typename IT>
__global__ void fp8_scale_kernel(const IT* src, float* scales, int64_t n, int32_t p, int32_t p_pad) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p_pad) return;
  if (j >= p) {
    scales[j] = 1.0f;
    return;
  }
  float amax = 0.0f;
  for (int64_t r = 0; r < n; ++r) amax = fmaxf(amax, fabsf(float(src[r * p + j])));
  scales[j] = (amax == 0.0f) ? 1.0f : amax / 448.0f;
}

__global__ void check_labels_kernel(const int32_t* y, int64_t n, int32_t K, int* err) {
  int bad = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    if (y[i] < 0 || y[i] >= K) bad = 1;
  if (bad) atomicOr(err, ERR_BAD_LABEL);
}

__global__ void init_stats_kernel(hmc_chain_stats* s, int chains) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < chains) s[c] = hmc_chain_stats{0, 0, 0, 0.0, 0.0};
}

int grid_for(int64_t work, int cap = 4096) {
  int64_t g = (work + kThreads - 1) / kThreads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return int(g);
}

}  // namespace

int update_group_lanes(int64_t per_chain, int chains, int nparts, int nsm) {
  // Lanes sharing one coefficient's split-K sum: more where few coefficients
  // meet many partials (a small call waits for about nparts / 8 dependent load
  // rounds), while the threads stay within half a wave.
  int G = 1;
  while (G < 32 && nparts >= 16 * G && per_chain * chains * G * 2 <= int64_t(nsm) * 2048) G *= 2;
  return G;
}

int update_blocks_per_chain(int64_t per_chain) {
  // About one coefficient (times its group lanes) per thread: the split-K sum
  // is latency-bound.
  int64_t g = (per_chain + kThreads - 1) / kThreads;
  if (g < 1) g = 1;
  if (g > 1024) g = 1024;
  return int(g);
}

cudaError_t launch_reduce_update(int st, const UpdateArgs& a, int mode, cudaStream_t s) {
  dim3 grid(a.nblk, a.chains);
  const bool grp = a.glanes > 1;
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  if (st == HMC_F64) {
    if (grp) reduce_update_kernel<double, true, false><<<grid, kThreads, 0, s>>>(a, mode);
    else reduce_update_kernel<double, false, false><<<grid, kThreads, 0, s>>>(a, mode);
  } else if (grp) {
    reduce_update_kernel<float, true, false><<<grid, kThreads, 0, s>>>(a, mode);
  } else if (a.p_pad % 4 == 0 && a.gpart_cstride % 4 == 0 && al16(a.gpart) && al16(a.beta) && al16(a.eta) &&
             al16(a.grad)) {
    // four coefficients per thread: a quarter of the blocks (their partial
    // slots and the last-block ticket follow gridDim.x)
    grid.x = std::max(1, (a.nblk + 3) / 4);
    reduce_update_kernel<float, false, true><<<grid, kThreads, 0, s>>>(a, mode);
  } else {
    reduce_update_kernel<float, false, false><<<grid, kThreads, 0, s>>>(a, mode);
  }
  return cudaGetLastError();
}

cudaError_t launch_traj_start(int st, const UpdateArgs& a, cudaStream_t s) {
  dim3 grid(a.nblk, a.chains);
  if (st == HMC_F64)
    traj_start_kernel<double><<<grid, kThreads, 0, s>>>(a);
  else
    traj_start_kernel<float><<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_select(int st, const UpdateArgs& a, unsigned int* ticket_all, cudaStream_t s) {
  dim3 grid(a.nblk, a.chains);
  if (st == HMC_F64)
    select_kernel<double><<<grid, kThreads, 0, s>>>(a, ticket_all);
  else
    select_kernel<float><<<grid, kThreads, 0, s>>>(a, ticket_all);
  return cudaGetLastError();
}

cudaError_t launch_leap_start(int st, const UpdateArgs& a, cudaStream_t s) {
  const int64_t total = int64_t(a.chains) * a.Km1 * a.p_pad;
  if (st == HMC_F64)
    leap_start_kernel<double><<<grid_for(total), kThreads, 0, s>>>(a, total);
  else
    leap_start_kernel<float><<<grid_for(total), kThreads, 0, s>>>(a, total);
  return cudaGetLastError();
}

cudaError_t launch_pack(int st, const void* src, void* dst, int64_t chains, int32_t ku, int32_t km1, int32_t p,
                        int32_t p_pad, cudaStream_t s) {
  const int g = grid_for(chains * km1 * p_pad);
  if (st == HMC_F64)
    pack_kernel<double><<<g, kThreads, 0, s>>>(static_cast<const double*>(src), static_cast<double*>(dst), chains, ku,
                                               km1, p, p_pad);
  else
    pack_kernel<float><<<g, kThreads, 0, s>>>(static_cast<const float*>(src), static_cast<float*>(dst), chains, ku, km1,
                                              p, p_pad);
  return cudaGetLastError();
}

cudaError_t launch_unpack(int st, const void* src, void* dst, int64_t chains, int32_t ku, int32_t km1, int32_t p,
                          int32_t p_pad, cudaStream_t s) {
  const int g = grid_for(chains * ku * p);
  if (st == HMC_F64)
    unpack_kernel<double><<<g, kThreads, 0, s>>>(static_cast<const double*>(src), static_cast<double*>(dst), chains, ku,
                                                 km1, p, p_pad);
  else
    unpack_kernel<float><<<g, kThreads, 0, s>>>(static_cast<const float*>(src), static_cast<float*>(dst), chains, ku,
                                                km1, p, p_pad);
  return cudaGetLastError();
}

template <typename IT>
static cudaError_t convert_from(const IT* src, int xt, void* dst, const float* scales, int64_t n, int32_t p, int32_t p_pad,
                                int* err, cudaStream_t s) {
  const int g = grid_for(n * p_pad, 8192);
  switch (xt) {
    case HMC_F64:
      convert_x_kernel<IT, double><<<g, kThreads, 0, s>>>(src, static_cast<double*>(dst), scales, n, p, p_pad, err);
      break;
    case HMC_F32:
      convert_x_kernel<IT, float><<<g, kThreads, 0, s>>>(src, static_cast<float*>(dst), scales, n, p, p_pad, err);
      break;
    case HMC_BF16:
      convert_x_kernel<IT, __nv_bfloat16><<<g, kThreads, 0, s>>>(src, static_cast<__nv_bfloat16*>(dst), scales, n, p,
                                                                   p_pad, err);
      break;
    default:
      convert_x_kernel<IT, __nv_fp8_e4m3><<<g, kThreads, 0, s>>>(src, static_cast<__nv_fp8_e4m3*>(dst), scales, n, p,
                                                                   p_pad, err);
  }
  return cudaGetLastError();
}

cudaError_t launch_convert_x(int in_dtype, const void* src, int xt, void* dst, const float* scales, int64_t n, int32_t p,
                             int32_t p_pad, int* err, cudaStream_t s) {
  if (in_dtype == HMC_F64) return convert_from(static_cast<const double*>(src), xt, dst, scales, n, p, p_pad, err, s);
  return convert_from(static_cast<const float*>(src), xt, dst, scales, n, p, p_pad, err, s);
}

cudaError_t launch_fp8_scales(int in_dtype, const void* src, float* scales, int64_t n, int32_t p, int32_t p_pad,
                              cudaStream_t s) {
  const int g = (p_pad + kThreads - 1) / kThreads;
  if (in_dtype == HMC_F64)
    fp8_scale_kernel<double><<<g, kThreads, 0, s>>>(static_cast<const double*>(src), scales, n, p, p_pad);
  else
    fp8_scale_kernel<float><<<g, kThreads, 0, s>>>(static_cast<const float*>(src), scales, n, p, p_pad);
  return cudaGetLastError();
}

cudaError_t launch_check_labels(const int32_t* y, int64_t n, int32_t K, int* err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  check_labels_kernel<<<grid_for(n), kThreads, 0, s>>>(y, n, K, err);
  return cudaGetLastError();
}

cudaError_t launch_init_stats(void* stats, int chains, cudaStream_t s) {
  init_stats_kernel<<<(chains + 127) / 128, 128, 0, s>>>(static_cast<hmc_chain_stats*>(stats), chains);
  return cudaGetLastError();
}

}  // namespace hmc
