// Posterior predictive class probabilities (Sec. 3.2: the predicted class is
// the one with the highest average softmax value over the posterior samples).
//
// For every new row x_i and every posterior draw B_d the kernel forms the
// logits z_idk = x_i . beta_dk of the draw's free classes (plus the implied
// zero logit of class K in the identifiable layouts), the softmax psi_id
// (Eq. softmax), and adds it to an FP64 running sum in draw order; the mean
// over draws and its argmax (lowest class on a tie) are the outputs.
//
// Work split: a block of 8 warps takes 8 rows, one warp per row; the warp's
// lanes stride over the p features, each lane keeping one partial dot product
// per class in registers, and a butterfly reduction gives every lane the full
// logits.  Lane k keeps the FP64 sum of class k.  The row of X stays in L1
// across the draws; every draw's coefficients are read once per block (L2).
// Not on the sampler's hot path: it runs once, after sampling.
#include <cmath>

#include "device_common.cuh"
#include "internal.h"

namespace hmc {
namespace {

constexpr int kWarps = 8;
constexpr int kMaxFree = 32;   // free classes a warp handles (class <-> lane)

template <typename AT>
__device__ __forceinline__ AT ex(AT x);
template <>
__device__ __forceinline__ float ex<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double ex<double>(double x) { return exp(x); }

template <typename IT, typename AT, int KB>
__global__ void __launch_bounds__(32 * kWarps) predict_kernel(const IT* __restrict__ X, int64_t n, int32_t p,
                                                               const AT* __restrict__ draws, int64_t ndraws,
                                                               int32_t ku, int32_t km1, int32_t zlogit, int32_t K,
                                                               double* __restrict__ prob, int32_t* __restrict__ cls) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = int64_t(blockIdx.x) * kWarps + warp;
  if (i >= n) return;
  const IT* xr = X + size_t(i) * p;
  double acc = 0.0;   // lane k: sum over draws of psi_ik
  for (int64_t d = 0; d < ndraws; ++d) {
    const AT* bd = draws + size_t(d) * ku * p;
    AT z[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) z[k] = AT(0);
    for (int j = lane; j < p; j += 32) {
      const AT xv = AT(xr[j]);
#pragma unroll
      for (int k = 0; k < KB; ++k)
        if (k < km1) z[k] = fma(xv, bd[size_t(k) * p + j], z[k]);
    }
#pragma unroll
    for (int k = 0; k < KB; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) z[k] += __shfl_xor_sync(0xffffffffu, z[k], o);
    // Every lane now holds all logits; lane k takes class k.
    AT mine = AT(0), m = zlogit ? AT(0) : AT(-INFINITY);
#pragma unroll
    for (int k = 0; k < KB; ++k)
      if (k < km1) {
        m = max(m, z[k]);
        if (k == lane) mine = z[k];
      }
    AT s = zlogit ? ex<AT>(-m) : AT(0);
#pragma unroll
    for (int k = 0; k < KB; ++k)
      if (k < km1) s += ex<AT>(z[k] - m);
    if (lane < K) acc += double(ex<AT>(mine - m) / s);   // lane km1 (zero logit) has mine = 0
  }
  const double mean = acc / double(ndraws);
  if (prob && lane < K) prob[size_t(i) * K + lane] = mean;
  if (cls) {
    // Fixed-order argmax over the K lanes: strictly greater wins, so a tie keeps
    // the lowest class.
    int best = 0;
    double bv = __shfl_sync(0xffffffffu, mean, 0);
    for (int k = 1; k < K; ++k) {
      const double v = __shfl_sync(0xffffffffu, mean, k);
      if (v > bv) {
        bv = v;
        best = k;
      }
    }
    if (lane == 0) cls[i] = best;
  }
}

template <typename IT, typename AT>
cudaError_t launch_t(const void* X, int64_t n, int32_t p, const void* draws, int64_t ndraws, int32_t ku, int32_t km1,
                     int32_t zlogit, int32_t K, double* prob, int32_t* cls, cudaStream_t s) {
  const int64_t blocks = (n + kWarps - 1) / kWarps;
  const IT* x = static_cast<const IT*>(X);
  const AT* b = static_cast<const AT*>(draws);
  // The class bound is a template parameter so the logits stay in registers.
  if (km1 <= 4)
    predict_kernel<IT, AT, 4><<<dim3(unsigned(blocks)), 32 * kWarps, 0, s>>>(x, n, p, b, ndraws, ku, km1, zlogit, K, prob, cls);
  else if (km1 <= 10)
    predict_kernel<IT, AT, 10><<<dim3(unsigned(blocks)), 32 * kWarps, 0, s>>>(x, n, p, b, ndraws, ku, km1, zlogit, K, prob, cls);
  else if (km1 <= 20)
    predict_kernel<IT, AT, 20><<<dim3(unsigned(blocks)), 32 * kWarps, 0, s>>>(x, n, p, b, ndraws, ku, km1, zlogit, K, prob, cls);
  else
    predict_kernel<IT, AT, kMaxFree><<<dim3(unsigned(blocks)), 32 * kWarps, 0, s>>>(x, n, p, b, ndraws, ku, km1, zlogit, K, prob,
                                                                                  cls);
  return cudaGetLastError();
}

}  // namespace

int predict_max_classes() { return kMaxFree; }

cudaError_t launch_predict(int st, int in_dtype, const void* X, int64_t n, int32_t p, const void* draws, int64_t ndraws,
                           int32_t ku, int32_t km1, int32_t zlogit, int32_t K, double* prob, int32_t* cls,
                           cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (st == HMC_F64)
    return in_dtype == HMC_F64 ? launch_t<double, double>(X, n, p, draws, ndraws, ku, km1, zlogit, K, prob, cls, s)
                               : launch_t<float, double>(X, n, p, draws, ndraws, ku, km1, zlogit, K, prob, cls, s);
  return in_dtype == HMC_F64 ? launch_t<double, float>(X, n, p, draws, ndraws, ku, km1, zlogit, K, prob, cls, s)
                             : launch_t<float, float>(X, n, p, draws, ndraws, ku, km1, zlogit, K, prob, cls, s);
}

}  // namespace hmc
