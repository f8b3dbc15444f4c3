// hmc_logpost_grad_noalloc: log K and its gradient for callers that cannot
// allocate device memory at call time.
//
// Who needs it: programs that hand (nearly) all device memory to their own
// pool allocator at start-up, so a library cudaMalloc would fail or force the
// pool to shrink; and code that must not pay cudaMalloc's implicit device-wide
// synchronisation inside a latency-critical loop.  Such callers own X, the
// labels, the coefficients and the outputs; this entry point brings the
// intermediate buffers itself.
//
// The intermediates of the usual path (packed coefficients, the fused pass's
// per-cluster partial gradients and log-likelihoods, the reduction's block
// partials and tickets, the padded gradient) live here in one file-scope
// __device__ array of kScratchBytes.  Every GPU that loads the library holds
// that array until the process exits.  All calls share it: two calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on it and give wrong results.  The array keeps the previous call's
// contents; the only state that must start at zero (the last-block tickets)
// is cleared at the start of every call.
//
// The kernels are the library's own (fused pass, pack, reduce, unpack); only
// where their scratch lives differs.  Nothing here calls cudaMalloc,
// cudaFree or an allocating library routine.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "device_common.cuh"
#include "internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

hmc_status nfail(hmc_status s, const std::string& m) {
  hmc::set_last_error(m);
  return s;
}

#define NA_CUDA(call)                                                                             \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return nfail(HMC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in: a kernel must be given the address returned by
// cudaGetSymbolAddress, taken once per device with that device current.
hmc_status scratch_address(void** out) {
  int dev = 0;
  NA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return nfail(HMC_EUNSUPPORTED, "device ordinal beyond the supported range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return nfail(HMC_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HMC_OK;
}

size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

extern "C" hmc_status hmc_logpost_grad_noalloc(const float* X, int64_t ldx, const int32_t* y, int64_t n, int64_t p,
                                               int32_t K, hmc_prior_kind prior, double prior_scale,
                                               const float* beta, int32_t chains, double* logpost, float* grad,
                                               void* stream_ptr) {
  using namespace hmc;
  hmc::set_last_error(std::string());
  if (n < 0 || p < 1 || K < 2 || K > 1024 || chains < 1) return nfail(HMC_EINVAL, "need n >= 0, p >= 1, 2 <= K <= 1024, chains >= 1");
  if (ldx < p || ldx % 16 != 0) return nfail(HMC_EINVAL, "ldx must be a multiple of 16 and >= p");
  if ((n > 0 && (!X || !y)) || !beta || !logpost || !grad) return nfail(HMC_EINVAL, "NULL pointer argument");
  if (prior != HMC_PRIOR_GAUSSIAN && prior != HMC_PRIOR_CAUCHY) return nfail(HMC_EINVAL, "unknown prior kind");
  if (!(prior_scale > 0.0) || !std::isfinite(prior_scale)) return nfail(HMC_EINVAL, "prior_scale must be finite and > 0");
  const int Km1 = K - 1;
  const int C = chains * Km1;
  if (C > simt_max_ct(HMC_F32))
    return nfail(HMC_EINVAL, "chains * (K-1) = " + std::to_string(C) + " exceeds " + std::to_string(simt_max_ct(HMC_F32)));
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);

  // Tile: cluster size S with column slice PC = ldx / S (no repacking of X).
  const int64_t ntiles = (n + kSimtRows - 1) / kSimtRows;
  SimtTile tile{};
  NA_CUDA(simt_choose(HMC_F32, C, p, ntiles, 0, 0, ldx, &tile));
  if (!tile.S)
    return nfail(HMC_EINVAL, "no tile fits ldx = " + std::to_string(ldx) + " (use a multiple of 256 up to 20480)");
  const int S = tile.S, PC = tile.PC, NT = tile.NT, NS = tile.NSTAGE, maxclu = tile.maxclu;
  const size_t smem = tile.smem;

  // Scratch layout (bytes, 256-aligned pieces).
  const size_t elems = size_t(C) * size_t(ldx);
  const int nblk = update_blocks_per_chain(int64_t(Km1) * ldx);
  size_t off = 0;
  const size_t o_err = off;     off = al256(off + sizeof(int));
  const size_t o_tick = off;    off = al256(off + size_t(chains + 1) * sizeof(unsigned int));
  const size_t o_logk = off;    off = al256(off + size_t(chains) * sizeof(double));
  const size_t o_scal = off;    off = al256(off + size_t(chains) * nblk * 2 * sizeof(double));
  const size_t o_beta = off;    off = al256(off + elems * sizeof(float));
  const size_t o_grad = off;    off = al256(off + elems * sizeof(float));
  const size_t fixed = off;
  // Every cluster of the fused pass writes one partial gradient slice (C x ldx
  // floats), so the array also caps the clusters launched, at about
  // 16 MiB / (4 C ldx) - 2.  Within the tile limits (C <= 12 columns up to
  // ldx = 20480, C <= 20 up to 10240) that is at least 15 slices, more than the
  // 7-9 clusters that fit the GPU at the widest tiles; it can bind only for
  // narrower problems with many row tiles and many resident clusters, which
  // then run on fewer clusters than the occupancy limit allows.
  const size_t per_cluster = al256(elems * sizeof(float)) + al256(size_t(chains) * sizeof(double));
  const int64_t nclu_cap = fixed < kScratchBytes ? int64_t((kScratchBytes - fixed) / per_cluster) : 0;
  if (nclu_cap < 1)
    return nfail(HMC_EINVAL, "problem needs " + std::to_string(fixed + per_cluster) +
                                 " bytes of scratch; the static maximum is " + std::to_string(kScratchBytes));
  int64_t nclu = std::min<int64_t>(maxclu, std::max<int64_t>(ntiles, 1));
  nclu = std::min<int64_t>(nclu, nclu_cap);
  const size_t o_gpart = off;   off = al256(off + size_t(nclu) * elems * sizeof(float));
  const size_t o_lpart = off;   off = al256(off + size_t(nclu) * chains * sizeof(double));
  if (off > kScratchBytes) return nfail(HMC_EINVAL, "scratch layout exceeds the static maximum");

  void* base = nullptr;
  {
    hmc_status s = scratch_address(&base);
    if (s != HMC_OK) return s;
  }
  unsigned char* sc = static_cast<unsigned char*>(base);
  int* err = reinterpret_cast<int*>(sc + o_err);
  unsigned int* tickets = reinterpret_cast<unsigned int*>(sc + o_tick);
  double* logk = reinterpret_cast<double*>(sc + o_logk);
  double* scal = reinterpret_cast<double*>(sc + o_scal);
  float* bpad = reinterpret_cast<float*>(sc + o_beta);
  float* gpad = reinterpret_cast<float*>(sc + o_grad);
  float* gpart = reinterpret_cast<float*>(sc + o_gpart);
  double* lpart = reinterpret_cast<double*>(sc + o_lpart);

  NA_CUDA(cudaMemsetAsync(sc, 0, o_logk, stream));  // error word and tickets start at zero
  NA_CUDA(launch_pack(HMC_F32, beta, bpad, chains, Km1, Km1, int32_t(p), int32_t(ldx), stream));
  if (n > 0) {
    LpgArgs a{};
    a.X = X;
    a.y = y;
    a.xscale = nullptr;
    a.beta = bpad;
    a.gpart = gpart;
    a.gpart_cstride = int64_t(elems);
    a.lpart = lpart;
    a.lpart_cstride = chains;
    a.err = err;
    a.n = n;
    a.p_pad = int32_t(ldx);
    a.PC = PC;
    a.C = C;
    a.Km1 = Km1;
    a.zlogit = 1;
    a.chains = chains;
    a.BM = kSimtRows;
    a.CR = kSimtRows;
    a.S = S;
    a.NT = NT;
    a.NWL = tile.NWL;
    a.NSTAGE = NS;
    a.nclusters = int32_t(nclu);
    a.ntiles = ntiles;
    a.spin_limit = 1ll << 22;
    a.inject_timeout = 0;
    NA_CUDA(simt_launch(HMC_F32, HMC_F32, a, smem, stream, 0));
  }
  UpdateArgs u{};
  u.beta = bpad;
  u.eta = nullptr;
  u.grad = gpad;
  u.gpart = gpart;
  u.gpart_cstride = int64_t(elems);
  u.nparts = n > 0 ? int32_t(nclu) : 0;
  u.nlparts = u.nparts;
  u.lpart = lpart;
  u.lpart_cstride = chains;
  u.logk = logk;
  u.scal = scal;
  u.tickets = tickets;
  u.err = err;
  u.p = int32_t(p);
  u.p_pad = int32_t(ldx);
  u.Km1 = Km1;
  u.ku = Km1;
  u.chains = chains;
  u.nblk = nblk;
  u.prior_kind = prior;
  u.prior_scale = prior_scale;
  NA_CUDA(launch_reduce_update(HMC_F32, u, UPD_SCALARS, stream));
  NA_CUDA(launch_unpack(HMC_F32, gpad, grad, chains, Km1, Km1, int32_t(p), int32_t(ldx), stream));
  NA_CUDA(cudaMemcpyAsync(logpost, logk, size_t(chains) * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  int herr = 0;
  NA_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  NA_CUDA(cudaStreamSynchronize(stream));
  if (herr & ERR_BAD_LABEL)
    return nfail(HMC_ENONFINITE, "a label outside [0, K) (error bits " + std::to_string(herr) + "); outputs are invalid");
  if (herr) return nfail(HMC_ETIMEOUT, "a bounded device wait ran out (error bits " + std::to_string(herr) + ")");
  return HMC_OK;
}
