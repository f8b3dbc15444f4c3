// Host side of the CUDA-core fused pass: instantiation lookup, shared-memory
// sizing, function attributes, occupancy query and the cluster launch.
#include "lpg_simt.cuh"

#include <algorithm>

namespace hmc {
namespace simt {

using KernelFn = void (*)(const LpgArgs);
using BatchedFn = void (*)(const LpgArgs*, const int*, int, int);
int table_batched_f64(const int** cts, const BatchedFn** fns);
int table_batched_f32(const int** cts, const BatchedFn** fns);
int table_batched_bf16(const int** cts, const BatchedFn** fns);
int table_batched_fp8(const int** cts, const BatchedFn** fns);

static BatchedFn pick_batched(int xt, int C, int* ct) {
  const int* cts;
  const BatchedFn* fns;
  int m = 0;
  switch (xt) {
    case HMC_F64: m = table_batched_f64(&cts, &fns); break;
    case HMC_F32: m = table_batched_f32(&cts, &fns); break;
    case HMC_BF16: m = table_batched_bf16(&cts, &fns); break;
    default: m = table_batched_fp8(&cts, &fns);
  }
  for (int i = 0; i < m; ++i)
    if (cts[i] >= C) {
      *ct = cts[i];
      return fns[i];
    }
  *ct = 0;
  return nullptr;
}
int table_f64(const int** cts, const KernelFn** fns);
int table_f32(const int** cts, const KernelFn** fns);
int table_bf16(const int** cts, const KernelFn** fns);
int table_fp8(const int** cts, const KernelFn** fns);

static int table(int xt, const int** cts, const KernelFn** fns) {
  switch (xt) {
    case HMC_F64: return table_f64(cts, fns);
    case HMC_F32: return table_f32(cts, fns);
    case HMC_BF16: return table_bf16(cts, fns);
    default: return table_fp8(cts, fns);
  }
}

// Smallest instantiated class bound >= C; returns the kernel (nullptr if none).
static KernelFn pick(int xt, int C, int* ct) {
  const int* cts;
  const KernelFn* fns;
  const int m = table(xt, &cts, &fns);
  for (int i = 0; i < m; ++i)
    if (cts[i] >= C) {
      *ct = cts[i];
      return fns[i];
    }
  *ct = 0;
  return nullptr;
}

}  // namespace simt

int simt_ct_of(int xt, int C) {
  int ct = 0;
  simt::pick(xt, C, &ct);
  return ct;
}

int simt_max_grad_warps(int xt, int C) {
  const int ct = simt_ct_of(xt, C);
  return simt::max_grad_warps(xt == HMC_F64 ? 8 : 4, ct);
}

int simt_logit_warps(int nwc) { return simt::logit_warps(nwc); }

int simt_max_ct(int xt) {
  const int* cts;
  const simt::KernelFn* fns;
  const int m = simt::table(xt, &cts, &fns);
  return cts[m - 1];
}

size_t simt_smem_bytes(int xt, int /*st*/, int C, int PC, int S, int NWL, int NSTAGE) {
  int ct = 0;
  if (!simt::pick(xt, C, &ct)) return ~size_t(0);
  const int xbytes = xt == HMC_F64 ? 8 : xt == HMC_F32 ? 4 : xt == HMC_BF16 ? 2 : 1;
  const int abytes = xt == HMC_F64 ? 8 : 4;
  const simt::ShapeRT sh = simt::shape_rt(abytes, ct);
  return simt::layout(xbytes, abytes, ct, sh.CTP, sh.V, sh.A, PC, S, NWL, NSTAGE).total;
}

cudaError_t simt_prepare(int xt, int /*st*/, int C, size_t smem, int S) {
  int ct = 0;
  simt::KernelFn fn = simt::pick(xt, C, &ct);
  if (!fn) return cudaErrorInvalidValue;
  // The opt-in is a per-function upper bound shared by every handle: set it to
  // the device maximum so no handle can lower it below another's need.
  int dev = 0, smem_max = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smem > size_t(smem_max)) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e != cudaSuccess) return e;
  if (S > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

static void fill_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int grid, int S, int NT, size_t smem,
                        cudaStream_t stream) {
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cfg.numAttrs = 0;
  cfg.attrs = attr;
  if (S > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.numAttrs = 1;
  }
}

cudaError_t simt_max_active_clusters(int xt, int /*st*/, int C, size_t smem, int S, int NT, int* out) {
  int ct = 0;
  simt::KernelFn fn = simt::pick(xt, C, &ct);
  if (!fn) return cudaErrorInvalidValue;
  if (S == 1) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *out = per_sm * sms;
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, S, S, NT, smem, nullptr);
  return cudaOccupancyMaxActiveClusters(out, fn, &cfg);
}

static int xbytes_of(int xt) { return xt == HMC_F64 ? 8 : xt == HMC_F32 ? 4 : xt == HMC_BF16 ? 2 : 1; }

cudaError_t simt_choose(int xt, int C, int64_t p, int64_t ntiles, int force_S, int force_NS, int64_t exact_ld,
                        SimtTile* out) {
  *out = SimtTile{};
  int dev = 0, smem_max = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const int64_t want = std::max<int64_t>(1, ntiles);
  int nsm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int64_t best_active = -1;
  // Without a forced size, a cluster is no wider than gives each CTA ~256 real
  // columns: below that the extra CTAs hold mostly padding and every tile pays
  // a wider logit exchange (p = 50: 10.3 us per pass at S = 1 against 15.0 us at
  // the S = 12 the occupancy model alone would pick; p = 100: 11.2 against 15.0).
  const int64_t s_cap = (force_S || exact_ld > 0) ? 16 : std::max<int64_t>(1, (p + 255) / 256);
  for (int S : {1, 2, 3, 4, 5, 6, 8, 10, 12, 16}) {
    if (force_S && S != force_S) continue;
    if (S > s_cap) continue;
    int64_t PC;
    if (exact_ld > 0) {
      if (exact_ld % (16 * S)) continue;
      PC = exact_ld / S;
    } else {
      // Slices start on 128-byte boundaries: bulk copies from unaligned
      // slices stream far slower.
      const int64_t al = std::max(16, 128 / xbytes_of(xt));
      PC = ((p + S - 1) / S + al - 1) / al * al;
    }
    if (PC < 16) PC = 16;
    const int NWC = int((PC + 127) / 128);
    if (NWC > simt_max_grad_warps(xt, C)) continue;
    const int NWL = simt_logit_warps(NWC);
    const int NT = 32 * (NWC + NWL + 1);
    for (int NS = 6; NS >= 2; --NS) {
      if (force_NS && NS != force_NS) continue;
      const size_t smem = simt_smem_bytes(xt, 0, C, int(PC), S, NWL, NS);
      if (smem > size_t(smem_max)) continue;
      e = simt_prepare(xt, 0, C, smem, S);
      if (e != cudaSuccess) return e;
      int maxclu = 0;
      e = simt_max_active_clusters(xt, 0, C, smem, S, NT, &maxclu);
      if (e != cudaSuccess) {
        cudaGetLastError();
        break;
      }
      if (maxclu < 1) break;
      // Most SMs streaming X (CTAs that share an SM share its issue slots and
      // bandwidth, so they count once), then the smaller cluster (fewer logit
      // exchanges).
      int per_sm = 1;
      {
        int ct = 0;
        simt::KernelFn fn = simt::pick(xt, C, &ct);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem) != cudaSuccess || per_sm < 1) {
          cudaGetLastError();
          per_sm = 1;
        }
      }
      const int64_t active = std::min<int64_t>(nsm, (std::min<int64_t>(maxclu, want) * S + per_sm - 1) / per_sm);
      if (active > best_active) {
        best_active = active;
        *out = SimtTile{S, int(PC), NWC, NWL, NT, NS, smem, maxclu};
      }
      break;  // deepest ring that fits for this cluster size
    }
  }
  return cudaSuccess;
}

cudaError_t simt_prepare_batched(int xt, int C, int S) {
  int ct = 0;
  simt::BatchedFn fn = simt::pick_batched(xt, C, &ct);
  if (!fn) return cudaErrorInvalidValue;
  int dev = 0, smem_max = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max - 1024);
  if (e == cudaSuccess && S > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t simt_max_active_clusters_batched(int xt, int C, size_t smem, int S, int NT, int* out) {
  int ct = 0;
  simt::BatchedFn fn = simt::pick_batched(xt, C, &ct);
  if (!fn) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, S, S, NT, smem, nullptr);
  if (S == 1) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *out = per_sm * sms;
    return cudaSuccess;
  }
  return cudaOccupancyMaxActiveClusters(out, fn, &cfg);
}

cudaError_t simt_launch_batched(int xt, int C, const LpgArgs* table, const int* first, int nprob, int chains,
                                int total_clusters, int S, int NT, size_t smem, cudaStream_t stream) {
  int ct = 0;
  simt::BatchedFn fn = simt::pick_batched(xt, C, &ct);
  if (!fn) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, total_clusters * S, S, NT, smem, stream);
  return cudaLaunchKernelEx(&cfg, fn, table, first, nprob, chains);
}

cudaError_t simt_launch(int xt, int /*st*/, const LpgArgs& a, size_t smem, cudaStream_t stream, int C_kernel) {
  int ct = 0;
  simt::KernelFn fn = simt::pick(xt, C_kernel > a.C ? C_kernel : a.C, &ct);
  if (!fn) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, a.nclusters * a.S, a.S, a.NT, smem, stream);
  return cudaLaunchKernelEx(&cfg, fn, a);
}

}  // namespace hmc
