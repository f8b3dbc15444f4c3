// Instantiations of the CUDA-core fused pass for X stored as __nv_fp8_e4m3.
#include "lpg_simt.cuh"

namespace hmc {
namespace simt {

using KernelFn = void (*)(const LpgArgs);

int table_fp8(const int** cts, const KernelFn** fns) {
  static const int kCT[] = {1,2,3,4,6,9,12,16,20};
  static const KernelFn kFn[] = {
      lpg_kernel<__nv_fp8_e4m3, float, 1>,
      lpg_kernel<__nv_fp8_e4m3, float, 2>,
      lpg_kernel<__nv_fp8_e4m3, float, 3>,
      lpg_kernel<__nv_fp8_e4m3, float, 4>,
      lpg_kernel<__nv_fp8_e4m3, float, 6>,
      lpg_kernel<__nv_fp8_e4m3, float, 9>,
      lpg_kernel<__nv_fp8_e4m3, float, 12>,
      lpg_kernel<__nv_fp8_e4m3, float, 16>,
      lpg_kernel<__nv_fp8_e4m3, float, 20>,
  };
  *cts = kCT;
  *fns = kFn;
  return int(sizeof(kCT) / sizeof(kCT[0]));
}


using BatchedFn = void (*)(const LpgArgs*, const int*, int, int);

int table_batched_fp8(const int** cts, const BatchedFn** fns) {
  static const int kCT[] = {1,2,3,4,6,9,12,16,20};
  static const BatchedFn kFn[] = {
      lpg_kernel_batched<__nv_fp8_e4m3, float, 1>,
      lpg_kernel_batched<__nv_fp8_e4m3, float, 2>,
      lpg_kernel_batched<__nv_fp8_e4m3, float, 3>,
      lpg_kernel_batched<__nv_fp8_e4m3, float, 4>,
      lpg_kernel_batched<__nv_fp8_e4m3, float, 6>,
      lpg_kernel_batched<__nv_fp8_e4m3, float, 9>,
      lpg_kernel_batched<__nv_fp8_e4m3, float, 12>,
      lpg_kernel_batched<__nv_fp8_e4m3, float, 16>,
      lpg_kernel_batched<__nv_fp8_e4m3, float, 20>,
  };
  *cts = kCT;
  *fns = kFn;
  return int(sizeof(kCT) / sizeof(kCT[0]));
}

}  // namespace simt
}  // namespace hmc
