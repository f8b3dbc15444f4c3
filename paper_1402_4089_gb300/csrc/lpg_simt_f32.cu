// Instantiations of the CUDA-core fused pass for X stored as float.
#include "lpg_simt.cuh"

namespace hmc {
namespace simt {

using KernelFn = void (*)(const LpgArgs);

int table_f32(const int** cts, const KernelFn** fns) {
  static const int kCT[] = {1,2,3,4,6,9,12,16,20};
  static const KernelFn kFn[] = {
      lpg_kernel<float, float, 1>,
      lpg_kernel<float, float, 2>,
      lpg_kernel<float, float, 3>,
      lpg_kernel<float, float, 4>,
      lpg_kernel<float, float, 6>,
      lpg_kernel<float, float, 9>,
      lpg_kernel<float, float, 12>,
      lpg_kernel<float, float, 16>,
      lpg_kernel<float, float, 20>,
  };
  *cts = kCT;
  *fns = kFn;
  return int(sizeof(kCT) / sizeof(kCT[0]));
}


using BatchedFn = void (*)(const LpgArgs*, const int*, int, int);

int table_batched_f32(const int** cts, const BatchedFn** fns) {
  static const int kCT[] = {1,2,3,4,6,9,12,16,20};
  static const BatchedFn kFn[] = {
      lpg_kernel_batched<float, float, 1>,
      lpg_kernel_batched<float, float, 2>,
      lpg_kernel_batched<float, float, 3>,
      lpg_kernel_batched<float, float, 4>,
      lpg_kernel_batched<float, float, 6>,
      lpg_kernel_batched<float, float, 9>,
      lpg_kernel_batched<float, float, 12>,
      lpg_kernel_batched<float, float, 16>,
      lpg_kernel_batched<float, float, 20>,
  };
  *cts = kCT;
  *fns = kFn;
  return int(sizeof(kCT) / sizeof(kCT[0]));
}

}  // namespace simt
}  // namespace hmc
