// Instantiations of the CUDA-core fused pass for X stored as double.
#include "lpg_simt.cuh"

namespace hmc {
namespace simt {

using KernelFn = void (*)(const LpgArgs);

int table_f64(const int** cts, const KernelFn** fns) {
  static const int kCT[] = {1,2,3,4,6,9,12};
  static const KernelFn kFn[] = {
      lpg_kernel<double, double, 1>,
      lpg_kernel<double, double, 2>,
      lpg_kernel<double, double, 3>,
      lpg_kernel<double, double, 4>,
      lpg_kernel<double, double, 6>,
      lpg_kernel<double, double, 9>,
      lpg_kernel<double, double, 12>,
  };
  *cts = kCT;
  *fns = kFn;
  return int(sizeof(kCT) / sizeof(kCT[0]));
}


using BatchedFn = void (*)(const LpgArgs*, const int*, int, int);

int table_batched_f64(const int** cts, const BatchedFn** fns) {
  static const int kCT[] = {1,2,3,4,6,9,12};
  static const BatchedFn kFn[] = {
      lpg_kernel_batched<double, double, 1>,
      lpg_kernel_batched<double, double, 2>,
      lpg_kernel_batched<double, double, 3>,
      lpg_kernel_batched<double, double, 4>,
      lpg_kernel_batched<double, double, 6>,
      lpg_kernel_batched<double, double, 9>,
      lpg_kernel_batched<double, double, 12>,
  };
  *cts = kCT;
  *fns = kFn;
  return int(sizeof(kCT) / sizeof(kCT[0]));
}

}  // namespace simt
}  // namespace hmc
