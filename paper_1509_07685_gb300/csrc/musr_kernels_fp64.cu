// musr_kernels_fp64.cu -- instantiates the FP64-path kernels of musr_kernels.cuh.
#include "musr_kernels.cuh"

namespace musr {

int launch_group_fp64(int mode, int grad, const Job* j, int n, int items, int sms, cudaStream_t s, LaunchInfo* info) {
  return kern::dispatch_mode<0, 0>(mode, grad, j, n, items, sms, s, info);
}
int occupancy_group_fp64(int mode, int grad) { return kern::occupancy_mode<0, 0>(mode, grad); }

}  // namespace musr
