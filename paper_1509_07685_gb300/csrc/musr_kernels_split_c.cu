// musr_kernels_split_c.cu -- instantiates the SPLIT (kShapeT2m, kShapeT2N1m) kernels of musr_kernels.cuh.
#include "musr_kernels.cuh"

namespace musr {

int launch_group_c(int shape, int mode, int grad, const Job* j, int n, int items, int sms, cudaStream_t s,
                     LaunchInfo* info) {
  switch (shape) {
    case kShapeT2m:
      return kern::dispatch_mode<1, kShapeT2m>(mode, grad, j, n, items, sms, s, info);
    case kShapeT2N1m:
      return kern::dispatch_mode<1, kShapeT2N1m>(mode, grad, j, n, items, sms, s, info);
    default:
      return -1;
  }
}
int occupancy_group_c(int shape, int mode, int grad) {
  switch (shape) {
    case kShapeT2m:
      return kern::occupancy_mode<1, kShapeT2m>(mode, grad);
    case kShapeT2N1m:
      return kern::occupancy_mode<1, kShapeT2N1m>(mode, grad);
    default:
      return 0;
  }
}

}  // namespace musr
