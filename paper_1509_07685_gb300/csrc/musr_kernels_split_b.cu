// musr_kernels_split_b.cu -- instantiates the SPLIT (kShapeT2, kShapeT2N1) kernels of musr_kernels.cuh.
#include "musr_kernels.cuh"

namespace musr {

int launch_group_b(int shape, int mode, int grad, const Job* j, int n, int items, int sms, cudaStream_t s,
                     LaunchInfo* info) {
  switch (shape) {
    case kShapeT2:
      return kern::dispatch_mode<1, kShapeT2>(mode, grad, j, n, items, sms, s, info);
    case kShapeT2N1:
      return kern::dispatch_mode<1, kShapeT2N1>(mode, grad, j, n, items, sms, s, info);
    default:
      return -1;
  }
}
int occupancy_group_b(int shape, int mode, int grad) {
  switch (shape) {
    case kShapeT2:
      return kern::occupancy_mode<1, kShapeT2>(mode, grad);
    case kShapeT2N1:
      return kern::occupancy_mode<1, kShapeT2N1>(mode, grad);
    default:
      return 0;
  }
}

}  // namespace musr
