// musr_kernels_vg_a.cu -- instantiates the vector-group SPLIT kernels of musr_kernels.cuh for the
// shapes kShapeT1, kShapeN1, kShapeT1N1, kShapeT2.
#include "musr_kernels.cuh"

namespace musr {

int launch_vg_group_a(int shape, int mode, int grad, const Job* j, int n, int items, int sms, cudaStream_t s,
                      LaunchInfo* info) {
  switch (shape) {
    case kShapeT1:
      return kern::dispatch_vg<kShapeT1>(mode, grad, j, n, items, sms, s, info);
    case kShapeN1:
      return kern::dispatch_vg<kShapeN1>(mode, grad, j, n, items, sms, s, info);
    case kShapeT1N1:
      return kern::dispatch_vg<kShapeT1N1>(mode, grad, j, n, items, sms, s, info);
    case kShapeT2:
      return kern::dispatch_vg<kShapeT2>(mode, grad, j, n, items, sms, s, info);
    default:
      return -1;
  }
}

}  // namespace musr
