// musr_kernels_vg_b.cu -- instantiates the vector-group SPLIT kernels of musr_kernels.cuh for the
// shapes kShapeT2N1, kShapeT2m, kShapeT2N1m.
#include "musr_kernels.cuh"

namespace musr {

int launch_vg_group_b(int shape, int mode, int grad, const Job* j, int n, int items, int sms, cudaStream_t s,
                      LaunchInfo* info) {
  switch (shape) {
    case kShapeT2N1:
      return kern::dispatch_vg<kShapeT2N1>(mode, grad, j, n, items, sms, s, info);
    case kShapeT2m:
      return kern::dispatch_vg<kShapeT2m>(mode, grad, j, n, items, sms, s, info);
    case kShapeT2N1m:
      return kern::dispatch_vg<kShapeT2N1m>(mode, grad, j, n, items, sms, s, info);
    default:
      return -1;
  }
}

}  // namespace musr
