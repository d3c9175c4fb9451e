// musr_kernels_split_a.cu -- instantiates the SPLIT (kShapeGeneric, kShapeT1, kShapeN1, kShapeT1N1, kShapeList, kShapeListS) kernels of musr_kernels.cuh.
#include "musr_kernels.cuh"

namespace musr {

int launch_group_a(int shape, int mode, int grad, const Job* j, int n, int items, int sms, cudaStream_t s,
                     LaunchInfo* info) {
  switch (shape) {
    case kShapeGeneric:
      return kern::dispatch_mode<1, kShapeGeneric>(mode, grad, j, n, items, sms, s, info);
    case kShapeT1:
      return kern::dispatch_mode<1, kShapeT1>(mode, grad, j, n, items, sms, s, info);
    case kShapeN1:
      return kern::dispatch_mode<1, kShapeN1>(mode, grad, j, n, items, sms, s, info);
    case kShapeT1N1:
      return kern::dispatch_mode<1, kShapeT1N1>(mode, grad, j, n, items, sms, s, info);
    case kShapeList:
      return kern::dispatch_mode<1, kShapeList>(mode, grad, j, n, items, sms, s, info);
    case kShapeListS:
      return kern::dispatch_mode<1, kShapeListS>(mode, grad, j, n, items, sms, s, info);
    default:
      return -1;
  }
}
int occupancy_group_a(int shape, int mode, int grad) {
  switch (shape) {
    case kShapeGeneric:
      return kern::occupancy_mode<1, kShapeGeneric>(mode, grad);
    case kShapeT1:
      return kern::occupancy_mode<1, kShapeT1>(mode, grad);
    case kShapeN1:
      return kern::occupancy_mode<1, kShapeN1>(mode, grad);
    case kShapeT1N1:
      return kern::occupancy_mode<1, kShapeT1N1>(mode, grad);
    case kShapeList:
      return kern::occupancy_mode<1, kShapeList>(mode, grad);
    case kShapeListS:
      return kern::occupancy_mode<1, kShapeListS>(mode, grad);
    default:
      return 0;
  }
}

}  // namespace musr
