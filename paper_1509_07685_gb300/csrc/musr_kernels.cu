// musr_kernels.cu -- host-side dispatch of the evaluation kernels (musr_kernels.cuh): the
// launcher of each precision and SPLIT shape lives in the translation unit of its group.
#include "musr_kernels.cuh"

namespace musr {
namespace {

int shape_group_of(int shape) {
  switch (shape) {
    case kShapeT2:
    case kShapeT2N1:
      return 1;
    case kShapeT2m:
    case kShapeT2N1m:
      return 2;
    default:
      return 0;  // generic, T1, N1, T1N1
  }
}

}  // namespace

int shape_group(int shape) {
  if (shape == kShapeList || shape == kShapeListS) return 1;
  switch (shape) {
#define MUSR_CASE(S) \
  case S:            \
    return kern::Basis<S>::G;
    MUSR_CASE(kShapeT1)
    MUSR_CASE(kShapeN1)
    MUSR_CASE(kShapeT1N1)
    MUSR_CASE(kShapeT2)
    MUSR_CASE(kShapeT2N1)
    MUSR_CASE(kShapeT2m)
    MUSR_CASE(kShapeT2N1m)
#undef MUSR_CASE
    default:
      return kern::Basis<kShapeGeneric>::G;
  }
}

int shape_channels(int shape) {
  if (shape == kShapeList || shape == kShapeListS) return kFp64Channels;
  switch (shape) {
#define MUSR_CASE(S) \
  case S:            \
    return kern::Basis<S>::NCH;
    MUSR_CASE(kShapeT1)
    MUSR_CASE(kShapeN1)
    MUSR_CASE(kShapeT1N1)
    MUSR_CASE(kShapeT2)
    MUSR_CASE(kShapeT2N1)
    MUSR_CASE(kShapeT2m)
    MUSR_CASE(kShapeT2N1m)
#undef MUSR_CASE
    default:
      return kern::Basis<kShapeGeneric>::NCH;
  }
}

int launch_eval(int precision, int shape, int mode, int grad, const Job* d_jobs, int njobs,
                int total_items, int num_sms, void* stream, LaunchInfo* info) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == 0) return launch_group_fp64(mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
  switch (shape_group_of(shape)) {
    case 1:
      return launch_group_b(shape, mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
    case 2:
      return launch_group_c(shape, mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
    default:
      return launch_group_a(shape, mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
  }
}

int max_ctas_per_sm(int precision, int shape, int mode, int grad) {
  if (precision == 0) return occupancy_group_fp64(mode, grad);
  switch (shape_group_of(shape)) {
    case 1:
      return occupancy_group_b(shape, mode, grad);
    case 2:
      return occupancy_group_c(shape, mode, grad);
    default:
      return occupancy_group_a(shape, mode, grad);
  }
}

}  // namespace musr
