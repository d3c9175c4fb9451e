// musr_info.cu -- what the loaded code was built for (a build check; no counterpart in the paper).
#include <cuda_runtime.h>

#include "musr.h"

namespace {

// A kernel of this translation unit (compiled with the library's flags) whose attributes
// report the architecture of the code the runtime loaded.
__global__ void build_probe_kernel() {}

}  // namespace

extern "C" int musr_binary_version(int device, int* out) {
  if (!out) return MUSR_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MUSR_EINVAL;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  cudaFuncAttributes a;
  const cudaError_t e = cudaFuncGetAttributes(&a, build_probe_kernel);
  if (prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) return MUSR_ECUDA;
  *out = a.binaryVersion;
  return MUSR_OK;
}
