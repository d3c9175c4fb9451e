// musr_selftest.cu -- self-check of the bounded waits of the evaluation kernels.
//
// Every staging wait of the SPLIT kernels waits on a shared-memory mbarrier for a bulk copy
// with a time limit of 100 ms on the global timer (mbar_wait in musr_kernels.cuh).  A copy that never lands makes
// the wait give up, the CTA records an error status, the evaluation's value comes back NaN
// and the call returns MUSR_ETIMEOUT.  The GPU is never faulted, trapped or hung for that.
// musr_check_bounded_wait exercises the wait itself with an mbarrier that nothing arrives on:
// the wait must give up within its limit, and the same wait must succeed once the phase
// has completed.
#include <cuda_runtime.h>

#include "musr.h"
#include "musr_kernels.cuh"

namespace musr {
namespace kern {
namespace {

// One thread.  out[0]: ns per unsatisfied try_wait (256 tries); out[1]: ns of the
// evaluation kernels' wait on the unsatisfied phase (-1: not run).  status bits: 1 a
// try_wait saw the unsatisfied phase complete; 2 the wait did not give up; 4 the wait was
// not run (a try saw the phase complete); 8 the completed phase was not seen.  The wait is
// bounded by the global timer (kWaitLimitNs), so it ends whatever a try costs.
__global__ void bounded_wait_kernel(double* out, unsigned* status) {
  __shared__ unsigned long long bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_init_fence();
  unsigned st = 0;
  unsigned long long t0 = global_ns();
  bool seen = false;
  for (int i = 0; i < 256; ++i) seen |= mbar_try_wait(&bar, 0);
  unsigned long long t1 = global_ns();
  const double per_try = static_cast<double>(t1 - t0) / 256.0;
  out[0] = per_try;
  if (seen) st |= 1u;
  if (!seen) {
    t0 = global_ns();
    const bool done = mbar_wait(&bar, 0);
    t1 = global_ns();
    out[1] = static_cast<double>(t1 - t0);
    if (done) st |= 2u;
  } else {
    out[1] = -1.0;
    st |= 4u;
  }
  // The one expected arrival completes phase 0.
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  if (!mbar_wait(&bar, 0)) st |= 8u;
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
  *status = st;
}

}  // namespace
}  // namespace kern
}  // namespace musr

extern "C" int musr_check_bounded_wait(int device, double* out_try_s, double* out_wait_s) {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MUSR_EINVAL;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  double* d_out = nullptr;
  unsigned* d_status = nullptr;
  cudaStream_t s = nullptr;
  double h_out[2] = {-1.0, -1.0};
  unsigned h_status = ~0u;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(unsigned));
  if (e == cudaSuccess) {
    musr::kern::bounded_wait_kernel<<<1, 32, 0, s>>>(d_out, d_status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_out, sizeof(h_out), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, d_status, sizeof(h_status), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (d_out) cudaFree(d_out);
  if (d_status) cudaFree(d_status);
  if (s) cudaStreamDestroy(s);
  if (prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) return MUSR_ECUDA;
  if (out_try_s) *out_try_s = h_out[0] * 1e-9;
  if (out_wait_s) *out_wait_s = h_out[1] < 0.0 ? -1.0 : h_out[1] * 1e-9;
  return h_status == 0 ? MUSR_OK : MUSR_ESTATE;
}

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
  const cudaError_t e = cudaFuncGetAttributes(&a, musr::kern::bounded_wait_kernel);
  if (prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) return MUSR_ECUDA;
  *out = a.binaryVersion;
  return MUSR_OK;
}
