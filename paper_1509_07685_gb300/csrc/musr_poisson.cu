// musr_poisson.cu -- the particle-mesh Poisson solve of Section 3 ("FFT Based Particle-Mesh
// Solver") on the GPU, Hockney's method for an isolated charge density: the density on the
// M = mx x my x mz mesh is zero-padded to the doubled mesh N = 2M, and
//     phi = hx hy hz FT^-1{ FT{rho} (x) FT{G} }   restricted to M        (Eq. oneterm)
// is the discretised convolution of Eq. openbruteforceconv, with G_{a,b,c} = 1/r on the
// doubled mesh (distances folded: G(N - a) = G(a), so the circular convolution of length N
// equals the linear one on M).  G is even, so FT{G} is real; it is computed once per solver
// and kept as N_x N_y (N_z / 2 + 1) reals.  The transforms are cuFFT, in FP64 (D2Z, Z2D) or,
// at MUSR_SPLIT precision, in FP32 (R2C, C2R; FP64 density in and potential out): GB300's
// FP64 rate makes the FP64 transforms arithmetic-bound, the FP32 ones are memory-bound;
// padding, the Green's function, the Hadamard product (with the 1/N^3 of the inverse
// transform and hx hy hz folded in) and the extraction are kernels of this file.  The padded
// density's zeros are written once (solves write the M block only).
// Reading: G_{0,0,0}, where 1/r is singular, is 1 / min(hx, hy, hz).
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "musr.h"

struct musr_poisson {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int precision = MUSR_FP64;  // MUSR_FP64: double transforms; MUSR_SPLIT: float transforms
  int mx = 0, my = 0, mz = 0;
  int nx = 0, ny = 0, nz = 0;  // doubled mesh
  double hx = 0, hy = 0, hz = 0;
  cufftHandle fwd = 0, inv = 0;
  bool have_fwd = false, have_inv = false;
  void* pad = nullptr;   // [nx][ny][nz] real: the padded density (its zeros written once)
  void* out = nullptr;   // [nx][ny][nz] real: the inverse transform's result
  void* hat = nullptr;   // [nx][ny][nz / 2 + 1] complex
  void* ghat = nullptr;  // FT{G}, real, [nx][ny][nz / 2 + 1]
  double* rho = nullptr;  // [mx][my][mz] staging of the host entry point
  double* phi = nullptr;
  int num_sms = 1;
  std::string err;
};

namespace {

thread_local std::string g_poisson_create_error;

int64_t grid_for(int64_t n, int num_sms) {
  const int64_t want = (n + 255) / 256;
  return want < 8LL * num_sms ? (want > 0 ? want : 1) : 8LL * num_sms;
}

// Threads of a row-wise kernel: one per work unit of the row, a multiple of 32, at most 256.
int row_block(int units) { return units >= 256 ? 256 : ((units + 31) / 32) * 32; }

// Grid of the row-wise kernels: x over the inner row index (ny or my <= 2^11 here), y over
// the outer one, up to about 32 CTAs per SM in all.
dim3 rows_grid(int inner, int outer, int num_sms) {
  const int want = (32 * num_sms + inner - 1) / inner;
  return dim3(static_cast<unsigned>(inner), static_cast<unsigned>(want < outer ? (want > 0 ? want : 1) : outer));
}

template <class R>
struct Cx;  // the complex type of each real type
template <>
struct Cx<double> {
  using type = cufftDoubleComplex;
};
template <>
struct Cx<float> {
  using type = cufftComplex;
};

// G on the doubled mesh, distances folded per axis (evaluated in FP64, stored as R).
template <class R>
__global__ void green_kernel(R* g, int nx, int ny, int nz, double hx, double hy, double hz, double g0) {
  const int64_t total = static_cast<int64_t>(nx) * ny * nz;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t a = e / (static_cast<int64_t>(ny) * nz), r = e - a * ny * static_cast<int64_t>(nz);
    const int64_t b = r / nz, c = r - b * nz;
    const int64_t da = a <= nx - a ? a : nx - a, db = b <= ny - b ? b : ny - b, dc = c <= nz - c ? c : nz - c;
    const double u = static_cast<double>(da) * hx, v = static_cast<double>(db) * hy, w = static_cast<double>(dc) * hz;
    g[e] = static_cast<R>((da | db | dc) == 0 ? g0 : 1.0 / sqrt(u * u + v * v + w * w));
  }
}

template <class R>
__global__ void real_part_kernel(const typename Cx<R>::type* in, R* out, int64_t n) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[e] = in[e].x;
}

template <class R>
struct Pair;  // two consecutive reals, one vector store
template <>
struct Pair<double> {
  using type = double2;
};
template <>
struct Pair<float> {
  using type = float2;
};

// rho [mx][my][mz] (FP64) into the M block of the doubled mesh.  The rest of the doubled
// mesh holds zeros written once: the forward transform is out of place and leaves its
// input as it is (the inverse writes to a buffer of its own).  CTA (b, y0) takes the rows
// (a, b) for a = y0, y0 + gridDim.y, ... < mx.
template <class R>
__global__ void pad_kernel(const double* __restrict__ rho, R* __restrict__ pad, int mx, int my, int mz, int ny,
                           int nz) {
  const int b = blockIdx.x;
  for (int a = blockIdx.y; a < mx; a += gridDim.y) {
    R* dst = pad + (static_cast<int64_t>(a) * ny + b) * nz;
    const double* src = rho + (static_cast<int64_t>(a) * my + b) * mz;
    for (int c = threadIdx.x; c < mz; c += blockDim.x) dst[c] = static_cast<R>(src[c]);
  }
}

// hat *= FT{G} * scale (scale = hx hy hz / (nx ny nz), the inverse transform's normalisation).
template <class R>
__global__ void hadamard_kernel(typename Cx<R>::type* __restrict__ hat, const R* __restrict__ ghat, int64_t n,
                                R scale) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const R s = ghat[e] * scale;
    typename Cx<R>::type v = hat[e];
    v.x *= s;
    v.y *= s;
    hat[e] = v;
  }
}

// The M block of the doubled mesh, as FP64.  CTA (j, y0) takes the rows (i, j) of M for
// i = y0, y0 + gridDim.y, ...
template <class R>
__global__ void extract_kernel(const R* __restrict__ pad, double* __restrict__ phi, int mx, int my, int mz, int ny,
                               int nz) {
  const int j = blockIdx.x;
  for (int i = blockIdx.y; i < mx; i += gridDim.y) {
    const R* src = pad + (static_cast<int64_t>(i) * ny + j) * nz;
    double* dst = phi + (static_cast<int64_t>(i) * my + j) * mz;
    for (int k = threadIdx.x; k < mz; k += blockDim.x) dst[k] = static_cast<double>(src[k]);
  }
}

int pfail(musr_poisson* ps, int code, const std::string& msg) {
  ps->err = msg;
  return code;
}

int cuda_err(musr_poisson* ps, cudaError_t e, const char* what) {
  cudaGetLastError();
  return pfail(ps, e == cudaErrorMemoryAllocation ? MUSR_ENOMEM : MUSR_ECUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

int fft_err(musr_poisson* ps, cufftResult r, const char* what) {
  return pfail(ps, r == CUFFT_ALLOC_FAILED ? MUSR_ENOMEM : MUSR_ECUDA,
               std::string(what) + ": cuFFT status " + std::to_string(static_cast<int>(r)));
}

struct DevScope {
  int prev = 0;
  explicit DevScope(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DevScope() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != prev) cudaSetDevice(prev);
  }
};

void release(musr_poisson* ps) {
  if (ps->have_fwd) cufftDestroy(ps->fwd);
  if (ps->have_inv) cufftDestroy(ps->inv);
  cudaFree(ps->pad);
  cudaFree(ps->out);
  cudaFree(ps->hat);
  cudaFree(ps->ghat);
  cudaFree(ps->rho);
  cudaFree(ps->phi);
  if (ps->own_stream && ps->stream) cudaStreamDestroy(ps->stream);
}

cufftResult exec_fwd(musr_poisson* ps) {
  return ps->precision == MUSR_FP64
             ? cufftExecD2Z(ps->fwd, static_cast<double*>(ps->pad), static_cast<cufftDoubleComplex*>(ps->hat))
             : cufftExecR2C(ps->fwd, static_cast<float*>(ps->pad), static_cast<cufftComplex*>(ps->hat));
}

cufftResult exec_inv(musr_poisson* ps) {
  return ps->precision == MUSR_FP64
             ? cufftExecZ2D(ps->inv, static_cast<cufftDoubleComplex*>(ps->hat), static_cast<double*>(ps->out))
             : cufftExecC2R(ps->inv, static_cast<cufftComplex*>(ps->hat), static_cast<float*>(ps->out));
}

// Enqueues one solve: d_rho [mx][my][mz] -> d_phi [mx][my][mz].
template <class R>
int enqueue_solve_t(musr_poisson* ps, const double* d_rho, double* d_phi) {
  const int64_t total = static_cast<int64_t>(ps->nx) * ps->ny * ps->nz;
  const int64_t nhat = static_cast<int64_t>(ps->nx) * ps->ny * (ps->nz / 2 + 1);
  R* pad = static_cast<R*>(ps->pad);
  auto* hat = static_cast<typename Cx<R>::type*>(ps->hat);
  pad_kernel<R><<<rows_grid(ps->my, ps->mx, ps->num_sms), row_block(ps->mz), 0, ps->stream>>>(
      d_rho, pad, ps->mx, ps->my, ps->mz, ps->ny, ps->nz);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ps, e, "pad kernel");
  cufftResult r = exec_fwd(ps);
  if (r != CUFFT_SUCCESS) return fft_err(ps, r, "forward FFT");
  const double scale = ps->hx * ps->hy * ps->hz / static_cast<double>(total);
  hadamard_kernel<R><<<grid_for(nhat, ps->num_sms), 256, 0, ps->stream>>>(hat, static_cast<const R*>(ps->ghat), nhat,
                                                                          static_cast<R>(scale));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ps, e, "hadamard kernel");
  r = exec_inv(ps);
  if (r != CUFFT_SUCCESS) return fft_err(ps, r, "inverse FFT");
  extract_kernel<R><<<rows_grid(ps->my, ps->mx, ps->num_sms), row_block(ps->mz), 0, ps->stream>>>(
      static_cast<const R*>(ps->out), d_phi, ps->mx, ps->my, ps->mz, ps->ny, ps->nz);
  e = cudaGetLastError();
  return e == cudaSuccess ? MUSR_OK : cuda_err(ps, e, "extract kernel");
}

int enqueue_solve(musr_poisson* ps, const double* d_rho, double* d_phi) {
  return ps->precision == MUSR_FP64 ? enqueue_solve_t<double>(ps, d_rho, d_phi)
                                    : enqueue_solve_t<float>(ps, d_rho, d_phi);
}

// FT{G}, once: G into the padded buffer, forward transform, keep the real part.
template <class R>
int setup_green(musr_poisson* ps) {
  const int64_t total = static_cast<int64_t>(ps->nx) * ps->ny * ps->nz;
  const int64_t nhat = static_cast<int64_t>(ps->nx) * ps->ny * (ps->nz / 2 + 1);
  const double g0 = 1.0 / std::fmin(ps->hx, std::fmin(ps->hy, ps->hz));
  green_kernel<R><<<grid_for(total, ps->num_sms), 256, 0, ps->stream>>>(static_cast<R*>(ps->pad), ps->nx, ps->ny,
                                                                        ps->nz, ps->hx, ps->hy, ps->hz, g0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ps, e, "green kernel");
  const cufftResult r = exec_fwd(ps);
  if (r != CUFFT_SUCCESS) return fft_err(ps, r, "forward FFT of G");
  real_part_kernel<R><<<grid_for(nhat, ps->num_sms), 256, 0, ps->stream>>>(
      static_cast<const typename Cx<R>::type*>(ps->hat), static_cast<R*>(ps->ghat), nhat);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(ps, e, "real-part kernel");
  // the padded density's zeros, once (solves write only the M block)
  if ((e = cudaMemsetAsync(ps->pad, 0, sizeof(R) * total, ps->stream)) != cudaSuccess)
    return cuda_err(ps, e, "cudaMemsetAsync(pad)");
  if ((e = cudaStreamSynchronize(ps->stream)) != cudaSuccess) return cuda_err(ps, e, "Green setup");
  return MUSR_OK;
}

}  // namespace

extern "C" {

int musr_poisson_create(musr_poisson** out, int device, int mx, int my, int mz, double hx, double hy, double hz,
                        int precision, void* cuda_stream) {
  if (!out) return MUSR_EINVAL;
  *out = nullptr;
  if (precision != MUSR_FP64 && precision != MUSR_SPLIT) {
    g_poisson_create_error = "precision must be MUSR_FP64 or MUSR_SPLIT";
    return MUSR_EINVAL;
  }
  if (mx < 1 || my < 1 || mz < 1) {
    g_poisson_create_error = "mesh sizes must be >= 1";
    return MUSR_EINVAL;
  }
  if (8.0 * mx * my * mz >= 2147483648.0) {  // in double: 2 * mx may not fit an int
    g_poisson_create_error = "the doubled mesh must hold fewer than 2^31 points";
    return MUSR_EINVAL;
  }
  if (!(hx > 0.0) || !(hy > 0.0) || !(hz > 0.0) || !std::isfinite(hx) || !std::isfinite(hy) || !std::isfinite(hz)) {
    g_poisson_create_error = "mesh spacings must be finite and > 0";
    return MUSR_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    g_poisson_create_error = "no such CUDA device";
    return MUSR_ECUDA;
  }
  DevScope ds(device);
  auto* ps = new musr_poisson();
  ps->device = device;
  ps->precision = precision;
  ps->mx = mx, ps->my = my, ps->mz = mz;
  ps->nx = 2 * mx, ps->ny = 2 * my, ps->nz = 2 * mz;
  ps->hx = hx, ps->hy = hy, ps->hz = hz;
  cudaDeviceGetAttribute(&ps->num_sms, cudaDevAttrMultiProcessorCount, device);
  auto fail_create = [&](int code) {
    g_poisson_create_error = ps->err;
    release(ps);
    delete ps;
    return code;
  };
  if (cuda_stream) {
    ps->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&ps->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail_create(cuda_err(ps, e, "cudaStreamCreate"));
    ps->own_stream = true;
  }
  const size_t rsz = precision == MUSR_FP64 ? sizeof(double) : sizeof(float);
  const int64_t total = static_cast<int64_t>(ps->nx) * ps->ny * ps->nz;
  const int64_t nhat = static_cast<int64_t>(ps->nx) * ps->ny * (ps->nz / 2 + 1);
  const int64_t nm = static_cast<int64_t>(mx) * my * mz;
  cudaError_t e = cudaMalloc(&ps->pad, rsz * total);
  if (e == cudaSuccess) e = cudaMalloc(&ps->out, rsz * total);
  if (e == cudaSuccess) e = cudaMalloc(&ps->hat, 2 * rsz * nhat);
  if (e == cudaSuccess) e = cudaMalloc(&ps->ghat, rsz * nhat);
  if (e == cudaSuccess) e = cudaMalloc(&ps->rho, sizeof(double) * nm);
  if (e == cudaSuccess) e = cudaMalloc(&ps->phi, sizeof(double) * nm);
  if (e != cudaSuccess) return fail_create(cuda_err(ps, e, "cudaMalloc"));
  cufftResult r = cufftPlan3d(&ps->fwd, ps->nx, ps->ny, ps->nz, precision == MUSR_FP64 ? CUFFT_D2Z : CUFFT_R2C);
  if (r != CUFFT_SUCCESS) return fail_create(fft_err(ps, r, "cufftPlan3d(forward)"));
  ps->have_fwd = true;
  r = cufftPlan3d(&ps->inv, ps->nx, ps->ny, ps->nz, precision == MUSR_FP64 ? CUFFT_Z2D : CUFFT_C2R);
  if (r != CUFFT_SUCCESS) return fail_create(fft_err(ps, r, "cufftPlan3d(inverse)"));
  ps->have_inv = true;
  if ((r = cufftSetStream(ps->fwd, ps->stream)) != CUFFT_SUCCESS ||
      (r = cufftSetStream(ps->inv, ps->stream)) != CUFFT_SUCCESS)
    return fail_create(fft_err(ps, r, "cufftSetStream"));
  const int rc = precision == MUSR_FP64 ? setup_green<double>(ps) : setup_green<float>(ps);
  if (rc) return fail_create(rc);
  g_poisson_create_error.clear();
  *out = ps;
  return MUSR_OK;
}

void musr_poisson_destroy(musr_poisson* ps) {
  if (!ps) return;
  DevScope ds(ps->device);
  cudaStreamSynchronize(ps->stream);
  release(ps);
  delete ps;
}

const char* musr_poisson_last_error(const musr_poisson* ps) {
  return ps ? ps->err.c_str() : g_poisson_create_error.c_str();
}

int musr_poisson_solve_device(musr_poisson* ps, const double* d_rho, double* d_phi) {
  if (!ps) return MUSR_EINVAL;
  if (!d_rho || !d_phi) return pfail(ps, MUSR_EINVAL, "d_rho and d_phi must not be NULL");
  DevScope ds(ps->device);
  return enqueue_solve(ps, d_rho, d_phi);
}

int musr_poisson_solve(musr_poisson* ps, const double* rho, double* phi) {
  if (!ps) return MUSR_EINVAL;
  if (!rho || !phi) return pfail(ps, MUSR_EINVAL, "rho and phi must not be NULL");
  DevScope ds(ps->device);
  const size_t bytes = sizeof(double) * static_cast<size_t>(ps->mx) * ps->my * ps->mz;
  cudaError_t e = cudaMemcpyAsync(ps->rho, rho, bytes, cudaMemcpyHostToDevice, ps->stream);
  if (e != cudaSuccess) return cuda_err(ps, e, "cudaMemcpyAsync(rho)");
  int rc = enqueue_solve(ps, ps->rho, ps->phi);
  if (rc) return rc;
  e = cudaMemcpyAsync(phi, ps->phi, bytes, cudaMemcpyDeviceToHost, ps->stream);
  if (e != cudaSuccess) return cuda_err(ps, e, "cudaMemcpyAsync(phi)");
  e = cudaStreamSynchronize(ps->stream);
  return e == cudaSuccess ? MUSR_OK : cuda_err(ps, e, "cudaStreamSynchronize");
}

}  // extern "C"
