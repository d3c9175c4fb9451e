// musr_counts.cu -- the device image of uploaded histograms and asymmetry data (the measured counts d_n^j of
// Eq. chi2 and Eq. mlh, Section 4.1): the rows arrive from the host as they are, one row
// per histogram at the device row stride; this kernel converts them in place to the stored
// type, zeroes each row's padding and flags values the store cannot hold, so the host makes
// one copy and no pass over the data.
#include <cstdint>
#include <type_traits>

#include "musr.h"
#include "musr_dev.h"

namespace musr {
namespace {

// One thread per element of [H][stride], grid-stride.  INT32 counts become FP32 (exact
// below 2^24); FP32 and FP64 are checked for finiteness.  A bad element writes seq to
// *flag (host-mapped memory), which the host compares after the stream has finished.
template <int DTYPE>
__global__ void __launch_bounds__(256) prepare_counts_kernel(void* buf, int64_t nbins, int64_t stride,
                                                             int64_t total, unsigned* flag, unsigned seq) {
  bool bad = false;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const bool pad = e % stride >= nbins;
    if (DTYPE == MUSR_DTYPE_INT32) {
      int32_t* p = static_cast<int32_t*>(buf) + e;
      const int32_t v = pad ? 0 : *p;
      bad |= v >= (1 << 24) || v <= -(1 << 24);
      *reinterpret_cast<float*>(p) = static_cast<float>(v);
    } else if (DTYPE == MUSR_DTYPE_FP32) {
      float* p = static_cast<float*>(buf) + e;
      if (pad) {
        *p = 0.0f;
      } else {
        const float v = *p;
        bad |= !(fabsf(v) <= 3.4028234663852886e38f);
      }
    } else {
      double* p = static_cast<double*>(buf) + e;
      if (pad) {
        *p = 0.0;
      } else {
        const double v = *p;
        bad |= !(fabs(v) <= 1.7976931348623157e308);
      }
    }
  }
  if (bad) *reinterpret_cast<volatile unsigned*>(flag) = seq;
}

// The same from a packed copy of the rows ([nhist][nbins], dtype as uploaded) into the
// image, row h moved left by shift[h] bins: img[h][j] = raw[h][j + shift[h]] while that
// bin exists, else 0.  Every raw value is checked, also those the shift leaves out.
template <int DTYPE>
__global__ void __launch_bounds__(256) prepare_shifted_kernel(const void* raw, void* img, const int64_t* shift,
                                                              int64_t nbins, int64_t stride, int64_t total,
                                                              int64_t nraw, unsigned* flag, unsigned seq) {
  using Out = typename std::conditional<DTYPE == MUSR_DTYPE_FP64, double, float>::type;
  using In = typename std::conditional<DTYPE == MUSR_DTYPE_INT32, int32_t,
                                       typename std::conditional<DTYPE == MUSR_DTYPE_FP64, double, float>::type>::type;
  const In* src = static_cast<const In*>(raw);
  Out* dst = static_cast<Out*>(img);
  const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t first = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  for (int64_t e = first; e < total; e += step) {
    const int64_t h = e / stride, j = e - h * stride, n = j + shift[h];
    dst[e] = j < nbins && n < nbins ? static_cast<Out>(src[h * nbins + n]) : Out(0);
  }
  bool bad = false;
  for (int64_t e = first; e < nraw; e += step) {
    const In v = src[e];
    if (DTYPE == MUSR_DTYPE_INT32)
      bad |= v >= (1 << 24) || v <= -(1 << 24);
    else if (DTYPE == MUSR_DTYPE_FP32)
      bad |= !(fabsf(static_cast<float>(v)) <= 3.4028234663852886e38f);
    else
      bad |= !(fabs(static_cast<double>(v)) <= 1.7976931348623157e308);
  }
  if (bad) *reinterpret_cast<volatile unsigned*>(flag) = seq;
}

// Asymmetry data from packed forward / backward rows (raw: F [nhist][nbins], then B; dtype
// as uploaded) into a and w ([nhist][stride], FP64), row h moved left by shift[h] bins:
//   f = F - bkg_f, b = B - bkg_b, D = f + alpha b,
//   a = (f - alpha b) / D,  w = 1 / sigma_a^2,
//   sigma_a^2 = 4 alpha^2 (b^2 max(F, 1) + f^2 max(B, 1)) / D^4
// (first-order propagation of the Poisson errors of F and B), a = w = 0 where D <= 0 and
// in the padding.  par holds alpha, bkg_f, bkg_b ([3][nhist]).  a32 and w32 receive FP32
// copies (the SPLIT kernels' operands).  Every raw count is checked.
template <int DTYPE>
__global__ void __launch_bounds__(256) prepare_asymmetry_kernel(const void* raw, const int64_t* shift,
                                                                const double* par, int nhist, int64_t nbins,
                                                                int64_t stride, double* a, double* w,
                                                                float* a32, float* w32, unsigned* flag,
                                                                unsigned seq) {
  using In = typename std::conditional<DTYPE == MUSR_DTYPE_INT32, int32_t,
                                       typename std::conditional<DTYPE == MUSR_DTYPE_FP64, double, float>::type>::type;
  const In* F = static_cast<const In*>(raw);
  const In* Bk = F + static_cast<int64_t>(nhist) * nbins;
  const int64_t total = static_cast<int64_t>(nhist) * stride, nraw = 2 * static_cast<int64_t>(nhist) * nbins;
  const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t first = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  for (int64_t e = first; e < total; e += step) {
    const int64_t h = e / stride, j = e - h * stride, n = j + shift[h];
    double av = 0.0, wv = 0.0;
    if (j < nbins && n < nbins) {
      const double Fc = static_cast<double>(F[h * nbins + n]), Bc = static_cast<double>(Bk[h * nbins + n]);
      const double al = par[h], f = Fc - par[nhist + h], b = Bc - par[2 * nhist + h];
      const double D = f + al * b;
      if (D > 0.0) {
        av = (f - al * b) / D;
        const double D2 = D * D;
        const double var = 4.0 * al * al * (b * b * fmax(Fc, 1.0) + f * f * fmax(Bc, 1.0)) / (D2 * D2);
        wv = var > 0.0 ? 1.0 / var : 0.0;
      }
    }
    a[e] = av;
    w[e] = wv;
    a32[e] = static_cast<float>(av);
    w32[e] = static_cast<float>(wv);
  }
  bool bad = false;
  for (int64_t e = first; e < nraw; e += step) {
    const In v = F[e];  // F and B are contiguous
    if (DTYPE == MUSR_DTYPE_INT32)
      bad |= v >= (1 << 24) || v <= -(1 << 24);
    else if (DTYPE == MUSR_DTYPE_FP32)
      bad |= !(fabsf(static_cast<float>(v)) <= 3.4028234663852886e38f);
    else
      bad |= !(fabs(static_cast<double>(v)) <= 1.7976931348623157e308);
  }
  if (bad) *reinterpret_cast<volatile unsigned*>(flag) = seq;
}

}  // namespace

int launch_prepare_asymmetry(const void* raw, const int64_t* shift, const double* par, int dtype, int nhist,
                             int64_t nbins, int64_t stride, double* a, double* w, float* a32, float* w32,
                             unsigned* flag, unsigned seq, int num_sms, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const int64_t total = static_cast<int64_t>(nhist) * stride;
  if (total <= 0) return 0;
  const int64_t want = (total + 255) / 256;
  const int grid = static_cast<int>(want < 8LL * num_sms ? want : 8LL * num_sms);
  switch (dtype) {
    case MUSR_DTYPE_INT32:
      prepare_asymmetry_kernel<MUSR_DTYPE_INT32>
          <<<grid, 256, 0, stream>>>(raw, shift, par, nhist, nbins, stride, a, w, a32, w32, flag, seq);
      break;
    case MUSR_DTYPE_FP32:
      prepare_asymmetry_kernel<MUSR_DTYPE_FP32>
          <<<grid, 256, 0, stream>>>(raw, shift, par, nhist, nbins, stride, a, w, a32, w32, flag, seq);
      break;
    default:
      prepare_asymmetry_kernel<MUSR_DTYPE_FP64>
          <<<grid, 256, 0, stream>>>(raw, shift, par, nhist, nbins, stride, a, w, a32, w32, flag, seq);
      break;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_prepare_counts_shifted(const void* raw, void* img, const int64_t* shift, int dtype, int nhist,
                                  int64_t nbins, int64_t stride, unsigned* flag, unsigned seq, int num_sms,
                                  void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const int64_t total = static_cast<int64_t>(nhist) * stride, nraw = static_cast<int64_t>(nhist) * nbins;
  if (total <= 0) return 0;
  const int64_t want = (total + 255) / 256;
  const int grid = static_cast<int>(want < 8LL * num_sms ? want : 8LL * num_sms);
  switch (dtype) {
    case MUSR_DTYPE_INT32:
      prepare_shifted_kernel<MUSR_DTYPE_INT32>
          <<<grid, 256, 0, stream>>>(raw, img, shift, nbins, stride, total, nraw, flag, seq);
      break;
    case MUSR_DTYPE_FP32:
      prepare_shifted_kernel<MUSR_DTYPE_FP32>
          <<<grid, 256, 0, stream>>>(raw, img, shift, nbins, stride, total, nraw, flag, seq);
      break;
    default:
      prepare_shifted_kernel<MUSR_DTYPE_FP64>
          <<<grid, 256, 0, stream>>>(raw, img, shift, nbins, stride, total, nraw, flag, seq);
      break;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_prepare_counts(void* buf, int dtype, int nhist, int64_t nbins, int64_t stride, unsigned* flag,
                          unsigned seq, int num_sms, void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const int64_t total = static_cast<int64_t>(nhist) * stride;
  if (total <= 0) return 0;
  const int64_t want = (total + 255) / 256;
  const int grid = static_cast<int>(want < 8LL * num_sms ? want : 8LL * num_sms);
  switch (dtype) {
    case MUSR_DTYPE_INT32:
      prepare_counts_kernel<MUSR_DTYPE_INT32><<<grid, 256, 0, stream>>>(buf, nbins, stride, total, flag, seq);
      break;
    case MUSR_DTYPE_FP32:
      prepare_counts_kernel<MUSR_DTYPE_FP32><<<grid, 256, 0, stream>>>(buf, nbins, stride, total, flag, seq);
      break;
    default:
      prepare_counts_kernel<MUSR_DTYPE_FP64><<<grid, 256, 0, stream>>>(buf, nbins, stride, total, flag, seq);
      break;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace musr
