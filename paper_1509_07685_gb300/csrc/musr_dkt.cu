// musr_dkt.cu -- tables of the dynamic Gaussian Kubo-Toyabe relaxation (primitive DKT).
//
// Strong-collision model: the muon's local field is drawn from the isotropic Gaussian of
// width Delta / gamma_mu and drawn anew at the events of a Poisson process of rate nu; between
// two events the spin precesses in a static field, which on average multiplies the
// polarisation by the static function g(s) = 1/3 + 2/3 (1 - Delta^2 s^2) exp(-Delta^2 s^2 / 2).
// Summing over the number of events gives the renewal (Volterra) equation
//     G(t) = f(t) + nu int_0^t f(s) G(t - s) ds,   f(t) = g(t) exp(-nu t),
// whose solution G is the relaxation (no closed form).  It is one of the "user defined
// functions" of Section 4.1's fits, not written in the paper.
//
// Per evaluation and per distinct (Delta, nu) pair, one CTA solves the equation on the grid
// t_k = k h over [0, span] by the trapezoidal rule (f_0 = G_0 = 1),
//     a G_k - c sum_{i=1}^{k-1} f_{k-i} G_i = b f_k,   a = 1 - nu h/2, b = 1 + nu h/2, c = nu h,
// on that grid and on its halving, and keeps the Richardson extrapolation (4 G_{h/2} - G_h) / 3
// at the coarse points (the rule's h^2 error term removed).  The derivatives with respect to
// Delta and nu satisfy the same equation with other right-hand sides (the recursion
// differentiated), so three solves share one operator.
//
// Blocked solve: the points are taken in blocks of 256, one thread per point.  Each thread
// sums the block's history (the terms with i before the block) -- the O(K^2) part, in
// parallel -- and the block's own lower-triangular Toeplitz system, a I - c L with
// L_{rs} = f_{r-s}, is solved by multiplying with its inverse, again lower-triangular
// Toeplitz, whose first column is computed once per grid by one warp.  The arithmetic type is
// that of the path the table serves: FP64 for the plain path, FP32 for the SPLIT path.
#include <cuda_runtime.h>

#include "musr_dev.h"

namespace musr {
namespace {

constexpr int kB = 256;  // threads per CTA, points per block of the solve

template <class T>
struct DktSmem {
  T tinv[kB];  // first column of the inverse of the block's Toeplitz matrix
  T rhs[kB];
};

__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float dexp(float x) { return expf(x); }

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum_{i=1}^{n-1} w[n - i] x[i] with four partial sums (independent FMA chains).
template <class T>
__device__ __forceinline__ T conv_sum(const T* w, const T* x, int n) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  int i = 1;
  for (; i + 3 < n; i += 4) {
    s0 = fma(w[n - i], x[i], s0);
    s1 = fma(w[n - i - 1], x[i + 1], s1);
    s2 = fma(w[n - i - 2], x[i + 2], s2);
    s3 = fma(w[n - i - 3], x[i + 3], s3);
  }
  for (; i < n; ++i) s0 = fma(w[n - i], x[i], s0);
  return (s0 + s1) + (s2 + s3);
}

// X[k], k = 1..K, holds the right-hand side R_k on entry and the solution of
// a X_k - c sum_{i=1}^{k-1} f_{k-i} X_i = R_k on exit (X[0] is not read).
template <class T>
__device__ void solve_blocks(const T* f, T* X, int K, T c, DktSmem<T>& sm) {
  const int r = threadIdx.x;
  for (int k0 = 1; k0 <= K; k0 += kB) {
    const int k = k0 + r;
    T rhs = T(0);
    if (k <= K) rhs = X[k] + c * conv_sum(f + (k - k0), X, k0);
    sm.rhs[r] = rhs;
    __syncthreads();
    if (k <= K) {
      T x = T(0);
      for (int s = 0; s <= r; ++s) x = fma(sm.tinv[r - s], sm.rhs[s], x);
      X[k] = x;
    }
    __syncthreads();
  }
}

// One grid: K intervals of width h.  f, fD, fN: the kernel and its Delta- and nu-derivatives;
// G, GD, GN: the solution and its derivatives (K + 1 values each).
template <class T>
__device__ void solve_grid(T D, T nu, T h, int K, T* f, T* fD, T* fN, T* G, T* GD, T* GN, DktSmem<T>& sm) {
  const int tid = threadIdx.x;
  const T a = T(1) - nu * (T(0.5) * h), b = T(1) + nu * (T(0.5) * h), c = nu * h;
  for (int k = tid; k <= K; k += kB) {
    const T t = static_cast<T>(k) * h;
    const T u = (D * t) * (D * t), gg = dexp(T(-0.5) * u), e = dexp(-nu * t);
    const T g = T(1) / T(3) + (T(2) / T(3)) * (T(1) - u) * gg;
    f[k] = g * e;
    fD[k] = (T(2) / T(3)) * D * t * t * gg * (u - T(3)) * e;
    fN[k] = -t * g * e;
  }
  __syncthreads();
  // t_0 = 1/a, t_r = (c/a) sum_{s<r} f_{r-s} t_s (warp 0; the block never reaches past K)
  if (tid < 32) {
    const int nr = K + 1 < kB ? K + 1 : kB;
    if (tid == 0) sm.tinv[0] = T(1) / a;
    __syncwarp();
    for (int rr = 1; rr < nr; ++rr) {
      T acc = T(0);
      for (int s = tid; s < rr; s += 32) acc = fma(f[rr - s], sm.tinv[s], acc);
      acc = warp_sum(acc);
      if (tid == 0) sm.tinv[rr] = (c / a) * acc;
      __syncwarp();
    }
  }
  // G: right-hand side b f_k (G_0 = 1 enters it through the trapezoid's end term)
  for (int k = tid; k <= K; k += kB) G[k] = k == 0 ? T(1) : b * f[k];
  __syncthreads();
  solve_blocks(f, G, K, c, sm);
  // right-hand sides of the derivatives, from the whole G:
  //   Delta: b fD_k + c sum fD_{k-i} G_i
  //   nu:    (h/2)(G_k + f_k) + b fN_k + h sum f_{k-i} G_i + c sum fN_{k-i} G_i
  for (int k = tid; k <= K; k += kB) {
    if (k == 0) {
      GD[0] = T(0);
      GN[0] = T(0);
      continue;
    }
    GD[k] = b * fD[k] + c * conv_sum(fD, G, k);
    GN[k] = T(0.5) * h * (G[k] + f[k]) + b * fN[k] + h * conv_sum(f, G, k) + c * conv_sum(fN, G, k);
  }
  __syncthreads();
  solve_blocks(f, GD, K, c, sm);
  solve_blocks(f, GN, K, c, sm);
}

template <class T>
__global__ void __launch_bounds__(kB) dkt_table_kernel(const Job* __restrict__ jobs, int ndkt) {
  __shared__ DktSmem<T> sm;
  const Job& job = jobs[blockIdx.x / ndkt];
  const int src = blockIdx.x % ndkt;
  const HistSet& hs = *job.hs;
  auto value = [&](int m) { return m >= 0 ? job.params[m] : hs.consts[-1 - m]; };
  const double Dd = value(hs.dkt_src[src].x), nd = value(hs.dkt_src[src].y);
  const double rate = fmax(fmax(fabs(Dd), fabs(nd)), 0.05);
  const double span = hs.dkt_span > 0.0 ? hs.dkt_span : 1.0;
  double kf = ceil(span * rate / (sizeof(T) == sizeof(float) ? kDktStep32 : kDktStep));
  if (!(kf >= kDktMinK)) kf = kDktMinK;  // also NaN parameters
  if (kf > kDktMaxK) kf = kDktMaxK;
  const int K = static_cast<int>(kf);
  const double h = span / K;
  T* tab = static_cast<T*>(job.dkt) + static_cast<size_t>(src) * kDktTable;
  T* w = static_cast<T*>(job.dkt_work) + static_cast<size_t>(src) * kDktWork;
  constexpr int L = 2 * kDktMaxK + 1;
  T *f = w, *fD = w + L, *fN = w + 2 * L, *G2 = w + 3 * L, *GD2 = w + 4 * L, *GN2 = w + 5 * L;
  T* G = tab + kDktHeader;
  T* GD = G + (kDktMaxK + 1);
  T* GN = GD + (kDktMaxK + 1);
  const T D = static_cast<T>(Dd), nu = static_cast<T>(nd);
  solve_grid<T>(D, nu, static_cast<T>(0.5 * h), 2 * K, f, fD, fN, G2, GD2, GN2, sm);  // halved grid
  __syncthreads();
  solve_grid<T>(D, nu, static_cast<T>(h), K, f, fD, fN, G, GD, GN, sm);
  __syncthreads();
  for (int k = threadIdx.x; k <= K; k += kB) {  // Richardson extrapolation at the coarse points
    G[k] = (T(4) * G2[2 * k] - G[k]) / T(3);
    GD[k] = (T(4) * GD2[2 * k] - GD[k]) / T(3);
    GN[k] = (T(4) * GN2[2 * k] - GN[k]) / T(3);
  }
  if (threadIdx.x == 0) {
    tab[0] = static_cast<T>(h);
    tab[1] = static_cast<T>(1.0 / h);
    tab[2] = static_cast<T>(K);
    tab[3] = T(0);
  }
}

}  // namespace

int launch_dkt_tables(int precision, const Job* d_jobs, int njobs, int ndkt, void* stream) {
  if (ndkt <= 0 || njobs <= 0) return 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == 0)
    dkt_table_kernel<double><<<njobs * ndkt, kB, 0, s>>>(d_jobs, ndkt);
  else
    dkt_table_kernel<float><<<njobs * ndkt, kB, 0, s>>>(d_jobs, ndkt);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace musr
