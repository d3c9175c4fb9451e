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
// Per evaluation and per distinct (Delta, nu) pair, two CTAs solve the equation on the grid
// t_k = k h over [0, span] by the trapezoidal rule (f_0 = G_0 = 1),
//     a G_k - c sum_{i=1}^{k-1} f_{k-i} G_i = b f_k,   a = 1 - nu h/2, b = 1 + nu h/2, c = nu h,
// on that grid and on its halving (one CTA each), and keeps the Richardson extrapolation
// (4 G_{h/2} - G_h) / 3 at the coarse points (the rule's h^2 error term removed).  The derivatives with respect to
// Delta and nu satisfy the same equation with other right-hand sides (the recursion
// differentiated), so three solves share one operator.
//
// Blocked solve: the points are taken in blocks of 256, four threads per point (1024 per
// CTA).  The block's history (the terms with i before the block) -- the O(K^2) part -- is
// summed in parallel, each of a point's threads taking a fixed quarter of it, and the
// block's own lower-triangular Toeplitz system, a I - c L with L_{rs} = f_{r-s}, is solved by
// multiplying with its inverse, again lower-triangular Toeplitz, whose first column is
// computed once per grid by one warp; the quarters' partial sums are added in a fixed order.
// The arithmetic type is that of the path the table serves: FP64 for the plain path, FP32 for
// the SPLIT path.
#include <cuda_runtime.h>

#include "musr_dev.h"

namespace musr {
namespace {

constexpr int kB = 256;       // points per block of the solve
constexpr int kQ = 4;         // threads per point
constexpr int kT = kB * kQ;   // threads per CTA

template <class T>
struct DktSmem {
  T tinv[kB];          // first column of the inverse of the block's Toeplitz matrix
  T rhs[kB];
  T part[kQ][3][kB];   // partial sums of the quarters of a point's threads
};

__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float dexp(float x) { return expf(x); }

// Quarter q of [lo, hi): the range [lo + q n / kQ, lo + (q + 1) n / kQ), n = hi - lo.
__device__ __forceinline__ void quarter(int lo, int hi, int q, int* b, int* e) {
  const int n = hi > lo ? hi - lo : 0;
  *b = lo + (q * n) / kQ;
  *e = lo + ((q + 1) * n) / kQ;
}

// sum_{i=b}^{e-1} w[n - i] x[i] with four partial sums (independent FMA chains).
template <class T>
__device__ __forceinline__ T conv_range(const T* w, const T* x, int n, int b, int e) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  int i = b;
  for (; i + 3 < e; i += 4) {
    s0 = fma(w[n - i], x[i], s0);
    s1 = fma(w[n - i - 1], x[i + 1], s1);
    s2 = fma(w[n - i - 2], x[i + 2], s2);
    s3 = fma(w[n - i - 3], x[i + 3], s3);
  }
  for (; i < e; ++i) s0 = fma(w[n - i], x[i], s0);
  return (s0 + s1) + (s2 + s3);
}

// X[k], k = 1..K, holds the right-hand side R_k on entry and the solution of
// a X_k - c sum_{i=1}^{k-1} f_{k-i} X_i = R_k on exit (X[0] is not read).
template <class T>
__device__ void solve_blocks(const T* f, T* X, int K, T c, DktSmem<T>& sm) {
  const int r = threadIdx.x % kB, q = threadIdx.x / kB;
  for (int k0 = 1; k0 <= K; k0 += kB) {
    const int k = k0 + r;
    int b, e;
    quarter(1, k0, q, &b, &e);  // this thread's quarter of the history i = 1 .. k0 - 1
    sm.part[q][0][r] = k <= K ? conv_range(f, X, k, b, e) : T(0);
    __syncthreads();
    if (q == 0)
      sm.rhs[r] = k <= K ? X[k] + c * ((sm.part[0][0][r] + sm.part[1][0][r]) + (sm.part[2][0][r] + sm.part[3][0][r]))
                         : T(0);
    __syncthreads();
    quarter(0, r + 1, q, &b, &e);  // this thread's quarter of s = 0 .. r
    T x = T(0);
    for (int s = b; s < e; ++s) x = fma(sm.tinv[r - s], sm.rhs[s], x);
    sm.part[q][0][r] = x;
    __syncthreads();
    if (q == 0 && k <= K) X[k] = (sm.part[0][0][r] + sm.part[1][0][r]) + (sm.part[2][0][r] + sm.part[3][0][r]);
    __syncthreads();
  }
}

// One grid: K intervals of width h.  f, fD, fN: the kernel and its Delta- and nu-derivatives;
// G, GD, GN: the solution and its derivatives (K + 1 values each).
template <class T>
__device__ void solve_grid(T D, T nu, T h, int K, T* f, T* fD, T* fN, T* G, T* GD, T* GN, DktSmem<T>& sm) {
  const int tid = threadIdx.x;
  const T a = T(1) - nu * (T(0.5) * h), b = T(1) + nu * (T(0.5) * h), c = nu * h;
  for (int k = tid; k <= K; k += kT) {
    const T t = static_cast<T>(k) * h;
    const T u = (D * t) * (D * t), gg = dexp(T(-0.5) * u), e = dexp(-nu * t);
    const T g = T(1) / T(3) + (T(2) / T(3)) * (T(1) - u) * gg;
    f[k] = g * e;
    fD[k] = (T(2) / T(3)) * D * t * t * gg * (u - T(3)) * e;
    fN[k] = -t * g * e;
  }
  __syncthreads();
  // t_0 = 1/a, t_r = (c/a) sum_{s<r} f_{r-s} t_s (warp 0; the block never reaches past K),
  // 32 entries at a time: each lane first sums the finished entries s < r0 for its r, then the
  // chunk's entries become final in order, each broadcast to the lanes above it.
  if (tid < 32) {
    const int nr = K + 1 < kB ? K + 1 : kB;
    const T ca = c / a;
    for (int r0 = 0; r0 < nr; r0 += 32) {
      const int rr = r0 + tid;
      const bool live = rr < nr;
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      if (live) {
        int q = 0;
        for (; q + 3 < r0; q += 4) {
          s0 = fma(f[rr - q], sm.tinv[q], s0);
          s1 = fma(f[rr - q - 1], sm.tinv[q + 1], s1);
          s2 = fma(f[rr - q - 2], sm.tinv[q + 2], s2);
          s3 = fma(f[rr - q - 3], sm.tinv[q + 3], s3);
        }
        for (; q < r0; ++q) s0 = fma(f[rr - q], sm.tinv[q], s0);
      }
      T acc = (s0 + s1) + (s2 + s3), tr = T(0);
      for (int j = 0; j < 32 && r0 + j < nr; ++j) {
        if (tid == j) tr = rr == 0 ? T(1) / a : ca * acc;
        const T tj = __shfl_sync(0xffffffffu, tr, j);
        if (live && tid > j) acc = fma(f[tid - j], tj, acc);
      }
      if (live) sm.tinv[rr] = tr;
      __syncwarp();
    }
  }
  // G: right-hand side b f_k (G_0 = 1 enters it through the trapezoid's end term)
  for (int k = tid; k <= K; k += kT) G[k] = k == 0 ? T(1) : b * f[k];
  __syncthreads();
  solve_blocks(f, G, K, c, sm);
  // right-hand sides of the derivatives, from the whole G:
  //   Delta: b fD_k + c sum fD_{k-i} G_i
  //   nu:    (h/2)(G_k + f_k) + b fN_k + h sum f_{k-i} G_i + c sum fN_{k-i} G_i
  const int r = tid % kB, q = tid / kB;
  for (int k0 = 0; k0 <= K; k0 += kB) {  // the point's four threads each sum a quarter
    const int k = k0 + r;
    int lo, hi;
    quarter(1, k, q, &lo, &hi);
    T sD = T(0), sf = T(0), sN = T(0);
    if (k <= K) {
      sD = conv_range(fD, G, k, lo, hi);
      sf = conv_range(f, G, k, lo, hi);
      sN = conv_range(fN, G, k, lo, hi);
    }
    sm.part[q][0][r] = sD;
    sm.part[q][1][r] = sf;
    sm.part[q][2][r] = sN;
    __syncthreads();
    if (q == 0 && k <= K) {
      auto sum4 = [&](int v) { return (sm.part[0][v][r] + sm.part[1][v][r]) + (sm.part[2][v][r] + sm.part[3][v][r]); };
      if (k == 0) {
        GD[0] = T(0);
        GN[0] = T(0);
      } else {
        GD[k] = b * fD[k] + c * sum4(0);
        GN[k] = T(0.5) * h * (G[k] + f[k]) + b * fN[k] + h * sum4(1) + c * sum4(2);
      }
    }
    __syncthreads();
  }
  solve_blocks(f, GD, K, c, sm);
  solve_blocks(f, GN, K, c, sm);
}

// Counter increment with acquire-release semantics at GPU scope, and the matching fence
// (documented PTX instructions).
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Two CTAs per (evaluation, source): part 0 solves the halved grid, part 1 the grid itself
// (each with its own kernel arrays), and whichever finishes second forms the Richardson
// extrapolation.  The source's counter gains 2 per solve (it starts at 0), so an odd value
// before the increment means the other part is done.  Release: the CTA barrier orders every
// thread's writes before thread 0's acquire-release increment; acquire: that increment and a
// fence by every thread of the finishing CTA (no CTA waits for the other).
template <class T>
__global__ void __launch_bounds__(kT) dkt_table_kernel(const Job* __restrict__ jobs, int ndkt) {
  __shared__ DktSmem<T> sm;
  __shared__ int second;
  const int pair = blockIdx.x >> 1, part = blockIdx.x & 1;
  const Job& job = jobs[pair / ndkt];
  const int src = pair % ndkt;
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
  constexpr int L = 2 * kDktMaxK + 1, Lc = kDktMaxK + 1;
  T *G2 = w + 3 * L, *GD2 = w + 4 * L, *GN2 = w + 5 * L;
  T* G = tab + kDktHeader;
  T* GD = G + (kDktMaxK + 1);
  T* GN = GD + (kDktMaxK + 1);
  const T D = static_cast<T>(Dd), nu = static_cast<T>(nd);
  if (part == 0) {
    solve_grid<T>(D, nu, static_cast<T>(0.5 * h), 2 * K, w, w + L, w + 2 * L, G2, GD2, GN2, sm);  // halved grid
  } else {
    T* fc = w + 6 * L;
    solve_grid<T>(D, nu, static_cast<T>(h), K, fc, fc + Lc, fc + 2 * Lc, G, GD, GN, sm);
  }
  __syncthreads();
  if (threadIdx.x == 0) second = (atom_add_acq_rel_u32(job.dkt_count + src, 1u) & 1u) != 0u;
  __syncthreads();
  if (!second) return;
  fence_acq_rel_gpu();
  for (int k = threadIdx.x; k <= K; k += kT) {  // Richardson extrapolation at the coarse points
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
    dkt_table_kernel<double><<<2 * njobs * ndkt, kT, 0, s>>>(d_jobs, ndkt);
  else
    dkt_table_kernel<float><<<2 * njobs * ndkt, kT, 0, s>>>(d_jobs, ndkt);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears the error
}

}  // namespace musr
