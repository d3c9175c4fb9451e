// musr_kernels.cu -- evaluation kernels of libmusr (sm_103a).
//
// The cost of Section 4.1 of arXiv 1509.07685 is a map-reduce over every bin
// of every histogram: Eq. positron_histo gives the expected count N, Eq. chisq
// or Eq. log-likelihood turns (d, N) into a per-bin term, and the terms are
// summed.  The gradient is the same reduction of (dcost/dN) * (dN/dslot).
// No tensor cores: nothing here is a contraction.
//
// Two paths:
//   * FP64 ("plain"): one CTA per (histogram, tile); every per-bin operation in
//     FP64 with the term list interpreted as given (any product of primitives).
//   * SPLIT: one CTA per (chunk of <= 8 histograms sharing the time grid and
//     every time-dependent parameter, tile).  For each bin the time-only factors
//     (muon decay, relaxations, Kubo-Toyabe, the precession's cos/sin) are
//     computed once and reused by the chunk's histograms; the per-histogram
//     phase enters by a rotation.  Per-bin work is FP32 (hardware ex2, lg2, rcp,
//     sin, cos); the precession phase is range-reduced in FP64 once per tile
//     and carried per bin as an exact FP32 split of the phase step; thread sums
//     are FP32 (Kahan-compensated for the cost value), every sum above the warp
//     (block, job) is FP64.
//
// Both paths write one FP64 partial row per work item; the CTA that completes
// a job's last item sums the rows in item order (deterministic) and scatters
// slot derivatives to global parameters through the map.
#include <cuda_runtime.h>

#include <cstdint>

#include "musr_dev.h"

namespace musr {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kLog2eF = 1.44269504088896340736f;
constexpr float kLn2F = 0.69314718055994530942f;
constexpr int kMaxChan = 96;

// ---------------------------------------------------------------------------------------------
// PTX approximate transcendentals (documented PTX ISA instructions, FTZ).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2a(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcpa(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sina(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cosa(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// Round to nearest integer for |x| < 2^22 with two exact-rounding adds.
__device__ __forceinline__ float rint_small(float x) {
  return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Local value of slot s of histogram h.
__device__ __forceinline__ double slot_value(const HistSet& hs, const double* x, int h, int s) {
  int m = hs.map[static_cast<int64_t>(h) * hs.nslots + s];
  return m >= 0 ? x[m] : hs.consts[-1 - m];
}

// ---------------------------------------------------------------------------------------------
// Shared memory
// ---------------------------------------------------------------------------------------------
struct FinSmem {
  double wred[kWarps];
  int last;
  int bad;
};

struct Fp64Smem {
  double loc[kMaxSlots];
  double red[kWarps][36];
  int h, nlo, nhi, tile_start;
  double t0;
};

struct SplitSmem {
  float n0[kGroupMax], bkg[kGroupMax];
  float amp[kMaxTerms][kGroupMax], cph[kMaxTerms][kGroupMax], sph[kMaxTerms][kGroupMax];
  int row[kGroupMax];
  double loc[kGroupMax][kMaxSlots];
  float ca[kMaxTerms], cb[kMaxTerms];  // EX_k = ex2(-(ca t + cb t^2))  (includes 1/tau)
  float dh[kMaxTerms], d2[kMaxTerms];  // KT: g = ex2(-dh t^2), u = d2 t^2
  float shi[kMaxTerms], slo[kMaxTerms], sstep[kMaxTerms], base[kMaxTerms];
  int kinds[kMaxTerms];
  float aE, tbase, dt;
  int nlo, nhi, tile_start, nh, nterms;
  double red[kWarps][kMaxChan];
  double chan[kMaxChan];
};

union KernelSmem {
  Fp64Smem f64;
  SplitSmem split;
};

// ---------------------------------------------------------------------------------------------
// Job completion: the CTA that finishes the last item of a job reduces its rows.
// ---------------------------------------------------------------------------------------------
__device__ double block_sum_fixed(double v, FinSmem& fs) {
  v = warp_sum_d(v);
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) fs.wred[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kWarps; ++i) s += fs.wred[i];
    fs.wred[0] = s;
  }
  __syncthreads();
  s = fs.wred[0];
  __syncthreads();
  return s;
}

__device__ void finalize_job(const Job& job, const HistSet& hs, FinSmem& fs) {
  const int ps = hs.pstride;
  const double* part = job.partials;
  double v = 0.0;
  for (int i = threadIdx.x; i < hs.nitems; i += kBlock) v += __ldcg(part + static_cast<int64_t>(i) * ps);
  double value = block_sum_fixed(v, fs);
  bool finite = isfinite(value);
  if (job.grad) {
    for (int c = threadIdx.x; c < hs.ncols; c += kBlock) {
      const Chunk ch = hs.chunks[hs.col_chunk[c]];
      int local = c - ch.col0;
      double s = 0.0;
      for (int t = 0; t < ch.ntiles; ++t)
        s += __ldcg(part + static_cast<int64_t>(ch.item0 + t) * ps + 1 + local);
      job.colsum[c] = s;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < hs.P; p += kBlock) {
      double g = 0.0;
      for (int j = hs.p_ptr[p]; j < hs.p_ptr[p + 1]; ++j) g += job.colsum[hs.p_cols[j]];
      job.out[1 + p] = finite ? g : 0.0;
    }
  }
  if (threadIdx.x == 0) {
    job.out[0] = value;
    *job.counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------------
// FP64 path: one histogram per item, every operation in FP64, term list as given.
// ---------------------------------------------------------------------------------------------
template <int MODE, bool GRAD>
__device__ void fp64_item(const Job& job, const HistSet& hs, int item, Fp64Smem& sm, FinSmem& fs) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    int2 it = hs.items[item];
    const Chunk ch = hs.chunks[it.x];
    sm.h = hs.hist_index[ch.first];
    sm.nlo = ch.nlo;
    sm.nhi = ch.nhi;
    sm.tile_start = ch.tile0 + it.y * hs.tile_bins;
    sm.t0 = ch.t0;
  }
  __syncthreads();
  if (tid < hs.nslots) sm.loc[tid] = slot_value(hs, job.params, sm.h, tid);
  __syncthreads();

  const int h = sm.h, nlo = sm.nlo, nhi = sm.nhi, ts = sm.tile_start;
  const double t0 = sm.t0, dt = hs.dt_us;
  const int nterms = hs.nterms;
  const double N0 = sm.loc[0], Nbkg = sm.loc[1];
  const float* rowf = static_cast<const float*>(hs.counts) + static_cast<int64_t>(h) * hs.stride;
  const double* rowd = static_cast<const double*>(hs.counts) + static_cast<int64_t>(h) * hs.stride;

  double acc_v = 0.0, acc_n0 = 0.0, acc_bkg = 0.0;
  double acc_p[kMaxTerms][kMaxPrims][2];
#pragma unroll
  for (int k = 0; k < kMaxTerms; ++k)
#pragma unroll
    for (int m = 0; m < kMaxPrims; ++m) acc_p[k][m][0] = acc_p[k][m][1] = 0.0;
  int bad = 0;
  const int store = hs.store;

  const int end = min(nhi, ts + hs.tile_bins);
  for (int n = ts + tid; n < end; n += kBlock) {
    if (n < nlo) continue;
    // Bin time (Section 4.1: t = n dt, shifted by t0).
    const double t = (static_cast<double>(n) - t0) * dt;
    const double d = store == kStoreF64 ? rowd[n] : static_cast<double>(rowf[n]);
    const double E = exp(-t / kTauMuUs);
    // gd[k][m][q]: derivative of term k with respect to slot q of primitive m.
    double gd[kMaxTerms][kMaxPrims][2];
    double A = 0.0;
#pragma unroll
    for (int k = 0; k < kMaxTerms; ++k) {
      double f[kMaxPrims], df[kMaxPrims][2];
      const int np = k < nterms ? hs.raw[k].nprim : 0;
      double term = 1.0;
#pragma unroll
      for (int m = 0; m < kMaxPrims; ++m) {
        f[m] = 1.0;
        df[m][0] = df[m][1] = 0.0;
        if (m >= np) continue;
        const int kind = hs.raw[k].kind[m];
        const double p0 = sm.loc[hs.raw[k].slot[m][0]];
        if (kind == kAmp) {
          f[m] = p0;
          df[m][0] = 1.0;
        } else if (kind == kExp) {
          const double e = exp(-p0 * t);
          f[m] = e;
          df[m][0] = -t * e;
        } else if (kind == kGauss) {
          const double e = exp(-0.5 * (p0 * t) * (p0 * t));
          f[m] = e;
          df[m][0] = -p0 * t * t * e;
        } else if (kind == kKT) {
          const double u = (p0 * t) * (p0 * t);
          const double g = exp(-0.5 * u);
          f[m] = 1.0 / 3.0 + (2.0 / 3.0) * (1.0 - u) * g;
          df[m][0] = (2.0 / 3.0) * p0 * t * t * g * (u - 3.0);
        } else if (kind == kTFCos) {
          const double p1 = sm.loc[hs.raw[k].slot[m][1]];
          // Phase in turns, range-reduced exactly before sin/cos.
          const double x = p0 * t + p1 / 360.0;
          const double r = x - rint(x);
          double s, c;
          sincospi(2.0 * r, &s, &c);
          f[m] = c;
          df[m][0] = -s * kTwoPi * t;
          df[m][1] = -s * kTwoPi / 360.0;
        }
        term *= f[m];
      }
      if (np > 0) A += term;
      if (GRAD) {
#pragma unroll
        for (int m = 0; m < kMaxPrims; ++m) {
          double rest = 1.0;
#pragma unroll
          for (int q = 0; q < kMaxPrims; ++q)
            if (q != m) rest *= f[q];
          gd[k][m][0] = df[m][0] * rest;
          gd[k][m][1] = df[m][1] * rest;
        }
      }
    }
    const double N = N0 * E * (1.0 + A) + Nbkg;
    double v, W;  // per-bin cost and dcost/dN
    if (MODE == 0) {
      const double r = d - N;
      const double iv = 1.0 / fmax(d, 1.0);
      v = r * r * iv;
      W = -2.0 * r * iv;
    } else if (d > 0.0) {
      if (N <= 0.0) {
        bad = 1;
        v = 0.0;
        W = 0.0;
      } else {
        v = 2.0 * ((N - d) + d * log(d / N));
        W = 2.0 * (1.0 - d / N);
      }
    } else {
      v = 2.0 * (N - d);
      W = 2.0;
    }
    acc_v += v;
    if (GRAD) {
      acc_n0 += W * E * (1.0 + A);
      acc_bkg += W;
      const double wNE = W * N0 * E;
#pragma unroll
      for (int k = 0; k < kMaxTerms; ++k)
#pragma unroll
        for (int m = 0; m < kMaxPrims; ++m) {
          acc_p[k][m][0] += wNE * gd[k][m][0];
          acc_p[k][m][1] += wNE * gd[k][m][1];
        }
    }
  }

  // Block reduction in FP64 (warp shuffle, then warps in a fixed order).
  bad = __syncthreads_or(bad);
  const int w = tid >> 5, lane = tid & 31;
  double r0 = warp_sum_d(acc_v);
  if (lane == 0) sm.red[w][0] = r0;
  if (GRAD) {
    double r1 = warp_sum_d(acc_n0), r2 = warp_sum_d(acc_bkg);
    if (lane == 0) {
      sm.red[w][1] = r1;
      sm.red[w][2] = r2;
    }
#pragma unroll
    for (int k = 0; k < kMaxTerms; ++k)
#pragma unroll
      for (int m = 0; m < kMaxPrims; ++m)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          double r = warp_sum_d(acc_p[k][m][q]);
          if (lane == 0) sm.red[w][3 + (k * kMaxPrims + m) * 2 + q] = r;
        }
  }
  __syncthreads();
  double* row = job.partials + static_cast<int64_t>(item) * hs.pstride;
  if (tid == 0) {
    double s = 0.0;
    for (int i = 0; i < kWarps; ++i) s += sm.red[i][0];
    row[0] = bad ? __longlong_as_double(0x7ff0000000000000LL) : s;
  }
  if (GRAD && tid < hs.nslots) {
    // Channel -> slot: N0 is slot 0, Nbkg slot 1, primitives add to their slots.
    double tot[3 + kMaxTerms * kMaxPrims * 2];
    for (int c = 0; c < 3 + kMaxTerms * kMaxPrims * 2; ++c) {
      double s = 0.0;
      for (int i = 0; i < kWarps; ++i) s += sm.red[i][c];
      tot[c] = s;
    }
    double g = 0.0;
    if (tid == 0) g += tot[1];
    if (tid == 1) g += tot[2];
    for (int k = 0; k < nterms; ++k)
      for (int m = 0; m < hs.raw[k].nprim; ++m) {
        if (hs.raw[k].slot[m][0] == tid) g += tot[3 + (k * kMaxPrims + m) * 2 + 0];
        if (hs.raw[k].kind[m] == kTFCos && hs.raw[k].slot[m][1] == tid)
          g += tot[3 + (k * kMaxPrims + m) * 2 + 1];
      }
    row[1 + tid] = g;
  }
}

// ---------------------------------------------------------------------------------------------
// SPLIT path
// ---------------------------------------------------------------------------------------------
template <int S>
struct ShapeT;
template <>
struct ShapeT<kShapeGeneric> {
  static constexpr int NT = 4, G = 4;
  __device__ static int kind(const SplitSmem& sm, int k) { return sm.kinds[k]; }
  __device__ static int nterms(const SplitSmem& sm) { return sm.nterms; }
};
template <>
struct ShapeT<kShapeTF1> {
  static constexpr int NT = 1, G = 8;
  __device__ static constexpr int kind(const SplitSmem&, int) { return kTermTF; }
  __device__ static constexpr int nterms(const SplitSmem&) { return 1; }
};
template <>
struct ShapeT<kShapeTF2> {
  static constexpr int NT = 2, G = 8;
  __device__ static constexpr int kind(const SplitSmem&, int) { return kTermTF; }
  __device__ static constexpr int nterms(const SplitSmem&) { return 2; }
};
template <>
struct ShapeT<kShapeKT1> {
  static constexpr int NT = 1, G = 8;
  __device__ static constexpr int kind(const SplitSmem&, int) { return kTermKT; }
  __device__ static constexpr int nterms(const SplitSmem&) { return 1; }
};
template <>
struct ShapeT<kShapeTF2KT1> {
  static constexpr int NT = 3, G = 4;
  __device__ static constexpr int kind(const SplitSmem&, int k) { return k < 2 ? kTermTF : kTermKT; }
  __device__ static constexpr int nterms(const SplitSmem&) { return 3; }
};

// Per-item set-up: local slot values, per-histogram FP32 constants and the
// shared time-factor coefficients of the chunk, including the FP64 range
// reduction of each precession phase at the tile's first bin.
template <int SHAPE>
__device__ void split_prologue(const Job& job, const HistSet& hs, int item, SplitSmem& sm) {
  using Sh = ShapeT<SHAPE>;
  const int tid = threadIdx.x;
  __shared__ int s_first;
  __shared__ double s_t0;
  if (tid == 0) {
    int2 it = hs.items[item];
    const Chunk ch = hs.chunks[it.x];
    sm.nh = ch.nh;
    sm.nlo = ch.nlo;
    sm.nhi = ch.nhi;
    sm.tile_start = ch.tile0 + it.y * hs.tile_bins;
    sm.nterms = hs.nterms;
    s_first = ch.first;
    s_t0 = ch.t0;
  }
  __syncthreads();
  const int nh = sm.nh, nsl = hs.nslots;
  for (int i = tid; i < nh * nsl; i += kBlock) {
    int hl = i / nsl, s = i - hl * nsl;
    int h = hs.hist_index[s_first + hl];
    sm.loc[hl][s] = slot_value(hs, job.params, h, s);
    if (s == 0) sm.row[hl] = h;
  }
  if (tid < kMaxTerms) sm.kinds[tid] = tid < hs.nterms ? hs.canon[tid].kind : kTermNone;
  __syncthreads();
  const double dt = hs.dt_us;
  const double t_start = (static_cast<double>(sm.tile_start) - s_t0) * dt;
  if (tid < nh) {
    const int hl = tid;
    sm.n0[hl] = static_cast<float>(sm.loc[hl][0]);
    sm.bkg[hl] = static_cast<float>(sm.loc[hl][1]);
#pragma unroll
    for (int k = 0; k < kMaxTerms; ++k) {
      float a = 0.0f, c = 1.0f, s = 0.0f;
      if (k < hs.nterms) {
        const CanonTerm& ct = hs.canon[k];
        a = ct.amp_slot >= 0 ? static_cast<float>(sm.loc[hl][ct.amp_slot]) : 1.0f;
        if (ct.kind == kTermTF) {
          double x = sm.loc[hl][ct.phi_slot] / 360.0;  // phase in turns
          double r = x - rint(x);
          sincospif(2.0f * static_cast<float>(r), &s, &c);
        }
      }
      sm.amp[k][hl] = a;
      sm.cph[k][hl] = c;
      sm.sph[k][hl] = s;
    }
  } else if (tid >= 32 && tid < 32 + kMaxTerms) {
    const int k = tid - 32;
    if (k < hs.nterms) {
      const CanonTerm& ct = hs.canon[k];
      double lam = 0.0, S = 0.0;
      for (int i = 0; i < ct.nexp; ++i) lam += sm.loc[0][ct.exp_slot[i]];
      for (int i = 0; i < ct.ngauss; ++i) {
        double sg = sm.loc[0][ct.gauss_slot[i]];
        S += sg * sg;
      }
      sm.ca[k] = static_cast<float>(1.4426950408889634 * (1.0 / kTauMuUs + lam));
      sm.cb[k] = static_cast<float>(1.4426950408889634 * 0.5 * S);
      if (ct.kind == kTermKT) {
        double D = sm.loc[0][ct.kt_slot];
        sm.d2[k] = static_cast<float>(D * D);
        sm.dh[k] = static_cast<float>(1.4426950408889634 * 0.5 * D * D);
      } else {
        sm.d2[k] = sm.dh[k] = 0.0f;
      }
      if (ct.kind == kTermTF) {
        const double nu = sm.loc[0][ct.nu_slot];
        const double step = nu * dt;  // turns per bin
        // Exact split: hi keeps 11 significant bits, so (bin offset < 2^13) * hi is exact in FP32.
        double hi = 0.0;
        if (step != 0.0) {
          int e;
          frexp(step, &e);
          double sc = ldexp(1.0, 11 - e);
          hi = trunc(step * sc) / sc;
        }
        sm.shi[k] = static_cast<float>(hi);
        sm.slo[k] = static_cast<float>(step - hi);
        sm.sstep[k] = static_cast<float>(step);
        double x = nu * t_start;  // FP64 range reduction at the tile's first bin
        sm.base[k] = static_cast<float>(x - rint(x));
      } else {
        sm.shi[k] = sm.slo[k] = sm.sstep[k] = sm.base[k] = 0.0f;
      }
    }
  } else if (tid == 64) {
    sm.aE = static_cast<float>(1.4426950408889634 / kTauMuUs);
    sm.tbase = static_cast<float>(t_start);
    sm.dt = static_cast<float>(dt);
  }
  __syncthreads();
  (void)Sh::NT;
}

template <int SHAPE, int MODE, bool GRAD>
__device__ void split_item(const Job& job, const HistSet& hs, int item, SplitSmem& sm, FinSmem& fs) {
  using Sh = ShapeT<SHAPE>;
  constexpr int NT = Sh::NT;
  constexpr int G = Sh::G;
  constexpr int NPH = 2 + 2 * NT;  // per-histogram channels: N0, bkg, amp[k], phi[k]
  constexpr int NSH = 4 * NT;      // shared channels per term: lambda, S, nu, Delta
  static_assert(G * NPH + NSH <= kMaxChan, "channel count");

  split_prologue<SHAPE>(job, hs, item, sm);

  const int tid = threadIdx.x;
  const int nh = sm.nh, nlo = sm.nlo, nhi = sm.nhi, ts = sm.tile_start;
  const int nterms = Sh::nterms(sm);
  const float aE = sm.aE, tbase = sm.tbase, dtf = sm.dt;
  const void* __restrict__ counts = hs.counts;
  const int64_t stride = hs.stride;
  const int store = hs.store;

  float acc_v = 0.0f, acc_c = 0.0f;  // Kahan-compensated cost value
  float ph[G][NPH];
  float sh[NT][4];
#pragma unroll
  for (int i = 0; i < G; ++i)
#pragma unroll
    for (int q = 0; q < NPH; ++q) ph[i][q] = 0.0f;
#pragma unroll
  for (int k = 0; k < NT; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) sh[k][q] = 0.0f;
  int bad = 0;

  const int iters = hs.tile_bins / (kBlock * kBinsPerThread);
  for (int it = 0; it < iters; ++it) {
    const int m0 = it * kBlock * kBinsPerThread + tid * kBinsPerThread;  // offset in tile (< 2^13)
    const int n0 = ts + m0;
    if (n0 >= nhi) break;
    float t[4];
    bool valid[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      t[j] = fmaf(static_cast<float>(m0 + j), dtf, tbase);
      valid[j] = (n0 + j >= nlo) && (n0 + j < nhi);
    }
    // Time-only factors of the chunk.
    float E[4], EXK[NT][4], cs[NT][4], sn[NT][4], dk[NT][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) E[j] = ex2a(-aE * t[j]);
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const int kk = Sh::kind(sm, k);
      if (k >= nterms) {
#pragma unroll
        for (int j = 0; j < 4; ++j) EXK[k][j] = cs[k][j] = sn[k][j] = dk[k][j] = 0.0f;
        continue;
      }
      const float ca = sm.ca[k], cb = sm.cb[k];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float ex = ex2a(-fmaf(cb, t[j], ca) * t[j]);
        EXK[k][j] = ex;
        cs[k][j] = 1.0f;
        sn[k][j] = 0.0f;
        dk[k][j] = 0.0f;
        if (kk == kTermKT) {
          const float tt = t[j] * t[j];
          const float g = ex2a(-sm.dh[k] * tt);
          const float u = sm.d2[k] * tt;
          EXK[k][j] = ex * fmaf((2.0f / 3.0f) * (1.0f - u), g, 1.0f / 3.0f);
          dk[k][j] = ex * tt * g * (u - 3.0f);
        }
      }
      if (kk == kTermTF) {
        // Phase (turns) of the thread's first bin: base + m0 * step, reduced exactly.
        float f = static_cast<float>(m0) * sm.shi[k];
        f = __fsub_rn(f, rint_small(f));
        float r = fmaf(static_cast<float>(m0), sm.slo[k], sm.base[k]) + f;
        r = __fsub_rn(r, rint_small(r));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float rj = fmaf(static_cast<float>(j), sm.sstep[k], r);
          rj = __fsub_rn(rj, rint_small(rj));  // |rj| <= 1/2: sin/cos arguments in [-pi, pi]
          const float a = rj * kTwoPiF;
          cs[k][j] = cosa(a);
          sn[k][j] = sina(a);
        }
      }
    }
    float U[NT][4], V[NT][4];
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
      for (int j = 0; j < 4; ++j) U[k][j] = V[k][j] = 0.0f;

#pragma unroll
    for (int hl = 0; hl < G; ++hl) {
      if (hl >= nh) break;
      float d[4];
      const int64_t off = static_cast<int64_t>(sm.row[hl]) * stride + n0;
      if (store == kStoreF32) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(counts) + off));
        d[0] = q.x;
        d[1] = q.y;
        d[2] = q.z;
        d[3] = q.w;
      } else {
        const double2* p = reinterpret_cast<const double2*>(static_cast<const double*>(counts) + off);
        const double2 q0 = __ldg(p), q1 = __ldg(p + 1);
        d[0] = static_cast<float>(q0.x);
        d[1] = static_cast<float>(q0.y);
        d[2] = static_cast<float>(q1.x);
        d[3] = static_cast<float>(q1.y);
      }
      const float N0 = sm.n0[hl], Nb = sm.bkg[hl];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float C[NT], Sn[NT], Q[NT];
        float M = E[j];
#pragma unroll
        for (int k = 0; k < NT; ++k) {
          if (k >= nterms) {
            C[k] = Sn[k] = Q[k] = 0.0f;
            continue;
          }
          if (Sh::kind(sm, k) == kTermTF) {
            const float cp = sm.cph[k][hl], sp = sm.sph[k][hl];
            C[k] = fmaf(cs[k][j], cp, -sn[k][j] * sp);  // cos(theta + phi)
            Sn[k] = fmaf(sn[k][j], cp, cs[k][j] * sp);  // sin(theta + phi)
          } else {
            C[k] = 1.0f;
            Sn[k] = 0.0f;
          }
          Q[k] = EXK[k][j] * C[k];
          M = fmaf(sm.amp[k][hl], Q[k], M);
        }
        const float N = fmaf(N0, M, Nb);
        const float dd = d[j];
        float v, w;  // per-bin cost (chi^2, or half the deviance) and d(cost/2)/dN
        if (MODE == 0) {
          const float iv = rcpa(fmaxf(dd, 1.0f));
          const float r = N - dd;
          w = r * iv;
          v = r * w;
        } else {
          if (dd > 0.0f) {
            if (N <= 0.0f) {
              bad = 1;
              v = 0.0f;
              w = 0.0f;
            } else {
              // d [y - ln(1 + y)], y = (N - d)/d: a series in z = y/(2+y) where |z| < 0.2,
              // y - ln(1+y) = z (y - 2 z^2 (1/3 + z^2/5 + ...)), else y - ln(1 + y) directly.
              const float y = (N - dd) * rcpa(dd);
              const float z = y * rcpa(2.0f + y);
              const float z2 = z * z;
              float pz = fmaf(z2, 1.0f / 13.0f, 1.0f / 11.0f);
              pz = fmaf(z2, pz, 1.0f / 9.0f);
              pz = fmaf(z2, pz, 1.0f / 7.0f);
              pz = fmaf(z2, pz, 1.0f / 5.0f);
              pz = fmaf(z2, pz, 1.0f / 3.0f);
              const float phs = z * fmaf(-2.0f * z2, pz, y);
              const float phl = y - lg2a(1.0f + y) * kLn2F;
              v = dd * (fabsf(z) < 0.2f ? phs : phl);
              w = (N - dd) * rcpa(N);
            }
          } else {
            v = N - dd;
            w = 1.0f;
          }
        }
        if (!valid[j]) {
          v = 0.0f;
          w = 0.0f;
        }
        {
          const float y = v - acc_c;
          const float tsum = acc_v + y;
          acc_c = (tsum - acc_v) - y;
          acc_v = tsum;
        }
        if (GRAD) {
          ph[hl][0] = fmaf(w, M, ph[hl][0]);
          ph[hl][1] += w;
          const float wN0 = w * N0;
#pragma unroll
          for (int k = 0; k < NT; ++k) {
            if (k >= nterms) continue;
            ph[hl][2 + k] = fmaf(w, Q[k], ph[hl][2 + k]);
            const float P = wN0 * sm.amp[k][hl];
            U[k][j] = fmaf(P, C[k], U[k][j]);
            if (Sh::kind(sm, k) == kTermTF) {
              ph[hl][2 + NT + k] = fmaf(w * Sn[k], EXK[k][j], ph[hl][2 + NT + k]);
              V[k][j] = fmaf(P, Sn[k], V[k][j]);
            }
          }
        }
      }
    }
    if (GRAD) {
      // Shared channels: time-only factor times the chunk's per-bin sums.
#pragma unroll
      for (int k = 0; k < NT; ++k) {
        if (k >= nterms) continue;
        const int kk = Sh::kind(sm, k);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float ue = U[k][j] * EXK[k][j];
          sh[k][0] = fmaf(-t[j], ue, sh[k][0]);               // d/dLambda
          sh[k][1] = fmaf(-0.5f * t[j] * t[j], ue, sh[k][1]);  // d/dS
          if (kk == kTermTF) sh[k][2] = fmaf(-kTwoPiF * t[j] * EXK[k][j], V[k][j], sh[k][2]);
          if (kk == kTermKT) sh[k][3] = fmaf(U[k][j], dk[k][j], sh[k][3]);
        }
      }
    }
  }

  // ---- reduction: thread (FP32) -> warp (FP32 for gradient channels, FP64 for the value)
  //      -> block (FP64, warps in fixed order) -> one FP64 row per item.
  bad = __syncthreads_or(bad);
  const int w = tid >> 5, lane = tid & 31;
  double vt = static_cast<double>(acc_v) - static_cast<double>(acc_c);
  vt = warp_sum_d(vt);
  constexpr int VCH = G * NPH + NSH;
  if (lane == 0) sm.red[w][VCH] = vt;
  if (GRAD) {
#pragma unroll
    for (int hl = 0; hl < G; ++hl)
#pragma unroll
      for (int q = 0; q < NPH; ++q) {
        float r = warp_sum_f(ph[hl][q]);
        if (lane == 0) sm.red[w][hl * NPH + q] = static_cast<double>(r);
      }
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float r = warp_sum_f(sh[k][q]);
        if (lane == 0) sm.red[w][G * NPH + k * 4 + q] = static_cast<double>(r);
      }
  }
  __syncthreads();
  for (int c = tid; c <= (GRAD ? VCH : 0); c += kBlock) {
    const int cc = GRAD ? c : VCH;
    double s = 0.0;
    for (int i = 0; i < kWarps; ++i) s += sm.red[i][cc];
    sm.chan[cc] = s;
  }
  __syncthreads();
  double* row = job.partials + static_cast<int64_t>(item) * hs.pstride;
  if (tid == 0) {
    const double val = sm.chan[VCH] * (MODE == 1 ? 2.0 : 1.0);
    row[0] = bad ? __longlong_as_double(0x7ff0000000000000LL) : val;
  }
  if (GRAD) {
    const int nsl = hs.nslots;
    for (int i = tid; i < G * nsl; i += kBlock) {
      const int hl = i / nsl, s = i - hl * nsl;
      double g = 0.0;
      if (hl < nh) {
        const double N0 = sm.loc[hl][0];
        for (int e = 0; e < hs.ncontrib; ++e) {
          const Contrib c = hs.contrib[e];
          if (c.slot != s) continue;
          const int k = c.term;
          switch (c.kind) {
            case kCN0:
              g += 2.0 * sm.chan[hl * NPH + 0];
              break;
            case kCBkg:
              g += 2.0 * sm.chan[hl * NPH + 1];
              break;
            case kCAmp:
              g += 2.0 * N0 * sm.chan[hl * NPH + 2 + k];
              break;
            case kCPhi: {
              const int as = hs.canon[k].amp_slot;
              const double a = as >= 0 ? sm.loc[hl][as] : 1.0;
              g += 2.0 * N0 * a * (-kTwoPi / 360.0) * sm.chan[hl * NPH + 2 + NT + k];
              break;
            }
            case kCLam:
              if (hl == 0) g += 2.0 * sm.chan[G * NPH + k * 4 + 0];
              break;
            case kCSig:
              if (hl == 0) g += 4.0 * sm.loc[0][s] * sm.chan[G * NPH + k * 4 + 1];
              break;
            case kCNu:
              if (hl == 0) g += 2.0 * sm.chan[G * NPH + k * 4 + 2];
              break;
            case kCDel:
              if (hl == 0) g += (4.0 / 3.0) * sm.loc[0][s] * sm.chan[G * NPH + k * 4 + 3];
              break;
            default:
              break;
          }
        }
      }
      row[1 + i] = g;
    }
  }
  (void)fs;
}

// ---------------------------------------------------------------------------------------------
// Persistent kernel: items of all jobs, strided over the grid.
// ---------------------------------------------------------------------------------------------
template <int PREC, int SHAPE, int MODE, bool GRAD>
__global__ void __launch_bounds__(kBlock) eval_kernel(const Job* __restrict__ jobs, int njobs,
                                                      int total_items) {
  __shared__ KernelSmem sm;
  __shared__ FinSmem fs;
  for (int gi = blockIdx.x; gi < total_items; gi += gridDim.x) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].item_begin <= gi)
        lo = mid;
      else
        hi = mid - 1;
    }
    const Job job = jobs[lo];
    const HistSet& hs = *job.hs;
    const int item = gi - job.item_begin;
    if (PREC == 0)
      fp64_item<MODE, GRAD>(job, hs, item, sm.f64, fs);
    else
      split_item<SHAPE, MODE, GRAD>(job, hs, item, sm.split, fs);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned prev = atomicAdd(job.counter, 1u);
      fs.last = (prev == static_cast<unsigned>(hs.nitems - 1));
    }
    __syncthreads();
    if (fs.last) {
      __threadfence();
      finalize_job(job, hs, fs);
    }
    __syncthreads();
  }
}

template <int PREC, int SHAPE, int MODE, bool GRAD>
int launch_one(const Job* d_jobs, int njobs, int total_items, int num_sms, cudaStream_t stream,
               LaunchInfo* info) {
  auto kern = eval_kernel<PREC, SHAPE, MODE, GRAD>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0) != cudaSuccess) return -1;
  if (per_sm < 1) per_sm = 1;
  int grid = num_sms * per_sm;
  if (grid > total_items) grid = total_items;
  if (grid < 1) grid = 1;
  kern<<<grid, kBlock, 0, stream>>>(d_jobs, njobs, total_items);
  if (info) {
    info->grid = grid;
    info->block = kBlock;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int PREC, int SHAPE, int MODE, bool GRAD>
int occupancy_one() {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eval_kernel<PREC, SHAPE, MODE, GRAD>, kBlock, 0);
  return per_sm;
}

template <int PREC, int SHAPE>
int dispatch_mode(int mode, int grad, const Job* j, int n, int items, int sms, cudaStream_t s,
                  LaunchInfo* info) {
  if (mode == 0)
    return grad ? launch_one<PREC, SHAPE, 0, true>(j, n, items, sms, s, info)
                : launch_one<PREC, SHAPE, 0, false>(j, n, items, sms, s, info);
  return grad ? launch_one<PREC, SHAPE, 1, true>(j, n, items, sms, s, info)
              : launch_one<PREC, SHAPE, 1, false>(j, n, items, sms, s, info);
}

template <int PREC, int SHAPE>
int occupancy_mode(int mode, int grad) {
  if (mode == 0) return grad ? occupancy_one<PREC, SHAPE, 0, true>() : occupancy_one<PREC, SHAPE, 0, false>();
  return grad ? occupancy_one<PREC, SHAPE, 1, true>() : occupancy_one<PREC, SHAPE, 1, false>();
}

}  // namespace

int shape_group(int shape) {
  switch (shape) {
    case kShapeTF1:
      return ShapeT<kShapeTF1>::G;
    case kShapeTF2:
      return ShapeT<kShapeTF2>::G;
    case kShapeKT1:
      return ShapeT<kShapeKT1>::G;
    case kShapeTF2KT1:
      return ShapeT<kShapeTF2KT1>::G;
    default:
      return ShapeT<kShapeGeneric>::G;
  }
}

int launch_eval(int precision, int shape, int mode, int grad, const Job* d_jobs, int njobs,
                int total_items, int num_sms, void* stream, LaunchInfo* info) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == 0) return dispatch_mode<0, 0>(mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
  switch (shape) {
    case kShapeTF1:
      return dispatch_mode<1, kShapeTF1>(mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
    case kShapeTF2:
      return dispatch_mode<1, kShapeTF2>(mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
    case kShapeKT1:
      return dispatch_mode<1, kShapeKT1>(mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
    case kShapeTF2KT1:
      return dispatch_mode<1, kShapeTF2KT1>(mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
    default:
      return dispatch_mode<1, kShapeGeneric>(mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
  }
}

int max_ctas_per_sm(int precision, int shape, int mode, int grad) {
  if (precision == 0) return occupancy_mode<0, 0>(mode, grad);
  switch (shape) {
    case kShapeTF1:
      return occupancy_mode<1, kShapeTF1>(mode, grad);
    case kShapeTF2:
      return occupancy_mode<1, kShapeTF2>(mode, grad);
    case kShapeKT1:
      return occupancy_mode<1, kShapeKT1>(mode, grad);
    case kShapeTF2KT1:
      return occupancy_mode<1, kShapeTF2KT1>(mode, grad);
    default:
      return occupancy_mode<1, kShapeGeneric>(mode, grad);
  }
}

}  // namespace musr
