// musr_kernels.cu -- evaluation kernels of libmusr (sm_103a).
//
// The cost of Section 4.1 of arXiv 1509.07685 is a map-reduce over every bin
// of every histogram: Eq. positron_histo gives the expected count N, Eq. chisq
// or Eq. log-likelihood turns (d, N) into a per-bin term, and the terms are
// summed.  The gradient is the same reduction of (dcost/dN) * (dN/dslot).
// No tensor cores: nothing here is a contraction.
//
// Two paths:
//   * FP64 ("plain"): one work item is a tile of one histogram; every per-bin
//     operation in FP64, the term list interpreted as given (any product of
//     primitives).
//   * SPLIT: one work item is a tile of a chunk of <= 8 histograms that share
//     the time grid and every time-dependent parameter.  For each bin the
//     time-only factors (muon decay, relaxations, Kubo-Toyabe, the precession's
//     cos/sin) are computed once and reused by the chunk's histograms; the
//     per-histogram phase enters by a rotation.  Per-bin work is FP32 (hardware
//     ex2, lg2, rcp, sin, cos); the precession phase is range-reduced in FP64
//     once per tile and carried per bin as an exact FP32 split of the phase step.
//
// Reductions.  FP64 runs ~60x slower than FP32 per warp instruction on this
// GPU, so it is kept where it buys accuracy and out of every per-bin and
// per-lane path: thread sums are FP32 (the cost value Kahan-compensated), warp
// sums FP32 (the value as a compensated float-float pair), the sum over the
// CTA's warps is FP64, and so is every sum over work items, chunks and the
// final scatter to parameters.
//
// Completion.  Each item writes one FP64 row of channel sums.  The CTA that
// completes a chunk's last item sums the chunk's rows in item order and turns
// channels into slot derivatives; the CTA that completes a job's last chunk
// sums the chunks in chunk order and scatters slots to parameters through the
// map.  The result depends on neither the CTA that ran an item nor on other
// jobs in the launch.
#include <cuda_runtime.h>

#include <cstdint>

#include "musr_dev.h"

namespace musr {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kLn2F = 0.69314718055994530942f;
constexpr float kLog2eF = 1.44269504088896340736f;
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
// Round to nearest integer for |x| < 2^22 with two exactly rounded adds.
__device__ __forceinline__ float rint_small(float x) {
  return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
}

// ---------------------------------------------------------------------------------------------
// TMA bulk copies global -> shared with mbarrier completion (documented PTX ISA).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of the barrier; false when the iteration limit ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  for (int i = 0; i < (1 << 20); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
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
// Warp sum of a float-float pair (hi, lo): Knuth's TwoSum on the hi parts.
__device__ __forceinline__ void warp_sum_ff(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = __fadd_rn(hi, h2);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(l2, e));
  }
}

// Local value of slot s of histogram h.
__device__ __forceinline__ double slot_value(const HistSet& hs, const double* x, int h, int s) {
  const int m = hs.map[static_cast<int64_t>(h) * hs.nslots + s];
  return m >= 0 ? x[m] : hs.consts[-1 - m];
}

// ---------------------------------------------------------------------------------------------
// Shared memory
// ---------------------------------------------------------------------------------------------

// Chunk-level constants, cached while a CTA stays on one chunk of one job.
struct ChunkCache {
  int job, chunk;  // cache key (-1: empty)
  int nh, nlo, nhi, tile0, item0, ntiles, col0, first;
  double t0;
  int row[kGroupMax];
  const void* rowp[kGroupMax];       // first count of each histogram's row
  double loc[kGroupMax][kMaxSlots];  // local slot values (FP64)
  // SPLIT per-histogram FP32 constants
  float n0[kGroupMax], bkg[kGroupMax];
  float amp[kMaxTerms][kGroupMax], cph[kMaxTerms][kGroupMax], sph[kMaxTerms][kGroupMax];
  // SPLIT per-term constants of the chunk
  int kinds[kMaxTerms];
  float ca[kMaxTerms], cb[kMaxTerms];  // E*X_k = ex2(-(ca t + cb t^2))  (ca includes 1/tau)
  float dh[kMaxTerms], d2[kMaxTerms];  // KT: g = ex2(-dh t^2), u = d2 t^2
  float shi[kMaxTerms], slo[kMaxTerms], sstep[kMaxTerms];
  double nu[kMaxTerms];
  float aE, dt;
};

struct TileState {
  int tile_start;
  float tbase;
  float base[kMaxTerms];  // phase (turns, in [-1/2, 1/2]) of each TF term at the tile's first bin
};

struct Smem {
  // SPLIT, FP32 counts: the rows of the current and the next CTA iteration, staged
  // by TMA bulk copies (one per histogram row segment), one mbarrier per buffer.
  alignas(128) float stage[2][kGroupMax][kBlock * kBinsPerThread];
  unsigned long long bar[2];
  ChunkCache cc;
  TileState ts;
  float cred[kWarps][kMaxChan];  // per-warp FP32 channel sums
  float vred[kWarps][2];         // per-warp float-float value
  double dred[kWarps][kFp64Channels + 2];
  double tot[kMaxChan + 1];      // chunk totals in the chunk finalize
  double wsum[kWarps];
  int flag;
  int bad;
};

// ---------------------------------------------------------------------------------------------
// Chunk cache fill (only when a CTA moves to another chunk or job).
// ---------------------------------------------------------------------------------------------
__device__ void load_chunk(const Job& job, const HistSet& hs, int job_index, int chunk_index, int prec,
                           Smem& sm) {
  ChunkCache& cc = sm.cc;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const Chunk ch = hs.chunks[chunk_index];
    cc.job = job_index;
    cc.chunk = chunk_index;
    cc.nh = ch.nh;
    cc.nlo = ch.nlo;
    cc.nhi = ch.nhi;
    cc.tile0 = ch.tile0;
    cc.item0 = ch.item0;
    cc.ntiles = ch.ntiles;
    cc.col0 = ch.col0;
    cc.first = ch.first;
    cc.t0 = ch.t0;
  }
  __syncthreads();
  const int nh = cc.nh, nsl = hs.nslots;
  for (int i = tid; i < nh * nsl; i += kBlock) {
    const int hl = i / nsl, s = i - hl * nsl;
    const int h = hs.hist_index[cc.first + hl];
    cc.loc[hl][s] = slot_value(hs, job.params, h, s);
    if (s == 0) {
      cc.row[hl] = h;
      const size_t esz = hs.store == kStoreF64 ? sizeof(double) : sizeof(float);
      cc.rowp[hl] = static_cast<const char*>(hs.counts) + static_cast<size_t>(h) * hs.stride * esz;
    }
  }
  __syncthreads();
  if (prec == 0) return;
  const double dt = hs.dt_us;
  if (tid < nh) {
    const int hl = tid;
    cc.n0[hl] = static_cast<float>(cc.loc[hl][0]);
    cc.bkg[hl] = static_cast<float>(cc.loc[hl][1]);
#pragma unroll
    for (int k = 0; k < kMaxTerms; ++k) {
      float a = 0.0f, c = 1.0f, s = 0.0f;
      if (k < hs.nterms) {
        const CanonTerm& ct = hs.canon[k];
        a = ct.amp_slot >= 0 ? static_cast<float>(cc.loc[hl][ct.amp_slot]) : 1.0f;
        if (ct.kind == kTermTF) {
          const double x = cc.loc[hl][ct.phi_slot] * (1.0 / 360.0);  // phase in turns (FP64)
          const float r = static_cast<float>(x - rint(x));
          sincospif(2.0f * r, &s, &c);
        }
      }
      cc.amp[k][hl] = a;
      cc.cph[k][hl] = c;
      cc.sph[k][hl] = s;
    }
  } else if (tid >= 32 && tid < 32 + kMaxTerms) {
    const int k = tid - 32;
    cc.kinds[k] = k < hs.nterms ? hs.canon[k].kind : kTermNone;
    if (k < hs.nterms) {
      const CanonTerm& ct = hs.canon[k];
      float lam = 0.0f, S = 0.0f;
      for (int i = 0; i < ct.nexp; ++i) lam += static_cast<float>(cc.loc[0][ct.exp_slot[i]]);
      for (int i = 0; i < ct.ngauss; ++i) {
        const float sg = static_cast<float>(cc.loc[0][ct.gauss_slot[i]]);
        S = fmaf(sg, sg, S);
      }
      cc.ca[k] = kLog2eF * (static_cast<float>(1.0 / kTauMuUs) + lam);
      cc.cb[k] = kLog2eF * 0.5f * S;
      if (ct.kind == kTermKT) {
        const float D = static_cast<float>(cc.loc[0][ct.kt_slot]);
        cc.d2[k] = D * D;
        cc.dh[k] = kLog2eF * 0.5f * D * D;
      } else {
        cc.d2[k] = cc.dh[k] = 0.0f;
      }
      if (ct.kind == kTermTF) {
        const double nu = cc.loc[0][ct.nu_slot];
        const double step = nu * dt;  // turns per bin (FP64)
        // Exact split: hi keeps 10 significant bits, so (bin offset < 2^14) * hi is exact in FP32.
        const float hi = __uint_as_float(__float_as_uint(static_cast<float>(step)) & 0xFFFFC000u);
        cc.shi[k] = hi;
        cc.slo[k] = static_cast<float>(step - static_cast<double>(hi));
        cc.sstep[k] = static_cast<float>(step);
        cc.nu[k] = nu;
      } else {
        cc.shi[k] = cc.slo[k] = cc.sstep[k] = 0.0f;
        cc.nu[k] = 0.0;
      }
    }
  } else if (tid == 64) {
    cc.aE = static_cast<float>(1.4426950408889634 / kTauMuUs);
    cc.dt = static_cast<float>(dt);
  }
  __syncthreads();
}

// Tile-level constants: the tile's first bin time and, in FP64, each precession
// phase at that bin reduced to [-1/2, 1/2] turns.
__device__ void load_tile(const HistSet& hs, int tile, int prec, Smem& sm) {
  const int tid = threadIdx.x;
  if (tid == 0) sm.ts.tile_start = sm.cc.tile0 + tile * hs.tile_bins;
  if (prec == 1 && tid >= 32 && tid < 32 + kMaxTerms) {
    const int k = tid - 32;
    const int ts = sm.cc.tile0 + tile * hs.tile_bins;
    const double t_start = (static_cast<double>(ts) - sm.cc.t0) * hs.dt_us;
    if (k == 0) sm.ts.tbase = static_cast<float>(t_start);
    float b = 0.0f;
    if (sm.cc.kinds[k] == kTermTF) {
      const double x = sm.cc.nu[k] * t_start;
      b = static_cast<float>(x - rint(x));
    }
    sm.ts.base[k] = b;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// FP64 path: one histogram per chunk, every operation in FP64, term list as given.
// Row: [value, N0, Nbkg, d/d(term k, primitive m, slot q)...].
// ---------------------------------------------------------------------------------------------
template <int MODE, bool GRAD>
__device__ void fp64_item(const Job& job, const HistSet& hs, int item, Smem& sm) {
  const int tid = threadIdx.x;
  const ChunkCache& cc = sm.cc;
  const int h = cc.row[0], nlo = cc.nlo, nhi = cc.nhi, ts = sm.ts.tile_start;
  const double t0 = cc.t0, dt = hs.dt_us;
  const int nterms = hs.nterms;
  const double N0 = cc.loc[0][0], Nbkg = cc.loc[0][1];
  const float* rowf = static_cast<const float*>(hs.counts) + static_cast<int64_t>(h) * hs.stride;
  const double* rowd = static_cast<const double*>(hs.counts) + static_cast<int64_t>(h) * hs.stride;
  const int store = hs.store;

  double acc_v = 0.0, acc_n0 = 0.0, acc_bkg = 0.0;
  double acc_p[kMaxTerms][kMaxPrims][2];
#pragma unroll
  for (int k = 0; k < kMaxTerms; ++k)
#pragma unroll
    for (int m = 0; m < kMaxPrims; ++m) acc_p[k][m][0] = acc_p[k][m][1] = 0.0;
  int bad = 0;

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
        const double p0 = cc.loc[0][hs.raw[k].slot[m][0]];
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
          const double p1 = cc.loc[0][hs.raw[k].slot[m][1]];
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

  // Warp (FP64 shuffles), then the CTA's warps in a fixed order (FP64).
  bad = __syncthreads_or(bad);
  const int w = tid >> 5, lane = tid & 31;
  const double r0 = warp_sum_d(acc_v);
  if (lane == 0) sm.dred[w][0] = r0;
  if (GRAD) {
    const double r1 = warp_sum_d(acc_n0), r2 = warp_sum_d(acc_bkg);
    if (lane == 0) {
      sm.dred[w][1] = r1;
      sm.dred[w][2] = r2;
    }
#pragma unroll
    for (int k = 0; k < kMaxTerms; ++k)
#pragma unroll
      for (int m = 0; m < kMaxPrims; ++m)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const double r = warp_sum_d(acc_p[k][m][q]);
          if (lane == 0) sm.dred[w][3 + (k * kMaxPrims + m) * 2 + q] = r;
        }
  }
  __syncthreads();
  double* row = job.partials + static_cast<int64_t>(item) * hs.pstride;
  const int nout = GRAD ? 1 + kFp64Channels : 1;
  for (int c = tid; c < nout; c += kBlock) {
    double s = 0.0;
    for (int i = 0; i < kWarps; ++i) s += sm.dred[i][c];
    if (c == 0 && bad) s = __longlong_as_double(0x7ff0000000000000LL);
    row[c] = s;
  }
}

// FP64 channels -> slot derivatives of the chunk's histogram.
__device__ double fp64_slot(const HistSet& hs, const double* tot, int s) {
  double g = 0.0;
  if (s == 0) g += tot[1];
  if (s == 1) g += tot[2];
  for (int k = 0; k < hs.nterms; ++k)
    for (int m = 0; m < hs.raw[k].nprim; ++m) {
      if (hs.raw[k].slot[m][0] == s) g += tot[3 + (k * kMaxPrims + m) * 2 + 0];
      if (hs.raw[k].kind[m] == kTFCos && hs.raw[k].slot[m][1] == s) g += tot[3 + (k * kMaxPrims + m) * 2 + 1];
    }
  return g;
}

// ---------------------------------------------------------------------------------------------
// SPLIT path
// ---------------------------------------------------------------------------------------------
template <int S>
struct ShapeT;
// NT: terms; G: histograms per chunk; AMP: whether amplitude channels are kept
// (the "c" shapes drop them: every amplitude is a constant); NTF: phase channels;
// phi(k): the phase channel of cosine term k (the "c" shapes also require one
// phase slot shared by all cosine terms, so a single channel holds their sum).
template <>
struct ShapeT<kShapeGeneric> {
  static constexpr int NT = 4, G = 2, NTF = 4;
  static constexpr bool AMP = true;
  __device__ static int kind(const ChunkCache& cc, int k) { return cc.kinds[k]; }
  __device__ static int nterms(const HistSet& hs) { return hs.nterms; }
  __device__ static constexpr int phi(int k) { return k; }
};
template <>
struct ShapeT<kShapeTF1> {
  static constexpr int NT = 1, G = 8, NTF = 1;
  static constexpr bool AMP = true;
  __device__ static constexpr int kind(const ChunkCache&, int) { return kTermTF; }
  __device__ static constexpr int nterms(const HistSet&) { return 1; }
  __device__ static constexpr int phi(int k) { return k; }
};
template <>
struct ShapeT<kShapeTF2> {
  static constexpr int NT = 2, G = 8, NTF = 2;
  static constexpr bool AMP = true;
  __device__ static constexpr int kind(const ChunkCache&, int) { return kTermTF; }
  __device__ static constexpr int nterms(const HistSet&) { return 2; }
  __device__ static constexpr int phi(int k) { return k; }
};
template <>
struct ShapeT<kShapeTF2c> {
  static constexpr int NT = 2, G = 8, NTF = 1;
  static constexpr bool AMP = false;
  __device__ static constexpr int kind(const ChunkCache&, int) { return kTermTF; }
  __device__ static constexpr int nterms(const HistSet&) { return 2; }
  __device__ static constexpr int phi(int) { return 0; }  // one phase slot for both cosines
};
template <>
struct ShapeT<kShapeKT1> {
  static constexpr int NT = 1, G = 8, NTF = 0;
  static constexpr bool AMP = true;
  __device__ static constexpr int kind(const ChunkCache&, int) { return kTermKT; }
  __device__ static constexpr int nterms(const HistSet&) { return 1; }
  __device__ static constexpr int phi(int) { return 0; }
};
template <>
struct ShapeT<kShapeTF2KT1> {
  static constexpr int NT = 3, G = 4, NTF = 2;
  static constexpr bool AMP = true;
  __device__ static constexpr int kind(const ChunkCache&, int k) { return k < 2 ? kTermTF : kTermKT; }
  __device__ static constexpr int nterms(const HistSet&) { return 3; }
  __device__ static constexpr int phi(int k) { return k; }
};
template <>
struct ShapeT<kShapeTF2KT1c> {
  static constexpr int NT = 3, G = 8, NTF = 1;
  static constexpr bool AMP = false;
  __device__ static constexpr int kind(const ChunkCache&, int k) { return k < 2 ? kTermTF : kTermKT; }
  __device__ static constexpr int nterms(const HistSet&) { return 3; }
  __device__ static constexpr int phi(int) { return 0; }  // one phase slot for both cosines
};
template <int S>
struct ShapeChan {
  // per histogram: N0, bkg, [amp of each term], phase of each cosine term
  static constexpr int AMP0 = 2;
  static constexpr int PHI0 = 2 + (ShapeT<S>::AMP ? ShapeT<S>::NT : 0);
  static constexpr int NPH = PHI0 + ShapeT<S>::NTF;
  static constexpr int NSH = 4 * ShapeT<S>::NT;  // shared per term: Lambda, S, nu, Delta
  static constexpr int N = ShapeT<S>::G * NPH + NSH;
  static_assert(N <= kMaxChan, "channel count");
};

template <int SHAPE, int MODE, bool GRAD>
__device__ void split_item(const Job& job, const HistSet& hs, int item, Smem& sm, uint32_t& parity) {
  using Sh = ShapeT<SHAPE>;
  constexpr int NT = Sh::NT;
  constexpr int G = Sh::G;
  constexpr int NPH = ShapeChan<SHAPE>::NPH;
  constexpr int PHI0 = ShapeChan<SHAPE>::PHI0;
  constexpr int NCH = ShapeChan<SHAPE>::N;
  constexpr int BPT = kBinsPerThread;  // consecutive bins per thread per iteration
  static_assert(BPT == 2, "the loads below read float2 / double2");

  const ChunkCache& cc = sm.cc;
  const int tid = threadIdx.x;
  const int nh = cc.nh, nlo = cc.nlo, nhi = cc.nhi, ts = sm.ts.tile_start;
  const int nterms = Sh::nterms(hs);
  const float aE = cc.aE, tbase = sm.ts.tbase, dtf = cc.dt;
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

  constexpr int CHUNK_BINS = kBlock * BPT;  // bins of one CTA iteration
  // Iterations of this tile that hold any bin of the fit range (the same for every thread).
  const int iters = min(hs.tile_bins / CHUNK_BINS, (nhi - ts + CHUNK_BINS - 1) / CHUNK_BINS);
  // FP32 counts are staged into shared memory one iteration ahead by TMA bulk copies.
  const bool staged = store == kStoreF32;
  const int64_t stride = hs.stride;
  auto issue = [&](int itn, int b) {  // one thread: the rows of iteration itn into buffer b
    const int64_t nstart = ts + static_cast<int64_t>(itn) * CHUNK_BINS;
    const int64_t avail = stride - nstart;  // > 0: nstart < nhi <= stride
    const unsigned bytes = static_cast<unsigned>((avail < CHUNK_BINS ? avail : CHUNK_BINS) * sizeof(float));
    mbar_expect_tx(&sm.bar[b], bytes * nh);
    for (int hl = 0; hl < nh; ++hl)
      tma_load_1d(&sm.stage[b][hl][0], static_cast<const float*>(cc.rowp[hl]) + nstart, bytes, &sm.bar[b]);
  };
  int stall = 0;
  if (staged && tid == 0 && iters > 0) issue(0, 0);
  // The bin offset in the tile is carried as an exact float (integers < 2^24): an
  // int-to-float conversion per bin would occupy this GPU's slow FP64/conversion pipe.
  float fm0 = static_cast<float>(tid * BPT);
  for (int it = 0; it < iters; ++it, fm0 += static_cast<float>(CHUNK_BINS)) {
    const int m0 = it * CHUNK_BINS + tid * BPT;  // offset in the tile (< 2^14)
    const int n0 = ts + m0;
    const int b = it & 1;
    if (staged) {
      if (it + 1 < iters) {
        __syncthreads();  // every thread is done with buffer b ^ 1 (iteration it - 1)
        if (tid == 0) issue(it + 1, b ^ 1);
      }
      if (!mbar_wait(&sm.bar[b], (parity >> b) & 1u)) stall = 1;
      parity ^= 1u << b;
    }
    float t[BPT];
    bool valid[BPT];
#pragma unroll
    for (int j = 0; j < BPT; ++j) {
      t[j] = fmaf(fm0 + static_cast<float>(j), dtf, tbase);
      valid[j] = (n0 + j >= nlo) && (n0 + j < nhi);
    }
    // Time-only factors of the chunk: E = exp(-t/tau), EXK_k = E X_k K_k, and the
    // precession (cos, sin) of each TF term without the per-histogram phase.
    float E[BPT], EXK[NT][BPT], cs[NT][BPT], sn[NT][BPT], dk[NT][BPT];
#pragma unroll
    for (int j = 0; j < BPT; ++j) E[j] = ex2a(-aE * t[j]);
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const int kk = Sh::kind(cc, k);
#pragma unroll
      for (int j = 0; j < BPT; ++j) EXK[k][j] = cs[k][j] = sn[k][j] = dk[k][j] = 0.0f;
      if (k >= nterms) continue;
      const float ca = cc.ca[k], cb = cc.cb[k];
#pragma unroll
      for (int j = 0; j < BPT; ++j) {
        const float ex = ex2a(-fmaf(cb, t[j], ca) * t[j]);
        EXK[k][j] = ex;
        cs[k][j] = 1.0f;
        if (kk == kTermKT) {
          const float tt = t[j] * t[j];
          const float g = ex2a(-cc.dh[k] * tt);
          const float u = cc.d2[k] * tt;
          EXK[k][j] = ex * fmaf((2.0f / 3.0f) * (1.0f - u), g, 1.0f / 3.0f);
          dk[k][j] = ex * tt * g * (u - 3.0f);
        }
      }
      if (kk == kTermTF) {
        // Phase (turns) of the thread's first bin: base + m0 * step, reduced exactly.
        float f = fm0 * cc.shi[k];
        f = __fsub_rn(f, rint_small(f));
        float r = fmaf(fm0, cc.slo[k], sm.ts.base[k]) + f;
        r = __fsub_rn(r, rint_small(r));
#pragma unroll
        for (int j = 0; j < BPT; ++j) {
          float rj = fmaf(static_cast<float>(j), cc.sstep[k], r);
          rj = __fsub_rn(rj, rint_small(rj));  // |rj| <= 1/2: sin/cos arguments in [-pi, pi]
          const float a = rj * kTwoPiF;
          cs[k][j] = cosa(a);
          sn[k][j] = sina(a);
        }
      }
    }
    float U[NT][BPT], V[NT][BPT];
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
      for (int j = 0; j < BPT; ++j) U[k][j] = V[k][j] = 0.0f;
    float vit = 0.0f;  // this iteration's cost terms (at most 2 G of them)

#pragma unroll
    for (int hl = 0; hl < G; ++hl) {
      if (hl >= nh) break;
      float d[BPT];
      if (staged) {
        const float2 q = *reinterpret_cast<const float2*>(&sm.stage[b][hl][tid * BPT]);
        d[0] = q.x;
        d[1] = q.y;
      } else {
        const double2 q = __ldg(reinterpret_cast<const double2*>(static_cast<const double*>(cc.rowp[hl]) + n0));
        d[0] = static_cast<float>(q.x);
        d[1] = static_cast<float>(q.y);
      }
      const float N0 = cc.n0[hl], Nb = cc.bkg[hl];
#pragma unroll
      for (int j = 0; j < BPT; ++j) {
        float C[NT], Sn[NT], Q[NT];
        float M = E[j];
#pragma unroll
        for (int k = 0; k < NT; ++k) {
          C[k] = Sn[k] = Q[k] = 0.0f;
          if (k >= nterms) continue;
          if (Sh::kind(cc, k) == kTermTF) {
            const float cp = cc.cph[k][hl], sp = cc.sph[k][hl];
            C[k] = fmaf(cs[k][j], cp, -sn[k][j] * sp);  // cos(theta + phi)
            Sn[k] = fmaf(sn[k][j], cp, cs[k][j] * sp);  // sin(theta + phi)
          } else {
            C[k] = 1.0f;
          }
          Q[k] = EXK[k][j] * C[k];
          M = fmaf(cc.amp[k][hl], Q[k], M);
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
          const float r = N - dd;
          if (dd > 0.0f) {
            if (N <= 0.0f) {
              bad |= valid[j] ? 1 : 0;
              v = 0.0f;
              w = 0.0f;
            } else {
              // Half deviance (N - d) - d ln(N/d) with z = (N - d)/(N + d): since
              // ln(N/d) = 2 atanh(z), it equals z ((N - d) - 2 d z^2 (1/3 + z^2/5 + ...)),
              // summed to z^10 for |z| < 0.1 (relative truncation < 1e-12); beyond that the
              // logarithms are taken directly, where no cancellation is left.
              const float z = r * rcpa(N + dd);
              if (fabsf(z) < 0.1f) {
                const float z2 = z * z;
                float pz = fmaf(z2, 1.0f / 11.0f, 1.0f / 9.0f);
                pz = fmaf(z2, pz, 1.0f / 7.0f);
                pz = fmaf(z2, pz, 1.0f / 5.0f);
                pz = fmaf(z2, pz, 1.0f / 3.0f);
                v = z * fmaf(-2.0f * dd * z2, pz, r);
              } else {
                v = fmaf(-dd * kLn2F, lg2a(N) - lg2a(dd), r);
              }
              w = r * rcpa(N);
            }
          } else {
            v = r;
            w = 1.0f;
          }
        }
        if (!valid[j]) {
          v = 0.0f;
          w = 0.0f;
        }
        vit += v;
        if (GRAD) {
          ph[hl][0] = fmaf(w, M, ph[hl][0]);
          ph[hl][1] += w;
          const float wN0 = w * N0;
#pragma unroll
          for (int k = 0; k < NT; ++k) {
            if (k >= nterms) continue;
            if (Sh::AMP) ph[hl][2 + k] = fmaf(w, Q[k], ph[hl][2 + k]);
            const float P = wN0 * cc.amp[k][hl];
            U[k][j] = fmaf(P, C[k], U[k][j]);
            if (Sh::kind(cc, k) == kTermTF) {
              const int pc = PHI0 + Sh::phi(k);
              const float PS = P * Sn[k];
              ph[hl][pc] = fmaf(PS, EXK[k][j], ph[hl][pc]);  // w N0 a sin(theta + phi) E X
              V[k][j] += PS;
            }
          }
        }
      }
    }
    {  // Kahan-compensated running sum of the per-iteration partials
      const float y = vit - acc_c;
      const float tsum = acc_v + y;
      acc_c = (tsum - acc_v) - y;
      acc_v = tsum;
    }
    if (GRAD) {
      // Shared channels: time-only factor times the chunk's per-bin sums.
#pragma unroll
      for (int k = 0; k < NT; ++k) {
        if (k >= nterms) continue;
        const int kk = Sh::kind(cc, k);
#pragma unroll
        for (int j = 0; j < BPT; ++j) {
          const float ue = U[k][j] * EXK[k][j];
          sh[k][0] = fmaf(-t[j], ue, sh[k][0]);               // d/dLambda
          sh[k][1] = fmaf(-0.5f * t[j] * t[j], ue, sh[k][1]);  // d/dS
          if (kk == kTermTF) sh[k][2] = fmaf(-kTwoPiF * t[j] * EXK[k][j], V[k][j], sh[k][2]);
          if (kk == kTermKT) sh[k][3] = fmaf(U[k][j], dk[k][j], sh[k][3]);
        }
      }
    }
  }

  // ---- thread (FP32) -> warp (FP32; the value as float-float) -> CTA (FP64 trees) -> row.
  bad = __syncthreads_or(bad);
  stall = __syncthreads_or(stall);
  const int w = tid >> 5, lane = tid & 31;
  float vh = acc_v, vl = -acc_c;
  warp_sum_ff(vh, vl);
  if (lane == 0) {
    sm.vred[w][0] = vh;
    sm.vred[w][1] = vl;
  }
  if (GRAD) {
#pragma unroll
    for (int hl = 0; hl < G; ++hl)
#pragma unroll
      for (int q = 0; q < NPH; ++q) {
        const float r = warp_sum_f(ph[hl][q]);
        if (lane == 0) sm.cred[w][hl * NPH + q] = r;
      }
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float r = warp_sum_f(sh[k][q]);
        if (lane == 0) sm.cred[w][G * NPH + k * 4 + q] = r;
      }
  }
  __syncthreads();
  static_assert(kWarps == 8, "the FP64 trees below sum 8 warps");
  double* row = job.partials + static_cast<int64_t>(item) * hs.pstride;
  if (GRAD && tid < NCH) {
    double a[kWarps];
#pragma unroll
    for (int i = 0; i < kWarps; ++i) a[i] = static_cast<double>(sm.cred[i][tid]);
    row[1 + tid] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  }
  if (tid >= kBlock - 32) {  // the last warp: one lane per warp's float-float value, FP64 tree
    static_assert(NCH <= kBlock - 32, "value warp overlaps a channel thread");
    const int l = tid - (kBlock - 32);
    double a = l < kWarps ? static_cast<double>(sm.vred[l][0]) + static_cast<double>(sm.vred[l][1]) : 0.0;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    // +inf: undefined likelihood; NaN: a staging wait ran out (the host reports a timeout)
    if (l == 0)
      row[0] = stall ? __longlong_as_double(0x7ff8000000000000LL)
                     : (bad ? __longlong_as_double(0x7ff0000000000000LL) : a * (MODE == 1 ? 2.0 : 1.0));
  }
}

// SPLIT channels -> derivative of local slot s of chunk histogram hl.
template <int SHAPE>
__device__ double split_slot(const HistSet& hs, const ChunkCache& cc, const double* tot, int hl, int s) {
  constexpr int NT = ShapeT<SHAPE>::NT;
  constexpr int G = ShapeT<SHAPE>::G;
  constexpr int NPH = ShapeChan<SHAPE>::NPH;
  constexpr int PHI0 = ShapeChan<SHAPE>::PHI0;
  const double* ch = tot + 1;
  const double N0 = cc.loc[hl][0];
  double g = 0.0;
  for (int e = 0; e < hs.ncontrib; ++e) {
    const Contrib c = hs.contrib[e];
    if (c.slot != s) continue;
    const int k = c.term;
    switch (c.kind) {
      case kCN0:
        g += 2.0 * ch[hl * NPH + 0];
        break;
      case kCBkg:
        g += 2.0 * ch[hl * NPH + 1];
        break;
      case kCAmp:
        if (ShapeT<SHAPE>::AMP) g += 2.0 * N0 * ch[hl * NPH + 2 + k];
        break;
      case kCPhi:  // the channel already holds w N0 a sin(theta + phi) E X
        g += 2.0 * (-kTwoPi / 360.0) * ch[hl * NPH + PHI0 + ShapeT<SHAPE>::phi(k)];
        break;
      case kCLam:
        if (hl == 0) g += 2.0 * ch[G * NPH + k * 4 + 0];
        break;
      case kCSig:
        if (hl == 0) g += 4.0 * cc.loc[0][s] * ch[G * NPH + k * 4 + 1];
        break;
      case kCNu:
        if (hl == 0) g += 2.0 * ch[G * NPH + k * 4 + 2];
        break;
      case kCDel:
        if (hl == 0) g += (4.0 / 3.0) * cc.loc[0][s] * ch[G * NPH + k * 4 + 3];
        break;
      default:
        break;
    }
  }
  return g;
}

// ---------------------------------------------------------------------------------------------
// Completion: chunk finalize, then job finalize.
// ---------------------------------------------------------------------------------------------
template <int PREC, int SHAPE, bool GRAD>
__device__ void chunk_finalize(const Job& job, const HistSet& hs, Smem& sm) {
  const ChunkCache& cc = sm.cc;
  const int tid = threadIdx.x;
  const int ps = hs.pstride;
  const int nout = GRAD ? 1 + hs.nch : 1;
  const double* part = job.partials + static_cast<int64_t>(cc.item0) * ps;
  for (int c = tid; c < nout; c += kBlock) {
    double s = 0.0;
    for (int t = 0; t < cc.ntiles; ++t) s += __ldcg(part + static_cast<int64_t>(t) * ps + c);
    sm.tot[c] = s;
  }
  __syncthreads();
  if (GRAD) {
    const int nsl = hs.nslots;
    for (int i = tid; i < cc.nh * nsl; i += kBlock) {
      const int hl = i / nsl, s = i - hl * nsl;
      double g;
      if (PREC == 0)
        g = fp64_slot(hs, sm.tot, s);
      else
        g = split_slot<SHAPE>(hs, cc, sm.tot, hl, s);
      job.colsum[cc.col0 + i] = g;
    }
  }
  if (tid == 0) {
    job.chunk_val[cc.chunk] = sm.tot[0];
    job.chunk_count[cc.chunk] = 0u;
  }
}

__device__ void job_finalize(const Job& job, const HistSet& hs, Smem& sm) {
  const int tid = threadIdx.x;
  double v = 0.0;
  for (int c = tid; c < hs.nchunks; c += kBlock) v += __ldcg(job.chunk_val + c);
  v = warp_sum_d(v);
  if ((tid & 31) == 0) sm.wsum[tid >> 5] = v;
  __syncthreads();
  double value = 0.0;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) value += sm.wsum[i];
  const bool finite = isfinite(value);
  if (job.grad) {
    for (int p = tid; p < hs.P; p += kBlock) {
      double g = 0.0;
      for (int j = hs.p_ptr[p]; j < hs.p_ptr[p + 1]; ++j) g += __ldcg(job.colsum + hs.p_cols[j]);
      job.out[1 + p] = finite ? g : 0.0;
    }
  }
  if (tid == 0) {
    job.out[0] = value;
    *job.counter = 0u;
  }
}

template <int PREC, int SHAPE, bool GRAD>
__device__ void complete_item(const Job& job, const HistSet& hs, Smem& sm) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(job.chunk_count + sm.cc.chunk, 1u);
    sm.flag = prev == static_cast<unsigned>(sm.cc.ntiles - 1);
  }
  __syncthreads();
  if (!sm.flag) return;
  __threadfence();
  chunk_finalize<PREC, SHAPE, GRAD>(job, hs, sm);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(job.counter, 1u);
    sm.flag = prev == static_cast<unsigned>(hs.nchunks - 1);
  }
  __syncthreads();
  if (!sm.flag) return;
  __threadfence();
  job_finalize(job, hs, sm);
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// Persistent kernel: each CTA takes a contiguous range of the launch's items.
// ---------------------------------------------------------------------------------------------
template <int PREC, int SHAPE, int MODE, bool GRAD>
__global__ void __launch_bounds__(kBlock, PREC == 1 ? 2 : 1) eval_kernel(const Job* __restrict__ jobs, int njobs,
                                                      int total_items) {
  __shared__ Smem sm;
  const int per = (total_items + gridDim.x - 1) / gridDim.x;
  const int beg = blockIdx.x * per;
  const int end = min(total_items, beg + per);
  if (threadIdx.x == 0) {
    sm.cc.job = -1;
    sm.cc.chunk = -1;
    if (PREC == 1) {
      mbar_init(&sm.bar[0], 1);
      mbar_init(&sm.bar[1], 1);
      mbar_init_fence();
    }
  }
  __syncthreads();
  uint32_t parity = 0;  // phase parity of each staging barrier (bit b: buffer b)
  int ji = -1;
  Job job;
  for (int gi = beg; gi < end; ++gi) {
    if (ji < 0 || gi >= job.item_begin + job.hs->nitems) {
      int lo = 0, hi = njobs - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].item_begin <= gi)
          lo = mid;
        else
          hi = mid - 1;
      }
      ji = lo;
      job = jobs[ji];
    }
    const HistSet& hs = *job.hs;
    const int item = gi - job.item_begin;
    if (sm.cc.job != ji || item < sm.cc.item0 || item >= sm.cc.item0 + sm.cc.ntiles) {
      __syncthreads();
      load_chunk(job, hs, ji, hs.items[item].x, PREC, sm);
    }
    load_tile(hs, item - sm.cc.item0, PREC, sm);
    if (PREC == 0)
      fp64_item<MODE, GRAD>(job, hs, item, sm);
    else
      split_item<SHAPE, MODE, GRAD>(job, hs, item, sm, parity);
    complete_item<PREC, SHAPE, GRAD>(job, hs, sm);
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
    case kShapeTF2c:
      return ShapeT<kShapeTF2c>::G;
    case kShapeTF2KT1c:
      return ShapeT<kShapeTF2KT1c>::G;
    default:
      return ShapeT<kShapeGeneric>::G;
  }
}

int shape_channels(int shape) {
  switch (shape) {
    case kShapeTF1:
      return ShapeChan<kShapeTF1>::N;
    case kShapeTF2:
      return ShapeChan<kShapeTF2>::N;
    case kShapeKT1:
      return ShapeChan<kShapeKT1>::N;
    case kShapeTF2KT1:
      return ShapeChan<kShapeTF2KT1>::N;
    case kShapeTF2c:
      return ShapeChan<kShapeTF2c>::N;
    case kShapeTF2KT1c:
      return ShapeChan<kShapeTF2KT1c>::N;
    default:
      return ShapeChan<kShapeGeneric>::N;
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
    case kShapeTF2c:
      return dispatch_mode<1, kShapeTF2c>(mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
    case kShapeTF2KT1c:
      return dispatch_mode<1, kShapeTF2KT1c>(mode, grad, d_jobs, njobs, total_items, num_sms, s, info);
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
    case kShapeTF2c:
      return occupancy_mode<1, kShapeTF2c>(mode, grad);
    case kShapeTF2KT1c:
      return occupancy_mode<1, kShapeTF2KT1c>(mode, grad);
    default:
      return occupancy_mode<1, kShapeGeneric>(mode, grad);
  }
}

}  // namespace musr
