// musr_kernels.cuh -- evaluation kernels of libmusr (sm_103a): the device code, included
// by the translation units that instantiate it (musr_kernels_*.cu, grouped by precision
// and shape so that they compile in parallel) and by the dispatch (musr_kernels.cu).
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
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "musr_dev.h"

namespace musr {
namespace kern {
namespace {  // every translation unit gets its own copy

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kLn2F = 0.69314718055994530942f;
constexpr float kLog2eF = 1.44269504088896340736f;
constexpr int kMaxChan = 96;
constexpr int kGamStride = 12;  // floats per histogram row of SPLIT coefficients (M <= 9, plus Nbkg)

// ---------------------------------------------------------------------------------------------
// The half Poisson deviance of a bin, (N - d) + d ln(d/N) = N phi(u) with u = (N - d)/N and
// phi(u) = u + (1 - u) ln(1 - u) = sum_{k>=2} u^k / (k (k - 1)), is taken from a polynomial
// for |u| < 0.2 (no cancellation) and from the logarithm otherwise.  phi_u2(u) = phi(u) / u^2 is
// the degree-6 polynomial through phi(u)/u^2 at the 7 Chebyshev nodes of [-0.2, 0.2], power
// coefficients (lowest first) rounded to FP32: relative error at most 1.3e-8 on the interval,
// below FP32's unit roundoff (the truncated series needs degree 8 for the same accuracy).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float phi_u2(float u) {
  float p = fmaf(u, 1.871784963e-02f, 2.473613620e-02f);
  p = fmaf(u, p, 3.331322595e-02f);
  p = fmaf(u, p, 4.998297244e-02f);
  p = fmaf(u, p, 8.333347738e-02f);
  p = fmaf(u, p, 1.666667461e-01f);
  return fmaf(u, p, 5.000000000e-01f);
}
// The same polynomial on two bins at once (packed FP32x2, the same rounding per component).
__device__ __forceinline__ float2 phi_u2(float2 u) {
  float2 p = __ffma2_rn(u, make_float2(1.871784963e-02f, 1.871784963e-02f),
                        make_float2(2.473613620e-02f, 2.473613620e-02f));
  p = __ffma2_rn(u, p, make_float2(3.331322595e-02f, 3.331322595e-02f));
  p = __ffma2_rn(u, p, make_float2(4.998297244e-02f, 4.998297244e-02f));
  p = __ffma2_rn(u, p, make_float2(8.333347738e-02f, 8.333347738e-02f));
  p = __ffma2_rn(u, p, make_float2(1.666667461e-01f, 1.666667461e-01f));
  return __ffma2_rn(u, p, make_float2(5.000000000e-01f, 5.000000000e-01f));
}

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
// Shared-memory addresses, asynchronous copies, atomics (documented PTX ISA).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Per-thread asynchronous copy global -> shared (cp.async, documented PTX ISA): 16 bytes
// through the L2 only (.cg), both addresses 16-byte aligned, zero-filled beyond src_bytes;
// completion tracked per thread in commit groups.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, unsigned src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)),
               "l"(__cvta_generic_to_global(src)), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Counter increment with acquire-release semantics at GPU scope (PTX atom.acq_rel).
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

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

// Dynamic Kubo-Toyabe relaxation of one (Delta, nu) source at time t from its table (header
// {h, 1/h, K}, then G, dG/dDelta, dG/dnu on the grid k h): the cubic through the four nearest
// grid points; 1 with zero derivatives for t <= 0 (the relaxation starts at time zero).
__device__ __forceinline__ double dkt_floor(double x) { return floor(x); }
__device__ __forceinline__ float dkt_floor(float x) { return floorf(x); }
template <class T>
__device__ __forceinline__ void dkt_lookup(const T* tab, T t, T* G, T* dD, T* dN) {
  if (!(t > T(0))) {
    *G = T(1);
    *dD = *dN = T(0);
    return;
  }
  int K = static_cast<int>(tab[2]);  // written by the table kernel earlier on the stream
  K = K < 4 ? 4 : (K > kDktMaxK ? kDktMaxK : K);
  const T x = t * tab[1];
  int i = x < T(K) ? static_cast<int>(dkt_floor(x)) - 1 : K - 3;
  i = i < 0 ? 0 : (i > K - 3 ? K - 3 : i);
  const T u = x - static_cast<T>(i);
  const T u1 = u - T(1), u2 = u - T(2), u3 = u - T(3);
  const T w0 = -u1 * u2 * u3 * (T(1) / T(6)), w1 = u * u2 * u3 * T(0.5), w2 = -u * u1 * u3 * T(0.5),
          w3 = u * u1 * u2 * (T(1) / T(6));
  const T* g = tab + kDktHeader + i;
  *G = fma(w0, g[0], fma(w1, g[1], fma(w2, g[2], w3 * g[3])));
  g += kDktMaxK + 1;
  *dD = fma(w0, g[0], fma(w1, g[1], fma(w2, g[2], w3 * g[3])));
  g += kDktMaxK + 1;
  *dN = fma(w0, g[0], fma(w1, g[1], fma(w2, g[2], w3 * g[3])));
}

// Checks of the checking build: true when cond holds; otherwise the check's bit goes into
// the error word w (when there is one) and the caller skips the access.  Always true in the
// release build (the checks compile away).
__device__ __forceinline__ bool dbg_ok(unsigned* w, bool cond, unsigned code) {
#ifdef MUSR_DEBUG_CHECKS
  if (!cond && w) atomicOr(w, code);
  return cond;
#else
  (void)w;
  (void)cond;
  (void)code;
  return true;
#endif
}

// Local value of slot s of histogram h.
__device__ __forceinline__ double slot_value(const HistSet& hs, const double* x, int h, int s,
                                             unsigned* dbg = nullptr) {
  const int m = hs.map[static_cast<int64_t>(h) * hs.nslots + s];
  if (!dbg_ok(dbg, m >= 0 ? m < hs.P : -1 - m < hs.nconsts, kDbgMap)) return 0.0;
  return m >= 0 ? x[m] : hs.consts[-1 - m];
}

// ---------------------------------------------------------------------------------------------
// Shared memory
// ---------------------------------------------------------------------------------------------

// One evaluation's constants of the SPLIT basis kernels on one chunk and tile: what the
// per-bin loop reads (kept in the chunk cache).
struct VecConst {
  // [Nbkg, Gam_0 .. Gam_{M-1}] of each histogram (16-byte rows: vector loads)
  alignas(16) float gam[kGroupMax][kGamStride];
  int kinds[kMaxTerms];
  float ca[kMaxTerms], cb[kMaxTerms];  // E*X_k = ex2(-(ca t + cb t^2))  (ca includes 1/tau)
  float dh[kMaxTerms], d2[kMaxTerms];  // KT: g = ex2(-dh t^2), u = d2 t^2
  float shi[kMaxTerms], slo[kMaxTerms], sstep[kMaxTerms];
  float bamp[kMaxTerms];               // amplitude carried by the basis (merged shapes), else 1
  float base[kMaxTerms];               // phase (turns, in [-1/2, 1/2]) of each TF term at the tile's first bin
  int dkt_src[kMaxTerms];              // dynamic Kubo-Toyabe term: its table in the evaluation's set
  float tbase;                         // time of the tile's first bin
  float aE, dt;
};

// Chunk-level constants, cached while a CTA stays on one chunk of one job.
struct ChunkCache {
  int job, chunk;  // cache key (-1: empty)
  int nh, nlo, nhi, tile0, item0, ntiles, col0, first;
  double t0;
  int row[kGroupMax];
  const void* rowp[kGroupMax];       // first count of each histogram's row
  const void* roww[kGroupMax];       // first chi^2 weight of the row (asymmetry data), else nullptr
  double loc[kGroupMax][kMaxSlots];  // local slot values (FP64)
  double ldir[kGroupMax][kMaxSlots]; // local slot components of a Gauss-Newton direction (else 0)
  double cph[kGroupMax][kMaxTerms], sph[kGroupMax][kMaxTerms];  // cos, sin of each cosine term's phase
  // SPLIT Gauss-Newton products: [v_Nbkg, dGam_0 .. dGam_{M-1}] along the direction v, and per
  // term the directional derivatives of its exponent rates (-t dLambda - t^2 dSigma), of its
  // frequency and (scaled by 2/3 Delta) of its Kubo-Toyabe width
  alignas(16) float gdot[kGroupMax][kGamStride];
  // term lists without a basis form (list_item), per (term k, primitive m) = k * kMaxPrims + m:
  // the phase step per bin of a cosine or Bessel primitive in turns, split so that
  // (bin offset < 2^15) * lhi is exact in FP32
  float lhi[kMaxTerms * kMaxPrims], llo[kMaxTerms * kMaxPrims], lstep[kMaxTerms * kMaxPrims];
  float dlam[kMaxTerms], dsig[kMaxTerms], dnu[kMaxTerms], ddel[kMaxTerms];
  double nu[kMaxTerms];
  VecConst v;  // the SPLIT basis kernels' constants of this job
};

struct TileState {
  int tile_start;
  // term lists without a basis form: the tile's first bin time, and per (term, primitive) the
  // cosine's phase at the tile's first bin (turns, in [-1/2, 1/2]) or the Bessel argument there
  // (radians)
  float tbase;
  float lbase[kMaxTerms * kMaxPrims];
};

struct Smem {
  // SPLIT, FP32 counts: the rows of the current and the next CTA iteration, each thread's two
  // bins of every histogram copied by that thread (cp.async)
  alignas(128) float stage[2][kGroupMax][kBlock * kBinsPerThread];
  __device__ float* stage_slot(int b, int hl, int bin) { return &stage[b][hl][bin]; }
  ChunkCache cc;
  TileState ts;
  float dkn[kMaxTerms][kBinsPerThread][kBlock];  // d/dnu factors of dynamic Kubo-Toyabe terms, per thread
  float cred[kWarps][kMaxChan];  // per-warp FP32 channel sums
  float vred[kWarps][2];         // per-warp float-float value
  double dred[kWarps][kFp64Channels + 2];
  double tot[kMaxChan + 1];      // chunk totals in the chunk finalize
  double wsum[kWarps];
  int flag;
  int bad;
};

// ---------------------------------------------------------------------------------------------
// SPLIT shapes (basis form, see musr_dev.h): NT terms, the first NTF with a cosine (NTF < 0:
// kinds known at run time only, every term owning two basis functions), M basis functions,
// at most G histograms per chunk; MERGED: the amplitudes live in the basis, one phase per
// histogram.  Per work item each histogram keeps NPH = M + 1 channels (G_m = sum u B_m, and
// W = sum u) and each term 4 shared channels (Lambda, S, nu, Delta).
// ---------------------------------------------------------------------------------------------
template <int NT_, int NTF_, int M_, int G_, bool MERGED_>
struct BasisBase {
  static constexpr int NT = NT_, NTF = NTF_, M = M_, G = G_;
  static constexpr bool MERGED = MERGED_;
  // Whether a term may carry a dynamic Kubo-Toyabe factor: every unmerged shape (the planner
  // does not merge a theory that has one, so the merged kernels carry no code for it).
  static constexpr bool DKT = !MERGED_;
  static constexpr int NPH = M + 1;
  static constexpr int NCH = G * NPH + 4 * NT;
  // Basis function of term k's cosine part (or of the whole term), and of its sine part.
  __host__ __device__ static constexpr int bc(int k) {
    return MERGED ? (k < NTF ? 1 : 0) : (NTF < 0 ? 1 + 2 * k : (k < NTF ? 1 + 2 * k : 1 + 2 * NTF + (k - NTF)));
  }
  __host__ __device__ static constexpr int bs(int k) { return MERGED ? 2 : (2 + 2 * k < M ? 2 + 2 * k : M - 1); }
  // Whether term k has a cosine (compile-time for the fixed shapes).
  __device__ static bool tf(const int* kinds, int k) { return NTF < 0 ? kinds[k] == kTermTF : k < NTF; }
  static_assert(NCH <= kMaxChan, "channel count");
  static_assert(M + 1 <= kGamStride, "coefficient row");
};
template <int S>
struct Basis;
template <>
struct Basis<kShapeGeneric> : BasisBase<4, -1, 9, 2, false> {};
template <>
struct Basis<kShapeT1> : BasisBase<1, 1, 3, 8, false> {};
template <>
struct Basis<kShapeN1> : BasisBase<1, 0, 2, 8, false> {};
template <>
struct Basis<kShapeT1N1> : BasisBase<2, 1, 4, 8, false> {};
template <>
struct Basis<kShapeT2> : BasisBase<2, 2, 5, 8, false> {};
template <>
struct Basis<kShapeT2N1> : BasisBase<3, 2, 6, 6, false> {};
template <>
struct Basis<kShapeT2m> : BasisBase<2, 2, 3, 8, true> {};
template <>
struct Basis<kShapeT2N1m> : BasisBase<3, 2, 3, 8, true> {};
// Term lists without a basis form (list_item): the traits only let the shared setup code
// compile; that code does not run for them.
template <>
struct Basis<kShapeList> : BasisBase<1, 0, 2, 1, false> {};
template <>
struct Basis<kShapeListS> : BasisBase<1, 0, 2, 1, false> {};
__host__ __device__ constexpr bool is_list(int shape) { return shape == kShapeList || shape == kShapeListS; }

// cos and sin of a phase given in degrees: reduced to [-1/2, 1/2] turns in FP64, then
// evaluated in FP32 (the SPLIT coefficients and their derivatives need no more; FP64
// sincospi is slow on this GPU and sits on the latency path of every chunk).
__device__ __forceinline__ void phase_cs(double phi_deg, double* c, double* s) {
  const double x = phi_deg * (1.0 / 360.0);
  float sf, cf;
  sincospif(2.0f * static_cast<float>(x - rint(x)), &sf, &cf);
  *c = cf;
  *s = sf;
}

// Coefficients [Nbkg, Gam_0 .. Gam_{M-1}] of one histogram's basis expansion from its slot
// values slot(s), computed in FP64 and rounded once; cos and sin of each cosine term's phase.
template <int SHAPE, class Slot>
__device__ void coef_row(const HistSet& hs, Slot slot, float* gam, double* cph, double* sph) {
  using Bs = Basis<SHAPE>;
  double g[kGamStride];
#pragma unroll
  for (int i = 0; i < kGamStride; ++i) g[i] = 0.0;
  const double N0 = slot(0);
  g[0] = slot(1);
  g[1] = hs.envelope ? N0 : 0.0;  // the basis function E carries the 1 of (1 + A)
#pragma unroll
  for (int k = 0; k < kMaxTerms; ++k) {
    double c = 1.0, sn = 0.0;
    if (k < hs.nterms && hs.canon[k].kind == kTermTF) phase_cs(slot(hs.canon[k].phi_slot), &c, &sn);
    cph[k] = c;
    sph[k] = sn;
  }
  if (Bs::MERGED) {  // one phase per histogram: that of the first cosine term
    g[2] = N0 * cph[0];
    g[3] = -N0 * sph[0];
  } else {
#pragma unroll
    for (int k = 0; k < Bs::NT; ++k) {
      if (k >= hs.nterms) break;
      const CanonTerm& ct = hs.canon[k];
      const double a = ct.amp_slot >= 0 ? slot(ct.amp_slot) : 1.0;
      if (ct.kind == kTermTF) {
        g[1 + Bs::bc(k)] = N0 * a * cph[k];
        g[1 + Bs::bs(k)] = -N0 * a * sph[k];
      } else {
        g[1 + Bs::bc(k)] = N0 * a;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kGamStride; ++i) gam[i] = static_cast<float>(g[i]);
}

// Constants of term k shared by a chunk's histograms (from the slot values slot(s) of its
// first histogram): its kind, exponent rates, Kubo-Toyabe width and phase step per bin.
// Returns the term's frequency (MHz; 0 without a cosine).
template <class Slot>
__device__ double term_consts(const HistSet& hs, Slot slot, int k, VecConst& v) {
  v.kinds[k] = k < hs.nterms ? hs.canon[k].kind : kTermNone;
  v.ca[k] = v.cb[k] = v.d2[k] = v.dh[k] = v.shi[k] = v.slo[k] = v.sstep[k] = 0.0f;
  v.bamp[k] = 1.0f;
  if (k >= hs.nterms) return 0.0;
  const CanonTerm& ct = hs.canon[k];
  float lam = 0.0f, S = 0.0f;
  for (int i = 0; i < ct.nexp; ++i) lam += static_cast<float>(slot(ct.exp_slot[i]));
  for (int i = 0; i < ct.ngauss; ++i) {
    const float sg = static_cast<float>(slot(ct.gauss_slot[i]));
    S = fmaf(sg, sg, S);
  }
  v.bamp[k] = hs.bamp[k];
  // the term's exponent carries the decay envelope E = exp(-t / tau_mu) (none for the
  // asymmetry model)
  v.ca[k] = kLog2eF * ((hs.envelope ? static_cast<float>(1.0 / kTauMuUs) : 0.0f) + lam);
  v.cb[k] = kLog2eF * 0.5f * S;
  if (ct.kind == kTermKT) {
    const float D = static_cast<float>(slot(ct.kt_slot));
    v.d2[k] = D * D;
    v.dh[k] = kLog2eF * 0.5f * D * D;
  } else if (ct.kind == kTermLKT) {  // g = ex2(-dh t) = exp(-a t), u = d2 t = a t
    const float a = static_cast<float>(slot(ct.kt_slot));
    v.d2[k] = a;
    v.dh[k] = kLog2eF * a;
  }
  if (ct.kind != kTermTF) return 0.0;
  const double nu = slot(ct.nu_slot);
  const double step = nu * hs.dt_us;  // turns per bin (FP64)
  // Exact split: hi keeps 9 significant bits, so (bin offset < 2^15) * hi is exact in FP32.
  const float hi = __uint_as_float(__float_as_uint(static_cast<float>(step)) & 0xFFFF8000u);
  v.shi[k] = hi;
  v.slo[k] = static_cast<float>(step - static_cast<double>(hi));
  v.sstep[k] = static_cast<float>(step);
  return nu;
}

// Phase (turns, reduced to [-1/2, 1/2] in FP64) of a cosine of frequency nu at time t_start.
__device__ __forceinline__ float tile_phase(double nu, double t_start) {
  const double x = nu * t_start;
  return static_cast<float>(x - rint(x));
}

// ---------------------------------------------------------------------------------------------
// Chunk cache fill (only when a CTA moves to another chunk or job).
// ---------------------------------------------------------------------------------------------
template <int SHAPE, class SM>
__device__ void load_chunk(const Job& job, const HistSet& hs, int job_index, int chunk_index, int prec,
                           SM& sm) {
  using Bs = Basis<SHAPE>;
  ChunkCache& cc = sm.cc;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const Chunk ch = hs.chunks[dbg_ok(job.dbg, chunk_index >= 0 && chunk_index < hs.nchunks, kDbgChunk) ? chunk_index : 0];
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
    int h = hs.hist_index[cc.first + hl];
    if (!dbg_ok(job.dbg, h >= 0 && h < hs.H, kDbgHist)) h = 0;
    cc.loc[hl][s] = slot_value(hs, job.params, h, s, job.dbg);
    const int mi = hs.map[static_cast<int64_t>(h) * hs.nslots + s];
    cc.ldir[hl][s] = job.dir && mi >= 0 ? job.dir[mi] : 0.0;
    if (s == 0) {
      cc.row[hl] = h;
      const size_t esz = hs.store == kStoreF64 ? sizeof(double) : sizeof(float);
      cc.rowp[hl] = static_cast<const char*>(hs.counts) + static_cast<size_t>(h) * hs.stride * esz;
      cc.roww[hl] = hs.weights ? static_cast<const char*>(hs.weights) + static_cast<size_t>(h) * hs.stride * esz
                               : nullptr;
    }
  }
  __syncthreads();
  if (prec == 0) return;
  const double dt = hs.dt_us;
  if (tid < nh) {
    const int hl = tid;
    coef_row<SHAPE>(hs, [&](int q) { return cc.loc[hl][q]; }, cc.v.gam[hl], cc.cph[hl], cc.sph[hl]);
    const double N0 = cc.loc[hl][0];
    // Directional derivative of the coefficients along a Gauss-Newton direction (zeros without).
    double gd[kGamStride];
#pragma unroll
    for (int i = 0; i < kGamStride; ++i) gd[i] = 0.0;
    if (job.dir) {
      constexpr double kDeg = kTwoPi / 360.0;
      const double vN0 = cc.ldir[hl][0];
      gd[0] = cc.ldir[hl][1];
      gd[1] = hs.envelope ? vN0 : 0.0;
      if (Bs::MERGED) {
        const double vph = cc.ldir[hl][hs.canon[0].phi_slot] * kDeg;
        const double c = cc.cph[hl][0], sn = cc.sph[hl][0];
        gd[2] = vN0 * c - N0 * sn * vph;
        gd[3] = -vN0 * sn - N0 * c * vph;
      } else {
#pragma unroll
        for (int k = 0; k < Bs::NT; ++k) {
          if (k >= hs.nterms) break;
          const CanonTerm& ct = hs.canon[k];
          const double a = ct.amp_slot >= 0 ? cc.loc[hl][ct.amp_slot] : 1.0;
          const double va = ct.amp_slot >= 0 ? cc.ldir[hl][ct.amp_slot] : 0.0;
          const double dNa = vN0 * a + N0 * va;  // d(N0 a) along v
          if (ct.kind == kTermTF) {
            const double vph = cc.ldir[hl][ct.phi_slot] * kDeg;
            const double c = cc.cph[hl][k], sn = cc.sph[hl][k];
            gd[1 + Bs::bc(k)] = dNa * c - N0 * a * sn * vph;
            gd[1 + Bs::bs(k)] = -dNa * sn - N0 * a * c * vph;
          } else {
            gd[1 + Bs::bc(k)] = dNa;
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kGamStride; ++i) cc.gdot[hl][i] = static_cast<float>(gd[i]);
  } else if (tid >= 32 && tid < 32 + kMaxTerms) {
    const int k = tid - 32;
    cc.nu[k] = term_consts(hs, [&](int q) { return cc.loc[0][q]; }, k, cc.v);
    int src = -1;
    if (k < hs.nterms && hs.canon[k].kind == kTermDKT) {  // the chunk's histograms share (Delta, nu)
      const CanonTerm& ct = hs.canon[k];
      src = hs.dkt_of[(static_cast<int64_t>(cc.row[0]) * kMaxTerms + ct.dkt_term) * kMaxPrims + ct.dkt_prim];
      if (!dbg_ok(job.dbg, src >= 0 && src < hs.ndkt, kDbgDkt)) src = -1;
    }
    cc.v.dkt_src[k] = src;
    if (k < hs.nterms) {  // directional derivatives of the term's shared parameters (Gauss-Newton products)
      const CanonTerm& ct = hs.canon[k];
      double dl = 0.0, ds = 0.0;
      for (int i = 0; i < ct.nexp; ++i) dl += cc.ldir[0][ct.exp_slot[i]];
      for (int i = 0; i < ct.ngauss; ++i) ds += cc.loc[0][ct.gauss_slot[i]] * cc.ldir[0][ct.gauss_slot[i]];
      cc.dlam[k] = static_cast<float>(dl);
      cc.dsig[k] = static_cast<float>(ds);
      cc.dnu[k] = ct.kind == kTermTF || ct.kind == kTermDKT ? static_cast<float>(cc.ldir[0][ct.nu_slot]) : 0.0f;
      cc.ddel[k] = ct.kind == kTermKT
                       ? static_cast<float>((2.0 / 3.0) * cc.loc[0][ct.kt_slot] * cc.ldir[0][ct.kt_slot])
                       : (ct.kind == kTermLKT ? static_cast<float>((2.0 / 3.0) * cc.ldir[0][ct.kt_slot])
                                              : (ct.kind == kTermDKT ? static_cast<float>(cc.ldir[0][ct.kt_slot])
                                                                     : 0.0f));
    }
  } else if (tid == 64) {
    // log2(e) / tau_mu: E = 2^(-aE t); without the decay envelope E = 1
    cc.v.aE = hs.envelope ? static_cast<float>(1.4426950408889634 / kTauMuUs) : 0.0f;
    cc.v.dt = static_cast<float>(dt);
  }
  __syncthreads();
}

// Tile-level constants for a tile (or piece) starting at bin ts: its first bin time and, in
// FP64, each precession phase at that bin reduced to [-1/2, 1/2] turns.
template <class SM>
__device__ void load_tile_at(int ts, const HistSet& hs, int prec, SM& sm) {
  const int tid = threadIdx.x;
  if (tid == 0) sm.ts.tile_start = ts;
  if (prec == 1 && tid >= 32 && tid < 32 + kMaxTerms) {
    const int k = tid - 32;
    const double t_start = (static_cast<double>(ts) - sm.cc.t0) * hs.dt_us;
    if (k == 0) sm.cc.v.tbase = static_cast<float>(t_start);
    sm.cc.v.base[k] = sm.cc.v.kinds[k] == kTermTF ? tile_phase(sm.cc.nu[k], t_start) : 0.0f;
  }
  __syncthreads();
}
template <class SM>
__device__ void load_tile(const HistSet& hs, int tile, int prec, SM& sm) {
  load_tile_at(sm.cc.tile0 + tile * hs.tile_bins, hs, prec, sm);
}

// ---------------------------------------------------------------------------------------------
// FP64 path: one histogram per chunk, every operation in FP64, term list as given.
// Row: [value, N0, Nbkg, d/d(term k, primitive m, slot q)...].
// ---------------------------------------------------------------------------------------------
// MODE 2 and 3: the Gauss-Newton product H v of chi^2 and -2lnL for the direction v of the
// job: per bin N' = J v (the directional derivative of N) and dcost/dN replaced by
// (d^2 cost/dN^2) N', so that the gradient channels accumulate H v; the value is v^T H v.
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
    if (!dbg_ok(job.dbg, n < hs.stride, kDbgRow)) continue;
    const double d = store == kStoreF64 ? rowd[n] : static_cast<double>(rowf[n]);
    const double E = hs.envelope ? exp(-t / kTauMuUs) : 1.0;
    // chi^2 weight: 1 / max(d, 1) for counts (Eq. chisq), given for asymmetry data
    const double iv = hs.weights ? static_cast<const double*>(hs.weights)[static_cast<int64_t>(h) * hs.stride + n]
                                 : 1.0 / fmax(d, 1.0);
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
        } else if (kind == kLKT) {
          const double u = p0 * t;
          const double g = exp(-u);
          f[m] = 1.0 / 3.0 + (2.0 / 3.0) * (1.0 - u) * g;
          df[m][0] = (2.0 / 3.0) * t * g * (u - 2.0);
        } else if (kind == kStrExp) {  // exp(-(|lambda| t)^beta) for t > 0, else 1
          const double p1 = cc.loc[0][hs.raw[k].slot[m][1]];
          const double lam = fabs(p0), x = lam * t;
          if (t > 0.0 && x > 0.0) {
            const double xb = pow(x, p1), e = exp(-xb);
            f[m] = e;
            df[m][0] = (p0 < 0.0 ? -1.0 : 1.0) * (-p1 * xb / lam) * e;
            df[m][1] = -xb * log(x) * e;
          }
        } else if (kind == kBessel) {  // J0(2 pi (nu t + phi / 360)); J0' = -J1
          const double p1 = cc.loc[0][hs.raw[k].slot[m][1]];
          const double x = kTwoPi * (p0 * t + p1 / 360.0);
          f[m] = j0(x);
          const double j1x = j1(x);
          df[m][0] = -j1x * kTwoPi * t;
          df[m][1] = -j1x * kTwoPi / 360.0;
        } else if (kind == kDKT) {  // dynamic Kubo-Toyabe: this evaluation's table of the pair
          const int src = hs.dkt_of[(h * kMaxTerms + k) * kMaxPrims + m];
          if (!dbg_ok(job.dbg, src >= 0 && src < hs.ndkt, kDbgDkt)) continue;
          dkt_lookup(static_cast<const double*>(job.dkt) + static_cast<size_t>(src) * kDktTable, t, &f[m],
                     &df[m][0], &df[m][1]);
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
    const double Ae = hs.envelope ? 1.0 + A : A;  // (1 + A), or A for the asymmetry model
    const double N = N0 * E * Ae + Nbkg;
    double v, W;  // per-bin cost and dcost/dN
    if (MODE == 2 || MODE == 3) {  // Gauss-Newton product: N' = J v, W = (d^2 cost/dN^2) N', v = W N'
      double Nd = E * Ae * cc.ldir[0][0] + cc.ldir[0][1];
#pragma unroll
      for (int k = 0; k < kMaxTerms; ++k) {
        const int np = k < nterms ? hs.raw[k].nprim : 0;
#pragma unroll
        for (int m = 0; m < kMaxPrims; ++m) {
          if (m >= np) continue;
          Nd += N0 * E * gd[k][m][0] * cc.ldir[0][hs.raw[k].slot[m][0]];
          if (prim_nslots(hs.raw[k].kind[m]) == 2) Nd += N0 * E * gd[k][m][1] * cc.ldir[0][hs.raw[k].slot[m][1]];
        }
      }
      double c2;
      if (MODE == 2) {
        c2 = 2.0 * iv;
      } else if (d > 0.0) {
        if (N <= 0.0) bad = 1;
        c2 = N > 0.0 ? 2.0 * d / (N * N) : 0.0;
      } else {
        c2 = 0.0;
      }
      W = c2 * Nd;
      v = W * Nd;
    } else if (MODE == 0) {
      const double r = d - N;
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
      acc_n0 += W * E * Ae;
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
  if (!dbg_ok(job.dbg, item >= 0 && item < job.nrows, kDbgPartial)) return;
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
      if (prim_nslots(hs.raw[k].kind[m]) == 2 && hs.raw[k].slot[m][1] == s) g += tot[3 + (k * kMaxPrims + m) * 2 + 1];
    }
  return g;
}

// Term lists without a basis form: per (term, primitive) with a phase, its step per bin in
// turns (FP64, then split so that (bin offset < 2^15) * lhi is exact in FP32; the Bessel
// step in radians), once per chunk.
__device__ void load_chunk_list(const HistSet& hs, Smem& sm) {
  const int tid = threadIdx.x;
  if (tid < kMaxTerms * kMaxPrims) {
    const int k = tid / kMaxPrims, m = tid - k * kMaxPrims;
    float hi = 0.0f, lo = 0.0f, st = 0.0f;
    if (k < hs.nterms && m < hs.raw[k].nprim &&
        (hs.raw[k].kind[m] == kTFCos || hs.raw[k].kind[m] == kBessel)) {
      const double step = sm.cc.loc[0][hs.raw[k].slot[m][0]] * hs.dt_us;
      hi = __uint_as_float(__float_as_uint(static_cast<float>(step)) & 0xFFFF8000u);
      lo = static_cast<float>(step - static_cast<double>(hi));
      st = static_cast<float>(hs.raw[k].kind[m] == kBessel ? kTwoPi * step : step);
    }
    sm.cc.lhi[tid] = hi;
    sm.cc.llo[tid] = lo;
    sm.cc.lstep[tid] = st;
  }
  __syncthreads();
}

// ... and the phase at the tile's first bin (FP64, then rounded once), and the tile's time.
__device__ void load_tile_list(const HistSet& hs, Smem& sm) {
  const int tid = threadIdx.x;
  const double t_start = (static_cast<double>(sm.ts.tile_start) - sm.cc.t0) * hs.dt_us;
  if (tid == 0) sm.ts.tbase = static_cast<float>(t_start);
  if (tid < kMaxTerms * kMaxPrims) {
    const int k = tid / kMaxPrims, m = tid - k * kMaxPrims;
    float b = 0.0f;
    if (k < hs.nterms && m < hs.raw[k].nprim &&
        (hs.raw[k].kind[m] == kTFCos || hs.raw[k].kind[m] == kBessel)) {
      const double x = fma(sm.cc.loc[0][hs.raw[k].slot[m][0]], t_start,
                           sm.cc.loc[0][hs.raw[k].slot[m][1]] * (1.0 / 360.0));  // turns
      b = static_cast<float>(hs.raw[k].kind[m] == kTFCos ? x - rint(x) : kTwoPi * x);
    }
    sm.ts.lbase[tid] = b;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// SPLIT path for term lists without a basis form (a stretched exponential, a Bessel
// precession, two cosines in one term): the FP64 path's per-bin evaluation of the term list
// in FP32 arithmetic, except the bin time and the phase argument, formed in FP64 (the cosine
// reduced to [-1/2, 1/2] turns there, the Bessel argument rounded once); FP32 sums per
// thread (the value Kahan-compensated), FP64 from the warp on; the row layout of the FP64
// path.  MODE 0 (chi^2), 1 (-2lnL), 4 (weighted chi^2 of asymmetry data).
// ---------------------------------------------------------------------------------------------
template <int MODE, bool GRAD, int LT, int LP>
__device__ void list_item(const Job& job, const HistSet& hs, int item, Smem& sm) {
  const int tid = threadIdx.x;
  const ChunkCache& cc = sm.cc;
  const int h = cc.row[0], nlo = cc.nlo, nhi = cc.nhi, ts = sm.ts.tile_start;
  const double dt = hs.dt_us;
  const int nterms = hs.nterms;
  const float N0 = static_cast<float>(cc.loc[0][0]), Nbkg = static_cast<float>(cc.loc[0][1]);
  const float* rowf = static_cast<const float*>(hs.counts) + static_cast<int64_t>(h) * hs.stride;
  const double* rowd = static_cast<const double*>(hs.counts) + static_cast<int64_t>(h) * hs.stride;
  const float* roww =
      hs.weights ? static_cast<const float*>(hs.weights) + static_cast<int64_t>(h) * hs.stride : nullptr;
  const int store = hs.store;
  const float rate = hs.envelope ? static_cast<float>(1.0 / kTauMuUs) : 0.0f;
  const float tbase = sm.ts.tbase, dtf = static_cast<float>(dt);

  float acc_v = 0.0f, acc_c = 0.0f, acc_n0 = 0.0f, acc_bkg = 0.0f;
  float acc_p[LT][LP][2];  // per (term, primitive, slot) of the first LT terms' first LP primitives
#pragma unroll
  for (int k = 0; k < LT; ++k)
#pragma unroll
    for (int m = 0; m < LP; ++m) acc_p[k][m][0] = acc_p[k][m][1] = 0.0f;
  int bad = 0;

  const int end = min(nhi, ts + hs.tile_bins);
  // The bin offset in the tile is carried as an exact float (< 2^15 here): time and phases
  // come from the tile's FP64 bases plus FP32 increments, with no FP64 work per bin.
  float fm = static_cast<float>(tid);
  for (int n = ts + tid; n < end; n += kBlock, fm += static_cast<float>(kBlock)) {
    if (n < nlo) continue;
    const float tf = fmaf(fm, dtf, tbase);  // Section 4.1: t = n dt, shifted by t0
    if (!dbg_ok(job.dbg, n < hs.stride, kDbgRow)) continue;
    const float d = store == kStoreF64 ? static_cast<float>(rowd[n]) : rowf[n];
    const float E = __expf(-rate * tf);
    float gd[LT][LP][2];
    float A = 0.0f;
#pragma unroll
    for (int k = 0; k < LT; ++k) {
      float f[LP], df[LP][2];
      const int np = k < nterms ? hs.raw[k].nprim : 0;
      float term = 1.0f;
#pragma unroll
      for (int m = 0; m < LP; ++m) {
        f[m] = 1.0f;
        df[m][0] = df[m][1] = 0.0f;
        if (m >= np) continue;
        const int kind = hs.raw[k].kind[m];
        const float p0 = static_cast<float>(cc.loc[0][hs.raw[k].slot[m][0]]);
        if (kind == kAmp) {
          f[m] = p0;
          df[m][0] = 1.0f;
        } else if (kind == kExp) {
          const float e = __expf(-p0 * tf);
          f[m] = e;
          df[m][0] = -tf * e;
        } else if (kind == kGauss) {
          const float x = p0 * tf, e = __expf(-0.5f * x * x);
          f[m] = e;
          df[m][0] = -p0 * tf * tf * e;
        } else if (kind == kKT) {
          const float u = (p0 * tf) * (p0 * tf), g = __expf(-0.5f * u);
          f[m] = 1.0f / 3.0f + (2.0f / 3.0f) * (1.0f - u) * g;
          df[m][0] = (2.0f / 3.0f) * p0 * tf * tf * g * (u - 3.0f);
        } else if (kind == kLKT) {
          const float u = p0 * tf, g = __expf(-u);
          f[m] = 1.0f / 3.0f + (2.0f / 3.0f) * (1.0f - u) * g;
          df[m][0] = (2.0f / 3.0f) * tf * g * (u - 2.0f);
        } else if (kind == kStrExp) {  // exp(-(|lambda| t)^beta) for t > 0, else 1
          const float p1 = static_cast<float>(cc.loc[0][hs.raw[k].slot[m][1]]);
          const float lam = fabsf(p0), x = lam * tf;
          if (tf > 0.0f && x > 0.0f) {
            const float lx = logf(x), xb = __expf(p1 * lx), e = __expf(-xb);
            f[m] = e;
            df[m][0] = (p0 < 0.0f ? -1.0f : 1.0f) * (-p1 * xb / lam) * e;
            df[m][1] = -xb * lx * e;
          }
        } else if (kind == kTFCos) {  // phase: tile base + fm * step, reduced exactly
          const int j = k * kMaxPrims + m;
          float fr = __fmul_rn(fm, cc.lhi[j]);
          fr = __fsub_rn(fr, rint_small(fr));
          float r = __fadd_rn(fmaf(fm, cc.llo[j], sm.ts.lbase[j]), fr);
          r = __fsub_rn(r, rint_small(r));
          float sn, cs;
          sincospif(2.0f * r, &sn, &cs);
          f[m] = cs;
          df[m][0] = -sn * kTwoPiF * tf;
          df[m][1] = -sn * (kTwoPiF / 360.0f);
        } else if (kind == kDKT) {  // dynamic Kubo-Toyabe: this evaluation's FP32 table of the pair
          const int src = hs.dkt_of[(h * kMaxTerms + k) * kMaxPrims + m];
          if (!dbg_ok(job.dbg, src >= 0 && src < hs.ndkt, kDbgDkt)) continue;
          dkt_lookup(static_cast<const float*>(job.dkt) + static_cast<size_t>(src) * kDktTable, tf, &f[m],
                     &df[m][0], &df[m][1]);
        } else if (kind == kBessel) {  // J0' = -J1; the argument (not periodic) in radians
          const int j = k * kMaxPrims + m;
          const float X = fmaf(fm, cc.lstep[j], sm.ts.lbase[j]), j1x = j1f(X);
          f[m] = j0f(X);
          df[m][0] = -j1x * kTwoPiF * tf;
          df[m][1] = -j1x * (kTwoPiF / 360.0f);
        }
        term *= f[m];
      }
      if (np > 0) A += term;
      if (GRAD) {
#pragma unroll
        for (int m = 0; m < LP; ++m) {
          float rest = 1.0f;
#pragma unroll
          for (int q = 0; q < LP; ++q)
            if (q != m) rest *= f[q];
          gd[k][m][0] = df[m][0] * rest;
          gd[k][m][1] = df[m][1] * rest;
        }
      }
    }
    const float Ae = hs.envelope ? 1.0f + A : A;
    const float N = N0 * E * Ae + Nbkg;
    float v, W;  // per-bin cost and dcost/dN
    if (MODE == 0 || MODE == 4) {
      const float w = MODE == 4 ? roww[n] : 1.0f / fmaxf(d, 1.0f);
      const float r = d - N;
      v = r * r * w;
      W = -2.0f * r * w;
    } else if (d > 0.0f) {
      if (!(N > 0.0f)) {
        bad = 1;
        v = W = 0.0f;
      } else {
        // (N - d) + d ln(d/N) = N phi(u), u = (N - d)/N: the polynomial for small |u|
        // (no cancellation), the logarithm otherwise
        const float r = N - d, u = r / N;
        if (fabsf(u) < 0.2f) {
          v = 2.0f * r * u * phi_u2(u);
        } else {
          v = 2.0f * (r + d * logf(d / N));
        }
        W = 2.0f * u;
      }
    } else {
      v = 2.0f * (N - d);
      W = 2.0f;
    }
    {  // Kahan-compensated running sum
      const float y = v - acc_c;
      const float s = acc_v + y;
      acc_c = (s - acc_v) - y;
      acc_v = s;
    }
    if (GRAD) {
      acc_n0 += W * E * Ae;
      acc_bkg += W;
      const float wNE = W * N0 * E;
#pragma unroll
      for (int k = 0; k < LT; ++k)
#pragma unroll
        for (int m = 0; m < LP; ++m) {
          acc_p[k][m][0] = fmaf(wNE, gd[k][m][0], acc_p[k][m][0]);
          acc_p[k][m][1] = fmaf(wNE, gd[k][m][1], acc_p[k][m][1]);
        }
    }
  }

  // Warp (FP64 shuffles), then the CTA's warps in a fixed order (FP64): the FP64 path's rows.
  bad = __syncthreads_or(bad);
  const int w = tid >> 5, lane = tid & 31;
  const double r0 = warp_sum_d(static_cast<double>(acc_v) - static_cast<double>(acc_c));
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
        for (int q = 0; q < 2; ++q) {  // the FP64 path's row layout; slots beyond LT x LP are 0
          const double r = k < LT && m < LP ? warp_sum_d(acc_p[k < LT ? k : 0][m < LP ? m : 0][q]) : 0.0;
          if (lane == 0) sm.dred[w][3 + (k * kMaxPrims + m) * 2 + q] = r;
        }
  }
  __syncthreads();
  if (!dbg_ok(job.dbg, item >= 0 && item < job.nrows, kDbgPartial)) return;
  double* row = job.partials + static_cast<int64_t>(item) * hs.pstride;
  const int nout = GRAD ? 1 + kFp64Channels : 1;
  for (int c = tid; c < nout; c += kBlock) {
    double s = 0.0;
    for (int i = 0; i < kWarps; ++i) s += sm.dred[i][c];
    if (c == 0 && bad) s = __longlong_as_double(0x7ff0000000000000LL);
    row[c] = s;
  }
}

// ---------------------------------------------------------------------------------------------
// SPLIT path (basis form).  Per bin, the time-only parts: E = exp(-t/tau) and, per term,
// the piece P_k = a E X_k [KT] (a: the basis amplitude) with its cosine and sine parts for a
// cosine term.  Per (histogram, bin): N = Nbkg + sum_m Gam_m B_m (M FMAs), the cost term and
// u = d(cost/2)/dN, then the channels G_m += u B_m, W += u and the per-bin sums
// V_m = sum_j u_j Gam_jm that carry the shared time parameters' derivatives.
// ---------------------------------------------------------------------------------------------
// vc: the job's constants on this chunk and tile.
template <int SHAPE, int MODE, bool GRAD>
__device__ void split_item(const Job& job, const HistSet& hs, int item, Smem& sm, const VecConst& vc, int nit = -1) {
  using Bs = Basis<SHAPE>;
  constexpr int NT = Bs::NT;
  constexpr int M = Bs::M;
  constexpr int G = Bs::G;
  constexpr int NPH = Bs::NPH;
  constexpr int NCH = Bs::NCH;
  constexpr int NG4 = (M + 1 + 3) / 4;  // float4 loads per coefficient row
  constexpr int BPT = kBinsPerThread;   // consecutive bins per thread per iteration
  static_assert(BPT == 2, "the loads below read float2 / double2");

  const ChunkCache& cc = sm.cc;
  const int tid = threadIdx.x;
  const int nh = cc.nh, nlo = cc.nlo, nhi = cc.nhi, ts = sm.ts.tile_start;
  const int nterms = Bs::NTF < 0 ? hs.nterms : NT;
  const float aE = vc.aE, tbase = vc.tbase, dtf = vc.dt;
  const int lane = tid & 31, w = tid >> 5;
  const int tb = tid;  // the thread's position in an iteration's bins
  const int store = hs.store;

  float acc_v = 0.0f, acc_c = 0.0f;  // Kahan-compensated cost value
  float gacc[G][NPH];                // per histogram: G_m (m < M), W
  float sh[NT][4];                   // per term: Lambda, S, nu, Delta
#pragma unroll
  for (int i = 0; i < G; ++i)
#pragma unroll
    for (int q = 0; q < NPH; ++q) gacc[i][q] = 0.0f;
#pragma unroll
  for (int k = 0; k < NT; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) sh[k][q] = 0.0f;

  constexpr int CHUNK_BINS = kBlock * BPT;  // bins of one CTA iteration
  // Iterations of this tile that hold any bin of the fit range (the same for every thread);
  // a piece of a launch-level partition brings its own count.
  const int iters = nit >= 0 ? nit : min(hs.tile_bins / CHUNK_BINS, (nhi - ts + CHUNK_BINS - 1) / CHUNK_BINS);
  // FP32 counts are staged into shared memory one iteration ahead by 16-byte cp.async copies,
  // each pair of lanes copying the 4 bins it reads of every histogram (half the histograms
  // each) and meeting at a warp barrier: no CTA-wide barrier per iteration, the warps run
  // independently through the tile.  Borrowed rows are 16-byte aligned with a stride of a
  // multiple of 4, and tiles start at multiples of 4 bins, so every copy is aligned.
  const bool staged = store == kStoreF32;
  const int64_t stride = hs.stride;
  // Lanes 2q and 2q + 1 of a warp share the 16-byte block of bins [4q, 4q + 4) of the
  // iteration: the even lane copies it for the even histograms, the odd lane for the odd.
  const int par = tb & 1, q4 = (tb >> 1) * 4;
  auto issue = [&](int itn) {  // bins [4q, 4q + 4) of iteration itn into buffer itn & 1
    if (itn < iters) {
      // n is a multiple of 4 and so is stride, so n < stride means all 4 bins lie in the row
      const int64_t n = ts + static_cast<int64_t>(itn) * CHUNK_BINS + q4;
      const bool in = n < stride;
#pragma unroll
      for (int i = 0; i < (G + 1) / 2; ++i) {
        const int hl = 2 * i + par;
        if (hl >= nh) break;
        const bool ok = dbg_ok(job.dbg, cc.row[hl] >= 0 && cc.row[hl] < hs.H && n >= 0, kDbgHist);
        cp_async16(sm.stage_slot(itn & 1, hl, q4),
                   static_cast<const float*>(cc.rowp[hl]) + (in && ok ? n : 0), in && ok ? 16u : 0u);
      }
    }
    cp_async_commit();  // one group per iteration (empty past the tile's end)
  };
  if (staged) issue(0);
  // The bin offset in the tile is carried as an exact float (integers < 2^24): an
  // int-to-float conversion per bin would occupy this GPU's slow FP64/conversion pipe.
  float fm0 = static_cast<float>(tb * BPT);
  for (int it = 0; it < iters; ++it, fm0 += static_cast<float>(CHUNK_BINS)) {
    const int m0 = it * CHUNK_BINS + tb * BPT;  // offset in the tile (< 2^15)
    const int n0 = ts + m0;
    const int b = it & 1;
    if (staged) {
      // buffer b ^ 1 was read by this lane and its partner in iteration it - 1: once both
      // are past it, refill it for it + 1, then wait for this lane's copies of iteration it
      // (all but the newest group) and for the partner's
      __syncwarp();
      issue(it + 1);
      cp_async_wait<1>();
      __syncwarp();
    }
    float t[BPT];
    bool valid[BPT];
#pragma unroll
    for (int j = 0; j < BPT; ++j) {
      t[j] = fmaf(__fadd_rn(fm0, static_cast<float>(j)), dtf, tbase);
      valid[j] = (n0 + j >= nlo) && (n0 + j < nhi);
    }
    // Time-only parts of the bin.  Every operation that reaches the cost value is an
    // explicitly rounded intrinsic: no contraction into FMAs that could differ between the
    // value-only and the value+gradient instantiations, so both return the same value.
    // dK: the derivative factor of a Kubo-Toyabe term (static: along Delta, scaled; dynamic:
    // d/dDelta).  d/dnu of a dynamic Kubo-Toyabe term waits in shared memory (sm.dkn) for the
    // shared channels after the histogram loop, so that no register is held for it there.
    float E[BPT], Pc[NT][BPT], Ps[NT][BPT], dK[NT][BPT];
#pragma unroll
    for (int j = 0; j < BPT; ++j) E[j] = ex2a(__fmul_rn(-aE, t[j]));
#pragma unroll
    for (int k = 0; k < NT; ++k) {
#pragma unroll
      for (int j = 0; j < BPT; ++j) Pc[k][j] = Ps[k][j] = dK[k][j] = 0.0f;
      if (k >= nterms) continue;
      const float ca = vc.ca[k], cb = vc.cb[k], ba = vc.bamp[k];
      const bool istf = Bs::tf(vc.kinds, k);
      const bool iskt = !istf && vc.kinds[k] == kTermKT;
      const bool islkt = !istf && vc.kinds[k] == kTermLKT;
      const bool isdkt = Bs::DKT && !istf && vc.kinds[k] == kTermDKT;
#pragma unroll
      for (int j = 0; j < BPT; ++j) {
        float X = __fmul_rn(ba, ex2a(__fmul_rn(-fmaf(cb, t[j], ca), t[j])));  // a E X_k
        if (iskt) {
          const float tt = __fmul_rn(t[j], t[j]);
          const float g = ex2a(__fmul_rn(-vc.dh[k], tt));
          const float u = __fmul_rn(vc.d2[k], tt);
          dK[k][j] = X * tt * g * (u - 3.0f);
          X = __fmul_rn(X, fmaf(__fmul_rn(2.0f / 3.0f, __fsub_rn(1.0f, u)), g, 1.0f / 3.0f));
        } else if (islkt) {  // static Lorentzian Kubo-Toyabe
          const float g = ex2a(__fmul_rn(-vc.dh[k], t[j]));
          const float u = __fmul_rn(vc.d2[k], t[j]);
          dK[k][j] = X * t[j] * g * (u - 2.0f);
          X = __fmul_rn(X, fmaf(__fmul_rn(2.0f / 3.0f, __fsub_rn(1.0f, u)), g, 1.0f / 3.0f));
        } else if (isdkt) {  // dynamic Kubo-Toyabe: the cubic through the evaluation's table
          const int src = vc.dkt_src[k];
          float G = 1.0f, gD = 0.0f, gN = 0.0f;
          if (src >= 0)
            dkt_lookup(static_cast<const float*>(job.dkt) + static_cast<size_t>(src) * kDktTable, t[j], &G, &gD, &gN);
          dK[k][j] = X * gD;
          sm.dkn[k][j][tid] = X * gN;
          X = __fmul_rn(X, G);
        }
        Pc[k][j] = X;
      }
      if (istf) {
        // Phase (turns) of the thread's first bin: base + m0 * step, reduced exactly.
        float f = __fmul_rn(fm0, vc.shi[k]);
        f = __fsub_rn(f, rint_small(f));
        float r = __fadd_rn(fmaf(fm0, vc.slo[k], vc.base[k]), f);
        r = __fsub_rn(r, rint_small(r));
#pragma unroll
        for (int j = 0; j < BPT; ++j) {
          float rj = fmaf(static_cast<float>(j), vc.sstep[k], r);
          rj = __fsub_rn(rj, rint_small(rj));  // |rj| <= 1/2: sin/cos arguments in [-pi, pi]
          const float a = __fmul_rn(rj, kTwoPiF);
          Ps[k][j] = __fmul_rn(Pc[k][j], sina(a));
          Pc[k][j] = __fmul_rn(Pc[k][j], cosa(a));
        }
      }
    }
    // Basis functions.
    float B[M][BPT];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int j = 0; j < BPT; ++j) B[m][j] = m == 0 ? E[j] : 0.0f;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      if (k >= nterms) continue;
      const bool istf = Bs::tf(vc.kinds, k);
#pragma unroll
      for (int j = 0; j < BPT; ++j) {
        if (Bs::MERGED) {
          if (istf) {
            B[1][j] = __fadd_rn(B[1][j], Pc[k][j]);
            B[2][j] = __fadd_rn(B[2][j], Ps[k][j]);
          } else {
            B[0][j] = __fadd_rn(B[0][j], Pc[k][j]);
          }
        } else {
          B[Bs::bc(k)][j] = Pc[k][j];
          if (Bs::NTF < 0 || k < Bs::NTF) B[Bs::bs(k)][j] = Ps[k][j];
        }
      }
    }

    // Gauss-Newton products: the basis functions' directional derivatives along v.
    constexpr bool GN = MODE == 2 || MODE == 3;
    float Bd[GN ? M : 1][BPT];
    if (GN) {
#pragma unroll
      for (int m = 0; m < (GN ? M : 1); ++m)
#pragma unroll
        for (int j = 0; j < BPT; ++j) Bd[m][j] = 0.0f;
#pragma unroll
      for (int k = 0; k < NT; ++k) {
        if (k >= nterms) continue;
        const bool istf = Bs::tf(vc.kinds, k);
#pragma unroll
        for (int j = 0; j < BPT; ++j) {
          const float g = -t[j] * fmaf(t[j], cc.dsig[k], cc.dlam[k]);  // d ln(X_k) along v
          const float w = kTwoPiF * t[j] * cc.dnu[k];                    // d theta_k along v
          const float dc = fmaf(Pc[k][j], g, -Ps[k][j] * w);
          const float ds = fmaf(Ps[k][j], g, Pc[k][j] * w);
          const float dN = Bs::DKT && !istf && vc.kinds[k] == kTermDKT ? sm.dkn[k][j][tid] : 0.0f;
          const float dn = fmaf(Pc[k][j], g, fmaf(cc.ddel[k], dK[k][j], cc.dnu[k] * dN));  // no cosine
          if (Bs::MERGED) {
            if (istf) {
              Bd[1 % (GN ? M : 1)][j] += dc;
              Bd[2 % (GN ? M : 1)][j] += ds;
            } else {
              Bd[0][j] += dn;
            }
          } else if (Bs::NTF < 0 || k < Bs::NTF) {
            if (istf) {
              Bd[Bs::bc(k) % (GN ? M : 1)][j] = dc;
              Bd[Bs::bs(k) % (GN ? M : 1)][j] = ds;
            } else {
              Bd[Bs::bc(k) % (GN ? M : 1)][j] = dn;
            }
          } else {
            Bd[Bs::bc(k) % (GN ? M : 1)][j] = dn;
          }
        }
      }
    }

    float V[M][BPT];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int j = 0; j < BPT; ++j) V[m][j] = 0.0f;
    float vit = 0.0f;  // this iteration's cost terms
    float2 vit2 = make_float2(0.0f, 0.0f);  // ... per bin of the thread

    // Per (histogram, bin).  Away from the ends of the fit range every bin of the warp is
    // valid and the loop runs without masks.
    const bool all_valid = __all_sync(0xffffffffu, valid[0] && valid[1]);
    // The counts and the coefficient row of histogram hl (rows past nh are read but unused).
    auto fetch_dot = [&](int hl, float (&gd)[4 * NG4]) {
#pragma unroll
      for (int q = 0; q < NG4; ++q) {
        const float4 x = *reinterpret_cast<const float4*>(&cc.gdot[hl][4 * q]);
        gd[4 * q] = x.x;
        gd[4 * q + 1] = x.y;
        gd[4 * q + 2] = x.z;
        gd[4 * q + 3] = x.w;
      }
    };
    auto fetch = [&](int hl, float (&d)[BPT], float (&gm)[4 * NG4]) {
      if (staged) {
        const float2 q = *reinterpret_cast<const float2*>(sm.stage_slot(b, hl, tb * BPT));
        d[0] = q.x;
        d[1] = q.y;
      } else if (hl < nh) {
        // n0 is even and the row stride a multiple of 64: n0 < stride holds both bins
        const double2 q = n0 < stride ? __ldg(reinterpret_cast<const double2*>(
                                            static_cast<const double*>(cc.rowp[hl]) + n0))
                                      : make_double2(0.0, 0.0);
        d[0] = static_cast<float>(q.x);
        d[1] = static_cast<float>(q.y);
      }
#pragma unroll
      for (int q = 0; q < NG4; ++q) {
        const float4 x = *reinterpret_cast<const float4*>(&vc.gam[hl][4 * q]);
        gm[4 * q] = x.x;
        gm[4 * q + 1] = x.y;
        gm[4 * q + 2] = x.z;
        gm[4 * q + 3] = x.w;
      }
    };
    auto fetch_w = [&](int hl) {  // the thread's two weights of histogram hl < nh (0 past the row)
      return n0 < stride ? __ldg(reinterpret_cast<const float2*>(static_cast<const float*>(cc.roww[hl]) + n0))
                         : make_float2(0.0f, 0.0f);
    };
    auto hist_loop = [&](auto masked_tag, auto full_tag) {
      constexpr bool MASKED = decltype(masked_tag)::value;
      constexpr bool FULL = decltype(full_tag)::value;  // nh == G: no per-histogram exit test
      // No explicit prefetch of the next histogram's loads: holding them costs 6 registers at
      // the 128-register cap of two CTAs per SM, and the unrolled loop lets the compiler
      // schedule the loads itself (measured 1-4 % faster on the merged shapes).
#pragma unroll
      for (int hl = 0; hl < G; ++hl) {
        if (!FULL && hl >= nh) break;
        float d[BPT], gm[4 * NG4];  // counts; Nbkg, Gam_0 .. Gam_{M-1}
        fetch(hl, d, gm);
        const float2 wc = MODE == 4 ? fetch_w(hl) : make_float2(0.0f, 0.0f);
        if (GN) {  // Gauss-Newton product: N' = J v, u = (d^2 (cost/2)/dN^2) N', value u N'
          float gdv[4 * NG4];
          fetch_dot(hl, gdv);
#pragma unroll
          for (int j = 0; j < BPT; ++j) {
            float N = gm[0], Nd = gdv[0];
#pragma unroll
            for (int m = 0; m < M; ++m) {
              N = fmaf(gm[1 + m], B[m][j], N);
              Nd = fmaf(gdv[1 + m], B[m][j], fmaf(gm[1 + m], Bd[m % (GN ? M : 1)][j], Nd));
            }
            const float dd = d[j];
            float w;
            bool undefined = false;
            if (MODE == 2) {
              w = rcpa(fmaxf(dd, 1.0f));
            } else {
              const float rN = rcpa(N);
              undefined = dd > 0.0f && !(N > 0.0f);
              w = dd > 0.0f ? dd * rN * rN : 0.0f;
            }
            float u = w * Nd;
            float v = undefined ? __int_as_float(0x7f800000) : u * Nd;
            if (MASKED && !valid[j]) u = v = 0.0f;
            vit2.x += v;
#pragma unroll
            for (int m = 0; m < M; ++m) gacc[hl][m] = fmaf(u, B[m][j], gacc[hl][m]);
            gacc[hl][M] += u;
#pragma unroll
            for (int m = 0; m < M; ++m) V[m][j] = fmaf(u, gm[1 + m], V[m][j]);
          }
          continue;
        }
        {  // the thread's two bins as one float2: packed FP32 (two lanes' work per instruction)
          const float2 dd2 = make_float2(d[0], d[1]);
          float2 N2 = make_float2(gm[0], gm[0]);
#pragma unroll
          for (int m = 0; m < M; ++m)
            N2 = __ffma2_rn(make_float2(gm[1 + m], gm[1 + m]), make_float2(B[m][0], B[m][1]), N2);
          const float2 r2 = __fadd2_rn(N2, make_float2(-dd2.x, -dd2.y));
          float2 v2, u2;
          if (MODE == 0 || MODE == 4) {
            // chi^2 weight: 1 / max(d, 1) (Eq. chisq), or the asymmetry data's own (MODE 4)
            float2 iv2;
            if (MODE == 4) {  // FP32 weights beside FP32 asymmetry values
              iv2 = wc;
            } else {
              iv2 = make_float2(rcpa(fmaxf(dd2.x, 1.0f)), rcpa(fmaxf(dd2.y, 1.0f)));
            }
            u2 = __fmul2_rn(r2, iv2);
            v2 = __fmul2_rn(r2, u2);
          } else {
            const float2 rN2 = make_float2(rcpa(N2.x), rcpa(N2.y));
            const float2 uu2 = __fmul2_rn(r2, rN2);
            const float2 vs2 = __fmul2_rn(r2, __fmul2_rn(uu2, phi_u2(uu2)));
            const float2 x2 = __fmul2_rn(dd2, rN2);
            const float2 vl2 = __ffma2_rn(__fmul2_rn(dd2, make_float2(kLn2F, kLn2F)),
                                          make_float2(lg2a(x2.x), lg2a(x2.y)), r2);
            const bool p0 = dd2.x > 0.0f, p1 = dd2.y > 0.0f;
            v2.x = p0 ? (fabsf(uu2.x) < 0.2f ? vs2.x : vl2.x) : r2.x;
            v2.y = p1 ? (fabsf(uu2.y) < 0.2f ? vs2.y : vl2.y) : r2.y;
            u2.x = p0 ? uu2.x : 1.0f;
            u2.y = p1 ? uu2.y : 1.0f;
          }
          if (MASKED) {
            if (!valid[0]) v2.x = u2.x = 0.0f;
            if (!valid[1]) v2.y = u2.y = 0.0f;
          }
          vit2 = __fadd2_rn(vit2, v2);
          if (GRAD) {
#pragma unroll
            for (int m = 0; m < M; ++m) gacc[hl][m] = fmaf(u2.y, B[m][1], fmaf(u2.x, B[m][0], gacc[hl][m]));
            gacc[hl][M] = (gacc[hl][M] + u2.x) + u2.y;
#pragma unroll
            for (int m = 0; m < M; ++m) {
              const float2 Vm = __ffma2_rn(u2, make_float2(gm[1 + m], gm[1 + m]), make_float2(V[m][0], V[m][1]));
              V[m][0] = Vm.x;
              V[m][1] = Vm.y;
            }
          }
        }
      }
    };
    if (nh == G) {
      if (all_valid)
        hist_loop(std::false_type{}, std::true_type{});
      else
        hist_loop(std::true_type{}, std::true_type{});
    } else {
      if (all_valid)
        hist_loop(std::false_type{}, std::false_type{});
      else
        hist_loop(std::true_type{}, std::false_type{});
    }
    vit = __fadd_rn(vit2.x, vit2.y);
    {  // Kahan-compensated running sum of the per-iteration partials
      const float y = __fsub_rn(vit, acc_c);
      const float tsum = __fadd_rn(acc_v, y);
      acc_c = __fsub_rn(__fsub_rn(tsum, acc_v), y);
      acc_v = tsum;
    }
    if (GRAD) {
      // Shared channels: derivatives of the time-only pieces against the chunk's per-bin sums.
#pragma unroll
      for (int j = 0; j < BPT; ++j) {
        const float mt = -t[j], mh = -0.5f * t[j] * t[j], tp = kTwoPiF * t[j];
#pragma unroll
        for (int k = 0; k < NT; ++k) {
          if (k >= nterms) continue;
          const bool istf = Bs::tf(vc.kinds, k);
          const float Vc = V[Bs::bc(k)][j];
          float D;
          if (Bs::NTF < 0 || k < Bs::NTF) {
            const float Vs = V[Bs::bs(k)][j];
            D = fmaf(Vc, Pc[k][j], Vs * Ps[k][j]);
            if (istf) sh[k][2] = fmaf(tp, fmaf(Vs, Pc[k][j], -Vc * Ps[k][j]), sh[k][2]);
          } else {
            D = Vc * Pc[k][j];
          }
          if (!istf) sh[k][3] = fmaf(Vc, dK[k][j], sh[k][3]);  // zero unless Kubo-Toyabe
          if (Bs::DKT && !istf && vc.kinds[k] == kTermDKT) sh[k][2] = fmaf(Vc, sm.dkn[k][j][tid], sh[k][2]);
          sh[k][0] = fmaf(mt, D, sh[k][0]);
          sh[k][1] = fmaf(mh, D, sh[k][1]);
        }
      }
    }
  }

  // Every copy of this thread has landed before the staging space is used again.
  if (staged) cp_async_wait<0>();
  float vh = acc_v, vl = -acc_c;
  warp_sum_ff(vh, vl);
  // ---- thread (FP32) -> warp (FP32; the value as float-float) -> CTA (FP64 trees) -> row.
  __syncthreads();
  if (lane == 0) {
    sm.vred[w][0] = vh;
    sm.vred[w][1] = vl;
  }
  if (GRAD) {
#pragma unroll
    for (int hl = 0; hl < G; ++hl)
#pragma unroll
      for (int q = 0; q < NPH; ++q) {
        const float r = warp_sum_f(gacc[hl][q]);
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
  if (!dbg_ok(job.dbg, item >= 0 && item < job.nrows, kDbgPartial)) return;
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
    // +inf: the likelihood is undefined (N <= 0 where d > 0) or the parameters were not finite.
    if (l == 0)
      row[0] = isfinite(a) ? a * (MODE == 0 || MODE == 4 ? 1.0 : 2.0) : __longlong_as_double(0x7ff0000000000000LL);
  }
}

// SPLIT channels -> derivative of local slot s of chunk histogram hl.
template <int SHAPE>
__device__ double split_slot(const HistSet& hs, const ChunkCache& cc, const double* tot, int hl, int s) {
  using Bs = Basis<SHAPE>;
  const double* gch = tot + 1 + hl * Bs::NPH;  // G_m (m < M), W
  const double* sch = tot + 1 + Bs::G * Bs::NPH;
  const double N0 = cc.loc[hl][0];
  constexpr double kDeg = kTwoPi / 360.0;
  double g = 0.0;
  for (int e = 0; e < hs.ncontrib; ++e) {
    const Contrib c = hs.contrib[e];
    if (c.slot != s) continue;
    const int k = c.term;
    const CanonTerm& ct = hs.canon[k];
    switch (c.kind) {
      case kCN0: {  // sum_m (dGam_m / dN0) G_m
        double a = hs.envelope ? gch[0] : 0.0;  // Gam_0 = N0 only with the decay envelope
        if (Bs::MERGED) {
          a += cc.cph[hl][0] * gch[1] - cc.sph[hl][0] * gch[2];
        } else {
          for (int kk = 0; kk < hs.nterms && kk < Bs::NT; ++kk) {
            const CanonTerm& q = hs.canon[kk];
            const double amp = q.amp_slot >= 0 ? cc.loc[hl][q.amp_slot] : 1.0;
            if (q.kind == kTermTF) {
              a += amp * (cc.cph[hl][kk] * gch[Bs::bc(kk)] - cc.sph[hl][kk] * gch[Bs::bs(kk)]);
            } else {
              a += amp * gch[Bs::bc(kk)];
            }
          }
        }
        g += 2.0 * a;
        break;
      }
      case kCBkg:
        g += 2.0 * gch[Bs::M];
        break;
      case kCAmp:  // unmerged shapes only
        if (!Bs::MERGED) {
          if (ct.kind == kTermTF) {
            g += 2.0 * N0 * (cc.cph[hl][k] * gch[Bs::bc(k)] - cc.sph[hl][k] * gch[Bs::bs(k)]);
          } else {
            g += 2.0 * N0 * gch[Bs::bc(k)];
          }
        }
        break;
      case kCPhi: {
        const double amp = !Bs::MERGED && ct.amp_slot >= 0 ? cc.loc[hl][ct.amp_slot] : 1.0;
        g += 2.0 * N0 * amp * kDeg * (-cc.sph[hl][k] * gch[Bs::bc(k)] - cc.cph[hl][k] * gch[Bs::bs(k)]);
        break;
      }
      case kCLam:
        if (hl == 0) g += 2.0 * sch[k * 4 + 0];
        break;
      case kCSig:
        if (hl == 0) g += 4.0 * cc.loc[0][s] * sch[k * 4 + 1];
        break;
      case kCNu:
        if (hl == 0) g += 2.0 * sch[k * 4 + 2];
        break;
      case kCLkt:
        if (hl == 0) g += (4.0 / 3.0) * sch[k * 4 + 3];
        break;
      case kCDktD:
        if (hl == 0) g += 2.0 * sch[k * 4 + 3];
        break;
      case kCDktN:
        if (hl == 0) g += 2.0 * sch[k * 4 + 2];
        break;
      case kCDel:
        if (hl == 0) g += (4.0 / 3.0) * cc.loc[0][s] * sch[k * 4 + 3];
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
template <int PREC, int SHAPE, bool GRAD, class SM>
__device__ void chunk_finalize(const Job& job, const HistSet& hs, SM& sm) {
  const ChunkCache& cc = sm.cc;
  const int tid = threadIdx.x;
  const int ps = hs.pstride;
  const int nout = GRAD ? 1 + hs.nch : 1;
  if (!dbg_ok(job.dbg, cc.item0 >= 0 && cc.item0 + cc.ntiles <= job.nrows, kDbgPartial)) return;
  const double* part = job.partials + static_cast<int64_t>(cc.item0) * ps;
  // The chunk's item rows, summed per column in a fixed order: each column's rows are cut
  // into `tpc` contiguous segments, one thread sums a segment (its loads all in flight),
  // then the segment sums are added in segment order.  The order depends only on the
  // chunk's tile count, not on which CTA ran which item.
  static_assert(kMaxChan + 1 <= kBlock, "one thread per column");
  // (the segmentation follows the value+gradient row width in both kernels, so that the
  // value-only kernel sums the value column in the same order)
  const int tpc = max(1, min(kBlock / (1 + hs.nch), cc.ntiles));  // threads (segments) per column
  double* seg = reinterpret_cast<double*>(&sm.stage[0][0][0]);  // [nout][tpc], idle staging space
  if (tid < nout * tpc) {
    const int c = tid / tpc, k = tid - c * tpc;
    const int t0 = static_cast<int>(static_cast<int64_t>(cc.ntiles) * k / tpc);
    const int t1 = static_cast<int>(static_cast<int64_t>(cc.ntiles) * (k + 1) / tpc);
    double a = 0.0;
    for (int t = t0; t < t1; t += 8) {  // eight rows' loads in flight, added in row order
      double x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = t + q < t1 ? __ldcg(part + static_cast<int64_t>(t + q) * ps + c) : 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (t + q < t1) a += x[q];
    }
    seg[c * tpc + k] = a;
  }
  __syncthreads();
  if (tid < nout) {
    double a = 0.0;
    for (int k = 0; k < tpc; ++k) a += seg[tid * tpc + k];
    sm.tot[tid] = a;
  }
  __syncthreads();
  if (GRAD) {
    const int nsl = hs.nslots;
    for (int i = tid; i < cc.nh * nsl; i += kBlock) {
      const int hl = i / nsl, s = i - hl * nsl;
      double g;
      if constexpr (PREC == 0 || is_list(SHAPE))
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

template <class SM>
__device__ void job_finalize(const Job& job, const HistSet& hs, SM& sm) {
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
      const int j1 = hs.p_ptr[p + 1];
      for (int j = hs.p_ptr[p]; j < j1; j += 8) {  // eight loads in flight, summed in column order
        double x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int col = j + q < j1 ? hs.p_cols[j + q] : 0;
          x[q] = j + q < j1 && dbg_ok(job.dbg, col >= 0 && col < hs.ncols, kDbgCol) ? __ldcg(job.colsum + col) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (j + q < j1) g += x[q];
      }
      job.out[1 + p] = finite ? g : 0.0;
    }
  }
  if (tid == 0) {
    job.out[0] = value;
    *job.counter = 0u;
  }
}

// The chunk of a job whose last row has just been published: the CTA sums the chunk's rows
// (chunk finalize) and, if that chunk was the job's last, the job's chunks (job finalize).
// Acquire: every thread fences after the acquire-release counter increment that found the
// chunk complete.
template <int PREC, int SHAPE, bool GRAD, class SM>
__device__ void finish_chunk(const Job& job, const HistSet& hs, SM& sm) {
  fence_acq_rel();
  chunk_finalize<PREC, SHAPE, GRAD>(job, hs, sm);
  __syncthreads();
  if (hs.nchunks == 1) {  // the chunk was the job's only one: no second counter
    job_finalize(job, hs, sm);
    __syncthreads();
    return;
  }
  if (threadIdx.x == 0) {
    const unsigned prev = atom_add_acq_rel(job.counter, 1u);
    sm.flag = prev == static_cast<unsigned>(hs.nchunks - 1);
  }
  __syncthreads();
  if (!sm.flag) return;
  fence_acq_rel();
  job_finalize(job, hs, sm);
  __syncthreads();
}

// Publishes the item's row; the CTA that completes a chunk's last item finalizes the
// chunk, and the one that completes a job's last chunk finalizes the job.  Release: the
// CTA barrier orders every thread's row writes before thread 0's acquire-release counter
// increment (cumulative over what the barrier ordered before it); acquire: that same
// atomic, and a fence by every thread of the finalizing CTA.
template <int PREC, int SHAPE, bool GRAD>
__device__ void complete_item(const Job& job, const HistSet& hs, Smem& sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atom_add_acq_rel(job.chunk_count + sm.cc.chunk, 1u);
    sm.flag = prev == static_cast<unsigned>(sm.cc.ntiles - 1);
  }
  __syncthreads();
  if (!sm.flag) return;
  finish_chunk<PREC, SHAPE, GRAD>(job, hs, sm);
}

// ---------------------------------------------------------------------------------------------
// Persistent kernel: each CTA takes a contiguous range of the launch's items.
// ---------------------------------------------------------------------------------------------
template <int PREC, int SHAPE, int MODE, bool GRAD>
__global__ void __launch_bounds__(kBlock, PREC == 1 && SHAPE != kShapeList ? 2 : 1) eval_kernel(
    const Job* __restrict__ jobs, int njobs,
                                                      int total_items) {
  __shared__ Smem sm;
  const int per = (total_items + gridDim.x - 1) / gridDim.x;
  const int beg = blockIdx.x * per;
  const int end = min(total_items, beg + per);
  if (threadIdx.x == 0) {
    sm.cc.job = -1;
    sm.cc.chunk = -1;
  }
  __syncthreads();
  if constexpr (PREC == 1 && !is_list(SHAPE)) {
    if (jobs[0].pieces) {  // launch-level partition: this CTA's pieces, in order
      if (static_cast<int>(blockIdx.x) >= jobs[0].npiece_ctas) return;
      const int pb = jobs[0].piece_cta[blockIdx.x], pe = jobs[0].piece_cta[blockIdx.x + 1];
      for (int p = pb; p < pe; ++p) {
        const Piece pc = jobs[0].pieces[p];
        if (!dbg_ok(jobs[0].dbg, pc.job >= 0 && pc.job < njobs, kDbgJob)) continue;
        const Job job = jobs[pc.job];
        const HistSet& hs = *job.hs;
        if (sm.cc.job != pc.job || sm.cc.chunk != pc.chunk) {
          __syncthreads();
          load_chunk<SHAPE>(job, hs, pc.job, pc.chunk, PREC, sm);
          if (threadIdx.x == 0) {  // the chunk's rows in this partition (load_tile_at's barrier publishes them)
            const int2 r = job.chunk_rows[pc.chunk];
            sm.cc.item0 = r.x;
            sm.cc.ntiles = r.y;
          }
        }
        load_tile_at(sm.cc.tile0 + pc.it0 * (kBlock * kBinsPerThread), hs, PREC, sm);
        split_item<SHAPE, MODE, GRAD>(job, hs, pc.row, sm, sm.cc.v, pc.nit);
        complete_item<PREC, SHAPE, GRAD>(job, hs, sm);
      }
      return;
    }
  }
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
    // term lists without a basis form take the FP64 path's chunk and tile setup
    constexpr int kSetupPrec = is_list(SHAPE) ? 0 : PREC;
    if (sm.cc.job != ji || item < sm.cc.item0 || item >= sm.cc.item0 + sm.cc.ntiles) {
      __syncthreads();
      load_chunk<SHAPE>(job, hs, ji, hs.items[item].x, kSetupPrec, sm);
      if constexpr (PREC == 1 && is_list(SHAPE)) load_chunk_list(hs, sm);
    }
    load_tile(hs, item - sm.cc.item0, kSetupPrec, sm);
    if constexpr (PREC == 1 && is_list(SHAPE)) load_tile_list(hs, sm);
    if constexpr (PREC == 0)
      fp64_item<MODE, GRAD>(job, hs, item, sm);
    else if constexpr (SHAPE == kShapeList)
      list_item<MODE, GRAD, kMaxTerms, kMaxPrims>(job, hs, item, sm);
    else if constexpr (SHAPE == kShapeListS)  // at most 2 terms of at most 3 primitives
      list_item<MODE, GRAD, 2, 3>(job, hs, item, sm);
    else
      split_item<SHAPE, MODE, GRAD>(job, hs, item, sm, sm.cc.v);
    complete_item<PREC, SHAPE, GRAD>(job, hs, sm);
  }
}

// Resident CTAs per SM of one instantiation (the occupancy query, made once: a driver call
// per launch would add its latency to every single evaluation).
template <int PREC, int SHAPE, int MODE, bool GRAD>
int resident_ctas() {
  static const int per_sm = [] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, eval_kernel<PREC, SHAPE, MODE, GRAD>, kBlock, 0) !=
        cudaSuccess)
      return -1;
    return n;
  }();
  return per_sm;
}

template <int PREC, int SHAPE, int MODE, bool GRAD>
int launch_one(const Job* d_jobs, int njobs, int total_items, int num_sms, cudaStream_t stream,
               LaunchInfo* info) {
  auto kern = eval_kernel<PREC, SHAPE, MODE, GRAD>;
  int per_sm = resident_ctas<PREC, SHAPE, MODE, GRAD>();
  if (per_sm < 0) return -1;
  if (per_sm < 1) per_sm = 1;
  int grid = num_sms * per_sm;
  if (grid > total_items) grid = total_items;
  if (grid < 1) grid = 1;
  kern<<<grid, kBlock, 0, stream>>>(d_jobs, njobs, total_items);
  if (info) {
    info->grid = grid;
    info->block = kBlock;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears the error
}

template <int PREC, int SHAPE, int MODE, bool GRAD>
int occupancy_one() {
  const int per_sm = resident_ctas<PREC, SHAPE, MODE, GRAD>();
  return per_sm < 0 ? 0 : per_sm;
}

template <int PREC, int SHAPE>
int dispatch_mode(int mode, int grad, const Job* j, int n, int items, int sms, cudaStream_t s,
                  LaunchInfo* info) {
  if constexpr (is_list(SHAPE)) {  // no Gauss-Newton kernels for term lists (FP64 path)
    if (mode == 2 || mode == 3) return -1;
  } else {
    if (mode == 2) return launch_one<PREC, SHAPE, 2, true>(j, n, items, sms, s, info);
    if (mode == 3) return launch_one<PREC, SHAPE, 3, true>(j, n, items, sms, s, info);
  }
  if (PREC == 1 && mode == 4)  // weighted chi^2 of asymmetry data (SPLIT)
    return grad ? launch_one<PREC, SHAPE, PREC == 1 ? 4 : 0, true>(j, n, items, sms, s, info)
                : launch_one<PREC, SHAPE, PREC == 1 ? 4 : 0, false>(j, n, items, sms, s, info);
  if (mode == 0)
    return grad ? launch_one<PREC, SHAPE, 0, true>(j, n, items, sms, s, info)
                : launch_one<PREC, SHAPE, 0, false>(j, n, items, sms, s, info);
  return grad ? launch_one<PREC, SHAPE, 1, true>(j, n, items, sms, s, info)
              : launch_one<PREC, SHAPE, 1, false>(j, n, items, sms, s, info);
}

template <int PREC, int SHAPE>
int occupancy_mode(int mode, int grad) {
  if constexpr (is_list(SHAPE)) {
    if (mode == 2 || mode == 3) return 0;
  } else {
    if (mode == 2) return occupancy_one<PREC, SHAPE, 2, true>();
    if (mode == 3) return occupancy_one<PREC, SHAPE, 3, true>();
  }
  if (PREC == 1 && mode == 4)
    return grad ? occupancy_one<PREC, SHAPE, PREC == 1 ? 4 : 0, true>()
                : occupancy_one<PREC, SHAPE, PREC == 1 ? 4 : 0, false>();
  if (mode == 0) return grad ? occupancy_one<PREC, SHAPE, 0, true>() : occupancy_one<PREC, SHAPE, 0, false>();
  return grad ? occupancy_one<PREC, SHAPE, 1, true>() : occupancy_one<PREC, SHAPE, 1, false>();
}

}  // namespace
}  // namespace kern

// Per-group launchers and occupancy queries (one translation unit each).
int launch_group_fp64(int mode, int grad, const Job* j, int n, int items, int sms, cudaStream_t s, LaunchInfo* info);
int occupancy_group_fp64(int mode, int grad);
#define MUSR_DECLARE_GROUP(G)                                                                                \
  int launch_group_##G(int shape, int mode, int grad, const Job* j, int n, int items, int sms, cudaStream_t s, \
                       LaunchInfo* info);                                                                   \
  int occupancy_group_##G(int shape, int mode, int grad);
MUSR_DECLARE_GROUP(a)
MUSR_DECLARE_GROUP(b)
MUSR_DECLARE_GROUP(c)
#undef MUSR_DECLARE_GROUP

}  // namespace musr
