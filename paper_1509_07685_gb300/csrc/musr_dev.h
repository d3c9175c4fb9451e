// musr_dev.h -- descriptors shared by the host side of libmusr and its kernels.
//
// Work decomposition (both precisions):
//   * a HistSet is one uploaded set of histograms plus theory and map, compiled
//     for one precision: its histograms are split into chunks, each tiled along
//     the bin axis; one work item = (chunk, tile) and is processed by one CTA;
//   * a Job is one evaluation of one parameter vector on one HistSet;
//   * a launch processes the items of one or more jobs with a persistent grid;
//     each item writes one row of FP64 partial sums, and the CTA that finishes a
//     job's last item sums that job's rows in a fixed order (deterministic: the
//     result does not depend on which CTA ran which item, nor on other jobs).
//
// FP64 path: a chunk is one histogram.  SPLIT path: a chunk is up to
// kGroupMax histograms that share t0 and every time-dependent parameter
// (relaxation rates, Kubo-Toyabe width, frequencies), so that the time-only
// factors of a bin are evaluated once and reused across the chunk.
#pragma once

#include <cstdint>

namespace musr {

constexpr double kTauMuUs = 2.197019;  // muon lifetime, microseconds
constexpr int kBlock = 256;            // threads per CTA
constexpr int kWarps = kBlock / 32;
constexpr int kBinsPerThread = 2;      // SPLIT: one 8-byte load of FP32 counts per histogram
constexpr int kMaxTileBins = 16384;    // SPLIT phase split: bin offsets in a tile stay below 2^14
constexpr int kGroupMax = 8;           // histograms per SPLIT chunk
constexpr int kMaxTerms = 4;
constexpr int kMaxPrims = 4;
constexpr int kMaxSlots = 32;
constexpr int kMaxContrib = 64;

enum StoreType : int { kStoreF32 = 1, kStoreF64 = 2 };
enum PrimKind : int { kAmp = 1, kExp = 2, kGauss = 3, kKT = 4, kTFCos = 5 };
enum TermKind : int { kTermNone = 0, kTermPlain = 1, kTermTF = 2, kTermKT = 3 };

// SPLIT shape identifiers (which compile-time specialisation runs a HistSet).
// The "c" shapes are the same term lists with every amplitude a constant (no
// amplitude gradient channels).
enum Shape : int {
  kShapeGeneric = 0,
  kShapeTF1 = 1,
  kShapeTF2 = 2,
  kShapeKT1 = 3,
  kShapeTF2KT1 = 4,
  kShapeTF2c = 5,
  kShapeTF2KT1c = 6
};

// A term as given: the product of nprim primitives (FP64 path).
struct RawTerm {
  int nprim;
  int kind[kMaxPrims];
  int slot[kMaxPrims][2];
};

// A term in canonical form (SPLIT path):
//   a * exp(-Lambda t - S t^2 / 2) * [KT(Delta, t)] * [cos(2 pi (nu t + phi / 360))]
// with Lambda the sum of its EXP rates and S the sum of its squared GAUSS widths.
struct CanonTerm {
  int kind;  // kTermPlain, kTermTF, kTermKT
  int amp_slot;  // -1: no AMP factor
  int nexp;
  int exp_slot[kMaxPrims];
  int ngauss;
  int gauss_slot[kMaxPrims];
  int kt_slot;   // kTermKT
  int nu_slot;   // kTermTF
  int phi_slot;  // kTermTF
};

// True when no amplitude slot of the canonical terms maps to a parameter.
inline bool amplitudes_constant(const CanonTerm* canon, int nterms, const int32_t* map, int H, int nslots) {
  for (int k = 0; k < nterms; ++k) {
    if (canon[k].amp_slot < 0) continue;
    for (int h = 0; h < H; ++h)
      if (map[static_cast<int64_t>(h) * nslots + canon[k].amp_slot] >= 0) return false;
  }
  return true;
}

// True when, for every histogram, all cosine terms take their phase from one
// parameter (or one constant value).
inline bool phases_shared(const CanonTerm* canon, int nterms, const int32_t* map, const double* consts, int H,
                          int nslots) {
  for (int h = 0; h < H; ++h) {
    int first = -1;
    for (int k = 0; k < nterms; ++k) {
      if (canon[k].kind != kTermTF) continue;
      const int32_t m = map[static_cast<int64_t>(h) * nslots + canon[k].phi_slot];
      if (first < 0) {
        first = k;
        continue;
      }
      const int32_t m0 = map[static_cast<int64_t>(h) * nslots + canon[first].phi_slot];
      const bool same = (m >= 0 || m0 >= 0) ? m == m0 : consts[-1 - m] == consts[-1 - m0];
      if (!same) return false;
    }
  }
  return true;
}

// Shape of a canonical term list whose amplitudes are all constants and whose
// cosines share one phase: the "c" variants of TF2 and TF2KT1.
inline int constant_amplitude_shape(int shape, const CanonTerm* canon, int nterms, const int32_t* map,
                                    const double* consts, int H, int nslots) {
  if (shape != kShapeTF2 && shape != kShapeTF2KT1) return shape;
  if (!amplitudes_constant(canon, nterms, map, H, nslots)) return shape;
  if (!phases_shared(canon, nterms, map, consts, H, nslots)) return shape;
  return shape == kShapeTF2 ? kShapeTF2c : kShapeTF2KT1c;
}

// How a SPLIT channel turns into the derivative of one local slot.
enum ContribKind : int {
  kCN0 = 0,    // d/dN0                 = 2 * ch_N0
  kCBkg = 1,   // d/dNbkg               = 2 * ch_bkg
  kCAmp = 2,   // d/da_k                = 2 * N0 * ch_amp[k]
  kCPhi = 3,   // d/dphi_k              = 2 * N0 * a_k * (-2 pi / 360) * ch_phi[k]
  kCLam = 4,   // d/dlambda (EXP of k)  = 2 * ch_lam[k]           (shared)
  kCSig = 5,   // d/dsigma  (GAUSS of k)= 4 * sigma * ch_S[k]     (shared)
  kCNu = 6,    // d/dnu_k               = 2 * ch_nu[k]            (shared)
  kCDel = 7    // d/dDelta_k            = (4/3) * Delta * ch_D[k] (shared)
};
struct Contrib {
  int slot;
  int kind;
  int term;
};

// Only chunks with at least one bin in the fit range are listed.
struct Chunk {
  int first;      // index into HistSet::hist_index of its first histogram
  int nh;         // number of histograms (<= kGroupMax, 1 on the FP64 path)
  int nlo, nhi;   // bins [nlo, nhi) in the fit (shared by the chunk)
  int item0;      // first work item of the chunk (HistSet-local)
  int ntiles;
  int col0;       // first finalize column of the chunk
  int tile0;      // first bin of tile 0 (nlo rounded down to a multiple of 4)
  double t0;      // time-zero bin shared by the chunk
};

struct HistSet {
  // histograms: [H][stride] in FP32 or FP64
  const void* counts;
  int store;
  int H;
  int64_t stride;
  double dt_us;
  // theory
  int nterms;
  RawTerm raw[kMaxTerms];
  CanonTerm canon[kMaxTerms];
  int shape;
  int ncontrib;
  Contrib contrib[kMaxContrib];
  // parameter map
  const int32_t* map;  // [H][nslots]
  int nslots;
  const double* consts;
  int P;
  // decomposition
  const Chunk* chunks;
  int nchunks;
  const int* hist_index;   // histograms of the chunks, chunk by chunk
  const int2* items;       // (chunk, tile) per work item
  int nitems;
  int tile_bins;           // bins per tile
  int group;               // histograms per chunk at most
  int nch;                 // reduction channels per item (SPLIT: per shape; FP64: 2 + 32)
  int pstride;             // doubles per partial row: 1 + nch
  int ncols;               // slot columns: sum over chunks of nh * nslots
  const int* col_chunk;    // [ncols] chunk of each column
  const int* p_ptr;        // [P + 1] CSR: columns contributing to parameter p
  const int* p_cols;
};

struct Job {
  const HistSet* hs;
  const double* params;      // [P]
  double* out;               // [1 + P]
  double* partials;          // [hs->nitems][hs->pstride]
  double* colsum;            // [hs->ncols]
  double* chunk_val;         // [hs->nchunks]
  unsigned int* chunk_count; // [hs->nchunks], zero between launches
  unsigned int* counter;     // zero between launches
  int item_begin;            // first global item of this job in the launch
  int mode;                  // 0 chi^2, 1 -2lnL
  int grad;                  // 0: value only
  int prec;                  // 0 FP64, 1 SPLIT
};

// Launchers (host side of musr_kernels.cu).  All enqueue on `stream`.
struct LaunchInfo {
  int grid;
  int block;
};
int launch_eval(int precision, int shape, int mode, int grad, const Job* d_jobs, int njobs,
                int total_items, int num_sms, void* stream, LaunchInfo* info);
int max_ctas_per_sm(int precision, int shape, int mode, int grad);
// Decompositions compiled per precision: tile v holds (bins per CTA iteration) << v
// bins -- SPLIT 512 ... 16384 (the phase-split limit), FP64 256 ... 8192.
constexpr int kVariants = 6;
inline int bins_per_iteration(int precision) { return precision == 1 ? kBlock * kBinsPerThread : kBlock; }

// The decomposition of a launch of nvec evaluations: the largest tiles that
// still give every resident CTA about four items (items[v] = items per
// evaluation of decomposition v), else the smallest tiles.
inline int pick_decomposition(const int* items, int64_t nvec, int num_sms) {
  const int64_t target = 4LL * 2 * num_sms;
  for (int v = kVariants - 1; v > 0; --v)
    if (nvec * items[v] >= target) return v;
  return 0;
}

// Histograms per chunk, and reduction channels per work item, of a SPLIT shape.
int shape_group(int shape);
int shape_channels(int shape);
constexpr int kFp64Channels = 2 + kMaxTerms * kMaxPrims * 2;

}  // namespace musr
