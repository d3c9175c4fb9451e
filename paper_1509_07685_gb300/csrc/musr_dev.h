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
constexpr int kMaxTileBins = 32768;    // SPLIT phase split: bin offsets in a tile stay below 2^15
constexpr int kGroupMax = 8;           // histograms per SPLIT chunk
constexpr int kMaxTerms = 4;
constexpr int kMaxPrims = 4;
constexpr int kMaxSlots = 32;
constexpr int kMaxContrib = 64;

enum StoreType : int { kStoreF32 = 1, kStoreF64 = 2 };
enum PrimKind : int {
  kAmp = 1, kExp = 2, kGauss = 3, kKT = 4, kTFCos = 5, kLKT = 6, kStrExp = 7, kBessel = 8, kDKT = 9
};
// Parameter slots of a primitive: frequency and phase (TFCOS, BESSEL), rate and exponent
// (STREXP), static width and fluctuation rate (DKT), else one.
__host__ __device__ inline int prim_nslots(int kind) {
  return kind == kTFCos || kind == kStrExp || kind == kBessel || kind == kDKT ? 2 : 1;
}

// Dynamic Kubo-Toyabe relaxation (DKT): the renewal equation G = f + nu f * G of the
// strong-collision model is solved per evaluation and per distinct (Delta, nu) pair (a
// "source") on a grid of K + 1 points over [0, span] (trapezoidal rule, Richardson
// extrapolation from the grid and its halving), K = ceil(span max(Delta, nu, 0.05) / step)
// clamped to [kDktMinK, kDktMaxK]; the bins interpolate the table with the cubic through the
// four nearest points.  Table of one source: header {h, 1/h, K} then G, dG/dDelta, dG/dnu,
// each kDktMaxK + 1 values, in the path's arithmetic type.  The step (grid spacing times the
// faster of Delta and nu) is 0.02 for FP64 tables; FP32 tables cannot resolve more than a few
// 1e-7 of G, and at 0.03 their discretisation and interpolation error stays below that
// rounding (a model of the scheme against the oracle: at most 6e-7, against 8e-7 at 0.02 and
// 4e-6 at 0.04), at (2/3)^2 of the work.
constexpr int kMaxDkt = 8;        // distinct (Delta, nu) sources of one histogram set
constexpr int kDktMaxK = 4096;
constexpr int kDktMinK = 64;
constexpr double kDktStep = 0.02;    // FP64 tables
constexpr double kDktStep32 = 0.03;  // FP32 tables (SPLIT)
constexpr int kDktHeader = 4;
constexpr int kDktTable = kDktHeader + 3 * (kDktMaxK + 1);   // values per source table
// scratch values per source: the finer grid's kernel and solution (6 arrays of 2 kDktMaxK + 1),
// the coarse grid's kernel (3 arrays of kDktMaxK + 1) and room to spare
constexpr int kDktWork = 8 * (2 * kDktMaxK + 1);
enum TermKind : int { kTermNone = 0, kTermPlain = 1, kTermTF = 2, kTermKT = 3, kTermLKT = 4, kTermDKT = 5 };

// SPLIT shapes.  Every model the SPLIT path accepts is, for each histogram j of a
// chunk, a linear combination of M time-only basis functions B_m(t) with
// per-histogram coefficients (Eq. positron_histo with A(t) expanded):
//   N_j(t) = Nbkg_j + sum_m Gam_jm B_m(t),   B_0 = E = exp(-t / tau_mu),
//   a cosine term k (relaxation R_k):  E R_k cos(2 pi nu_k t), E R_k sin(2 pi nu_k t)
//                                      with Gam = N0 a_k cos(phi_k), -N0 a_k sin(phi_k);
//   any other term k:                  E R_k with Gam = N0 a_k.
// A shape fixes the number of cosine terms (they come first) and other terms at
// compile time.  The merged ("m") shapes serve term lists whose amplitudes are
// constants shared by all histograms and whose cosines share one phase per
// histogram: the amplitudes move into the basis and the terms collapse into
// M = 3 functions (E + the other terms, the cosine parts, the sine parts).
enum Shape : int {
  kShapeGeneric = 0,  // up to 4 terms of any kind, two basis functions per term (M = 9)
  kShapeT1 = 1,       // one cosine term (M = 3)
  kShapeN1 = 2,       // one term without cosine (M = 2)
  kShapeT1N1 = 3,     // cosine + other (M = 4)
  kShapeT2 = 4,       // two cosine terms (M = 5)
  kShapeT2N1 = 5,     // two cosine terms + other (M = 6)
  kShapeT2m = 6,      // merged two cosine terms (M = 3)
  kShapeT2N1m = 7,    // merged two cosine terms + other (M = 3)
  kShapeList = 8,     // no basis form: the term list per bin in FP32 (one histogram per chunk)
  kShapeListS = 9     // the same for at most 2 terms of at most 3 primitives (fewer registers)
};

// A term as given: the product of nprim primitives (FP64 path).
struct RawTerm {
  int nprim;
  int kind[kMaxPrims];
  int slot[kMaxPrims][2];
};

// A term in canonical form (SPLIT path):
//   a * exp(-Lambda t - S t^2 / 2) * [KT(Delta, t) or LKT(a, t)] * [cos(2 pi (nu t + phi / 360))]
// with Lambda the sum of its EXP rates and S the sum of its squared GAUSS widths.
struct CanonTerm {
  int kind;  // kTermPlain, kTermTF, kTermKT, kTermLKT, kTermDKT
  int amp_slot;  // -1: no AMP factor
  int nexp;
  int exp_slot[kMaxPrims];
  int ngauss;
  int gauss_slot[kMaxPrims];
  int kt_slot;   // kTermKT, kTermDKT: Delta; kTermLKT: a
  int nu_slot;   // kTermTF: the frequency; kTermDKT: the fluctuation rate
  int phi_slot;  // kTermTF
  int dkt_term, dkt_prim;  // kTermDKT: the factor's term and primitive in the theory as given
};

// How a SPLIT channel turns into the derivative of one local slot.
enum ContribKind : int {
  // per histogram, from G_m = sum_n u B_m and W = sum_n u (u = d(cost/2)/dN):
  kCN0 = 0,    // d/dN0     = 2 sum_m (Gam_m / N0) G_m
  kCBkg = 1,   // d/dNbkg   = 2 W
  kCAmp = 2,   // d/da_k    = 2 sum over the term's basis functions of (dGam/da_k) G
  kCPhi = 3,   // d/dphi_k  = 2 sum over the term's basis functions of (dGam/dphi_k) G
  // shared by the chunk (time-only), from the per-term channels:
  kCLam = 4,   // d/dlambda = 2 ch_Lambda[k]
  kCSig = 5,   // d/dsigma  = 4 sigma ch_S[k]
  kCNu = 6,    // d/dnu     = 2 ch_nu[k]
  kCDel = 7,   // d/dDelta  = (4/3) Delta ch_Delta[k]
  kCLkt = 8,   // d/da (Lorentzian KT) = (4/3) ch_Delta[k]
  kCDktD = 9,  // d/dDelta (dynamic KT) = 2 ch_Delta[k]
  kCDktN = 10  // d/dnu (dynamic KT)    = 2 ch_nu[k]
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
  // asymmetry data (forward / backward pairs): counts holds the asymmetry a and weights the
  // chi^2 weight w = 1 / sigma_a^2 ([H][stride]; FP64 on the FP64 path, FP32 on the SPLIT
  // path, in the store's type); nullptr for counts
  const void* weights;
  int envelope;  // 1: N0 exp(-t / tau_mu) (1 + A) + Nbkg; 0: the asymmetry model N0 A + Nbkg
  int H;
  int64_t stride;
  double dt_us;
  // theory
  int nterms;
  RawTerm raw[kMaxTerms];
  CanonTerm canon[kMaxTerms];  // SPLIT: cosine terms first
  int shape;
  int merged;                  // SPLIT merged shape: amplitudes folded into the basis
  float bamp[kMaxTerms];       // SPLIT basis amplitude of each term (its constant if merged, else 1)
  int ncontrib;
  Contrib contrib[kMaxContrib];
  // dynamic Kubo-Toyabe sources: map entries of (Delta, nu) of each, and per (histogram,
  // term, primitive) the source index or -1 ([H][kMaxTerms][kMaxPrims]); span of the tables
  int ndkt;
  int2 dkt_src[kMaxDkt];
  const int* dkt_of;
  double dkt_span;
  // parameter map
  const int32_t* map;  // [H][nslots]
  int nslots;
  const double* consts;
  int nconsts;
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

// A work piece of a launch-level partition (SPLIT basis kernels, batches): nit CTA iterations
// of chunk `chunk` of job `job`, from iteration it0 of the chunk, into the job's partial row
// `row`.  Pieces are cut from one contiguous range of the batch's iterations per CTA.
struct Piece {
  int job, chunk, it0, nit, row;
};

struct Job {
  const HistSet* hs;
  const double* params;      // [P]
  double* out;               // [1 + P]
  double* partials;          // [nrows][hs->pstride]
  int nrows;                 // partial rows of this job: hs->nitems, or its pieces' count
  double* colsum;            // [hs->ncols]
  double* chunk_val;         // [hs->nchunks]
  unsigned int* chunk_count; // [hs->nchunks], zero between launches
  unsigned int* counter;     // zero between launches
  int item_begin;            // first global item of this job in the launch
  int mode;                  // 0 chi^2, 1 -2lnL; 2, 3: their Gauss-Newton product (needs dir)
  int grad;                  // 0: value only
  int prec;                  // 0 FP64, 1 SPLIT
  const double* dir;         // [P] direction v of a Gauss-Newton product, else nullptr
  void* dkt;                 // [ndkt][kDktTable] tables of this evaluation (double: FP64 path, float: SPLIT)
  void* dkt_work;            // [ndkt][kDktWork] scratch of the table solve, same type
  unsigned* dkt_count;       // [ndkt] completion counters of the table solve's two grids
  unsigned* dbg;             // checking build: the context's error word (bits of DebugCheck), else nullptr
  // Launch-level partition (read from the launch's first job; nullptr: the decomposition's
  // items): the pieces, CTA b's pieces [piece_cta[b], piece_cta[b + 1]) for b < npiece_ctas,
  // and per chunk of this job its first partial row and row count.
  const Piece* pieces;
  const int* piece_cta;
  int npiece_ctas;
  const int2* chunk_rows;
};

// Index checks of the checking build (compiled with MUSR_DEBUG_CHECKS): a kernel that finds a
// computed index out of its bounds ORs the check's bit into the evaluation's error word and
// skips the access (no trap); musr_debug_word reads the word.
enum DebugCheck : unsigned {
  kDbgRow = 1u,       // a count, weight or staging index beyond the histogram row
  kDbgHist = 2u,      // a histogram index >= H
  kDbgChunk = 4u,     // a chunk or work-item index beyond the decomposition
  kDbgPartial = 8u,   // a partial row beyond the job's rows
  kDbgMap = 16u,      // a parameter-map entry beyond the parameters or constants
  kDbgDkt = 32u,      // a dynamic Kubo-Toyabe source beyond the tables
  kDbgCol = 64u,      // a finalize column beyond the job's columns
  kDbgJob = 128u      // a job index beyond the launch's jobs
};

// Launchers (host side of musr_kernels.cu).  All enqueue on `stream`.
struct LaunchInfo {
  int grid;
  int block;
};
int launch_eval(int precision, int shape, int mode, int grad, const Job* d_jobs, int njobs,
                int total_items, int num_sms, void* stream, LaunchInfo* info);
int max_ctas_per_sm(int precision, int shape, int mode, int grad);
// The dynamic Kubo-Toyabe tables of njobs evaluations of one histogram set (precision 0:
// FP64, 1: FP32), two CTAs per (job, source); enqueued on `stream` before the evaluation.
int launch_dkt_tables(int precision, const Job* d_jobs, int njobs, int ndkt, void* stream);
// Turns raw histogram rows copied to buf ([nhist][stride], dtype as uploaded) into the
// stored image in place: INT32 -> FP32, zero padding beyond nbins; writes seq to *flag
// (host-mapped) if a count is not representable (|INT32| >= 2^24, non-finite float).
int launch_prepare_counts(void* buf, int dtype, int nhist, int64_t nbins, int64_t stride, unsigned* flag,
                          unsigned seq, int num_sms, void* stream);
// The same from packed raw rows ([nhist][nbins]) into img ([nhist][stride]), row h moved
// left by shift[h] >= 0 bins (device array): img[h][j] = raw[h][j + shift[h]] or 0.
// Asymmetry a and chi^2 weight w ([nhist][stride], FP64) of forward / backward pairs from
// packed raw rows (F then B, [nhist][nbins] each), row h moved left by shift[h] bins;
// par = alpha, bkg_f, bkg_b ([3][nhist], device); a32, w32: FP32 copies.  Flags counts the
// store cannot hold.
int launch_prepare_asymmetry(const void* raw, const int64_t* shift, const double* par, int dtype, int nhist,
                             int64_t nbins, int64_t stride, double* a, double* w, float* a32, float* w32,
                             unsigned* flag, unsigned seq, int num_sms, void* stream);
int launch_prepare_counts_shifted(const void* raw, void* img, const int64_t* shift, int dtype, int nhist,
                                  int64_t nbins, int64_t stride, unsigned* flag, unsigned seq, int num_sms,
                                  void* stream);
// Decompositions compiled per precision: tile v holds (bins per CTA iteration) << v
// bins -- SPLIT 512 ... 32768 (the phase-split limit), FP64 256 ... 16384.
constexpr int kVariants = 7;
inline int bins_per_iteration(int precision) { return precision == 1 ? kBlock * kBinsPerThread : kBlock; }

// The decomposition of a launch of nvec evaluations (items[v]: work items of one
// evaluation with decomposition v).  Each CTA of the persistent grid takes
// ceil(items / grid) consecutive items; an item costs its iterations (1 << v for tiles of
// decomposition v) plus a fixed overhead worth item_cost iterations (row reduction,
// completion, staging start-up).  The pick minimises the busiest CTA's time; ties go to
// the smaller tiles.
inline int pick_decomposition(const int* items, int64_t nvec, int grid, double item_cost) {
  int best = 0;
  double best_t = 0.0;
  for (int v = 0; v < kVariants; ++v) {
    const int64_t total = nvec * items[v];
    const int64_t per = (total + grid - 1) / grid;
    const double t = static_cast<double>(per) * (static_cast<double>(1 << v) + item_cost);
    if (v == 0 || t < best_t) {
      best = v;
      best_t = t;
    }
  }
  return best;
}
// Per-item overhead in CTA iterations (measured on GB300), and the persistent grid: the
// SPLIT kernels run two CTAs per SM, the FP64 kernels one.
constexpr double kSplitItemCost = 1.3;
constexpr double kFp64ItemCost = 0.1;
inline int persistent_grid(int precision, int num_sms) { return num_sms * (precision == 1 ? 2 : 1); }
inline int pick_decomposition(const int* items, int64_t nvec, int precision, int num_sms) {
  return pick_decomposition(items, nvec, persistent_grid(precision, num_sms),
                            precision == 1 ? kSplitItemCost : kFp64ItemCost);
}

// Histograms per chunk, and reduction channels per work item, of a SPLIT shape.
int shape_group(int shape);
int shape_channels(int shape);
constexpr int kFp64Channels = 2 + kMaxTerms * kMaxPrims * 2;

}  // namespace musr
