// musr_noalloc.cu -- musr_eval_noalloc: one cost evaluation that allocates no memory.
//
// Some callers cannot allocate device memory at all: code running inside a
// framework that owns every byte of the GPU through its own pool (and forbids
// cudaMalloc behind its back), plugins loaded into a host that pre-reserves
// HBM, or real-time loops where an allocation's implicit synchronisation is not
// allowed.  Such callers cannot create a musr_ctx either, since a context
// allocates its tables and scratch.  This entry point takes everything from the
// caller (device histograms, device parameters, device output; host copies of
// the small configuration) and puts the evaluation's scratch -- work
// decomposition tables, per-item partial rows, per-chunk sums, completion
// counters -- in one file-scope __device__ array of fixed size.
//
// The work decomposition is built as a context builds it for a single evaluation (the
// same grouping of histograms, the same tiles, the same kernels), so for histograms on one
// time grid the result equals musr_eval's for the same inputs and device.  A context also
// moves histograms whose time zeros differ by whole bins onto one grid at upload; the
// borrowed rows here stay as they are, so such histograms form chunks of their own and
// the sums run in another order (equal within the precision's tolerance).
//
// The tables are staged in a host buffer that every call overwrites, and copied from
// there on the caller's stream.  A copy recorded into a CUDA graph would read that
// buffer when the graph is replayed, by then holding another call's tables, so a call
// on a stream that is capturing is refused.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "musr.h"
#include "musr_dev.h"
#include "musr_host.h"
#include "musr_plan.h"

namespace musr {
namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;  // MUSR_NOALLOC_SCRATCH_BYTES
constexpr int kNaMaxHist = 64;
constexpr int kNaMaxParams = 1024;
constexpr int kNaMaxConsts = 256;
constexpr int kNaMaxItems = 8192;
constexpr int kNaMaxCols = kNaMaxHist * kMaxSlots;
constexpr int kMaxDevices = 64;

// The scratch every call on a device shares (held by that device until exit).
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, set up once per device.
void* g_scratch_ptr[kMaxDevices];
std::mutex g_mutex;  // guards the host staging buffer and the set-up

// Host staging of the tables (copied to the scratch on every call).
struct Tables {
  HistSet hs;
  Job job;
  int32_t map[kNaMaxHist * kMaxSlots];
  double consts[kNaMaxConsts];
  Chunk chunks[kNaMaxHist];
  int hist_index[kNaMaxHist];
  int2 items[kNaMaxItems];
  int col_chunk[kNaMaxCols];
  int p_ptr[kNaMaxParams + 1];
  int p_cols[kNaMaxCols];
};
Tables g_tab;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Rejections return MUSR_EINVAL and leave the reason for musr_last_error(NULL).
int na_fail(const char* why) {
  set_thread_error(std::string("musr_eval_noalloc: ") + why);
  return MUSR_EINVAL;
}
int na_cuda(cudaError_t e, const char* what) {
  set_thread_error(std::string("musr_eval_noalloc: ") + what + ": " + cudaGetErrorString(e));
  return MUSR_ECUDA;
}

int64_t tiles_total(const Chunk* ch, int n, int64_t T) {
  int64_t s = 0;
  for (int i = 0; i < n; ++i) s += (ch[i].nhi - ch[i].tile0 + T - 1) / T;
  return s;
}

}  // namespace
}  // namespace musr

using namespace musr;

extern "C" int musr_eval_noalloc(const void* d_counts, int dtype, int nhist, int64_t nbins, int64_t row_stride,
                                 const double* t0, double bin_width_ns, const double fit_range_us[2],
                                 const musr_term* terms, int nterms, const int32_t* map, int nslots, int nparams,
                                 const double* consts, int nconsts, const double* d_params, int mode,
                                 int precision, int with_grad, double* d_out, void* cuda_stream) {
  // ---- argument checks (limits of the fixed scratch)
  if (!d_counts || !t0 || !fit_range_us || !map || !d_params || !d_out || (nterms > 0 && !terms))
    return na_fail("NULL pointer argument");
  if (dtype != MUSR_DTYPE_FP32 && dtype != MUSR_DTYPE_FP64) return na_fail("dtype must be MUSR_DTYPE_FP32 or _FP64");
  if (nhist < 1 || nhist > kNaMaxHist) return na_fail("nhist must be in [1, 64] for musr_eval_noalloc");
  if (nbins < 1 || nbins >= (int64_t(1) << 30)) return na_fail("nbins must be in [1, 2^30)");
  if (row_stride < nbins || row_stride % 4 != 0) return na_fail("row_stride must be >= nbins and a multiple of 4");
  if (reinterpret_cast<uintptr_t>(d_counts) % 16 != 0) return na_fail("d_counts must be 16-byte aligned");
  if (nslots < 2 || nslots > MUSR_MAX_SLOTS) return na_fail("nslots must be in [2, 32]");
  if (nparams < 0 || nparams > kNaMaxParams) return na_fail("nparams must be in [0, 1024] for musr_eval_noalloc");
  if (nconsts < 0 || nconsts > kNaMaxConsts || (nconsts > 0 && !consts))
    return na_fail("nconsts must be in [0, 256] for musr_eval_noalloc");
  if (nterms < 0 || nterms > MUSR_MAX_TERMS) return na_fail("nterms must be in [0, 4]");
  if (mode != MUSR_CHI2 && mode != MUSR_MLE) return na_fail("mode must be MUSR_CHI2 or MUSR_MLE");
  if (precision != MUSR_FP64 && precision != MUSR_SPLIT) return na_fail("precision must be MUSR_FP64 or MUSR_SPLIT");
  if (!(bin_width_ns > 0.0) || !std::isfinite(bin_width_ns)) return na_fail("bin_width_ns must be finite and > 0");
  if (!std::isfinite(fit_range_us[0]) || !std::isfinite(fit_range_us[1]) || fit_range_us[0] > fit_range_us[1])
    return na_fail("fit range must be finite with lo <= hi");
  for (int k = 0; k < nterms; ++k) {
    if (terms[k].nprim < 1 || terms[k].nprim > MUSR_MAX_PRIMS) return na_fail("a term needs 1..4 primitives");
    for (int m = 0; m < terms[k].nprim; ++m) {
      if (terms[k].kind[m] == MUSR_PRIM_DKT)
        return na_fail("the dynamic Kubo-Toyabe primitive needs tables solved per evaluation: use a context");
      if (terms[k].kind[m] < MUSR_PRIM_AMP || terms[k].kind[m] > MUSR_PRIM_BESSEL) return na_fail("unknown primitive");
      for (int q = 0; q < prim_nslots(terms[k].kind[m]); ++q)
        if (terms[k].slot[m][q] < 0 || terms[k].slot[m][q] >= nslots) return na_fail("slot index out of range");
    }
  }
  for (int i = 0; i < nhist * nslots; ++i)
    if (map[i] >= nparams || (map[i] < 0 && -1 - map[i] >= nconsts)) return na_fail("map entry out of range");
  for (int h = 0; h < nhist; ++h)
    if (!std::isfinite(t0[h])) return na_fail("t0 must be finite");

  set_thread_error("");
  std::lock_guard<std::mutex> lock(g_mutex);
  // ---- tables (same decomposition as a context's single evaluation); host work only
  Tables& T = g_tab;
  HistSet& hs = T.hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.store = dtype == MUSR_DTYPE_FP64 ? kStoreF64 : kStoreF32;
  hs.envelope = 1;  // histograms of counts (Eq. positron_histo)
  hs.H = nhist;
  hs.stride = row_stride;
  hs.dt_us = bin_width_ns / 1000.0;
  hs.nterms = nterms;
  hs.nslots = nslots;
  hs.P = nparams;
  hs.nconsts = nconsts;
  for (int k = 0; k < nterms; ++k) {
    hs.raw[k].nprim = terms[k].nprim;
    for (int m = 0; m < kMaxPrims; ++m) {
      hs.raw[k].kind[m] = m < terms[k].nprim ? terms[k].kind[m] : 0;
      hs.raw[k].slot[m][0] = m < terms[k].nprim ? terms[k].slot[m][0] : 0;
      hs.raw[k].slot[m][1] = m < terms[k].nprim && prim_nslots(terms[k].kind[m]) == 2 ? terms[k].slot[m][1] : 0;
    }
  }
  int nlo[kNaMaxHist], nhi[kNaMaxHist];
  for (int h = 0; h < nhist; ++h) fit_bins(t0[h], hs.dt_us, nbins, fit_range_us[0], fit_range_us[1], &nlo[h], &nhi[h]);
  int group_of[kNaMaxHist];
  int ngroups = 0;
  int group_cap = 1;
  // Theories without a basis form evaluate their term list per bin in FP32 (one histogram
  // per chunk), as a context does.
  const bool basis = precision == MUSR_SPLIT && !plan_split(terms, nterms, map, nhist, nslots, consts, &hs);
  if (precision == MUSR_SPLIT && !basis) {
    bool small = nterms <= 2;
    for (int k = 0; k < nterms; ++k) small = small && terms[k].nprim <= 3;
    hs.shape = small ? kShapeListS : kShapeList;
  }
  if (basis) {
    group_cap = shape_group(hs.shape);
    // Group histograms sharing t0 (to 2^-24 bins), the fit window and every time-dependent
    // parameter, in order of first appearance: the key a context builds.
    int64_t keys[kNaMaxHist][6 + 2 * MUSR_MAX_TERMS * 10];
    int keylen[kNaMaxHist];
    for (int h = 0; h < nhist; ++h) {
      int n = 0;
      const double q = std::nearbyint(t0[h] * 16777216.0);
      if (std::fabs(q) < 4e18) {
        keys[h][n++] = 0;
        keys[h][n++] = static_cast<int64_t>(q);
      } else {
        int64_t tb;
        std::memcpy(&tb, &t0[h], sizeof(tb));
        keys[h][n++] = 1;
        keys[h][n++] = tb;
      }
      keys[h][n++] = nlo[h];
      keys[h][n++] = nhi[h];
      auto push = [&](int s) {
        const int32_t m = map[h * nslots + s];
        if (m >= 0) {
          keys[h][n++] = 0;
          keys[h][n++] = m;
        } else {
          int64_t bits;
          std::memcpy(&bits, &consts[-1 - m], sizeof(bits));
          keys[h][n++] = 1;
          keys[h][n++] = bits;
        }
      };
      for (int k = 0; k < nterms; ++k) {
        const CanonTerm& ct = hs.canon[k];
        for (int i = 0; i < ct.nexp; ++i) push(ct.exp_slot[i]);
        for (int i = 0; i < ct.ngauss; ++i) push(ct.gauss_slot[i]);
        if (ct.kind == kTermKT || ct.kind == kTermLKT) push(ct.kt_slot);
        if (ct.kind == kTermTF) push(ct.nu_slot);
      }
      keylen[h] = n;
      group_of[h] = -1;
      for (int g = 0; g < h && group_of[h] < 0; ++g) {
        if (keylen[g] != n || group_of[g] < 0) continue;
        bool eq = true;
        for (int i = 0; i < n && eq; ++i) eq = keys[g][i] == keys[h][i];
        // the first histogram of an existing group with this key
        if (eq) group_of[h] = group_of[g];
      }
      if (group_of[h] < 0) group_of[h] = ngroups++;
    }
  } else {
    for (int h = 0; h < nhist; ++h) group_of[h] = h;
    ngroups = nhist;
  }
  // Chunks (skipping histograms without a bin in the fit range).
  int nchunks = 0, nidx = 0;
  for (int g = 0; g < ngroups; ++g) {
    int members[kNaMaxHist], nm = 0;
    for (int h = 0; h < nhist; ++h)
      if (group_of[h] == g) members[nm++] = h;
    for (int i = 0; i < nm; i += group_cap) {
      if (nhi[members[i]] <= nlo[members[i]]) continue;
      Chunk& ch = T.chunks[nchunks++];
      std::memset(&ch, 0, sizeof(ch));
      ch.first = nidx;
      ch.nh = nm - i < group_cap ? nm - i : group_cap;
      for (int j = 0; j < ch.nh; ++j) T.hist_index[nidx++] = members[i + j];
      ch.nlo = nlo[members[i]];
      ch.nhi = nhi[members[i]];
      ch.t0 = t0[members[i]];
      ch.tile0 = ch.nlo & ~3;
    }
  }
  // ---- device set-up: once per device, with that device current (the first call on a
  // device looks up the scratch array's address; with lazy module loading, that is also
  // when the library's module, and with it the array, is loaded onto the device)
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return na_cuda(e, "cudaStreamIsCapturing");
  if (cap != cudaStreamCaptureStatusNone)
    return na_fail("cuda_stream is capturing: the tables are staged in a host buffer that later calls "
                   "overwrite, so a recorded copy would read another call's tables");
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_cuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return na_fail("device index beyond 63");
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return na_cuda(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_ptr[dev] = ptr;
  }
  unsigned char* scratch = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  int num_sms = 1;
  e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return na_cuda(e, "cudaDeviceGetAttribute");

  if (nchunks == 0) {  // no bin in the fit range
    e = cudaMemsetAsync(d_out, 0, sizeof(double) * (1 + nparams), stream);
    return e == cudaSuccess ? MUSR_OK : na_cuda(e, "cudaMemsetAsync(out)");
  }
  // The decomposition a context picks for one evaluation.
  int items_per_var[kVariants];
  for (int v = 0; v < kVariants; ++v)
    items_per_var[v] = static_cast<int>(tiles_total(T.chunks, nchunks, int64_t(bins_per_iteration(precision)) << v));
  hs.tile_bins = bins_per_iteration(precision) << pick_decomposition(items_per_var, 1, precision, num_sms);
  const int64_t nitems64 = tiles_total(T.chunks, nchunks, hs.tile_bins);
  if (nitems64 > kNaMaxItems) return na_fail("problem needs more than 8192 work items (too many bins for musr_eval_noalloc)");
  int nitems = 0, col = 0;
  for (int ci = 0; ci < nchunks; ++ci) {
    Chunk& ch = T.chunks[ci];
    ch.item0 = nitems;
    ch.ntiles = static_cast<int>((ch.nhi - ch.tile0 + hs.tile_bins - 1) / hs.tile_bins);
    for (int t = 0; t < ch.ntiles; ++t) T.items[nitems++] = make_int2(ci, t);
    ch.col0 = col;
    col += ch.nh * nslots;
  }
  hs.group = group_cap;
  hs.nch = precision == MUSR_SPLIT ? shape_channels(hs.shape) : kFp64Channels;
  hs.pstride = 1 + hs.nch;
  hs.ncols = col;
  hs.nchunks = nchunks;
  hs.nitems = nitems;
  // CSR: parameter -> columns, in column order.
  int count[kNaMaxParams + 1];
  for (int p = 0; p <= nparams; ++p) count[p] = 0;
  for (int ci = 0; ci < nchunks; ++ci)
    for (int hl = 0; hl < T.chunks[ci].nh; ++hl)
      for (int s = 0; s < nslots; ++s) {
        const int cc = T.chunks[ci].col0 + hl * nslots + s;
        T.col_chunk[cc] = ci;
        const int32_t m = map[T.hist_index[T.chunks[ci].first + hl] * nslots + s];
        if (m >= 0) ++count[m];
      }
  T.p_ptr[0] = 0;
  for (int p = 0; p < nparams; ++p) T.p_ptr[p + 1] = T.p_ptr[p] + count[p];
  for (int p = 0; p < nparams; ++p) count[p] = T.p_ptr[p];
  for (int cc = 0; cc < col; ++cc) {
    const Chunk& ch = T.chunks[T.col_chunk[cc]];
    const int local = cc - ch.col0, hl = local / nslots, s = local - hl * nslots;
    const int32_t m = map[T.hist_index[ch.first + hl] * nslots + s];
    if (m >= 0) T.p_cols[count[m]++] = cc;
  }
  std::memcpy(T.map, map, sizeof(int32_t) * nhist * nslots);
  for (int i = 0; i < nconsts; ++i) T.consts[i] = consts[i];

  // ---- scratch layout: [tables][partials][colsum][chunk_val][chunk_count][counter]
  const size_t tab_bytes = align256(sizeof(Tables));
  const size_t part_bytes = align256(sizeof(double) * size_t(nitems) * hs.pstride);
  const size_t cols_bytes = align256(sizeof(double) * size_t(col > 0 ? col : 1));
  const size_t cval_bytes = align256(sizeof(double) * size_t(nchunks));
  const size_t zero_bytes = align256(sizeof(unsigned) * size_t(nchunks + 1));
  const size_t total = tab_bytes + part_bytes + cols_bytes + cval_bytes + zero_bytes;
  if (total > kScratchBytes) return na_fail("problem exceeds the 8 MiB scratch of musr_eval_noalloc");
  unsigned char* d_tab = scratch;
  double* d_part = reinterpret_cast<double*>(scratch + tab_bytes);
  double* d_cols = reinterpret_cast<double*>(scratch + tab_bytes + part_bytes);
  double* d_cval = reinterpret_cast<double*>(scratch + tab_bytes + part_bytes + cols_bytes);
  unsigned* d_zero = reinterpret_cast<unsigned*>(scratch + tab_bytes + part_bytes + cols_bytes + cval_bytes);
  const Tables* dT = reinterpret_cast<const Tables*>(d_tab);
  hs.counts = d_counts;
  hs.map = dT->map;
  hs.consts = dT->consts;
  hs.chunks = dT->chunks;
  hs.hist_index = dT->hist_index;
  hs.items = dT->items;
  hs.col_chunk = dT->col_chunk;
  hs.p_ptr = dT->p_ptr;
  hs.p_cols = dT->p_cols;
  Job& job = T.job;
  std::memset(&job, 0, sizeof(job));
  job.hs = &dT->hs;
  job.params = d_params;
  job.out = d_out;
  job.partials = d_part;
  job.nrows = nitems;
  job.colsum = d_cols;
  job.chunk_val = d_cval;
  job.chunk_count = d_zero;
  job.counter = d_zero + nchunks;
  job.item_begin = 0;
  job.mode = mode;
  job.grad = with_grad ? 1 : 0;
  job.prec = precision;

  // Pageable source: the copy has consumed the staging buffer when the call returns.
  e = cudaMemcpyAsync(d_tab, &T, sizeof(Tables), cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return na_cuda(e, "cudaMemcpyAsync(tables)");
  // The completion counters must start at zero; the previous call's values stay otherwise.
  e = cudaMemsetAsync(d_zero, 0, sizeof(unsigned) * (nchunks + 1), stream);
  if (e != cudaSuccess) return na_cuda(e, "cudaMemsetAsync(counters)");
  LaunchInfo info;
  if (launch_eval(precision, hs.shape, mode, job.grad, &dT->job, 1, nitems, num_sms, cuda_stream, &info))
    return na_cuda(cudaGetLastError(), "kernel launch");
  return MUSR_OK;
}
