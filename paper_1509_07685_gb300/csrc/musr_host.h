// musr_host.h -- the context object behind the opaque musr_ctx of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <set>
#include <mutex>
#include <string>
#include <vector>

#include "musr.h"
#include "musr_dev.h"

namespace musr {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  bool from_arena = false;
};

// A device memory arena: one cudaMalloc of the HBM budget, carved best-fit in
// 256-byte units.  Allocation fails (nullptr) when no free range is large enough,
// which is how the serving loop admits fits by budget.  Thread-safe.
class Arena {
 public:
  ~Arena();
  int init(size_t bytes);  // MUSR_OK / MUSR_ENOMEM
  void* alloc(size_t bytes);
  void release(void* p);
  size_t capacity() const { return cap_; }
  size_t used() const;

 private:
  void insert_free(size_t off, size_t size);
  void erase_free(std::map<size_t, size_t>::iterator it);

  char* base_ = nullptr;
  size_t cap_ = 0, used_ = 0;
  // Free ranges twice: by offset (to merge neighbours on release) and by (size, offset)
  // (best fit in O(log n): the smallest range that holds the request, lowest offset first).
  std::map<size_t, size_t> free_;              // offset -> size
  std::set<std::pair<size_t, size_t>> by_size_;  // (size, offset)
  std::map<size_t, size_t> live_;              // offset -> size
  mutable std::mutex mu_;
};

// The theory and map of one precision, compiled to a work decomposition.
// The tables are planned on the host when the map is set and copied to the
// device (one allocation, one copy) the first time a launch needs them.
struct Compiled {
  bool planned = false;  // compile() has run since the map was set
  bool valid = false;
  std::string reason;  // why this precision is unavailable (valid == false)
  HistSet hs{};        // host copy (device pointers inside once uploaded)
  std::vector<Chunk> chunks;
  std::vector<int2> items;
  std::vector<int> hist_index, col_chunk, p_ptr, p_cols;
  std::vector<int> dkt_of;  // [H][kMaxTerms][kMaxPrims] dynamic Kubo-Toyabe source or -1
  bool uploaded = false;
  DevBuf tables;        // HistSet + all tables + map + consts, 256-byte aligned pieces
  std::vector<char> blob;  // host image of `tables`, the source of their copy
  const HistSet* d_hs = nullptr;
};

// Buffers of the eval entry points and the cached job table of the last launch.
struct EvalBufs {
  DevBuf params, out, partials, colsum, chunk_val, chunk_count, counters, jobs, dirs;
  DevBuf dkt, dkt_work;  // dynamic Kubo-Toyabe tables and their solve's scratch, per evaluation
  DevBuf dkt_count;      // their completion counters (zeroed once; each solve adds 2)
  DevBuf part;           // a launch-level partition: chunk rows, CTA offsets, pieces
  double* h_in = nullptr;
  double* h_out = nullptr;
  size_t h_in_bytes = 0, h_out_bytes = 0;
  bool key_valid = false;
  int k_prec = -1, k_var = -1, k_mode = -1, k_grad = -1, k_nvec = -1;
  const double* k_params = nullptr;
  const double* k_dirs = nullptr;
  bool k_pieces = false;
  int k_grid = 0;  // the partition's grid (k_pieces)
  double* k_out = nullptr;
};

// RAII: make `dev` current, restore the caller's device on exit.
class DeviceScope {
 public:
  explicit DeviceScope(int dev);
  ~DeviceScope();

 private:
  int prev_ = 0;
};

int fail(musr_ctx* ctx, int code, const std::string& msg);
// The calling thread's error text for calls without a context (musr_last_error(NULL)).
void set_thread_error(const std::string& msg);
int cuda_fail(musr_ctx* ctx, cudaError_t e, const char* what);
int dalloc(musr_ctx* ctx, DevBuf& b, size_t bytes);
void dfree(musr_ctx* ctx, DevBuf& b);
void fit_bins(double t0, double dt_us, int64_t B, double lo, double hi, int* nlo, int* nhi);
int wait_stream(musr_ctx* ctx, int timeout_ms);
int check_ready(musr_ctx* ctx, int mode, int prec);
// Plans one decomposition the first time a launch needs it (host work only).
int ensure_compiled(musr_ctx* ctx, int prec, int var);
// Evaluation buffers of a context for nvec vectors of one decomposition, and the
// job descriptors of such a launch (written to `jobs`, items numbered from
// item_begin).  Used by the context's own launches and by the serving loop.
int ensure_eval(musr_ctx* ctx, int prec, int var, int nvec);
// Reads the device check of the last histogram upload once the stream it ran on has
// finished: MUSR_EINVAL (and no histograms) if a count was not representable.  Uploads
// made with setup_stream set leave the check for the caller to read.
int finish_upload_check(musr_ctx* ctx);
void fill_jobs(musr_ctx* ctx, int prec, int var, int mode, int grad, int nvec, const double* d_params,
               double* d_out, Job* jobs, int item_begin, const double* d_dirs = nullptr);

}  // namespace musr

struct musr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 1;
  size_t budget = 0, used = 0;
  std::string err;
  // histograms
  bool have_hist = false;
  musr::DevBuf counts_own;
  const void* d_counts = nullptr;
  int store = musr::kStoreF32;
  int H = 0;
  int64_t B = 0, stride = 0;
  std::vector<double> t0;
  double bin_width_ns = 0.0, dt_us = 0.0, lo = 0.0, hi = 0.0;
  std::vector<int> nlo, nhi;
  // theory
  bool have_theory = false;
  std::vector<musr_term> terms;
  // parameter map
  bool have_map = false;
  std::vector<int32_t> map;
  int nslots = 0, P = 0;
  std::string split_reason;  // why the theory has no basis form (empty: it has); SPLIT then
                             // evaluates the term list per bin (list_item)
  std::vector<double> consts;
  // [precision][decomposition]: tiles of (bins per CTA iteration) << v bins; a
  // launch picks the largest that still fills the GPU (pick_decomposition).
  musr::Compiled comp[2][musr::kVariants];
  musr::EvalBufs ev;
  musr::DevBuf dbg_word;  // checking build: the error word of the kernels' index checks
  int last_grid = 0;
  musr::Arena* arena = nullptr;  // when set, device memory comes from it (serving)
  // Stream of one-time setup work (histogram copy and check, tables, zeroed buffers);
  // null: the histogram upload waits on the calling thread's stream and the rest goes
  // on `stream`.  The serving loop sets it while it configures a fit, then waits once.
  cudaStream_t setup_stream = nullptr;
  // Set by an owner that has already waited for all of this context's device work (the
  // serving loop, which shares one stream among many contexts): destroy does not wait.
  bool owner_waited = false;
  // Device check of the last histogram upload, not read yet (see finish_upload_check).
  const unsigned* check_flag = nullptr;
  musr::DevBuf upload_scratch;     // packed rows of a shifted upload, until the check is read
  // asymmetry data (musr_upload_asymmetry): d_counts holds a, weights_own the chi^2 weights
  bool asym = false;
  musr::DevBuf weights_own;
  musr::DevBuf asym32_own;         // FP32 a and w ([2][H][stride]) for the SPLIT path
  std::vector<double> asym_par;    // alpha, bkg_f, bkg_b of the pairs, the source of their copy
  std::vector<int64_t> shift;      // whole bins each histogram's row moved left on the device
  unsigned check_seq = 0;
  int check_dtype = 0;
};
