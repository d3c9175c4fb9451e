// musr_ctx.cpp -- host side of the libmusr C ABI (include/musr.h).
//
// The context owns the device copies of the histograms (uploaded once, as the
// offload of Section 4 does), the compiled theory/map of each precision (work
// decomposition, finalize tables) and the per-evaluation buffers.  Every step
// of the cost runs in the kernels of musr_kernels.cu; this file validates
// arguments, lays out memory, builds the work decomposition and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "musr.h"
#include "musr_dev.h"
#include "musr_host.h"
#include "musr_partition.h"
#include "musr_plan.h"

using musr::Chunk;
using musr::HistSet;
using musr::Job;

namespace {

thread_local std::string g_create_error;

constexpr int64_t kRowAlign = 64;  // elements: rows start on 256-byte boundaries (FP32)

}  // namespace

namespace musr {

int fail(musr_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

void set_thread_error(const std::string& msg) { g_create_error = msg; }

int cuda_fail(musr_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, MUSR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

Arena::~Arena() {
  if (base_) cudaFree(base_);
}

int Arena::init(size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (cudaMalloc(reinterpret_cast<void**>(&base_), bytes) != cudaSuccess) {
    cudaGetLastError();
    base_ = nullptr;
    return MUSR_ENOMEM;
  }
  cap_ = bytes;
  free_.clear();
  by_size_.clear();
  live_.clear();
  insert_free(0, bytes);
  used_ = 0;
  return MUSR_OK;
}

void Arena::insert_free(size_t off, size_t size) {
  free_[off] = size;
  by_size_.insert({size, off});
}

void Arena::erase_free(std::map<size_t, size_t>::iterator it) {
  by_size_.erase({it->second, it->first});
  free_.erase(it);
}

void* Arena::alloc(size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  std::lock_guard<std::mutex> lock(mu_);
  const auto best = by_size_.lower_bound({bytes, 0});
  if (best == by_size_.end()) return nullptr;
  const size_t off = best->second, rest = best->first - bytes;
  erase_free(free_.find(off));
  if (rest) insert_free(off + bytes, rest);
  live_[off] = bytes;
  used_ += bytes;
  return base_ + off;
}

void Arena::release(void* p) {
  std::lock_guard<std::mutex> lock(mu_);
  const size_t off = static_cast<size_t>(static_cast<char*>(p) - base_);
  auto it = live_.find(off);
  if (it == live_.end()) return;
  size_t start = off, size = it->second;
  used_ -= size;
  live_.erase(it);
  auto next = free_.lower_bound(start);
  if (next != free_.end() && next->first == start + size) {  // merge with the following range
    size += next->second;
    erase_free(next);
  }
  auto prev = free_.lower_bound(start);
  if (prev != free_.begin()) {
    --prev;
    if (prev->first + prev->second == start) {  // merge with the preceding range
      start = prev->first;
      size += prev->second;
      erase_free(prev);
    }
  }
  insert_free(start, size);
}

size_t Arena::used() const {
  std::lock_guard<std::mutex> lock(mu_);
  return used_;
}

int dalloc(musr_ctx* ctx, DevBuf& b, size_t bytes) {
  dfree(ctx, b);
  if (bytes == 0) bytes = 16;
  if (ctx->arena) {
    b.p = ctx->arena->alloc(bytes);
    if (!b.p) return fail(ctx, MUSR_ENOMEM, "device memory budget exceeded (serving arena full)");
    b.bytes = bytes;
    b.from_arena = true;
    ctx->used += bytes;
    return MUSR_OK;
  }
  if (ctx->budget && ctx->used + bytes > ctx->budget)
    return fail(ctx, MUSR_ENOMEM, "device memory budget exceeded (" + std::to_string(ctx->used + bytes) +
                                      " > " + std::to_string(ctx->budget) + " bytes)");
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    cudaGetLastError();
    return fail(ctx, MUSR_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  b.bytes = bytes;
  ctx->used += bytes;
  return MUSR_OK;
}

void dfree(musr_ctx* ctx, DevBuf& b) {
  if (b.p) {
    if (b.from_arena)
      ctx->arena->release(b.p);
    else
      cudaFree(b.p);
    ctx->used -= b.bytes;
  }
  b.p = nullptr;
  b.bytes = 0;
  b.from_arena = false;
}

// Host -> device copy on the calling thread's own stream, complete on return.  Uploads
// from several threads (the serving loop admits fits in parallel) then overlap instead of
// queueing on the legacy default stream, and never wait for a context's evaluations.
cudaError_t copy_h2d(void* dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cudaStreamPerThread);
  return e == cudaSuccess ? cudaStreamSynchronize(cudaStreamPerThread) : e;
}

// A host-mapped word per thread that device-side checks of an upload write to: each check
// gets a new sequence number, so a word left from an earlier upload never matches.
struct CheckFlag {
  unsigned* host = nullptr;
  unsigned* dev = nullptr;
  unsigned seq = 0;
  ~CheckFlag() {
    if (host) cudaFreeHost(host);
  }
  bool ready() {
    if (host) return true;
    void* p = nullptr;
    if (cudaHostAlloc(&p, 64, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) return false;
    host = static_cast<unsigned*>(p);
    *host = 0;
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) {
      cudaFreeHost(p);
      host = nullptr;
      return false;
    }
    dev = static_cast<unsigned*>(d);
    return true;
  }
  unsigned next() { return ++seq == 0 ? ++seq : seq; }
  bool raised(unsigned s) const { return *static_cast<volatile unsigned*>(host) == s; }
};
thread_local CheckFlag tl_flag;

// A pinned staging buffer of the calling thread for uploads made with setup_stream set (the
// serving loop's helper threads).  Copies from pageable memory go through the driver's own
// staging, which concurrent threads share; each helper instead copies the rows into its own
// pinned buffer (host memcpy, in parallel on the host cores) and the device reads them from
// there asynchronously.  The helper waits for its stream before its next upload, so the
// buffer is free again by then.  Requests larger than kMaxBounce take the pageable copy.
struct Bounce {
  static constexpr size_t kMaxBounce = size_t(256) << 20;
  void* p = nullptr;
  size_t cap = 0;
  ~Bounce() {
    if (p) cudaFreeHost(p);
  }
  void* get(size_t bytes) {
    if (bytes > kMaxBounce) return nullptr;
    if (bytes <= cap) return p;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max(bytes, size_t(16) << 20);
    if (cudaHostAlloc(&p, want, cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return nullptr;
    }
    cap = want;
    return p;
  }
};
thread_local Bounce tl_bounce;

// The host rows `counts` ([nhist][nbins] of esz bytes) as the source of an asynchronous copy:
// the thread's pinned staging buffer when the upload is a serving helper's, else as given.
const void* stage_rows(musr_ctx* ctx, const void* counts, size_t bytes) {
  if (!ctx->setup_stream) return counts;
  void* b = tl_bounce.get(bytes);
  if (!b) return counts;
  std::memcpy(b, counts, bytes);
  return b;
}

DeviceScope::DeviceScope(int dev) {
  cudaGetDevice(&prev_);
  if (prev_ != dev) cudaSetDevice(dev);
}
DeviceScope::~DeviceScope() {
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != prev_) cudaSetDevice(prev_);
}

// Bins [nlo, nhi) of a histogram whose times t_n = (n - t0) * dt satisfy lo <= t_n <= hi.
void fit_bins(double t0, double dt_us, int64_t B, double lo, double hi, int* nlo, int* nhi) {
  auto tn = [&](int64_t n) { return (static_cast<double>(n) - t0) * dt_us; };
  auto first_at_least = [&](double v) -> int64_t {  // first n with t_n >= v
    double est = std::ceil(v / dt_us + t0);
    int64_t n = est < 0 ? 0 : (est > static_cast<double>(B) ? B : static_cast<int64_t>(est));
    while (n > 0 && tn(n - 1) >= v) --n;
    while (n < B && tn(n) < v) ++n;
    return n;
  };
  auto first_above = [&](double v) -> int64_t {  // first n with t_n > v
    double est = std::floor(v / dt_us + t0) + 1.0;
    int64_t n = est < 0 ? 0 : (est > static_cast<double>(B) ? B : static_cast<int64_t>(est));
    while (n > 0 && tn(n - 1) > v) --n;
    while (n < B && tn(n) <= v) ++n;
    return n;
  };
  int64_t a = first_at_least(lo), b = first_above(hi);
  if (b < a) b = a;
  *nlo = static_cast<int>(a);
  *nhi = static_cast<int>(b);
}

// Whole-bin shifts that put histograms on a common time grid: histogram h moves left by
// floor(t0_h) - min_h floor(t0_h) bins (histograms whose t0 have equal fractions then
// share t0), never past its first bin in the fit window (no fitted bin is dropped).
// Histograms without a bin in the window stay.
std::vector<int64_t> grid_shifts(const musr_ctx* ctx) {
  std::vector<int64_t> shift(ctx->H, 0);
  double fmin = 0.0;
  bool any = false;
  for (int h = 0; h < ctx->H; ++h)
    if (ctx->nhi[h] > ctx->nlo[h]) {
      const double f = std::floor(ctx->t0[h]);
      fmin = any ? std::min(fmin, f) : f;
      any = true;
    }
  for (int h = 0; h < ctx->H && any; ++h)
    if (ctx->nhi[h] > ctx->nlo[h]) {
      const double d = std::floor(ctx->t0[h]) - fmin;  // >= 0
      shift[h] = std::min<int64_t>(d < 1e18 ? static_cast<int64_t>(d) : ctx->nlo[h], ctx->nlo[h]);
    }
  return shift;
}

void free_compiled(musr_ctx* ctx, Compiled& c) {
  dfree(ctx, c.tables);
  std::vector<char>().swap(c.blob);
  c.d_hs = nullptr;
  c.uploaded = false;
  c.chunks.clear();
  c.items.clear();
  c.hist_index.clear();
  c.col_chunk.clear();
  c.p_ptr.clear();
  c.p_cols.clear();
  c.dkt_of.clear();
  c.valid = false;
  c.planned = false;
  c.reason.clear();
}

// Builds the decomposition and finalize tables of one precision and one
// decomposition (0: tiles small enough that one evaluation fills the GPU;
// 1: the largest tiles, for batched launches).
int compile(musr_ctx* ctx, int prec, int var) {
  Compiled& c = ctx->comp[prec][var];
  free_compiled(ctx, c);
  HistSet hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.counts = ctx->d_counts;
  hs.store = ctx->store;
  hs.weights = ctx->asym ? ctx->weights_own.p : nullptr;
  hs.envelope = ctx->asym ? 0 : 1;
  if (ctx->asym && prec == MUSR_SPLIT) {  // FP32 copies: a staged like counts, w beside it
    hs.counts = ctx->asym32_own.p;
    hs.store = kStoreF32;
    hs.weights = static_cast<const float*>(ctx->asym32_own.p) + static_cast<size_t>(ctx->H) * ctx->stride;
  }
  hs.H = ctx->H;
  hs.stride = ctx->stride;
  hs.dt_us = ctx->dt_us;
  hs.nterms = static_cast<int>(ctx->terms.size());
  hs.nslots = ctx->nslots;
  hs.P = ctx->P;  // map and consts: device copies in the tables (ensure_uploaded)
  hs.nconsts = static_cast<int>(ctx->consts.size());
  for (int k = 0; k < hs.nterms; ++k) {
    const musr_term& t = ctx->terms[k];
    hs.raw[k].nprim = t.nprim;
    for (int m = 0; m < musr::kMaxPrims; ++m) {
      hs.raw[k].kind[m] = m < t.nprim ? t.kind[m] : 0;
      hs.raw[k].slot[m][0] = m < t.nprim ? t.slot[m][0] : 0;
      hs.raw[k].slot[m][1] = m < t.nprim && musr::prim_nslots(t.kind[m]) == 2 ? t.slot[m][1] : 0;
    }
  }
  const int H = ctx->H;
  // Dynamic Kubo-Toyabe sources: the distinct (Delta, nu) map entries of every DKT factor.
  std::vector<int> dkt_of(static_cast<size_t>(H) * musr::kMaxTerms * musr::kMaxPrims, -1);
  hs.ndkt = 0;
  for (int h = 0; h < H; ++h)
    for (int k = 0; k < hs.nterms; ++k)
      for (int m = 0; m < ctx->terms[k].nprim; ++m) {
        if (ctx->terms[k].kind[m] != MUSR_PRIM_DKT) continue;
        const int32_t* row = ctx->map.data() + static_cast<size_t>(h) * ctx->nslots;
        const int2 key = make_int2(row[ctx->terms[k].slot[m][0]], row[ctx->terms[k].slot[m][1]]);
        int src = -1;
        for (int q = 0; q < hs.ndkt && src < 0; ++q)
          if (hs.dkt_src[q].x == key.x && hs.dkt_src[q].y == key.y) src = q;
        if (src < 0 && hs.ndkt < musr::kMaxDkt) {
          src = hs.ndkt++;
          hs.dkt_src[src] = key;
        }
        dkt_of[(static_cast<size_t>(h) * musr::kMaxTerms + k) * musr::kMaxPrims + m] = src;
      }
  // the tables span the last in-fit time of every histogram
  hs.dkt_span = 0.0;
  for (int h = 0; h < H; ++h)
    if (ctx->nhi[h] > ctx->nlo[h])
      hs.dkt_span = std::max(hs.dkt_span, (static_cast<double>(ctx->nhi[h] - 1) - ctx->t0[h]) * ctx->dt_us);
  std::vector<std::vector<int>> groups;
  int group_cap = 1;
  const bool basis = prec == MUSR_SPLIT &&
                     !musr::plan_split(ctx->terms.data(), hs.nterms, ctx->map.data(), H, ctx->nslots,
                                       ctx->consts.data(), &hs, !ctx->asym);
  if (prec == MUSR_SPLIT && !basis) {  // the term list per bin in FP32
    bool small = hs.nterms <= 2;
    for (int k = 0; k < hs.nterms; ++k) small = small && ctx->terms[k].nprim <= 3;
    hs.shape = small ? musr::kShapeListS : musr::kShapeList;
  }
  if (basis) {
    group_cap = musr::shape_group(hs.shape);
    // Group histograms that share t0, the fit window and every time-dependent parameter.
    std::map<std::vector<int64_t>, int> key_to_group;
    // A slot's identity across histograms: the global parameter, or the constant's value.
    auto push_entry = [&](std::vector<int64_t>& key, int h, int s) {
      const int32_t m = ctx->map[static_cast<size_t>(h) * ctx->nslots + s];
      if (m >= 0) {
        key.push_back(0);
        key.push_back(m);
      } else {
        const double v = ctx->consts[-1 - m];
        int64_t bits;
        std::memcpy(&bits, &v, sizeof(bits));
        key.push_back(1);
        key.push_back(bits);
      }
    };
    for (int h = 0; h < H; ++h) {
      std::vector<int64_t> key;
      int64_t tb;
      // t0 to 2^-24 bins: a smaller difference in time zero (below 2^-24 bin widths in
      // every time) is far below the FP32 resolution of the shared per-bin factors
      const double q = std::nearbyint(ctx->t0[h] * 16777216.0);
      if (std::fabs(q) < 4e18) {
        key.push_back(0);
        key.push_back(static_cast<int64_t>(q));
      } else {
        std::memcpy(&tb, &ctx->t0[h], sizeof(tb));
        key.push_back(1);
        key.push_back(tb);
      }
      key.push_back(ctx->nlo[h]);
      key.push_back(ctx->nhi[h]);
      for (int k = 0; k < hs.nterms; ++k) {
        const CanonTerm& ct = hs.canon[k];
        for (int i = 0; i < ct.nexp; ++i) push_entry(key, h, ct.exp_slot[i]);
        for (int i = 0; i < ct.ngauss; ++i) push_entry(key, h, ct.gauss_slot[i]);
        if (ct.kind == musr::kTermKT || ct.kind == musr::kTermLKT || ct.kind == musr::kTermDKT)
          push_entry(key, h, ct.kt_slot);
        if (ct.kind == musr::kTermTF || ct.kind == musr::kTermDKT) push_entry(key, h, ct.nu_slot);
      }
      auto it = key_to_group.find(key);
      if (it == key_to_group.end()) {
        key_to_group.emplace(key, static_cast<int>(groups.size()));
        groups.push_back({h});
      } else {
        groups[it->second].push_back(h);
      }
    }
  } else {
    for (int h = 0; h < H; ++h) groups.push_back({h});
  }
  // Chunks of at most group_cap histograms; histograms without a bin in the fit
  // range contribute nothing and get no chunk.
  std::vector<Chunk> chunks;
  std::vector<int> hist_index;
  for (const auto& g : groups)
    for (size_t i = 0; i < g.size(); i += group_cap) {
      if (ctx->nhi[g[i]] <= ctx->nlo[g[i]]) continue;
      Chunk ch;
      std::memset(&ch, 0, sizeof(ch));
      ch.first = static_cast<int>(hist_index.size());
      ch.nh = static_cast<int>(std::min<size_t>(group_cap, g.size() - i));
      for (int j = 0; j < ch.nh; ++j) hist_index.push_back(g[i + j]);
      ch.nlo = ctx->nlo[g[i]];
      ch.nhi = ctx->nhi[g[i]];
      ch.t0 = ctx->t0[g[i]];
      ch.tile0 = ch.nlo & ~3;
      chunks.push_back(ch);
    }
  // Tiles: at most 64 iterations of the CTA per tile (the SPLIT phase split
  // needs tile offsets below 2^15 bins).
  std::vector<int64_t> ranges;
  for (const auto& ch : chunks) ranges.push_back(ch.nhi - ch.tile0);
  hs.tile_bins = musr::bins_per_iteration(prec) << var;
  std::vector<int2> items;
  int col = 0;
  for (size_t ci = 0; ci < chunks.size(); ++ci) {
    Chunk& ch = chunks[ci];
    ch.item0 = static_cast<int>(items.size());
    ch.ntiles = static_cast<int>((ranges[ci] + hs.tile_bins - 1) / hs.tile_bins);
    for (int t = 0; t < ch.ntiles; ++t) items.push_back(make_int2(static_cast<int>(ci), t));
    ch.col0 = col;
    col += ch.nh * ctx->nslots;
  }
  hs.group = group_cap;
  hs.nch = prec == MUSR_SPLIT ? musr::shape_channels(hs.shape) : musr::kFp64Channels;
  hs.pstride = 1 + hs.nch;
  hs.ncols = col;
  hs.nchunks = static_cast<int>(chunks.size());
  hs.nitems = static_cast<int>(items.size());
  std::vector<int> col_chunk(std::max(col, 1));
  std::vector<std::vector<int>> pcols(ctx->P);
  for (size_t ci = 0; ci < chunks.size(); ++ci) {
    const Chunk& ch = chunks[ci];
    for (int hl = 0; hl < ch.nh; ++hl) {
      const int h = hist_index[ch.first + hl];
      for (int s = 0; s < ctx->nslots; ++s) {
        const int cc = ch.col0 + hl * ctx->nslots + s;
        col_chunk[cc] = static_cast<int>(ci);
        const int32_t m = ctx->map[static_cast<size_t>(h) * ctx->nslots + s];
        if (m >= 0) pcols[m].push_back(cc);
      }
    }
  }
  std::vector<int> p_ptr(ctx->P + 1, 0), p_cols;
  for (int p = 0; p < ctx->P; ++p) {
    p_ptr[p] = static_cast<int>(p_cols.size());
    p_cols.insert(p_cols.end(), pcols[p].begin(), pcols[p].end());
  }
  p_ptr[ctx->P] = static_cast<int>(p_cols.size());
  if (p_cols.empty()) p_cols.push_back(0);
  if (items.empty()) items.push_back(make_int2(0, 0));
  if (chunks.empty()) chunks.push_back(Chunk{});
  if (hist_index.empty()) hist_index.push_back(0);
  c.dkt_of = std::move(dkt_of);
  c.chunks = std::move(chunks);
  c.items = std::move(items);
  c.hist_index = std::move(hist_index);
  c.col_chunk = std::move(col_chunk);
  c.p_ptr = std::move(p_ptr);
  c.p_cols = std::move(p_cols);
  c.hs = hs;
  c.valid = true;
  c.planned = true;
  c.uploaded = false;
  return MUSR_OK;
}

// Plans one decomposition the first time a launch needs it (host work only).
int ensure_compiled(musr_ctx* ctx, int prec, int var) {
  return ctx->comp[prec][var].planned ? MUSR_OK : compile(ctx, prec, var);
}

// Copies one decomposition's tables to the device (first use only): one allocation
// holding the HistSet, every table and the parameter map and constants, one copy,
// enqueued on the context's stream ahead of the launches that read it.
int ensure_uploaded(musr_ctx* ctx, int prec, int var) {
  Compiled& c = ctx->comp[prec][var];
  if (c.uploaded) return MUSR_OK;
  int crc = ensure_compiled(ctx, prec, var);
  if (crc) return crc;
  size_t off = 0;
  auto place = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t nconsts = std::max<size_t>(ctx->consts.size(), 1);
  const size_t o_hs = place(sizeof(HistSet));
  const size_t o_ch = place(sizeof(Chunk) * c.chunks.size());
  const size_t o_it = place(sizeof(int2) * c.items.size());
  const size_t o_hi = place(sizeof(int) * c.hist_index.size());
  const size_t o_cc = place(sizeof(int) * c.col_chunk.size());
  const size_t o_pp = place(sizeof(int) * c.p_ptr.size());
  const size_t o_pc = place(sizeof(int) * c.p_cols.size());
  const size_t o_mp = place(sizeof(int32_t) * ctx->map.size());
  const size_t o_cs = place(sizeof(double) * nconsts);
  const size_t o_dk = place(sizeof(int) * std::max<size_t>(c.dkt_of.size(), 1));
  int rc = dalloc(ctx, c.tables, off);
  if (rc) return rc;
  char* base = static_cast<char*>(c.tables.p);
  HistSet& hs = c.hs;
  hs.chunks = reinterpret_cast<const Chunk*>(base + o_ch);
  hs.items = reinterpret_cast<const int2*>(base + o_it);
  hs.hist_index = reinterpret_cast<const int*>(base + o_hi);
  hs.col_chunk = reinterpret_cast<const int*>(base + o_cc);
  hs.p_ptr = reinterpret_cast<const int*>(base + o_pp);
  hs.p_cols = reinterpret_cast<const int*>(base + o_pc);
  hs.map = reinterpret_cast<const int32_t*>(base + o_mp);
  hs.consts = reinterpret_cast<const double*>(base + o_cs);
  hs.dkt_of = reinterpret_cast<const int*>(base + o_dk);
  std::vector<char>& blob = c.blob;  // kept until the tables are freed: the copy's source
  blob.assign(off, 0);
  std::memcpy(blob.data() + o_hs, &hs, sizeof(hs));
  std::memcpy(blob.data() + o_ch, c.chunks.data(), sizeof(Chunk) * c.chunks.size());
  std::memcpy(blob.data() + o_it, c.items.data(), sizeof(int2) * c.items.size());
  std::memcpy(blob.data() + o_hi, c.hist_index.data(), sizeof(int) * c.hist_index.size());
  std::memcpy(blob.data() + o_cc, c.col_chunk.data(), sizeof(int) * c.col_chunk.size());
  std::memcpy(blob.data() + o_pp, c.p_ptr.data(), sizeof(int) * c.p_ptr.size());
  std::memcpy(blob.data() + o_pc, c.p_cols.data(), sizeof(int) * c.p_cols.size());
  std::memcpy(blob.data() + o_mp, ctx->map.data(), sizeof(int32_t) * ctx->map.size());
  if (!ctx->consts.empty()) std::memcpy(blob.data() + o_cs, ctx->consts.data(), sizeof(double) * ctx->consts.size());
  if (!c.dkt_of.empty()) std::memcpy(blob.data() + o_dk, c.dkt_of.data(), sizeof(int) * c.dkt_of.size());
  cudaError_t e = cudaMemcpyAsync(base, blob.data(), off, cudaMemcpyHostToDevice,
                                  ctx->setup_stream ? ctx->setup_stream : ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpyAsync(tables)");
  c.d_hs = reinterpret_cast<const HistSet*>(base + o_hs);
  c.uploaded = true;
  return MUSR_OK;
}

void invalidate_eval(musr_ctx* ctx) { ctx->ev.key_valid = false; }

// Decomposition for a launch of nvec evaluations: the large tiles when the
// batch still gives every resident CTA a few items, else the small ones.
int pick_variant(musr_ctx* ctx, int prec, int nvec) {
  int items[musr::kVariants];
  for (int v = 0; v < musr::kVariants; ++v) {
    ensure_compiled(ctx, prec, v);
    items[v] = ctx->comp[prec][v].hs.nitems;
  }
  return musr::pick_decomposition(items, nvec, prec, ctx->num_sms);
}

// Buffers for nvec evaluations; rebuilds the job table when the launch's key
// (precision, decomposition, mode, grad, nvec, pointers) changes.
int ensure_eval(musr_ctx* ctx, int prec, int var, int nvec) {
  EvalBufs& ev = ctx->ev;
  int urc = ensure_uploaded(ctx, prec, var);
  if (urc) return urc;
  const HistSet& hs = ctx->comp[prec][var].hs;
  const size_t part = static_cast<size_t>(nvec) * hs.nitems * hs.pstride;
  const size_t cols = static_cast<size_t>(nvec) * std::max(hs.ncols, 1);
  const size_t nck = static_cast<size_t>(nvec) * std::max(hs.nchunks, 1);
  int rc;
  auto grow = [&](DevBuf& b, size_t bytes, bool zero) -> int {
    if (b.bytes >= bytes) return MUSR_OK;
    int r = dalloc(ctx, b, bytes);
    if (r) return r;
    ev.key_valid = false;
    if (zero) {
      cudaError_t e = cudaMemsetAsync(b.p, 0, b.bytes, ctx->setup_stream ? ctx->setup_stream : ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync");
    }
    return MUSR_OK;
  };
  if ((rc = grow(ev.partials, part * sizeof(double), false))) return rc;
  if ((rc = grow(ev.colsum, cols * sizeof(double), false))) return rc;
  if ((rc = grow(ev.chunk_val, nck * sizeof(double), false))) return rc;
  if ((rc = grow(ev.chunk_count, nck * sizeof(unsigned), true))) return rc;
  if ((rc = grow(ev.counters, nvec * sizeof(unsigned), true))) return rc;
#ifdef MUSR_DEBUG_CHECKS
  if (!ctx->dbg_word.p && (rc = grow(ctx->dbg_word, sizeof(unsigned), true))) return rc;
#endif
  if (hs.ndkt > 0) {
    const size_t nt = static_cast<size_t>(nvec) * hs.ndkt;
    if ((rc = grow(ev.dkt, nt * musr::kDktTable * sizeof(double), false))) return rc;
    if ((rc = grow(ev.dkt_work, nt * musr::kDktWork * sizeof(double), false))) return rc;
    if ((rc = grow(ev.dkt_count, nt * sizeof(unsigned), true))) return rc;
  }
  return MUSR_OK;
}

void fill_jobs(musr_ctx* ctx, int prec, int var, int mode, int grad, int nvec, const double* d_params,
               double* d_out, Job* jobs, int item_begin, const double* d_dirs) {
  EvalBufs& ev = ctx->ev;
  const HistSet& hs = ctx->comp[prec][var].hs;
  const HistSet* d_hs = ctx->comp[prec][var].d_hs;
  for (int v = 0; v < nvec; ++v) {
    Job& j = jobs[v];
    std::memset(&j, 0, sizeof(j));
    j.hs = d_hs;
    j.params = d_params + static_cast<size_t>(v) * ctx->P;
    j.out = d_out + static_cast<size_t>(v) * (1 + ctx->P);
    j.partials = static_cast<double*>(ev.partials.p) + static_cast<size_t>(v) * hs.nitems * hs.pstride;
    j.nrows = hs.nitems;
    j.colsum = static_cast<double*>(ev.colsum.p) + static_cast<size_t>(v) * std::max(hs.ncols, 1);
    j.chunk_val = static_cast<double*>(ev.chunk_val.p) + static_cast<size_t>(v) * std::max(hs.nchunks, 1);
    j.chunk_count = static_cast<unsigned*>(ev.chunk_count.p) + static_cast<size_t>(v) * std::max(hs.nchunks, 1);
    j.counter = static_cast<unsigned*>(ev.counters.p) + v;
    j.item_begin = item_begin + v * hs.nitems;
    j.mode = mode;
    j.grad = grad;
    j.prec = prec;
    j.dir = d_dirs ? d_dirs + static_cast<size_t>(v) * ctx->P : nullptr;
    j.dbg = static_cast<unsigned*>(ctx->dbg_word.p);  // checking build only (else null)
    if (hs.ndkt > 0) {  // tables of this evaluation: FP64 values for prec 0, FP32 for SPLIT
      const size_t esz = prec == MUSR_SPLIT ? sizeof(float) : sizeof(double);
      j.dkt = static_cast<char*>(ev.dkt.p) + static_cast<size_t>(v) * hs.ndkt * musr::kDktTable * esz;
      j.dkt_work = static_cast<char*>(ev.dkt_work.p) + static_cast<size_t>(v) * hs.ndkt * musr::kDktWork * esz;
      j.dkt_count = static_cast<unsigned*>(ev.dkt_count.p) + static_cast<size_t>(v) * hs.ndkt;
    }
  }
}

using musr::Partition;
constexpr int kMaxPieceIters = musr::kMaxTileBins / (musr::kBlock * musr::kBinsPerThread);

// Fills `part` (the launch-level partition of musr_partition.h) and returns true when the
// busiest CTA of its equal-iteration cut beats the compiled decomposition `var` by 3 % or
// more.  Costs in CTA
// iterations: the iterations, a fixed cost per item or piece (row reduction, completion,
// staging start-up: kSplitItemCost) and a cost per change of chunk within a CTA (the chunk's
// FP64 coefficients and constants: 2.4 iterations of a full chunk of 8 histograms, more for
// fewer); both fixed costs weigh 1.5x for the chi^2 kernels, whose iterations are shorter
// (measured on GB300).  Below 8 iterations per CTA a launch is latency, not work: the
// decomposition stays.
bool plan_partition(musr_ctx* ctx, int prec, int var, int mode, int grad, int nvec, Partition* part) {
  const Compiled& c = ctx->comp[prec][var];
  const HistSet& hs = c.hs;
  const int per_sm = musr::max_ctas_per_sm(prec, hs.shape, mode, grad);
  if (per_sm < 1) return false;
  const int G = ctx->num_sms * per_sm;
  const int bpi = musr::bins_per_iteration(prec);
  const int nck = static_cast<int>(c.chunks.size());
  if (nck == 0) return false;
  const double scale = mode == MUSR_MLE ? 1.0 : 1.5;
  const double item_cost = musr::kSplitItemCost * scale;
  std::vector<int64_t> it(nck);
  std::vector<double> load(nck);
  int64_t S = 0;
  double max_load = 0.0;
  int min_tiles = INT32_MAX;
  for (int k = 0; k < nck; ++k) {
    it[k] = (static_cast<int64_t>(c.chunks[k].nhi) - c.chunks[k].tile0 + bpi - 1) / bpi;
    S += it[k];
    load[k] = 2.4 * scale * musr::kGroupMax / std::max(c.chunks[k].nh, 1);
    max_load = std::max(max_load, load[k]);
    min_tiles = std::min(min_tiles, c.chunks[k].ntiles);
  }
  if (S <= 0 || S * nvec < 8 * static_cast<int64_t>(G)) return false;
  // The choice weighs the equal-iteration cut (measured against the decomposition on GB300);
  // the layout may then take ranges of equal cost (musr_partition.h).
  const double equal = musr::equal_cut_worst(it, load, nvec, G, kMaxPieceIters, item_cost);
  if (equal >= 0.97 * musr::items_cost(hs.nitems, nvec, G, hs.tile_bins / bpi, min_tiles, item_cost, max_load))
    return false;
  musr::cut_partition(it, load, nvec, G, kMaxPieceIters, item_cost, part);
  return true;
}

int prepare_jobs(musr_ctx* ctx, int prec, int var, int mode, int grad, int nvec, const double* d_params,
                 double* d_out, const double* d_dirs, const Partition* part = nullptr) {
  EvalBufs& ev = ctx->ev;
  int rc;
  if ((rc = ensure_eval(ctx, prec, var, nvec))) return rc;
  if (ev.jobs.bytes < nvec * sizeof(Job)) {
    if ((rc = dalloc(ctx, ev.jobs, nvec * sizeof(Job)))) return rc;
    ev.key_valid = false;
  }
  const bool pieces = part != nullptr;
  if (ev.key_valid && ev.k_prec == prec && ev.k_var == var && ev.k_mode == mode && ev.k_grad == grad &&
      ev.k_nvec == nvec && ev.k_params == d_params && ev.k_out == d_out && ev.k_dirs == d_dirs &&
      ev.k_pieces == pieces)
    return MUSR_OK;
  std::vector<Job> jobs(nvec);
  fill_jobs(ctx, prec, var, mode, grad, nvec, d_params, d_out, jobs.data(), 0, d_dirs);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
  if (pieces) {  // the partition's rows, tables and the jobs' pointers into them
    const HistSet& hs = ctx->comp[prec][var].hs;
    size_t total_rows = 0;
    for (int r : part->rows) total_rows += static_cast<size_t>(r);
    if (ev.partials.bytes < total_rows * hs.pstride * sizeof(double)) {
      if ((rc = dalloc(ctx, ev.partials, total_rows * hs.pstride * sizeof(double)))) return rc;
    }
    const size_t b_rows = part->chunk_rows.size() * sizeof(int2);
    const size_t b_cta = ((part->cta.size() * sizeof(int)) + 15) & ~size_t(15);
    const size_t b_pcs = part->pieces.size() * sizeof(musr::Piece);
    const size_t o_cta = (b_rows + 15) & ~size_t(15), o_pcs = o_cta + b_cta;
    if (ev.part.bytes < o_pcs + b_pcs) {
      if ((rc = dalloc(ctx, ev.part, o_pcs + b_pcs))) return rc;
    }
    std::vector<char> blob(o_pcs + b_pcs, 0);
    std::memcpy(blob.data(), part->chunk_rows.data(), b_rows);
    std::memcpy(blob.data() + o_cta, part->cta.data(), part->cta.size() * sizeof(int));
    std::memcpy(blob.data() + o_pcs, part->pieces.data(), b_pcs);
    char* base = static_cast<char*>(ev.part.p);
    size_t row0 = 0;
    for (int v = 0; v < nvec; ++v) {
      Job& j = jobs[v];
      j.partials = static_cast<double*>(ev.partials.p) + row0 * hs.pstride;
      j.nrows = part->rows[v];
      j.chunk_rows = reinterpret_cast<const int2*>(base) + static_cast<size_t>(v) * hs.nchunks;
      j.piece_cta = reinterpret_cast<const int*>(base + o_cta);
      j.pieces = reinterpret_cast<const musr::Piece*>(base + o_pcs);
      j.npiece_ctas = part->grid;
      row0 += static_cast<size_t>(part->rows[v]);
    }
    e = cudaMemcpy(ev.part.p, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy(partition)");
  }
  e = copy_h2d(ev.jobs.p, jobs.data(), sizeof(Job) * nvec);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpyAsync(jobs)");
  ev.key_valid = true;
  ev.k_prec = prec;
  ev.k_var = var;
  ev.k_mode = mode;
  ev.k_grad = grad;
  ev.k_nvec = nvec;
  ev.k_params = d_params;
  ev.k_out = d_out;
  ev.k_dirs = d_dirs;
  ev.k_pieces = pieces;
  ev.k_grid = pieces ? part->grid : 0;
  return MUSR_OK;
}

int check_ready(musr_ctx* ctx, int mode, int prec) {
  if (!ctx->have_hist) return fail(ctx, MUSR_ESTATE, "no histograms uploaded");
  if (!ctx->have_theory) return fail(ctx, MUSR_ESTATE, "no theory set");
  if (!ctx->have_map) return fail(ctx, MUSR_ESTATE, "no parameter map set");
  if (mode != MUSR_CHI2 && mode != MUSR_MLE) return fail(ctx, MUSR_EINVAL, "mode must be MUSR_CHI2 or MUSR_MLE");
  if (prec != MUSR_FP64 && prec != MUSR_SPLIT)
    return fail(ctx, MUSR_EINVAL, "precision must be MUSR_FP64 or MUSR_SPLIT");
  if (ctx->asym && mode != MUSR_CHI2)
    return fail(ctx, MUSR_EINVAL, "asymmetry data have the chi^2 cost only (MUSR_CHI2)");
  return MUSR_OK;
}

// Enqueues one launch of nvec evaluations reading d_params, writing d_out.
// One evaluation launch in two steps: the host's planning (decomposition, partition, job
// table; it may synchronise the stream and copy) and the issue of its asynchronous work alone
// (the dynamic Kubo-Toyabe tables, the evaluation kernel).
struct LaunchPlan {
  int prec = 0, mode = 0, grad = 0, nvec = 0, var = 0;
  bool empty = false, pieces = false;
  int grid = 0;
  double* d_out = nullptr;
};

int plan_launch(musr_ctx* ctx, int prec, int mode, int grad, int nvec, const double* d_params, double* d_out,
                const double* d_dirs, LaunchPlan* L) {
  if (ctx->asym && prec == MUSR_SPLIT && mode == MUSR_CHI2) mode = 4;  // SPLIT kernels: weighted chi^2
  L->prec = prec;
  L->mode = mode;
  L->grad = grad;
  L->nvec = nvec;
  L->d_out = d_out;
  L->var = pick_variant(ctx, prec, nvec);
  const HistSet& hs = ctx->comp[prec][L->var].hs;
  L->empty = hs.nitems == 0;  // no bin in the fit range: cost 0, gradient 0
  if (L->empty) return MUSR_OK;
  musr::max_ctas_per_sm(prec, hs.shape, mode, grad);  // the occupancy query, before any capture
  const EvalBufs& ev = ctx->ev;
  if (ev.key_valid && ev.k_prec == prec && ev.k_var == L->var && ev.k_mode == mode && ev.k_grad == grad &&
      ev.k_nvec == nvec && ev.k_params == d_params && ev.k_out == d_out && ev.k_dirs == d_dirs) {
    L->pieces = ev.k_pieces;  // the job table and partition on the device are this launch's
    L->grid = ev.k_grid;
    return MUSR_OK;
  }
  // Batches of plain evaluations on the SPLIT basis kernels may take a launch-level partition.
  Partition part;
  L->pieces = prec == MUSR_SPLIT && nvec >= 2 && (mode == 0 || mode == 1 || mode == 4) &&
              hs.shape != musr::kShapeList && hs.shape != musr::kShapeListS &&
              plan_partition(ctx, prec, L->var, mode, grad, nvec, &part);
  L->grid = L->pieces ? part.grid : 0;
  return prepare_jobs(ctx, prec, L->var, mode, grad, nvec, d_params, d_out, d_dirs, L->pieces ? &part : nullptr);
}

int issue_launch(musr_ctx* ctx, const LaunchPlan& L) {
  const HistSet& hs = ctx->comp[L.prec][L.var].hs;
  if (L.empty) {
    cudaError_t e = cudaMemsetAsync(L.d_out, 0, sizeof(double) * L.nvec * (1 + ctx->P), ctx->stream);
    return e == cudaSuccess ? MUSR_OK : cuda_fail(ctx, e, "cudaMemsetAsync");
  }
  musr::LaunchInfo info;
  if (hs.ndkt > 0 &&
      musr::launch_dkt_tables(L.prec, static_cast<const Job*>(ctx->ev.jobs.p), L.nvec, hs.ndkt, ctx->stream)) {
    cudaError_t e = cudaGetLastError();
    ctx->ev.key_valid = false;
    return cuda_fail(ctx, e, "dynamic Kubo-Toyabe table launch");
  }
  if (musr::launch_eval(L.prec, hs.shape, L.mode, L.grad, static_cast<const Job*>(ctx->ev.jobs.p), L.nvec,
                        L.pieces ? L.grid : L.nvec * hs.nitems, ctx->num_sms, ctx->stream, &info)) {
    cudaError_t e = cudaGetLastError();
    ctx->ev.key_valid = false;
    return cuda_fail(ctx, e, "kernel launch");
  }
  if (L.pieces && info.grid != L.grid) {  // every CTA range of the partition must run
    ctx->ev.key_valid = false;
    return fail(ctx, MUSR_ECUDA, "launch grid differs from the partition's");
  }
  ctx->last_grid = info.grid;
  return MUSR_OK;
}

int enqueue_eval(musr_ctx* ctx, int prec, int mode, int grad, int nvec, const double* d_params,
                 double* d_out, const double* d_dirs = nullptr) {
  LaunchPlan L;
  int rc = plan_launch(ctx, prec, mode, grad, nvec, d_params, d_out, d_dirs, &L);
  return rc ? rc : issue_launch(ctx, L);
}

int wait_stream(musr_ctx* ctx, int timeout_ms) {
  if (timeout_ms <= 0) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? MUSR_OK : cuda_fail(ctx, e, "cudaStreamSynchronize");
  }
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventCreate");
  cudaEventRecord(ev, ctx->stream);
  auto t_end = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  int rc = MUSR_OK;
  for (;;) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      rc = cuda_fail(ctx, e, "cudaEventQuery");
      break;
    }
    if (std::chrono::steady_clock::now() > t_end) {
      rc = fail(ctx, MUSR_ETIMEOUT, "wait timed out");
      break;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  return rc;
}

int ensure_host(musr_ctx* ctx, double** buf, size_t* have, size_t bytes) {
  if (*have >= bytes) return MUSR_OK;
  if (*buf) cudaFreeHost(*buf);
  *buf = nullptr;
  *have = 0;
  cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(buf), bytes);
  if (e != cudaSuccess) return fail(ctx, MUSR_ENOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
  *have = bytes;
  return MUSR_OK;
}

}  // namespace musr

using namespace musr;

extern "C" {

int musr_ctx_create(musr_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream) {
  if (!out) return MUSR_EINVAL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return MUSR_ECUDA;
  }
  if (device < 0 || device >= ndev) {
    g_create_error = "device index out of range";
    return MUSR_EINVAL;
  }
  musr_ctx* ctx = new musr_ctx();
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  DeviceScope ds(device);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    ctx->own_stream = false;
  } else {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      g_create_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
      delete ctx;
      return MUSR_ECUDA;
    }
    ctx->own_stream = true;
  }
  g_create_error.clear();
  *out = ctx;
  return MUSR_OK;
}

void musr_ctx_destroy(musr_ctx* ctx) {
  if (!ctx) return;
  DeviceScope ds(ctx->device);
  if (!ctx->owner_waited) cudaStreamSynchronize(ctx->stream);
  for (auto& pc : ctx->comp)
    for (auto& c : pc) free_compiled(ctx, c);
  dfree(ctx, ctx->counts_own);
  dfree(ctx, ctx->upload_scratch);
  dfree(ctx, ctx->weights_own);
  dfree(ctx, ctx->asym32_own);
  EvalBufs& ev = ctx->ev;
  dfree(ctx, ev.params);
  dfree(ctx, ev.out);
  dfree(ctx, ev.partials);
  dfree(ctx, ev.colsum);
  dfree(ctx, ev.chunk_val);
  dfree(ctx, ev.chunk_count);
  dfree(ctx, ev.counters);
  dfree(ctx, ev.jobs);
  dfree(ctx, ev.dirs);
  dfree(ctx, ev.dkt);
  dfree(ctx, ev.dkt_work);
  dfree(ctx, ev.dkt_count);
  dfree(ctx, ev.part);
  dfree(ctx, ctx->dbg_word);
  if (ev.h_in) cudaFreeHost(ev.h_in);
  if (ev.h_out) cudaFreeHost(ev.h_out);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* musr_last_error(const musr_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

static int upload_common(musr_ctx* ctx, int nhist, int64_t nbins, const double* t0, double bin_width_ns,
                         const double* fit_range_us) {
  if (nhist < 1 || nbins < 1) return fail(ctx, MUSR_EINVAL, "nhist and nbins must be >= 1");
  if (nbins > (int64_t(1) << 30)) return fail(ctx, MUSR_EINVAL, "nbins must be < 2^30");
  if (!t0 || !fit_range_us) return fail(ctx, MUSR_EINVAL, "t0 and fit_range_us must not be NULL");
  if (!(bin_width_ns > 0.0) || !std::isfinite(bin_width_ns))
    return fail(ctx, MUSR_EINVAL, "bin_width_ns must be finite and > 0");
  if (!std::isfinite(fit_range_us[0]) || !std::isfinite(fit_range_us[1]) || fit_range_us[0] > fit_range_us[1])
    return fail(ctx, MUSR_EINVAL, "fit range must be finite with lo <= hi");
  for (int h = 0; h < nhist; ++h)
    if (!std::isfinite(t0[h])) return fail(ctx, MUSR_EINVAL, "t0 must be finite");
  ctx->check_flag = nullptr;
  dfree(ctx, ctx->upload_scratch);
  ctx->shift.clear();
  ctx->asym = false;
  dfree(ctx, ctx->weights_own);
  dfree(ctx, ctx->asym32_own);
  ctx->H = nhist;
  ctx->B = nbins;
  ctx->t0.assign(t0, t0 + nhist);
  ctx->bin_width_ns = bin_width_ns;
  ctx->dt_us = bin_width_ns / 1000.0;
  ctx->lo = fit_range_us[0];
  ctx->hi = fit_range_us[1];
  ctx->nlo.resize(nhist);
  ctx->nhi.resize(nhist);
  for (int h = 0; h < nhist; ++h)
    fit_bins(ctx->t0[h], ctx->dt_us, nbins, ctx->lo, ctx->hi, &ctx->nlo[h], &ctx->nhi[h]);
  return MUSR_OK;
}

// Waits for launches that may still read the current configuration; a context that
// has no map yet has never launched, so nothing is waited for (the serving loop
// configures new fits while other fits run on the same stream).
static void quiesce(musr_ctx* ctx) {
  if (ctx->have_map) cudaStreamSynchronize(ctx->stream);
}

static void drop_config(musr_ctx* ctx) {
  for (auto& pc : ctx->comp)
    for (auto& c : pc) free_compiled(ctx, c);
  ctx->have_map = false;
  ctx->have_hist = false;
  invalidate_eval(ctx);
}

int musr_upload_histograms(musr_ctx* ctx, const void* counts, int dtype, int nhist, int64_t nbins,
                           const double* t0, double bin_width_ns, const double fit_range_us[2]) {
  if (!ctx) return MUSR_EINVAL;
  DeviceScope ds(ctx->device);
  if (!counts) return fail(ctx, MUSR_EINVAL, "counts must not be NULL");
  if (dtype != MUSR_DTYPE_INT32 && dtype != MUSR_DTYPE_FP32 && dtype != MUSR_DTYPE_FP64)
    return fail(ctx, MUSR_EINVAL, "dtype must be MUSR_DTYPE_INT32, _FP32 or _FP64");
  quiesce(ctx);
  drop_config(ctx);
  int rc = upload_common(ctx, nhist, nbins, t0, bin_width_ns, fit_range_us);
  if (rc) return rc;
  const int64_t stride = (nbins + kRowAlign - 1) / kRowAlign * kRowAlign;
  const size_t esz = dtype == MUSR_DTYPE_FP64 ? 8 : 4;
  const size_t total = static_cast<size_t>(nhist) * stride * esz;
  // Rows whose time-zero bins differ by whole bins are moved onto one grid (the time
  // factors of histograms on a common grid are evaluated once for all of them).
  std::vector<int64_t> shift = grid_shifts(ctx);
  const bool shifted = std::any_of(shift.begin(), shift.end(), [](int64_t v) { return v != 0; });
  // The rows go to the device as they are, in one copy; a kernel then converts INT32 to
  // FP32, zeroes the padding and flags counts the store cannot hold.  The host makes no
  // pass over the data.  Unshifted rows go straight to the device image at its row
  // stride (converted in place); shifted ones to a packed scratch copy first.
  if ((rc = dalloc(ctx, ctx->counts_own, total))) return rc;
  cudaStream_t st = ctx->setup_stream ? ctx->setup_stream : cudaStreamPerThread;
  const size_t row = static_cast<size_t>(nbins) * esz;
  CheckFlag& flag = tl_flag;
  if (!flag.ready()) return cuda_fail(ctx, cudaGetLastError(), "cudaHostAlloc(check flag)");
  const unsigned seq = flag.next();
  cudaError_t e;
  const void* src = stage_rows(ctx, counts, row * static_cast<size_t>(nhist));
  if (!shifted) {
    e = stride == nbins ? cudaMemcpyAsync(ctx->counts_own.p, src, total, cudaMemcpyHostToDevice, st)
                        : cudaMemcpy2DAsync(ctx->counts_own.p, static_cast<size_t>(stride) * esz, src, row, row,
                                            static_cast<size_t>(nhist), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpyAsync(counts)");
    if (launch_prepare_counts(ctx->counts_own.p, dtype, nhist, nbins, stride, flag.dev, seq, ctx->num_sms, st))
      return cuda_fail(ctx, cudaGetLastError(), "prepare_counts launch");
  } else {
    const size_t raw = (row * nhist + 255) & ~size_t(255);
    if ((rc = dalloc(ctx, ctx->upload_scratch, raw + sizeof(int64_t) * nhist))) return rc;
    char* sp = static_cast<char*>(ctx->upload_scratch.p);
    ctx->shift = std::move(shift);  // the copy's source, kept until the check is read
    e = cudaMemcpyAsync(sp, src, row * nhist, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sp + raw, ctx->shift.data(), sizeof(int64_t) * nhist, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpyAsync(counts)");
    if (launch_prepare_counts_shifted(sp, ctx->counts_own.p, reinterpret_cast<const int64_t*>(sp + raw), dtype,
                                      nhist, nbins, stride, flag.dev, seq, ctx->num_sms, st))
      return cuda_fail(ctx, cudaGetLastError(), "prepare_counts launch");
    // the device grid: t0 and the fit window move with the row (whole bins, exact)
    for (int h = 0; h < nhist; ++h) {
      ctx->t0[h] -= static_cast<double>(ctx->shift[h]);
      ctx->nlo[h] -= static_cast<int>(ctx->shift[h]);
      ctx->nhi[h] -= static_cast<int>(ctx->shift[h]);
    }
  }
  ctx->check_flag = flag.host;
  ctx->check_seq = seq;
  ctx->check_dtype = dtype;
  ctx->d_counts = ctx->counts_own.p;
  ctx->store = dtype == MUSR_DTYPE_FP64 ? kStoreF64 : kStoreF32;
  ctx->stride = stride;
  ctx->have_hist = true;
  if (ctx->setup_stream) return MUSR_OK;  // the caller waits and reads the check
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "prepare_counts");
  return finish_upload_check(ctx);
}

}  // extern "C"

int musr::finish_upload_check(musr_ctx* ctx) {
  if (!ctx->check_flag) return MUSR_OK;
  const bool bad = *static_cast<const volatile unsigned*>(ctx->check_flag) == ctx->check_seq;
  ctx->check_flag = nullptr;
  dfree(ctx, ctx->upload_scratch);
  if (!bad) return MUSR_OK;
  drop_config(ctx);
  dfree(ctx, ctx->counts_own);
  dfree(ctx, ctx->weights_own);
  dfree(ctx, ctx->asym32_own);
  ctx->asym = false;
  ctx->d_counts = nullptr;
  return fail(ctx, MUSR_EINVAL,
              ctx->check_dtype == MUSR_DTYPE_INT32 ? "INT32 counts must satisfy |count| < 2^24 (exact in FP32)"
                                                   : "counts must be finite");
}

extern "C" {

int musr_upload_asymmetry(musr_ctx* ctx, const void* forward, const void* backward, int dtype, int npairs,
                          int64_t nbins, const double* t0, double bin_width_ns, const double fit_range_us[2],
                          const double* alpha, const double* bkg_forward, const double* bkg_backward) {
  if (!ctx) return MUSR_EINVAL;
  DeviceScope ds(ctx->device);
  if (!forward || !backward) return fail(ctx, MUSR_EINVAL, "forward and backward must not be NULL");
  if (!alpha || !bkg_forward || !bkg_backward)
    return fail(ctx, MUSR_EINVAL, "alpha, bkg_forward and bkg_backward must not be NULL");
  if (dtype != MUSR_DTYPE_INT32 && dtype != MUSR_DTYPE_FP32 && dtype != MUSR_DTYPE_FP64)
    return fail(ctx, MUSR_EINVAL, "dtype must be MUSR_DTYPE_INT32, _FP32 or _FP64");
  quiesce(ctx);
  drop_config(ctx);
  int rc = upload_common(ctx, npairs, nbins, t0, bin_width_ns, fit_range_us);
  if (rc) return rc;
  for (int h = 0; h < npairs; ++h)
    if (!(alpha[h] > 0.0) || !std::isfinite(alpha[h]) || !std::isfinite(bkg_forward[h]) ||
        !std::isfinite(bkg_backward[h]))
      return fail(ctx, MUSR_EINVAL, "alpha must be finite and > 0, the backgrounds finite");
  const int64_t stride = (nbins + kRowAlign - 1) / kRowAlign * kRowAlign;
  const size_t esz = dtype == MUSR_DTYPE_FP64 ? 8 : 4;
  const size_t row = static_cast<size_t>(nbins) * esz, H = static_cast<size_t>(npairs);
  const size_t image = H * stride * sizeof(double);
  if ((rc = dalloc(ctx, ctx->counts_own, image))) return rc;
  if ((rc = dalloc(ctx, ctx->weights_own, image))) return rc;
  if ((rc = dalloc(ctx, ctx->asym32_own, image))) return rc;  // [2][H][stride] FP32
  // Scratch: the raw forward rows, the raw backward rows, the row shifts, alpha and the
  // backgrounds; one kernel turns them into a and w on the device (FP64).
  const size_t raw = (2 * row * H + 255) & ~size_t(255), o_par = raw + ((8 * H + 255) & ~size_t(255));
  if ((rc = dalloc(ctx, ctx->upload_scratch, o_par + 3 * sizeof(double) * H))) return rc;
  char* sp = static_cast<char*>(ctx->upload_scratch.p);
  ctx->shift = grid_shifts(ctx);
  ctx->asym_par.assign(alpha, alpha + H);
  ctx->asym_par.insert(ctx->asym_par.end(), bkg_forward, bkg_forward + H);
  ctx->asym_par.insert(ctx->asym_par.end(), bkg_backward, bkg_backward + H);
  cudaStream_t st = ctx->setup_stream ? ctx->setup_stream : cudaStreamPerThread;
  cudaError_t e = cudaMemcpyAsync(sp, forward, row * H, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sp + row * H, backward, row * H, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sp + raw, ctx->shift.data(), 8 * H, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sp + o_par, ctx->asym_par.data(), 3 * sizeof(double) * H, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpyAsync(asymmetry pairs)");
  CheckFlag& flag = tl_flag;
  if (!flag.ready()) return cuda_fail(ctx, cudaGetLastError(), "cudaHostAlloc(check flag)");
  const unsigned seq = flag.next();
  if (launch_prepare_asymmetry(sp, reinterpret_cast<const int64_t*>(sp + raw),
                               reinterpret_cast<const double*>(sp + o_par), dtype, npairs, nbins, stride,
                               static_cast<double*>(ctx->counts_own.p), static_cast<double*>(ctx->weights_own.p),
                               static_cast<float*>(ctx->asym32_own.p),
                               static_cast<float*>(ctx->asym32_own.p) + H * stride, flag.dev, seq, ctx->num_sms, st))
    return cuda_fail(ctx, cudaGetLastError(), "prepare_asymmetry launch");
  for (int h = 0; h < npairs; ++h) {  // the device grid (see musr_upload_histograms)
    ctx->t0[h] -= static_cast<double>(ctx->shift[h]);
    ctx->nlo[h] -= static_cast<int>(ctx->shift[h]);
    ctx->nhi[h] -= static_cast<int>(ctx->shift[h]);
  }
  ctx->check_flag = flag.host;
  ctx->check_seq = seq;
  ctx->check_dtype = dtype;
  ctx->d_counts = ctx->counts_own.p;
  ctx->store = kStoreF64;
  ctx->stride = stride;
  ctx->asym = true;
  ctx->have_hist = true;
  if (ctx->setup_stream) return MUSR_OK;  // the caller waits and reads the check
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "prepare_asymmetry");
  return finish_upload_check(ctx);
}

int musr_upload_histograms_device(musr_ctx* ctx, const void* d_counts, int dtype, int nhist, int64_t nbins,
                                  int64_t row_stride, const double* t0, double bin_width_ns,
                                  const double fit_range_us[2]) {
  if (!ctx) return MUSR_EINVAL;
  DeviceScope ds(ctx->device);
  if (!d_counts) return fail(ctx, MUSR_EINVAL, "d_counts must not be NULL");
  if (dtype != MUSR_DTYPE_FP32 && dtype != MUSR_DTYPE_FP64)
    return fail(ctx, MUSR_EINVAL, "device histograms must be MUSR_DTYPE_FP32 or _FP64");
  if (reinterpret_cast<uintptr_t>(d_counts) % 16 != 0)
    return fail(ctx, MUSR_EINVAL, "d_counts must be 16-byte aligned");
  if (row_stride < nbins || row_stride % 4 != 0)
    return fail(ctx, MUSR_EINVAL, "row_stride must be >= nbins and a multiple of 4");
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, d_counts) != cudaSuccess || attr.type != cudaMemoryTypeDevice ||
      attr.device != ctx->device) {
    cudaGetLastError();
    return fail(ctx, MUSR_EINVAL, "d_counts is not device memory of the context's device");
  }
  quiesce(ctx);
  drop_config(ctx);
  dfree(ctx, ctx->counts_own);
  int rc = upload_common(ctx, nhist, nbins, t0, bin_width_ns, fit_range_us);
  if (rc) return rc;
  ctx->d_counts = d_counts;
  ctx->store = dtype == MUSR_DTYPE_FP64 ? kStoreF64 : kStoreF32;
  ctx->stride = row_stride;
  ctx->have_hist = true;
  return MUSR_OK;
}

int musr_set_theory(musr_ctx* ctx, const musr_term* terms, int nterms) {
  if (!ctx) return MUSR_EINVAL;
  DeviceScope ds(ctx->device);
  if (nterms < 0 || nterms > MUSR_MAX_TERMS) return fail(ctx, MUSR_EINVAL, "nterms must be in [0, 4]");
  if (nterms > 0 && !terms) return fail(ctx, MUSR_EINVAL, "terms must not be NULL");
  for (int k = 0; k < nterms; ++k) {
    const musr_term& t = terms[k];
    if (t.nprim < 1 || t.nprim > MUSR_MAX_PRIMS) return fail(ctx, MUSR_EINVAL, "a term needs 1..4 primitives");
    for (int m = 0; m < t.nprim; ++m) {
      if (t.kind[m] < MUSR_PRIM_AMP || t.kind[m] > MUSR_PRIM_DKT)
        return fail(ctx, MUSR_EINVAL, "unknown primitive kind");
      const int ns = musr::prim_nslots(t.kind[m]);
      for (int q = 0; q < ns; ++q)
        if (t.slot[m][q] < 0 || t.slot[m][q] >= MUSR_MAX_SLOTS)
          return fail(ctx, MUSR_EINVAL, "slot index out of range");
    }
  }
  quiesce(ctx);
  for (auto& pc : ctx->comp)
    for (auto& c : pc) free_compiled(ctx, c);
  ctx->have_map = false;
  invalidate_eval(ctx);
  ctx->terms.assign(terms, terms + nterms);
  ctx->have_theory = true;
  return MUSR_OK;
}

int musr_set_map(musr_ctx* ctx, const int32_t* map, int nslots, int nparams, const double* consts,
                 int nconsts) {
  if (!ctx) return MUSR_EINVAL;
  DeviceScope ds(ctx->device);
  if (!ctx->have_hist) return fail(ctx, MUSR_ESTATE, "upload histograms before the map");
  if (!ctx->have_theory) return fail(ctx, MUSR_ESTATE, "set the theory before the map");
  if (!map) return fail(ctx, MUSR_EINVAL, "map must not be NULL");
  if (nslots < 2 || nslots > MUSR_MAX_SLOTS) return fail(ctx, MUSR_EINVAL, "nslots must be in [2, 32]");
  if (nparams < 0 || nparams > MUSR_MAX_PARAMS) return fail(ctx, MUSR_EINVAL, "nparams out of range");
  if (nconsts < 0 || (nconsts > 0 && !consts)) return fail(ctx, MUSR_EINVAL, "bad consts");
  for (const auto& t : ctx->terms)
    for (int m = 0; m < t.nprim; ++m)
      for (int q = 0; q < musr::prim_nslots(t.kind[m]); ++q)
        if (t.slot[m][q] >= nslots) return fail(ctx, MUSR_EINVAL, "theory references a slot >= nslots");
  {  // at most kMaxDkt distinct (Delta, nu) pairs of dynamic Kubo-Toyabe factors
    std::vector<std::pair<int32_t, int32_t>> src;
    for (int h = 0; h < ctx->H; ++h)
      for (const auto& t : ctx->terms)
        for (int m = 0; m < t.nprim; ++m) {
          if (t.kind[m] != MUSR_PRIM_DKT) continue;
          const std::pair<int32_t, int32_t> key(map[static_cast<size_t>(h) * nslots + t.slot[m][0]],
                                                map[static_cast<size_t>(h) * nslots + t.slot[m][1]]);
          if (std::find(src.begin(), src.end(), key) == src.end()) src.push_back(key);
        }
    if (static_cast<int>(src.size()) > musr::kMaxDkt)
      return fail(ctx, MUSR_EINVAL, "at most 8 distinct (Delta, nu) pairs of dynamic Kubo-Toyabe factors");
  }
  for (int i = 0; i < nconsts; ++i)
    if (!std::isfinite(consts[i])) return fail(ctx, MUSR_EINVAL, "consts must be finite");
  const size_t n = static_cast<size_t>(ctx->H) * nslots;
  for (size_t i = 0; i < n; ++i) {
    const int32_t m = map[i];
    if (m >= nparams || (m < 0 && -1 - m >= nconsts))
      return fail(ctx, MUSR_EINVAL, "map entry " + std::to_string(i) + " out of range");
  }
  quiesce(ctx);
  for (auto& pc : ctx->comp)
    for (auto& c : pc) free_compiled(ctx, c);
  invalidate_eval(ctx);
  ctx->map.assign(map, map + n);
  ctx->nslots = nslots;
  ctx->P = nparams;
  ctx->consts.assign(consts, consts + nconsts);
  // Decompositions are planned when a launch first needs one; whether the SPLIT path
  // can run this theory at all is decided now.
  {
    HistSet probe;
    std::memset(&probe, 0, sizeof(probe));
    const char* why = musr::plan_split(ctx->terms.data(), static_cast<int>(ctx->terms.size()), ctx->map.data(),
                                       ctx->H, ctx->nslots, ctx->consts.data(), &probe, !ctx->asym);
    ctx->split_reason = why ? why : "";
  }
  ctx->have_map = true;
  return MUSR_OK;
}

int musr_eval_batch(musr_ctx* ctx, const double* params, int nvec, int nparams, int mode, int precision,
                    double* out_values, double* out_grads) {
  if (!ctx) return MUSR_EINVAL;
  DeviceScope ds(ctx->device);
  int rc = check_ready(ctx, mode, precision);
  if (rc) return rc;
  if (nvec < 1) return fail(ctx, MUSR_EINVAL, "nvec must be >= 1");
  if (nparams != ctx->P) return fail(ctx, MUSR_EINVAL, "nparams does not match the map");
  if (!params || !out_values) return fail(ctx, MUSR_EINVAL, "params and out_values must not be NULL");
  const size_t P = ctx->P, np = static_cast<size_t>(nvec) * P, no = static_cast<size_t>(nvec) * (1 + P);
  for (size_t i = 0; i < np; ++i)
    if (!std::isfinite(params[i])) return fail(ctx, MUSR_EINVAL, "parameters must be finite");
  EvalBufs& ev = ctx->ev;
  if ((rc = ensure_host(ctx, &ev.h_in, &ev.h_in_bytes, std::max<size_t>(np, 1) * sizeof(double)))) return rc;
  if ((rc = ensure_host(ctx, &ev.h_out, &ev.h_out_bytes, no * sizeof(double)))) return rc;
  if (ev.params.bytes < std::max<size_t>(np, 1) * sizeof(double)) {
    if ((rc = dalloc(ctx, ev.params, std::max<size_t>(np, 1) * sizeof(double)))) return rc;
    ev.key_valid = false;
  }
  if (ev.out.bytes < no * sizeof(double)) {
    if ((rc = dalloc(ctx, ev.out, no * sizeof(double)))) return rc;
    ev.key_valid = false;
  }
  const int grad = out_grads != nullptr;
  std::memcpy(ev.h_in, params, np * sizeof(double));
  LaunchPlan L;
  if ((rc = plan_launch(ctx, precision, mode, grad, nvec, static_cast<const double*>(ev.params.p),
                        static_cast<double*>(ev.out.p), nullptr, &L)))
    return rc;
  cudaError_t e = cudaMemcpyAsync(ev.params.p, ev.h_in, np * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpyAsync(params)");
  if ((rc = issue_launch(ctx, L))) return rc;
  e = cudaMemcpyAsync(ev.h_out, ev.out.p, no * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpyAsync(out)");
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
  bool nonfinite = false;
  for (int v = 0; v < nvec; ++v) {
    const double* o = ev.h_out + static_cast<size_t>(v) * (1 + P);
    out_values[v] = o[0];
    if (!std::isfinite(o[0])) nonfinite = true;
    if (out_grads) {
      double* g = out_grads + static_cast<size_t>(v) * P;
      if (std::isfinite(o[0]))
        std::memcpy(g, o + 1, P * sizeof(double));
      else
        std::memset(g, 0, P * sizeof(double));
    }
  }
  if (nonfinite)
    return fail(ctx, MUSR_ENONFINITE, "cost not finite: N <= 0 in a bin with d > 0 (-2lnL), or a parameter not finite");
  return MUSR_OK;
}

int musr_gn_product(musr_ctx* ctx, const double* params, int nparams, const double* dirs, int ndir, int mode,
                    int precision, double* out) {
  if (!ctx) return MUSR_EINVAL;
  DeviceScope ds(ctx->device);
  int rc = check_ready(ctx, mode, precision);
  if (rc) return rc;
  if (ctx->asym && precision == MUSR_SPLIT)
    return fail(ctx, MUSR_EINVAL, "Gauss-Newton products of asymmetry data run at MUSR_FP64 precision");
  if (!ctx->split_reason.empty() && precision == MUSR_SPLIT)
    return fail(ctx, MUSR_EINVAL,
                "Gauss-Newton products of a theory without a basis form run at MUSR_FP64 precision (" +
                    ctx->split_reason + ")");
  if (ndir < 1) return fail(ctx, MUSR_EINVAL, "ndir must be >= 1");
  if (nparams != ctx->P) return fail(ctx, MUSR_EINVAL, "nparams does not match the map");
  if (!params || !dirs || !out) return fail(ctx, MUSR_EINVAL, "params, dirs and out must not be NULL");
  const size_t P = ctx->P, nd = static_cast<size_t>(ndir) * P, no = static_cast<size_t>(ndir) * (1 + P);
  for (size_t i = 0; i < P; ++i)
    if (!std::isfinite(params[i])) return fail(ctx, MUSR_EINVAL, "parameters must be finite");
  for (size_t i = 0; i < nd; ++i)
    if (!std::isfinite(dirs[i])) return fail(ctx, MUSR_EINVAL, "directions must be finite");
  EvalBufs& ev = ctx->ev;
  // params repeated for every direction (one job each), then the directions
  const size_t nin = std::max<size_t>(2 * nd, 1);
  if ((rc = ensure_host(ctx, &ev.h_in, &ev.h_in_bytes, nin * sizeof(double)))) return rc;
  if ((rc = ensure_host(ctx, &ev.h_out, &ev.h_out_bytes, no * sizeof(double)))) return rc;
  if (ev.params.bytes < std::max<size_t>(nd, 1) * sizeof(double)) {
    if ((rc = dalloc(ctx, ev.params, std::max<size_t>(nd, 1) * sizeof(double)))) return rc;
    ev.key_valid = false;
  }
  if (ev.dirs.bytes < std::max<size_t>(nd, 1) * sizeof(double)) {
    if ((rc = dalloc(ctx, ev.dirs, std::max<size_t>(nd, 1) * sizeof(double)))) return rc;
    ev.key_valid = false;
  }
  if (ev.out.bytes < no * sizeof(double)) {
    if ((rc = dalloc(ctx, ev.out, no * sizeof(double)))) return rc;
    ev.key_valid = false;
  }
  for (int v = 0; v < ndir; ++v) std::memcpy(ev.h_in + static_cast<size_t>(v) * P, params, P * sizeof(double));
  std::memcpy(ev.h_in + nd, dirs, nd * sizeof(double));
  cudaError_t e = cudaMemcpyAsync(ev.params.p, ev.h_in, nd * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ev.dirs.p, ev.h_in + nd, nd * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpyAsync(params, dirs)");
  if ((rc = enqueue_eval(ctx, precision, mode + 2, 1, ndir, static_cast<const double*>(ev.params.p),
                         static_cast<double*>(ev.out.p), static_cast<const double*>(ev.dirs.p))))
    return rc;
  e = cudaMemcpyAsync(ev.h_out, ev.out.p, no * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpyAsync(out)");
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
  bool nonfinite = false;
  for (int v = 0; v < ndir; ++v) {
    const double* o = ev.h_out + static_cast<size_t>(v) * (1 + P);
    double* r = out + static_cast<size_t>(v) * (1 + P);
    r[0] = o[0];
    if (!std::isfinite(o[0])) {
      nonfinite = true;
      std::memset(r + 1, 0, P * sizeof(double));
    } else {
      std::memcpy(r + 1, o + 1, P * sizeof(double));
    }
  }
  if (nonfinite) return fail(ctx, MUSR_ENONFINITE, "-2lnL undefined: N <= 0 in a bin with d > 0, or a parameter not finite");
  return MUSR_OK;
}

int musr_gauss_newton(musr_ctx* ctx, const double* params, int nparams, int mode, int precision, double* out) {
  if (!ctx) return MUSR_EINVAL;
  if (!out) return fail(ctx, MUSR_EINVAL, "out must not be NULL");
  if (nparams != ctx->P || nparams < 1) return fail(ctx, MUSR_EINVAL, "nparams does not match the map");
  const size_t P = nparams;
  std::vector<double> dirs(P * P, 0.0), prod(P * (P + 1));
  for (size_t i = 0; i < P; ++i) dirs[i * P + i] = 1.0;
  const int rc = musr_gn_product(ctx, params, nparams, dirs.data(), nparams, mode, precision, prod.data());
  if (rc) return rc;
  for (size_t i = 0; i < P; ++i)
    for (size_t j = 0; j < P; ++j)  // column j of H is the product with unit vector j
      out[i * P + j] = 0.5 * (prod[j * (P + 1) + 1 + i] + prod[i * (P + 1) + 1 + j]);
  return MUSR_OK;
}

int musr_eval(musr_ctx* ctx, const double* params, int nparams, int mode, int precision, double* out_value,
              double* out_grad) {
  return musr_eval_batch(ctx, params, 1, nparams, mode, precision, out_value, out_grad);
}

int musr_eval_device(musr_ctx* ctx, const double* d_params, int nvec, int mode, int precision, int with_grad,
                     double* d_out) {
  if (!ctx) return MUSR_EINVAL;
  DeviceScope ds(ctx->device);
  int rc = check_ready(ctx, mode, precision);
  if (rc) return rc;
  if (nvec < 1) return fail(ctx, MUSR_EINVAL, "nvec must be >= 1");
  if (!d_params || !d_out) return fail(ctx, MUSR_EINVAL, "d_params and d_out must not be NULL");
  return enqueue_eval(ctx, precision, mode, with_grad ? 1 : 0, nvec, d_params, d_out);
}

int musr_sync(musr_ctx* ctx, int timeout_ms) {
  if (!ctx) return MUSR_EINVAL;
  DeviceScope ds(ctx->device);
  return wait_stream(ctx, timeout_ms);
}

int musr_bins_in_fit(musr_ctx* ctx, int64_t* out) {
  if (!ctx || !out) return MUSR_EINVAL;
  if (!ctx->have_hist) return fail(ctx, MUSR_ESTATE, "no histograms uploaded");
  int64_t s = 0;
  for (int h = 0; h < ctx->H; ++h) s += ctx->nhi[h] - ctx->nlo[h];
  *out = s;
  return MUSR_OK;
}

int musr_debug_word(musr_ctx* ctx, uint32_t* out) {
  if (!ctx || !out) return MUSR_EINVAL;
  *out = 0;
#ifdef MUSR_DEBUG_CHECKS
  DeviceScope ds(ctx->device);
  if (!ctx->dbg_word.p) return MUSR_OK;  // no evaluation yet
  unsigned w = 0;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpy(&w, ctx->dbg_word.p, sizeof(w), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "musr_debug_word");
  *out = w;
  return MUSR_OK;
#else
  return fail(ctx, MUSR_ESTATE, "this library was built without the index checks (MUSR_DEBUG_CHECKS)");
#endif
}

int musr_launches_per_eval(musr_ctx* ctx, int* out) {
  if (!ctx || !out) return MUSR_EINVAL;
  bool dkt = false;  // a dynamic Kubo-Toyabe factor adds the launch that solves its tables
  for (const auto& t : ctx->terms)
    for (int m = 0; m < t.nprim; ++m) dkt = dkt || t.kind[m] == MUSR_PRIM_DKT;
  *out = dkt ? 2 : 1;
  return MUSR_OK;
}

}  // extern "C"
