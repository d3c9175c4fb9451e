// musr_partition.h -- host-side launch-level partition of a batch for the SPLIT basis kernels.
//
// A compiled decomposition hands out whole items (a chunk's tile for one parameter vector), so
// a batch whose items do not divide evenly over the persistent grid leaves CTAs idle or with
// an extra item.  The partition cuts the batch's CTA iterations -- in the order job, chunk,
// iteration -- into one contiguous range per CTA (equal in iterations or in modelled cost, see
// cut_partition); a range's share of a chunk becomes
// pieces of at most max_piece iterations (the phase split's limit), each with a partial row
// of its own.  A job's rows follow its pieces' order, so every chunk's rows are contiguous and
// are summed in a fixed order.  Pure host logic (no CUDA call): the context plans with it and
// the host tests check its invariants.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

#include "musr_dev.h"

namespace musr {

struct Partition {
  int grid = 0;
  std::vector<Piece> pieces;
  std::vector<int> cta;          // [grid + 1] first piece of each CTA
  std::vector<int2> chunk_rows;  // [nvec][nchunks] first row, rows
  std::vector<int> rows;         // [nvec] rows of each job
};

// Iterations that a CTA with cost budget b takes from a chunk of r remaining iterations and
// chunk load `load`, starting on it: n iterations cost n, item_cost per piece of at most
// max_piece iterations and the load.  0 when not one iteration fits.
inline int64_t fit_iterations(int64_t r, double b, double load, int max_piece, double item_cost) {
  const double room = b - load;
  int64_t n = std::min<int64_t>(r, static_cast<int64_t>(room - item_cost));
  while (n > 0) {  // fewer iterations may need fewer pieces: shrink until the cost fits
    const int64_t pieces = (n + max_piece - 1) / max_piece;
    const int64_t m = std::min<int64_t>(n, static_cast<int64_t>(room - item_cost * static_cast<double>(pieces)));
    if (m == n) break;
    n = m;
  }
  return std::max<int64_t>(n, 0);
}

// Greedy cut of the job-chunk-iteration order into CTA ranges of cost at most T, each range
// as long as its budget allows; bounds gets each range's first iteration and the end.
// Returns the number of ranges, or G + 1 when G ranges do not cover the batch.  The cost of
// a range does not grow when its start moves later, so no cut into G ranges of cost at most
// T exists when this one needs more.
inline int greedy_bounds(const std::vector<int64_t>& iters, const std::vector<double>& load, int nvec, int G,
                         int max_piece, double item_cost, double T, std::vector<int64_t>* bounds) {
  const int nck = static_cast<int>(iters.size());
  bounds->clear();
  int j = 0, k = 0;
  int64_t i0 = 0, q = 0;  // iteration i0 of chunk k of job j; q in the batch order
  while (j < nvec) {
    if (static_cast<int>(bounds->size()) == G) return G + 1;
    bounds->push_back(q);
    double b = T;
    bool took = false;
    while (j < nvec) {
      const int64_t n = fit_iterations(iters[k] - i0, b, load[k], max_piece, item_cost);
      if (n == 0) break;
      took = true;
      b -= static_cast<double>(n) + load[k] + item_cost * static_cast<double>((n + max_piece - 1) / max_piece);
      q += n;
      i0 += n;
      if (i0 < iters[k]) break;  // the budget ended inside the chunk
      i0 = 0;
      if (++k == nck) {
        k = 0;
        ++j;
      }
    }
    if (!took) return G + 1;  // T below the cost of a single iteration
  }
  const int used = static_cast<int>(bounds->size());
  bounds->push_back(q);
  return used;
}

// Cost of the CTA range [lo, hi) of the batch order over chunks with prefix sums pre
// (pre[k] = iterations before chunk k of a job, pre[nck] = S): its iterations, item_cost per
// piece (cut at max_piece from the range's start in each chunk) and load[k] for each chunk k
// it starts on.  Walks the chunks the range crosses, not its pieces.
inline double range_cost(const std::vector<int64_t>& pre, const std::vector<double>& load, int max_piece,
                         double item_cost, int64_t lo, int64_t hi) {
  const int64_t S = pre.back();
  double c = static_cast<double>(hi - lo);
  for (int64_t q = lo; q < hi;) {
    const int64_t j = q / S, off = q - j * S;
    const int k = static_cast<int>(std::upper_bound(pre.begin(), pre.end(), off) - pre.begin()) - 1;
    const int64_t n = std::min<int64_t>(hi - q, pre[k + 1] - off);
    c += load[k] + item_cost * static_cast<double>((n + max_piece - 1) / max_piece);
    q += n;
  }
  return c;
}

// The busiest CTA's cost when G CTAs take equal iteration counts (floor(I b / G) onwards).
inline double equal_cut_worst(const std::vector<int64_t>& iters, const std::vector<double>& load, int nvec, int G,
                              int max_piece, double item_cost) {
  std::vector<int64_t> pre(iters.size() + 1, 0);
  for (size_t k = 0; k < iters.size(); ++k) pre[k + 1] = pre[k] + iters[k];
  const int64_t I = pre.back() * nvec;
  double w = 0.0;
  for (int b = 0; b < G; ++b)
    w = std::max(w, range_cost(pre, load, max_piece, item_cost, I * b / G, I * (b + 1) / G));
  return w;
}

// Cuts nvec jobs over chunks of iters[k] CTA iterations (k < nck) into G CTA ranges.
// Returns the busiest CTA's cost in iterations: its iterations, item_cost per piece and
// load[k] each time the CTA starts on chunk k of another job or chunk; *equal_worst (if
// given) gets the same for ranges of equal iteration counts.  The ranges hold
// equal iteration counts, unless ranges of equal cost (those that give the CTAs which
// cross into another chunk fewer iterations) lower the busiest CTA's cost by 5 % or more;
// below that the model's error is larger than its gain (measured on GB300: 5 % faster on
// 8 x 65536 bins at 64 vectors for a model gain of 8 %, 1.5 % slower on 16 x 81920 for 2 %).
inline double cut_partition(const std::vector<int64_t>& iters, const std::vector<double>& load, int nvec, int G,
                            int max_piece, double item_cost, Partition* part, double* equal_worst = nullptr) {
  const int nck = static_cast<int>(iters.size());
  std::vector<int64_t> pre(nck + 1, 0);
  for (int k = 0; k < nck; ++k) pre[k + 1] = pre[k] + iters[k];
  const int64_t S = pre[nck], I = S * nvec;
  std::vector<int64_t> bounds(G + 1);
  for (int b = 0; b <= G; ++b) bounds[b] = I * b / G;
  const double equal = equal_cut_worst(iters, load, nvec, G, max_piece, item_cost);
  if (equal_worst) *equal_worst = equal;
  std::vector<int64_t> gb;
  double lo_t = static_cast<double>(I) / G, hi_t = equal;  // infeasible, feasible
  for (int it = 0; it < 40 && hi_t - lo_t > 1e-3; ++it) {
    const double mid = 0.5 * (lo_t + hi_t);
    (greedy_bounds(iters, load, nvec, G, max_piece, item_cost, mid, &gb) <= G ? hi_t : lo_t) = mid;
  }
  if (hi_t <= 0.95 * equal) {
    const int used = greedy_bounds(iters, load, nvec, G, max_piece, item_cost, hi_t, &gb);
    for (int b = 0; b <= G; ++b) bounds[b] = gb[std::min(b, used)];  // CTAs past the last range: none
  }
  part->grid = G;
  part->pieces.clear();
  part->cta.assign(G + 1, 0);
  part->chunk_rows.assign(static_cast<size_t>(nvec) * nck, int2{0, 0});
  part->rows.assign(nvec, 0);
  double worst = 0.0;
  for (int b = 0; b < G; ++b) {
    part->cta[b] = static_cast<int>(part->pieces.size());
    const int64_t lo = bounds[b], hi = bounds[b + 1];
    double cost = static_cast<double>(hi - lo);
    int pj = -1, pk = -1;
    for (int64_t q = lo; q < hi;) {
      const int j = static_cast<int>(q / S);
      const int64_t off = q - static_cast<int64_t>(j) * S;
      const int k = static_cast<int>(std::upper_bound(pre.begin(), pre.end(), off) - pre.begin()) - 1;
      const int64_t i0 = off - pre[k];
      const int64_t n = std::min<int64_t>({hi - q, iters[k] - i0, static_cast<int64_t>(max_piece)});
      int2& cr = part->chunk_rows[static_cast<size_t>(j) * nck + k];
      if (cr.y == 0) cr.x = part->rows[j];
      ++cr.y;
      part->pieces.push_back({j, k, static_cast<int>(i0), static_cast<int>(n), part->rows[j]++});
      cost += item_cost + (j != pj || k != pk ? load[k] : 0.0);
      pj = j;
      pk = k;
      q += n;
    }
    worst = std::max(worst, cost);
  }
  part->cta[G] = static_cast<int>(part->pieces.size());
  return worst;
}

// The compiled decomposition's busiest CTA in the same units: ceil(items / G) whole items of
// tile_iters iterations in a row, loading a chunk for the first and again each time the row
// crosses into another chunk (at most every min_tiles items).
inline double items_cost(int64_t nitems, int nvec, int G, int tile_iters, int min_tiles, double item_cost,
                         double max_load) {
  const int64_t per = (static_cast<int64_t>(nvec) * nitems + G - 1) / G;
  const int64_t mt = std::max(min_tiles, 1);
  const double switches = static_cast<double>(1 + (per - 1 + mt - 1) / mt);
  return static_cast<double>(per) * (tile_iters + item_cost) + switches * max_load;
}

}  // namespace musr
