// musr_partition.h -- host-side launch-level partition of a batch for the SPLIT basis kernels.
//
// A compiled decomposition hands out whole items (a chunk's tile for one parameter vector), so
// a batch whose items do not divide evenly over the persistent grid leaves CTAs idle or with
// an extra item.  The partition cuts the batch's CTA iterations -- in the order job, chunk,
// iteration -- into one contiguous, equal range per CTA; a range's share of a chunk becomes
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

// Cuts nvec jobs over chunks of iters[k] CTA iterations (k < nck) into G CTA ranges.
// Returns the busiest CTA's cost in iterations: its iterations, item_cost per piece and
// load[k] each time the CTA starts on chunk k of another job or chunk.
inline double cut_partition(const std::vector<int64_t>& iters, const std::vector<double>& load, int nvec, int G,
                            int max_piece, double item_cost, Partition* part) {
  const int nck = static_cast<int>(iters.size());
  std::vector<int64_t> pre(nck + 1, 0);
  for (int k = 0; k < nck; ++k) pre[k + 1] = pre[k] + iters[k];
  const int64_t S = pre[nck], I = S * nvec;
  part->grid = G;
  part->pieces.clear();
  part->cta.assign(G + 1, 0);
  part->chunk_rows.assign(static_cast<size_t>(nvec) * nck, int2{0, 0});
  part->rows.assign(nvec, 0);
  double worst = 0.0;
  for (int b = 0; b < G; ++b) {
    part->cta[b] = static_cast<int>(part->pieces.size());
    const int64_t lo = I * b / G, hi = I * (b + 1) / G;
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
