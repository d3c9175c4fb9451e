// host_logic.cpp -- drives the library's host-only headers on the CPU for
// tests/test_host_logic.py: the BFGS state machine (musr_bfgs.h), SPLIT planning
// (musr_plan.h) and the decomposition cost model (musr_dev.h).  No GPU, no CUDA
// runtime: the headers are compiled by g++ with the CUDA vector types only.
#include <vector_types.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "musr.h"
#include "musr_bfgs.h"
#include "musr_dev.h"
#include "musr_partition.h"
#include "musr_plan.h"

using musr::Bfgs;

namespace {

// Runs the state machine on f with analytic gradient; prints one JSON object.
template <class F>
void run_bfgs(const char* name, std::vector<double> x0, F f, double gtol, int maxit) {
  const int P = static_cast<int>(x0.size());
  Bfgs b;
  b.start(x0.data(), P, gtol, maxit, 0.0, 1e-14);
  std::vector<double> pts, vals, grads;
  std::vector<int> sizes;
  while (!b.done()) {
    const int n = b.request(&pts);
    sizes.push_back(n);
    vals.assign(n, 0.0);
    grads.assign(static_cast<size_t>(n) * P, 0.0);
    for (int i = 0; i < n; ++i) vals[i] = f(pts.data() + static_cast<size_t>(i) * P, grads.data() + static_cast<size_t>(i) * P);
    b.deliver(vals.data(), grads.data());
  }
  std::printf("{\"name\": \"%s\", \"status\": %d, \"iters\": %d, \"nfev\": %d, \"f\": %.17g, \"x\": [", name, b.status(),
              b.iters(), b.nfev(), std::isfinite(b.f()) ? b.f() : -1.0);
  for (int i = 0; i < P; ++i) std::printf("%s%.17g", i ? ", " : "", b.x()[i]);
  std::printf("], \"first_requests\": [");
  for (size_t i = 0; i < sizes.size() && i < 4; ++i) std::printf("%s%d", i ? ", " : "", sizes[i]);
  std::printf("]}\n");
}

void bfgs_cases() {
  // Quadratic with a known minimum a and an SPD matrix A.
  const double a[4] = {1.5, -2.0, 0.25, 3.0};
  const double A[4][4] = {{4.0, 1.0, 0.0, 0.2}, {1.0, 3.0, 0.5, 0.0}, {0.0, 0.5, 2.0, 0.3}, {0.2, 0.0, 0.3, 1.0}};
  run_bfgs("quadratic", {0.0, 0.0, 0.0, 0.0},
           [&](const double* x, double* g) {
             double f = 0.0;
             for (int i = 0; i < 4; ++i) {
               g[i] = 0.0;
               for (int j = 0; j < 4; ++j) g[i] += A[i][j] * (x[j] - a[j]);
               f += 0.5 * (x[i] - a[i]) * g[i];
             }
             return f;
           },
           1e-12, 200);
  // Rosenbrock: minimum 0 at (1, 1).
  run_bfgs("rosenbrock", {-1.2, 1.0},
           [](const double* x, double* g) {
             const double u = x[1] - x[0] * x[0], v = 1.0 - x[0];
             g[0] = -400.0 * x[0] * u - 2.0 * v;
             g[1] = 200.0 * u;
             return 100.0 * u * u + v * v;
           },
           1e-10, 500);
  // A start where the cost is not finite ends at once with status 1.
  run_bfgs("nonfinite", {1.0},
           [](const double*, double* g) {
             g[0] = 0.0;
             return INFINITY;
           },
           1e-8, 10);
}

musr_term term(std::initializer_list<std::pair<int, std::pair<int, int>>> prims) {
  musr_term t;
  std::memset(&t, 0, sizeof(t));
  for (const auto& p : prims) {
    t.kind[t.nprim] = p.first;
    t.slot[t.nprim][0] = p.second.first;
    t.slot[t.nprim][1] = p.second.second;
    ++t.nprim;
  }
  return t;
}

void plan_case(const char* name, const std::vector<musr_term>& terms, const std::vector<int32_t>& map, int H,
               int nslots, const std::vector<double>& consts) {
  musr::HistSet hs;
  std::memset(&hs, 0, sizeof(hs));
  const char* why = musr::plan_split(terms.data(), static_cast<int>(terms.size()), map.data(), H, nslots,
                                     consts.empty() ? nullptr : consts.data(), &hs);
  std::printf("{\"name\": \"%s\", \"ok\": %s, \"shape\": %d, \"merged\": %d, \"kinds\": [", name, why ? "false" : "true",
              why ? -1 : hs.shape, why ? 0 : hs.merged);
  for (int k = 0; k < (why ? 0 : hs.nterms); ++k) std::printf("%s%d", k ? ", " : "", hs.canon[k].kind);
  std::printf("], \"bamp\": [");
  for (int k = 0; k < (why ? 0 : hs.nterms); ++k) std::printf("%s%.17g", k ? ", " : "", hs.bamp[k]);
  std::printf("], \"contrib\": [");
  for (int e = 0; e < (why ? 0 : hs.ncontrib); ++e)
    std::printf("%s[%d, %d, %d]", e ? ", " : "", hs.contrib[e].slot, hs.contrib[e].kind, hs.contrib[e].term);
  std::printf("]}\n");
}

void plan_cases() {
  const int A = MUSR_PRIM_AMP, E = MUSR_PRIM_EXP, G = MUSR_PRIM_GAUSS, K = MUSR_PRIM_KT, T = MUSR_PRIM_TFCOS,
            L = MUSR_PRIM_LKT;
  // Two cosine terms, constant equal amplitudes, one phase per histogram: merged.
  const std::vector<musr_term> tf2 = {term({{A, {2, 0}}, {E, {3, 0}}, {T, {4, 5}}}),
                                      term({{A, {6, 0}}, {G, {7, 0}}, {T, {8, 5}}})};
  std::vector<int32_t> m2;
  for (int h = 0; h < 3; ++h) {
    const int32_t row[9] = {10 + 2 * h, 11 + 2 * h, -1, 0, 1, 16 + h, -2, 2, 3};
    m2.insert(m2.end(), row, row + 9);
  }
  plan_case("tf2_merged", tf2, m2, 3, 9, {0.125, 0.1});
  // The same with the second cosine on its own phase slot: not merged.
  std::vector<int32_t> m2b = m2;
  const std::vector<musr_term> tf2b = {term({{A, {2, 0}}, {E, {3, 0}}, {T, {4, 5}}}),
                                       term({{A, {6, 0}}, {G, {7, 0}}, {T, {8, 2}}})};
  plan_case("tf2_own_phases", tf2b, m2b, 3, 9, {0.125, 0.1});
  // Amplitude constants that differ between histograms: not merged.
  std::vector<int32_t> m2c = m2;
  m2c[9 + 2] = -3;
  plan_case("tf2_amp_per_hist", tf2, m2c, 3, 9, {0.125, 0.1, 0.2});
  // Terms given non-cosine first are reordered, cosine first.
  const std::vector<musr_term> mix = {term({{A, {2, 0}}, {K, {3, 0}}}), term({{A, {4, 0}}, {E, {5, 0}}, {T, {6, 7}}})};
  const std::vector<int32_t> mm = {0, 1, 2, 3, 4, 5, 6, 7};
  plan_case("kt_then_tf", mix, mm, 1, 8, {});
  const std::vector<musr_term> lkt = {term({{A, {2, 0}}, {L, {3, 0}}, {E, {4, 0}}})};
  const std::vector<int32_t> ml = {0, 1, 2, 3, 4};
  plan_case("lkt", lkt, ml, 1, 5, {});
  // Two cosines in one term cannot be split into basis functions.
  const std::vector<musr_term> bad = {term({{A, {2, 0}}, {T, {3, 4}}, {T, {5, 4}}})};
  const std::vector<int32_t> mb = {0, 1, 2, 3, 4, 5};
  plan_case("two_cosines", bad, mb, 1, 6, {});
  // Four terms without a common shape: generic.
  const std::vector<musr_term> gen = {term({{A, {2, 0}}, {E, {3, 0}}}), term({{A, {4, 0}}, {G, {5, 0}}}),
                                      term({{A, {6, 0}}, {K, {7, 0}}}), term({{A, {8, 0}}, {T, {9, 10}}})};
  const std::vector<int32_t> mg = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10};
  plan_case("generic4", gen, mg, 1, 11, {});
  // A dynamic Kubo-Toyabe factor is a time-only factor like the static one: a basis term
  // with a Delta and a nu contribution, reordered after the cosine.
  const int D = MUSR_PRIM_DKT;
  const std::vector<musr_term> dkt = {term({{A, {2, 0}}, {D, {3, 4}}, {E, {5, 0}}}),
                                      term({{A, {6, 0}}, {T, {7, 8}}})};
  const std::vector<int32_t> md = {0, 1, 2, 3, 4, 5, 6, 7, 8};
  plan_case("dkt_then_tf", dkt, md, 1, 9, {});
  // ... but not beside a cosine in the same term.
  const std::vector<musr_term> dkt_tf = {term({{A, {2, 0}}, {D, {3, 4}}, {T, {5, 6}}})};
  const std::vector<int32_t> mdt = {0, 1, 2, 3, 4, 5, 6};
  plan_case("dkt_times_cosine", dkt_tf, mdt, 1, 7, {});
}

void pick_cases() {
  // Items of one evaluation for tiles of 512 << v bins.
  const int cfg2[musr::kVariants] = {128, 64, 32, 16, 8, 4, 2};
  for (int nvec : {1, 8, 64, 152}) {
    std::printf("{\"name\": \"pick\", \"nvec\": %d, \"v\": %d, \"costs\": [", nvec,
                musr::pick_decomposition(cfg2, nvec, 304, 1.3));
    for (int v = 0; v < musr::kVariants; ++v) {
      const long long per = (static_cast<long long>(nvec) * cfg2[v] + 303) / 304;
      std::printf("%s%.6g", v ? ", " : "", per * ((1 << v) + 1.3));
    }
    std::printf("]}\n");
  }
}

void partition_case(const char* name, const std::vector<int64_t>& iters, const std::vector<double>& load, int nvec,
                    int G, int max_piece, double item_cost) {
  musr::Partition part;
  double equal = 0.0;
  const double worst = musr::cut_partition(iters, load, nvec, G, max_piece, item_cost, &part, &equal);
  std::printf("{\"name\": \"%s\", \"worst\": %.17g, \"equal\": %.17g, \"grid\": %d, \"pieces\": [", name, worst,
              equal, part.grid);
  for (size_t i = 0; i < part.pieces.size(); ++i) {
    const musr::Piece& p = part.pieces[i];
    std::printf("%s[%d, %d, %d, %d, %d]", i ? ", " : "", p.job, p.chunk, p.it0, p.nit, p.row);
  }
  std::printf("], \"cta\": [");
  for (size_t i = 0; i < part.cta.size(); ++i) std::printf("%s%d", i ? ", " : "", part.cta[i]);
  std::printf("], \"chunk_rows\": [");
  for (size_t i = 0; i < part.chunk_rows.size(); ++i)
    std::printf("%s[%d, %d]", i ? ", " : "", part.chunk_rows[i].x, part.chunk_rows[i].y);
  std::printf("], \"rows\": [");
  for (size_t i = 0; i < part.rows.size(); ++i) std::printf("%s%d", i ? ", " : "", part.rows[i]);
  std::printf("], \"items_cost\": %.17g}\n", musr::items_cost(10, nvec, G, 8, 5, item_cost, 2.4));
}

void partition_cases() {
  partition_case("paper_64", {160, 160}, {2.4, 2.4}, 64, 304, 64, 1.3);
  partition_case("cfg2_64", {128}, {2.4}, 64, 304, 64, 1.3);
  partition_case("uneven", {7, 100, 33}, {1.0, 2.0, 3.0}, 5, 13, 16, 1.3);
  partition_case("long", {2048, 2048, 2048}, {2.4, 2.4, 2.4}, 3, 7, 64, 1.3);
  partition_case("tiny", {3, 5}, {1.0, 2.0}, 3, 4, 2, 0.5);
  partition_case("cfg2_64_chi2", {128}, {3.6}, 64, 304, 64, 1.95);
  partition_case("paper_8", {160, 160}, {2.4, 2.4}, 8, 304, 64, 1.3);
}

// One case per line of standard input: nck, then nck chunk iterations, nck loads, nvec, G,
// the largest piece and the piece cost; the cases are named by their line number.
void partition_stdin() {
  int nck, line = 0;
  while (std::scanf("%d", &nck) == 1 && nck > 0) {
    std::vector<int64_t> iters(nck);
    std::vector<double> load(nck);
    for (auto& v : iters) {
      long long x = 0;
      if (std::scanf("%lld", &x) != 1) return;
      v = x;
    }
    for (auto& v : load)
      if (std::scanf("%lf", &v) != 1) return;
    int nvec, G, max_piece;
    double item_cost;
    if (std::scanf("%d %d %d %lf", &nvec, &G, &max_piece, &item_cost) != 4) return;
    const std::string name = std::to_string(line++);
    partition_case(name.c_str(), iters, load, nvec, G, max_piece, item_cost);
  }
}

}  // namespace

int main(int argc, char** argv) {
  const std::string what = argc > 1 ? argv[1] : "";
  if (what == "bfgs") bfgs_cases();
  if (what == "plan") plan_cases();
  if (what == "pick") pick_cases();
  if (what == "partition") partition_cases();
  if (what == "partition_stdin") partition_stdin();
  return 0;
}
