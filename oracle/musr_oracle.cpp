// musr_oracle.cpp -- plain, slow, single-threaded FP64 CPU oracle for the
// muSR chi^2 / Poisson -2lnL cost of arXiv 1509.07685, Section 4.
//
// TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path is
// checked against.  Only the test suite, the smoke check and the CPU-baseline
// leg of the benchmark may load it.  It shares no code, header, table or
// constant generator with the CUDA library; the two agree only through the
// definitions of the paper restated below.
//
// What it computes (Section 4.1):
//   Eq. positron_histo   N^j(t) = N0^j exp(-t/tau_mu) [1 + A^j(p, t)] + Nbkg^j
//                        at discrete times t = n * dt (here t_n = (n - t0_j) * dt)
//   Eq. chisq            chi^2 = sum_j sum_n (d - N)^2 / d_err^2,  d_err^2 = d
//                        (read as max(d, 1) so that empty bins are defined)
//   Eq. log-likelihood   L = 2 sum_j sum_n { (N - d) + d log(d/N)   d > 0
//                                            (N - d)                d <= 0 }
//                        (the Poisson deviance; minimised, zero iff N == d)
//   Eq. asymmetry        A(t) = A0 exp(-(sigma t)^2 / 2) cos(gamma_mu B t + phi)
//                        generalised to a sum of terms, each a product of the
//                        primitives AMP, EXP, GAUSS, KT (static Gaussian
//                        Kubo-Toyabe), TFCOS.
//
// Readings of the paper that this oracle fixes (the paper leaves them open):
//   * tau_mu = 2.197019 us.
//   * t_n = (n - t0_j) * (bin_width_ns / 1000.0) in microseconds, t0_j in
//     (possibly fractional) bins; bin n is in the fit when lo <= t_n <= hi.
//   * TFCOS(nu, phi) = cos(2 pi (nu t + phi / 360)), nu in MHz, phi in degrees
//     (gamma_mu B = 2 pi nu).
//   * GAUSS(sigma) = exp(-(sigma t)^2 / 2), EXP(lambda) = exp(-lambda t).
//   * KT(Delta) = 1/3 + 2/3 (1 - Delta^2 t^2) exp(-Delta^2 t^2 / 2).
//   * LKT(a) = 1/3 + 2/3 (1 - a t) exp(-a t), the static Lorentzian Kubo-Toyabe
//     relaxation (a: the Lorentzian field width times gamma_mu).
//   * STREXP(lambda, beta) = exp(-(|lambda| t)^beta) for t > 0 and 1 for t <= 0 (the
//     relaxation starts at time zero), the stretched exponential.
//   * BESSEL(nu, phi) = J0(2 pi (nu t + phi / 360)), precession in an incommensurate
//     field distribution, the phase inside the argument like TFCOS.
//   * DKT(Delta, nu): the dynamic Gaussian Kubo-Toyabe relaxation of the strong-collision
//     model, the solution of a renewal equation (see dkt_solve below); 1 for t <= 0.
//   * Local slot 0 is N0, slot 1 is Nbkg; terms reference any slot.
//   * MLE with N <= 0 in a bin with d > 0 is +infinity (status 1).
//
// Asymmetry data (the form A(t) of Eq. asymmetry is measured directly): a forward /
// backward histogram pair (F, B) with relative efficiency alpha and constant backgrounds
// gives, with f = F - bkg_F and b = B - bkg_B,
//     a = (f - alpha b) / (f + alpha b),
//     sigma_a^2 = 4 alpha^2 (b^2 var F + f^2 var B) / (f + alpha b)^4
// (first-order propagation of Poisson errors, each count's variance read as
// max(count, 1) like Eq. chisq's d_err^2), weight w = 1 / sigma_a^2, and w = 0 where
// f + alpha b <= 0.  The model of asymmetry data drops the decay envelope:
//     T(t) = N0 A(t) + Nbkg   (N0 a scale, usually the constant 1; Nbkg a baseline),
// and the cost is chi^2 = sum w (a - T)^2.  -2lnL is not defined for it (status 2).
//
// The file also holds the direct-summation oracle of the paper's particle-mesh Poisson
// solve (Section 3, Eq. openbruteforceconv), at its end.
//
// Summation: every sum over bins is Neumaier-compensated, in bin order
// (histogram-major), so that the oracle's own rounding stays far below the
// 1e-12 relative tolerance used against the GPU path.
//
// The value function is a template on the scalar type so that the same code,
// instantiated on std::complex<double>, yields the complex-step derivative
// (Squire & Trapp 1998) used to pin the analytic gradient.

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <tuple>
#include <vector>

namespace {

constexpr double kTauMu = 2.197019;  // muon lifetime in microseconds
constexpr double kPi = 3.14159265358979323846;

enum PrimKind { kAmp = 1, kExp = 2, kGauss = 3, kKT = 4, kTFCos = 5, kLKT = 6, kStrExp = 7, kBessel = 8, kDKT = 9 };
constexpr int kMaxPrim = 4;

using cplx = std::complex<double>;

inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }

// Neumaier's improvement of Kahan summation, one real accumulator.
struct Neumaier {
  double s = 0.0, c = 0.0;
  void add(double x) {
    double t = s + x;
    if (std::fabs(s) >= std::fabs(x))
      c += (s - t) + x;
    else
      c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

// Complex accumulator: real and imaginary parts compensated separately.
struct NeumaierC {
  Neumaier r, i;
  void add(const cplx& x) { r.add(x.real()); i.add(x.imag()); }
  void add(double x) { r.add(x); }
  cplx value() const { return cplx(r.value(), i.value()); }
};

template <class T> struct AccFor;
template <> struct AccFor<double> { using type = Neumaier; };
template <> struct AccFor<cplx> { using type = NeumaierC; };

struct Theory {
  int nterms;
  const int32_t* nprim;  // [nterms]
  const int32_t* kind;   // [nterms][kMaxPrim]
  const int32_t* slot;   // [nterms][kMaxPrim][2]
};

struct Problem {
  const double* data;  // [H][B], histogram-major (counts, or asymmetry values)
  const double* weight;  // [H][B] chi^2 weights of asymmetry data; nullptr for counts
  int envelope;          // 1: Eq. positron_histo; 0: asymmetry model N0 A + Nbkg
  int H;
  int64_t B;
  const double* t0;  // [H], in bins
  double dt_us;
  double lo, hi;  // fit range, microseconds, closed
  Theory th;
  const int32_t* map;  // [H][nslots]: >= 0 global parameter, < 0 -> consts[-1-k]
  int nslots;
  const double* consts;
  int nconsts;
  int P;
};

// Time of bin n of histogram h (Section 4.1, t = n * dt, shifted by t0).
inline double bin_time(const Problem& pb, int h, int64_t n) {
  return (static_cast<double>(n) - pb.t0[h]) * pb.dt_us;
}

inline bool in_fit(const Problem& pb, double t) { return pb.lo <= t && t <= pb.hi; }

// Value of local slot s of histogram h for parameter vector x.
template <class T>
T slot_value(const Problem& pb, const T* x, int h, int s) {
  int32_t m = pb.map[static_cast<int64_t>(h) * pb.nslots + s];
  if (m >= 0) return x[m];
  return T(pb.consts[-1 - m]);
}

// J0 and J1 (C++17 special functions, defined for x >= 0; J0 is even and J1 odd).
inline double bessel_j0(double x) { return std::cyl_bessel_j(0.0, std::fabs(x)); }
inline double bessel_j1(double x) { return x < 0.0 ? -std::cyl_bessel_j(1.0, -x) : std::cyl_bessel_j(1.0, x); }
// J0 at a complex argument x + i y with |y| tiny (the complex step): J0(x) - i y J1(x),
// exact to O(y^2).
inline cplx bessel_j0(const cplx& z) { return cplx(bessel_j0(z.real()), -z.imag() * bessel_j1(z.real())); }

// ---------------------------------------------------------------------------------------
// Dynamic Gaussian Kubo-Toyabe relaxation, strong-collision model (primitive DKT; slot 0 the
// static width Delta, slot 1 the fluctuation rate nu, both in 1/us).  Not in the paper: one
// of the "user defined functions" of Section 4.1.  The local field is drawn from the
// isotropic Gaussian of width Delta / gamma_mu and drawn anew at the events of a Poisson
// process of rate nu.  Between two events the muon precesses in a static field; averaged
// over that field, an interval of length s multiplies the polarisation by the static
// function g(s) = 1/3 + 2/3 (1 - Delta^2 s^2) exp(-Delta^2 s^2 / 2).  Summing over the
// number of events gives the renewal (Volterra) equation of the second kind
//     G(t) = f(t) + nu int_0^t f(s) G(t - s) ds,    f(t) = g(t) exp(-nu t),
// whose solution G is the relaxation.  It has no closed form.  The oracle solves it on the
// uniform grid t_k = k h of [0, span] by the trapezoidal rule (f_0 = G_0 = 1):
//     (1 - nu h / 2) G_k = (1 + nu h / 2) f_k + nu h sum_{j=1}^{k-1} f_j G_{k-j},
// removes the rule's h^2 error term by Richardson extrapolation, (4 G_{h/2} - G_h) / 3 at the
// points of the coarser grid, and interpolates with the cubic through the four nearest grid
// points.  The derivatives with respect to Delta and nu solve the same recursion
// differentiated (df/dDelta = dg/dDelta exp(-nu t), df/dnu = -t f).  For t <= 0 the
// relaxation is 1: it starts at time zero.
// ---------------------------------------------------------------------------------------

// The grid's end (microseconds): the last time in the fit of the problem being evaluated
// (set by every entry point; the oracle is single-threaded).
double g_dkt_span = 1.0;

// The static function g and its Delta-derivative at time t.
template <class T>
T dkt_static(const T& D, double t) {
  const T u = (D * t) * (D * t);
  return 1.0 / 3.0 + (2.0 / 3.0) * (1.0 - u) * std::exp(-0.5 * u);
}
inline double dkt_static_dD(double D, double t) {
  const double u = (D * t) * (D * t);
  return (2.0 / 3.0) * D * t * t * std::exp(-0.5 * u) * (u - 3.0);
}

// Trapezoidal solution on K + 1 points t_k = k h: G, and when dG is given the derivatives
// dG[0] (Delta) and dG[1] (nu) (real arithmetic only).
template <class T>
void dkt_solve(const T& D, const T& nu, double h, int K, std::vector<T>* G, std::vector<double>* dG) {
  std::vector<T> f(K + 1);
  for (int k = 0; k <= K; ++k) f[k] = dkt_static(D, k * h) * std::exp(-nu * (k * h));
  const T a = 1.0 - nu * (0.5 * h), b = 1.0 + nu * (0.5 * h), c = nu * h;
  G->assign(K + 1, T(0.0));
  (*G)[0] = T(1.0);
  std::vector<double> S;  // S_k = sum_{j=1}^{k-1} f_j G_{k-j}, kept for the nu-derivative
  if (dG) S.assign(K + 1, 0.0);
  for (int k = 1; k <= K; ++k) {
    T sk = T(0.0);
    for (int j = 1; j < k; ++j) sk = sk + f[j] * (*G)[k - j];
    (*G)[k] = (b * f[k] + c * sk) / a;
    if (dG) S[k] = re(sk);
  }
  if (!dG) return;
  const double Dr = re(D), nr = re(nu), ar = re(a), br = re(b), cr = re(c);
  std::vector<double> fD(K + 1), fn(K + 1);
  for (int k = 0; k <= K; ++k) {
    fD[k] = dkt_static_dD(Dr, k * h) * std::exp(-nr * (k * h));
    fn[k] = -(k * h) * re(f[k]);
  }
  dG[0].assign(K + 1, 0.0);
  dG[1].assign(K + 1, 0.0);
  for (int k = 1; k <= K; ++k) {
    double sD = 0.0, sn = 0.0;
    for (int j = 1; j < k; ++j) {
      sD += fD[j] * re((*G)[k - j]) + re(f[j]) * dG[0][k - j];
      sn += fn[j] * re((*G)[k - j]) + re(f[j]) * dG[1][k - j];
    }
    dG[0][k] = (br * fD[k] + cr * sD) / ar;
    // d/dnu of a G_k = b f_k + c S_k, with da/dnu = -h/2, db/dnu = h/2, dc/dnu = h
    dG[1][k] = (0.5 * h * (re((*G)[k]) + re(f[k])) + br * fn[k] + h * S[k] + cr * sn) / ar;
  }
}

// Points of the coarse grid over [0, span]: enough that h max(Delta, nu) stays near 0.004.
inline int dkt_points(double D, double nu, double span) {
  const double rate = std::fmax(std::fmax(std::fabs(D), std::fabs(nu)), 0.05);
  const double k = std::ceil(span * rate / 0.004);
  return static_cast<int>(std::fmin(std::fmax(k, 1024.0), 32768.0));
}

template <class T>
struct DktTable {
  double h = 0.0;
  int K = 0;
  std::vector<T> G;      // Richardson-extrapolated values at t_k = k h, k = 0..K
  std::vector<double> dG[2];  // derivatives (real tables only)
};

template <class T>
std::shared_ptr<DktTable<T>> dkt_build(const T& D, const T& nu, double span, bool derivs) {
  auto tab = std::make_shared<DktTable<T>>();
  const int K = dkt_points(re(D), re(nu), span);
  const double h = span / K;
  std::vector<T> Gh, Gh2;
  std::vector<double> dh[2], dh2[2];
  dkt_solve(D, nu, h, K, &Gh, derivs ? dh : nullptr);
  dkt_solve(D, nu, 0.5 * h, 2 * K, &Gh2, derivs ? dh2 : nullptr);
  tab->h = h;
  tab->K = K;
  tab->G.resize(K + 1);
  for (int k = 0; k <= K; ++k) tab->G[k] = (4.0 * Gh2[2 * k] - Gh[k]) / 3.0;
  if (derivs)
    for (int q = 0; q < 2; ++q) {
      tab->dG[q].resize(K + 1);
      for (int k = 0; k <= K; ++k) tab->dG[q][k] = (4.0 * dh2[q][2 * k] - dh[q][k]) / 3.0;
    }
  return tab;
}

// Cubic through the four grid points nearest to t (one-sided at the ends of the grid).
template <class T, class V>
T dkt_interp(const V& y, double h, int K, double t) {
  const double x = t / h;
  int i = static_cast<int>(std::floor(x)) - 1;  // stencil i .. i + 3 around [i + 1, i + 2]
  if (i < 0) i = 0;
  if (i > K - 3) i = K - 3;
  const double u = x - i;  // position in units of h from point i
  const double w0 = -(u - 1.0) * (u - 2.0) * (u - 3.0) / 6.0, w1 = u * (u - 2.0) * (u - 3.0) / 2.0;
  const double w2 = -u * (u - 1.0) * (u - 3.0) / 2.0, w3 = u * (u - 1.0) * (u - 2.0) / 6.0;
  return w0 * y[i] + w1 * y[i + 1] + w2 * y[i + 2] + w3 * y[i + 3];
}

inline double key_im(double) { return 0.0; }
inline double key_im(const cplx& z) { return z.imag(); }

// The table of (Delta, nu) over [0, span], built on first use (a cache of recent ones).
template <class T>
std::shared_ptr<DktTable<T>> dkt_table(const T& D, const T& nu, double span, bool derivs) {
  using Key = std::tuple<double, double, double, double, double, bool>;
  static std::map<Key, std::shared_ptr<DktTable<T>>> cache;
  const Key key(re(D), key_im(D), re(nu), key_im(nu), span, derivs);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  if (cache.size() > 64) cache.clear();
  auto tab = dkt_build(D, nu, span, derivs);
  cache[key] = tab;
  return tab;
}

template <class T>
T dkt_value(const T& D, const T& nu, double t) {
  if (!(t > 0.0)) return T(1.0);
  const double span = std::fmax(g_dkt_span, t);
  auto tab = dkt_table(D, nu, span, false);
  return dkt_interp<T>(tab->G, tab->h, tab->K, t);
}

inline void dkt_derivs(double D, double nu, double t, double* dD, double* dnu) {
  if (!(t > 0.0)) {
    *dD = *dnu = 0.0;
    return;
  }
  const double span = std::fmax(g_dkt_span, t);
  auto tab = dkt_table(D, nu, span, true);
  *dD = dkt_interp<double>(tab->dG[0], tab->h, tab->K, t);
  *dnu = dkt_interp<double>(tab->dG[1], tab->h, tab->K, t);
}

// |lambda| for the stretched exponential: the sign folded analytically on each side.
inline double fold_sign(double v) { return v < 0.0 ? -v : v; }
inline cplx fold_sign(const cplx& v) { return v.real() < 0.0 ? -v : v; }

// One primitive factor of a term of A(t) (Eq. asymmetry and its generalisation).
template <class T>
T primitive(int kind, const T& p0, const T& p1, double t) {
  switch (kind) {
    case kAmp:
      return p0;
    case kExp:
      return std::exp(-p0 * t);
    case kGauss:
      return std::exp(-0.5 * (p0 * t) * (p0 * t));
    case kKT: {
      T u = (p0 * t) * (p0 * t);
      return 1.0 / 3.0 + (2.0 / 3.0) * (1.0 - u) * std::exp(-0.5 * u);
    }
    case kTFCos:
      return std::cos(2.0 * kPi * (p0 * t + p1 / 360.0));
    case kLKT: {
      T u = p0 * t;
      return 1.0 / 3.0 + (2.0 / 3.0) * (1.0 - u) * std::exp(-u);
    }
    case kStrExp: {
      const T x = fold_sign(p0) * t;
      if (!(t > 0.0) || re(x) == 0.0) return T(1.0);
      return std::exp(-std::pow(x, p1));
    }
    case kBessel:
      return bessel_j0(2.0 * kPi * (p0 * t + p1 / 360.0));
    case kDKT:
      return dkt_value(p0, p1, t);
    default:
      return T(std::numeric_limits<double>::quiet_NaN());
  }
}

// Derivatives of one primitive with respect to its first and second slot.
inline void primitive_deriv(int kind, double p0, double p1, double t, double* d0, double* d1) {
  *d0 = 0.0;
  *d1 = 0.0;
  switch (kind) {
    case kAmp:
      *d0 = 1.0;
      break;
    case kExp:
      *d0 = -t * std::exp(-p0 * t);
      break;
    case kGauss:
      *d0 = -p0 * t * t * std::exp(-0.5 * (p0 * t) * (p0 * t));
      break;
    case kKT: {
      double u = (p0 * t) * (p0 * t);
      *d0 = (2.0 / 3.0) * p0 * t * t * std::exp(-0.5 * u) * (u - 3.0);
      break;
    }
    case kTFCos: {
      double s = std::sin(2.0 * kPi * (p0 * t + p1 / 360.0));
      *d0 = -s * 2.0 * kPi * t;
      *d1 = -s * 2.0 * kPi / 360.0;
      break;
    }
    case kLKT: {
      double u = p0 * t;
      *d0 = (2.0 / 3.0) * t * std::exp(-u) * (u - 2.0);
      break;
    }
    case kStrExp: {
      const double lam = std::fabs(p0), x = lam * t;
      if (!(t > 0.0) || x == 0.0) break;
      const double xb = std::pow(x, p1), f = std::exp(-xb);
      *d0 = (p0 < 0.0 ? -1.0 : 1.0) * (-p1 * xb / lam) * f;  // d/dlambda
      *d1 = -xb * std::log(x) * f;                             // d/dbeta
      break;
    }
    case kBessel: {
      const double j1 = bessel_j1(2.0 * kPi * (p0 * t + p1 / 360.0));  // J0' = -J1
      *d0 = -j1 * 2.0 * kPi * t;
      *d1 = -j1 * 2.0 * kPi / 360.0;
      break;
    }
    case kDKT:
      dkt_derivs(p0, p1, t, d0, d1);
      break;
    default:
      break;
  }
}

inline int nslots_of(int kind) {
  return kind == kTFCos || kind == kStrExp || kind == kBessel || kind == kDKT ? 2 : 1;
}

// Eq. positron_histo for histogram h at time t.
template <class T>
T model(const Problem& pb, const T* x, int h, double t) {
  T A = T(0.0);
  for (int k = 0; k < pb.th.nterms; ++k) {
    T term = T(1.0);
    for (int m = 0; m < pb.th.nprim[k]; ++m) {
      int kind = pb.th.kind[k * kMaxPrim + m];
      const int32_t* sl = pb.th.slot + (k * kMaxPrim + m) * 2;
      T p0 = slot_value(pb, x, h, sl[0]);
      T p1 = nslots_of(kind) == 2 ? slot_value(pb, x, h, sl[1]) : T(0.0);
      term = term * primitive(kind, p0, p1, t);
    }
    A = A + term;
  }
  T N0 = slot_value(pb, x, h, 0);
  T Nbkg = slot_value(pb, x, h, 1);
  if (!pb.envelope) return N0 * A + Nbkg;
  return N0 * std::exp(-t / kTauMu) * (1.0 + A) + Nbkg;
}

// One bin's contribution to Eq. chisq (mode 0) or Eq. log-likelihood (mode 1).
// w >= 0 is the given chi^2 weight of asymmetry data (w < 0: counts).
// Sets *bad when the likelihood is undefined (N <= 0 where d > 0).
template <class T>
T bin_cost(int mode, double d, double w, const T& N, bool* bad) {
  if (mode == 0) {
    T r = d - N;
    if (w >= 0.0) return w * r * r;
    return r * r / std::fmax(d, 1.0);
  }
  if (d > 0.0) {
    if (re(N) <= 0.0) {
      *bad = true;
      return T(0.0);
    }
    return 2.0 * ((N - d) + d * std::log(d / N));
  }
  return 2.0 * (N - d);
}

// The chi^2 weight of bin n of histogram h: given for asymmetry data, else -1.
inline double bin_weight(const Problem& pb, int h, int64_t n) {
  return pb.weight ? pb.weight[static_cast<int64_t>(h) * pb.B + n] : -1.0;
}

template <class T>
int cost_value(const Problem& pb, const T* x, int mode, T* out) {
  typename AccFor<T>::type acc;
  bool bad = false;
  if (pb.weight && mode != 0) return 2;
  for (int h = 0; h < pb.H; ++h) {
    const double* row = pb.data + static_cast<int64_t>(h) * pb.B;
    for (int64_t n = 0; n < pb.B; ++n) {
      double t = bin_time(pb, h, n);
      if (!in_fit(pb, t)) continue;
      T N = model(pb, x, h, t);
      acc.add(bin_cost(mode, row[n], bin_weight(pb, h, n), N, &bad));
    }
  }
  if (bad) {
    *out = T(std::numeric_limits<double>::infinity());
    return 1;
  }
  *out = acc.value();
  return 0;
}

// Expected count N of histogram h at time t (Eq. positron_histo) and its derivative with
// respect to every local slot, through the product rule of each term.
double model_and_slot_derivs(const Problem& pb, const double* x, int h, double t, double* dslot) {
  const double N0 = slot_value(pb, x, h, 0);
  const double E = pb.envelope ? std::exp(-t / kTauMu) : 1.0;
  std::fill(dslot, dslot + pb.nslots, 0.0);
  double A = 0.0;
  for (int k = 0; k < pb.th.nterms; ++k) {
    int np = pb.th.nprim[k];
    double f[kMaxPrim], p0[kMaxPrim], p1[kMaxPrim];
    for (int m = 0; m < np; ++m) {
      int kind = pb.th.kind[k * kMaxPrim + m];
      const int32_t* sl = pb.th.slot + (k * kMaxPrim + m) * 2;
      p0[m] = slot_value(pb, x, h, sl[0]);
      p1[m] = nslots_of(kind) == 2 ? slot_value(pb, x, h, sl[1]) : 0.0;
      f[m] = primitive(kind, p0[m], p1[m], t);
    }
    double term = 1.0;
    for (int m = 0; m < np; ++m) term *= f[m];
    A += term;
    for (int m = 0; m < np; ++m) {
      int kind = pb.th.kind[k * kMaxPrim + m];
      const int32_t* sl = pb.th.slot + (k * kMaxPrim + m) * 2;
      double rest = 1.0;
      for (int q = 0; q < np; ++q)
        if (q != m) rest *= f[q];
      double d0, d1;
      primitive_deriv(kind, p0[m], p1[m], t, &d0, &d1);
      dslot[sl[0]] += N0 * E * d0 * rest;
      if (nslots_of(kind) == 2) dslot[sl[1]] += N0 * E * d1 * rest;
    }
  }
  if (!pb.envelope) {  // asymmetry model N0 A + Nbkg
    dslot[0] += A;
    dslot[1] += 1.0;
    return N0 * A + slot_value(pb, x, h, 1);
  }
  dslot[0] += E * (1.0 + A);
  dslot[1] += 1.0;
  return N0 * E * (1.0 + A) + slot_value(pb, x, h, 1);
}

// Value plus analytic gradient: dcost/dx_p = sum over bins of
// (dcost/dN) * sum over (slot s of hist h mapped to p) dN/d(slot s).
// gscale[p] accumulates sum |per-bin contribution|, the scale against which
// the GPU gradient tolerance is stated.
int cost_grad(const Problem& pb, const double* x, int mode, double* value, double* grad,
              double* gscale) {
  Neumaier acc;
  std::vector<Neumaier> g(pb.P), gs(pb.P);
  std::vector<double> dslot(pb.nslots);
  bool bad = false;
  if (pb.weight && mode != 0) return 2;
  for (int h = 0; h < pb.H; ++h) {
    const double* row = pb.data + static_cast<int64_t>(h) * pb.B;
    for (int64_t n = 0; n < pb.B; ++n) {
      double t = bin_time(pb, h, n);
      if (!in_fit(pb, t)) continue;
      double d = row[n];
      double N = model_and_slot_derivs(pb, x, h, t, dslot.data());
      double W;  // dcost / dN for this bin
      const double w = bin_weight(pb, h, n);
      if (mode == 0 && w >= 0.0) {  // asymmetry data: the given weight
        double r = d - N;
        acc.add(w * r * r);
        W = -2.0 * w * r;
      } else if (mode == 0) {
        double r = d - N;
        acc.add(r * r / std::fmax(d, 1.0));
        W = -2.0 * r / std::fmax(d, 1.0);
      } else if (d > 0.0) {
        if (N <= 0.0) {
          bad = true;
          continue;
        }
        acc.add(2.0 * ((N - d) + d * std::log(d / N)));
        W = 2.0 * (1.0 - d / N);
      } else {
        acc.add(2.0 * (N - d));
        W = 2.0;
      }
      for (int s = 0; s < pb.nslots; ++s) {
        int32_t m = pb.map[static_cast<int64_t>(h) * pb.nslots + s];
        if (m < 0) continue;
        double c = W * dslot[s];
        g[m].add(c);
        gs[m].add(std::fabs(c));
      }
    }
  }
  for (int p = 0; p < pb.P; ++p) {
    if (grad) grad[p] = bad ? 0.0 : g[p].value();
    if (gscale) gscale[p] = gs[p].value();
  }
  if (bad) {
    *value = std::numeric_limits<double>::infinity();
    return 1;
  }
  *value = acc.value();
  return 0;
}

// Gauss-Newton matrix of the cost: sum over bins of (d^2 cost / dN^2) J J^T, with J the
// parameter gradient of N (the second-derivative term of N dropped).  d^2/dN^2 of the bin
// cost is 2 / max(d, 1) for Eq. chisq and 2 d / N^2 for Eq. log-likelihood (0 when d <= 0).
// gn is [P][P]; returns 1 (gn zeros) when the likelihood is undefined.
int gauss_newton(const Problem& pb, const double* x, int mode, double* gn) {
  const int P = pb.P;
  std::vector<Neumaier> acc(static_cast<size_t>(P) * P);
  std::vector<double> dslot(pb.nslots), J(P);
  if (pb.weight && mode != 0) return 2;
  for (int h = 0; h < pb.H; ++h) {
    const double* row = pb.data + static_cast<int64_t>(h) * pb.B;
    for (int64_t n = 0; n < pb.B; ++n) {
      double t = bin_time(pb, h, n);
      if (!in_fit(pb, t)) continue;
      double d = row[n];
      double N = model_and_slot_derivs(pb, x, h, t, dslot.data());
      double c2;
      const double w = bin_weight(pb, h, n);
      if (mode == 0 && w >= 0.0) {
        c2 = 2.0 * w;
      } else if (mode == 0) {
        c2 = 2.0 / std::fmax(d, 1.0);
      } else if (d > 0.0) {
        if (N <= 0.0) {
          std::fill(gn, gn + static_cast<size_t>(P) * P, 0.0);
          return 1;
        }
        c2 = 2.0 * d / (N * N);
      } else {
        c2 = 0.0;
      }
      std::fill(J.begin(), J.end(), 0.0);
      for (int s = 0; s < pb.nslots; ++s) {
        int32_t m = pb.map[static_cast<int64_t>(h) * pb.nslots + s];
        if (m >= 0) J[m] += dslot[s];
      }
      for (int p = 0; p < P; ++p) {
        if (J[p] == 0.0) continue;
        for (int q = p; q < P; ++q) acc[static_cast<size_t>(p) * P + q].add(c2 * J[p] * J[q]);
      }
    }
  }
  for (int p = 0; p < P; ++p)
    for (int q = p; q < P; ++q) gn[static_cast<size_t>(p) * P + q] = gn[static_cast<size_t>(q) * P + p] =
                                    acc[static_cast<size_t>(p) * P + q].value();
  return 0;
}

Problem make_problem(const double* data, int H, int64_t B, const double* t0, double bin_width_ns,
                     double lo, double hi, int nterms, const int32_t* nprim, const int32_t* kind,
                     const int32_t* slot, const int32_t* map, int nslots, const double* consts,
                     int nconsts, int P, const double* weight, int envelope) {
  Problem pb;
  pb.data = data;
  pb.weight = weight;
  pb.envelope = envelope;
  pb.H = H;
  pb.B = B;
  pb.t0 = t0;
  pb.dt_us = bin_width_ns / 1000.0;
  pb.lo = lo;
  pb.hi = hi;
  pb.th.nterms = nterms;
  pb.th.nprim = nprim;
  pb.th.kind = kind;
  pb.th.slot = slot;
  pb.map = map;
  pb.nslots = nslots;
  pb.consts = consts;
  pb.nconsts = nconsts;
  pb.P = P;
  return pb;
}

// The dynamic Kubo-Toyabe grid spans the problem's fit times: up to its last in-fit time.
void set_dkt_span(const Problem& pb) {
  double span = 0.0;
  for (int h = 0; h < pb.H; ++h) {
    const double t_last = bin_time(pb, h, pb.B - 1);
    span = std::fmax(span, std::fmin(t_last, pb.hi));
  }
  g_dkt_span = span > 0.0 ? span : 1.0;
}

double inf_norm(const std::vector<double>& v) {
  double m = 0.0;
  for (double a : v) m = std::fmax(m, std::fabs(a));
  return m;
}

}  // namespace

#define ORACLE_PROBLEM_ARGS                                                                  \
  const double *data, int H, int64_t B, const double *t0, double bin_width_ns, double lo,   \
      double hi, int nterms, const int32_t *nprim, const int32_t *kind, const int32_t *slot, \
      const int32_t *map, int nslots, const double *consts, int nconsts, int P, const double *weight,  \
      int envelope
#define ORACLE_PROBLEM                                                                                  \
  make_problem(data, H, B, t0, bin_width_ns, lo, hi, nterms, nprim, kind, slot, map, nslots, consts, nconsts, P, \
               weight, envelope);                                                                               \
  set_dkt_span(pb)

extern "C" {

// One primitive at time t (Section 4.1, Eq. asymmetry and its generalisation).
double oracle_primitive(int kind, double p0, double p1, double t) {
  if (kind == kDKT) g_dkt_span = t;  // a grid over [0, t]
  return primitive<double>(kind, p0, p1, t);
}

// Eq. positron_histo of histogram h at time t (microseconds).
double oracle_model(ORACLE_PROBLEM_ARGS, const double* x, int h, double t) {
  Problem pb = ORACLE_PROBLEM;
  return model<double>(pb, x, h, t);
}

// The whole cost (Eq. chisq for mode 0, Eq. log-likelihood for mode 1) and,
// when grad != NULL, its analytic gradient.  Returns 0, or 1 when the
// likelihood is +infinity (then *value = +inf and grad is all zeros).
int oracle_cost(ORACLE_PROBLEM_ARGS, const double* x, int mode, double* value, double* grad,
                double* gscale) {
  Problem pb = ORACLE_PROBLEM;
  if (grad == nullptr && gscale == nullptr) return cost_value<double>(pb, x, mode, value);
  return cost_grad(pb, x, mode, value, grad, gscale);
}

// Complex-step derivative of the cost along direction v:
// Im(cost(x + i h v)) / h, the same value code evaluated in complex arithmetic.
int oracle_cost_cstep(ORACLE_PROBLEM_ARGS, const double* x, const double* v, double h, int mode,
                      double* deriv) {
  Problem pb = ORACLE_PROBLEM;
  std::vector<cplx> xc(P);
  for (int p = 0; p < P; ++p) xc[p] = cplx(x[p], h * v[p]);
  cplx out;
  int st = cost_value<cplx>(pb, xc.data(), mode, &out);
  *deriv = out.imag() / h;
  return st;
}

// Hessian by central differences of the analytic gradient, symmetrised.
// step[p] is the difference step of parameter p.  hess is [P][P].
int oracle_hessian(ORACLE_PROBLEM_ARGS, const double* x, const double* step, int mode,
                   double* hess) {
  Problem pb = ORACLE_PROBLEM;
  std::vector<double> xp(x, x + P), gp(P), gm(P);
  double f;
  for (int j = 0; j < P; ++j) {
    xp[j] = x[j] + step[j];
    if (cost_grad(pb, xp.data(), mode, &f, gp.data(), nullptr)) return 1;
    xp[j] = x[j] - step[j];
    if (cost_grad(pb, xp.data(), mode, &f, gm.data(), nullptr)) return 1;
    xp[j] = x[j];
    for (int i = 0; i < P; ++i) hess[i * P + j] = (gp[i] - gm[i]) / (2.0 * step[j]);
  }
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < i; ++j) {
      double a = 0.5 * (hess[i * P + j] + hess[j * P + i]);
      hess[i * P + j] = hess[j * P + i] = a;
    }
  return 0;
}

// Gauss-Newton matrix [P][P] at x (see gauss_newton above).
int oracle_gauss_newton(ORACLE_PROBLEM_ARGS, const double* x, int mode, double* gn) {
  Problem pb = ORACLE_PROBLEM;
  return gauss_newton(pb, x, mode, gn);
}

// BFGS minimisation standing in for Minuit2's migrad (Section 4: the
// minimiser runs on the host and calls the cost once per trial point).
//   * initial inverse Hessian: diag(1/h_ii) from forward differences of the
//     analytic gradient (step fd_step[p]); |h_ii| is used, and 1 when h_ii == 0;
//   * direction p = -Hinv g; if not a descent direction, Hinv is reset;
//   * backtracking line search from alpha = 1, halving, until the Armijo
//     condition f_new <= f + 1e-4 alpha g.p holds with f_new finite;
//   * BFGS inverse update when s.y > 0;
//   * stop when max|g| <= gtol * max(1, |f|), when a step changes no
//     parameter, or after maxit iterations.
// Returns 0 on convergence, 2 when maxit was reached, 3 when the line search
// failed, 1 when the cost was +inf at the start.
int oracle_fit(ORACLE_PROBLEM_ARGS, int mode, const double* x0, const double* fd_step, int maxit,
               double gtol, double* x_out, double* f_out, double* g_out, int* iters_out) {
  Problem pb = ORACLE_PROBLEM;
  std::vector<double> x(x0, x0 + P), g(P), xn(P), gn(P), p(P), s(P), y(P), Hy(P);
  std::vector<double> Hinv(static_cast<size_t>(P) * P, 0.0);
  double f;
  int status = 2;
  int it = 0;
  if (cost_grad(pb, x.data(), mode, &f, g.data(), nullptr)) {
    *f_out = f;
    *iters_out = 0;
    return 1;
  }
  auto reset_hinv = [&]() {
    std::fill(Hinv.begin(), Hinv.end(), 0.0);
    for (int j = 0; j < P; ++j) {
      std::vector<double> xs(x);
      xs[j] += fd_step[j];
      double fs;
      std::vector<double> gsj(P);
      double hjj = 0.0;
      if (cost_grad(pb, xs.data(), mode, &fs, gsj.data(), nullptr) == 0)
        hjj = std::fabs((gsj[j] - g[j]) / fd_step[j]);
      Hinv[static_cast<size_t>(j) * P + j] = hjj > 0.0 ? 1.0 / hjj : 1.0;
    }
  };
  reset_hinv();
  for (it = 0; it < maxit; ++it) {
    if (inf_norm(g) <= gtol * std::fmax(1.0, std::fabs(f))) {
      status = 0;
      break;
    }
    double gp = 0.0;
    for (int i = 0; i < P; ++i) {
      double a = 0.0;
      for (int j = 0; j < P; ++j) a -= Hinv[static_cast<size_t>(i) * P + j] * g[j];
      p[i] = a;
      gp += a * g[i];
    }
    if (!(gp < 0.0)) {
      reset_hinv();
      gp = 0.0;
      for (int i = 0; i < P; ++i) {
        p[i] = -Hinv[static_cast<size_t>(i) * P + i] * g[i];
        gp += p[i] * g[i];
      }
    }
    double alpha = 1.0, fn = 0.0;
    bool ok = false;
    for (int ls = 0; ls < 80; ++ls) {
      for (int i = 0; i < P; ++i) xn[i] = x[i] + alpha * p[i];
      int st = cost_grad(pb, xn.data(), mode, &fn, gn.data(), nullptr);
      if (st == 0 && std::isfinite(fn) && fn <= f + 1e-4 * alpha * gp) {
        ok = true;
        break;
      }
      alpha *= 0.5;
    }
    if (!ok) {
      status = 3;
      break;
    }
    bool moved = false;
    double sy = 0.0;
    for (int i = 0; i < P; ++i) {
      s[i] = xn[i] - x[i];
      y[i] = gn[i] - g[i];
      sy += s[i] * y[i];
      if (xn[i] != x[i]) moved = true;
    }
    x.swap(xn);
    g.swap(gn);
    f = fn;
    if (!moved) {
      status = 0;
      break;
    }
    if (sy > 0.0) {
      // Hinv <- (I - rho s y^T) Hinv (I - rho y s^T) + rho s s^T
      double rho = 1.0 / sy;
      double yHy = 0.0;
      for (int i = 0; i < P; ++i) {
        double a = 0.0;
        for (int j = 0; j < P; ++j) a += Hinv[static_cast<size_t>(i) * P + j] * y[j];
        Hy[i] = a;
        yHy += y[i] * a;
      }
      for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j)
          Hinv[static_cast<size_t>(i) * P + j] +=
              -rho * (Hy[i] * s[j] + s[i] * Hy[j]) + (rho * rho * yHy + rho) * s[i] * s[j];
    }
  }
  std::memcpy(x_out, x.data(), sizeof(double) * P);
  if (g_out) std::memcpy(g_out, g.data(), sizeof(double) * P);
  *f_out = f;
  *iters_out = it;
  return status;
}

// Asymmetry a and chi^2 weight w of npairs forward / backward histogram pairs (see the
// header): F, B, a, w are [npairs][nbins]; alpha, bkg_f, bkg_b are [npairs].
void oracle_asymmetry(const double* F, const double* B, int npairs, int64_t nbins, const double* alpha,
                      const double* bkg_f, const double* bkg_b, double* a, double* w) {
  for (int k = 0; k < npairs; ++k)
    for (int64_t n = 0; n < nbins; ++n) {
      const int64_t i = static_cast<int64_t>(k) * nbins + n;
      const double f = F[i] - bkg_f[k], b = B[i] - bkg_b[k], al = alpha[k];
      const double D = f + al * b;
      if (!(D > 0.0)) {
        a[i] = 0.0;
        w[i] = 0.0;
        continue;
      }
      a[i] = (f - al * b) / D;
      const double var = 4.0 * al * al * (b * b * std::fmax(F[i], 1.0) + f * f * std::fmax(B[i], 1.0)) / (D * D * D * D);
      w[i] = var > 0.0 ? 1.0 / var : 0.0;
    }
}

// ---------------------------------------------------------------------------------------
// The particle-mesh Poisson solve of Section 3 (the second workload): the discretised
// convolution of Eq. openbruteforceconv for an isolated (open-boundary) charge density,
//   phi_{i,j,k} = hx hy hz sum_{i',j',k'} rho_{i',j',k'} G_{i-i',j-j',k-k'},
//   G_{a,b,c} = 1 / sqrt((a hx)^2 + (b hy)^2 + (c hz)^2),
// summed directly (no FFT).  Reading: G_{0,0,0}, where 1/r is singular, is 1 / min(h).
// Arrays are [mx][my][mz], z fastest.
// ---------------------------------------------------------------------------------------
double poisson_green(int a, int b, int c, double hx, double hy, double hz) {
  if (a == 0 && b == 0 && c == 0) return 1.0 / std::fmin(hx, std::fmin(hy, hz));
  const double u = a * hx, v = b * hy, w = c * hz;
  return 1.0 / std::sqrt(u * u + v * v + w * w);
}

double poisson_at(const double* rho, int mx, int my, int mz, double hx, double hy, double hz, int i, int j,
                  int k) {
  Neumaier acc;
  for (int a = 0; a < mx; ++a)
    for (int b = 0; b < my; ++b)
      for (int c = 0; c < mz; ++c) {
        const double q = rho[(static_cast<int64_t>(a) * my + b) * mz + c];
        if (q != 0.0) acc.add(q * poisson_green(std::abs(i - a), std::abs(j - b), std::abs(k - c), hx, hy, hz));
      }
  return hx * hy * hz * acc.value();
}

// phi on the whole mesh.
void oracle_poisson_direct(const double* rho, int mx, int my, int mz, double hx, double hy, double hz,
                           double* phi) {
  for (int i = 0; i < mx; ++i)
    for (int j = 0; j < my; ++j)
      for (int k = 0; k < mz; ++k)
        phi[(static_cast<int64_t>(i) * my + j) * mz + k] = poisson_at(rho, mx, my, mz, hx, hy, hz, i, j, k);
}

// phi at npts mesh points ijk[npts][3] only (for samples of large meshes).
void oracle_poisson_points(const double* rho, int mx, int my, int mz, double hx, double hy, double hz,
                           const int32_t* ijk, int npts, double* out) {
  for (int p = 0; p < npts; ++p)
    out[p] = poisson_at(rho, mx, my, mz, hx, hy, hz, ijk[3 * p], ijk[3 * p + 1], ijk[3 * p + 2]);
}

// The dynamic Kubo-Toyabe relaxation of (Delta, nu) on the grid over [0, span], at the n
// times ts: G[n], and its derivatives dD[n] (Delta), dnu[n] (nu) when those are not NULL.
// Returns the number of coarse grid intervals used.
int oracle_dkt(double D, double nu, double span, const double* ts, int n, double* G, double* dD, double* dnu) {
  g_dkt_span = span;
  for (int i = 0; i < n; ++i) {
    G[i] = dkt_value<double>(D, nu, ts[i]);
    if (dD || dnu) {
      double a, b;
      dkt_derivs(D, nu, ts[i], &a, &b);
      if (dD) dD[i] = a;
      if (dnu) dnu[i] = b;
    }
  }
  return dkt_points(D, nu, span);
}

// Neumaier-compensated sum of n doubles, exposed so that the summation itself
// can be pinned against an exactly rounded sum.
double oracle_neumaier_sum(const double* v, int64_t n) {
  Neumaier a;
  for (int64_t i = 0; i < n; ++i) a.add(v[i]);
  return a.value();
}

}  // extern "C"
