// musr_bfgs.h -- the host minimiser as a state machine (the role migrad plays in
// Section 4: the minimiser runs on the host, each trial point costs one device
// evaluation).  A state machine rather than a loop, so that the serving loop can
// advance many fits by one step each per launch.
//
// Algorithm (the same as paper_1509_07685_gb300/fit.py):
//   * H0 = diag(1/|h_ii|), h_ii forward differences of the analytic gradient along
//     each axis (steps max(1e-5 |x_i|, 1e-4); the P points are one batched request);
//   * p = -H g, reset to the diagonal when p is not a descent direction;
//   * backtracking from alpha = 1 (halving, at most 60 trials) until
//     f_new <= f + 1e-4 alpha g.p, or -- for a cost with rounding noise f_noise --
//     the predicted gain is below the noise, f_new within f_noise of that bound and
//     |g_new| < |g|;
//   * BFGS inverse update when s.y > 0;
//   * stop when max|g| <= gtol max(1, |f|), when EDM = -g.p/2 < edm_tol after at
//     least two updates, when a step leaves x unchanged, or after maxit iterations.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace musr {

class Bfgs {
 public:
  enum Status { kConverged = 0, kNonFinite = 1, kMaxIter = 2, kLineSearch = 3, kRunning = -1 };

  Bfgs() = default;
  void start(const double* x0, int P, double gtol, int maxit, double f_noise, double edm_tol) {
    P_ = P;
    x_.assign(x0, x0 + P);
    g_.assign(P, 0.0);
    H_.assign(static_cast<size_t>(P) * P, 0.0);
    p_.assign(P, 0.0);
    xn_.assign(P, 0.0);
    steps_.resize(P);
    for (int i = 0; i < P; ++i) steps_[i] = std::max(1e-5 * std::fabs(x0[i]), 1e-4);
    gtol_ = gtol;
    maxit_ = maxit;
    f_noise_ = f_noise;
    edm_tol_ = edm_tol;
    it_ = 0;
    updates_ = 0;
    nfev_ = 0;
    status_ = kRunning;
    phase_ = kStart;
  }

  bool done() const { return status_ != kRunning; }
  int status() const { return status_; }
  int iters() const { return it_; }
  int nfev() const { return nfev_; }
  double f() const { return f_; }
  double edm() const { return edm_; }
  const std::vector<double>& x() const { return x_; }
  void set_f_noise(double v) { f_noise_ = v; }

  // Points to evaluate next, row-major [n][P]; returns n (0 when done).
  int request(std::vector<double>* pts) {
    pts->clear();
    if (done()) return 0;
    switch (phase_) {
      case kStart:
        pts->assign(x_.begin(), x_.end());
        return 1;
      case kDiag:
        pts->resize(static_cast<size_t>(P_) * P_);
        for (int j = 0; j < P_; ++j) {
          std::copy(x_.begin(), x_.end(), pts->begin() + static_cast<size_t>(j) * P_);
          (*pts)[static_cast<size_t>(j) * P_ + j] += steps_[j];
        }
        return P_;
      case kTrial:
        for (int i = 0; i < P_; ++i) xn_[i] = x_[i] + alpha_ * p_[i];
        pts->assign(xn_.begin(), xn_.end());
        return 1;
    }
    return 0;
  }

  // Values f[n] and gradients g[n][P] of the points of the last request.
  void deliver(const double* f, const double* g) {
    if (done()) return;
    switch (phase_) {
      case kStart:
        nfev_ += 1;
        f_ = f[0];
        if (!std::isfinite(f_)) {
          status_ = kNonFinite;
          return;
        }
        std::memcpy(g_.data(), g, sizeof(double) * P_);
        phase_ = kDiag;
        return;
      case kDiag:
        nfev_ += P_;
        std::fill(H_.begin(), H_.end(), 0.0);
        for (int j = 0; j < P_; ++j) {
          const double h = std::fabs((g[static_cast<size_t>(j) * P_ + j] - g_[j]) / steps_[j]);
          H_[static_cast<size_t>(j) * P_ + j] = h > 0.0 ? 1.0 / h : 1.0;
        }
        updates_ = 0;
        next_direction(true);
        return;
      case kTrial: {
        nfev_ += 1;
        const double fn = f[0];
        bool ok = false;
        if (std::isfinite(fn)) {
          const double armijo = f_ + 1e-4 * alpha_ * gp_;
          const bool small = -alpha_ * gp_ < 10.0 * f_noise_;
          ok = fn <= armijo || (small && fn <= armijo + f_noise_ && norm(g) < gnorm_);
        }
        if (ok) {
          accept(fn, g);
          return;
        }
        if (-alpha_ * gp_ < 0.01 * f_noise_ || ++ls_ >= 60) {
          status_ = (f_noise_ > 0.0 && edm_ < 100.0 * edm_tol_) ? kConverged : kLineSearch;
          return;
        }
        alpha_ *= 0.5;
        return;
      }
    }
  }

 private:
  enum Phase { kStart, kDiag, kTrial };

  double norm(const double* v) const {
    double s = 0.0;
    for (int i = 0; i < P_; ++i) s += v[i] * v[i];
    return std::sqrt(s);
  }

  // Convergence checks at the current point, then the next search direction.
  void next_direction(bool after_reset) {
    double gmax = 0.0;
    for (int i = 0; i < P_; ++i) gmax = std::max(gmax, std::fabs(g_[i]));
    if (gmax <= gtol_ * std::max(1.0, std::fabs(f_))) {
      status_ = kConverged;
      return;
    }
    gp_ = 0.0;
    for (int i = 0; i < P_; ++i) {
      double a = 0.0;
      const double* row = H_.data() + static_cast<size_t>(i) * P_;
      for (int j = 0; j < P_; ++j) a -= row[j] * g_[j];
      p_[i] = a;
      gp_ += a * g_[i];
    }
    if (!(gp_ < 0.0)) {
      if (after_reset) {  // a diagonal with positive entries always gives descent; guard anyway
        status_ = kLineSearch;
        return;
      }
      phase_ = kDiag;  // reset to the diagonal estimate at this point
      return;
    }
    edm_ = -0.5 * gp_;
    if (updates_ >= 2 && edm_ < edm_tol_) {
      status_ = kConverged;
      return;
    }
    alpha_ = 1.0;
    ls_ = 0;
    gnorm_ = norm(g_.data());
    phase_ = kTrial;
  }

  void accept(double fn, const double* gn) {
    std::vector<double> s(P_), y(P_), Hy(P_);
    bool moved = false;
    double sy = 0.0;
    for (int i = 0; i < P_; ++i) {
      s[i] = xn_[i] - x_[i];
      y[i] = gn[i] - g_[i];
      sy += s[i] * y[i];
      if (xn_[i] != x_[i]) moved = true;
    }
    x_ = xn_;
    std::memcpy(g_.data(), gn, sizeof(double) * P_);
    f_ = fn;
    ++it_;
    if (!moved) {
      status_ = kConverged;
      return;
    }
    if (sy > 0.0) {
      ++updates_;
      const double rho = 1.0 / sy;
      double yHy = 0.0;
      for (int i = 0; i < P_; ++i) {
        double a = 0.0;
        const double* row = H_.data() + static_cast<size_t>(i) * P_;
        for (int j = 0; j < P_; ++j) a += row[j] * y[j];
        Hy[i] = a;
        yHy += y[i] * a;
      }
      for (int i = 0; i < P_; ++i) {
        double* row = H_.data() + static_cast<size_t>(i) * P_;
        for (int j = 0; j < P_; ++j)
          row[j] += -rho * (Hy[i] * s[j] + s[i] * Hy[j]) + (rho * rho * yHy + rho) * s[i] * s[j];
      }
    }
    if (it_ >= maxit_) {
      status_ = kMaxIter;
      return;
    }
    next_direction(false);
  }

  int P_ = 0;
  std::vector<double> x_, g_, H_, p_, xn_, steps_;
  double f_ = 0.0, gp_ = 0.0, alpha_ = 1.0, gnorm_ = 0.0, edm_ = 0.0;
  double gtol_ = 1e-8, f_noise_ = 0.0, edm_tol_ = 1e-7;
  int maxit_ = 1000, it_ = 0, updates_ = 0, nfev_ = 0, ls_ = 0;
  int status_ = kRunning;
  Phase phase_ = kStart;
};

}  // namespace musr
