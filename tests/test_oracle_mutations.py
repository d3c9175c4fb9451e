"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/musr_oracle.cpp (a dropped term, a
wrong sign or index, a transposed operand, a wrong constant), builds it into a
temporary library on the CPU, and runs the pin tests against it: every mutant must
fail at least one pin.  Nothing here touches the GPU or the CUDA library.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "musr_oracle.cpp")

MUTANTS = {
    "gauss drops the 1/2": ("return std::exp(-0.5 * (p0 * t) * (p0 * t));", "return std::exp(-(p0 * t) * (p0 * t));"),
    "phase sign": ("return std::cos(2.0 * kPi * (p0 * t + p1 / 360.0));",
                   "return std::cos(2.0 * kPi * (p0 * t - p1 / 360.0));"),
    "phase in radians": ("return std::cos(2.0 * kPi * (p0 * t + p1 / 360.0));",
                         "return std::cos(2.0 * kPi * p0 * t + p1);"),
    "muon lifetime": ("constexpr double kTauMu = 2.197019;", "constexpr double kTauMu = 2.19703;"),
    "log argument transposed": ("return 2.0 * ((N - d) + d * std::log(d / N));",
                                "return 2.0 * ((N - d) + d * std::log(N / d));"),
    "background dropped": ("return N0 * std::exp(-t / kTauMu) * (1.0 + A) + Nbkg;",
                           "return N0 * std::exp(-t / kTauMu) * (1.0 + A);"),
    "t0 sign": ("return (static_cast<double>(n) - pb.t0[h]) * pb.dt_us;",
                "return (static_cast<double>(n) + pb.t0[h]) * pb.dt_us;"),
    "fit range open": ("return pb.lo <= t && t <= pb.hi;", "return pb.lo < t && t < pb.hi;"),
    "chi2 variance off by one": ("return r * r / std::fmax(d, 1.0);", "return r * r / std::fmax(d + 1.0, 1.0);"),
    "KT derivative misses a t": ("*d0 = (2.0 / 3.0) * p0 * t * t * std::exp(-0.5 * u) * (u - 3.0);",
                                 "*d0 = (2.0 / 3.0) * p0 * t * std::exp(-0.5 * u) * (u - 3.0);"),
    "cosine derivative sign": ("*d0 = -s * 2.0 * kPi * t;", "*d0 = s * 2.0 * kPi * t;"),
    "phase derivative scale": ("*d1 = -s * 2.0 * kPi / 360.0;", "*d1 = -s * 2.0 * kPi;"),
    "KT sign": ("return 1.0 / 3.0 + (2.0 / 3.0) * (1.0 - u) * std::exp(-0.5 * u);",
                "return 1.0 / 3.0 + (2.0 / 3.0) * (1.0 + u) * std::exp(-0.5 * u);"),
    "no compensation": ("      c += (s - t) + x;\n    else\n      c += (x - t) + s;",
                        "      c += 0.0;\n    else\n      c += 0.0;"),
    "map scatter to the wrong index": ("        g[m].add(c);", "        g[(m + 1) % pb.P].add(c);"),
    "N0 derivative drops the asymmetry": ("  dslot[0] += E * (1.0 + A);", "  dslot[0] += E;"),
    "Lorentzian KT sign": ("return 1.0 / 3.0 + (2.0 / 3.0) * (1.0 - u) * std::exp(-u);",
                           "return 1.0 / 3.0 + (2.0 / 3.0) * (1.0 + u) * std::exp(-u);"),
    "Lorentzian KT derivative": ("*d0 = (2.0 / 3.0) * t * std::exp(-u) * (u - 2.0);",
                                 "*d0 = (2.0 / 3.0) * t * std::exp(-u) * (u - 3.0);"),
    "Gauss-Newton weight of -2lnL": ("        c2 = 2.0 * d / (N * N);", "        c2 = 2.0 / N;"),
    "Bessel argument misses 2 pi": ("return bessel_j0(2.0 * kPi * (p0 * t + p1 / 360.0));",
                                    "return bessel_j0(p0 * t + p1 / 360.0);"),
    "Bessel derivative sign": ("      *d0 = -j1 * 2.0 * kPi * t;", "      *d0 = j1 * 2.0 * kPi * t;"),
    "stretched exponent derivative drops the log": ("*d1 = -xb * std::log(x) * f;", "*d1 = -xb * f;"),
    "stretched rate derivative drops beta": ("(-p1 * xb / lam) * f;", "(-xb / lam) * f;"),
    "Poisson spacings transposed": ("const double u = a * hx, v = b * hy, w = c * hz;",
                                    "const double u = a * hy, v = b * hx, w = c * hz;"),
    "Poisson volume factor dropped": ("return hx * hy * hz * acc.value();", "return acc.value();"),
    "Poisson self term": ("return 1.0 / std::fmin(hx, std::fmin(hy, hz));", "return 0.0;"),
    "Poisson source offset": ("std::abs(i - a), std::abs(j - b), std::abs(k - c)",
                              "std::abs(i - a), std::abs(j - b), std::abs(k - c + 1)"),
    "asymmetry variance drops the 4": ("const double var = 4.0 * al * al *", "const double var = al * al *"),
    "asymmetry alpha on the forward count": ("a[i] = (f - al * b) / D;", "a[i] = (al * f - b) / D;"),
    "asymmetry variances exchanged": ("(b * b * std::fmax(F[i], 1.0) + f * f * std::fmax(B[i], 1.0))",
                                      "(b * b * std::fmax(B[i], 1.0) + f * f * std::fmax(F[i], 1.0))"),
    "asymmetry model keeps the envelope": ("  if (!pb.envelope) return N0 * A + Nbkg;\n", ""),
    "asymmetry slot derivatives keep the envelope": ("const double E = pb.envelope ? std::exp(-t / kTauMu) : 1.0;",
                                                     "const double E = std::exp(-t / kTauMu);"),
    "asymmetry weight missing from the gradient": ("        W = -2.0 * w * r;", "        W = -2.0 * r;"),
    "asymmetry scale derivative": ("    dslot[0] += A;", "    dslot[0] += 1.0 + A;"),
    "Gauss-Newton weight of chi^2": ("        c2 = 2.0 / std::fmax(d, 1.0);", "        c2 = 1.0 / std::fmax(d, 1.0);"),
    "-2lnL gradient weight inverted": ("        W = 2.0 * (1.0 - d / N);", "        W = 2.0 * (1.0 - N / d);"),
    "chi^2 gradient weight sign": ("        W = -2.0 * r / std::fmax(d, 1.0);", "        W = 2.0 * r / std::fmax(d, 1.0);"),
    "exponential derivative sign": ("      *d0 = -t * std::exp(-p0 * t);", "      *d0 = t * std::exp(-p0 * t);"),
    "Gaussian derivative drops sigma": ("      *d0 = -p0 * t * t * std::exp(-0.5 * (p0 * t) * (p0 * t));",
                                        "      *d0 = -t * t * std::exp(-0.5 * (p0 * t) * (p0 * t));"),
    "-2lnL empty bin halved": ("        acc.add(2.0 * (N - d));", "        acc.add(N - d);"),
    "-2lnL empty-bin gradient halved": ("        W = 2.0;", "        W = 1.0;"),
    "stretched exponential is 0 before time zero": ("if (!(t > 0.0) || re(x) == 0.0) return T(1.0);",
                                                    "if (!(t > 0.0) || re(x) == 0.0) return T(0.0);"),
    "asymmetry Gauss-Newton weight": ("        c2 = 2.0 * w;", "        c2 = 2.0;"),
    "Gauss-Newton Jacobian overwrites a parameter read by two slots": (
        "        if (m >= 0) J[m] += dslot[s];", "        if (m >= 0) J[m] = dslot[s];"),
    "product rule drops the other factors": ("      dslot[sl[0]] += N0 * E * d0 * rest;",
                                             "      dslot[sl[0]] += N0 * E * d0;"),
    "second slot's derivative to the first slot": (
        "      if (nslots_of(kind) == 2) dslot[sl[1]] += N0 * E * d1 * rest;",
        "      if (nslots_of(kind) == 2) dslot[sl[0]] += N0 * E * d1 * rest;"),
    "background derivative carries the decay": ("  dslot[0] += E * (1.0 + A);\n  dslot[1] += 1.0;",
                                                 "  dslot[0] += E * (1.0 + A);\n  dslot[1] += E;"),
    "product rule keeps the differentiated factor": ("        if (q != m) rest *= f[q];", "        rest *= f[q];"),
    "dynamic KT drops the trapezoid's end weights": (
        "const T a = 1.0 - nu * (0.5 * h), b = 1.0 + nu * (0.5 * h), c = nu * h;",
        "const T a = 1.0, b = 1.0, c = nu * h;"),
    "dynamic KT without Richardson extrapolation": ("tab->G[k] = (4.0 * Gh2[2 * k] - Gh[k]) / 3.0;", "tab->G[k] = Gh[k];"),
    "dynamic KT kernel misses the renewal decay": ("f[k] = dkt_static(D, k * h) * std::exp(-nu * (k * h));",
                                                  "f[k] = dkt_static(D, k * h);"),
    "dynamic KT convolution lags one point": ("sk = sk + f[j] * (*G)[k - j];", "sk = sk + f[j] * (*G)[k - j - 1];"),
    "dynamic KT nu-derivative drops the convolution": ("+ h * S[k] + cr * sn) / ar;", "+ cr * sn) / ar;"),
    "dynamic KT Delta-derivative misses a t": (
        "return (2.0 / 3.0) * D * t * t * std::exp(-0.5 * u) * (u - 3.0);",
        "return (2.0 / 3.0) * D * t * std::exp(-0.5 * u) * (u - 3.0);"),
    "dynamic KT interpolation weights exchanged": (
        "return w0 * y[i] + w1 * y[i + 1] + w2 * y[i + 2] + w3 * y[i + 3];",
        "return w0 * y[i] + w2 * y[i + 1] + w1 * y[i + 2] + w3 * y[i + 3];"),
}


SCRATCH = os.path.join(ROOT, "tests", "_mutants")  # git-ignored


def _run_mutant(name):
    """Builds the mutant and runs the pins against it; returns (caught, pytest output tail)."""
    old, new = MUTANTS[name]
    src = open(SRC).read()
    if src.count(old) < 1:
        return None, f"mutation site not found: {name}"
    mutated = src.replace(old, new, 1)
    tag = "".join(c if c.isalnum() else "_" for c in name)
    cpp = os.path.join(SCRATCH, tag + ".cpp")
    lib = os.path.join(SCRATCH, tag + ".so")
    with open(cpp, "w") as f:
        f.write(mutated)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                           "-o", str(lib), str(cpp)])
    env = dict(os.environ, MUSR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode != 0, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes():
    """Every mutant built and pinned once, several at a time (each in its own processes)."""
    from concurrent.futures import ThreadPoolExecutor
    os.makedirs(SCRATCH, exist_ok=True)
    names = sorted(MUTANTS)
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(zip(names, ex.map(_run_mutant, names)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, outcomes):
    caught, tail = outcomes[name]
    assert caught is not None, tail
    assert caught, f"no pin caught the mutant '{name}':\n{tail}"
