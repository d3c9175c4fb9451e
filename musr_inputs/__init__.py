"""Seeded synthetic muSR inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the fitted method: it neither evaluates the
positron-histogram model nor any cost.  Histograms come from an event-level
Monte Carlo of a muSR run (Section 4.1 describes the experiment):

  * each muon decays at t ~ Exponential(tau_mu);
  * it belongs to one signal component k with probability amp_k / sum(amp);
  * its spin precesses in its own local field: transverse-field (TF)
    components draw a frequency omega = 2 pi nu + sigma z (z ~ N(0, 1)), so the
    ensemble dephases; zero-field (ZF) components draw a 3-D static field
    b ~ N(0, Delta^2 I) and the spin component along the initial polarisation
    follows (b_z^2 + (b_x^2 + b_y^2) cos(|b| t)) / |b|^2;
  * dynamic zero-field (DZF) components draw such a field anew at the events of a
    Poisson process of rate nu (strong collisions); between events the spin vector
    precesses about the current field (a rotation by |b| times the interval);
  * a component with rate lambda loses its polarisation at an
    Exponential(1/lambda) time;
  * the positron is counted by detector j with probability
    (1 + a s) / (1 + a), a = sum(amp), s the spin projection on the detector axis
    (phase phi_j for TF);
  * a flat Poisson background Nbkg per bin is added.

The relaxation functions (exponential, Gaussian, Kubo-Toyabe) are therefore
never written down here: they emerge from the field distributions, which is
what makes fits of these histograms an independent check of the model.  An
event at time t lands in bin floor(t / dt + t0 + 1/2), so the expected count
of bin n is the model at the bin's left-edge time t_n = (n - t0) dt to second
order in dt.

All generators are seeded (numpy PCG64).  Problem descriptions (term lists and
parameter maps) are plain data consumed by both the oracle and the GPU binding.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

TAU_MU_US = 2.197019  # muon lifetime in microseconds (the paper gives no value; this one is used throughout)

# --------------------------------------------------------------------------------------------
# Problem description (plain data)
# --------------------------------------------------------------------------------------------

Term = Sequence[Tuple[str, Tuple[int, ...]]]


@dataclasses.dataclass
class Problem:
    """One fit: histograms, time grid, theory term list and parameter map.

    ``terms``: list of terms, each a list of (kind, slots), kind one of AMP,
    EXP, GAUSS, KT, TFCOS.  Local slot 0 is N0 and slot 1 is Nbkg.
    ``map``: int32 [H][nslots]; entry >= 0 is a global parameter index, entry
    < 0 selects ``consts[-1 - entry]``.
    """

    counts: np.ndarray  # [H][B]
    t0: np.ndarray  # [H] in bins
    bin_width_ns: float
    fit_range_us: Tuple[float, float]
    terms: List[Term]
    map: np.ndarray
    consts: np.ndarray
    nparams: int
    truth: np.ndarray
    names: List[str]
    name: str = ""

    @property
    def H(self) -> int:
        return int(self.counts.shape[0])

    @property
    def B(self) -> int:
        return int(self.counts.shape[1])

    @property
    def nslots(self) -> int:
        return int(self.map.shape[1])

    def with_counts(self, counts) -> "Problem":
        return dataclasses.replace(self, counts=counts)


@dataclasses.dataclass
class Component:
    """One physical signal component of the simulated run."""

    amp: float
    # "TF", "ZF" (static Gaussian fields), "ZFL" (static Lorentzian fields), "DZF" (Gaussian
    # fields drawn anew at the events of a Poisson process of rate nu_c), "INC" (fields of an
    # incommensurate structure, gamma B = 2 pi nu cos(U), U uniform) or "LF" (no precession)
    kind: str = "TF"
    nu_mhz: float = 0.0
    sigma: float = 0.0  # TF field-width (Gaussian dephasing rate), 1/us
    lam: float = 0.0  # depolarisation rate, 1/us
    delta: float = 0.0  # ZF / ZFL static field width, 1/us
    levy: float = 0.0  # depolarisation at a rate r = levy / (2 Z^2), Z ~ N(0, 1) per muon, 1/us
    nu_c: float = 0.0  # DZF: rate of the field's renewals, 1/us


@dataclasses.dataclass
class Detector:
    n0: float  # counts per bin at t = 0 without asymmetry
    nbkg: float  # background counts per bin
    phase_deg: float
    t0: float = 0.0


# --------------------------------------------------------------------------------------------
# Event-level Monte Carlo
# --------------------------------------------------------------------------------------------

def simulate_histogram(rng: np.random.Generator, det: Detector, comps: Sequence[Component],
                       nbins: int, bin_width_ns: float, chunk: int = 1 << 22) -> np.ndarray:
    """Counts of one detector, int64 [nbins]."""
    dt_us = bin_width_ns / 1000.0
    a_tot = float(sum(c.amp for c in comps))
    if a_tot < 0:
        raise ValueError("component amplitudes must be non-negative")
    probs = np.array([c.amp for c in comps], dtype=np.float64)
    probs = probs / probs.sum() if a_tot > 0 else np.full(len(comps), 1.0 / max(len(comps), 1))
    n_muons = rng.poisson(det.n0 * (TAU_MU_US / dt_us) * (1.0 + a_tot))
    counts = np.zeros(nbins, dtype=np.int64)
    phase = math.radians(det.phase_deg)
    done = 0
    while done < n_muons:
        m = min(chunk, n_muons - done)
        done += m
        t = rng.exponential(TAU_MU_US, m)
        which = rng.choice(len(comps), size=m, p=probs) if len(comps) > 1 else np.zeros(m, np.int64)
        s = np.zeros(m)
        for k, c in enumerate(comps):
            sel = np.nonzero(which == k)[0]
            if sel.size == 0:
                continue
            tk = t[sel]
            if c.kind == "TF":
                omega = 2.0 * math.pi * c.nu_mhz + c.sigma * rng.standard_normal(sel.size)
                sk = np.cos(omega * tk + phase)
            elif c.kind == "INC":
                omega = 2.0 * math.pi * c.nu_mhz * np.cos(rng.uniform(0.0, 2.0 * math.pi, sel.size))
                sk = np.cos(omega * tk + phase)
            elif c.kind == "LF":
                sk = np.ones(sel.size)
            elif c.kind in ("ZF", "ZFL"):
                # fields in units of gamma_mu: Gaussian, or the 3-D Lorentzian of dilute moments
                # (a multivariate Cauchy: a Gaussian vector divided by |N(0, 1)|)
                b = c.delta * rng.standard_normal((sel.size, 3))
                if c.kind == "ZFL":
                    b /= np.abs(rng.standard_normal((sel.size, 1)))
                b2 = np.einsum("ij,ij->i", b, b)
                bt2 = b[:, 0] ** 2 + b[:, 1] ** 2
                sk = (b[:, 2] ** 2 + bt2 * np.cos(np.sqrt(b2) * tk)) / np.maximum(b2, 1e-300)
            elif c.kind == "DZF":
                sk = _dynamic_spin_z(rng, tk, c.delta, c.nu_c)
            else:
                raise ValueError(c.kind)
            if c.lam > 0:
                alive = rng.exponential(1.0 / c.lam, sel.size) > tk
                sk = np.where(alive, sk, 0.0)
            if c.levy > 0:  # a one-sided Levy distribution of rates
                z = rng.standard_normal(sel.size)
                rate = c.levy / (2.0 * np.maximum(z * z, 1e-300))
                alive = rng.exponential(1.0, sel.size) > rate * tk
                sk = np.where(alive, sk, 0.0)
            s[sel] = sk
        keep = rng.random(m) * (1.0 + a_tot) < 1.0 + a_tot * s
        n = np.floor(t[keep] / dt_us + det.t0 + 0.5).astype(np.int64)
        n = n[(n >= 0) & (n < nbins)]
        counts += np.bincount(n, minlength=nbins)[:nbins]
    if det.nbkg > 0:
        counts += rng.poisson(det.nbkg, nbins)
    return counts


def _dynamic_spin_z(rng: np.random.Generator, t: np.ndarray, delta: float, nu_c: float) -> np.ndarray:
    """Spin component along the initial polarisation (z) at times t of muons whose local
    field, drawn from N(0, delta^2 I) (in units of gamma_mu), is drawn anew at the events of
    a Poisson process of rate nu_c: the spin vector is rotated about each interval's field by
    |b| times the interval's length (Rodrigues' formula)."""
    m = t.size
    S = np.zeros((m, 3))
    S[:, 2] = 1.0
    left = t.astype(np.float64).copy()
    active = np.nonzero(left > 0.0)[0]
    while active.size:
        seg = left[active]
        if nu_c > 0.0:
            seg = np.minimum(seg, rng.exponential(1.0 / nu_c, active.size))
        b = delta * rng.standard_normal((active.size, 3))
        bn = np.sqrt(np.einsum("ij,ij->i", b, b))
        k = b / np.maximum(bn, 1e-300)[:, None]
        th = bn * seg
        c, s_ = np.cos(th)[:, None], np.sin(th)[:, None]
        v = S[active]
        kv = np.einsum("ij,ij->i", k, v)[:, None]
        S[active] = v * c + np.cross(k, v) * s_ + k * kv * (1.0 - c)
        left[active] -= seg
        active = active[left[active] > 0.0]
    return S[:, 2]


def simulate(seed: int, dets: Sequence[Detector], comps_per_det: Sequence[Sequence[Component]],
             nbins: int, bin_width_ns: float, dtype=np.float32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = np.empty((len(dets), nbins), dtype=dtype)
    for j, (d, comps) in enumerate(zip(dets, comps_per_det)):
        out[j] = simulate_histogram(rng, d, comps, nbins, bin_width_ns)
    return out


def jitter(truth: np.ndarray, n: int, seed: int, lo: float = 0.8, hi: float = 1.2) -> np.ndarray:
    """n parameter vectors truth * U(lo, hi), componentwise (seeded)."""
    rng = np.random.default_rng(seed)
    return truth[None, :] * rng.uniform(lo, hi, size=(n, truth.size))


def start_point(p: "Problem", seed: int, rel: float = 0.02, nu_rel: float = 0.002,
                phase_deg: float = 5.0) -> np.ndarray:
    """A fit start near the truth, as a muSR analyst would give it: every parameter within
    +-rel (relative), frequencies within +-nu_rel (a frequency read off an FFT of the run)
    and phases within +-phase_deg degrees."""
    rng = np.random.default_rng(seed)
    x = p.truth.astype(np.float64).copy()
    for i, n in enumerate(p.names):
        if n.startswith("nu"):
            x[i] *= 1.0 + rng.uniform(-nu_rel, nu_rel)
        elif n.startswith("phi"):
            x[i] += rng.uniform(-phase_deg, phase_deg)
        else:
            x[i] *= 1.0 + rng.uniform(-rel, rel)
    return x


# --------------------------------------------------------------------------------------------
# The configurations (sizes and truths of the paper-shaped workloads)
# --------------------------------------------------------------------------------------------

def _full_range(nbins: int, bin_width_ns: float) -> Tuple[float, float]:
    """Every bin after the first: the bin at t = 0 only collects events from half its width."""
    dt_us = bin_width_ns / 1000.0
    return (0.5 * dt_us, nbins * dt_us)


def _jittered(truth, jitter_seed):
    truth = np.array(truth, dtype=np.float64)
    if jitter_seed is not None:
        truth = truth * np.random.default_rng(jitter_seed).uniform(0.8, 1.2, truth.size)
    return truth


def cfg1(nbins: int = 16384, bin_width_ns: float = 0.5, seed: int = 0, dtype=np.int32,
         n0: float = 300.0, jitter_seed: Optional[int] = None) -> Problem:
    """Single histogram, A = A0 exp(-lambda t) cos(2 pi nu t + phi); 6 parameters."""
    names = ["N0", "Nbkg", "A0", "lambda", "nu", "phi"]
    truth = _jittered([n0, 2.0, 0.25, 0.5, 5.0, 10.0], jitter_seed)
    terms = [[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))]]
    mp = np.array([[0, 1, 2, 3, 4, 5]], np.int32)
    det = Detector(truth[0], truth[1], truth[5])
    comp = Component(truth[2], "TF", nu_mhz=truth[4], lam=truth[3])
    counts = simulate(seed, [det], [[comp]], nbins, bin_width_ns, dtype)
    return Problem(counts, np.zeros(1), bin_width_ns, _full_range(nbins, bin_width_ns), terms, mp,
                   np.zeros(0), 6, truth, names, "cfg1")


def _tf2_map(H: int, first: int, shared: dict, with_kt: bool):
    """Map rows for the two-term TF model (+ optional KT term)."""
    rows = []
    # consts: -1 -> A1 = 0.125, -2 -> A2 = 0.125, -3 -> A3 = 0.05
    for j in range(H):
        base = first + 3 * j
        row = [base + 0, base + 1, -1, shared["lambda"], shared["nu1"], base + 2, -2,
               shared["sigma"], shared["nu2"]]
        if with_kt:
            row += [-3, shared["delta"]]
        rows.append(row)
    return np.array(rows, np.int32)


def cfg2(nhist: int = 8, nbins: int = 65536, bin_width_ns: float = 0.1953125, seed: int = 2,
         dtype=np.float32, n0: float = 300.0, jitter_seed: Optional[int] = None) -> Problem:
    """Global two-term TF fit: shared lambda, sigma, nu1, nu2; per-histogram N0, Nbkg, phase.

    A_j = A1 e^{-lambda t} cos(2 pi (nu1 t + phi_j/360)) + A2 e^{-(sigma t)^2/2} cos(2 pi (nu2 t + phi_j/360)),
    A1 = A2 = 0.125 fixed; 4 + 3 H parameters (28 for H = 8).
    """
    terms = [[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))],
             [("AMP", (6,)), ("GAUSS", (7,)), ("TFCOS", (8, 5))]]
    shared = {"lambda": 0, "sigma": 1, "nu1": 2, "nu2": 3}
    mp = _tf2_map(nhist, 4, shared, False)
    names = ["lambda", "sigma", "nu1", "nu2"]
    truth = [0.5, 0.3, 5.0, 5.5]
    for j in range(nhist):
        ph = (45.0 * j) % 360.0 if nhist <= 8 else 360.0 * j / nhist
        names += [f"N0_{j}", f"Nbkg_{j}", f"phi_{j}"]
        truth += [n0, 2.0, ph]
    truth = _jittered(truth, jitter_seed)
    dets, comps = [], []
    for j in range(nhist):
        b = 4 + 3 * j
        dets.append(Detector(truth[b], truth[b + 1], truth[b + 2]))
        comps.append([Component(0.125, "TF", nu_mhz=truth[2], lam=truth[0]),
                      Component(0.125, "TF", nu_mhz=truth[3], sigma=truth[1])])
    counts = simulate(seed, dets, comps, nbins, bin_width_ns, dtype)
    return Problem(counts, np.zeros(nhist), bin_width_ns, _full_range(nbins, bin_width_ns), terms,
                   mp, np.array([0.125, 0.125]), len(truth), truth, names, "cfg2")


def cfg3(nhist: int = 4, nbins: int = 32768, bin_width_ns: float = 0.390625, seed: int = 3,
         dtype=np.float32, n0: float = 300.0, jitter_seed: Optional[int] = None) -> Problem:
    """Zero-field static Gaussian Kubo-Toyabe times an exponential: A = A0 KT(Delta, t) e^{-lambda t}.

    Shared A0, Delta, lambda; per-histogram N0, Nbkg: 3 + 2 H parameters (11 for H = 4).
    """
    terms = [[("AMP", (2,)), ("KT", (3,)), ("EXP", (4,))]]
    rows = [[3 + 2 * j, 4 + 2 * j, 0, 1, 2] for j in range(nhist)]
    names = ["A0", "Delta", "lambda"]
    truth = [0.25, 0.3, 0.1]
    for j in range(nhist):
        names += [f"N0_{j}", f"Nbkg_{j}"]
        truth += [n0, 2.0]
    truth = _jittered(truth, jitter_seed)
    dets, comps = [], []
    for j in range(nhist):
        dets.append(Detector(truth[3 + 2 * j], truth[4 + 2 * j], 0.0))
        comps.append([Component(truth[0], "ZF", delta=truth[1], lam=truth[2])])
    counts = simulate(seed, dets, comps, nbins, bin_width_ns, dtype)
    return Problem(counts, np.zeros(nhist), bin_width_ns, _full_range(nbins, bin_width_ns), terms,
                   np.array(rows, np.int32), np.zeros(0), len(truth), truth, names, "cfg3")


def lkt_zf(nhist: int = 2, nbins: int = 1600, bin_width_ns: float = 8.0, seed: int = 7,
           dtype=np.float64, n0: float = 3000.0) -> Problem:
    """Zero-field static Lorentzian Kubo-Toyabe: A = A0 LKT(a, t); shared A0, a; per-histogram
    N0, Nbkg (2 + 2 H parameters)."""
    terms = [[("AMP", (2,)), ("LKT", (3,))]]
    rows = [[2 + 2 * j, 3 + 2 * j, 0, 1] for j in range(nhist)]
    names = ["A0", "a"]
    truth = [0.22, 0.6]
    for j in range(nhist):
        names += [f"N0_{j}", f"Nbkg_{j}"]
        truth += [n0, 2.0]
    dets = [Detector(truth[2 + 2 * j], truth[3 + 2 * j], 0.0) for j in range(nhist)]
    comps = [[Component(truth[0], "ZFL", delta=truth[1])] for _ in range(nhist)]
    counts = simulate(seed, dets, comps, nbins, bin_width_ns, dtype)
    return Problem(counts, np.zeros(nhist), bin_width_ns, _full_range(nbins, bin_width_ns), terms,
                   np.array(rows, np.int32), np.zeros(0), len(truth), np.array(truth), names, "lkt_zf")


def cfg5(nhist: int = 64, nbins: int = 1 << 20, bin_width_ns: Optional[float] = None, seed: int = 5,
         dtype=np.float32, n0: float = 2.0, nbkg: float = 0.01) -> Problem:
    """Large single fit: two-term TF (as cfg2) plus 0.05 KT(Delta, t); 5 + 3 H parameters (197 for H = 64).

    Low statistics (N0 = 2 counts per bin), the maximum-likelihood regime.
    """
    if bin_width_ns is None:
        bin_width_ns = 12800.0 / nbins
    terms = [[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))],
             [("AMP", (6,)), ("GAUSS", (7,)), ("TFCOS", (8, 5))],
             [("AMP", (9,)), ("KT", (10,))]]
    shared = {"lambda": 0, "sigma": 1, "nu1": 2, "nu2": 3, "delta": 4}
    mp = _tf2_map(nhist, 5, shared, True)
    names = ["lambda", "sigma", "nu1", "nu2", "Delta"]
    truth = [0.5, 0.3, 5.0, 5.5, 0.3]
    dets, comps = [], []
    for j in range(nhist):
        ph = 360.0 * j / nhist
        names += [f"N0_{j}", f"Nbkg_{j}", f"phi_{j}"]
        truth += [n0, nbkg, ph]
        dets.append(Detector(n0, nbkg, ph))
        comps.append([Component(0.125, "TF", nu_mhz=5.0, lam=0.5),
                      Component(0.125, "TF", nu_mhz=5.5, sigma=0.3),
                      Component(0.05, "ZF", delta=0.3)])
    counts = simulate(seed, dets, comps, nbins, bin_width_ns, dtype)
    return Problem(counts, np.zeros(nhist), bin_width_ns, _full_range(nbins, bin_width_ns), terms,
                   mp, np.array([0.125, 0.125, 0.05]), len(truth), np.array(truth), names, "cfg5")


def paper_tf16(nhist: int = 16, nbins: int = 81920, bin_width_ns: Optional[float] = None,
               seed: int = 16, dtype=np.float32, n0: float = 300.0) -> Problem:
    """The paper's benchmark model (Eq. asymmetry): A_j = A0_j exp(-(sigma t)^2/2) cos(2 pi nu t + phi_j).

    Per detector N0, Nbkg, A0, phi; shared sigma and nu: 4 H + 2 parameters (66 for 16 detectors).
    """
    if bin_width_ns is None:
        bin_width_ns = 12800.0 / nbins
    terms = [[("AMP", (2,)), ("GAUSS", (3,)), ("TFCOS", (4, 5))]]
    rows = [[2 + 4 * j, 3 + 4 * j, 4 + 4 * j, 0, 1, 5 + 4 * j] for j in range(nhist)]
    names = ["sigma", "nu"]
    truth = [0.3, 10.0]
    dets, comps = [], []
    for j in range(nhist):
        ph = 360.0 * j / nhist
        a0 = 0.2 + 0.002 * j
        names += [f"N0_{j}", f"Nbkg_{j}", f"A0_{j}", f"phi_{j}"]
        truth += [n0, 2.0, a0, ph]
        dets.append(Detector(n0, 2.0, ph))
        comps.append([Component(a0, "TF", nu_mhz=10.0, sigma=0.3)])
    counts = simulate(seed, dets, comps, nbins, bin_width_ns, dtype)
    return Problem(counts, np.zeros(nhist), bin_width_ns, _full_range(nbins, bin_width_ns), terms,
                   np.array(rows, np.int32), np.zeros(0), len(truth), np.array(truth), names,
                   "paper_tf16")


def inc_bessel(nhist: int = 2, nbins: int = 1600, bin_width_ns: float = 8.0, seed: int = 8, n0: float = 3000.0,
               dtype=np.float32) -> Problem:
    """Incommensurate magnetic order: fields gamma B = 2 pi nu cos(U) with U uniform give the
    polarisation J0(2 pi nu t) (detector phase 0; the second detector at 180 degrees sees
    -J0).  Model A_j = A0_j J0(2 pi nu t) e^{-lambda t} (BESSEL phase fixed at 0 through a
    constant); per detector N0, Nbkg, A0; shared nu, lambda."""
    dets, comps, names, truth = [], [], ["nu", "lambda"], [2.5, 0.3]
    rows = []
    for j in range(nhist):
        ph = 0.0 if j % 2 == 0 else 180.0
        dets.append(Detector(n0, 2.0, ph))
        comps.append([Component(0.22, "INC", nu_mhz=2.5, lam=0.3)])
        names += [f"N0_{j}", f"Nbkg_{j}", f"A0_{j}"]
        truth += [n0, 2.0, 0.22 if ph == 0.0 else -0.22]
        rows.append([2 + 3 * j, 3 + 3 * j, 4 + 3 * j, 0, -1, 1])
    counts = simulate(seed, dets, comps, nbins, bin_width_ns, dtype)
    terms = [[("AMP", (2,)), ("BESSEL", (3, 4)), ("EXP", (5,))]]
    return Problem(counts, np.zeros(nhist), bin_width_ns, _full_range(nbins, bin_width_ns), terms,
                   np.array(rows, np.int32), np.array([0.0]), len(truth), np.array(truth), names, "inc_bessel")


def levy_lf(nhist: int = 2, nbins: int = 1600, bin_width_ns: float = 8.0, seed: int = 9, n0: float = 3000.0,
            dtype=np.float32) -> Problem:
    """Depolarisation at rates drawn from a one-sided Levy distribution (r = lambda / (2 Z^2)),
    whose average exp(-r t) is exp(-(lambda t)^(1/2)): model A = A0 exp(-(lambda t)^beta) with
    beta fitted (truth 1/2); shared A0, lambda, beta; per detector N0, Nbkg."""
    dets = [Detector(n0, 2.0, 0.0) for _ in range(nhist)]
    comps = [[Component(0.25, "LF", levy=0.8)] for _ in range(nhist)]
    counts = simulate(seed, dets, comps, nbins, bin_width_ns, dtype)
    terms = [[("AMP", (2,)), ("STREXP", (3, 4))]]
    rows = [[3 + 2 * j, 4 + 2 * j, 0, 1, 2] for j in range(nhist)]
    names = ["A0", "lambda", "beta"] + [n for j in range(nhist) for n in (f"N0_{j}", f"Nbkg_{j}")]
    truth = [0.25, 0.8, 0.5] + [v for _ in range(nhist) for v in (n0, 2.0)]
    return Problem(counts, np.zeros(nhist), bin_width_ns, _full_range(nbins, bin_width_ns), terms,
                   np.array(rows, np.int32), np.zeros(0), len(truth), np.array(truth), names, "levy_lf")


def dkt_zf(nhist: int = 2, nbins: int = 1600, bin_width_ns: float = 8.0, seed: int = 10, n0: float = 3000.0,
           delta: float = 0.4, nu_c: float = 0.8, dtype=np.float32) -> Problem:
    """Zero-field run in fluctuating Gaussian fields (strong collisions at rate nu_c): model
    A = A0 DKT(Delta, nu) with shared A0, Delta, nu; per detector N0, Nbkg."""
    dets = [Detector(n0, 2.0, 0.0) for _ in range(nhist)]
    comps = [[Component(0.25, "DZF", delta=delta, nu_c=nu_c)] for _ in range(nhist)]
    counts = simulate(seed, dets, comps, nbins, bin_width_ns, dtype)
    terms = [[("AMP", (2,)), ("DKT", (3, 4))]]
    rows = [[3 + 2 * j, 4 + 2 * j, 0, 1, 2] for j in range(nhist)]
    names = ["A0", "Delta", "nu"] + [n for j in range(nhist) for n in (f"N0_{j}", f"Nbkg_{j}")]
    truth = [0.25, delta, nu_c] + [v for _ in range(nhist) for v in (n0, 2.0)]
    return Problem(counts, np.zeros(nhist), bin_width_ns, _full_range(nbins, bin_width_ns), terms,
                   np.array(rows, np.int32), np.zeros(0), len(truth), np.array(truth), names, "dkt_zf")


@dataclasses.dataclass
class AsymmetryProblem:
    """A fit of asymmetry data: forward / backward histogram pairs ([H][B] each) with the
    relative efficiency alpha and constant backgrounds of each pair; theory and map as for
    histograms, with local slot 0 the scale and slot 1 the baseline of T = N0 A(t) + Nbkg."""

    forward: np.ndarray
    backward: np.ndarray
    alpha: np.ndarray  # [H]
    bkg_f: np.ndarray  # [H] counts per bin
    bkg_b: np.ndarray
    t0: np.ndarray
    bin_width_ns: float
    fit_range_us: Tuple[float, float]
    terms: List[Term]
    map: np.ndarray
    consts: np.ndarray
    nparams: int
    truth: np.ndarray
    names: List[str]
    name: str = ""

    @property
    def H(self) -> int:
        return int(self.forward.shape[0])

    @property
    def B(self) -> int:
        return int(self.forward.shape[1])

    @property
    def nslots(self) -> int:
        return int(self.map.shape[1])


def asym_tf(npairs: int = 2, nbins: int = 8192, bin_width_ns: float = 1.0, seed: int = 21, n0: float = 400.0,
            eff_b: float = 0.85, nbkg: float = 3.0, dtype=np.float32) -> AsymmetryProblem:
    """Transverse-field asymmetry fit: detector pairs at phases phi_k and phi_k + 180 deg, the
    backward detector with efficiency eff_b (so alpha = 1 / eff_b), one TF component with
    Gaussian damping.  Model A = A0 exp(-(sigma t)^2 / 2) cos(2 pi (nu t + phi_k / 360)),
    shared A0, sigma, nu, a phase per pair; scale 1 and baseline 0 (constants)."""
    comps = [Component(0.22, "TF", nu_mhz=3.0, sigma=0.4)]
    dets, cps, phis = [], [], []
    for k in range(npairs):
        ph = 20.0 + 90.0 * k
        phis.append(ph)
        dets += [Detector(n0, nbkg, ph), Detector(n0 * eff_b, nbkg, ph + 180.0)]
        cps += [comps, comps]
    h = simulate(seed, dets, cps, nbins, bin_width_ns, dtype)
    terms = [[("AMP", (2,)), ("GAUSS", (3,)), ("TFCOS", (4, 5))]]
    rows = [[-1, -2, 0, 1, 2, 3 + k] for k in range(npairs)]
    names = ["A0", "sigma", "nu"] + [f"phi_{k}" for k in range(npairs)]
    truth = [0.22, 0.4, 3.0] + phis
    return AsymmetryProblem(np.ascontiguousarray(h[0::2]), np.ascontiguousarray(h[1::2]),
                            np.full(npairs, 1.0 / eff_b), np.full(npairs, nbkg), np.full(npairs, nbkg),
                            np.zeros(npairs), bin_width_ns, _full_range(nbins, bin_width_ns), terms,
                            np.array(rows, np.int32), np.array([1.0, 0.0]), len(truth), np.array(truth), names,
                            "asym_tf")


CONFIGS = {"cfg1": cfg1, "cfg2": cfg2, "cfg3": cfg3, "cfg5": cfg5, "paper_tf16": paper_tf16}


# --------------------------------------------------------------------------------------------
# Serving request stream (the continuous-batching workload)
# --------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Request:
    arrival_s: float
    problem: Problem
    x0: np.ndarray
    mode: int  # 0 chi^2, 1 -2lnL


def _pool_member(spec) -> Problem:
    kind, H, B, dtw, n0, sub, jit, dtype = spec
    if kind == 0:
        return cfg1(nbins=B, bin_width_ns=dtw, seed=sub, dtype=dtype, n0=n0, jitter_seed=jit)
    if kind == 1:
        return cfg2(nhist=H, nbins=B, bin_width_ns=dtw, seed=sub, dtype=dtype, n0=n0, jitter_seed=jit)
    return cfg3(nhist=H, nbins=B, bin_width_ns=dtw, seed=sub, dtype=dtype, n0=n0, jitter_seed=jit)


def serving_pool(n_pool: int, seed: int = 4, hist_range=(1, 64), bin_range=(4096, 262144),
                 span_ns: float = 12800.0, dtype=np.float32, workers: int = 1) -> List[Problem]:
    """A pool of distinct fits: H ~ logU(hist_range), B ~ logU(bin_range), theory drawn from
    cfg1/cfg2/cfg3, truths jittered by U(0.8, 1.2), each fit its own seeded Monte Carlo.

    N0 is scaled by min(1, 4096 / B) so that every histogram holds about the same
    number of events whatever its binning (a fixed-length run binned finer).  With
    workers > 1 the fits are simulated by that many spawned processes (the same fits).
    """
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n_pool):
        H = int(round(math.exp(rng.uniform(math.log(hist_range[0]), math.log(hist_range[1])))))
        B = int(round(math.exp(rng.uniform(math.log(bin_range[0]), math.log(bin_range[1])))))
        kind = int(rng.integers(0, 3))
        dtw = span_ns / B
        n0 = 300.0 * min(1.0, 4096.0 / B)
        sub = int(rng.integers(0, 2**31))
        jit = int(rng.integers(0, 2**31))
        specs.append((kind, H, B, dtw, n0, sub, jit, dtype))
    if workers > 1 and n_pool > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, n_pool)) as pool:
            return pool.map(_pool_member, specs, chunksize=1)
    return [_pool_member(sp) for sp in specs]


def request_stream(pool: Sequence[Problem], n_requests: int, rate_per_s: float, seed: int = 4,
                   mode_mix: float = 0.5) -> List[Request]:
    """Poisson arrivals at ``rate_per_s`` (0 or inf: all at t = 0); start points from
    :func:`start_point` around each fit's (jittered) truth."""
    rng = np.random.default_rng(seed + 1)
    t = 0.0
    out = []
    for i in range(n_requests):
        if rate_per_s and math.isfinite(rate_per_s):
            t += rng.exponential(1.0 / rate_per_s)
        p = pool[i % len(pool)]
        x0 = start_point(p, int(rng.integers(0, 2**31)))
        mode = int(rng.random() < mode_mix)
        out.append(Request(t, p, x0, mode))
    return out
