// musr_plan.h -- host-side planning of the SPLIT path: canonical terms, shape,
// basis amplitudes and the slot -> channel contributions (Section 4.1 model,
// Eq. positron_histo and Eq. asymmetry).  Heap-free, so that the allocation-free
// entry point can use it too.
#pragma once

#include <cstdint>
#include <cstring>

#include "musr.h"
#include "musr_dev.h"

namespace musr {

// Canonical form of one term; false if the term is not
// a * exp(-Lambda t - S t^2/2) * [KT, LKT, DKT or TFCOS] with at most one AMP.
inline bool canonical_term(const musr_term& t, CanonTerm* ct) {
  std::memset(ct, 0, sizeof(*ct));
  ct->amp_slot = ct->kt_slot = ct->nu_slot = ct->phi_slot = ct->dkt_term = ct->dkt_prim = -1;
  int namp = 0, nkt = 0, nlkt = 0, ntf = 0, ndkt = 0;
  for (int m = 0; m < t.nprim; ++m) {
    switch (t.kind[m]) {
      case MUSR_PRIM_AMP:
        ct->amp_slot = t.slot[m][0];
        ++namp;
        break;
      case MUSR_PRIM_EXP:
        ct->exp_slot[ct->nexp++] = t.slot[m][0];
        break;
      case MUSR_PRIM_GAUSS:
        ct->gauss_slot[ct->ngauss++] = t.slot[m][0];
        break;
      case MUSR_PRIM_KT:
        ct->kt_slot = t.slot[m][0];
        ++nkt;
        break;
      case MUSR_PRIM_TFCOS:
        ct->nu_slot = t.slot[m][0];
        ct->phi_slot = t.slot[m][1];
        ++ntf;
        break;
      case MUSR_PRIM_LKT:
        ct->kt_slot = t.slot[m][0];
        ++nlkt;
        break;
      case MUSR_PRIM_DKT:  // a time-only factor, read per bin from the evaluation's table
        ct->kt_slot = t.slot[m][0];
        ct->nu_slot = t.slot[m][1];
        ct->dkt_prim = m;
        ++ndkt;
        break;
      default:  // STREXP, BESSEL: no basis form (the SPLIT path evaluates the term list)
        return false;
    }
  }
  if (namp > 1 || nkt + nlkt + ntf + ndkt > 1) return false;
  ct->kind = ntf ? kTermTF : (nkt ? kTermKT : (nlkt ? kTermLKT : (ndkt ? kTermDKT : kTermPlain)));
  return true;
}

// The value a slot of histogram h takes if it maps to a constant; false if it maps
// to a parameter.
inline bool slot_constant(const int32_t* map, const double* consts, int nslots, int h, int s, double* v) {
  const int32_t m = map[static_cast<int64_t>(h) * nslots + s];
  if (m >= 0) return false;
  *v = consts[-1 - m];
  return true;
}

// True when, for every histogram, all cosine terms take their phase from one
// parameter (or equal constants).
inline bool phases_shared(const CanonTerm* canon, int nterms, const int32_t* map, const double* consts, int H,
                          int nslots) {
  for (int h = 0; h < H; ++h) {
    int first = -1;
    for (int k = 0; k < nterms; ++k) {
      if (canon[k].kind != kTermTF) continue;
      if (first < 0) {
        first = k;
        continue;
      }
      const int32_t m = map[static_cast<int64_t>(h) * nslots + canon[k].phi_slot];
      const int32_t m0 = map[static_cast<int64_t>(h) * nslots + canon[first].phi_slot];
      const bool same = (m >= 0 || m0 >= 0) ? m == m0 : consts[-1 - m] == consts[-1 - m0];
      if (!same) return false;
    }
  }
  return true;
}

// Amplitude of term k if it is the same constant for every histogram (1 without
// an AMP factor); false if some histogram maps it to a parameter or the constants differ.
inline bool shared_constant_amplitude(const CanonTerm& ct, const int32_t* map, const double* consts, int H,
                                      int nslots, double* a) {
  if (ct.amp_slot < 0) {
    *a = 1.0;
    return true;
  }
  double v0 = 0.0;
  for (int h = 0; h < H; ++h) {
    double v;
    if (!slot_constant(map, consts, nslots, h, ct.amp_slot, &v)) return false;
    if (h == 0)
      v0 = v;
    else if (v != v0)
      return false;
  }
  *a = v0;
  return true;
}

// Plans the SPLIT path of a theory and map into hs (canon in cosine-first order,
// nterms, shape, merged, bamp, contributions).  Returns nullptr, or why the theory has no
// basis form (the SPLIT path then evaluates its term list per bin).
// Without the decay envelope (asymmetry data) no shape is merged: a merged shape folds the
// non-cosine terms into the basis function that carries the 1 of (1 + A).
inline const char* plan_split(const musr_term* terms, int nterms, const int32_t* map, int H, int nslots,
                              const double* consts, HistSet* hs, bool envelope = true) {
  if (nterms > kMaxTerms) return "at most 4 terms";
  CanonTerm canon[kMaxTerms];
  for (int k = 0; k < nterms; ++k) {
    if (!canonical_term(terms[k], &canon[k]))
      return "SPLIT precision needs every term to hold at most one AMP, and at most one of KT, LKT, DKT or "
             "TFCOS (STREXP and BESSEL have no basis form)";
    if (canon[k].kind == kTermDKT) canon[k].dkt_term = k;
  }
  // Cosine terms first (the model is a sum: the order of its terms is free).
  int ntf = 0, nn = 0;
  hs->nterms = nterms;
  for (int k = 0; k < nterms; ++k)
    if (canon[k].kind == kTermTF) hs->canon[ntf++] = canon[k];
  for (int k = 0; k < nterms; ++k)
    if (canon[k].kind != kTermTF) hs->canon[ntf + nn++] = canon[k];
  // Merged: every amplitude one shared constant, one phase per histogram, and no dynamic
  // Kubo-Toyabe factor (the merged kernels, the fastest, carry no code for its table).
  double amp[kMaxTerms];
  bool merged = envelope && ntf == 2 && nn <= 1 && phases_shared(hs->canon, nterms, map, consts, H, nslots);
  for (int k = 0; k < nterms; ++k) merged = merged && hs->canon[k].kind != kTermDKT;
  for (int k = 0; k < nterms && merged; ++k)
    merged = shared_constant_amplitude(hs->canon[k], map, consts, H, nslots, &amp[k]);
  hs->merged = merged ? 1 : 0;
  for (int k = 0; k < kMaxTerms; ++k) hs->bamp[k] = merged && k < nterms ? static_cast<float>(amp[k]) : 1.0f;
  if (merged)
    hs->shape = nn == 0 ? kShapeT2m : kShapeT2N1m;
  else if (ntf == 1 && nn == 0)
    hs->shape = kShapeT1;
  else if (ntf == 0 && nn == 1)
    hs->shape = kShapeN1;
  else if (ntf == 1 && nn == 1)
    hs->shape = kShapeT1N1;
  else if (ntf == 2 && nn == 0)
    hs->shape = kShapeT2;
  else if (ntf == 2 && nn == 1)
    hs->shape = kShapeT2N1;
  else
    hs->shape = kShapeGeneric;
  // Slot -> channel contributions.
  hs->ncontrib = 0;
  auto add = [&](int slot, int kind, int term) {
    hs->contrib[hs->ncontrib].slot = slot;
    hs->contrib[hs->ncontrib].kind = kind;
    hs->contrib[hs->ncontrib].term = term;
    ++hs->ncontrib;
  };
  add(0, kCN0, 0);
  add(1, kCBkg, 0);
  for (int k = 0; k < nterms; ++k) {
    const CanonTerm& ct = hs->canon[k];
    if (ct.amp_slot >= 0 && !merged) add(ct.amp_slot, kCAmp, k);
    for (int i = 0; i < ct.nexp; ++i) add(ct.exp_slot[i], kCLam, k);
    for (int i = 0; i < ct.ngauss; ++i) add(ct.gauss_slot[i], kCSig, k);
    if (ct.kind == kTermKT) add(ct.kt_slot, kCDel, k);
    if (ct.kind == kTermLKT) add(ct.kt_slot, kCLkt, k);
    if (ct.kind == kTermDKT) {
      add(ct.kt_slot, kCDktD, k);
      add(ct.nu_slot, kCDktN, k);
    }
    if (ct.kind == kTermTF) {
      add(ct.nu_slot, kCNu, k);
      // merged: one phase per histogram, whose slot receives the derivative once
      if (!merged || k == 0) add(ct.phi_slot, kCPhi, k);
    }
  }
  return nullptr;
}

}  // namespace musr
