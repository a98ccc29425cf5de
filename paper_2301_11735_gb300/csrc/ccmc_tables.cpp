// ccmc_tables.cpp -- host-side parameter tables of the sweep.  Compiled with
// -ffp-contract=off so every FP64 operation rounds in the order written.
#include <cmath>
#include <cstdint>

#include "ccmc_internal.h"

namespace ccmc {

namespace {
// Site values of the four codes (Sec. 2.1): S, and sigma = 2 (1 - S^2) s.
constexpr int kS[4] = {0, 0, 1, -1};
constexpr int kSigma[4] = {1, -1, 0, 0};

// Metropolis acceptance threshold of an energy change (Sec. 3.1): the move is
// accepted iff the threshold is 0xFFFFFFFF or a uniform 32-bit word lies below
// it, i.e. with probability min(1, exp(-beta dE)) to within 2^-32.
uint32_t threshold(double beta, double Delta, double V, double J, int dQ, int dBV, int dBJ) {
  const double eQ = Delta * static_cast<double>(dQ);
  const double eV = V * static_cast<double>(dBV);
  const double eQV = eQ + eV;
  const double quarterJ = 0.25 * J;
  const double eJ = quarterJ * static_cast<double>(dBJ);
  const double dE = eQV + eJ;  // Eq. (3): Delta dQ + V dBV + (J/4) dBJ
  if (dE <= 0.0) return 0xFFFFFFFFu;
  const double p = std::exp(-beta * dE);
  if (p >= 1.0) return 0xFFFFFFFFu;
  const double scaled = std::floor(std::ldexp(p, 32));
  if (scaled >= 4294967295.0) return 0xFFFFFFFEu;
  return static_cast<uint32_t>(scaled);
}
}  // namespace

void build_thresholds(double beta, double Delta, double V, double J, uint32_t *thr32) {
  for (int dqi = 0; dqi < 3; ++dqi)
    for (int dBV = -kDB; dBV <= kDB; ++dBV)
      for (int dBJ = -kDB; dBJ <= kDB; ++dBJ)
        thr32[(dqi * kNB + dBV + kDB) * kNB + dBJ + kDB] =
            threshold(beta, Delta, V, J, 2 * dqi - 2, dBV, dBJ);
}

// Move entries (see the phase kernel).  For choice class r = v mod 12, kind
// near (the partner is a nearest neighbour) and pair state pc = 4 a + b, the
// proposed state is the (r mod |set|)-th configuration of the pair's q-set in
// the paper's order (Sec. 3.1); frozen pairs (|q| = 2) propose themselves.  dE
// of the move:
//   dBV = dS_a sum_<a> S + dS_b sum_<b> S + m dS_a dS_b
//   dBJ = dsig_a sum_<a> sigma + dsig_b sum_<b> sigma + m dsig_a dsig_b
// with neighbour sums over old states (partner included) and m = near the number
// of a-b bonds.  As dS_b = -dS_a, the threshold index
//   ((dQ + 2)/2 * 41 + dBV + 20) * 41 + dBJ + 20
// is an affine function of the biased sums D8 = sum_<a> S - sum_<b> S + 8,
// GA = sum_<a> sigma + 4, GB = sum_<b> sigma + 4:
//   index = base + (41 dS_a) D8 + dsig_a GA + dsig_b GB.
// Entry (2 r + near) * 16 + (pc XOR r): word 0 holds base; word 1 the signed byte
// coefficients (41 dS_a, dsig_a, dsig_b) and, in bits 24-27 (byte 3, which
// the phase kernel multiplies by zero; bits 28-31 stay clear), pc XOR npc.
namespace {
constexpr int kSetN[3] = {4, 6, 4};  // q = +1, 0, -1
constexpr int kSets[3][6][2] = {
    {{2, 0}, {2, 1}, {0, 2}, {1, 2}, {0, 0}, {0, 0}},  // q = +1
    {{2, 3}, {3, 2}, {0, 0}, {1, 1}, {0, 1}, {1, 0}},  // q = 0
    {{3, 0}, {3, 1}, {0, 3}, {1, 3}, {0, 0}, {0, 0}},  // q = -1
};
}  // namespace

bool build_transitions(uint32_t *trans) {
  int lo = 1 << 30, hi = -(1 << 30);
  for (int pc = 0; pc < 16; ++pc) {
    const int ca = pc >> 2, cb = pc & 3;
    const int q = kS[ca] + kS[cb];
    for (int r = 0; r < 12; ++r) {
      int na = ca, nb = cb;
      if (q >= -1 && q <= 1) {
        const int qi = 1 - q;
        na = kSets[qi][r % kSetN[qi]][0];
        nb = kSets[qi][r % kSetN[qi]][1];
      }
      const int dQ = kS[na] * kS[na] + kS[nb] * kS[nb] - kS[ca] * kS[ca] - kS[cb] * kS[cb];
      const int dSa = kS[na] - kS[ca], dSb = kS[nb] - kS[cb];
      const int dGa = kSigma[na] - kSigma[ca], dGb = kSigma[nb] - kSigma[cb];
      const int mulS = kNB * dSa;
      const int base = (dQ + 2) / 2 * kNB * kNB + kDB * kNB + kDB - 4 * (dGa + dGb) - 8 * mulS;
      const int near_base = base + kNB * dSa * dSb + dGa * dGb;
      const uint32_t x = (uint32_t)(((ca ^ na) << 2) | (cb ^ nb));
      const uint32_t coef = ((uint32_t)mulS & 0xFFu) | (((uint32_t)dGa & 0xFFu) << 8) |
                            (((uint32_t)dGb & 0xFFu) << 16) | (x << 24);
      for (int near = 0; near < 2; ++near) {
        const int e = (2 * r + near) * 16 + (pc ^ r);  // bank-spread (see the phase kernel)
        trans[2 * e] = (uint32_t)(near ? near_base : base);
        trans[2 * e + 1] = coef;
      }
      // every index an entry can form, over all possible neighbour sums
      // (D8 in [0, 16], GA and GB in [0, 8]), must stay inside the table
      for (int b0 : {base, near_base})
        for (int D8 : {0, 16})
          for (int ga : {0, 8})
            for (int gb : {0, 8}) {
              const int idx = b0 + mulS * D8 + dGa * ga + dGb * gb;
              lo = idx < lo ? idx : lo;
              hi = idx > hi ? idx : hi;
            }
    }
  }
  return lo >= 0 && hi < kTableN;
}

}  // namespace ccmc
