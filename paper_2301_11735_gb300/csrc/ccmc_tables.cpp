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

// Transition entries for pc = 4 a + b -> npc (see trans_index in the device
// header).  dE of a pair move (Sec. 3.1):
//   dBV = dS_a sum_<a> S + dS_b sum_<b> S + m dS_a dS_b
//   dBJ = dsig_a sum_<a> sigma + dsig_b sum_<b> sigma + m dsig_a dsig_b
// with neighbour sums over old states (partner included) and m the number of
// a-b bonds (0 or 1 here).  Because dS_b = -dS_a the V term is
// dS_a (SA - SB) in the biased sums SA = sum S + 4; the sigma biases and the
// m-term are folded into the base index.
void build_transitions(int32_t *trans_far, int32_t *trans_near) {
  for (int pc = 0; pc < 16; ++pc) {
    for (int npc = 0; npc < 16; ++npc) {
      const int ca = pc >> 2, cb = pc & 3, na = npc >> 2, nb = npc & 3;
      const int q0 = kS[ca] + kS[cb], q1 = kS[na] + kS[nb];
      int32_t far = 0, nearv = 0;
      if (q0 == q1 && q0 >= -1 && q0 <= 1) {
        const int dQ = kS[na] * kS[na] + kS[nb] * kS[nb] - kS[ca] * kS[ca] - kS[cb] * kS[cb];
        const int dSa = kS[na] - kS[ca], dSb = kS[nb] - kS[cb];
        const int dGa = kSigma[na] - kSigma[ca], dGb = kSigma[nb] - kSigma[cb];
        const int dqi = (dQ + 2) / 2;
        const int base = dqi * kNB * kNB + kDB * kNB + kDB - 4 * (dGa + dGb);
        const int near_base = base + kNB * dSa * dSb + dGa * dGb;
        const uint32_t fields = ((static_cast<uint32_t>(kNB * dSa) & 0xFFu) << 13) |
                                ((static_cast<uint32_t>(dGa) & 0xFu) << 21) |
                                ((static_cast<uint32_t>(dGb) & 0xFu) << 25);
        far = static_cast<int32_t>((static_cast<uint32_t>(base) & 0x1FFFu) | fields);
        nearv = static_cast<int32_t>((static_cast<uint32_t>(near_base) & 0x1FFFu) | fields);
      }
      trans_far[pc * 16 + npc] = far;
      trans_near[pc * 16 + npc] = nearv;
    }
  }
}

}  // namespace ccmc
