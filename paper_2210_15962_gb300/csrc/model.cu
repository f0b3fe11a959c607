// The paper's predictive model (Section 4.1, Eq. 6, Eq. 7): host arithmetic
// behind the C ABI.  The run lengths (solution evaluations) that reach an
// optimal skew-symmetric sequence are exponentially distributed with rate
// lambda(L) = 0.006753 * 0.8617^L, the authors' fit on L = 71..119.
#include <cmath>
#include <cstdint>

#include "labs.h"

namespace {

bool model_L(int32_t L) { return L >= LABS_L_MIN && L <= LABS_L_MAX && (L & 1); }

}  // namespace

extern "C" double labs_model_lambda(int32_t L) {
  if (!model_L(L)) return NAN;
  return 0.006753 * std::pow(0.8617, (double)L);
}

extern "C" double labs_model_nses_limit(int32_t L, double P, int32_t N) {
  if (!model_L(L) || !(P >= 0.0 && P < 1.0) || N < 1) return NAN;
  return std::log1p(-P) / (-labs_model_lambda(L) * (double)N);  // Eq. 6
}

extern "C" double labs_model_p_optimal(int32_t L, double nses) {
  if (!model_L(L) || !(nses >= 0.0)) return NAN;
  return -std::expm1(-labs_model_lambda(L) * nses);  // Eq. 7
}

extern "C" double labs_model_nses_of_evals(int32_t L, uint64_t evals) {
  if (!model_L(L)) return NAN;
  const double D = (double)((L + 1) / 2);
  return (double)evals * (D - 1.0) / D;
}

extern "C" uint64_t labs_model_budget(int32_t L, double P) {
  const double nses = labs_model_nses_limit(L, P, 1);
  if (!(nses >= 0.0)) return 0;
  const double D = (double)((L + 1) / 2);
  const double evals = std::ceil(nses * D / (D - 1.0));
  if (evals >= 18446744073709551615.0) return UINT64_MAX;
  return evals < 1.0 ? 1u : (uint64_t)evals;
}
