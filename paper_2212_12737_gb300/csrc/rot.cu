// Preconditioner size from the runtime model of Sec. 4.3 (host arithmetic, no device work).
//
// The model (Eq. 7, without its n^3 factor) is
//     cost(k) = (k_min / k)^m + (k / n)^2,
// the PCG term falling as a power law in the number k of inducing columns and the
// preconditioner term growing as k^2 n.  Eq. 8 picks the k in [1, n] that minimises it.
// Its stationary point solves m k_min^m k^-(m+1) = 2 k / n^2, i.e.
//     k* = (m k_min^m n^2 / 2)^(1 / (2 + m)),
// and cost is convex for k > 0 (both terms are), so the best integer is floor(k*) or
// ceil(k*), clamped to [1, n]; a tie goes to the smaller one.
#include <cmath>
#include <string>

#include "common.cuh"

using namespace gdml;

namespace {

double rot_cost(double k, double n, double m, double k_min) {
  const double r = k / n;
  return std::pow(k_min / k, m) + r * r;
}

}  // namespace

extern "C" gdml_status gdml_rule_of_thumb_k(int64_t n, double m, double k_min, int64_t* k_out) {
  if (!k_out) return fail(GDML_ERR_ARG, "rule_of_thumb_k: k_out is NULL");
  if (n < 1 || !(m > 0.0) || !std::isfinite(m) || !(k_min > 0.0) || !std::isfinite(k_min))
    return fail(GDML_ERR_ARG, "rule_of_thumb_k: need n >= 1, finite m > 0 and finite k_min > 0");
  const double nd = (double)n;
  // k* in logarithms: no overflow of k_min^m n^2 for large n or m
  const double ls = (std::log(m) + m * std::log(k_min) + 2.0 * std::log(nd) - std::log(2.0)) / (2.0 + m);
  const double ks = std::exp(ls);
  int64_t lo = ks >= nd ? n : (int64_t)std::floor(ks);
  if (lo < 1) lo = 1;
  const int64_t hi = lo < n ? lo + 1 : n;
  *k_out = rot_cost((double)hi, nd, m, k_min) < rot_cost((double)lo, nd, m, k_min) ? hi : lo;
  return GDML_OK;
}
