// advise.cu -- sketch-size advisor (Section 6: optimized sketch size and complexity).
// Host-only arithmetic: the sketch size m* that minimises the paper's flop model of PCG,
// the model's cost ratio to the classical choice, and the predicted iteration count
// T = ceil(log(4/eps) / log(m* / m_delta)) (Section 6, with rho = m_delta / m).
#include <math.h>

#include "common.cuh"

namespace {

// principal branch of the Lambert W function for a > 0: Halley's iteration on w e^w = a
// (Corless, Gonnet, Hare, Jeffrey, Knuth, "On the Lambert W function", 1996)
double lambert_w0(double a) {
  double w = a < 2.718281828459045 ? a / (1.0 + a) : log(a) - log(log(a));
  for (int it = 0; it < 64; ++it) {
    const double ew = exp(w);
    const double f = w * ew - a;
    const double step = f / (ew * (w + 1.0) - (w + 2.0) * f / (2.0 * w + 2.0));
    w -= step;
    if (fabs(step) <= 1e-15 * (1.0 + fabs(w))) break;
  }
  return w;
}

}  // namespace

extern "C" lsq_status lsq_advise_sketch_size(int64_t n, int64_t d, double eps, int32_t sketch_type, lsq_advice* out) {
  if (!out || n < 1 || d < 2 || !(eps > 0.0) || !(eps < 1.0)) return LSQ_ERR_ARG;
  const double nd = (double)n, dd = (double)d;
  if (nd <= dd * dd) return LSQ_ERR_ARG;  // the analysis assumes n > d^2
  const double L = log(1.0 / eps), Lr = log(nd / (dd * dd));
  double m_star, cost, cost_cl, m_delta;
  if (sketch_type == LSQ_SKETCH_GAUSS) {
    // Theorem theoremoptimalcomplexitygaussian: alpha* log alpha* = (n/d^2) log(1/eps)
    const double alpha = exp(lambert_w0(nd / (dd * dd) * L));
    m_star = dd * alpha;
    m_delta = dd;
    cost = nd * dd * L / Lr;  // O(nd log(1/eps) / log(n/d^2)), constants dropped
    cost_cl = nd * dd * L;    // m = O(d): O(nd log(1/eps))
    out->regime = 0;
  } else if (sketch_type == LSQ_SKETCH_SRHT) {
    // Theorem theoremoptimalcomplexitysrht, cases (i) and (ii)
    const double logd = log(dd);
    m_delta = dd * logd;
    if (sqrt(L) < Lr) {
      m_star = exp(sqrt(L)) * dd * logd;
      cost = nd * dd * (logd + sqrt(L));
      out->regime = 1;
    } else {
      m_star = nd / dd * fmax(logd, L / Lr);
      cost = nd * dd * (logd + L / Lr);
      out->regime = 2;
    }
    cost_cl = nd * dd * (logd + L);  // m = O(d log d)
  } else {
    return LSQ_ERR_ARG;  // the paper gives no sketch-size result for the SJLT
  }
  out->m_star = m_star;
  out->cost_ratio = cost / cost_cl;
  out->predicted_iters = m_star > m_delta ? ceil(log(4.0 / eps) / log(m_star / m_delta)) : -1.0;
  return LSQ_OK;
}
