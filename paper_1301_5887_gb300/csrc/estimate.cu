// estimate.cu — FP64 estimators over the integer tallies (wedge_estimate).
//
// Per bin (Thm 3.2, Thm 3.3): c_b = (q1+q2+q3)/k_b, t_b = p_b (q1 + q2/2 + q3/3)/k_b,
// with the Hoeffding half-width eps_b = sqrt(ln(2/delta)/(2 k_b)) (Thm 3.1).
// Global from bins, Eq. (global_est): c_hat = sum_b (p_b/p) c_b, t_hat = c_hat p/3.
// Global stream (one bin of all degrees >= 2): c = closed/k, t = c p/3 (Eq. CC).
#include <math.h>
#include <string.h>

#include "runtime.h"

using namespace wedge;

extern "C" wedge_status wedge_estimate(const wedge_counts* c, double delta, wedge_estimates* out) {
  clear_error();
  if (!c || !out) return fail(WEDGE_EINVAL, "wedge_estimate: NULL argument");
  if (!(delta > 0.0 && delta < 1.0)) return fail(WEDGE_EINVAL, "wedge_estimate: delta must lie in (0, 1)");
  if (c->n_bins > WEDGE_MAX_BINS) return fail(WEDGE_EINVAL, "wedge_estimate: n_bins > WEDGE_MAX_BINS");
  memset(out, 0, sizeof(*out));
  out->n_bins = c->n_bins;
  const double p = (double)c->p_total;
  out->p_total = p;
  const double log_term = log(2.0 / delta);
  double c_hat = 0.0;
  for (uint32_t b = 0; b < c->n_bins; ++b) {
    const uint64_t k = c->k_b[b];
    if (k == 0) continue;
    const double kd = (double)k;
    const double q1 = (double)c->q[b][1], q2 = (double)c->q[b][2], q3 = (double)c->q[b][3];
    out->c_b[b] = (q1 + q2 + q3) / kd;
    out->t_b[b] = (double)c->p_b[b] * (q1 + q2 / 2.0 + q3 / 3.0) / kd;
    out->eps_b[b] = sqrt(log_term / (2.0 * kd));
    if (p > 0.0) c_hat += ((double)c->p_b[b] / p) * out->c_b[b];
  }
  out->c_hat = c_hat;
  out->t_hat = c_hat * p / 3.0;
  if (c->k_global > 0) {
    const double kg = (double)c->k_global;
    out->c_hat_global = (double)c->closed_global / kg;
    out->t_hat_global = out->c_hat_global * p / 3.0;
    out->eps_global = sqrt(log_term / (2.0 * kg));
  }
  return WEDGE_OK;
}
