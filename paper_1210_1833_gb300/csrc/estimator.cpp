// estimator.cpp -- correlation-function estimators on exact pair counts
// (Sec. 2.2) and the angle -> chord helper.  Host FP64 arithmetic only,
// compiled without floating-point contraction.
#include "cute_internal.h"

#include <cmath>

extern "C" {

cute_status cute_estimator(cute_estimator_kind k, const uint64_t *DD, const uint64_t *DR,
                           const uint64_t *RR, int64_t Nd, int64_t Nr, int32_t nbins,
                           const double *edges, double box_L, double *xi_out) {
  if (!DD || !xi_out || nbins < 1) return CUTE_E_INVALID;
  if (k == CUTE_EST_PERIODIC) {
    // Eq. 13 with unique pairs: the expected count of uniform points in the
    // shell [e_b, e_b+1) of a periodic box is N(N-1)/2 * V_shell / L^3
    if (!edges || !(box_L > 0) || Nd < 2) return CUTE_E_INVALID;
    const double pi = 3.14159265358979323846;
    const double pairs = 0.5 * (double)Nd * (double)(Nd - 1);
    const double box = box_L * box_L * box_L;
    for (int b = 0; b < nbins; b++) {
      const double lo = edges[b], hi = edges[b + 1];
      const double vshell = (4.0 * pi / 3.0) * (hi * hi * hi - lo * lo * lo);
      const double expect = pairs * vshell / box;
      xi_out[b] = expect > 0 ? (double)DD[b] / expect - 1.0 : NAN;
    }
    return CUTE_OK;
  }
  if (!RR || Nd < 2 || Nr < 2) return CUTE_E_INVALID;
  // ratio of unique random pairs to unique data pairs
  const double f = ((double)Nr * (double)(Nr - 1)) / ((double)Nd * (double)(Nd - 1));
  if (k == CUTE_EST_NATURAL) {  // Eq. 14
    for (int b = 0; b < nbins; b++)
      xi_out[b] = RR[b] ? f * (double)DD[b] / (double)RR[b] - 1.0 : NAN;
    return CUTE_OK;
  }
  if (k == CUTE_EST_LS) {  // Eq. 15
    if (!DR) return CUTE_E_INVALID;
    const double g = (double)(Nr - 1) / (double)Nd;
    for (int b = 0; b < nbins; b++) {
      if (!RR[b]) { xi_out[b] = NAN; continue; }
      const double rr = (double)RR[b];
      xi_out[b] = (f * (double)DD[b] - g * (double)DR[b] + rr) / rr;
    }
    return CUTE_OK;
  }
  return CUTE_E_INVALID;
}

cute_status cute_theta_to_chord(const double *theta_deg, int32_t n, double *chord_out) {
  if (!theta_deg || !chord_out || n < 0) return CUTE_E_INVALID;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; i++) {
    if (!(theta_deg[i] >= 0 && theta_deg[i] <= 180)) return CUTE_E_INVALID;
    chord_out[i] = 2.0 * std::sin(0.5 * theta_deg[i] * (pi / 180.0));
  }
  return CUTE_OK;
}

}  // extern "C"
