// estimator.cpp -- correlation-function estimators on exact pair counts
// (Sec. 2.2), multipoles of xi(r, mu) (Sec. 2.1, Eq. 3-4) and the angle ->
// chord helper.  Host FP64 arithmetic only,
// compiled without floating-point contraction.
#include "cute_internal.h"

#include <cmath>
#include <vector>

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

// Legendre polynomials P_0..P_{lmax}(x) by Bonnet's recurrence
// (n + 1) P_{n+1} = (2n + 1) x P_n - n P_{n-1}.
static void legendre_all(double x, int lmax, double *P) {
  P[0] = 1.0;
  if (lmax >= 1) P[1] = x;
  for (int n = 1; n < lmax; n++) P[n + 1] = ((2.0 * n + 1.0) * x * P[n] - n * P[n - 1]) / (n + 1.0);
}

cute_status cute_multipoles(const double *xi, int32_t n_r, int32_t n_mu, const double *mu_edges,
                            int32_t n_ell, const int32_t *ells, double *out) {
  if (!xi || !mu_edges || !ells || !out || n_r < 1 || n_mu < 1 || n_ell < 1) return CUTE_E_INVALID;
  if (mu_edges[0] != 0.0 || mu_edges[n_mu] != 1.0) return CUTE_E_INVALID;
  for (int k = 0; k < n_mu; k++)
    if (!(mu_edges[k + 1] > mu_edges[k])) return CUTE_E_INVALID;
  int lmax = 0;
  for (int q = 0; q < n_ell; q++) {
    if (ells[q] < 0 || ells[q] > 16 || (ells[q] & 1)) return CUTE_E_INVALID;
    lmax = ells[q] > lmax ? ells[q] : lmax;
  }
  // weights c[q][k]: (2l + 1) times the integral of P_l over mu bin k
  std::vector<double> P0(lmax + 2), P1(lmax + 2), c((size_t)n_ell * n_mu);
  for (int k = 0; k < n_mu; k++) {
    legendre_all(mu_edges[k], lmax + 1, P0.data());
    legendre_all(mu_edges[k + 1], lmax + 1, P1.data());
    for (int q = 0; q < n_ell; q++) {
      const int l = ells[q];
      c[(size_t)q * n_mu + k] = l == 0 ? mu_edges[k + 1] - mu_edges[k]
                                       : (P1[l + 1] - P1[l - 1]) - (P0[l + 1] - P0[l - 1]);
    }
  }
  for (int q = 0; q < n_ell; q++)
    for (int i = 0; i < n_r; i++) {
      double s = 0.0;
      for (int k = 0; k < n_mu; k++) s += xi[(size_t)i * n_mu + k] * c[(size_t)q * n_mu + k];
      out[(size_t)q * n_r + i] = s;
    }
  return CUTE_OK;
}

cute_status cute_estimator_weighted(cute_estimator_kind k, const double *DD, const double *DR,
                                    const double *RR, double s_d, double q_d, double s_r,
                                    double q_r, int32_t nbins, double *xi_out) {
  if (!DD || !RR || !xi_out || nbins < 1) return CUTE_E_INVALID;
  if (k != CUTE_EST_NATURAL && k != CUTE_EST_LS) return CUTE_E_INVALID;
  const double ndd = 0.5 * (s_d * s_d - q_d), nrr = 0.5 * (s_r * s_r - q_r), ndr = s_d * s_r;
  if (!(ndd > 0) || !(nrr > 0) || !(ndr > 0)) return CUTE_E_INVALID;
  if (k == CUTE_EST_LS && !DR) return CUTE_E_INVALID;
  for (int b = 0; b < nbins; b++) {
    const double rr = RR[b] / nrr;
    if (!(RR[b] != 0.0)) {
      xi_out[b] = NAN;
    } else if (k == CUTE_EST_NATURAL) {  // Eq. 14
      xi_out[b] = (DD[b] / ndd) / rr - 1.0;
    } else {  // Eq. 15
      xi_out[b] = (DD[b] / ndd - 2.0 * (DR[b] / ndr) + rr) / rr;
    }
  }
  return CUTE_OK;
}

}  // extern "C"
