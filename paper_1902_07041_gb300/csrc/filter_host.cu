// Host-side mathematics of the filter: Chebyshev coefficients of the piecewise quadratic
// target (eq. (fct_f)) and of the characteristic function, evaluated with the closed-form
// integrals of App. A; damping factors (Sec. 2.3); the degree criterion (eq. (thresh)); and
// the top eigenpair of the small Lanczos tridiagonal matrix.  All FP64, all tiny.
#include <cmath>

#include "pfe_internal.h"

namespace pfe {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// Integral of T_n(x) / sqrt(1 - x^2) over [lo, hi] within [-1, 1]: with x = cos(t) it is the
// integral of cos(n t) over t in [acos(hi), acos(lo)].
double weighted_integral_T(int64_t n, double t_lo, double t_hi) {
  if (n == 0) return t_hi - t_lo;
  const double dn = (double)n;
  return (std::sin(dn * t_hi) - std::sin(dn * t_lo)) / dn;
}

// One quadratic piece P(x) = c0 + c1 x + c2 x^2 on [lo, hi]: write P = a0 T_0 + a1 T_1 + a2 T_2
// (x = T_1, x^2 = (T_0 + T_2)/2) and integrate T_l T_j with 2 T_l T_j = T_{l+j} + T_{|l-j|}.
void add_piece(double c0, double c1, double c2, double lo, double hi, int32_t m, std::vector<double> &acc) {
  lo = std::max(lo, -1.0);
  hi = std::min(hi, 1.0);
  if (!(lo < hi)) return;
  const double t_lo = std::acos(hi), t_hi = std::acos(lo);
  const double a[3] = {c0 + 0.5 * c2, c1, 0.5 * c2};
  for (int32_t j = 0; j <= m; ++j) {
    double s = 0.0;
    for (int l = 0; l < 3; ++l) {
      if (a[l] == 0.0) continue;
      if (l == 0) {
        s += a[0] * weighted_integral_T(j, t_lo, t_hi);
      } else {
        const int64_t sum = (int64_t)l + j, dif = std::llabs((int64_t)l - j);
        s += a[l] * 0.5 * (weighted_integral_T(sum, t_lo, t_hi) + weighted_integral_T(dif, t_lo, t_hi));
      }
    }
    acc[j] += s;
  }
}

}  // namespace

void pq_coefficients(double xi, double eta, double eps, int32_t m, std::vector<double> &gamma) {
  gamma.assign((size_t)m + 1, 0.0);
  const double ie2 = 1.0 / (eps * eps);
  // rising flank (x - (xi - eps))^2 / eps^2 on [xi - eps, xi]
  const double l = xi - eps;
  add_piece(l * l * ie2, -2.0 * l * ie2, ie2, xi - eps, xi, m, gamma);
  // plateau 1 + ((eta - xi)^2 - (2x - xi - eta)^2) / (2 eps (eta - xi)) on [xi, eta]
  const double w = eta - xi, s = xi + eta, k = 1.0 / (2.0 * eps * w);
  add_piece(1.0 + (w * w - s * s) * k, 4.0 * s * k, -4.0 * k, xi, eta, m, gamma);
  // falling flank (x - (eta + eps))^2 / eps^2 on [eta, eta + eps]
  const double r = eta + eps;
  add_piece(r * r * ie2, -2.0 * r * ie2, ie2, eta, eta + eps, m, gamma);
  // divide by <T_j, T_j> = pi (j = 0), pi/2 (j > 0)
  for (int32_t j = 0; j <= m; ++j) gamma[j] *= (j == 0) ? 1.0 / kPi : 2.0 / kPi;
}

void chi_coefficients(double xi, double eta, int32_t m, std::vector<double> &gamma) {
  gamma.assign((size_t)m + 1, 0.0);
  add_piece(1.0, 0.0, 0.0, xi, eta, m, gamma);
  for (int32_t j = 0; j <= m; ++j) gamma[j] *= (j == 0) ? 1.0 / kPi : 2.0 / kPi;
}

void damping_factors(int kind, int32_t m, std::vector<double> &g) {
  g.assign((size_t)m + 1, 1.0);
  if (kind == 1) {  // Jackson, alpha = pi / (m + 2)
    const double al = kPi / (m + 2.0), cot = std::cos(al) / std::sin(al);
    for (int32_t j = 0; j <= m; ++j)
      g[j] = (1.0 - j / (m + 2.0)) * std::cos(j * al) + cot * std::sin(j * al) / (m + 2.0);
  } else if (kind == 2) {  // Lanczos sigma factors, theta = pi / (m + 1)
    const double th = kPi / (m + 1.0);
    for (int32_t j = 1; j <= m; ++j) g[j] = std::sin(j * th) / (j * th);
  }
}

double chebyshev_value(const std::vector<double> &c, int32_t m, double x) {
  double t0 = 1.0, t1 = x, v = c[0];
  if (m >= 1) v += c[1] * x;
  for (int32_t j = 2; j <= m; ++j) {
    const double t2 = 2.0 * x * t1 - t0;
    v += c[j] * t2;
    t0 = t1;
    t1 = t2;
  }
  return v;
}

int32_t choose_degree(double xi, double eta, double eps, double r, int kind, int32_t kmax) {
  std::vector<double> gamma;
  pq_coefficients(xi, eta, eps, kmax, gamma);
  // T_j at the four test points, tabulated once by the recurrence
  const double pts[4] = {xi - eps, eta + eps, xi, eta};
  std::vector<double> T[4];
  for (int p = 0; p < 4; ++p) {
    T[p].resize((size_t)kmax + 1);
    T[p][0] = 1.0;
    if (kmax >= 1) T[p][1] = pts[p];
    for (int32_t j = 2; j <= kmax; ++j) T[p][j] = 2.0 * pts[p] * T[p][j - 1] - T[p][j - 2];
  }
  std::vector<double> g;
  for (int32_t k = 1; k <= kmax; ++k) {
    damping_factors(kind, k, g);
    double v[4] = {0, 0, 0, 0};
    for (int32_t j = 0; j <= k; ++j) {
      const double c = g[j] * gamma[j];
      for (int p = 0; p < 4; ++p) v[p] += c * T[p][j];
    }
    if (std::max(v[0], v[1]) <= r * std::min(v[2], v[3])) return k;
  }
  return -1;
}

// ---- the Dirac filter of eq. (cheby-delta.1): rho(x) = sum_j g_j T_j(gamma) T_j(x) / <T_j, T_j>
void dirac_coefficients(double gamma, int32_t m, int kind, std::vector<double> &c) {
  damping_factors(kind, m, c);
  // T_j(gamma) by the three-term recurrence
  double t0 = 1.0, t1 = gamma;
  for (int32_t j = 0; j <= m; ++j) {
    double tj;
    if (j == 0) tj = 1.0;
    else if (j == 1) tj = gamma;
    else {
      tj = 2.0 * gamma * t1 - t0;
      t0 = t1;
      t1 = tj;
    }
    c[j] *= tj * ((j == 0) ? 1.0 / kPi : 2.0 / kPi);
  }
}

// The centre gamma in (xi, eta) with rho(xi) = rho(eta).  rho_gamma(xi) - rho_gamma(eta) is the
// Chebyshev series sum_j d_j T_j(gamma) with d_j = g_j w_j (T_j(xi) - T_j(eta)); it is positive
// while gamma lies too close to xi.  Its sign change in (xi, eta) is found by bisection.
double dirac_center(double xi, double eta, int32_t m, int kind) {
  std::vector<double> d;
  damping_factors(kind, m, d);
  double a0 = 1.0, a1 = xi, b0 = 1.0, b1 = eta;
  for (int32_t j = 0; j <= m; ++j) {
    double ta, tb;
    if (j == 0) {
      ta = tb = 1.0;
    } else if (j == 1) {
      ta = xi;
      tb = eta;
    } else {
      ta = 2.0 * xi * a1 - a0;
      a0 = a1;
      a1 = ta;
      tb = 2.0 * eta * b1 - b0;
      b0 = b1;
      b1 = tb;
    }
    d[j] *= (ta - tb) * ((j == 0) ? 1.0 / kPi : 2.0 / kPi);
  }
  double lo = xi, hi = eta;
  for (int it = 0; it < 80 && hi - lo > 1e-17; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (chebyshev_value(d, m, mid) > 0.0) lo = mid;
    else hi = mid;
  }
  return 0.5 * (lo + hi);
}

namespace {
// rho(xi) / rho(gamma) of the balanced degree-m filter
double dirac_edge_ratio(double xi, double eta, int32_t m, int kind) {
  const double g = dirac_center(xi, eta, m, kind);
  std::vector<double> c((size_t)m + 1);
  dirac_coefficients(g, m, kind, c);
  return chebyshev_value(c, m, xi) / chebyshev_value(c, m, g);
}
}  // namespace

int32_t choose_dirac_degree(double xi, double eta, double phi, int kind, int32_t kmax) {
  // the edge ratio falls with the degree: bracket by doubling, bisect, then step down while the
  // next lower degree still qualifies
  int32_t hi = 2;
  while (hi <= kmax && dirac_edge_ratio(xi, eta, hi, kind) > phi) hi *= 2;
  if (hi > kmax) {
    hi = kmax;
    if (dirac_edge_ratio(xi, eta, hi, kind) > phi) return -1;
  }
  int32_t lo = std::max(2, hi / 2);  // lo fails (or is the start), hi qualifies
  if (lo == hi || dirac_edge_ratio(xi, eta, lo, kind) <= phi) {
    hi = lo;
  } else {
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) / 2;
      if (dirac_edge_ratio(xi, eta, mid, kind) <= phi) hi = mid;
      else lo = mid;
    }
  }
  while (hi > 2 && dirac_edge_ratio(xi, eta, hi - 1, kind) <= phi) --hi;
  return hi;
}

void tridiag_top(const std::vector<double> &alpha, const std::vector<double> &beta, double *theta, double *last) {
  const int n = (int)alpha.size();
  // Gershgorin bounds
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(beta[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(beta[i]) : 0.0);
    lo = std::min(lo, alpha[i] - r);
    hi = std::max(hi, alpha[i] + r);
  }
  auto below = [&](double x) {  // number of eigenvalues < x (Sturm sequence)
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < n; ++i) {
      q = alpha[i] - x - (i > 0 ? beta[i - 1] * beta[i - 1] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  // largest eigenvalue: smallest x with below(x) == n
  double a = lo - 1e-12 * std::fabs(lo) - 1e-300, b = hi + 1e-12 * std::fabs(hi) + 1e-300;
  for (int it = 0; it < 300 && b - a > 1e-15 * std::max(std::fabs(a), std::fabs(b)); ++it) {
    const double mid = 0.5 * (a + b);
    if (below(mid) >= n) b = mid;
    else a = mid;
  }
  const double th = 0.5 * (a + b);
  *theta = th;
  // inverse iteration with (T - (th + delta) I), negative definite: LU without pivoting is stable
  const double shift = th + 1e-10 * std::max(std::fabs(th), 1e-300);
  std::vector<double> z((size_t)n, 1.0), dd((size_t)n), ll((size_t)n);
  for (int i = 0; i < n; ++i) {
    dd[i] = alpha[i] - shift - (i > 0 ? beta[i - 1] * ll[i - 1] : 0.0);
    if (dd[i] == 0.0) dd[i] = -1e-300;
    if (i + 1 < n) ll[i] = beta[i] / dd[i];
  }
  for (int it = 0; it < 4; ++it) {
    for (int i = 1; i < n; ++i) z[i] -= ll[i - 1] * z[i - 1];  // L y = z
    z[n - 1] /= dd[n - 1];
    for (int i = n - 2; i >= 0; --i) z[i] = (z[i] - beta[i] * z[i + 1]) / dd[i];  // D L^T x = y
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) nrm += z[i] * z[i];
    nrm = std::sqrt(nrm);
    for (int i = 0; i < n; ++i) z[i] /= nrm;
  }
  *last = z[n - 1];
}

// Largest |p(x)| outside the margin window [xi - eps, eta + eps] over the smallest p(x) in [xi, eta],
// for p = sum c_j T_j: the factor by which one filter application shrinks the components a subspace
// holding the window does not capture (eq. (thresh) bounds it at the two margin points only).  The
// outside is sampled in theta = arccos x with a step of pi / (6 m), fine enough for the oscillations
// of a degree-m series; the inside at 65 points including both edges.
double filter_ratio(const std::vector<double> &c, int32_t m, double xi, double eta, double eps) {
  const double kPi = 3.14159265358979323846;
  const double lo = std::max(-1.0, xi - eps), hi = std::min(1.0, eta + eps);
  double out = 0.0;
  const double h = kPi / (6.0 * std::max(m, 1));
  const double th_hi = std::acos(hi), th_lo = std::acos(lo);  // x in [hi, 1] <-> theta in [0, th_hi]
  for (double th = 0.0; th <= th_hi; th += h) out = std::max(out, std::fabs(chebyshev_value(c, m, std::cos(th))));
  if (hi < 1.0) out = std::max(out, std::fabs(chebyshev_value(c, m, hi)));
  for (double th = th_lo; th <= kPi; th += h) out = std::max(out, std::fabs(chebyshev_value(c, m, std::cos(th))));
  if (lo > -1.0) out = std::max(out, std::fabs(chebyshev_value(c, m, lo)));
  double in = 1e300;
  for (int i = 0; i <= 64; ++i) in = std::min(in, chebyshev_value(c, m, xi + (eta - xi) * i / 64.0));
  return in > 0.0 ? out / in : 1e300;
}

// The degree in [m0, 4 m0] (steps of 5 %) that minimises the modelled work of the subspace iteration:
// iterations log(tol) / log(ratio(m)) times the work of one, m filter steps plus the dense steps, the
// latter as dense_steps equivalent filter steps (work of CholQR2, Rayleigh-Ritz and locking over the
// work of one filter step on the block).  m0 when no candidate beats it.
int32_t choose_degree_cost(double xi, double eta, double eps, int kind, int32_t m0, double tol, double dense_steps) {
  if (m0 < 1 || !(tol > 0.0 && tol < 1.0)) return m0;
  int32_t best = m0;
  double best_cost = 1e300;
  std::vector<double> gam, g, c;
  for (int32_t m = m0; m <= 4 * m0 && m <= 60000; m = std::max(m + 1, (int32_t)std::lround(m * 1.05))) {
    pq_coefficients(xi, eta, eps, m, gam);
    damping_factors(kind, m, g);
    c.resize((size_t)m + 1);
    for (int32_t j = 0; j <= m; ++j) c[j] = gam[j] * g[j];
    const double r = filter_ratio(c, m, xi, eta, eps);
    if (!(r > 0.0 && r < 1.0)) continue;
    const double cost = std::log(tol) / std::log(r) * ((double)m + dense_steps);
    if (cost < best_cost) {
      best_cost = cost;
      best = m;
    }
  }
  return best;
}

}  // namespace pfe

// ---- the filter design without a context (host only, callable without a GPU)
extern "C" pfe_status pfe_design_filter(int kind, double xi, double eta, double eps, double r, double phi, int damping,
                                        int32_t degree, int32_t cap, int32_t *m_out, double *coeffs) {
  using namespace pfe;
  // explicit degrees share the automatic search's limit of 60000
  if (!m_out || (kind != 0 && kind != 1) || (damping < 0 || damping > 2) || degree < 0 || degree > 60000)
    return PFE_E_ARG;
  if (!(xi >= -1.0 && xi < eta && eta <= 1.0)) return PFE_E_ARG;
  if (kind == 0 && !(eps > 0.0 && r > 0.0 && r < 1.0)) return PFE_E_ARG;
  if (kind == 1 && !(phi > 0.0 && phi < 1.0)) return PFE_E_ARG;
  int32_t m = degree;
  if (m == 0) {
    m = (kind == 0) ? choose_degree(xi, eta, eps, r, damping, 60000) : choose_dirac_degree(xi, eta, phi, damping, 60000);
    if (m < 0) return PFE_E_ARG;
  }
  *m_out = m;
  if (!coeffs) return PFE_OK;
  if ((int64_t)cap < (int64_t)m + 1) return PFE_E_CAPACITY;
  std::vector<double> c;
  if (kind == 0) {
    std::vector<double> gam, g;
    pq_coefficients(xi, eta, eps, m, gam);
    damping_factors(damping, m, g);
    c.resize((size_t)m + 1);
    for (int32_t j = 0; j <= m; ++j) c[j] = gam[j] * g[j];
  } else {
    c.resize((size_t)m + 1);
    dirac_coefficients(dirac_center(xi, eta, m, damping), m, damping, c);
  }
  std::copy(c.begin(), c.end(), coeffs);
  return PFE_OK;
}

