// Host-side contour arithmetic: the trapezoid rule of Eq. 7, the scalar rational
// function it defines, the extreme eigenvalues of a Lanczos tridiagonal matrix and
// the choice of ellipse from spectral bounds.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ov_internal.h"

// Eq. 7: theta_j = 2 pi (j - 1/2) / n_q, z_j = gamma + rho (cos + i alpha sin),
// w_j = alpha cos + i sin; P_Gamma ~ (1/n_q) sum_j rho w_j (z_j - H)^-1.
void ellipse_rule(int n_q, double gamma, double rho, double alpha, int form, std::vector<double2>& z,
                  std::vector<double2>& c, double2& c0) {
  z.clear();
  c.clear();
  const int ncont = (form == OV_CONTOUR_PAIR) ? 2 : 1;
  for (int k = 0; k < ncont; ++k) {
    const double centre = (k == 0) ? gamma : -gamma;
    // single contour: 2 P - 1; pair: + P_{Gamma+} - P_{Gamma-}
    const double scale = (form == OV_CONTOUR_PAIR) ? (k == 0 ? 1.0 : -1.0) : 2.0;
    for (int j = 1; j <= n_q; ++j) {
      const double th = 2.0 * M_PI * (j - 0.5) / n_q;
      const double ct = std::cos(th), sn = std::sin(th);
      z.push_back(make_double2(centre + rho * ct, rho * alpha * sn));
      c.push_back(make_double2(scale * rho * alpha * ct / n_q, scale * rho * sn / n_q));
    }
  }
  c0 = make_double2(form == OV_CONTOUR_PAIR ? 0.0 : -1.0, 0.0);
}

// Re r_N(lambda) = Re [c0 + sum_j c_j / (z_j - lambda)] for real lambda.
double rational_value(double lam, const std::vector<double2>& z, const std::vector<double2>& c, double2 c0) {
  double re = c0.x;
  for (size_t j = 0; j < z.size(); ++j) {
    const double dr = z[j].x - lam, di = z[j].y;
    const double den = dr * dr + di * di;
    re += (c[j].x * dr + c[j].y * di) / den;
  }
  return re;
}

namespace {

// Number of eigenvalues of the symmetric tridiagonal (a, b) smaller than x (Sturm count).
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  const int k = (int)a.size();
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < k; ++i) {
    const double qq = (q == 0.0) ? 1e-300 : q;
    q = a[i] - x - b[i - 1] * b[i - 1] / qq;
    if (q < 0) ++cnt;
  }
  return cnt;
}

double kth_eig(const std::vector<double>& a, const std::vector<double>& b, int idx, double lo, double hi) {
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(a, b, mid) > idx)
      hi = mid;
    else
      lo = mid;
    if (hi - lo <= 1e-15 * std::max(1.0, std::fabs(mid))) break;
  }
  return 0.5 * (lo + hi);
}

// |last component| of the normalised eigenvector of (a, b) for eigenvalue th (inverse iteration).
double last_component(const std::vector<double>& a, const std::vector<double>& b, double th) {
  const int k = (int)a.size();
  std::vector<double> v(k, 1.0), dd(k), ee(k), y(k);
  const double shift = th + 1e-10 * std::max(1.0, std::fabs(th));
  for (int rep = 0; rep < 3; ++rep) {
    // solve (T - shift) y = v by Gaussian elimination without pivoting (Thomas)
    dd[0] = a[0] - shift;
    y[0] = v[0];
    for (int i = 1; i < k; ++i) {
      const double m = b[i - 1] / (dd[i - 1] == 0.0 ? 1e-300 : dd[i - 1]);
      dd[i] = a[i] - shift - m * b[i - 1];
      y[i] = v[i] - m * y[i - 1];
    }
    v[k - 1] = y[k - 1] / (dd[k - 1] == 0.0 ? 1e-300 : dd[k - 1]);
    for (int i = k - 2; i >= 0; --i) v[i] = (y[i] - b[i] * v[i + 1]) / (dd[i] == 0.0 ? 1e-300 : dd[i]);
    double nrm = 0.0;
    for (double x : v) nrm += x * x;
    nrm = std::sqrt(nrm);
    for (double& x : v) x /= nrm;
  }
  return std::fabs(v[k - 1]);
}

}  // namespace

// Extreme Ritz values of the k x k tridiagonal with diagonal a[0..k) and
// off-diagonals b[0..k-1); b[k-1] is the next Lanczos coefficient beta_k, used for
// the Ritz residual bounds beta_k |s_k| (lo_resid, hi_resid).
void tridiag_extreme_eigs(const std::vector<double>& a, const std::vector<double>& b, double* lo, double* hi,
                          double* lo_resid, double* hi_resid) {
  const int k = (int)a.size();
  double gl = a[0], gh = a[0];
  for (int i = 0; i < k; ++i) {
    const double rad = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < k - 1 ? std::fabs(b[i]) : 0.0);
    gl = std::min(gl, a[i] - rad);
    gh = std::max(gh, a[i] + rad);
  }
  std::vector<double> bb(b.begin(), b.begin() + std::max(0, k - 1));
  *lo = kth_eig(a, bb, 0, gl - 1.0, gh + 1.0);
  *hi = kth_eig(a, bb, k - 1, gl - 1.0, gh + 1.0);
  const double bk = (int)b.size() >= k ? std::fabs(b[k - 1]) : 0.0;
  *lo_resid = bk * last_component(a, bb, *lo);
  *hi_resid = bk * last_component(a, bb, *hi);
}
