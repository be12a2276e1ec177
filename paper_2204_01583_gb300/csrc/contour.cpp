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

// ------------------------------------------------------------ Zolotarev node set
// Complete elliptic integral K(m) = pi / (2 AGM(1, sqrt(1 - m))) and the Jacobi elliptic
// functions sn, cn of parameter m by the arithmetic-geometric-mean scheme (descending
// Landen transformation; Abramowitz & Stegun 16.4 and 17.6), in double precision.
double ellip_K(double m) {
  double a = 1.0, b = std::sqrt(1.0 - m);
  for (int it = 0; it < 64 && std::fabs(a - b) > 1e-16 * a; ++it) {
    const double an = 0.5 * (a + b);
    b = std::sqrt(a * b);
    a = an;
  }
  return M_PI / (2.0 * a);
}

void ellip_sn_cn(double u, double m, double* sn, double* cn) {
  double a[40], c[40];
  a[0] = 1.0;
  double b = std::sqrt(1.0 - m);
  c[0] = std::sqrt(m);
  int n = 0;
  while (n < 38 && std::fabs(c[n]) > 1e-17) {
    a[n + 1] = 0.5 * (a[n] + b);
    c[n + 1] = 0.5 * (a[n] - b);
    b = std::sqrt(a[n] * b);
    ++n;
  }
  double phi = std::ldexp(a[n] * u, n);  // 2^n a_n u
  for (int k = n; k > 0; --k) {
    const double q = std::max(-1.0, std::min(1.0, c[k] * std::sin(phi) / a[k]));
    phi = 0.5 * (phi + std::asin(q));
  }
  *sn = std::sin(phi);
  *cn = std::cos(phi);
}

// Zolotarev's optimal rational approximation of sgn on [-lmax, -lmin] u [lmin, lmax] as a
// resolvent sum: with x = lambda / lmin, b = lmax / lmin, m' = 1 - 1/b^2, K' = K(m') and
// c_l = sn^2 / cn^2 (l K' / 2n | m'), the function
//   R(x) = d0 x prod_{i<n} (x^2 + c_{2i}) / prod_{i<=n} (x^2 + c_{2i-1}) = x sum_l b_l / (x^2 + c_{2l-1})
// equioscillates about 1 on [1, b] with amplitude delta for the right d0 (taken from the
// extreme values of R / d0, located on a log grid and refined by golden-section search).
// lambda / (lambda^2 + s^2) = -1/2 [1/(is - lambda) + 1/(-is - lambda)], so each pole pair
// gives nodes +-i s_l, s_l = lmin sqrt(c_{2l-1}), with coefficient -b_l lmin / 2.
int zolotarev_rule(int n, double lmin, double lmax, std::vector<double2>& z, std::vector<double2>& c, double2& c0,
                   double* delta) {
  if (n < 1 || n > 128 || !(lmin > 0.0) || !(lmax > lmin) || !std::isfinite(lmax)) return OV_ERR_INVALID_ARG;
  const double bb = lmax / lmin, m1 = 1.0 - 1.0 / (bb * bb), K1 = ellip_K(m1);
  std::vector<double> cl(2 * n);
  for (int l = 1; l < 2 * n; ++l) {
    double sn, cn;
    ellip_sn_cn(l * K1 / (2.0 * n), m1, &sn, &cn);
    cl[l] = (sn * sn) / (cn * cn);
  }
  auto Rt = [&](double x) {  // R / d0
    double r = x;
    for (int i = 1; i <= n; ++i) r /= (x * x + cl[2 * i - 1]);
    for (int i = 1; i < n; ++i) r *= (x * x + cl[2 * i]);
    return r;
  };
  // extreme values of R / d0 on [1, b]: endpoints and refined interior extrema
  const int M = 400 * n + 400;
  const double lb = std::log(bb);
  std::vector<double> v(M + 1);
  for (int k = 0; k <= M; ++k) v[k] = Rt(std::exp(lb * k / M));
  double lo = std::min(v[0], v[M]), hi = std::max(v[0], v[M]);
  for (int k = 1; k < M; ++k) {
    const bool mx = v[k] >= v[k - 1] && v[k] >= v[k + 1], mn = v[k] <= v[k - 1] && v[k] <= v[k + 1];
    if (!mx && !mn) continue;
    const double sg = mx ? 1.0 : -1.0;  // maximise sg * R
    double ta = lb * (k - 1) / M, tb = lb * (k + 1) / M;
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    double t1 = tb - gr * (tb - ta), t2 = ta + gr * (tb - ta);
    double f1 = sg * Rt(std::exp(t1)), f2 = sg * Rt(std::exp(t2));
    for (int it = 0; it < 80; ++it) {
      if (f1 > f2) {
        tb = t2; t2 = t1; f2 = f1; t1 = tb - gr * (tb - ta); f1 = sg * Rt(std::exp(t1));
      } else {
        ta = t1; t1 = t2; f1 = f2; t2 = ta + gr * (tb - ta); f2 = sg * Rt(std::exp(t2));
      }
    }
    const double best = std::max({sg * v[k], f1, f2}) * sg;
    lo = std::min(lo, best);
    hi = std::max(hi, best);
  }
  const double d0 = 2.0 / (lo + hi);
  if (delta) *delta = (hi - lo) / (hi + lo);
  std::vector<double> bl(n), s(n);
  for (int l = 1; l <= n; ++l) {
    const double co = cl[2 * l - 1];
    double num = d0, den = 1.0;
    for (int i = 1; i < n; ++i) num *= (cl[2 * i] - co);
    for (int i = 1; i <= n; ++i)
      if (i != l) den *= (cl[2 * i - 1] - co);
    bl[l - 1] = num / den;
    s[l - 1] = lmin * std::sqrt(co);
  }
  z.clear();
  c.clear();
  for (int l = 0; l < n; ++l) {
    z.push_back(make_double2(0.0, s[l]));
    c.push_back(make_double2(-0.5 * lmin * bl[l], 0.0));
  }
  for (int l = n - 1; l >= 0; --l) {
    z.push_back(make_double2(0.0, -s[l]));
    c.push_back(make_double2(-0.5 * lmin * bl[l], 0.0));
  }
  c0 = make_double2(0.0, 0.0);
  return OV_OK;
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
