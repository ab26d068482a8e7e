// Host-side FP64 coefficients: E(a), growth factors D1 / D2 and their
// momentum growth, the FastPM leapfrog factors, and the linear power table.
//
// Sec. 2.2.1 item 1 (linear P(k) of the fiducial cosmology) and item 2 (2LPT
// initial condition, leapfrog PM steps of constant da).  Units: H0 = 1,
// Mpc/h, h/Mpc.
#include "host_cosmo.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace pmhost {

double efunc(double a, double om) { return std::sqrt(om / (a * a * a) + (1.0 - om)); }

// y = (D1, dD1/dln a, D2, dD2/dln a); in ln a the growth equations read
//   D'' + (2 - 1.5 Om(a)) D' = 1.5 Om(a) D            (linear)
//   D2'' + (2 - 1.5 Om(a)) D2' = 1.5 Om(a) (D2 - D1^2) (second order)
static void rhs(double lna, const double *y, double om, double *dy) {
  const double a = std::exp(lna);
  const double e2 = om / (a * a * a) + (1.0 - om);
  const double oma = om / (a * a * a) / e2;
  const double damp = 2.0 - 1.5 * oma;
  dy[0] = y[1];
  dy[1] = -damp * y[1] + 1.5 * oma * y[0];
  dy[2] = y[3];
  dy[3] = -damp * y[3] + 1.5 * oma * (y[2] - y[0] * y[0]);
}

void growth(double om, int n, const double *a_in, GrowthPoint *out) {
  // integrate once through the sorted scale factors (plus a = 1 for the
  // normalisation), from the Einstein-de Sitter growing mode at a = 1e-5
  std::vector<double> pts(a_in, a_in + n);
  pts.push_back(1.0);
  std::sort(pts.begin(), pts.end());
  pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
  const double a0 = 1e-5;
  const double steps_per_efold = 2000.0;
  double lna = std::log(a0);
  double y[4] = {a0, a0, -3.0 / 7.0 * a0 * a0, -6.0 / 7.0 * a0 * a0};
  std::vector<std::array<double, 4>> st(pts.size());
  for (size_t i = 0; i < pts.size(); ++i) {
    const double end = std::log(pts[i]);
    const int m = std::max(1, (int)std::ceil((end - lna) * steps_per_efold));
    const double h = (end - lna) / m;
    for (int s = 0; s < m; ++s) {
      double k1[4], k2[4], k3[4], k4[4], t[4];
      rhs(lna, y, om, k1);
      for (int j = 0; j < 4; ++j) t[j] = y[j] + 0.5 * h * k1[j];
      rhs(lna + 0.5 * h, t, om, k2);
      for (int j = 0; j < 4; ++j) t[j] = y[j] + 0.5 * h * k2[j];
      rhs(lna + 0.5 * h, t, om, k3);
      for (int j = 0; j < 4; ++j) t[j] = y[j] + h * k3[j];
      rhs(lna + h, t, om, k4);
      for (int j = 0; j < 4; ++j) y[j] += h / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
      lna += h;
    }
    lna = end;
    for (int j = 0; j < 4; ++j) st[i][j] = y[j];
  }
  const double norm = st.back()[0];  // a = 1 is the largest point
  for (int i = 0; i < n; ++i) {
    const size_t j = std::lower_bound(pts.begin(), pts.end(), a_in[i]) - pts.begin();
    const double a = a_in[i];
    const double e = efunc(a, om);
    const double d1 = st[j][0] / norm, u1 = st[j][1] / norm;
    const double d2 = st[j][2] / (norm * norm), u2 = st[j][3] / (norm * norm);
    out[i].D1 = d1;
    out[i].D2 = d2;
    out[i].Gp1 = a * a * e * u1;  // a^3 E dD/da = a^2 E dD/dln a
    out[i].Gp2 = a * a * e * u2;
  }
}

Schedule leapfrog(double om, double a_init, int n_steps) {
  // a_k = a_init + k da, midpoints a_{k+1/2}; FastPM factors
  //   kick  K(a->b; c) = [Gp(b) - Gp(a)] / Gf(c), Gf = 1.5 Om D1
  //   drift Dr(a->b; c) = [D1(b) - D1(a)] / Gp(c)
  Schedule sc;
  const double da = (1.0 - a_init) / n_steps;
  std::vector<double> a(n_steps + 1), ah(n_steps);
  for (int k = 0; k <= n_steps; ++k) a[k] = a_init + da * k;
  a[n_steps] = 1.0;
  for (int k = 0; k < n_steps; ++k) ah[k] = 0.5 * (a[k] + a[k + 1]);
  std::vector<GrowthPoint> ga(n_steps + 1), gh(n_steps);
  growth(om, n_steps + 1, a.data(), ga.data());
  growth(om, n_steps, ah.data(), gh.data());
  sc.a = a;
  sc.Ka.resize(n_steps);
  sc.Kb.resize(n_steps);
  sc.Dr.resize(n_steps);
  for (int k = 0; k < n_steps; ++k) {
    sc.Ka[k] = (gh[k].Gp1 - ga[k].Gp1) / (1.5 * om * ga[k].D1);
    sc.Kb[k] = (ga[k + 1].Gp1 - gh[k].Gp1) / (1.5 * om * ga[k + 1].D1);
    sc.Dr[k] = (ga[k + 1].D1 - ga[k].D1) / gh[k].Gp1;
  }
  sc.lpt = ga[0];
  sc.e_final = efunc(1.0, om);
  return sc;
}

// Eisenstein & Hu (1998) transfer function without baryon oscillations,
// k in h/Mpc (their Eqs. 26, 28-31).
double eh98_nowiggle(double k, double om, double ob, double h, double tcmb) {
  const double omh2 = om * h * h, obh2 = ob * h * h, fb = ob / om;
  const double theta = tcmb / 2.7;
  const double s = 44.5 * std::log(9.83 / omh2) / std::sqrt(1.0 + 10.0 * std::pow(obh2, 0.75));
  const double alpha = 1.0 - 0.328 * std::log(431.0 * omh2) * fb + 0.38 * std::log(22.3 * omh2) * fb * fb;
  const double ks = 0.43 * k * h * s;
  const double gamma = om * h * (alpha + (1.0 - alpha) / (1.0 + ks * ks * ks * ks));
  const double q = k * theta * theta / gamma;
  const double l0 = std::log(2.0 * M_E + 1.8 * q);
  const double c0 = 14.2 + 731.0 / (1.0 + 62.5 * q);
  return l0 / (l0 + c0 * q * q);
}

static double tophat(double x) {
  if (std::fabs(x) < 1e-3) return 1.0 - x * x / 10.0;
  return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}

void power_table(double om, double ob, double h, double sigma8, double ns, double kmin, double kmax,
                 int nk, double *lnk, double *lnp) {
  // sigma(8)^2 of the unnormalised shape k^ns T^2 by composite Simpson in ln k
  auto shape = [&](double k) {
    const double t = eh98_nowiggle(k, om, ob, h, 2.7255);
    return std::pow(k, ns) * t * t;
  };
  const double lo = std::log(1e-7), hi = std::log(1e3);
  const int m = 400000;
  const double dx = (hi - lo) / m;
  double acc = 0.0;
  for (int i = 0; i <= m; ++i) {
    const double k = std::exp(lo + dx * i);
    const double w = tophat(8.0 * k);
    const double f = k * k * k * shape(k) * w * w;
    acc += f * ((i == 0 || i == m) ? 1.0 : ((i & 1) ? 4.0 : 2.0));
  }
  const double sig2 = acc * dx / 3.0 / (2.0 * M_PI * M_PI);
  const double amp = sigma8 * sigma8 / sig2;
  const double l0 = std::log(kmin), l1 = std::log(kmax);
  for (int i = 0; i < nk; ++i) {
    const double lk = (nk == 1) ? l0 : l0 + (l1 - l0) * i / (nk - 1);
    lnk[i] = lk;
    lnp[i] = std::log(amp * shape(std::exp(lk)));
  }
}

void distance_table(double om, double a_min, int n, double *a, double *chi) {
  // 8-point Gauss-Legendre on each grid interval (the integrand is smooth on
  // [a_min, 1], so each interval's rule is exact to rounding), accumulated
  // from a = 1 downward
  static const double xg[4] = {0.18343464249564980494, 0.52553240991632898582, 0.79666647741362673959,
                               0.96028985649753623168};
  static const double wg[4] = {0.36268378337836198297, 0.31370664587788728734, 0.22238103445337447054,
                               0.10122853629037625915};
  const double da = (1.0 - a_min) / (n - 1);
  for (int j = 0; j < n; ++j) a[j] = j == n - 1 ? 1.0 : a_min + j * da;
  chi[n - 1] = 0.0;
  for (int j = n - 2; j >= 0; --j) {
    const double lo = a[j], hi = a[j + 1], mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
    double s = 0.0;
    for (int g = 0; g < 4; ++g) {
      for (int sg = -1; sg <= 1; sg += 2) {
        const double x = mid + sg * half * xg[g];
        s += wg[g] / (x * x * efunc(x, om));
      }
    }
    chi[j] = chi[j + 1] + kCOverH0 * half * s;
  }
}

}  // namespace pmhost
