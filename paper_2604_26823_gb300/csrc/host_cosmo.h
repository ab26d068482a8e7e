// Host FP64 cosmology coefficients used to build a plan (no GPU code).
#pragma once
#include <array>
#include <vector>

namespace pmhost {

struct GrowthPoint {
  double D1, D2, Gp1, Gp2;  // growth factors and a^3 E dD/da
};

struct Schedule {
  std::vector<double> a;   // n_steps + 1 scale factors
  std::vector<double> Ka;  // first half-kick factor of step k
  std::vector<double> Kb;  // second half-kick factor of step k
  std::vector<double> Dr;  // drift factor of step k
  GrowthPoint lpt;         // growth at a_init
  double e_final;          // E(a = 1)
};

double efunc(double a, double om);
void growth(double om, int n, const double *a, GrowthPoint *out);
Schedule leapfrog(double om, double a_init, int n_steps);
double eh98_nowiggle(double k, double om, double ob, double h, double tcmb);
void power_table(double om, double ob, double h, double sigma8, double ns, double kmin, double kmax,
                 int nk, double *lnk, double *lnp);
// Comoving distance table of the lightcone: chi_j = (c/H0) int_{a_j}^1 da / (a^2 E)
// (Mpc/h) on the uniform grid a_j = a_min + j (1 - a_min)/(n - 1), j = 0..n-1.
constexpr double kCOverH0 = 2997.92458;  // Mpc/h
void distance_table(double om, double a_min, int n, double *a, double *chi);

}  // namespace pmhost
