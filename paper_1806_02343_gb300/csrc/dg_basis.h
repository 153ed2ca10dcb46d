// Host-side generation of the DG basis and quadrature tables in double precision.
//
// Legendre products P_k, |k| <= d (Sec. 3.2, eq. legendre-3d), mode order: total
// degree, then k1 descending, then k2 descending; l_k(1) = 1.
// LDF vector basis of degree <= d (Sec. 3.3, App. A.2): curls of Legendre-product
// potentials of degree 1..d+1 (2D: stream function; 3D: x-, then y-, then
// z-directed potentials), stable-sorted by degree, unnormalised Gram-Schmidt under
// the L2 product of eq. innerp; N_div = D n(d) - n(d-1) (eq. dimVdiv).
// Gauss-Legendre rules from Newton iteration on l_n (Sec. 3.5).
#pragma once
#include <array>
#include <vector>

namespace dgmhd {

// Polynomial in D <= 3 variables as dense coefficients over monomials of total
// degree <= maxdeg; the monomial list is shared by a Basis.
struct MonoSet {
  int D = 3, maxdeg = 0;
  std::vector<std::array<int, 3>> exps;
  int index(int a, int b, int c) const;
  std::vector<int> lut;  // (maxdeg+1)^3 -> index or -1
  void build(int D_, int maxdeg_);
};

struct Basis {
  int D = 3, d = 0;
  int n = 0;     // Legendre modes n(d)
  int ndiv = 0;  // LDF vectors N_div
  std::vector<std::array<int, 3>> modes;
  MonoSet ms;                                    // monomials of degree <= d+1
  std::vector<std::vector<double>> leg;          // [mode][mono]
  std::vector<std::array<std::vector<double>, 3>> ldf;  // [j][comp][mono]
  std::vector<int> ldf_deg;
  std::vector<double> leg_mass, ldf_mass;

  bool build(int D_, int d_, bool with_ldf);
  double eval(const std::vector<double>& poly, const double* x) const;
  double eval_deriv(const std::vector<double>& poly, int axis, const double* x) const;
};

// n-point Gauss-Legendre nodes (ascending) and weights on [-1, 1].
void gauss_legendre(int npts, std::vector<double>& x, std::vector<double>& w);

int n_modes(int D, int d);

}  // namespace dgmhd
