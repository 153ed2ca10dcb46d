// Host basis generation (double precision). See dg_basis.h for the conventions.
#include "dg_basis.h"

#include <algorithm>
#include <cmath>

namespace dgmhd {

int n_modes(int D, int d) {
  if (d < 0) return 0;
  if (D == 2) return (d + 1) * (d + 2) / 2;
  return (d + 1) * (d + 2) * (d + 3) / 6;
}

void MonoSet::build(int D_, int maxdeg_) {
  D = D_;
  maxdeg = maxdeg_;
  exps.clear();
  int m = maxdeg + 1;
  lut.assign(m * m * m, -1);
  for (int deg = 0; deg <= maxdeg; ++deg)
    for (int a = deg; a >= 0; --a)
      for (int b = deg - a; b >= 0; --b) {
        int c = deg - a - b;
        if (D == 2 && c != 0) continue;
        lut[(a * m + b) * m + c] = (int)exps.size();
        exps.push_back({a, b, c});
      }
}

int MonoSet::index(int a, int b, int c) const {
  int m = maxdeg + 1;
  if (a < 0 || b < 0 || c < 0 || a > maxdeg || b > maxdeg || c > maxdeg) return -1;
  return lut[(a * m + b) * m + c];
}

// 1D Legendre coefficients by Bonnet's recurrence.
static std::vector<double> legendre1d(int k) {
  std::vector<double> p0{1.0}, p1{0.0, 1.0};
  if (k == 0) return p0;
  for (int j = 1; j < k; ++j) {
    std::vector<double> p2(j + 2, 0.0);
    for (int i = 0; i <= j; ++i) p2[i + 1] += (2.0 * j + 1.0) / (j + 1.0) * p1[i];
    for (int i = 0; i < j; ++i) p2[i] -= (double)j / (j + 1.0) * p0[i];
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

static double mono_int1d(int k) { return (k & 1) ? 0.0 : 2.0 / (k + 1.0); }

using Poly = std::vector<double>;
using VPoly = std::array<Poly, 3>;

static Poly poly_deriv(const MonoSet& ms, const Poly& p, int axis) {
  Poly out(ms.exps.size(), 0.0);
  for (size_t i = 0; i < ms.exps.size(); ++i) {
    if (p[i] == 0.0) continue;
    auto e = ms.exps[i];
    if (e[axis] == 0) continue;
    double c = p[i] * e[axis];
    e[axis] -= 1;
    out[ms.index(e[0], e[1], e[2])] += c;
  }
  return out;
}

static double poly_dot(const MonoSet& ms, const Poly& a, const Poly& b) {
  double s = 0.0;
  for (size_t i = 0; i < ms.exps.size(); ++i) {
    if (a[i] == 0.0) continue;
    for (size_t j = 0; j < ms.exps.size(); ++j) {
      if (b[j] == 0.0) continue;
      const auto& ei = ms.exps[i];
      const auto& ej = ms.exps[j];
      double v = 1.0;
      for (int ax = 0; ax < ms.D; ++ax) v *= mono_int1d(ei[ax] + ej[ax]);
      s += a[i] * b[j] * v;
    }
  }
  return s;
}

static int poly_degree(const MonoSet& ms, const Poly& p) {
  int deg = -1;
  for (size_t i = 0; i < ms.exps.size(); ++i)
    if (p[i] != 0.0) deg = std::max(deg, ms.exps[i][0] + ms.exps[i][1] + ms.exps[i][2]);
  return deg;
}

bool Basis::build(int D_, int d_, bool with_ldf) {
  D = D_;
  d = d_;
  n = n_modes(D, d);
  ms.build(D, d + 1);
  const size_t nm = ms.exps.size();
  // Legendre products of degree <= d+1 (potentials) in mode order
  std::vector<std::array<int, 3>> all;
  for (int deg = 0; deg <= d + 1; ++deg)
    for (int a = deg; a >= 0; --a)
      for (int b = deg - a; b >= 0; --b) {
        int c = deg - a - b;
        if (D == 2 && c != 0) continue;
        all.push_back({a, b, c});
      }
  auto product = [&](const std::array<int, 3>& k) {
    Poly p(nm, 0.0);
    auto la = legendre1d(k[0]), lb = legendre1d(k[1]), lc = legendre1d(k[2]);
    for (size_t i = 0; i < la.size(); ++i)
      for (size_t j = 0; j < lb.size(); ++j)
        for (size_t l = 0; l < lc.size(); ++l) {
          double c = la[i] * lb[j] * lc[l];
          if (c != 0.0) p[ms.index((int)i, (int)j, (int)l)] += c;
        }
    return p;
  };
  modes.clear();
  leg.clear();
  leg_mass.clear();
  for (auto& k : all) {
    if (k[0] + k[1] + k[2] > d) break;
    modes.push_back(k);
    leg.push_back(product(k));
    double m = 1.0;
    for (int ax = 0; ax < D; ++ax) m *= 2.0 / (2.0 * k[ax] + 1.0);
    leg_mass.push_back(m);
  }
  if ((int)modes.size() != n) return false;
  ldf.clear();
  ldf_deg.clear();
  ldf_mass.clear();
  ndiv = 0;
  if (!with_ldf) return true;
  const int target = D * n_modes(D, d) - n_modes(D, d - 1);
  // pool of curls, each tagged with its degree, in pool order
  std::vector<std::pair<int, VPoly>> pool;
  std::vector<std::array<int, 3>> pots;
  for (auto& k : all)
    if (k[0] + k[1] + k[2] >= 1) pots.push_back(k);
  Poly zero(nm, 0.0);
  auto push = [&](VPoly v) {
    int deg = -1;
    for (int c = 0; c < D; ++c) deg = std::max(deg, poly_degree(ms, v[c]));
    if (deg >= 0) pool.push_back({deg, v});
  };
  if (D == 2) {
    for (auto& k : pots) {
      Poly Q = product(k);
      Poly dy = poly_deriv(ms, Q, 1), dx = poly_deriv(ms, Q, 0);
      for (auto& c : dx) c = -c;
      push({dy, dx, zero});
    }
  } else {
    for (int dir = 0; dir < 3; ++dir)
      for (auto& k : pots) {
        Poly Q = product(k);
        VPoly v{zero, zero, zero};
        if (dir == 0) {  // (Q,0,0) -> (0, dQ/dz, -dQ/dy)
          v[1] = poly_deriv(ms, Q, 2);
          v[2] = poly_deriv(ms, Q, 1);
          for (auto& c : v[2]) c = -c;
        } else if (dir == 1) {  // (0,Q,0) -> (-dQ/dz, 0, dQ/dx)
          v[0] = poly_deriv(ms, Q, 2);
          for (auto& c : v[0]) c = -c;
          v[2] = poly_deriv(ms, Q, 0);
        } else {  // (0,0,Q) -> (dQ/dy, -dQ/dx, 0)
          v[0] = poly_deriv(ms, Q, 1);
          v[1] = poly_deriv(ms, Q, 0);
          for (auto& c : v[1]) c = -c;
        }
        push(v);
      }
  }
  std::stable_sort(pool.begin(), pool.end(),
                   [](const std::pair<int, VPoly>& a, const std::pair<int, VPoly>& b) {
                     return a.first < b.first;
                   });
  auto vdot = [&](const VPoly& a, const VPoly& b) {
    double s = 0.0;
    for (int c = 0; c < D; ++c) s += poly_dot(ms, a[c], b[c]);
    return s;
  };
  for (auto& pv : pool) {
    if ((int)ldf.size() == target) break;
    VPoly r = pv.second;
    double n0 = vdot(r, r);
    // modified Gram-Schmidt against the accepted vectors
    for (size_t j = 0; j < ldf.size(); ++j) {
      double c = vdot(r, ldf[j]) / ldf_mass[j];
      if (c != 0.0)
        for (int comp = 0; comp < D; ++comp)
          for (size_t i = 0; i < nm; ++i) r[comp][i] -= c * ldf[j][comp][i];
    }
    double nr = vdot(r, r);
    if (nr <= 1e-20 * n0) continue;  // linearly dependent on earlier curls
    // clean round-off dust so that exact zeros stay zero
    for (int comp = 0; comp < D; ++comp)
      for (size_t i = 0; i < nm; ++i)
        if (std::fabs(r[comp][i]) < 1e-13) r[comp][i] = 0.0;
    ldf.push_back(r);
    ldf_mass.push_back(vdot(r, r));
    ldf_deg.push_back(pv.first);
  }
  ndiv = (int)ldf.size();
  return ndiv == target;
}

double Basis::eval(const Poly& p, const double* x) const {
  double s = 0.0;
  for (size_t i = 0; i < ms.exps.size(); ++i) {
    if (p[i] == 0.0) continue;
    double t = p[i];
    for (int ax = 0; ax < D; ++ax)
      for (int e = 0; e < ms.exps[i][ax]; ++e) t *= x[ax];
    s += t;
  }
  return s;
}

double Basis::eval_deriv(const Poly& p, int axis, const double* x) const {
  return eval(poly_deriv(ms, p, axis), x);
}

void gauss_legendre(int npts, std::vector<double>& x, std::vector<double>& w) {
  x.assign(npts, 0.0);
  w.assign(npts, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < npts; ++i) {
    double z = std::cos(pi * (i + 0.75) / (npts + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < npts; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (npts == 1) { p1 = z; p0 = 1.0; }
      dp = npts * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged root
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < npts; ++k) {
      double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    if (npts == 1) { p1 = z; p0 = 1.0; }
    dp = npts * (z * p1 - p0) / (z * z - 1.0);
    x[npts - 1 - i] = z;
    w[npts - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace dgmhd

// ------------------------------------------------------------------ C ABI

#include "../../include/dg_mhd.h"

extern "C" int dg_mhd_basis_values(int dim, int degree, int divB_scheme, int64_t npts, const double* xi,
                                   int64_t cap, double* out, int* n_rows, int* n_vars) {
  if (!n_rows || !n_vars || (dim != 2 && dim != 3) || degree < 0 || degree > 3 ||
      (divB_scheme != DG_DIVB_POWELL && divB_scheme != DG_DIVB_GLM) || npts < 0 || npts > (1 << 24) ||
      (npts > 0 && !xi))
    return DG_E_ARG;
  const bool glm = divB_scheme == DG_DIVB_GLM;
  dgmhd::Basis B;
  if (!B.build(dim, degree, !glm)) return DG_E_ARG;
  const int n = B.n, V = glm ? 9 : 8;
  const int R = glm ? 9 * n : 5 * n + B.ndiv + (dim == 2 ? n : 0);
  *n_rows = R;
  *n_vars = V;
  if (!out) return DG_OK;  // size query
  if (cap < (int64_t)R * V * npts) return DG_E_ARG;
  std::fill(out, out + (int64_t)R * V * npts, 0.0);
  auto at = [&](int r, int v, int64_t p) -> double& { return out[((int64_t)r * V + v) * npts + p]; };
  for (int64_t p = 0; p < npts; ++p) {
    double x[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < dim; ++a) x[a] = xi[p * dim + a];
    std::vector<double> leg(n);
    for (int l = 0; l < n; ++l) leg[l] = B.eval(B.leg[l], x);
    const int nleg = glm ? 9 : 5;  // variables carried by Legendre rows in row order
    for (int v = 0; v < nleg; ++v)
      for (int l = 0; l < n; ++l) at(v * n + l, v, p) = leg[l];
    if (!glm) {
      for (int j = 0; j < B.ndiv; ++j)
        for (int c = 0; c < dim; ++c) at(5 * n + j, 5 + c, p) = B.eval(B.ldf[j][c], x);
      if (dim == 2)
        for (int l = 0; l < n; ++l) at(5 * n + B.ndiv + l, 7, p) = leg[l];
    }
  }
  return DG_OK;
}
