// Host precomputation of the float-float coefficient arrays of the 2D FP64 apply (apply_ff2d.cuh):
// cell mu, 1/(lambda+mu), node mu (the mean of the four cells around a node, clamped at the
// boundary; A_e of Sec. 3.1) and the complex face masses m_f = rho_f omega^2 (1 - i (gamma +
// gamma_ABL(x_f))) of the unshifted operator.
#pragma once
#include <algorithm>
#include <vector>

#include "apply_ff2d.cuh"

namespace ff2 {

inline f2 to_f2(double v) {
  f2 r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

struct HostFF2 {
  std::vector<f2> mu, cp, mun;
  std::vector<c2> m1, m2;
};

// lam, mu, rho: FP64 cell arrays (x fastest); h: cell size; ablL, ablG: absorbing layer thickness
// (physical, 0 = none) and gamma at the boundary; Lx, Ly: domain lengths; gamma: attenuation.
inline void build_host(HostFF2& o, int nx, int ny, double h, const double* lam, const double* mu, const double* rho,
                       double omega, double gamma, double ablL, double ablG, double Lx, double Ly) {
  const size_t N = (size_t)nx * ny;
  auto M = [&](const double* f, int i, int j) {
    return f[(size_t)std::min(std::max(j, 0), ny - 1) * nx + std::min(std::max(i, 0), nx - 1)];
  };
  auto abl = [&](double x, double y) {
    if (ablL <= 0.0) return 0.0;
    return ablG * (abl_axis(x, ablL, Lx) + abl_axis(y, ablL, Ly)) / (ablL * ablL);
  };
  o.mu.resize(N);
  o.cp.resize(N);
  o.m1.resize(N);
  o.m2.resize(N);
  o.mun.resize((size_t)(nx + 1) * (ny + 1));
  const double w2 = omega * omega;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const size_t k = (size_t)j * nx + i;
      o.mu[k] = to_f2(mu[k]);
      o.cp[k] = to_f2(1.0 / (lam[k] + mu[k]));
      const double a1 = 0.5 * (M(rho, i - 1, j) + M(rho, i, j)) * w2;
      const double g1 = gamma + abl(i * h, (j + 0.5) * h);
      o.m1[k] = {to_f2(a1), to_f2(-a1 * g1)};
      const double a2 = 0.5 * (M(rho, i, j - 1) + M(rho, i, j)) * w2;
      const double g2 = gamma + abl((i + 0.5) * h, j * h);
      o.m2[k] = {to_f2(a2), to_f2(-a2 * g2)};
    }
  for (int Y = 0; Y <= ny; ++Y)
    for (int X = 0; X <= nx; ++X)
      o.mun[(size_t)Y * (nx + 1) + X] =
          to_f2(0.25 * (M(mu, X - 1, Y - 1) + M(mu, X, Y - 1) + M(mu, X - 1, Y) + M(mu, X, Y)));
}

// The kernel's descriptor for the arrays of o (host or device copies), the operator's shift.
inline FineFF make(const f2* mu, const f2* mun, const f2* cp, const c2* m1, const c2* m2, int nx, int ny, double h,
                   double beta, double alpha) {
  FineFF g;
  g.nx = nx;
  g.ny = ny;
  g.ih = to_f2(1.0 / h);
  g.ih2 = to_f2(1.0 / (h * h));
  g.t0 = to_f2(0.5 * (1.0 + beta));
  g.t1 = to_f2(0.25 * (1.0 - beta));
  g.ht2[0] = g.ht2[2] = to_f2(0.25 * (1.0 - beta) / (h * h));
  g.ht2[1] = to_f2(0.5 * (1.0 + beta) / (h * h));
  g.ht1[0] = g.ht1[2] = to_f2(0.25 * (1.0 - beta) / h);
  g.ht1[1] = to_f2(0.5 * (1.0 + beta) / h);
  g.beta = to_f2(beta);
  g.sm = to_f2(0.25 * (1.0 - beta));
  g.alpha = to_f2(alpha);
  g.mu = mu;
  g.mun = mun;
  g.cp = cp;
  g.m1 = m1;
  g.m2 = m2;
  return g;
}

}  // namespace ff2
