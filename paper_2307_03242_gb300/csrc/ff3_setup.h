// Host precomputation of the float-float coefficient arrays of the 3D FP64 apply (apply_ff3d.cuh).
#pragma once
#include <algorithm>
#include <vector>

#include "apply_ff3d.cuh"

namespace ff3 {

inline f2 to_f2(double v) {
  f2 r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

struct HostFF3 {
  std::vector<f2> mu, cp, edge[3];
  std::vector<c2> m[3];
};

// lam, mu, rho: FP64 cell arrays (x fastest); h: cell size; abl: absorbing layer thickness
// (physical, 0 = none) and gamma at the boundary; L: domain lengths; gamma: attenuation.
inline void build_host(HostFF3& o, int nx, int ny, int nz, double h, const double* lam, const double* mu,
                       const double* rho, double omega, double gamma, double ablL, double ablG, const double L[3]) {
  const size_t N = (size_t)nx * ny * nz, NL = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  auto lin = [&](int i, int j, int k) { return ((size_t)k * ny + j) * nx + i; };
  auto M = [&](const double* f, int i, int j, int k) {
    return f[lin(std::min(std::max(i, 0), nx - 1), std::min(std::max(j, 0), ny - 1), std::min(std::max(k, 0), nz - 1))];
  };
  auto abl = [&](double x, double y, double z) {
    if (ablL <= 0.0) return 0.0;
    return ablG * (abl_axis(x, ablL, L[0]) + abl_axis(y, ablL, L[1]) + abl_axis(z, ablL, L[2])) / (ablL * ablL);
  };
  o.mu.resize(N);
  o.cp.resize(N);
  for (int c = 0; c < 3; ++c) {
    o.m[c].resize(N);
    o.edge[c].assign(NL, {0.f, 0.f});
  }
  const double w2 = omega * omega;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t q = lin(i, j, k);
        o.mu[q] = to_f2(mu[q]);
        o.cp[q] = to_f2(1.0 / (lam[q] + mu[q]));
        for (int c = 0; c < 3; ++c) {
          const int s[3] = {c == 0, c == 1, c == 2};
          const double a = 0.5 * (M(rho, i - s[0], j - s[1], k - s[2]) + M(rho, i, j, k)) * w2;
          const double g = gamma + abl((i + (c == 0 ? 0.0 : 0.5)) * h, (j + (c == 1 ? 0.0 : 0.5)) * h,
                                       (k + (c == 2 ? 0.0 : 0.5)) * h);
          o.m[c][q] = {to_f2(a), to_f2(-a * g)};
        }
      }
  // edge mu: edges parallel to axis r sit at integer positions along the two other axes
  for (int r = 0; r < 3; ++r) {
    const int c = (r + 1) % 3, e = (r + 2) % 3;
    const int sc[3] = {c == 0, c == 1, c == 2}, se[3] = {e == 0, e == 1, e == 2};
    for (int k = 0; k <= nz; ++k)
      for (int j = 0; j <= ny; ++j)
        for (int i = 0; i <= nx; ++i) {
          const double v = 0.25 * (M(mu, i, j, k) + M(mu, i - sc[0], j - sc[1], k - sc[2]) +
                                   M(mu, i - se[0], j - se[1], k - se[2]) +
                                   M(mu, i - sc[0] - se[0], j - sc[1] - se[1], k - sc[2] - se[2]));
          o.edge[r][((size_t)k * (ny + 1) + j) * (nx + 1) + i] = to_f2(v);
        }
  }
}

inline FineFF3 make(const HostFF3& o, const f2* mu, const f2* cp, const f2* const edge[3], const c2* const m[3], int nx,
                    int ny, int nz, double h, double beta, double alpha) {
  FineFF3 g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.ih = to_f2(1.0 / h);
  g.ih2 = to_f2(1.0 / (h * h));
  g.beta = to_f2(beta);
  g.sm = to_f2((1.0 - beta) / 6.0);
  g.kap = to_f2((1.0 - beta) / 16.0);
  g.alpha = to_f2(alpha);
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b) {
      const double wa = a == 0 ? 2.0 : 1.0, wb = b == 0 ? 2.0 : 1.0;
      g.W[a + 1][b + 1] = to_f2((a == 0 && b == 0 ? beta : 0.0) + (1.0 - beta) * wa * wb / 16.0);
    }
  g.mu = mu;
  g.cp = cp;
  for (int r = 0; r < 3; ++r) {
    g.edge[r] = edge[r];
    g.m[r] = m[r];
  }
  (void)o;
  return g;
}

}  // namespace ff3
