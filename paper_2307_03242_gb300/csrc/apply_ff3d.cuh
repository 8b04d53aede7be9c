// FP64 operator apply of the outer solve (3D), evaluated in double-FP32 arithmetic.
//
// Section 5.3: the 3D beta-spread derivative (Eq. dxSkew3D, with 1/h) spreads a difference along
// axis e over the two other axes with the weights W(a, b) = beta [a = b = 0] + (1-beta)/16
// [1 2 1]_a [1 2 1]_b; the mass spreads to the 6 neighbours with (1-beta)/6 (Eq. massHO3D). The
// row of u_c at face q expands to a 27-point sum
//   sum_delta C(delta) u_c(q + delta),  C(delta) = sum_e part_e(delta_e) W(delta_t1(e), delta_t2(e)),
// with part_e = (-mu_a, mu_a + mu_b, -mu_b): mu_a, mu_b the mu of the two derivative points beside
// q along e -- cell centres for e = c, edge centres (mean of 4 cells, A_e) for e != c. FP64
// coefficients are precomputed on the host as float-float pairs: cell mu, 1/(lambda+mu), edge mu
// for the three edge orientations, and the complex face masses of the unshifted operator.
#pragma once
#include "apply_ff2d.cuh"

namespace ff3 {

using df::f2;
using ff2::c2;
using ff2::cacc;
using ff2::ld;
using ff2::mul;
using ff2::add;
using ff2::fneg;
constexpr int BX = 32, BY = 4, BZ = 2;

struct FineFF3 {
  int nx, ny, nz;
  f2 ih, ih2, beta, sm, alpha;
  f2 W[3][3];          // W[a+1][b+1]
  const f2* mu;        // cells
  const f2* cp;        // cells
  const f2* edge[3];   // edge[r]: edges parallel to axis r, lattice (nx+1)(ny+1)(nz+1)
  const c2* m[3];      // face masses of u_c, cells
};

HD size_t lat(const FineFF3& g, int i, int j, int k) { return ((size_t)k * (g.ny + 1) + j) * (g.nx + 1) + i; }
HD size_t lin(const FineFF3& g, int i, int j, int k) { return ((size_t)k * g.ny + j) * g.nx + i; }

template <typename TI>
HD void cell_rows(const FineFF3& g, const cx<TI>* x, const cx<double>* b, double bscale, cx<double>* y, int i, int j,
                  int k) {
  const int n[3] = {g.nx, g.ny, g.nz};
  const int q[3] = {i, j, k};
  const size_t N = (size_t)g.nx * g.ny * g.nz, kq = lin(g, i, j, k);
  auto inside = [&](int a, int bb, int c) { return a >= 0 && a < g.nx && bb >= 0 && bb < g.ny && c >= 0 && c < g.nz; };
  auto mclamp = [&](int a, int bb, int c) {
    return g.mu[lin(g, iclamp(a, 0, g.nx - 1), iclamp(bb, 0, g.ny - 1), iclamp(c, 0, g.nz - 1))];
  };
  auto mshift = [&](c2 m) {
    if (g.alpha.hi != 0.f) m.im = add(m.im, fneg(mul(g.alpha, m.re)));
    return m;
  };
  cx<double> out[4];
  for (int c = 0; c < 3; ++c) {
    cacc r;
    if (q[c] >= 1) {
      // part_e for the three derivative axes
      f2 part[3][3];
      for (int e = 0; e < 3; ++e) {
        f2 ma, mb;
        int s[3] = {0, 0, 0};
        s[e] = 1;
        if (e == c) {
          ma = mclamp(i - s[0], j - s[1], k - s[2]);
          mb = mclamp(i, j, k);
        } else {
          const int rr = 3 - c - e;
          ma = g.edge[rr][lat(g, i, j, k)];
          mb = g.edge[rr][lat(g, i + s[0], j + s[1], k + s[2])];
        }
        part[e][0] = fneg(ma);
        part[e][1] = add(ma, mb);
        part[e][2] = fneg(mb);
      }
      const cx<TI>* u = x + c * N;
      for (int dk = -1; dk <= 1; ++dk)
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) {
            const int a = i + di, bb = j + dj, cc = k + dk;
            const int qa[3] = {a, bb, cc};
            if (!inside(a, bb, cc) || qa[c] < 1) continue;
            const int dl[3] = {di, dj, dk};
            f2 C = {0.f, 0.f};
            for (int e = 0; e < 3; ++e) {
              const int t1 = (e + 1) % 3, t2 = (e + 2) % 3;
              C = add(C, mul(part[e][dl[e] + 1], g.W[dl[t1] + 1][dl[t2] + 1]));
            }
            C = mul(g.ih2, C);
            const cx<TI> uv = u[lin(g, a, bb, cc)];
            const f2 ur = ld(uv.re), ui = ld(uv.im);
            r.rterm(C, ur, ui);
            const int nz0 = (di != 0) + (dj != 0) + (dk != 0);
            if (nz0 <= 1) {
              const c2 m = mshift(g.m[c][lin(g, a, bb, cc)]);
              const f2 f = nz0 == 0 ? g.beta : g.sm;
              r.cterm({fneg(mul(f, m.re)), fneg(mul(f, m.im))}, ur, ui);
            }
          }
      int s[3] = {0, 0, 0};
      s[c] = 1;
      const cx<TI>* p = x + 3 * N;
      const cx<TI> pc = p[kq], pm = p[lin(g, i - s[0], j - s[1], k - s[2])];
      r.rterm(g.ih, ld(pc.re), ld(pc.im));
      r.rterm(fneg(g.ih), ld(pm.re), ld(pm.im));
      out[c] = mkc<double>(r.re.to_double(), r.im.to_double());
    } else {
      out[c] = czero<double>();
    }
  }
  {
    cacc r;
    for (int c = 0; c < 3; ++c) {
      const int t1 = (c + 1) % 3, t2 = (c + 2) % 3;
      const cx<TI>* u = x + c * N;
      for (int a = -1; a <= 1; ++a)
        for (int bb = -1; bb <= 1; ++bb) {
          int o[3] = {0, 0, 0};
          o[t1] = a;
          o[t2] = bb;
          const f2 wgt = mul(g.ih, g.W[a + 1][bb + 1]);
          // + u_c(q + s_c + o), - u_c(q + o)
          int hi[3] = {i + o[0], j + o[1], k + o[2]};
          int lo[3] = {hi[0], hi[1], hi[2]};
          hi[c] += 1;
          if (inside(hi[0], hi[1], hi[2]) && hi[c] >= 1) {
            const cx<TI> uv = u[lin(g, hi[0], hi[1], hi[2])];
            r.rterm(wgt, ld(uv.re), ld(uv.im));
          }
          if (inside(lo[0], lo[1], lo[2]) && lo[c] >= 1) {
            const cx<TI> uv = u[lin(g, lo[0], lo[1], lo[2])];
            r.rterm(fneg(wgt), ld(uv.re), ld(uv.im));
          }
        }
    }
    const cx<TI> pc = x[3 * N + kq];
    r.rterm(g.cp[kq], ld(pc.re), ld(pc.im));
    out[3] = mkc<double>(r.re.to_double(), r.im.to_double());
  }
  for (int c = 0; c < 4; ++c) {
    cx<double> v = out[c];
    if (b) v = (c < 3 && q[c] < 1) ? czero<double>() : bscale * b[c * N + kq] - v;
    y[c * N + kq] = v;
  }
  (void)n;
}

template <typename TI>
__global__ void __launch_bounds__(BX * BY * BZ) apply(FineFF3 g, const cx<TI>* __restrict__ x,
                                                     const cx<double>* __restrict__ b, double bscale,
                                                     cx<double>* __restrict__ y) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z * BZ + threadIdx.z;
  if (i >= g.nx || j >= g.ny || k >= g.nz) return;
  cell_rows(g, x, b, bscale, y, i, j, k);
}

}  // namespace ff3
