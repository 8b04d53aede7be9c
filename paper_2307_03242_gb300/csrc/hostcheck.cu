// Host build of per-cell functions of the kernels, for CPU checks against the FP64 oracle: the
// same source the GPU kernels run (the adjoint rows and material derivative of adjoint.cuh; the
// 2D red-black half-sweep of vanka2d_fast.cuh and the residual and restriction of
// residual2d_fast.cuh, the 3D residual of residual3d.cuh, with the kernels' choice among their
// interior and attenuation-free variants; the 3D float-float FP64 apply of apply_ff3d.cuh on the
// library's host-built coefficients), looped over the cells on the host. Not part of the solve path;
// libemg_hostcheck.so holds no device code that runs.
#include <cmath>
#include <limits>
#include <vector>

#include "adjoint.cuh"
#include "adjoint_ff3.cuh"
#include "dfloat.cuh"
#include "ff2_setup.h"
#include "ff3_setup.h"
#include "residual2d_fast.cuh"
#include "residual3d.cuh"
#include "vanka3d_tile.cuh"
#include "sweep2d_tile.cuh"
#include "residual2d_tile.cuh"
#include "vanka2d_fast.cuh"
#include "kaczmarz.cuh"
#include "emg.h"

#include <algorithm>
#include <array>
#include <cstddef>

namespace {

Grid<double> host_grid(int dim, const int* n, double h, double beta, double omega, double att, double abl_len,
                       double abl_gmax, const double* mu, const double* rho, const double* cp) {
  Grid<double> g;
  g.nx = n[0];
  g.ny = n[1];
  g.nz = dim == 3 ? n[2] : 1;
  g.h = h;
  g.ih = 1.0 / h;
  g.beta = beta;
  g.sm = (1.0 - beta) / (2.0 * dim);
  g.w2 = omega * omega;
  g.att = att;
  g.ablL = abl_len;
  g.ablG = abl_gmax;
  g.Lx = n[0] * h;
  g.Ly = n[1] * h;
  g.Lz = dim == 3 ? n[2] * h : 0.0;
  g.mu = mu;
  g.rho = rho;
  g.cp = cp;
  g.abl_tab[0] = g.abl_tab[1] = g.abl_tab[2] = nullptr;
  return g;
}

template <int D>
void apply_all(const Grid<double>& g, const cx<double>* x, cx<double>* y) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const cx<double>* xs[4];
  for (int c = 0; c <= D; ++c) xs[c] = x + (size_t)c * N;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const size_t idx = adj::lin(g, i, j, k);
        for (int c = 0; c < D; ++c) y[(size_t)c * N + idx] = adj::row_u<D, double, double>(c, xs, g, i, j, k);
        y[(size_t)D * N + idx] = adj::row_p<D, double, double>(xs, g, i, j, k);
      }
}

template <int D>
void gradient_all(const Grid<double>& g, const cx<double>* u, const cx<double>* a, double* gl, double* gm, double* gr) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const cx<double>* us[4];
  const cx<double>* as[4];
  for (int c = 0; c <= D; ++c) {
    us[c] = u + (size_t)c * N;
    as[c] = a + (size_t)c * N;
  }
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const size_t idx = adj::lin(g, i, j, k);
        adj::gradient<D, double, double>(us, as, g, i, j, k, gl[idx], gm[idx], gr[idx]);
      }
}

// A 2D (D = 2) or 3D level as the library sets it up: material in precision T, the per-axis
// absorbing-layer tables at k h and (k + 1/2) h for k = -2 .. n + 2 and the attenuation-free
// lattice range.
template <typename T, int D = 2>
struct Level2 {
  Grid<T> g;
  std::vector<T> mu, rho, cp, tab[3];
  Level2(const int* n, double h, double beta, double omega, double att, double abl_len, double abl_gmax, double Lx,
         double Ly, const double* mu64, const double* rho64, const double* cp64, double Lz = 0.0) {
    const size_t N = (size_t)n[0] * n[1] * (D == 3 ? n[2] : 1);
    mu.assign(mu64, mu64 + N);
    rho.assign(rho64, rho64 + N);
    cp.assign(cp64, cp64 + N);
    g.nx = n[0];
    g.ny = n[1];
    g.nz = D == 3 ? n[2] : 1;
    g.h = (T)h;
    g.ih = (T)(1.0 / h);
    g.beta = (T)beta;
    g.sm = (T)((1.0 - beta) / (2.0 * D));
    g.w2 = (T)(omega * omega);
    g.att = (T)att;
    g.ablL = (T)abl_len;
    g.ablG = (T)abl_gmax;
    g.Lx = (T)Lx;
    g.Ly = (T)Ly;
    g.Lz = (T)Lz;
    g.mu = mu.data();
    g.rho = rho.data();
    g.cp = cp.data();
    g.abl_tab[2] = nullptr;
    const double X[3] = {Lx, Ly, Lz};
    for (int a = 0; a < D; ++a) {
      tab[a].assign(2 * (n[a] + 5), T(0));
      for (int k = -2; k <= n[a] + 2; ++k)
        for (int half = 0; half < 2; ++half) {
          const double x = (k + 0.5 * half) * h;
          tab[a][2 * (k + 2) + half] = (T)(abl_len > 0.0 ? abl_gmax * abl_axis(x, abl_len, X[a]) / (abl_len * abl_len) : 0.0);
        }
      auto zero_at = [&](int k) { return tab[a][2 * (k + 2)] == T(0) && tab[a][2 * (k + 2) + 1] == T(0); };
      int lo = n[a] / 2, hi = n[a] / 2 - 1;
      if (zero_at(n[a] / 2)) {
        lo = hi = n[a] / 2;
        while (lo > -2 && zero_at(lo - 1)) --lo;
        while (hi < n[a] + 2 && zero_at(hi + 1)) ++hi;
      }
      g.abl_tab[a] = tab[a].data();
      g.zlo[a] = lo;
      g.zhi[a] = hi;
    }
  }
};

template <typename T>
std::vector<cx<T>> to_cx(const double* v, size_t n) {
  std::vector<cx<T>> out(n);
  for (size_t k = 0; k < n; ++k) out[k] = mkc<T>((T)v[2 * k], (T)v[2 * k + 1]);
  return out;
}
template <typename T>
void from_cx(const std::vector<cx<T>>& v, double* out) {
  for (size_t k = 0; k < v.size(); ++k) {
    out[2 * k] = (double)v[k].re;
    out[2 * k + 1] = (double)v[k].im;
  }
}

// One red-black half-sweep of colour `colour` over every cell, choosing the variant as k2::vanka_fast does
template <typename T>
void half_sweep2(const Grid<T>& g, const cx<T>* b, const cx<T>* uin, cx<T>* uout, cx<T>* p, int colour, T w, int zin) {
  for (int j = 0; j < g.ny; ++j)
    for (int ip = 0; ip < (g.nx + 1) / 2; ++ip) {
      const int i = 2 * ip + ((colour + j) & 1);
      if (!zin && i >= 2 && i + 3 <= g.nx && j >= 2 && j + 3 <= g.ny) {
        if (g.abl_free(0, i - 1, i + 2) && g.abl_free(1, j - 1, j + 2))
          k2::vanka_cell<T, true, true>(g, b, uin, uout, p, colour, w, zin, ip, j);
        else
          k2::vanka_cell<T, true>(g, b, uin, uout, p, colour, w, zin, ip, j);
      } else {
        k2::vanka_cell<T, false>(g, b, uin, uout, p, colour, w, zin, ip, j);
      }
    }
}

// `sweeps` full sweeps with the library's buffer protocol: colour 0 reads x and writes the
// displacements into alt, colour 1 reads alt and writes them back into x; p is updated in place.
template <typename T>
void sweeps2(const Level2<T>& L, const double* b64, double* x64, double w, int sweeps, int zero_first) {
  const size_t N = (size_t)L.g.nx * L.g.ny;
  std::vector<cx<T>> b = to_cx<T>(b64, 3 * N), x = to_cx<T>(x64, 3 * N), alt(2 * N, czero<T>());
  cx<T>* p = x.data() + 2 * N;
  for (int s = 0; s < sweeps; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      const cx<T>* uin = colour == 0 ? x.data() : alt.data();
      cx<T>* uout = colour == 0 ? alt.data() : x.data();
      half_sweep2<T>(L.g, b.data(), uin, uout, p, colour, (T)w, (zero_first && s == 0 && colour == 0) ? 1 : 0);
    }
  from_cx(x, x64);
}

// r = b - H_s x with the variant choice of k2::residual_fast, then b_c = R r (k2::restrict_r)
template <typename T>
void residual_restrict2(const Level2<T>& L, const double* b64, const double* x64, double* bc64) {
  const int nx = L.g.nx, ny = L.g.ny, nxc = nx / 2, nyc = ny / 2;
  const size_t N = (size_t)nx * ny;
  std::vector<cx<T>> b = to_cx<T>(b64, 3 * N), x = to_cx<T>(x64, 3 * N), r(3 * N), bc(3 * (size_t)nxc * nyc);
  const Grid<T>& g = L.g;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      if (i >= 2 && i + 3 <= nx && j >= 2 && j + 3 <= ny) {
        if (g.abl_free(0, i - 1, i + 2) && g.abl_free(1, j - 1, j + 2))
          k2::residual_cell<T, true, true>(g, b.data(), x.data(), r.data(), i, j);
        else
          k2::residual_cell<T, true>(g, b.data(), x.data(), r.data(), i, j);
      } else {
        k2::residual_cell<T, false>(g, b.data(), x.data(), r.data(), i, j);
      }
    }
  for (int J = 0; J < nyc; ++J)
    for (int I = 0; I < nxc; ++I) k2::restrict_r_cell<T>(r.data(), bc.data(), nx, ny, nxc, nyc, I, J);
  from_cx(bc, bc64);
}

// r = b - H_s x in 3D with the variant choice of k3::residual (interior cells: the register
// cube, with or without the absorbing layer; cells next to the boundary: the reference rows)
template <typename T>
void residual3(const Level2<T, 3>& L, const double* b64, const double* x64, double* r64) {
  const Grid<T>& g = L.g;
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  std::vector<cx<T>> b = to_cx<T>(b64, 4 * N), x = to_cx<T>(x64, 4 * N), r(4 * N);
  const cx<T>* u[3] = {x.data(), x.data() + N, x.data() + 2 * N};
  const cx<T>* p = x.data() + 3 * N;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        if (i >= 2 && i + 3 <= g.nx && j >= 2 && j + 3 <= g.ny && k >= 2 && k + 3 <= g.nz) {
          if (g.abl_free(0, i - 1, i + 2) && g.abl_free(1, j - 1, j + 2) && g.abl_free(2, k - 1, k + 2))
            k3::residual_cell3<T, true>(g, b.data(), x.data(), r.data(), i, j, k);
          else
            k3::residual_cell3<T, false>(g, b.data(), x.data(), r.data(), i, j, k);
          continue;
        }
        const size_t q = s3::lin(g, i, j, k);
        const int idx[3] = {i, j, k};
        for (int c = 0; c < 3; ++c)
          r[c * N + q] = idx[c] >= 1 ? b[c * N + q] - s3::row_u(c, u[c], p, g, i, j, k) : czero<T>();
        r[3 * N + q] = b[3 * N + q] - s3::row_p(u, p, g, i, j, k);
      }
  from_cx(r, r64);
}

// 3D red-black Vanka sweeps with the shared-memory tile kernel (k3t::vanka_tile) on the host:
// per half-sweep every block's tile_load over its NT lanes, then its tile_compute over them, with
// the library's ping-pong of the displacements (colour 0 reads x and writes alt, colour 1 reads
// alt and writes x; p in place). Blocks run one after another, which gives the kernel's result
// because a half-sweep reads no value that another block writes in it. Needs n >= (16, 8, 4), the
// kernel's own condition; returns -1 otherwise.
template <typename T>
void sweeps3_tile(const Level2<T, 3>& L, const double* b64, double* x64, double w, int sweeps, int zero_first) {
  const Grid<T>& g = L.g;
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  std::vector<cx<T>> b = to_cx<T>(b64, 4 * N), x = to_cx<T>(x64, 4 * N), alt(4 * N, czero<T>());
  std::vector<k3t::Tile<T>> tile(1);
  cx<T>* p = x.data() + 3 * N;
  for (int s = 0; s < sweeps; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      const cx<T>* uin = colour == 0 ? x.data() : alt.data();
      cx<T>* uout = colour == 0 ? alt.data() : x.data();
      const int zin = (zero_first && s == 0 && colour == 0) ? 1 : 0;
      for (int z0 = 0; z0 < g.nz; z0 += k3t::TZ)
        for (int y0 = 0; y0 < g.ny; y0 += k3t::TY)
          for (int x0 = 0; x0 < g.nx; x0 += k3t::TX) {
            for (int t = 0; t < k3t::NT; ++t) k3t::tile_load(tile[0], g, b.data(), uin, p, zin, x0, y0, z0, t);
            for (int t = 0; t < k3t::NT; ++t) k3t::tile_compute(tile[0], g, uout, p, colour, (T)w, zin, x0, y0, z0, t);
          }
    }
  from_cx(x, x64);
}

// One full sweep of the one-pass tiled kernel (k2t::sweep_tile) on the host: the same tiles, the
// same shared-region contents (zeros outside the grid as the TMA copies give them, clamped
// material and zeroed boundary faces on boundary tiles) and the same colour-0 / colour-1 phases
// and lane mapping. Shared entries the kernel never writes before reading are poisoned with NaN
// (the colour-0 faces of interior tiles), so a read of one shows in the result.
template <int TYV>
void sweep_tiled(const Grid<float>& g, const cx<float>* b, const cx<float>* xin, cx<float>* xout, float w, int zero_in,
                 const cx<float>* e = nullptr, int nxc = 0, int nyc = 0) {
  using namespace k2t;
  using G = Geo<TYV>;
  constexpr int TY = G::TY, PLANE = G::PLANE, EX = G::EX, EPLANE = G::EPLANE;
  const size_t N = (size_t)g.nx * g.ny;
  const float nan = std::numeric_limits<float>::quiet_NaN();
  std::vector<cx<float>> U(3 * PLANE), V(2 * PLANE);
  std::vector<float> MU(PLANE), RHO(PLANE);
  const int tx = (g.nx + TX - 1) / TX, ty = (g.ny + TY - 1) / TY;
  for (int by = 0; by < ty; ++by)
    for (int bx = 0; bx < tx; ++bx) {
      const Tile t = tile_of<G>(g, bx, by);
      for (int q = 0; q < PLANE; ++q) {
        const int gx = t.x0 - HALO + q % DX, gy = t.y0 - HALO + q / DX;
        const bool in = gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny;
        const size_t k = (size_t)gy * g.nx + gx;
        for (int c = 0; c < 3; ++c) U[c * PLANE + q] = (in && !zero_in) ? xin[c * N + k] : czero<float>();
        MU[q] = in ? g.mu[k] : 0.f;
        RHO[q] = in ? g.rho[k] : 0.f;
      }
      if (e) {
        // the coarse box as the TMA copy gives it: zeros outside the coarse grid, NaN beyond the box
        for (auto& v : V) v = mkc<float>(nan, nan);
        const int ex0 = t.x0 / 2 - 4, ey0 = t.y0 / 2 - 3;
        const size_t Nc = (size_t)nxc * nyc;
        for (int c = 0; c < 3; ++c)
          for (int q = 0; q < EPLANE; ++q) {
            const int I = ex0 + q % EX, J = ey0 + q / EX;
            const bool in = I >= 0 && I < nxc && J >= 0 && J < nyc;
            V[c * EPLANE + q] = in ? e[c * Nc + (size_t)J * nxc + I] : czero<float>();
          }
        if (t.fast) add_prolonged<G, true>(g, t, U.data(), V.data(), nxc, nyc, 0, 1);
        else add_prolonged<G, false>(g, t, U.data(), V.data(), nxc, nyc, 0, 1);
      }
      for (auto& v : V) v = t.boundary ? czero<float>() : mkc<float>(nan, nan);
      if (t.boundary) fix_boundary<G>(g, t, U.data(), MU.data(), RHO.data(), 0, 1);
      View s{U.data(), U.data() + PLANE, U.data() + 2 * PLANE, MU.data(), RHO.data()};
      cx<float>* v1 = V.data();
      cx<float>* v2 = V.data() + PLANE;
      for (int patch = 0; patch < G::C0_PATCHES; ++patch)
        for (int lane = 0; lane < 32; ++lane) {
          int lx, ly;
          c0_pos(patch, lane, lx, ly);
          if (t.fast) {
            if (zero_in) relax_c0<true, true>(g, t, s, v1, v2, b, w, lx, ly);
            else relax_c0<true, false>(g, t, s, v1, v2, b, w, lx, ly);
          } else {
            if (zero_in) relax_c0<false, true>(g, t, s, v1, v2, b, w, lx, ly);
            else relax_c0<false, false>(g, t, s, v1, v2, b, w, lx, ly);
          }
        }
      const View s1{v1, v2, U.data() + 2 * PLANE, MU.data(), RHO.data()};
      for (int patch = 0; patch < G::C1_PATCHES; ++patch)
        for (int lane = 0; lane < 32; ++lane) {
          int lx, ly;
          if (!c1_pos(patch, lane, lx, ly)) continue;
          if (t.fast) relax_c1<true>(g, t, s1, b, xout, w, lx, ly);
          else relax_c1<false>(g, t, s1, b, xout, w, lx, ly);
        }
    }
}

// The one-pass residual + restriction (k2t::resid_restrict_tile) on the host: the same tiles,
// shared-region contents, phases and work order; unwritten shared entries are NaN.
template <int TYV>
void resid_restrict_tiled(const Grid<float>& g, const cx<float>* b, const cx<float>* x, cx<float>* bc, int nxc,
                          int nyc) {
  using namespace k2t;
  using G = Geo<TYV>;
  constexpr int TY = G::TY, PLANE = G::PLANE;
  const size_t N = (size_t)g.nx * g.ny;
  const float nan = std::numeric_limits<float>::quiet_NaN();
  std::vector<cx<float>> U(3 * PLANE), V(2 * PLANE);
  std::vector<float> MU(PLANE), RHO(PLANE);
  for (int by = 0; by < (g.ny + TY - 1) / TY; ++by)
    for (int bx = 0; bx < (g.nx + TX - 1) / TX; ++bx) {
      const Tile t = tile_of<G>(g, bx, by);
      for (int q = 0; q < PLANE; ++q) {
        const int gx = t.x0 - HALO + q % DX, gy = t.y0 - HALO + q / DX;
        const bool in = gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny;
        const size_t k = (size_t)gy * g.nx + gx;
        for (int c = 0; c < 3; ++c) U[c * PLANE + q] = in ? x[c * N + k] : czero<float>();
        MU[q] = in ? g.mu[k] : 0.f;
        RHO[q] = in ? g.rho[k] : 0.f;
      }
      for (auto& v : V) v = mkc<float>(nan, nan);
      if (t.boundary) fix_boundary<G>(g, t, U.data(), MU.data(), RHO.data(), 0, 1);
      const View s{U.data(), U.data() + PLANE, U.data() + 2 * PLANE, MU.data(), RHO.data()};
      constexpr int EW = TX + 1, EH = TY + 1;
      for (int q = 0; q < EW * EH; ++q) {
        const int lx = HALO - 1 + q % EW, ly = HALO - 1 + q / EW;
        if (t.noabl) resid_phase1<true>(g, t, s, V.data(), V.data() + PLANE, b, lx, ly);
        else resid_phase1<false>(g, t, s, V.data(), V.data() + PLANE, b, lx, ly);
      }
      for (int q = 0; q < (TX / 2) * (TY / 2); ++q)
        restrict_phase2(g, t, s, V.data(), V.data() + PLANE, b, bc, nxc, nyc, q % (TX / 2), q / (TX / 2));
    }
}

}  // namespace

namespace {

// H_s x of one level on the host, row by row as the level's apply kernels evaluate it.
template <int D>
void level_apply(const Grid<double>& g, const cx<double>* x, cx<double>* y) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const size_t q = kz::cell_of(std::array<int, 3>{g.nx, g.ny, g.nz}.data(), D, i, j, k);
        if (D == 3) {
          const cx<double>* u[3] = {x, x + N, x + 2 * N};
          const int idx[3] = {i, j, k};
          for (int c = 0; c < 3; ++c)
            y[c * N + q] = idx[c] >= 1 ? s3::row_u<double, double>(c, u[c], x + 3 * N, g, i, j, k) : czero<double>();
          y[3 * N + q] = s3::row_p<double, double>(u, x + 3 * N, g, i, j, k);
        } else {
          y[q] = i >= 1 ? s2::row_u1<double, double>(x, x + 2 * N, g, i, j) : czero<double>();
          y[N + q] = j >= 1 ? s2::row_u2<double, double>(x + N, x + 2 * N, g, i, j) : czero<double>();
          y[2 * N + q] = s2::row_p<double, double>(x, x + N, x + 2 * N, g, i, j);
        }
      }
}

// The Kaczmarz solve's set-up on the host: the Schur rows by probing the level operator.
template <int D>
void kz_probe_host(const Grid<double>& g, cx<double>* coef) {
  const int n[3] = {g.nx, g.ny, g.nz};
  const size_t N = (size_t)n[0] * n[1] * n[2];
  std::fill(coef, coef + (size_t)D * N * kz::Shape<D>::NE, czero<double>());
  std::vector<cx<double>> e((D + 1) * N), y((D + 1) * N);
  for (int c2 = 0; c2 < D; ++c2)
    for (int q2 = 0; q2 < (D == 3 ? kz::PER : 1); ++q2)
      for (int q1 = 0; q1 < kz::PER; ++q1)
        for (int q0 = 0; q0 < kz::PER; ++q0) {
          const int q[3] = {q0, q1, q2};
          for (size_t t = 0; t < e.size(); ++t) e[t] = kz::probe_value<double, D>(c2, q, n, t);
          level_apply<D>(g, e.data(), y.data());
          for (size_t r = 0; r < (size_t)D * N; ++r) kz::probe_take_row<double, D>(g, y.data(), c2, q, r, coef);
        }
}

// `steps` Kaczmarz steps (sweep of every box, then the component average) with the kernel's
// index tables and loop order, lanes taken one after another. Returns the number of region
// indices that fell outside a box's region or did not map back to the entry's unknown (0).
template <int D>
long kz_steps_host(const kz::Boxes& B, const cx<double>* coef, const cx<double>* rhs, cx<double>* x, int steps,
                   double w) {
  constexpr int NE = kz::Shape<D>::NE, SL = kz::Shape<D>::SL;
  const size_t N = (size_t)B.n[0] * B.n[1] * B.n[2];
  std::vector<kz::LaneTab<D>> tab(kz::HW);
  for (int lane = 0; lane < kz::HW; ++lane) tab[lane].init(B, lane);
  std::vector<double> in2((size_t)D * N);
  for (size_t r = 0; r < in2.size(); ++r) in2[r] = kz::inv_row_norm<double, D>(coef, r);
  std::vector<cx<double>> copies((size_t)B.nboxes * B.RS), reg(B.RS);
  long bad = 0;
  for (int s = 0; s < steps; ++s) {
    for (int bx = 0; bx < B.nboxes; ++bx) {
      int lo[3];
      kz::box_lo(B, bx, lo);
      // the region through the kernel's layout table (kz::region_code), checked against region_cell
      for (int t = 0; t < B.RS; ++t) {
        int m[3];
        const int c2 = kz::region_cell(B, t, lo, m);
        const int code = kz::region_code(B, t);
        const int cc = code & 3;
        const int mm[3] = {lo[0] - kz::reach_lo(cc, 0) + ((code >> 2) & 255), lo[1] - kz::reach_lo(cc, 1) + ((code >> 10) & 255),
                           D == 3 ? lo[2] - kz::reach_lo(cc, 2) + ((code >> 18) & 255) : 0};
        if (cc != c2 || mm[0] != m[0] || mm[1] != m[1] || mm[2] != m[2]) ++bad;
        bool in = true;
        for (int a = 0; a < D; ++a) in = in && m[a] >= 0 && m[a] < B.n[a];
        reg[t] = (in && m[c2] >= 1) ? x[(size_t)c2 * N + kz::cell_of(B.n, D, m[0], m[1], m[2])] : czero<double>();
      }
      // rows in the kernel's order: an odometer cursor (the boxes-of-2 and general variants)
      kz::Cursor cu, cu2;
      const int Q = D * B.box[0] * B.box[1] * B.box[2];
      const bool two = B.box[0] == 2 && B.box[1] == 2 && (D == 2 || B.box[2] == 2);
      const bool one = B.box[0] == 1 && B.box[1] == 1 && (D == 2 || B.box[2] == 1);
      kz::Cursor cu1;
      for (int q = 0; q < Q; ++q) {
        const int c = cu.c;
        const int lz = cu.l[2], ly = cu.l[1], lx = cu.l[0];
        const long long rr = kz::cursor_row<D>(B, cu, lo, (unsigned)N);
        cu.advance<D, 0>(B);
        if (two) {
          if (cu2.c != c || cu2.l[0] != lx || cu2.l[1] != ly || cu2.l[2] != lz) ++bad;
          cu2.advance<D, 2>(B);
        }
        if (one) {
          if (cu1.c != c || cu1.l[0] != lx || cu1.l[1] != ly || cu1.l[2] != lz) ++bad;
          cu1.advance<D, 1>(B);
        }
        {
              const int k[3] = {lo[0] + lx, lo[1] + ly, lo[2] + lz};
              const bool valid = !(k[0] >= B.n[0] || k[1] >= B.n[1] || k[2] >= B.n[2] || k[c] < 1);
              if (valid != (rr >= 0)) ++bad;
              if (!valid) continue;
              const size_t r = (size_t)c * N + kz::cell_of(B.n, D, k[0], k[1], k[2]);
              if ((long long)r != rr) ++bad;
              if (in2[r] == 0.0) continue;
              cx<double> dot = czero<double>();
              std::vector<int> idx(kz::HW * SL, -1);
              for (int lane = 0; lane < kz::HW; ++lane)
                for (int t = 0; t < SL; ++t) {
                  const int pk = tab[lane].get(c, t);
                  if (pk < 0) continue;
                  const int cc = kz::pk_c2(pk);
                  const int id = kz::pk_off(pk) + (lz * B.ry[cc] + ly) * B.rx[cc] + lx;
                  int m[3];
                  const bool ok = id >= 0 && id < B.RS && kz::region_cell(B, id, lo, m) == cc &&
                                  m[0] == k[0] + kz::pk_o(pk, 0) && m[1] == k[1] + kz::pk_o(pk, 1) &&
                                  m[2] == k[2] + kz::pk_o(pk, 2);
                  if (!ok) {
                    ++bad;
                    continue;
                  }
                  idx[lane * SL + t] = id;
                  dot = dot + coef[r * NE + lane + kz::HW * t] * reg[id];
                }
              const cx<double> sc = (w * in2[r]) * (rhs[r] - dot);
              for (int lane = 0; lane < kz::HW; ++lane)
                for (int t = 0; t < SL; ++t) {
                  const int id = idx[lane * SL + t];
                  if (id >= 0) reg[id] = reg[id] + sc * cconj(coef[r * NE + lane + kz::HW * t]);
                }
        }
      }
      std::copy(reg.begin(), reg.end(), copies.begin() + (size_t)bx * B.RS);
    }
    for (size_t q = 0; q < (size_t)D * N; ++q) {
      const int c2 = (int)(q / N);
      const size_t cell = q % N;
      const int m[3] = {(int)(cell % B.n[0]), (int)((cell / B.n[0]) % B.n[1]), (int)(cell / ((size_t)B.n[0] * B.n[1]))};
      if (m[c2] < 1) {
        x[q] = czero<double>();
        continue;
      }
      int blo[3], bhi[3];
      kz::reach_boxes(B, c2, m, blo, bhi);
      for (int a = 0; a < 3; ++a)
        if (bhi[a] - blo[a] > (B.box[a] == 1 ? 3 : 2)) ++bad;  // the kernel's candidates per axis
      cx<double> acc = czero<double>();
      int cnt = 0;
      for (int bz = blo[2]; bz <= bhi[2]; ++bz)
        for (int by = blo[1]; by <= bhi[1]; ++by)
          for (int bxx = blo[0]; bxx <= bhi[0]; ++bxx) {
            const int box = (bz * B.nb[1] + by) * B.nb[0] + bxx;
            const int loc = kz::reach_local(B, c2, m, bxx, by, bz);
            int lo[3], mm[3];
            kz::box_lo(B, box, lo);
            if (loc < 0 || loc >= B.RS || kz::region_cell(B, loc, lo, mm) != c2 || mm[0] != m[0] || mm[1] != m[1] ||
                mm[2] != m[2]) {
              ++bad;
              continue;
            }
            acc = acc + copies[(size_t)box * B.RS + loc];
            ++cnt;
          }
      x[q] = cnt ? mkc<double>(acc.re / cnt, acc.im / cnt) : czero<double>();
    }
  }
  return bad;
}

}  // namespace

extern "C" {

// Layout of emg_params as this compiler sees it: sizeof, then the offsets of dim, n, h, damping,
// coarse_solver, level_alpha, smoother, sweep_path, kaczmarz_box, kaczmarz_steps,
// kaczmarz_damping, coarse_tol, coarse_restart, kaczmarz_max.
int emg_hc_params_layout(long* out) {
  out[0] = sizeof(emg_params);
  out[1] = offsetof(emg_params, dim);
  out[2] = offsetof(emg_params, n);
  out[3] = offsetof(emg_params, h);
  out[4] = offsetof(emg_params, damping);
  out[5] = offsetof(emg_params, coarse_solver);
  out[6] = offsetof(emg_params, level_alpha);
  out[7] = offsetof(emg_params, smoother);
  out[8] = offsetof(emg_params, sweep_path);
  out[9] = offsetof(emg_params, kaczmarz_box);
  out[10] = offsetof(emg_params, kaczmarz_steps);
  out[11] = offsetof(emg_params, kaczmarz_damping);
  out[12] = offsetof(emg_params, coarse_tol);
  out[13] = offsetof(emg_params, coarse_restart);
  out[14] = offsetof(emg_params, kaczmarz_max);
  return 0;
}

// Entry of the Kaczmarz solve's stored Schur row of component c for the column of component c2
// at offsets o (-1: outside the footprint).
int emg_hc_kz_slot(int dim, int c, int c2, int o0, int o1, int o2) {
  const int o[3] = {o0, o1, o2};
  for (int a = 0; a < dim; ++a)
    if (o[a] < kz::foot_lo(c, c2, a) || o[a] > 1) return -1;
  if (dim == 2 && o2 != 0) return -1;
  return dim == 3 ? kz::slot_of<3>(c, c2, o) : kz::slot_of<2>(c, c2, o);
}

// Schur rows (complex128, dim N x NE) of one level by probing its operator (att = gamma + shift).
int emg_hc_kz_probe(int dim, const int* n, double h, double beta, double omega, double att, double abl_len,
                    double abl_gmax, double Lx, double Ly, double Lz, const double* mu, const double* rho,
                    const double* cp, double* coef) {
  if (dim == 3) {
    Level2<double, 3> L(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp, Lz);
    kz_probe_host<3>(L.g, (cx<double>*)coef);
  } else if (dim == 2) {
    Level2<double, 2> L(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp);
    kz_probe_host<2>(L.g, (cx<double>*)coef);
  } else {
    return -1;
  }
  return 0;
}

// `steps` parallel hybrid Kaczmarz steps for S x = rhs (complex128 vectors of dim N: the
// displacement components, boundary faces 0) from x, with boxes of box[a] cells. Returns the
// number of bad region indices (0), or -1 for a bad dim.
long emg_hc_kz_steps(int dim, const int* n, const int* box, const double* coef, const double* rhs, double* x,
                     int steps, double w) {
  if (dim != 2 && dim != 3) return -1;
  const kz::Boxes B = kz::make_boxes(dim, n, box);
  if (dim == 3) return kz_steps_host<3>(B, (const cx<double>*)coef, (const cx<double>*)rhs, (cx<double>*)x, steps, w);
  return kz_steps_host<2>(B, (const cx<double>*)coef, (const cx<double>*)rhs, (cx<double>*)x, steps, w);
}

// One-pass tiled residual + restriction (FP32) of a 2D level: bc (complex128, 3 (nx/2)(ny/2)) =
// R (b - H_s x); the arguments of emg_hc_residual_restrict2 without prec, then the tile height.
int emg_hc_resid_restrict_tiled(const int* n, double h, double beta, double omega, double att, double abl_len,
                                double abl_gmax, double Lx, double Ly, const double* mu, const double* rho,
                                const double* cp, const double* b64, const double* x64, double* bc64, int ty) {
  if (n[0] % 4 || n[0] < 4 || n[1] < 2 || (ty != 24 && ty != 8 && ty != 4)) return -1;
  Level2<float> L(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp);
  const size_t N = (size_t)n[0] * n[1];
  const int nxc = n[0] / 2, nyc = n[1] / 2;
  std::vector<cx<float>> b = to_cx<float>(b64, 3 * N), x = to_cx<float>(x64, 3 * N),
                         bc(3 * (size_t)nxc * nyc, mkc<float>(std::numeric_limits<float>::quiet_NaN(), 0.f));
  if (ty == 24) resid_restrict_tiled<24>(L.g, b.data(), x.data(), bc.data(), nxc, nyc);
  else if (ty == 8) resid_restrict_tiled<8>(L.g, b.data(), x.data(), bc.data(), nxc, nyc);
  else resid_restrict_tiled<4>(L.g, b.data(), x.data(), bc.data(), nxc, nyc);
  from_cx(bc, bc64);
  return 0;
}

// 2D FP64 apply of the outer solve in float-float arithmetic (ff2::apply_cell over every cell), with
// the coefficient arrays built as the library builds them (ff2::build_host, ff2::make):
// y = H x (shift 0) or H_s x; x FP64 (x32 = 0) or rounded to FP32 first (x32 = 1).
int emg_hc_apply_ff2(const int* n, double h, double beta, double omega, double gamma, double shift, double abl_len,
                     double abl_gmax, const double* lam, const double* mu, const double* rho, const double* x,
                     double* y, int x32) {
  ff2::HostFF2 o;
  ff2::build_host(o, n[0], n[1], h, lam, mu, rho, omega, gamma, abl_len, abl_gmax, n[0] * h, n[1] * h);
  const ff2::FineFF g = ff2::make(o.mu.data(), o.mun.data(), o.cp.data(), o.m1.data(), o.m2.data(), n[0], n[1], h,
                                  beta, shift);
  const size_t N = (size_t)n[0] * n[1];
  std::vector<cx<double>> xd(3 * N);
  std::vector<cx<float>> xf(3 * N);
  for (size_t k = 0; k < 3 * N; ++k) {
    xd[k] = mkc<double>(x[2 * k], x[2 * k + 1]);
    xf[k] = mkc<float>((float)x[2 * k], (float)x[2 * k + 1]);
  }
  for (int j = 0; j < n[1]; ++j)
    for (int i = 0; i < n[0]; ++i) {
      cx<double> out[3];
      if (x32) ff2::apply_cell<float>(g, xf.data(), nullptr, 0.0, i, j, out);
      else ff2::apply_cell<double>(g, xd.data(), nullptr, 0.0, i, j, out);
      for (int c = 0; c < 3; ++c) {
        const size_t q = c * N + (size_t)j * n[0] + i;
        y[2 * q] = out[c].re;
        y[2 * q + 1] = out[c].im;
      }
    }
  return 0;
}

// The float-float split and join of the FP64 outer kernels (dfloat.cuh) on n doubles.
int emg_hc_split_join(const double* x, int n, float* hi, float* lo, double* joined, double* widened) {
  for (int k = 0; k < n; ++k) {
    const df::f2 r = df::split(x[k]);
    hi[k] = r.hi;
    lo[k] = r.lo;
    joined[k] = df::join(r.hi, r.lo);
    widened[k] = df::widen(r.hi);
  }
  return 0;
}

// df::join on n arbitrary float pairs (the FP64 value of hi + lo).
int emg_hc_join(const float* hi, const float* lo, int n, double* out) {
  for (int k = 0; k < n; ++k) out[k] = df::join(hi[k], lo[k]);
  return 0;
}

// x += P e, then `sweeps` one-pass tiled sweeps with the correction added by the first one's tile
// loads (the fused post-smoothing of the cycle); e: complex128 coarse vector of 3 (nx/2)(ny/2).
int emg_hc_prolong_sweep_tiled(const int* n, double h, double beta, double omega, double att, double abl_len,
                               double abl_gmax, double Lx, double Ly, const double* mu, const double* rho,
                               const double* cp, const double* b64, const double* e64, double* x64, double w,
                               int sweeps, int ty) {
  if (ty != 24 && ty != 8 && ty != 4) return -1;
  if (n[0] % 4 || n[0] < 4 || n[1] < 2 || sweeps < 1) return -1;
  Level2<float> L(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp);
  const size_t N = (size_t)n[0] * n[1];
  const int nxc = n[0] / 2, nyc = n[1] / 2;
  std::vector<cx<float>> b = to_cx<float>(b64, 3 * N), x = to_cx<float>(x64, 3 * N), y(3 * N),
                         e = to_cx<float>(e64, 3 * (size_t)nxc * nyc);
  const float nan = std::numeric_limits<float>::quiet_NaN();
  for (int s = 0; s < sweeps; ++s) {
    for (auto& v : y) v = mkc<float>(nan, nan);
    if (ty == 24) sweep_tiled<24>(L.g, b.data(), x.data(), y.data(), (float)w, 0, s == 0 ? e.data() : nullptr, nxc, nyc);
    else if (ty == 8) sweep_tiled<8>(L.g, b.data(), x.data(), y.data(), (float)w, 0, s == 0 ? e.data() : nullptr, nxc, nyc);
    else sweep_tiled<4>(L.g, b.data(), x.data(), y.data(), (float)w, 0, s == 0 ? e.data() : nullptr, nxc, nyc);
    std::swap(x, y);
  }
  from_cx(x, x64);
  return 0;
}

// `sweeps` one-pass tiled sweeps (FP32) of a 2D level, complex128 b and x (x in/out), with the
// arguments of emg_hc_vanka2_sweeps; returns the number of tiles whose shared region lies
// inside the grid without attenuation (the kernel's interior, attenuation-free variant), or -1
// if the grid does not meet the kernel's rules.
int emg_hc_sweep_tiled(const int* n, double h, double beta, double omega, double att, double abl_len, double abl_gmax,
                       double Lx, double Ly, const double* mu, const double* rho, const double* cp, const double* b64,
                       double* x64, double w, int sweeps, int zero_first, int ty) {
  if (n[0] % 4 || n[0] < 4 || n[1] < 2 || (ty != 24 && ty != 8 && ty != 4)) return -1;
  Level2<float> L(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp);
  const size_t N = (size_t)n[0] * n[1];
  std::vector<cx<float>> b = to_cx<float>(b64, 3 * N), x = to_cx<float>(x64, 3 * N), y(3 * N);
  const float nan = std::numeric_limits<float>::quiet_NaN();
  for (int s = 0; s < sweeps; ++s) {
    for (auto& v : y) v = mkc<float>(nan, nan);  // every entry must be written
    if (ty == 24) sweep_tiled<24>(L.g, b.data(), x.data(), y.data(), (float)w, (zero_first && s == 0) ? 1 : 0);
    else if (ty == 8) sweep_tiled<8>(L.g, b.data(), x.data(), y.data(), (float)w, (zero_first && s == 0) ? 1 : 0);
    else sweep_tiled<4>(L.g, b.data(), x.data(), y.data(), (float)w, (zero_first && s == 0) ? 1 : 0);
    std::swap(x, y);
  }
  from_cx(x, x64);
  int interior = 0;
  for (int by = 0; by < (n[1] + ty - 1) / ty; ++by)
    for (int bx = 0; bx < (n[0] + k2t::TX - 1) / k2t::TX; ++bx) {
      const k2t::Tile t = ty == 24 ? k2t::tile_of<k2t::Geo<24>>(L.g, bx, by)
                                   : (ty == 8 ? k2t::tile_of<k2t::Geo<8>>(L.g, bx, by) : k2t::tile_of<k2t::Geo<4>>(L.g, bx, by));
      interior += t.fast ? 1 : 0;
    }
  return interior;
}

// 3D FP64 apply of the outer solve in float-float arithmetic: y = H x (shift 0) or H_s x, with
// the coefficient arrays built as the library builds them (ff3::build_host, ff3::make).
int emg_hc_apply_ff3(const int* n, double h, double beta, double omega, double gamma, double shift, double abl_len,
                     double abl_gmax, const double* L, const double* lam, const double* mu, const double* rho,
                     const double* x, double* y) {
  ff3::HostFF3 o;
  ff3::build_host(o, n[0], n[1], n[2], h, lam, mu, rho, omega, gamma, abl_len, abl_gmax, L);
  const df::f2* edge[3] = {o.edge[0].data(), o.edge[1].data(), o.edge[2].data()};
  const ff2::c2* m[3] = {o.m[0].data(), o.m[1].data(), o.m[2].data()};
  const ff3::FineFF3 g = ff3::make(o, o.mu.data(), o.cp.data(), edge, m, n[0], n[1], n[2], h, beta, shift);
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i)
        ff3::cell_rows<double>(g, (const cx<double>*)x, nullptr, 0.0, (cx<double>*)y, i, j, k);
  return 0;
}

// The outer solve's residual form y = bscale * b - H x in float-float arithmetic, 2D (d = 2, L
// unused) or 3D (ff2::apply_cell / ff3::cell_rows), x FP64 (x32 = 0) or rounded to FP32 first
// (x32 = 1); b == NULL gives y = H x.
int emg_hc_residual_ff(int d, const int* n, double h, double beta, double omega, double gamma, double abl_len,
                       double abl_gmax, const double* L, const double* lam, const double* mu, const double* rho,
                       const double* x, const double* b, double bscale, double* y, int x32) {
  const size_t N = (size_t)n[0] * n[1] * (d == 3 ? n[2] : 1), nv = (size_t)(d + 1) * N;
  std::vector<cx<double>> xd(nv);
  std::vector<cx<float>> xf(nv);
  for (size_t k = 0; k < nv; ++k) {
    xd[k] = mkc<double>(x[2 * k], x[2 * k + 1]);
    xf[k] = mkc<float>((float)x[2 * k], (float)x[2 * k + 1]);
  }
  const cx<double>* bb = (const cx<double>*)b;
  if (d == 2) {
    ff2::HostFF2 o;
    ff2::build_host(o, n[0], n[1], h, lam, mu, rho, omega, gamma, abl_len, abl_gmax, n[0] * h, n[1] * h);
    const ff2::FineFF g = ff2::make(o.mu.data(), o.mun.data(), o.cp.data(), o.m1.data(), o.m2.data(), n[0], n[1], h,
                                    beta, 0.0);
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        cx<double> out[3];
        if (x32) ff2::apply_cell<float>(g, xf.data(), bb, bscale, i, j, out);
        else ff2::apply_cell<double>(g, xd.data(), bb, bscale, i, j, out);
        for (int c = 0; c < 3; ++c) {
          const size_t q = c * N + (size_t)j * n[0] + i;
          y[2 * q] = out[c].re;
          y[2 * q + 1] = out[c].im;
        }
      }
    return 0;
  }
  ff3::HostFF3 o;
  ff3::build_host(o, n[0], n[1], n[2], h, lam, mu, rho, omega, gamma, abl_len, abl_gmax, L);
  const df::f2* edge[3] = {o.edge[0].data(), o.edge[1].data(), o.edge[2].data()};
  const ff2::c2* m[3] = {o.m[0].data(), o.m[1].data(), o.m[2].data()};
  const ff3::FineFF3 g = ff3::make(o, o.mu.data(), o.cp.data(), edge, m, n[0], n[1], n[2], h, beta, 0.0);
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        if (x32) ff3::cell_rows<float>(g, xf.data(), bb, bscale, (cx<double>*)y, i, j, k);
        else ff3::cell_rows<double>(g, xd.data(), bb, bscale, (cx<double>*)y, i, j, k);
      }
  return 0;
}

// 3D y = H^H x in float-float arithmetic on the same coefficient arrays (adjoint_ff3.cuh).
int emg_hc_apply_adjoint_ff3(const int* n, double h, double beta, double omega, double gamma, double abl_len,
                             double abl_gmax, const double* L, const double* lam, const double* mu, const double* rho,
                             const double* x, double* y) {
  ff3::HostFF3 o;
  ff3::build_host(o, n[0], n[1], n[2], h, lam, mu, rho, omega, gamma, abl_len, abl_gmax, L);
  const df::f2* edge[3] = {o.edge[0].data(), o.edge[1].data(), o.edge[2].data()};
  const ff2::c2* m[3] = {o.m[0].data(), o.m[1].data(), o.m[2].data()};
  const ff3::FineFF3 g = ff3::make(o, o.mu.data(), o.cp.data(), edge, m, n[0], n[1], n[2], h, beta, 0.0);
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i)
        ff3::cell_rows_adjoint<double>(g, (const cx<double>*)x, nullptr, 0.0, (cx<double>*)y, i, j, k);
  return 0;
}

// 3D residual of one level: r (complex128, 4 nx ny nz) = b - H_s x.
int emg_hc_residual3(int prec, const int* n, double h, double beta, double omega, double att, double abl_len,
                     double abl_gmax, double Lx, double Ly, double Lz, const double* mu, const double* rho,
                     const double* cp, const double* b, const double* x, double* r) {
  if (prec == 64) residual3<double>(Level2<double, 3>(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp, Lz),
                                    b, x, r);
  else if (prec == 32) residual3<float>(Level2<float, 3>(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp, Lz),
                                        b, x, r);
  else return 1;
  return 0;
}

// 3D tile half-sweeps (sweeps3_tile); -1 for a grid below one tile.
int emg_hc_vanka3_tile_sweeps(int prec, const int* n, double h, double beta, double omega, double att, double abl_len,
                              double abl_gmax, double Lx, double Ly, double Lz, const double* mu, const double* rho,
                              const double* cp, const double* b, double* x, double w, int sweeps, int zero_first) {
  if (n[0] < k3t::TX || n[1] < k3t::TY || n[2] < k3t::TZ) return -1;
  if (prec == 64)
    sweeps3_tile<double>(Level2<double, 3>(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp, Lz), b, x, w,
                         sweeps, zero_first);
  else if (prec == 32)
    sweeps3_tile<float>(Level2<float, 3>(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp, Lz), b, x, w,
                        sweeps, zero_first);
  else return 1;
  return 0;
}

// 2D red-black Vanka sweeps of one level (prec 32 or 64), complex128 b and x (x in/out);
// att = gamma + the level's shift; abl_len, Lx, Ly physical (the finest grid's).
int emg_hc_vanka2_sweeps(int prec, const int* n, double h, double beta, double omega, double att, double abl_len,
                         double abl_gmax, double Lx, double Ly, const double* mu, const double* rho, const double* cp,
                         const double* b, double* x, double w, int sweeps, int zero_first) {
  if (prec == 64) sweeps2<double>(Level2<double>(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp), b, x, w,
                                  sweeps, zero_first);
  else if (prec == 32) sweeps2<float>(Level2<float>(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp), b, x,
                                      w, sweeps, zero_first);
  else return 1;
  return 0;
}

// 2D residual and restriction of one level: bc (complex128, 3 (nx/2)(ny/2)) = R (b - H_s x).
int emg_hc_residual_restrict2(int prec, const int* n, double h, double beta, double omega, double att, double abl_len,
                              double abl_gmax, double Lx, double Ly, const double* mu, const double* rho,
                              const double* cp, const double* b, const double* x, double* bc) {
  if (prec == 64) residual_restrict2<double>(Level2<double>(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho, cp),
                                             b, x, bc);
  else if (prec == 32) residual_restrict2<float>(Level2<float>(n, h, beta, omega, att, abl_len, abl_gmax, Lx, Ly, mu, rho,
                                                               cp), b, x, bc);
  else return 1;
  return 0;
}


// y = H^H x for complex128 x, y of (dim+1) * n_x n_y (n_z) values; att = gamma + shift.
int emg_hc_adjoint_apply(int dim, const int* n, double h, double beta, double omega, double att, double abl_len,
                         double abl_gmax, const double* mu, const double* rho, const double* cp, const double* x,
                         double* y) {
  const Grid<double> g = host_grid(dim, n, h, beta, omega, att, abl_len, abl_gmax, mu, rho, cp);
  if (dim == 2) apply_all<2>(g, (const cx<double>*)x, (cx<double>*)y);
  else if (dim == 3) apply_all<3>(g, (const cx<double>*)x, (cx<double>*)y);
  else return 1;
  return 0;
}

// -Re a^H (dH/dm) u per cell for m = lambda, mu, rho (unshifted operator: att = gamma).
int emg_hc_material_gradient(int dim, const int* n, double h, double beta, double omega, double att, double abl_len,
                             double abl_gmax, const double* mu, const double* rho, const double* cp, const double* u,
                             const double* a, double* glam, double* gmu, double* grho) {
  const Grid<double> g = host_grid(dim, n, h, beta, omega, att, abl_len, abl_gmax, mu, rho, cp);
  if (dim == 2) gradient_all<2>(g, (const cx<double>*)u, (const cx<double>*)a, glam, gmu, grho);
  else if (dim == 3) gradient_all<3>(g, (const cx<double>*)u, (const cx<double>*)a, glam, gmu, grho);
  else return 1;
  return 0;
}

}  // extern "C"
