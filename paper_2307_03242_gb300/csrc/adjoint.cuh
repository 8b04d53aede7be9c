// Conjugate-transposed operator and the material derivative of a^H H u, for the adjoint-state
// misfit gradient of frequency-domain inversion (the adjoint-state method, Plessix 2006), in 2D
// and 3D (D). __host__ __device__ so the same per-DOF functions run in the GPU kernels and in a
// host build that the tests compare with the FP64 oracle.
//
// Operator (Eq. 3.10 with the coupling sign of Eq. 4.4; 3D Sec. 5.3):
//   u_c row at face q: (1/h) sum_e [y_e(q) - y_e(q + s_e)] - (M^beta (m u_c))(q) + (p(q) - p(q - s_c))/h
//   p row at cell q:   sum_c (D^beta_c u_c)(q) + p(q) / (lambda + mu)
// with y_e(pt) = mu_e(pt) (D^beta_e u_c)(pt) at the derivative points pt (between pt - s_e and
// pt), D^beta the beta-spread difference (beta at the centre line plus (1-beta) [1 2 1]/4 across
// in 2D, Eq. 3.5; (1-beta)/16 [1 2 1] x [1 2 1] across in 3D, Eq. dxSkew3D), mu_e the cell mu
// for e = c and the mean of the 2 x 2 cells around the node / edge otherwise, and the face mass
// m = rho_f omega^2 (1 - i att), rho_f the mean of the two adjacent cells.
//
// Transpose. Summation by parts over the derivative points turns the Laplacian into
// (1/h) sum_e sum_o w(o) [Y_e(q + o) - Y_e(q + o + s_e)] with Y_e(pt) = mu_e(pt) (u_c(pt) -
// u_c(pt - s_e))/h (the spread moves to the outer difference; w is symmetric), the mass into
// m(q) (M^beta u_c)(q), the divergence into (1/h) sum_o w(o) [p(q + o - s_c) - p(q + o)] and the
// gradient into sum_c (u_c(q) - u_c(q + s_c))/h. Every coefficient but m is real, so H^H is H^T
// with conj(m). Values outside the domain and on boundary faces are zero, exactly as in H, so the
// sums need no range checks; boundary faces (index 0 along their axis) are not unknowns and get
// zero rows.
//
// Material derivative, -Re a^H (dH/dm_k) u for the finest level (unshifted operator):
//   mu:  sum over the derivative points whose mu average contains cell k (with the clamping of
//        the average at the boundary) of weight * conj(D_e a_c)(pt) (D^beta_e u_c)(pt), plus the
//        continuity term -conj(a_p) u_p / (lambda + mu)^2;
//   lam: the continuity term;
//   rho: -sum over the faces whose density average contains k of weight * conj(M^beta a_c)(f)
//        omega^2 (1 - i att_f) u_c(f).
#pragma once
#include "emg_types.cuh"

namespace adj {

HD void unit(int a, int& di, int& dj, int& dk) {
  di = a == 0;
  dj = a == 1;
  dk = a == 2;
}
template <typename T> HD size_t lin(const Grid<T>& g, int i, int j, int k) {
  return ((size_t)k * g.ny + j) * g.nx + i;
}
template <typename T> HD bool inside(const Grid<T>& g, int i, int j, int k) {
  return i >= 0 && i < g.nx && j >= 0 && j < g.ny && k >= 0 && k < g.nz;
}
// component c at face (i,j,k): zero outside the domain and on the boundary faces of its axis
template <typename T, typename TI>
HD cx<T> U(int c, const cx<TI>* u, const Grid<T>& g, int i, int j, int k) {
  const int kc = c == 0 ? i : (c == 1 ? j : k);
  return (inside(g, i, j, k) && kc >= 1) ? ccast<T>(u[lin(g, i, j, k)]) : czero<T>();
}
template <typename T, typename TI>
HD cx<T> P(const cx<TI>* p, const Grid<T>& g, int i, int j, int k) {
  return inside(g, i, j, k) ? ccast<T>(p[lin(g, i, j, k)]) : czero<T>();
}
HD int clampi(int v, int n) { return v < 0 ? 0 : (v > n - 1 ? n - 1 : v); }
template <typename T> HD T mat(const T* f, const Grid<T>& g, int i, int j, int k) {
  return f[lin(g, clampi(i, g.nx), clampi(j, g.ny), clampi(k, g.nz))];
}

// mu at the derivative point pt of d_e u_c: the cell pt - s_c for e == c, the mean of the four
// cells pt, pt - s_c, pt - s_e, pt - s_c - s_e otherwise
template <typename T> HD T mu_pt(const Grid<T>& g, int c, int e, int i, int j, int k) {
  int ci, cj, ck;
  unit(c, ci, cj, ck);
  if (e == c) return mat(g.mu, g, i - ci, j - cj, k - ck);
  int ei, ej, ek;
  unit(e, ei, ej, ek);
  return T(0.25) * (mat(g.mu, g, i, j, k) + mat(g.mu, g, i - ci, j - cj, k - ck) + mat(g.mu, g, i - ei, j - ej, k - ek) +
                    mat(g.mu, g, i - ci - ei, j - cj - ej, k - ck - ek));
}

// omega^2 (1 - i att_f) at face u_c(i,j,k), att_f = g.att + absorbing layer (Grid::ablL > 0)
template <int D, typename T> HD cx<T> mass_unit(const Grid<T>& g, int c, int i, int j, int k) {
  T att = g.att;
  if (g.ablL > T(0)) {
    const T x = (T(i) + (c == 0 ? T(0) : T(0.5))) * g.h;
    const T y = (T(j) + (c == 1 ? T(0) : T(0.5))) * g.h;
    T s = abl_axis(x, g.ablL, g.Lx) + abl_axis(y, g.ablL, g.Ly);
    if (D == 3) s += abl_axis((T(k) + (c == 2 ? T(0) : T(0.5))) * g.h, g.ablL, g.Lz);
    att += g.ablG * s / (g.ablL * g.ablL);
  }
  return mkc<T>(g.w2, -g.w2 * att);
}
// rho_f at face u_c(i,j,k): mean of the cells on both sides (clamped)
template <typename T> HD T rho_face(const Grid<T>& g, int c, int i, int j, int k) {
  int ci, cj, ck;
  unit(c, ci, cj, ck);
  return T(0.5) * (mat(g.rho, g, i - ci, j - cj, k - ck) + mat(g.rho, g, i, j, k));
}

// Offsets across axis e of the spread difference and their weights: n_off() offsets; offset t
// gives (oi, oj, ok) and its weight.
template <int D> HD int n_off() { return D == 3 ? 9 : 3; }
template <int D, typename T>
HD T offset(int e, int t, T beta, int& oi, int& oj, int& ok) {
  if (D == 2) {
    const int a = t - 1, p = 1 - e;
    oi = p == 0 ? a : 0;
    oj = p == 1 ? a : 0;
    ok = 0;
    return (a == 0 ? beta : T(0)) + (T(1) - beta) * (a == 0 ? T(0.5) : T(0.25));
  }
  const int a = t / 3 - 1, b = t % 3 - 1;
  const int p = (e + 1) % 3, r = (e + 2) % 3;
  int pi, pj, pk, ri, rj, rk;
  unit(p, pi, pj, pk);
  unit(r, ri, rj, rk);
  oi = a * pi + b * ri;
  oj = a * pj + b * rj;
  ok = a * pk + b * rk;
  const T wa = a == 0 ? T(2) : T(1), wb = b == 0 ? T(2) : T(1);
  return (a == 0 && b == 0 ? beta : T(0)) + (T(1) - beta) * wa * wb * T(0.0625);
}

// beta-spread difference of u_c along e at point (i,j,k) (between pt - s_e and pt), times 1/h
template <int D, typename T, typename TI>
HD cx<T> dspread(int c, int e, const cx<TI>* u, const Grid<T>& g, int i, int j, int k) {
  int ei, ej, ek;
  unit(e, ei, ej, ek);
  cx<T> acc = czero<T>();
  for (int t = 0; t < n_off<D>(); ++t) {
    int oi, oj, ok;
    const T w = offset<D, T>(e, t, g.beta, oi, oj, ok);
    acc = acc + w * (U(c, u, g, i + oi, j + oj, k + ok) - U(c, u, g, i + oi - ei, j + oj - ej, k + ok - ek));
  }
  return g.ih * acc;
}
// plain difference of u_c along e at point (i,j,k), times 1/h
template <typename T, typename TI>
HD cx<T> dplain(int c, int e, const cx<TI>* u, const Grid<T>& g, int i, int j, int k) {
  int ei, ej, ek;
  unit(e, ei, ej, ek);
  return g.ih * (U(c, u, g, i, j, k) - U(c, u, g, i - ei, j - ej, k - ek));
}
// (M^beta v_c)(face): beta v(f) + sm * (sum of the 2D same-component neighbours)
template <int D, typename T, typename TI>
HD cx<T> mspread(int c, const cx<TI>* v, const Grid<T>& g, int i, int j, int k) {
  cx<T> nb = czero<T>();
  for (int a = 0; a < D; ++a) {
    int ai, aj, ak;
    unit(a, ai, aj, ak);
    nb = nb + U(c, v, g, i - ai, j - aj, k - ak) + U(c, v, g, i + ai, j + aj, k + ak);
  }
  return g.beta * U(c, v, g, i, j, k) + g.sm * nb;
}

// (H^H x) at face u_c(i,j,k); x[0..D-1] displacement components, x[D] pressure
template <int D, typename T, typename TI>
HD cx<T> row_u(int c, const cx<TI>* const* x, const Grid<T>& g, int i, int j, int k) {
  const int kc = c == 0 ? i : (c == 1 ? j : k);
  if (kc < 1) return czero<T>();
  cx<T> lap = czero<T>();
  for (int e = 0; e < D; ++e) {
    int ei, ej, ek;
    unit(e, ei, ej, ek);
    for (int t = 0; t < n_off<D>(); ++t) {
      int oi, oj, ok;
      const T w = offset<D, T>(e, t, g.beta, oi, oj, ok);
      const int a = i + oi, b = j + oj, q = k + ok;
      const cx<T> y0 = mu_pt(g, c, e, a, b, q) * dplain(c, e, x[c], g, a, b, q);
      const cx<T> y1 = mu_pt(g, c, e, a + ei, b + ej, q + ek) * dplain(c, e, x[c], g, a + ei, b + ej, q + ek);
      lap = lap + w * (y0 - y1);
    }
  }
  lap = g.ih * lap;
  const cx<T> m = rho_face(g, c, i, j, k) * mass_unit<D>(g, c, i, j, k);
  const cx<T> mass = cconj(m) * mspread<D>(c, x[c], g, i, j, k);
  int ci, cj, ck;
  unit(c, ci, cj, ck);
  cx<T> dv = czero<T>();
  for (int t = 0; t < n_off<D>(); ++t) {
    int oi, oj, ok;
    const T w = offset<D, T>(c, t, g.beta, oi, oj, ok);
    dv = dv + w * (P(x[D], g, i + oi - ci, j + oj - cj, k + ok - ck) - P(x[D], g, i + oi, j + oj, k + ok));
  }
  return lap - mass + g.ih * dv;
}

// (H^H x) at the centre of cell (i,j,k)
template <int D, typename T, typename TI>
HD cx<T> row_p(const cx<TI>* const* x, const Grid<T>& g, int i, int j, int k) {
  cx<T> s = czero<T>();
  for (int c = 0; c < D; ++c) {
    int ci, cj, ck;
    unit(c, ci, cj, ck);
    s = s + (U(c, x[c], g, i, j, k) - U(c, x[c], g, i + ci, j + cj, k + ck));
  }
  return g.ih * s + mat(g.cp, g, i, j, k) * P(x[D], g, i, j, k);
}

// number of the corners {0, -1} along c (and along e, if e >= 0) of point (i,j,k) whose clamped
// cell is (ki,kj,kk)
template <typename T>
HD int corners_at(const Grid<T>& g, int c, int e, int i, int j, int k, int ki, int kj, int kk) {
  int ci, cj, ck, ei = 0, ej = 0, ek = 0;
  unit(c, ci, cj, ck);
  if (e >= 0) unit(e, ei, ej, ek);
  int cnt = 0;
  for (int x = 0; x < 2; ++x)
    for (int y = 0; y < (e >= 0 ? 2 : 1); ++y) {
      const int a = clampi(i - x * ci - y * ei, g.nx), b = clampi(j - x * cj - y * ej, g.ny),
                q = clampi(k - x * ck - y * ek, g.nz);
      cnt += (a == ki && b == kj && q == kk);
    }
  return cnt;
}

// -Re a^H (dH/dm) u at cell (i,j,k) for m = lam, mu, rho (u[0..D], a[0..D] as in row_u)
template <int D, typename T, typename TI>
HD void gradient(const cx<TI>* const* u, const cx<TI>* const* a, const Grid<T>& g, int i, int j, int k, T& glam,
                 T& gmu, T& grho) {
  cx<T> dmu = czero<T>(), drho = czero<T>();
  for (int c = 0; c < D; ++c) {
    int ci, cj, ck;
    unit(c, ci, cj, ck);
    // e == c: the derivative point of cell (i,j,k) itself
    dmu = dmu + cconj(dplain(c, c, a[c], g, i + ci, j + cj, k + ck)) * dspread<D>(c, c, u[c], g, i + ci, j + cj, k + ck);
    for (int e = 0; e < D; ++e) {
      if (e == c) continue;
      int ei, ej, ek;
      unit(e, ei, ej, ek);
      for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) {
          const int pi = i + x * ci + y * ei, pj = j + x * cj + y * ej, pk = k + x * ck + y * ek;
          const int cnt = corners_at(g, c, e, pi, pj, pk, i, j, k);
          if (cnt == 0) continue;
          dmu = dmu + (T(0.25) * T(cnt)) * (cconj(dplain(c, e, a[c], g, pi, pj, pk)) * dspread<D>(c, e, u[c], g, pi, pj, pk));
        }
    }
    for (int x = 0; x < 2; ++x) {
      const int fi = i + x * ci, fj = j + x * cj, fk = k + x * ck;
      const int cnt = corners_at(g, c, -1, fi, fj, fk, i, j, k);
      if (cnt == 0) continue;
      const cx<T> ma = cconj(mspread<D>(c, a[c], g, fi, fj, fk));
      drho = drho - (T(0.5) * T(cnt)) * (ma * mass_unit<D>(g, c, fi, fj, fk) * U(c, u[c], g, fi, fj, fk));
    }
  }
  const T cp = mat(g.cp, g, i, j, k);
  const cx<T> pp = (-cp * cp) * (cconj(P(a[D], g, i, j, k)) * P(u[D], g, i, j, k));
  glam = -pp.re;
  gmu = -(dmu.re + pp.re);
  grho = -drho.re;
}

}  // namespace adj
