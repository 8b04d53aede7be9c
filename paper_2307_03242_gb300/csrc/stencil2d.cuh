// 2D operator rows of the beta-spread MAC discretisation (Eq. 3.10 with the sign of Eq. 4.4),
// written as __host__ __device__ functions so that the host can assemble the dense coarsest
// operator from exactly the formulas the kernels use.
//
// Storage: component arrays of nx*ny complex values, index j*nx + i. u1(i,j) is the x1-face at
// x = i h, y = (j+1/2) h; u2(i,j) the x2-face at x = (i+1/2) h, y = j h; p(i,j) the cell centre.
// Faces with i = 0 (u1) or j = 0 (u2) are on the boundary and are not unknowns; every value
// outside the domain is zero; material outside the domain is clamped to the nearest cell.
#pragma once
#include "emg_types.cuh"

namespace s2 {

template <typename T, typename TI>
HD cx<T> U1(const cx<TI>* u, const Grid<T>& g, int i, int j) {
  return (i >= 1 && i < g.nx && j >= 0 && j < g.ny) ? ccast<T>(u[(size_t)j * g.nx + i]) : czero<T>();
}
template <typename T, typename TI>
HD cx<T> U2(const cx<TI>* u, const Grid<T>& g, int i, int j) {
  return (j >= 1 && j < g.ny && i >= 0 && i < g.nx) ? ccast<T>(u[(size_t)j * g.nx + i]) : czero<T>();
}
template <typename T, typename TI>
HD cx<T> PP(const cx<TI>* p, const Grid<T>& g, int i, int j) {
  return (i >= 0 && i < g.nx && j >= 0 && j < g.ny) ? ccast<T>(p[(size_t)j * g.nx + i]) : czero<T>();
}
template <typename T> HD T mat(const T* f, const Grid<T>& g, int i, int j) {
  i = iclamp(i, 0, g.nx - 1);
  j = iclamp(j, 0, g.ny - 1);
  return f[(size_t)j * g.nx + i];
}
// mu at the lattice point (X h, Y h): mean of the four cells around it (A_e, Sec. 3.1).
template <typename T> HD T mu_node(const Grid<T>& g, int X, int Y) {
  return T(0.25) * (mat(g.mu, g, X - 1, Y - 1) + mat(g.mu, g, X, Y - 1) + mat(g.mu, g, X - 1, Y) + mat(g.mu, g, X, Y));
}
// Mass coefficient m_f = rho_f omega^2 (1 - i (gamma + shift + gamma_ABL(x_f))) at u1 / u2 faces.
template <typename T> HD cx<T> m1(const Grid<T>& g, int i, int j) {
  T rf = T(0.5) * (mat(g.rho, g, i - 1, j) + mat(g.rho, g, i, j));
  T att = g.att;
  if (g.ablL > T(0)) {
    T x = T(i) * g.h, y = (T(j) + T(0.5)) * g.h;
    att += g.ablG * (abl_axis(x, g.ablL, g.Lx) + abl_axis(y, g.ablL, g.Ly)) / (g.ablL * g.ablL);
  }
  T a = rf * g.w2;
  return mkc<T>(a, -a * att);
}
template <typename T> HD cx<T> m2(const Grid<T>& g, int i, int j) {
  T rf = T(0.5) * (mat(g.rho, g, i, j - 1) + mat(g.rho, g, i, j));
  T att = g.att;
  if (g.ablL > T(0)) {
    T x = (T(i) + T(0.5)) * g.h, y = T(j) * g.h;
    att += g.ablG * (abl_axis(x, g.ablL, g.Lx) + abl_axis(y, g.ablL, g.Ly)) / (g.ablL * g.ablL);
  }
  T a = rf * g.w2;
  return mkc<T>(a, -a * att);
}

// beta-spread derivatives (Eq. 3.5). t0 = (1+beta)/2 on the centre line, t1 = (1-beta)/4 on the
// two lines beside it.
// d/dx1 of u1 at the centre of cell (c, j):
template <typename T, typename TI> HD cx<T> G1(const cx<TI>* u1, const Grid<T>& g, int c, int j, T t0, T t1) {
  cx<T> a = U1(u1, g, c + 1, j - 1) - U1(u1, g, c, j - 1);
  cx<T> b = U1(u1, g, c + 1, j) - U1(u1, g, c, j);
  cx<T> d = U1(u1, g, c + 1, j + 1) - U1(u1, g, c, j + 1);
  return g.ih * (t1 * (a + d) + t0 * b);
}
// d/dx2 of u1 at the lattice point (i h, k h):
template <typename T, typename TI> HD cx<T> G2(const cx<TI>* u1, const Grid<T>& g, int i, int k, T t0, T t1) {
  cx<T> a = U1(u1, g, i - 1, k) - U1(u1, g, i - 1, k - 1);
  cx<T> b = U1(u1, g, i, k) - U1(u1, g, i, k - 1);
  cx<T> d = U1(u1, g, i + 1, k) - U1(u1, g, i + 1, k - 1);
  return g.ih * (t1 * (a + d) + t0 * b);
}
// d/dx1 of u2 at the lattice point (k h, j h):
template <typename T, typename TI> HD cx<T> H1(const cx<TI>* u2, const Grid<T>& g, int k, int j, T t0, T t1) {
  cx<T> a = U2(u2, g, k, j - 1) - U2(u2, g, k - 1, j - 1);
  cx<T> b = U2(u2, g, k, j) - U2(u2, g, k - 1, j);
  cx<T> d = U2(u2, g, k, j + 1) - U2(u2, g, k - 1, j + 1);
  return g.ih * (t1 * (a + d) + t0 * b);
}
// d/dx2 of u2 at the centre of cell (i, c):
template <typename T, typename TI> HD cx<T> H2(const cx<TI>* u2, const Grid<T>& g, int i, int c, T t0, T t1) {
  cx<T> a = U2(u2, g, i - 1, c + 1) - U2(u2, g, i - 1, c);
  cx<T> b = U2(u2, g, i, c + 1) - U2(u2, g, i, c);
  cx<T> d = U2(u2, g, i + 1, c + 1) - U2(u2, g, i + 1, c);
  return g.ih * (t1 * (a + d) + t0 * b);
}

// (H x) at the u1 face (i, j), 1 <= i < nx: grad_h^T A_e(mu) grad_h^beta u1 - M^beta(m u1) + d/dx1 p.
template <typename T, typename TI>
HD cx<T> row_u1(const cx<TI>* u1, const cx<TI>* p, const Grid<T>& g, int i, int j) {
  const T t0 = T(0.5) * (T(1) + g.beta), t1 = T(0.25) * (T(1) - g.beta);
  cx<T> lap = g.ih * (mat(g.mu, g, i - 1, j) * G1(u1, g, i - 1, j, t0, t1) - mat(g.mu, g, i, j) * G1(u1, g, i, j, t0, t1)
                      + mu_node(g, i, j) * G2(u1, g, i, j, t0, t1) - mu_node(g, i, j + 1) * G2(u1, g, i, j + 1, t0, t1));
  cx<T> mass = g.beta * (m1(g, i, j) * U1(u1, g, i, j))
             + g.sm * (m1(g, i - 1, j) * U1(u1, g, i - 1, j) + m1(g, i + 1, j) * U1(u1, g, i + 1, j)
                       + m1(g, i, j - 1) * U1(u1, g, i, j - 1) + m1(g, i, j + 1) * U1(u1, g, i, j + 1));
  cx<T> grad = g.ih * (PP(p, g, i, j) - PP(p, g, i - 1, j));
  return lap - mass + grad;
}
// (H x) at the u2 face (i, j), 1 <= j < ny.
template <typename T, typename TI>
HD cx<T> row_u2(const cx<TI>* u2, const cx<TI>* p, const Grid<T>& g, int i, int j) {
  const T t0 = T(0.5) * (T(1) + g.beta), t1 = T(0.25) * (T(1) - g.beta);
  cx<T> lap = g.ih * (mu_node(g, i, j) * H1(u2, g, i, j, t0, t1) - mu_node(g, i + 1, j) * H1(u2, g, i + 1, j, t0, t1)
                      + mat(g.mu, g, i, j - 1) * H2(u2, g, i, j - 1, t0, t1) - mat(g.mu, g, i, j) * H2(u2, g, i, j, t0, t1));
  cx<T> mass = g.beta * (m2(g, i, j) * U2(u2, g, i, j))
             + g.sm * (m2(g, i - 1, j) * U2(u2, g, i - 1, j) + m2(g, i + 1, j) * U2(u2, g, i + 1, j)
                       + m2(g, i, j - 1) * U2(u2, g, i, j - 1) + m2(g, i, j + 1) * U2(u2, g, i, j + 1));
  cx<T> grad = g.ih * (PP(p, g, i, j) - PP(p, g, i, j - 1));
  return lap - mass + grad;
}
// (H x) at the centre of cell (i, j): (div)_h^beta u + p / (lambda + mu).
template <typename T, typename TI>
HD cx<T> row_p(const cx<TI>* u1, const cx<TI>* u2, const cx<TI>* p, const Grid<T>& g, int i, int j) {
  const T t0 = T(0.5) * (T(1) + g.beta), t1 = T(0.25) * (T(1) - g.beta);
  return G1(u1, g, i, j, t0, t1) + H2(u2, g, i, j, t0, t1) + mat(g.cp, g, i, j) * PP(p, g, i, j);
}

// The cell's 5x5 Vanka block (Sec. 2.3; Remark 3.1: the u block is two 2x2 blocks) for the DOFs
// (W = u1(i,j), E = u1(i+1,j), S = u2(i,j), N = u2(i,j+1), p(i,j)):
//   [A1 0 Gu1] A1 = [dW oWE; oEW dE], A2 = [dS oSN; oNS dN]
//   [0 A2 Gu2] G = (+1/h, -1/h, +1/h, -1/h) (gradient), B = t0/h (-1, +1, -1, +1) (divergence)
//   [B    cp ]
template <typename T>
HD void block_u1(const Grid<T>& g, int i, int j, cx<T>& dW, cx<T>& oWE, cx<T>& oEW, cx<T>& dE) {
  const T t0 = T(0.5) * (T(1) + g.beta), t1 = T(0.25) * (T(1) - g.beta);
  const T ih2 = g.ih * g.ih;
  T mc = mat(g.mu, g, i, j);
  T nA = mu_node(g, i, j), nB = mu_node(g, i, j + 1), nC = mu_node(g, i + 1, j), nD = mu_node(g, i + 1, j + 1);
  cx<T> mW = m1(g, i, j), mE = m1(g, i + 1, j);
  dW = mkc<T>(t0 * ih2 * (mat(g.mu, g, i - 1, j) + mc + nA + nB), T(0)) - g.beta * mW;
  dE = mkc<T>(t0 * ih2 * (mc + mat(g.mu, g, i + 1, j) + nC + nD), T(0)) - g.beta * mE;
  oWE = mkc<T>(ih2 * (-t0 * mc + t1 * (nA + nB)), T(0)) - g.sm * mE;
  oEW = mkc<T>(ih2 * (-t0 * mc + t1 * (nC + nD)), T(0)) - g.sm * mW;
}
template <typename T>
HD void block_u2(const Grid<T>& g, int i, int j, cx<T>& dS, cx<T>& oSN, cx<T>& oNS, cx<T>& dN) {
  const T t0 = T(0.5) * (T(1) + g.beta), t1 = T(0.25) * (T(1) - g.beta);
  const T ih2 = g.ih * g.ih;
  T mc = mat(g.mu, g, i, j);
  T nA = mu_node(g, i, j), nB = mu_node(g, i + 1, j), nC = mu_node(g, i, j + 1), nD = mu_node(g, i + 1, j + 1);
  cx<T> mS = m2(g, i, j), mN = m2(g, i, j + 1);
  dS = mkc<T>(t0 * ih2 * (nA + nB + mat(g.mu, g, i, j - 1) + mc), T(0)) - g.beta * mS;
  dN = mkc<T>(t0 * ih2 * (nC + nD + mc + mat(g.mu, g, i, j + 1)), T(0)) - g.beta * mN;
  oSN = mkc<T>(ih2 * (-t0 * mc + t1 * (nA + nB)), T(0)) - g.sm * mN;
  oNS = mkc<T>(ih2 * (-t0 * mc + t1 * (nC + nD)), T(0)) - g.sm * mS;
}

}  // namespace s2
