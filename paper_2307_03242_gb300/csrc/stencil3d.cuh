// 3D operator rows of the beta-spread MAC discretisation (Section 5.3: Eq. dxSkew3D spread
// derivatives with the 1/h of the 2D form, Eq. massHO3D spread mass; block form of Eq. 3.10 with
// the sign of Eq. 4.4). __host__ __device__ so the host can assemble the dense coarsest operator.
//
// Storage: arrays of nx*ny*nz complex values, index (k*ny + j)*nx + i. u_c(i,j,k) is the face
// normal to axis c on the low side of cell (i,j,k); p at the cell centre. Faces whose index along
// their own axis is 0 are boundary faces (not unknowns); values outside the domain are zero;
// material outside the domain is clamped.
#pragma once
#include "emg_types.cuh"

namespace s3 {

template <typename T> HD size_t lin(const Grid<T>& g, int i, int j, int k) {
  return ((size_t)k * g.ny + j) * g.nx + i;
}
template <typename T> HD bool inside(const Grid<T>& g, int i, int j, int k) {
  return i >= 0 && i < g.nx && j >= 0 && j < g.ny && k >= 0 && k < g.nz;
}
template <typename T, typename TI>
HD cx<T> U(int c, const cx<TI>* u, const Grid<T>& g, int i, int j, int k) {
  const int kc = c == 0 ? i : (c == 1 ? j : k);
  return (inside(g, i, j, k) && kc >= 1) ? ccast<T>(u[lin(g, i, j, k)]) : czero<T>();
}
template <typename T, typename TI>
HD cx<T> PP(const cx<TI>* p, const Grid<T>& g, int i, int j, int k) {
  return inside(g, i, j, k) ? ccast<T>(p[lin(g, i, j, k)]) : czero<T>();
}
template <typename T> HD T mat(const T* f, const Grid<T>& g, int i, int j, int k) {
  return f[lin(g, iclamp(i, 0, g.nx - 1), iclamp(j, 0, g.ny - 1), iclamp(k, 0, g.nz - 1))];
}

HD void unit(int a, int& di, int& dj, int& dk) {
  di = a == 0;
  dj = a == 1;
  dk = a == 2;
}

// mu at the lattice point with integer positions along axes c and e (c != e) and the index
// (i,j,k): mean of the four cells around that edge (A_e, Sec. 3.1).
template <typename T> HD T mu_edge(const Grid<T>& g, int c, int e, int i, int j, int k) {
  int ci, cj, ck, ei, ej, ek;
  unit(c, ci, cj, ck);
  unit(e, ei, ej, ek);
  return T(0.25) * (mat(g.mu, g, i, j, k) + mat(g.mu, g, i - ci, j - cj, k - ck) + mat(g.mu, g, i - ei, j - ej, k - ek) +
                    mat(g.mu, g, i - ci - ei, j - cj - ej, k - ck - ek));
}

// m_f = rho_f omega^2 (1 - i (gamma + shift + gamma_ABL(x_f))) at the face u_c(i,j,k).
template <typename T> HD cx<T> mcoef(const Grid<T>& g, int c, int i, int j, int k) {
  int ci, cj, ck;
  unit(c, ci, cj, ck);
  T rf = T(0.5) * (mat(g.rho, g, i - ci, j - cj, k - ck) + mat(g.rho, g, i, j, k));
  T att = g.att;
  if (g.ablL > T(0)) {
    T x = (T(i) + (c == 0 ? T(0) : T(0.5))) * g.h;
    T y = (T(j) + (c == 1 ? T(0) : T(0.5))) * g.h;
    T z = (T(k) + (c == 2 ? T(0) : T(0.5))) * g.h;
    att += g.ablG * (abl_axis(x, g.ablL, g.Lx) + abl_axis(y, g.ablL, g.Ly) + abl_axis(z, g.ablL, g.Lz)) / (g.ablL * g.ablL);
  }
  T a = rf * g.w2;
  return mkc<T>(a, -a * att);
}

// Transverse weights of Eq. dxSkew3D: beta at the centre line plus (1-beta)/16 [1 2 1]x[1 2 1].
template <typename T> HD T wt(T beta, int a, int b) {
  const T wa = a == 0 ? T(2) : T(1), wb = b == 0 ? T(2) : T(1);
  return (a == 0 && b == 0 ? beta : T(0)) + (T(1) - beta) * wa * wb * T(0.0625);
}

// beta-spread derivative along axis e of u_c, between the points q - s_e and q, where
// s_e = unit(e) and q = (i,j,k); spread over the two axes other than e.
template <typename T, typename TI>
HD cx<T> dspread(int c, int e, const cx<TI>* u, const Grid<T>& g, int i, int j, int k) {
  const int p = (e + 1) % 3, r = (e + 2) % 3;
  int ei, ej, ek, pi, pj, pk, ri, rj, rk;
  unit(e, ei, ej, ek);
  unit(p, pi, pj, pk);
  unit(r, ri, rj, rk);
  cx<T> acc = czero<T>();
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b) {
      const int oi = a * pi + b * ri, oj = a * pj + b * rj, ok = a * pk + b * rk;
      cx<T> dif = U(c, u, g, i + oi, j + oj, k + ok) - U(c, u, g, i + oi - ei, j + oj - ej, k + ok - ek);
      acc = acc + wt(g.beta, a, b) * dif;
    }
  return g.ih * acc;
}

// (H x) at the face u_c(i,j,k) (index along c >= 1).
template <typename T, typename TI>
HD cx<T> row_u(int c, const cx<TI>* u, const cx<TI>* p, const Grid<T>& g, int i, int j, int k) {
  int ci, cj, ck;
  unit(c, ci, cj, ck);
  // e == c: derivative lives at cell centres q - s_c and q
  cx<T> lap = mat(g.mu, g, i - ci, j - cj, k - ck) * dspread(c, c, u, g, i, j, k) -
              mat(g.mu, g, i, j, k) * dspread(c, c, u, g, i + ci, j + cj, k + ck);
  for (int e = 0; e < 3; ++e) {
    if (e == c) continue;
    int ei, ej, ek;
    unit(e, ei, ej, ek);
    lap = lap + mu_edge(g, c, e, i, j, k) * dspread(c, e, u, g, i, j, k) -
          mu_edge(g, c, e, i + ei, j + ej, k + ek) * dspread(c, e, u, g, i + ei, j + ej, k + ek);
  }
  lap = g.ih * lap;
  cx<T> nb = czero<T>();
  for (int a = 0; a < 3; ++a) {
    int ai, aj, ak;
    unit(a, ai, aj, ak);
    nb = nb + mcoef(g, c, i - ai, j - aj, k - ak) * U(c, u, g, i - ai, j - aj, k - ak) +
         mcoef(g, c, i + ai, j + aj, k + ak) * U(c, u, g, i + ai, j + aj, k + ak);
  }
  cx<T> mass = g.beta * (mcoef(g, c, i, j, k) * U(c, u, g, i, j, k)) + g.sm * nb;
  cx<T> grad = g.ih * (PP(p, g, i, j, k) - PP(p, g, i - ci, j - cj, k - ck));
  return lap - mass + grad;
}

// (H x) at the centre of cell (i,j,k): (div)^beta u + p/(lambda+mu). u[c] points to component c.
template <typename T, typename TI>
HD cx<T> row_p(const cx<TI>* const u[3], const cx<TI>* p, const Grid<T>& g, int i, int j, int k) {
  cx<T> d = dspread(0, 0, u[0], g, i + 1, j, k) + dspread(1, 1, u[1], g, i, j + 1, k) + dspread(2, 2, u[2], g, i, j, k + 1);
  return d + mat(g.cp, g, i, j, k) * PP(p, g, i, j, k);
}

// 2x2 Vanka block of u_c for the faces lo = u_c(q) and hi = u_c(q + s_c) of cell q
// (Remark 3.1): [d_lo o_lh; o_hl d_hi].
template <typename T>
HD void block_u(const Grid<T>& g, int c, int i, int j, int k, cx<T>& dlo, cx<T>& olh, cx<T>& ohl, cx<T>& dhi) {
  int ci, cj, ck;
  unit(c, ci, cj, ck);
  const T w00 = wt(g.beta, 0, 0), w10 = wt(g.beta, 1, 0);
  const T ih2 = g.ih * g.ih;
  const T mq = mat(g.mu, g, i, j, k);
  T elo = T(0), ehi = T(0);
  for (int e = 0; e < 3; ++e) {
    if (e == c) continue;
    int ei, ej, ek;
    unit(e, ei, ej, ek);
    elo += mu_edge(g, c, e, i, j, k) + mu_edge(g, c, e, i + ei, j + ej, k + ek);
    ehi += mu_edge(g, c, e, i + ci, j + cj, k + ck) + mu_edge(g, c, e, i + ci + ei, j + cj + ej, k + ck + ek);
  }
  cx<T> mlo = mcoef(g, c, i, j, k), mhi = mcoef(g, c, i + ci, j + cj, k + ck);
  dlo = mkc<T>(ih2 * w00 * (mat(g.mu, g, i - ci, j - cj, k - ck) + mq + elo), T(0)) - g.beta * mlo;
  dhi = mkc<T>(ih2 * w00 * (mq + mat(g.mu, g, i + ci, j + cj, k + ck) + ehi), T(0)) - g.beta * mhi;
  olh = mkc<T>(ih2 * (-w00 * mq + w10 * elo), T(0)) - g.sm * mhi;
  ohl = mkc<T>(ih2 * (-w00 * mq + w10 * ehi), T(0)) - g.sm * mlo;
}

}  // namespace s3
