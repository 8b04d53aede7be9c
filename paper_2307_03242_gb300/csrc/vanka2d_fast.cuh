// 2D red-black half-sweep with the cell's whole neighbourhood held in registers.
//
// Same arithmetic as k2::vanka (Eq. 3.10 rows with the sign of Eq. 4.4, the cell's 5x5 block of
// Sec. 2.3 solved by block elimination, Remark 3.1), but every input value is loaded once per
// thread and every shared quantity -- the six beta-spread derivatives of each component
// (Eq. 3.5), the node averages of mu, the face masses m_f u_f -- is computed once per cell.
// Thread layout: one thread per cell of the colour; a warp covers 32 cells of one grid row.
#pragma once
#include "kernels2d.cuh"

namespace k2 {

template <typename T> HD T abl_term(const Grid<T>& g, T x, T L) {
  return g.ablL > T(0) ? g.ablG * abl_axis(x, g.ablL, L) / (g.ablL * g.ablL) : T(0);
}

// ABL attenuation along axis a at lattice position k (half = 0) or k + 1/2 (half = 1).
template <typename T> HD T abl_at(const Grid<T>& g, int a, int k, int half, T L) {
  if (g.abl_tab[a]) return ldg(g.abl_tab[a] + 2 * (k + 2) + half);
  return abl_term(g, (T(k) + (half ? T(0.5) : T(0))) * g.h, L);
}

// INTERIOR: the caller guarantees 2 <= i <= nx-3 and 2 <= j <= ny-3 (no bounds checks, no clamps,
// no excluded faces). NOABL: the caller guarantees the attenuation is zero on lattice positions
// i-1 .. i+2 and j-1 .. j+2 (Grid::abl_free), so the absorbing-layer terms are dropped.
// COH: u and p are read through L2 (ldcg) because other blocks of the same launch wrote them
// before a grid-wide barrier (the cooperative coarse solve); otherwise u takes the read-only path.
template <typename T, bool INTERIOR = false, bool NOABL = false, bool COH = false>
HD void vanka_cell(const Grid<T>& g, const cx<T>* __restrict__ b, const cx<T>* __restrict__ uin,
                   cx<T>* __restrict__ uout, cx<T>* p, int colour, T w, int zero_in, int ip, int j) {
  const int nx = g.nx, ny = g.ny;
  if (j >= ny) return;
  const int par = (colour + j) & 1;
  const int i = 2 * ip + par;
  if (zero_in) {
    const int io = 2 * ip + 1 - par;
    if (io < nx) p[(size_t)j * nx + io] = czero<T>();
  }
  if (i >= nx) return;
  const size_t N = (size_t)nx * ny, k = (size_t)j * nx + i;
  auto ldu = [](const cx<T>* q) { return COH ? ldcg(q) : ldg(q); };
  auto ldp = [](const cx<T>* q) { return COH ? ldcg(q) : *q; };
  const cx<T>* u1 = uin;
  const cx<T>* u2 = uin + N;
  const T t0 = T(0.5) * (T(1) + g.beta), t1 = T(0.25) * (T(1) - g.beta);
  const T ih = g.ih, ih2 = g.ih * g.ih;
  const bool exW = INTERIOR ? false : i == 0, exE = INTERIOR ? false : i + 1 >= nx;
  const bool exS = INTERIOR ? false : j == 0, exN = INTERIOR ? false : j + 1 >= ny;

  // ---- material: mu on the 3x3 cells around (i, j); rho on the cells the face masses need
  auto cl = [&](int ii, int jj) -> size_t {
    if (INTERIOR) return (size_t)jj * nx + ii;
    return (size_t)iclamp(jj, 0, ny - 1) * nx + iclamp(ii, 0, nx - 1);
  };
  T mu9[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) mu9[r][c] = ldg(g.mu + cl(i - 1 + c, j - 1 + r));
  // node mu at (X, Y), X in {i, i+1}, Y in {j, j+1}: mean of cells (X-1..X, Y-1..Y)
  const T mnA = T(0.25) * (mu9[0][0] + mu9[0][1] + mu9[1][0] + mu9[1][1]);  // (i,   j)
  const T mnB = T(0.25) * (mu9[0][1] + mu9[0][2] + mu9[1][1] + mu9[1][2]);  // (i+1, j)
  const T mnC = T(0.25) * (mu9[1][0] + mu9[1][1] + mu9[2][0] + mu9[2][1]);  // (i,   j+1)
  const T mnD = T(0.25) * (mu9[1][1] + mu9[1][2] + mu9[2][1] + mu9[2][2]);  // (i+1, j+1)
  T R0[5], Rm[3], Rp[3];
#pragma unroll
  for (int c = 0; c < 5; ++c) R0[c] = ldg(g.rho + cl(i - 2 + c, j));
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Rm[c] = ldg(g.rho + cl(i - 1 + c, j - 1));
    Rp[c] = ldg(g.rho + cl(i - 1 + c, j + 1));
  }
  const T rS2 = ldg(g.rho + cl(i, j - 2)), rN2 = ldg(g.rho + cl(i, j + 2));
  // absorbing layer, separable in x and y: gx at face (X h) and cell ((X+1/2) h) positions, etc.
  T gxf[4], gxc[3], gyf[4], gyc[3];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    gxf[c] = NOABL ? T(0) : abl_at(g, 0, i - 1 + c, 0, g.Lx);
    gyf[c] = NOABL ? T(0) : abl_at(g, 1, j - 1 + c, 0, g.Ly);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    gxc[c] = NOABL ? T(0) : abl_at(g, 0, i - 1 + c, 1, g.Lx);
    gyc[c] = NOABL ? T(0) : abl_at(g, 1, j - 1 + c, 1, g.Ly);
  }
  const T w2 = g.w2, att = g.att;
  // m1 at u1 face (X, Y) with rho_f = (rho(X-1,Y) + rho(X,Y))/2; offsets relative to (i, j)
  auto m1 = [&](T rf, int ox, int oy) -> cx<T> {
    T a = rf * w2;
    return mkc<T>(a, -a * (att + gxf[ox + 1] + gyc[oy + 1]));
  };
  auto m2 = [&](T rf, int ox, int oy) -> cx<T> {
    T a = rf * w2;
    return mkc<T>(a, -a * (att + gxc[ox + 1] + gyf[oy + 1]));
  };
  const T h5 = T(0.5);
  const cx<T> mW = m1(h5 * (R0[1] + R0[2]), 0, 0), mE = m1(h5 * (R0[2] + R0[3]), 1, 0);
  const cx<T> mS = m2(h5 * (Rm[1] + R0[2]), 0, 0), mN = m2(h5 * (R0[2] + Rp[1]), 0, 1);

  cx<T> r[5];
  const cx<T> z = czero<T>();
  if (zero_in) {
    r[0] = exW ? z : b[k];
    r[1] = exE ? z : b[k + 1];
    r[2] = exS ? z : b[N + k];
    r[3] = exN ? z : b[N + k + nx];
    r[4] = b[2 * N + k];
  } else {
    const cx<T> pC = ldp(p + k);
    const cx<T> pW = (INTERIOR || i > 0) ? ldp(p + k - 1) : z, pE = (INTERIOR || i + 1 < nx) ? ldp(p + k + 1) : z;
    const cx<T> pS = (INTERIOR || j > 0) ? ldp(p + k - nx) : z, pN = (INTERIOR || j + 1 < ny) ? ldp(p + k + nx) : z;
    cx<T> G1m, G1c, G1p;  // d1 u1 at cells i-1, i, i+1 (needed by the p row too)
    {
      // u1 on faces i-1..i+2, rows j-1..j+1
      cx<T> A[3][4];
#pragma unroll
      for (int rr = 0; rr < 3; ++rr) {
        const int jj = j - 1 + rr;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int ii = i - 1 + c;
          A[rr][c] = (INTERIOR || (ii >= 1 && ii < nx && jj >= 0 && jj < ny)) ? ldu(u1 + (size_t)jj * nx + ii) : z;
        }
      }
      auto g1 = [&](int c) { return ih * (t1 * ((A[0][c + 1] - A[0][c]) + (A[2][c + 1] - A[2][c])) + t0 * (A[1][c + 1] - A[1][c])); };
      // node derivative at (X = i-1+cx0+1, Y): rows ry (Y) and ry-1
      auto g2 = [&](int c0, int ry) {
        return ih * (t1 * ((A[ry][c0] - A[ry - 1][c0]) + (A[ry][c0 + 2] - A[ry - 1][c0 + 2])) + t0 * (A[ry][c0 + 1] - A[ry - 1][c0 + 1]));
      };
      G1m = g1(0);
      G1c = g1(1);
      G1p = g1(2);
      const cx<T> G2A = g2(0, 1), G2C = g2(0, 2), G2B = g2(1, 1), G2D = g2(1, 2);
      const cx<T> lapW = ih * (mu9[1][0] * G1m - mu9[1][1] * G1c + mnA * G2A - mnC * G2C);
      const cx<T> lapE = ih * (mu9[1][1] * G1c - mu9[1][2] * G1p + mnB * G2B - mnD * G2D);
      cx<T> massW, massE;  // the spread face-mass terms of the two u1 rows
      if (NOABL) {
        // every face mass is rho_f omega^2 (1 - i att): weight u by the density sums first and
        // scale by the common complex factor once
        const cx<T> cm = mkc<T>(h5 * w2, -(h5 * w2) * att);
        const cx<T> Vw = (R0[1] + R0[2]) * A[1][1], Ve = (R0[2] + R0[3]) * A[1][2];
        const cx<T> Vww = (R0[0] + R0[1]) * A[1][0], Vee = (R0[3] + R0[4]) * A[1][3];
        const cx<T> Vws = (Rm[0] + Rm[1]) * A[0][1], Vwn = (Rp[0] + Rp[1]) * A[2][1];
        const cx<T> Ves = (Rm[1] + Rm[2]) * A[0][2], Ven = (Rp[1] + Rp[2]) * A[2][2];
        massW = cm * (g.beta * Vw + g.sm * (Vww + Ve + Vws + Vwn));
        massE = cm * (g.beta * Ve + g.sm * (Vw + Vee + Ves + Ven));
      } else {
        // face masses m u at the u1 faces the two rows need
        const cx<T> MUw = mW * A[1][1], MUe = mE * A[1][2];
        const cx<T> MUww = m1(h5 * (R0[0] + R0[1]), -1, 0) * A[1][0];
        const cx<T> MUee = m1(h5 * (R0[3] + R0[4]), 2, 0) * A[1][3];
        const cx<T> MUws = m1(h5 * (Rm[0] + Rm[1]), 0, -1) * A[0][1];
        const cx<T> MUwn = m1(h5 * (Rp[0] + Rp[1]), 0, 1) * A[2][1];
        const cx<T> MUes = m1(h5 * (Rm[1] + Rm[2]), 1, -1) * A[0][2];
        const cx<T> MUen = m1(h5 * (Rp[1] + Rp[2]), 1, 1) * A[2][2];
        massW = g.beta * MUw + g.sm * (MUww + MUe + MUws + MUwn);
        massE = g.beta * MUe + g.sm * (MUw + MUee + MUes + MUen);
      }
      r[0] = exW ? z : b[k] - (lapW - massW + ih * (pC - pW));
      r[1] = exE ? z : b[k + 1] - (lapE - massE + ih * (pE - pC));
    }
    cx<T> H2c;
    {
      // u2 on faces rows j-1..j+2, columns i-1..i+1
      cx<T> B[4][3];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int jj = j - 1 + rr;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int ii = i - 1 + c;
          B[rr][c] = (INTERIOR || (jj >= 1 && jj < ny && ii >= 0 && ii < nx)) ? ldu(u2 + (size_t)jj * nx + ii) : z;
        }
      }
      // d2 u2 at cell (i, Y): rows ry+1 (Y+1) and ry (Y)
      auto h2 = [&](int ry) { return ih * (t1 * ((B[ry + 1][0] - B[ry][0]) + (B[ry + 1][2] - B[ry][2])) + t0 * (B[ry + 1][1] - B[ry][1])); };
      // d1 u2 at node (X, Y): columns cx0+1 (X) and cx0 (X-1), rows ry-1..ry+1 (Y-1..Y+1)
      auto h1 = [&](int c0, int ry) {
        return ih * (t1 * ((B[ry - 1][c0 + 1] - B[ry - 1][c0]) + (B[ry + 1][c0 + 1] - B[ry + 1][c0])) + t0 * (B[ry][c0 + 1] - B[ry][c0]));
      };
      const cx<T> H2m = h2(0);
      H2c = h2(1);
      const cx<T> H2p = h2(2);
      const cx<T> H1A = h1(0, 1), H1B = h1(1, 1), H1C = h1(0, 2), H1D = h1(1, 2);
      const cx<T> lapS = ih * (mnA * H1A - mnB * H1B + mu9[0][1] * H2m - mu9[1][1] * H2c);
      const cx<T> lapN = ih * (mnC * H1C - mnD * H1D + mu9[1][1] * H2c - mu9[2][1] * H2p);
      cx<T> massS, massN;  // the spread face-mass terms of the two u2 rows
      if (NOABL) {
        const cx<T> cm = mkc<T>(h5 * w2, -(h5 * w2) * att);
        const cx<T> Vs = (Rm[1] + R0[2]) * B[1][1], Vn = (R0[2] + Rp[1]) * B[2][1];
        const cx<T> Vss = (rS2 + Rm[1]) * B[0][1], Vnn = (Rp[1] + rN2) * B[3][1];
        const cx<T> Vsw = (Rm[0] + R0[1]) * B[1][0], Vse = (Rm[2] + R0[3]) * B[1][2];
        const cx<T> Vnw = (R0[1] + Rp[0]) * B[2][0], Vne = (R0[3] + Rp[2]) * B[2][2];
        massS = cm * (g.beta * Vs + g.sm * (Vsw + Vse + Vss + Vn));
        massN = cm * (g.beta * Vn + g.sm * (Vnw + Vne + Vs + Vnn));
      } else {
        const cx<T> MUs = mS * B[1][1], MUn = mN * B[2][1];
        const cx<T> MUss = m2(h5 * (rS2 + Rm[1]), 0, -1) * B[0][1];
        const cx<T> MUnn = m2(h5 * (Rp[1] + rN2), 0, 2) * B[3][1];
        const cx<T> MUsw = m2(h5 * (Rm[0] + R0[1]), -1, 0) * B[1][0];
        const cx<T> MUse = m2(h5 * (Rm[2] + R0[3]), 1, 0) * B[1][2];
        const cx<T> MUnw = m2(h5 * (R0[1] + Rp[0]), -1, 1) * B[2][0];
        const cx<T> MUne = m2(h5 * (R0[3] + Rp[2]), 1, 1) * B[2][2];
        massS = g.beta * MUs + g.sm * (MUsw + MUse + MUss + MUn);
        massN = g.beta * MUn + g.sm * (MUnw + MUne + MUs + MUnn);
      }
      r[2] = exS ? z : b[N + k] - (lapS - massS + ih * (pC - pS));
      r[3] = exN ? z : b[N + k + nx] - (lapN - massN + ih * (pN - pC));
    }
    r[4] = b[2 * N + k] - (G1c + H2c + ldg(g.cp + k) * pC);
  }

  // ---- the cell's block (same entries as s2::block_u1 / block_u2)
  cx<T> a1[4], a2[4], d[5];
  const T mc = mu9[1][1];
  a1[0] = mkc<T>(t0 * ih2 * (mu9[1][0] + mc + mnA + mnC), T(0)) - g.beta * mW;
  a1[3] = mkc<T>(t0 * ih2 * (mc + mu9[1][2] + mnB + mnD), T(0)) - g.beta * mE;
  a1[1] = mkc<T>(ih2 * (-t0 * mc + t1 * (mnA + mnC)), T(0)) - g.sm * mE;
  a1[2] = mkc<T>(ih2 * (-t0 * mc + t1 * (mnB + mnD)), T(0)) - g.sm * mW;
  a2[0] = mkc<T>(t0 * ih2 * (mnA + mnB + mu9[0][1] + mc), T(0)) - g.beta * mS;
  a2[3] = mkc<T>(t0 * ih2 * (mnC + mnD + mc + mu9[2][1]), T(0)) - g.beta * mN;
  a2[1] = mkc<T>(ih2 * (-t0 * mc + t1 * (mnA + mnB)), T(0)) - g.sm * mN;
  a2[2] = mkc<T>(ih2 * (-t0 * mc + t1 * (mnC + mnD)), T(0)) - g.sm * mS;
  if (g.economic) a1[1] = a1[2] = a2[1] = a2[2] = czero<T>();
  const bool ex[4] = {exW, exE, exS, exN};
  cell_solve(a1, a2, ex, ih, t0, ldg(g.cp + k), r, d);

  cx<T>* o1 = uout;
  cx<T>* o2 = uout + N;
  if (zero_in) {
    o1[k] = exW ? z : w * d[0];
    if (!exE) o1[k + 1] = w * d[1];
    o2[k] = exS ? z : w * d[2];
    if (!exN) o2[k + nx] = w * d[3];
    p[k] = w * d[4];
  } else {
    o1[k] = exW ? z : ldu(u1 + k) + w * d[0];
    if (!exE) o1[k + 1] = ldu(u1 + k + 1) + w * d[1];
    o2[k] = exS ? z : ldu(u2 + k) + w * d[2];
    if (!exN) o2[k + nx] = ldu(u2 + k + nx) + w * d[3];
    p[k] = ldp(p + k) + w * d[4];
  }
  if (!INTERIOR && i == 1) o1[k - 1] = z;
  if (!INTERIOR && j == 1) o2[k - nx] = z;
}

template <typename T>
__global__ void __launch_bounds__(BX * BY, sizeof(T) == 4 ? 2 : 1) vanka_fast(Grid<T> g, const cx<T>* __restrict__ b,
                                                                             const cx<T>* __restrict__ uin,
                                                                             cx<T>* __restrict__ uout, cx<T>* p, int colour,
                                                                             T w, int zero_in) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int ip = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int i = 2 * ip + ((colour + j) & 1);
  if (!zero_in && i >= 2 && i + 3 <= g.nx && j >= 2 && j + 3 <= g.ny) {
    if (g.abl_free(0, i - 1, i + 2) && g.abl_free(1, j - 1, j + 2))
      vanka_cell<T, true, true>(g, b, uin, uout, p, colour, w, zero_in, ip, j);
    else
      vanka_cell<T, true>(g, b, uin, uout, p, colour, w, zero_in, ip, j);
  } else
    vanka_cell<T, false>(g, b, uin, uout, p, colour, w, zero_in, ip, j);
}

}  // namespace k2
