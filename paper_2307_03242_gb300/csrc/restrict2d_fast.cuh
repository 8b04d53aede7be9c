// 2D fused residual + restriction with the fine neighbourhood of one coarse cell in registers.
//
// Same result as k2::restrict_residual: b_c = R (b - H_s x) with R_u1 = [1 2 1]/4 along x1 x
// [1 1]/2 along x2, R_u2 rotated, R_p the mean of the 4 children (Eq. 2.11-2.13); the fine rows
// are Eq. 3.10 with the sign of Eq. 4.4. One thread per coarse cell (I, J); the fine u1 values on
// faces 2I-2..2I+2, rows 2J-1..2J+2 and the u2 values on columns 2I-1..2I+2, rows 2J-2..2J+2 are
// loaded once; derivatives shared by neighbouring fine rows are computed once.
#pragma once
#include "vanka2d_fast.cuh"

namespace k2 {

// INTERIOR: the caller guarantees the fine window (cells 2I-3 .. 2I+3, 2J-3 .. 2J+3) lies inside
// the grid, so no bounds checks or clamps are needed.
template <typename T, bool INTERIOR = false>
HD void restrict_cell(const Grid<T>& g, const cx<T>* __restrict__ b, const cx<T>* __restrict__ x,
                      cx<T>* __restrict__ bc, int nxc, int nyc, int I, int J) {
  const int nx = g.nx, ny = g.ny;
  const size_t N = (size_t)nx * ny, Nc = (size_t)nxc * nyc, kc = (size_t)J * nxc + I;
  const int i0 = 2 * I, j0 = 2 * J;
  const cx<T>* u1 = x;
  const cx<T>* u2 = x + N;
  const cx<T>* p = x + 2 * N;
  const T t0 = T(0.5) * (T(1) + g.beta), t1 = T(0.25) * (T(1) - g.beta);
  const T ih = g.ih, w2 = g.w2, att = g.att, h5 = T(0.5);
  const cx<T> z = czero<T>();
  auto cl = [&](int ii, int jj) -> size_t {
    if (INTERIOR) return (size_t)jj * nx + ii;
    return (size_t)iclamp(jj, 0, ny - 1) * nx + iclamp(ii, 0, nx - 1);
  };
  auto MU = [&](int ii, int jj) -> T { return ldg(g.mu + cl(ii, jj)); };
  auto RHO = [&](int ii, int jj) -> T { return ldg(g.rho + cl(ii, jj)); };
  auto MUN = [&](int X, int Y) -> T { return T(0.25) * (MU(X - 1, Y - 1) + MU(X, Y - 1) + MU(X - 1, Y) + MU(X, Y)); };
  auto P = [&](int ii, int jj) -> cx<T> {
    return (INTERIOR || (ii >= 0 && ii < nx && jj >= 0 && jj < ny)) ? ldg(p + (size_t)jj * nx + ii) : z;
  };
  auto m1 = [&](int ii, int jj) -> cx<T> {
    const T a = h5 * (RHO(ii - 1, jj) + RHO(ii, jj)) * w2;
    const T at = att + abl_at(g, 0, ii, 0, g.Lx) + abl_at(g, 1, jj, 1, g.Ly);
    return mkc<T>(a, -a * at);
  };
  auto m2 = [&](int ii, int jj) -> cx<T> {
    const T a = h5 * (RHO(ii, jj - 1) + RHO(ii, jj)) * w2;
    const T at = att + abl_at(g, 0, ii, 1, g.Lx) + abl_at(g, 1, jj, 0, g.Ly);
    return mkc<T>(a, -a * at);
  };
  cx<T> G1c[2][2], H2c[2][2];  // d1 u1 and d2 u2 at the 4 child cells (rows j0..j0+1, cols i0..i0+1)
  cx<T> c1 = z, c2 = z;
  {
    // u1 faces i0-2..i0+2 (col c = i - (i0-2)), rows j0-1..j0+2 (row r = j - (j0-1))
    cx<T> A[4][5];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int jj = j0 - 1 + r;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const int ii = i0 - 2 + c;
        A[r][c] = (INTERIOR || (ii >= 1 && ii < nx && jj >= 0 && jj < ny)) ? ldg(u1 + (size_t)jj * nx + ii) : z;
      }
    }
    // d1 u1 at cell (i0-2+c, j0-1+r) uses faces c, c+1 (c = 0..3), rows r-1..r+1 (r = 1, 2)
    auto g1 = [&](int r, int c) {
      return ih * (t1 * ((A[r - 1][c + 1] - A[r - 1][c]) + (A[r + 1][c + 1] - A[r + 1][c])) + t0 * (A[r][c + 1] - A[r][c]));
    };
    // d2 u1 at node (X = i0-2+c, Y = j0-1+r) uses rows r, r-1, columns c-1..c+1
    auto g2 = [&](int r, int c) {
      return ih * (t1 * ((A[r][c - 1] - A[r - 1][c - 1]) + (A[r][c + 1] - A[r - 1][c + 1])) + t0 * (A[r][c] - A[r - 1][c]));
    };
    cx<T> G1[2][4], G2[3][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) G1[r][c] = g1(r + 1, c);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) G2[r][c] = g2(r + 1, c + 1);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      G1c[r][0] = G1[r][2];
      G1c[r][1] = G1[r][3];
    }
    if (INTERIOR || I >= 1) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int j = j0 + r;
#pragma unroll
        for (int q = 0; q < 3; ++q) {   // faces i = i0-1+q, A column c = q+1
          const int i = i0 - 1 + q, c = q + 1, ra = r + 1;
          const cx<T> lap = ih * (MU(i - 1, j) * G1[r][q] - MU(i, j) * G1[r][q + 1] + MUN(i, j) * G2[r][q] -
                                  MUN(i, j + 1) * G2[r + 1][q]);
          const cx<T> mass = g.beta * (m1(i, j) * A[ra][c]) +
                             g.sm * (m1(i - 1, j) * A[ra][c - 1] + m1(i + 1, j) * A[ra][c + 1] + m1(i, j - 1) * A[ra - 1][c] +
                                     m1(i, j + 1) * A[ra + 1][c]);
          const cx<T> res = b[(size_t)j * nx + i] - (lap - mass + ih * (P(i, j) - P(i - 1, j)));
          c1 = c1 + (q == 1 ? T(2) : T(1)) * res;
        }
      }
      c1 = T(0.125) * c1;
    }
  }
  {
    // u2 faces: columns i0-1..i0+2 (col c = i - (i0-1)), rows j0-2..j0+2 (row r = j - (j0-2))
    cx<T> B[5][4];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const int jj = j0 - 2 + r;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int ii = i0 - 1 + c;
        B[r][c] = (INTERIOR || (jj >= 1 && jj < ny && ii >= 0 && ii < nx)) ? ldg(u2 + (size_t)jj * nx + ii) : z;
      }
    }
    // d2 u2 at cell (X = i0-1+c, Y = j0-2+r) uses rows r, r+1 (r = 0..3), columns c-1..c+1 (c = 1, 2)
    auto h2 = [&](int r, int c) {
      return ih * (t1 * ((B[r + 1][c - 1] - B[r][c - 1]) + (B[r + 1][c + 1] - B[r][c + 1])) + t0 * (B[r + 1][c] - B[r][c]));
    };
    // d1 u2 at node (X = i0-1+c, Y = j0-2+r) uses columns c, c-1, rows r-1..r+1
    auto h1 = [&](int r, int c) {
      return ih * (t1 * ((B[r - 1][c] - B[r - 1][c - 1]) + (B[r + 1][c] - B[r + 1][c - 1])) + t0 * (B[r][c] - B[r][c - 1]));
    };
    cx<T> H2[4][2], H1[3][3];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) H2[r][c] = h2(r, c + 1);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) H1[r][c] = h1(r + 1, c + 1);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      H2c[0][c] = H2[2][c];
      H2c[1][c] = H2[3][c];
    }
    if (INTERIOR || J >= 1) {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int i = i0 + a;
#pragma unroll
        for (int q = 0; q < 3; ++q) {   // faces j = j0-1+q, B row r = q+1
          const int j = j0 - 1 + q, r = q + 1, cb = a + 1;
          const cx<T> lap = ih * (MUN(i, j) * H1[q][a] - MUN(i + 1, j) * H1[q][a + 1] + MU(i, j - 1) * H2[q][a] -
                                  MU(i, j) * H2[q + 1][a]);
          const cx<T> mass = g.beta * (m2(i, j) * B[r][cb]) +
                             g.sm * (m2(i - 1, j) * B[r][cb - 1] + m2(i + 1, j) * B[r][cb + 1] + m2(i, j - 1) * B[r - 1][cb] +
                                     m2(i, j + 1) * B[r + 1][cb]);
          const cx<T> res = b[N + (size_t)j * nx + i] - (lap - mass + ih * (P(i, j) - P(i, j - 1)));
          c2 = c2 + (q == 1 ? T(2) : T(1)) * res;
        }
      }
      c2 = T(0.125) * c2;
    }
  }
  cx<T> cpv = z;
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const size_t k = (size_t)(j0 + r) * nx + i0 + a;
      cpv = cpv + (b[2 * N + k] - (G1c[r][a] + H2c[r][a] + ldg(g.cp + k) * p[k]));
    }
  bc[kc] = c1;
  bc[Nc + kc] = c2;
  bc[2 * Nc + kc] = T(0.25) * cpv;
}

template <typename T>
__global__ void __launch_bounds__(BX * BY, sizeof(T) == 4 ? 2 : 1) restrict_fast(Grid<T> g, const cx<T>* __restrict__ b,
                                                                                const cx<T>* __restrict__ x,
                                                                                cx<T>* __restrict__ bc, int nxc, int nyc) {
  const int I = blockIdx.x * BX + threadIdx.x;
  const int J = blockIdx.y * BY + threadIdx.y;
  if (I >= nxc || J >= nyc) return;
  if (2 * I >= 3 && 2 * I + 4 <= g.nx && 2 * J >= 3 && 2 * J + 4 <= g.ny)
    restrict_cell<T, true>(g, b, x, bc, nxc, nyc, I, J);
  else
    restrict_cell<T, false>(g, b, x, bc, nxc, nyc, I, J);
}

}  // namespace k2
