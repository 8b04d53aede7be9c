// 2D residual r = b - H_s x with one thread per fine cell (its u1 row, u2 row and p row), and the
// restriction b_c = R r from that residual (Eq. 2.11-2.13). Used where the fused per-coarse-cell
// kernel is latency-bound (small levels): four times as many threads, each with a short chain.
#pragma once
#include "vanka2d_fast.cuh"

namespace k2 {

// INTERIOR: 2 <= i <= nx-3 and 2 <= j <= ny-3. NOABL: zero attenuation on i-1 .. i+2, j-1 .. j+2.
template <typename T, bool INTERIOR = false, bool NOABL = false>
HD void residual_cell(const Grid<T>& g, const cx<T>* __restrict__ b, const cx<T>* __restrict__ x, cx<T>* __restrict__ r,
                      int i, int j) {
  const int nx = g.nx, ny = g.ny;
  const size_t N = (size_t)nx * ny, k = (size_t)j * nx + i;
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
  auto P = [&](int ii, int jj) -> cx<T> {
    return (INTERIOR || (ii >= 0 && ii < nx && jj >= 0 && jj < ny)) ? ldg(p + (size_t)jj * nx + ii) : z;
  };
  T mu9[3][3];
#pragma unroll
  for (int rr = 0; rr < 3; ++rr)
#pragma unroll
    for (int c = 0; c < 3; ++c) mu9[rr][c] = MU(i - 1 + c, j - 1 + rr);
  const T mnA = T(0.25) * (mu9[0][0] + mu9[0][1] + mu9[1][0] + mu9[1][1]);  // node (i, j)
  const T mnB = T(0.25) * (mu9[0][1] + mu9[0][2] + mu9[1][1] + mu9[1][2]);  // node (i+1, j)
  const T mnC = T(0.25) * (mu9[1][0] + mu9[1][1] + mu9[2][0] + mu9[2][1]);  // node (i, j+1)
  auto m1 = [&](int ii, int jj) -> cx<T> {
    const T a = h5 * (RHO(ii - 1, jj) + RHO(ii, jj)) * w2;
    return mkc<T>(a, NOABL ? -a * att : -a * (att + abl_at(g, 0, ii, 0, g.Lx) + abl_at(g, 1, jj, 1, g.Ly)));
  };
  auto m2 = [&](int ii, int jj) -> cx<T> {
    const T a = h5 * (RHO(ii, jj - 1) + RHO(ii, jj)) * w2;
    return mkc<T>(a, NOABL ? -a * att : -a * (att + abl_at(g, 0, ii, 1, g.Lx) + abl_at(g, 1, jj, 0, g.Ly)));
  };
  const cx<T> pC = P(i, j);
  cx<T> G1c, H2c;
  {
    cx<T> A[3][3];  // u1 faces i-1..i+1, rows j-1..j+1
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int ii = i - 1 + c, jj = j - 1 + rr;
        A[rr][c] = (INTERIOR || (ii >= 1 && ii < nx && jj >= 0 && jj < ny)) ? ldg(u1 + (size_t)jj * nx + ii) : z;
      }
    auto g1 = [&](int c) {  // d1 u1 at cell (i-1+c, j), faces c, c+1
      return ih * (t1 * ((A[0][c + 1] - A[0][c]) + (A[2][c + 1] - A[2][c])) + t0 * (A[1][c + 1] - A[1][c]));
    };
    auto g2 = [&](int ry) {  // d2 u1 at node (i, j-1+ry), rows ry, ry-1
      return ih * (t1 * ((A[ry][0] - A[ry - 1][0]) + (A[ry][2] - A[ry - 1][2])) + t0 * (A[ry][1] - A[ry - 1][1]));
    };
    const cx<T> G1m = g1(0);
    G1c = g1(1);
    if (INTERIOR || i >= 1) {
      const cx<T> lap = ih * (mu9[1][0] * G1m - mu9[1][1] * G1c + mnA * g2(1) - mnC * g2(2));
      cx<T> mass;
      if (NOABL) {  // every face mass is rho_f omega^2 (1 - i att): one complex scaling at the end
        auto rs = [&](int ii, int jj) { return RHO(ii - 1, jj) + RHO(ii, jj); };
        mass = mkc<T>(h5 * w2, -(h5 * w2) * att) *
               (g.beta * (rs(i, j) * A[1][1]) +
                g.sm * (rs(i - 1, j) * A[1][0] + rs(i + 1, j) * A[1][2] + rs(i, j - 1) * A[0][1] + rs(i, j + 1) * A[2][1]));
      } else {
        mass = g.beta * (m1(i, j) * A[1][1]) +
               g.sm * (m1(i - 1, j) * A[1][0] + m1(i + 1, j) * A[1][2] + m1(i, j - 1) * A[0][1] + m1(i, j + 1) * A[2][1]);
      }
      r[k] = ldg(b + k) - (lap - mass + ih * (pC - P(i - 1, j)));
    } else {
      r[k] = z;
    }
  }
  {
    cx<T> B[3][3];  // u2 faces rows j-1..j+1, columns i-1..i+1
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int ii = i - 1 + c, jj = j - 1 + rr;
        B[rr][c] = (INTERIOR || (jj >= 1 && jj < ny && ii >= 0 && ii < nx)) ? ldg(u2 + (size_t)jj * nx + ii) : z;
      }
    auto h2 = [&](int ry) {  // d2 u2 at cell (i, j-1+ry), rows ry, ry+1
      return ih * (t1 * ((B[ry + 1][0] - B[ry][0]) + (B[ry + 1][2] - B[ry][2])) + t0 * (B[ry + 1][1] - B[ry][1]));
    };
    auto h1 = [&](int c0) {  // d1 u2 at node (i-1+c0+1, j), columns c0+1, c0
      return ih * (t1 * ((B[0][c0 + 1] - B[0][c0]) + (B[2][c0 + 1] - B[2][c0])) + t0 * (B[1][c0 + 1] - B[1][c0]));
    };
    const cx<T> H2m = h2(0);
    H2c = (INTERIOR || j + 1 < ny) ? h2(1) : ih * (t1 * ((z - B[1][0]) + (z - B[1][2])) + t0 * (z - B[1][1]));
    if (INTERIOR || j >= 1) {
      const cx<T> lap = ih * (mnA * h1(0) - mnB * h1(1) + mu9[0][1] * H2m - mu9[1][1] * H2c);
      cx<T> mass;
      if (NOABL) {
        auto rs = [&](int ii, int jj) { return RHO(ii, jj - 1) + RHO(ii, jj); };
        mass = mkc<T>(h5 * w2, -(h5 * w2) * att) *
               (g.beta * (rs(i, j) * B[1][1]) +
                g.sm * (rs(i - 1, j) * B[1][0] + rs(i + 1, j) * B[1][2] + rs(i, j - 1) * B[0][1] + rs(i, j + 1) * B[2][1]));
      } else {
        mass = g.beta * (m2(i, j) * B[1][1]) +
               g.sm * (m2(i - 1, j) * B[1][0] + m2(i + 1, j) * B[1][2] + m2(i, j - 1) * B[0][1] + m2(i, j + 1) * B[2][1]);
      }
      r[N + k] = ldg(b + N + k) - (lap - mass + ih * (pC - P(i, j - 1)));
    } else {
      r[N + k] = z;
    }
  }
  r[2 * N + k] = ldg(b + 2 * N + k) - (G1c + H2c + ldg(g.cp + k) * pC);
}

// Four blocks of 256 per SM (64 registers, a few spilled): the kernel is latency-bound, and the
// extra warps hide more than the spills cost (2048^2 residual + restriction 137 -> 124 us).
template <typename T>
__global__ void __launch_bounds__(BX * BY, 4) residual_fast(Grid<T> g, const cx<T>* __restrict__ b,
                                                        const cx<T>* __restrict__ x, cx<T>* __restrict__ r) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  if (i >= 2 && i + 3 <= g.nx && j >= 2 && j + 3 <= g.ny) {
    if (g.abl_free(0, i - 1, i + 2) && g.abl_free(1, j - 1, j + 2))
      residual_cell<T, true, true>(g, b, x, r, i, j);
    else
      residual_cell<T, true>(g, b, x, r, i, j);
  } else
    residual_cell<T, false>(g, b, x, r, i, j);
}

// b_c = R r: one thread per coarse cell (I, J) reading 6 + 6 + 4 fine residuals.
template <typename T>
HD void restrict_r_cell(const cx<T>* __restrict__ r, cx<T>* __restrict__ bc, int nx, int ny, int nxc, int nyc, int I,
                        int J) {
  const size_t N = (size_t)nx * ny, Nc = (size_t)nxc * nyc, kc = (size_t)J * nxc + I;
  const int i0 = 2 * I, j0 = 2 * J;
  auto R = [&](int c, int ii, int jj) { return ldg(r + c * N + (size_t)jj * nx + ii); };
  cx<T> c1 = czero<T>(), c2 = czero<T>();
  if (I >= 1) {
    for (int bb = 0; bb < 2; ++bb) c1 = c1 + R(0, i0 - 1, j0 + bb) + T(2) * R(0, i0, j0 + bb) + R(0, i0 + 1, j0 + bb);
    c1 = T(0.125) * c1;
  }
  if (J >= 1) {
    for (int a = 0; a < 2; ++a) c2 = c2 + R(1, i0 + a, j0 - 1) + T(2) * R(1, i0 + a, j0) + R(1, i0 + a, j0 + 1);
    c2 = T(0.125) * c2;
  }
  const cx<T> cp = T(0.25) * (R(2, i0, j0) + R(2, i0 + 1, j0) + R(2, i0, j0 + 1) + R(2, i0 + 1, j0 + 1));
  bc[kc] = c1;
  bc[Nc + kc] = c2;
  bc[2 * Nc + kc] = cp;
}

template <typename T>
__global__ void __launch_bounds__(BX * BY) restrict_r(const cx<T>* __restrict__ r, cx<T>* __restrict__ bc, int nx, int ny,
                                                     int nxc, int nyc) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int I = blockIdx.x * BX + threadIdx.x;
  const int J = blockIdx.y * BY + threadIdx.y;
  if (I >= nxc || J >= nyc) return;
  restrict_r_cell(r, bc, nx, ny, nxc, nyc, I, J);
}

}  // namespace k2
