// 3D residual r = b - H_s x with one thread per fine cell (its three face rows and its pressure
// row, Eq. 3.10 with the 3D spread derivatives and mass of Sec. 5.3 and the sign of Eq. 4.4),
// and the restriction b_c = R r from that residual (3D tensor-product transfer: R_u_c =
// [1 2 1]/4 along c x [1 1]/2 x [1 1]/2, R_p the mean of the 8 children). Each fine row is
// evaluated once; a kernel with one thread per coarse cell evaluates the rows it needs itself,
// about 1.4 times each, on an 8 times smaller grid of threads.
#pragma once
#include "kernels3d.cuh"

namespace k3 {

// Attenuation of the absorbing layer along axis a at lattice position kk (half = 0) or kk + 1/2
// (half = 1): the level's table, or the profile itself when there is none.
template <typename T> HD T abl3(const Grid<T>& g, int a, int kk, int half) {
  if (g.abl_tab[a]) return ldg(g.abl_tab[a] + 2 * (kk + 2) + half);
  if (!(g.ablL > T(0))) return T(0);
  const T L = a == 0 ? g.Lx : (a == 1 ? g.Ly : g.Lz);
  return g.ablG * abl_axis((T(kk) + (half ? T(0.5) : T(0))) * g.h, g.ablL, L) / (g.ablL * g.ablL);
}

// The four rows of an interior cell (2 <= i <= nx-3, likewise j, k), the same arithmetic as
// s3::row_u / s3::row_p, with every value loaded once: a 3x3x3 cube of mu around the cell, per
// component a 3x3x3 cube of u_c around the face u_c(i,j,k) (its 27-point stencil), the density of
// the cells the seven face masses need, and p on the cell and its three low neighbours.
// NOABL: the attenuation is zero on lattice positions i-1 .. i+2 (likewise j, k).
template <typename T, bool NOABL>
HD void residual_cell3(const Grid<T>& g, const cx<T>* __restrict__ b, const cx<T>* __restrict__ x,
                       cx<T>* __restrict__ r, int i, int j, int k) {
  const int nx = g.nx, ny = g.ny;
  const size_t N = (size_t)nx * ny * g.nz, sy = (size_t)nx, sz = (size_t)nx * ny;
  const size_t q = (size_t)k * sz + (size_t)j * sy + i;
  const size_t st[3] = {1, sy, sz};
  const cx<T>* p = x + 3 * N;
  const T ih = g.ih, w2 = g.w2, att = g.att, h5 = T(0.5);
  T MU[3][3][3];  // mu at cell q + (di, dj, dk), indexed [dk+1][dj+1][di+1]
#pragma unroll
  for (int dk = -1; dk <= 1; ++dk)
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
      for (int di = -1; di <= 1; ++di) MU[dk + 1][dj + 1][di + 1] = ldg(g.mu + q + dk * sz + dj * sy + di);
  auto mu_at = [&](const int o[3]) { return MU[o[2] + 1][o[1] + 1][o[0] + 1]; };
  const cx<T> pq = ldg(p + q);
  const int pos[3] = {i, j, k};
  cx<T> div = czero<T>();  // (div)^beta u at the cell centre, built component by component
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<T>* uc = x + c * N;
    cx<T> U[3][3][3];  // u_c at face q + (di, dj, dk)
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk)
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
        for (int di = -1; di <= 1; ++di) U[dk + 1][dj + 1][di + 1] = ldg(uc + q + dk * sz + dj * sy + di);
    auto u_at = [&](const int o[3]) { return U[o[2] + 1][o[1] + 1][o[0] + 1]; };
    // beta-spread derivative along e between face planes s-1 and s (s = 0: at q, s = 1: at q + s_e)
    auto dsp = [&](int e, int s) {
      const int pa = (e + 1) % 3, ra = (e + 2) % 3;
      cx<T> acc = czero<T>();
#pragma unroll
      for (int a = -1; a <= 1; ++a)
#pragma unroll
        for (int bb = -1; bb <= 1; ++bb) {
          int o1[3] = {0, 0, 0}, o0[3] = {0, 0, 0};
          o1[e] = s;
          o0[e] = s - 1;
          o1[pa] += a;
          o0[pa] += a;
          o1[ra] += bb;
          o0[ra] += bb;
          acc = acc + s3::wt(g.beta, a, bb) * (u_at(o1) - u_at(o0));
        }
      return ih * acc;
    };
    // mu on the edge (integer along c and e) at q + s*s_e: mean of its four cells
    auto mu_edge = [&](int e, int s) {
      int o0[3] = {0, 0, 0}, o1[3] = {0, 0, 0}, o2[3] = {0, 0, 0}, o3[3] = {0, 0, 0};
      o0[e] += s; o1[e] += s; o2[e] += s; o3[e] += s;
      o1[c] -= 1; o2[e] -= 1; o3[c] -= 1; o3[e] -= 1;
      return T(0.25) * (mu_at(o0) + mu_at(o1) + mu_at(o2) + mu_at(o3));
    };
    int oc[3] = {0, 0, 0};
    oc[c] = -1;
    cx<T> lap = mu_at(oc) * dsp(c, 0) - MU[1][1][1] * dsp(c, 1);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      if (e == c) continue;
      lap = lap + mu_edge(e, 0) * dsp(e, 0) - mu_edge(e, 1) * dsp(e, 1);
    }
    lap = ih * lap;
    // face mass m_f at face q + o of component c: density of the two cells beside it
    auto mass_at = [&](const int o[3]) -> cx<T> {
      const size_t f = q + o[0] + o[1] * sy + o[2] * sz;
      const T rf = h5 * (ldg(g.rho + f - st[c]) + ldg(g.rho + f));
      T at = att;
      if (!NOABL)
#pragma unroll
        for (int a = 0; a < 3; ++a) at += abl3(g, a, pos[a] + o[a], a == c ? 0 : 1);
      const T m = rf * w2;
      return mkc<T>(m, -m * at);
    };
    const int o0[3] = {0, 0, 0};
    cx<T> nb = czero<T>();
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int om[3] = {0, 0, 0}, op[3] = {0, 0, 0};
      om[a] = -1;
      op[a] = 1;
      nb = nb + mass_at(om) * u_at(om) + mass_at(op) * u_at(op);
    }
    const cx<T> mass = g.beta * (mass_at(o0) * U[1][1][1]) + g.sm * nb;
    const cx<T> grad = ih * (pq - ldg(p + q - st[c]));
    r[c * N + q] = ldg(b + c * N + q) - (lap - mass + grad);
    div = div + dsp(c, 1);
  }
  r[3 * N + q] = ldg(b + 3 * N + q) - (div + ldg(g.cp + q) * pq);
}

// Two blocks of 256 per SM (128 registers): measured against one (176 registers, 6.7 ms per
// 256^3 residual + restriction) and three (80 registers with spills, 5.4 ms): 5.0 ms.
template <typename T>
__global__ void __launch_bounds__(BX * BY * BZ, 2) residual(Grid<T> g, const cx<T>* __restrict__ b,
                                                        const cx<T>* __restrict__ x, cx<T>* __restrict__ r) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z * BZ + threadIdx.z;
  if (i >= g.nx || j >= g.ny || k >= g.nz) return;
  if (i >= 2 && i + 3 <= g.nx && j >= 2 && j + 3 <= g.ny && k >= 2 && k + 3 <= g.nz) {
    if (g.abl_free(0, i - 1, i + 2) && g.abl_free(1, j - 1, j + 2) && g.abl_free(2, k - 1, k + 2))
      residual_cell3<T, true>(g, b, x, r, i, j, k);
    else
      residual_cell3<T, false>(g, b, x, r, i, j, k);
    return;
  }
  // cells next to the boundary: the reference rows (bounds checks, excluded faces, clamped media)
  const size_t N = (size_t)g.nx * g.ny * g.nz, q = s3::lin(g, i, j, k);
  const cx<T>* u[3] = {x, x + N, x + 2 * N};
  const cx<T>* p = x + 3 * N;
  const int idx[3] = {i, j, k};
#pragma unroll
  for (int c = 0; c < 3; ++c)
    r[c * N + q] = idx[c] >= 1 ? b[c * N + q] - s3::row_u(c, u[c], p, g, i, j, k) : czero<T>();
  r[3 * N + q] = b[3 * N + q] - s3::row_p(u, p, g, i, j, k);
}

template <typename T>
__global__ void __launch_bounds__(BX * BY * BZ) restrict_r(const cx<T>* __restrict__ r, cx<T>* __restrict__ bc,
                                                          int nx, int ny, int nz, int nxc, int nyc, int nzc) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int I = blockIdx.x * BX + threadIdx.x;
  const int J = blockIdx.y * BY + threadIdx.y;
  const int K = blockIdx.z * BZ + threadIdx.z;
  if (I >= nxc || J >= nyc || K >= nzc) return;
  const size_t N = (size_t)nx * ny * nz, Nc = (size_t)nxc * nyc * nzc;
  const size_t qc = ((size_t)K * nyc + J) * nxc + I;
  auto R = [&](int c, int fi, int fj, int fk) { return r[c * N + ((size_t)fk * ny + fj) * nx + fi]; };
  const int IC[3] = {I, J, K};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cx<T> acc = czero<T>();
    if (IC[c] >= 1) {
      const int o1 = (c + 1) % 3, o2 = (c + 2) % 3;
      for (int s = -1; s <= 1; ++s) {
        const T ws = s == 0 ? T(2) : T(1);
        for (int a = 0; a < 2; ++a)
          for (int bb = 0; bb < 2; ++bb) {
            int f[3] = {2 * I, 2 * J, 2 * K};
            f[c] += s;
            f[o1] += a;
            f[o2] += bb;
            acc = acc + ws * R(c, f[0], f[1], f[2]);
          }
      }
      acc = T(0.0625) * acc;
    }
    bc[c * Nc + qc] = acc;
  }
  cx<T> acc = czero<T>();
  for (int c3 = 0; c3 < 2; ++c3)
    for (int c2 = 0; c2 < 2; ++c2)
      for (int c1 = 0; c1 < 2; ++c1) acc = acc + R(3, 2 * I + c1, 2 * J + c2, 2 * K + c3);
  bc[3 * Nc + qc] = T(0.125) * acc;
}

}  // namespace k3
