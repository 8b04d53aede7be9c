// 2D building blocks: the Vanka cell solve, the operator apply (one thread per cell) and the
// prolongation + correction (one thread per fine cell). The half-sweep is in vanka2d_fast.cuh,
// the residual and restriction in residual2d_fast.cuh.
#pragma once
#include "stencil2d.cuh"

namespace k2 {

constexpr int BX = 32, BY = 8;

// Exact solve of one cell's Vanka block by block elimination (Remark 3.1):
// A = blockdiag(A1, A2) (2x2 each), gradient column G, divergence row B, scalar cp.
//   S = cp - B A^{-1} G,  dp = (r_p - B A^{-1} r_u) / S,  du = A^{-1} (r_u - G dp).
// Excluded DOFs (boundary faces, faces outside the domain) carry an identity row/column and a
// zero residual, so their correction is zero.
template <typename T>
HD void cell_solve(cx<T> a1[4], cx<T> a2[4], const bool ex[4], T ih, T t0, T cp,
                   cx<T> r[5], cx<T> d[5]) {
  T G[4] = {ih, -ih, ih, -ih};
  T B[4] = {-t0 * ih, t0 * ih, -t0 * ih, t0 * ih};
  cx<T>* A[2] = {a1, a2};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (ex[k]) {
      r[k] = czero<T>();
      G[k] = T(0);
      B[k] = T(0);
    }
  }
  cx<T> y1[4], y2[4];
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    cx<T>* a = A[blk];
    const int k0 = 2 * blk, k1 = 2 * blk + 1;
    if (ex[k0]) { a[0] = mkc<T>(T(1), T(0)); a[1] = czero<T>(); a[2] = czero<T>(); }
    if (ex[k1]) { a[3] = mkc<T>(T(1), T(0)); a[1] = czero<T>(); a[2] = czero<T>(); }
    cx<T> idet = cinv(a[0] * a[3] - a[1] * a[2]);
    // inverse = idet * [a3 -a1; -a2 a0]
    y1[k0] = idet * (a[3] * r[k0] - a[1] * r[k1]);
    y1[k1] = idet * (a[0] * r[k1] - a[2] * r[k0]);
    y2[k0] = idet * (G[k0] * a[3] - G[k1] * a[1]);
    y2[k1] = idet * (G[k1] * a[0] - G[k0] * a[2]);
  }
  cx<T> S = mkc<T>(cp, T(0));
  cx<T> rp = r[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    S = S - B[k] * y2[k];
    rp = rp - B[k] * y1[k];
  }
  d[4] = rp * cinv(S);
#pragma unroll
  for (int k = 0; k < 4; ++k) d[k] = y1[k] - y2[k] * d[4];
}

// y = H x (b == nullptr) or y = bscale * b - H x. Component pointers: x + c*N.
template <typename T, typename TI>
__global__ void __launch_bounds__(BX * BY) apply(Grid<T> g, const cx<TI>* __restrict__ x,
                                                const cx<T>* __restrict__ b, T bscale, cx<T>* __restrict__ y) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const size_t N = (size_t)g.nx * g.ny, k = (size_t)j * g.nx + i;
  const cx<TI>* u1 = x;
  const cx<TI>* u2 = x + N;
  const cx<TI>* p = x + 2 * N;
  cx<T> y1 = i >= 1 ? s2::row_u1(u1, p, g, i, j) : czero<T>();
  cx<T> y2 = j >= 1 ? s2::row_u2(u2, p, g, i, j) : czero<T>();
  cx<T> yp = s2::row_p(u1, u2, p, g, i, j);
  if (b) {
    y1 = i >= 1 ? bscale * b[k] - y1 : czero<T>();
    y2 = j >= 1 ? bscale * b[N + k] - y2 : czero<T>();
    yp = bscale * b[2 * N + k] - yp;
  }
  y[k] = y1;
  y[N + k] = y2;
  y[2 * N + k] = yp;
}

// x += P e, one thread per fine cell (i, j). P_u1: linear along x1 ([1 2 1]/2 transposed) x
// [1 3 3 1]/4 transposed along x2; P_u2 rotated; P_p bilinear (Eq. 2.11, 2.12).
template <typename T>
HD cx<T> ec_u1(const cx<T>* e, int I, int J, int nxc, int nyc) {
  return (I >= 1 && I < nxc && J >= 0 && J < nyc) ? e[(size_t)J * nxc + I] : czero<T>();
}
template <typename T>
HD cx<T> ec_u2(const cx<T>* e, int I, int J, int nxc, int nyc) {
  return (J >= 1 && J < nyc && I >= 0 && I < nxc) ? e[(size_t)J * nxc + I] : czero<T>();
}
template <typename T>
HD cx<T> ec_p(const cx<T>* e, int I, int J, int nxc, int nyc) {
  return (I >= 0 && I < nxc && J >= 0 && J < nyc) ? e[(size_t)J * nxc + I] : czero<T>();
}

template <typename T>
__global__ void __launch_bounds__(BX * BY) prolong_add(const cx<T>* __restrict__ e, cx<T>* __restrict__ x,
                                                      int nx, int ny, int nxc, int nyc) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const size_t N = (size_t)nx * ny, Nc = (size_t)nxc * nyc, k = (size_t)j * nx + i;
  const int I = i >> 1, J = j >> 1;
  // cell-centred axis: fine 2K -> 3/4 K + 1/4 (K-1); fine 2K+1 -> 3/4 K + 1/4 (K+1)
  const int Io = (i & 1) ? I + 1 : I - 1;
  const int Jo = (j & 1) ? J + 1 : J - 1;
  const T a = T(0.75), c = T(0.25);
  // u1: along x1 faces: even i -> coarse face I; odd -> mean of faces I, I+1
  if (i >= 1) {
    cx<T> v;
    if ((i & 1) == 0)
      v = a * ec_u1(e, I, J, nxc, nyc) + c * ec_u1(e, I, Jo, nxc, nyc);
    else
      v = T(0.5) * (a * ec_u1(e, I, J, nxc, nyc) + c * ec_u1(e, I, Jo, nxc, nyc)
                    + a * ec_u1(e, I + 1, J, nxc, nyc) + c * ec_u1(e, I + 1, Jo, nxc, nyc));
    x[k] = x[k] + v;
  } else {
    x[k] = czero<T>();
  }
  const cx<T>* e2 = e + Nc;
  if (j >= 1) {
    cx<T> v;
    if ((j & 1) == 0)
      v = a * ec_u2(e2, I, J, nxc, nyc) + c * ec_u2(e2, Io, J, nxc, nyc);
    else
      v = T(0.5) * (a * ec_u2(e2, I, J, nxc, nyc) + c * ec_u2(e2, Io, J, nxc, nyc)
                    + a * ec_u2(e2, I, J + 1, nxc, nyc) + c * ec_u2(e2, Io, J + 1, nxc, nyc));
    x[N + k] = x[N + k] + v;
  } else {
    x[N + k] = czero<T>();
  }
  const cx<T>* ep = e + 2 * Nc;
  cx<T> v = a * (a * ec_p(ep, I, J, nxc, nyc) + c * ec_p(ep, Io, J, nxc, nyc))
          + c * (a * ec_p(ep, I, Jo, nxc, nyc) + c * ec_p(ep, Io, Jo, nxc, nyc));
  x[2 * N + k] = x[2 * N + k] + v;
}

}  // namespace k2
