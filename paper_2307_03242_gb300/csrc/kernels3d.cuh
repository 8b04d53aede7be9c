// 3D kernels of the V-cycle and of the FP64 operator apply (same structure as the 2D ones).
#pragma once
#include "stencil3d.cuh"

namespace k3 {

constexpr int BX = 32, BY = 4, BZ = 2;

// Exact solve of one cell's 7x7 Vanka block by block elimination: three 2x2 displacement blocks
// (Remark 3.1), gradient column G = ih(+1,-1, ..), divergence row B = w00 ih (-1,+1, ..).
template <typename T>
HD void cell_solve(cx<T> a[3][4], const bool ex[6], T ih, T w00, T cp, cx<T> r[7], cx<T> d[7]) {
  T G[6], B[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const T s = (q & 1) ? T(-1) : T(1);
    G[q] = ex[q] ? T(0) : s * ih;
    B[q] = ex[q] ? T(0) : -s * w00 * ih;
    if (ex[q]) r[q] = czero<T>();
  }
  cx<T> y1[6], y2[6];
#pragma unroll
  for (int blk = 0; blk < 3; ++blk) {
    cx<T>* m = a[blk];
    const int k0 = 2 * blk, k1 = 2 * blk + 1;
    if (ex[k0]) { m[0] = mkc<T>(T(1), T(0)); m[1] = czero<T>(); m[2] = czero<T>(); }
    if (ex[k1]) { m[3] = mkc<T>(T(1), T(0)); m[1] = czero<T>(); m[2] = czero<T>(); }
    cx<T> idet = cinv(m[0] * m[3] - m[1] * m[2]);
    y1[k0] = idet * (m[3] * r[k0] - m[1] * r[k1]);
    y1[k1] = idet * (m[0] * r[k1] - m[2] * r[k0]);
    y2[k0] = idet * (G[k0] * m[3] - G[k1] * m[1]);
    y2[k1] = idet * (G[k1] * m[0] - G[k0] * m[2]);
  }
  cx<T> S = mkc<T>(cp, T(0));
  cx<T> rp = r[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    S = S - B[q] * y2[q];
    rp = rp - B[q] * y1[q];
  }
  d[6] = rp * cinv(S);
#pragma unroll
  for (int q = 0; q < 6; ++q) d[q] = y1[q] - y2[q] * d[6];
}

template <typename T, typename TI>
__global__ void __launch_bounds__(BX * BY * BZ) apply(Grid<T> g, const cx<TI>* __restrict__ x,
                                                     const cx<T>* __restrict__ b, T bscale, cx<T>* __restrict__ y) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z * BZ + threadIdx.z;
  if (i >= g.nx || j >= g.ny || k >= g.nz) return;
  const size_t N = (size_t)g.nx * g.ny * g.nz, q = s3::lin(g, i, j, k);
  const cx<TI>* u[3] = {x, x + N, x + 2 * N};
  const cx<TI>* p = x + 3 * N;
  const int idx[3] = {i, j, k};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cx<T> v = idx[c] >= 1 ? s3::row_u(c, u[c], p, g, i, j, k) : czero<T>();
    if (b) v = idx[c] >= 1 ? bscale * b[c * N + q] - v : czero<T>();
    y[c * N + q] = v;
  }
  cx<T> v = s3::row_p(u, p, g, i, j, k);
  if (b) v = bscale * b[3 * N + q] - v;
  y[3 * N + q] = v;
}

template <typename T>
__global__ void __launch_bounds__(BX * BY * BZ) vanka(Grid<T> g, const cx<T>* __restrict__ b,
                                                     const cx<T>* __restrict__ uin, cx<T>* __restrict__ uout,
                                                     cx<T>* p, int colour, T w, int zero_in) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int ip = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z * BZ + threadIdx.z;
  if (j >= g.ny || k >= g.nz) return;
  const int par = (colour + j + k) & 1;
  const int i = 2 * ip + par;
  if (zero_in) {
    const int io = 2 * ip + 1 - par;
    if (io < g.nx) p[s3::lin(g, io, j, k)] = czero<T>();
  }
  if (i >= g.nx) return;
  const size_t N = (size_t)g.nx * g.ny * g.nz, q = s3::lin(g, i, j, k);
  const cx<T>* u[3] = {uin, uin + N, uin + 2 * N};
  const int idx[3] = {i, j, k};
  const int nn[3] = {g.nx, g.ny, g.nz};
  const size_t stride[3] = {1, (size_t)g.nx, (size_t)g.nx * g.ny};
  bool ex[6];
  cx<T> r[7], a[3][4], d[7];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ex[2 * c] = idx[c] == 0;
    ex[2 * c + 1] = idx[c] + 1 >= nn[c];
    int ci, cj, ck;
    s3::unit(c, ci, cj, ck);
    if (zero_in) {
      r[2 * c] = ex[2 * c] ? czero<T>() : b[c * N + q];
      r[2 * c + 1] = ex[2 * c + 1] ? czero<T>() : b[c * N + q + stride[c]];
    } else {
      r[2 * c] = ex[2 * c] ? czero<T>() : b[c * N + q] - s3::row_u(c, u[c], (const cx<T>*)p, g, i, j, k);
      r[2 * c + 1] = ex[2 * c + 1] ? czero<T>()
                                   : b[c * N + q + stride[c]] - s3::row_u(c, u[c], (const cx<T>*)p, g, i + ci, j + cj, k + ck);
    }
    s3::block_u(g, c, i, j, k, a[c][0], a[c][1], a[c][2], a[c][3]);
    if (g.economic) a[c][1] = a[c][2] = czero<T>();
  }
  r[6] = zero_in ? b[3 * N + q] : b[3 * N + q] - s3::row_p(u, (const cx<T>*)p, g, i, j, k);
  cell_solve(a, ex, g.ih, s3::wt(g.beta, 0, 0), s3::mat(g.cp, g, i, j, k), r, d);
  const cx<T> z = czero<T>();
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cx<T>* o = uout + c * N;
    const cx<T>* ui = u[c];
    if (zero_in) {
      o[q] = ex[2 * c] ? z : w * d[2 * c];
      if (!ex[2 * c + 1]) o[q + stride[c]] = w * d[2 * c + 1];
    } else {
      o[q] = ex[2 * c] ? z : ui[q] + w * d[2 * c];
      if (!ex[2 * c + 1]) o[q + stride[c]] = ui[q + stride[c]] + w * d[2 * c + 1];
    }
    if (idx[c] == 1) o[q - stride[c]] = z;  // boundary face owned by a cell of the other colour
  }
  p[q] = zero_in ? w * d[6] : p[q] + w * d[6];
}

// x += P e: P_u_c = [1 2 1]/2 (transposed) along c x [1 3 3 1]/4 (transposed) along the others;
// P_p trilinear.
template <typename T>
__global__ void __launch_bounds__(BX * BY * BZ) prolong_add(const cx<T>* __restrict__ e, cx<T>* __restrict__ x,
                                                           int nx, int ny, int nz, int nxc, int nyc, int nzc) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z * BZ + threadIdx.z;
  if (i >= nx || j >= ny || k >= nz) return;
  const size_t N = (size_t)nx * ny * nz, Nc = (size_t)nxc * nyc * nzc;
  const size_t q = ((size_t)k * ny + j) * nx + i;
  const int f[3] = {i, j, k};
  const int nc[3] = {nxc, nyc, nzc};
  // per-axis cell-type interpolation: two coarse indices with weights 3/4, 1/4
  int ci[3][2];
  T cw[3][2];
  // every loop is unrolled, so that no array is indexed at run time (no local memory)
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int K0 = f[a] >> 1;
    ci[a][0] = K0;
    ci[a][1] = (f[a] & 1) ? K0 + 1 : K0 - 1;
    cw[a][0] = T(0.75);
    cw[a][1] = T(0.25);
  }
  auto ev = [&](const cx<T>* ec, int comp, int I, int J, int K) -> cx<T> {
    if (I < 0 || I >= nxc || J < 0 || J >= nyc || K < 0 || K >= nzc) return czero<T>();
    const int IC[3] = {I, J, K};
    if (comp < 3 && IC[comp] == 0) return czero<T>();
    return ec[((size_t)K * nyc + J) * nxc + I];
  };
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const cx<T>* ec = e + c * Nc;
    if (c < 3 && f[c] == 0) {
      x[c * N + q] = czero<T>();
      continue;
    }
    // index lists per axis
    int idx[3][2];
    T wgt[3][2];
    int cnt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == c) {  // face axis: even -> coarse face f/2; odd -> mean of f/2 and f/2+1
        idx[a][0] = f[a] >> 1;
        wgt[a][0] = (f[a] & 1) ? T(0.5) : T(1);
        idx[a][1] = (f[a] >> 1) + 1;
        wgt[a][1] = T(0.5);
        cnt[a] = (f[a] & 1) ? 2 : 1;
      } else {
        idx[a][0] = ci[a][0];
        idx[a][1] = ci[a][1];
        wgt[a][0] = cw[a][0];
        wgt[a][1] = cw[a][1];
        cnt[a] = 2;
      }
    }
    cx<T> acc = czero<T>();
#pragma unroll
    for (int s2_ = 0; s2_ < 2; ++s2_)
#pragma unroll
      for (int s1 = 0; s1 < 2; ++s1)
#pragma unroll
        for (int s0 = 0; s0 < 2; ++s0)
          if (s2_ < cnt[2] && s1 < cnt[1] && s0 < cnt[0])
            acc = acc + (wgt[0][s0] * wgt[1][s1] * wgt[2][s2_]) * ev(ec, c, idx[0][s0], idx[1][s1], idx[2][s2_]);
    x[c * N + q] = x[c * N + q] + acc;
  }
  (void)nc;
}

}  // namespace k3
