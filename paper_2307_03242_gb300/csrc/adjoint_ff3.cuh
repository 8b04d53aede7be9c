// 3D y = H^H x (or y = bscale b - H^H x) in double-FP32 arithmetic, on the float-float
// coefficient arrays of the forward FP64 apply (apply_ff3d.cuh): cell mu, 1/(lambda+mu), edge mu
// per orientation, face masses. Same operator as adj::row_u / adj::row_p (adjoint.cuh), arranged
// as the transpose of the forward 27-point expansion: the forward row of u_c at q' has the
// coefficient C_q'(delta) = (1/h^2) sum_e part_e(q')(delta_e) W(delta across e), with
// part_e(q') = (-mu_a, mu_a + mu_b, -mu_b) from the mu of the two derivative points beside q'
// along e; row q of the transpose takes C_{q+delta}(-delta) for every delta. The mass term is
// conj(m_q) (M^beta x)(q), the spread divergence turns into the spread difference of p, the
// gradient of p into minus the plain divergence.
#pragma once
#include "apply_ff3d.cuh"

namespace ff3 {

template <typename TI, bool FFO = false>
HD void cell_rows_adjoint(const FineFF3& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y, int i, int j,
                          int k) {
  const int q[3] = {i, j, k};
  const size_t N = (size_t)g.nx * g.ny * g.nz, kq = lin(g, i, j, k);
  auto inside = [&](int a, int bb, int c) { return a >= 0 && a < g.nx && bb >= 0 && bb < g.ny && c >= 0 && c < g.nz; };
  auto mclamp = [&](int a, int bb, int c) {
    return g.mu[lin(g, iclamp(a, 0, g.nx - 1), iclamp(bb, 0, g.ny - 1), iclamp(c, 0, g.nz - 1))];
  };
  // mu of the derivative point of d_e u_c between p - s_e and p (lattice position p)
  auto mu_pt = [&](int c, int e, int a, int bb, int cc) -> f2 {
    if (e == c) {
      int s[3] = {0, 0, 0};
      s[c] = 1;
      return mclamp(a - s[0], bb - s[1], cc - s[2]);
    }
    // edges parallel to the third axis, at integer positions along c and e; outside the lattice
    // the point is never used with a non-zero displacement difference
    if (a < 0 || bb < 0 || cc < 0 || a > g.nx || bb > g.ny || cc > g.nz) return f2{0.f, 0.f};
    return g.edge[3 - c - e][lat(g, a, bb, cc)];
  };
  cx<double> out[4];
  // every loop is unrolled, so that no array is indexed at run time (no local memory)
  #pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (q[c] < 1) {
      out[c] = czero<double>();
      continue;
    }
    cacc r;
    const cx<TI>* u = x + c * N;
    #pragma unroll
    for (int dk = -1; dk <= 1; ++dk)
      #pragma unroll
      for (int dj = -1; dj <= 1; ++dj)
        #pragma unroll
        for (int di = -1; di <= 1; ++di) {
          const int a = i + di, bb = j + dj, cc = k + dk;
          const int qa[3] = {a, bb, cc};
          if (!inside(a, bb, cc) || qa[c] < 1) continue;
          const int dl[3] = {di, dj, dk};
          f2 C = {0.f, 0.f};
          #pragma unroll
          for (int e = 0; e < 3; ++e) {
            // part_e of row q + delta at offset -delta_e
            int s[3] = {0, 0, 0};
            s[e] = 1;
            const f2 ma = mu_pt(c, e, a, bb, cc);                          // beside q + delta, low side
            const f2 mb = mu_pt(c, e, a + s[0], bb + s[1], cc + s[2]);     // high side
            f2 part;
            if (dl[e] == 1) part = fneg(ma);
            else if (dl[e] == 0) part = add(ma, mb);
            else part = fneg(mb);
            const int t1 = (e + 1) % 3, t2 = (e + 2) % 3;
            C = add(C, mul(part, g.W[dl[t1] + 1][dl[t2] + 1]));
          }
          C = mul(g.ih2, C);
          const cx<TI> uv = u[lin(g, a, bb, cc)];
          r.rterm(C, ld(uv.re), ld(uv.im));
        }
    // - conj(m_q) (M^beta x_c)(q)
    {
      c2 m = g.m[c][kq];
      if (g.alpha.hi != 0.f) m.im = add(m.im, fneg(mul(g.alpha, m.re)));
      cacc s;
      const cx<TI> u0 = u[kq];
      s.rterm(g.beta, ld(u0.re), ld(u0.im));
      #pragma unroll
      for (int t = 0; t < 3; ++t)
        #pragma unroll
        for (int sg = -1; sg <= 1; sg += 2) {
          int o[3] = {i, j, k};
          o[t] += sg;
          if (!inside(o[0], o[1], o[2]) || o[c] < 1) continue;
          const cx<TI> uv = u[lin(g, o[0], o[1], o[2])];
          s.rterm(g.sm, ld(uv.re), ld(uv.im));
        }
      const f2 sr = s.re.norm(), si = s.im.norm();
      // conj(m) * s = (m.re - i m.im)(sr + i si)
      r.re.fms_ff(m.re, sr);
      r.re.fms_ff(m.im, si);
      r.im.fms_ff(m.re, si);
      r.im.fma_ff(m.im, sr);
    }
    // (1/h) sum_o W(o) [p(q + o - s_c) - p(q + o)], o across c
    {
      const int t1 = (c + 1) % 3, t2 = (c + 2) % 3;
      const cx<TI>* p = x + 3 * N;
      #pragma unroll
      for (int a = -1; a <= 1; ++a)
        #pragma unroll
        for (int bb = -1; bb <= 1; ++bb) {
          int o[3] = {i, j, k};
          o[t1] += a;
          o[t2] += bb;
          const f2 wgt = mul(g.ih, g.W[a + 1][bb + 1]);
          int lo[3] = {o[0], o[1], o[2]};
          lo[c] -= 1;
          if (inside(lo[0], lo[1], lo[2])) {
            const cx<TI> pv = p[lin(g, lo[0], lo[1], lo[2])];
            r.rterm(wgt, ld(pv.re), ld(pv.im));
          }
          if (inside(o[0], o[1], o[2])) {
            const cx<TI> pv = p[lin(g, o[0], o[1], o[2])];
            r.rterm(fneg(wgt), ld(pv.re), ld(pv.im));
          }
        }
    }
    out[c] = mkc<double>(r.re.to_double(), r.im.to_double());
  }
  {
    // p row: (1/h) sum_c (x_c(q) - x_c(q + s_c)) + cp(q) p(q)
    cacc r;
    #pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cx<TI>* u = x + c * N;
      if (q[c] >= 1) {
        const cx<TI> uv = u[kq];
        r.rterm(g.ih, ld(uv.re), ld(uv.im));
      }
      int hi[3] = {i, j, k};
      hi[c] += 1;
      if (inside(hi[0], hi[1], hi[2])) {
        const cx<TI> uv = u[lin(g, hi[0], hi[1], hi[2])];
        r.rterm(fneg(g.ih), ld(uv.re), ld(uv.im));
      }
    }
    const cx<TI> pc = x[3 * N + kq];
    r.rterm(g.cp[kq], ld(pc.re), ld(pc.im));
    out[3] = mkc<double>(r.re.to_double(), r.im.to_double());
  }
  #pragma unroll
  for (int c = 0; c < 4; ++c) {
    cx<double> v = out[c];
    if (b) v = (c < 3 && q[c] < 1) ? czero<double>() : bscale * b[c * N + kq] - v;
    ff2::store_val<FFO>(y, c * N + kq, v);
  }
}

template <typename TI, bool FFO>
__global__ void __launch_bounds__(BX * BY * BZ) apply_adjoint(FineFF3 g, const cx<TI>* __restrict__ x,
                                                             const cx<double>* __restrict__ b, double bscale,
                                                             void* __restrict__ y) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z * BZ + threadIdx.z;
  if (i >= g.nx || j >= g.ny || k >= g.nz) return;
  cell_rows_adjoint<TI, FFO>(g, x, b, bscale, y, i, j, k);
}

}  // namespace ff3
