// FP64 operator apply of the outer solve (2D), evaluated in double-FP32 arithmetic.
//
// y = H x (Eq. 3.10 with the sign of Eq. 4.4) or y = bscale*b - H x, with x in FP32 (the cycle's
// output, exact floats) or FP64 (the iterate), y in FP64. The FP64 coefficients are precomputed
// once on the host and stored as float-float pairs: cell mu and 1/(lambda+mu), node mu
// (A_e, the mean of the four cells around a node), and the complex face masses
// m_f = rho_f omega^2 (1 - i (gamma + gamma_ABL(x_f))) of the unshifted operator; the shifted
// operator uses m_f - i alpha Re(m_f). Each row is then
//   Laplacian: sum over the 3x3 faces of C(di, dj) u(i+di, j+dj) with
//              C = cell(di) t(dj) + node(dj) t(di),  t = ((1-beta)/4, (1+beta)/2, (1-beta)/4),
//              cell = (-mu_W, mu_W + mu_E, -mu_E) (the two cells beside the face),
//              node = (-mu_S, mu_S + mu_N, -mu_N) (the two nodes beside it) -- the expansion of
//              grad_h^T A_e(mu) grad_h^beta (Eq. 3.4-3.6);
//   mass:      beta m_f u_f + (1-beta)/4 sum of the 4 neighbours' m u (Eq. 3.3);
//   gradient:  (p_+ - p_-) / h;   continuity row: (div)^beta u + p/(lambda+mu).
#pragma once
#include "dfloat.cuh"
#include "emg_types.cuh"

namespace ff2 {

using df::f2;
constexpr int BX = 32, BY = 8;

struct c2 {
  f2 re, im;
};

struct FineFF {
  int nx, ny;
  f2 ih2, ih;        // 1/h^2, 1/h
  f2 t0, t1;         // (1+beta)/2, (1-beta)/4
  f2 ht2[3], ht1[3]; // t / h^2 and t / h with t = (t1, t0, t1)
  f2 beta, sm;       // beta, (1-beta)/4
  f2 alpha;          // shift added to the attenuation (0 for H, alpha for H_s)
  const f2* mu;      // nx*ny cells
  const f2* mun;     // (nx+1)*(ny+1) nodes, node (X, Y) at X h, Y h
  const f2* cp;      // nx*ny cells
  const c2* m1;      // nx*ny u1 faces
  const c2* m2;      // nx*ny u2 faces
};

HD f2 ld(float v) { return {v, 0.f}; }
HD f2 ld(double v) { return df::split(v); }
HD f2 fneg(f2 a) { return {-a.hi, -a.lo}; }

// float-float product / sum with normalisation (used for the few coefficient combinations)
HD f2 mul(f2 a, f2 b) {
  float p = a.hi * b.hi;
  float e = std::fma(a.hi, b.hi, -p);
  e = std::fma(a.hi, b.lo, e);
  e = std::fma(a.lo, b.hi, e);
  f2 r;
  df::two_sum(p, e, r.hi, r.lo);
  return r;
}
HD f2 add(f2 a, f2 b) {
  float s, t;
  df::two_sum(a.hi, b.hi, s, t);
  t += a.lo + b.lo;
  f2 r;
  df::two_sum(s, t, r.hi, r.lo);
  return r;
}

struct cacc {
  df::acc re, im;
  // += c * u (c real)
  HD void rterm(f2 c, f2 ur, f2 ui) {
    re.fma_ff(c, ur);
    im.fma_ff(c, ui);
  }
  // += m * u (m complex)
  HD void cterm(const c2& m, f2 ur, f2 ui) {
    re.fma_ff(m.re, ur);
    re.fms_ff(m.im, ui);
    im.fma_ff(m.re, ui);
    im.fma_ff(m.im, ur);
  }
};

// y at cell (i, j): the u1 row at face i, the u2 row at face j and the continuity row, each as
// H x (b == nullptr) or bscale * b - H x, as float-float accumulators; rows of faces that are not
// unknowns are 0.
template <typename TI>
HD void apply_cell_acc(const FineFF& g, const cx<TI>* __restrict__ x, const cx<double>* __restrict__ b, double bscale,
                       int i, int j, cacc out3[3]) {
  const int nx = g.nx, ny = g.ny;
  const size_t N = (size_t)nx * ny, k = (size_t)j * nx + i;
  const cx<TI>* u1 = x;
  const cx<TI>* u2 = x + N;
  const cx<TI>* p = x + 2 * N;
  const f2 z = {0.f, 0.f};
  auto clampc = [&](int ii, int jj) { return (size_t)iclamp(jj, 0, ny - 1) * nx + iclamp(ii, 0, nx - 1); };
  const f2 muC = g.mu[k];
  auto mshift = [&](c2 m) {  // m - i alpha Re(m)
    if (g.alpha.hi != 0.f) m.im = add(m.im, fneg(mul(g.alpha, m.re)));
    return m;
  };
  // ---- u1 row at face (i, j)
  cacc r1;
  if (i >= 1) {
    const f2 muW = g.mu[clampc(i - 1, j)];
    const f2 nS = g.mun[(size_t)j * (nx + 1) + i], nN = g.mun[(size_t)(j + 1) * (nx + 1) + i];
    const f2 cell[3] = {fneg(muW), add(muW, muC), fneg(muC)};
    const f2 node[3] = {fneg(nS), add(nS, nN), fneg(nN)};
    cacc a0, a4;
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
      const int jj = j + dj;
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        const int ii = i + di;
        if (ii < 1 || ii >= nx || jj < 0 || jj >= ny) continue;
        const cx<TI> u = u1[(size_t)jj * nx + ii];
        const f2 C = add(mul(cell[di + 1], g.ht2[dj + 1]), mul(node[dj + 1], g.ht2[di + 1]));
        const f2 ur = ld(u.re), ui = ld(u.im);
        r1.rterm(C, ur, ui);
        // mass: m u at the face (a0) and at the 4 neighbours (a4)
        if (di == 0 || dj == 0) (di == 0 && dj == 0 ? a0 : a4).cterm(mshift(g.m1[(size_t)jj * nx + ii]), ur, ui);
      }
    }
    // - beta a0 - sm a4
    r1.re.fms_ff(g.beta, a0.re.norm());
    r1.im.fms_ff(g.beta, a0.im.norm());
    r1.re.fms_ff(g.sm, a4.re.norm());
    r1.im.fms_ff(g.sm, a4.im.norm());
    // + (p(i,j) - p(i-1,j)) / h
    const cx<TI> pc = p[k], pw = p[k - 1];
    r1.rterm(g.ih, ld(pc.re), ld(pc.im));
    r1.rterm(fneg(g.ih), ld(pw.re), ld(pw.im));
  }
  // ---- u2 row at face (i, j)
  cacc r2;
  if (j >= 1) {
    const f2 muS = g.mu[clampc(i, j - 1)];
    const f2 nW = g.mun[(size_t)j * (nx + 1) + i], nE = g.mun[(size_t)j * (nx + 1) + i + 1];
    const f2 cell[3] = {fneg(muS), add(muS, muC), fneg(muC)};  // along x2 (dj)
    const f2 node[3] = {fneg(nW), add(nW, nE), fneg(nE)};      // along x1 (di)
    cacc a0, a4;
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
      const int jj = j + dj;
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        const int ii = i + di;
        if (jj < 1 || jj >= ny || ii < 0 || ii >= nx) continue;
        const cx<TI> u = u2[(size_t)jj * nx + ii];
        const f2 C = add(mul(cell[dj + 1], g.ht2[di + 1]), mul(node[di + 1], g.ht2[dj + 1]));
        const f2 ur = ld(u.re), ui = ld(u.im);
        r2.rterm(C, ur, ui);
        if (di == 0 || dj == 0) (di == 0 && dj == 0 ? a0 : a4).cterm(mshift(g.m2[(size_t)jj * nx + ii]), ur, ui);
      }
    }
    r2.re.fms_ff(g.beta, a0.re.norm());
    r2.im.fms_ff(g.beta, a0.im.norm());
    r2.re.fms_ff(g.sm, a4.re.norm());
    r2.im.fms_ff(g.sm, a4.im.norm());
    const cx<TI> pc = p[k], ps = p[k - nx];
    r2.rterm(g.ih, ld(pc.re), ld(pc.im));
    r2.rterm(fneg(g.ih), ld(ps.re), ld(ps.im));
  }
  // ---- continuity row at cell (i, j): d1^beta u1 + d2^beta u2 + cp p
  cacc rp;
  {
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
      const int jj = j + dj;
      if (jj < 0 || jj >= ny) continue;
      const f2 c = g.ht1[dj + 1];
      if (i + 1 < nx) {
        const cx<TI> a = u1[(size_t)jj * nx + i + 1];
        rp.rterm(c, ld(a.re), ld(a.im));
      }
      if (i >= 1) {
        const cx<TI> a = u1[(size_t)jj * nx + i];
        rp.rterm(fneg(c), ld(a.re), ld(a.im));
      }
    }
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const int ii = i + di;
      if (ii < 0 || ii >= nx) continue;
      const f2 c = g.ht1[di + 1];
      if (j + 1 < ny) {
        const cx<TI> a = u2[(size_t)(j + 1) * nx + ii];
        rp.rterm(c, ld(a.re), ld(a.im));
      }
      if (j >= 1) {
        const cx<TI> a = u2[(size_t)j * nx + ii];
        rp.rterm(fneg(c), ld(a.re), ld(a.im));
      }
    }
    const cx<TI> pc = p[k];
    rp.rterm(g.cp[k], ld(pc.re), ld(pc.im));
  }
  const cacc zero{};
  if (b) {
    // bscale * b - H x in float-float when bscale is a power of two in the float range
    const float bs = df::pow2_float(bscale);
    auto res = [&](const cacc& a, cx<double> bv) {
      cacc t;
      t.re = df::scaled_sub_acc(bv.re, bs, bscale, a.re);
      t.im = df::scaled_sub_acc(bv.im, bs, bscale, a.im);
      return t;
    };
    out3[0] = i >= 1 ? res(r1, b[k]) : zero;
    out3[1] = j >= 1 ? res(r2, b[N + k]) : zero;
    out3[2] = res(rp, b[2 * N + k]);
  } else {
    out3[0] = i >= 1 ? r1 : zero;
    out3[1] = j >= 1 ? r2 : zero;
    out3[2] = rp;
  }
  (void)z;
}

// The same rows as FP64 values.
template <typename TI>
HD void apply_cell(const FineFF& g, const cx<TI>* __restrict__ x, const cx<double>* __restrict__ b, double bscale, int i,
                   int j, cx<double> out3[3]) {
  cacc a[3];
  apply_cell_acc<TI>(g, x, b, bscale, i, j, a);
  for (int c = 0; c < 3; ++c) out3[c] = mkc<double>(a[c].re.to_double(), a[c].im.to_double());
}

// Stores a row: as a complex double, or (FFO) as a float-float pair (df::cff).
template <bool FFO>
HD void store_row(void* y, size_t at, const cacc& a) {
  if constexpr (FFO) static_cast<df::cff*>(y)[at] = df::to_cff(a.re, a.im);
  else static_cast<cx<double>*>(y)[at] = mkc<double>(a.re.to_double(), a.im.to_double());
}
// Stores an FP64 value: as it is, or (FFO) split into a float-float pair.
template <bool FFO>
HD void store_val(void* y, size_t at, cx<double> v) {
  if constexpr (FFO) static_cast<df::cff*>(y)[at] = df::to_cff(v.re, v.im);
  else static_cast<cx<double>*>(y)[at] = v;
}

// y (complex double, or with FFO float-float pairs) = H x or bscale * b - H x.
template <typename TI, bool FFO>
__global__ void __launch_bounds__(BX * BY) apply(FineFF g, const cx<TI>* __restrict__ x, const cx<double>* __restrict__ b,
                                                double bscale, void* __restrict__ y) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const size_t N = (size_t)g.nx * g.ny, k = (size_t)j * g.nx + i;
  cacc out[3];
  apply_cell_acc<TI>(g, x, b, bscale, i, j, out);
  store_row<FFO>(y, k, out[0]);
  store_row<FFO>(y, N + k, out[1]);
  store_row<FFO>(y, 2 * N + k, out[2]);
}

}  // namespace ff2
