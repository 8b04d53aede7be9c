// FP64 operator apply of the outer solve (3D), evaluated in double-FP32 arithmetic.
//
// Section 5.3: the 3D beta-spread derivative (Eq. dxSkew3D, with 1/h) spreads a difference along
// axis e over the two other axes with the weights W(a, b) = beta [a = b = 0] + (1-beta)/16
// [1 2 1]_a [1 2 1]_b; the mass spreads to the 6 neighbours with (1-beta)/6 (Eq. massHO3D). The
// row of u_c at face q is the 27-point sum (evaluated in a factored form, see cell_rows)
//   sum_delta C(delta) u_c(q + delta),  C(delta) = sum_e part_e(delta_e) W(delta_t1(e), delta_t2(e)),
// with part_e = (-mu_a, mu_a + mu_b, -mu_b): mu_a, mu_b the mu of the two derivative points beside
// q along e -- cell centres for e = c, edge centres (mean of 4 cells, A_e) for e != c. FP64
// coefficients are precomputed on the host as float-float pairs: cell mu, 1/(lambda+mu), edge mu
// for the three edge orientations, and the complex face masses of the unshifted operator.
#pragma once
#include "apply_ff2d.cuh"

namespace ff3 {

using df::f2;
using ff2::c2;
using ff2::cacc;
using ff2::ld;
using ff2::mul;
using ff2::add;
using ff2::fneg;
constexpr int BX = 32, BY = 4, BZ = 2;

struct FineFF3 {
  int nx, ny, nz;
  f2 ih, ih2, beta, sm, alpha;
  f2 kap;              // (1-beta)/16
  f2 W[3][3];          // W[a+1][b+1]
  const f2* mu;        // cells
  const f2* cp;        // cells
  const f2* edge[3];   // edge[r]: edges parallel to axis r, lattice (nx+1)(ny+1)(nz+1)
  const c2* m[3];      // face masses of u_c, cells
};

HD size_t lat(const FineFF3& g, int i, int j, int k) { return ((size_t)k * (g.ny + 1) + j) * (g.nx + 1) + i; }
HD size_t lin(const FineFF3& g, int i, int j, int k) { return ((size_t)k * g.ny + j) * g.nx + i; }

// One of three values selected by a run-time index without an indexed array (an array indexed at
// run time would be placed in local memory).
template <typename V>
HD V sel3(int c, V a, V b, V d) {
  return c == 0 ? a : (c == 1 ? b : d);
}

// A loaded complex value ready for float-float use: floats as they are, doubles split once.
template <typename TI>
struct Val;
template <>
struct Val<float> {
  float re, im;
};
template <>
struct Val<double> {
  f2 re, im;
};
HD Val<float> val(cx<float> v) { return {v.re, v.im}; }
HD Val<double> val(cx<double> v) { return {df::split(v.re), df::split(v.im)}; }
HD f2 asf2(float v) { return {v, 0.f}; }
HD f2 asf2(f2 v) { return v; }
// a * b for float-float a and a float or float-float b (normalised).
HD f2 mulv(f2 a, float b) {
  const float p = a.hi * b;
  float e = std::fma(a.hi, b, -p);
  e = std::fma(a.lo, b, e);
  f2 r;
  df::two_sum(p, e, r.hi, r.lo);
  return r;
}
HD f2 mulv(f2 a, f2 b) { return mul(a, b); }
// (ar, ai) += w v with w = 1, 2 or 4 (the scaling is exact)
HD void wadd(df::acc& ar, df::acc& ai, Val<float> v, float w) {
  ar.add(v.re * w);
  ai.add(v.im * w);
}
HD void wadd(df::acc& ar, df::acc& ai, Val<double> v, float w) {
  ar.add(f2{v.re.hi * w, v.re.lo * w});
  ai.add(f2{v.im.hi * w, v.im.lo * w});
}
HD c2 csub(c2 a, c2 b) { return {add(a.re, fneg(b.re)), add(a.im, fneg(b.im))}; }

// The rows of cell (i, j, k): u_c at its low face for c = 0, 1, 2 (zero for a boundary face,
// which is not an unknown) and the continuity row, as H x or bscale * b - H x.
//
// The 27-point row of u_c is evaluated in its factored form: with W(a, b) = beta [a = b = 0] +
// kappa w_a w_b, kappa = (1-beta)/16, w = (1, 2, 1), the slab sums
//   S_e(d) = sum_{a,b} W(a, b) u_c(q + d e_e + a e_t1 + b e_t2) = beta u_c(q + d e_e) + kappa T_e(d)
// (T_e(d) the sum with the integer weights w_a w_b, exact scalings by 1, 2 or 4) turn the row into
//   ih2 sum_e [mu_a (S_e(0) - S_e(-1)) + mu_b (S_e(0) - S_e(+1))],
// the same sum as sum_delta C(delta) u_c(q + delta) up to the order of the additions. Each of the
// 27 values is loaded once and added into the three slab families it belongs to. The continuity
// row's spread divergence of u_c is ih (S_c(+1) - S_c(0)) with the same slab sums.
template <typename TI, bool FFO = false>
HD void cell_rows_factored(const FineFF3& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y, int i, int j,
                           int k) {
  const size_t N = (size_t)g.nx * g.ny * g.nz, kq = lin(g, i, j, k);
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  const long long sl[3] = {1, sy, sz};
  auto inside = [&](int a, int bb, int c) { return a >= 0 && a < g.nx && bb >= 0 && bb < g.ny && c >= 0 && c < g.nz; };
  auto mshift = [&](c2 m) {
    if (g.alpha.hi != 0.f) m.im = add(m.im, fneg(mul(g.alpha, m.re)));
    return m;
  };
  const float bs = b ? df::pow2_float(bscale) : 0.f;
  auto finish = [&](const cacc& r, size_t at) {
    if (!b) {
      ff2::store_row<FFO>(y, at, r);
      return;
    }
    cacc t;
    t.re = df::scaled_sub_acc(b[at].re, bs, bscale, r.re);
    t.im = df::scaled_sub_acc(b[at].im, bs, bscale, r.im);
    ff2::store_row<FFO>(y, at, t);
  };
  cacc dv;  // spread divergence sum_c (S_c(+1) - S_c(0)), without the 1/h
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    const int qc = sel3(c, i, j, k);
    const cx<TI>* u = x + c * N + kq;
    // slab sums with integer weights: T[e][d+1]; the 7 values on the axes through q: v7
    df::acc tr[3][3], ti[3][3];
    Val<TI> v7[7];  // centre, then -e0, +e0, -e1, +e1, -e2, +e2
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const bool ok = inside(i + dx, j + dy, k + dz) && qc + sel3(c, dx, dy, dz) >= 1;
          const Val<TI> v = val(ok ? u[dx + dy * sy + dz * sz] : czero<TI>());
          const float wx = dx == 0 ? 2.f : 1.f, wy = dy == 0 ? 2.f : 1.f, wz = dz == 0 ? 2.f : 1.f;
          wadd(tr[0][dx + 1], ti[0][dx + 1], v, wy * wz);
          wadd(tr[1][dy + 1], ti[1][dy + 1], v, wx * wz);
          wadd(tr[2][dz + 1], ti[2][dz + 1], v, wx * wy);
          const int nz0 = (dx != 0) + (dy != 0) + (dz != 0);
          if (nz0 == 0) v7[0] = v;
          if (nz0 == 1) v7[dx != 0 ? (dx < 0 ? 1 : 2) : dy != 0 ? (dy < 0 ? 3 : 4) : (dz < 0 ? 5 : 6)] = v;
        }
    // S_e(d) = beta v(axis point) + kappa T_e(d)
    c2 S[3][3];
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
      for (int d = -1; d <= 1; ++d) {
        const Val<TI> va = d == 0 ? v7[0] : v7[1 + 2 * e + (d > 0)];
        S[e][d + 1] = {add(mulv(g.beta, va.re), mul(g.kap, tr[e][d + 1].norm())),
                       add(mulv(g.beta, va.im), mul(g.kap, ti[e][d + 1].norm()))};
      }
    {
      const c2 Sc0 = sel3(c, S[0][1], S[1][1], S[2][1]), Sc1 = sel3(c, S[0][2], S[1][2], S[2][2]);
      const c2 dd = csub(Sc1, Sc0);
      dv.re.add(dd.re);
      dv.im.add(dd.im);
    }
    if (qc < 1) {
      ff2::store_row<FFO>(y, c * N + kq, cacc{});
    } else {
      // mu beside q along each derivative axis: cell centres for e = c, edge means otherwise
      df::acc lr, li;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        f2 ma, mb;
        if (e == c) {
          ma = g.mu[lin(g, iclamp(i - (e == 0), 0, g.nx - 1), iclamp(j - (e == 1), 0, g.ny - 1),
                        iclamp(k - (e == 2), 0, g.nz - 1))];
          mb = g.mu[kq];
        } else {
          const int rr = 3 - c - e;
          const f2* E = sel3(rr, g.edge[0], g.edge[1], g.edge[2]);
          ma = E[lat(g, i, j, k)];
          mb = E[lat(g, i + (e == 0), j + (e == 1), k + (e == 2))];
        }
        const c2 dA = csub(S[e][1], S[e][0]), dB = csub(S[e][1], S[e][2]);
        lr.fma_ff(ma, dA.re);
        lr.fma_ff(mb, dB.re);
        li.fma_ff(ma, dA.im);
        li.fma_ff(mb, dB.im);
      }
      cacc r;
      r.re.add(mul(g.ih2, lr.norm()));
      r.im.add(mul(g.ih2, li.norm()));
      // mass: -(beta m u) at the face, -(sm m u) at its 6 neighbours (Eq. massHO3D), summed as
      // -beta A0 - sm A6 with A0 = m u at the face and A6 the sum over the neighbours
      const c2* mc = sel3(c, g.m[0], g.m[1], g.m[2]);
      cacc a0, a6;
#pragma unroll
      for (int t = 0; t < 7; ++t) {
        const int ax = (t - 1) / 2, sg = (t & 1) ? -1 : 1;
        const int dx = t > 0 && ax == 0 ? sg : 0, dy = t > 0 && ax == 1 ? sg : 0, dz = t > 0 && ax == 2 ? sg : 0;
        const bool ok = inside(i + dx, j + dy, k + dz) && qc + sel3(c, dx, dy, dz) >= 1;
        if (!ok) continue;
        const c2 m = mshift(mc[(long long)kq + dx + dy * sy + dz * sz]);
        (t == 0 ? a0 : a6).cterm(m, asf2(v7[t].re), asf2(v7[t].im));
      }
      r.re.fms_ff(g.beta, a0.re.norm());
      r.im.fms_ff(g.beta, a0.im.norm());
      r.re.fms_ff(g.sm, a6.re.norm());
      r.im.fms_ff(g.sm, a6.im.norm());
      // gradient: + (p(q) - p(q - e_c)) / h
      const cx<TI>* p = x + 3 * N + kq;
      const Val<TI> pc = val(p[0]), pm = val(p[-sel3(c, sl[0], sl[1], sl[2])]);
      r.rterm(g.ih, asf2(pc.re), asf2(pc.im));
      r.rterm(fneg(g.ih), asf2(pm.re), asf2(pm.im));
      finish(r, c * N + kq);
    }
  }
  {
    cacc r;
    r.re.add(mul(g.ih, dv.re.norm()));
    r.im.add(mul(g.ih, dv.im.norm()));
    const Val<TI> pc = val(x[3 * N + kq]);
    r.rterm(g.cp[kq], asf2(pc.re), asf2(pc.im));
    finish(r, 3 * N + kq);
  }
}

// The same rows in their direct 27-point form: the coefficient C(delta) of every point formed in
// float-float from part_e and W, then the products. About twice the instructions of the factored
// form, but 63 registers: for FP64 input, whose split values double the factored form's live
// registers (150, one block per SM), it is the faster form (10.7 against ~19 ms per 256^3 launch).
template <typename TI, bool FFO = false>
HD void cell_rows_direct(const FineFF3& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y, int i, int j,
                         int k) {
  const int q[3] = {i, j, k};
  const size_t N = (size_t)g.nx * g.ny * g.nz, kq = lin(g, i, j, k);
  auto inside = [&](int a, int bb, int c) { return a >= 0 && a < g.nx && bb >= 0 && bb < g.ny && c >= 0 && c < g.nz; };
  auto mclamp = [&](int a, int bb, int c) {
    return g.mu[lin(g, iclamp(a, 0, g.nx - 1), iclamp(bb, 0, g.ny - 1), iclamp(c, 0, g.nz - 1))];
  };
  auto mshift = [&](c2 m) {
    if (g.alpha.hi != 0.f) m.im = add(m.im, fneg(mul(g.alpha, m.re)));
    return m;
  };
  const float bs = b ? df::pow2_float(bscale) : 0.f;
  auto finish = [&](const cacc& r, size_t at) {
    if (!b) {
      ff2::store_row<FFO>(y, at, r);
      return;
    }
    cacc t;
    t.re = df::scaled_sub_acc(b[at].re, bs, bscale, r.re);
    t.im = df::scaled_sub_acc(b[at].im, bs, bscale, r.im);
    ff2::store_row<FFO>(y, at, t);
  };
  for (int c = 0; c < 3; ++c) {
    if (q[c] < 1) {
      ff2::store_row<FFO>(y, c * N + kq, cacc{});
      continue;
    }
    cacc r;
    // part_e for the three derivative axes
    f2 part[3][3];
    for (int e = 0; e < 3; ++e) {
      f2 ma, mb;
      int s[3] = {0, 0, 0};
      s[e] = 1;
      if (e == c) {
        ma = mclamp(i - s[0], j - s[1], k - s[2]);
        mb = mclamp(i, j, k);
      } else {
        const int rr = 3 - c - e;
        ma = g.edge[rr][lat(g, i, j, k)];
        mb = g.edge[rr][lat(g, i + s[0], j + s[1], k + s[2])];
      }
      part[e][0] = fneg(ma);
      part[e][1] = add(ma, mb);
      part[e][2] = fneg(mb);
    }
    const cx<TI>* u = x + c * N;
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          const int a = i + di, bb = j + dj, cc = k + dk;
          const int qa[3] = {a, bb, cc};
          if (!inside(a, bb, cc) || qa[c] < 1) continue;
          const int dl[3] = {di, dj, dk};
          f2 C = {0.f, 0.f};
          for (int e = 0; e < 3; ++e) {
            const int t1 = (e + 1) % 3, t2 = (e + 2) % 3;
            C = add(C, mul(part[e][dl[e] + 1], g.W[dl[t1] + 1][dl[t2] + 1]));
          }
          C = mul(g.ih2, C);
          const cx<TI> uv = u[lin(g, a, bb, cc)];
          const f2 ur = ld(uv.re), ui = ld(uv.im);
          r.rterm(C, ur, ui);
          const int nz0 = (di != 0) + (dj != 0) + (dk != 0);
          if (nz0 <= 1) {
            const c2 m = mshift(g.m[c][lin(g, a, bb, cc)]);
            const f2 f = nz0 == 0 ? g.beta : g.sm;
            r.cterm({fneg(mul(f, m.re)), fneg(mul(f, m.im))}, ur, ui);
          }
        }
    int s[3] = {0, 0, 0};
    s[c] = 1;
    const cx<TI>* p = x + 3 * N;
    const cx<TI> pc = p[kq], pm = p[lin(g, i - s[0], j - s[1], k - s[2])];
    r.rterm(g.ih, ld(pc.re), ld(pc.im));
    r.rterm(fneg(g.ih), ld(pm.re), ld(pm.im));
    finish(r, c * N + kq);
  }
  {
    cacc r;
    for (int c = 0; c < 3; ++c) {
      const int t1 = (c + 1) % 3, t2 = (c + 2) % 3;
      const cx<TI>* u = x + c * N;
      for (int a = -1; a <= 1; ++a)
        for (int bb = -1; bb <= 1; ++bb) {
          int o[3] = {0, 0, 0};
          o[t1] = a;
          o[t2] = bb;
          const f2 wgt = mul(g.ih, g.W[a + 1][bb + 1]);
          // + u_c(q + s_c + o), - u_c(q + o)
          int hi[3] = {i + o[0], j + o[1], k + o[2]};
          int lo[3] = {hi[0], hi[1], hi[2]};
          hi[c] += 1;
          if (inside(hi[0], hi[1], hi[2]) && hi[c] >= 1) {
            const cx<TI> uv = u[lin(g, hi[0], hi[1], hi[2])];
            r.rterm(wgt, ld(uv.re), ld(uv.im));
          }
          if (inside(lo[0], lo[1], lo[2]) && lo[c] >= 1) {
            const cx<TI> uv = u[lin(g, lo[0], lo[1], lo[2])];
            r.rterm(fneg(wgt), ld(uv.re), ld(uv.im));
          }
        }
    }
    const cx<TI> pc = x[3 * N + kq];
    r.rterm(g.cp[kq], ld(pc.re), ld(pc.im));
    finish(r, 3 * N + kq);
  }
}

// The rows as the kernel evaluates them: the factored form for FP32 input (the cycle's output,
// every iteration), the direct form for FP64 input (the iterate, at restarts).
template <typename TI, bool FFO = false>
HD void cell_rows(const FineFF3& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y, int i, int j, int k) {
  if constexpr (sizeof(TI) == 8) cell_rows_direct<TI, FFO>(g, x, b, bscale, y, i, j, k);
  else cell_rows_factored<TI, FFO>(g, x, b, bscale, y, i, j, k);
}

template <typename TI, bool FFO>
__global__ void __launch_bounds__(BX * BY * BZ) apply(FineFF3 g, const cx<TI>* __restrict__ x,
                                                     const cx<double>* __restrict__ b, double bscale,
                                                     void* __restrict__ y) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z * BZ + threadIdx.z;
  if (i >= g.nx || j >= g.ny || k >= g.nz) return;
  cell_rows<TI, FFO>(g, x, b, bscale, y, i, j, k);
}

}  // namespace ff3
