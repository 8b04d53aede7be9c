// 2D residual and restriction in one pass, FP32: b_2h = R (b - H_s x) (Eq. 2.11-2.13, Alg. 1
// step 2) without writing the fine residual to memory.
//
// A block owns a coarse tile of TX/2 x TY/2 coarse cells, i.e. the fine tile of the one-pass sweep
// (k2t::Geo<TY>), and loads the same shared region: x, mu and rho of the fine tile plus a ring of
// HALO cells, by TMA, with the same boundary handling (zeros outside the domain, clamped material,
// zeroed boundary faces). Phase 1 forms the displacement rows of the fine residual on every fine
// cell that the restriction of the tile reads (the tile and one more column and row on the low
// sides, for R_u's [1 2 1] weights) into shared memory; phase 2 restricts them, R_u = [1 2 1]/4
// along the face normal x [1 1]/2 across, and forms the pressure residual of the four children of
// each coarse cell on the fly for R_p (their mean). Rows: Eq. 3.10 with the sign of Eq. 4.4, the
// same arithmetic as k2::residual_cell.
#pragma once
#include "sweep2d_tile.cuh"

namespace k2t {

// The u1 row at face (gi, gj) and the u2 row at face (gi, gj) of the residual of the state in s,
// for the cell at local (lx, ly); excluded faces (not unknowns) get 0.
template <bool NOABL>
HD void resid_u_rows(const Grid<float>& g, const View& s, int lx, int ly, int gi, int gj, const cx<float>* __restrict__ b,
                     cx<float>& r1, cx<float>& r2) {
  using T = float;
  const int nx = g.nx, ny = g.ny;
  const size_t N = (size_t)nx * ny, k = (size_t)gj * nx + gi;
  const int c0 = ly * DX + lx;
  const T t0 = T(0.5) * (T(1) + g.beta), t1 = T(0.25) * (T(1) - g.beta);
  const T ih = g.ih, ih2 = g.ih * g.ih, w2 = g.w2, att = g.att, h5 = T(0.5);
  const cx<T> z = czero<T>();
  const bool ex1 = gi == 0, ex2 = gj == 0;
  const cx<T> b1 = ex1 ? z : ldg(b + k), b2 = ex2 ? z : ldg(b + N + k);
  T mu9[3][3];
#pragma unroll
  for (int rr = 0; rr < 3; ++rr)
#pragma unroll
    for (int c = 0; c < 3; ++c) mu9[rr][c] = lds(s.mu + c0 + (rr - 1) * DX + (c - 1));
  const T mnA = T(0.25) * (mu9[0][0] + mu9[0][1] + mu9[1][0] + mu9[1][1]);  // node (i, j)
  const T mnB = T(0.25) * (mu9[0][1] + mu9[0][2] + mu9[1][1] + mu9[1][2]);  // node (i+1, j)
  const T mnC = T(0.25) * (mu9[1][0] + mu9[1][1] + mu9[2][0] + mu9[2][1]);  // node (i, j+1)
  auto RHO = [&](int dx, int dy) { return lds(s.rho + c0 + dy * DX + dx); };
  // face masses m_f = rho_f omega^2 (1 - i (att + gamma_ABL)) at u1 face (gi+dx, gj+dy) / u2 face
  auto m1 = [&](int dx, int dy) -> cx<T> {
    const T a = h5 * (RHO(dx - 1, dy) + RHO(dx, dy)) * w2;
    return mkc<T>(a, NOABL ? -a * att
                           : -a * (att + k2::abl_at(g, 0, gi + dx, 0, g.Lx) + k2::abl_at(g, 1, gj + dy, 1, g.Ly)));
  };
  auto m2 = [&](int dx, int dy) -> cx<T> {
    const T a = h5 * (RHO(dx, dy - 1) + RHO(dx, dy)) * w2;
    return mkc<T>(a, NOABL ? -a * att
                           : -a * (att + k2::abl_at(g, 0, gi + dx, 1, g.Lx) + k2::abl_at(g, 1, gj + dy, 0, g.Ly)));
  };
  const cx<T> pC = lds(s.p + c0);
  const cx<T> cm = mkc<T>(h5 * w2, -(h5 * w2) * att);
  {
    cx<T> A[3][3];  // u1 faces i-1..i+1, rows j-1..j+1
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
      for (int c = 0; c < 3; ++c) A[rr][c] = lds(s.u1 + c0 + (rr - 1) * DX + (c - 1));
    auto g1 = [&](int c) {  // d1 u1 at cell (i-1+c, j) without 1/h
      return pfma(t1, padd(psub(A[0][c + 1], A[0][c]), psub(A[2][c + 1], A[2][c])), pscl(t0, psub(A[1][c + 1], A[1][c])));
    };
    auto g2 = [&](int ry) {  // d2 u1 at node (i, j-1+ry) without 1/h
      return pfma(t1, padd(psub(A[ry][0], A[ry - 1][0]), psub(A[ry][2], A[ry - 1][2])), pscl(t0, psub(A[ry][1], A[ry - 1][1])));
    };
    const cx<T> lap = pscl(ih2, padd(psub(pscl(mu9[1][0], g1(0)), pscl(mu9[1][1], g1(1))),
                                     psub(pscl(mnA, g2(1)), pscl(mnC, g2(2)))));
    cx<T> mass;
    if (NOABL) {
      auto rs = [&](int dx, int dy) { return RHO(dx - 1, dy) + RHO(dx, dy); };
      mass = cm * pfma(g.beta, pscl(rs(0, 0), A[1][1]),
                       pscl(g.sm, padd(padd(pscl(rs(-1, 0), A[1][0]), pscl(rs(1, 0), A[1][2])),
                                       padd(pscl(rs(0, -1), A[0][1]), pscl(rs(0, 1), A[2][1])))));
    } else {
      mass = pfma(g.beta, m1(0, 0) * A[1][1],
                  pscl(g.sm, padd(padd(m1(-1, 0) * A[1][0], m1(1, 0) * A[1][2]), padd(m1(0, -1) * A[0][1], m1(0, 1) * A[2][1]))));
    }
    r1 = ex1 ? z : psub(b1, pfma(ih, psub(pC, lds(s.p + c0 - 1)), psub(lap, mass)));
  }
  {
    cx<T> B[3][3];  // u2 faces rows j-1..j+1, columns i-1..i+1
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
      for (int c = 0; c < 3; ++c) B[rr][c] = lds(s.u2 + c0 + (rr - 1) * DX + (c - 1));
    auto h2 = [&](int ry) {  // d2 u2 at cell (i, j-1+ry) without 1/h
      return pfma(t1, padd(psub(B[ry + 1][0], B[ry][0]), psub(B[ry + 1][2], B[ry][2])), pscl(t0, psub(B[ry + 1][1], B[ry][1])));
    };
    auto h1 = [&](int c) {  // d1 u2 at node (i-1+c+1, j) without 1/h
      return pfma(t1, padd(psub(B[0][c + 1], B[0][c]), psub(B[2][c + 1], B[2][c])), pscl(t0, psub(B[1][c + 1], B[1][c])));
    };
    const cx<T> lap = pscl(ih2, padd(psub(pscl(mnA, h1(0)), pscl(mnB, h1(1))),
                                     psub(pscl(mu9[0][1], h2(0)), pscl(mu9[1][1], h2(1)))));
    cx<T> mass;
    if (NOABL) {
      auto rs = [&](int dx, int dy) { return RHO(dx, dy - 1) + RHO(dx, dy); };
      mass = cm * pfma(g.beta, pscl(rs(0, 0), B[1][1]),
                       pscl(g.sm, padd(padd(pscl(rs(-1, 0), B[1][0]), pscl(rs(1, 0), B[1][2])),
                                       padd(pscl(rs(0, -1), B[0][1]), pscl(rs(0, 1), B[2][1])))));
    } else {
      mass = pfma(g.beta, m2(0, 0) * B[1][1],
                  pscl(g.sm, padd(padd(m2(-1, 0) * B[1][0], m2(1, 0) * B[1][2]), padd(m2(0, -1) * B[0][1], m2(0, 1) * B[2][1]))));
    }
    r2 = ex2 ? z : psub(b2, pfma(ih, psub(pC, lds(s.p + c0 - DX)), psub(lap, mass)));
  }
}

// The pressure row of the residual at cell (gi, gj): b_p - (div^beta u + p / (lambda + mu)).
HD cx<float> resid_p_row(const Grid<float>& g, const View& s, int lx, int ly, int gi, int gj,
                         const cx<float>* __restrict__ b) {
  const size_t N = (size_t)g.nx * g.ny, k = (size_t)gj * g.nx + gi;
  const int c0 = ly * DX + lx;
  const float t0 = 0.5f * (1.f + g.beta), t1 = 0.25f * (1.f - g.beta);
  auto U1 = [&](int dx, int dy) { return lds(s.u1 + c0 + dy * DX + dx); };
  auto U2 = [&](int dx, int dy) { return lds(s.u2 + c0 + dy * DX + dx); };
  // d1 u1 and d2 u2 at the cell centre (Eq. 3.5), faces (i, i+1) resp. (j, j+1)
  const cx<float> G1 = pfma(t1, padd(psub(U1(1, -1), U1(0, -1)), psub(U1(1, 1), U1(0, 1))), pscl(t0, psub(U1(1, 0), U1(0, 0))));
  const cx<float> H2 = pfma(t1, padd(psub(U2(-1, 1), U2(-1, 0)), psub(U2(1, 1), U2(1, 0))), pscl(t0, psub(U2(0, 1), U2(0, 0))));
  return psub(ldg(b + 2 * N + k), pfma(ldg(g.cp + k), lds(s.p + c0), pscl(g.ih, padd(G1, H2))));
}

// Phase 1 on fine cell (lx, ly) of the extended tile [HALO-1, HALO+TX) x [HALO-1, HALO+TY):
// its two displacement residual rows into R1, R2 (zero outside the domain).
template <bool NOABL>
HD void resid_phase1(const Grid<float>& g, const Tile& t, const View& s, cx<float>* R1, cx<float>* R2,
                     const cx<float>* b, int lx, int ly) {
  const int gi = t.x0 - HALO + lx, gj = t.y0 - HALO + ly;
  const int c0 = ly * DX + lx;
  cx<float> r1 = czero<float>(), r2 = czero<float>();
  if (gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny) resid_u_rows<NOABL>(g, s, lx, ly, gi, gj, b, r1, r2);
  sts(R1 + c0, r1);
  sts(R2 + c0, r2);
}

// Phase 2 on coarse cell (ci, cj) of the tile: b_2h = R r (R_u1 = (1/8) [1 2 1; 1 2 1] over the fine
// u1 faces 2I-1 .. 2I+1 of rows 2J, 2J+1; R_u2 rotated; R_p the mean of the 4 children).
HD void restrict_phase2(const Grid<float>& g, const Tile& t, const View& s, const cx<float>* R1, const cx<float>* R2,
                        const cx<float>* b, cx<float>* bc, int nxc, int nyc, int ci, int cj) {
  const int I = t.x0 / 2 + ci, J = t.y0 / 2 + cj;
  if (I >= nxc || J >= nyc) return;
  const int fx = HALO + 2 * ci, fy = HALO + 2 * cj, c0 = fy * DX + fx;
  const cx<float> z = czero<float>();
  cx<float> c1 = z, c2 = z, cp = z;
  if (I >= 1) {
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
      const int q = c0 + bb * DX;
      c1 = padd(c1, padd(padd(lds(R1 + q - 1), lds(R1 + q + 1)), pscl(2.f, lds(R1 + q))));
    }
    c1 = pscl(0.125f, c1);
  }
  if (J >= 1) {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int q = c0 + a;
      c2 = padd(c2, padd(padd(lds(R2 + q - DX), lds(R2 + q + DX)), pscl(2.f, lds(R2 + q))));
    }
    c2 = pscl(0.125f, c2);
  }
  const int gi = t.x0 - HALO + fx, gj = t.y0 - HALO + fy;
#pragma unroll
  for (int bb = 0; bb < 2; ++bb)
#pragma unroll
    for (int a = 0; a < 2; ++a) cp = padd(cp, resid_p_row(g, s, fx + a, fy + bb, gi + a, gj + bb, b));
  cp = pscl(0.25f, cp);
  const size_t Nc = (size_t)nxc * nyc, kc = (size_t)J * nxc + I;
  bc[kc] = c1;
  bc[Nc + kc] = c2;
  bc[2 * Nc + kc] = cp;
}

}  // namespace k2t

#ifdef __CUDACC__
namespace k2t {

struct RArgs {
  Grid<float> g;
  const cx<float>* b;  // fine right-hand side (3 components)
  cx<float>* bc;       // coarse right-hand side (3 components of nxc x nyc)
  int nxc, nyc;
  int* err;            // device status word: bit 0 is set if a TMA wait timed out
};

// One block per coarse tile (the fine tile of Geo<TY_>); grid (ceil(nx / TX), ceil(ny / TY)).
template <int TY_>
__global__ void __launch_bounds__(NT, 2) resid_restrict_tile(const __grid_constant__ CUtensorMap tm_x,
                                                             const __grid_constant__ CUtensorMap tm_mu,
                                                             const __grid_constant__ CUtensorMap tm_rho, const RArgs a) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  using G = Geo<TY_>;
  constexpr int PLANE = G::PLANE;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  cx<float>* U = (cx<float>*)(base + G::OFF_U);
  cx<float>* V = (cx<float>*)(base + G::OFF_V);
  float* MU = (float*)(base + G::OFF_MU);
  float* RHO = (float*)(base + G::OFF_RHO);
  const unsigned bar = (unsigned)__cvta_generic_to_shared(base + G::OFF_BAR);
  const Tile t = tile_of<G>(a.g, blockIdx.x, blockIdx.y);
  const int tid = threadIdx.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(G::BYTES_X + G::BYTES_MAT)
                 : "memory");
    tma_3d(U, &tm_x, 2 * (t.x0 - HALO), t.y0 - HALO, 0, bar);
    tma_2d(MU, &tm_mu, t.x0 - HALO, t.y0 - HALO, bar);
    tma_2d(RHO, &tm_rho, t.x0 - HALO, t.y0 - HALO, bar);
  }
  const bool ok = wait_parity(bar, 0);
  if (!__syncthreads_and(ok)) {
    if (tid == 0) atomicOr(a.err, 1);
    wait_parity(bar, 0);  // let copies still in flight land before the block's memory is released
    return;
  }
  if (t.boundary) {
    fix_boundary<G>(a.g, t, U, MU, RHO, tid, NT);
    __syncthreads();
  }
  const View s{U, U + PLANE, U + 2 * PLANE, MU, RHO};
  cx<float>* R1 = V;
  cx<float>* R2 = V + PLANE;
  constexpr int EW = TX + 1, EH = G::TY + 1;  // extended tile
  for (int q = tid; q < EW * EH; q += NT) {
    const int lx = HALO - 1 + q % EW, ly = HALO - 1 + q / EW;
    if (t.noabl) resid_phase1<true>(a.g, t, s, R1, R2, a.b, lx, ly);
    else resid_phase1<false>(a.g, t, s, R1, R2, a.b, lx, ly);
  }
  __syncthreads();
  constexpr int CW = TX / 2, CH = G::TY / 2;
  for (int q = tid; q < CW * CH; q += NT) restrict_phase2(a.g, t, s, R1, R2, a.b, a.bc, a.nxc, a.nyc, q % CW, q / CW);
}

}  // namespace k2t
#endif
