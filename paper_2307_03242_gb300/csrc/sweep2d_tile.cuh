// One full 2D red-black Vanka sweep (colour 0, then colour 1) in a single pass, FP32.
//
// Same arithmetic as two launches of k2::vanka_fast (Eq. 3.10 rows with the sign of Eq. 4.4, the
// cell's 5x5 block of Sec. 2.3 solved by block elimination, Remark 3.1; Jacobi within a colour,
// colour 0 before colour 1, Sec. 3.2), but x, b and the material pass through DRAM once per
// sweep instead of once per half-sweep.
//
// Tiling (overlapped, no communication between blocks). A block owns an output tile of TX x TY
// cells and loads the tile plus a ring of HALO = 4 cells of x (u1, u2, p), mu and rho into shared
// memory with three TMA copies. It relaxes the colour-0 cells of the tile plus a 2-cell ring
// (every colour-0 cell whose result a colour-1 cell of the tile reads: the faces of the colour-1
// cell's 3x4 / 4x3 neighbourhoods and its four pressure neighbours lie at most 2 cells away)
// into a second shared copy of the faces, then relaxes the tile's colour-1 cells from it and
// writes the result to global memory. The ring's colour-0 cells are recomputed by the
// neighbouring blocks (about 1/4 more colour-0 cell solves); their halo loads hit L2.
//
// Work mapping: a warp relaxes a patch of 2 rows x 16 cells of one colour; each half-warp takes 8
// cells of each row (lanes 0-7 and 16-23 on the first row, 8-15 and 24-31 on the second), so that
// the 64-bit shared loads of a half-warp, which the hardware serves together, fall in distinct
// banks (same-colour cells of one row are 2 complex words apart; the second row is offset by an
// odd number of complex words, which moves it to the other half of the banks).
//
// Boundary handling is done once per block in shared memory: TMA fills positions outside the
// grid with zeros (the displacement and pressure outside the domain are zero), material outside
// the domain is replaced by the nearest cell's (clamping), and the boundary faces (u1 at i = 0,
// u2 at j = 0), which are not unknowns, are zeroed.
//
// Complex additions and real-by-complex products use the packed FP32x2 instructions of sm_100+
// (add/mul/fma .rn.f32x2): one instruction per complex operation instead of two.
#pragma once
#include <cmath>

#include "kernels2d.cuh"
#include "vanka2d_fast.cuh"

namespace k2t {

constexpr int TX = 60, HALO = 4;
constexpr int DX = TX + 2 * HALO;  // shared region width (68 cells)
constexpr int NT = 256;            // threads per block (8 warps)
constexpr int C0_PER_ROW = (DX - 4) / 2;  // 32 colour-0 cells per row of the ring-extended region
constexpr int C1_PER_ROW = TX / 2;        // 30 colour-1 cells per tile row
static_assert(DX % 4 == 0, "TMA boxes: the inner extent must be a multiple of 16 bytes");
static_assert(TX % 4 == 0, "tile origins must keep x aligned to 16 bytes and the colour parity");

// Geometry of a tile of TX x TY_ cells. Large grids use TY_ = 24 (less halo per cell); grids
// with few tiles use TY_ = 8 (more blocks and shorter per-warp chains for the same grid).
// colour-0 region: local rows and columns [2, DX-2) x [2, DY-2); colour-1 region (the tile):
// [HALO, HALO+TX) x [HALO, HALO+TY).
template <int TY_>
struct Geo {
  static constexpr int TY = TY_;
  static constexpr int DY = TY + 2 * HALO;
  static constexpr int PLANE = DX * DY;  // elements of one shared array
  static constexpr int C0_ROWS = DY - 4;
  static constexpr int C0_PATCHES = (C0_ROWS / 2) * ((C0_PER_ROW + 15) / 16);
  static constexpr int C1_PATCHES = (TY / 2) * ((C1_PER_ROW + 15) / 16);
  // Shared-memory layout (bytes from the 128-byte aligned base): u1, u2, p (one 3D TMA box), the
  // colour-0 faces v1, v2, then mu and rho (2D TMA boxes), then the mbarrier.
  static constexpr int OFF_U = 0;
  static constexpr int OFF_V = OFF_U + 3 * PLANE * 8;
  static constexpr int OFF_MU = OFF_V + 2 * PLANE * 8;
  static constexpr int OFF_RHO = (OFF_MU + PLANE * 4 + 127) / 128 * 128;  // 128-byte aligned for TMA
  static constexpr int OFF_BAR = OFF_RHO + PLANE * 4;
  static constexpr int SMEM_BYTES = OFF_BAR + 16 + 128;  // + slack for aligning the base
  static constexpr unsigned BYTES_X = 3u * PLANE * 8u, BYTES_MAT = 2u * PLANE * 4u;
  // The coarse correction of the first post-sweep, staged in the colour-0 face arrays: 3 planes
  // of EX x EY coarse values from coarse origin (x0/2 - 4, y0/2 - 3) (one 3D TMA box; the start
  // column is even so that it is 16-byte aligned), covering every coarse value P reads for a fine
  // position of the shared region: columns x0/2 - 3 .. x0/2 + 33, rows y0/2 - 3 .. y0/2 + TY/2 + 2.
  static constexpr int EX = 40, EY = TY / 2 + 6, EPLANE = EX * EY;
  static constexpr unsigned BYTES_E = 3u * EPLANE * 8u;
  static_assert(TY % 2 == 0, "tile origins must keep the colour parity");
  static_assert(OFF_MU % 128 == 0 && OFF_RHO % 128 == 0, "TMA destinations must be 128-byte aligned");
  static_assert(BYTES_E <= 2u * PLANE * 8u, "E is staged in the colour-0 face arrays, which are written later");
};

// ---- packed complex arithmetic (FP32x2 on the device, plain on the host)
HD cx<float> padd(cx<float> a, cx<float> b) {
#ifdef __CUDA_ARCH__
  cx<float> r;
  asm("{.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\tadd.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;}"
      : "=f"(r.re), "=f"(r.im) : "f"(a.re), "f"(a.im), "f"(b.re), "f"(b.im));
  return r;
#else
  return mkc<float>(a.re + b.re, a.im + b.im);
#endif
}
HD cx<float> psub(cx<float> a, cx<float> b) {
#ifdef __CUDA_ARCH__
  cx<float> r;
  asm("{.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\tsub.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;}"
      : "=f"(r.re), "=f"(r.im) : "f"(a.re), "f"(a.im), "f"(b.re), "f"(b.im));
  return r;
#else
  return mkc<float>(a.re - b.re, a.im - b.im);
#endif
}
// s * a for real s
HD cx<float> pscl(float s, cx<float> a) {
#ifdef __CUDA_ARCH__
  cx<float> r;
  asm("{.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %2};\n\tmov.b64 y, {%3, %4};\n\tmul.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;}"
      : "=f"(r.re), "=f"(r.im) : "f"(s), "f"(a.re), "f"(a.im));
  return r;
#else
  return mkc<float>(s * a.re, s * a.im);
#endif
}
// s * a + c for real s
HD cx<float> pfma(float s, cx<float> a, cx<float> c) {
#ifdef __CUDA_ARCH__
  cx<float> r;
  asm("{.reg .b64 x, y, z, d;\n\tmov.b64 x, {%2, %2};\n\tmov.b64 y, {%3, %4};\n\tmov.b64 z, {%5, %6};\n\tfma.rn.f32x2 d, x, y, z;\n\t"
      "mov.b64 {%0, %1}, d;}"
      : "=f"(r.re), "=f"(r.im) : "f"(s), "f"(a.re), "f"(a.im), "f"(c.re), "f"(c.im));
  return r;
#else
  return mkc<float>(std::fma(s, a.re, c.re), std::fma(s, a.im, c.im));
#endif
}

// Shared-memory accesses through the 32-bit shared window (ld/st.shared with an immediate
// offset) rather than generic 64-bit addresses; plain accesses on the host. volatile keeps them in
// program order relative to the block barriers.
HD cx<float> lds(const cx<float>* p) {
#ifdef __CUDA_ARCH__
  cx<float> v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.re), "=f"(v.im) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
#else
  return *p;
#endif
}
HD float lds(const float* p) {
#ifdef __CUDA_ARCH__
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
#else
  return *p;
#endif
}
HD void sts(cx<float>* p, cx<float> v) {
#ifdef __CUDA_ARCH__
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"((unsigned)__cvta_generic_to_shared(p)), "f"(v.re), "f"(v.im)
               : "memory");
#else
  *p = v;
#endif
}

// Views of the shared arrays, row stride DX, local (lx, ly) = global (x0 - HALO + lx, y0 - HALO + ly).
struct View {
  const cx<float>* u1;
  const cx<float>* u2;
  cx<float>* p;
  const float* mu;
  const float* rho;
};

// k2::cell_solve for a cell with no excluded face, using the structure of the block's coupling
// columns: the gradient column is (1, -1, 1, -1)/h and the divergence row t0 (-1, 1, -1, 1)/h, so
// A^{-1} G needs only the sums of the 2x2 blocks' columns (Remark 3.1; same elimination order).
HD void cell_solve_interior(const cx<float> a1[4], const cx<float> a2[4], float ih, float t0, float cp,
                            const cx<float> r[5], cx<float> d[5]) {
  const cx<float>* A[2] = {a1, a2};
  cx<float> y1[4], q[4];
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    const cx<float>* a = A[blk];
    const int k0 = 2 * blk, k1 = 2 * blk + 1;
    const cx<float> idet = cinv(a[0] * a[3] - a[1] * a[2]);
    y1[k0] = idet * (a[3] * r[k0] - a[1] * r[k1]);
    y1[k1] = idet * (a[0] * r[k1] - a[2] * r[k0]);
    // (A^{-1} G) h = idet [a3 + a1, -(a0 + a2)]
    q[k0] = idet * padd(a[3], a[1]);
    q[k1] = -(idet * padd(a[0], a[2]));
  }
  // S = cp - B A^{-1} G, rp = r_p - B A^{-1} r_u with B = t0/h (-1, 1, -1, 1)
  const float c2 = t0 * ih * ih;
  const cx<float> S = pfma(c2, padd(psub(q[0], q[1]), psub(q[2], q[3])), mkc<float>(cp, 0.f));
  const cx<float> rp = pfma(t0 * ih, padd(psub(y1[0], y1[1]), psub(y1[2], y1[3])), r[4]);
  d[4] = rp * cinv(S);
  const cx<float> dq = pscl(ih, d[4]);
#pragma unroll
  for (int k = 0; k < 4; ++k) d[k] = y1[k] - q[k] * dq;
}

// Relaxes the cell at local (lx, ly) = global (gi, gj), which lies inside the domain: its 5x5
// block against the residual of the state in `s` (faces from s.u1/s.u2, pressures from s.p).
// Returns the new values of its DOFs (u1 W, u1 E, u2 S, u2 N, p); excluded faces get 0.
// ZERO: the state is zero (first half-sweep from a zero guess), so r = b on the cell's DOFs.
// FAST: the cell lies in an interior tile without attenuation (no excluded face, no
// absorbing-layer terms).
template <bool FAST, bool ZERO>
HD void cell(const Grid<float>& g, const View& s, int lx, int ly, int gi, int gj, const cx<float>* __restrict__ b,
             float w, cx<float> out[5]) {
  using T = float;
  const int nx = g.nx, ny = g.ny;
  const size_t N = (size_t)nx * ny, k = (size_t)gj * nx + gi;
  const int c0 = ly * DX + lx;
  const T t0 = T(0.5) * (T(1) + g.beta), t1 = T(0.25) * (T(1) - g.beta);
  const T ih = g.ih, ih2 = g.ih * g.ih;
  const bool exW = !FAST && gi == 0, exE = !FAST && gi + 1 >= nx, exS = !FAST && gj == 0, exN = !FAST && gj + 1 >= ny;
  constexpr bool NOABL = FAST;
  const cx<T> z = czero<T>();
  // b of the cell's DOFs (global), issued first
  cx<T> r[5];
  r[0] = exW ? z : ldg(b + k);
  r[1] = exE ? z : ldg(b + k + 1);
  r[2] = exS ? z : ldg(b + N + k);
  r[3] = exN ? z : ldg(b + N + k + nx);
  r[4] = ldg(b + 2 * N + k);
  const T cpc = ldg(g.cp + k);
  // material from shared memory
  T mu9[3][3];
#pragma unroll
  for (int rr = 0; rr < 3; ++rr)
#pragma unroll
    for (int c = 0; c < 3; ++c) mu9[rr][c] = lds(s.mu + c0 + (rr - 1) * DX + (c - 1));
  const T mnA = T(0.25) * (mu9[0][0] + mu9[0][1] + mu9[1][0] + mu9[1][1]);  // node (i,   j)
  const T mnB = T(0.25) * (mu9[0][1] + mu9[0][2] + mu9[1][1] + mu9[1][2]);  // node (i+1, j)
  const T mnC = T(0.25) * (mu9[1][0] + mu9[1][1] + mu9[2][0] + mu9[2][1]);  // node (i,   j+1)
  const T mnD = T(0.25) * (mu9[1][1] + mu9[1][2] + mu9[2][1] + mu9[2][2]);  // node (i+1, j+1)
  T R0[5], Rm[3], Rp[3];
#pragma unroll
  for (int c = 0; c < 5; ++c) R0[c] = lds(s.rho + c0 + (c - 2));
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Rm[c] = lds(s.rho + c0 - DX + (c - 1));
    Rp[c] = lds(s.rho + c0 + DX + (c - 1));
  }
  const T rS2 = lds(s.rho + c0 - 2 * DX), rN2 = lds(s.rho + c0 + 2 * DX);
  T gxf[4], gxc[3], gyf[4], gyc[3];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    gxf[c] = NOABL ? T(0) : k2::abl_at(g, 0, gi - 1 + c, 0, g.Lx);
    gyf[c] = NOABL ? T(0) : k2::abl_at(g, 1, gj - 1 + c, 0, g.Ly);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    gxc[c] = NOABL ? T(0) : k2::abl_at(g, 0, gi - 1 + c, 1, g.Lx);
    gyc[c] = NOABL ? T(0) : k2::abl_at(g, 1, gj - 1 + c, 1, g.Ly);
  }
  const T w2 = g.w2, att = g.att, h5 = T(0.5);
  auto m1 = [&](T rf, int ox, int oy) -> cx<T> {
    const T a = rf * w2;
    return mkc<T>(a, -a * (att + gxf[ox + 1] + gyc[oy + 1]));
  };
  auto m2 = [&](T rf, int ox, int oy) -> cx<T> {
    const T a = rf * w2;
    return mkc<T>(a, -a * (att + gxc[ox + 1] + gyf[oy + 1]));
  };
  const cx<T> mW = m1(h5 * (R0[1] + R0[2]), 0, 0), mE = m1(h5 * (R0[2] + R0[3]), 1, 0);
  const cx<T> mS = m2(h5 * (Rm[1] + R0[2]), 0, 0), mN = m2(h5 * (R0[2] + Rp[1]), 0, 1);
  cx<T> A11 = z, A12 = z, B11 = z, B21 = z, pC = z;  // the cell's current DOF values
  if (!ZERO) {
    pC = lds(s.p + c0);
    const cx<T> pW = lds(s.p + c0 - 1), pE = lds(s.p + c0 + 1), pS = lds(s.p + c0 - DX), pN = lds(s.p + c0 + DX);
    cx<T> G1c, H2c;
    {
      // u1 on faces i-1..i+2, rows j-1..j+1
      cx<T> A[3][4];
#pragma unroll
      for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int c = 0; c < 4; ++c) A[rr][c] = lds(s.u1 + c0 + (rr - 1) * DX + (c - 1));
      A11 = A[1][1];
      A12 = A[1][2];
      // spread derivatives (Eq. 3.5) without the 1/h, which is applied once per row
      auto g1 = [&](int c) {
        return pfma(t1, padd(psub(A[0][c + 1], A[0][c]), psub(A[2][c + 1], A[2][c])), pscl(t0, psub(A[1][c + 1], A[1][c])));
      };
      auto g2 = [&](int c0_, int ry) {
        return pfma(t1, padd(psub(A[ry][c0_], A[ry - 1][c0_]), psub(A[ry][c0_ + 2], A[ry - 1][c0_ + 2])),
                    pscl(t0, psub(A[ry][c0_ + 1], A[ry - 1][c0_ + 1])));
      };
      const cx<T> G1m = g1(0);
      G1c = g1(1);
      const cx<T> G1p = g1(2);
      const cx<T> G2A = g2(0, 1), G2C = g2(0, 2), G2B = g2(1, 1), G2D = g2(1, 2);
      // ih^2 (mu G1 - mu G1 + mu_node G2 - mu_node G2); the p row keeps G1c / h
      const cx<T> lapW = pscl(ih2, padd(psub(pscl(mu9[1][0], G1m), pscl(mu9[1][1], G1c)), psub(pscl(mnA, G2A), pscl(mnC, G2C))));
      const cx<T> lapE = pscl(ih2, padd(psub(pscl(mu9[1][1], G1c), pscl(mu9[1][2], G1p)), psub(pscl(mnB, G2B), pscl(mnD, G2D))));
      cx<T> massW, massE;
      if (NOABL) {
        const cx<T> cm = mkc<T>(h5 * w2, -(h5 * w2) * att);
        const cx<T> Vw = pscl(R0[1] + R0[2], A[1][1]), Ve = pscl(R0[2] + R0[3], A[1][2]);
        const cx<T> Vww = pscl(R0[0] + R0[1], A[1][0]), Vee = pscl(R0[3] + R0[4], A[1][3]);
        const cx<T> Vws = pscl(Rm[0] + Rm[1], A[0][1]), Vwn = pscl(Rp[0] + Rp[1], A[2][1]);
        const cx<T> Ves = pscl(Rm[1] + Rm[2], A[0][2]), Ven = pscl(Rp[1] + Rp[2], A[2][2]);
        massW = cm * pfma(g.beta, Vw, pscl(g.sm, padd(padd(Vww, Ve), padd(Vws, Vwn))));
        massE = cm * pfma(g.beta, Ve, pscl(g.sm, padd(padd(Vw, Vee), padd(Ves, Ven))));
      } else {
        const cx<T> MUw = mW * A[1][1], MUe = mE * A[1][2];
        const cx<T> MUww = m1(h5 * (R0[0] + R0[1]), -1, 0) * A[1][0];
        const cx<T> MUee = m1(h5 * (R0[3] + R0[4]), 2, 0) * A[1][3];
        const cx<T> MUws = m1(h5 * (Rm[0] + Rm[1]), 0, -1) * A[0][1];
        const cx<T> MUwn = m1(h5 * (Rp[0] + Rp[1]), 0, 1) * A[2][1];
        const cx<T> MUes = m1(h5 * (Rm[1] + Rm[2]), 1, -1) * A[0][2];
        const cx<T> MUen = m1(h5 * (Rp[1] + Rp[2]), 1, 1) * A[2][2];
        massW = pfma(g.beta, MUw, pscl(g.sm, padd(padd(MUww, MUe), padd(MUws, MUwn))));
        massE = pfma(g.beta, MUe, pscl(g.sm, padd(padd(MUw, MUee), padd(MUes, MUen))));
      }
      if (!exW) r[0] = psub(r[0], pfma(ih, psub(pC, pW), psub(lapW, massW)));
      if (!exE) r[1] = psub(r[1], pfma(ih, psub(pE, pC), psub(lapE, massE)));
    }
    {
      // u2 on faces rows j-1..j+2, columns i-1..i+1
      cx<T> B[4][3];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr)
#pragma unroll
        for (int c = 0; c < 3; ++c) B[rr][c] = lds(s.u2 + c0 + (rr - 1) * DX + (c - 1));
      B11 = B[1][1];
      B21 = B[2][1];
      auto h2 = [&](int ry) {
        return pfma(t1, padd(psub(B[ry + 1][0], B[ry][0]), psub(B[ry + 1][2], B[ry][2])), pscl(t0, psub(B[ry + 1][1], B[ry][1])));
      };
      auto h1 = [&](int c0_, int ry) {
        return pfma(t1, padd(psub(B[ry - 1][c0_ + 1], B[ry - 1][c0_]), psub(B[ry + 1][c0_ + 1], B[ry + 1][c0_])),
                    pscl(t0, psub(B[ry][c0_ + 1], B[ry][c0_])));
      };
      const cx<T> H2m = h2(0);
      H2c = h2(1);
      const cx<T> H2p = h2(2);
      const cx<T> H1A = h1(0, 1), H1B = h1(1, 1), H1C = h1(0, 2), H1D = h1(1, 2);
      const cx<T> lapS = pscl(ih2, padd(psub(pscl(mnA, H1A), pscl(mnB, H1B)), psub(pscl(mu9[0][1], H2m), pscl(mu9[1][1], H2c))));
      const cx<T> lapN = pscl(ih2, padd(psub(pscl(mnC, H1C), pscl(mnD, H1D)), psub(pscl(mu9[1][1], H2c), pscl(mu9[2][1], H2p))));
      cx<T> massS, massN;
      if (NOABL) {
        const cx<T> cm = mkc<T>(h5 * w2, -(h5 * w2) * att);
        const cx<T> Vs = pscl(Rm[1] + R0[2], B[1][1]), Vn = pscl(R0[2] + Rp[1], B[2][1]);
        const cx<T> Vss = pscl(rS2 + Rm[1], B[0][1]), Vnn = pscl(Rp[1] + rN2, B[3][1]);
        const cx<T> Vsw = pscl(Rm[0] + R0[1], B[1][0]), Vse = pscl(Rm[2] + R0[3], B[1][2]);
        const cx<T> Vnw = pscl(R0[1] + Rp[0], B[2][0]), Vne = pscl(R0[3] + Rp[2], B[2][2]);
        massS = cm * pfma(g.beta, Vs, pscl(g.sm, padd(padd(Vsw, Vse), padd(Vss, Vn))));
        massN = cm * pfma(g.beta, Vn, pscl(g.sm, padd(padd(Vnw, Vne), padd(Vs, Vnn))));
      } else {
        const cx<T> MUs = mS * B[1][1], MUn = mN * B[2][1];
        const cx<T> MUss = m2(h5 * (rS2 + Rm[1]), 0, -1) * B[0][1];
        const cx<T> MUnn = m2(h5 * (Rp[1] + rN2), 0, 2) * B[3][1];
        const cx<T> MUsw = m2(h5 * (Rm[0] + R0[1]), -1, 0) * B[1][0];
        const cx<T> MUse = m2(h5 * (Rm[2] + R0[3]), 1, 0) * B[1][2];
        const cx<T> MUnw = m2(h5 * (R0[1] + Rp[0]), -1, 1) * B[2][0];
        const cx<T> MUne = m2(h5 * (R0[3] + Rp[2]), 1, 1) * B[2][2];
        massS = pfma(g.beta, MUs, pscl(g.sm, padd(padd(MUsw, MUse), padd(MUss, MUn))));
        massN = pfma(g.beta, MUn, pscl(g.sm, padd(padd(MUnw, MUne), padd(MUs, MUnn))));
      }
      if (!exS) r[2] = psub(r[2], pfma(ih, psub(pC, pS), psub(lapS, massS)));
      if (!exN) r[3] = psub(r[3], pfma(ih, psub(pN, pC), psub(lapN, massN)));
    }
    r[4] = psub(r[4], pfma(cpc, pC, pscl(ih, padd(G1c, H2c))));
  }

  // ---- the cell's block (the entries of s2::block_u1 / block_u2)
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
  if (g.economic) a1[1] = a1[2] = a2[1] = a2[2] = z;
  if (FAST) {
    cell_solve_interior(a1, a2, ih, t0, cpc, r, d);
  } else {
    const bool ex[4] = {exW, exE, exS, exN};
    k2::cell_solve(a1, a2, ex, ih, t0, cpc, r, d);
  }
  out[0] = exW ? z : pfma(w, d[0], A11);
  out[1] = exE ? z : pfma(w, d[1], A12);
  out[2] = exS ? z : pfma(w, d[2], B11);
  out[3] = exN ? z : pfma(w, d[3], B21);
  out[4] = pfma(w, d[4], pC);
}

// Tile origin and the per-block variant choice.
struct Tile {
  int x0, y0;       // global index of local (HALO, HALO)
  bool boundary;    // the shared region reaches outside the domain
  bool noabl;       // no attenuation on any lattice position of the shared region
  bool fast;        // interior and without attenuation: the cells take the specialised variant
};

template <class G>
HD Tile tile_of(const Grid<float>& g, int bx, int by) {
  Tile t;
  t.x0 = bx * TX;
  t.y0 = by * G::TY;
  t.boundary = t.x0 - HALO < 0 || t.y0 - HALO < 0 || t.x0 + TX + HALO > g.nx || t.y0 + G::TY + HALO > g.ny;
  t.noabl = g.abl_free(0, t.x0 - HALO, t.x0 + TX + HALO) && g.abl_free(1, t.y0 - HALO, t.y0 + G::TY + HALO);
  t.fast = t.noabl && !t.boundary;
  return t;
}

// Boundary fix-up of a loaded shared region: material outside the domain takes the nearest
// cell's value (the clamped material of the rows), and the faces that are not unknowns are zero.
// Thread t of nthr handles every nthr-th position.
template <class G>
HD void fix_boundary(const Grid<float>& g, const Tile& t, cx<float>* U, float* MU, float* RHO, int tid, int nthr) {
  constexpr int PLANE = G::PLANE;
  for (int q = tid; q < PLANE; q += nthr) {
    const int lx = q % DX, ly = q / DX;
    const int gx = t.x0 - HALO + lx, gy = t.y0 - HALO + ly;
    const bool out = gx < 0 || gx >= g.nx || gy < 0 || gy >= g.ny;
    if (out) {
      const int cx_ = iclamp(gx, 0, g.nx - 1) - (t.x0 - HALO), cy_ = iclamp(gy, 0, g.ny - 1) - (t.y0 - HALO);
      MU[q] = MU[cy_ * DX + cx_];
      RHO[q] = RHO[cy_ * DX + cx_];
    }
    if (gx == 0) U[q] = czero<float>();              // u1 boundary face
    if (gy == 0) U[PLANE + q] = czero<float>();      // u2 boundary face
  }
}

// ---- prolongation + correction on load (the first post-sweep of a cycle)
// State += P e on every in-domain position of the shared region (Eq. 2.11-2.12): P_u linear
// along the face normal and [1 3 3 1]/4 across, P_p bilinear; fine boundary faces (i = 0 for u1,
// j = 0 for u2) are not unknowns and coarse boundary faces carry nothing. Work item: one coarse
// cell (I, J) and its 2 x 2 fine cells (the shared region starts on an even fine index in both
// directions), from the 21 coarse values around it. FAST (interior tiles): every fine position is
// inside the domain and every coarse value P reads exists, so no test is made.
template <class G, bool FAST>
HD void add_prolonged(const Grid<float>& g, const Tile& t, cx<float>* U, const cx<float>* E, int nxc, int nyc, int tid,
                      int nthr) {
  constexpr int PLANE = G::PLANE, EX = G::EX, EPLANE = G::EPLANE;
  constexpr int BX = DX / 2, BY = G::DY / 2;  // coarse cells of the shared region
  const float a = 0.75f, c = 0.25f, hf = 0.5f;
  const int I0 = (t.x0 - HALO) / 2, J0 = (t.y0 - HALO) / 2;  // coarse cell of the region's first fine cell
  const int ex0 = t.x0 / 2 - 4, ey0 = t.y0 / 2 - 3;
  for (int q = tid; q < BX * BY; q += nthr) {
    const int m = q % BX, n = q / BX;
    const int I = I0 + m, J = J0 + n;
    const cx<float> z = czero<float>();
    // coarse values at (I + di, J + dj), di, dj in {-1, 0, 1}; zero where the coarse DOF does not exist
    auto ld = [&](int comp, int di, int dj) -> cx<float> {
      const int II = I + di, JJ = J + dj;
      if (!FAST) {
        const bool okx = comp == 0 ? (II >= 1 && II < nxc) : (II >= 0 && II < nxc);
        const bool oky = comp == 1 ? (JJ >= 1 && JJ < nyc) : (JJ >= 0 && JJ < nyc);
        if (!okx || !oky) return z;
      }
      return lds(E + comp * EPLANE + (JJ - ey0) * EX + (II - ex0));
    };
    const int lx = 2 * m, ly = 2 * n, c0 = ly * DX + lx;
    const int gx = t.x0 - HALO + lx, gy = t.y0 - HALO + ly;
    // which of the 2 x 2 fine cells lie inside the domain (all of them in interior tiles)
    const bool in00 = FAST || (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny);
    const bool in10 = FAST || (gx + 1 >= 0 && gx + 1 < g.nx && gy >= 0 && gy < g.ny);
    const bool in01 = FAST || (gx >= 0 && gx < g.nx && gy + 1 >= 0 && gy + 1 < g.ny);
    const bool in11 = FAST || (gx + 1 >= 0 && gx + 1 < g.nx && gy + 1 >= 0 && gy + 1 < g.ny);
    auto add = [&](int off, bool in, cx<float> v) {
      if (in) sts(U + off, padd(lds(U + off), v));
    };
    {  // u1: faces 2I (coarse face I) and 2I+1 (mean of faces I, I+1); rows 2J (with J-1) and 2J+1 (with J+1)
      const cx<float> fm = ld(0, 0, -1), f0 = ld(0, 0, 0), fp = ld(0, 0, 1);
      const cx<float> gm = ld(0, 1, -1), g0 = ld(0, 1, 0), gp = ld(0, 1, 1);
      const cx<float> aS = pfma(a, f0, pscl(c, fm)), aN = pfma(a, f0, pscl(c, fp));
      const cx<float> bS = pfma(a, g0, pscl(c, gm)), bN = pfma(a, g0, pscl(c, gp));
      add(c0, in00, aS);
      add(c0 + 1, in10, pscl(hf, padd(aS, bS)));
      add(c0 + DX, in01, aN);
      add(c0 + DX + 1, in11, pscl(hf, padd(aN, bN)));
    }
    {  // u2: rows 2J (coarse face J) and 2J+1 (mean of J, J+1); columns 2I (with I-1) and 2I+1 (with I+1)
      const cx<float> fm = ld(1, -1, 0), f0 = ld(1, 0, 0), fp = ld(1, 1, 0);
      const cx<float> gm = ld(1, -1, 1), g0 = ld(1, 0, 1), gp = ld(1, 1, 1);
      const cx<float> aW = pfma(a, f0, pscl(c, fm)), aE = pfma(a, f0, pscl(c, fp));
      const cx<float> bW = pfma(a, g0, pscl(c, gm)), bE = pfma(a, g0, pscl(c, gp));
      add(PLANE + c0, in00, aW);
      add(PLANE + c0 + 1, in10, aE);
      add(PLANE + c0 + DX, in01, pscl(hf, padd(aW, bW)));
      add(PLANE + c0 + DX + 1, in11, pscl(hf, padd(aE, bE)));
    }
    {  // p: bilinear, 3/4 on the own coarse cell, 1/4 on the neighbour towards the fine cell
      cx<float> e[3][3];
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
        for (int di = -1; di <= 1; ++di) e[dj + 1][di + 1] = ld(2, di, dj);
      const cx<float> rW = pfma(a, e[1][1], pscl(c, e[1][0])), rE = pfma(a, e[1][1], pscl(c, e[1][2]));
      const cx<float> sW = pfma(a, e[0][1], pscl(c, e[0][0])), sE = pfma(a, e[0][1], pscl(c, e[0][2]));
      const cx<float> nW = pfma(a, e[2][1], pscl(c, e[2][0])), nE = pfma(a, e[2][1], pscl(c, e[2][2]));
      add(2 * PLANE + c0, in00, pfma(a, rW, pscl(c, sW)));
      add(2 * PLANE + c0 + 1, in10, pfma(a, rE, pscl(c, sE)));
      add(2 * PLANE + c0 + DX, in01, pfma(a, rW, pscl(c, nW)));
      add(2 * PLANE + c0 + DX + 1, in11, pfma(a, rE, pscl(c, nE)));
    }
  }
}

// Local position of the colour-0 cell of patch `patch`, lane `lane` (valid if the cell exists).
HD void c0_pos(int patch, int lane, int& lx, int& ly) {
  const int rp = patch >> 1, half = patch & 1;
  ly = 2 + 2 * rp + ((lane >> 3) & 1);
  const int kk = 16 * half + (lane & 7) + 8 * (lane >> 4);
  lx = 2 + (ly & 1) + 2 * kk;
}
// Local position of the colour-1 cell of patch `patch`, lane `lane`; false past the row's end.
HD bool c1_pos(int patch, int lane, int& lx, int& ly) {
  const int rp = patch >> 1, half = patch & 1;
  ly = HALO + 2 * rp + ((lane >> 3) & 1);
  const int kk = 16 * half + (lane & 7) + 8 * (lane >> 4);
  lx = HALO + ((ly + 1) & 1) + 2 * kk;
  return kk < C1_PER_ROW;
}

// Colour-0 relaxation of one cell of the ring-extended region into v1/v2 (faces) and p (in place).
template <bool FAST, bool ZERO>
HD void relax_c0(const Grid<float>& g, const Tile& t, const View& s, cx<float>* v1, cx<float>* v2,
                 const cx<float>* b, float w, int lx, int ly) {
  const int gi = t.x0 - HALO + lx, gj = t.y0 - HALO + ly;
  if (!FAST && (gi < 0 || gi >= g.nx || gj < 0 || gj >= g.ny)) return;
  cx<float> o[5];
  cell<FAST, ZERO>(g, s, lx, ly, gi, gj, b, w, o);
  const int c0 = ly * DX + lx;
  sts(v1 + c0, o[0]);
  sts(v1 + c0 + 1, o[1]);
  sts(v2 + c0, o[2]);
  sts(v2 + c0 + DX, o[3]);
  sts(s.p + c0, o[4]);
}

// Colour-1 relaxation of one tile cell from the colour-0 state; writes its faces, its pressure
// and its colour-0 partner's pressure (the aligned pair) to the global result.
template <bool FAST>
HD void relax_c1(const Grid<float>& g, const Tile& t, const View& s, const cx<float>* b, cx<float>* xout, float w,
                 int lx, int ly) {
  const int gi = t.x0 - HALO + lx, gj = t.y0 - HALO + ly;
  if (!FAST && (gi >= g.nx || gj >= g.ny)) return;
  cx<float> o[5];
  cell<FAST, false>(g, s, lx, ly, gi, gj, b, w, o);
  const int nx = g.nx;
  const size_t N = (size_t)nx * g.ny, k = (size_t)gj * nx + gi;
  cx<float>* o1 = xout;
  cx<float>* o2 = xout + N;
  cx<float>* op = xout + 2 * N;
  o1[k] = o[0];
  if (FAST || gi + 1 < nx) o1[k + 1] = o[1];
  o2[k] = o[2];
  if (FAST || gj + 1 < g.ny) o2[k + nx] = o[3];
  // faces no colour-1 cell owns: the boundary face west of a colour-0 cell at i = 0 (resp. south of one at j = 0)
  if (!FAST && gi == 1) o1[k - 1] = czero<float>();
  if (!FAST && gj == 1) o2[k - nx] = czero<float>();
  const int c0 = ly * DX + lx;
  const int pi = gi ^ 1;  // the other cell of the aligned pair (2m, 2m+1), colour 0
  if (FAST || pi < nx) {
    const cx<float> pp = lds(s.p + c0 + (pi - gi));
    op[k + (pi - gi)] = pp;
  }
  op[k] = o[4];
}

}  // namespace k2t

#ifdef __CUDACC__
#include <cuda.h>  // CUtensorMap (the tensor maps are encoded by the launcher)

namespace k2t {

struct Args {
  Grid<float> g;
  const cx<float>* b;  // right-hand side of the level (3 components)
  cx<float>* xout;     // the swept state; must not alias the input the tensor map describes
  float w;             // damping
  int zero_in;         // the input state is zero: x is not read
  int* err;            // device status word: bit 0 is set if a TMA wait timed out
  int pro;             // add P e (e: the coarse correction of the tensor map tm_e) to x first
  int nxc, nyc;        // coarse grid of e
};

// An mbarrier wait that gives up after about 2 s (4e9 SM cycles): a copy that never lands must
// not hang the GPU. Returns false on timeout.
__device__ __forceinline__ bool wait_parity(unsigned bar, unsigned parity) {
  const long long start = clock64();
  for (;;) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - start > 4000000000LL) return false;
    __nanosleep(64);  // yield the issue slots to the other block's warps while the copy is in flight
  }
}

__device__ __forceinline__ void tma_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      :
      : "r"((unsigned)__cvta_generic_to_shared(dst)), "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int c0, int c1, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      :
      : "r"((unsigned)__cvta_generic_to_shared(dst)), "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

template <class G, bool FAST, bool ZERO>
__device__ __forceinline__ void phase_c0(const Args& a, const Tile& t, const View& s, cx<float>* v1, cx<float>* v2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int patch = warp; patch < G::C0_PATCHES; patch += NT / 32) {
    int lx, ly;
    c0_pos(patch, lane, lx, ly);
    relax_c0<FAST, ZERO>(a.g, t, s, v1, v2, a.b, a.w, lx, ly);
  }
}
template <class G, bool FAST>
__device__ __forceinline__ void phase_c1(const Args& a, const Tile& t, const View& s) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int patch = warp; patch < G::C1_PATCHES; patch += NT / 32) {
    int lx, ly;
    if (c1_pos(patch, lane, lx, ly)) relax_c1<FAST>(a.g, t, s, a.b, a.xout, a.w, lx, ly);
  }
}

// One block per output tile; grid (ceil(nx / TX), ceil(ny / TY)).
template <int TY_>
__global__ void __launch_bounds__(NT, 2) sweep_tile(const __grid_constant__ CUtensorMap tm_x,
                                                    const __grid_constant__ CUtensorMap tm_mu,
                                                    const __grid_constant__ CUtensorMap tm_rho,
                                                    const __grid_constant__ CUtensorMap tm_e, const Args a) {
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
    const unsigned bytes = (a.zero_in ? 0u : G::BYTES_X) + G::BYTES_MAT + (a.pro ? G::BYTES_E : 0u);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    // x is a 3D float tensor (2 nx, ny, 3): the start column 2 (x0 - HALO) is a multiple of 8 floats
    if (!a.zero_in) tma_3d(U, &tm_x, 2 * (t.x0 - HALO), t.y0 - HALO, 0, bar);
    tma_2d(MU, &tm_mu, t.x0 - HALO, t.y0 - HALO, bar);
    tma_2d(RHO, &tm_rho, t.x0 - HALO, t.y0 - HALO, bar);
    // e (2 nxc, nyc, 3) into the colour-0 face arrays: start column 2 (x0/2 - 4), a multiple of 4 floats
    if (a.pro) tma_3d(V, &tm_e, 2 * (t.x0 / 2 - 4), t.y0 / 2 - 3, 0, bar);
  }
  // while the copies are in flight: zero what is not loaded
  if (a.zero_in)
    for (int q = tid; q < 3 * PLANE; q += NT) U[q] = czero<float>();
  if (t.boundary && !a.pro)
    for (int q = tid; q < 2 * PLANE; q += NT) V[q] = czero<float>();
  const bool ok = wait_parity(bar, 0);
  if (!__syncthreads_and(ok)) {
    if (tid == 0) atomicOr(a.err, 1);
    wait_parity(bar, 0);  // let copies still in flight land before the block's memory is released
    return;
  }
  if (a.pro) {
    if (t.fast) add_prolonged<G, true>(a.g, t, U, V, a.nxc, a.nyc, tid, NT);
    else add_prolonged<G, false>(a.g, t, U, V, a.nxc, a.nyc, tid, NT);
    __syncthreads();  // E (in V) has been read
    if (t.boundary)
      for (int q = tid; q < 2 * PLANE; q += NT) V[q] = czero<float>();
  }
  if (t.boundary) {
    fix_boundary<G>(a.g, t, U, MU, RHO, tid, NT);
    __syncthreads();
  }
  View s{U, U + PLANE, U + 2 * PLANE, MU, RHO};
  cx<float>* v1 = V;
  cx<float>* v2 = V + PLANE;
  if (t.fast) {
    if (a.zero_in) phase_c0<G, true, true>(a, t, s, v1, v2);
    else phase_c0<G, true, false>(a, t, s, v1, v2);
  } else {
    if (a.zero_in) phase_c0<G, false, true>(a, t, s, v1, v2);
    else phase_c0<G, false, false>(a, t, s, v1, v2);
  }
  __syncthreads();
  const View s1{v1, v2, U + 2 * PLANE, MU, RHO};
  if (t.fast) phase_c1<G, true>(a, t, s1);
  else phase_c1<G, false>(a, t, s1);
}

}  // namespace k2t
#endif
