// 3D red-black half-sweep with a shared-memory tile.
//
// Same arithmetic as k3::vanka (rows of Eq. 3.10 with the sign of Eq. 4.4 in the 3D form of
// Sec. 5.3; the cell's 7x7 block solved by block elimination, Remark 3.1). A block of 256 threads
// owns TX x TY x TZ = 16 x 8 x 4 cells, one thread per cell of the colour. Phase 1 stages u1..u3,
// p, mu and the complex face masses on a halo box [-2, TX+2) x [-1, TY+2) x [-1, TZ+2) around
// the tile, and b on the tile's faces, with the boundary handled at load time. Phase 2 has no
// bounds checks. Columns (x) are stored de-interleaved by parity.
#pragma once
#include "kernels3d.cuh"

namespace k3t {

constexpr int TX = 16, TY = 8, TZ = 4, NT = 256;
constexpr int WX = TX + 4, HX = WX / 2, WY = TY + 3, WZ = TZ + 3;  // halo box extents
constexpr int NS = WX * WY * WZ;
// b_c staged on the tile faces: along c one extra layer
constexpr int B0 = (TX + 1) * TY * TZ, B1 = TX * (TY + 1) * TZ, B2 = TX * TY * (TZ + 1), BP = TX * TY * TZ;

template <typename T>
struct Tile {
  cx<T> u[3][NS];
  cx<T> p[NS];
  cx<T> m[3][NS];
  T mu[NS];
  cx<T> b0[B0], b1[B1], b2[B2], bp[BP];
};

HD int colx(int cxx) { return (cxx & 1) * HX + (cxx >> 1); }
// slot of the halo-box coordinates (cxx = x - (x0-2), cy = y - (y0-1), cz = z - (z0-1))
HD int slot(int cxx, int cy, int cz) { return (cz * WY + cy) * WX + colx(cxx); }

template <typename T> HD T ablt(const Grid<T>& g, T x, T L) {
  return g.ablL > T(0) ? g.ablG * abl_axis(x, g.ablL, L) / (g.ablL * g.ablL) : T(0);
}

template <typename T>
HD void tile_load(Tile<T>& s, const Grid<T>& g, const cx<T>* b, const cx<T>* uin, const cx<T>* p, int zero_in, int x0,
                  int y0, int z0, int tid) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const size_t N = (size_t)nx * ny * nz;
  const cx<T> z = czero<T>();
  const T h5 = T(0.5), w2 = g.w2, att = g.att;
  auto cl = [&](int i, int j, int k) {
    return ((size_t)iclamp(k, 0, nz - 1) * ny + iclamp(j, 0, ny - 1)) * nx + iclamp(i, 0, nx - 1);
  };
  for (int e = tid; e < NS; e += NT) {
    const int cxx = e % WX, cy = (e / WX) % WY, cz = e / (WX * WY);
    const int x = x0 - 2 + cxx, y = y0 - 1 + cy, zz = z0 - 1 + cz;
    const int sl = slot(cxx, cy, cz);
    const bool in = x >= 0 && x < nx && y >= 0 && y < ny && zz >= 0 && zz < nz;
    const size_t q = in ? ((size_t)zz * ny + y) * nx + x : 0;
    const int idx[3] = {x, y, zz};
#pragma unroll
    for (int c = 0; c < 3; ++c) s.u[c][sl] = (!zero_in && in && idx[c] >= 1) ? uin[c * N + q] : z;
    s.p[sl] = (!zero_in && in) ? p[q] : z;
    s.mu[sl] = ldg(g.mu + cl(x, y, zz));
    const T rq = ldg(g.rho + cl(x, y, zz));
    const T gx0 = ablt(g, T(x) * g.h, g.Lx), gx5 = ablt(g, (T(x) + h5) * g.h, g.Lx);
    const T gy0 = ablt(g, T(y) * g.h, g.Ly), gy5 = ablt(g, (T(y) + h5) * g.h, g.Ly);
    const T gz0 = ablt(g, T(zz) * g.h, g.Lz), gz5 = ablt(g, (T(zz) + h5) * g.h, g.Lz);
    {
      const T a = h5 * (ldg(g.rho + cl(x - 1, y, zz)) + rq) * w2;
      s.m[0][sl] = mkc<T>(a, -a * (att + gx0 + gy5 + gz5));
    }
    {
      const T a = h5 * (ldg(g.rho + cl(x, y - 1, zz)) + rq) * w2;
      s.m[1][sl] = mkc<T>(a, -a * (att + gx5 + gy0 + gz5));
    }
    {
      const T a = h5 * (ldg(g.rho + cl(x, y, zz - 1)) + rq) * w2;
      s.m[2][sl] = mkc<T>(a, -a * (att + gx5 + gy5 + gz0));
    }
  }
  // b on the tile's faces (component c: one extra layer along c)
  for (int e = tid; e < B0 + B1 + B2 + BP; e += NT) {
    int c, r, ex, ey;
    if (e < B0) { c = 0; r = e; ex = TX + 1; ey = TY; }
    else if (e < B0 + B1) { c = 1; r = e - B0; ex = TX; ey = TY + 1; }
    else if (e < B0 + B1 + B2) { c = 2; r = e - B0 - B1; ex = TX; ey = TY; }
    else { c = 3; r = e - B0 - B1 - B2; ex = TX; ey = TY; }
    const int lx = r % ex, ly = (r / ex) % ey, lz = r / (ex * ey);
    const int x = x0 + lx, y = y0 + ly, zz = z0 + lz;
    const bool in = x < nx && y < ny && zz < nz;
    const int idx[3] = {x, y, zz};
    cx<T> v = z;
    if (in && (c == 3 || idx[c] >= 1)) v = b[c * N + ((size_t)zz * ny + y) * nx + x];
    if (c == 0) s.b0[r] = v;
    else if (c == 1) s.b1[r] = v;
    else if (c == 2) s.b2[r] = v;
    else s.bp[r] = v;
  }
}

template <typename T>
HD void tile_compute(const Tile<T>& s, const Grid<T>& g, cx<T>* uout, cx<T>* p, int colour, T w, int zero_in, int x0,
                     int y0, int z0, int tid) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int qx = tid % (TX / 2), jr = (tid / (TX / 2)) % TY, kr = tid / ((TX / 2) * TY);
  const int j = y0 + jr, k = z0 + kr;
  if (j >= ny || k >= nz) return;
  const int par = (colour + j + k) & 1;
  const int lx = 2 * qx + par, i = x0 + lx;
  if (zero_in) {
    const int io = x0 + 2 * qx + 1 - par;
    if (io < nx) p[((size_t)k * ny + j) * nx + io] = czero<T>();
  }
  if (i >= nx) return;
  const size_t N = (size_t)nx * ny * nz, q = ((size_t)k * ny + j) * nx + i;
  const int bx = lx + 2, by = jr + 1, bz = kr + 1;  // halo-box coordinates of cell q
  const int idx[3] = {i, j, k};
  const int nn[3] = {nx, ny, nz};
  const size_t stride[3] = {1, (size_t)nx, (size_t)nx * ny};
  const T ih = g.ih, ih2 = ih * ih;
  const T w00 = s3::wt(g.beta, 0, 0), w10 = s3::wt(g.beta, 1, 0), w11 = s3::wt(g.beta, 1, 1);
  auto U = [&](int c, int dx, int dy, int dz) { return s.u[c][slot(bx + dx, by + dy, bz + dz)]; };
  auto M = [&](int c, int dx, int dy, int dz) { return s.m[c][slot(bx + dx, by + dy, bz + dz)]; };
  auto MU = [&](int dx, int dy, int dz) { return s.mu[slot(bx + dx, by + dy, bz + dz)]; };
  auto PS = [&](int dx, int dy, int dz) { return s.p[slot(bx + dx, by + dy, bz + dz)]; };
  const cx<T> z = czero<T>();
  cx<T> r[7], a[3][4], d[7];
  bool ex[6];
  cx<T> Dcell[3];  // d_c^beta u_c at cell q (for the p row)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    int sc[3] = {0, 0, 0};
    sc[c] = 1;
    const int t1 = (c + 1) % 3, t2 = (c + 2) % 3;
    // beta-spread derivative of u_c along e between (o - s_e) and o, o = offset from q
    auto D = [&](int e, int ox, int oy, int oz) {
      const int p1 = (e + 1) % 3, p2 = (e + 2) % 3;
      cx<T> acc = z;
#pragma unroll
      for (int aa = -1; aa <= 1; ++aa)
#pragma unroll
        for (int bb = -1; bb <= 1; ++bb) {
          int o[3] = {ox, oy, oz};
          o[p1] += aa;
          o[p2] += bb;
          int om[3] = {o[0], o[1], o[2]};
          om[e] -= 1;
          const T wgt = (aa == 0 && bb == 0) ? w00 : ((aa == 0 || bb == 0) ? w10 : w11);
          acc = acc + wgt * (U(c, o[0], o[1], o[2]) - U(c, om[0], om[1], om[2]));
        }
      return ih * acc;
    };
    // mu at the derivative point between (o - s_e) and o: cell centre (e == c) or edge (e != c)
    auto MUE = [&](int e, int ox, int oy, int oz) -> T {
      if (e == c) return MU(ox - sc[0], oy - sc[1], oz - sc[2]);
      int se[3] = {0, 0, 0};
      se[e] = 1;
      return T(0.25) * (MU(ox, oy, oz) + MU(ox - sc[0], oy - sc[1], oz - sc[2]) + MU(ox - se[0], oy - se[1], oz - se[2]) +
                        MU(ox - sc[0] - se[0], oy - sc[1] - se[1], oz - sc[2] - se[2]));
    };
    // rows of the lo (f = q) and hi (f = q + s_c) faces
    cx<T> res[2];
    const cx<T> bq[2] = {c == 0 ? s.b0[(kr * TY + jr) * (TX + 1) + lx] : c == 1 ? s.b1[(kr * (TY + 1) + jr) * TX + lx]
                                                                       : s.b2[(kr * TY + jr) * TX + lx],
                         c == 0 ? s.b0[(kr * TY + jr) * (TX + 1) + lx + 1] : c == 1 ? s.b1[(kr * (TY + 1) + jr + 1) * TX + lx]
                                                                             : s.b2[((kr + 1) * TY + jr) * TX + lx]};
    T elo = T(0), ehi = T(0);
    const cx<T> Dc_mid = D(c, sc[0], sc[1], sc[2]);  // derivative at cell q
    Dcell[c] = Dc_mid;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int f[3] = {h * sc[0], h * sc[1], h * sc[2]};
      cx<T> lap = z;
      // e == c: points f and f + s_c
      {
        const cx<T> Da = h == 0 ? D(c, 0, 0, 0) : Dc_mid;
        const cx<T> Db = h == 0 ? Dc_mid : D(c, 2 * sc[0], 2 * sc[1], 2 * sc[2]);
        lap = lap + MUE(c, f[0], f[1], f[2]) * Da - MUE(c, f[0] + sc[0], f[1] + sc[1], f[2] + sc[2]) * Db;
      }
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        if (e == c) continue;
        int se[3] = {0, 0, 0};
        se[e] = 1;
        const T ma = MUE(e, f[0], f[1], f[2]), mb = MUE(e, f[0] + se[0], f[1] + se[1], f[2] + se[2]);
        if (h == 0) elo += ma + mb;
        else ehi += ma + mb;
        lap = lap + ma * D(e, f[0], f[1], f[2]) - mb * D(e, f[0] + se[0], f[1] + se[1], f[2] + se[2]);
      }
      lap = ih * lap;
      cx<T> nb = z;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        int sa[3] = {0, 0, 0};
        sa[ax] = 1;
        nb = nb + M(c, f[0] - sa[0], f[1] - sa[1], f[2] - sa[2]) * U(c, f[0] - sa[0], f[1] - sa[1], f[2] - sa[2]) +
             M(c, f[0] + sa[0], f[1] + sa[1], f[2] + sa[2]) * U(c, f[0] + sa[0], f[1] + sa[1], f[2] + sa[2]);
      }
      const cx<T> mass = g.beta * (M(c, f[0], f[1], f[2]) * U(c, f[0], f[1], f[2])) + g.sm * nb;
      const cx<T> grad = ih * (PS(f[0], f[1], f[2]) - PS(f[0] - sc[0], f[1] - sc[1], f[2] - sc[2]));
      res[h] = bq[h] - (lap - mass + grad);
    }
    ex[2 * c] = idx[c] == 0;
    ex[2 * c + 1] = idx[c] + 1 >= nn[c];
    r[2 * c] = ex[2 * c] ? z : (zero_in ? bq[0] : res[0]);
    r[2 * c + 1] = ex[2 * c + 1] ? z : (zero_in ? bq[1] : res[1]);
    // the 2x2 block of u_c (same entries as s3::block_u)
    const T mq = MU(0, 0, 0);
    const cx<T> mlo = M(c, 0, 0, 0), mhi = M(c, sc[0], sc[1], sc[2]);
    a[c][0] = mkc<T>(ih2 * w00 * (MU(-sc[0], -sc[1], -sc[2]) + mq + elo), T(0)) - g.beta * mlo;
    a[c][3] = mkc<T>(ih2 * w00 * (mq + MU(sc[0], sc[1], sc[2]) + ehi), T(0)) - g.beta * mhi;
    a[c][1] = mkc<T>(ih2 * (-w00 * mq + w10 * elo), T(0)) - g.sm * mhi;
    a[c][2] = mkc<T>(ih2 * (-w00 * mq + w10 * ehi), T(0)) - g.sm * mlo;
    if (g.economic) a[c][1] = a[c][2] = czero<T>();
    (void)t1;
    (void)t2;
  }
  const cx<T> pC = PS(0, 0, 0);
  const T cpq = ldg(g.cp + q);
  r[6] = zero_in ? s.bp[(kr * TY + jr) * TX + lx] : s.bp[(kr * TY + jr) * TX + lx] - (Dcell[0] + Dcell[1] + Dcell[2] + cpq * pC);
  k3::cell_solve(a, ex, ih, w00, cpq, r, d);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    int sc[3] = {0, 0, 0};
    sc[c] = 1;
    cx<T>* o = uout + c * N;
    o[q] = ex[2 * c] ? z : U(c, 0, 0, 0) + w * d[2 * c];
    if (!ex[2 * c + 1]) o[q + stride[c]] = U(c, sc[0], sc[1], sc[2]) + w * d[2 * c + 1];
    if (idx[c] == 1) o[q - stride[c]] = z;
  }
  p[q] = pC + w * d[6];
}

template <typename T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) vanka_tile(Grid<T> g, const cx<T>* __restrict__ b, const cx<T>* __restrict__ uin,
                                                   cx<T>* __restrict__ uout, cx<T>* p, int colour, T w, int zero_in) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tile<T>& s = *reinterpret_cast<Tile<T>*>(smem_raw);
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  tile_load(s, g, b, uin, p, zero_in, x0, y0, z0, threadIdx.x);
  __syncthreads();
  tile_compute(s, g, uout, p, colour, w, zero_in, x0, y0, z0, threadIdx.x);
}

}  // namespace k3t
