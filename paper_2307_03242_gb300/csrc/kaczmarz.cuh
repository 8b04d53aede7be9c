// Hybrid Kaczmarz-GMRES solve of the coarsest level (Sections 3.2 and 5.3) in one cooperative
// launch.
//
// The coarsest system H_s x = b is reduced to the displacements by the Schur complement that
// eliminates p through the diagonal p-p block C = diag(1/(lambda+mu)):
//   S u = f,  S = A_uu - A_up C^-1 A_pu,  f = b_u - A_up C^-1 b_p,  then p = C^-1 (b_p - A_pu u).
// S is solved by FGMRES(m) from zero (Arnoldi with modified Gram-Schmidt, complex Givens
// rotations, the true residual recomputed at every restart), preconditioned by a fixed number of
// parallel hybrid Kaczmarz steps from zero: the cells are divided into boxes (sub-regions); each
// box sweeps the Schur rows of its faces (component by component, x fastest) with damped row
// projections x += w (rhs_i - a_i x) / ||a_i||^2 conj(a_i) on a private copy of the unknowns it
// reaches, every box starting from the same iterate; each unknown then becomes the mean of the
// copies of the boxes whose reach holds it (component averaging). The reach of a box for
// component c2 is the box dilated by 1 cell below along x_c2, 2 cells below along the other
// axes and 1 cell above: the footprint of the Schur stencil.
//
// Rows of S are stored densely over their footprint (NE = 75 entries in 3D, 17 in 2D); they are
// formed at set-up by probing the level's own operator: for a component c2 and a residue class q
// of cells modulo 4 per axis, e = 1 on the active c2 faces of class q, and
// S e = (H_s e)_u - grad(C^-1 (H_s e)_p); a row's footprint holds at most one column of each class.
//
// GPU mapping: one block per SM, all blocks co-resident (cooperative launch), meeting at a
// grid-wide barrier whose waits are bounded (a timeout sets bit 1 of the status word and every
// block returns). A box is swept by one half-warp (two boxes per warp, in lock-step: a row that
// one half lacks is a zero row there): its 16 lanes take the row's entries, the row's dot product
// is a butterfly reduction (every lane ends with the same bits), the next rows' entries are
// loaded two rows ahead, and the private copy lives in shared memory. Dot products accumulate in FP64 and are summed over blocks in a fixed order, so
// the solve is deterministic; the Hessenberg matrix and rotations are FP64, computed identically
// by every block. The index helpers are __host__ __device__ so that the host can check them.
#pragma once
#include "emg_types.cuh"
#include "stencil2d.cuh"
#include "stencil3d.cuh"

namespace kz {

constexpr int NT = 512, NW = NT / 32, HW = 16;  // threads, warps per block; lanes per box
constexpr int MAXM = 8;          // largest restart length
constexpr int PER = 4;           // probe period per axis
constexpr long long WAIT_CYCLES = 4000000000LL;  // bound of one barrier wait (about 2 s)

template <int D>
struct Shape {
  static constexpr int NE = D == 3 ? 75 : 17;  // Schur row entries
  static constexpr int SL = (NE + HW - 1) / HW;  // entries per lane of a half-warp
};

// Footprint of a row of component c in component c2 along axis a: [foot_lo, 1].
HD int foot_lo(int c, int c2, int a) { return c2 == c ? -1 : (a == c ? -2 : (a == c2 ? 0 : -1)); }
// Reach of a box for component c2 below it along axis a (above it: 1 cell).
HD int reach_lo(int c2, int a) { return a == c2 ? 1 : 2; }

HD int pmod(int a, int m) {
  const int r = a % m;
  return r < 0 ? r + m : r;
}

// Entry s of a row of component c -> component c2 and offsets o (entries run over c2 = 0..D-1,
// each footprint box with x fastest). false: s >= NE.
template <int D>
HD bool slot_decode(int c, int s, int& c2, int o[3]) {
  o[0] = o[1] = o[2] = 0;
  for (int cc = 0; cc < D; ++cc) {
    int w[3] = {1, 1, 1}, cnt = 1;
    for (int a = 0; a < D; ++a) {
      w[a] = 2 - foot_lo(c, cc, a);
      cnt *= w[a];
    }
    if (s < cnt) {
      c2 = cc;
      for (int a = 0; a < D; ++a) {
        o[a] = foot_lo(c, cc, a) + s % w[a];
        s /= w[a];
      }
      return true;
    }
    s -= cnt;
  }
  return false;
}

template <int D>
HD int slot_of(int c, int c2, const int o[3]) {
  int base = 0;
  for (int cc = 0; cc < c2; ++cc) {
    int cnt = 1;
    for (int a = 0; a < D; ++a) cnt *= 2 - foot_lo(c, cc, a);
    base += cnt;
  }
  int s = 0, mul = 1;
  for (int a = 0; a < D; ++a) {
    s += (o[a] - foot_lo(c, c2, a)) * mul;
    mul *= 2 - foot_lo(c, c2, a);
  }
  return base + s;
}

// Box geometry: boxes of box[a] cells, nb[a] per axis; the reach region of a box holds, for
// each component c2, an rx[c2] x ry[c2] (x rz[c2]) block starting at rbase[c2].
struct Boxes {
  int dim, n[3], box[3], nb[3], nboxes;
  int rx[3], ry[3], rz[3], rbase[3], RS;
};

inline Boxes make_boxes(int dim, const int n[3], const int box[3]) {
  Boxes B{};
  B.dim = dim;
  B.nboxes = 1;
  for (int a = 0; a < 3; ++a) {
    B.n[a] = a < dim ? n[a] : 1;
    B.box[a] = a < dim ? box[a] : 1;
    B.nb[a] = (B.n[a] + B.box[a] - 1) / B.box[a];
    B.nboxes *= B.nb[a];
  }
  int base = 0;
  for (int c2 = 0; c2 < dim; ++c2) {
    B.rx[c2] = B.box[0] + reach_lo(c2, 0) + 1;
    B.ry[c2] = B.box[1] + reach_lo(c2, 1) + 1;
    B.rz[c2] = dim == 3 ? B.box[2] + reach_lo(c2, 2) + 1 : 1;
    B.rbase[c2] = base;
    base += B.rx[c2] * B.ry[c2] * B.rz[c2];
  }
  B.RS = base;
  return B;
}

// Lowest cell of box bx.
HD void box_lo(const Boxes& B, int bx, int lo[3]) {
  lo[0] = (bx % B.nb[0]) * B.box[0];
  lo[1] = ((bx / B.nb[0]) % B.nb[1]) * B.box[1];
  lo[2] = (bx / (B.nb[0] * B.nb[1])) * B.box[2];
}

// Region value t of the box with lowest cell lo -> component and cell (may lie outside).
HD int region_cell(const Boxes& B, int t, const int lo[3], int m[3]) {
  int c2 = 0;
  while (c2 + 1 < B.dim && t >= B.rbase[c2 + 1]) ++c2;
  int r = t - B.rbase[c2];
  m[0] = lo[0] - reach_lo(c2, 0) + r % B.rx[c2];
  r /= B.rx[c2];
  m[1] = lo[1] - reach_lo(c2, 1) + r % B.ry[c2];
  m[2] = B.dim == 3 ? lo[2] - reach_lo(c2, 2) + r / B.ry[c2] : 0;
  return c2;
}

// Position in a box's region of the entry (c2, o) of the row at local cell (lx, ly, lz).
HD int region_index(const Boxes& B, int c2, const int o[3], int lx, int ly, int lz) {
  const int z = B.dim == 3 ? lz + o[2] + reach_lo(c2, 2) : 0;
  return B.rbase[c2] + (z * B.ry[c2] + ly + o[1] + reach_lo(c2, 1)) * B.rx[c2] + lx + o[0] + reach_lo(c2, 0);
}

// Boxes whose reach holds the face of component c2 in cell m: [blo, bhi] per axis.
HD void reach_boxes(const Boxes& B, int c2, const int m[3], int blo[3], int bhi[3]) {
  for (int a = 0; a < 3; ++a) {
    if (a >= B.dim) {
      blo[a] = bhi[a] = 0;
      continue;
    }
    const int bb = B.box[a];
    const int lo = (m[a] + bb - 1) / bb - 1;
    const int hi = (m[a] + reach_lo(c2, a)) / bb;
    blo[a] = lo < 0 ? 0 : lo;
    bhi[a] = hi > B.nb[a] - 1 ? B.nb[a] - 1 : hi;
  }
}

// Position of that face in the region of box (bxx, by, bz).
HD int reach_local(const Boxes& B, int c2, const int m[3], int bxx, int by, int bz) {
  const int lz = B.dim == 3 ? m[2] - (bz * B.box[2] - reach_lo(c2, 2)) : 0;
  const int ly = m[1] - (by * B.box[1] - reach_lo(c2, 1));
  const int lx = m[0] - (bxx * B.box[0] - reach_lo(c2, 0));
  return B.rbase[c2] + (lz * B.ry[c2] + ly) * B.rx[c2] + lx;
}

HD size_t cell_of(const int n[3], int dim, int i, int j, int k) {
  return dim == 3 ? ((size_t)k * n[1] + j) * n[0] + i : (size_t)j * n[0] + i;
}

// ---------------------------------------------------------------- set-up: probing
// Probe value at position t of a (D+1) N vector: 1 on the active c2 faces of class q.
template <typename T, int D>
HD cx<T> probe_value(int c2, const int q[3], const int n[3], size_t t) {
  const size_t N = (size_t)n[0] * n[1] * (D == 3 ? n[2] : 1);
  const int c = (int)(t / N);
  const size_t cell = t % N;
  const int idx[3] = {(int)(cell % n[0]), (int)((cell / n[0]) % n[1]), D == 3 ? (int)(cell / ((size_t)n[0] * n[1])) : 0};
  bool on = c == c2 && idx[c2] >= 1;
  for (int a = 0; a < D; ++a) on = on && pmod(idx[a] - q[a], PER) == 0;
  return mkc<T>(on ? T(1) : T(0), T(0));
}

// y = H_s e of a probe: the entry of row r (component c, cell k) of S for its class-q column of
// component c2, stored at coef[r NE + slot] (rows without such a column: nothing written).
template <typename T, int D>
HD void probe_take_row(const Grid<T>& g, const cx<T>* y, int c2, const int q[3], size_t r, cx<T>* coef) {
  constexpr int NE = Shape<D>::NE;
  const int n[3] = {g.nx, g.ny, D == 3 ? g.nz : 1};
  const size_t N = (size_t)n[0] * n[1] * n[2];
  const int c = (int)(r / N);
  const size_t cell = r % N;
  const int kk[3] = {(int)(cell % n[0]), (int)((cell / n[0]) % n[1]), D == 3 ? (int)(cell / ((size_t)n[0] * n[1])) : 0};
  if (kk[c] < 1) return;  // boundary face: not an unknown
  int o[3] = {0, 0, 0}, m[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) {
    const int lo = foot_lo(c, c2, a);
    o[a] = lo + pmod(q[a] - kk[a] - lo, PER);
    if (o[a] > 1) return;  // no column of this class in the footprint
    m[a] = kk[a] + o[a];
    if (m[a] < 0 || m[a] >= n[a]) return;
  }
  if (m[c2] < 1) return;  // the column is a boundary face
  int pm[3] = {kk[0], kk[1], kk[2]};
  pm[c] -= 1;
  const size_t km = cell_of(n, D, pm[0], pm[1], pm[2]);
  const cx<T>* yp = y + (size_t)D * N;
  const cx<T> gp = (T(1) / g.cp[cell]) * yp[cell] - (T(1) / g.cp[km]) * yp[km];
  coef[r * NE + slot_of<D>(c, c2, o)] = y[r] - g.ih * gp;
}

template <typename T, int D>
HD T inv_row_norm(const cx<T>* coef, size_t r) {
  constexpr int NE = Shape<D>::NE;
  T s = T(0);
  for (int e = 0; e < NE; ++e) {
    const cx<T> v = coef[r * NE + e];
    s += v.re * v.re + v.im * v.im;
  }
  return s > T(0) ? T(1) / s : T(0);
}

// f = b_u - A_up C^-1 b_p at Schur row q (0 on boundary faces).
template <typename T, int D>
HD cx<T> schur_rhs(const Grid<T>& g, const cx<T>* b, size_t q) {
  const int n[3] = {g.nx, g.ny, D == 3 ? g.nz : 1};
  const size_t N = (size_t)n[0] * n[1] * n[2];
  const int c = (int)(q / N);
  const size_t cell = q % N;
  const int k[3] = {(int)(cell % n[0]), (int)((cell / n[0]) % n[1]), D == 3 ? (int)(cell / ((size_t)n[0] * n[1])) : 0};
  if ((c == 0 ? k[0] : (c == 1 ? k[1] : k[2])) < 1) return czero<T>();
  const cx<T>* bp = b + (size_t)D * N;
  const size_t km = cell_of(n, D, k[0] - (c == 0), k[1] - (c == 1), k[2] - (c == 2));
  const cx<T> gq = (T(1) / g.cp[cell]) * bp[cell] - (T(1) / g.cp[km]) * bp[km];
  return b[q] - g.ih * gq;
}

template <typename T>
struct Args {
  Grid<T> g;                 // the coarsest level's operator H_s
  Boxes B;                   // sub-region boxes
  size_t N;                  // cells
  int warps_a;               // half-warps per block that own a region in shared memory (even)
  const cx<T>* coef;         // D N rows x NE entries
  const T* inv_n2;           // 1 / ||row||^2 (0: no row)
  const cx<T>* b;            // (D+1) N right-hand side
  cx<T>* x;                  // (D+1) N solution
  cx<T>* f;                  // D N: Schur right-hand side
  cx<T>* u;                  // D N: Schur iterate
  cx<T>* w;                  // D N: Arnoldi / residual work vector
  cx<T>* V;                  // (m+1) D N
  cx<T>* Z;                  // m D N
  cx<T>* copies;             // nboxes RS
  double* part;              // 2 x gridDim x 2 partial sums
  unsigned* bar;             // barrier count, generation
  int* err;                  // status word (bit 1: a barrier wait timed out)
  double* stats;             // FGMRES iterations, relative Schur residual, Kaczmarz steps
  T damping;
  int steps, restart, max_its;
  double tol;
};

#ifdef __CUDACC__
template <typename T, int D>
__global__ void probe_set(cx<T>* __restrict__ e, int c2, int q0, int q1, int q2, int nx, int ny, int nz) {
  const int n[3] = {nx, ny, nz}, q[3] = {q0, q1, q2};
  const size_t N = (size_t)nx * ny * nz;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (size_t)(D + 1) * N) e[t] = probe_value<T, D>(c2, q, n, t);
}

template <typename T, int D>
__global__ void probe_take(Grid<T> g, const cx<T>* __restrict__ y, int c2, int q0, int q1, int q2,
                           cx<T>* __restrict__ coef) {
  const int q[3] = {q0, q1, q2};
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < (size_t)D * N) probe_take_row<T, D>(g, y, c2, q, r, coef);
}

template <typename T, int D>
__global__ void row_norms(const cx<T>* __restrict__ coef, T* __restrict__ inv_n2, size_t rows) {
  const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows) inv_n2[r] = inv_row_norm<T, D>(coef, r);
}

// ---------------------------------------------------------------- the solve
__device__ __forceinline__ void st_cg(cx<float>* p, cx<float> v) { __stcg(reinterpret_cast<float2*>(p), make_float2(v.re, v.im)); }
__device__ __forceinline__ void st_cg(cx<double>* p, cx<double> v) {
  __stcg(reinterpret_cast<double2*>(p), make_double2(v.re, v.im));
}

// Grid-wide barrier with bounded waits. Returns false (on every thread of the block) once any
// block has recorded a timeout; the caller then returns.
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err, int* sh_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile int* verr = err;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned prev = atomicAdd(bar, 1u);
    if (prev == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (*verr & 2) break;
        if (clock64() - t0 > WAIT_CYCLES) {
          atomicOr(err, 2);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    *sh_ok = (*verr & 2) ? 0 : 1;
  }
  __syncthreads();
  return *(volatile int*)sh_ok != 0;
}

struct Shared {
  double red[2 * NW + 4];
  cx<double> H[(MAXM + 1) * MAXM];
  cx<double> cs[MAXM], sn[MAXM], gv[MAXM + 1], y[MAXM];
  double scal[4];
  int ok;
};

__device__ __forceinline__ cx<double> cdd(double r, double i) { return mkc<double>(r, i); }
__device__ __forceinline__ double cabs2(cx<double> a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ cx<double> cdiv_real(cx<double> a, double s) { return mkc<double>(a.re / s, a.im / s); }

// Sum over the grid of the per-thread (re, im); the same bits on every thread of every block.
// One barrier. parity alternates the partial-sum buffer between consecutive reductions.
__device__ __forceinline__ bool grid_sum(double re, double im, double* part, unsigned* bar, int* err, Shared& sh,
                                         int& parity, cx<double>& out) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, m);
    im += __shfl_xor_sync(0xffffffffu, im, m);
  }
  if (lane == 0) {
    sh.red[2 * wib] = re;
    sh.red[2 * wib + 1] = im;
  }
  __syncthreads();
  double* P = part + (size_t)parity * 2 * gridDim.x;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < NW; ++k) {
      a += sh.red[2 * k];
      b += sh.red[2 * k + 1];
    }
    __stcg(P + 2 * blockIdx.x, a);
    __stcg(P + 2 * blockIdx.x + 1, b);
  }
  parity ^= 1;
  if (!grid_sync(bar, err, &sh.ok)) return false;
  if (wib == 0) {
    double a = 0.0, b = 0.0;
    for (int k = lane; k < (int)gridDim.x; k += 32) {
      a += __ldcg(P + 2 * k);
      b += __ldcg(P + 2 * k + 1);
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, m);
      b += __shfl_xor_sync(0xffffffffu, b, m);
    }
    if (lane == 0) {
      sh.scal[0] = a;
      sh.scal[1] = b;
    }
  }
  __syncthreads();
  out = cdd(sh.scal[0], sh.scal[1]);
  __syncthreads();
  return true;
}

// Per-lane table of a row's entries: for component c and slot t of half-warp lane l (entry
// l + 16 t), -1 (no entry) or the packed entry: component c2 (bits 0-1), offsets + 2 (3 bits each
// from bit 2) and the region position for the row cell at local (0, 0, 0) (from bit 11).
template <int D>
struct LaneTab {
  int pk[D][Shape<D>::SL];
  HD void init(const Boxes& B, int hl) {
    for (int c = 0; c < D; ++c)
      for (int t = 0; t < Shape<D>::SL; ++t) {
        int cc = -1, oo[3];
        if (slot_decode<D>(c, hl + HW * t, cc, oo))
          pk[c][t] = cc | (oo[0] + 2) << 2 | (oo[1] + 2) << 5 | (oo[2] + 2) << 8 | region_index(B, cc, oo, 0, 0, 0) << 11;
        else
          pk[c][t] = -1;
      }
  }
  // (selects instead of an indexed load keep the table in registers)
  HD int get(int c, int t) const {
    int v = pk[0][t];
    if (D > 1 && c == 1) v = pk[1][t];
    if (D > 2 && c == 2) v = pk[D - 1][t];
    return v;
  }
};
// The lane tables of a block in shared memory: entry (c, t) of lane l at [(c SL + t) HW + l];
// after them, at the same index + D SL HW, the entry's region strides rx | (rx ry) << 16, so that
// the sweep finds an entry's position without reading the box geometry at a lane-dependent index.
template <int D>
struct LaneTabSm {
  const int* v;
  __device__ __forceinline__ int get(int c, int t) const {
    return v[(c * Shape<D>::SL + t) * HW + (threadIdx.x & (HW - 1))];
  }
  __device__ __forceinline__ int strides(int c, int t) const {
    return v[(D * Shape<D>::SL + c * Shape<D>::SL + t) * HW + (threadIdx.x & (HW - 1))];
  }
};
HD int pk_c2(int v) { return v & 3; }
HD int pk_o(int v, int a) { return ((v >> (2 + 3 * a)) & 7) - 2; }
HD int pk_off(int v) { return v >> 11; }

// Row q of a box in sweep order (component, then cells with x fastest) -> component and local cell.
HD int box_row(const Boxes& B, int q, int l[3]) {
  const int per = B.box[0] * B.box[1] * B.box[2];
  const int c = q / per;
  int r = q - c * per;
  l[0] = r % B.box[0];
  r /= B.box[0];
  l[1] = r % B.box[1];
  l[2] = r / B.box[1];
  return c;
}

// Global row of box row q (lowest box cell lo), or -1 if the row is outside the grid or a
// boundary face.
HD long long box_row_global(const Boxes& B, int q, const int lo[3], int& c, int l[3]) {
  c = box_row(B, q, l);
  const int k[3] = {lo[0] + l[0], lo[1] + l[1], lo[2] + l[2]};
  if (k[0] >= B.n[0] || k[1] >= B.n[1] || k[2] >= B.n[2] || k[c] < 1) return -1;
  const size_t N = (size_t)B.n[0] * B.n[1] * B.n[2];
  return (long long)((size_t)c * N + cell_of(B.n, B.dim, k[0], k[1], k[2]));
}

// Asynchronous global -> shared copies (cp.async; each thread's copies form groups that it
// commits and waits for).
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Rows in flight per half-warp (the ring of row slots in shared memory after its region). A slot
// holds the row's NE entries, its right-hand side and 1 / ||row||^2 (in the real part of one more
// complex value).
constexpr int PD = 4;
template <int D>
struct Ring {
  static constexpr int SLOT = Shape<D>::NE + 2;  // complex values per slot
};
// Complex values of shared memory a half-warp uses: its region and its ring.
HD int half_warp_smem(const Boxes& B, int D) { return B.RS + PD * ((D == 3 ? Shape<3>::NE : Shape<2>::NE) + 2); }

// Per-component region extents in registers, for the component average, which indexes them by a
// component known only at run time (indexing the kernel-parameter copy that way puts it in
// local memory).
struct RegGeo {
  int rx0, rx1, rx2, ry0, ry1, ry2, rb0, rb1, rb2;
  __device__ __forceinline__ explicit RegGeo(const Boxes& B)
      : rx0(B.rx[0]), rx1(B.rx[1]), rx2(B.rx[2]), ry0(B.ry[0]), ry1(B.ry[1]), ry2(B.ry[2]), rb0(B.rbase[0]),
        rb1(B.rbase[1]), rb2(B.rbase[2]) {}
  __device__ __forceinline__ int rx(int c) const { return c == 0 ? rx0 : (c == 1 ? rx1 : rx2); }
  __device__ __forceinline__ int ry(int c) const { return c == 0 ? ry0 : (c == 1 ? ry1 : ry2); }
  __device__ __forceinline__ int rbase(int c) const { return c == 0 ? rb0 : (c == 1 ? rb1 : rb2); }
};

// Box extent along axis a: FIXB cells on every axis of the grid when FIXB > 0 (boxes of 1 or 2
// cells; the compiler then turns the index arithmetic's divisions into shifts), else the run-time
// boxes (at least 2 cells per axis).
template <int D, int FIXB>
HD int bsz(const Boxes& B, int a) {
  return FIXB ? (a < D ? FIXB : 1) : B.box[a];
}

// A box row in sweep order (component, then cells with x fastest), advanced like an odometer.
struct Cursor {
  int c = 0, l[3] = {0, 0, 0};
  template <int D, int FIXB>
  HD void advance(const Boxes& B) {
    if (++l[0] == bsz<D, FIXB>(B, 0)) {
      l[0] = 0;
      if (++l[1] == bsz<D, FIXB>(B, 1)) {
        l[1] = 0;
        if (++l[2] == bsz<D, FIXB>(B, 2)) {
          l[2] = 0;
          ++c;
        }
      }
    }
  }
};

// Global row of the cursor's row in the box with lowest cell lo, or -1 (outside the grid or a
// boundary face).
template <int D>
HD long long cursor_row(const Boxes& B, const Cursor& u, const int lo[3], unsigned N) {
  const int k0 = lo[0] + u.l[0], k1 = lo[1] + u.l[1], k2 = lo[2] + u.l[2];
  const int kc = u.c == 0 ? k0 : (u.c == 1 ? k1 : k2);
  if (k0 >= B.n[0] || k1 >= B.n[1] || (D == 3 && k2 >= B.n[2]) || kc < 1) return -1;
  const unsigned cell = D == 3 ? ((unsigned)k2 * B.n[1] + k1) * B.n[0] + k0 : (unsigned)k1 * B.n[0] + k0;
  return (long long)u.c * N + cell;
}

// Starts the copy of row r into ring slot `slot` (this lane's entries; lane 0 also the right-hand
// side and the norm), or zero-fills the slot for a missing row (r < 0); commits one group.
template <typename T, int D>
__device__ __forceinline__ void stage_row(const Args<T>& a, const LaneTabSm<D>& tab, const cx<T>* rhs, long long r,
                                          int c, int hl, cx<T>* slot) {
  constexpr int NE = Shape<D>::NE, SL = Shape<D>::SL;
  if (r >= 0) {
#pragma unroll
    for (int t = 0; t < SL; ++t)
      if (hl + HW * t < NE) cp_async(slot + hl + HW * t, a.coef + (size_t)r * NE + hl + HW * t, (int)sizeof(cx<T>));
    if (hl == 0) {
      cp_async(slot + NE, rhs + r, (int)sizeof(cx<T>));
      cp_async(&slot[NE + 1].re, a.inv_n2 + r, (int)sizeof(T));
    }
  } else {
#pragma unroll
    for (int t = 0; t < SL; ++t)
      if (hl + HW * t < NE) slot[hl + HW * t] = czero<T>();
    if (hl == 0) {
      slot[NE] = czero<T>();
      slot[NE + 1] = czero<T>();
    }
  }
  (void)c;
  (void)tab;
  cp_commit();
}

// Region layout of a box (the same for every box, relative to its lowest cell): entry t is
// component c2 (bits 0-1) at offsets (bits 2-9, 10-17, 18-25) from the region's lowest cell.
HD int region_code(const Boxes& B, int t) {
  const int lo[3] = {0, 0, 0};
  int m[3];
  const int c2 = region_cell(B, t, lo, m);
  return c2 | (m[0] + reach_lo(c2, 0)) << 2 | (m[1] + reach_lo(c2, 1)) << 10 |
         (B.dim == 3 ? m[2] + reach_lo(c2, 2) : 0) << 18;
}

// One sweep of every box: rhs -> copies, starting from xin (nullptr: zero). Half-warp h of the
// grid takes boxes h, h + nhw, ...; both halves of a warp run the same number of box rounds.
// reg: the half-warp's region, followed by its ring of PD row slots; rtab: region_code of every
// region entry (shared by the block).
template <typename T, int D, int FIXB>
__device__ void sweep_boxes(const Args<T>& a, const LaneTabSm<D>& tab, const cx<T>* rhs, const cx<T>* xin, cx<T>* reg,
                            const int* rtab, int ghw, int nhw) {
  constexpr int NE = Shape<D>::NE, SL = Shape<D>::SL, SLOT = Ring<D>::SLOT;
  constexpr int RB = D == 3 ? 4 : 8;  // region loads in flight per lane (fewer in 3D: registers)
  const int hl = threadIdx.x & (HW - 1);
  const Boxes& B = a.B;
  const unsigned N = (unsigned)a.N;
  cx<T>* ring = reg + B.RS;
  const int Q = D * bsz<D, FIXB>(B, 0) * bsz<D, FIXB>(B, 1) * bsz<D, FIXB>(B, 2);
  const int ghw0 = ghw & ~1;  // the warp's first half-warp: both halves run the same rounds
  for (int rd_i = 0; ghw0 + rd_i * nhw < B.nboxes; ++rd_i) {
    const int bx = ghw + rd_i * nhw;
    const bool live = bx < B.nboxes;
    int lo[3] = {0, 0, 0};
    if (live) {
      lo[0] = (bx % B.nb[0]) * bsz<D, FIXB>(B, 0);
      lo[1] = ((bx / B.nb[0]) % B.nb[1]) * bsz<D, FIXB>(B, 1);
      lo[2] = (bx / (B.nb[0] * B.nb[1])) * bsz<D, FIXB>(B, 2);
    }
    // the first PD - 1 rows start copying while the region loads
    Cursor st;
    int staged = 0;
    auto stage_next = [&](cx<T>* slot) {
      long long r = -1;
      if (staged < Q) {
        if (live) r = cursor_row<D>(B, st, lo, N);
        st.advance<D, FIXB>(B);
      }
      ++staged;
      stage_row<T, D>(a, tab, rhs, r, 0, hl, slot);
    };
    for (int q = 0; q < PD - 1; ++q) stage_next(ring + q * SLOT);
    // the region from xin, RB independent loads in flight per lane
    for (int t0 = hl; t0 < B.RS; t0 += RB * HW) {
      cx<T> v[RB];
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        const int t = t0 + u * HW;
        v[u] = czero<T>();
        if (live && xin && t < B.RS) {
          const int code = rtab[t];
          const int c2 = code & 3;
          const int m0 = lo[0] - reach_lo(c2, 0) + ((code >> 2) & 255);
          const int m1 = lo[1] - reach_lo(c2, 1) + ((code >> 10) & 255);
          const int m2 = D == 3 ? lo[2] - reach_lo(c2, 2) + ((code >> 18) & 255) : 0;
          const int mc = c2 == 0 ? m0 : (c2 == 1 ? m1 : m2);
          const bool in = m0 >= 0 && m0 < B.n[0] && m1 >= 0 && m1 < B.n[1] && (D == 2 || (m2 >= 0 && m2 < B.n[2]));
          if (in && mc >= 1) {
            const unsigned cell = D == 3 ? ((unsigned)m2 * B.n[1] + m1) * B.n[0] + m0 : (unsigned)m1 * B.n[0] + m0;
            v[u] = ldcg(xin + (size_t)c2 * N + cell);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < RB; ++u)
        if (t0 + u * HW < B.RS) reg[t0 + u * HW] = v[u];
    }
    Cursor cu;
    for (int q = 0; q < Q; ++q) {
      stage_next(ring + ((q + PD - 1) % PD) * SLOT);
      cp_wait<PD - 1>();  // this lane's copies of row q have landed
      __syncwarp();       // ... and every lane's (the right-hand side and norm come from lane 0)
      const cx<T>* sl = ring + (q % PD) * SLOT;
      const int c = cu.c;
      int idx[SL];
      cx<T> co[SL];
      T sr = T(0), si = T(0);
#pragma unroll
      for (int t = 0; t < SL; ++t) {
        const int pk = tab.get(c, t);
        idx[t] = -1;
        co[t] = czero<T>();
        if (pk >= 0) {
          const int cc = pk_c2(pk);
          const int st2 = tab.strides(c, t);
          idx[t] = pk_off(pk) + cu.l[2] * (st2 >> 16) + cu.l[1] * (st2 & 0xffff) + cu.l[0];
          (void)cc;
          co[t] = sl[hl + HW * t];
          const cx<T> xv = reg[idx[t]];
          sr += co[t].re * xv.re - co[t].im * xv.im;
          si += co[t].re * xv.im + co[t].im * xv.re;
        }
      }
#pragma unroll
      for (int m = HW / 2; m >= 1; m >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, m);
        si += __shfl_xor_sync(0xffffffffu, si, m);
      }
      const cx<T> bv = sl[NE];
      const T in2 = sl[NE + 1].re;
      const T s_re = a.damping * in2 * (bv.re - sr), s_im = a.damping * in2 * (bv.im - si);
#pragma unroll
      for (int t = 0; t < SL; ++t) {
        if (idx[t] >= 0) {  // += s conj(a)
          cx<T> v = reg[idx[t]];
          v.re += s_re * co[t].re + s_im * co[t].im;
          v.im += s_im * co[t].re - s_re * co[t].im;
          reg[idx[t]] = v;
        }
      }
      cu.advance<D, FIXB>(B);
      __syncwarp();  // the region's updates and the slot's reads are done before the slot refills
    }
    cp_wait<0>();
    if (live) {
      cx<T>* out = a.copies + (size_t)bx * B.RS;
      for (int t = hl; t < B.RS; t += HW) st_cg(out + t, reg[t]);
    }
    __syncwarp();
  }
}

// Component average of the copies -> out (D N; boundary faces 0). At most 3 boxes per axis hold
// an unknown when boxes have at least 2 cells per axis, at most 4 for boxes of one cell.
template <typename T, int D, int FIXB>
__device__ void average(const Args<T>& a, cx<T>* out, size_t tid, size_t nthr) {
  const Boxes& B = a.B;
  const RegGeo rg(B);
  const unsigned N = (unsigned)a.N, n0 = (unsigned)B.n[0], n1 = (unsigned)B.n[1];
  const unsigned DN = (unsigned)D * N;
  for (unsigned q = (unsigned)tid; q < DN; q += (unsigned)nthr) {
    const int c2 = (int)(q / N);
    const unsigned cell = q - (unsigned)c2 * N;
    const unsigned t = cell / n0;
    const int m[3] = {(int)(cell - t * n0), (int)(D == 3 ? t % n1 : t), D == 3 ? (int)(t / n1) : 0};
    if ((c2 == 0 ? m[0] : (c2 == 1 ? m[1] : m[2])) < 1) {  // (selects: no run-time-indexed array)
      out[q] = czero<T>();
      continue;
    }
    int blo[3], bhi[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if (ax >= D) {
        blo[ax] = bhi[ax] = 0;
        continue;
      }
      const int bb = bsz<D, FIXB>(B, ax);
      const int lo = (m[ax] + bb - 1) / bb - 1;
      const int hi = (m[ax] + reach_lo(c2, ax)) / bb;
      blo[ax] = lo < 0 ? 0 : lo;
      bhi[ax] = hi > B.nb[ax] - 1 ? B.nb[ax] - 1 : hi;
    }
    const int rx = rg.rx(c2), ry = rg.ry(c2), rb = rg.rbase(c2);
    // the candidate boxes in box order, CA per axis (4 for boxes of one cell, else 3); the loop is
    // unrolled, so the loads are independent and the compiler issues them ahead of the sums
    constexpr int CA = FIXB == 1 ? 4 : 3;
    constexpr int NZ = D == 3 ? CA : 1;
    T sr = T(0), si = T(0);
    int cnt = 0;
#pragma unroll
    for (int dz = 0; dz < NZ; ++dz)
#pragma unroll
      for (int dy = 0; dy < CA; ++dy)
#pragma unroll
        for (int dx = 0; dx < CA; ++dx) {
          const int bz = blo[2] + dz, by = blo[1] + dy, bxx = blo[0] + dx;
          if (bz <= bhi[2] && by <= bhi[1] && bxx <= bhi[0]) {
            const int box = (bz * B.nb[1] + by) * B.nb[0] + bxx;
            const int lz = D == 3 ? m[2] - (bz * bsz<D, FIXB>(B, 2) - reach_lo(c2, 2)) : 0;
            const int ly = m[1] - (by * bsz<D, FIXB>(B, 1) - reach_lo(c2, 1));
            const int lx = m[0] - (bxx * bsz<D, FIXB>(B, 0) - reach_lo(c2, 0));
            const cx<T> w = ldcg(a.copies + (size_t)box * B.RS + rb + (lz * ry + ly) * rx + lx);
            sr += w.re;
            si += w.im;
            ++cnt;
          }
        }
    out[q] = mkc<T>(sr / T(cnt), si / T(cnt));
  }
}

// S z at row r (or 0 for r < 0) as this half-warp's lanes' shares summed over the half-warp.
template <typename T, int D>
__device__ __forceinline__ cx<T> row_dot(const Args<T>& a, const LaneTabSm<D>& tab, const cx<T>* z, long long r, int hl) {
  constexpr int NE = Shape<D>::NE, SL = Shape<D>::SL;
  const Boxes& B = a.B;
  const size_t N = a.N;
  T sr = T(0), si = T(0);
  if (r >= 0) {
    const int c = (int)(r / N);
    const size_t cell = r % N;
    const int k[3] = {(int)(cell % B.n[0]), (int)((cell / B.n[0]) % B.n[1]), D == 3 ? (int)(cell / ((size_t)B.n[0] * B.n[1])) : 0};
    if ((c == 0 ? k[0] : (c == 1 ? k[1] : k[2])) >= 1) {
#pragma unroll
      for (int t = 0; t < SL; ++t) {
        const int pk = tab.get(c, t);
        if (pk < 0) continue;
        const int cc = pk_c2(pk);
        const int m[3] = {k[0] + pk_o(pk, 0), k[1] + pk_o(pk, 1), k[2] + pk_o(pk, 2)};
        bool in = true;
        for (int q = 0; q < D; ++q) in = in && m[q] >= 0 && m[q] < B.n[q];
        if (!in) continue;
        const cx<T> co = ldg(a.coef + (size_t)r * NE + hl + HW * t);
        const cx<T> zv = ldcg(z + (size_t)cc * N + cell_of(B.n, D, m[0], m[1], m[2]));
        sr += co.re * zv.re - co.im * zv.im;
        si += co.re * zv.im + co.im * zv.re;
      }
    }
  }
#pragma unroll
  for (int m = HW / 2; m >= 1; m >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, m);
    si += __shfl_xor_sync(0xffffffffu, si, m);
  }
  return mkc<T>(sr, si);
}

// w = S z (or rhs - S z), one row per half-warp and two rows in flight; adds this thread's share
// of sum conj(v) w (v given) or of |w|^2 (v == nullptr) to (dre, dim_).
template <typename T, int D>
__device__ void matvec(const Args<T>& a, const LaneTabSm<D>& tab, const cx<T>* z, const cx<T>* rhs, cx<T>* w,
                       const cx<T>* v, double& dre, double& dim_, int ghw, int nhw) {
  const int hl = threadIdx.x & (HW - 1);
  const long long rows = (long long)D * a.N;
  const long long per = 2LL * nhw;
  const long long ghw0 = ghw & ~1;
  for (long long base = 0; base + ghw0 < rows; base += per) {
    const long long r0 = base + ghw, r1 = base + nhw + ghw;
    const long long q0 = r0 < rows ? r0 : -1, q1 = r1 < rows ? r1 : -1;
    const cx<T> s0 = row_dot<T, D>(a, tab, z, q0, hl);
    const cx<T> s1 = row_dot<T, D>(a, tab, z, q1, hl);
    if (hl == 0) {
      const long long qq[2] = {q0, q1};
      const cx<T> ss[2] = {s0, s1};
      for (int u = 0; u < 2; ++u) {
        if (qq[u] < 0) continue;
        cx<T> wv = ss[u];
        if (rhs) {
          const cx<T> bv = ldcg(rhs + qq[u]);
          wv = mkc<T>(bv.re - wv.re, bv.im - wv.im);
        }
        st_cg(w + qq[u], wv);
        if (v) {
          const cx<T> vv = ldcg(v + qq[u]);
          dre += (double)vv.re * wv.re + (double)vv.im * wv.im;
          dim_ += (double)vv.re * wv.im - (double)vv.im * wv.re;
        } else {
          dre += (double)wv.re * wv.re + (double)wv.im * wv.im;
        }
      }
    }
  }
}

// The parameter block is __grid_constant__: the kernels index its box geometry by components known
// only at run time, which on an ordinary parameter makes the compiler copy it to local memory.
template <typename T, int D, int FIXB>
__global__ void __launch_bounds__(NT, 1) solve(const __grid_constant__ Args<T> a) {
  extern __shared__ __align__(16) unsigned char kz_smem[];
  __shared__ Shared sh;
  const int hwb = threadIdx.x / HW;  // half-warp in the block
  // a.warps_a counts half-warps that own a private region (an even number)
  cx<T>* reg = reinterpret_cast<cx<T>*>(kz_smem) + (size_t)(hwb < a.warps_a ? hwb : 0) * half_warp_smem(a.B, D);
  const size_t tid = (size_t)blockIdx.x * NT + threadIdx.x, nthr = (size_t)gridDim.x * NT;
  const int ghw_all = blockIdx.x * (NT / HW) + hwb, nhw_all = gridDim.x * (NT / HW);
  // box-sweeping half-warps numbered block-fastest, so that a grid with few boxes still spreads
  // them over every SM; the two halves of a warp stay consecutive (they run in lock-step)
  const int ghw_a = ((hwb >> 1) * gridDim.x + blockIdx.x) * 2 + (hwb & 1), nhw_a = gridDim.x * a.warps_a;
  const size_t N = a.N, DN = (size_t)D * N;
  const Grid<T>& g = a.g;
  // the region layout and the lane tables, after the half-warps' regions and rings (read after
  // the first barrier)
  int* rtab = reinterpret_cast<int*>(reinterpret_cast<cx<T>*>(kz_smem) + (size_t)a.warps_a * half_warp_smem(a.B, D));
  for (int t = threadIdx.x; t < a.B.RS; t += NT) rtab[t] = region_code(a.B, t);
  int* ltab = rtab + a.B.RS;
  if (threadIdx.x < HW) {
    LaneTab<D> lt;
    lt.init(a.B, threadIdx.x);
    for (int c = 0; c < D; ++c)
      for (int t = 0; t < Shape<D>::SL; ++t) {
        const int pk = lt.pk[c][t];
        ltab[(c * Shape<D>::SL + t) * HW + threadIdx.x] = pk;
        const int cc = pk >= 0 ? pk_c2(pk) : 0;
        ltab[(D * Shape<D>::SL + c * Shape<D>::SL + t) * HW + threadIdx.x] = a.B.rx[cc] | (a.B.rx[cc] * a.B.ry[cc]) << 16;
      }
  }
  const LaneTabSm<D> tab{ltab};
  int parity = 0;
  cx<double> red;

  // f = b_u - A_up C^-1 b_p, u = 0, ||f||^2
  double acc = 0.0;
  for (size_t q = tid; q < DN; q += nthr) {
    const cx<T> fv = schur_rhs<T, D>(g, a.b, q);
    st_cg(a.f + q, fv);
    st_cg(a.u + q, czero<T>());
    acc += (double)fv.re * fv.re + (double)fv.im * fv.im;
  }
  if (!grid_sum(acc, 0.0, a.part, a.bar, a.err, sh, parity, red)) return;
  const double bnorm = sqrt(red.re);
  double beta = bnorm;
  int its = 0;
  const int m = a.restart;
  if (bnorm > 0.0) {
    for (size_t q = tid; q < DN; q += nthr) {  // V_0 = f / beta
      const cx<T> fv = ldcg(a.f + q);
      st_cg(a.V + q, mkc<T>((T)(fv.re / beta), (T)(fv.im / beta)));
    }
    while (beta / bnorm > a.tol && its < a.max_its) {
      if (threadIdx.x == 0) {
        for (int i = 0; i <= MAXM; ++i) sh.gv[i] = cdd(0.0, 0.0);
        sh.gv[0] = cdd(beta, 0.0);
      }
      int kdone = 0;
      for (int j = 0; j < m; ++j) {
        const cx<T>* Vj = a.V + (size_t)j * DN;
        cx<T>* Zj = a.Z + (size_t)j * DN;
        if (!grid_sync(a.bar, a.err, &sh.ok)) return;
        // Z_j = K(V_j): Kaczmarz steps from zero
        for (int s = 0; s < a.steps; ++s) {
          if (hwb < a.warps_a) sweep_boxes<T, D, FIXB>(a, tab, Vj, s == 0 ? nullptr : Zj, reg, rtab, ghw_a, nhw_a);
          if (!grid_sync(a.bar, a.err, &sh.ok)) return;
          average<T, D, FIXB>(a, Zj, tid, nthr);
          if (!grid_sync(a.bar, a.err, &sh.ok)) return;
        }
        // w = S Z_j, h_0j = <V_0, w>
        double dre = 0.0, dim_ = 0.0;
        matvec<T, D>(a, tab, Zj, nullptr, a.w, a.V, dre, dim_, ghw_all, nhw_all);
        if (!grid_sum(dre, dim_, a.part, a.bar, a.err, sh, parity, red)) return;
        if (threadIdx.x == 0) sh.H[j] = red;
        __syncthreads();
        // modified Gram-Schmidt: w -= h_{i-1,j} V_{i-1}, then h_ij = <V_i, w> (i <= j) or ||w||
        for (int i = 1; i <= j + 1; ++i) {
          const cx<double> hp = sh.H[(i - 1) * MAXM + j];
          const cx<T> h = mkc<T>((T)hp.re, (T)hp.im);
          const cx<T>* Vp = a.V + (size_t)(i - 1) * DN;
          const cx<T>* Vi = a.V + (size_t)i * DN;
          double pr = 0.0, pi = 0.0;
          for (size_t q = tid; q < DN; q += nthr) {
            const cx<T> wv = ldcg(a.w + q) - h * ldcg(Vp + q);
            st_cg(a.w + q, wv);
            if (i <= j) {
              const cx<T> vv = ldcg(Vi + q);
              pr += (double)vv.re * wv.re + (double)vv.im * wv.im;
              pi += (double)vv.re * wv.im - (double)vv.im * wv.re;
            } else {
              pr += (double)wv.re * wv.re + (double)wv.im * wv.im;
            }
          }
          if (!grid_sum(pr, pi, a.part, a.bar, a.err, sh, parity, red)) return;
          if (threadIdx.x == 0) sh.H[i * MAXM + j] = i <= j ? red : cdd(sqrt(red.re), 0.0);
          __syncthreads();
        }
        const double hn = sh.H[(j + 1) * MAXM + j].re;
        if (hn != 0.0) {  // V_{j+1} = w / h_{j+1,j}
          cx<T>* Vn = a.V + (size_t)(j + 1) * DN;
          for (size_t q = tid; q < DN; q += nthr) {
            const cx<T> wv = ldcg(a.w + q);
            st_cg(Vn + q, mkc<T>((T)(wv.re / hn), (T)(wv.im / hn)));
          }
        }
        // Givens rotations (FP64, the same on every block)
        if (threadIdx.x == 0) {
          cx<double>* Hc = sh.H;
          for (int i = 0; i < j; ++i) {
            const cx<double> hij = Hc[i * MAXM + j], hi1 = Hc[(i + 1) * MAXM + j];
            const cx<double> t = sh.cs[i] * hij + sh.sn[i] * hi1;
            Hc[(i + 1) * MAXM + j] = (-cconj(sh.sn[i])) * hij + cconj(sh.cs[i]) * hi1;
            Hc[i * MAXM + j] = t;
          }
          const cx<double> av = Hc[j * MAXM + j], bv = Hc[(j + 1) * MAXM + j];
          const double den = sqrt(cabs2(av) + cabs2(bv));
          if (den == 0.0) {
            sh.cs[j] = cdd(1.0, 0.0);
            sh.sn[j] = cdd(0.0, 0.0);
          } else {
            sh.cs[j] = cconj(cdiv_real(av, den));
            sh.sn[j] = cconj(cdiv_real(bv, den));
          }
          Hc[j * MAXM + j] = sh.cs[j] * av + sh.sn[j] * bv;
          Hc[(j + 1) * MAXM + j] = cdd(0.0, 0.0);
          sh.gv[j + 1] = (-cconj(sh.sn[j])) * sh.gv[j];
          sh.gv[j] = sh.cs[j] * sh.gv[j];
        }
        __syncthreads();
        ++its;
        kdone = j + 1;
        const cx<double> hjj = sh.H[j * MAXM + j];
        if (sqrt(cabs2(sh.gv[j + 1])) / bnorm <= a.tol || its >= a.max_its || (hjj.re == 0.0 && hjj.im == 0.0)) break;
      }
      // y = H^-1 g (upper triangular), u += Z y
      if (threadIdx.x == 0) {
        for (int i = kdone - 1; i >= 0; --i) {
          cx<double> s = sh.gv[i];
          for (int l = i + 1; l < kdone; ++l) s = s - sh.H[i * MAXM + l] * sh.y[l];
          const cx<double> d = sh.H[i * MAXM + i];
          sh.y[i] = cdiv_real(s * cconj(d), cabs2(d));
        }
      }
      __syncthreads();
      for (size_t q = tid; q < DN; q += nthr) {
        cx<T> uv = ldcg(a.u + q);
        for (int l = 0; l < kdone; ++l) {
          const cx<double> yl = sh.y[l];
          uv = uv + mkc<T>((T)yl.re, (T)yl.im) * ldcg(a.Z + (size_t)l * DN + q);
        }
        st_cg(a.u + q, uv);
      }
      if (!grid_sync(a.bar, a.err, &sh.ok)) return;
      // true residual r = f - S u -> w, beta
      double dre = 0.0, dim_ = 0.0;
      matvec<T, D>(a, tab, a.u, a.f, a.w, nullptr, dre, dim_, ghw_all, nhw_all);
      if (!grid_sum(dre, 0.0, a.part, a.bar, a.err, sh, parity, red)) return;
      beta = sqrt(red.re);
      if (beta / bnorm > a.tol && its < a.max_its) {
        for (size_t q = tid; q < DN; q += nthr) {  // V_0 = r / beta
          const cx<T> wv = ldcg(a.w + q);
          st_cg(a.V + q, mkc<T>((T)(wv.re / beta), (T)(wv.im / beta)));
        }
      }
    }
  }
  // recover (u, p): x_u = u, x_p = C^-1 (b_p - A_pu u)
  for (size_t q = tid; q < DN; q += nthr) st_cg(a.x + q, ldcg(a.u + q));
  for (size_t q = tid; q < N; q += nthr) st_cg(a.x + DN + q, czero<T>());
  if (!grid_sync(a.bar, a.err, &sh.ok)) return;
  for (size_t q = tid; q < N; q += nthr) {
    const int i = (int)(q % g.nx), j = (int)((q / g.nx) % g.ny), k = D == 3 ? (int)(q / ((size_t)g.nx * g.ny)) : 0;
    cx<T> dv;
    if (D == 3) {
      const cx<T>* uu[3] = {a.x, a.x + N, a.x + 2 * N};
      dv = s3::row_p<T, T>(uu, a.x + DN, g, i, j, k);
    } else {
      dv = s2::row_p<T, T>(a.x, a.x + N, a.x + DN, g, i, j);
    }
    st_cg(a.x + DN + q, (T(1) / g.cp[q]) * (a.b[DN + q] - dv));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.stats[0] = its;
    a.stats[1] = bnorm > 0.0 ? beta / bnorm : 0.0;
    a.stats[2] = (double)its * a.steps;
  }
}
#endif  // __CUDACC__

}  // namespace kz
