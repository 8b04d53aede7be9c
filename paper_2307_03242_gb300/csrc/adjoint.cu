// Kernels of the adjoint-state gradient: y = H^H x (or y = s b - H^H x) on the finest level in
// FP64, the material derivative -Re a^H (dH/dm) u per cell, and the sign-and-conjugation map
// z <- S conj(z) (S = diag(I, -I): displacements kept, pressure negated) that turns the forward
// cycle into a preconditioner for H^H. One thread per cell, grid-stride; the per-cell arithmetic
// is adjoint.cuh, which the tests also run in a host build against the FP64 oracle.
#include "adjoint.cuh"
#include "apply_ff2d.cuh"
#include "launch.h"

namespace adjk {

constexpr int RT = 256;

inline int blocks_for(size_t n) {
  const size_t b = (n + RT - 1) / RT;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

template <int D, typename TI, bool FFO>
__global__ void __launch_bounds__(RT) apply(Grid<double> g, const cx<TI>* __restrict__ x, const cx<double>* b,
                                           double bscale, void* __restrict__ y) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const cx<TI>* xs[4];
  for (int c = 0; c <= D; ++c) xs[c] = x + (size_t)c * N;
  for (size_t idx = (size_t)blockIdx.x * RT + threadIdx.x; idx < N; idx += (size_t)gridDim.x * RT) {
    const int i = (int)(idx % g.nx), j = (int)((idx / g.nx) % g.ny), k = (int)(idx / ((size_t)g.nx * g.ny));
    for (int c = 0; c < D; ++c) {
      const cx<double> r = adj::row_u<D, double, TI>(c, xs, g, i, j, k);
      ff2::store_val<FFO>(y, (size_t)c * N + idx, b ? bscale * b[(size_t)c * N + idx] - r : r);
    }
    const cx<double> r = adj::row_p<D, double, TI>(xs, g, i, j, k);
    ff2::store_val<FFO>(y, (size_t)D * N + idx, b ? bscale * b[(size_t)D * N + idx] - r : r);
  }
}

template <int D>
__global__ void __launch_bounds__(RT) gradient(Grid<double> g, const cx<double>* __restrict__ u,
                                              const cx<double>* __restrict__ a, double* __restrict__ glam,
                                              double* __restrict__ gmu, double* __restrict__ grho, int accumulate) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const cx<double>* us[4];
  const cx<double>* as[4];
  for (int c = 0; c <= D; ++c) {
    us[c] = u + (size_t)c * N;
    as[c] = a + (size_t)c * N;
  }
  for (size_t idx = (size_t)blockIdx.x * RT + threadIdx.x; idx < N; idx += (size_t)gridDim.x * RT) {
    const int i = (int)(idx % g.nx), j = (int)((idx / g.nx) % g.ny), k = (int)(idx / ((size_t)g.nx * g.ny));
    double gl, gm, gr;
    adj::gradient<D, double, double>(us, as, g, i, j, k, gl, gm, gr);
    if (accumulate) {
      glam[idx] += gl;
      gmu[idx] += gm;
      grho[idx] += gr;
    } else {
      glam[idx] = gl;
      gmu[idx] = gm;
      grho[idx] = gr;
    }
  }
}

// z <- S conj(z): the first nu entries (displacements) conjugated, the rest (pressure) negated too
__global__ void __launch_bounds__(RT) sconj(cx<float>* z, size_t nu, size_t n) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  for (size_t t = (size_t)blockIdx.x * RT + threadIdx.x; t < n; t += (size_t)gridDim.x * RT) {
    const cx<float> v = z[t];
    z[t] = t < nu ? mkc<float>(v.re, -v.im) : mkc<float>(-v.re, v.im);
  }
}

}  // namespace adjk

template <int D, typename TI>
void launch_adjoint_apply(const Grid<double>& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y,
                          bool ffo, cudaStream_t st) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  if (ffo) launch_dep(adjk::apply<D, TI, true>, dim3(adjk::blocks_for(N)), dim3(adjk::RT), 0, st, g, x, b, bscale, y);
  else launch_dep(adjk::apply<D, TI, false>, dim3(adjk::blocks_for(N)), dim3(adjk::RT), 0, st, g, x, b, bscale, y);
}

template <int D>
void launch_adjoint_gradient(const Grid<double>& g, const cx<double>* u, const cx<double>* a, double* glam,
                             double* gmu, double* grho, int accumulate, cudaStream_t st) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  launch_dep(adjk::gradient<D>, dim3(adjk::blocks_for(N)), dim3(adjk::RT), 0, st, g, u, a, glam, gmu, grho, accumulate);
}

void launch_sconj(cx<float>* z, size_t nu, size_t n, cudaStream_t st) {
  launch_dep(adjk::sconj, dim3(adjk::blocks_for(n)), dim3(adjk::RT), 0, st, z, nu, n);
}

template void launch_adjoint_apply<2, float>(const Grid<double>&, const cx<float>*, const cx<double>*, double, void*,
                                              bool, cudaStream_t);
template void launch_adjoint_apply<2, double>(const Grid<double>&, const cx<double>*, const cx<double>*, double, void*,
                                              bool, cudaStream_t);
template void launch_adjoint_apply<3, float>(const Grid<double>&, const cx<float>*, const cx<double>*, double, void*,
                                              bool, cudaStream_t);
template void launch_adjoint_apply<3, double>(const Grid<double>&, const cx<double>*, const cx<double>*, double, void*,
                                              bool, cudaStream_t);
template void launch_adjoint_gradient<2>(const Grid<double>&, const cx<double>*, const cx<double>*, double*, double*,
                                         double*, int, cudaStream_t);
template void launch_adjoint_gradient<3>(const Grid<double>&, const cx<double>*, const cx<double>*, double*, double*,
                                         double*, int, cudaStream_t);
