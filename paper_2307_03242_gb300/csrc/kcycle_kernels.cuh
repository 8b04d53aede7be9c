// Vector kernels of the K-cycle's coarse-level Krylov steps (GCR(2), Sec. 2.2). The scalars
// (<a, b> / <a, a>) are reduced on the device and read back by the next kernel from device
// memory, so a cycle needs no host synchronisation.
#pragma once
#include "vector_kernels.cuh"

namespace kc {

constexpr int RT = 256;

// part[blk] = (Re, Im) of sum conj(a) b and sum |a|^2 over the block's elements (FP64 partials).
template <typename T>
__global__ void __launch_bounds__(RT) dot_parts(const cx<T>* __restrict__ a, const cx<T>* __restrict__ b, size_t n,
                                                double* part) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  double acc[3] = {0.0, 0.0, 0.0};
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < n; e += (size_t)gridDim.x * RT) {
    const cx<T> x = a[e], y = b[e];
    acc[0] += (double)x.re * y.re + (double)x.im * y.im;
    acc[1] += (double)x.re * y.im - (double)x.im * y.re;
    acc[2] += (double)x.re * x.re + (double)x.im * x.im;
  }
  kv::block_reduce_store<3>(acc, part);
}

// coef = <a, b> / <a, a> from the partials (fixed summation order), stored as (re, im).
__global__ void finalize_coef(const double* __restrict__ part, int nblk, double* __restrict__ coef) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  __shared__ double s[3][kv::RP];
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblk; b += kv::RP)
    for (int r = 0; r < 3; ++r) v[r] += part[(size_t)b * 3 + r];
  for (int r = 0; r < 3; ++r) s[r][threadIdx.x] = v[r];
  __syncthreads();
  for (int st = kv::RP / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int r = 0; r < 3; ++r) s[r][threadIdx.x] += s[r][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nn = s[2][0];
    coef[0] = nn > 0.0 ? s[0][0] / nn : 0.0;
    coef[1] = nn > 0.0 ? s[1][0] / nn : 0.0;
  }
}

// y = x0 + sgn * coef * x  (x0 may alias y)
template <typename T>
__global__ void axpy_coef(cx<T>* y, const cx<T>* x0, const cx<T>* __restrict__ x, const double* __restrict__ coef,
                          T sgn, size_t n) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const cx<T> c = mkc<T>((T)coef[0] * sgn, (T)coef[1] * sgn);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const cx<T> v = x0 ? x0[e] : czero<T>();
    y[e] = v + c * x[e];
  }
}

}  // namespace kc
