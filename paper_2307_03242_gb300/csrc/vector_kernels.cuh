// Dimension-independent kernels: FP64 Krylov reductions and updates, precision casts, and the
// dense coarsest-level inverse applied as a matrix-vector product.
#pragma once
#include "emg_types.cuh"

namespace kv {

constexpr int RT = 256;           // threads per reduction block
constexpr int MAXV = 16;          // vectors per multi-dot pass

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce NR doubles per thread into part[blockIdx.x * NR + r] (deterministic order).
template <int NR>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NR], double* part) {
  __shared__ double sh[RT / 32][NR];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    double v = warp_sum(acc[r]);
    if (lane == 0) sh[wid][r] = v;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      double v = lane < RT / 32 ? sh[lane][r] : 0.0;
      v = warp_sum(v);
      if (lane == 0) part[(size_t)blockIdx.x * NR + r] = v;
    }
  }
}

// part[blk][2i], part[blk][2i+1] = Re/Im of sum conj(V_i) w over the block's elements (i < NV),
// part[blk][2NV] = sum |w|^2.
template <int NV>
__global__ void __launch_bounds__(RT) mdot(const cx<double>* __restrict__ V, size_t ldv,
                                           const cx<double>* __restrict__ w, size_t n, double* part) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  double acc[2 * NV + 1];
#pragma unroll
  for (int r = 0; r < 2 * NV + 1; ++r) acc[r] = 0.0;
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < n; e += (size_t)gridDim.x * RT) {
    cx<double> we = w[e];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      cx<double> a = V[v * ldv + e];
      acc[2 * v] += a.re * we.re + a.im * we.im;
      acc[2 * v + 1] += a.re * we.im - a.im * we.re;
    }
    acc[2 * NV] += we.re * we.re + we.im * we.im;
  }
  block_reduce_store<2 * NV + 1>(acc, part);
}

struct Coefs { cx<double> c[64]; };

// w -= sum_i h_i V_i (i < cnt); part[blk] = sum |w_new|^2.
__global__ void __launch_bounds__(RT) update_norm(cx<double>* __restrict__ w, const cx<double>* __restrict__ V,
                                                  size_t ldv, int cnt, Coefs h, size_t n, double* part) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  double acc[1] = {0.0};
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < n; e += (size_t)gridDim.x * RT) {
    cx<double> we = w[e];
    for (int v = 0; v < cnt; ++v) we = we - h.c[v] * V[v * ldv + e];
    w[e] = we;
    acc[0] += we.re * we.re + we.im * we.im;
  }
  block_reduce_store<1>(acc, part);
}

// Sum per-block partials column-wise: out[r] = sum_b part[b*nr + r]. One block per column; each
// thread sums a fixed strided subset, then a fixed tree combines them (deterministic).
constexpr int RP = 256;
__global__ void __launch_bounds__(RP) reduce_parts(const double* __restrict__ part, int nblk, int nr,
                                                   double* __restrict__ out) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int r = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += RP) s += part[(size_t)b * nr + r];
  __shared__ double sh[RP / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < RP / 32 ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) out[r] = v;
  }
}

__global__ void scale(cx<double>* __restrict__ dst, const cx<double>* __restrict__ src, double s, size_t n) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = s * src[e];
}

// x += sum_i y_i Z_i, Z in the cycle precision.
template <typename TZ>
__global__ void combine(cx<double>* __restrict__ x, const cx<TZ>* __restrict__ Z, size_t ldz, int cnt, Coefs y,
                        size_t n) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    cx<double> a = x[e];
    for (int v = 0; v < cnt; ++v) a = a + y.c[v] * ccast<double>(Z[v * ldz + e]);
    x[e] = a;
  }
}

template <typename TD, typename TS>
__global__ void cast(cx<TD>* __restrict__ dst, const cx<TS>* __restrict__ src, size_t n) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = ccast<TD>(src[e]);
}

// x = Ainv b for the coarsest level (Ainv dense, n x n, row-major); one warp per row.
template <typename T>
__global__ void dense_gemv(const cx<T>* __restrict__ Ainv, const cx<T>* __restrict__ b, cx<T>* __restrict__ x,
                           int n) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const cx<T>* a = Ainv + (size_t)row * n;
  T re = 0, im = 0;
  for (int c = lane; c < n; c += 32) {
    cx<T> v = a[c] * b[c];
    re += v.re;
    im += v.im;
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane == 0) x[row] = mkc<T>(re, im);
}

}  // namespace kv
