// FP64 Krylov vector kernels evaluated in double-FP32 arithmetic (dfloat.cuh): every product and
// sum is carried with ~48 significant bits on the FP32 pipe. The Krylov basis and the applied
// vector w are stored as float-float pairs (df::cff, 16 bytes per complex value like a complex
// double), so that these kernels neither split nor assemble doubles; the iterate x stays IEEE
// FP64 and is split and assembled with integer operations. No FP64 instruction runs per element
// (this part's FP64 pipe is ~57x slower than its FP32 pipe).
#pragma once
#include "dfloat.cuh"
#include "vector_kernels.cuh"

namespace kf {

using df::cff;
using df::f2;
constexpr int RT = kv::RT;

// Elements per thread and loop iteration: their loads are issued together, so that enough bytes
// are in flight per thread to cover the HBM latency (the vectors are 100s of MB).
constexpr int UPD = 4;

// Warp sum of float-float values by an XOR butterfly; TwoSum is exact and symmetric in its
// operands, so every lane ends with the same sum.
__device__ __forceinline__ f2 warp_sum_ff(f2 v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, v.hi, off), l = __shfl_xor_sync(0xffffffffu, v.lo, off);
    float s, t;
    df::two_sum(v.hi, h, s, t);
    t += v.lo + l;
    df::two_sum(s, t, v.hi, v.lo);
  }
  return v;
}

// Block sums of every thread's accumulators, in float-float on the FP32 pipe; part[blk][r] is the
// block's sum r as a double (assembled without FP64 instructions).
template <int NR>
__device__ __forceinline__ void block_reduce_store_ff(const df::acc (&a)[NR], double* part) {
  __shared__ f2 sh[RT / 32][NR];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const f2 v = warp_sum_ff(a[r].norm());
    if (lane == 0) sh[wid][r] = v;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const f2 v = warp_sum_ff(lane < RT / 32 ? sh[lane][r] : f2{0.f, 0.f});
      if (lane == 0) part[(size_t)blockIdx.x * NR + r] = df::join(v.hi, v.lo);
    }
  }
}

// part[blk][2i], [2i+1] = Re, Im of sum conj(V_i) w (i < NV); part[blk][2NV] = sum |w|^2.
template <int NV>
__global__ void __launch_bounds__(RT) mdot(const cff* __restrict__ V, size_t ldv, const cff* __restrict__ w, size_t n,
                                           double* part) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  constexpr int U = NV <= 2 ? 4 : (NV <= 6 ? 2 : 1);
  df::acc are[NV > 0 ? NV : 1], aim[NV > 0 ? NV : 1], ann;
  const size_t stride = (size_t)gridDim.x * RT;
  const cff z = {0.f, 0.f, 0.f, 0.f};
  for (size_t e0 = (size_t)blockIdx.x * RT + threadIdx.x; e0 < n; e0 += U * stride) {
    cff we[U], a[U][NV > 0 ? NV : 1];
    // every load is issued before any arithmetic (indices clamped into the vector); elements
    // past the end are then replaced by zeros, which add nothing
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const size_t e = e0 + u * stride < n ? e0 + u * stride : n - 1;
      we[u] = w[e];
#pragma unroll
      for (int v = 0; v < NV; ++v) a[u][v] = V[v * ldv + e];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (e0 + u * stride < n) continue;
      we[u] = z;
#pragma unroll
      for (int v = 0; v < NV; ++v) a[u][v] = z;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const f2 wr = {we[u].rh, we[u].rl}, wi = {we[u].ih, we[u].il};
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const f2 ar = {a[u][v].rh, a[u][v].rl}, ai = {a[u][v].ih, a[u][v].il};
        are[v].fma_ff(ar, wr);
        are[v].fma_ff(ai, wi);
        aim[v].fma_ff(ar, wi);
        aim[v].fms_ff(ai, wr);
      }
      ann.fma_ff(wr, wr);
      ann.fma_ff(wi, wi);
    }
  }
  df::acc all[2 * NV + 1];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    all[2 * v] = are[v];
    all[2 * v + 1] = aim[v];
  }
  all[2 * NV] = ann;
  block_reduce_store_ff<2 * NV + 1>(all, part);
}

// Complex float-float coefficient.
struct c2 {
  f2 re, im;
};
struct Coefs {
  c2 c[64];
};

// w <- s * (w - sum_i h_i V_i) (i < cnt), written back in place; optionally also written to
// outc, the next cycle's right-hand side, in FP32 (outk = 1) or FP64 (outk = 2);
// part[blk] = sum |w_new|^2.
__global__ void __launch_bounds__(RT) update_scale(cff* __restrict__ w, const cff* __restrict__ V, size_t ldv, int cnt,
                                                   Coefs h, f2 s, size_t n, void* __restrict__ outc, int outk,
                                                   double* part) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  df::acc nn;
  const size_t stride = (size_t)gridDim.x * RT;
  const cff z = {0.f, 0.f, 0.f, 0.f};
  for (size_t e0 = (size_t)blockIdx.x * RT + threadIdx.x; e0 < n; e0 += UPD * stride) {
    df::acc re[UPD], im[UPD];
#pragma unroll
    for (int u = 0; u < UPD; ++u) {
      const size_t e = e0 + u * stride;
      const cff we = e < n ? w[e] : z;
      re[u].add(f2{we.rh, we.rl});
      im[u].add(f2{we.ih, we.il});
    }
    for (int v = 0; v < cnt; ++v) {
      cff a[UPD];
#pragma unroll
      for (int u = 0; u < UPD; ++u) a[u] = V[v * ldv + (e0 + u * stride < n ? e0 + u * stride : n - 1)];
#pragma unroll
      for (int u = 0; u < UPD; ++u)
        if (e0 + u * stride >= n) a[u] = z;
      const c2 hv = h.c[v];
#pragma unroll
      for (int u = 0; u < UPD; ++u) {
        const f2 ar = {a[u].rh, a[u].rl}, ai = {a[u].ih, a[u].il};
        // (hr + i hi)(ar + i ai) = (hr ar - hi ai) + i (hr ai + hi ar)
        re[u].fms_ff(hv.re, ar);
        re[u].fma_ff(hv.im, ai);
        im[u].fms_ff(hv.re, ai);
        im[u].fms_ff(hv.im, ar);
      }
    }
#pragma unroll
    for (int u = 0; u < UPD; ++u) {
      const size_t e = e0 + u * stride;
      if (e >= n) break;
      df::acc ore, oim;
      ore.fma_ff(re[u].norm(), s);
      oim.fma_ff(im[u].norm(), s);
      const f2 fr = ore.norm(), fi = oim.norm();
      w[e] = {fr.hi, fr.lo, fi.hi, fi.lo};
      if (outk == 1) static_cast<cx<float>*>(outc)[e] = mkc<float>(fr.hi, fi.hi);
      else if (outk == 2) static_cast<cx<double>*>(outc)[e] = mkc<double>(df::join(fr.hi, fr.lo), df::join(fi.hi, fi.lo));
      nn.fma_ff(fr, fr);
      nn.fma_ff(fi, fi);
    }
  }
  const df::acc all[1] = {nn};
  block_reduce_store_ff<1>(all, part);
}

// x += sum_i y_i Z_i with Z in FP32 (exact floats) or FP64.
template <typename TZ>
__global__ void __launch_bounds__(RT) combine(cx<double>* __restrict__ x, const cx<TZ>* __restrict__ Z, size_t ldz,
                                              int cnt, Coefs y, size_t n) {
  grid_dependency_wait();  // launched with programmatic stream serialisation
  const size_t stride = (size_t)gridDim.x * RT;
  for (size_t e0 = (size_t)blockIdx.x * RT + threadIdx.x; e0 < n; e0 += UPD * stride) {
    df::acc re[UPD], im[UPD];
#pragma unroll
    for (int u = 0; u < UPD; ++u) {
      const size_t e = e0 + u * stride;
      const cx<double> xe = e < n ? x[e] : czero<double>();
      re[u].add(df::split(xe.re));
      im[u].add(df::split(xe.im));
    }
    for (int v = 0; v < cnt; ++v) {
      cx<TZ> zv[UPD];
#pragma unroll
      for (int u = 0; u < UPD; ++u) zv[u] = Z[v * ldz + (e0 + u * stride < n ? e0 + u * stride : n - 1)];
#pragma unroll
      for (int u = 0; u < UPD; ++u)
        if (e0 + u * stride >= n) zv[u] = czero<TZ>();
      const c2 yv = y.c[v];
#pragma unroll
      for (int u = 0; u < UPD; ++u) {
        f2 zr, zi;
        if constexpr (sizeof(TZ) == 4) {
          zr = {(float)zv[u].re, 0.f};
          zi = {(float)zv[u].im, 0.f};
        } else {
          zr = df::split((double)zv[u].re);
          zi = df::split((double)zv[u].im);
        }
        re[u].fma_ff(yv.re, zr);
        re[u].fms_ff(yv.im, zi);
        im[u].fma_ff(yv.re, zi);
        im[u].fma_ff(yv.im, zr);
      }
    }
#pragma unroll
    for (int u = 0; u < UPD; ++u) {
      const size_t e = e0 + u * stride;
      if (e >= n) break;
      const f2 fr = re[u].norm(), fi = im[u].norm();
      x[e] = mkc<double>(df::join(fr.hi, fr.lo), df::join(fi.hi, fi.lo));
    }
  }
}

}  // namespace kf
