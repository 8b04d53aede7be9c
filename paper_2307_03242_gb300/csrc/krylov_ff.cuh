// FP64 Krylov vector kernels evaluated in double-FP32 arithmetic (dfloat.cuh): the vectors are
// IEEE FP64 in memory, every product and sum is carried with ~48 significant bits on the FP32
// pipe, and only per-thread partial sums and final stores touch the FP64 pipe.
#pragma once
#include "dfloat.cuh"
#include "vector_kernels.cuh"

namespace kf {

using df::f2;
constexpr int RT = kv::RT;

// part[blk][2i], [2i+1] = Re, Im of sum conj(V_i) w (i < NV); part[blk][2NV] = sum |w|^2.
template <int NV>
__global__ void __launch_bounds__(RT) mdot(const cx<double>* __restrict__ V, size_t ldv,
                                           const cx<double>* __restrict__ w, size_t n, double* part) {
  df::acc are[NV > 0 ? NV : 1], aim[NV > 0 ? NV : 1], ann;
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < n; e += (size_t)gridDim.x * RT) {
    const cx<double> we = w[e];
    const f2 wr = df::split(we.re), wi = df::split(we.im);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const cx<double> a = V[v * ldv + e];
      const f2 ar = df::split(a.re), ai = df::split(a.im);
      are[v].fma_ff(ar, wr);
      are[v].fma_ff(ai, wi);
      aim[v].fma_ff(ar, wi);
      aim[v].fms_ff(ai, wr);
    }
    ann.fma_ff(wr, wr);
    ann.fma_ff(wi, wi);
  }
  double acc[2 * NV + 1];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    acc[2 * v] = are[v].to_double();
    acc[2 * v + 1] = aim[v].to_double();
  }
  acc[2 * NV] = ann.to_double();
  kv::block_reduce_store<2 * NV + 1>(acc, part);
}

// Complex float-float coefficient.
struct c2 {
  f2 re, im;
};
struct Coefs {
  c2 c[64];
};

// w <- s * (w - sum_i h_i V_i) (i < cnt), written back as FP64; optionally also written in FP32
// to out32 (the next cycle's right-hand side); part[blk] = sum |w_new|^2.
__global__ void __launch_bounds__(RT) update_scale(cx<double>* __restrict__ w, const cx<double>* __restrict__ V,
                                                   size_t ldv, int cnt, Coefs h, f2 s, size_t n,
                                                   cx<float>* __restrict__ out32, double* part) {
  df::acc nn;
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < n; e += (size_t)gridDim.x * RT) {
    const cx<double> we = w[e];
    df::acc re, im;
    re.add(df::split(we.re));
    im.add(df::split(we.im));
    for (int v = 0; v < cnt; ++v) {
      const cx<double> a = V[v * ldv + e];
      const f2 ar = df::split(a.re), ai = df::split(a.im);
      const c2 hv = h.c[v];
      // (hr + i hi)(ar + i ai) = (hr ar - hi ai) + i (hr ai + hi ar)
      re.fms_ff(hv.re, ar);
      re.fma_ff(hv.im, ai);
      im.fms_ff(hv.re, ai);
      im.fms_ff(hv.im, ar);
    }
    df::acc ore, oim;
    ore.fma_ff(re.norm(), s);
    oim.fma_ff(im.norm(), s);
    const f2 fr = ore.norm(), fi = oim.norm();
    w[e] = mkc<double>((double)fr.hi + (double)fr.lo, (double)fi.hi + (double)fi.lo);
    if (out32) out32[e] = mkc<float>(fr.hi, fi.hi);
    nn.fma_ff(fr, fr);
    nn.fma_ff(fi, fi);
  }
  double acc[1] = {nn.to_double()};
  kv::block_reduce_store<1>(acc, part);
}

// x += sum_i y_i Z_i with Z in FP32 (exact floats) or FP64.
template <typename TZ>
__global__ void __launch_bounds__(RT) combine(cx<double>* __restrict__ x, const cx<TZ>* __restrict__ Z, size_t ldz,
                                              int cnt, Coefs y, size_t n) {
  for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < n; e += (size_t)gridDim.x * RT) {
    const cx<double> xe = x[e];
    df::acc re, im;
    re.add(df::split(xe.re));
    im.add(df::split(xe.im));
    for (int v = 0; v < cnt; ++v) {
      const cx<TZ> z = Z[v * ldz + e];
      f2 zr, zi;
      if constexpr (sizeof(TZ) == 4) {
        zr = {(float)z.re, 0.f};
        zi = {(float)z.im, 0.f};
      } else {
        zr = df::split((double)z.re);
        zi = df::split((double)z.im);
      }
      const c2 yv = y.c[v];
      re.fma_ff(yv.re, zr);
      re.fms_ff(yv.im, zi);
      im.fma_ff(yv.re, zi);
      im.fma_ff(yv.im, zr);
    }
    const f2 fr = re.norm(), fi = im.norm();
    x[e] = mkc<double>((double)fr.hi + (double)fr.lo, (double)fi.hi + (double)fi.lo);
  }
}

}  // namespace kf
