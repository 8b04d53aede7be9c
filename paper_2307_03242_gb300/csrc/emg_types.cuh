// Complex arithmetic and per-level grid descriptors shared by the kernels and the host code.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#define HD __host__ __device__ __forceinline__

#include "pdl.cuh"

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

template <typename T> HD cx<T> mkc(T r, T i) { cx<T> z; z.re = r; z.im = i; return z; }
// read-only loads of complex values (one 8- or 16-byte load)
HD cx<float> ldg(const cx<float>* p) {
#ifdef __CUDA_ARCH__
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return mkc<float>(v.x, v.y);
#else
  return *p;
#endif
}
HD cx<double> ldg(const cx<double>* p) {
#ifdef __CUDA_ARCH__
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return mkc<double>(v.x, v.y);
#else
  return *p;
#endif
}
// L2-coherent loads (cached in L2 only): for values that other blocks of the same launch wrote
// before a grid-wide barrier, which the read-only path may not see.
HD cx<float> ldcg(const cx<float>* p) {
#ifdef __CUDA_ARCH__
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return mkc<float>(v.x, v.y);
#else
  return *p;
#endif
}
HD cx<double> ldcg(const cx<double>* p) {
#ifdef __CUDA_ARCH__
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return mkc<double>(v.x, v.y);
#else
  return *p;
#endif
}
template <typename T> HD cx<T> czero() { return mkc<T>(T(0), T(0)); }
template <typename T> HD cx<T> operator+(cx<T> a, cx<T> b) { return mkc<T>(a.re + b.re, a.im + b.im); }
template <typename T> HD cx<T> operator-(cx<T> a, cx<T> b) { return mkc<T>(a.re - b.re, a.im - b.im); }
template <typename T> HD cx<T> operator-(cx<T> a) { return mkc<T>(-a.re, -a.im); }
template <typename T> HD cx<T> operator*(cx<T> a, cx<T> b) {
  return mkc<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> HD cx<T> operator*(T s, cx<T> a) { return mkc<T>(s * a.re, s * a.im); }
template <typename T> HD cx<T> cconj(cx<T> a) { return mkc<T>(a.re, -a.im); }
template <typename T> HD T cabs2(cx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T> HD cx<T> cinv(cx<T> a) {
  T d = T(1) / cabs2(a);
  return mkc<T>(a.re * d, -a.im * d);
}
template <typename T, typename S> HD cx<T> ccast(cx<S> a) { return mkc<T>((T)a.re, (T)a.im); }

HD int iclamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Read-only load: the texture/read-only path on the device, a plain load on the host.
template <typename T> HD T ldg(const T* p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}

// Geometry and coefficients of one level, by value in every kernel launch.
//   t0 = (1+beta)/2, t1 = (1-beta)/4: weights of the beta-spread derivative across one axis
//     (2D, Eq. 3.5: beta*[-1 1] + (1-beta)/4*[1 2 1] x [-1 1]);
//   in 3D the transverse weights are beta*delta + (1-beta)/16*[1 2 1]x[1 2 1] (Eq. dxSkew3D);
//   sm = (1-beta)/(2d): mass spread weight (Eq. 3.3 / massHO3D).
template <typename T>
struct Grid {
  int nx, ny, nz;           // nz = 1 in 2D
  T h, ih;                  // cell size, 1/h
  T beta, sm;               // beta, mass spread weight
  T w2;                     // omega^2
  T att;                    // gamma + shift (alpha in the cycle, 0 outside)
  T ablL, ablG;             // absorbing layer: physical thickness (0: none), gamma at the boundary
  T Lx, Ly, Lz;             // physical domain lengths
  const T* mu;              // cell-centred mu
  const T* rho;             // cell-centred rho
  const T* cp;              // cell-centred 1/(lambda + mu)
  // Absorbing-layer attenuation along each axis, tabulated per level (nullptr: evaluate the
  // profile): tab[a][2*(k+2)] at the lattice position k h, tab[a][2*(k+2)+1] at (k+1/2) h, for
  // k = -2 .. n_a+2 (the values outside the domain only ever multiply zero displacements).
  const T* abl_tab[3];
  // Per axis, the lattice range [zlo, zhi] on which the tabulated attenuation is exactly zero at
  // both k h and (k+1/2) h (empty when zlo > zhi). Kernels whose whole window lies inside it take
  // a variant that skips the absorbing-layer terms; the result is the same.
  int zlo[3] = {1, 1, 1}, zhi[3] = {0, 0, 0};
  // Economic Vanka: the cell block's displacement part is replaced by its diagonal (Sec. 2.3).
  int economic = 0;
  HD bool abl_free(int a, int lo, int hi) const { return lo >= zlo[a] && hi <= zhi[a]; }
};

// Absorbing-layer attenuation at a physical position: gamma_max * sum_a (delta_a / L)^2.
template <typename T>
HD T abl_axis(T x, T L, T X) {
  T a = L - x;
  T b = x - (X - L);
  T d = (a > T(0) ? a : T(0)) + (b > T(0) ? b : T(0));
  return d * d;
}
