// 2D kernel launchers (explicit instantiations for the FP32 and FP64 cycles and the FP64 apply).
#include "residual2d_fast.cuh"
#include "coarse2d_coop.cuh"
#include "launch.h"

#include <atomic>
#include "apply_ff2d.cuh"

namespace {
constexpr int kMaxDevices = 64;
dim3 g2(int nx, int ny) { return dim3((nx + k2::BX - 1) / k2::BX, (ny + k2::BY - 1) / k2::BY); }
}  // namespace

template <typename T, typename TI>
void launch_apply2(const Grid<T>& g, const cx<TI>* x, const cx<T>* b, T bscale, cx<T>* y, cudaStream_t st) {
  k2::apply<T, TI><<<g2(g.nx, g.ny), dim3(k2::BX, k2::BY), 0, st>>>(g, x, b, bscale, y);
}
template <typename T>
void launch_vanka2(const Grid<T>& g, const cx<T>* b, const cx<T>* uin, cx<T>* uout, cx<T>* p, int colour, T w,
                   int zero_in, cudaStream_t st) {
  k2::vanka_fast<T><<<g2((g.nx + 1) / 2, g.ny), dim3(k2::BX, k2::BY), 0, st>>>(g, b, uin, uout, p, colour, w, zero_in);
}
template <typename T>
void launch_restrict2(const Grid<T>& g, const cx<T>* b, const cx<T>* x, cx<T>* bc, const int nc[3], cx<T>* r,
                      cudaStream_t st) {
  k2::residual_fast<T><<<g2(g.nx, g.ny), dim3(k2::BX, k2::BY), 0, st>>>(g, b, x, r);
  k2::restrict_r<T><<<g2(nc[0], nc[1]), dim3(k2::BX, k2::BY), 0, st>>>(r, bc, g.nx, g.ny, nc[0], nc[1]);
}
template <typename T>
void launch_prolong2(const cx<T>* e, cx<T>* x, const int n[3], const int nc[3], cudaStream_t st) {
  k2::prolong_add<T><<<g2(n[0], n[1]), dim3(k2::BX, k2::BY), 0, st>>>(e, x, n[0], n[1], nc[0], nc[1]);
}

template void launch_apply2<float, float>(const Grid<float>&, const cx<float>*, const cx<float>*, float, cx<float>*, cudaStream_t);
template void launch_apply2<double, double>(const Grid<double>&, const cx<double>*, const cx<double>*, double, cx<double>*, cudaStream_t);
template void launch_apply2<double, float>(const Grid<double>&, const cx<float>*, const cx<double>*, double, cx<double>*, cudaStream_t);
#define INST(T)                                                                                                   \
  template void launch_vanka2<T>(const Grid<T>&, const cx<T>*, const cx<T>*, cx<T>*, cx<T>*, int, T, int, cudaStream_t); \
  template void launch_restrict2<T>(const Grid<T>&, const cx<T>*, const cx<T>*, cx<T>*, const int*, cx<T>*, cudaStream_t); \
  template void launch_prolong2<T>(const cx<T>*, cx<T>*, const int*, const int*, cudaStream_t);
INST(float)
INST(double)

template <typename TI>
void launch_apply_ff2(const ff2::FineFF& g, const cx<TI>* x, const cx<double>* b, double bscale, cx<double>* y,
                      cudaStream_t st) {
  ff2::apply<TI><<<g2(g.nx, g.ny), dim3(ff2::BX, ff2::BY), 0, st>>>(g, x, b, bscale, y);
}
template void launch_apply_ff2<float>(const ff2::FineFF&, const cx<float>*, const cx<double>*, double, cx<double>*, cudaStream_t);
template void launch_apply_ff2<double>(const ff2::FineFF&, const cx<double>*, const cx<double>*, double, cx<double>*, cudaStream_t);

// All sweeps of one coarsest-level solve in one cooperative launch (x starts from zero).
// Cooperative sweeps on a small level: 64-thread blocks spread the few cells over as many SMs as
// possible (fewer warps per SM shortens each thread's latency chain), capped at what is
// co-resident.
template <typename T>
cudaError_t launch_sweeps_coop2(const Grid<T>& g, const cx<T>* b, cx<T>* x, cx<T>* alt, int sweeps, T w,
                                int zero_first, cudaStream_t st) {
  constexpr int threads = 64;
  static std::atomic<int> caps[kMaxDevices];  // co-resident blocks of this instantiation, per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  int cap = caps[dev].load();
  if (cap == 0) {
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2::sweeps_coop<T>, threads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    cap = sms * per_sm;
    caps[dev].store(cap);
  }
  const long long items = (long long)((g.nx + 1) / 2) * g.ny;
  const long long want = (items + threads - 1) / threads;
  int blocks = (int)(want < cap ? want : cap);
  Grid<T> gg = g;
  const cx<T>* bb = b;
  cx<T>* xx = x;
  cx<T>* aa = alt;
  int sw = sweeps, zf = zero_first;
  T ww = w;
  void* args[] = {&gg, &bb, &xx, &aa, &sw, &ww, &zf};
  return cudaLaunchCooperativeKernel((const void*)k2::sweeps_coop<T>, dim3(blocks), dim3(threads), args, 0, st);
}
template cudaError_t launch_sweeps_coop2<float>(const Grid<float>&, const cx<float>*, cx<float>*, cx<float>*, int, float, int, cudaStream_t);
template cudaError_t launch_sweeps_coop2<double>(const Grid<double>&, const cx<double>*, cx<double>*, cx<double>*, int, double, int, cudaStream_t);
