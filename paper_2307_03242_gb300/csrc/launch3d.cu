// 3D kernel launchers (explicit instantiations for the FP32 and FP64 cycles and the FP64 apply).
#include "vanka3d_tile.cuh"
#include "residual3d.cuh"
#include "launch.h"
#include "adjoint_ff3.cuh"

#include <atomic>

namespace {
dim3 g3(int nx, int ny, int nz) {
  return dim3((nx + k3::BX - 1) / k3::BX, (ny + k3::BY - 1) / k3::BY, (nz + k3::BZ - 1) / k3::BZ);
}
dim3 b3() { return dim3(k3::BX, k3::BY, k3::BZ); }
}  // namespace

template <typename T, typename TI>
void launch_apply3(const Grid<T>& g, const cx<TI>* x, const cx<T>* b, T bscale, cx<T>* y, cudaStream_t st) {
  launch_dep(k3::apply<T, TI>, dim3(g3(g.nx, g.ny, g.nz)), dim3(b3()), 0, st, g, x, b, bscale, y);
}
template <typename T>
void launch_vanka3(const Grid<T>& g, const cx<T>* b, const cx<T>* uin, cx<T>* uout, cx<T>* p, int colour, T w,
                   int zero_in, cudaStream_t st) {
  if (g.nx >= 16 && g.ny >= 8 && g.nz >= 4) {
    // the dynamic shared memory limit is a per-device function attribute: set it once per device
    static std::atomic<bool> attr_set[64];
    const size_t smem = sizeof(k3t::Tile<T>);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev].load()) {
      cudaFuncSetAttribute(k3t::vanka_tile<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (dev >= 0 && dev < 64) attr_set[dev].store(true);
    }
    dim3 grid((g.nx + k3t::TX - 1) / k3t::TX, (g.ny + k3t::TY - 1) / k3t::TY, (g.nz + k3t::TZ - 1) / k3t::TZ);
    launch_dep(k3t::vanka_tile<T>, dim3(grid), dim3(k3t::NT), smem, st, g, b, uin, uout, p, colour, w, zero_in);
  } else {
    launch_dep(k3::vanka<T>, dim3(g3((g.nx + 1) / 2, g.ny, g.nz)), dim3(b3()), 0, st, g, b, uin, uout, p, colour, w, zero_in);
  }
}
template <typename T>
void launch_restrict3(const Grid<T>& g, const cx<T>* b, const cx<T>* x, cx<T>* bc, const int nc[3], cx<T>* r,
                      cudaStream_t st) {
  launch_dep(k3::residual<T>, dim3(g3(g.nx, g.ny, g.nz)), dim3(b3()), 0, st, g, b, x, r);
  launch_dep(k3::restrict_r<T>, dim3(g3(nc[0], nc[1], nc[2])), dim3(b3()), 0, st, r, bc, g.nx, g.ny, g.nz, nc[0], nc[1], nc[2]);
}
template <typename T>
void launch_prolong3(const cx<T>* e, cx<T>* x, const int n[3], const int nc[3], cudaStream_t st) {
  launch_dep(k3::prolong_add<T>, dim3(g3(n[0], n[1], n[2])), dim3(b3()), 0, st, e, x, n[0], n[1], n[2], nc[0], nc[1], nc[2]);
}

template void launch_apply3<float, float>(const Grid<float>&, const cx<float>*, const cx<float>*, float, cx<float>*, cudaStream_t);
template void launch_apply3<double, double>(const Grid<double>&, const cx<double>*, const cx<double>*, double, cx<double>*, cudaStream_t);
template void launch_apply3<double, float>(const Grid<double>&, const cx<float>*, const cx<double>*, double, cx<double>*, cudaStream_t);
#define INST(T)                                                                                                   \
  template void launch_vanka3<T>(const Grid<T>&, const cx<T>*, const cx<T>*, cx<T>*, cx<T>*, int, T, int, cudaStream_t); \
  template void launch_restrict3<T>(const Grid<T>&, const cx<T>*, const cx<T>*, cx<T>*, const int*, cx<T>*, cudaStream_t); \
  template void launch_prolong3<T>(const cx<T>*, cx<T>*, const int*, const int*, cudaStream_t);
INST(float)
INST(double)

template <typename TI>
void launch_apply_ff3(const ff3::FineFF3& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y, bool ffo,
                      cudaStream_t st) {
  dim3 grid((g.nx + ff3::BX - 1) / ff3::BX, (g.ny + ff3::BY - 1) / ff3::BY, (g.nz + ff3::BZ - 1) / ff3::BZ);
  if (ffo) launch_dep(ff3::apply<TI, true>, dim3(grid), dim3(ff3::BX, ff3::BY, ff3::BZ), 0, st, g, x, b, bscale, y);
  else launch_dep(ff3::apply<TI, false>, dim3(grid), dim3(ff3::BX, ff3::BY, ff3::BZ), 0, st, g, x, b, bscale, y);
}
template void launch_apply_ff3<float>(const ff3::FineFF3&, const cx<float>*, const cx<double>*, double, void*, bool,
                                      cudaStream_t);
template void launch_apply_ff3<double>(const ff3::FineFF3&, const cx<double>*, const cx<double>*, double, void*, bool,
                                       cudaStream_t);

// y = H^H x (or bscale b - H^H x) of the finest 3D operator in float-float arithmetic on the
// forward apply's coefficient arrays (adjoint_ff3.cuh).
template <typename TI>
void launch_apply_adjoint_ff3(const ff3::FineFF3& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y,
                              bool ffo, cudaStream_t st) {
  dim3 grid((g.nx + ff3::BX - 1) / ff3::BX, (g.ny + ff3::BY - 1) / ff3::BY, (g.nz + ff3::BZ - 1) / ff3::BZ);
  if (ffo) launch_dep(ff3::apply_adjoint<TI, true>, dim3(grid), dim3(ff3::BX, ff3::BY, ff3::BZ), 0, st, g, x, b, bscale, y);
  else launch_dep(ff3::apply_adjoint<TI, false>, dim3(grid), dim3(ff3::BX, ff3::BY, ff3::BZ), 0, st, g, x, b, bscale, y);
}
template void launch_apply_adjoint_ff3<float>(const ff3::FineFF3&, const cx<float>*, const cx<double>*, double, void*,
                                              bool, cudaStream_t);
template void launch_apply_adjoint_ff3<double>(const ff3::FineFF3&, const cx<double>*, const cx<double>*, double,
                                               void*, bool, cudaStream_t);
