// 3D kernel launchers (explicit instantiations for the FP32 and FP64 cycles and the FP64 apply).
#include "kernels3d.cuh"
#include "launch.h"

namespace {
dim3 g3(int nx, int ny, int nz) {
  return dim3((nx + k3::BX - 1) / k3::BX, (ny + k3::BY - 1) / k3::BY, (nz + k3::BZ - 1) / k3::BZ);
}
dim3 b3() { return dim3(k3::BX, k3::BY, k3::BZ); }
}  // namespace

template <typename T, typename TI>
void launch_apply3(const Grid<T>& g, const cx<TI>* x, const cx<T>* b, T bscale, cx<T>* y, cudaStream_t st) {
  k3::apply<T, TI><<<g3(g.nx, g.ny, g.nz), b3(), 0, st>>>(g, x, b, bscale, y);
}
template <typename T>
void launch_vanka3(const Grid<T>& g, const cx<T>* b, const cx<T>* uin, cx<T>* uout, cx<T>* p, int colour, T w,
                   int zero_in, cudaStream_t st) {
  k3::vanka<T><<<g3((g.nx + 1) / 2, g.ny, g.nz), b3(), 0, st>>>(g, b, uin, uout, p, colour, w, zero_in);
}
template <typename T>
void launch_restrict3(const Grid<T>& g, const cx<T>* b, const cx<T>* x, cx<T>* bc, const int nc[3], int zero_x,
                      cudaStream_t st) {
  k3::restrict_residual<T><<<g3(nc[0], nc[1], nc[2]), b3(), 0, st>>>(g, b, x, bc, nc[0], nc[1], nc[2], zero_x);
}
template <typename T>
void launch_prolong3(const cx<T>* e, cx<T>* x, const int n[3], const int nc[3], cudaStream_t st) {
  k3::prolong_add<T><<<g3(n[0], n[1], n[2]), b3(), 0, st>>>(e, x, n[0], n[1], n[2], nc[0], nc[1], nc[2]);
}

template void launch_apply3<float, float>(const Grid<float>&, const cx<float>*, const cx<float>*, float, cx<float>*, cudaStream_t);
template void launch_apply3<double, double>(const Grid<double>&, const cx<double>*, const cx<double>*, double, cx<double>*, cudaStream_t);
template void launch_apply3<double, float>(const Grid<double>&, const cx<float>*, const cx<double>*, double, cx<double>*, cudaStream_t);
#define INST(T)                                                                                                   \
  template void launch_vanka3<T>(const Grid<T>&, const cx<T>*, const cx<T>*, cx<T>*, cx<T>*, int, T, int, cudaStream_t); \
  template void launch_restrict3<T>(const Grid<T>&, const cx<T>*, const cx<T>*, cx<T>*, const int*, int, cudaStream_t); \
  template void launch_prolong3<T>(const cx<T>*, cx<T>*, const int*, const int*, cudaStream_t);
INST(float)
INST(double)
