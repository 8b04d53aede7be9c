// Set-up and launch of the hybrid Kaczmarz-GMRES coarsest solve (kaczmarz.cuh).
#include "kaczmarz.cuh"
#include "launch.h"

#include <atomic>

namespace {
constexpr int kMaxDev = 64;
constexpr size_t kRegionBudget = 200 * 1024;  // dynamic shared memory for the boxes' private copies

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T, int D>
cudaError_t probe_all(const Grid<T>& g, cx<T>* coef, T* inv_n2, cx<T>* e, cx<T>* y, cudaStream_t st) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  cudaError_t err = cudaMemsetAsync(coef, 0, (size_t)D * N * kz::Shape<D>::NE * sizeof(cx<T>), st);
  if (err != cudaSuccess) return err;
  for (int c2 = 0; c2 < D; ++c2)
    for (int q2 = 0; q2 < (D == 3 ? kz::PER : 1); ++q2)
      for (int q1 = 0; q1 < kz::PER; ++q1)
        for (int q0 = 0; q0 < kz::PER; ++q0) {
          kz::probe_set<T, D><<<nblk((D + 1) * N, 256), 256, 0, st>>>(e, c2, q0, q1, q2, g.nx, g.ny, g.nz);
          if (D == 3) launch_apply3<T, T>(g, e, nullptr, T(0), y, st);
          else launch_apply2<T, T>(g, e, nullptr, T(0), y, st);
          kz::probe_take<T, D><<<nblk(D * N, 256), 256, 0, st>>>(g, y, c2, q0, q1, q2, coef);
          err = cudaGetLastError();
          if (err != cudaSuccess) return err;
        }
  kz::row_norms<T, D><<<nblk(D * N, 256), 256, 0, st>>>(coef, inv_n2, D * N);
  return cudaGetLastError();
}

// The solve kernel for boxes of 1 or 2 cells per axis (fixb = 1, 2) or of at least 2 (fixb = 0).
template <typename T, int D>
const void* solve_fn(int fixb) {
  return fixb == 2 ? (const void*)kz::solve<T, D, 2>
                   : (fixb == 1 ? (const void*)kz::solve<T, D, 1> : (const void*)kz::solve<T, D, 0>);
}

template <typename T, int D>
cudaError_t plan_solve(int sms, int RS, const int box[3], KzLaunch& out) {
  // half-warps with a private region: as many as fit beside the block's region-layout table, an
  // even number (both halves of a warp)
  const size_t per_hw = (size_t)(RS + kz::PD * kz::Ring<D>::SLOT) * sizeof(cx<T>);
  const size_t table = ((size_t)(RS + 2 * D * kz::Shape<D>::SL * kz::HW) * sizeof(int) + 15) / 16 * 16;
  if (table >= kRegionBudget) return cudaErrorInvalidValue;
  int warps = (int)((kRegionBudget - table) / per_hw);
  if (warps > kz::NT / kz::HW) warps = kz::NT / kz::HW;
  warps &= ~1;
  if (warps < 2) return cudaErrorInvalidValue;
  const size_t smem = (size_t)warps * per_hw + table;
  bool two = true, one = true;
  for (int a = 0; a < D; ++a) {
    two = two && box[a] == 2;
    one = one && box[a] == 1;
  }
  const int fixb = two ? 2 : (one ? 1 : 0);
  static std::atomic<bool> attr_set[kMaxDev];
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  if (!attr_set[dev].load()) {
    for (int f : {0, 1, 2}) {
      err = cudaFuncSetAttribute(solve_fn<T, D>(f), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRegionBudget);
      if (err != cudaSuccess) return err;
    }
    attr_set[dev].store(true);
  }
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_fn<T, D>(fixb), kz::NT, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  out.blocks = sms * per_sm;
  out.warps = warps;
  out.smem = smem;
  out.fixb = fixb;
  return cudaSuccess;
}
}  // namespace

template <typename T>
cudaError_t launch_kz_probe(const Grid<T>& g, int dim, cx<T>* coef, T* inv_n2, cx<T>* e, cx<T>* y, cudaStream_t st) {
  return dim == 3 ? probe_all<T, 3>(g, coef, inv_n2, e, y, st) : probe_all<T, 2>(g, coef, inv_n2, e, y, st);
}

template <typename T>
cudaError_t plan_kz_solve(int dim, int sms, int RS, const int box[3], KzLaunch& out) {
  return dim == 3 ? plan_solve<T, 3>(sms, RS, box, out) : plan_solve<T, 2>(sms, RS, box, out);
}

template <typename T>
cudaError_t launch_kz_solve(const kz::Args<T>& a, int dim, const KzLaunch& L, cudaStream_t st) {
  kz::Args<T> args = a;
  args.warps_a = L.warps;
  void* params[] = {&args};
  const void* fn = dim == 3 ? solve_fn<T, 3>(L.fixb) : solve_fn<T, 2>(L.fixb);
  return cudaLaunchCooperativeKernel(fn, dim3(L.blocks), dim3(kz::NT), params, L.smem, st);
}

#define INST(T)                                                                                                    \
  template cudaError_t launch_kz_probe<T>(const Grid<T>&, int, cx<T>*, T*, cx<T>*, cx<T>*, cudaStream_t);         \
  template cudaError_t plan_kz_solve<T>(int, int, int, const int*, KzLaunch&);                                                \
  template cudaError_t launch_kz_solve<T>(const kz::Args<T>&, int, const KzLaunch&, cudaStream_t);
INST(float)
INST(double)
