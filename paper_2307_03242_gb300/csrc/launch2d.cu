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
  launch_dep(k2::apply<T, TI>, dim3(g2(g.nx, g.ny)), dim3(k2::BX, k2::BY), 0, st, g, x, b, bscale, y);
}
template <typename T>
void launch_vanka2(const Grid<T>& g, const cx<T>* b, const cx<T>* uin, cx<T>* uout, cx<T>* p, int colour, T w,
                   int zero_in, cudaStream_t st) {
  launch_dep(k2::vanka_fast<T>, dim3(g2((g.nx + 1) / 2, g.ny)), dim3(k2::BX, k2::BY), 0, st, g, b, uin, uout, p, colour, w, zero_in);
}
template <typename T>
void launch_restrict2(const Grid<T>& g, const cx<T>* b, const cx<T>* x, cx<T>* bc, const int nc[3], cx<T>* r,
                      cudaStream_t st) {
  launch_dep(k2::residual_fast<T>, dim3(g2(g.nx, g.ny)), dim3(k2::BX, k2::BY), 0, st, g, b, x, r);
  launch_dep(k2::restrict_r<T>, dim3(g2(nc[0], nc[1])), dim3(k2::BX, k2::BY), 0, st, r, bc, g.nx, g.ny, nc[0], nc[1]);
}
template <typename T>
void launch_prolong2(const cx<T>* e, cx<T>* x, const int n[3], const int nc[3], cudaStream_t st) {
  launch_dep(k2::prolong_add<T>, dim3(g2(n[0], n[1])), dim3(k2::BX, k2::BY), 0, st, e, x, n[0], n[1], nc[0], nc[1]);
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
void launch_apply_ff2(const ff2::FineFF& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y, bool ffo,
                      cudaStream_t st) {
  if (ffo) launch_dep(ff2::apply<TI, true>, dim3(g2(g.nx, g.ny)), dim3(ff2::BX, ff2::BY), 0, st, g, x, b, bscale, y);
  else launch_dep(ff2::apply<TI, false>, dim3(g2(g.nx, g.ny)), dim3(ff2::BX, ff2::BY), 0, st, g, x, b, bscale, y);
}
template void launch_apply_ff2<float>(const ff2::FineFF&, const cx<float>*, const cx<double>*, double, void*, bool,
                                      cudaStream_t);
template void launch_apply_ff2<double>(const ff2::FineFF&, const cx<double>*, const cx<double>*, double, void*, bool,
                                       cudaStream_t);

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

// ---------------------------------------------------------------- one-pass red-black sweep (FP32)
#include "sweep2d_tile.cuh"
#include "residual2d_tile.cuh"

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime (no link-time dependency on the driver library).
EncodeTiled encode_fn() {
  static std::atomic<EncodeTiled> fn{nullptr};
  EncodeTiled f = fn.load();
  if (f) return f;
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  f = (EncodeTiled)p;
  fn.store(f);
  return f;
}

// A float tensor of rank 2 or 3 with inner extent d0 (contiguous), read in boxes of b0 x b1 (x b2).
bool encode(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides_bytes,
            const cuuint32_t* box) {
  EncodeTiled f = encode_fn();
  if (!f) return false;
  const cuuint32_t es[3] = {1, 1, 1};
  return f(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base), dims, strides_bytes, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

bool sweep_tile_fits(const Grid<float>& g, const void* b, const void* xin, const void* xout) {
  const uintptr_t a = (uintptr_t)b | (uintptr_t)xin | (uintptr_t)xout | (uintptr_t)g.mu | (uintptr_t)g.rho;
  return g.nz == 1 && g.nx % 4 == 0 && g.nx >= 4 && g.ny >= 2 && (a % 16) == 0 && xin != xout;
}

namespace {
template <int TY>
cudaError_t launch_sweep_tile_ty(const Grid<float>& g, const cx<float>* b, const cx<float>* xin, cx<float>* xout,
                                 float w, int zero_in, const cx<float>* e, int nxc, int nyc, int* err,
                                 cudaStream_t st) {
  using G = k2t::Geo<TY>;
  static std::atomic<int> attr_set[kMaxDevices];
  int dev = 0;
  cudaError_t err_ = cudaGetDevice(&dev);
  if (err_ != cudaSuccess) return err_;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!attr_set[dev].load()) {
    err_ = cudaFuncSetAttribute(k2t::sweep_tile<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
    if (err_ == cudaSuccess)
      err_ = cudaFuncSetAttribute(k2t::sweep_tile<TY>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared);
    if (err_ != cudaSuccess) return err_;
    attr_set[dev].store(1);
  }
  const cuuint64_t nx = (cuuint64_t)g.nx, ny = (cuuint64_t)g.ny;
  CUtensorMap tx, tmu, trho;
  {
    // x: floats (2 nx, ny, 3): the u1, u2 and p planes, re/im interleaved
    const cuuint64_t dims[3] = {2 * nx, ny, 3}, strides[2] = {nx * 8, nx * ny * 8};
    const cuuint32_t box[3] = {2 * k2t::DX, (cuuint32_t)G::DY, 3};
    // with a zero input x is not read; the map still has to be valid
    if (!encode(&tx, zero_in ? (const void*)xout : (const void*)xin, 3, dims, strides, box)) return cudaErrorInvalidValue;
  }
  {
    const cuuint64_t dims[2] = {nx, ny}, strides[1] = {nx * 4};
    const cuuint32_t box[2] = {k2t::DX, (cuuint32_t)G::DY};
    if (!encode(&tmu, g.mu, 2, dims, strides, box) || !encode(&trho, g.rho, 2, dims, strides, box))
      return cudaErrorInvalidValue;
  }
  CUtensorMap te = tx;  // a valid map in every case; read only with a correction
  if (e) {
    const cuuint64_t nc = (cuuint64_t)nxc, mc = (cuuint64_t)nyc;
    const cuuint64_t dims[3] = {2 * nc, mc, 3}, strides[2] = {nc * 8, nc * mc * 8};
    const cuuint32_t box[3] = {2 * G::EX, (cuuint32_t)G::EY, 3};
    if (!encode(&te, e, 3, dims, strides, box)) return cudaErrorInvalidValue;
  }
  k2t::Args a{g, b, xout, w, zero_in, err, e ? 1 : 0, nxc, nyc};
  const dim3 grid((g.nx + k2t::TX - 1) / k2t::TX, (g.ny + TY - 1) / TY);
  return launch_dep(k2t::sweep_tile<TY>, grid, dim3(k2t::NT), G::SMEM_BYTES, st, tx, tmu, trho, te, a);
}
}  // namespace

cudaError_t launch_sweep_tile(const Grid<float>& g, const cx<float>* b, const cx<float>* xin, cx<float>* xout, float w,
                              int zero_in, const cx<float>* e, int nxc, int nyc, int ty, int* err, cudaStream_t st) {
  if (e && (zero_in || nxc * 2 != g.nx || nyc * 2 != g.ny || ((uintptr_t)e % 16))) return cudaErrorInvalidValue;
  if (ty == 24) return launch_sweep_tile_ty<24>(g, b, xin, xout, w, zero_in, e, nxc, nyc, err, st);
  if (ty == 8) return launch_sweep_tile_ty<8>(g, b, xin, xout, w, zero_in, e, nxc, nyc, err, st);
  if (ty == 4) return launch_sweep_tile_ty<4>(g, b, xin, xout, w, zero_in, e, nxc, nyc, err, st);
  return cudaErrorInvalidValue;
}

namespace {
template <int TY>
cudaError_t launch_resid_restrict_tile_ty(const Grid<float>& g, const cx<float>* b, const cx<float>* x, cx<float>* bc,
                                          int nxc, int nyc, int* err, cudaStream_t st) {
  using G = k2t::Geo<TY>;
  static std::atomic<int> attr_set[kMaxDevices];
  int dev = 0;
  cudaError_t err_ = cudaGetDevice(&dev);
  if (err_ != cudaSuccess) return err_;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!attr_set[dev].load()) {
    err_ = cudaFuncSetAttribute(k2t::resid_restrict_tile<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_BYTES);
    if (err_ == cudaSuccess)
      err_ = cudaFuncSetAttribute(k2t::resid_restrict_tile<TY>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared);
    if (err_ != cudaSuccess) return err_;
    attr_set[dev].store(1);
  }
  const cuuint64_t nx = (cuuint64_t)g.nx, ny = (cuuint64_t)g.ny;
  CUtensorMap tx, tmu, trho;
  {
    const cuuint64_t dims[3] = {2 * nx, ny, 3}, strides[2] = {nx * 8, nx * ny * 8};
    const cuuint32_t box[3] = {2 * k2t::DX, (cuuint32_t)G::DY, 3};
    if (!encode(&tx, x, 3, dims, strides, box)) return cudaErrorInvalidValue;
  }
  {
    const cuuint64_t dims[2] = {nx, ny}, strides[1] = {nx * 4};
    const cuuint32_t box[2] = {k2t::DX, (cuuint32_t)G::DY};
    if (!encode(&tmu, g.mu, 2, dims, strides, box) || !encode(&trho, g.rho, 2, dims, strides, box))
      return cudaErrorInvalidValue;
  }
  k2t::RArgs a{g, b, bc, nxc, nyc, err};
  const dim3 grid((g.nx + k2t::TX - 1) / k2t::TX, (g.ny + TY - 1) / TY);
  return launch_dep(k2t::resid_restrict_tile<TY>, grid, dim3(k2t::NT), G::SMEM_BYTES, st, tx, tmu, trho, a);
}
}  // namespace

cudaError_t launch_resid_restrict_tile(const Grid<float>& g, const cx<float>* b, const cx<float>* x, cx<float>* bc,
                                       int nxc, int nyc, int ty, int* err, cudaStream_t st) {
  if (nxc * 2 != g.nx || nyc * 2 != g.ny) return cudaErrorInvalidValue;
  if (ty == 24) return launch_resid_restrict_tile_ty<24>(g, b, x, bc, nxc, nyc, err, st);
  if (ty == 8) return launch_resid_restrict_tile_ty<8>(g, b, x, bc, nxc, nyc, err, st);
  if (ty == 4) return launch_resid_restrict_tile_ty<4>(g, b, x, bc, nxc, nyc, err, st);
  return cudaErrorInvalidValue;
}
