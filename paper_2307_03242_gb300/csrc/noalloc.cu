// Allocation-free red-black Vanka smoothing for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is being captured into a
// stream that must not allocate, applications whose memory is fully reserved by their own pool,
// and hosts that link this library only for a fixed-size inner solve. emg_smooth_noalloc gives
// them the smoother of emg_smooth without a handle: the caller passes the material, b and x; the
// only work array -- the ping-pong copy of the displacement components that the red-black
// half-sweeps need -- is a fixed file-scope device array, so nothing is allocated.
#include <cuda.h>  // driver API types only; the two context queries are resolved at run time
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "emg.h"
#include "launch.h"

namespace {

// Ping-pong buffer of the u components: 2 x EMG_NOALLOC_MAX_CELLS complex FP32 values (4 MiB).
// Every GPU that loads the library holds it until the process exits.
__device__ __align__(256) cx<float> g_noalloc_alt[2 * EMG_NOALLOC_MAX_CELLS];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
// Per device: the array's device address and the ID of the context it was looked up in.
void* g_alt_addr[kMaxDevices] = {nullptr};
unsigned long long g_alt_ctx[kMaxDevices] = {0};

// Unique ID of the calling thread's current context (cuCtxGetCurrent + cuCtxGetId, resolved through
// the runtime so the library needs no link-time dependency on the driver library). A context
// created after a device reset has a new ID, so a cached address is never reused across contexts.
// Returns false when the ID cannot be determined; the caller then looks the address up again.
bool current_context_id(unsigned long long* id) {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {  // under g_mutex
    resolved = true;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_current, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      get_current = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      get_id = nullptr;
    cudaGetLastError();
  }
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

emg_status fail(emg_status s, const std::string& m) {
  emg_set_last_error(m);  // reported by emg_last_error()
  return s;
}

}  // namespace

extern "C" emg_status emg_smooth_noalloc(const emg_params* p, const float* mu, const float* rho, const float* cp,
                                         const void* b, void* x, int sweeps, void* cuda_stream) {
  if (!p) return fail(EMG_ERR_INVALID, "params is NULL");
  // the checks emg_create makes of one level (h, omega, gamma, alpha, beta, level_alpha, abl_cells, ...)
  std::string why;
  const emg_status ps = emg_validate_level_params(p, &why);
  if (ps != EMG_OK) return fail(ps, why);
  if (!std::isfinite(p->damping[0]) || !std::isfinite(p->abl_gamma_max))
    return fail(EMG_ERR_INVALID, "non-finite damping[0] or abl_gamma_max");
  if (!mu || !rho || !cp || !b || !x) return fail(EMG_ERR_INVALID, "NULL argument");
  if (p->dim != 2) return fail(EMG_ERR_INVALID, "emg_smooth_noalloc supports dim = 2 only");
  if (p->cycle_precision != 32) return fail(EMG_ERR_INVALID, "emg_smooth_noalloc works on FP32 cycle vectors");
  if (sweeps < 0) return fail(EMG_ERR_INVALID, "sweeps < 0");
  if (p->n[0] < 2 || p->n[1] < 2) return fail(EMG_ERR_INVALID, "n must be >= 2");
  const long long cells = (long long)p->n[0] * p->n[1];
  if (cells > EMG_NOALLOC_MAX_CELLS)
    return fail(EMG_ERR_INVALID, "grid has " + std::to_string(cells) + " cells; emg_smooth_noalloc is limited to " +
                                     std::to_string(EMG_NOALLOC_MAX_CELLS));
  if ((reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(x)) % 16)
    return fail(EMG_ERR_INVALID, "b and x must be 16-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(EMG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(EMG_ERR_INVALID, "device index out of range");
  void* alt = nullptr;
  {
    // First call on a device (or in a new context of it, e.g. after cudaDeviceReset): look up the
    // device address of the file-scope array (the host-side symbol is only a stand-in and must not
    // be passed to a kernel).
    std::lock_guard<std::mutex> lock(g_mutex);
    unsigned long long ctx = 0;
    const bool known = current_context_id(&ctx);
    if (!g_alt_addr[dev] || !known || g_alt_ctx[dev] != ctx) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_alt);
      if (e != cudaSuccess) return fail(EMG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      // the lookup makes the device's primary context current if no context was yet
      g_alt_addr[dev] = current_context_id(&ctx) ? ptr : nullptr;
      g_alt_ctx[dev] = ctx;
      alt = ptr;
    } else {
      alt = g_alt_addr[dev];
    }
  }
  // Level-0 grid of the hierarchy the parameters describe (same coefficients as emg_smooth).
  Grid<float> g;
  g.nx = p->n[0];
  g.ny = p->n[1];
  g.nz = 1;
  g.h = (float)p->h;
  g.ih = (float)(1.0 / p->h);
  g.beta = (float)p->beta;
  g.sm = (float)((1.0 - p->beta) / 4.0);
  g.w2 = (float)(p->omega * p->omega);
  const double a0 = p->level_alpha[0] > 0.0 ? p->level_alpha[0] : p->alpha;
  g.att = (float)(p->gamma + a0);
  g.ablL = (float)(p->abl_cells > 0 ? p->abl_cells * p->h : 0.0);
  g.ablG = (float)p->abl_gamma_max;
  g.Lx = (float)(p->n[0] * p->h);
  g.Ly = (float)(p->n[1] * p->h);
  g.Lz = 0.f;
  g.mu = mu;
  g.rho = rho;
  g.cp = cp;
  g.abl_tab[0] = g.abl_tab[1] = g.abl_tab[2] = nullptr;  // profile evaluated in the kernel
  g.economic = p->smoother == EMG_VANKA_ECONOMIC ? 1 : 0;
  double w = p->damping[0];
  if (!(w > 0.0)) w = p->levels <= 2 ? 0.55 : p->levels == 3 ? 0.35 : p->levels == 4 ? 0.25 : 0.2;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t N = (size_t)cells;
  cx<float>* xv = (cx<float>*)x;
  cx<float>* av = (cx<float>*)alt;
  for (int s = 0; s < sweeps; ++s) {
    // colour 0 writes every face of the scratch copy, so nothing in it has to start at zero
    launch_vanka2<float>(g, (const cx<float>*)b, xv, av, xv + 2 * N, 0, (float)w, 0, st);
    launch_vanka2<float>(g, (const cx<float>*)b, av, xv, xv + 2 * N, 1, (float)w, 0, st);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(EMG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return EMG_OK;
}
