// Host side of the emg library: hierarchy setup, V-cycle recursion, FGMRES outer solve, C ABI.
//
// Paper: Yovel & Treister, arXiv 2307.03242. The V-cycle is Algorithm 1 applied recursively with
// one recursive call (Section 2.2) on the shifted operator H_s (Eq. 2.9: alpha added to the
// attenuation), re-discretised on every level (Remark 2.1, Section 3.2). The outer solver is
// right-preconditioned restarted flexible GMRES (Sections 3.2, 5) in FP64; the cycle runs in the
// precision chosen at creation (FP32 for the mixed-precision solve of Section 5.3).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <memory>
#include <type_traits>
#include <cstring>
#include <string>
#include <vector>
#include <cstdlib>
#include <atomic>
#include <map>
#include <thread>
#include <mutex>
#include <tuple>

#include <nvtx3/nvToolsExt.h>  // header-only; inert unless a profiler is attached

#include "emg.h"
#include "launch.h"
#include "ff2_setup.h"
#include "ff3_setup.h"
#include "stencil2d.cuh"
#include "stencil3d.cuh"
#include "krylov_ff.cuh"
#include "kcycle_kernels.cuh"
#include "vector_kernels.cuh"

namespace {

thread_local std::string g_err;

struct EmgError {
  emg_status s;
  std::string msg;
};

[[noreturn]] void raise(emg_status s, const std::string& m) { throw EmgError{s, m}; }

#define CK(x)                                                                                   \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) raise(EMG_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define CKL() CK(cudaGetLastError())
#define LAUNCHED(c) ((c).launches++)

// Device buffer owned by the handle.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t nbytes) {
    release();
    if (nbytes == 0) return;
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      raise(EMG_ERR_NOMEM, "cudaMalloc(" + std::to_string(nbytes) + " bytes): " + cudaGetErrorString(e));
    }
    bytes = nbytes;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

struct Level {
  int n[3] = {1, 1, 1};
  double h = 1.0;
  size_t ncell = 0;
  double w = 0.5;                         // Vanka damping on this level
  std::vector<double> lam_h, mu_h, rho_h;  // host FP64 material (setup, dense coarse assembly)
  DBuf mu, rho, cp;                        // device material in the cycle precision
  DBuf b, x, alt;                          // cycle vectors: b, x hold dim+1 components, alt dim
  DBuf abl_tab[3];                         // absorbing-layer attenuation per axis (cycle precision)
  int zlo[3] = {1, 1, 1}, zhi[3] = {0, 0, 0};  // lattice range where that attenuation is zero
  DBuf kz1, kz2, kq1, kq2, kr2, kpart, kcoef;  // K-cycle work vectors (levels 1 .. L-2)
  int path = EMG_SWEEP_HALF;  // how the level's sweeps run (EMG_SWEEP_*)
  double tuned_us = 0.0;      // measured time of one smoothing call when the path was timed
};

}  // namespace

struct emg_ctx {
  emg_params prm{};
  int dim = 2, L = 1, prec = 32, sms = 148;
  int dev = 0;  // the device the handle was created on
  cudaStream_t st = nullptr;
  std::vector<Level> lv;
  DBuf mu64, rho64, cp64;  // finest material in FP64 for the outer operator
  DBuf ff_mu, ff_mun, ff_cp, ff_m1, ff_m2;  // 2D: FP64 coefficients as float-float pairs
  DBuf ff3_edge[3], ff3_m[3];              // 3D: edge mu per orientation, face masses
  DBuf cinv;               // dense inverse of the coarsest operator (cycle precision)
  // hybrid Kaczmarz-GMRES coarsest solve (EMG_COARSE_KACZMARZ): Schur rows, 1/||row||^2, Schur
  // vectors, the boxes' private copies, reduction partials, grid barrier, statistics
  DBuf kz_coef, kz_n2, kz_f, kz_u, kz_w, kz_V, kz_Z, kz_copies, kz_part, kz_bar, kz_stats;
  kz::Boxes kz_B{};
  KzLaunch kz_launch{};
  DBuf rscr;               // the fine residual between the residual and restriction kernels
  DBuf dev_err;            // device status word of bounded waits (bit 0: a tile load timed out)
  int cn = 0;
  // Krylov workspace
  int km = 0;
  DBuf V, Z, part, red, wk64, hb, hx;
  double* hred = nullptr;  // pinned
  size_t hb_bytes = 0;
  // instrumentation
  struct Rec { int cls; cudaEvent_t a, b; double bytes; };
  bool prof = false;
  bool prof_coarse = false;  // also time the kernels of the levels below the finest (EMG_K_COARSE)
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  double pms[EMG_K_COUNT] = {0};
  int64_t pn[EMG_K_COUNT] = {0};
  double pbytes[EMG_K_COUNT] = {0};
  int64_t launches = 0;  // every kernel launch, any level
  // The preconditioner cycle as CUDA graphs, one per (right-hand side, output) pair: the cycle's
  // launch sequence depends only on the parameters, so it is captured once and replayed, one
  // graph launch instead of ~50-170 kernel launches per FGMRES iteration.
  struct CycleGraph {
    const void* b;
    void* z;
    int timed;                  // captured with the instrumentation's event pairs as graph nodes
                                // (1: finest level, 2: every level; 0: none)
    int uses;                   // eager runs before capture (the first one warms lazy set-up)
    cudaGraphExec_t exec;
    int64_t kernels;            // kernel launches one replay stands for
    std::vector<Rec> recs;      // timed: the event pairs every replay records
    bool unread;                // timed: the last replay's events have not been read yet
  };
  std::vector<CycleGraph> graphs;
  bool graphs_ok = true;       // false once a capture failed: the cycle then runs eagerly
  std::vector<Rec>* capture_recs = nullptr;  // during a timed capture: where its event pairs go

  size_t nvec() const { return (size_t)(dim + 1) * lv[0].ncell; }
  ~emg_ctx() {
    for (auto& g : graphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      for (auto& r : g.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    }
    if (hred) cudaFreeHost(hred);
    for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

namespace {

double default_damping(int levels) {
  switch (levels) {
    case 1: case 2: return 0.55;
    case 3: return 0.35;
    case 4: return 0.25;
    default: return 0.2;
  }
}

double level_alpha(const emg_params& p, int l) { return p.level_alpha[l] > 0.0 ? p.level_alpha[l] : p.alpha; }

// EMG_COARSE_KACZMARZ settings with the paper's values for the zero fields (Sec. 5.3).
struct KzCfg {
  int box[3];
  int steps, restart, max_steps;
  double damping, tol;
};
KzCfg kz_cfg(const emg_params& p) {
  KzCfg k;
  for (int a = 0; a < 3; ++a) k.box[a] = p.kaczmarz_box[a];  // all zero: chosen at set-up
  k.steps = p.kaczmarz_steps > 0 ? p.kaczmarz_steps : 10;
  k.restart = p.coarse_restart > 0 ? p.coarse_restart : 5;
  k.max_steps = p.kaczmarz_max > 0 ? p.kaczmarz_max : 250;
  k.damping = p.kaczmarz_damping > 0.0 ? p.kaczmarz_damping : 0.8;
  k.tol = p.coarse_tol > 0.0 ? p.coarse_tol : 0.1;
  return k;
}

// Half-warps per block whose box region and row ring fit beside the region-layout table in the
// Kaczmarz kernel's 200 KB of shared memory (an even number; < 2: the box does not fit).
int kz_region_halfwarps(int dim, const int n[3], const int box[3], size_t cb) {
  const kz::Boxes B = kz::make_boxes(dim, n, box);
  const size_t per_hw = (size_t)kz::half_warp_smem(B, dim) * cb;
  const size_t table = ((size_t)(B.RS + 2 * dim * (dim == 3 ? kz::Shape<3>::SL : kz::Shape<2>::SL) * kz::HW) * 4 + 15) / 16 * 16;
  if (table >= 200 * 1024) return 0;
  int w = (int)((200 * 1024 - table) / per_hw);
  if (w > kz::NT / kz::HW) w = kz::NT / kz::HW;
  return w & ~1;
}

// The automatic box: the smallest cube of 2, 4, ... cells whose boxes the resident
// half-warps (one block per SM) can all sweep at once, so that a Kaczmarz step's sequential part
// is one box's rows; the largest that fits if none does.
void kz_auto_box(int dim, const int n[3], int sms, size_t cb, int box[3]) {
  int pick = 0;
  // from 2 cells: boxes of one cell need about twice the steps (3D) or stall (2D), which costs
  // more than their shorter sweeps save
  for (int b = 2; b <= 64; b *= 2) {
    const int bb[3] = {b, b, b};
    const int hw = kz_region_halfwarps(dim, n, bb, cb);
    if (hw < 2) break;
    pick = b;
    if ((long long)kz::make_boxes(dim, n, bb).nboxes <= (long long)sms * hw) break;
  }
  if (pick == 0) pick = 1;
  for (int a = 0; a < 3; ++a) box[a] = pick;
}

template <typename T>
Grid<T> make_grid(const emg_ctx& c, int l, bool shifted, const void* mu, const void* rho, const void* cp) {
  const Level& L = c.lv[l];
  const emg_params& p = c.prm;
  Grid<T> g;
  g.nx = L.n[0];
  g.ny = L.n[1];
  g.nz = c.dim == 3 ? L.n[2] : 1;
  g.h = (T)L.h;
  g.ih = (T)(1.0 / L.h);
  g.beta = (T)p.beta;
  g.sm = (T)((1.0 - p.beta) / (2.0 * c.dim));
  g.w2 = (T)(p.omega * p.omega);
  g.att = (T)(p.gamma + (shifted ? level_alpha(p, l) : 0.0));
  g.ablL = (T)(p.abl_cells > 0 ? p.abl_cells * p.h : 0.0);
  g.ablG = (T)p.abl_gamma_max;
  g.Lx = (T)(p.n[0] * p.h);
  g.Ly = (T)(p.n[1] * p.h);
  g.Lz = (T)(c.dim == 3 ? p.n[2] * p.h : 0.0);
  g.mu = (const T*)mu;
  g.rho = (const T*)rho;
  g.cp = (const T*)cp;
  g.abl_tab[0] = g.abl_tab[1] = g.abl_tab[2] = nullptr;
  for (int a = 0; a < 3; ++a) { g.zlo[a] = 1; g.zhi[a] = 0; }
  g.economic = p.smoother == EMG_VANKA_ECONOMIC ? 1 : 0;
  return g;
}

template <typename T> Grid<T> level_grid(const emg_ctx& c, int l) {
  const Level& L = c.lv[l];
  Grid<T> g = make_grid<T>(c, l, true, L.mu.p, L.rho.p, L.cp.p);
  for (int a = 0; a < c.dim; ++a) {
    g.abl_tab[a] = L.abl_tab[a].as<const T>();
    g.zlo[a] = L.zlo[a];
    g.zhi[a] = L.zhi[a];
  }
  return g;
}

// ---------------------------------------------------------------- instrumentation
// An NVTX range over each ABI call (emg_create, emg_solve, emg_vcycle, ...), so that profilers
// can select the kernels of one kind of call (ncu --nvtx --nvtx-include "emg_solve/").
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct ProfScope {
  emg_ctx& c;
  int cls;
  double bytes;
  bool on;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(emg_ctx& c_, int cls_, int level, double bytes_) : c(c_), cls(cls_), bytes(bytes_) {
    on = c.prof && (level == 0 || c.prof_coarse);
    if (level > 0) cls = EMG_K_COARSE;
    if (!on) return;
    a = take();
    b = take();
    CK(record(a));
  }
  // In a stream capture a plain event record only expresses a dependency inside the graph; an
  // external record becomes a node that records the event each time the graph runs.
  cudaError_t record(cudaEvent_t e) {
    return c.capture_recs ? cudaEventRecordWithFlags(e, c.st, cudaEventRecordExternal) : cudaEventRecord(e, c.st);
  }
  cudaEvent_t take() {
    if (!c.pool.empty()) { cudaEvent_t e = c.pool.back(); c.pool.pop_back(); return e; }
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    return e;
  }
  ~ProfScope() {
    if (!on) return;
    record(b);
    (c.capture_recs ? *c.capture_recs : c.recs).push_back({cls, a, b, bytes});
  }
};

// Adds the times of a timed graph's last replay (complete: the caller has synchronised since).
void harvest(emg_ctx& c, emg_ctx::CycleGraph& g) {
  if (!g.unread) return;
  for (auto& r : g.recs) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    c.pms[r.cls] += ms;
    c.pn[r.cls] += 1;
    c.pbytes[r.cls] += r.bytes;
  }
  g.unread = false;
}

void prof_flush(emg_ctx& c) {
  bool any = !c.recs.empty();
  for (auto& g : c.graphs) any = any || g.unread;
  if (!any) return;
  CK(cudaStreamSynchronize(c.st));
  for (auto& g : c.graphs) harvest(c, g);
  for (auto& r : c.recs) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    c.pms[r.cls] += ms;
    c.pn[r.cls] += 1;
    c.pbytes[r.cls] += r.bytes;
    c.pool.push_back(r.a);
    c.pool.push_back(r.b);
  }
  c.recs.clear();
}

// ---------------------------------------------------------------- launch helpers
int vec_blocks(const emg_ctx& c, size_t n) {
  size_t b = (n + 255) / 256;
  return (int)std::max<size_t>(1, std::min<size_t>(b, (size_t)c.sms * 8));
}

// Algorithmic bytes (minimum traffic) of the fine-level kernels, per cell, used by the
// instrumentation: a half-sweep reads x, b on the colour's DOFs, 3 material reals and writes
// every face plus the colour's pressures.
template <typename T> double half_sweep_bytes(const emg_ctx& c) {
  const double cw = 2.0 * sizeof(T), rw = sizeof(T);
  const int d = c.dim;
  return (double)c.lv[0].ncell * ((d + 1) * cw + (d + 0.5) * cw + 3 * rw + (d + 0.5) * cw);
}

// ---------------------------------------------------------------- cycle pieces
template <typename T>
void launch_apply(emg_ctx& c, const Grid<T>& g, const void* x, bool x32, const cx<T>* b, T bscale, cx<T>* y) {
  if (x32) {
    if constexpr (std::is_same<T, double>::value) {
      if (c.dim == 2) launch_apply2<double, float>(g, (const cx<float>*)x, b, bscale, y, c.st);
      else launch_apply3<double, float>(g, (const cx<float>*)x, b, bscale, y, c.st);
    } else {
      raise(EMG_ERR_INVALID, "FP32 input requires the FP64 operator");
    }
  } else {
    if (c.dim == 2) launch_apply2<T, T>(g, (const cx<T>*)x, b, bscale, y, c.st);
    else launch_apply3<T, T>(g, (const cx<T>*)x, b, bscale, y, c.st);
  }
  CKL();
  LAUNCHED(c);
}

// 2D levels below the finest with at most this many cells per colour run all their sweeps in one
// cooperative launch (measured on the 2048^2 hierarchy: 128^2 to 512^2 gain 15-45 %, 1024^2 loses).
constexpr long long kCoopMaxColourCells = 1 << 17;

// Whether level l's sweeps run as one-pass tiled sweeps (k2t::sweep_tile).
bool tiled_level(const emg_ctx& c, int l) {
  const int p = c.lv[l].path;
  return p == EMG_SWEEP_TILE24 || p == EMG_SWEEP_TILE8 || p == EMG_SWEEP_TILE4;
}

// Tile height of a one-pass tiled path.
int tile_height(int path) { return path == EMG_SWEEP_TILE24 ? 24 : (path == EMG_SWEEP_TILE8 ? 8 : 4); }

// Whether a sweep path can run level l.
bool path_ok(const emg_ctx& c, int l, int path) {
  const Level& L = c.lv[l];
  switch (path) {
    case EMG_SWEEP_HALF: return true;
    case EMG_SWEEP_COOP: return c.dim == 2;
    case EMG_SWEEP_TILE24:
    case EMG_SWEEP_TILE8:
    case EMG_SWEEP_TILE4: return c.dim == 2 && c.prec == 32 && L.n[0] % 4 == 0 && L.n[0] >= 4;
    default: return false;
  }
}

// The path without timing: the cooperative launch for the 2D levels below the finest with few
// cells, one launch per colour otherwise.
int default_path(const emg_ctx& c, int l) {
  const Level& L = c.lv[l];
  if (c.dim == 2 && l > 0 && (long long)((L.n[0] + 1) / 2) * L.n[1] <= kCoopMaxColourCells) return EMG_SWEEP_COOP;
  return EMG_SWEEP_HALF;
}

// Algorithmic bytes of one one-pass sweep of level l: read x (unless it is zero), b and the three
// material reals, write x.
double tiled_sweep_bytes(const emg_ctx& c, int l, bool zero_in) {
  const double S = (c.dim + 1) * 8.0;
  return (double)c.lv[l].ncell * ((zero_in ? 2.0 : 3.0) * S + 3 * 4.0);
}

// `sweeps` red-black sweeps on level l starting from the state in `cur`; `other` is a second
// vector of (d+1) n values. Returns the buffer that holds the result: one-pass tiled sweeps
// cannot work in place, so they alternate between cur and other; every other path works in
// place in cur and uses other as its ping-pong copy of the displacements.
template <typename T>
void prolong_correct(emg_ctx& c, int l, const cx<T>* e, cx<T>* x);

// e: a coarse correction (level l+1) to add, x += P e, before the first sweep; the one-pass
// sweep adds it while loading its tiles (prolongation + correction fused into the sweep).
template <typename T>
cx<T>* smooth2(emg_ctx& c, int l, const cx<T>* b, cx<T>* cur, cx<T>* other, int sweeps, double w, bool zero_first,
               const cx<T>* e = nullptr) {
  Level& L = c.lv[l];
  Grid<T> g = level_grid<T>(c, l);
  const size_t N = L.ncell;
  if (e && (sweeps == 0 || zero_first || !std::is_same<T, float>::value || !tiled_level(c, l))) {
    prolong_correct<T>(c, l, e, cur);
    e = nullptr;
  }
  if (sweeps == 0) {
    if (zero_first) CK(cudaMemsetAsync(cur, 0, (c.dim + 1) * N * sizeof(cx<T>), c.st));
    return cur;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (tiled_level(c, l)) {
      const int ty = tile_height(L.path);
      if (!sweep_tile_fits(g, b, cur, other)) raise(EMG_ERR_INVALID, "sweep buffers are not 16-byte aligned");
      for (int s = 0; s < sweeps; ++s) {
        const bool zin = zero_first && s == 0;
        const cx<float>* es = s == 0 ? (const cx<float>*)e : nullptr;
        const Level* C = es ? &c.lv[l + 1] : nullptr;
        {
          // with a correction, the sweep also reads e (3 coarse values per 4 fine cells)
          ProfScope ps(c, EMG_K_SMOOTH, l, tiled_sweep_bytes(c, l, zin) + (es ? C->ncell * 3 * 8.0 : 0.0));
          CK(launch_sweep_tile(g, b, cur, other, (float)w, zin ? 1 : 0, es, C ? C->n[0] : 0, C ? C->n[1] : 0, ty,
                               c.dev_err.as<int>(), c.st));
          LAUNCHED(c);
        }
        std::swap(cur, other);
      }
      return cur;
    }
  }
  cx<T>* alt = other;
  cx<T>* x = cur;
  cx<T>* p = x + (size_t)c.dim * N;
  const double bytes = l == 0 ? half_sweep_bytes<T>(c) : 0.0;
  if (c.dim == 2 && L.path == EMG_SWEEP_COOP) {
    ProfScope ps(c, EMG_K_SMOOTH, l, 0.0);
    CK(launch_sweeps_coop2<T>(g, b, x, alt, sweeps, (T)w, zero_first ? 1 : 0, c.st));
    LAUNCHED(c);
    return cur;
  }
  for (int s = 0; s < sweeps; ++s) {
    for (int colour = 0; colour < 2; ++colour) {
      const cx<T>* uin = colour == 0 ? x : alt;
      cx<T>* uout = colour == 0 ? alt : x;
      const int zin = (zero_first && s == 0 && colour == 0) ? 1 : 0;
      ProfScope ps(c, EMG_K_SMOOTH, l, bytes);
      if (c.dim == 2) launch_vanka2<T>(g, b, uin, uout, p, colour, (T)w, zin, c.st);
      else launch_vanka3<T>(g, b, uin, uout, p, colour, (T)w, zin, c.st);
      CKL();
      LAUNCHED(c);
    }
  }
  return cur;
}

// Sweeps with the result in x (the level's alternate vector serves as the second buffer).
template <typename T>
void smooth(emg_ctx& c, int l, const cx<T>* b, cx<T>* x, int sweeps, double w, bool zero_first) {
  cx<T>* alt = c.lv[l].alt.as<cx<T>>();
  cx<T>* r = smooth2<T>(c, l, b, x, alt, sweeps, w, zero_first);
  if (r != x) CK(cudaMemcpyAsync(x, r, (c.dim + 1) * c.lv[l].ncell * sizeof(cx<T>), cudaMemcpyDeviceToDevice, c.st));
}

// ---------------------------------------------------------------- sweep-path autotuner
// A level's smoothing call (its sweep count) is timed on each path that can run it, on the level's
// own buffers (right after set-up, outside any stream capture), and the fastest is kept. Choices
// are cached per device, grid, sweep count and smoother for the life of the process, so handles
// of the same sizes (a batch of instances) tune once.
struct TuneKey {
  int dev, nx, ny, sweeps, economic;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, nx, ny, sweeps, economic) < std::tie(o.dev, o.nx, o.ny, o.sweeps, o.economic);
  }
};
std::mutex g_tune_mutex;
std::map<TuneKey, std::pair<int, double>> g_tune_cache;

// Mean time of one smoothing call of `sweeps` sweeps on level l along its current path, in us.
double time_smoothing(emg_ctx& c, int l, int sweeps, double w) {
  Level& L = c.lv[l];
  cx<float>* b = L.b.as<cx<float>>();
  cx<float>* cur = L.x.as<cx<float>>();
  cx<float>* oth = L.alt.as<cx<float>>();
  auto call = [&]() {
    cx<float>* r = smooth2<float>(c, l, b, cur, oth, sweeps, w, false);
    if (r != cur) std::swap(cur, oth);
  };
  call();
  call();
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  constexpr int reps = 5, trials = 3;
  double best = 0.0;
  for (int t = 0; t < trials; ++t) {  // the fastest of three trials: a trial disturbed by other work is dropped
    CK(cudaEventRecord(e0, c.st));
    for (int r = 0; r < reps; ++r) call();
    CK(cudaEventRecord(e1, c.st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    const double us = 1e3 * ms / reps;
    if (t == 0 || us < best) best = us;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

void choose_sweep_paths(emg_ctx& c) {
  for (int l = 0; l < c.L; ++l) {
    Level& L = c.lv[l];
    L.path = default_path(c, l);
    L.tuned_us = 0.0;
    const bool coarsest = l == c.L - 1;
    if (c.dim != 2 || c.prec != 32 || (coarsest && c.prm.coarse_solver != EMG_COARSE_SMOOTH)) continue;
    const int forced = c.prm.sweep_path;
    if (forced != EMG_SWEEP_AUTO) {
      if (path_ok(c, l, forced)) L.path = forced;
      continue;
    }
    const int sweeps = coarsest ? c.prm.coarse_sweeps : std::max(1, std::max(c.prm.nu_pre, c.prm.nu_post));
    const double w = coarsest ? c.prm.coarse_damping : L.w;
    const TuneKey key{c.dev, L.n[0], L.n[1], sweeps, c.prm.smoother};
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        L.path = it->second.first;
        L.tuned_us = it->second.second;
        continue;
      }
    }
    // candidates in a fixed order of preference; a later one replaces the current choice only
    // when it is at least 5 % faster, so that near-ties (timing noise) resolve the same way in
    // every process
    const long long colour_cells = (long long)((L.n[0] + 1) / 2) * L.n[1];
    std::vector<int> cand;
    for (int p : {EMG_SWEEP_TILE24, EMG_SWEEP_TILE8, EMG_SWEEP_TILE4})
      if (path_ok(c, l, p)) cand.push_back(p);
    if (colour_cells <= (1 << 19)) cand.push_back(EMG_SWEEP_COOP);
    cand.push_back(EMG_SWEEP_HALF);
    int best = L.path;
    double best_us = 0.0;
    for (int p : cand) {
      L.path = p;
      const double us = time_smoothing(c, l, sweeps, w);
      if (best_us == 0.0 || us < 0.95 * best_us) {
        best = p;
        best_us = us;
      }
    }
    L.path = best;
    L.tuned_us = best_us;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = {best, best_us};
  }
  // the timing runs swept zero vectors; leave the level buffers as set-up left them
  for (auto& L : c.lv) {
    CK(cudaMemsetAsync(L.x.p, 0, L.x.bytes, c.st));
    CK(cudaMemsetAsync(L.alt.p, 0, L.alt.bytes, c.st));
  }
  CK(cudaStreamSynchronize(c.st));
  c.launches = 0;
}

template <typename T>
void residual_restrict(emg_ctx& c, int l, const cx<T>* b, const cx<T>* x, cx<T>* bc) {
  Level& L = c.lv[l];
  Level& C = c.lv[l + 1];
  Grid<T> g = level_grid<T>(c, l);
  const double cw = 2.0 * sizeof(T);
  ProfScope ps(c, EMG_K_RESTRICT, l, (double)L.ncell * (2 * (c.dim + 1) * cw + 3 * sizeof(T)) + C.ncell * (c.dim + 1) * cw);
  if constexpr (std::is_same<T, float>::value) {
    // 2D FP32 levels whose rows meet the tile kernel's alignment rule: one pass, no fine residual
    // in memory; the tallest tiles (60 x 24, 60 x 8, 60 x 4) that still fill the GPU twice over
    if (c.dim == 2 && path_ok(c, l, EMG_SWEEP_TILE24) &&
        !(((uintptr_t)b | (uintptr_t)x | (uintptr_t)bc) % 16)) {
      const long long cols = (L.n[0] + 59) / 60;
      const int ty = cols * ((L.n[1] + 23) / 24) >= 2LL * c.sms ? 24 : (cols * ((L.n[1] + 7) / 8) >= 2LL * c.sms ? 8 : 4);
      CK(launch_resid_restrict_tile(g, b, x, bc, C.n[0], C.n[1], ty, c.dev_err.as<int>(), c.st));
      LAUNCHED(c);
      return;
    }
  }
  if (c.dim == 2) launch_restrict2<T>(g, b, x, bc, C.n, c.rscr.as<cx<T>>(), c.st);
  else launch_restrict3<T>(g, b, x, bc, C.n, c.rscr.as<cx<T>>(), c.st);
  CKL();
  LAUNCHED(c);  // residual, then restriction
  LAUNCHED(c);
}

template <typename T>
void prolong_correct(emg_ctx& c, int l, const cx<T>* e, cx<T>* x) {
  Level& L = c.lv[l];
  Level& C = c.lv[l + 1];
  const double cw = 2.0 * sizeof(T);
  ProfScope ps(c, EMG_K_PROLONG, l, (double)L.ncell * 2 * (c.dim + 1) * cw + C.ncell * (c.dim + 1) * cw);
  if (c.dim == 2) launch_prolong2<T>(e, x, L.n, C.n, c.st);
  else launch_prolong3<T>(e, x, L.n, C.n, c.st);
  CKL();
  LAUNCHED(c);
}

template <typename T>
kz::Args<T> kz_args(emg_ctx& c, const cx<T>* b, cx<T>* x);

template <typename T>
void coarse_solve(emg_ctx& c, const cx<T>* b, cx<T>* x) {
  const int l = c.L - 1;
  if (c.prm.coarse_solver == EMG_COARSE_DENSE) {
    ProfScope ps(c, EMG_K_SMOOTH, l, 0.0);
    const int n = c.cn;
    launch_dep(kv::dense_gemv<T>, dim3((n + 7) / 8), dim3(256), 0, c.st, c.cinv.as<cx<T>>(), b, x, n);
    CKL();
  LAUNCHED(c);
  } else if (c.prm.coarse_solver == EMG_COARSE_KACZMARZ) {
    ProfScope ps(c, EMG_K_SMOOTH, l, 0.0);
    CK(launch_kz_solve<T>(kz_args<T>(c, b, x), c.dim, c.kz_launch, c.st));
    LAUNCHED(c);
  } else {
    smooth<T>(c, l, b, x, c.prm.coarse_sweeps, c.prm.coarse_damping, true);
  }
}

template <typename T>
void vcycle(emg_ctx& c, int l, const cx<T>* b, cx<T>* x, bool zero_guess);

// coef (device) = <a, b> / <a, a> on level m
template <typename T>
void kcoef(emg_ctx& c, int m, const cx<T>* a, const cx<T>* b, double* coef) {
  Level& M = c.lv[m];
  const size_t n = (c.dim + 1) * M.ncell;
  const int nblk = vec_blocks(c, n);
  launch_dep(kc::dot_parts<T>, dim3(nblk), dim3(kc::RT), 0, c.st, a, b, n, M.kpart.as<double>());
  CKL();
  LAUNCHED(c);
  launch_dep(kc::finalize_coef, dim3(1), dim3(kv::RP), 0, c.st, M.kpart.as<double>(), nblk, coef);
  CKL();
  LAUNCHED(c);
}

template <typename T>
void kaxpy(emg_ctx& c, size_t n, cx<T>* y, const cx<T>* x0, const cx<T>* x, const double* coef, T sgn) {
  launch_dep(kc::axpy_coef<T>, dim3(vec_blocks(c, n)), dim3(256), 0, c.st, y, x0, x, coef, sgn, n);
  CKL();
  LAUNCHED(c);
}

// K-cycle coarse correction on level m (1 <= m < L-1): two GCR steps for H_s e = r, each
// preconditioned by one recursive cycle on level m; e is written to e_out.
template <typename T>
void kcycle_correction(emg_ctx& c, int m, const cx<T>* r, cx<T>* e_out) {
  Level& M = c.lv[m];
  const size_t n = (c.dim + 1) * M.ncell;
  cx<T>* z1 = M.kz1.as<cx<T>>();
  cx<T>* z2 = M.kz2.as<cx<T>>();
  cx<T>* q1 = M.kq1.as<cx<T>>();
  cx<T>* q2 = M.kq2.as<cx<T>>();
  cx<T>* r2 = M.kr2.as<cx<T>>();
  double* cf = M.kcoef.as<double>();  // cf[0..1] a1, cf[2..3] beta, cf[4..5] a2
  Grid<T> g = level_grid<T>(c, m);
  vcycle<T>(c, m, r, z1, true);
  launch_apply<T>(c, g, z1, false, nullptr, T(0), q1);
  LAUNCHED(c);
  kcoef<T>(c, m, q1, r, cf);
  kaxpy<T>(c, n, r2, r, q1, cf, T(-1));      // r2 = r - a1 q1
  kaxpy<T>(c, n, e_out, nullptr, z1, cf, T(1));  // e = a1 z1
  vcycle<T>(c, m, r2, z2, true);
  launch_apply<T>(c, g, z2, false, nullptr, T(0), q2);
  LAUNCHED(c);
  kcoef<T>(c, m, q1, q2, cf + 2);
  kaxpy<T>(c, n, q2, q2, q1, cf + 2, T(-1));  // q2 -= beta q1
  kaxpy<T>(c, n, z2, z2, z1, cf + 2, T(-1));  // z2 -= beta z1
  kcoef<T>(c, m, q2, r2, cf + 4);
  kaxpy<T>(c, n, e_out, e_out, z2, cf + 4, T(1));  // e += a2 z2
}

template <typename T>
void vcycle(emg_ctx& c, int l, const cx<T>* b, cx<T>* x, bool zero_guess) {
  if (l == c.L - 1) {
    coarse_solve<T>(c, b, x);
    return;
  }
  Level& L = c.lv[l];
  Level& C = c.lv[l + 1];
  // the level's state moves between x and the level's alternate vector (one-pass sweeps do not
  // work in place); it ends in x
  cx<T>* alt = L.alt.as<cx<T>>();
  cx<T>* cur = smooth2<T>(c, l, b, x, alt, c.prm.nu_pre, L.w, zero_guess);
  residual_restrict<T>(c, l, b, cur, C.b.as<cx<T>>());
  if (c.prm.cycle_type == EMG_CYCLE_K && l + 1 < c.L - 1) {
    kcycle_correction<T>(c, l + 1, C.b.as<cx<T>>(), C.x.as<cx<T>>());
  } else {
    vcycle<T>(c, l + 1, C.b.as<cx<T>>(), C.x.as<cx<T>>(), true);
    if (c.prm.cycle_type == EMG_CYCLE_W && l + 1 < c.L - 1) vcycle<T>(c, l + 1, C.b.as<cx<T>>(), C.x.as<cx<T>>(), false);
  }
  // prolongation + correction, fused into the first post-sweep where the sweep is one pass
  cur = smooth2<T>(c, l, b, cur, cur == x ? alt : x, c.prm.nu_post, L.w, false, C.x.as<const cx<T>>());
  if (cur != x) CK(cudaMemcpyAsync(x, cur, (c.dim + 1) * L.ncell * sizeof(cx<T>), cudaMemcpyDeviceToDevice, c.st));
}

// ---------------------------------------------------------------- host assembly of the coarsest operator
// Column-by-column application of the same stencil functions the kernels use, restricted to the
// neighbourhood of each unit vector; then a Gauss-Jordan inverse with partial pivoting in FP64.
void assemble_dense(const emg_ctx& c, std::vector<std::complex<double>>& A, std::vector<int>& act) {
  const int l = c.L - 1;
  const Level& L = c.lv[l];
  const int d = c.dim;
  std::vector<double> cph(L.ncell);
  for (size_t k = 0; k < L.ncell; ++k) cph[k] = 1.0 / (L.lam_h[k] + L.mu_h[k]);
  Grid<double> g = make_grid<double>(c, l, true, L.mu_h.data(), L.rho_h.data(), cph.data());
  const int nx = L.n[0], ny = L.n[1], nz = d == 3 ? L.n[2] : 1;
  const size_t N = L.ncell, NF = (d + 1) * N;
  act.assign(NF, 1);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t q = ((size_t)k * ny + j) * nx + i;
        if (i == 0) act[q] = 0;
        if (j == 0) act[N + q] = 0;
        if (d == 3 && k == 0) act[2 * N + q] = 0;
      }
  A.assign(NF * NF, 0.0);
  std::vector<cx<double>> x(NF);
  for (size_t col = 0; col < NF; ++col) {
    if (!act[col]) continue;
    std::fill(x.begin(), x.end(), czero<double>());
    x[col] = mkc(1.0, 0.0);
    const size_t q = col % N;
    const int ci = (int)(q % nx), cj = (int)((q / nx) % ny), ck = (int)(q / ((size_t)nx * ny));
    for (int k = std::max(0, ck - 2); k <= std::min(nz - 1, ck + 2); ++k)
      for (int j = std::max(0, cj - 2); j <= std::min(ny - 1, cj + 2); ++j)
        for (int i = std::max(0, ci - 2); i <= std::min(nx - 1, ci + 2); ++i) {
          size_t r = ((size_t)k * ny + j) * nx + i;
          cx<double> y[4];
          if (d == 2) {
            y[0] = i >= 1 ? s2::row_u1(x.data(), x.data() + 2 * N, g, i, j) : czero<double>();
            y[1] = j >= 1 ? s2::row_u2(x.data() + N, x.data() + 2 * N, g, i, j) : czero<double>();
            y[2] = s2::row_p(x.data(), x.data() + N, x.data() + 2 * N, g, i, j);
          } else {
            const cx<double>* u[3] = {x.data(), x.data() + N, x.data() + 2 * N};
            for (int cc = 0; cc < 3; ++cc)
              y[cc] = (cc == 0 ? i : cc == 1 ? j : k) >= 1 ? s3::row_u(cc, u[cc], x.data() + 3 * N, g, i, j, k)
                                                         : czero<double>();
            y[3] = s3::row_p(u, x.data() + 3 * N, g, i, j, k);
          }
          for (int cc = 0; cc <= d; ++cc) {
            size_t row = cc * N + r;
            if (act[row]) A[row * NF + col] = std::complex<double>(y[cc].re, y[cc].im);
          }
        }
  }
}

void invert_dense(std::vector<std::complex<double>>& A, const std::vector<int>& act, std::vector<std::complex<double>>& Ainv) {
  const size_t NF = act.size();
  std::vector<size_t> idx;
  for (size_t i = 0; i < NF; ++i)
    if (act[i]) idx.push_back(i);
  const size_t n = idx.size();
  std::vector<std::complex<double>> M(n * 2 * n, 0.0);
  for (size_t r = 0; r < n; ++r) {
    for (size_t s = 0; s < n; ++s) M[r * 2 * n + s] = A[idx[r] * NF + idx[s]];
    M[r * 2 * n + n + r] = 1.0;
  }
  const size_t W = 2 * n;
  for (size_t k = 0; k < n; ++k) {
    size_t piv = k;
    double best = std::abs(M[k * W + k]);
    for (size_t r = k + 1; r < n; ++r)
      if (std::abs(M[r * W + k]) > best) { best = std::abs(M[r * W + k]); piv = r; }
    if (!(best > 0.0) || !std::isfinite(best)) raise(EMG_ERR_INVALID, "coarsest operator is singular");
    if (piv != k)
      for (size_t s = 0; s < W; ++s) std::swap(M[k * W + s], M[piv * W + s]);
    std::complex<double> ip = 1.0 / M[k * W + k];
    for (size_t s = 0; s < W; ++s) M[k * W + s] *= ip;
    for (size_t r = 0; r < n; ++r) {
      if (r == k) continue;
      std::complex<double> f = M[r * W + k];
      if (f == 0.0) continue;
      std::complex<double>* dst = &M[r * W];
      const std::complex<double>* src = &M[k * W];
      for (size_t s = 0; s < W; ++s) dst[s] -= f * src[s];
    }
  }
  Ainv.assign(NF * NF, 0.0);
  for (size_t r = 0; r < n; ++r)
    for (size_t s = 0; s < n; ++s) Ainv[idx[r] * NF + idx[s]] = M[r * W + n + s];
}

// ---------------------------------------------------------------- setup
template <typename T>
void upload_material(emg_ctx& c, Level& L) {
  std::vector<T> mu(L.ncell), rho(L.ncell), cp(L.ncell);
  for (size_t k = 0; k < L.ncell; ++k) {
    mu[k] = (T)L.mu_h[k];
    rho[k] = (T)L.rho_h[k];
    cp[k] = (T)(1.0 / (L.lam_h[k] + L.mu_h[k]));
  }
  L.mu.alloc(L.ncell * sizeof(T));
  L.rho.alloc(L.ncell * sizeof(T));
  L.cp.alloc(L.ncell * sizeof(T));
  CK(cudaMemcpy(L.mu.p, mu.data(), L.ncell * sizeof(T), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(L.rho.p, rho.data(), L.ncell * sizeof(T), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(L.cp.p, cp.data(), L.ncell * sizeof(T), cudaMemcpyHostToDevice));
}

void coarsen_material(const emg_ctx& c, const Level& F, Level& C) {
  const int d = c.dim;
  C.lam_h.assign(C.ncell, 0.0);
  C.mu_h.assign(C.ncell, 0.0);
  C.rho_h.assign(C.ncell, 0.0);
  const int nz = d == 3 ? C.n[2] : 1;
  const double inv = 1.0 / (d == 3 ? 8.0 : 4.0);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < C.n[1]; ++j)
      for (int i = 0; i < C.n[0]; ++i) {
        double sl = 0, sm = 0, sr = 0;
        for (int c3 = 0; c3 < (d == 3 ? 2 : 1); ++c3)
          for (int c2 = 0; c2 < 2; ++c2)
            for (int c1 = 0; c1 < 2; ++c1) {
              size_t f = ((size_t)(d == 3 ? 2 * k + c3 : 0) * F.n[1] + (2 * j + c2)) * F.n[0] + (2 * i + c1);
              sl += F.lam_h[f];
              sm += F.mu_h[f];
              sr += F.rho_h[f];
            }
        size_t q = ((size_t)k * C.n[1] + j) * C.n[0] + i;
        C.lam_h[q] = sl * inv;
        C.mu_h[q] = sm * inv;
        C.rho_h[q] = sr * inv;
      }
}

df::f2 to_f2(double v) {
  df::f2 r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

// FP64 coefficients of the finest 2D operator as float-float pairs for ff2::apply (ff2_setup.h).
void build_ff2(emg_ctx& c) {
  const Level& F = c.lv[0];
  const emg_params& p = c.prm;
  ff2::HostFF2 o;
  ff2::build_host(o, F.n[0], F.n[1], F.h, F.lam_h.data(), F.mu_h.data(), F.rho_h.data(), p.omega, p.gamma,
                  p.abl_cells > 0 ? p.abl_cells * p.h : 0.0, p.abl_gamma_max, p.n[0] * p.h, p.n[1] * p.h);
  auto up = [&](DBuf& d, const void* src, size_t bytes) {
    d.alloc(bytes);
    CK(cudaMemcpy(d.p, src, bytes, cudaMemcpyHostToDevice));
  };
  up(c.ff_mu, o.mu.data(), o.mu.size() * sizeof(df::f2));
  up(c.ff_cp, o.cp.data(), o.cp.size() * sizeof(df::f2));
  up(c.ff_mun, o.mun.data(), o.mun.size() * sizeof(df::f2));
  up(c.ff_m1, o.m1.data(), o.m1.size() * sizeof(ff2::c2));
  up(c.ff_m2, o.m2.data(), o.m2.size() * sizeof(ff2::c2));
}

// FP64 coefficients of the finest 3D operator as float-float pairs for ff3::apply.
void build_ff3(emg_ctx& c) {
  const Level& F = c.lv[0];
  const emg_params& p = c.prm;
  ff3::HostFF3 o;
  const double L[3] = {p.n[0] * p.h, p.n[1] * p.h, p.n[2] * p.h};
  ff3::build_host(o, F.n[0], F.n[1], F.n[2], F.h, F.lam_h.data(), F.mu_h.data(), F.rho_h.data(), p.omega, p.gamma,
                  p.abl_cells > 0 ? p.abl_cells * p.h : 0.0, p.abl_gamma_max, L);
  auto up = [&](DBuf& d, const void* src, size_t bytes) {
    d.alloc(bytes);
    CK(cudaMemcpy(d.p, src, bytes, cudaMemcpyHostToDevice));
  };
  up(c.ff_mu, o.mu.data(), o.mu.size() * sizeof(df::f2));
  up(c.ff_cp, o.cp.data(), o.cp.size() * sizeof(df::f2));
  for (int r = 0; r < 3; ++r) {
    up(c.ff3_edge[r], o.edge[r].data(), o.edge[r].size() * sizeof(df::f2));
    up(c.ff3_m[r], o.m[r].data(), o.m[r].size() * sizeof(ff2::c2));
  }
}

// Absorbing-layer attenuation along axis a of a level, at k h and (k + 1/2) h for k = -2 .. n+2.
template <typename T>
void upload_abl_tables(emg_ctx& c, Level& L) {
  const emg_params& p = c.prm;
  const double Lab = p.abl_cells > 0 ? p.abl_cells * p.h : 0.0;
  for (int a = 0; a < c.dim; ++a) {
    const int n = L.n[a];
    const double X = p.n[a] * p.h;
    std::vector<T> tab(2 * (n + 5));
    for (int k = -2; k <= n + 2; ++k)
      for (int half = 0; half < 2; ++half) {
        const double x = (k + 0.5 * half) * L.h;
        tab[2 * (k + 2) + half] = (T)(Lab > 0.0 ? p.abl_gamma_max * abl_axis(x, Lab, X) / (Lab * Lab) : 0.0);
      }
    // the attenuation-free range: k with both entries zero, contiguous around the middle
    auto zero_at = [&](int k) { return tab[2 * (k + 2)] == T(0) && tab[2 * (k + 2) + 1] == T(0); };
    int lo = n / 2, hi = n / 2 - 1;
    if (zero_at(n / 2)) {
      lo = hi = n / 2;
      while (lo > -2 && zero_at(lo - 1)) --lo;
      while (hi < n + 2 && zero_at(hi + 1)) ++hi;
    }
    L.zlo[a] = lo;
    L.zhi[a] = hi;
    L.abl_tab[a].alloc(tab.size() * sizeof(T));
    CK(cudaMemcpy(L.abl_tab[a].p, tab.data(), tab.size() * sizeof(T), cudaMemcpyHostToDevice));
  }
}

// EMG_COARSE_KACZMARZ set-up (Sec. 3.2, 5.3): the Schur rows of the coarsest level by probing
// its operator, the Schur and Krylov vectors, the boxes' private copies and the launch shape.
template <typename T>
void setup_kaczmarz(emg_ctx& c) {
  const int d = c.dim, l = c.L - 1;
  const Level& C = c.lv[l];
  const KzCfg k = kz_cfg(c.prm);
  int box[3] = {k.box[0], k.box[1], k.box[2]};
  if (box[0] == 0) kz_auto_box(d, C.n, c.sms, sizeof(cx<T>), box);
  c.kz_B = kz::make_boxes(d, C.n, box);
  const size_t N = C.ncell, DN = (size_t)d * N, cb = sizeof(cx<T>);
  const int NE = d == 3 ? kz::Shape<3>::NE : kz::Shape<2>::NE;
  c.kz_coef.alloc(DN * NE * cb);
  c.kz_n2.alloc(DN * sizeof(T));
  {
    DBuf e, y;
    e.alloc((d + 1) * N * cb);
    y.alloc((d + 1) * N * cb);
    CK(launch_kz_probe<T>(level_grid<T>(c, l), d, c.kz_coef.as<cx<T>>(), c.kz_n2.as<T>(), e.as<cx<T>>(),
                          y.as<cx<T>>(), c.st));
    CK(cudaStreamSynchronize(c.st));  // e and y are released here
  }
  c.kz_f.alloc(DN * cb);
  c.kz_u.alloc(DN * cb);
  c.kz_w.alloc(DN * cb);
  c.kz_V.alloc((size_t)(k.restart + 1) * DN * cb);
  c.kz_Z.alloc((size_t)k.restart * DN * cb);
  c.kz_copies.alloc((size_t)c.kz_B.nboxes * c.kz_B.RS * cb);
  CK(plan_kz_solve<T>(d, c.sms, c.kz_B.RS, c.kz_B.box, c.kz_launch));
  c.kz_part.alloc((size_t)4 * c.kz_launch.blocks * sizeof(double));
  c.kz_bar.alloc(2 * sizeof(unsigned));
  CK(cudaMemset(c.kz_bar.p, 0, c.kz_bar.bytes));
  c.kz_stats.alloc(4 * sizeof(double));
  CK(cudaMemset(c.kz_stats.p, 0, c.kz_stats.bytes));
}

template <typename T>
kz::Args<T> kz_args(emg_ctx& c, const cx<T>* b, cx<T>* x) {
  const int l = c.L - 1;
  const KzCfg k = kz_cfg(c.prm);
  kz::Args<T> a{};
  a.g = level_grid<T>(c, l);
  a.B = c.kz_B;
  a.N = c.lv[l].ncell;
  a.warps_a = c.kz_launch.warps;
  a.coef = c.kz_coef.as<const cx<T>>();
  a.inv_n2 = c.kz_n2.as<const T>();
  a.b = b;
  a.x = x;
  a.f = c.kz_f.as<cx<T>>();
  a.u = c.kz_u.as<cx<T>>();
  a.w = c.kz_w.as<cx<T>>();
  a.V = c.kz_V.as<cx<T>>();
  a.Z = c.kz_Z.as<cx<T>>();
  a.copies = c.kz_copies.as<cx<T>>();
  a.part = c.kz_part.as<double>();
  a.bar = c.kz_bar.as<unsigned>();
  a.err = c.dev_err.as<int>();
  a.stats = c.kz_stats.as<double>();
  a.damping = (T)k.damping;
  a.steps = k.steps;
  a.restart = k.restart;
  a.max_its = std::max(1, k.max_steps / k.steps);
  a.tol = k.tol;
  return a;
}

template <typename T>
void build(emg_ctx& c) {
  const int d = c.dim;
  for (int l = 0; l < c.L; ++l) {
    Level& L = c.lv[l];
    if (l > 0) coarsen_material(c, c.lv[l - 1], L);
    upload_material<T>(c, L);
    upload_abl_tables<T>(c, L);
    L.b.alloc((d + 1) * L.ncell * sizeof(cx<T>));
    L.x.alloc((d + 1) * L.ncell * sizeof(cx<T>));
    L.alt.alloc((d + 1) * L.ncell * sizeof(cx<T>));  // a whole second state (one-pass sweeps alternate)
    if (c.prm.cycle_type == EMG_CYCLE_K && l >= 1 && l < c.L - 1) {
      const size_t vb = (d + 1) * L.ncell * sizeof(cx<T>);
      L.kz1.alloc(vb);
      L.kz2.alloc(vb);
      L.kq1.alloc(vb);
      L.kq2.alloc(vb);
      L.kr2.alloc(vb);
      L.kpart.alloc((size_t)vec_blocks(c, (d + 1) * L.ncell) * 3 * sizeof(double));
      L.kcoef.alloc(8 * sizeof(double));
    }
    CK(cudaMemset(L.b.p, 0, L.b.bytes));
    CK(cudaMemset(L.x.p, 0, L.x.bytes));
    CK(cudaMemset(L.alt.p, 0, L.alt.bytes));
  }
  if (c.L > 1) c.rscr.alloc((d + 1) * c.lv[0].ncell * sizeof(cx<T>));
  c.dev_err.alloc(16);
  CK(cudaMemset(c.dev_err.p, 0, c.dev_err.bytes));
  // finest material in FP64 for the outer operator
  Level& F = c.lv[0];
  std::vector<double> cp(F.ncell);
  for (size_t k = 0; k < F.ncell; ++k) cp[k] = 1.0 / (F.lam_h[k] + F.mu_h[k]);
  c.mu64.alloc(F.ncell * 8);
  c.rho64.alloc(F.ncell * 8);
  c.cp64.alloc(F.ncell * 8);
  CK(cudaMemcpy(c.mu64.p, F.mu_h.data(), F.ncell * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c.rho64.p, F.rho_h.data(), F.ncell * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c.cp64.p, cp.data(), F.ncell * 8, cudaMemcpyHostToDevice));
  if (c.dim == 2) build_ff2(c);
  else build_ff3(c);
  if (c.prm.coarse_solver == EMG_COARSE_DENSE) {
    std::vector<std::complex<double>> A, Ainv;
    std::vector<int> act;
    assemble_dense(c, A, act);
    invert_dense(A, act, Ainv);
    const size_t NF = act.size();
    std::vector<cx<T>> h(NF * NF);
    for (size_t k = 0; k < NF * NF; ++k) h[k] = mkc<T>((T)Ainv[k].real(), (T)Ainv[k].imag());
    c.cinv.alloc(NF * NF * sizeof(cx<T>));
    CK(cudaMemcpy(c.cinv.p, h.data(), NF * NF * sizeof(cx<T>), cudaMemcpyHostToDevice));
    c.cn = (int)NF;
  }
  if (c.prm.coarse_solver == EMG_COARSE_KACZMARZ) setup_kaczmarz<T>(c);
  CK(cudaDeviceSynchronize());
  choose_sweep_paths(c);
}

// ---------------------------------------------------------------- FP64 Krylov helpers
void ensure_krylov(emg_ctx& c, int m) {
  const size_t n = c.nvec();
  const size_t cb = c.prec == 32 ? 8 : 16;
  if (c.km < m) {
    c.V.alloc((size_t)(m + 1) * n * 16);
    c.Z.alloc((size_t)m * n * cb);
    c.km = m;
  }
  if (!c.wk64.p) c.wk64.alloc(n * 16);
  const int nblk = vec_blocks(c, n);
  const size_t need = (size_t)nblk * (2 * kv::MAXV + 1) * 16 * sizeof(double);
  if (c.part.bytes < need) c.part.alloc(need);
  if (!c.red.p) c.red.alloc(4096 * sizeof(double));
  if (!c.hred) CK(cudaMallocHost(&c.hred, 4096 * sizeof(double)));
}

// Launch one multi-dot pass over NV vectors: native FP64 (exact) on complex doubles, or float-float
// (ff) on float-float pairs (df::cff, the Krylov basis and the applied vector).
template <int NV>
void launch_mdot(emg_ctx& c, bool ff, const cx<double>* V, size_t ldv, const cx<double>* w, size_t n, double* part,
                 int nblk) {
  if (ff)
    launch_dep(kf::mdot<NV>, dim3(nblk), dim3(kv::RT), 0, c.st, reinterpret_cast<const df::cff*>(V), ldv,
               reinterpret_cast<const df::cff*>(w), n, part);
  else launch_dep(kv::mdot<NV>, dim3(nblk), dim3(kv::RT), 0, c.st, V, ldv, w, n, part);
  CKL();
  LAUNCHED(c);
}

// h[i] = V_i^H w for i < cnt, and ||w||^2; one device->host transfer, one synchronisation.
void mdots(emg_ctx& c, bool ff, const cx<double>* V, size_t ldv, int cnt, const cx<double>* w, size_t n,
           std::vector<std::complex<double>>& h, double& wn2) {
  const int nblk = vec_blocks(c, n);
  double* part = c.part.as<double>();
  double* red = c.red.as<double>();
  int off = 0, s = 0;
  std::vector<std::pair<int, int>> chunks;  // (first vector, count)
  const double vbytes = (double)n * 16;
  do {
    int nv = std::min(kv::MAXV, cnt - s);
    {
      ProfScope ps(c, EMG_K_KRYLOV, 0, vbytes * (nv + 1));
      switch (nv) {
        case 0: launch_mdot<0>(c, ff, V, ldv, w, n, part, nblk); break;
        case 1: launch_mdot<1>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 2: launch_mdot<2>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 3: launch_mdot<3>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 4: launch_mdot<4>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 5: launch_mdot<5>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 6: launch_mdot<6>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 7: launch_mdot<7>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 8: launch_mdot<8>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 9: launch_mdot<9>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 10: launch_mdot<10>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 11: launch_mdot<11>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 12: launch_mdot<12>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 13: launch_mdot<13>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 14: launch_mdot<14>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        case 15: launch_mdot<15>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
        default: launch_mdot<16>(c, ff, V + s * ldv, ldv, w, n, part, nblk); break;
      }
    }
    const int nr = 2 * nv + 1;
    launch_dep(kv::reduce_parts, dim3(nr), dim3(kv::RP), 0, c.st, part, nblk, nr, red + off);
    CKL();
    LAUNCHED(c);
    chunks.push_back({s, nv});
    off += nr;
    s += nv;
  } while (s < cnt);
  CK(cudaMemcpyAsync(c.hred, red, off * sizeof(double), cudaMemcpyDeviceToHost, c.st));
  CK(cudaStreamSynchronize(c.st));
  h.assign(cnt, 0.0);
  off = 0;
  for (auto& ch : chunks) {
    for (int v = 0; v < ch.second; ++v) h[ch.first + v] = std::complex<double>(c.hred[off + 2 * v], c.hred[off + 2 * v + 1]);
    wn2 = c.hred[off + 2 * ch.second];
    off += 2 * ch.second + 1;
  }
  for (auto& z : h)
    if (!std::isfinite(z.real()) || !std::isfinite(z.imag())) raise(EMG_ERR_NONFINITE, "non-finite Krylov inner product");
  if (!std::isfinite(wn2)) raise(EMG_ERR_NONFINITE, "non-finite Krylov norm");
}

// w <- s (w - sum_i h_i V_i) on float-float vectors, optionally also written to outc (the next
// cycle's right-hand side) in FP32 (outk 1) or FP64 (outk 2). With want_norm, returns
// ||w_new||^2 (one reduction and a synchronisation); otherwise returns 0 and does not wait.
double update_scale(emg_ctx& c, cx<double>* w, const cx<double>* V, size_t ldv,
                    const std::vector<std::complex<double>>& h, double s, size_t n, void* outc, int outk,
                    bool want_norm = false) {
  const int nblk = vec_blocks(c, n);
  kf::Coefs co;
  const int cnt = (int)h.size();
  for (int i = 0; i < cnt; ++i) co.c[i] = {to_f2(h[i].real()), to_f2(h[i].imag())};
  {
    ProfScope ps(c, EMG_K_KRYLOV, 0, (double)n * 16 * (cnt + 2) + (double)n * 8.0 * outk);
    launch_dep(kf::update_scale, dim3(nblk), dim3(kv::RT), 0, c.st, reinterpret_cast<df::cff*>(w),
               reinterpret_cast<const df::cff*>(V), ldv, cnt, co, to_f2(s), n, outc, outk, c.part.as<double>());
    CKL();
    LAUNCHED(c);
  }
  if (!want_norm) return 0.0;
  launch_dep(kv::reduce_parts, dim3(1), dim3(kv::RP), 0, c.st, c.part.as<double>(), nblk, 1, c.red.as<double>());
  CKL();
  LAUNCHED(c);
  CK(cudaMemcpyAsync(c.hred, c.red.p, sizeof(double), cudaMemcpyDeviceToHost, c.st));
  CK(cudaStreamSynchronize(c.st));
  if (!std::isfinite(c.hred[0])) raise(EMG_ERR_NONFINITE, "non-finite Krylov norm");
  return c.hred[0];
}

// y = H x (unshifted or shifted) or y = bscale*b - H x on the finest level in FP64; x in FP64 or FP32.
// ffo: y is one of the outer solve's float-float vectors (df::cff) instead of complex doubles.
void outer_apply(emg_ctx& c, const void* x, bool x32, const cx<double>* b, double bscale, cx<double>* y, bool shifted,
                 bool ffo = false) {
  const double cw = 16.0;
  if (c.dim == 2) {
    // float-float evaluation from precomputed FP64 coefficients (x, b, y + mu, node mu, cp, 2 masses)
    ProfScope ps(c, EMG_K_APPLY64, 0, (double)c.lv[0].ncell * (3 * ((x32 ? 8.0 : 16.0) + cw + (b ? cw : 0.0)) + 3 * 8.0 + 2 * 16.0));
    const Level& F = c.lv[0];
    const ff2::FineFF g = ff2::make(c.ff_mu.as<df::f2>(), c.ff_mun.as<df::f2>(), c.ff_cp.as<df::f2>(),
                                    c.ff_m1.as<ff2::c2>(), c.ff_m2.as<ff2::c2>(), F.n[0], F.n[1], F.h, c.prm.beta,
                                    shifted ? level_alpha(c.prm, 0) : 0.0);
    if (x32) launch_apply_ff2<float>(g, (const cx<float>*)x, b, bscale, y, ffo, c.st);
    else launch_apply_ff2<double>(g, (const cx<double>*)x, b, bscale, y, ffo, c.st);
    CKL();
    LAUNCHED(c);
    return;
  }
  // 3D: float-float evaluation from precomputed FP64 coefficients
  ProfScope ps(c, EMG_K_APPLY64, 0, (double)c.lv[0].ncell * (4 * ((x32 ? 8.0 : 16.0) + cw + (b ? cw : 0.0)) + 2 * 8.0 + 3 * 8.0 + 3 * 16.0));
  const Level& F = c.lv[0];
  const df::f2* ed[3] = {c.ff3_edge[0].as<df::f2>(), c.ff3_edge[1].as<df::f2>(), c.ff3_edge[2].as<df::f2>()};
  const ff2::c2* ms[3] = {c.ff3_m[0].as<ff2::c2>(), c.ff3_m[1].as<ff2::c2>(), c.ff3_m[2].as<ff2::c2>()};
  ff3::HostFF3 none;
  ff3::FineFF3 g = ff3::make(none, c.ff_mu.as<df::f2>(), c.ff_cp.as<df::f2>(), ed, ms, F.n[0], F.n[1], F.n[2], F.h,
                             c.prm.beta, shifted ? level_alpha(c.prm, 0) : 0.0);
  if (x32) launch_apply_ff3<float>(g, (const cx<float>*)x, b, bscale, y, ffo, c.st);
  else launch_apply_ff3<double>(g, (const cx<double>*)x, b, bscale, y, ffo, c.st);
  CKL();
  LAUNCHED(c);
}

// y = H^H x (the unshifted finest operator, conjugate-transposed) or y = bscale*b - H^H x, FP64;
// x in FP64 or FP32.
void outer_apply_adjoint(emg_ctx& c, const void* x, bool x32, const cx<double>* b, double bscale, cx<double>* y,
                         bool ffo = false) {
  const Level& F = c.lv[0];
  ProfScope ps(c, EMG_K_APPLY64, 0,
               (double)F.ncell * ((c.dim + 1) * ((x32 ? 8.0 : 16.0) + 16.0 + (b ? 16.0 : 0.0)) + 3 * 8.0));
  const Grid<double> g = make_grid<double>(c, 0, false, c.mu64.p, c.rho64.p, c.cp64.p);
  if (c.dim == 2) {
    if (x32) launch_adjoint_apply<2, float>(g, (const cx<float>*)x, b, bscale, y, ffo, c.st);
    else launch_adjoint_apply<2, double>(g, (const cx<double>*)x, b, bscale, y, ffo, c.st);
  } else {
    // float-float on the forward apply's coefficients (the FP64 pipe is ~57x slower)
    const df::f2* ed[3] = {c.ff3_edge[0].as<df::f2>(), c.ff3_edge[1].as<df::f2>(), c.ff3_edge[2].as<df::f2>()};
    const ff2::c2* ms[3] = {c.ff3_m[0].as<ff2::c2>(), c.ff3_m[1].as<ff2::c2>(), c.ff3_m[2].as<ff2::c2>()};
    ff3::HostFF3 none;
    const ff3::FineFF3 gf = ff3::make(none, c.ff_mu.as<df::f2>(), c.ff_cp.as<df::f2>(), ed, ms, F.n[0], F.n[1], F.n[2],
                                      F.h, c.prm.beta, 0.0);
    if (x32) launch_apply_adjoint_ff3<float>(gf, (const cx<float>*)x, b, bscale, y, ffo, c.st);
    else launch_apply_adjoint_ff3<double>(gf, (const cx<double>*)x, b, bscale, y, ffo, c.st);
  }
  CKL();
  LAUNCHED(c);
}

// z <- S conj(z) on an FP32 cycle vector (S = diag(I, -I)): maps the forward cycle onto a
// preconditioner for H^H (emg_solve_adjoint).
template <typename T>
void sconj_cycle_vector(emg_ctx& c, cx<T>* z) {
  if constexpr (std::is_same<T, float>::value) {
    launch_sconj(z, (size_t)c.dim * c.lv[0].ncell, c.nvec(), c.st);
    CKL();
    LAUNCHED(c);
  } else {
    (void)z;
    raise(EMG_ERR_INVALID, "adjoint solves need the FP32 cycle");
  }
}

// Capture vcycle(0, b, z) into a graph; nullptr (and graphs off for this handle) if the capture
// or the instantiation fails, e.g. because the runtime cannot capture a launch kind.
template <typename T>
cudaGraphExec_t capture_cycle(emg_ctx& c, const cx<T>* b, cx<T>* z, int64_t& kernels,
                              std::vector<emg_ctx::Rec>* recs) {
  const int64_t l0 = c.launches;
  if (cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  bool ok = true;
  c.capture_recs = recs;  // with the instrumentation on, its event pairs become graph nodes
  try {
    vcycle<T>(c, 0, b, z, true);
  } catch (const EmgError&) {
    ok = false;
  }
  c.capture_recs = nullptr;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c.st, &g);
  kernels = c.launches - l0;
  c.launches = l0;  // nothing ran yet
  cudaGraphExec_t exec = nullptr;
  if (ok && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();  // a failed capture leaves no error behind for the next call
  return exec;
}

template <typename T>
void precondition(emg_ctx& c, const cx<double>* v, cx<T>* z) {
  Level& F = c.lv[0];
  // the cycle's right-hand side was written in its precision to F.b by the update that produced v
  (void)v;
  const cx<T>* b = F.b.as<cx<T>>();
  if (c.graphs_ok) {
    // with the instrumentation on, a graph that records its own event pairs (they are graph
    // nodes, so every replay times its kernels); otherwise one without
    const int timed = c.prof ? (c.prof_coarse ? 2 : 1) : 0;
    emg_ctx::CycleGraph* cg = nullptr;
    for (auto& g : c.graphs)
      if (g.b == b && g.z == z && g.timed == timed) cg = &g;
    if (!cg) {
      c.graphs.push_back({b, z, timed, 0, nullptr, 0, {}, false});
      cg = &c.graphs.back();
    }
    if (!cg->exec && cg->uses >= 1) {
      cg->exec = capture_cycle<T>(c, b, z, cg->kernels, timed ? &cg->recs : nullptr);
      if (!cg->exec) {
        c.graphs_ok = false;
        for (auto& r : cg->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        cg->recs.clear();
      }
    }
    if (cg->exec) {
      harvest(c, *cg);  // the previous replay of this graph finished: the loop has synchronised since
      CK(cudaGraphLaunch(cg->exec, c.st));
      c.launches += cg->kernels;
      cg->unread = timed && !cg->recs.empty();
      return;
    }
    ++cg->uses;
  }
  vcycle<T>(c, 0, b, z, true);
}

// Reads the device status word of the bounded waits (after a synchronisation): a tile load that
// timed out left the sweep's result unusable.
void check_device_status(emg_ctx& c) {
  int flags = 0;
  CK(cudaMemcpy(&flags, c.dev_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (flags) {
    CK(cudaMemset(c.dev_err.p, 0, sizeof(int)));
    if (c.kz_bar.p) CK(cudaMemset(c.kz_bar.p, 0, c.kz_bar.bytes));
    raise(EMG_ERR_TIMEOUT, (flags & 2) ? "a grid-wide barrier of the Kaczmarz coarsest solve timed out"
                                       : "a shared-memory tile load of the one-pass sweep timed out");
  }
}

// Re-orthogonalise when ||w'||^2 < kReorth ||w||^2. At that ratio the Pythagorean norm keeps
// ~13 correct digits (its absolute error is ~eps ||w||^2) and one classical Gram-Schmidt pass
// leaves the new vector orthogonal to ~eps ||w||/||w'|| ~ 1e-14, far below what a 1e-6 solve
// needs; the true residual is recomputed at every restart regardless.
constexpr double kReorth = 1e-3;

// Right-preconditioned restarted FGMRES(m), Saad (1993). Classical Gram-Schmidt with the
// Pythagorean norm ||w'||^2 = ||w||^2 - sum |h_i|^2 and one re-orthogonalisation pass when it
// cancels (kReorth); the update of the new basis vector is deferred into a fused
// pass that also normalises it and writes the next cycle's FP32 right-hand side. All vectors are
// scaled by a power of two so that ||b|| ~ 1 (exact), which keeps them inside the float exponent
// range of the float-float kernels; x is unscaled on exit.
template <typename T>
emg_status solve_impl(emg_ctx& c, const cx<double>* b, cx<double>* x, double tol, int max_iter, int m, emg_stats* st,
                      bool adj = false) {
  const size_t n = c.nvec();
  ensure_krylov(c, m);
  const bool f32 = std::is_same<T, float>::value;
  cx<double>* V = c.V.as<cx<double>>();
  cx<T>* Z = c.Z.as<cx<T>>();
  cx<double>* r = c.wk64.as<cx<double>>();
  // the Krylov vectors V (and r) are float-float pairs; each finished V_j is also written to the
  // cycle's right-hand side in the cycle's precision
  void* bcyc = c.lv[0].b.p;
  const int bk = f32 ? 1 : 2;
  int hist = 0;
  auto push_hist = [&](double v) {
    if (st && st->history && hist < st->history_cap) st->history[hist] = v;
    ++hist;
  };
  std::vector<std::complex<double>> h, h2;
  double bn2 = 0;
  mdots(c, false, nullptr, 0, 0, b, n, h, bn2);  // exact FP64 norm of the caller's b
  const double bnorm = std::sqrt(bn2);
  if (!(bnorm > 0.0)) {
    CK(cudaMemsetAsync(x, 0, n * 16, c.st));
    CK(cudaStreamSynchronize(c.st));
    if (st) { st->iterations = 0; st->restarts = 0; st->rel_residual = 0.0; st->history_len = 0; }
    return EMG_OK;
  }
  const double sc = std::ldexp(1.0, -std::ilogb(bnorm));  // power of two: sc*||b|| in [1, 2)
  const double bhat = sc * bnorm;
  launch_dep(kv::scale, dim3(vec_blocks(c, n)), dim3(256), 0, c.st, x, x, sc, n);
  CKL();
  LAUNCHED(c);
  auto true_residual = [&]() {
    if (adj) outer_apply_adjoint(c, x, false, b, sc, r, true);  // r = sc*b - H^H (sc*x)
    else outer_apply(c, x, false, b, sc, r, false, true);     // r = sc*b - H (sc*x)
    double rn2 = 0;
    mdots(c, true, nullptr, 0, 0, r, n, h, rn2);
    return std::sqrt(rn2);
  };
  double beta = true_residual();
  push_hist(beta / bhat);
  int its = 0, restarts = 0;
  std::vector<std::complex<double>> Hh((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1);
  while (beta / bhat > tol && its < max_iter) {
    // V_0 = r / beta (and its FP32 copy for the first cycle)
    CK(cudaMemcpyAsync(V, r, n * 16, cudaMemcpyDeviceToDevice, c.st));
    update_scale(c, V, V, n, {}, 1.0 / beta, n, bcyc, bk);
    std::fill(Hh.begin(), Hh.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    std::vector<std::complex<double>> pend;  // deferred coefficients of V_j
    double pend_norm = 1.0;
    for (int j = 0; j < m; ++j) {
      cx<double>* vj = V + (size_t)j * n;
      if (j > 0) update_scale(c, vj, V, n, pend, 1.0 / pend_norm, n, bcyc, bk);  // finish V_j
      cx<double>* w = V + (size_t)(j + 1) * n;
      if (adj) sconj_cycle_vector<T>(c, c.lv[0].b.as<cx<T>>());  // the cycle solves with conj(S v_j)
      precondition<T>(c, vj, Z + (size_t)j * n);
      if (adj) {
        sconj_cycle_vector<T>(c, Z + (size_t)j * n);  // z_j = S conj(M conj(S v_j))
        outer_apply_adjoint(c, Z + (size_t)j * n, f32, nullptr, 0.0, w, true);
      } else {
        outer_apply(c, Z + (size_t)j * n, f32, nullptr, 0.0, w, false, true);
      }
      double wn2 = 0;
      mdots(c, true, V, n, j + 1, w, n, h, wn2);
      double hh = 0;
      for (auto& z : h) hh += std::norm(z);
      double nn2 = wn2 - hh;
      pend = h;
      if (nn2 < kReorth * wn2) {  // cancellation: apply the projection now and orthogonalise again
        update_scale(c, w, V, n, h, 1.0, n, nullptr, 0);
        double wn2b = 0;
        mdots(c, true, V, n, j + 1, w, n, h2, wn2b);
        double hh2 = 0;
        for (auto& z : h2) hh2 += std::norm(z);
        nn2 = wn2b - hh2;
        if (nn2 < kReorth * wn2b) {  // still cancelling: materialise and measure exactly
          nn2 = update_scale(c, w, V, n, h2, 1.0, n, nullptr, 0, true);
          h2.assign(j + 1, 0.0);
        }
        for (int i = 0; i <= j; ++i) h[i] += h2[i];
        pend = h2;
      }
      const double hn = std::sqrt(std::max(nn2, 0.0));
      pend_norm = hn > 0.0 ? hn : 1.0;
      for (int i = 0; i <= j; ++i) Hh[(size_t)i * m + j] = h[i];
      Hh[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        std::complex<double> a = Hh[(size_t)i * m + j], bb = Hh[(size_t)(i + 1) * m + j];
        Hh[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        Hh[(size_t)(i + 1) * m + j] = -std::conj(sn[i]) * a + std::conj(cs[i]) * bb;
      }
      std::complex<double> a = Hh[(size_t)j * m + j], bb = Hh[(size_t)(j + 1) * m + j];
      const double den = std::sqrt(std::norm(a) + std::norm(bb));
      if (den == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
      else { cs[j] = std::conj(a / den); sn[j] = std::conj(bb / den); }
      Hh[(size_t)j * m + j] = cs[j] * a + sn[j] * bb;
      Hh[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -std::conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      k = j + 1;
      push_hist(std::abs(g[j + 1]) / bhat);
      if (std::abs(g[j + 1]) / bhat <= tol || its >= max_iter || hn == 0.0) break;
    }
    // y = R^{-1} g, x += Z y
    std::vector<std::complex<double>> y(k);
    for (int i = k - 1; i >= 0; --i) {
      std::complex<double> s = g[i];
      for (int q = i + 1; q < k; ++q) s -= Hh[(size_t)i * m + q] * y[q];
      y[i] = s / Hh[(size_t)i * m + i];
    }
    kf::Coefs co;
    for (int i = 0; i < k; ++i) co.c[i] = {to_f2(y[i].real()), to_f2(y[i].imag())};
    {
      ProfScope ps(c, EMG_K_KRYLOV, 0, (double)n * (32.0 + k * (f32 ? 8.0 : 16.0)));
      launch_dep(kf::combine<T>, dim3(vec_blocks(c, n)), dim3(kv::RT), 0, c.st, x, Z, n, k, co, n);
      CKL();
      LAUNCHED(c);
    }
    beta = true_residual();
    ++restarts;
  }
  launch_dep(kv::scale, dim3(vec_blocks(c, n)), dim3(256), 0, c.st, x, x, 1.0 / sc, n);
  CKL();
  LAUNCHED(c);
  CK(cudaStreamSynchronize(c.st));
  check_device_status(c);
  if (st) {
    st->iterations = its;
    st->restarts = restarts;
    st->rel_residual = beta / bhat;
    st->history_len = std::min(hist, st->history ? st->history_cap : 0);
  }
  return beta / bhat <= tol ? EMG_OK : EMG_NOT_CONVERGED;
}

// The checks that concern one level's operator and smoother (grid, coefficients, precision).
void check_level_params(const emg_params* p) {
  if (!p) raise(EMG_ERR_INVALID, "params is NULL");
  if (p->dim != 2 && p->dim != 3) raise(EMG_ERR_INVALID, "dim must be 2 or 3");
  if (p->levels < 1 || p->levels > EMG_MAX_LEVELS) raise(EMG_ERR_INVALID, "levels out of range");
  for (int a = 0; a < p->dim; ++a)
    if (p->n[a] < 2) raise(EMG_ERR_INVALID, "each n must be >= 2");
  if (!(p->h > 0) || !std::isfinite(p->h)) raise(EMG_ERR_INVALID, "h must be positive");
  if (!std::isfinite(p->omega) || !std::isfinite(p->gamma) || !std::isfinite(p->alpha) || !std::isfinite(p->beta))
    raise(EMG_ERR_INVALID, "non-finite omega/gamma/alpha/beta");
  for (int l = 0; l < EMG_MAX_LEVELS; ++l)
    if (!std::isfinite(p->level_alpha[l])) raise(EMG_ERR_INVALID, "non-finite level_alpha");
  if (p->abl_cells < 0) raise(EMG_ERR_INVALID, "abl_cells must be >= 0");
  if (p->nu_pre < 0 || p->nu_post < 0) raise(EMG_ERR_INVALID, "negative smoothing count");
  if (p->cycle_precision != 32 && p->cycle_precision != 64) raise(EMG_ERR_INVALID, "cycle_precision must be 32 or 64");
  if (p->cycle_type != EMG_CYCLE_V && p->cycle_type != EMG_CYCLE_W && p->cycle_type != EMG_CYCLE_K)
    raise(EMG_ERR_INVALID, "unknown cycle_type");
  if (p->smoother != EMG_VANKA_FULL && p->smoother != EMG_VANKA_ECONOMIC) raise(EMG_ERR_INVALID, "unknown smoother");
  if (p->sweep_path < EMG_SWEEP_AUTO || p->sweep_path > EMG_SWEEP_TILE4) raise(EMG_ERR_INVALID, "unknown sweep_path");
}

// Every check of emg_create: one level's, then the hierarchy's.
void check_params(const emg_params* p) {
  check_level_params(p);
  const int div = 1 << (p->levels - 1);
  for (int a = 0; a < p->dim; ++a) {
    if (p->n[a] % div) raise(EMG_ERR_INVALID, "n[" + std::to_string(a) + "] not divisible by 2^(levels-1)");
    if (p->n[a] / div < 2) raise(EMG_ERR_INVALID, "coarsest grid must have >= 2 cells per axis");
  }
  if (p->coarse_solver != EMG_COARSE_DENSE && p->coarse_solver != EMG_COARSE_SMOOTH &&
      p->coarse_solver != EMG_COARSE_KACZMARZ)
    raise(EMG_ERR_INVALID, "unknown coarse_solver");
  if (p->coarse_solver == EMG_COARSE_KACZMARZ) {
    const KzCfg k = kz_cfg(*p);
    bool zero = true, ones = true, big = true;
    for (int a = 0; a < p->dim; ++a) {
      zero = zero && k.box[a] == 0;
      ones = ones && k.box[a] == 1;
      big = big && k.box[a] >= 2 && k.box[a] <= 64;
    }
    if (!zero && !ones && !big)
      raise(EMG_ERR_INVALID, "kaczmarz_box: all 0 (automatic), all 1, or each in 2..64");
    if (p->kaczmarz_steps < 0 || p->coarse_restart < 0 || p->kaczmarz_max < 0 || k.restart > kz::MAXM)
      raise(EMG_ERR_INVALID, "kaczmarz_steps, kaczmarz_max must be >= 0 and coarse_restart in 0..8");
    if (!std::isfinite(p->kaczmarz_damping) || p->kaczmarz_damping < 0.0 || k.damping >= 2.0)
      raise(EMG_ERR_INVALID, "kaczmarz_damping must be in (0, 2) (0: 0.8)");
    if (!std::isfinite(p->coarse_tol) || p->coarse_tol < 0.0) raise(EMG_ERR_INVALID, "coarse_tol must be >= 0");
    int nc[3] = {1, 1, 1};
    for (int a = 0; a < p->dim; ++a) nc[a] = p->n[a] / div;
    const size_t cb = p->cycle_precision == 32 ? 8 : 16;
    if (!zero && kz_region_halfwarps(p->dim, nc, k.box, cb) < 2)
      raise(EMG_ERR_INVALID, "kaczmarz_box too large for shared memory");
  }
  if (p->coarse_solver == EMG_COARSE_SMOOTH && p->coarse_sweeps < 1 && p->levels > 0)
    raise(EMG_ERR_INVALID, "coarse_sweeps must be >= 1");
  size_t nc = 1;
  for (int a = 0; a < p->dim; ++a) nc *= (size_t)(p->n[a] / div);
  if (p->coarse_solver == EMG_COARSE_DENSE && nc * (p->dim + 1) > 4096)
    raise(EMG_ERR_INVALID, "dense coarsest solve limited to 4096 unknowns");
}

emg_ctx* checked(emg_handle h) {
  if (!h) raise(EMG_ERR_INVALID, "NULL handle");
  return h;
}

void check_level(emg_ctx& c, int level, bool need_coarser) {
  if (level < 0 || level >= c.L || (need_coarser && level >= c.L - 1)) raise(EMG_ERR_INVALID, "level out of range");
}

void check_ptr(const void* p, const char* what) {
  if (!p) raise(EMG_ERR_INVALID, std::string(what) + " is NULL");
  if (reinterpret_cast<uintptr_t>(p) % 16) raise(EMG_ERR_INVALID, std::string(what) + " is not 16-byte aligned");
}

}  // namespace

#define ABI_TRY try {
#define ABI_CATCH                                                   \
  }                                                                 \
  catch (const EmgError& e) { g_err = e.msg; return e.s; }          \
  catch (const std::bad_alloc&) { g_err = "host allocation failed"; return EMG_ERR_NOMEM; } \
  catch (const std::exception& e) { g_err = e.what(); return EMG_ERR_INVALID; }

void emg_set_last_error(const std::string& msg) { g_err = msg; }

emg_status emg_validate_level_params(const emg_params* p, std::string* why) {
  try {
    check_level_params(p);
  } catch (const EmgError& e) {
    if (why) *why = e.msg;
    return e.s;
  }
  return EMG_OK;
}



extern "C" {

const char* emg_last_error(void) { return g_err.c_str(); }

emg_status emg_create(const emg_params* params, const double* lam, const double* mu, const double* rho, int on_device,
                      void* cuda_stream, emg_handle* out) {
  NvtxRange nvtx_range("emg_create");
  ABI_TRY
  if (!out) raise(EMG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  check_params(params);
  if (!lam || !mu || !rho) raise(EMG_ERR_INVALID, "material pointer is NULL");
  std::unique_ptr<emg_ctx> c(new emg_ctx());
  c->prm = *params;
  c->dim = params->dim;
  c->L = params->levels;
  c->prec = params->cycle_precision;
  c->st = (cudaStream_t)cuda_stream;
  c->lv.resize(c->L);
  for (int l = 0; l < c->L; ++l) {
    Level& L = c->lv[l];
    L.ncell = 1;
    for (int a = 0; a < 3; ++a) {
      L.n[a] = a < c->dim ? params->n[a] >> l : 1;
      L.ncell *= (size_t)L.n[a];
    }
    L.h = params->h * (double)(1 << l);
    const double w = params->damping[l];
    L.w = w > 0.0 ? w : default_damping(c->L);
  }
  Level& F = c->lv[0];
  F.lam_h.resize(F.ncell);
  F.mu_h.resize(F.ncell);
  F.rho_h.resize(F.ncell);
  if (on_device) {
    CK(cudaMemcpy(F.lam_h.data(), lam, F.ncell * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(F.mu_h.data(), mu, F.ncell * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(F.rho_h.data(), rho, F.ncell * 8, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(F.lam_h.data(), lam, F.ncell * 8);
    std::memcpy(F.mu_h.data(), mu, F.ncell * 8);
    std::memcpy(F.rho_h.data(), rho, F.ncell * 8);
  }
  for (size_t k = 0; k < F.ncell; ++k) {
    if (!std::isfinite(F.lam_h[k]) || !std::isfinite(F.mu_h[k]) || !std::isfinite(F.rho_h[k]) || !(F.mu_h[k] > 0) ||
        !(F.rho_h[k] > 0) || !(F.lam_h[k] + F.mu_h[k] > 0))
      raise(EMG_ERR_INVALID, "material must be finite with mu > 0, rho > 0, lambda + mu > 0 (cell " + std::to_string(k) + ")");
  }
  // every argument check above needs no device; from here on the device is used
  CK(cudaGetDevice(&c->dev));
  CK(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev));
  if (c->prec == 32) build<float>(*c);
  else build<double>(*c);
  *out = c.release();
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_destroy(emg_handle h) {
  ABI_TRY
  if (h) {
    if (h->st) cudaStreamSynchronize(h->st);
    else cudaDeviceSynchronize();
    delete h;
  }
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_level_info(emg_handle h, int level, int32_t n[3], double* cell_size) {
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_level(c, level, false);
  for (int a = 0; a < 3; ++a) n[a] = c.lv[level].n[a];
  if (cell_size) *cell_size = c.lv[level].h;
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_sweep_path(emg_handle h, int level, int32_t* path, double* us_per_call) {
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_level(c, level, false);
  if (!path) raise(EMG_ERR_INVALID, "path is NULL");
  *path = c.lv[level].path;
  if (us_per_call) *us_per_call = c.lv[level].tuned_us;
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_apply(emg_handle h, int shifted, const void* x, void* y) {
  NvtxRange nvtx_range("emg_apply");
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_ptr(x, "x");
  check_ptr(y, "y");
  outer_apply(c, x, false, nullptr, 0.0, (cx<double>*)y, shifted != 0);
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_vcycle(emg_handle h, const void* b, void* x, int zero_guess) {
  NvtxRange nvtx_range("emg_vcycle");
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_ptr(b, "b");
  check_ptr(x, "x");
  if (c.prec == 32) vcycle<float>(c, 0, (const cx<float>*)b, (cx<float>*)x, zero_guess != 0);
  else vcycle<double>(c, 0, (const cx<double>*)b, (cx<double>*)x, zero_guess != 0);
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_smooth(emg_handle h, int level, const void* b, void* x, int sweeps) {
  NvtxRange nvtx_range("emg_smooth");
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_level(c, level, false);
  check_ptr(b, "b");
  check_ptr(x, "x");
  if (sweeps < 0) raise(EMG_ERR_INVALID, "sweeps < 0");
  const double w = c.lv[level].w;
  if (c.prec == 32) smooth<float>(c, level, (const cx<float>*)b, (cx<float>*)x, sweeps, w, false);
  else smooth<double>(c, level, (const cx<double>*)b, (cx<double>*)x, sweeps, w, false);
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_residual_restrict(emg_handle h, int level, const void* b, const void* x, void* bc) {
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_level(c, level, true);
  check_ptr(b, "b");
  check_ptr(x, "x");
  check_ptr(bc, "b_coarse");
  if (c.prec == 32) residual_restrict<float>(c, level, (const cx<float>*)b, (const cx<float>*)x, (cx<float>*)bc);
  else residual_restrict<double>(c, level, (const cx<double>*)b, (const cx<double>*)x, (cx<double>*)bc);
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_prolong_correct(emg_handle h, int level, const void* e, void* x) {
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_level(c, level, true);
  check_ptr(e, "e_coarse");
  check_ptr(x, "x");
  if (c.prec == 32) prolong_correct<float>(c, level, (const cx<float>*)e, (cx<float>*)x);
  else prolong_correct<double>(c, level, (const cx<double>*)e, (cx<double>*)x);
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_coarse_solve(emg_handle h, const void* b, void* x) {
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_ptr(b, "b");
  check_ptr(x, "x");
  if (c.prec == 32) coarse_solve<float>(c, (const cx<float>*)b, (cx<float>*)x);
  else coarse_solve<double>(c, (const cx<double>*)b, (cx<double>*)x);
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_coarse_stats(emg_handle h, double out[3]) {
  ABI_TRY
  emg_ctx& c = *checked(h);
  if (!out) raise(EMG_ERR_INVALID, "out is NULL");
  if (c.prm.coarse_solver != EMG_COARSE_KACZMARZ) raise(EMG_ERR_INVALID, "the coarsest solver is not EMG_COARSE_KACZMARZ");
  CK(cudaStreamSynchronize(c.st));
  check_device_status(c);
  double s[4];
  CK(cudaMemcpy(s, c.kz_stats.p, 4 * sizeof(double), cudaMemcpyDeviceToHost));
  for (int i = 0; i < 3; ++i) out[i] = s[i];
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_coarse_schur_rows(emg_handle h, void* rows_host) {
  ABI_TRY
  emg_ctx& c = *checked(h);
  if (!rows_host) raise(EMG_ERR_INVALID, "rows_host is NULL");
  if (c.prm.coarse_solver != EMG_COARSE_KACZMARZ) raise(EMG_ERR_INVALID, "the coarsest solver is not EMG_COARSE_KACZMARZ");
  CK(cudaStreamSynchronize(c.st));
  CK(cudaMemcpy(rows_host, c.kz_coef.p, c.kz_coef.bytes, cudaMemcpyDeviceToHost));
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_solve(emg_handle h, const void* b, void* x, double tol, int max_iter, int restart, emg_stats* stats) {
  NvtxRange nvtx_range("emg_solve");
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_ptr(b, "b");
  check_ptr(x, "x");
  if (restart < 1 || restart > 64) raise(EMG_ERR_INVALID, "restart must be in 1..64");
  if (max_iter < 0) raise(EMG_ERR_INVALID, "max_iter < 0");
  if (!(tol >= 0.0)) raise(EMG_ERR_INVALID, "tol must be >= 0");
  if (c.prec == 32) return solve_impl<float>(c, (const cx<double>*)b, (cx<double>*)x, tol, max_iter, restart, stats);
  return solve_impl<double>(c, (const cx<double>*)b, (cx<double>*)x, tol, max_iter, restart, stats);
  ABI_CATCH
}

emg_status emg_apply_adjoint(emg_handle h, const void* x, void* y) {
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_ptr(x, "x");
  check_ptr(y, "y");
  outer_apply_adjoint(c, x, false, nullptr, 0.0, (cx<double>*)y);
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_solve_adjoint(emg_handle h, const void* b, void* x, double tol, int max_iter, int restart,
                             emg_stats* stats) {
  NvtxRange nvtx_range("emg_solve_adjoint");
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_ptr(b, "b");
  check_ptr(x, "x");
  if (restart < 1 || restart > 64) raise(EMG_ERR_INVALID, "restart must be in 1..64");
  if (max_iter < 0) raise(EMG_ERR_INVALID, "max_iter < 0");
  if (!(tol >= 0.0)) raise(EMG_ERR_INVALID, "tol must be >= 0");
  if (c.prec != 32) raise(EMG_ERR_INVALID, "emg_solve_adjoint needs cycle_precision 32");
  return solve_impl<float>(c, (const cx<double>*)b, (cx<double>*)x, tol, max_iter, restart, stats, true);
  ABI_CATCH
}

emg_status emg_material_gradient(emg_handle h, const void* u, const void* a, double* g_lam, double* g_mu,
                                 double* g_rho, int accumulate) {
  ABI_TRY
  emg_ctx& c = *checked(h);
  check_ptr(u, "u");
  check_ptr(a, "a");
  for (const double* gp : {g_lam, g_mu, g_rho})
    if (!gp || reinterpret_cast<uintptr_t>(gp) % 8) raise(EMG_ERR_INVALID, "gradient arrays must be 8-byte aligned device arrays");
  const Grid<double> g = make_grid<double>(c, 0, false, c.mu64.p, c.rho64.p, c.cp64.p);
  {
    ProfScope ps(c, EMG_K_APPLY64, 0, (double)c.lv[0].ncell * (2 * (c.dim + 1) * 16.0 + 3 * 8.0 * (accumulate ? 2 : 1)));
    if (c.dim == 2)
      launch_adjoint_gradient<2>(g, (const cx<double>*)u, (const cx<double>*)a, g_lam, g_mu, g_rho, accumulate, c.st);
    else
      launch_adjoint_gradient<3>(g, (const cx<double>*)u, (const cx<double>*)a, g_lam, g_mu, g_rho, accumulate, c.st);
    CKL();
    LAUNCHED(c);
  }
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_solve_batch(const emg_handle* handles, int count, const void* const* b, void* const* x, double tol,
                           int max_iter, int restart, emg_stats* stats, int workers, emg_status* status) {
  NvtxRange nvtx_range("emg_solve_batch");
  ABI_TRY
  if (count < 0) raise(EMG_ERR_INVALID, "count < 0");
  if (count == 0) return EMG_OK;
  if (!handles || !b || !x) raise(EMG_ERR_INVALID, "handles, b or x is NULL");
  if (restart < 1 || restart > 64) raise(EMG_ERR_INVALID, "restart must be in 1..64");
  if (max_iter < 0) raise(EMG_ERR_INVALID, "max_iter < 0");
  if (!(tol >= 0.0)) raise(EMG_ERR_INVALID, "tol must be >= 0");
  if (workers < 0) raise(EMG_ERR_INVALID, "workers < 0");
  // Jobs whose handles share a stream (in particular jobs of one handle, which also share its
  // workspaces) run one after another on one worker: a stream is driven by one thread at a time,
  // and a cycle capture on it must not see another thread's launches.
  std::map<cudaStream_t, std::vector<int>> by_stream;
  std::vector<std::vector<int>> groups;
  for (int k = 0; k < count; ++k) {
    emg_ctx* c = checked(handles[k]);
    check_ptr(b[k], "b[k]");
    check_ptr(x[k], "x[k]");
    by_stream[c->st].push_back(k);
  }
  for (auto& kv : by_stream) groups.push_back(kv.second);
  // The largest systems first, so that the last ones to start are short.
  std::sort(groups.begin(), groups.end(), [&](const std::vector<int>& a, const std::vector<int>& g) {
    return handles[a[0]]->nvec() * a.size() > handles[g[0]]->nvec() * g.size();
  });
  const int nw = std::max(1, std::min<int>(workers > 0 ? workers : (int)groups.size(), std::min<int>((int)groups.size(), 64)));
  std::vector<emg_status> st(count, EMG_OK);
  std::vector<std::string> msg(count);
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int gi = next.fetch_add(1); gi < (int)groups.size(); gi = next.fetch_add(1)) {
      for (int k : groups[gi]) {
        emg_ctx& c = *handles[k];
        try {
          CK(cudaSetDevice(c.dev));
          emg_stats* sk = stats ? &stats[k] : nullptr;
          st[k] = c.prec == 32 ? solve_impl<float>(c, (const cx<double>*)b[k], (cx<double>*)x[k], tol, max_iter, restart, sk)
                               : solve_impl<double>(c, (const cx<double>*)b[k], (cx<double>*)x[k], tol, max_iter, restart, sk);
        } catch (const EmgError& e) {
          st[k] = e.s;
          msg[k] = e.msg;
        } catch (const std::bad_alloc&) {
          st[k] = EMG_ERR_NOMEM;
          msg[k] = "host allocation failed";
        } catch (const std::exception& e) {
          st[k] = EMG_ERR_INVALID;
          msg[k] = e.what();
        }
      }
    }
  };
  int dev0 = 0;
  CK(cudaGetDevice(&dev0));
  std::vector<std::thread> pool;
  pool.reserve(nw);
  try {
    for (int t = 1; t < nw; ++t) pool.emplace_back(work);
  } catch (...) {
    // fewer threads than asked for: the ones that started and the calling thread do the rest
  }
  work();  // the calling thread is one of the workers
  for (auto& t : pool) t.join();
  CK(cudaSetDevice(dev0));
  if (status)
    for (int k = 0; k < count; ++k) status[k] = st[k];
  // the first error (by job index) wins; otherwise EMG_NOT_CONVERGED if any job did not converge
  emg_status worst = EMG_OK;
  for (int k = 0; k < count; ++k) {
    if (st[k] != EMG_OK && st[k] != EMG_NOT_CONVERGED) {
      g_err = "job " + std::to_string(k) + ": " + msg[k];
      return st[k];
    }
    if (st[k] == EMG_NOT_CONVERGED) worst = EMG_NOT_CONVERGED;
  }
  return worst;
  ABI_CATCH
}

emg_status emg_solve_host(emg_handle h, const double* b_host, double* x_host, double tol, int max_iter, int restart,
                          emg_stats* stats) {
  NvtxRange nvtx_range("emg_solve_host");
  ABI_TRY
  emg_ctx& c = *checked(h);
  if (!b_host || !x_host) raise(EMG_ERR_INVALID, "host vector is NULL");
  const size_t bytes = c.nvec() * 16;
  if (c.hb_bytes < bytes) {
    c.hb.alloc(bytes);
    c.hx.alloc(bytes);
    c.hb_bytes = bytes;
  }
  CK(cudaMemcpyAsync(c.hb.p, b_host, bytes, cudaMemcpyHostToDevice, c.st));
  CK(cudaMemcpyAsync(c.hx.p, x_host, bytes, cudaMemcpyHostToDevice, c.st));
  emg_status s = emg_solve(h, c.hb.p, c.hx.p, tol, max_iter, restart, stats);
  if (s != EMG_OK && s != EMG_NOT_CONVERGED) return s;
  CK(cudaMemcpyAsync(x_host, c.hx.p, bytes, cudaMemcpyDeviceToHost, c.st));
  CK(cudaStreamSynchronize(c.st));
  return s;
  ABI_CATCH
}

emg_status emg_profile(emg_handle h, int enable) {
  ABI_TRY
  emg_ctx& c = *checked(h);
  prof_flush(c);
  c.prof = enable != 0;
  c.prof_coarse = enable == 2;
  ABI_CATCH
  return EMG_OK;
}

emg_status emg_profile_read(emg_handle h, int cls, double* total_ms, int64_t* launches, double* bytes) {
  ABI_TRY
  emg_ctx& c = *checked(h);
  if (cls < 0 || cls > EMG_K_ALL) raise(EMG_ERR_INVALID, "kernel class out of range");
  if (cls == EMG_K_ALL) {
    if (total_ms) *total_ms = 0.0;
    if (launches) *launches = c.launches;
    if (bytes) *bytes = 0.0;
    c.launches = 0;
    return EMG_OK;
  }
  prof_flush(c);
  if (total_ms) *total_ms = c.pms[cls];
  if (launches) *launches = c.pn[cls];
  if (bytes) *bytes = c.pbytes[cls];
  c.pms[cls] = 0;
  c.pn[cls] = 0;
  c.pbytes[cls] = 0;
  ABI_CATCH
  return EMG_OK;
}

}  // extern "C"
