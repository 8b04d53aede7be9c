// Launchers of the stencil kernels; each dimension lives in its own translation unit
// (launch2d.cu, launch3d.cu) so that the library builds in parallel.
#pragma once
#include "emg.h"
#include "emg_types.cuh"
#include "apply_ff2d.cuh"
#include "apply_ff3d.cuh"
#include "kaczmarz.cuh"

#include <string>

// Sets the message that emg_last_error() returns on the calling thread.
void emg_set_last_error(const std::string& msg);
// The checks emg_create makes of one level's grid, coefficients, precision and smoother (not of
// the hierarchy): EMG_OK, or EMG_ERR_INVALID with the reason in *why.
emg_status emg_validate_level_params(const emg_params* p, std::string* why);

template <typename T, typename TI>
void launch_apply2(const Grid<T>& g, const cx<TI>* x, const cx<T>* b, T bscale, cx<T>* y, cudaStream_t st);
template <typename T>
void launch_vanka2(const Grid<T>& g, const cx<T>* b, const cx<T>* uin, cx<T>* uout, cx<T>* p, int colour, T w,
                   int zero_in, cudaStream_t st);
template <typename T>
void launch_restrict2(const Grid<T>& g, const cx<T>* b, const cx<T>* x, cx<T>* bc, const int nc[3], cx<T>* r,
                      cudaStream_t st);  // r: fine-level scratch of (d+1) n_x n_y values (the residual)  // r: fine-level scratch for the two-kernel path, or nullptr
template <typename T>
void launch_prolong2(const cx<T>* e, cx<T>* x, const int n[3], const int nc[3], cudaStream_t st);

template <typename T, typename TI>
void launch_apply3(const Grid<T>& g, const cx<TI>* x, const cx<T>* b, T bscale, cx<T>* y, cudaStream_t st);
template <typename T>
void launch_vanka3(const Grid<T>& g, const cx<T>* b, const cx<T>* uin, cx<T>* uout, cx<T>* p, int colour, T w,
                   int zero_in, cudaStream_t st);
template <typename T>
void launch_restrict3(const Grid<T>& g, const cx<T>* b, const cx<T>* x, cx<T>* bc, const int nc[3], cx<T>* r,
                      cudaStream_t st);  // r: fine-level scratch of (d+1) n_x n_y n_z values (the residual)
template <typename T>
void launch_prolong3(const cx<T>* e, cx<T>* x, const int n[3], const int nc[3], cudaStream_t st);

// The FP64 outer applies write y as complex doubles, or with ffo as float-float pairs (df::cff,
// the outer solve's internal Krylov vectors).
template <typename TI>
void launch_apply_ff2(const ff2::FineFF& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y, bool ffo,
                      cudaStream_t st);

// One full red-black sweep of a 2D FP32 level in one pass (k2t::sweep_tile): xin -> xout, which
// must be distinct buffers of (d+1) n_x n_y values; zero_in: xin is taken as zero and not read;
// e (nullptr: none): a coarse correction on the nxc x nyc grid added as xin + P e before the
// sweep (prolongation + correction fused into the first post-sweep).
// err: a device status word (bit 0 set if a tile load timed out). sweep_tile_fits says whether
// the grid and pointers meet the kernel's alignment rules (n_x a multiple of 4, 16-byte aligned
// buffers); otherwise the two half-sweep launches are used.
bool sweep_tile_fits(const Grid<float>& g, const void* b, const void* xin, const void* xout);
// ty: the tile height, 24 or 8 (more, smaller tiles for small grids).
cudaError_t launch_sweep_tile(const Grid<float>& g, const cx<float>* b, const cx<float>* xin, cx<float>* xout, float w,
                              int zero_in, const cx<float>* e, int nxc, int nyc, int ty, int* err, cudaStream_t st);

// b_c = R (b - H_s x) of a 2D FP32 level in one pass (k2t::resid_restrict_tile): no fine residual
// is written. Same tile geometry and alignment rules as launch_sweep_tile.
cudaError_t launch_resid_restrict_tile(const Grid<float>& g, const cx<float>* b, const cx<float>* x, cx<float>* bc,
                                       int nxc, int nyc, int ty, int* err, cudaStream_t st);

template <typename T>
cudaError_t launch_sweeps_coop2(const Grid<T>& g, const cx<T>* b, cx<T>* x, cx<T>* alt, int sweeps, T w,
                                int zero_first, cudaStream_t st);

template <typename TI>
void launch_apply_ff3(const ff3::FineFF3& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y, bool ffo,
                      cudaStream_t st);

template <typename TI>
void launch_apply_adjoint_ff3(const ff3::FineFF3& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y,
                              bool ffo, cudaStream_t st);

// Adjoint-state gradient (adjoint.cu): y = H^H x or y = bscale b - H^H x on the finest level,
// the per-cell material derivative, and z <- S conj(z) on an FP32 vector (nu displacement
// entries, then the pressure).
template <int D, typename TI>
void launch_adjoint_apply(const Grid<double>& g, const cx<TI>* x, const cx<double>* b, double bscale, void* y,
                          bool ffo, cudaStream_t st);
template <int D>
void launch_adjoint_gradient(const Grid<double>& g, const cx<double>* u, const cx<double>* a, double* glam,
                             double* gmu, double* grho, int accumulate, cudaStream_t st);
void launch_sconj(cx<float>* z, size_t nu, size_t n, cudaStream_t st);

// Hybrid Kaczmarz-GMRES coarsest solve (kaczmarz.cu / kaczmarz.cuh). launch_kz_probe fills the
// Schur rows (D N rows x NE entries, zero where a row has no column) and their inverse squared
// norms by probing the level operator of g; e and y are scratch vectors of (D+1) N values.
// plan_kz_solve sizes the cooperative launch (one block per SM, the warps whose private copies
// fit in shared memory); launch_kz_solve runs one solve described by a.
struct KzLaunch {
  int blocks = 0, warps = 0;
  size_t smem = 0;
  int fixb = 0;  // 2: the kernel built for boxes of 2 cells per axis; 0: any box
};
template <typename T>
cudaError_t launch_kz_probe(const Grid<T>& g, int dim, cx<T>* coef, T* inv_n2, cx<T>* e, cx<T>* y, cudaStream_t st);
template <typename T>
cudaError_t plan_kz_solve(int dim, int sms, int RS, const int box[3], KzLaunch& out);
template <typename T>
cudaError_t launch_kz_solve(const kz::Args<T>& a, int dim, const KzLaunch& L, cudaStream_t st);
