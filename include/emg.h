/*
 * emg -- matrix-free shifted-Laplacian multigrid for the elastic Helmholtz equation in mixed
 * (u, p) form on a beta-spread staggered (MAC) grid, for one NVIDIA GB300 (sm_103a).
 *
 * Method: Yovel & Treister, "LFA-tuned matrix-free multigrid method for the elastic Helmholtz
 * equation" (arXiv 2307.03242). Section and equation numbers below refer to that paper.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid: n[0] x n[1] (x n[2]) cells of size h; x1 is the fastest-varying index; the last axis is
 * depth. A field vector holds dim+1 complex components (u_1, .., u_dim, p), each an array of
 * n[0]*n[1](*n[2]) complex numbers in that order (component-major, x1 fastest, real and
 * imaginary parts interleaved). u_d[k] is the displacement on the face normal to x_d on the LOW
 * side of cell k (position x_d = k_d h, cell-centred in the other coordinates); p[k] sits at the
 * cell centre (Section 2.3, Fig. 2.1). The faces u_d with k_d = 0 lie on the domain boundary and
 * are not unknowns: inputs there are ignored and outputs there are written as zero.
 *
 * Precision: "FP64 vector" = complex128 (2 x double per entry); "cycle vector" = complex64 when
 * the handle was created with cycle_precision = 32, complex128 when 64.
 *
 * Memory: unless an entry point says "host", every vector pointer is a DEVICE pointer on the
 * current CUDA device, owned by the caller, at least 16-byte aligned, and not aliased with any
 * other argument. The library owns the hierarchy (material copies, level vectors, Krylov basis);
 * it allocates all of it in emg_create and frees it in emg_destroy.
 *
 * Streams: every call is ordered on the stream given to emg_create and returns without
 * synchronising the stream, except where stated (emg_solve and emg_solve_host synchronise,
 * because the Krylov loop reads reductions on the host).
 *
 * Errors: no exception crosses the ABI. Every call returns an emg_status; on failure
 * emg_last_error() returns a message for the calling thread. Invalid arguments are rejected
 * before any work is enqueued.
 */
#ifndef EMG_H
#define EMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EMG_MAX_LEVELS 10

typedef struct emg_ctx* emg_handle;

typedef enum {
  EMG_OK = 0,
  EMG_ERR_INVALID = 1,    /* bad argument, unsupported size, non-finite or non-positive material */
  EMG_ERR_NOMEM = 2,      /* device allocation failed */
  EMG_ERR_CUDA = 3,       /* a CUDA call failed (message from the runtime) */
  EMG_ERR_NONFINITE = 4,  /* NaN/Inf met in a Krylov reduction */
  EMG_NOT_CONVERGED = 5,  /* emg_solve stopped at max_iter; x holds the last iterate */
  EMG_ERR_TIMEOUT = 6     /* reserved for bounded device-side waits */
} emg_status;

/* Coarsest-level solvers (Sec. 3.2): EMG_COARSE_DENSE, the exact solve (the paper's 2D choice);
 * EMG_COARSE_SMOOTH, coarse_sweeps red-black Vanka sweeps from zero; EMG_COARSE_KACZMARZ, the
 * paper's 3D choice (Sec. 3.2, 5.3): FGMRES on the Schur complement that eliminates p (the p-p
 * block is diagonal), preconditioned by parallel hybrid Kaczmarz steps, until a relative drop of
 * the Schur residual (the kaczmarz_* and coarse_* fields of emg_params). */
enum { EMG_COARSE_DENSE = 0, EMG_COARSE_SMOOTH = 1, EMG_COARSE_KACZMARZ = 2 };
enum { EMG_CYCLE_V = 0, EMG_CYCLE_W = 1, EMG_CYCLE_K = 2 };
enum { EMG_VANKA_FULL = 0, EMG_VANKA_ECONOMIC = 1 };
/* How a level's red-black sweeps run (emg_params.sweep_path). EMG_SWEEP_AUTO: chosen per level at
 * creation by timing the candidates below on the level's own buffers (cached per device, grid
 * size and sweep count for the life of the process). The others force one path on every 2D FP32
 * level that can take it (the others keep their automatic choice): EMG_SWEEP_HALF: one launch per
 * colour; EMG_SWEEP_COOP: all sweeps of a call in one cooperative launch; EMG_SWEEP_TILE24 /
 * EMG_SWEEP_TILE8 / EMG_SWEEP_TILE4: one launch per sweep, both colours in shared-memory tiles of
 * 60 x 24 / 60 x 8 / 60 x 4 cells (n[0] of the level a multiple of 4; the smaller tiles give
 * small levels more blocks with shorter latency chains). Every path computes the same sweeps
 * (Sec. 3.2); FP32 rounding differs. FP64 cycles and 3D levels ignore the field. */
enum {
  EMG_SWEEP_AUTO = 0,
  EMG_SWEEP_HALF = 1,
  EMG_SWEEP_COOP = 2,
  EMG_SWEEP_TILE24 = 3,
  EMG_SWEEP_TILE8 = 4,
  EMG_SWEEP_TILE4 = 5
};

/* Solver description. All lengths in the same unit as h. */
typedef struct {
  int32_t dim;              /* 2 or 3 */
  int32_t n[3];             /* cells per axis (x1 first); every n[a] divisible by 2^(levels-1) */
  double h;                 /* finest cell size */
  double omega;             /* angular frequency (Eq. 2.1) */
  double gamma;             /* physical attenuation of the unshifted operator (Sec. 5: 0.01) */
  double alpha;             /* complex shift of the cycle operator, added to gamma (Eq. 2.9) */
  double beta;              /* stencil spread weight, Eq. 3.2-3.5 (LFA-tuned: 2/3) */
  int32_t abl_cells;        /* absorbing layer thickness in finest cells, on all sides (0: none) */
  double abl_gamma_max;     /* attenuation added at the outer boundary; profile gamma_max*(d/L)^2 */
  int32_t levels;           /* multigrid levels, 1..EMG_MAX_LEVELS */
  int32_t nu_pre, nu_post;  /* pre- and post-smoothing sweeps (Alg. 1) */
  double damping[EMG_MAX_LEVELS]; /* Vanka damping w per level; 0 selects the default by depth */
  int32_t coarse_solver;    /* EMG_COARSE_DENSE (exact, host LU) or EMG_COARSE_SMOOTH */
  int32_t coarse_sweeps;    /* red-black sweeps on the coarsest level for EMG_COARSE_SMOOTH */
  double coarse_damping;    /* Vanka damping on the coarsest level for EMG_COARSE_SMOOTH */
  int32_t cycle_precision;  /* 32: FP32 cycle with FP64 outer solve; 64: everything in FP64 */
  int32_t cycle_type;       /* EMG_CYCLE_V (one recursive call, Alg. 1), EMG_CYCLE_W (two calls, the
                               second from the first one's result; Sec. 2.2, the paper's 2D choice)
                               or EMG_CYCLE_K (the two calls precondition two GCR steps for the coarse
                               problem; Sec. 2.2, the paper's 3D choice); the coarsest level is
                               solved once per visit */
  double level_alpha[EMG_MAX_LEVELS]; /* shift of level l's cycle operator when > 0, else alpha (the
                               paper raises the shift as levels are added, Sec. 5.2; a deeper shift on
                               the coarsest level keeps its smoothing iteration convergent) */
  int32_t smoother;         /* EMG_VANKA_FULL: each cell's whole (2d+1)^2 block is inverted (the
                               paper's solves); EMG_VANKA_ECONOMIC: its displacement part is replaced
                               by its diagonal (the paper's LFA variant, Sec. 2.3), in red-black
                               order here */
  int32_t sweep_path;       /* EMG_SWEEP_*: how the sweeps of 2D FP32 levels run (0: autotuned) */
  /* EMG_COARSE_KACZMARZ (Sec. 3.2, 5.3). The Schur system S u = f is solved by FGMRES(coarse_restart)
   * from zero, each preconditioner application being kaczmarz_steps parallel hybrid Kaczmarz steps
   * from zero with damping kaczmarz_damping: the coarsest cells are divided into boxes of
   * kaczmarz_box cells per axis; every box sweeps its faces' rows (component by component, x
   * fastest) with damped row projections on a private copy of the unknowns its rows reach (the box
   * dilated by 2 cells below, 1 along the component's own axis, and 1 cell above), all boxes from
   * the same iterate, and each unknown becomes the mean of the boxes' copies of it. The solve stops
   * when ||f - S u|| <= coarse_tol ||f|| or after kaczmarz_max / kaczmarz_steps FGMRES iterations.
   * Zero selects the paper's value: restart 5, 10 steps, damping 0.8, drop 0.1, at most 250 steps.
   * kaczmarz_box: all 0 (automatic: the smallest cube of 2, 4, ... cells whose boxes the GPU can
   * all sweep at once), all 1, or each in 2..64. coarse_restart <= 8; kaczmarz_damping in
   * (0, 2). */
  int32_t kaczmarz_box[3];
  int32_t kaczmarz_steps;
  double kaczmarz_damping;
  double coarse_tol;
  int32_t coarse_restart;
  int32_t kaczmarz_max;
} emg_params;

typedef struct {
  int32_t iterations;       /* preconditioned FGMRES iterations (= V-cycles) */
  int32_t restarts;
  double rel_residual;      /* true ||b - H x||_2 / ||b||_2 at exit, in FP64 */
  double* history;          /* optional, caller-owned host array: estimated relative residual
                               after each iteration (history[0] = initial) */
  int32_t history_cap;      /* capacity of history (0: none) */
  int32_t history_len;      /* entries written */
} emg_stats;

/* Build the multigrid hierarchy (Sec. 3.2: re-discretisation on every level; coarse media are
 * the mean of the 2^dim children). lam, mu, rho: FP64 cell-centred arrays of n[0]*n[1](*n[2])
 * values, on the host (on_device = 0) or on the device (on_device = 1); they are copied.
 * cuda_stream: a cudaStream_t, or NULL for the legacy default stream.
 * Rejects: dim not 2/3; n not divisible by 2^(levels-1); a coarsest grid below 2 cells per
 * axis; non-finite or non-positive mu, rho, lam+mu; EMG_COARSE_DENSE with more than 4096
 * coarsest unknowns; EMG_COARSE_KACZMARZ settings out of range (a box's private copy must fit in
 * 200 KB of shared memory). On success *out is a new handle. */
emg_status emg_create(const emg_params* params, const double* lam, const double* mu,
                      const double* rho, int on_device, void* cuda_stream, emg_handle* out);

/* Free every device and host resource of the handle. NULL is accepted. */
emg_status emg_destroy(emg_handle h);

/* Message describing the last failure on the calling thread ("" if none). */
const char* emg_last_error(void);

/* y = H x (shifted = 0) or y = H_s x (shifted = 1) on the finest level in FP64, Eq. 3.10 with the
 * sign of Eq. 4.4; H_s adds alpha to the attenuation (Eq. 2.9). x, y: FP64 vectors. */
emg_status emg_apply(emg_handle h, int shifted, const void* x, void* y);

/* x <- one V(nu_pre, nu_post)-cycle (or W-cycle, per cycle_type) for H_s x = b on the finest
 * level (Alg. 1 applied recursively). zero_guess = 1 ignores the input x. b, x: cycle vectors. */
emg_status emg_vcycle(emg_handle h, const void* b, void* x, int zero_guess);

/* Solve H x = b (unshifted, FP64) by right-preconditioned restarted FGMRES(restart) with one
 * V-cycle as preconditioner (Sec. 3.2, 5). x: in = initial guess, out = solution. Stops when the
 * true relative residual ||b - H x|| / ||b|| <= tol or after max_iter iterations
 * (EMG_NOT_CONVERGED; x then holds the last iterate). restart in 1..64. b, x: FP64 vectors.
 * stats may be NULL. Synchronises the stream. On a stream other than the legacy default stream
 * the preconditioner cycle is captured into a CUDA graph on the second use of each Krylov slot
 * and replayed from then on (same kernels, bitwise the same result); while profiling is on, or
 * if a capture fails, it runs launch by launch. So no other thread may launch work into the
 * handle's stream during the call. */
emg_status emg_solve(emg_handle h, const void* b, void* x, double tol, int max_iter, int restart,
                     emg_stats* stats);

/* emg_solve with HOST vectors: b_host and x_host are host arrays of (dim+1)*ncell complex128
 * (pinned or pageable). The copies to and from the device are part of the call. */
emg_status emg_solve_host(emg_handle h, const double* b_host, double* x_host, double tol,
                          int max_iter, int restart, emg_stats* stats);

/* A batch of independent solves, each exactly emg_solve(handles[k], b[k], x[k], ...): many
 * grids, media, frequencies or sources at once (the batched use the paper's Sec. 5 experiments
 * imply -- one solve per source and frequency -- but do not describe; no counterpart in the
 * paper's solver itself). Small grids cannot fill the GPU on their own, so the solves run
 * concurrently: up to `workers` host threads (0: one per distinct stream, at most 64) each drive
 * the solves of one stream's handles, and the GPU interleaves the kernels of the streams. Give
 * every handle its own stream to get the overlap; jobs whose handles share a stream, and
 * repeated handles (several right-hand sides of one system), run one after another on one
 * worker. b[k], x[k]: FP64 device vectors of
 * handle k's size; stats and status: arrays of count entries, or NULL. Returns EMG_OK, the first
 * (lowest k) error, or EMG_NOT_CONVERGED if any job stopped at max_iter; status[k] holds each
 * job's own result. The handles must not be used by other threads during the call. */
emg_status emg_solve_batch(const emg_handle* handles, int count, const void* const* b,
                           void* const* x, double tol, int max_iter, int restart,
                           emg_stats* stats, int workers, emg_status* status);

/* ---- Adjoint-state gradient (frequency-domain inversion; the adjoint-state method, e.g.
 * Plessix 2006; the paper's solver is the forward solver of such an inversion, Sec. 1 and 5). ----
 * For a data misfit J = 1/2 sum_s |S u_s - d_s|^2 with u_s = H^-1 q_s, the gradient with respect
 * to the cell fields is -Re sum_s a_s^H (dH/dm) u_s with the adjoint fields a_s = H^-H S^T
 * (S u_s - d_s). H is the unshifted finest-level operator of this handle. Vectors are FP64
 * complex device vectors of (dim+1)*ncell values in the layout of emg_apply. */

/* y = H^H x (conjugate transpose of the unshifted operator), FP64. */
emg_status emg_apply_adjoint(emg_handle h, const void* x, void* y);

/* Solve H^H x = b by the FGMRES of emg_solve with H^H as the operator. The preconditioner is
 * the handle's cycle mapped through z = S conj(M(conj(S r))), S = diag(I, -I) (displacements
 * kept, pressure negated): with beta = 1 the operator satisfies H^H = S conj(H) S exactly, with
 * the beta-spread stencils up to the spread of the coupling blocks, so the mapped cycle is a
 * close preconditioner. Requires cycle_precision 32 (EMG_ERR_INVALID otherwise); arguments,
 * statuses and stats as emg_solve. */
emg_status emg_solve_adjoint(emg_handle h, const void* b, void* x, double tol, int max_iter,
                             int restart, emg_stats* stats);

/* Per cell k: g_lam[k] = -Re a^H (dH/dlambda_k) u, and likewise g_mu, g_rho (FP64 device
 * arrays of ncell values, cell index x fastest). accumulate != 0 adds to the arrays (summing
 * over sources); otherwise they are overwritten. u: forward field, a: adjoint field. */
emg_status emg_material_gradient(emg_handle h, const void* u, const void* a, double* g_lam,
                                 double* g_mu, double* g_rho, int accumulate);

/* ---- Per-step entry points (one row of the cycle each; used for parity checks). ----
 * `level` 0 is the finest. Vectors are cycle vectors of that level's size. */

/* Grid of a level: cells per axis and cell size. */
emg_status emg_level_info(emg_handle h, int level, int32_t n[3], double* cell_size);

/* x <- `sweeps` red-black full Vanka sweeps on H_s of `level` (Sec. 2.3, 3.2): colour 0 then
 * colour 1, each cell's (2d+1)x(2d+1) block solved exactly and damped by the level's w. */
emg_status emg_smooth(emg_handle h, int level, const void* b, void* x, int sweeps);

/* b_coarse <- R (b - H_s x) from `level` to level+1 (Eq. 2.11-2.13, Alg. 1 step 2). */
emg_status emg_residual_restrict(emg_handle h, int level, const void* b, const void* x,
                                 void* b_coarse);

/* x <- x + P e_coarse from level+1 to `level` (Eq. 2.11-2.13, Alg. 1 step 4). */
emg_status emg_prolong_correct(emg_handle h, int level, const void* e_coarse, void* x);

/* x <- coarsest-level solve of H_s x = b (exact for EMG_COARSE_DENSE, coarse_sweeps red-black
 * sweeps from zero for EMG_COARSE_SMOOTH, the hybrid Kaczmarz-GMRES solve for
 * EMG_COARSE_KACZMARZ). b, x: cycle vectors of the coarsest level. */
emg_status emg_coarse_solve(emg_handle h, const void* b, void* x);

/* EMG_COARSE_KACZMARZ diagnostics (Sec. 3.2, 5.3). emg_coarse_stats synchronises the handle's
 * stream and writes, for the last coarsest solve: out[0] FGMRES iterations, out[1] the relative
 * Schur residual ||f - S u|| / ||f|| at exit, out[2] Kaczmarz steps spent. emg_coarse_schur_rows
 * copies the stored Schur rows to the caller's host buffer: dim N_c rows (component-major, x
 * fastest; N_c coarsest cells), each of 75 (3D) or 17 (2D) complex entries in the cycle precision,
 * over the row's footprint: for c2 = 0 .. dim-1, offsets o along each axis a from -2 (a = c != c2),
 * 0 (a = c2 != c) or -1 (otherwise) to +1, x fastest; entries outside the grid or on boundary
 * faces are 0, and rows of boundary faces are all 0. EMG_ERR_INVALID for other coarse solvers. */
emg_status emg_coarse_stats(emg_handle h, double out[3]);
emg_status emg_coarse_schur_rows(emg_handle h, void* rows_host);

/* ---- Instrumentation. ----
 * While enabled, the library records a CUDA event pair on its stream around every launch of
 * the listed kernel classes on the finest level (enable = 1), and with enable = 2 also around
 * every launch on the coarser levels, which count as EMG_K_COARSE. emg_profile_read synchronises the stream and
 * returns the summed event time, the launch count and the algorithmic bytes of those launches,
 * then resets the counters. kernel_class is one of EMG_K_* (EMG_K_ALL: launch count only). */
enum { EMG_K_SMOOTH = 0, EMG_K_RESTRICT = 1, EMG_K_PROLONG = 2, EMG_K_APPLY64 = 3,
       EMG_K_KRYLOV = 4, EMG_K_COARSE = 5 /* every kernel of the levels below the finest (enable = 2) */,
       EMG_K_COUNT = 6,
       EMG_K_ALL = 6 /* emg_profile_read(EMG_K_ALL): launches = every kernel launched by the handle
                        on any level since the last read (counted even when profiling is off) */ };
emg_status emg_profile(emg_handle h, int enable);
emg_status emg_profile_read(emg_handle h, int kernel_class, double* total_ms, int64_t* launches,
                            double* bytes);

/* The sweep path level `level` took (EMG_SWEEP_HALF .. EMG_SWEEP_TILE4) and, when it was chosen
 * by timing, the measured time of one smoothing call of the level in microseconds (else 0).
 * No counterpart in the paper: it reports the autotuner's choice. */
emg_status emg_sweep_path(emg_handle h, int level, int32_t* path, double* us_per_call);

/* ---- Allocation-free smoothing. ----
 * No counterpart in the paper: this entry point exists for callers that cannot allocate device
 * memory -- code that runs while a stream is being captured into a CUDA graph and must not
 * allocate, applications whose device memory is fully reserved by their own allocator, and hosts
 * that embed a fixed-size smoother. It performs exactly what emg_smooth does on level 0 of the
 * hierarchy that `params` describes (2D, FP32 cycle vectors): `sweeps` red-black full Vanka
 * sweeps on H_s x = b, with the damping damping[0] (or the default by depth) and the shift
 * level_alpha[0] (or alpha). It needs no handle and allocates nothing: the caller passes the
 * finest-level material in FP32 -- mu, rho and cp = 1/(lambda + mu), n[0]*n[1] device values each
 * -- and b, x (FP32 cycle vectors, device, 16-byte aligned); the only work array, the ping-pong
 * copy of the displacement components, is a fixed file-scope device array of
 * 2 * EMG_NOALLOC_MAX_CELLS complex FP32 values (4 MiB), which every GPU that loads the library
 * holds until the process exits.
 * Limits and behaviour: level parameters that emg_create would reject (h, omega, gamma, alpha,
 * beta, level_alpha, abl_cells, levels, ...), a non-finite damping[0] or abl_gamma_max, grids with more
 * than EMG_NOALLOC_MAX_CELLS cells, dim != 2 or cycle_precision != 32 are rejected with
 * EMG_ERR_INVALID before any work. The first call on a device looks up the device address of the
 * work array (cudaGetSymbolAddress); make that first call before any stream capture. The address
 * is cached per device and context: after a device reset (cudaDeviceReset) or any other teardown
 * of the context, the next call looks it up again, so that call, too, belongs before any stream
 * capture. Every call shares the one work array: calls that overlap on the
 * GPU (different streams, or other threads) race and give wrong results; serialise them. The
 * array keeps the last call's contents; nothing in it needs to start at zero, because each
 * sweep's first half writes every entry before the second half reads it. Enqueued on
 * cuda_stream (NULL: the legacy default stream); returns without synchronising. */
#define EMG_NOALLOC_MAX_CELLS 262144
emg_status emg_smooth_noalloc(const emg_params* params, const float* mu, const float* rho,
                              const float* cp, const void* b, void* x, int sweeps,
                              void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* EMG_H */
