// Host build of the per-cell adjoint functions (adjoint.cuh), for CPU checks against the FP64
// oracle: the same source the GPU kernels run, looped over the cells on the host. Not part of
// the solve path; libemg_hostcheck.so holds no device code that runs.
#include "adjoint.cuh"

namespace {

Grid<double> host_grid(int dim, const int* n, double h, double beta, double omega, double att, double abl_len,
                       double abl_gmax, const double* mu, const double* rho, const double* cp) {
  Grid<double> g;
  g.nx = n[0];
  g.ny = n[1];
  g.nz = dim == 3 ? n[2] : 1;
  g.h = h;
  g.ih = 1.0 / h;
  g.beta = beta;
  g.sm = (1.0 - beta) / (2.0 * dim);
  g.w2 = omega * omega;
  g.att = att;
  g.ablL = abl_len;
  g.ablG = abl_gmax;
  g.Lx = n[0] * h;
  g.Ly = n[1] * h;
  g.Lz = dim == 3 ? n[2] * h : 0.0;
  g.mu = mu;
  g.rho = rho;
  g.cp = cp;
  g.abl_tab[0] = g.abl_tab[1] = g.abl_tab[2] = nullptr;
  return g;
}

template <int D>
void apply_all(const Grid<double>& g, const cx<double>* x, cx<double>* y) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const cx<double>* xs[4];
  for (int c = 0; c <= D; ++c) xs[c] = x + (size_t)c * N;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const size_t idx = adj::lin(g, i, j, k);
        for (int c = 0; c < D; ++c) y[(size_t)c * N + idx] = adj::row_u<D, double, double>(c, xs, g, i, j, k);
        y[(size_t)D * N + idx] = adj::row_p<D, double, double>(xs, g, i, j, k);
      }
}

template <int D>
void gradient_all(const Grid<double>& g, const cx<double>* u, const cx<double>* a, double* gl, double* gm, double* gr) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const cx<double>* us[4];
  const cx<double>* as[4];
  for (int c = 0; c <= D; ++c) {
    us[c] = u + (size_t)c * N;
    as[c] = a + (size_t)c * N;
  }
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const size_t idx = adj::lin(g, i, j, k);
        adj::gradient<D, double, double>(us, as, g, i, j, k, gl[idx], gm[idx], gr[idx]);
      }
}

}  // namespace

extern "C" {

// y = H^H x for complex128 x, y of (dim+1) * n_x n_y (n_z) values; att = gamma + shift.
int emg_hc_adjoint_apply(int dim, const int* n, double h, double beta, double omega, double att, double abl_len,
                         double abl_gmax, const double* mu, const double* rho, const double* cp, const double* x,
                         double* y) {
  const Grid<double> g = host_grid(dim, n, h, beta, omega, att, abl_len, abl_gmax, mu, rho, cp);
  if (dim == 2) apply_all<2>(g, (const cx<double>*)x, (cx<double>*)y);
  else if (dim == 3) apply_all<3>(g, (const cx<double>*)x, (cx<double>*)y);
  else return 1;
  return 0;
}

// -Re a^H (dH/dm) u per cell for m = lambda, mu, rho (unshifted operator: att = gamma).
int emg_hc_material_gradient(int dim, const int* n, double h, double beta, double omega, double att, double abl_len,
                             double abl_gmax, const double* mu, const double* rho, const double* cp, const double* u,
                             const double* a, double* glam, double* gmu, double* grho) {
  const Grid<double> g = host_grid(dim, n, h, beta, omega, att, abl_len, abl_gmax, mu, rho, cp);
  if (dim == 2) gradient_all<2>(g, (const cx<double>*)u, (const cx<double>*)a, glam, gmu, grho);
  else if (dim == 3) gradient_all<3>(g, (const cx<double>*)u, (const cx<double>*)a, glam, gmu, grho);
  else return 1;
  return 0;
}

}  // extern "C"
