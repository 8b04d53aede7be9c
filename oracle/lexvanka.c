/* Lexicographic block relaxation for the oracle (test infrastructure only; never linked into the
 * product library).
 *
 * One sweep visits the cells in lexicographic order (x1 fastest) and relaxes each one at once:
 *   x[dofs(c)] += w * Vinv(c) * (b - H x)[dofs(c)]
 * with the residual taken from the CURRENT x, so a cell sees the updates of the cells before it
 * (Gauss-Seidel over cells; the paper's lexicographic Vanka of Sec. 3.2). H is the assembled
 * operator in CSR form; complex numbers are stored as interleaved (re, im) doubles. Vinv(c) is
 * the inverse of the cell's local block (full or economic), computed by the caller. dofs(c) lists
 * the cell's k degrees of freedom; -1 marks one that is not an unknown (its correction is zero). */
#include <stddef.h>

void lex_block_sweep(int ncell, int k, const int* dofs, const double* vinv, const int* indptr, const int* indices,
                     const double* data, const double* b, double* x, double w) {
  double r[2 * 16], d[2 * 16];
  for (int c = 0; c < ncell; ++c) {
    const int* dc = dofs + (size_t)c * k;
    for (int a = 0; a < k; ++a) {
      r[2 * a] = r[2 * a + 1] = 0.0;
      const int row = dc[a];
      if (row < 0) continue;
      double re = b[2 * (size_t)row], im = b[2 * (size_t)row + 1];
      for (int j = indptr[row]; j < indptr[row + 1]; ++j) {
        const double hr = data[2 * (size_t)j], hi = data[2 * (size_t)j + 1];
        const double xr = x[2 * (size_t)indices[j]], xi = x[2 * (size_t)indices[j] + 1];
        re -= hr * xr - hi * xi;
        im -= hr * xi + hi * xr;
      }
      r[2 * a] = re;
      r[2 * a + 1] = im;
    }
    const double* V = vinv + (size_t)c * k * k * 2;
    for (int a = 0; a < k; ++a) {
      double re = 0.0, im = 0.0;
      for (int e = 0; e < k; ++e) {
        const double vr = V[2 * (a * k + e)], vi = V[2 * (a * k + e) + 1];
        re += vr * r[2 * e] - vi * r[2 * e + 1];
        im += vr * r[2 * e + 1] + vi * r[2 * e];
      }
      d[2 * a] = re;
      d[2 * a + 1] = im;
    }
    for (int a = 0; a < k; ++a) {
      const int row = dc[a];
      if (row < 0) continue;
      x[2 * (size_t)row] += w * d[2 * a];
      x[2 * (size_t)row + 1] += w * d[2 * a + 1];
    }
  }
}
