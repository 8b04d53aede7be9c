/* One step of the parallel hybrid Kaczmarz method (oracle; test infrastructure only).
 *
 * Sections 3.2 and 5.3 (coarsest grid solution), after Gordon and Gordon's component-averaged
 * row projections: the rows of the system are divided among sub-regions. Every sub-region takes
 * its own copy of the unknowns in its reach (a declared set that holds every unknown its rows
 * touch), runs one Kaczmarz sweep over its rows in the given order on that copy, starting from the
 * same iterate x as all other sub-regions (the sub-regions are independent, i.e. parallel), and
 * every unknown is then set to the mean of the copies of the sub-regions whose reach holds it;
 * unknowns in no reach keep their value.
 * The Kaczmarz update of row i with damping w, for complex rows a_i:
 *     x <- x + w (rhs_i - a_i x) / ||a_i||^2 conj(a_i)^T
 * (for w = 1 the orthogonal projection onto the row's hyperplane a_i x = rhs_i).
 *
 * Matrix in CSR with complex values interleaved (re, im); vectors likewise. Plain loops, no
 * blocking or reordering. work, acc: 2 * ncols doubles; cnt, mark: ncols ints (scratch).
 * Returns 0, or -1 if a row touches an unknown outside its sub-region's reach. */
#include <string.h>

int carp_step(int ncols, const int* rp, const int* ci, const double* v, const double* rhs, double* x, int nparts,
              const int* part_ptr, const int* part_rows, const int* reach_ptr, const int* reach_cols, double w,
              double* work, double* acc, int* cnt, int* mark) {
  memset(acc, 0, sizeof(double) * 2 * (size_t)ncols);
  memset(cnt, 0, sizeof(int) * (size_t)ncols);
  for (int j = 0; j < ncols; ++j) mark[j] = -1;
  for (int p = 0; p < nparts; ++p) {
    /* the sub-region's copy of its reach, taken from x */
    for (int t = reach_ptr[p]; t < reach_ptr[p + 1]; ++t) {
      const int j = reach_cols[t];
      mark[j] = p;
      work[2 * j] = x[2 * j];
      work[2 * j + 1] = x[2 * j + 1];
    }
    for (int t = part_ptr[p]; t < part_ptr[p + 1]; ++t) {
      const int i = part_rows[t];
      double rr = rhs[2 * i], ri = rhs[2 * i + 1], nn = 0.0;
      for (int q = rp[i]; q < rp[i + 1]; ++q) {
        const int j = ci[q];
        if (mark[j] != p) return -1;
        const double ar = v[2 * q], ai = v[2 * q + 1];
        rr -= ar * work[2 * j] - ai * work[2 * j + 1];
        ri -= ar * work[2 * j + 1] + ai * work[2 * j];
        nn += ar * ar + ai * ai;
      }
      if (nn == 0.0) continue;
      const double sr = w * rr / nn, si = w * ri / nn;
      /* work += s conj(a) */
      for (int q = rp[i]; q < rp[i + 1]; ++q) {
        const int j = ci[q];
        const double ar = v[2 * q], ai = -v[2 * q + 1];
        work[2 * j] += sr * ar - si * ai;
        work[2 * j + 1] += sr * ai + si * ar;
      }
    }
    for (int t = reach_ptr[p]; t < reach_ptr[p + 1]; ++t) {
      const int j = reach_cols[t];
      acc[2 * j] += work[2 * j];
      acc[2 * j + 1] += work[2 * j + 1];
      cnt[j] += 1;
    }
  }
  for (int j = 0; j < ncols; ++j)
    if (cnt[j] > 0) {
      x[2 * j] = acc[2 * j] / cnt[j];
      x[2 * j + 1] = acc[2 * j + 1] / cnt[j];
    }
  return 0;
}
