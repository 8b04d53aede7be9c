// Red-black Vanka sweeps of one small 2D level in a single cooperative launch.
//
// On small grids (the coarsest level, and the levels just above it) a half-sweep has too few
// cells to fill the GPU, so separate launches per half-sweep are dominated by launch and drain
// latency. Here all co-resident blocks run every half-sweep and meet at a grid-wide barrier
// between half-sweeps (the next colour reads the faces the previous one wrote). Arithmetic:
// vanka_cell, i.e. the same as emg_smooth; u and p, written by other blocks of this launch, are
// read through L2 (COH), never through the read-only path.
#pragma once
#include <cooperative_groups.h>

#include "vanka2d_fast.cuh"

namespace k2 {

// sweeps full red-black sweeps; zero_first: x enters as zero (the first half-sweep then reads
// neither x nor the ping-pong copy).
template <typename T>
__global__ void __launch_bounds__(BX * BY) sweeps_coop(Grid<T> g, const cx<T>* __restrict__ b, cx<T>* x, cx<T>* alt,
                                                       int sweeps, T w, int zero_first) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int nx = g.nx, ny = g.ny;
  const size_t N = (size_t)nx * ny;
  const int npx = (nx + 1) / 2;
  const long long items = (long long)npx * ny;
  const int nthreads = blockDim.x * blockDim.y;
  const long long tid = (long long)blockIdx.x * nthreads + threadIdx.y * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * nthreads;
  for (int s = 0; s < sweeps; ++s) {
    for (int colour = 0; colour < 2; ++colour) {
      const cx<T>* uin = colour == 0 ? x : alt;
      cx<T>* uout = colour == 0 ? alt : x;
      const int zin = (zero_first && s == 0 && colour == 0) ? 1 : 0;
      for (long long it = tid; it < items; it += stride) {
        const int ip = (int)(it % npx), j = (int)(it / npx);
        vanka_cell<T, false, false, true>(g, b, uin, uout, x + 2 * N, colour, w, zin, ip, j);
      }
      grid.sync();
    }
  }
}

}  // namespace k2
