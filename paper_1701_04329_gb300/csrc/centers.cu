// Leaf cell centres written straight into device memory (the device form of
// afg_cell_centers): a set-up kernel, not part of the solve.
#include <algorithm>

#include "grid.h"

namespace afg {

namespace {
// geo: per leaf box its lower corner (x, y, z) and cell size; cells of a box
// lexicographic with x fastest, boxes in canonical order, D values per cell
__global__ void k_cell_centers(const double *geo, int D, int N, long long ncells, double *xyz) {
    const long long per_box = D == 2 ? (long long)N * N : (long long)N * N * N;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncells;
         q += (long long)gridDim.x * blockDim.x) {
        const long long b = q / per_box;
        const int c = (int)(q - b * per_box);
        const int ci[3] = {c % N, (c / N) % N, c / (N * N)};
        const double *g = geo + 4 * b;
        for (int a = 0; a < D; ++a) xyz[q * D + a] = g[a] + (ci[a] + 0.5) * g[3];
    }
}
}  // namespace

void launch_cell_centers(const Grid &g, double *xyz, cudaStream_t s) {
    if (g.n_leaf_cells == 0) return;
    const int threads = 256;
    const long long want = (g.n_leaf_cells + threads - 1) / threads;
    const int blocks = (int)std::min<long long>(want, 152LL * 16);
    k_cell_centers<<<blocks, threads, 0, s>>>(g.d_leaf_geo, g.D, g.N, g.n_leaf_cells, xyz);
    ++g_launches;
    check(cudaGetLastError(), "k_cell_centers");
}

}  // namespace afg
