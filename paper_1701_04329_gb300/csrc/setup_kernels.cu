// Set-up kernels, not part of the solve: leaf cell centres written straight
// into device memory (the device form of afg_cell_centers), and the FP32
// copy of a field (the coefficient of the variable-coefficient operators).
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
// refinement flags from a leaf field f: +1 where |f| h^power > tau_refine,
// -1 where |f| h^power < tau_coarsen, 0 elsewhere (h the cell size)
__global__ void k_flag(const double *geo, int D, int N, long long ncells, const double *f, int power, double tau_ref,
                       double tau_de, signed char *flags) {
    const long long per_box = D == 2 ? (long long)N * N : (long long)N * N * N;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncells;
         q += (long long)gridDim.x * blockDim.x) {
        const double h = geo[4 * (q / per_box) + 3];
        double hp = 1.0;
        for (int e = 0; e < power; ++e) hp *= h;
        const double v = fabs(f[q]) * hp;
        flags[q] = v > tau_ref ? 1 : (v < tau_de ? -1 : 0);
    }
}

__global__ void k_to_f32(const double *src, float *dst, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        dst[q] = (float)src[q];
}
}  // namespace

void launch_to_f32(const double *src, float *dst, long long n, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    k_to_f32<<<blocks, 256, 0, s>>>(src, dst, n);
    ++g_launches;
    check(cudaGetLastError(), "k_to_f32");
}

void launch_flag(const Grid &g, const double *f, int power, double tau_ref, double tau_de, signed char *flags,
                 cudaStream_t s) {
    if (g.n_leaf_cells == 0) return;
    const int blocks = (int)std::min<long long>((g.n_leaf_cells + 255) / 256, 152LL * 16);
    k_flag<<<blocks, 256, 0, s>>>(g.d_leaf_geo, g.D, g.N, g.n_leaf_cells, f, power, tau_ref, tau_de, flags);
    ++g_launches;
    check(cudaGetLastError(), "k_flag");
}

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
