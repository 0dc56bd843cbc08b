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

// Volume-weighted sums over the leaves, deterministic (fixed grid, fixed
// reduction order).  Pass 1: block k sums over leaf boxes k, k + grid, ...:
// h^D f (f in the box layout), h^D, and h^(D-1) b over the Neumann faces of
// the leaves (bc != null).  Pass 2 (one block) adds the partials in order.
constexpr int kSumBlocks = 1024;

__device__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void k_leaf_vsum(BoxMeta A, const int *leaves, int nleaf, const double *geo, int D, int N,
                            const double *f, const double *bc, double *partials) {
    __shared__ double sh[256];
    const int C = D == 2 ? N * N : N * N * N, F = D == 2 ? N : N * N;
    double sf = 0.0, sv = 0.0, sb = 0.0;
    for (int li = blockIdx.x; li < nleaf; li += gridDim.x) {
        const double h = geo[4 * li + 3];
        const double vol = D == 2 ? h * h : h * h * h, area = D == 2 ? h : h * h;
        const int b = leaves[li];
        const long long cb = A.coff[b];
        for (int q = threadIdx.x; q < C; q += blockDim.x) sf += vol * f[cb + q];
        if (threadIdx.x == 0) sv += vol * C;
        if (bc)
            for (int s = 0; s < 2 * D; ++s)
                if ((A.nmask[b] >> s) & 1)
                    for (int q = threadIdx.x; q < F; q += blockDim.x) sb += area * bc[A.bcoff[b * 2 * D + s] + q];
    }
    sf = block_sum(sf, sh);
    sv = block_sum(sv, sh);
    sb = block_sum(sb, sh);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x] = sf;
        partials[3 * blockIdx.x + 1] = sv;
        partials[3 * blockIdx.x + 2] = sb;
    }
}

// out = (sum f - sum b) / sum vol
__global__ void k_vsum_final(const double *partials, int nb, double *out) {
    __shared__ double sh[256];
    double sf = 0.0, sv = 0.0, sb = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        sf += partials[3 * k];
        sv += partials[3 * k + 1];
        sb += partials[3 * k + 2];
    }
    sf = block_sum(sf, sh);
    sv = block_sum(sv, sh);
    sb = block_sum(sb, sh);
    if (threadIdx.x == 0) *out = (sf - sb) / sv;
}

// f -= *c on the leaf boxes (box layout)
__global__ void k_leaf_shift(BoxMeta A, const int *leaves, int nleaf, int C, double *f, const double *c) {
    const double v = *c;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)nleaf * C;
         e += (long long)gridDim.x * blockDim.x) {
        const int li = (int)(e / C), q = (int)(e - (long long)li * C);
        f[A.coff[leaves[li]] + q] -= v;
    }
}

// Forests: block t forms tree t's constant from its own leaves, in a fixed
// order (0 for a tree with a Dirichlet side, or one masked out by active).
__global__ void k_tree_vsum(BoxMeta A, const int *leaves, const int *leaf0, const char *sing, const int *active,
                            const double *geo, int D, int N, const double *f, const double *bc, double *c) {
    __shared__ double sh[256];
    const int t = blockIdx.x;
    const bool on = sing[t] && (!active || active[t]);
    const int C = D == 2 ? N * N : N * N * N, F = D == 2 ? N : N * N;
    double sf = 0.0, sv = 0.0, sb = 0.0;
    if (on)
        for (int li = leaf0[t]; li < leaf0[t + 1]; ++li) {
            const double h = geo[4 * li + 3];
            const double vol = D == 2 ? h * h : h * h * h, area = D == 2 ? h : h * h;
            const int b = leaves[li];
            const long long cb = A.coff[b];
            for (int q = threadIdx.x; q < C; q += blockDim.x) sf += vol * f[cb + q];
            if (threadIdx.x == 0) sv += vol * C;
            if (bc)
                for (int s = 0; s < 2 * D; ++s)
                    if ((A.nmask[b] >> s) & 1)
                        for (int q = threadIdx.x; q < F; q += blockDim.x) sb += area * bc[A.bcoff[b * 2 * D + s] + q];
        }
    sf = block_sum(sf, sh);
    sv = block_sum(sv, sh);
    sb = block_sum(sb, sh);
    if (threadIdx.x == 0) c[t] = on ? (sf - sb) / sv : 0.0;
}

// f -= c[tree] on the leaf boxes (box layout)
__global__ void k_tree_shift(BoxMeta A, const int *leaves, int nleaf, int C, double *f, const double *c) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)nleaf * C;
         e += (long long)gridDim.x * blockDim.x) {
        const int li = (int)(e / C), q = (int)(e - (long long)li * C);
        const int b = leaves[li];
        const double v = c[A.tree[b]];
        if (v != 0.0) f[A.coff[b] + q] -= v;
    }
}

__global__ void k_to_f64(const float *src, double *dst, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        dst[q] = (double)src[q];
}

__global__ void k_to_f32(const double *src, float *dst, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        dst[q] = (float)src[q];
}
}  // namespace

void launch_to_f64(const float *src, double *dst, long long n, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    k_to_f64<<<blocks, 256, 0, s>>>(src, dst, n);
    ++g_launches;
    check(cudaGetLastError(), "k_to_f64");
}

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

// f -= (sum_leaves h^D f - [sum Neumann faces h^(D-1) b]) / sum h^D on the leaves
void launch_leaf_center(const Grid &g, double *f, bool with_flux, cudaStream_t s) {
    if (g.n_leaf_boxes == 0) return;
    if (g.T > 1) {  // forests: one constant per singular tree
        const int C = g.D == 2 ? g.N * g.N : g.N * g.N * g.N;
        k_tree_vsum<<<g.T, 256, 0, s>>>(g.meta, g.d_leaves, g.d_tree_leaf0, g.d_tree_sing, nullptr, g.d_leaf_geo, g.D,
                                        g.N, f, with_flux ? g.d_bc : nullptr, g.d_tree_c);
        const int blocks = (int)std::min<long long>(((long long)g.n_leaf_boxes * C + 255) / 256, 152LL * 16);
        k_tree_shift<<<blocks, 256, 0, s>>>(g.meta, g.d_leaves, g.n_leaf_boxes, C, f, g.d_tree_c);
        g_launches += 2;
        check(cudaGetLastError(), "k_tree_vsum");
        return;
    }
    const int nb = std::min(kSumBlocks, g.n_leaf_boxes);
    static_assert(3 * kSumBlocks <= kPartials, "partials buffer");
    k_leaf_vsum<<<nb, 256, 0, s>>>(g.meta, g.d_leaves, g.n_leaf_boxes, g.d_leaf_geo, g.D, g.N, f,
                                   with_flux ? g.d_bc : nullptr, g.d_partials);
    k_vsum_final<<<1, 256, 0, s>>>(g.d_partials, nb, g.d_scalar);
    const int C = g.D == 2 ? g.N * g.N : g.N * g.N * g.N;
    const int blocks = (int)std::min<long long>(((long long)g.n_leaf_boxes * C + 255) / 256, 152LL * 16);
    k_leaf_shift<<<blocks, 256, 0, s>>>(g.meta, g.d_leaves, g.n_leaf_boxes, C, f, g.d_scalar);
    g_launches += 3;
    check(cudaGetLastError(), "k_leaf_vsum");
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
