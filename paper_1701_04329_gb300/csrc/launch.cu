// Dimension dispatch of the launch layer and the occupancy cache.
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "launch_impl.cuh"

namespace afg {

extern template struct DimOps<2>;
extern template struct DimOps<3>;
extern template struct PrecOps<2, double>;
extern template struct PrecOps<2, float>;
extern template struct PrecOps<3, double>;
extern template struct PrecOps<3, float>;

unsigned long long g_launches = 0;

namespace {
int device_attr(cudaDeviceAttr a, int fallback) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> cache;  // (device, attribute) -> value
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(dev, (int)a);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, a, dev) != cudaSuccess || v < 1) v = fallback;
    cache[key] = v;
    return v;
}
}  // namespace

int sm_count() { return device_attr(cudaDevAttrMultiProcessorCount, 1); }

size_t max_smem_optin() { return (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin, 48 * 1024); }

int occupancy(const void *kernel, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, size_t>, int> cache;  // per device: the attribute is too
    // the shared-memory limit set so far per kernel: it only grows, so that a
    // launch with less shared memory never lowers it under a larger one
    static std::map<std::pair<int, const void *>, size_t> limit;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(dev, kernel, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    size_t &lim = limit[std::make_pair(dev, kernel)];
    if (smem > 48 * 1024 && smem > lim) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        lim = smem;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, smem) != cudaSuccess || occ < 1) occ = 1;
    cache[key] = occ;
    return occ;
}

#define AFG_BY_DIM(FN, ...) \
    do { if (c.D == 2) DimOps<2>::FN(__VA_ARGS__); else DimOps<3>::FN(__VA_ARGS__); } while (0)

void launch_bottom(const LaunchCfg &c, const BoxMeta &A, int ntrees, int N, int lmin, int ltop, int top, int mode,
                   void *u, void *rho, void *vold, int nd, int nu, int nb, int hom, const int *lvl_b0) {
    AFG_BY_DIM(bottom, c, A, ntrees, N, lmin, ltop, top, mode, u, rho, vold, nd, nu, nb, hom, lvl_b0);
}
size_t bottom_smem(int D, bool fp64, int top_m) {
    if (D == 2) return fp64 ? bottom_smem<2, double>(top_m) : bottom_smem<2, float>(top_m);
    return fp64 ? bottom_smem<3, double>(top_m) : bottom_smem<3, float>(top_m);
}
void launch_bottom_block(const LaunchCfg &c, const BoxMeta &A, const int *nroot, const int *bct, const int *root_box,
                         int N, int mode, void *u, void *rho, void *vold, int nd, int nu, int nb, int hom) {
    AFG_BY_DIM(bottom_block, c, A, nroot, bct, root_box, N, mode, u, rho, vold, nd, nu, nb, hom);
}
size_t bottom_block_smem(int D, bool fp64, int N, const int *nroot, const int *bct) {
    BlockTree B;
    for (int a = 0; a < 3; ++a) B.nroot[a] = a < D ? nroot[a] : 1;
    for (int s = 0; s < 6; ++s) B.bct[s] = s < 2 * D ? bct[s] : 0;
    B.root_box = nullptr;
    if (D == 2) return fp64 ? block_bottom_smem<2, double>(N, B) : block_bottom_smem<2, float>(N, B);
    return fp64 ? block_bottom_smem<3, double>(N, B) : block_bottom_smem<3, float>(N, B);
}
void launch_smooth(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u, const void *rho,
                   const void *rhoh, double h2, int colour, int hom) {
    AFG_BY_DIM(smooth, c, A, b0, n, list, u, rho, rhoh, h2, colour, hom);
}
void launch_rho_hat(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *rho, void *rhoh) {
    AFG_BY_DIM(rho_hat, c, A, list, n, rho, rhoh);
}
void launch_resid_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, void *rho, void *vold,
                           double ih2, int hom) { AFG_BY_DIM(resid_restrict, c, A, b0, n, u, rho, vold, ih2, hom); }
void launch_fas(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const void *u, void *rho, void *vold, double ih2,
                int hom, void *rhoh) { AFG_BY_DIM(fas, c, A, b0, n, u, rho, vold, ih2, hom, rhoh); }
void launch_correct(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *vold) {
    AFG_BY_DIM(correct, c, A, b0, n, u, vold);
}
void launch_restrict_u(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u) {
    AFG_BY_DIM(restrict_u, c, A, b0, n, list, u);
}
void launch_leaf_residual(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *u, const void *rho,
                          int hom, unsigned long long *rmax, unsigned long long *pmax, void *rout, bool rout_f32) {
    AFG_BY_DIM(leaf_residual, c, A, list, n, u, rho, hom, rmax, pmax, rout, rout_f32);
}

// Per-tree convergence mask of a batched solve: a tree stays active while
// max|r| > tol * max|rho|; counts the active trees.
__global__ void k_mask_update(const unsigned long long *norms, int T, const double *tolp, int *active,
                              int *nactive) {
    const double tol = *tolp;
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int local = 0;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const double r = __longlong_as_double((long long)norms[t]);
        const double p = __longlong_as_double((long long)norms[T + t]);
        const int a = active[t] && (p > 0.0 ? r > tol * p : r > tol);
        active[t] = a;
        local += a;
    }
    atomicAdd(&cnt, local);
    __syncthreads();
    if (threadIdx.x == 0) *nactive = cnt;
}

// FP64 issue-rate probe: 8 independent FMA chains per thread, 64 FMAs per
// iteration; the result is consumed so nothing is optimised away.
__global__ void __launch_bounds__(kThreads) k_fp64_probe(double *out, double a, double b, int iters) {
    double x[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) x[r] = threadIdx.x * 1e-3 + r;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int rep = 0; rep < 8; ++rep)
#pragma unroll
            for (int r = 0; r < 8; ++r) x[r] = fma(x[r], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < 8; ++r) s += x[r];
    if (s == -12345.0) out[0] = s;
}

double launch_fp64_probe(cudaStream_t s, double *scratch, int iters) {
    const int blocks = sm_count() * 8;
    k_fp64_probe<<<blocks, kThreads, 0, s>>>(scratch, 0.999999, 1e-7, iters);
    ++g_launches;
    return 2.0 * 64.0 * (double)blocks * kThreads * iters;  // flops (FMA = 2)
}

void launch_mask_update(cudaStream_t s, const unsigned long long *norms, int T, const double *tol, int *active,
                        int *nactive) {
    k_mask_update<<<1, kThreads, 0, s>>>(norms, T, tol, active, nactive);
    ++g_launches;
}
void launch_leaf_set(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const double *src, void *dst) {
    AFG_BY_DIM(leaf_set, c, A, list, n, src, dst);
}
void launch_leaf_get(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *src, double *dst) {
    AFG_BY_DIM(leaf_get, c, A, list, n, src, dst);
}
void launch_bc_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, double *bc) { AFG_BY_DIM(bc_restrict, c, A, b0, n, bc); }
void launch_mixed_update(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, double *x, const float *e) {
    AFG_BY_DIM(mixed_update, c, A, list, n, x, e);
}
void launch_adjoint_apply(const LaunchCfg &c, const BoxMeta &A, const int *child, const double *hb, const int *list,
                          int n, const double *lam, double *out) {
    AFG_BY_DIM(adjoint_apply, c, A, child, hb, list, n, lam, out);
}
void launch_adjoint_db(const LaunchCfg &c, const BoxMeta &A, const double *hb, const int *list, int n,
                       const double *lam, double *db) { AFG_BY_DIM(adjoint_db, c, A, hb, list, n, lam, db); }
void launch_leaf_axpbypcz(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, double *out, double a,
                          const double *x, double b, const double *y, double cc, const double *z) {
    AFG_BY_DIM(axpbypcz, c, A, list, n, out, a, x, b, y, cc, z);
}
void launch_leaf_scale(const LaunchCfg &c, const BoxMeta &A, const double *hb, const int *list, int n, double *out,
                       const double *x, int power) { AFG_BY_DIM(scale, c, A, hb, list, n, out, x, power); }
void launch_leaf_dot(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const double *x, const double *y,
                     double *partials, double *result) { AFG_BY_DIM(reduce, c, A, list, n, x, y, 0, partials, result); }
void launch_leaf_absmax(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const double *x,
                        double *partials, double *result) { AFG_BY_DIM(reduce, c, A, list, n, x, nullptr, 1, partials, result); }

}  // namespace afg
