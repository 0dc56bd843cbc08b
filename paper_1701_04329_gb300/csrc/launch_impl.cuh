// Template side of the launch layer; instantiated per dimension (the
// dispatch, launch_d2.cu / launch_d3.cu) and per dimension and precision (the
// launches and their kernels, launch_d<D>_f64.cu / launch_d<D>_f32.cu), so
// that the six translation units compile in parallel.
#pragma once
#include <algorithm>
#include <stdexcept>
#include <string>

#include "kernels_leaf.cuh"
#include "kernels_smooth.cuh"
#include "kernels_full.cuh"
#include "kernels_bottom.cuh"
#include "kernels_block.cuh"
#include "launch.h"

namespace afg {

// FP64 half-sweeps: the staged half-row kernel (true) or the table-driven one
constexpr bool kStagedSmooth64 = true;

int sm_count();
// resident CTAs per SM of a kernel for a given dynamic shared memory size (cached)
int occupancy(const void *kernel, size_t smem);

// Persistent grid: (resident CTAs per SM) x SMs, capped by the work.
template <typename K>
int grid_for(K kernel, size_t smem, int work_ctas) {
    const int cap = occupancy(reinterpret_cast<const void *>(kernel), smem) * sm_count();
    return std::max(1, std::min(work_ctas, cap));
}

// Launch with programmatic stream serialization (PDL): the kernel may start
// while its predecessor drains; every kernel waits (griddepcontrol.wait)
// before reading data a predecessor wrote.
template <typename... KArgs, typename... Args>
void launch_pdl_block(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), int grid, size_t smem, cudaStream_t s, Args... args) {
    launch_pdl_block(kernel, grid, kThreads, smem, s, args...);
}

template <int D, int M>
inline int work_ctas(int nbox) { return (nbox + Geo<D, M>::BPC - 1) / Geo<D, M>::BPC; }

template <int D, int M, typename T>
void do_smooth(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u, const void *rho,
               const void *rhoh, double h2, int colour, int hom) {
    if (n <= 0) return;
    // FP32: the staged half-row kernel; FP64 keeps the table-driven one unless
    // kStagedSmooth64 is set
    if constexpr (SpCfg<D, M, T>::ok && (sizeof(T) == 4 || kStagedSmooth64)) {
        // FP32 with half the threads per box (two vectors per thread) on request
        if constexpr (sizeof(T) == 4 && SpCfg<D, M, T>::NV >= 2) {
            if (c.vpt == 2) {
                using S = SpCfg<D, M, T, 2>;
                const size_t smem = S::smem();
                auto k = k_smooth_p<D, M, T, 2>;
                launch_pdl(k, grid_for(k, smem, (n + S::BPC - 1) / S::BPC), smem, c.stream, A, b0, n, list, (T *)u,
                           (const T *)(rhoh ? rhoh : rho), T(h2), colour, hom, rhoh ? 1 : 0);
                ++g_launches;
                return;
            }
        }
        {
            using S = SpCfg<D, M, T>;
            const size_t smem = S::smem();
            auto k = k_smooth_p<D, M, T>;
            launch_pdl(k, grid_for(k, smem, (n + S::BPC - 1) / S::BPC), smem, c.stream, A, b0, n, list, (T *)u,
                       (const T *)(rhoh ? rhoh : rho), T(h2), colour, hom, rhoh ? 1 : 0);
            ++g_launches;
            return;
        }
    }
    using S = SmCfg<D, M, T>;
    const size_t smem = S::smem();
    auto k = k_smooth<D, M, T>;
    launch_pdl(k, grid_for(k, smem, (n + S::BPC - 1) / S::BPC), smem, c.stream, A, b0, n, list, (T *)u,
               (const T *)(rhoh ? rhoh : rho), T(h2), colour, hom, rhoh ? 1 : 0);
    ++g_launches;
}

// Whole-box kernels: the cp.async-staged versions wherever a half-row holds
// a 16-byte vector (all boxes of 8^D and 16^D cells, FP64 4^D), the
// table-driven ones otherwise.
template <int D, int M, int MP, typename T>
void do_resid_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, void *rho, void *vold,
                       double ih2, int hom) {
    if (n <= 0) return;
    if constexpr (FpCfg<D, M, T>::ok) {
        using F = FpCfg<D, M, T, rr_threads<D, M, T>()>;
        const size_t smem = F::smem();
        auto k = k_resid_restrict_p<D, M, MP, T>;
        launch_pdl(k, grid_for(k, smem, (n + F::BPC - 1) / F::BPC), smem, c.stream, A, b0, n, (T *)u, (T *)rho,
                   (T *)vold, T(ih2), hom);
    } else {
        const size_t smem = FullCfg<D, M, T>::smem();
        auto k = k_resid_restrict<D, M, MP, T>;
        launch_pdl(k, grid_for(k, smem, work_ctas<D, M>(n)), smem, c.stream, A, b0, n, (T *)u, (T *)rho,
                   (T *)vold, T(ih2), hom);
    }
    ++g_launches;
}

template <int D, int M, typename T>
void do_fas(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const void *u, void *rho, void *vold, double ih2,
            int hom, void *rhoh) {
    if (n <= 0) return;
    const T chat = T(-1.0 / (ih2 * 2 * D));  // -h^2 / (2D)
    if constexpr (FpCfg<D, M, T>::ok) {
        using F = FpCfg<D, M, T, fas_threads<D, M, T>()>;
        const size_t smem = F::smem();
        auto k = k_fas_p<D, M, T>;
        launch_pdl(k, grid_for(k, smem, (n + F::BPC - 1) / F::BPC), smem, c.stream, A, b0, n, (const T *)u,
                   (T *)rho, (T *)vold, T(ih2), hom, (T *)rhoh, chat);
    } else {
        const size_t smem = FullCfg<D, M, T>::smem();
        auto k = k_fas<D, M, T>;
        launch_pdl(k, grid_for(k, smem, work_ctas<D, M>(n)), smem, c.stream, A, b0, n, (const T *)u, (T *)rho,
                   (T *)vold, T(ih2), hom, (T *)rhoh, chat);
    }
    ++g_launches;
}

template <int D, int M, int MP, typename T>
void do_correct(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *vold) {
    if (n <= 0) return;
    // one CTA per parent: the parent staged once for its 2^D children
    if constexpr (PpCfg<D, M, T>::ok && MP == M) {
        if (c.sibs) {
            using S = PpCfg<D, M, T>;
            const size_t smem = S::smem();
            auto k = k_correct_pp<D, M, T>;
            launch_pdl(k, grid_for(k, smem, n / S::NC), smem, c.stream, A, b0, n, (T *)u, (const T *)vold);
            ++g_launches;
            return;
        }
    }
    // staged copies; in 3D the pair sums of a coarse cell are shared by its children
    if constexpr (CpCfg<D, M, T>::ok && MP == M) {
        using S = CpCfg<D, M, T>;
        const size_t smem = S::smem();
        auto k = k_correct_p<D, M, MP, T>;
        launch_pdl(k, grid_for(k, smem, (n + S::BPC - 1) / S::BPC), smem, c.stream, A, b0, n, (T *)u,
                   (const T *)vold);
        ++g_launches;
        return;
    }
    const size_t smem = CorrCfg<D, M>::template smem<T>();
    auto k = k_correct<D, M, MP, T>;
    launch_pdl(k, grid_for(k, smem, work_ctas<D, M>(n)), smem, c.stream, A, b0, n, (T *)u, (const T *)vold);
    ++g_launches;
}

template <int D, int M, int MP, typename T>
void do_restrict_u(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u) {
    if (n <= 0) return;
    auto k = k_restrict_u<D, M, MP, T>;
    launch_pdl(k, grid_for(k, 0, work_ctas<D, M>(n)), 0, c.stream, A, b0, n, list, (T *)u);
    ++g_launches;
}

template <int D, int M, typename T>
void do_leaf_residual(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *u, const void *rho,
                      int hom, unsigned long long *rmax, unsigned long long *pmax, void *rout,
                      bool rout_f32) {
    if (n <= 0) return;
    auto go = [&](auto k, size_t smem, int wc, auto *out) {
        launch_pdl(k, grid_for(k, smem, wc), smem, c.stream, A, list, n, (const T *)u, (const T *)rho, hom, rmax,
                   pmax, out);
    };
    if constexpr (FpCfg<D, M, T>::ok) {
        using F = FpCfg<D, M, T, leaf_threads<D, M, T>()>;
        const int wc = (n + F::BPC - 1) / F::BPC;
        if (rout_f32) go(k_leaf_residual_p<D, M, T, float>, F::smem(), wc, (float *)rout);
        else go(k_leaf_residual_p<D, M, T, double>, F::smem(), wc, (double *)rout);
    } else {
        const size_t smem = FullCfg<D, M, T>::smem();
        if (rout_f32) go(k_leaf_residual<D, M, T, float>, smem, work_ctas<D, M>(n), (float *)rout);
        else go(k_leaf_residual<D, M, T, double>, smem, work_ctas<D, M>(n), (double *)rout);
    }
    ++g_launches;
}

template <int D, int M, typename T>
void do_leaf_set(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const double *src, void *dst) {
    if (n <= 0) return;
    auto k = k_leaf_set<D, M, T>;
    launch_pdl(k, grid_for(k, 0, work_ctas<D, M>(n)), 0, c.stream, A, list, n, src, (T *)dst);
    ++g_launches;
}

template <int D, int M, typename T>
void do_leaf_get(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *src, double *dst) {
    if (n <= 0) return;
    auto k = k_leaf_get<D, M, T>;
    launch_pdl(k, grid_for(k, 0, work_ctas<D, M>(n)), 0, c.stream, A, list, n, (const T *)src, dst);
    ++g_launches;
}

template <int D, int M, int MP>
void do_bc_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, double *bc) {
    if (n <= 0) return;
    auto k = k_bc_restrict<D, M, MP>;
    launch_pdl(k, grid_for(k, 0, work_ctas<D, M>(n)), 0, c.stream, A, b0, n, bc);
    ++g_launches;
}

template <int D, int M>
void do_mixed_update(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, double *x, const float *e) {
    if (n <= 0) return;
    auto k = k_mixed_update<D, M>;
    launch_pdl(k, grid_for(k, 0, work_ctas<D, M>(n)), 0, c.stream, A, list, n, x, e);
    ++g_launches;
}

template <int D, int M>
void do_adjoint_apply(const LaunchCfg &c, const BoxMeta &A, const int *child, const double *hb, const int *list,
                      int n, const double *lam, double *out) {
    if (n <= 0) return;
    const size_t smem = sizeof(double) * Geo<D, M>::PC * Geo<D, M>::BPC;
    auto k = k_adjoint_apply<D, M>;
    launch_pdl(k, grid_for(k, smem, work_ctas<D, M>(n)), smem, c.stream, A, child, hb, list, n, lam, out);
    ++g_launches;
}

template <int D, int M>
void do_adjoint_db(const LaunchCfg &c, const BoxMeta &A, const double *hb, const int *list, int n, const double *lam,
                   double *db) {
    if (n <= 0) return;
    auto k = k_adjoint_db<D, M>;
    launch_pdl(k, grid_for(k, 0, work_ctas<D, M>(n)), 0, c.stream, A, hb, list, n, lam, db);
    ++g_launches;
}

template <int D, int M>
void do_axpbypcz(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, double *out, double a,
                 const double *x, double b, const double *y, double cc, const double *z) {
    if (n <= 0) return;
    auto k = k_leaf_axpbypcz<D, M>;
    launch_pdl(k, grid_for(k, 0, work_ctas<D, M>(n)), 0, c.stream, A, list, n, out, a, x, b, y, cc, z);
    ++g_launches;
}

template <int D, int M>
void do_scale(const LaunchCfg &c, const BoxMeta &A, const double *hb, const int *list, int n, double *out,
              const double *x, int power) {
    if (n <= 0) return;
    auto k = k_leaf_scale<D, M>;
    launch_pdl(k, grid_for(k, 0, work_ctas<D, M>(n)), 0, c.stream, A, hb, list, n, out, x, power);
    ++g_launches;
}

template <int D, int M>
void do_reduce(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const double *x, const double *y,
               int mode, double *partials, double *result) {
    auto k = k_leaf_reduce<D, M>;
    const int grid = std::min(kPartials, grid_for(k, 0, std::max(1, work_ctas<D, M>(n))));
    launch_pdl(k, grid, 0, c.stream, A, list, n, x, y, mode, partials);
    k_reduce_final<<<1, kThreads, 0, c.stream>>>(partials, grid, mode, result);
    g_launches += 2;
}

template <int D, int M, typename T>
void do_rho_hat(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *rho, void *rhoh) {
    if (n <= 0) return;
    auto k = k_rho_hat<D, M, T>;
    launch_pdl(k, grid_for(k, 0, work_ctas<D, M>(n)), 0, c.stream, A, list, n, (const T *)rho, (T *)rhoh);
    ++g_launches;
}

static_assert(kBottomLevels == kBottomMaxLevels, "bottom level count");

template <int D, typename T>
void do_bottom(const LaunchCfg &c, const BoxMeta &A, int ntrees, int N, int lmin, int ltop, int top, int mode,
               void *u, void *rho, void *vold, int nd, int nu, int nb, int hom, const int *lvl_b0) {
    const size_t smem = bottom_smem<D, T>(top == 2 ? 2 * N : N);
    auto k = k_bottom<D, T>;
    occupancy(reinterpret_cast<const void *>(k), smem);  // sets the shared-memory limit
    BottomArgs P = {};
    P.ntrees = ntrees;
    P.N = N;
    P.lmin = lmin;
    P.ltop = ltop;
    P.mode = mode;
    P.nd = nd;
    P.nu = nu;
    P.nb = nb;
    P.hom = hom;
    P.top = top;
    for (int li = 0; li <= top - lmin && li < kBottomMaxLevels; ++li) P.b0[li] = lvl_b0[li];
    launch_pdl_block(k, ntrees, kBottomThreads, smem, c.stream, A, P, (T *)u, (T *)rho, (T *)vold);
    ++g_launches;
}

template <int D, typename T>
void do_bottom_block(const LaunchCfg &c, const BoxMeta &A, const int *nroot, const int *bct, const int *root_box,
                     int N, int mode, void *u, void *rho, void *vold, int nd, int nu, int nb, int hom) {
    BlockTree B;
    for (int a = 0; a < 3; ++a) B.nroot[a] = a < D ? nroot[a] : 1;
    for (int s = 0; s < 6; ++s) B.bct[s] = s < 2 * D ? bct[s] : 0;
    B.root_box = root_box;
    const size_t smem = block_bottom_smem<D, T>(N, B);
    if (smem > max_smem_optin())
        throw std::runtime_error("the block of root boxes is too large for one CTA's shared memory (" +
                                 std::to_string(smem) + " bytes)");
    auto k = k_bottom_block<D, T>;
    occupancy(reinterpret_cast<const void *>(k), smem);  // sets the shared-memory limit once
    launch_pdl(k, 1, smem, c.stream, A, B, N, mode, (T *)u, (T *)rho, (T *)vold, nd, nu, nb, hom);
    ++g_launches;
}

// ---- dispatch over the box size --------------------------------------------
[[noreturn]] inline void bad_size(int M, int MP) {
    throw std::runtime_error("unsupported box size " + std::to_string(M) + "/" + std::to_string(MP));
}

#define AFG_SWITCH_M(M, BODY)                       \
    switch (M) {                                    \
        case 2: { constexpr int MM = 2; BODY; break; }   \
        case 4: { constexpr int MM = 4; BODY; break; }   \
        case 8: { constexpr int MM = 8; BODY; break; }   \
        case 16: { constexpr int MM = 16; BODY; break; } \
        default: bad_size(M, 0);                    \
    }

// (M, MP) pairs: same size (tree levels >= 2) or half size (root and below)
#define AFG_SWITCH_MMP(M, MP, BODY)                                                   \
    if ((M) == (MP)) {                                                                \
        switch (M) {                                                                  \
            case 4: { constexpr int MM = 4, PP = 4; BODY; break; }                    \
            case 8: { constexpr int MM = 8, PP = 8; BODY; break; }                    \
            case 16: { constexpr int MM = 16, PP = 16; BODY; break; }                 \
            default: bad_size(M, MP);                                                 \
        }                                                                             \
    } else if (2 * (MP) == (M)) {                                                     \
        switch (M) {                                                                  \
            case 4: { constexpr int MM = 4, PP = 2; BODY; break; }                    \
            case 8: { constexpr int MM = 8, PP = 4; BODY; break; }                    \
            case 16: { constexpr int MM = 16, PP = 8; BODY; break; }                  \
            default: bad_size(M, MP);                                                 \
        }                                                                             \
    } else bad_size(M, MP);

// The precision-specific launches, instantiated per (dimension, precision) in
// launch_d<D>_f64.cu / launch_d<D>_f32.cu so those compile in parallel.
template <int D, typename T>
struct PrecOps {
    static void rho_hat(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *rho, void *rhoh);
    static void bottom(const LaunchCfg &c, const BoxMeta &A, int ntrees, int N, int lmin, int ltop, int top, int mode,
                       void *u, void *rho, void *vold, int nd, int nu, int nb, int hom, const int *lvl_b0);
    static void bottom_block(const LaunchCfg &c, const BoxMeta &A, const int *nroot, const int *bct,
                             const int *root_box, int N, int mode, void *u, void *rho, void *vold, int nd, int nu,
                             int nb, int hom);
    static void smooth(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u,
                       const void *rho, const void *rhoh, double h2, int colour, int hom);
    static void resid_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, void *rho, void *vold,
                               double ih2, int hom);
    static void fas(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const void *u, void *rho, void *vold,
                    double ih2, int hom, void *rhoh);
    static void correct(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *vold);
    static void restrict_u(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u);
    static void leaf_residual(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *u,
                              const void *rho, int hom, unsigned long long *rmax,
                              unsigned long long *pmax, void *rout, bool rout_f32);
    static void leaf_set(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const double *src, void *dst);
    static void leaf_get(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *src, double *dst);
};

template <int D, typename T>
void PrecOps<D, T>::rho_hat(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *rho, void *rhoh) {
    AFG_SWITCH_M(c.M, (do_rho_hat<D, MM, T>(c, A, list, n, rho, rhoh)));
}

template <int D, typename T>
void PrecOps<D, T>::bottom(const LaunchCfg &c, const BoxMeta &A, int ntrees, int N, int lmin, int ltop, int top,
                           int mode, void *u, void *rho, void *vold, int nd, int nu, int nb, int hom,
                           const int *lvl_b0) {
    do_bottom<D, T>(c, A, ntrees, N, lmin, ltop, top, mode, u, rho, vold, nd, nu, nb, hom, lvl_b0);
}

template <int D, typename T>
void PrecOps<D, T>::bottom_block(const LaunchCfg &c, const BoxMeta &A, const int *nroot, const int *bct,
                                 const int *root_box, int N, int mode, void *u, void *rho, void *vold, int nd, int nu,
                                 int nb, int hom) {
    do_bottom_block<D, T>(c, A, nroot, bct, root_box, N, mode, u, rho, vold, nd, nu, nb, hom);
}

template <int D, typename T>
void PrecOps<D, T>::smooth(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u,
                           const void *rho, const void *rhoh, double h2, int colour, int hom) {
    AFG_SWITCH_M(c.M, (do_smooth<D, MM, T>(c, A, b0, n, list, u, rho, rhoh, h2, colour, hom)));
}

template <int D, typename T>
void PrecOps<D, T>::resid_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, void *rho, void *vold,
                                   double ih2, int hom) {
    AFG_SWITCH_MMP(c.M, c.MP, (do_resid_restrict<D, MM, PP, T>(c, A, b0, n, u, rho, vold, ih2, hom)));
}

template <int D, typename T>
void PrecOps<D, T>::fas(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const void *u, void *rho, void *vold,
                        double ih2, int hom, void *rhoh) {
    AFG_SWITCH_M(c.M, (do_fas<D, MM, T>(c, A, b0, n, u, rho, vold, ih2, hom, rhoh)));
}

template <int D, typename T>
void PrecOps<D, T>::correct(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *vold) {
    AFG_SWITCH_MMP(c.M, c.MP, (do_correct<D, MM, PP, T>(c, A, b0, n, u, vold)));
}

template <int D, typename T>
void PrecOps<D, T>::restrict_u(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u) {
    AFG_SWITCH_MMP(c.M, c.MP, (do_restrict_u<D, MM, PP, T>(c, A, b0, n, list, u)));
}

template <int D, typename T>
void PrecOps<D, T>::leaf_residual(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *u,
                                  const void *rho, int hom, unsigned long long *rmax,
                                  unsigned long long *pmax, void *rout, bool rout_f32) {
    AFG_SWITCH_M(c.M, (do_leaf_residual<D, MM, T>(c, A, list, n, u, rho, hom, rmax, pmax, rout, rout_f32)));
}

template <int D, typename T>
void PrecOps<D, T>::leaf_set(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const double *src, void *dst) {
    AFG_SWITCH_M(c.M, (do_leaf_set<D, MM, T>(c, A, list, n, src, dst)));
}

template <int D, typename T>
void PrecOps<D, T>::leaf_get(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *src, double *dst) {
    AFG_SWITCH_M(c.M, (do_leaf_get<D, MM, T>(c, A, list, n, src, dst)));
}

template <int D>
struct DimOps {
    static void rho_hat(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *rho, void *rhoh);
    static void bottom(const LaunchCfg &c, const BoxMeta &A, int ntrees, int N, int lmin, int ltop, int top, int mode,
                       void *u, void *rho, void *vold, int nd, int nu, int nb, int hom, const int *lvl_b0);
    static void bottom_block(const LaunchCfg &c, const BoxMeta &A, const int *nroot, const int *bct,
                             const int *root_box, int N, int mode, void *u, void *rho, void *vold, int nd, int nu,
                             int nb, int hom);
    static void smooth(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u,
                       const void *rho, const void *rhoh, double h2, int colour, int hom);
    static void resid_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, void *rho, void *vold,
                               double ih2, int hom);
    static void fas(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const void *u, void *rho, void *vold,
                    double ih2, int hom, void *rhoh);
    static void correct(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *vold);
    static void restrict_u(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u);
    static void leaf_residual(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *u,
                              const void *rho, int hom, unsigned long long *rmax,
                              unsigned long long *pmax, void *rout, bool rout_f32);
    static void leaf_set(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const double *src, void *dst);
    static void leaf_get(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *src, double *dst);
    static void bc_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, double *bc);
    static void mixed_update(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, double *x, const float *e);
    static void adjoint_apply(const LaunchCfg &c, const BoxMeta &A, const int *child, const double *hb,
                              const int *list, int n, const double *lam, double *out);
    static void adjoint_db(const LaunchCfg &c, const BoxMeta &A, const double *hb, const int *list, int n,
                           const double *lam, double *db);
    static void axpbypcz(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, double *out, double a,
                         const double *x, double b, const double *y, double cc, const double *z);
    static void scale(const LaunchCfg &c, const BoxMeta &A, const double *hb, const int *list, int n, double *out,
                      const double *x, int power);
    static void reduce(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const double *x,
                       const double *y, int mode, double *partials, double *result);
};

template <int D>
void DimOps<D>::rho_hat(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *rho, void *rhoh) {
    if (c.fp64) PrecOps<D, double>::rho_hat(c, A, list, n, rho, rhoh);
    else PrecOps<D, float>::rho_hat(c, A, list, n, rho, rhoh);
}

template <int D>
void DimOps<D>::bottom(const LaunchCfg &c, const BoxMeta &A, int ntrees, int N, int lmin, int ltop, int top,
                       int mode, void *u, void *rho, void *vold, int nd, int nu, int nb, int hom, const int *lvl_b0) {
    if (c.fp64)
        PrecOps<D, double>::bottom(c, A, ntrees, N, lmin, ltop, top, mode, u, rho, vold, nd, nu, nb, hom, lvl_b0);
    else
        PrecOps<D, float>::bottom(c, A, ntrees, N, lmin, ltop, top, mode, u, rho, vold, nd, nu, nb, hom, lvl_b0);
}

template <int D>
void DimOps<D>::bottom_block(const LaunchCfg &c, const BoxMeta &A, const int *nroot, const int *bct,
                             const int *root_box, int N, int mode, void *u, void *rho, void *vold, int nd, int nu,
                             int nb, int hom) {
    if (c.fp64) PrecOps<D, double>::bottom_block(c, A, nroot, bct, root_box, N, mode, u, rho, vold, nd, nu, nb, hom);
    else PrecOps<D, float>::bottom_block(c, A, nroot, bct, root_box, N, mode, u, rho, vold, nd, nu, nb, hom);
}

template <int D>
void DimOps<D>::smooth(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u,
                       const void *rho, const void *rhoh, double h2, int colour, int hom) {
    if (c.fp64) PrecOps<D, double>::smooth(c, A, b0, n, list, u, rho, rhoh, h2, colour, hom);
    else PrecOps<D, float>::smooth(c, A, b0, n, list, u, rho, rhoh, h2, colour, hom);
}

template <int D>
void DimOps<D>::resid_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, void *rho, void *vold,
                               double ih2, int hom) {
    if (c.fp64) PrecOps<D, double>::resid_restrict(c, A, b0, n, u, rho, vold, ih2, hom);
    else PrecOps<D, float>::resid_restrict(c, A, b0, n, u, rho, vold, ih2, hom);
}

template <int D>
void DimOps<D>::fas(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const void *u, void *rho, void *vold,
                    double ih2, int hom, void *rhoh) {
    if (c.fp64) PrecOps<D, double>::fas(c, A, b0, n, u, rho, vold, ih2, hom, rhoh);
    else PrecOps<D, float>::fas(c, A, b0, n, u, rho, vold, ih2, hom, rhoh);
}

template <int D>
void DimOps<D>::correct(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *vold) {
    if (c.fp64) PrecOps<D, double>::correct(c, A, b0, n, u, vold);
    else PrecOps<D, float>::correct(c, A, b0, n, u, vold);
}

template <int D>
void DimOps<D>::restrict_u(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *u) {
    if (c.fp64) PrecOps<D, double>::restrict_u(c, A, b0, n, list, u);
    else PrecOps<D, float>::restrict_u(c, A, b0, n, list, u);
}

template <int D>
void DimOps<D>::leaf_residual(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *u,
                              const void *rho, int hom, unsigned long long *rmax,
                              unsigned long long *pmax, void *rout, bool rout_f32) {
    if (c.fp64) PrecOps<D, double>::leaf_residual(c, A, list, n, u, rho, hom, rmax, pmax, rout, rout_f32);
    else PrecOps<D, float>::leaf_residual(c, A, list, n, u, rho, hom, rmax, pmax, rout, rout_f32);
}

template <int D>
void DimOps<D>::leaf_set(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const double *src, void *dst) {
    if (c.fp64) PrecOps<D, double>::leaf_set(c, A, list, n, src, dst);
    else PrecOps<D, float>::leaf_set(c, A, list, n, src, dst);
}

template <int D>
void DimOps<D>::leaf_get(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *src, double *dst) {
    if (c.fp64) PrecOps<D, double>::leaf_get(c, A, list, n, src, dst);
    else PrecOps<D, float>::leaf_get(c, A, list, n, src, dst);
}

template <int D>
void DimOps<D>::bc_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, double *bc) {
    AFG_SWITCH_MMP(c.M, c.MP, (do_bc_restrict<D, MM, PP>(c, A, b0, n, bc)));
}

template <int D>
void DimOps<D>::mixed_update(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, double *x, const float *e) {
    AFG_SWITCH_M(c.M, (do_mixed_update<D, MM>(c, A, list, n, x, e)));
}

template <int D>
void DimOps<D>::adjoint_apply(const LaunchCfg &c, const BoxMeta &A, const int *child, const double *hb,
                              const int *list, int n, const double *lam, double *out) {
    AFG_SWITCH_M(c.M, (do_adjoint_apply<D, MM>(c, A, child, hb, list, n, lam, out)));
}

template <int D>
void DimOps<D>::adjoint_db(const LaunchCfg &c, const BoxMeta &A, const double *hb, const int *list, int n,
                           const double *lam, double *db) {
    AFG_SWITCH_M(c.M, (do_adjoint_db<D, MM>(c, A, hb, list, n, lam, db)));
}

template <int D>
void DimOps<D>::axpbypcz(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, double *out, double a,
                         const double *x, double b, const double *y, double cc, const double *z) {
    AFG_SWITCH_M(c.M, (do_axpbypcz<D, MM>(c, A, list, n, out, a, x, b, y, cc, z)));
}

template <int D>
void DimOps<D>::scale(const LaunchCfg &c, const BoxMeta &A, const double *hb, const int *list, int n, double *out,
                      const double *x, int power) {
    AFG_SWITCH_M(c.M, (do_scale<D, MM>(c, A, hb, list, n, out, x, power)));
}

template <int D>
void DimOps<D>::reduce(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const double *x,
                       const double *y, int mode, double *partials, double *result) {
    AFG_SWITCH_M(c.M, (do_reduce<D, MM>(c, A, list, n, x, y, mode, partials, result)));
}


}  // namespace afg
