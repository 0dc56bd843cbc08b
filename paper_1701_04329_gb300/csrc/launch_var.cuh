// Launches of the variable-coefficient kernels (kernels_var.cuh), included
// by launch_var_d2.cu / launch_var_d3.cu (one translation unit per
// dimension, compiled in parallel).
#pragma once
#include "kernels_prolong.cuh"
#include "kernels_transfer.cuh"
#include "kernels_var.cuh"
#include "launch_impl.cuh"

namespace afg {

template <int D, int M, typename T>
void do_var_smooth(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *rho, const void *eps,
                   int colour, int hom, int op) {
    if (n <= 0) return;
    using S = VarCfg<D, M, T>;
    auto k = k_var_smooth<D, M, T>;
    launch_pdl(k, grid_for(k, S::smem(), (n + S::BPC - 1) / S::BPC), S::smem(), c.stream, A, b0, n, (T *)u,
               (const T *)rho, (const T *)eps, colour, hom, op);
    ++g_launches;
}

template <int D, int M, int MP, typename T>
void do_var_resid_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, void *rho, void *vold,
                           const void *eps, int hom, int op) {
    if (n <= 0) return;
    using S = VarCfg<D, M, T>;
    auto k = k_var_resid_restrict<D, M, MP, T>;
    launch_pdl(k, grid_for(k, S::smem(), (n + S::BPC - 1) / S::BPC), S::smem(), c.stream, A, b0, n, (T *)u, (T *)rho,
               (T *)vold, (const T *)eps, hom, op);
    ++g_launches;
}

template <int D, int M, typename T>
void do_var_fas(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const void *u, void *rho, void *vold,
                const void *eps, int hom, int op) {
    if (n <= 0) return;
    using S = VarCfg<D, M, T>;
    auto k = k_var_fas<D, M, T>;
    launch_pdl(k, grid_for(k, S::smem(), (n + S::BPC - 1) / S::BPC), S::smem(), c.stream, A, b0, n, (const T *)u,
               (T *)rho, (T *)vold, (const T *)eps, hom, op);
    ++g_launches;
}

template <int D, int M, typename T, typename Ro>
void do_var_leaf_residual(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *u,
                          const void *rho, const void *eps, int hom, int op, unsigned long long *rmax,
                          unsigned long long *pmax, void *rout) {
    if (n <= 0) return;
    using S = VarCfg<D, M, T>;
    auto k = k_var_leaf_residual<D, M, T, Ro>;
    launch_pdl(k, grid_for(k, S::smem(), (n + S::BPC - 1) / S::BPC), S::smem(), c.stream, A, list, n, (const T *)u,
               (const T *)rho, (const T *)eps, hom, op, rmax, pmax, (Ro *)rout);
    ++g_launches;
}

template <int D, int M, int MP, typename T>
void do_var_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *v, int op) {
    if (n <= 0) return;
    constexpr int NCO = D == 2 ? (M / 2) * (M / 2) : (M / 2) * (M / 2) * (M / 2);
    auto k = k_var_restrict<D, M, MP, T>;
    const long long work = ((long long)n * NCO + kThreads - 1) / kThreads;
    launch_pdl(k, grid_for(k, 0, (int)std::min<long long>(work, 1 << 20)), 0, c.stream, A, b0, n, list, (T *)v, op);
    ++g_launches;
}

template <int D, int M, int MP, typename T>
void do_correct_x(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *vold, const int *nball,
                  int scheme) {
    if (n <= 0) return;
    using S = PxCfg<D, M>;
    const size_t smem = S::template smem<T>();
    auto k = k_correct_x<D, M, MP, T>;
    launch_pdl(k, grid_for(k, smem, (n + S::BPC - 1) / S::BPC), smem, c.stream, A, b0, n, (T *)u, (const T *)vold,
               nball, scheme);
    ++g_launches;
}

template <int D, int M>
void do_transfer(cudaStream_t st, const BoxMeta &Ao, const double *uo, const int *nball_o, const BoxMeta &An,
                 double *un, const int *new_leaves, const int *src, const int *poff, int n, int scheme) {
    if (n <= 0) return;
    using S = TrCfg<D, M>;
    const size_t smem = S::template smem<double>();
    auto k = k_transfer<D, M, double>;
    launch_pdl(k, grid_for(k, smem, (n + S::BPC - 1) / S::BPC), smem, st, Ao, uo, nball_o, An, un, new_leaves, src,
               poff, n, scheme);
    ++g_launches;
}

template <int D>
struct VarOps {
    static void transfer(cudaStream_t st, int N, const BoxMeta &Ao, const double *uo, const int *nball_o,
                         const BoxMeta &An, double *un, const int *new_leaves, const int *src, const int *poff, int n,
                         int scheme) {
        switch (N) {
            case 4: do_transfer<D, 4>(st, Ao, uo, nball_o, An, un, new_leaves, src, poff, n, scheme); break;
            case 8: do_transfer<D, 8>(st, Ao, uo, nball_o, An, un, new_leaves, src, poff, n, scheme); break;
            case 16: do_transfer<D, 16>(st, Ao, uo, nball_o, An, un, new_leaves, src, poff, n, scheme); break;
            default: bad_size(N, 0);
        }
    }
    template <typename T>
    static void correct_x(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *vold,
                          const int *nball, int scheme) {
        AFG_SWITCH_MMP(c.M, c.MP, (do_correct_x<D, MM, PP, T>(c, A, b0, n, u, vold, nball, scheme)));
    }
    template <typename T>
    static void smooth(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *rho, const void *eps,
                       int colour, int hom, int op) {
        AFG_SWITCH_M(c.M, (do_var_smooth<D, MM, T>(c, A, b0, n, u, rho, eps, colour, hom, op)));
    }
    template <typename T>
    static void resid_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, void *rho, void *vold,
                               const void *eps, int hom, int op) {
        AFG_SWITCH_MMP(c.M, c.MP, (do_var_resid_restrict<D, MM, PP, T>(c, A, b0, n, u, rho, vold, eps, hom, op)));
    }
    template <typename T>
    static void fas(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const void *u, void *rho, void *vold,
                    const void *eps, int hom, int op) {
        AFG_SWITCH_M(c.M, (do_var_fas<D, MM, T>(c, A, b0, n, u, rho, vold, eps, hom, op)));
    }
    template <typename T>
    static void restrict_v(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *v, int op) {
        AFG_SWITCH_MMP(c.M, c.MP, (do_var_restrict<D, MM, PP, T>(c, A, b0, n, list, v, op)));
    }
    static void leaf_residual(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *u,
                              const void *rho, const void *eps, int hom, int op, unsigned long long *rmax,
                              unsigned long long *pmax, void *rout, bool rout_f32) {
        if (rout_f32) {
            AFG_SWITCH_M(c.M, (do_var_leaf_residual<D, MM, double, float>(c, A, list, n, u, rho, eps, hom, op, rmax,
                                                                          pmax, rout)));
        } else {
            AFG_SWITCH_M(c.M, (do_var_leaf_residual<D, MM, double, double>(c, A, list, n, u, rho, eps, hom, op, rmax,
                                                                           pmax, rout)));
        }
    }
};

// the entry points of launch.h for one dimension
#define AFG_VAR_LAUNCHES(DD)                                                                                          \
    void launch_var_smooth_d##DD(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *rho,       \
                                 const void *eps, int colour, int hom, int op) {                                      \
        if (c.fp64) VarOps<DD>::smooth<double>(c, A, b0, n, u, rho, eps, colour, hom, op);                            \
        else VarOps<DD>::smooth<float>(c, A, b0, n, u, rho, eps, colour, hom, op);                                    \
    }                                                                                                                 \
    void launch_var_resid_restrict_d##DD(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, void *rho,     \
                                         void *vold, const void *eps, int hom, int op) {                              \
        if (c.fp64) VarOps<DD>::resid_restrict<double>(c, A, b0, n, u, rho, vold, eps, hom, op);                      \
        else VarOps<DD>::resid_restrict<float>(c, A, b0, n, u, rho, vold, eps, hom, op);                              \
    }                                                                                                                 \
    void launch_var_fas_d##DD(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const void *u, void *rho,          \
                              void *vold, const void *eps, int hom, int op) {                                         \
        if (c.fp64) VarOps<DD>::fas<double>(c, A, b0, n, u, rho, vold, eps, hom, op);                                 \
        else VarOps<DD>::fas<float>(c, A, b0, n, u, rho, vold, eps, hom, op);                                         \
    }                                                                                                                 \
    void launch_var_restrict_d##DD(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *v,     \
                                   int op) {                                                                          \
        if (c.fp64) VarOps<DD>::restrict_v<double>(c, A, b0, n, list, v, op);                                        \
        else VarOps<DD>::restrict_v<float>(c, A, b0, n, list, v, op);                                                 \
    }                                                                                                                 \
    void launch_correct_x_d##DD(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *vold,      \
                                const int *nball, int scheme) {                                                       \
        if (c.fp64) VarOps<DD>::correct_x<double>(c, A, b0, n, u, vold, nball, scheme);                               \
        else VarOps<DD>::correct_x<float>(c, A, b0, n, u, vold, nball, scheme);                                       \
    }                                                                                                                 \
    void launch_transfer_d##DD(cudaStream_t st, int N, const BoxMeta &Ao, const double *uo, const int *nball_o,      \
                               const BoxMeta &An, double *un, const int *new_leaves, const int *src,                  \
                               const int *poff, int n, int scheme) {                                                  \
        VarOps<DD>::transfer(st, N, Ao, uo, nball_o, An, un, new_leaves, src, poff, n, scheme);                       \
    }                                                                                                                 \
    void launch_var_leaf_residual_d##DD(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *u,  \
                                        const void *rho, const void *eps, int hom, int op, unsigned long long *rmax,  \
                                        unsigned long long *pmax, void *rout, bool rout_f32) {                        \
        VarOps<DD>::leaf_residual(c, A, list, n, u, rho, eps, hom, op, rmax, pmax, rout, rout_f32);                   \
    }

}  // namespace afg
