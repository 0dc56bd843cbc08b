// Host-side launch interface of the multigrid kernels.  Every function
// enqueues one kernel on cfg.stream; grids are sized from the kernel's
// occupancy times the SM count (a persistent grid looping over boxes).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace afg {

struct LaunchCfg {
    cudaStream_t stream;
    int D;      // 2 or 3
    int M;      // cells per box side on this level
    int MP;     // cells per box side on the parent level (M or M/2)
    bool fp64;  // double (true) or float (false) field data
};

// counts launches of this library's kernels (host side)
extern unsigned long long g_launches;

// the levels at and below the root box in one launch (one CTA per tree):
// mode 0 = V-cycle from ltop (<= 1), mode 1 = the FMG steps up to level 1;
// lvl_b0[li] = first box of level lmin + li
void launch_bottom(const LaunchCfg &, const BoxMeta &, int ntrees, int N, int lmin, int ltop, int mode, void *u,
                   void *rho, void *vold, int nd, int nu, int nb, int hom, const int *lvl_b0);
// the levels at and below level 1 of one tree whose level 1 is a block of
// root boxes (one CTA): nroot[3] roots per axis, bct[6] side types,
// root_box (device) the box id of root ri + nroot0 (rj + nroot1 rk); mode 0 =
// V-cycle from level 1, mode 1 = the FMG steps up to level 1.  Throws when
// the block's grids do not fit one CTA's shared memory.
void launch_bottom_block(const LaunchCfg &, const BoxMeta &, const int *nroot, const int *bct, const int *root_box,
                         int N, int mode, void *u, void *rho, void *vold, int nd, int nu, int nb, int hom);
// shared memory that launch needs (bytes)
size_t bottom_block_smem(int D, bool fp64, int N, const int *nroot, const int *bct);
// opt-in shared memory per block of the current device (bytes)
size_t max_smem_optin();
// rhoh (may be null): use the pre-scaled source -h^2 rho/(2D) instead of rho
void launch_smooth(const LaunchCfg &, const BoxMeta &, int b0, int n, const int *list, void *u, const void *rho,
                   const void *rhoh, double h2, int colour, int hom);
void launch_resid_restrict(const LaunchCfg &, const BoxMeta &, int b0, int n, void *u, void *rho, void *vold,
                           double ih2, int hom);
// rhoh (may be null): also store the pre-scaled coarse source
void launch_fas(const LaunchCfg &, const BoxMeta &, int b0, int n, const void *u, void *rho, void *vold, double ih2,
                int hom, void *rhoh);
// rhoh = -h^2 rho / (2D) on a list of boxes
void launch_rho_hat(const LaunchCfg &, const BoxMeta &, const int *list, int n, const void *rho, void *rhoh);
void launch_correct(const LaunchCfg &, const BoxMeta &, int b0, int n, void *u, const void *vold);
// boxes b0..b0+n-1, or the n boxes of list (list != nullptr)
void launch_restrict_u(const LaunchCfg &, const BoxMeta &, int b0, int n, const int *list, void *u);
// residual rho - A u on leaf boxes (cell size from the box metadata); the
// residual is also stored into rout (float* when rout_f32, else double*) if
// rout is not null
void launch_leaf_residual(const LaunchCfg &, const BoxMeta &, const int *list, int n, const void *u, const void *rho,
                          int hom, unsigned long long *rmax, unsigned long long *pmax, void *rout,
                          bool rout_f32);
// canonical leaf data <-> box storage
void launch_leaf_set(const LaunchCfg &, const BoxMeta &, const int *list, int n, const double *src, void *dst);
void launch_leaf_get(const LaunchCfg &, const BoxMeta &, const int *list, int n, const void *src, double *dst);
// Dirichlet data of the boxes of a level -> their parents (face means)
void launch_bc_restrict(const LaunchCfg &, const BoxMeta &, int b0, int n, double *bc);
// FP64 FMA throughput probe; returns the flops of one launch (FMA = 2)
double launch_fp64_probe(cudaStream_t s, double *scratch, int iters);
// tol is read from device memory, so captured graphs do not bake it in
void launch_mask_update(cudaStream_t s, const unsigned long long *norms, int T, const double *tol, int *active,
                        int *nactive);
// x (double) += e (float) on leaf boxes
void launch_mixed_update(const LaunchCfg &, const BoxMeta &, const int *list, int n, double *x, const float *e);
// adjoint: out = K^T lam on leaf boxes (double); hb = cell size per box
void launch_adjoint_apply(const LaunchCfg &, const BoxMeta &, const int *child, const double *hb, const int *list,
                          int n, const double *lam, double *out);
// dL/db on leaf boundary faces: -(2/h^2) lam of the adjacent cell
void launch_adjoint_db(const LaunchCfg &, const BoxMeta &, const double *hb, const int *list, int n,
                       const double *lam, double *db);
// leaf vectors (double): out = a x + b y + c z (y, z may be null)
void launch_leaf_axpbypcz(const LaunchCfg &, const BoxMeta &, const int *list, int n, double *out, double a,
                          const double *x, double b, const double *y, double c, const double *z);
// out = x * h^(D*power) per box (power = +1 or -1)
void launch_leaf_scale(const LaunchCfg &, const BoxMeta &, const double *hb, const int *list, int n, double *out,
                       const double *x, int power);
// dot product / max norm over leaf cells into *result (device), deterministic
void launch_leaf_dot(const LaunchCfg &, const BoxMeta &, const int *list, int n, const double *x, const double *y,
                     double *partials, double *result);
void launch_leaf_absmax(const LaunchCfg &, const BoxMeta &, const int *list, int n, const double *x,
                        double *partials, double *result);
constexpr int kPartials = 4096;  // size of the partials buffer (doubles)

}  // namespace afg
