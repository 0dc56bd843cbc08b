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
    // the boxes of the range come in sibling groups: 2^D consecutive boxes
    // share a parent, child c of a group at offset bit a = (c >> a) & 1
    bool sibs = false;
    // FP32 half-sweep: 16-byte vectors per thread (1: one thread per vector of
    // a box's colour half; 2: half the threads per box)
    int vpt = 1;
};

// counts launches of this library's kernels (host side)
extern unsigned long long g_launches;

// the levels at and below the root box in one launch (one CTA per tree), and
// level 2 as well for one tree of one root box (top = 2; otherwise top = 1):
// mode 0 = V-cycle from ltop (<= top), mode 1 = the FMG steps up to level
// top; lvl_b0[li] = first box of level lmin + li (li = 0 .. top - lmin)
constexpr int kBottomLevels = 6;  // grids of 2 .. 64 cells per side
void launch_bottom(const LaunchCfg &, const BoxMeta &, int ntrees, int N, int lmin, int ltop, int top, int mode,
                   void *u, void *rho, void *vold, int nd, int nu, int nb, int hom, const int *lvl_b0);
// shared memory of that launch for grids of up to top_m cells per side (bytes)
size_t bottom_smem(int D, bool fp64, int top_m);
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

// Variable-coefficient operators (kernels_var.cuh): op 1 div(eps grad u),
// op 2 the same in (r,z) coordinates; eps in the field layout, same precision.
#define AFG_VAR_DECL(DD)                                                                                             \
    void launch_var_smooth_d##DD(const LaunchCfg &, const BoxMeta &, int b0, int n, void *u, const void *rho,        \
                                 const void *eps, int colour, int hom, int op);                                      \
    void launch_var_resid_restrict_d##DD(const LaunchCfg &, const BoxMeta &, int b0, int n, void *u, void *rho,      \
                                         void *vold, const void *eps, int hom, int op);                              \
    void launch_var_fas_d##DD(const LaunchCfg &, const BoxMeta &, int b0, int n, const void *u, void *rho,           \
                              void *vold, const void *eps, int hom, int op);                                         \
    void launch_var_restrict_d##DD(const LaunchCfg &, const BoxMeta &, int b0, int n, const int *list, void *v,      \
                                   int op);                                                                          \
    void launch_correct_x_d##DD(const LaunchCfg &, const BoxMeta &, int b0, int n, void *u, const void *vold,         \
                                const int *nball, int scheme);                                                        \
    void launch_transfer_d##DD(cudaStream_t st, int N, const BoxMeta &Ao, const double *uo, const int *nball_o,      \
                               const BoxMeta &An, double *un, const int *new_leaves, const int *src,                  \
                               const int *poff, int n, int scheme);                                                   \
    void launch_var_leaf_residual_d##DD(const LaunchCfg &, const BoxMeta &, const int *list, int n, const void *u,   \
                                        const void *rho, const void *eps, int hom, int op, unsigned long long *rmax, \
                                        unsigned long long *pmax, void *rout, bool rout_f32);
AFG_VAR_DECL(2)
AFG_VAR_DECL(3)
#undef AFG_VAR_DECL

inline void launch_var_smooth(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *rho,
                              const void *eps, int colour, int hom, int op) {
    if (c.D == 2) launch_var_smooth_d2(c, A, b0, n, u, rho, eps, colour, hom, op);
    else launch_var_smooth_d3(c, A, b0, n, u, rho, eps, colour, hom, op);
}
inline void launch_var_resid_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, void *rho,
                                      void *vold, const void *eps, int hom, int op) {
    if (c.D == 2) launch_var_resid_restrict_d2(c, A, b0, n, u, rho, vold, eps, hom, op);
    else launch_var_resid_restrict_d3(c, A, b0, n, u, rho, vold, eps, hom, op);
}
inline void launch_var_fas(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const void *u, void *rho, void *vold,
                           const void *eps, int hom, int op) {
    if (c.D == 2) launch_var_fas_d2(c, A, b0, n, u, rho, vold, eps, hom, op);
    else launch_var_fas_d3(c, A, b0, n, u, rho, vold, eps, hom, op);
}
// restriction of a field into the parents: the mean of the children (weighted by r when op == 2)
inline void launch_var_restrict(const LaunchCfg &c, const BoxMeta &A, int b0, int n, const int *list, void *v,
                                int op) {
    if (c.D == 2) launch_var_restrict_d2(c, A, b0, n, list, v, op);
    else launch_var_restrict_d3(c, A, b0, n, list, v, op);
}
// coarse-grid correction with the bi/trilinear (scheme 1) or zeroth-order
// (scheme 2) prolongation; nball: the same-level neighbour of every box in
// all 3^D - 1 directions (-1: none)
inline void launch_correct_x(const LaunchCfg &c, const BoxMeta &A, int b0, int n, void *u, const void *vold,
                             const int *nball, int scheme) {
    if (c.D == 2) launch_correct_x_d2(c, A, b0, n, u, vold, nball, scheme);
    else launch_correct_x_d3(c, A, b0, n, u, vold, nball, scheme);
}
// field transfer after mesh adaptation: new leaf li of the new grid copies
// old box src[li] (poff[li] < 0) or is prolonged from old leaf src[li] at
// offset poff[li] (8 bits per axis) with `scheme`
inline void launch_transfer(int D, cudaStream_t st, int N, const BoxMeta &Ao, const double *uo, const int *nball_o,
                            const BoxMeta &An, double *un, const int *new_leaves, const int *src, const int *poff,
                            int n, int scheme) {
    if (D == 2) launch_transfer_d2(st, N, Ao, uo, nball_o, An, un, new_leaves, src, poff, n, scheme);
    else launch_transfer_d3(st, N, Ao, uo, nball_o, An, un, new_leaves, src, poff, n, scheme);
}
inline void launch_var_leaf_residual(const LaunchCfg &c, const BoxMeta &A, const int *list, int n, const void *u,
                                     const void *rho, const void *eps, int hom, int op, unsigned long long *rmax,
                                     unsigned long long *pmax, void *rout, bool rout_f32) {
    if (c.D == 2) launch_var_leaf_residual_d2(c, A, list, n, u, rho, eps, hom, op, rmax, pmax, rout, rout_f32);
    else launch_var_leaf_residual_d3(c, A, list, n, u, rho, eps, hom, op, rmax, pmax, rout, rout_f32);
}

}  // namespace afg
