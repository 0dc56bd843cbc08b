// Device-resident multigrid hierarchy for one or more trees (a forest):
// box metadata, per-level box ranges and leaf lists, field workspaces, and
// the multigrid drivers (arXiv:1701.04329 Sec. 3.2) built on the kernels.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "host_tree.h"
#include "launch.h"

namespace afg {

struct CudaError : std::runtime_error {
    using std::runtime_error::runtime_error;
};
struct NoMem : std::runtime_error {
    using std::runtime_error::runtime_error;
};

void check(cudaError_t e, const char *what);

// Where device buffers come from: cudaMalloc/cudaFree, or the caller's
// callbacks (afg_set_allocator).  Process-wide; a buffer is returned to the
// allocator that made it.
struct Allocator {
    void *(*alloc)(size_t bytes, void *ctx) = nullptr;
    void (*dealloc)(void *ptr, void *ctx) = nullptr;
    void *ctx = nullptr;
};
Allocator &allocator();
// buffers made by a caller's allocator that are alive (the library synchronises
// the device before it hands one back)
extern int g_user_buffers;

// Makes `dev` the current device for the lifetime of the guard (the device a
// handle's data lives on) and restores the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};
int current_device();

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    Allocator from;
    DevBuf() = default;
    explicit DevBuf(size_t n);
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf();
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

struct Workspace {
    bool fp64 = true;
    std::unique_ptr<DevBuf> u, rho, vold;
    std::unique_ptr<DevBuf> rhoh;  // FP64 only: -h^2 rho / (2D), read by the half-sweep
    void *rhoh_p() const { return rhoh ? rhoh->p : nullptr; }
};

struct MgOpts {
    int n_down = 2, n_up = 2, n_base = 4;
};

class Grid {
  public:
    // levels_only: a tree of several root boxes keeps its coarse grids as
    // device boxes (the per-level kernels) even where they fit one CTA (the
    // variable-coefficient operators and the other prolongations run there)
    explicit Grid(const std::vector<const HostTree *> &trees, bool levels_only = false);
    ~Grid();
    int device = 0;  // the CUDA device holding this grid's data

    struct Level {
        int l, M, MP, b0, nb;  // MP = parent box size (0 at the bottom)
        double h;
        int *d_leaves = nullptr;
        int nleaves = 0;
        long long c0 = 0, ncell = 0;  // cell range of the level
        bool sibs = false;            // boxes in sibling groups (checked when the grid is built)
    };

    int D, N, T, lmin, lmax;
    // a single tree whose level 1 is a block of root boxes: no device boxes
    // below level 1 (the block bottom solve keeps those grids in shared memory)
    bool block = false;
    // highest level of the bottom launch (k_bottom) per precision: 1, or 2
    // for one tree of one root box whose level-2 grid fits one CTA's shared
    // memory (FP32), and in FP64 only while that grid holds at most 1024
    // cells (one SM's FP64 rate makes a larger one slower there than the
    // per-level kernels: 130 us per call for 16^3 against about 110 us)
    int btop32 = 1, btop64 = 1;
    int btop(const Workspace &w) const { return w.fp64 ? btop64 : btop32; }
    int block_nroot[3] = {1, 1, 1}, block_bct[6] = {0, 0, 0, 0, 0, 0};
    int *d_root_box = nullptr;  // box id of root ri + nroot0 (rj + nroot1 rk)
    std::vector<Level> lv;
    Level &L(int l) { return lv[l - lmin]; }
    int nbox = 0, n_leaf_boxes = 0;
    long long ncell = 0, n_leaf_cells = 0, n_bfaces = 0, nbc = 0;
    std::vector<long long> tree_cells, tree_faces;  // per tree
    std::vector<int> tree_top;                      // finest level per tree

    BoxMeta meta{};  // active = nullptr
    int *d_leaves = nullptr;  // all leaf boxes, canonical (tree-major) order
    double *d_leaf_geo = nullptr;  // per leaf box (canonical order): lower corner x, y, z and cell size
    int *d_cf_children = nullptr;  // children of parents that face a same-level leaf
    int n_cf_children = 0;
    int *d_child = nullptr;
    double *d_hb = nullptr;
    double *d_bc = nullptr;
    int *d_masks = nullptr;   // row r: active[tree] for FMG level lmin + r; last row: not converged
    int *d_converged_mask() const { return d_masks + (size_t)(lmax - lmin + 1) * T; }
    int *fmg_mask(int l) const { return d_masks + (size_t)(l - lmin) * T; }
    unsigned long long *d_norms = nullptr;  // 2*T: rmax[T], pmax[T]
    unsigned long long *h_norms = nullptr;  // pinned copy
    int *d_nactive = nullptr, *h_nactive = nullptr;
    double *d_partials = nullptr, *d_scalar = nullptr, *h_scalar = nullptr;

    std::vector<std::unique_ptr<DevBuf>> owned;  // metadata buffers
    Workspace ws64, ws32, wsadj;
    // operator (Sec. 3.4-3.5): 0 Laplacian, 1 div(eps grad u), 2 the same in (r,z);
    // eps on every level (leaves: the user's values, parents: restrictions) in both precisions
    int op = 0;
    std::unique_ptr<DevBuf> eps64, eps32;
    bool eps_set = false;
    double *d_x0 = nullptr;  // lower x coordinate of every box
    // prolongation of the coarse-grid correction (Sec. 2.5): 0 linear, 1 bi/trilinear, 2 zeroth order
    int prolong = 0;
    int *d_nball = nullptr;  // same-level neighbour of every box in all 3^D - 1 directions, -1 none
    // variable coefficients or another prolongation: every level on the per-level kernels
    bool levels_path() const { return op != 0 || prolong != 0 || roots_levels; }
    int vpt = 1;  // FP32 half-sweep: 16-byte vectors per thread (the threads-per-box option)
    // trees of several root boxes whose coarse grids are device boxes (one per
    // root and level): the cycle runs on the per-level kernels
    bool roots_levels = false;
    void correct(Workspace &w, int l, const int *active, cudaStream_t s);
    // a tree without a Dirichlet side: its source is made compatible and its
    // solution kept at zero volume-weighted mean
    bool singular = false;
    // forests: which trees are singular, each tree's first entry in d_leaves
    // (T + 1 offsets) and its constant (the source shift, then the mean)
    std::vector<char> tree_sing;
    char *d_tree_sing = nullptr;
    int *d_tree_leaf0 = nullptr;
    double *d_tree_c = nullptr;
    void make_compatible(cudaStream_t s);
    void remove_mean(Workspace &w, cudaStream_t s);
    const void *eps_of(const Workspace &w) const { return w.fp64 ? eps64->p : eps32->p; }
    void set_eps(const double *eps_leaf, cudaStream_t s);
    std::vector<std::unique_ptr<DevBuf>> bicg;  // adjoint vectors
    bool rhs_set = false;

    LaunchCfg cfg(int l, bool fp64, cudaStream_t s) {
        auto &v = L(l);
        return LaunchCfg{s, D, v.M, v.MP, fp64, v.sibs};
    }
    LaunchCfg leaf_cfg(bool fp64, cudaStream_t s) const { return LaunchCfg{s, D, N, N / 2, fp64}; }

    void alloc_ws(Workspace &w, bool fp64);
    // refresh rho_hat of the leaves after their source term changed
    void leaf_rho_hat(Workspace &w, cudaStream_t s);
    void ensure_mixed();
    void ensure_adjoint();

    // ---- multigrid building blocks ---------------------------------------
    void smooth(Workspace &w, int l, int steps, int hom, const int *active, cudaStream_t s);
    void down_step(Workspace &w, int l, int hom, const int *active, cudaStream_t s);
    void vcycle(Workspace &w, int ltop, const MgOpts &o, int hom, const int *active, cudaStream_t s);
    // levels lmin..1 (one box per tree): mode 0 V-cycle from ltop, mode 1 FMG steps lmin..1
    void bottom(Workspace &w, int ltop, int mode, const MgOpts &o, int hom, const int *active, cudaStream_t s);
    void fmg(Workspace &w, const MgOpts &o, int hom, bool masked, cudaStream_t s);
    void restrict_all(Workspace &w, cudaStream_t s);
    void restrict_cf(Workspace &w, cudaStream_t s);  // only what the composite residual reads
    // restriction of u from the boxes of level l (or a list) into their parents
    void restrict_u(Workspace &w, int l, int b0, int n, const int *list, cudaStream_t s);
    // the cycle on the per-level kernels down to the coarsest grid (no k_bottom)
    void vcycle_levels(Workspace &w, int ltop, const MgOpts &o, int hom, const int *active, cudaStream_t s);
    void fmg_low_levels(Workspace &w, const MgOpts &o, int hom, cudaStream_t s);
    // composite residual of ws64 (restriction + leaf residual), norms to host buffer (async)
    void norms_async(Workspace &w, int hom, void *rout, bool rout_f32, cudaStream_t s);
    // convergence mask update against the tolerance stored in d_tol
    void mask_update_async(cudaStream_t s);
    double *d_tol = nullptr;
    void set_tol(double tol, cudaStream_t s);

    // graphs keyed by a small tuple
    std::map<std::tuple<int, int, int, int, int>, cudaGraphExec_t> graphs;
    std::map<std::tuple<int, int, int, int, int>, int> graph_kernels;  // kernel nodes per graph
    void clear_graphs();
};

// leaf cell centres (canonical order, D doubles per cell) into device memory
void launch_cell_centers(const Grid &g, double *xyz, cudaStream_t s);
// refinement flags of the leaf cells from a leaf field (canonical order)
void launch_flag(const Grid &g, const double *f, int power, double tau_ref, double tau_de, signed char *flags,
                 cudaStream_t s);
// f -= (sum_leaves h^D f - [sum over Neumann leaf faces h^(D-1) b]) / sum h^D on the leaves
// (forests: per singular tree, over its own leaves; other trees unchanged)
void launch_leaf_center(const Grid &g, double *f, bool with_flux, cudaStream_t s);
// dst = (float) src, n values
void launch_to_f32(const double *src, float *dst, long long n, cudaStream_t s);
// dst = (double) src, n values
void launch_to_f64(const float *src, double *dst, long long n, cudaStream_t s);

}  // namespace afg
