// Grid construction (device metadata for a forest of trees) and the
// multigrid drivers of arXiv:1701.04329 Sec. 3.2 on top of the kernels.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <stdexcept>

#include "grid.h"

namespace afg {

void check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        throw NoMem(std::string(what) + ": out of device memory");
    }
    throw CudaError(std::string(what) + ": " + cudaGetErrorString(e));
}

Allocator &allocator() {
    static Allocator a;
    return a;
}
int g_user_buffers = 0;

DeviceGuard::DeviceGuard(int dev) {
    int cur = 0;
    check(cudaGetDevice(&cur), "cudaGetDevice");
    if (cur != dev) {
        check(cudaSetDevice(dev), "cudaSetDevice");
        prev = cur;
    }
}

DeviceGuard::~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
}

int current_device() {
    int d = 0;
    check(cudaGetDevice(&d), "cudaGetDevice");
    return d;
}

DevBuf::DevBuf(size_t n) : bytes(n), from(allocator()) {
    if (n == 0) return;
    if (!from.alloc) {
        check(cudaMalloc(&p, n), "cudaMalloc");
        return;
    }
    p = from.alloc(n, from.ctx);
    if (!p) throw NoMem("the allocator callback returned NULL for " + std::to_string(n) + " bytes");
    ++g_user_buffers;
    if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {
        from.dealloc(p, from.ctx);
        --g_user_buffers;
        p = nullptr;
        throw std::runtime_error("the allocator callback returned memory that is not 256-byte aligned");
    }
}

DevBuf::~DevBuf() {
    if (!p) return;
    if (from.alloc) {
        from.dealloc(p, from.ctx);
        --g_user_buffers;
    } else {
        cudaFree(p);
    }
}

namespace {
template <typename T>
T *upload(const std::vector<T> &v, std::vector<std::unique_ptr<DevBuf>> &owned) {
    owned.emplace_back(new DevBuf(std::max<size_t>(1, v.size()) * sizeof(T)));
    if (!v.empty()) check(cudaMemcpy(owned.back()->p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
    return owned.back()->as<T>();
}
}  // namespace

Grid::Grid(const std::vector<const HostTree *> &trees, bool levels_only) {
    device = current_device();
    D = trees[0]->D;
    N = trees[0]->N;
    T = (int)trees.size();
    // Below level 1 every root box has its coarse grids of N/2, ..., 2 cells
    // (Sec. 3.2), connected like the roots.  A single tree whose level 1 is a
    // block of root boxes small enough for one CTA's shared memory keeps them
    // there only (k_bottom_block); otherwise they are device boxes, one per
    // root and level, and the cycle runs on the per-level kernels down to the
    // coarsest grid (several roots: `roots_levels`), or, with one root per
    // tree, in one launch per cycle (k_bottom).
    bool multi = false;
    for (const HostTree *h : trees) multi |= h->nroots() != 1;
    block = T == 1 && multi && !levels_only &&
            bottom_block_smem(D, true, N, trees[0]->nr, trees[0]->bct) <= max_smem_optin();
    roots_levels = multi && !block;
    for (const HostTree *h : trees) {
        bool dir = false;
        for (int s2 = 0; s2 < 2 * D; ++s2) dir |= h->bct[s2] == 0;
        singular |= !dir;
        tree_sing.push_back(!dir);
    }
    if (singular && multi)
        throw std::runtime_error("problems without a Dirichlet side are solved for trees of one root box");
    int nsub = 0;
    if (!block)
        for (int m = N / 2; m >= 2; m /= 2) ++nsub;
    lmin = 1 - nsub;
    lmax = 1;
    tree_top.resize(T);
    for (int t = 0; t < T; ++t) {
        tree_top[t] = trees[t]->L;
        lmax = std::max(lmax, trees[t]->L);
        tree_cells.push_back(trees[t]->n_leaf_cells);
        tree_faces.push_back(trees[t]->n_bfaces);
    }
    // one tree of one root box: level 2 (the root's 2^D children, one grid of
    // 2N cells per side) joins the bottom launch where it fits shared memory
    if (T == 1 && !multi && lmax >= 2) {
        const long long cells2 = D == 2 ? 4LL * N * N : 8LL * N * N * N;
        btop32 = bottom_smem(D, false, 2 * N) <= max_smem_optin() ? 2 : 1;
        btop64 = cells2 <= 1024 && bottom_smem(D, true, 2 * N) <= max_smem_optin() ? 2 : 1;
    }
    // global box ids: level-major, then tree, then the tree's canonical order
    std::vector<std::vector<int>> gid(T), sub(T, std::vector<int>(nsub, -1));
    for (int t = 0; t < T; ++t) gid[t].assign(trees[t]->boxes.size(), -1);
    int next = 0;
    long long cells = 0;
    for (int l = lmin; l <= lmax; ++l) {
        Level v{};
        v.l = l;
        v.M = l <= 0 ? (N >> (1 - l)) : N;
        v.MP = l == lmin ? 0 : (l <= 1 ? v.M / 2 : N);
        v.h = 1.0 / std::ldexp((double)N, l - 1);
        v.b0 = next;
        cells = (cells + 63) / 64 * 64;  // 64-cell alignment keeps every box 16-byte aligned for vector loads
        v.c0 = cells;
        for (int t = 0; t < T; ++t) {
            if (l <= 0) {  // one box per root box of the tree, in the roots' order
                sub[t][l - lmin] = next;
                next += trees[t]->nroots();
                continue;
            }
            const HostTree &ht = *trees[t];
            if (l > ht.L) continue;
            for (int b = ht.lstart[l]; b < ht.lstart[l] + ht.lcount[l]; ++b) gid[t][b] = next++;
        }
        v.nb = next - v.b0;
        const long long cpb = D == 2 ? (long long)v.M * v.M : (long long)v.M * v.M * v.M;
        v.ncell = cpb * v.nb;
        cells += v.ncell;
        lv.push_back(v);
    }
    nbox = next;
    ncell = cells;
    const int S = 2 * D, NC = 1 << D;
    std::vector<int> nb(nbox * S, -1), parent(nbox, -1), poff(nbox, 0), tree(nbox, 0), child(nbox * NC, -1);
    const int NDIR = D == 2 ? 8 : 26;
    std::vector<int> nball((size_t)nbox * NDIR, -1);
    std::vector<long long> coff(nbox, 0);
    std::vector<unsigned char> bflag(nbox, 0);
    std::vector<double> hb(nbox, 0.0), x0(nbox, 0.0);  // x0: below level 1 the single root's origin, 0
    for (auto &v : lv) {
        const long long cpb = v.ncell / std::max(1, v.nb);
        for (int i = 0; i < v.nb; ++i) {
            coff[v.b0 + i] = v.c0 + i * cpb;
            hb[v.b0 + i] = v.h;
        }
    }
    for (int t = 0; t < T; ++t) {
        const HostTree &ht = *trees[t];
        const int r1 = ht.lstart[1];
        for (int i = 0; i < nsub; ++i)
            for (int r = 0; r < ht.nroots(); ++r) {
                const int g = sub[t][i] + r;
                const HBox &root = ht.boxes[r1 + r];
                parent[g] = i > 0 ? sub[t][i - 1] + r : -1;
                bflag[g] = BF_REFINED | BF_SPECIAL;
                tree[g] = t;
                x0[g] = root.idx[0] - 1;  // unit root boxes
                child[g * NC] = i + 1 < nsub ? sub[t][i + 1] + r : gid[t][r1 + r];
                for (int s = 0; s < S; ++s) {  // connected like the roots (a root is its own periodic neighbour)
                    const int q = root.nb[ht.side_dir(s)];
                    if (q >= 0) nb[g * S + s] = sub[t][i] + (q - r1);
                }
                for (int d = 0; d < NDIR; ++d)
                    if (root.nb[d] >= 0) nball[(size_t)g * NDIR + d] = sub[t][i] + (root.nb[d] - r1);
            }
        for (int b = 0; b < (int)ht.boxes.size(); ++b) {
            const HBox &hx = ht.boxes[b];
            const int g = gid[t][b];
            tree[g] = t;
            x0[g] = (hx.idx[0] - 1) * N * hb[g];
            if (hx.level == 1) {
                parent[g] = nsub > 0 ? sub[t][nsub - 1] + (b - ht.lstart[1]) : -1;
            } else {
                parent[g] = gid[t][hx.parent];
                int p = 0;
                for (int a = 0; a < D; ++a) p |= (((hx.idx[a] - 1) & 1) * (N / 2)) << (8 * a);
                poff[g] = p;
            }
            bool special = false;
            for (int s = 0; s < S; ++s) {
                const int q = hx.nb[ht.side_dir(s)];
                if (q >= 0) nb[g * S + s] = gid[t][q];
                else if (q == -2) { nb[g * S + s] = -1; special = true; }
                else {
                    const int cq = ht.boxes[hx.parent].nb[ht.side_dir(s)];
                    if (cq < 0) throw std::runtime_error("tree is not 2:1 balanced");
                    nb[g * S + s] = -2 - gid[t][cq];
                    special = true;
                }
            }
            bflag[g] = (hx.leaf() ? 0 : BF_REFINED) | (special ? BF_SPECIAL : 0);
            for (int d = 0; d < NDIR; ++d)
                if (hx.nb[d] >= 0) nball[(size_t)g * NDIR + d] = gid[t][hx.nb[d]];
            for (int c = 0; c < NC; ++c) child[g * NC + c] = hx.child[c] >= 0 ? gid[t][hx.child[c]] : -1;
        }
    }
    // sibling groups: on every level from 2 up the boxes of a parent are
    // consecutive (Morton order) with child c at offset bit a = (c >> a) & 1
    for (auto &v : lv) {
        if (v.l < 2 || v.nb % NC) continue;
        bool ok = true;
        for (int q = 0; ok && q < v.nb / NC; ++q)
            for (int c = 0; ok && c < NC; ++c) {
                const int g = v.b0 + NC * q + c;
                int want = 0;
                for (int a = 0; a < D; ++a) want |= (((c >> a) & 1) * (N / 2)) << (8 * a);
                ok = parent[g] == parent[v.b0 + NC * q] && poff[g] == want;
            }
        v.sibs = ok;
    }
    // Dirichlet storage: leaf faces first, in canonical (tree-major) order, so
    // that user face arrays map onto it directly; then the coarse boxes' faces.
    std::vector<int> bcoff(nbox * S, -1), leaves;
    long long off = 0;
    std::vector<double> leaf_geo;
    for (int t = 0; t < T; ++t)
        for (int b : trees[t]->leaves) {
            leaves.push_back(gid[t][b]);
            const HBox &hx = trees[t]->boxes[b];
            const double hh = 1.0 / std::ldexp((double)N, hx.level - 1);
            for (int a = 0; a < 3; ++a) leaf_geo.push_back(a < D ? (hx.idx[a] - 1) * N * hh : 0.0);
            leaf_geo.push_back(hh);
        }
    n_leaf_boxes = (int)leaves.size();
    const int F = D == 2 ? N : N * N;
    for (int g : leaves)
        for (int s = 0; s < S; ++s)
            if (nb[g * S + s] == -1) { bcoff[g * S + s] = (int)off; off += F; }
    n_bfaces = off;
    for (auto &v : lv) {
        const int Fl = D == 2 ? v.M : v.M * v.M;
        for (int g = v.b0; g < v.b0 + v.nb; ++g) {
            if (!(bflag[g] & BF_REFINED)) continue;
            for (int s = 0; s < S; ++s)
                if (nb[g * S + s] == -1) { bcoff[g * S + s] = (int)off; off += Fl; }
        }
    }
    nbc = off;
    // per side: the cells of the box a ghost reads from, or its Dirichlet data
    std::vector<long long> nbase(nbox * S, 0);
    for (int g = 0; g < nbox; ++g)
        for (int s = 0; s < S; ++s) {
            const int code = nb[g * S + s];
            if (code >= 0) nbase[g * S + s] = coff[code];
            else if (code == -1) nbase[g * S + s] = bcoff[g * S + s];
            else nbase[g * S + s] = coff[-2 - code];
        }
    n_leaf_cells = (long long)n_leaf_boxes * (D == 2 ? N * N : N * N * N);

    // Neumann domain sides of every box (bit s), from its tree's side types
    std::vector<unsigned char> nmask(nbox, 0);
    for (int g = 0; g < nbox; ++g) {
        for (int s = 0; s < S; ++s)
            if (nb[g * S + s] == -1 && trees[tree[g]]->bct[s] == 1) nmask[g] |= (unsigned char)(1u << s);
        bflag[g] |= (unsigned char)(nmask[g] << BF_NSHIFT);  // kernels read it with the flags
    }

    auto &own = owned;
    if (block) {  // the roots' box ids in block order
        const HostTree &ht = *trees[0];
        for (int a = 0; a < 3; ++a) block_nroot[a] = ht.nr[a];
        for (int s2 = 0; s2 < 6; ++s2) block_bct[s2] = ht.bct[s2];
        std::vector<int> rb(ht.nroots(), -1);
        for (int b = ht.lstart[1]; b < ht.lstart[1] + ht.lcount[1]; ++b) {
            const HBox &hx = ht.boxes[b];
            rb[(hx.idx[0] - 1) + ht.nr[0] * ((hx.idx[1] - 1) + ht.nr[1] * (D == 3 ? hx.idx[2] - 1 : 0))] = gid[0][b];
        }
        d_root_box = upload(rb, own);
    }
    meta.nb = upload(nb, own);
    meta.nmask = upload(nmask, own);
    std::vector<unsigned char> cfmask(nbox, 0);
    for (int g = 0; g < nbox; ++g)
        for (int s = 0; s < S; ++s)
            if (nb[g * S + s] <= -2) cfmask[g] |= (unsigned char)(1u << s);
    meta.cfmask = upload(cfmask, own);
    meta.parent = upload(parent, own);
    meta.poff = upload(poff, own);
    meta.coff = upload(coff, own);
    meta.bcoff = upload(bcoff, own);
    meta.bflag = upload(bflag, own);
    meta.tree = upload(tree, own);
    meta.hb = d_hb = upload(hb, own);
    meta.nbase = upload(nbase, own);
    meta.x0 = d_x0 = upload(x0, own);
    d_nball = upload(nball, own);
    std::vector<double> ih2(nbox);
    for (int b = 0; b < nbox; ++b) ih2[b] = 1.0 / (hb[b] * hb[b]);
    meta.ih2 = upload(ih2, own);
    meta.active = nullptr;
    d_child = upload(child, own);
    d_leaves = upload(leaves, own);
    d_leaf_geo = upload(leaf_geo, own);
    if (singular && T > 1) {  // forests: per-tree compatibility constants and means
        std::vector<int> leaf0(T + 1, 0);
        for (int t = 0; t < T; ++t) leaf0[t + 1] = leaf0[t] + (int)trees[t]->leaves.size();
        d_tree_leaf0 = upload(leaf0, own);
        d_tree_sing = upload(tree_sing, own);
        d_tree_c = upload(std::vector<double>(T, 0.0), own);
    }
    // boxes (level >= 2) whose parent has a same-level leaf across a face
    std::vector<int> cfc;
    for (auto &v : lv) {
        if (v.l < 2) continue;
        for (int g = v.b0; g < v.b0 + v.nb; ++g) {
            const int p = parent[g];
            bool faces_leaf = false;
            for (int s = 0; s < S; ++s) {
                const int q = nb[p * S + s];
                if (q >= 0 && !(bflag[q] & BF_REFINED)) faces_leaf = true;
            }
            if (faces_leaf) cfc.push_back(g);
        }
    }
    n_cf_children = (int)cfc.size();
    d_cf_children = cfc.empty() ? nullptr : upload(cfc, own);
    own.emplace_back(new DevBuf(std::max<long long>(1, nbc) * sizeof(double)));
    d_bc = own.back()->as<double>();
    check(cudaMemset(d_bc, 0, std::max<long long>(1, nbc) * sizeof(double)), "memset bc");
    meta.bc = d_bc;
    // FMG masks (tree active on FMG step l iff it reaches level l) + convergence mask
    std::vector<int> masks((size_t)(lmax - lmin + 2) * T, 1);
    for (int l = lmin; l <= lmax; ++l)
        for (int t = 0; t < T; ++t) masks[(size_t)(l - lmin) * T + t] = tree_top[t] >= l;
    d_masks = upload(masks, own);
    own.emplace_back(new DevBuf(2 * T * sizeof(unsigned long long)));
    d_norms = own.back()->as<unsigned long long>();
    own.emplace_back(new DevBuf(sizeof(int)));
    d_nactive = own.back()->as<int>();
    own.emplace_back(new DevBuf(kPartials * sizeof(double)));
    d_partials = own.back()->as<double>();
    own.emplace_back(new DevBuf(sizeof(double)));
    d_scalar = own.back()->as<double>();
    own.emplace_back(new DevBuf(sizeof(double)));
    d_tol = own.back()->as<double>();
    check(cudaMallocHost((void **)&h_norms, 2 * T * sizeof(unsigned long long)), "cudaMallocHost");
    check(cudaMallocHost((void **)&h_nactive, sizeof(int)), "cudaMallocHost");
    check(cudaMallocHost((void **)&h_scalar, sizeof(double)), "cudaMallocHost");
    alloc_ws(ws64, true);
}

Grid::~Grid() {
    // cudaFree waits for the device; a caller's deallocator may hand the
    // memory to other work at once, so wait for this grid's kernels first
    if (allocator().alloc || g_user_buffers > 0) cudaDeviceSynchronize();
    clear_graphs();
    if (h_norms) cudaFreeHost(h_norms);
    if (h_nactive) cudaFreeHost(h_nactive);
    if (h_scalar) cudaFreeHost(h_scalar);
}

void Grid::clear_graphs() {
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
}

void Grid::alloc_ws(Workspace &w, bool fp64) {
    const size_t bytes = (size_t)ncell * (fp64 ? 8 : 4);
    w.fp64 = fp64;
    w.u.reset(new DevBuf(bytes));
    w.rho.reset(new DevBuf(bytes));
    w.vold.reset(new DevBuf(bytes));
    check(cudaMemset(w.u->p, 0, bytes), "memset");
    check(cudaMemset(w.rho->p, 0, bytes), "memset");
    check(cudaMemset(w.vold->p, 0, bytes), "memset");
    if (fp64) {
        w.rhoh.reset(new DevBuf(bytes));
        check(cudaMemset(w.rhoh->p, 0, bytes), "memset");
    }
}

void Grid::leaf_rho_hat(Workspace &w, cudaStream_t s) {
    if (w.rhoh) launch_rho_hat(leaf_cfg(w.fp64, s), meta, d_leaves, n_leaf_boxes, w.rho->p, w.rhoh->p);
}

void Grid::ensure_mixed() {
    if (!ws32.u) alloc_ws(ws32, false);
}

void Grid::ensure_adjoint() {
    if (!wsadj.u) alloc_ws(wsadj, true);
    while (bicg.size() < 10) {
        bicg.emplace_back(new DevBuf((size_t)ncell * 8));
        check(cudaMemset(bicg.back()->p, 0, (size_t)ncell * 8), "memset");
    }
}

// ---- multigrid building blocks --------------------------------------------

void Grid::smooth(Workspace &w, int l, int steps, int hom, const int *active, cudaStream_t s) {
    Level &v = L(l);
    BoxMeta A = meta;
    A.active = active;
    LaunchCfg c = cfg(l, w.fp64, s);
    c.vpt = vpt;
    for (int it = 0; it < steps; ++it)
        for (int col = 0; col < 2; ++col) {
            if (op) launch_var_smooth(c, A, v.b0, v.nb, w.u->p, w.rho->p, eps_of(w), col, hom, op);
            else launch_smooth(c, A, v.b0, v.nb, nullptr, w.u->p, w.rho->p, w.rhoh_p(), v.h * v.h, col, hom);
        }
}

// Residual on level l restricted to l-1 with v_H <- I v_h, v'_H <- v_H, then
// rho_H <- I r_h + A_H(v_H) on the refined boxes of l-1 (Eq. residual,
// Eq. coarse-rhs); leaves of l-1 store v' too.
void Grid::down_step(Workspace &w, int l, int hom, const int *active, cudaStream_t s) {
    Level &v = L(l), &vc = L(l - 1);
    BoxMeta A = meta;
    A.active = active;
    if (op) {
        launch_var_resid_restrict(cfg(l, w.fp64, s), A, v.b0, v.nb, w.u->p, w.rho->p, w.vold->p, eps_of(w), hom, op);
        launch_var_fas(cfg(l - 1, w.fp64, s), A, vc.b0, vc.nb, w.u->p, w.rho->p, w.vold->p, eps_of(w), hom, op);
        return;
    }
    launch_resid_restrict(cfg(l, w.fp64, s), A, v.b0, v.nb, w.u->p, w.rho->p, w.vold->p, 1.0 / (v.h * v.h), hom);
    launch_fas(cfg(l - 1, w.fp64, s), A, vc.b0, vc.nb, w.u->p, w.rho->p, w.vold->p, 1.0 / (vc.h * vc.h), hom,
               w.rhoh_p());
}

void Grid::bottom(Workspace &w, int ltop, int mode, const MgOpts &o, int hom, const int *active, cudaStream_t s) {
    BoxMeta A = meta;
    A.active = active;
    if (block) {  // one tree: level 1 and the grids below it in one CTA
        launch_bottom_block(cfg(1, w.fp64, s), A, block_nroot, block_bct, d_root_box, N, mode, w.u->p, w.rho->p,
                            w.vold->p, o.n_down, o.n_up, o.n_base, hom);
        return;
    }
    const int top = btop(w);
    int b0[kBottomLevels] = {};
    for (int l = lmin; l <= top; ++l) b0[l - lmin] = L(l).b0;
    launch_bottom(cfg(1, w.fp64, s), A, T, N, lmin, ltop, top, mode, w.u->p, w.rho->p, w.vold->p, o.n_down, o.n_up,
                  o.n_base, hom, b0);
}

// FAS V-cycle (Sec. 3.2) from ltop down to the coarsest grid and back.  The
// levels at and below btop(w) (the root box, or level 2 of a one-root tree)
// run in one launch (k_bottom).
void Grid::vcycle(Workspace &w, int ltop, const MgOpts &o, int hom, const int *active, cudaStream_t s) {
    if (levels_path()) {
        vcycle_levels(w, ltop, o, hom, active, s);
        return;
    }
    const int top = btop(w);
    for (int l = ltop; l > top; --l) {
        smooth(w, l, o.n_down, hom, active, s);
        down_step(w, l, hom, active, s);
    }
    bottom(w, ltop < top ? ltop : top, 0, o, hom, active, s);
    for (int l = top + 1; l <= ltop; ++l) {
        correct(w, l, active, s);
        smooth(w, l, o.n_up, hom, active, s);
    }
}

// FMG cycle (Sec. 3.2): restrict the current solution down, set the coarse
// right-hand sides, then for l = coarsest..finest: store v'_l, correct from
// l-1 and run a V-cycle from l.  In a forest a tree leaves the loop after its
// own finest level (masked).
void Grid::fmg(Workspace &w, const MgOpts &o, int hom, bool masked, cudaStream_t s) {
    for (int l = lmax; l > lmin; --l) restrict_u(w, l, L(l).b0, L(l).nb, nullptr, s);
    for (int l = lmax; l > lmin; --l) down_step(w, l, hom, nullptr, s);
    const size_t es = w.fp64 ? 8 : 4;
    // steps l = lmin..btop in one launch (every tree reaches level btop)
    const int l0 = levels_path() ? 1 : btop(w);
    if (levels_path()) fmg_low_levels(w, o, hom, s);
    else bottom(w, l0, 1, o, hom, nullptr, s);
    for (int l = l0 + 1; l <= lmax; ++l) {
        Level &v = L(l);
        const int *active = masked ? fmg_mask(l) : nullptr;
        check(cudaMemcpyAsync((char *)w.vold->p + v.c0 * es, (char *)w.u->p + v.c0 * es, v.ncell * es,
                              cudaMemcpyDeviceToDevice, s), "copy v'");
        if (l > lmin) correct(w, l, active, s);
        vcycle(w, l, o, hom, active, s);
    }
}

// u restricted to every parent (levels lmax..2), so that leaves next to a
// refined same-level box see the mean of the fine cells.
void Grid::restrict_all(Workspace &w, cudaStream_t s) {
    for (int l = lmax; l >= 2; --l) restrict_u(w, l, L(l).b0, L(l).nb, nullptr, s);
}

// (r,z): every restriction is the mean weighted by the children's r
void Grid::restrict_u(Workspace &w, int l, int b0, int n, const int *list, cudaStream_t s) {
    if (op == 2) launch_var_restrict(cfg(l, w.fp64, s), meta, b0, n, list, w.u->p, op);
    else launch_restrict_u(cfg(l, w.fp64, s), meta, b0, n, list, w.u->p);
}

// Variable-coefficient operators: the V-cycle on the per-level kernels all
// the way down (the coarse grids below the root have one box per tree),
// N_base steps on the 2^D-cell grid.
void Grid::vcycle_levels(Workspace &w, int ltop, const MgOpts &o, int hom, const int *active, cudaStream_t s) {
    for (int l = ltop; l > lmin; --l) {
        smooth(w, l, o.n_down, hom, active, s);
        down_step(w, l, hom, active, s);
    }
    smooth(w, lmin, o.n_base, hom, active, s);
    for (int l = lmin + 1; l <= ltop; ++l) {
        correct(w, l, active, s);
        smooth(w, l, o.n_up, hom, active, s);
    }
}

// coarse-grid correction of level l from l-1 with the grid's prolongation
void Grid::correct(Workspace &w, int l, const int *active, cudaStream_t s) {
    Level &v = L(l);
    BoxMeta A = meta;
    A.active = active;
    if (prolong) launch_correct_x(cfg(l, w.fp64, s), A, v.b0, v.nb, w.u->p, w.vold->p, d_nball, prolong);
    else launch_correct(cfg(l, w.fp64, s), A, v.b0, v.nb, w.u->p, w.vold->p);
}

// the FMG steps l = lmin..1 (Sec. 3.2) for the variable-coefficient operators
void Grid::fmg_low_levels(Workspace &w, const MgOpts &o, int hom, cudaStream_t s) {
    const size_t es = w.fp64 ? 8 : 4;
    for (int l = lmin; l <= 1; ++l) {
        Level &v = L(l);
        check(cudaMemcpyAsync((char *)w.vold->p + v.c0 * es, (char *)w.u->p + v.c0 * es, v.ncell * es,
                              cudaMemcpyDeviceToDevice, s), "copy v'");
        if (l > lmin) correct(w, l, nullptr, s);
        vcycle_levels(w, l, o, hom, nullptr, s);
    }
}

// Problems without a Dirichlet side: A u = rho - c with c the volume-weighted
// mean of rho less the Neumann inflow per volume (idempotent: c = 0 for a
// compatible source), and the solution of zero volume-weighted mean.
void Grid::make_compatible(cudaStream_t s) {
    if (!singular) return;
    launch_leaf_center(*this, ws64.rho->as<double>(), true, s);
    leaf_rho_hat(ws64, s);
}

void Grid::remove_mean(Workspace &w, cudaStream_t s) {
    if (singular && w.fp64) launch_leaf_center(*this, w.u->as<double>(), false, s);
}

// eps on the leaves, restricted to every parent (level by level, finest
// first), and its FP32 copy
void Grid::set_eps(const double *eps_leaf, cudaStream_t s) {
    if (!eps64) {
        eps64.reset(new DevBuf((size_t)ncell * 8));
        check(cudaMemsetAsync(eps64->p, 0, (size_t)ncell * 8, s), "memset eps");
    }
    if (!eps32) eps32.reset(new DevBuf((size_t)ncell * 4));
    launch_leaf_set(leaf_cfg(true, s), meta, d_leaves, n_leaf_boxes, eps_leaf, eps64->p);
    for (int l = lmax; l > lmin; --l) launch_var_restrict(cfg(l, true, s), meta, L(l).b0, L(l).nb, nullptr, eps64->p, op);
    launch_to_f32(eps64->as<double>(), eps32->as<float>(), ncell, s);
    eps_set = true;
}

// The composite residual reads a parent's values only where the parent
// faces a same-level leaf; by 2:1 balance the children of such a parent are
// leaves, so one pass over their list restricts everything it reads.
void Grid::restrict_cf(Workspace &w, cudaStream_t s) {
    if (n_cf_children > 0) restrict_u(w, 2, 0, n_cf_children, d_cf_children, s);
}

void Grid::norms_async(Workspace &w, int hom, void *rout, bool rout_f32, cudaStream_t s) {
    restrict_cf(w, s);
    check(cudaMemsetAsync(d_norms, 0, 2 * T * sizeof(unsigned long long), s), "memset norms");
    if (op)
        launch_var_leaf_residual(leaf_cfg(w.fp64, s), meta, d_leaves, n_leaf_boxes, w.u->p, w.rho->p, eps_of(w), hom,
                                 op, d_norms, d_norms + T, rout, rout_f32);
    else
        launch_leaf_residual(leaf_cfg(w.fp64, s), meta, d_leaves, n_leaf_boxes, w.u->p, w.rho->p, hom, d_norms,
                             d_norms + T, rout, rout_f32);
    check(cudaMemcpyAsync(h_norms, d_norms, 2 * T * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s),
          "norms to host");
}

void Grid::set_tol(double tol, cudaStream_t s) {
    *h_scalar = tol;
    check(cudaMemcpyAsync(d_tol, h_scalar, sizeof(double), cudaMemcpyHostToDevice, s), "tol");
    check(cudaStreamSynchronize(s), "tol");
}

void Grid::mask_update_async(cudaStream_t s) {
    launch_mask_update(s, d_norms, T, d_tol, d_converged_mask(), d_nactive);
    check(cudaMemcpyAsync(h_nactive, d_nactive, sizeof(int), cudaMemcpyDeviceToHost, s), "nactive");
}

}  // namespace afg
