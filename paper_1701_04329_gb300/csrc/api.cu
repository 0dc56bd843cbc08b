// C interface of libafgpu (include/afgpu.h): handles, error reporting and the
// solve drivers -- FAS FMG + V-cycles (arXiv:1701.04329 Sec. 3.2), the
// mixed-precision defect correction, the adjoint solve and batched forests.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <memory>
#include <string>
#include <vector>

#include "../../include/afgpu.h"
#include "handles.h"

using afg::Grid;
using afg::HostTree;
using afg::HBox;

namespace {
thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define AFG_API_BEGIN try {
// inside AFG_API_BEGIN: run the rest of the call on the handle's device
#define AFG_ON_DEVICE(h) afg::DeviceGuard afg_device_guard_((h)->device_for_call())
#define AFG_ON_FOREST_DEVICE(f) afg::DeviceGuard afg_device_guard_((f)->device)
#define AFG_API_END                                                      \
    }                                                                    \
    catch (const afg::NoMem &e) { return fail(AFG_ERR_NOMEM, e.what()); } \
    catch (const afg::CudaError &e) { return fail(AFG_ERR_CUDA, e.what()); } \
    catch (const std::bad_alloc &) { return fail(AFG_ERR_NOMEM, "host allocation failed"); } \
    catch (const std::exception &e) { return fail(AFG_ERR_STATE, e.what()); }

using afg::check;

// The capture stream: graphs are recorded on a private non-blocking stream
// (capture is not allowed on the legacy default stream) and replayed on the
// caller's stream.
cudaStream_t capture_stream() {
    static thread_local cudaStream_t s = nullptr;
    if (!s) check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
    return s;
}

template <typename F>
void run(Grid &g, std::tuple<int, int, int, int, int> key, bool use_graph, cudaStream_t s, F &&body) {
    std::get<0>(key) += 1000 * g.vpt;  // a graph per threads-per-box choice
    if (!use_graph) {
        body(s);
        return;
    }
    auto it = g.graphs.find(key);
    if (it == g.graphs.end()) {
        cudaStream_t cs = capture_stream();
        check(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        try {
            body(cs);
        } catch (...) {
            cudaGraph_t gr = nullptr;
            cudaStreamEndCapture(cs, &gr);
            if (gr) cudaGraphDestroy(gr);
            cudaGetLastError();  // the invalidated capture's status must not reach the next call
            throw;
        }
        cudaGraph_t gr;
        check(cudaStreamEndCapture(cs, &gr), "cudaStreamEndCapture");
        size_t nn = 0;
        check(cudaGraphGetNodes(gr, nullptr, &nn), "cudaGraphGetNodes");
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) check(cudaGraphGetNodes(gr, nodes.data(), &nn), "cudaGraphGetNodes");
        int kernels = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            check(cudaGraphNodeGetType(nd, &ty), "cudaGraphNodeGetType");
            kernels += ty == cudaGraphNodeTypeKernel;
        }
        cudaGraphExec_t ex;
        cudaError_t e = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        check(e, "cudaGraphInstantiate");
        it = g.graphs.emplace(key, ex).first;
        g.graph_kernels[key] = kernels;
        afg::g_launches -= kernels;  // the capture itself launched nothing
    }
    check(cudaGraphLaunch(it->second, s), "cudaGraphLaunch");
    afg::g_launches += g.graph_kernels[key];
}

afg_mg_opts opts_or_default(const afg_mg_opts *o) {
    afg_mg_opts d;
    afg_default_opts(&d);
    return o ? *o : d;
}

// threads per box of the FP32 half-sweep: 0 or one per 16-byte vector of a
// box's colour half (vpt 1), or half as many (vpt 2)
int vpt_of(const Grid &g, const afg_mg_opts &o, int *vpt) {
    const int half = (g.D == 2 ? g.N * g.N : g.N * g.N * g.N) / 2;
    const int nv = std::min(half / 4, 256);
    if (o.threads_per_box == 0 || o.threads_per_box == nv) *vpt = 1;
    else if (o.threads_per_box == nv / 2 && nv >= 2) *vpt = 2;
    else return fail(AFG_ERR_ARG, "threads_per_box must be 0, " + std::to_string(nv) + " or " +
                                      std::to_string(nv / 2) + " for these boxes");
    return AFG_OK;
}

int validate(const afg_mg_opts &o) {
    if (o.n_down < 0 || o.n_up < 0 || o.n_base < 1 || o.n_down > 64 || o.n_up > 64 || o.n_base > 1024)
        return fail(AFG_ERR_ARG, "smoothing steps out of range");
    if (o.max_cycles < 1 || !(o.rel_tol >= 0.0)) return fail(AFG_ERR_ARG, "bad max_cycles / rel_tol");
    if (o.precision != AFG_FP64 && o.precision != AFG_MIXED) return fail(AFG_ERR_ARG, "bad precision");
    if (o.inner_vcycles < 0 || o.inner_vcycles > 16) return fail(AFG_ERR_ARG, "inner_vcycles out of range");
    if (o.threads_per_box < 0) return fail(AFG_ERR_ARG, "threads_per_box out of range");
    return AFG_OK;
}

Grid &grid_of(afg_tree *t) {
    if (!t->grid || t->grid_version != t->ht.version) {
        t->grid.reset();
        std::vector<const HostTree *> v{&t->ht};
        t->grid.reset(new Grid(v, t->op || t->prolong));
        t->grid_version = t->ht.version;
        t->grid->op = t->op;
        t->grid->prolong = t->prolong;
    }
    return *t->grid;
}

// the multigrid calls need rho, and eps for the variable-coefficient operators
int ready(const Grid &g) {
    if (!g.rhs_set) return fail(AFG_ERR_STATE, "no right-hand side set");
    if (g.op && !g.eps_set) return fail(AFG_ERR_STATE, "the variable-coefficient operator needs eps (afg_set_eps)");
    return AFG_OK;
}

double as_double(unsigned long long bits) {
    double d;
    std::memcpy(&d, &bits, sizeof d);
    return d;
}

double rel_of(const Grid &g, int t) {
    const double r = as_double(g.h_norms[t]);
    const double p = as_double(g.h_norms[g.T + t]);
    return p > 0.0 ? r / p : r;
}

void fill_stats(afg_stats *st, const Grid &g, int t, int cycles, double secs) {
    if (!st) return;
    st->cycles = cycles;
    st->max_residual = as_double(g.h_norms[t]);
    st->max_rho = as_double(g.h_norms[g.T + t]);
    st->rel_residual = rel_of(g, t);
    st->seconds = secs;
}

using clk = std::chrono::steady_clock;

}  // namespace

int afg::api_fail(int code, const std::string &msg) { return fail(code, msg); }

namespace {

// FMG then V-cycles (plain FP64), all trees of the grid together; a tree that
// reached rel_tol is masked out of later cycles.  Returns cycles done.
int solve_fp64(Grid &g, const afg_mg_opts &o, cudaStream_t s, std::vector<std::vector<double>> &hist,
               bool fmg_first) {
    const afg::MgOpts mo{o.n_down, o.n_up, o.n_base};
    const bool forest = g.T > 1;
    std::vector<int> ones(g.T, 1);
    check(cudaMemcpyAsync(g.d_converged_mask(), ones.data(), g.T * sizeof(int), cudaMemcpyHostToDevice, s), "mask");
    g.set_tol(o.rel_tol, s);
    int cycles = 0;
    hist.assign(g.T, {});
    auto record = [&]() {
        for (int t = 0; t < g.T; ++t)
            if (hist[t].empty() || hist[t].back() > o.rel_tol) hist[t].push_back(rel_of(g, t));
    };
    g.make_compatible(s);
    if (fmg_first) {
        run(g, {1, o.n_down, o.n_up, o.n_base, 0}, o.use_graph, s, [&](cudaStream_t cs) {
            g.fmg(g.ws64, mo, 0, forest, cs);
            g.remove_mean(g.ws64, cs);
            g.norms_async(g.ws64, 0, nullptr, false, cs);
            g.mask_update_async(cs);
        });
    } else {
        run(g, {3, 0, 0, 0, 0}, o.use_graph, s, [&](cudaStream_t cs) {
            g.norms_async(g.ws64, 0, nullptr, false, cs);
            g.mask_update_async(cs);
        });
    }
    check(cudaStreamSynchronize(s), "solve");
    cycles = fmg_first ? 1 : 0;
    record();
    while (*g.h_nactive > 0 && cycles < o.max_cycles) {
        run(g, {2, o.n_down, o.n_up, o.n_base, 0}, o.use_graph, s, [&](cudaStream_t cs) {
            g.vcycle(g.ws64, g.lmax, mo, 0, forest ? g.d_converged_mask() : nullptr, cs);
            g.remove_mean(g.ws64, cs);
            g.norms_async(g.ws64, 0, nullptr, false, cs);
            g.mask_update_async(cs);
        });
        check(cudaStreamSynchronize(s), "solve");
        ++cycles;
        record();
    }
    return cycles;
}

// Mixed precision (an addition to the paper's method): the FP64 composite
// residual r = rho - A x is formed on the leaves and cast to FP32; the FP32
// FAS multigrid solves A e = r with homogeneous boundary data (FMG on the
// first pass, inner_vcycles V-cycles afterwards); x += e in FP64.  Repeats
// until the FP64 relative residual reaches rel_tol.
int solve_mixed(Grid &g, const afg_mg_opts &o, cudaStream_t s, std::vector<std::vector<double>> &hist) {
    g.ensure_mixed();
    const afg::MgOpts mo{o.n_down, o.n_up, o.n_base};
    const bool forest = g.T > 1;
    std::vector<int> ones(g.T, 1);
    check(cudaMemcpyAsync(g.d_converged_mask(), ones.data(), g.T * sizeof(int), cudaMemcpyHostToDevice, s), "mask");
    g.set_tol(o.rel_tol, s);
    hist.assign(g.T, {});
    auto record = [&]() {
        for (int t = 0; t < g.T; ++t)
            if (hist[t].empty() || hist[t].back() > o.rel_tol) hist[t].push_back(rel_of(g, t));
    };
    const size_t bytes32 = (size_t)g.ncell * 4;
    g.make_compatible(s);
    auto residual = [&](cudaStream_t cs) {
        g.norms_async(g.ws64, 0, g.ws32.rho->p, true, cs);
        g.mask_update_async(cs);
    };
    run(g, {10, 0, 0, 0, 0}, o.use_graph, s, residual);
    check(cudaStreamSynchronize(s), "solve");
    // inner_vcycles 0, one tree: two V-cycles on the first step after FMG, then
    // as many as the reduction per V-cycle measured on the previous step says
    // reach the tolerance in this step (the FP64 residual passes are then as
    // few as the FP32 resolution allows); forests: two (trees converge at
    // different rates, and every active tree would take the worst one's count)
    auto worst = [&]() {
        double r = 0;
        for (int t = 0; t < g.T; ++t)
            if (!hist[t].empty() && hist[t].back() > o.rel_tol) r = std::max(r, hist[t].back());
        return r;
    };
    double rate = 0, r_prev = 0;  // reduction per V-cycle, measured
    int k_prev = 0;
    int cycles = 0;
    while (*g.h_nactive > 0 && cycles < o.max_cycles) {
        const bool first = cycles == 0;
        int k = o.inner_vcycles;
        if (!first && k == 0) {
            const double r = worst();
            if (k_prev > 0 && r_prev > 0 && r > 0)
                rate = std::min(0.5, std::max(0.01, std::pow(r / r_prev, 1.0 / k_prev)));
            k = 2;
            if (!forest && rate > 0) {
                const double need = r > o.rel_tol ? std::log(r / o.rel_tol) / -std::log(rate) : 1.0;
                // at most 1e-5 per pass: the FP32 solve's resolution bounds what one pass can gain
                const int kmax = std::max(1, (int)std::floor(std::log(1e-5) / std::log(rate)));
                k = std::min(kmax, std::max(1, (int)std::ceil(need - 1e-9)));
            }
            r_prev = r;
            k_prev = k;
        }
        run(g, {first ? 11 : 12, o.n_down, o.n_up, o.n_base, k}, o.use_graph, s,
            [&](cudaStream_t cs) {
                const int *active = forest ? g.d_converged_mask() : nullptr;
                check(cudaMemsetAsync(g.ws32.u->p, 0, bytes32, cs), "zero e");
                if (first) g.fmg(g.ws32, mo, 1, forest, cs);
                else
                    for (int q = 0; q < k; ++q) g.vcycle(g.ws32, g.lmax, mo, 1, active, cs);
                afg::BoxMeta A = g.meta;
                A.active = active;
                afg::launch_mixed_update(g.leaf_cfg(true, cs), A, g.d_leaves, g.n_leaf_boxes, g.ws64.u->as<double>(),
                                         g.ws32.u->as<float>());
                g.remove_mean(g.ws64, cs);
                residual(cs);
            });
        check(cudaStreamSynchronize(s), "solve");
        ++cycles;
        record();
    }
    return cycles;
}

double host_scalar(Grid &g, cudaStream_t s) {
    check(cudaMemcpyAsync(g.h_scalar, g.d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s), "scalar");
    check(cudaStreamSynchronize(s), "scalar");
    return *g.h_scalar;
}

// Adjoint (an addition to the paper's method): K^T lam = g for the
// transposed composite operator, by BiCGStab (van der Vorst 1992) with right
// preconditioner W M W^-1, where M is one linear FP64 V-cycle from zero with
// homogeneous boundary data and W the diagonal of cell volumes.  W K is
// symmetric up to the refinement-boundary terms, so W M W^-1 approximates
// K^-T.  Returns iterations; sets *rel to max|g - K^T lam| / max|g|.
int adjoint_solve(Grid &g, const afg_mg_opts &o, cudaStream_t s, const double *g_leaf, double *rel) {
    g.ensure_adjoint();
    const afg::MgOpts mo{o.n_down, o.n_up, o.n_base};
    const afg::LaunchCfg lc = g.leaf_cfg(true, s);
    const afg::BoxMeta &A = g.meta;
    const int *L = g.d_leaves;
    const int n = g.n_leaf_boxes;
    double *bvec = g.bicg[0]->as<double>(), *x = g.bicg[1]->as<double>(), *r = g.bicg[2]->as<double>(),
           *rh = g.bicg[3]->as<double>(), *p = g.bicg[4]->as<double>(), *v = g.bicg[5]->as<double>(),
           *sv = g.bicg[6]->as<double>(), *t = g.bicg[7]->as<double>(), *ph = g.bicg[8]->as<double>(),
           *sh = g.bicg[9]->as<double>();
    afg::launch_leaf_set(lc, A, L, n, g_leaf, bvec);
    auto dot = [&](const double *a, const double *b) {
        afg::launch_leaf_dot(lc, A, L, n, a, b, g.d_partials, g.d_scalar);
        return host_scalar(g, s);
    };
    auto amax = [&](const double *a) {
        afg::launch_leaf_absmax(lc, A, L, n, a, g.d_partials, g.d_scalar);
        return host_scalar(g, s);
    };
    const size_t bytes = (size_t)g.ncell * 8;
    // AFG_MIXED: M is one FP32 V-cycle (the BiCGStab recurrences and K^T stay FP64)
    const bool m32 = o.precision == AFG_MIXED;
    if (m32) g.ensure_mixed();
    auto precond = [&](const double *in, double *out, cudaStream_t cs) {
        afg::launch_leaf_scale(g.leaf_cfg(true, cs), A, g.d_hb, L, n, g.wsadj.rho->as<double>(), in, -1);
        if (m32) {
            afg::launch_to_f32(g.wsadj.rho->as<double>(), g.ws32.rho->as<float>(), g.ncell, cs);
            check(cudaMemsetAsync(g.ws32.u->p, 0, (size_t)g.ncell * 4, cs), "zero");
            g.vcycle(g.ws32, g.lmax, mo, 1, nullptr, cs);
            afg::launch_to_f64(g.ws32.u->as<float>(), g.wsadj.u->as<double>(), g.ncell, cs);
        } else {
            g.leaf_rho_hat(g.wsadj, cs);
            check(cudaMemsetAsync(g.wsadj.u->p, 0, bytes, cs), "zero");
            g.vcycle(g.wsadj, g.lmax, mo, 1, nullptr, cs);
        }
        afg::launch_leaf_scale(g.leaf_cfg(true, cs), A, g.d_hb, L, n, out, g.wsadj.u->as<double>(), 1);
    };
    auto apply_T = [&](const double *in, double *out) {
        afg::launch_adjoint_apply(lc, A, g.d_child, g.d_hb, L, n, in, out);
    };
    // graphs for the two preconditioner applications (fixed buffers)
    const int kp = m32 ? 22 : 20;
    auto P_p = [&]() {
        run(g, {kp, o.n_down, o.n_up, o.n_base, 0}, o.use_graph, s, [&](cudaStream_t cs) { precond(p, ph, cs); });
    };
    auto P_s = [&]() {
        run(g, {kp + 1, o.n_down, o.n_up, o.n_base, 0}, o.use_graph, s, [&](cudaStream_t cs) { precond(sv, sh, cs); });
    };

    const double bnorm = amax(bvec);
    check(cudaMemsetAsync(x, 0, bytes, s), "zero");
    if (bnorm == 0.0) {
        *rel = 0.0;
        return 0;
    }
    afg::launch_leaf_axpbypcz(lc, A, L, n, r, 1.0, bvec, 0.0, nullptr, 0.0, nullptr);
    afg::launch_leaf_axpbypcz(lc, A, L, n, rh, 1.0, bvec, 0.0, nullptr, 0.0, nullptr);
    check(cudaMemsetAsync(p, 0, bytes, s), "zero");
    check(cudaMemsetAsync(v, 0, bytes, s), "zero");
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    int it = 0;
    double res = 1.0;
    for (it = 1; it <= o.max_cycles; ++it) {
        const double rho_new = dot(rh, r);
        if (rho_new == 0.0) break;
        const double beta = (rho_new / rho_old) * (alpha / omega);
        afg::launch_leaf_axpbypcz(lc, A, L, n, p, 1.0, r, beta, p, -beta * omega, v);
        P_p();
        apply_T(ph, v);
        alpha = rho_new / dot(rh, v);
        afg::launch_leaf_axpbypcz(lc, A, L, n, sv, 1.0, r, -alpha, v, 0.0, nullptr);
        res = amax(sv) / bnorm;
        if (res <= o.rel_tol) {
            afg::launch_leaf_axpbypcz(lc, A, L, n, x, 1.0, x, alpha, ph, 0.0, nullptr);
            break;
        }
        P_s();
        apply_T(sh, t);
        const double tt = dot(t, t);
        omega = tt > 0.0 ? dot(t, sv) / tt : 0.0;
        afg::launch_leaf_axpbypcz(lc, A, L, n, x, 1.0, x, alpha, ph, omega, sh);
        afg::launch_leaf_axpbypcz(lc, A, L, n, r, 1.0, sv, -omega, t, 0.0, nullptr);
        res = amax(r) / bnorm;
        if (res <= o.rel_tol || omega == 0.0) break;
        rho_old = rho_new;
    }
    // true residual
    apply_T(x, t);
    afg::launch_leaf_axpbypcz(lc, A, L, n, r, 1.0, bvec, -1.0, t, 0.0, nullptr);
    *rel = amax(r) / bnorm;
    return std::min(it, o.max_cycles);
}

void set_dirichlet_dev(Grid &g, const double *b, cudaStream_t s) {
    if (g.n_bfaces > 0) {
        if (b) check(cudaMemcpyAsync(g.d_bc, b, g.n_bfaces * 8, cudaMemcpyDeviceToDevice, s), "copy b");
        else check(cudaMemsetAsync(g.d_bc, 0, g.n_bfaces * 8, s), "zero b");
    }
    for (int l = g.lmax; l > g.lmin; --l) {
        auto &v = g.L(l);
        afg::launch_bc_restrict(g.cfg(l, true, s), g.meta, v.b0, v.nb, g.d_bc);
    }
}

}  // namespace

extern "C" {

void afg_default_opts(afg_mg_opts *o) {
    if (!o) return;
    o->n_down = 2;
    o->n_up = 2;
    o->n_base = 4;
    o->max_cycles = 50;
    o->rel_tol = 1e-10;
    o->precision = AFG_FP64;
    o->inner_vcycles = 0;
    o->use_graph = 1;
    o->threads_per_box = 0;
}

const char *afg_last_error(void) { return g_err.c_str(); }

int afg_set_allocator(void *(*alloc)(size_t, void *), void (*dealloc)(void *, void *), void *ctx) {
    if ((alloc == nullptr) != (dealloc == nullptr)) return fail(AFG_ERR_ARG, "give both callbacks or neither");
    afg::Allocator &a = afg::allocator();
    a.alloc = alloc;
    a.dealloc = dealloc;
    a.ctx = alloc ? ctx : nullptr;
    return AFG_OK;
}

int afg_tree_create(int dim, int box_n, int max_level, afg_tree **out) {
    if (!out) return fail(AFG_ERR_ARG, "out is NULL");
    if (dim != 2 && dim != 3) return fail(AFG_ERR_ARG, "dim must be 2 or 3");
    if (box_n != 4 && box_n != 8 && box_n != 16) return fail(AFG_ERR_ARG, "box_n must be 4, 8 or 16");
    if (max_level < 1 || max_level > (dim == 3 ? 21 : 30)) return fail(AFG_ERR_ARG, "max_level out of range");
    AFG_API_BEGIN
    *out = new afg_tree(dim, box_n, max_level);
    return AFG_OK;
    AFG_API_END
}

int afg_tree_create_roots(int dim, int box_n, int max_level, const int *nroot, afg_tree **out) {
    if (!out || !nroot) return fail(AFG_ERR_ARG, "null argument");
    if (dim != 2 && dim != 3) return fail(AFG_ERR_ARG, "dim must be 2 or 3");
    if (box_n != 4 && box_n != 8 && box_n != 16) return fail(AFG_ERR_ARG, "box_n must be 4, 8 or 16");
    if (max_level < 1 || max_level > (dim == 3 ? 21 : 30)) return fail(AFG_ERR_ARG, "max_level out of range");
    for (int a = 0; a < dim; ++a) {
        if (nroot[a] < 1 || nroot[a] > 64) return fail(AFG_ERR_ARG, "root boxes per axis must be in [1, 64]");
        if (((long long)nroot[a] << (max_level - 1)) > (1LL << 21))
            return fail(AFG_ERR_ARG, "boxes per axis on max_level exceed 2^21 (Morton keys)");
    }
    AFG_API_BEGIN
    *out = new afg_tree(dim, box_n, max_level, nroot);
    return AFG_OK;
    AFG_API_END
}

int afg_tree_destroy(afg_tree *t) {
    delete t;
    return AFG_OK;
}

int afg_set_stream(afg_tree *t, void *stream) {
    if (!t) return fail(AFG_ERR_ARG, "null tree");
    t->stream = (cudaStream_t)stream;
    return AFG_OK;
}

int afg_refine_uniform(afg_tree *t, int level) {
    if (!t) return fail(AFG_ERR_ARG, "null tree");
    AFG_API_BEGIN
    std::string err;
    if (t->ht.refine_uniform(level, err)) return fail(AFG_ERR_ARG, err);
    return AFG_OK;
    AFG_API_END
}

int afg_cell_centers(const afg_tree *t, double *xyz) {
    if (!t || !xyz) return fail(AFG_ERR_ARG, "null argument");
    const HostTree &h = t->ht;
    const int N = h.N, D = h.D, nc = D == 2 ? N * N : N * N * N;
    long long o = 0;
    for (int b : h.leaves) {
        const double hh = 1.0 / std::ldexp((double)N, h.boxes[b].level - 1);
        for (int c = 0; c < nc; ++c, ++o) {
            const int ci[3] = {c % N, (c / N) % N, c / (N * N)};
            for (int a = 0; a < D; ++a) xyz[o * D + a] = ((h.boxes[b].idx[a] - 1) * N + ci[a] + 0.5) * hh;
        }
    }
    return AFG_OK;
}

int afg_cell_centers_device(afg_tree *t, double *xyz_dev) {
    if (!t || !xyz_dev) return fail(AFG_ERR_ARG, "null argument");
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &g = grid_of(t);
    afg::launch_cell_centers(g, xyz_dev, t->stream);
    return AFG_OK;
    AFG_API_END
}

int afg_face_centers(const afg_tree *t, double *xyz) {
    if (!t || !xyz) return fail(AFG_ERR_ARG, "null argument");
    const HostTree &h = t->ht;
    const int N = h.N, D = h.D, nf = D == 2 ? N : N * N;
    long long o = 0;
    for (int b : h.leaves) {
        const HBox &bx = h.boxes[b];
        const double hh = 1.0 / std::ldexp((double)N, bx.level - 1);
        for (int s = 0; s < 2 * D; ++s) {
            if (bx.nb[h.side_dir(s)] != -2) continue;
            const int a = s / 2;
            int ta[2] = {-1, -1}, k = 0;
            for (int e = 0; e < D; ++e)
                if (e != a) ta[k++] = e;
            for (int f = 0; f < nf; ++f, ++o) {
                double x[3];
                x[a] = (s & 1) ? (double)h.nr[a] : 0.0;
                x[ta[0]] = ((bx.idx[ta[0]] - 1) * N + f % N + 0.5) * hh;
                if (D == 3) x[ta[1]] = ((bx.idx[ta[1]] - 1) * N + f / N + 0.5) * hh;
                for (int e = 0; e < D; ++e) xyz[o * D + e] = x[e];
            }
        }
    }
    return AFG_OK;
}

int afg_leaf_levels(const afg_tree *t, int32_t *levels) {
    if (!t || !levels) return fail(AFG_ERR_ARG, "null argument");
    for (size_t i = 0; i < t->ht.leaves.size(); ++i) levels[i] = t->ht.boxes[t->ht.leaves[i]].level;
    return AFG_OK;
}

int afg_adapt(afg_tree *t, const int8_t *flags, int n_buf, int *n_added, int *n_removed) {
    if (!t || !flags) return fail(AFG_ERR_ARG, "null argument");
    AFG_API_BEGIN
    std::string err;
    const int rc = t->ht.adapt(flags, n_buf, n_added, n_removed, err);
    if (rc == -1) return fail(AFG_ERR_ARG, err);
    if (rc) return fail(AFG_ERR_STATE, err);
    return AFG_OK;
    AFG_API_END
}

int afg_adapt_transfer(afg_tree *t, const int8_t *flags, int n_buf, int scheme, int *n_added, int *n_removed) {
    if (!t || !flags) return fail(AFG_ERR_ARG, "null argument");
    if (scheme < 0 || scheme > 2) return fail(AFG_ERR_ARG, "scheme must be AFG_PROLONG_LINEAR, _MULTILINEAR or _ZEROTH");
    if (!t->grid || t->grid_version != t->ht.version)
        return fail(AFG_ERR_STATE, "no solution on the device to carry over (set or solve one first)");
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &old = *t->grid;
    cudaStream_t s = t->stream;
    old.restrict_all(old.ws64, s);  // a parent whose children go away becomes a leaf holding their mean
    const HostTree before(t->ht);
    std::string err;
    int added = 0, removed = 0;
    const int rc = t->ht.adapt(flags, n_buf, &added, &removed, err);
    if (rc == -1) return fail(AFG_ERR_ARG, err);
    if (rc) return fail(AFG_ERR_STATE, err);
    if (n_added) *n_added = added;
    if (n_removed) *n_removed = removed;
    std::unique_ptr<Grid> fresh;
    {
        std::vector<const HostTree *> v{&t->ht};
        fresh.reset(new Grid(v, t->op || t->prolong));
        fresh->op = t->op;
        fresh->prolong = t->prolong;
    }
    // per new leaf: the old box that holds its values, or the old leaf it is prolonged from
    const HostTree &now = t->ht;
    const int N = now.N, D = now.D, old_b1 = old.L(1).b0;
    std::vector<int> src(now.leaves.size()), poff(now.leaves.size());
    for (size_t li = 0; li < now.leaves.size(); ++li) {
        const HBox &nb = now.boxes[now.leaves[li]];
        const int same = before.find(nb.level, nb.idx);
        if (same >= 0) {
            src[li] = old_b1 + same;
            poff[li] = -1;
            continue;
        }
        int pidx[3] = {1, 1, 1}, po = 0;
        for (int a = 0; a < D; ++a) {
            pidx[a] = (nb.idx[a] + 1) / 2;
            po |= (((nb.idx[a] - 1) & 1) * (N / 2)) << (8 * a);
        }
        const int par = before.find(nb.level - 1, pidx);
        if (par < 0 || !before.boxes[par].leaf()) throw std::runtime_error("adapted leaf without a source box");
        src[li] = old_b1 + par;
        poff[li] = po;
    }
    afg::DevBuf d_src(src.size() * sizeof(int)), d_poff(poff.size() * sizeof(int));
    check(cudaMemcpyAsync(d_src.p, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice, s), "plan");
    check(cudaMemcpyAsync(d_poff.p, poff.data(), poff.size() * sizeof(int), cudaMemcpyHostToDevice, s), "plan");
    afg::launch_transfer(D, s, N, old.meta, old.ws64.u->as<double>(), old.d_nball, fresh->meta,
                         fresh->ws64.u->as<double>(), fresh->d_leaves, d_src.as<int>(), d_poff.as<int>(),
                         (int)src.size(), scheme);
    check(cudaGetLastError(), "afg_adapt_transfer");
    check(cudaStreamSynchronize(s), "afg_adapt_transfer");
    t->grid = std::move(fresh);
    t->grid_version = t->ht.version;
    return AFG_OK;
    AFG_API_END
}

int afg_flag_cells(afg_tree *t, const double *f_dev, int power, double tau_refine, double tau_coarsen,
                   int8_t *flags_dev) {
    if (!t || !f_dev || !flags_dev) return fail(AFG_ERR_ARG, "null argument");
    if (power < 0 || power > 8 || !(tau_coarsen <= tau_refine)) return fail(AFG_ERR_ARG, "bad power or thresholds");
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &g = grid_of(t);
    afg::launch_flag(g, f_dev, power, tau_refine, tau_coarsen, reinterpret_cast<signed char *>(flags_dev), t->stream);
    return AFG_OK;
    AFG_API_END
}

int afg_set_boundary_types(afg_tree *t, const int *types) {
    if (!t || !types) return fail(AFG_ERR_ARG, "null argument");
    if (t->op) {
        bool dir = false;
        for (int s2 = 0; s2 < 2 * t->ht.D; ++s2) dir |= types[s2] == 0;
        if (!dir) return fail(AFG_ERR_ARG, "the variable-coefficient operators need a Dirichlet side");
    }
    AFG_API_BEGIN
    std::string err;  // a change rebuilds the host tree (new version: the device grid follows)
    if (t->ht.set_boundary_types(types, err)) return fail(AFG_ERR_ARG, err);
    return AFG_OK;
    AFG_API_END
}

int afg_info(const afg_tree *t, afg_tree_info *out) {
    if (!t || !out) return fail(AFG_ERR_ARG, "null argument");
    const HostTree &h = t->ht;
    std::memset(out, 0, sizeof(*out));
    out->dim = h.D;
    out->box_n = h.N;
    out->max_level = h.max_level;
    out->highest_level = h.L;
    out->n_boxes = (int)h.boxes.size();
    out->n_leaves = (int)h.leaves.size();
    out->n_leaf_cells = h.n_leaf_cells;
    out->n_bfaces = h.n_bfaces;
    for (const auto &b : h.boxes)
        if (b.level < 32) {
            out->boxes_per_level[b.level]++;
            if (b.leaf()) out->leaves_per_level[b.level]++;
        }
    return AFG_OK;
}

int afg_export_tree(const afg_tree *t, int32_t *level, int32_t *idx, int32_t *parent, int32_t *children,
                    int32_t *neighbours) {
    if (!t) return fail(AFG_ERR_ARG, "null tree");
    const HostTree &h = t->ht;
    const int D = h.D, nc = 1 << D, nd = h.ndir();
    for (size_t i = 0; i < h.boxes.size(); ++i) {
        const HBox &b = h.boxes[i];
        if (level) level[i] = b.level;
        if (idx)
            for (int a = 0; a < D; ++a) idx[i * D + a] = b.idx[a];
        if (parent) parent[i] = b.parent;
        if (children)
            for (int c = 0; c < nc; ++c) children[i * nc + c] = b.child[c];
        if (neighbours)
            for (int d = 0; d < nd; ++d) neighbours[i * nd + d] = b.nb[d];
    }
    return AFG_OK;
}

int afg_set_rhs(afg_tree *t, const double *rho) {
    if (!t || !rho) return fail(AFG_ERR_ARG, "null argument");
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &g = grid_of(t);
    afg::launch_leaf_set(g.leaf_cfg(true, t->stream), g.meta, g.d_leaves, g.n_leaf_boxes, rho, g.ws64.rho->p);
    g.leaf_rho_hat(g.ws64, t->stream);
    check(cudaGetLastError(), "afg_set_rhs");
    g.rhs_set = true;
    return AFG_OK;
    AFG_API_END
}

int afg_set_operator(afg_tree *t, int op) {
    if (!t) return fail(AFG_ERR_ARG, "null tree");
    if (op < 0 || op > 2) return fail(AFG_ERR_ARG, "op must be AFG_OP_LAPLACE, AFG_OP_VAR or AFG_OP_VAR_RZ");
    if (op == 2 && t->ht.D != 2) return fail(AFG_ERR_ARG, "(r,z) coordinates need a 2D tree");
    if (op && t->grid && t->grid->block)
        return fail(AFG_ERR_STATE, "a tree of several root boxes takes its operator before its data");
    if (op == 2 && t->ht.bct[0] == 2) return fail(AFG_ERR_ARG, "(r,z): the -x side is the axis and cannot be periodic");
    bool dir = false;
    for (int s2 = 0; s2 < 2 * t->ht.D; ++s2) dir |= t->ht.bct[s2] == 0;
    if (op && !dir) return fail(AFG_ERR_ARG, "the variable-coefficient operators need a Dirichlet side");
    AFG_API_BEGIN
    t->op = op;
    if (t->grid) {  // the device data stays; the cycles change (graphs are recaptured) and eps is needed again
        afg::DeviceGuard dg(t->device);
        t->grid->op = op;
        t->grid->eps_set = false;
        t->grid->clear_graphs();
    }
    return AFG_OK;
    AFG_API_END
}

int afg_set_prolongation(afg_tree *t, int scheme) {
    if (!t) return fail(AFG_ERR_ARG, "null tree");
    if (scheme < 0 || scheme > 2) return fail(AFG_ERR_ARG, "scheme must be AFG_PROLONG_LINEAR, _MULTILINEAR or _ZEROTH");
    if (scheme && t->grid && t->grid->block)
        return fail(AFG_ERR_STATE, "a tree of several root boxes takes its prolongation before its data");
    AFG_API_BEGIN
    t->prolong = scheme;
    if (t->grid) {
        afg::DeviceGuard dg(t->device);
        t->grid->prolong = scheme;
        t->grid->clear_graphs();
    }
    return AFG_OK;
    AFG_API_END
}

int afg_set_eps(afg_tree *t, const double *eps) {
    if (!t || !eps) return fail(AFG_ERR_ARG, "null argument");
    if (!t->op) return fail(AFG_ERR_STATE, "eps needs a variable-coefficient operator (afg_set_operator)");
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &g = grid_of(t);
    g.set_eps(eps, t->stream);
    check(cudaGetLastError(), "afg_set_eps");
    return AFG_OK;
    AFG_API_END
}

int afg_forest_set_eps(afg_forest *f, const double *eps) {
    if (!f || !eps) return fail(AFG_ERR_ARG, "null argument");
    if (!f->grid->op) return fail(AFG_ERR_STATE, "eps needs a variable-coefficient operator (afg_set_operator)");
    AFG_API_BEGIN
    AFG_ON_FOREST_DEVICE(f);
    f->grid->set_eps(eps, f->stream);
    check(cudaGetLastError(), "afg_forest_set_eps");
    return AFG_OK;
    AFG_API_END
}

int afg_set_dirichlet(afg_tree *t, const double *b) {
    if (!t || !b) return fail(AFG_ERR_ARG, "null argument");
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &g = grid_of(t);
    set_dirichlet_dev(g, b, t->stream);
    check(cudaGetLastError(), "afg_set_dirichlet");
    return AFG_OK;
    AFG_API_END
}

int afg_set_solution(afg_tree *t, const double *u) {
    if (!t || !u) return fail(AFG_ERR_ARG, "null argument");
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &g = grid_of(t);
    afg::launch_leaf_set(g.leaf_cfg(true, t->stream), g.meta, g.d_leaves, g.n_leaf_boxes, u, g.ws64.u->p);
    check(cudaGetLastError(), "afg_set_solution");
    return AFG_OK;
    AFG_API_END
}

int afg_get_solution(const afg_tree *tc, double *u) {
    afg_tree *t = const_cast<afg_tree *>(tc);
    if (!t || !u) return fail(AFG_ERR_ARG, "null argument");
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &g = grid_of(t);
    afg::launch_leaf_get(g.leaf_cfg(true, t->stream), g.meta, g.d_leaves, g.n_leaf_boxes, g.ws64.u->p, u);
    check(cudaGetLastError(), "afg_get_solution");
    return AFG_OK;
    AFG_API_END
}

static int one_cycle(afg_tree *t, const afg_mg_opts *opts, afg_stats *st, bool fmg) {
    if (!t) return fail(AFG_ERR_ARG, "null tree");
    const afg_mg_opts o = opts_or_default(opts);
    if (int rc = validate(o)) return rc;
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &g = grid_of(t);
    if (int rc = ready(g)) return rc;
    if (int rc = vpt_of(g, o, &g.vpt)) return rc;
    const auto t0 = clk::now();
    const afg::MgOpts mo{o.n_down, o.n_up, o.n_base};
    g.make_compatible(t->stream);
    run(g, {fmg ? 30 : 31, o.n_down, o.n_up, o.n_base, 0}, o.use_graph, t->stream, [&](cudaStream_t cs) {
        if (fmg) g.fmg(g.ws64, mo, 0, false, cs);
        else g.vcycle(g.ws64, g.lmax, mo, 0, nullptr, cs);
        g.remove_mean(g.ws64, cs);
        g.norms_async(g.ws64, 0, nullptr, false, cs);
    });
    check(cudaStreamSynchronize(t->stream), "cycle");
    if (st) {
        std::memset(st, 0, sizeof(*st));
        fill_stats(st, g, 0, 1, std::chrono::duration<double>(clk::now() - t0).count());
        st->history[0] = st->rel_residual;
    }
    return AFG_OK;
    AFG_API_END
}

int afg_fmg(afg_tree *t, const afg_mg_opts *o, afg_stats *st) { return one_cycle(t, o, st, true); }
int afg_vcycle(afg_tree *t, const afg_mg_opts *o, afg_stats *st) { return one_cycle(t, o, st, false); }

int afg_solve(afg_tree *t, const afg_mg_opts *opts, afg_stats *st) {
    if (!t) return fail(AFG_ERR_ARG, "null tree");
    const afg_mg_opts o = opts_or_default(opts);
    if (int rc = validate(o)) return rc;
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &g = grid_of(t);
    if (int rc = ready(g)) return rc;
    if (int rc = vpt_of(g, o, &g.vpt)) return rc;
    const auto t0 = clk::now();
    std::vector<std::vector<double>> hist;
    const int cycles = o.precision == AFG_MIXED ? solve_mixed(g, o, t->stream, hist)
                                                : solve_fp64(g, o, t->stream, hist, true);
    const double secs = std::chrono::duration<double>(clk::now() - t0).count();
    if (st) {
        std::memset(st, 0, sizeof(*st));
        fill_stats(st, g, 0, cycles, secs);
        for (size_t i = 0; i < hist[0].size() && i < 64; ++i) st->history[i] = hist[0][i];
    }
    if (rel_of(g, 0) > o.rel_tol) return fail(AFG_ERR_NOT_CONVERGED, "max_cycles reached above rel_tol");
    return AFG_OK;
    AFG_API_END
}

int afg_residual_norm(afg_tree *t, double *max_abs_r, double *max_abs_rho) {
    if (!t) return fail(AFG_ERR_ARG, "null tree");
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &g = grid_of(t);
    if (g.op && !g.eps_set) return fail(AFG_ERR_STATE, "the variable-coefficient operator needs eps (afg_set_eps)");
    if (g.rhs_set) g.make_compatible(t->stream);
    g.norms_async(g.ws64, 0, nullptr, false, t->stream);
    check(cudaStreamSynchronize(t->stream), "residual norm");
    if (max_abs_r) *max_abs_r = as_double(g.h_norms[0]);
    if (max_abs_rho) *max_abs_rho = as_double(g.h_norms[g.T]);
    return AFG_OK;
    AFG_API_END
}

int afg_adjoint(afg_tree *t, const double *g_leaf, double *lambda_leaf, double *dL_db, const afg_mg_opts *opts,
                afg_stats *st) {
    if (!t || !g_leaf) return fail(AFG_ERR_ARG, "null argument");
    const afg_mg_opts o = opts_or_default(opts);
    if (int rc = validate(o)) return rc;
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    Grid &g = grid_of(t);
    if (g.op) return fail(AFG_ERR_STATE, "the adjoint is built for the Laplacian only");
    if (g.singular) return fail(AFG_ERR_STATE, "the adjoint needs a Dirichlet side");
    const auto t0 = clk::now();
    double rel = 0.0;
    const int its = adjoint_solve(g, o, t->stream, g_leaf, &rel);
    const afg::LaunchCfg lc = g.leaf_cfg(true, t->stream);
    double *x = g.bicg[1]->as<double>();
    if (lambda_leaf) afg::launch_leaf_get(lc, g.meta, g.d_leaves, g.n_leaf_boxes, x, lambda_leaf);
    if (dL_db) afg::launch_adjoint_db(lc, g.meta, g.d_hb, g.d_leaves, g.n_leaf_boxes, x, dL_db);
    check(cudaStreamSynchronize(t->stream), "adjoint");
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->cycles = its;
        st->rel_residual = rel;
        st->seconds = std::chrono::duration<double>(clk::now() - t0).count();
    }
    if (rel > o.rel_tol) return fail(AFG_ERR_NOT_CONVERGED, "adjoint did not reach rel_tol");
    return AFG_OK;
    AFG_API_END
}

// ---- forests ---------------------------------------------------------------

int afg_forest_create(int n, afg_tree *const *trees, afg_forest **out) {
    if (n < 1 || !trees || !out) return fail(AFG_ERR_ARG, "bad arguments");
    for (int i = 0; i < n; ++i)
        if (!trees[i] || trees[i]->ht.D != trees[0]->ht.D || trees[i]->ht.N != trees[0]->ht.N)
            return fail(AFG_ERR_ARG, "trees must exist and share dim and box_n");
    for (int i = 0; i < n; ++i) {
        if (trees[i]->op != trees[0]->op || trees[i]->prolong != trees[0]->prolong)
            return fail(AFG_ERR_ARG, "the trees of a forest must share the operator and the prolongation");
    }
    AFG_API_BEGIN
    std::unique_ptr<afg_forest> f(new afg_forest);
    f->device = afg::current_device();
    std::vector<const HostTree *> v;
    for (int i = 0; i < n; ++i) {
        f->trees.emplace_back(new HostTree(trees[i]->ht));
        v.push_back(f->trees.back().get());
    }
    f->grid.reset(new Grid(v));
    f->grid->op = trees[0]->op;
    f->grid->prolong = trees[0]->prolong;
    *out = f.release();
    return AFG_OK;
    AFG_API_END
}

int afg_forest_destroy(afg_forest *f) {
    delete f;
    return AFG_OK;
}

int afg_forest_set_stream(afg_forest *f, void *s) {
    if (!f) return fail(AFG_ERR_ARG, "null forest");
    f->stream = (cudaStream_t)s;
    return AFG_OK;
}

int afg_forest_counts(const afg_forest *f, long long *cells, long long *faces) {
    if (!f) return fail(AFG_ERR_ARG, "null forest");
    for (int t = 0; t < f->grid->T; ++t) {
        if (cells) cells[t] = f->grid->tree_cells[t];
        if (faces) faces[t] = f->grid->tree_faces[t];
    }
    return AFG_OK;
}

int afg_forest_set_rhs(afg_forest *f, const double *rho) {
    if (!f || !rho) return fail(AFG_ERR_ARG, "null argument");
    AFG_API_BEGIN
    AFG_ON_FOREST_DEVICE(f);
    Grid &g = *f->grid;
    afg::launch_leaf_set(g.leaf_cfg(true, f->stream), g.meta, g.d_leaves, g.n_leaf_boxes, rho, g.ws64.rho->p);
    g.leaf_rho_hat(g.ws64, f->stream);
    check(cudaGetLastError(), "afg_forest_set_rhs");
    g.rhs_set = true;
    return AFG_OK;
    AFG_API_END
}

int afg_forest_set_dirichlet(afg_forest *f, const double *b) {
    if (!f || !b) return fail(AFG_ERR_ARG, "null argument");
    AFG_API_BEGIN
    AFG_ON_FOREST_DEVICE(f);
    set_dirichlet_dev(*f->grid, b, f->stream);
    check(cudaGetLastError(), "afg_forest_set_dirichlet");
    return AFG_OK;
    AFG_API_END
}

int afg_forest_get_solution(const afg_forest *f, double *u) {
    if (!f || !u) return fail(AFG_ERR_ARG, "null argument");
    AFG_API_BEGIN
    AFG_ON_FOREST_DEVICE(f);
    Grid &g = *f->grid;
    afg::launch_leaf_get(g.leaf_cfg(true, f->stream), g.meta, g.d_leaves, g.n_leaf_boxes, g.ws64.u->p, u);
    check(cudaGetLastError(), "afg_forest_get_solution");
    return AFG_OK;
    AFG_API_END
}

int afg_forest_solve(afg_forest *f, const afg_mg_opts *opts, afg_stats *per_tree) {
    if (!f) return fail(AFG_ERR_ARG, "null forest");
    const afg_mg_opts o = opts_or_default(opts);
    if (int rc = validate(o)) return rc;
    AFG_API_BEGIN
    AFG_ON_FOREST_DEVICE(f);
    Grid &g = *f->grid;
    if (int rc = ready(g)) return rc;
    if (int rc = vpt_of(g, o, &g.vpt)) return rc;
    const auto t0 = clk::now();
    check(cudaMemsetAsync(g.ws64.u->p, 0, (size_t)g.ncell * 8, f->stream), "zero");
    std::vector<std::vector<double>> hist;
    const int cycles = o.precision == AFG_MIXED ? solve_mixed(g, o, f->stream, hist)
                                                : solve_fp64(g, o, f->stream, hist, true);
    const double secs = std::chrono::duration<double>(clk::now() - t0).count();
    bool all = true;
    for (int t = 0; t < g.T; ++t) {
        if (rel_of(g, t) > o.rel_tol) all = false;
        if (per_tree) {
            std::memset(&per_tree[t], 0, sizeof(afg_stats));
            fill_stats(&per_tree[t], g, t, (int)hist[t].size() - (o.precision == AFG_MIXED ? 1 : 0), secs);
            for (size_t i = 0; i < hist[t].size() && i < 64; ++i) per_tree[t].history[i] = hist[t][i];
        }
    }
    (void)cycles;
    if (!all) return fail(AFG_ERR_NOT_CONVERGED, "some trees did not reach rel_tol");
    return AFG_OK;
    AFG_API_END
}

int afg_kernel_launches(unsigned long long *count) {
    if (!count) return fail(AFG_ERR_ARG, "null argument");
    *count = afg::g_launches;
    return AFG_OK;
}

}  // extern "C"

namespace {
// times `reps` launches of one kernel of the solve on grid g (afg_time_kernel)
int time_kernel_on(Grid &g, cudaStream_t s, int kernel, int level, int fp64, int reps, double *avg_ms, double *bytes,
                   double *flops, long long *cells) {
    if (!g.rhs_set) return fail(AFG_ERR_STATE, "no right-hand side set");
    if (g.op) return fail(AFG_ERR_STATE, "kernel timing covers the Laplacian's kernels");
    if (kernel < 3 && (level < g.lmin || level > g.lmax)) return fail(AFG_ERR_ARG, "level out of range");
    if ((kernel == 1 || kernel == 2) && level < 2) return fail(AFG_ERR_ARG, "level must be >= 2");
    if (!fp64 || kernel == 3) g.ensure_mixed();
    afg::Workspace &w = fp64 ? g.ws64 : g.ws32;
    if (!fp64) {  // FP32 data from the FP64 source (values are irrelevant to timing)
        afg::launch_leaf_residual(g.leaf_cfg(true, s), g.meta, g.d_leaves, g.n_leaf_boxes, g.ws64.u->p,
                                  g.ws64.rho->p, 0, g.d_norms, g.d_norms + g.T, g.ws32.rho->p, true);
    }
    const double sz = fp64 ? 8.0 : 4.0;
    const int D = g.D;
    long long nc = 0;
    double by = 0, fl = 0;
    auto launch = [&](int i) {
        if (kernel == 0) {
            auto &v = g.L(level);
            // FP32 half-sweeps run with homogeneous boundary data, as in the mixed-precision solve
            afg::launch_smooth(g.cfg(level, fp64, s), g.meta, v.b0, v.nb, nullptr, w.u->p, w.rho->p, w.rhoh_p(), v.h * v.h,
                               i & 1, fp64 ? 0 : 1);
        } else if (kernel == 1) {
            auto &v = g.L(level);
            afg::launch_resid_restrict(g.cfg(level, fp64, s), g.meta, v.b0, v.nb, w.u->p, w.rho->p, w.vold->p,
                                       1.0 / (v.h * v.h), 0);
        } else if (kernel == 2) {
            auto &v = g.L(level);
            afg::launch_correct(g.cfg(level, fp64, s), g.meta, v.b0, v.nb, w.u->p, w.vold->p);
        } else if (kernel == 3) {
            afg::launch_leaf_residual(g.leaf_cfg(true, s), g.meta, g.d_leaves, g.n_leaf_boxes, g.ws64.u->p,
                                      g.ws64.rho->p, 0, g.d_norms, g.d_norms + g.T, g.ws32.rho->p, true);
        } else {
            fl = afg::launch_fp64_probe(s, g.d_partials, 2048);
        }
    };
    if (kernel == 4) {
        nc = 0;
        by = 0;
    } else if (kernel == 3) {
        nc = g.n_leaf_cells;
        by = nc * (2 * 8.0 + 4.0);
        fl = nc * (2.0 * D + 3);
    } else {
        nc = g.L(level).ncell;
        const double c2 = double(1 << D);
        // half-sweep, per update: 2D-1 additions and one FMA with the pre-scaled source (FP64),
        // or 2D-1 additions, one FMA and one multiplication (FP32)
        if (kernel == 0) { by = nc * 1.5 * sz; fl = nc * (2.0 * D + (w.rhoh_p() ? 1 : 2)) / 2; }
        if (kernel == 1) { by = nc * (2 * sz + 3 * sz / c2); fl = nc * (2.0 * D + 5); }
        if (kernel == 2) { by = nc * (2 * sz + 2 * sz / c2); fl = nc * 5.0; }
    }
    launch(0);
    cudaEvent_t e0, e1;
    check(cudaEventCreate(&e0), "event");
    check(cudaEventCreate(&e1), "event");
    check(cudaEventRecord(e0, s), "event");
    for (int i = 0; i < reps; ++i) launch(i + 1);
    check(cudaEventRecord(e1, s), "event");
    check(cudaEventSynchronize(e1), "event");
    float ms = 0.f;
    check(cudaEventElapsedTime(&ms, e0, e1), "event");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    check(cudaGetLastError(), "afg_time_kernel");
    if (avg_ms) *avg_ms = ms / reps;
    if (bytes) *bytes = by;
    if (flops) *flops = fl;
    if (cells) *cells = nc;
    return AFG_OK;
}
}  // namespace


extern "C" {

int afg_time_kernel(afg_tree *t, int kernel, int level, int fp64, int reps, double *avg_ms, double *bytes,
                    double *flops, long long *cells) {
    if (!t || reps < 1 || kernel < 0 || kernel > 4) return fail(AFG_ERR_ARG, "bad arguments");
    AFG_API_BEGIN
    AFG_ON_DEVICE(t);
    return time_kernel_on(grid_of(t), t->stream, kernel, level, fp64, reps, avg_ms, bytes, flops, cells);
    AFG_API_END
}

int afg_forest_time_kernel(afg_forest *f, int kernel, int level, int fp64, int reps, double *avg_ms, double *bytes,
                           double *flops, long long *cells) {
    if (!f || reps < 1 || kernel < 0 || kernel > 4) return fail(AFG_ERR_ARG, "bad arguments");
    AFG_API_BEGIN
    AFG_ON_FOREST_DEVICE(f);
    return time_kernel_on(*f->grid, f->stream, kernel, level, fp64, reps, avg_ms, bytes, flops, cells);
    AFG_API_END
}

}  // extern "C"

