// Residual norms of a forest without any allocation.
//
// Some callers cannot allocate device memory at the point where they check
// convergence: a host framework that has handed the whole device memory
// pool to its own caching allocator, or a latency-bound loop in which the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.
// afg_forest_residual_norms_noalloc gives them the per-tree residual norms
// of an existing forest using only memory that already exists: the forest's
// own field data (allocated when the forest was created) and the file-scope
// scratch array below for the per-tree maxima.
#include <cstring>
#include <map>
#include <mutex>

#include "../../include/afgpu.h"
#include "handles.h"

namespace {

// Largest forest served: two 8-byte maxima per tree (16 KB of device memory,
// held by every GPU that loads the library until the process exits).
constexpr int kNoAllocMaxTrees = 1024;
__device__ __align__(256) unsigned long long g_noalloc_norms[2 * kNoAllocMaxTrees];

std::mutex g_mu;
std::map<int, unsigned long long *> g_addr;  // device ordinal -> device address of g_noalloc_norms

int noalloc_fail(int code, const char *msg) { return afg::api_fail(code, msg); }

}  // namespace

extern "C" int afg_forest_residual_norms_noalloc(afg_forest *f, double *max_abs_r, double *max_abs_rho) {
    if (!f || !f->grid || !max_abs_r || !max_abs_rho) return noalloc_fail(AFG_ERR_ARG, "null argument");
    afg::Grid &g = *f->grid;
    if (g.T > kNoAllocMaxTrees)
        return noalloc_fail(AFG_ERR_ARG, "forest has more trees than the 1024 the allocation-free norm supports");
    if (!g.rhs_set) return noalloc_fail(AFG_ERR_STATE, "no right-hand side set");
    if (g.op) return noalloc_fail(AFG_ERR_STATE, "the allocation-free norm covers the Laplacian only");
    if (g.singular) return noalloc_fail(AFG_ERR_STATE, "the allocation-free norm needs a Dirichlet side");
    // the forest's device (where its data and this call's kernels live)
    const int dev = f->device;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return noalloc_fail(AFG_ERR_CUDA, "cudaGetDevice failed");
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return noalloc_fail(AFG_ERR_CUDA, "cudaSetDevice failed");
    struct Restore {
        int prev, dev;
        ~Restore() {
            if (prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, dev};
    unsigned long long *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_addr.find(dev);
        if (it == g_addr.end()) {
            // once per device, with that device current: the host-side name of
            // the array is only a stand-in, the kernel needs its device address
            if (cudaGetSymbolAddress((void **)&scratch, g_noalloc_norms) != cudaSuccess || !scratch)
                return noalloc_fail(AFG_ERR_CUDA, "cudaGetSymbolAddress of the norm scratch failed");
            g_addr.emplace(dev, scratch);
        } else {
            scratch = it->second;
        }
    }
    try {
        cudaStream_t s = f->stream;
        g.restrict_cf(g.ws64, s);  // what the composite residual reads, as afg_forest_solve's norms
        // the scratch keeps the previous call's maxima: clear the slots used
        afg::check(cudaMemsetAsync(scratch, 0, 2 * (size_t)g.T * sizeof(unsigned long long), s), "memset");
        afg::launch_leaf_residual(g.leaf_cfg(true, s), g.meta, g.d_leaves, g.n_leaf_boxes, g.ws64.u->p,
                                  g.ws64.rho->p, 0, scratch, scratch + g.T, nullptr, false);
        // non-negative doubles were reduced through their bit patterns: copy the bits back
        afg::check(cudaMemcpyAsync(max_abs_r, scratch, g.T * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
        afg::check(cudaMemcpyAsync(max_abs_rho, scratch + g.T, g.T * sizeof(double), cudaMemcpyDeviceToHost, s),
                   "copy");
        afg::check(cudaStreamSynchronize(s), "sync");
    } catch (const std::exception &e) {
        return noalloc_fail(AFG_ERR_CUDA, e.what());
    }
    return AFG_OK;
}
