// Opaque handle types of the C interface (include/afgpu.h).
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "grid.h"

namespace afg {
// destroys a grid with its own device current (never throws)
inline void release_on(int device, std::unique_ptr<Grid> &grid) {
    if (!grid) return;
    int cur = -1;
    const bool sw = device >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != device &&
                    cudaSetDevice(device) == cudaSuccess;
    grid.reset();
    if (sw) cudaSetDevice(cur);
}
}  // namespace afg

struct afg_tree {
    afg::HostTree ht;
    std::unique_ptr<afg::Grid> grid;
    int grid_version = -1;
    cudaStream_t stream = nullptr;
    int op = 0;       // operator: 0 Laplacian, 1 div(eps grad u), 2 the same in (r,z)
    int prolong = 0;  // correction's prolongation: 0 linear, 1 bi/trilinear, 2 zeroth order
    // CUDA device of the tree's field data: the device current at the first
    // field call; every later call runs there whatever device is current
    int device = -1;
    int device_for_call() {
        if (device < 0) device = afg::current_device();
        return device;
    }
    afg_tree(int d, int n, int m, const int *nroot = nullptr) : ht(d, n, m, nroot) {}
    ~afg_tree() { afg::release_on(device, grid); }
};

struct afg_forest {
    std::vector<std::unique_ptr<afg::HostTree>> trees;
    std::unique_ptr<afg::Grid> grid;
    cudaStream_t stream = nullptr;
    int device = 0;  // device current at afg_forest_create, where its data lives
    ~afg_forest() { afg::release_on(device, grid); }
};

namespace afg {
// records `msg` for afg_last_error() on this thread and returns `code`
int api_fail(int code, const std::string &msg);
}  // namespace afg
