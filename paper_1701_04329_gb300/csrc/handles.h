// Opaque handle types of the C interface (include/afgpu.h).
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "grid.h"

struct afg_tree {
    afg::HostTree ht;
    std::unique_ptr<afg::Grid> grid;
    int grid_version = -1;
    cudaStream_t stream = nullptr;
    afg_tree(int d, int n, int m, const int *nroot = nullptr) : ht(d, n, m, nroot) {}
};

struct afg_forest {
    std::vector<std::unique_ptr<afg::HostTree>> trees;
    std::unique_ptr<afg::Grid> grid;
    cudaStream_t stream = nullptr;
};

namespace afg {
// records `msg` for afg_last_error() on this thread and returns `code`
int api_fail(int code, const std::string &msg);
}  // namespace afg
