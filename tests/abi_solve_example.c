/* Plain C11 use of the C ABI for a whole solve on the GPU: the library's
 * device memory comes from a caller's allocator that counts its calls
 * (afg_set_allocator), the caller's own fields from cudaMalloc.  Writes the
 * solution (canonical leaf order, doubles) to the file named by argv[1] and
 * prints the counts, cycles and residual the test checks. */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "afgpu.h"

typedef struct {
    long allocs, frees, live;
    size_t bytes;
} counter;

static void *count_alloc(size_t bytes, void *ctx) {
    counter *c = (counter *)ctx;
    void *p = NULL;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return NULL;
    c->allocs++;
    c->live++;
    c->bytes += bytes;
    return p;
}

static void count_free(void *p, void *ctx) {
    counter *c = (counter *)ctx;
    c->frees++;
    c->live--;
    cudaFree(p);
}

int main(int argc, char **argv) {
    if (argc < 2) return 1;
    counter cnt = {0, 0, 0, 0};
    if (afg_set_allocator(count_alloc, NULL, &cnt) != AFG_ERR_ARG) return 2; /* both or neither */
    if (afg_set_allocator(count_alloc, count_free, &cnt) != AFG_OK) return 3;
    afg_tree *t = NULL;
    if (afg_tree_create(2, 8, 5, &t) != AFG_OK) return 4;
    if (afg_refine_uniform(t, 4) != AFG_OK) return 5;
    afg_tree_info info;
    if (afg_info(t, &info) != AFG_OK) return 6;
    const long long n = info.n_leaf_cells;
    double *xyz = malloc(sizeof(double) * 2 * (size_t)n), *rho = malloc(sizeof(double) * (size_t)n);
    double *u = malloc(sizeof(double) * (size_t)n);
    if (!xyz || !rho || !u) return 7;
    if (afg_cell_centers(t, xyz) != AFG_OK) return 8;
    for (long long i = 0; i < n; ++i) rho[i] = xyz[2 * i] * (1.0 - xyz[2 * i]) - xyz[2 * i + 1];
    double *d_rho = NULL, *d_u = NULL;
    if (cudaMalloc((void **)&d_rho, sizeof(double) * (size_t)n) != cudaSuccess) return 9;
    if (cudaMalloc((void **)&d_u, sizeof(double) * (size_t)n) != cudaSuccess) return 10;
    if (cudaMemcpy(d_rho, rho, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) return 11;
    if (afg_set_rhs(t, d_rho) != AFG_OK) return 12;
    afg_mg_opts o;
    afg_default_opts(&o);
    o.rel_tol = 1e-10;
    afg_stats st;
    if (afg_solve(t, &o, &st) != AFG_OK) return 13;
    if (afg_get_solution(t, d_u) != AFG_OK) return 14;
    if (cudaMemcpy(u, d_u, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess) return 15;
    const long allocs_during = cnt.allocs;
    afg_tree_destroy(t);
    if (afg_set_allocator(NULL, NULL, NULL) != AFG_OK) return 16;
    FILE *f = fopen(argv[1], "wb");
    if (!f || fwrite(u, sizeof(double), (size_t)n, f) != (size_t)n) return 17;
    fclose(f);
    printf("cells %lld\n", n);
    printf("solve %d %.3e\n", st.cycles, st.rel_residual);
    printf("allocator %ld %ld %ld %ld\n", allocs_during, cnt.allocs, cnt.frees, cnt.live);
    cudaFree(d_rho);
    cudaFree(d_u);
    free(xyz);
    free(rho);
    free(u);
    return 0;
}
