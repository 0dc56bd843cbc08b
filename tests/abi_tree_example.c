/* Plain C11 use of the C ABI (include/afgpu.h) for the tree calls, which need
 * no GPU: create, refine, adapt, query, export, errors, root blocks.  Prints
 * the figures the test compares with the oracle. */
#include <stdio.h>
#include <stdlib.h>

#include "afgpu.h"

int main(void) {
    afg_tree *t = NULL;
    if (afg_tree_create(2, 8, 5, &t) != AFG_OK) return 1;
    if (afg_refine_uniform(t, 3) != AFG_OK) return 2;
    afg_tree_info info;
    if (afg_info(t, &info) != AFG_OK) return 3;
    printf("uniform %d %lld %lld\n", info.n_boxes, info.n_leaf_cells, info.n_bfaces);
    int8_t *flags = calloc((size_t)info.n_leaf_cells, 1);
    if (!flags) return 4;
    flags[0] = 1; /* the first cell of the first leaf box */
    int added = 0, removed = 0;
    if (afg_adapt(t, flags, 2, &added, &removed) != AFG_OK) return 5;
    if (afg_info(t, &info) != AFG_OK) return 6;
    printf("adapted %d %d %d %lld %lld\n", added, removed, info.n_boxes, info.n_leaf_cells, info.n_bfaces);
    int32_t *level = malloc(sizeof(int32_t) * (size_t)info.n_boxes);
    int32_t *parent = malloc(sizeof(int32_t) * (size_t)info.n_boxes);
    if (!level || !parent) return 7;
    if (afg_export_tree(t, level, NULL, parent, NULL, NULL) != AFG_OK) return 8;
    int deepest = 0;
    for (int b = 0; b < info.n_boxes; ++b) deepest = level[b] > deepest ? level[b] : deepest;
    printf("export %d %d %d\n", level[0], parent[0], deepest);
    afg_tree *bad = NULL;
    int rc = afg_tree_create(4, 8, 3, &bad);
    printf("error %d %s\n", rc == AFG_ERR_ARG, afg_last_error());
    const int roots[2] = {3, 2};
    afg_tree *m = NULL;
    if (afg_tree_create_roots(2, 8, 3, roots, &m) != AFG_OK) return 9;
    if (afg_refine_uniform(m, 2) != AFG_OK) return 10;
    if (afg_info(m, &info) != AFG_OK) return 11;
    printf("roots %d %lld %lld\n", info.n_boxes, info.n_leaf_cells, info.n_bfaces);
    afg_tree_destroy(m);
    afg_tree_destroy(t);
    free(flags);
    free(level);
    free(parent);
    return 0;
}
