/*
 * afmg_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the method of Teunissen & Ebert,
 * "Afivo: a framework for quadtree/octree AMR with shared-memory
 * parallelization and geometric multigrid methods" (arXiv:1701.04329):
 * the quadtree/octree of boxes (Sec. 2.1-2.3), ghost cells (Sec. 2.4, 3.3),
 * prolongation/restriction (Sec. 2.5) and the FAS V-cycle / FMG multigrid
 * solver with red-black Gauss-Seidel smoothing (Sec. 3.1-3.2), on domains
 * of one or several root boxes (Sec. 2.2); also the parts the CUDA library
 * does not have yet: the variable-coefficient and (r,z) operators (Sec. 3.4-3.5),
 * edge/corner ghosts with the bilinear / trilinear and zeroth-order
 * prolongation (Sec. 2.4-2.5), and the field transfer of mesh adaptation
 * (Sec. 2.3).  Every function is pinned by the tests against values fixed
 * by the paper or the mathematics (tests/test_oracle_*.py).
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this file.  It shares no code, header or table with the CUDA
 * library.  It follows the paper's own data layout: every box stores one
 * ghost layer around its N^D cells, ghost cells are filled by a separate pass,
 * and all operators loop over boxes of one level (the paper's OpenMP scheme,
 * Sec. 2.6; the loops are independent per box, so results do not depend on
 * the thread count).
 *
 * Readings of points the paper leaves open are marked "Reading:".
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OMAXLEV 24
#define ONDIR 26

/* ---------------------------------------------------------------------- */
/* Tree: boxes, levels, spatial indices, parent/children/neighbours        */
/* (Sec. 2.1, 2.2).                                                        */
/* ---------------------------------------------------------------------- */

typedef struct {
    int level;          /* refinement level, 1 = the root box */
    int idx[3];         /* 1-based spatial index (Sec. 2.1) */
    uint64_t key;       /* Morton key of idx-1, x lowest (Sec. 2.3) */
    int parent;         /* box id or -1 */
    int child[8];       /* box ids or -1; child c has offset bit a = (c>>a)&1 */
    int nb[ONDIR];      /* same-level neighbour id, -1 = none, -2 = physical boundary */
} OBox;

/* multigrid face kinds */
#define K_SAME 0
#define K_PHYS 1
#define K_CF 2

typedef struct {
    int level, M;       /* level (<= 0 below the root) and cells per side */
    double h;
    int tbox;           /* tree box id, -1 for the boxes below the root */
    int parent;         /* multigrid box holding this box's restriction, -1 at the bottom */
    int poff[3];        /* offset (cells) of this box's region inside the parent */
    int refined;        /* 1 if finer boxes exist below it (values are FAS values) */
    int kind[6], nbid[6];
    int nball[26];      /* same-level neighbour (multigrid id) in every direction, -1 none */
    double x0[3];       /* lower corner of the box */
    double *u, *rho, *vold, *r, *rr, *d;
    double *eps;        /* coefficient of the variable-coefficient operators, ghosts included */
    double *bc[6];
} OMG;

typedef struct {
    int D, N, max_level;
    int nr[3];                      /* root boxes per axis (the domain is nr[0] x nr[1] x nr[2]) */
    int nbox;
    OBox *box;
    int L;                          /* highest level present */
    int lstart[OMAXLEV + 2], lcount[OMAXLEV + 2];
    /* leaves in canonical order */
    int nleaf;
    int *leaf;
    /* multigrid hierarchy */
    int mg_ready;
    int lmin;                        /* coarsest multigrid level */
    int nmg;
    OMG *mg;
    int mgstart[2 * OMAXLEV + 8], mgcount[2 * OMAXLEV + 8]; /* indexed by level - lmin */
    int hom;                         /* 1: homogeneous boundary data (defect equations) */
    int bct[6];                      /* per domain side (-x,+x,-y,+y,-z,+z): 0 Dirichlet, 1 Neumann, 2 periodic */
    int op;                          /* 0 Laplacian, 1 div(eps grad), 2 the same in (r,z) with r = x (2D) */
    int prolong;                     /* correction: 0 linear 2-1-1 / 1-1-1-1, 1 bi/trilinear, 2 zeroth order */
    int singular;                    /* no Dirichlet side: constants are the null space (see make_compatible) */
} OTree;

/* spatial index q along axis a at a level with `side` boxes per axis: on a
 * periodic axis it wraps around (Sec. 2.2: the box beyond the last one is
 * the first), elsewhere it is returned as is */
static int pwrap(const OTree *t, int a, int q, int side) {
    if (t->bct[2 * a] != 2) return q;
    return ((q - 1) % side + side) % side + 1;
}

static int ipow(int b, int e) { int r = 1; while (e-- > 0) r *= b; return r; }

/* boxes per axis a at a level: nr[a] root boxes, each split 2^(level-1) times */
static int side_of(const OTree *t, int a, int level) { return t->nr[a] << (level - 1); }

static uint64_t morton_key(int D, const int *idx) {
    uint64_t k = 0;
    for (int b = 0; b < 21; b++)
        for (int a = 0; a < D; a++)
            k |= (uint64_t)(((unsigned)(idx[a] - 1) >> b) & 1u) << (D * b + a);
    return k;
}

/* Neighbour direction n (0..3^D-2) -> offsets; lexicographic over (dz,dy,dx), x fastest. */
static void dir_offsets(int D, int n, int *off) {
    int full = n >= (ipow(3, D) - 1) / 2 ? n + 1 : n; /* skip the centre */
    for (int a = 0; a < 3; a++) off[a] = 0;
    for (int a = 0; a < D; a++) { off[a] = full % 3 - 1; full /= 3; }
}

/* face side s (-x,+x,-y,+y,-z,+z) -> neighbour direction index */
static int side_dir(int D, int s) {
    int off[3] = {0, 0, 0};
    off[s / 2] = (s % 2) ? 1 : -1;
    int full = 0, m = 1;
    for (int a = 0; a < D; a++) { full += (off[a] + 1) * m; m *= 3; }
    int centre = (ipow(3, D) - 1) / 2;
    return full > centre ? full - 1 : full;
}

typedef struct { int level; uint64_t key; int idx[3]; } OPos;

static int cmp_pos(const void *pa, const void *pb) {
    const OPos *a = pa, *b = pb;
    if (a->level != b->level) return a->level < b->level ? -1 : 1;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return 0;
}

/* binary search for (level, idx) in the canonical order; -1 when absent */
static int find_box(const OTree *t, int level, const int *idx) {
    if (level < 1 || level > t->L) return -1;
    for (int a = 0; a < t->D; a++)
        if (idx[a] < 1 || idx[a] > side_of(t, a, level)) return -1;
    uint64_t key = morton_key(t->D, idx);
    int lo = t->lstart[level], hi = lo + t->lcount[level] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (t->box[mid].key == key) return mid;
        if (t->box[mid].key < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static void free_mg(OTree *t);

/* Rebuild all connectivity from a list of box positions (Sec. 2.1, 2.3). */
static int rebuild(OTree *t, OPos *pos, int n) {
    qsort(pos, n, sizeof(OPos), cmp_pos);
    free(t->box);
    t->box = calloc((size_t)n, sizeof(OBox));
    if (!t->box) return -3;
    t->nbox = n;
    t->L = 0;
    for (int l = 0; l < OMAXLEV + 2; l++) { t->lstart[l] = 0; t->lcount[l] = 0; }
    for (int i = 0; i < n; i++) {
        OBox *b = &t->box[i];
        b->level = pos[i].level;
        for (int a = 0; a < 3; a++) b->idx[a] = a < t->D ? pos[i].idx[a] : 1;
        b->key = pos[i].key;
        if (t->lcount[b->level] == 0) t->lstart[b->level] = i;
        t->lcount[b->level]++;
        if (b->level > t->L) t->L = b->level;
    }
    int nd = ipow(3, t->D) - 1, nc = 1 << t->D;
    for (int i = 0; i < n; i++) {
        OBox *b = &t->box[i];
        int p[3] = {1, 1, 1};
        for (int a = 0; a < t->D; a++) p[a] = (b->idx[a] + 1) / 2;
        b->parent = b->level > 1 ? find_box(t, b->level - 1, p) : -1;
        for (int c = 0; c < 8; c++) b->child[c] = -1;
        for (int c = 0; c < nc; c++) {
            int q[3] = {1, 1, 1};
            for (int a = 0; a < t->D; a++) q[a] = 2 * b->idx[a] - 1 + ((c >> a) & 1);
            b->child[c] = find_box(t, b->level + 1, q);
        }
        for (int d = 0; d < ONDIR; d++) b->nb[d] = -1;
        for (int d = 0; d < nd; d++) {
            int off[3], q[3] = {1, 1, 1}, outside = 0;
            dir_offsets(t->D, d, off);
            for (int a = 0; a < t->D; a++) {
                int side = side_of(t, a, b->level);
                q[a] = pwrap(t, a, b->idx[a] + off[a], side);
                if (q[a] < 1 || q[a] > side) outside = 1;
            }
            b->nb[d] = outside ? -2 : find_box(t, b->level, q);
        }
    }
    free(t->leaf);
    t->nleaf = 0;
    t->leaf = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; i++)
        if (t->box[i].child[0] < 0) t->leaf[t->nleaf++] = i;
    free_mg(t);
    return 0;
}

/* the tree made of its root boxes alone (level 1), nr[0] x nr[1] (x nr[2]) */
static int rebuild_roots(OTree *t) {
    int R = t->nr[0] * t->nr[1] * t->nr[2];
    OPos *pos = malloc(sizeof(OPos) * (size_t)R);
    if (!pos) return -3;
    for (int r = 0; r < R; r++) {
        pos[r].level = 1;
        pos[r].idx[0] = r % t->nr[0] + 1;
        pos[r].idx[1] = (r / t->nr[0]) % t->nr[1] + 1;
        pos[r].idx[2] = r / (t->nr[0] * t->nr[1]) + 1;
        pos[r].key = morton_key(t->D, pos[r].idx);
    }
    int rc = rebuild(t, pos, R);
    free(pos);
    return rc;
}

/* A tree whose coarsest level is a rectangular block of root boxes, each the
 * unit square/cube (Sec. 2.2: a domain of several root boxes; the boxes
 * below them form several coarse boxes per level, Sec. 3.2). */
OTree *ot_create_roots(int D, int N, int max_level, const int *nroot) {
    if (D < 2 || D > 3 || N < 4 || N % 2 || N > 64 || max_level < 1) return NULL;
    if (max_level > (D == 3 ? 21 : OMAXLEV)) return NULL;
    for (int a = 0; a < 3; a++) {
        int r = a < D ? nroot[a] : 1;
        if (r < 1 || r > 64) return NULL;
        if (((long long)r << (max_level - 1)) > (1LL << 21)) return NULL;  /* Morton keys: 21 bits per axis */
    }
    OTree *t = calloc(1, sizeof(OTree));
    t->D = D; t->N = N; t->max_level = max_level;
    for (int a = 0; a < 3; a++) t->nr[a] = a < D ? nroot[a] : 1;
    rebuild_roots(t);
    return t;
}

OTree *ot_create(int D, int N, int max_level) {
    const int one[3] = {1, 1, 1};
    return ot_create_roots(D, N, max_level, one);
}

void ot_destroy(OTree *t) {
    if (!t) return;
    free_mg(t);
    free(t->box);
    free(t->leaf);
    free(t);
}

/* Refine every leaf below `level` until the tree is uniform up to `level`. */
int ot_refine_uniform(OTree *t, int level) {
    if (level > t->max_level) return -1;
    while (t->L < level) {
        int nc = 1 << t->D, n = 0, cap = t->nbox + t->nleaf * nc;
        OPos *pos = malloc(sizeof(OPos) * (size_t)cap);
        for (int i = 0; i < t->nbox; i++) {
            pos[n].level = t->box[i].level;
            memcpy(pos[n].idx, t->box[i].idx, sizeof(int) * 3);
            pos[n].key = t->box[i].key; n++;
        }
        for (int i = 0; i < t->nleaf; i++) {
            OBox *b = &t->box[t->leaf[i]];
            for (int c = 0; c < nc; c++) {
                pos[n].level = b->level + 1;
                for (int a = 0; a < 3; a++) pos[n].idx[a] = a < t->D ? 2 * b->idx[a] - 1 + ((c >> a) & 1) : 1;
                pos[n].key = morton_key(t->D, pos[n].idx); n++;
            }
        }
        int rc = rebuild(t, pos, n);
        free(pos);
        if (rc) return rc;
    }
    return 0;
}

int ot_nbox(const OTree *t) { return t->nbox; }
int ot_nleaf(const OTree *t) { return t->nleaf; }
int ot_highest_level(const OTree *t) { return t->L; }
long long ot_nleaf_cells(const OTree *t) { return (long long)t->nleaf * ipow(t->N, t->D); }

/* Export the tree in canonical order: level, spatial index (D per box),
 * parent, children (2^D per box) and neighbours (3^D-1 per box). */
void ot_export(const OTree *t, int *level, int *idx, int *parent, int *children, int *nbs) {
    int nc = 1 << t->D, nd = ipow(3, t->D) - 1;
    for (int i = 0; i < t->nbox; i++) {
        const OBox *b = &t->box[i];
        level[i] = b->level;
        for (int a = 0; a < t->D; a++) idx[i * t->D + a] = b->idx[a];
        parent[i] = b->parent;
        for (int c = 0; c < nc; c++) children[i * nc + c] = b->child[c];
        for (int d = 0; d < nd; d++) nbs[i * nd + d] = b->nb[d];
    }
}

static double cell_h(const OTree *t, int level) { return 1.0 / ((double)t->N * (double)(1 << (level - 1))); }

/* Leaf cell centres, canonical order (leaves, then cells with x fastest). */
void ot_cell_centers(const OTree *t, double *xyz) {
    int N = t->N, D = t->D, nc = ipow(N, D);
    long long o = 0;
    for (int li = 0; li < t->nleaf; li++) {
        const OBox *b = &t->box[t->leaf[li]];
        double h = cell_h(t, b->level);
        for (int c = 0; c < nc; c++) {
            int ci[3] = {c % N, (c / N) % N, c / (N * N)};
            for (int a = 0; a < D; a++) xyz[o * D + a] = ((b->idx[a] - 1) * N + ci[a] + 0.5) * h;
            o++;
        }
    }
}

/* Number of leaf boundary faces: leaves in canonical order, sides -x,+x,-y,..,
 * each physical side contributing N^(D-1) faces. */
long long ot_nbfaces(const OTree *t) {
    long long n = 0;
    for (int li = 0; li < t->nleaf; li++)
        for (int s = 0; s < 2 * t->D; s++)
            if (t->box[t->leaf[li]].nb[side_dir(t->D, s)] == -2) n += ipow(t->N, t->D - 1);
    return n;
}

/* tangential axes of side s */
static void tang_axes(int D, int s, int *t1, int *t2) {
    int a = s / 2, k = 0, ax[2] = {-1, -1};
    for (int b = 0; b < D; b++) if (b != a) ax[k++] = b;
    *t1 = ax[0]; *t2 = ax[1];
}

void ot_face_centers(const OTree *t, double *xyz) {
    int N = t->N, D = t->D, nf = ipow(N, D - 1);
    long long o = 0;
    for (int li = 0; li < t->nleaf; li++) {
        const OBox *b = &t->box[t->leaf[li]];
        double h = cell_h(t, b->level);
        for (int s = 0; s < 2 * D; s++) {
            if (b->nb[side_dir(D, s)] != -2) continue;
            int a = s / 2, t1, t2;
            tang_axes(D, s, &t1, &t2);
            for (int f = 0; f < nf; f++) {
                double x[3];
                x[a] = (s % 2) ? (double)t->nr[a] : 0.0;
                x[t1] = ((b->idx[t1] - 1) * N + f % N + 0.5) * h;
                if (t2 >= 0) x[t2] = ((b->idx[t2] - 1) * N + f / N + 0.5) * h;
                for (int c = 0; c < D; c++) xyz[o * D + c] = x[c];
                o++;
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Mesh adaptation (Sec. 2.3): cell flags +1 refine, 0 keep, -1 derefine.  */
/* ---------------------------------------------------------------------- */
int ot_adapt(OTree *t, const signed char *flags, int nbuf, int *n_added, int *n_removed) {
    int D = t->D, N = t->N, nc = 1 << D, nd = ipow(3, D) - 1, ncell = ipow(N, D);
    if (nbuf < 0 || nbuf > N) return -1;
    char *ref = calloc((size_t)t->nbox, 1), *rm = calloc((size_t)t->nbox, 1);
    char *isleaf = calloc((size_t)t->nbox, 1);
    int *leafpos = malloc(sizeof(int) * (size_t)t->nbox);
    for (int i = 0; i < t->nbox; i++) leafpos[i] = -1;
    for (int li = 0; li < t->nleaf; li++) { isleaf[t->leaf[li]] = 1; leafpos[t->leaf[li]] = li; }

    /* rule 1: a box with a cell flagged for refinement is refined; rule 2:
     * same-level leaves (diagonal ones included) within nbuf cells of such a
     * cell are refined too.  Reading: flags in boxes at max_level are ignored. */
    for (int li = 0; li < t->nleaf; li++) {
        int b = t->leaf[li];
        if (t->box[b].level >= t->max_level) continue;
        const signed char *f = flags + (long long)li * ncell;
        for (int c = 0; c < ncell; c++) {
            if (f[c] != 1) continue;
            ref[b] = 1;
            int ci[3] = {c % N + 1, (c / N) % N + 1, c / (N * N) + 1};
            for (int d = 0; d < nd; d++) {
                int off[3], near = 1;
                dir_offsets(D, d, off);
                for (int a = 0; a < D; a++) {
                    if (off[a] == -1 && !(ci[a] <= nbuf)) near = 0;
                    if (off[a] == 1 && !(ci[a] > N - nbuf)) near = 0;
                }
                int q = t->box[b].nb[d];
                if (near && q >= 0 && isleaf[q]) ref[q] = 1;
            }
        }
    }
    /* 2:1 balance: a box that gets refined needs all same-level neighbours
     * (diagonal ones included); a missing one is covered by a coarser leaf,
     * which is refined as well.  Levels are visited finest first. */
    for (int l = t->L; l >= 1; l--) {
        for (int b = t->lstart[l]; b < t->lstart[l] + t->lcount[l]; b++) {
            if (!ref[b]) continue;
            for (int d = 0; d < nd; d++) {
                if (t->box[b].nb[d] != -1) continue;
                int off[3], q[3] = {1, 1, 1};
                dir_offsets(D, d, off);
                for (int a = 0; a < D; a++) q[a] = (pwrap(t, a, t->box[b].idx[a] + off[a], side_of(t, a, l)) + 1) / 2;
                int c = find_box(t, l - 1, q);
                if (c < 0 || !isleaf[c]) { free(ref); free(rm); free(isleaf); free(leafpos); return -4; }
                ref[c] = 1;
            }
        }
    }
    /* derefinement: the 2^D children of a parent are removed when they are all
     * leaves, none is refined, every one of their cells is flagged -1, and no
     * same-level neighbour of the parent has a child that is (or becomes) refined. */
    int nrm = 0;
    for (int p = 0; p < t->nbox; p++) {
        if (isleaf[p]) continue;
        int ok = 1;
        for (int c = 0; c < nc && ok; c++) {
            int ch = t->box[p].child[c];
            if (!isleaf[ch] || ref[ch]) { ok = 0; break; }
            const signed char *f = flags + (long long)leafpos[ch] * ncell;
            for (int k = 0; k < ncell; k++) if (f[k] != -1) { ok = 0; break; }
        }
        for (int d = 0; d < nd && ok; d++) {
            int q = t->box[p].nb[d];
            if (q < 0 || isleaf[q]) continue;
            for (int c = 0; c < nc; c++) {
                int ch = t->box[q].child[c];
                if (!isleaf[ch] || ref[ch]) { ok = 0; break; }
            }
        }
        if (ok)
            for (int c = 0; c < nc; c++) { rm[t->box[p].child[c]] = 1; nrm++; }
    }
    int nadd = 0;
    for (int b = 0; b < t->nbox; b++) if (ref[b]) nadd += nc;
    OPos *pos = malloc(sizeof(OPos) * (size_t)(t->nbox + nadd));
    int n = 0;
    for (int b = 0; b < t->nbox; b++) {
        if (rm[b]) continue;
        pos[n].level = t->box[b].level;
        memcpy(pos[n].idx, t->box[b].idx, sizeof(int) * 3);
        pos[n].key = t->box[b].key; n++;
        if (ref[b])
            for (int c = 0; c < nc; c++) {
                pos[n].level = t->box[b].level + 1;
                for (int a = 0; a < 3; a++) pos[n].idx[a] = a < D ? 2 * t->box[b].idx[a] - 1 + ((c >> a) & 1) : 1;
                pos[n].key = morton_key(D, pos[n].idx); n++;
            }
    }
    int rc = rebuild(t, pos, n);
    free(pos); free(ref); free(rm); free(isleaf); free(leafpos);
    if (n_added) *n_added = nadd;
    if (n_removed) *n_removed = nrm;
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Multigrid hierarchy: tree levels plus the coarse grids below the root   */
/* (boxes of N/2, N/4, ..., 2 cells; Sec. 3.2 "V-cycle").                   */
/* ---------------------------------------------------------------------- */

static void free_mg(OTree *t) {
    if (!t->mg) { t->mg_ready = 0; return; }
    for (int i = 0; i < t->nmg; i++) {
        OMG *m = &t->mg[i];
        free(m->u); free(m->rho); free(m->vold); free(m->r); free(m->rr); free(m->d); free(m->eps);
        for (int s = 0; s < 6; s++) free(m->bc[s]);
    }
    free(t->mg);
    t->mg = NULL; t->nmg = 0; t->mg_ready = 0;
}

static int ncells_g(int D, int M) { return ipow(M + 2, D); }
/* index of cell (i,j,k), 0..M+1 each (0 and M+1 are ghosts) */
#define GI(M, i, j, k) ((((k) * ((M) + 2)) + (j)) * ((M) + 2) + (i))

int ot_mg_setup(OTree *t) {
    free_mg(t);
    int D = t->D, N = t->N;
    int nsub = 0;
    for (int M = N / 2; M >= 2; M /= 2) nsub++;
    /* R root boxes (the level-1 boxes, canonical order); below each of them
     * one box per coarse level, connected like the roots */
    const int R = t->lcount[1], r0 = t->lstart[1];
    const int nsubR = nsub * R;
    t->lmin = 1 - nsub;
    t->nmg = nsubR + t->nbox;
    t->mg = calloc((size_t)t->nmg, sizeof(OMG));
    for (int i = 0; i < 2 * OMAXLEV + 8; i++) { t->mgstart[i] = 0; t->mgcount[i] = 0; }
    /* boxes below the roots: level lmin .. 0, R each, in the roots' order */
    for (int i = 0; i < nsub; i++) {
        for (int r = 0; r < R; r++) {
            OMG *m = &t->mg[i * R + r];
            m->level = t->lmin + i;
            m->M = N >> (1 - m->level);
            m->h = 1.0 / m->M;
            m->tbox = -1;
            m->parent = i > 0 ? (i - 1) * R + r : -1;
            m->refined = 1;
            for (int a = 0; a < 3; a++) m->x0[a] = a < D ? (double)(t->box[r0 + r].idx[a] - 1) : 0.0;
            for (int s = 0; s < 2 * D; s++) {
                /* the root's neighbour across side s (itself across a periodic
                 * side of a one-root axis) */
                int q = t->box[r0 + r].nb[side_dir(D, s)];
                if (q >= 0) { m->kind[s] = K_SAME; m->nbid[s] = i * R + (q - r0); }
                else { m->kind[s] = K_PHYS; m->nbid[s] = -1; }
            }
            for (int d = 0; d < ONDIR; d++) {
                int q = d < ipow(3, D) - 1 ? t->box[r0 + r].nb[d] : -1;
                m->nball[d] = q >= 0 ? i * R + (q - r0) : -1;
            }
        }
        t->mgstart[i] = i * R; t->mgcount[i] = R;
    }
    for (int b = 0; b < t->nbox; b++) {
        OMG *m = &t->mg[nsubR + b];
        const OBox *tb = &t->box[b];
        m->level = tb->level; m->M = N; m->h = cell_h(t, tb->level);
        m->tbox = b;
        for (int a = 0; a < 3; a++) m->x0[a] = a < D ? (double)(tb->idx[a] - 1) * N * m->h : 0.0;
        m->refined = tb->child[0] >= 0;
        if (tb->level == 1) {
            m->parent = nsub > 0 ? (nsub - 1) * R + (b - r0) : -1;
            for (int a = 0; a < 3; a++) m->poff[a] = 0;
        } else {
            m->parent = nsubR + tb->parent;
            for (int a = 0; a < D; a++) m->poff[a] = ((tb->idx[a] - 1) & 1) * (N / 2);
        }
        for (int d = 0; d < ONDIR; d++) {
            int q = d < ipow(3, D) - 1 ? tb->nb[d] : -1;
            m->nball[d] = q >= 0 ? nsubR + q : -1;
        }
        for (int s = 0; s < 2 * D; s++) {
            int q = tb->nb[side_dir(D, s)];
            if (q >= 0) { m->kind[s] = K_SAME; m->nbid[s] = nsubR + q; }
            else if (q == -2) { m->kind[s] = K_PHYS; m->nbid[s] = -1; }
            else {
                /* refinement boundary: the coarse box is the parent's neighbour */
                int cq = t->box[tb->parent].nb[side_dir(D, s)];
                if (cq < 0) return -4;
                m->kind[s] = K_CF; m->nbid[s] = nsubR + cq;
            }
        }
        int li = tb->level - t->lmin;
        if (t->mgcount[li] == 0) t->mgstart[li] = nsubR + b;
        t->mgcount[li]++;
    }
    for (int i = 0; i < t->nmg; i++) {
        OMG *m = &t->mg[i];
        size_t ng = (size_t)ncells_g(D, m->M);
        m->u = calloc(ng, sizeof(double)); m->rho = calloc(ng, sizeof(double));
        m->vold = calloc(ng, sizeof(double)); m->r = calloc(ng, sizeof(double));
        m->rr = calloc(ng, sizeof(double)); m->d = calloc(ng, sizeof(double));
        m->eps = malloc(ng * sizeof(double));
        if (!m->u || !m->rho || !m->vold || !m->r || !m->rr || !m->d || !m->eps) return -3;
        for (size_t g = 0; g < ng; g++) m->eps[g] = 1.0;
        for (int s = 0; s < 2 * D; s++)
            if (m->kind[s] == K_PHYS) m->bc[s] = calloc((size_t)ipow(m->M, D - 1), sizeof(double));
    }
    t->mg_ready = 1;
    t->hom = 0;
    return 0;
}

static OMG *leaf_mg(OTree *t, int li) { return &t->mg[(t->nmg - t->nbox) + t->leaf[li]]; }

/* interior cell c (x fastest, 0-based) of an M-box -> ghosted index */
static int interior_index(int D, int M, int c) {
    int i = c % M + 1, j = (c / M) % M + 1, k = D == 3 ? c / (M * M) + 1 : 0;
    return GI(M, i, j, k);
}

void ot_set_rhs(OTree *t, const double *rho) {
    int D = t->D, nc = ipow(t->N, D);
    for (int li = 0; li < t->nleaf; li++) {
        OMG *m = leaf_mg(t, li);
        for (int c = 0; c < nc; c++) m->rho[interior_index(D, m->M, c)] = rho[(long long)li * nc + c];
    }
}

void ot_set_solution(OTree *t, const double *u) {
    int D = t->D, nc = ipow(t->N, D);
    for (int li = 0; li < t->nleaf; li++) {
        OMG *m = leaf_mg(t, li);
        for (int c = 0; c < nc; c++) m->u[interior_index(D, m->M, c)] = u[(long long)li * nc + c];
    }
}

void ot_get_solution(const OTree *t, double *u) {
    int D = t->D, nc = ipow(t->N, D);
    for (int li = 0; li < t->nleaf; li++) {
        OMG *m = leaf_mg((OTree *)t, li);
        for (int c = 0; c < nc; c++) u[(long long)li * nc + c] = m->u[interior_index(D, m->M, c)];
    }
}

/* Zero the solution on every level (a fresh start). */
void ot_zero_solution(OTree *t) {
    for (int i = 0; i < t->nmg; i++) memset(t->mg[i].u, 0, sizeof(double) * (size_t)ncells_g(t->D, t->mg[i].M));
}

/* Face cell f of side s: tangential coordinates (0-based) */
static void face_tc(int M, int f, int *c1, int *c2) { *c1 = f % M; *c2 = f / M; }

/* Boundary data on leaf boundary faces (canonical face order): values on
 * Dirichlet sides, outward normal derivatives on Neumann sides; coarse boxes
 * get the mean of the 2^(D-1) finer faces they cover.  Reading: the paper's
 * boundary routine is called per box; with data given only on leaf faces the
 * coarse values are their averages (they do not change the converged
 * composite solution). */
void ot_set_dirichlet(OTree *t, const double *b) {
    int D = t->D, nf = ipow(t->N, D - 1);
    long long o = 0;
    for (int li = 0; li < t->nleaf; li++) {
        OMG *m = leaf_mg(t, li);
        for (int s = 0; s < 2 * D; s++) {
            if (m->kind[s] != K_PHYS) continue;
            for (int f = 0; f < nf; f++) m->bc[s][f] = b[o++];
        }
    }
    /* coarse boxes: levels from finest to coarsest */
    for (int i = 0; i < t->nmg; i++)
        if (t->mg[i].refined)
            for (int s = 0; s < 2 * D; s++)
                if (t->mg[i].kind[s] == K_PHYS) memset(t->mg[i].bc[s], 0, sizeof(double) * (size_t)ipow(t->mg[i].M, D - 1));
    for (int l = t->L; l > t->lmin; l--) {
        int li = l - t->lmin;
        for (int i = t->mgstart[li]; i < t->mgstart[li] + t->mgcount[li]; i++) {
            OMG *m = &t->mg[i];
            OMG *p = &t->mg[m->parent];
            for (int s = 0; s < 2 * D; s++) {
                if (m->kind[s] != K_PHYS || p->kind[s] != K_PHYS) continue;
                int t1, t2;
                tang_axes(D, s, &t1, &t2);
                int mf = ipow(m->M, D - 1);
                for (int f = 0; f < mf; f++) {
                    int c1, c2;
                    face_tc(m->M, f, &c1, &c2);
                    int p1 = m->poff[t1] + c1 / 2, p2 = t2 >= 0 ? m->poff[t2] + c2 / 2 : 0;
                    p->bc[s][p2 * p->M + p1] += m->bc[s][f] / (double)(1 << (D - 1));
                }
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Ghost cells (Sec. 2.4 and the conservative scheme of Sec. 3.3).        */
/* ---------------------------------------------------------------------- */

/* position along axis a of the first interior cell next to side s, and of the ghost */
static void side_cells(int M, int s, int *inner, int *second, int *ghost) {
    if (s % 2 == 0) { *inner = 1; *second = 2; *ghost = 0; }
    else { *inner = M; *second = M - 1; *ghost = M + 1; }
}

/* Problems without a Dirichlet side (only Neumann and periodic sides) are
 * singular: constants are the null space of the composite operator, and
 * A u = rho has a solution only for a compatible source,
 *   sum_leaves h^D rho = sum_(Neumann leaf faces) h^(D-1) b
 * (the discrete divergence theorem: the conservative scheme of Sec. 3.3
 * makes the flux sums cancel between cells).  Sec. 4.4's gravity problem
 * subtracts the mean source.  Reading: the solver solves A u = rho - c with
 * c = (sum h^D rho - sum h^(D-1) b) / sum h^D -- the source less its
 * volume-weighted mean and the boundary inflow per volume (c = 0 for a
 * compatible source, so the step is idempotent) -- and picks the solution of
 * zero volume-weighted mean: after every cycle the leaf mean is subtracted
 * from the leaves.  Only the Laplacian (op 0). */
static void make_compatible(OTree *t) {
    if (!t->singular) return;
    int D = t->D, nc = ipow(t->N, D), nf = ipow(t->N, D - 1);
    double sr = 0.0, sb = 0.0, sv = 0.0;
    for (int li = 0; li < t->nleaf; li++) {
        OMG *m = leaf_mg(t, li);
        double vol = 1.0, area = 1.0;
        for (int a = 0; a < D; a++) vol *= m->h;
        for (int a = 0; a < D - 1; a++) area *= m->h;
        for (int c = 0; c < nc; c++) sr += vol * m->rho[interior_index(D, m->M, c)];
        sv += vol * nc;
        if (t->hom) continue;
        for (int s = 0; s < 2 * D; s++)
            if (m->kind[s] == K_PHYS && t->bct[s] == 1)
                for (int f = 0; f < nf; f++) sb += area * m->bc[s][f];
    }
    double c = (sr - sb) / sv;
    for (int li = 0; li < t->nleaf; li++) {
        OMG *m = leaf_mg(t, li);
        for (int q = 0; q < nc; q++) m->rho[interior_index(D, m->M, q)] -= c;
    }
}

/* the volume-weighted leaf mean of u, subtracted from the leaves */
static void remove_mean(OTree *t) {
    if (!t->singular) return;
    int D = t->D, nc = ipow(t->N, D);
    double su = 0.0, sv = 0.0;
    for (int li = 0; li < t->nleaf; li++) {
        OMG *m = leaf_mg(t, li);
        double vol = 1.0;
        for (int a = 0; a < D; a++) vol *= m->h;
        for (int c = 0; c < nc; c++) su += vol * m->u[interior_index(D, m->M, c)];
        sv += vol * nc;
    }
    double mean = su / sv;
    for (int li = 0; li < t->nleaf; li++) {
        OMG *m = leaf_mg(t, li);
        for (int c = 0; c < nc; c++) m->u[interior_index(D, m->M, c)] -= mean;
    }
}

/* Fill the side ghost cells of variable `which` (0 = u, 1 = d) of all boxes
 * of a level.  Same-level neighbour: copy.  Physical boundary, Dirichlet:
 * g = 2 b - u_1 (reading: b is the value at the face centre; the linear
 * extrapolation through it); Neumann: g = u_1 + h b (b the outward normal
 * derivative); for the correction d the data is homogeneous.
 * Refinement boundary: the paper's default two-point conservative scheme,
 *   2D: g = u_H/2 + u_1 - (u_t + u_2)/4,
 *   3D: g = u_H/2 + 5/4 u_1 - (u_2 + u_t1 + u_t2)/4,
 * with u_1 the cell next to the ghost, u_2 the next cell inward, u_t the
 * other fine cell(s) of this box under the same coarse face cell, and u_H the
 * coarse leaf cell across the face.  Edge/corner ghosts are not filled: the
 * (2D+1)-point operator, the scheme above and the 2-1-1 / 1-1-1-1
 * prolongation never read them. */
static void fill_ghosts(OTree *t, int level, int which) {
    int D = t->D, li = level - t->lmin;
    int i0 = t->mgstart[li], i1 = i0 + t->mgcount[li];
#pragma omp parallel for schedule(static)
    for (int i = i0; i < i1; i++) {
        OMG *m = &t->mg[i];
        int M = m->M;
        double *v = which == 0 ? m->u : which == 1 ? m->d : m->eps;
        for (int s = 0; s < 2 * D; s++) {
            int a = s / 2, t1, t2;
            tang_axes(D, s, &t1, &t2);
            int inner, second, ghost;
            side_cells(M, s, &inner, &second, &ghost);
            int nf = ipow(M, D - 1);
            for (int f = 0; f < nf; f++) {
                int c1, c2;
                face_tc(M, f, &c1, &c2);
                int pg[3] = {0, 0, 0}, p1[3], p2[3];
                pg[t1] = c1 + 1;
                if (t2 >= 0) pg[t2] = c2 + 1;
                memcpy(p1, pg, sizeof pg); memcpy(p2, pg, sizeof pg);
                pg[a] = ghost; p1[a] = inner; p2[a] = second;
                int gi = GI(M, pg[0], pg[1], pg[2]);
                int ii = GI(M, p1[0], p1[1], p1[2]);
                if (m->kind[s] == K_SAME) {
                    OMG *q = &t->mg[m->nbid[s]];
                    double *w = which == 0 ? q->u : which == 1 ? q->d : q->eps;
                    int pq[3]; memcpy(pq, pg, sizeof pg);
                    pq[a] = (s % 2 == 0) ? M : 1;
                    v[gi] = w[GI(M, pq[0], pq[1], pq[2])];
                } else if (m->kind[s] == K_PHYS && which == 2) {
                    v[gi] = v[ii];  /* the coefficient is mirrored: the face takes the cell's own */
                } else if (m->kind[s] == K_PHYS) {
                    double bval = (which == 0 && !t->hom) ? m->bc[s][f] : 0.0;
                    if (t->bct[s] == 1) v[gi] = v[ii] + m->h * bval;
                    else v[gi] = 2.0 * bval - v[ii];
                } else if (which != 1) {
                    /* coarse-fine; the correction d never needs this */
                    OMG *q = &t->mg[m->nbid[s]];
                    int pc[3] = {0, 0, 0};
                    pc[a] = (s % 2 == 0) ? q->M : 1;
                    pc[t1] = m->poff[t1] + c1 / 2 + 1;
                    if (t2 >= 0) pc[t2] = m->poff[t2] + c2 / 2 + 1;
                    if (which == 2) {  /* the coefficient of the coarse cell across the face */
                        v[gi] = q->eps[GI(q->M, pc[0], pc[1], pc[2])];
                        continue;
                    }
                    double uH = q->u[GI(q->M, pc[0], pc[1], pc[2])];
                    int pt[3]; memcpy(pt, p1, sizeof pt);
                    pt[t1] = (c1 % 2 == 0) ? c1 + 2 : c1; /* partner: 1-based c1+1 odd -> +1 */
                    double ut1 = v[GI(M, pt[0], pt[1], pt[2])];
                    double u2 = v[GI(M, p2[0], p2[1], p2[2])];
                    if (D == 2) {
                        v[gi] = 0.5 * uH + v[ii] - 0.25 * (ut1 + u2);
                    } else {
                        int pu[3]; memcpy(pu, p1, sizeof pu);
                        pu[t2] = (c2 % 2 == 0) ? c2 + 2 : c2;
                        double ut2 = v[GI(M, pu[0], pu[1], pu[2])];
                        v[gi] = 0.5 * uH + 1.25 * v[ii] - 0.25 * (u2 + ut1 + ut2);
                    }
                }
            }
        }
    }
}

/* Edge and corner ghost cells (Sec. 2.4) of variable `which` (0 = u, 1 = d)
 * of all boxes of a level, after the side ghosts: copied from the diagonal
 * neighbour when it exists at the same level, otherwise linearly
 * extrapolated -- in 2D the corner ghost gets b + c - a (b, c the two side
 * ghosts next to it, a the corner cell); in 3D an edge ghost likewise from
 * its two side ghosts and the edge cell, and a corner ghost from the edge
 * ghost next to it along x, the side ghost next to it along y-z and the
 * corner cell: f(p) = f(p + u) + f(p + w) - f(p + u + w) for the unit steps
 * u (into the box along the first ghost axis) and w (along the others), which
 * is exact for linear f.  Edges are filled before corners. */
static void fill_corner_ghosts(OTree *t, int level, int which) {
    int D = t->D, li = level - t->lmin, nd = ipow(3, D) - 1;
    int i0 = t->mgstart[li], i1 = i0 + t->mgcount[li];
    for (int pass = 2; pass <= D; pass++) {
#pragma omp parallel for schedule(static)
        for (int b = i0; b < i1; b++) {
            OMG *m = &t->mg[b];
            int M = m->M;
            double *v = which == 0 ? m->u : m->d;
            for (int d = 0; d < nd; d++) {
                int off[3];
                dir_offsets(D, d, off);
                int nz = 0, ax[3], na = 0;
                for (int a = 0; a < D; a++) if (off[a]) { nz++; ax[na++] = a; }
                if (nz != pass) continue;
                const OMG *q = m->nball[d] >= 0 ? &t->mg[m->nball[d]] : NULL;
                const double *w = q ? (which == 0 ? q->u : q->d) : NULL;
                int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
                for (int a = 0; a < D; a++) {
                    if (off[a] < 0) lo[a] = hi[a] = 0;
                    else if (off[a] > 0) lo[a] = hi[a] = M + 1;
                    else { lo[a] = 1; hi[a] = M; }
                }
                for (int k = lo[2]; k <= hi[2]; k++)
                    for (int j = lo[1]; j <= hi[1]; j++)
                        for (int i = lo[0]; i <= hi[0]; i++) {
                            int p[3] = {i, j, k};
                            if (w) {
                                int pq[3] = {i, j, k};
                                for (int a = 0; a < D; a++)
                                    if (off[a] < 0) pq[a] = M; else if (off[a] > 0) pq[a] = 1;
                                v[GI(M, p[0], p[1], p[2])] = w[GI(M, pq[0], pq[1], pq[2])];
                                continue;
                            }
                            int pu[3] = {i, j, k}, pw[3] = {i, j, k}, pa[3] = {i, j, k};
                            /* u: step in along the first ghost axis; w: along the others */
                            pu[ax[0]] = off[ax[0]] < 0 ? 1 : M;
                            for (int e = 1; e < na; e++) pw[ax[e]] = off[ax[e]] < 0 ? 1 : M;
                            for (int e = 0; e < na; e++) pa[ax[e]] = off[ax[e]] < 0 ? 1 : M;
                            v[GI(M, p[0], p[1], p[2])] = v[GI(M, pu[0], pu[1], pu[2])] + v[GI(M, pw[0], pw[1], pw[2])]
                                                         - v[GI(M, pa[0], pa[1], pa[2])];
                        }
            }
        }
    }
}

/* sum of the 2D face neighbours of cell g, order ((x-+x+)+(y-+y+))+(z-+z+) */
static double nbsum(int D, int M, const double *v, int i, int j, int k) {
    double s = (v[GI(M, i - 1, j, k)] + v[GI(M, i + 1, j, k)]) + (v[GI(M, i, j - 1, k)] + v[GI(M, i, j + 1, k)]);
    if (D == 3) s += v[GI(M, i, j, k - 1)] + v[GI(M, i, j, k + 1)];
    return s;
}

static void wsum(const OTree *t, const OMG *m, const double *v, int i, int j, int k, double *sv, double *sc);

/* One half-sweep of red-black Gauss-Seidel (Sec. 3.1) on all boxes of a
 * level.  Colour 0 (red) = cells whose 1-based indices sum to an even number.
 * For the Poisson operator the local solve is u = (sum nb - h^2 rho)/(2D). */
static void gsrb_half(OTree *t, int level, int colour) {
    int D = t->D, li = level - t->lmin;
    int i0 = t->mgstart[li], i1 = i0 + t->mgcount[li];
    double inv = 1.0 / (2.0 * D);
#pragma omp parallel for schedule(static)
    for (int b = i0; b < i1; b++) {
        OMG *m = &t->mg[b];
        int M = m->M, kmax = D == 3 ? M : 1;
        double h2 = m->h * m->h;
        for (int k = (D == 3 ? 1 : 0); k <= (D == 3 ? kmax : 0); k++)
            for (int j = 1; j <= M; j++)
                for (int i = 1; i <= M; i++) {
                    if ((i + j + k) % 2 != colour) continue;
                    int g = GI(M, i, j, k);
                    if (t->op) {  /* local solve of the variable-coefficient equation */
                        double sv, sc;
                        wsum(t, m, m->u, i, j, k, &sv, &sc);
                        m->u[g] = (sv - h2 * m->rho[g]) / sc;
                    } else {
                        m->u[g] = (nbsum(D, M, m->u, i, j, k) - h2 * m->rho[g]) * inv;
                    }
                }
    }
}

/* N smoothing steps: each is a red and a black half-sweep, the ghost cells
 * being refilled before every half-sweep (reading: ghosts are data that stay
 * fixed during one half-sweep). */
static void smooth(OTree *t, int level, int n) {
    for (int it = 0; it < n; it++)
        for (int c = 0; c < 2; c++) {
            fill_ghosts(t, level, 0);
            gsrb_half(t, level, c);
        }
}

/* A_h(u) at one cell (needs filled ghosts) */
static double lap(int D, int M, double h, const double *v, int i, int j, int k) {
    return (nbsum(D, M, v, i, j, k) - 2.0 * D * v[GI(M, i, j, k)]) / (h * h);
}

/* Variable-coefficient operators (Sec. 3.4-3.5), div(eps grad u) = rho:
 * the flux through the face between cells of coefficients e1 and e2 is the
 * harmonic mean 2 e1 e2 / (e1 + e2) times the difference quotient (Sec. 3.4:
 * the local reconstruction with a jump of eps at the face).  In (r,z)
 * coordinates (2D, r = x) the divergence is (1/r) d/dr (r eps du/dr) +
 * d/dz (eps du/dz), so the r-faces are also weighted by r_face / r_cell, and
 * the face on the axis r = 0 carries no flux.  c[s] is the coefficient of
 * side s (-x,+x,-y,+y,-z,+z) of cell (i,j,k) of box m (ghosts of eps filled). */
static void face_coef(const OTree *t, const OMG *m, int i, int j, int k, double *c) {
    const int D = t->D, M = m->M;
    const int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
    const double e0 = m->eps[GI(M, i, j, k)];
    for (int s = 0; s < 2 * D; s++) {
        const double en = m->eps[GI(M, nb[s][0], nb[s][1], nb[s][2])];
        c[s] = 2.0 * e0 * en / (e0 + en);
    }
    if (t->op == 2) {
        const double rc = m->x0[0] + (i - 0.5) * m->h;
        c[0] *= (m->x0[0] + (i - 1) * m->h) / rc;
        c[1] *= (m->x0[0] + i * m->h) / rc;
    }
}

/* sum_s c_s v_s and sum_s c_s over the faces of cell (i,j,k), in side order */
static void wsum(const OTree *t, const OMG *m, const double *v, int i, int j, int k, double *sv, double *sc) {
    const int D = t->D, M = m->M;
    const int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
    double c[6], a = 0.0, b = 0.0;
    face_coef(t, m, i, j, k, c);
    for (int s = 0; s < 2 * D; s++) {
        a += c[s] * v[GI(M, nb[s][0], nb[s][1], nb[s][2])];
        b += c[s];
    }
    *sv = a;
    *sc = b;
}

/* A_h(v) at one cell for the tree's operator (needs filled ghosts):
 * (sum_s c_s (v_s - v)) / h^2 */
static double op_apply(const OTree *t, const OMG *m, const double *v, int i, int j, int k) {
    if (t->op == 0) return lap(t->D, m->M, m->h, v, i, j, k);
    double sv, sc;
    wsum(t, m, v, i, j, k, &sv, &sc);
    return (sv - sc * v[GI(m->M, i, j, k)]) / (m->h * m->h);
}

/* residual r = rho - A_h(u) (Eq. residual) on all boxes of a level */
static void residual_level(OTree *t, int level) {
    int D = t->D, li = level - t->lmin;
    int i0 = t->mgstart[li], i1 = i0 + t->mgcount[li];
#pragma omp parallel for schedule(static)
    for (int b = i0; b < i1; b++) {
        OMG *m = &t->mg[b];
        int M = m->M;
        for (int k = (D == 3 ? 1 : 0); k <= (D == 3 ? M : 0); k++)
            for (int j = 1; j <= M; j++)
                for (int i = 1; i <= M; i++) {
                    int g = GI(M, i, j, k);
                    m->r[g] = m->rho[g] - op_apply(t, m, m->u, i, j, k);
                }
    }
}

/* Restriction by averaging the 2^D children (Sec. 2.5): every box of `level`
 * writes the mean of its cells into its region of the parent.  which: 0 = u
 * into u, 1 = r into rr, 2 = eps into eps. */
static void restrict_level(OTree *t, int level, int which) {
    int D = t->D, li = level - t->lmin;
    int i0 = t->mgstart[li], i1 = i0 + t->mgcount[li];
#pragma omp parallel for schedule(static)
    for (int b = i0; b < i1; b++) {
        OMG *m = &t->mg[b];
        OMG *p = &t->mg[m->parent];
        const double *src = which == 0 ? m->u : which == 1 ? m->r : m->eps;
        double *dst = which == 0 ? p->u : which == 1 ? p->rr : p->eps;
        int Mh = m->M / 2;
        for (int K = 0; K < (D == 3 ? Mh : 1); K++)
            for (int J = 0; J < Mh; J++)
                for (int I = 0; I < Mh; I++) {
                    int pk = D == 3 ? m->poff[2] + K + 1 : 0;
                    double *out = &dst[GI(p->M, m->poff[0] + I + 1, m->poff[1] + J + 1, pk)];
                    if (t->op == 2) {
                        /* (r,z): the mean weighted by the children's volumes, proportional to r */
                        double s = 0.0, w = 0.0;
                        for (int dy = 0; dy < 2; dy++)
                            for (int dx = 0; dx < 2; dx++) {
                                const double r = m->x0[0] + (2 * I + dx + 0.5) * m->h;
                                s += r * src[GI(m->M, 2 * I + 1 + dx, 2 * J + 1 + dy, 0)];
                                w += r;
                            }
                        *out = s / w;
                        continue;
                    }
                    double s = 0.0;
                    for (int dz = 0; dz < (D == 3 ? 2 : 1); dz++)
                        for (int dy = 0; dy < 2; dy++)
                            for (int dx = 0; dx < 2; dx++)
                                s += src[GI(m->M, 2 * I + 1 + dx, 2 * J + 1 + dy, D == 3 ? 2 * K + 1 + dz : 0)];
                    *out = s / (double)(1 << D);
                }
    }
}

/* Coarse update of the FAS V-cycle: v_H <- I v_h (already done), store v'_H,
 * rho_H <- I r_h + A_H(v_H) (Eq. coarse-rhs) on the refined boxes of `level`. */
static void fas_coarse(OTree *t, int level) {
    int D = t->D, li = level - t->lmin;
    int i0 = t->mgstart[li], i1 = i0 + t->mgcount[li];
    fill_ghosts(t, level, 0);
#pragma omp parallel for schedule(static)
    for (int b = i0; b < i1; b++) {
        OMG *m = &t->mg[b];
        int M = m->M;
        memcpy(m->vold, m->u, sizeof(double) * (size_t)ncells_g(D, M));
        if (!m->refined) continue;
        for (int k = (D == 3 ? 1 : 0); k <= (D == 3 ? M : 0); k++)
            for (int j = 1; j <= M; j++)
                for (int i = 1; i <= M; i++) {
                    int g = GI(M, i, j, k);
                    m->rho[g] = m->rr[g] + op_apply(t, m, m->u, i, j, k);
                }
    }
}

/* Coarse-grid correction u_h <- u_h + I_H^h (v_H - v'_H) (Eq. coarse-corr)
 * on all boxes of `level`, with the 2-1-1 (2D) / 1-1-1-1 (3D) linear
 * prolongation (Sec. 2.5).  Reading: "first order prolongation" in Sec. 4.1
 * is this linear scheme.  Ghosts of the difference: same-level copy, and the
 * homogeneous Dirichlet value at physical boundaries. */
static void correct_level(OTree *t, int level) {
    int D = t->D;
    int lc = level - 1 - t->lmin;
    int c0 = t->mgstart[lc], c1 = c0 + t->mgcount[lc];
    for (int b = c0; b < c1; b++) {
        OMG *m = &t->mg[b];
        int ng = ncells_g(D, m->M);
        for (int g = 0; g < ng; g++) m->d[g] = m->u[g] - m->vold[g];
    }
    fill_ghosts(t, level - 1, 1);
    if (t->prolong == 1) fill_corner_ghosts(t, level - 1, 1);
    int li = level - t->lmin;
    int i0 = t->mgstart[li], i1 = i0 + t->mgcount[li];
#pragma omp parallel for schedule(static)
    for (int b = i0; b < i1; b++) {
        OMG *m = &t->mg[b];
        OMG *p = &t->mg[m->parent];
        int M = m->M;
        for (int k = (D == 3 ? 1 : 0); k <= (D == 3 ? M : 0); k++)
            for (int j = 1; j <= M; j++)
                for (int i = 1; i <= M; i++) {
                    int f[3] = {i, j, k}, C[3] = {0, 0, 0}, sgn[3] = {0, 0, 0};
                    for (int a = 0; a < D; a++) {
                        C[a] = m->poff[a] + (f[a] + 1) / 2;
                        sgn[a] = (f[a] % 2 == 1) ? -1 : 1;
                    }
                    double d0 = p->d[GI(p->M, C[0], C[1], C[2])];
                    if (t->prolong == 2) {  /* zeroth order: the coarse value */
                        m->u[GI(M, i, j, k)] += d0;
                        continue;
                    }
                    if (t->prolong == 1) {
                        /* bi/trilinear: the 2^D nearest coarse cells, weight 3/4 per
                         * axis for the nearer one and 1/4 for the farther one */
                        double add = 0.0;
                        for (int c = 0; c < (1 << D); c++) {
                            int q[3] = {C[0], C[1], C[2]};
                            double wgt = 1.0;
                            for (int a = 0; a < D; a++) {
                                if ((c >> a) & 1) { q[a] += sgn[a]; wgt *= 0.25; }
                                else wgt *= 0.75;
                            }
                            add += wgt * p->d[GI(p->M, q[0], q[1], q[2])];
                        }
                        m->u[GI(M, i, j, k)] += add;
                        continue;
                    }
                    double dx = p->d[GI(p->M, C[0] + sgn[0], C[1], C[2])];
                    double dy = p->d[GI(p->M, C[0], C[1] + sgn[1], C[2])];
                    double add;
                    if (D == 2) add = 0.5 * d0 + 0.25 * (dx + dy);
                    else {
                        double dz = p->d[GI(p->M, C[0], C[1], C[2] + sgn[2])];
                        add = 0.25 * (((d0 + dx) + dy) + dz);
                    }
                    m->u[GI(M, i, j, k)] += add;
                }
    }
}

/* The FAS V-cycle of Sec. 3.2 from level `ltop` down to the coarsest grid
 * and back.  Reading: smoothing, residual and correction act on all boxes of
 * a level (parents and leaves); the coarse right-hand side is set on the
 * refined boxes only, leaves keep the user's source term. */
static void vcycle_from(OTree *t, int ltop, int nd, int nu, int nb) {
    for (int l = ltop; l > t->lmin; l--) {
        smooth(t, l, nd);
        fill_ghosts(t, l, 0);
        residual_level(t, l);
        restrict_level(t, l, 0);
        restrict_level(t, l, 1);
        fas_coarse(t, l - 1);
    }
    smooth(t, t->lmin, nb);
    for (int l = t->lmin + 1; l <= ltop; l++) {
        correct_level(t, l);
        smooth(t, l, nu);
    }
}

void ot_vcycle(OTree *t, int nd, int nu, int nb) {
    make_compatible(t);
    vcycle_from(t, t->L, nd, nu, nb);
    remove_mean(t);
}

/* FMG cycle (Sec. 3.2).  Reading: both start cases are handled by one rule:
 * the current leaf values (zero for a fresh start) are restricted down to
 * the coarsest grid, and Eq. coarse-rhs sets the coarse source terms. */
void ot_fmg(OTree *t, int nd, int nu, int nb) {
    make_compatible(t);
    for (int l = t->L; l > t->lmin; l--) restrict_level(t, l, 0);
    for (int l = t->L; l > t->lmin; l--) {
        fill_ghosts(t, l, 0);
        residual_level(t, l);
        restrict_level(t, l, 1);
        fas_coarse(t, l - 1);
    }
    for (int l = t->lmin; l <= t->L; l++) {
        int li = l - t->lmin;
        for (int b = t->mgstart[li]; b < t->mgstart[li] + t->mgcount[li]; b++)
            memcpy(t->mg[b].vold, t->mg[b].u, sizeof(double) * (size_t)ncells_g(t->D, t->mg[b].M));
        if (l > t->lmin) {
            /* correction from l-1 uses the copy stored at the start of step l-1 */
            correct_level(t, l);
        }
        vcycle_from(t, l, nd, nu, nb);
    }
    remove_mean(t);
}

/* Residual norms on the leaves.  Reading: "relative residual" =
 * max_leaf |rho - A u| / max_leaf |rho|; before evaluating it the solution is
 * restricted to every parent so that a leaf next to a refined same-level box
 * sees the mean of the fine cells (the composite operator). */
void ot_residual_norm(OTree *t, double *rmax, double *rhomax) {
    int D = t->D;
    make_compatible(t);
    for (int l = t->L; l > 1; l--) restrict_level(t, l, 0);
    for (int l = 1; l <= t->L; l++) fill_ghosts(t, l, 0);
    double rm = 0.0, pm = 0.0;
    for (int li = 0; li < t->nleaf; li++) {
        OMG *m = leaf_mg(t, li);
        int M = m->M;
        for (int k = (D == 3 ? 1 : 0); k <= (D == 3 ? M : 0); k++)
            for (int j = 1; j <= M; j++)
                for (int i = 1; i <= M; i++) {
                    int g = GI(M, i, j, k);
                    double r = fabs(m->rho[g] - op_apply(t, m, m->u, i, j, k));
                    if (r > rm) rm = r;
                    if (fabs(m->rho[g]) > pm) pm = fabs(m->rho[g]);
                }
    }
    *rmax = rm; *rhomax = pm;
}

/* Composite operator on leaf data: out = A(u) (boundary data included),
 * evaluated by the box machinery (restriction to parents, ghost fill,
 * stencil).  The solution stored in the tree is overwritten by u. */
void ot_apply_A(OTree *t, const double *u, double *out) {
    int D = t->D, nc = ipow(t->N, D);
    ot_set_solution(t, u);
    for (int l = t->L; l > 1; l--) restrict_level(t, l, 0);
    for (int l = 1; l <= t->L; l++) fill_ghosts(t, l, 0);
    for (int li = 0; li < t->nleaf; li++) {
        OMG *m = leaf_mg(t, li);
        for (int c = 0; c < nc; c++) {
            int M = m->M, i = c % M + 1, j = (c / M) % M + 1, k = D == 3 ? c / (M * M) + 1 : 0;
            out[(long long)li * nc + c] = op_apply(t, m, m->u, i, j, k);
        }
    }
}

void ot_set_homogeneous(OTree *t, int hom) { t->hom = hom; }

/* value at fine cell f (1-based, in a child box at offset poff of its
 * parent) prolonged from the parent's ghosted array p (M cells per side):
 * scheme 0 linear (1/2,1/4,1/4) / (1/4,1/4,1/4,1/4), 1 bi/trilinear, 2 copy */
static double prolong_value(int D, int M, const double *p, const int *poff, const int *f, int scheme) {
    int C[3] = {0, 0, 0}, sgn[3] = {0, 0, 0};
    for (int a = 0; a < D; a++) {
        C[a] = poff[a] + (f[a] + 1) / 2;
        sgn[a] = (f[a] % 2 == 1) ? -1 : 1;
    }
    double d0 = p[GI(M, C[0], C[1], C[2])];
    if (scheme == 2) return d0;
    if (scheme == 1) {
        double add = 0.0;
        for (int c = 0; c < (1 << D); c++) {
            int q[3] = {C[0], C[1], C[2]};
            double w = 1.0;
            for (int a = 0; a < D; a++) {
                if ((c >> a) & 1) { q[a] += sgn[a]; w *= 0.25; }
                else w *= 0.75;
            }
            add += w * p[GI(M, q[0], q[1], q[2])];
        }
        return add;
    }
    double dx = p[GI(M, C[0] + sgn[0], C[1], C[2])];
    double dy = p[GI(M, C[0], C[1] + sgn[1], C[2])];
    if (D == 2) return 0.5 * d0 + 0.25 * (dx + dy);
    double dz = p[GI(M, C[0], C[1], C[2] + sgn[2])];
    return 0.25 * (((d0 + dx) + dy) + dz);
}

/* Mesh adaptation with a leaf field carried along (Sec. 2.3: with
 * prolongation and restriction routines given, they are applied when the
 * mesh changes): u_old on the current leaves (canonical order) becomes u_new
 * on the adapted leaves.  A leaf that stays keeps its values; a parent whose
 * children are removed gets their mean (the restriction of Sec. 2.5); the
 * children of a refined leaf are prolonged from it with `scheme` (as
 * ot_set_prolong), its ghosts filled as in the solver (same-level copy, the
 * stored boundary data, the refinement-boundary scheme, and for the
 * bi/trilinear scheme the edge/corner ghosts).  The stored solution is
 * overwritten; the multigrid data is rebuilt afterwards. */
int ot_adapt_transfer(OTree *t, const signed char *flags, int nbuf, int scheme, const double *u_old,
                      double *u_new, int *n_added, int *n_removed) {
    if (scheme < 0 || scheme > 2) return -1;
    int D = t->D, N = t->N, nc = ipow(N, D), ng = ncells_g(D, N);
    if (!t->mg_ready && ot_mg_setup(t) != 0) return -3;
    ot_set_solution(t, u_old);
    for (int l = t->L; l > 1; l--) restrict_level(t, l, 0);
    for (int l = 1; l <= t->L; l++) {
        fill_ghosts(t, l, 0);
        if (scheme == 1) fill_corner_ghosts(t, l, 0);
    }
    int nold = t->nbox, nsub = t->nmg - t->nbox;
    int *olev = malloc(sizeof(int) * (size_t)nold);
    uint64_t *okey = malloc(sizeof(uint64_t) * (size_t)nold);
    double *odata = malloc(sizeof(double) * (size_t)nold * (size_t)ng);
    if (!olev || !okey || !odata) { free(olev); free(okey); free(odata); return -3; }
    for (int b = 0; b < nold; b++) {
        olev[b] = t->box[b].level;
        okey[b] = t->box[b].key;
        memcpy(odata + (size_t)b * ng, t->mg[nsub + b].u, sizeof(double) * (size_t)ng);
    }
    int rc = ot_adapt(t, flags, nbuf, n_added, n_removed);
    if (rc) { free(olev); free(okey); free(odata); return rc; }
    /* old boxes are in canonical order: binary search on (level, key) */
    for (int li = 0; li < t->nleaf; li++) {
        const OBox *nb = &t->box[t->leaf[li]];
        int found = -1, lo = 0, hi = nold - 1;
        while (lo <= hi) {
            int mid = (lo + hi) / 2;
            if (olev[mid] == nb->level && okey[mid] == nb->key) { found = mid; break; }
            if (olev[mid] < nb->level || (olev[mid] == nb->level && okey[mid] < nb->key)) lo = mid + 1;
            else hi = mid - 1;
        }
        double *out = u_new + (long long)li * nc;
        if (found >= 0) {  /* a leaf that stays, or a parent that became a leaf (restricted values) */
            for (int c = 0; c < nc; c++) out[c] = odata[(size_t)found * ng + interior_index(D, N, c)];
            continue;
        }
        /* a new child of a refined leaf */
        int pidx[3] = {1, 1, 1}, poff[3] = {0, 0, 0};
        for (int a = 0; a < D; a++) {
            pidx[a] = (nb->idx[a] + 1) / 2;
            poff[a] = ((nb->idx[a] - 1) & 1) * (N / 2);
        }
        uint64_t pkey = morton_key(D, pidx);
        int par = -1;
        lo = 0; hi = nold - 1;
        while (lo <= hi) {
            int mid = (lo + hi) / 2;
            if (olev[mid] == nb->level - 1 && okey[mid] == pkey) { par = mid; break; }
            if (olev[mid] < nb->level - 1 || (olev[mid] == nb->level - 1 && okey[mid] < pkey)) lo = mid + 1;
            else hi = mid - 1;
        }
        if (par < 0) { free(olev); free(okey); free(odata); return -4; }
        for (int c = 0; c < nc; c++) {
            int f[3] = {c % N + 1, (c / N) % N + 1, D == 3 ? c / (N * N) + 1 : 0};
            out[c] = prolong_value(D, N, odata + (size_t)par * ng, poff, f, scheme);
        }
    }
    free(olev); free(okey); free(odata);
    return 0;
}

/* Prolongation of the coarse-grid correction (Sec. 2.5 lists these schemes;
 * Sec. 4.1 notes that a higher order one lowers the convergence factor):
 * 0 linear with weights (1/2,1/4,1/4) / (1/4,1/4,1/4,1/4) (the default),
 * 1 bilinear / trilinear (it reads edge and corner ghosts of the coarse
 * difference), 2 zeroth order (the coarse value). */
int ot_set_prolong(OTree *t, int scheme) {
    if (scheme < 0 || scheme > 2) return -1;
    t->prolong = scheme;
    return 0;
}

/* Operator of the tree (Sec. 3.5): 0 the Laplacian, 1 div(eps grad u) with
 * harmonic-mean face coefficients, 2 the same in (r,z) coordinates (2D only;
 * r = x, the -x side of the domain is the axis r = 0).  Reading: eps is given
 * per leaf cell (ot_set_eps, after ot_set_operator); coarse cells take the
 * mean of their children (the restriction of Sec. 2.5; in (r,z) every
 * restriction is the mean weighted by the children's volumes, r at their
 * centres -- with the plain mean the (r,z) cycles stall), which keeps the
 * value when, as Sec. 3.4 requires, eps jumps only at faces of the coarsest
 * cells; ghost values are
 * copied from the same-level neighbour, taken from the coarse cell across a
 * refinement boundary, and mirrored at the domain boundary (a boundary face
 * takes its cell's coefficient).  Neumann data stays the normal derivative
 * of u, so the boundary flux is eps b. */
int ot_set_operator(OTree *t, int op) {
    if (op < 0 || op > 2 || (op == 2 && t->D != 2)) return -1;
    if (op && t->singular) return -1;  /* singular problems: the Laplacian only */
    t->op = op;
    return 0;
}

int ot_set_eps(OTree *t, const double *eps) {
    if (!t->mg_ready) return -1;
    int D = t->D, nc = ipow(t->N, D);
    for (int li = 0; li < t->nleaf; li++) {
        OMG *m = leaf_mg(t, li);
        for (int c = 0; c < nc; c++) {
            double e = eps[(long long)li * nc + c];
            if (!(e > 0.0)) return -1;
            m->eps[interior_index(D, m->M, c)] = e;
        }
    }
    for (int l = t->L; l > t->lmin; l--) restrict_level(t, l, 2);
    for (int l = t->lmin; l <= t->L; l++) fill_ghosts(t, l, 2);
    return 0;
}

/* Boundary type of each domain side (Sec. 2 lists Dirichlet, Neumann and
 * periodic conditions, given through ghost cells; Sec. 3 allows a mix).
 * Reading: Neumann data b is the outward normal derivative at the face
 * centre, and the ghost g = u_1 + h b makes the face flux (g - u_1)/h equal
 * to b.  Periodic (Sec. 2.2: the neighbour beyond the last box is the first)
 * applies to both sides of an axis; it changes the connectivity, so it can
 * only be switched on or off while the tree is its root boxes alone.  A tree
 * with no Dirichlet side is singular (make_compatible). */
int ot_set_bc_types(OTree *t, const int *types) {
    int any_dirichlet = 0, change = 0;
    for (int s = 0; s < 2 * t->D; s++) {
        if (types[s] < 0 || types[s] > 2) return -1;
        if ((types[s] == 2) != (types[s ^ 1] == 2)) return -1;
        any_dirichlet |= types[s] == 0;
        change |= (types[s] == 2) != (t->bct[s] == 2);
    }
    if (change && t->nbox != t->nr[0] * t->nr[1] * t->nr[2]) return -1;
    if (!any_dirichlet && t->op) return -1;
    for (int s = 0; s < 2 * t->D; s++) t->bct[s] = types[s];
    t->singular = !any_dirichlet;
    if (change) return rebuild_roots(t);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Composite operator as explicit rows: for leaf cell i the list of        */
/* (leaf cell j, coefficient) with (A u)_i = sum_j K_ij u_j + boundary     */
/* terms.  It restates the same ghost rules cell by cell, which gives the  */
/* transpose used by the adjoint.  Returns the number of entries; with     */
/* rows == NULL only counts.                                               */
/* ---------------------------------------------------------------------- */

static long long leaf_cell_id(OTree *t, int *leafpos, int mgb, int i, int j, int k) {
    OMG *m = &t->mg[mgb];
    int M = m->M;
    long long li = leafpos[m->tbox];
    return li * ipow(M, t->D) + ((long long)(t->D == 3 ? k - 1 : 0) * M + (j - 1)) * M + (i - 1);
}

long long ot_leaf_rows(OTree *t, int *row, int *col, double *val) {
    if (t->op != 0) return -1;  /* the rows restate the Laplacian's ghost rules only */
    int D = t->D, N = t->N, nc = ipow(N, D), nsub = t->nmg - t->nbox;
    int *leafpos = malloc(sizeof(int) * (size_t)t->nbox);
    for (int i = 0; i < t->nbox; i++) leafpos[i] = -1;
    for (int li = 0; li < t->nleaf; li++) leafpos[t->leaf[li]] = li;
    long long n = 0;
#define PUT(R, C, V) do { if (row) { row[n] = (int)(R); col[n] = (int)(C); val[n] = (V); } n++; } while (0)
    for (int li = 0; li < t->nleaf; li++) {
        int mb = nsub + t->leaf[li];
        OMG *m = &t->mg[mb];
        double ih2 = 1.0 / (m->h * m->h);
        for (int c = 0; c < nc; c++) {
            int p[3] = {c % N + 1, (c / N) % N + 1, D == 3 ? c / (N * N) + 1 : 0};
            long long me = (long long)li * nc + c;
            PUT(me, me, -2.0 * D * ih2);
            for (int s = 0; s < 2 * D; s++) {
                int a = s / 2, q[3];
                memcpy(q, p, sizeof q);
                q[a] += (s % 2) ? 1 : -1;
                if (q[a] >= 1 && q[a] <= N) { PUT(me, leaf_cell_id(t, leafpos, mb, q[0], q[1], q[2]), ih2); continue; }
                if (m->kind[s] == K_PHYS) { PUT(me, me, t->bct[s] == 1 ? ih2 : -ih2); continue; }
                if (m->kind[s] == K_SAME) {
                    OMG *nbm = &t->mg[m->nbid[s]];
                    int qq[3]; memcpy(qq, q, sizeof qq);
                    qq[a] = (s % 2) ? 1 : N;
                    if (!nbm->refined) { PUT(me, leaf_cell_id(t, leafpos, m->nbid[s], qq[0], qq[1], qq[2]), ih2); continue; }
                    /* refined same-level box: mean of the 2^D fine cells under that cell */
                    const OBox *nb = &t->box[nbm->tbox];
                    for (int cc = 0; cc < (1 << D); cc++) {
                        int fine[3] = {0, 0, 0}, cidx = 0;
                        for (int e = 0; e < D; e++) {
                            int fg = 2 * ((nb->idx[e] - 1) * N + qq[e] - 1) + ((cc >> e) & 1); /* 0-based global fine */
                            int bi = fg / N; fine[e] = fg % N + 1;
                            cidx |= (bi - 2 * (nb->idx[e] - 1)) << e;
                        }
                        int fb = nsub + nb->child[cidx];
                        PUT(me, leaf_cell_id(t, leafpos, fb, fine[0], fine[1], D == 3 ? fine[2] : 0), ih2 / (double)(1 << D));
                    }
                    continue;
                }
                /* coarse-fine: g = u_H/2 + c1 u_1 - (u_2 + sum u_t)/4 */
                OMG *q2 = &t->mg[m->nbid[s]];
                int t1, t2;
                tang_axes(D, s, &t1, &t2);
                int pc[3] = {0, 0, 0};
                pc[a] = (s % 2 == 0) ? q2->M : 1;
                pc[t1] = m->poff[t1] + (p[t1] - 1) / 2 + 1;
                if (t2 >= 0) pc[t2] = m->poff[t2] + (p[t2] - 1) / 2 + 1;
                PUT(me, leaf_cell_id(t, leafpos, m->nbid[s], pc[0], pc[1], pc[2]), 0.5 * ih2);
                PUT(me, me, (D == 2 ? 1.0 : 1.25) * ih2);
                int p2[3]; memcpy(p2, p, sizeof p2);
                p2[a] += (s % 2) ? -1 : 1;
                PUT(me, leaf_cell_id(t, leafpos, mb, p2[0], p2[1], p2[2]), -0.25 * ih2);
                int pt[3]; memcpy(pt, p, sizeof pt);
                pt[t1] = (p[t1] % 2 == 1) ? p[t1] + 1 : p[t1] - 1;
                PUT(me, leaf_cell_id(t, leafpos, mb, pt[0], pt[1], pt[2]), -0.25 * ih2);
                if (D == 3) {
                    int pu[3]; memcpy(pu, p, sizeof pu);
                    pu[t2] = (p[t2] % 2 == 1) ? p[t2] + 1 : p[t2] - 1;
                    PUT(me, leaf_cell_id(t, leafpos, mb, pu[0], pu[1], pu[2]), -0.25 * ih2);
                }
            }
        }
    }
#undef PUT
    free(leafpos);
    return n;
}

/* Ghosted copy of a multigrid box's variable (0 u, 1 rho, 2 vold, 3 r, 4 d), for tests. */
int ot_mg_nbox(const OTree *t) { return t->nmg; }
int ot_mg_lmin(const OTree *t) { return t->lmin; }
void ot_mg_box_info(const OTree *t, int b, int *info) {
    const OMG *m = &t->mg[b];
    info[0] = m->level; info[1] = m->M; info[2] = m->tbox; info[3] = m->parent; info[4] = m->refined;
    for (int s = 0; s < 6; s++) { info[5 + s] = m->kind[s]; info[11 + s] = m->nbid[s]; }
    for (int a = 0; a < 3; a++) info[17 + a] = m->poff[a];
}
void ot_mg_get(const OTree *t, int b, int var, double *out) {
    const OMG *m = &t->mg[b];
    const double *v = var == 0 ? m->u : var == 1 ? m->rho : var == 2 ? m->vold : var == 3 ? m->r : m->d;
    memcpy(out, v, sizeof(double) * (size_t)ncells_g(t->D, m->M));
}
void ot_mg_set(OTree *t, int b, int var, const double *in) {
    OMG *m = &t->mg[b];
    double *v = var == 0 ? m->u : var == 1 ? m->rho : var == 2 ? m->vold : var == 3 ? m->r : m->d;
    memcpy(v, in, sizeof(double) * (size_t)ncells_g(t->D, m->M));
}
void ot_fill_ghosts(OTree *t, int level, int which) { fill_ghosts(t, level, which); }
void ot_fill_corner_ghosts(OTree *t, int level, int which) { fill_corner_ghosts(t, level, which); }
void ot_smooth(OTree *t, int level, int n) { smooth(t, level, n); }
void ot_gsrb_half(OTree *t, int level, int colour) { gsrb_half(t, level, colour); }
void ot_restrict(OTree *t, int level, int which) { restrict_level(t, level, which); }
void ot_correct(OTree *t, int level) { correct_level(t, level); }
