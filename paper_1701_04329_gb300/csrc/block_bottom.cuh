// The levels at and below the root boxes of a tree whose level 1 is a block
// of r_x x r_y (x r_z) root boxes (arXiv:1701.04329 Sec. 2.2; Sec. 3.2: the
// coarse grids then hold several boxes, relaxed together).  Every box of
// those levels exists, so each level is one rectangular grid of r_a M cells
// along axis a (M = N at level 1, N/2, ..., 2 below), which is how these
// functions hold it: one array per field with a ghost layer, cells
// lexicographic with x fastest.
//
// Each function performs one step of the multigrid cycle on such grids with
// the arithmetic of the per-box operators (sums in the order
// ((x- + x+) + (y- + y+)) + (z- + z+), the same ghost rules), for any number
// of threads: a call handles the items tid, tid + nth, ... of its step, and
// the caller separates steps by a barrier (one CTA on the GPU, one thread on
// the host).  Ghost cells: Dirichlet g = 2b - u_1, Neumann g = u_1 + h b (b
// = 0 for homogeneous data and for the correction), periodic sides copy the
// cell at the other end of the row.  Edge and corner ghosts are not filled:
// nothing here reads them.
#pragma once

#ifdef __CUDACC__
#define AFG_BLK_HD __host__ __device__ __forceinline__
#else
#define AFG_BLK_HD inline
#endif

namespace afg {

struct BlkLevel {
    int D;
    int n[3];       // cells per axis (1 along z in 2D)
    int p[3];       // padded extents n + 2 (1 along z in 2D)
    double h;       // cell size
    long long cells, padded;
};

AFG_BLK_HD BlkLevel blk_level(int D, const int *nroot, int M) {
    BlkLevel L;
    L.D = D;
    L.cells = 1;
    L.padded = 1;
    for (int a = 0; a < 3; ++a) {
        L.n[a] = a < D ? nroot[a] * M : 1;
        L.p[a] = a < D ? L.n[a] + 2 : 1;
        L.cells *= L.n[a];
        L.padded *= L.p[a];
    }
    L.h = 1.0 / M;
    return L;
}

// index of (i, j, k), each in [0, n + 1] (k = 0 in 2D)
AFG_BLK_HD long long blk_at(const BlkLevel &L, int i, int j, int k) {
    return ((long long)k * L.p[1] + j) * L.p[0] + i;
}

// c-th interior cell (x fastest) as 1-based (i, j, k); k = 0 in 2D
AFG_BLK_HD void blk_cell(const BlkLevel &L, long long c, int &i, int &j, int &k) {
    i = (int)(c % L.n[0]) + 1;
    j = (int)((c / L.n[0]) % L.n[1]) + 1;
    k = L.D == 3 ? (int)(c / ((long long)L.n[0] * L.n[1])) + 1 : 0;
}

// Where a cell and a face cell of the block live in the per-box storage.
// Box storage is red-black split: the red half (0-based (i + j + k + D)
// even, i.e. 1-based indices summing to an even number), then the black
// half, each ordered (k, j, i >> 1) with i >> 1 fastest.
AFG_BLK_HD int blk_rbi(int D, int M, int i, int j, int k) {  // 0-based within the box
    const int H = (D == 2 ? M * M : M * M * M) / 2;
    return ((i + j + k + D) & 1) * H + (k * M + j) * (M / 2) + (i >> 1);
}

// cell (i, j, k) (1-based, block of boxes of M cells): root index ri +
// nroot0 (rj + nroot1 rk) and the cell's red-black index within that box
AFG_BLK_HD void blk_cell_home(int D, int M, const int *nroot, int i, int j, int k, int &root, int &q) {
    const int ri = (i - 1) / M, rj = (j - 1) / M, rk = D == 3 ? (k - 1) / M : 0;
    root = ri + nroot[0] * (rj + nroot[1] * rk);
    q = blk_rbi(D, M, (i - 1) % M, (j - 1) % M, D == 3 ? (k - 1) % M : 0);
}

// face cell f of side s of the block: root index and the face cell within
// that box's side (tangential axes lower first, lower fastest)
AFG_BLK_HD void blk_face_home(const BlkLevel &L, int M, const int *nroot, int s, int f, int &root, int &lf) {
    int t1, t2;
    const int a = s / 2;
    t1 = a == 0 ? 1 : 0;
    t2 = L.D == 3 ? (a == 2 ? 1 : 2) : -1;
    const int f1 = f % L.n[t1], f2 = f / L.n[t1];
    int r[3] = {0, 0, 0};
    r[a] = (s & 1) ? nroot[a] - 1 : 0;
    r[t1] = f1 / M;
    if (t2 >= 0) r[t2] = f2 / M;
    root = r[0] + nroot[0] * (r[1] + nroot[1] * r[2]);
    lf = (f1 % M) + M * (t2 >= 0 ? f2 % M : 0);
}

template <typename T>
AFG_BLK_HD T blk_nbsum(const BlkLevel &L, const T *v, int i, int j, int k) {
    T s = (v[blk_at(L, i - 1, j, k)] + v[blk_at(L, i + 1, j, k)]) + (v[blk_at(L, i, j - 1, k)] + v[blk_at(L, i, j + 1, k)]);
    if (L.D == 3) s += v[blk_at(L, i, j, k - 1)] + v[blk_at(L, i, j, k + 1)];
    return s;
}

// (sum_nb - 2D v) / h^2 at an interior cell
template <typename T>
AFG_BLK_HD T blk_lap(const BlkLevel &L, const T *v, int i, int j, int k) {
    const T h = T(L.h);
    return (blk_nbsum(L, v, i, j, k) - T(2.0 * L.D) * v[blk_at(L, i, j, k)]) / (h * h);
}

// number of face cells of side s and their tangential axes
AFG_BLK_HD int blk_faces(const BlkLevel &L, int s, int &t1, int &t2) {
    const int a = s / 2;
    t1 = a == 0 ? 1 : 0;
    t2 = L.D == 3 ? (a == 2 ? 1 : 2) : -1;
    return L.n[t1] * (t2 >= 0 ? L.n[t2] : 1);
}

// Side ghosts of v.  bct[s]: 0 Dirichlet, 1 Neumann, 2 periodic; bc[s]: face
// data of side s (face cell f1 + n[t1] f2), unused when zero_b or periodic.
template <typename T>
AFG_BLK_HD void blk_fill_ghosts(const BlkLevel &L, T *v, const T *const *bc, const int *bct, bool zero_b, int tid,
                                int nth) {
    for (int s = 0; s < 2 * L.D; ++s) {
        int t1, t2;
        const int nf = blk_faces(L, s, t1, t2), a = s / 2;
        for (int f = tid; f < nf; f += nth) {
            int q[3] = {0, 0, 0};
            q[t1] = f % L.n[t1] + 1;
            if (t2 >= 0) q[t2] = f / L.n[t1] + 1;
            int g[3] = {q[0], q[1], q[2]}, in[3] = {q[0], q[1], q[2]};
            g[a] = (s & 1) ? L.n[a] + 1 : 0;
            in[a] = (s & 1) ? L.n[a] : 1;
            T &gv = v[blk_at(L, g[0], g[1], g[2])];
            if (bct[s] == 2) {  // the cell at the other end of the row
                int o[3] = {q[0], q[1], q[2]};
                o[a] = (s & 1) ? 1 : L.n[a];
                gv = v[blk_at(L, o[0], o[1], o[2])];
                continue;
            }
            const T u1 = v[blk_at(L, in[0], in[1], in[2])];
            const T b = zero_b ? T(0) : bc[s][f];
            gv = bct[s] == 1 ? u1 + T(L.h) * b : T(2) * b - u1;
        }
    }
}

// red-black half-sweep: cells whose 1-based indices sum to colour's parity
template <typename T>
AFG_BLK_HD void blk_gsrb(const BlkLevel &L, T *u, const T *rho, int colour, int tid, int nth) {
    const T h2 = T(L.h) * T(L.h), inv = T(1) / T(2 * L.D);
    for (long long c = tid; c < L.cells; c += nth) {
        int i, j, k;
        blk_cell(L, c, i, j, k);
        if ((i + j + k) % 2 != colour) continue;
        const long long g = blk_at(L, i, j, k);
        u[g] = (blk_nbsum(L, u, i, j, k) - h2 * rho[g]) * inv;
    }
}

template <typename T>
AFG_BLK_HD void blk_residual(const BlkLevel &L, const T *u, const T *rho, T *r, int tid, int nth) {
    for (long long c = tid; c < L.cells; c += nth) {
        int i, j, k;
        blk_cell(L, c, i, j, k);
        const long long g = blk_at(L, i, j, k);
        r[g] = rho[g] - blk_lap(L, u, i, j, k);
    }
}

// coarse cell = mean of its 2^D children, summed z, y, x outer to inner
template <typename T>
AFG_BLK_HD void blk_restrict(const BlkLevel &F, const BlkLevel &C, const T *vf, T *vc, int tid, int nth) {
    const int D = F.D;
    for (long long c = tid; c < C.cells; c += nth) {
        int I, J, K;
        blk_cell(C, c, I, J, K);
        T s = T(0);
        for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx)
                    s += vf[blk_at(F, 2 * I - 1 + dx, 2 * J - 1 + dy, D == 3 ? 2 * K - 1 + dz : 0)];
        vc[blk_at(C, I, J, K)] = s / T(1 << D);
    }
}

// coarse right-hand side rho = I r + A(u) (Eq. coarse-rhs), ghosts of u filled
template <typename T>
AFG_BLK_HD void blk_fas(const BlkLevel &L, const T *u, const T *rr, T *rho, int tid, int nth) {
    for (long long c = tid; c < L.cells; c += nth) {
        int i, j, k;
        blk_cell(L, c, i, j, k);
        const long long g = blk_at(L, i, j, k);
        rho[g] = rr[g] + blk_lap(L, u, i, j, k);
    }
}

// dst = src over the padded arrays (v' = u, ghosts included)
template <typename T>
AFG_BLK_HD void blk_copy(const BlkLevel &L, T *dst, const T *src, int tid, int nth) {
    for (long long g = tid; g < L.padded; g += nth) dst[g] = src[g];
}

// d = u - v' over the padded arrays
template <typename T>
AFG_BLK_HD void blk_diff(const BlkLevel &L, T *d, const T *u, const T *vold, int tid, int nth) {
    for (long long g = tid; g < L.padded; g += nth) d[g] = u[g] - vold[g];
}

// u_fine += I d_coarse: weights (1/2,1/4,1/4) in 2D, (1/4,1/4,1/4,1/4) in 3D
// over the coarse cell and its neighbours towards the fine cell (Sec. 2.5);
// the coarse difference's ghosts filled
template <typename T>
AFG_BLK_HD void blk_correct(const BlkLevel &F, const BlkLevel &C, T *uf, const T *dc, int tid, int nth) {
    const int D = F.D;
    for (long long c = tid; c < F.cells; c += nth) {
        int f[3];
        blk_cell(F, c, f[0], f[1], f[2]);
        int P[3] = {0, 0, 0}, sg[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            P[a] = (f[a] + 1) / 2;
            sg[a] = (f[a] % 2 == 1) ? -1 : 1;
        }
        const T d0 = dc[blk_at(C, P[0], P[1], P[2])];
        const T dx = dc[blk_at(C, P[0] + sg[0], P[1], P[2])];
        const T dy = dc[blk_at(C, P[0], P[1] + sg[1], P[2])];
        T add;
        if (D == 2) {
            add = T(0.5) * d0 + T(0.25) * (dx + dy);
        } else {
            const T dz = dc[blk_at(C, P[0], P[1], P[2] + sg[2])];
            add = T(0.25) * (((d0 + dx) + dy) + dz);
        }
        uf[blk_at(F, f[0], f[1], f[2])] += add;
    }
}

// face data of the coarse level: each coarse face cell gets the mean of the
// 2^(D-1) fine face cells it covers, added in the fine order (x fastest)
template <typename T>
AFG_BLK_HD void blk_bc_restrict(const BlkLevel &F, const BlkLevel &C, int s, const T *bf, T *bcoarse, int tid,
                                int nth) {
    int t1, t2;
    const int nfc = blk_faces(C, s, t1, t2), D = F.D;
    const T w = T(1) / T(1 << (D - 1));
    for (int f = tid; f < nfc; f += nth) {
        const int p1 = f % C.n[t1], p2 = f / C.n[t1];
        T acc = T(0);
        for (int c2 = 0; c2 < (D == 3 ? 2 : 1); ++c2)
            for (int c1 = 0; c1 < 2; ++c1)
                acc += bf[(2 * p1 + c1) + F.n[t1] * (D == 3 ? 2 * p2 + c2 : 0)] * w;
        bcoarse[f] = acc;
    }
}

}  // namespace afg

// ---- variable coefficients (Sec. 3.4-3.5) ----------------------------------
// op 1: div(eps grad u) with face coefficient 2 e1 e2 / (e1 + e2); op 2: the
// same in (r,z) coordinates (2D, r = x, the -x side is the axis), r-faces
// weighted by r_face / r_cell and every restriction weighted by the
// children's volumes (r at their centres).  eps holds the coefficient with
// its ghosts (mirrored at the domain sides, wrapped on periodic ones).  M is
// the box size of the level: radii are formed from the cell's root box
// origin, as the per-box operators form them.

namespace afg {

// radius (x) of cell i (1-based over the block) and of its two x-faces
AFG_BLK_HD void blk_radii(const BlkLevel &L, int M, int i, double &rc, double &rm, double &rp) {
    const int ri = (i - 1) / M, il = (i - 1) % M + 1;
    const double x0 = (double)ri;
    rc = x0 + (il - 0.5) * L.h;
    rm = x0 + (il - 1) * L.h;
    rp = x0 + il * L.h;
}

template <typename T>
AFG_BLK_HD void blk_face_coef(const BlkLevel &L, int M, int op, const T *eps, int i, int j, int k, T *c) {
    const int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
    const T e0 = eps[blk_at(L, i, j, k)];
    for (int s = 0; s < 2 * L.D; ++s) {
        const T en = eps[blk_at(L, nb[s][0], nb[s][1], nb[s][2])];
        c[s] = T(2) * e0 * en / (e0 + en);
    }
    if (op == 2) {
        double rc, rm, rp;
        blk_radii(L, M, i, rc, rm, rp);
        c[0] *= T(rm / rc);
        c[1] *= T(rp / rc);
    }
}

// sum_s c_s v_s and sum_s c_s over the faces of cell (i,j,k), in side order
template <typename T>
AFG_BLK_HD void blk_wsum(const BlkLevel &L, int M, int op, const T *eps, const T *v, int i, int j, int k, T &sv,
                         T &sc) {
    const int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
    T c[6];
    blk_face_coef(L, M, op, eps, i, j, k, c);
    T a = T(0), b = T(0);
    for (int s = 0; s < 2 * L.D; ++s) {
        a += c[s] * v[blk_at(L, nb[s][0], nb[s][1], nb[s][2])];
        b += c[s];
    }
    sv = a;
    sc = b;
}

// (sum_s c_s (v_s - v)) / h^2, evaluated as (sum c_s v_s - sum c_s v) / h^2
template <typename T>
AFG_BLK_HD T blk_lap_v(const BlkLevel &L, int M, int op, const T *eps, const T *v, int i, int j, int k) {
    T sv, sc;
    blk_wsum(L, M, op, eps, v, i, j, k, sv, sc);
    const T h = T(L.h);
    return (sv - sc * v[blk_at(L, i, j, k)]) / (h * h);
}

// ghosts of the coefficient: mirrored at the domain sides, wrapped on periodic ones
template <typename T>
AFG_BLK_HD void blk_fill_eps_ghosts(const BlkLevel &L, T *eps, const int *bct, int tid, int nth) {
    for (int s = 0; s < 2 * L.D; ++s) {
        int t1, t2;
        const int nf = blk_faces(L, s, t1, t2), a = s / 2;
        for (int f = tid; f < nf; f += nth) {
            int q[3] = {0, 0, 0};
            q[t1] = f % L.n[t1] + 1;
            if (t2 >= 0) q[t2] = f / L.n[t1] + 1;
            int g[3] = {q[0], q[1], q[2]}, o[3] = {q[0], q[1], q[2]};
            g[a] = (s & 1) ? L.n[a] + 1 : 0;
            if (bct[s] == 2) o[a] = (s & 1) ? 1 : L.n[a];
            else o[a] = (s & 1) ? L.n[a] : 1;
            eps[blk_at(L, g[0], g[1], g[2])] = eps[blk_at(L, o[0], o[1], o[2])];
        }
    }
}

// local solve of the variable-coefficient equation: u = (sum c_s u_s - h^2 rho) / sum c_s
template <typename T>
AFG_BLK_HD void blk_gsrb_v(const BlkLevel &L, int M, int op, const T *eps, T *u, const T *rho, int colour, int tid,
                           int nth) {
    const T h2 = T(L.h) * T(L.h);
    for (long long c = tid; c < L.cells; c += nth) {
        int i, j, k;
        blk_cell(L, c, i, j, k);
        if ((i + j + k) % 2 != colour) continue;
        const long long g = blk_at(L, i, j, k);
        T sv, sc;
        blk_wsum(L, M, op, eps, u, i, j, k, sv, sc);
        u[g] = (sv - h2 * rho[g]) / sc;
    }
}

template <typename T>
AFG_BLK_HD void blk_residual_v(const BlkLevel &L, int M, int op, const T *eps, const T *u, const T *rho, T *r, int tid,
                               int nth) {
    for (long long c = tid; c < L.cells; c += nth) {
        int i, j, k;
        blk_cell(L, c, i, j, k);
        const long long g = blk_at(L, i, j, k);
        r[g] = rho[g] - blk_lap_v(L, M, op, eps, u, i, j, k);
    }
}

template <typename T>
AFG_BLK_HD void blk_fas_v(const BlkLevel &L, int M, int op, const T *eps, const T *u, const T *rr, T *rho, int tid,
                          int nth) {
    for (long long c = tid; c < L.cells; c += nth) {
        int i, j, k;
        blk_cell(L, c, i, j, k);
        const long long g = blk_at(L, i, j, k);
        rho[g] = rr[g] + blk_lap_v(L, M, op, eps, u, i, j, k);
    }
}

// restriction: the plain mean (op 0, 1) or, in (r,z), the mean weighted by
// the children's radii, summed y then x (Mf = the fine level's box size)
template <typename T>
AFG_BLK_HD void blk_restrict_v(const BlkLevel &F, const BlkLevel &C, int Mf, int op, const T *vf, T *vc, int tid,
                               int nth) {
    if (op != 2) {
        blk_restrict(F, C, vf, vc, tid, nth);
        return;
    }
    for (long long c = tid; c < C.cells; c += nth) {
        int I, J, K;
        blk_cell(C, c, I, J, K);
        T s = T(0), w = T(0);
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const int fi = 2 * I - 1 + dx;
                double rc, rm, rp;
                blk_radii(F, Mf, fi, rc, rm, rp);
                s += T(rc) * vf[blk_at(F, fi, 2 * J - 1 + dy, 0)];
                w += T(rc);
            }
        vc[blk_at(C, I, J, K)] = s / w;
    }
}

}  // namespace afg
