// The bottom of the multigrid hierarchy in one launch: levels 1 (the root
// box) and below (boxes of N/2, ..., 2 cells; arXiv:1701.04329 Sec. 3.2)
// hold exactly one box per tree, and all their sides are domain boundaries.
// For a tree of one root box, level 2 can run here too: the 2^D children of
// the root always exist together (a box is refined as a whole, Sec. 2.3), so
// level 2 is one grid of 2N cells per side that covers the domain, with no
// refinement boundary.
//
// One CTA per tree stages those grids in shared memory (solution and copy v'
// with a ghost layer, source term, domain face data) and runs the part of the
// FAS V-cycle below them -- red-black Gauss-Seidel (Sec. 3.1), residual and
// averaging restriction, the coarse right-hand side (Eq. coarse-rhs), the
// 2-1-1 / 1-1-1-1 correction (Eq. coarse-corr) -- with block barriers between
// the steps, then writes the grids back.  The arithmetic is that of the
// per-level kernels, step for step.
//
// The grid size M is a run-time value (a power of two, M = 2 << li for level
// index li): one copy of each step serves every level.  The kernel is
// latency bound (a few hundred cells per step, one CTA): with one inlined
// instantiation per grid size most of its time went to instruction fetch, so
// the steps are separate (not inlined) functions, shared by every level.
//
// mode 0: one V-cycle from level ltop down to the coarsest grid and back up
//         to ltop.
// mode 1: the FMG steps l = lmin..ltop: store v'_l, correct from l-1
//         (l > lmin), V-cycle from l.
#pragma once
#include <type_traits>

#include "kernels.cuh"

namespace afg {

constexpr int kBottomMaxLevels = 6;  // grids of 2 .. 64 cells per side
constexpr int kBottomThreads = 512;  // a level-2 grid of 8^3 boxes has 2048 cells per colour

struct BottomLevel {
    int M, lg;                    // M = 1 << lg cells per side
    int cells, padded, faces;     // faces = 2D * M^(D-1)
    int ou, ov, orho, obc;        // shared-memory offsets (elements)
    int b0;                       // first box of the level (tree 0)
    int kids;                     // 0: one box per tree; 1: the 2^D children of the root (one tree)
};

struct BottomArgs {
    int ntrees, N, lmin, ltop, mode, nd, nu, nb, hom;
    int top;                      // highest level held: 1, or 2 (level 2 of a one-root tree)
    int b0[kBottomMaxLevels];     // first box of level lmin + li
};

// 0-based red-black storage index in a box of M cells per side
__device__ __forceinline__ int rbi_rt(int D, int M, int i, int j, int k) {
    const int H = (D == 2 ? M * M : M * M * M) / 2;
    return ((i + j + k + D) & 1) * H + (k * M + j) * (M / 2) + (i >> 1);
}

template <int D>
__device__ __forceinline__ int pad_idx(int M, int i, int j, int k) {  // i,j,k in [-1, M]
    return D == 2 ? (j + 1) * (M + 2) + (i + 1) : ((k + 1) * (M + 2) + (j + 1)) * (M + 2) + (i + 1);
}

// cell c of an M^D grid in lexicographic order (i fastest)
template <int D>
__device__ __forceinline__ void cell_of(int M, int lg, int c, int &i, int &j, int &k) {
    i = c & (M - 1);
    j = (c >> lg) & (M - 1);
    k = D == 3 ? c >> (2 * lg) : 0;
}

// c-th cell of colour col (c < M^D / 2)
template <int D>
__device__ __forceinline__ void bt_cell(int M, int lg, int c, int col, int &i, int &j, int &k) {
    const int h = c & (M / 2 - 1), row = c >> (lg - 1);
    j = row & (M - 1);
    k = D == 3 ? row >> lg : 0;
    i = 2 * h + ((col + j + k + D) & 1);
}

// Every side of a bottom grid is a domain boundary, so a neighbour outside
// the grid is the ghost whose inner cell u_1 is the cell itself: Dirichlet
// g = 2b - u_1, Neumann (bit s of nm) g = u_1 + h b with h = 1/M (the grid
// spans the domain); b = 0 for homogeneous data.  Face data: side s, face
// cell (t2 << lg) + t1 with (t1, t2) the tangential coordinates, x first.
template <int D, typename T, bool BC>
__device__ __forceinline__ T bt_ghost(const T *bc, bool zero_b, int nm, int lg, T hM, int s, int t1, int t2,
                                      T self) {
    const T b = zero_b ? T(0) : bc[((s << (lg * (D - 1))) + (t2 << lg)) + t1];
    // g = a b + c u_1: (2, -1) Dirichlet, (h, 1) Neumann (2b and -u_1 are exact)
    const bool neu = BC && ((nm >> s) & 1);
    return fma(neu ? hM : T(2), b, neu ? self : -self);
}

// ((x- + x+) + (y- + y+)) + (z- + z+) around interior cell (i,j,k), ghosts
// folded in (FP64: the first four terms summed exactly, nb_sum6); on a
// periodic axis (bit a of pm) the grid is its own neighbour, so the value
// across the side is the cell at the other end of the row
template <int D, typename T, bool BC>
__device__ __forceinline__ T bt_sum(const T *v, const T *bc, bool zero_b, int nm, int pm, int M, int lg, T hM,
                                    int i, int j, int k, T self) {
    const T xm = i > 0 ? v[pad_idx<D>(M, i - 1, j, k)]
                       : (BC && (pm & 1)) ? v[pad_idx<D>(M, M - 1, j, k)]
                                          : bt_ghost<D, T, BC>(bc, zero_b, nm, lg, hM, 0, j, k, self);
    const T xp = i < M - 1 ? v[pad_idx<D>(M, i + 1, j, k)]
                           : (BC && (pm & 1)) ? v[pad_idx<D>(M, 0, j, k)]
                                              : bt_ghost<D, T, BC>(bc, zero_b, nm, lg, hM, 1, j, k, self);
    const T ym = j > 0 ? v[pad_idx<D>(M, i, j - 1, k)]
                       : (BC && (pm & 2)) ? v[pad_idx<D>(M, i, M - 1, k)]
                                          : bt_ghost<D, T, BC>(bc, zero_b, nm, lg, hM, 2, i, k, self);
    const T yp = j < M - 1 ? v[pad_idx<D>(M, i, j + 1, k)]
                           : (BC && (pm & 2)) ? v[pad_idx<D>(M, i, 0, k)]
                                              : bt_ghost<D, T, BC>(bc, zero_b, nm, lg, hM, 3, i, k, self);
    T zm = T(0), zp = T(0);
    if (D == 3) {
        zm = k > 0 ? v[pad_idx<D>(M, i, j, k - 1)]
                   : (BC && (pm & 4)) ? v[pad_idx<D>(M, i, j, M - 1)]
                                      : bt_ghost<D, T, BC>(bc, zero_b, nm, lg, hM, 4, i, j, self);
        zp = k < M - 1 ? v[pad_idx<D>(M, i, j, k + 1)]
                       : (BC && (pm & 4)) ? v[pad_idx<D>(M, i, j, 0)]
                                          : bt_ghost<D, T, BC>(bc, zero_b, nm, lg, hM, 5, i, j, self);
    }
    return nb_sum6<D, T>(xm, xp, ym, yp, zm, zp);
}

// one barrier per half-sweep: the colour-c cells read only colour 1-c cells
// and their own ghosts
template <int D, typename T, bool BC>
__device__ __noinline__ void bt_smooth(const BottomLevel &L, T *sm, int steps, int hom, int nm, int pm) {
    const int M = L.M, lg = L.lg, H = L.cells / 2;
    T *u = sm + L.ou;
    const T *rho = sm + L.orho, *bc = sm + L.obc;
    const T hM = T(1) / T(M), h2 = hM * hM, inv = T(1) / T(2 * D);
    for (int it = 0; it < steps; ++it)
        for (int col = 0; col < 2; ++col) {
            for (int c = threadIdx.x; c < H; c += blockDim.x) {
                int i, j, k;
                bt_cell<D>(M, lg, c, col, i, j, k);
                const int p = pad_idx<D>(M, i, j, k);
                const T sum = bt_sum<D, T, BC>(u, bc, hom, nm, pm, M, lg, hM, i, j, k, u[p]);
                u[p] = (sum - h2 * rho[(((k << lg) + j) << lg) + i]) * inv;
            }
            __syncthreads();
        }
}

// residual of level L (M cells per side) restricted into the coarse level C
// (M/2, the same domain), then the coarse right-hand side
template <int D, typename T, bool BC>
__device__ __noinline__ void bt_down(const BottomLevel &L, const BottomLevel &C, T *sm, int hom, int nm,
                                     int pm) {
    const int M = L.M, lg = L.lg, MC = C.M, lgc = C.lg;
    const T *u = sm + L.ou, *bcf = sm + L.obc;
    const T *rho = sm + L.orho;
    T *uc = sm + C.ou, *vc = sm + C.ov, *rc = sm + C.orho;
    const T hM = T(1) / T(M), hMC = T(1) / T(MC);
    const T ih2 = T(M) * T(M), ihc2 = T(MC) * T(MC), w = T(1) / T(1 << D);
    for (int c = threadIdx.x; c < C.cells; c += blockDim.x) {
        int X, Y, Z;
        cell_of<D>(MC, lgc, c, X, Y, Z);
        T su = T(0), sro = T(0), sout = T(0);
        for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int i = 2 * X + dx, j = 2 * Y + dy, k = D == 3 ? 2 * Z + dz : 0;
                    const T uu = u[pad_idx<D>(M, i, j, k)];
                    su += uu;
                    sro += rho[(((k << lg) + j) << lg) + i];
                    const int io = i + (dx ? 1 : -1), jo = j + (dy ? 1 : -1), ko = k + (dz ? 1 : -1);
                    const int iw = io & (M - 1), jw = jo & (M - 1), kw = ko & (M - 1);  // periodic wrap
                    sout += (io >= 0 && io < M) ? u[pad_idx<D>(M, io, j, k)]
                            : (BC && (pm & 1)) ? u[pad_idx<D>(M, iw, j, k)]
                                               : bt_ghost<D, T, BC>(bcf, hom, nm, lg, hM, dx, j, k, uu);
                    sout += (jo >= 0 && jo < M) ? u[pad_idx<D>(M, i, jo, k)]
                            : (BC && (pm & 2)) ? u[pad_idx<D>(M, i, jw, k)]
                                               : bt_ghost<D, T, BC>(bcf, hom, nm, lg, hM, 2 + dy, i, k, uu);
                    if (D == 3)
                        sout += (ko >= 0 && ko < M) ? u[pad_idx<D>(M, i, j, ko)]
                                : (BC && (pm & 4)) ? u[pad_idx<D>(M, i, j, kw)]
                                                   : bt_ghost<D, T, BC>(bcf, hom, nm, lg, hM, 4 + dz, i, j, uu);
                }
        const T mu = su * w;
        uc[pad_idx<D>(MC, X, Y, Z)] = mu;
        vc[pad_idx<D>(MC, X, Y, Z)] = mu;
        rc[c] = fma(-ih2, fma(T(-D), su, sout), sro) * w;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C.cells; c += blockDim.x) {
        int i, j, k;
        cell_of<D>(MC, lgc, c, i, j, k);
        const T uu = uc[pad_idx<D>(MC, i, j, k)];
        rc[c] = fma(ihc2, fma(T(-2 * D), uu, bt_sum<D, T, BC>(uc, sm + C.obc, hom, nm, pm, MC, lgc, hMC, i, j, k, uu)),
                    rc[c]);
    }
    __syncthreads();
}

// u_L += I (u_C - v'_C), 2-1-1 (2D) / 1-1-1-1 (3D); outside the grid the
// difference is the homogeneous ghost of the cell inside: -d across a
// Dirichlet side, d across a Neumann side; across a periodic side it is the
// difference at the other end of the row.
// dc: scratch for the difference (padded, coarse size)
template <int D, typename T, bool BC>
__device__ __noinline__ void bt_correct(const BottomLevel &L, const BottomLevel &C, T *sm, T *dc, int nm,
                                        int pm) {
    const int M = L.M, lg = L.lg, MC = C.M, lgc = C.lg;
    T *u = sm + L.ou;
    const T *uc = sm + C.ou, *vc = sm + C.ov;
    for (int c = threadIdx.x; c < C.cells; c += blockDim.x) {
        int i, j, k;
        cell_of<D>(MC, lgc, c, i, j, k);
        const int p = pad_idx<D>(MC, i, j, k);
        dc[p] = uc[p] - vc[p];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < L.cells; c += blockDim.x) {
        int i, j, k;
        cell_of<D>(M, lg, c, i, j, k);
        const int X = i >> 1, Y = j >> 1, Z = k >> 1;
        const int xs = X + ((i & 1) ? 1 : -1), ys = Y + ((j & 1) ? 1 : -1), zs = Z + ((k & 1) ? 1 : -1);
        const T d0 = dc[pad_idx<D>(MC, X, Y, Z)];
        auto outside = [&](int s) { return (BC && ((nm >> s) & 1)) ? d0 : -d0; };
        const T dx = (xs >= 0 && xs < MC) ? dc[pad_idx<D>(MC, xs, Y, Z)]
                     : (BC && (pm & 1)) ? dc[pad_idx<D>(MC, xs & (MC - 1), Y, Z)] : outside(xs < 0 ? 0 : 1);
        const T dy = (ys >= 0 && ys < MC) ? dc[pad_idx<D>(MC, X, ys, Z)]
                     : (BC && (pm & 2)) ? dc[pad_idx<D>(MC, X, ys & (MC - 1), Z)] : outside(ys < 0 ? 2 : 3);
        const int q = pad_idx<D>(M, i, j, k);
        if (D == 2) {
            u[q] = fma(T(0.25), dx + dy, fma(T(0.5), d0, u[q]));
        } else {
            const T dz = (zs >= 0 && zs < MC) ? dc[pad_idx<D>(MC, X, Y, zs)]
                         : (BC && (pm & 4)) ? dc[pad_idx<D>(MC, X, Y, zs & (MC - 1))] : outside(zs < 0 ? 4 : 5);
            u[q] = fma(T(0.25), ((d0 + dx) + dy) + dz, u[q]);
        }
    }
    __syncthreads();
}

template <int D, typename T, bool BC>
__device__ __noinline__ void bt_vcycle(const BottomLevel *Ls, int lmin, int ltop, T *sm, T *dc, int nd, int nu, int nb,
                                       int hom, int nm, int pm) {
    for (int l = ltop; l > lmin; --l) {
        const int li = l - lmin;
        bt_smooth<D, T, BC>(Ls[li], sm, nd, hom, nm, pm);
        bt_down<D, T, BC>(Ls[li], Ls[li - 1], sm, hom, nm, pm);
    }
    bt_smooth<D, T, BC>(Ls[0], sm, nb, hom, nm, pm);
    for (int l = lmin + 1; l <= ltop; ++l) {
        const int li = l - lmin;
        bt_correct<D, T, BC>(Ls[li], Ls[li - 1], sm, dc, nm, pm);
        bt_smooth<D, T, BC>(Ls[li], sm, nu, hom, nm, pm);
    }
}

// Global location of cell (i, j, k) of a staged grid.  A grid of the 2^D
// children of the root (kids) maps the cell to the child holding it (kb:
// child position (bit a set on the upper half along axis a) -> box) and to
// that box's own N-cell storage.
template <int D>
__device__ __forceinline__ long long bt_gcell(const BoxMeta &A, const BottomLevel &L, const int *kb, int t, int N,
                                              int lgN, int i, int j, int k) {
    if (!L.kids) return A.coff[L.b0 + t] + rbi_rt(D, L.M, i, j, k);
    const int ch = (i >> lgN) | ((j >> lgN) << 1) | (D == 3 ? (k >> lgN) << 2 : 0);
    return A.coff[kb[ch]] + rbi_rt(D, N, i & (N - 1), j & (N - 1), k & (N - 1));
}

// Dirichlet data of face cell x (side s, tangential (t1, t2)) of a staged
// grid, or 0 where there is none (homogeneous data, a periodic side)
template <int D, typename T>
__device__ __forceinline__ T bt_face(const BoxMeta &A, const BottomLevel &L, const int *kb, int t, int N, int lgN,
                                     int hom, int s, int t1, int t2) {
    int b = L.b0 + t, f = (t2 << L.lg) + t1;
    if (L.kids) {
        // the child on side s that holds the face cell: bit s/2 from the side,
        // the tangential bits from (t1, t2)
        const int a = s >> 1;
        const int a1 = a == 0 ? 1 : 0, a2 = a == 2 ? 1 : 2;
        int ch = (s & 1) << a;
        ch |= (t1 >> lgN) << a1;
        if (D == 3) ch |= (t2 >> lgN) << a2;
        b = kb[ch];
        f = ((t2 & (N - 1)) << lgN) + (t1 & (N - 1));
    }
    // face data exists on domain-boundary sides only (a periodic side's offset is a cell offset)
    const bool phys = A.nb[b * 2 * D + s] == -1;
    return (hom || !phys) ? T(0) : T(A.bc[A.nbase[b * 2 * D + s] + f]);
}

template <int D, typename T>
__global__ void __launch_bounds__(kBottomThreads) k_bottom(BoxMeta A, BottomArgs P, T *u, T *rho, T *vold) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int kb[8];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int t = blockIdx.x, N = P.N;
    const int lgN = 31 - __clz(N);
    BottomLevel Ls[kBottomMaxLevels];
    const int nl = P.top + 1 - P.lmin;
    int off = 0;
    for (int li = 0; li < nl; ++li) {
        BottomLevel &L = Ls[li];
        L.lg = li + 1;
        L.M = 1 << L.lg;
        L.cells = D == 2 ? L.M * L.M : L.M * L.M * L.M;
        L.padded = D == 2 ? (L.M + 2) * (L.M + 2) : (L.M + 2) * (L.M + 2) * (L.M + 2);
        L.faces = 2 * D * (D == 2 ? L.M : L.M * L.M);
        L.ou = off;
        off += L.padded;
        L.ov = off;
        off += L.padded;
        L.orho = off;
        off += L.cells;
        L.obc = off;
        off += L.faces;
        L.b0 = P.b0[li];
        L.kids = P.lmin + li == 2;
    }
    T *dc = sm + off;  // correction scratch: (M_top/2 + 2)^D values
    const int root = P.b0[1 - P.lmin] + t;
    pdl_trigger();
    if (P.top == 2 && threadIdx.x < (1 << D)) {  // child position -> box (box metadata: no wait needed)
        const int b = P.b0[2 - P.lmin] + threadIdx.x;
        const int po = A.poff[b];
        int ch = 0;
        for (int a = 0; a < D; ++a) ch |= (unpack_off(po, a) != 0) << a;
        kb[ch] = b;
    }
    pdl_wait();
    if (A.active && !A.active[t]) return;  // uniform per CTA: no barrier has been passed yet
    __syncthreads();
    const int nm = A.nmask[root];  // Neumann sides (the same for every grid below the root)
    int pm = 0;  // periodic axes: the root box is its own neighbour there
    for (int a = 0; a < D; ++a) pm |= (A.nb[root * 2 * D + 2 * a] >= 0) << a;
    // stage
    for (int li = 0; li < nl; ++li) {
        const BottomLevel &L = Ls[li];
        for (int c = threadIdx.x; c < L.cells; c += blockDim.x) {
            int i, j, k;
            cell_of<D>(L.M, L.lg, c, i, j, k);
            const long long g = bt_gcell<D>(A, L, kb, t, N, lgN, i, j, k);
            sm[L.ou + pad_idx<D>(L.M, i, j, k)] = u[g];
            sm[L.ov + pad_idx<D>(L.M, i, j, k)] = vold[g];
            sm[L.orho + c] = rho[g];
        }
        const int lf = L.lg * (D - 1);  // face cells per side: 1 << lf
        for (int x = threadIdx.x; x < L.faces; x += blockDim.x) {
            const int s = x >> lf, f = x & ((1 << lf) - 1);
            sm[L.obc + x] = bt_face<D, T>(A, L, kb, t, N, lgN, P.hom, s, f & (L.M - 1), f >> L.lg);
        }
    }
    __syncthreads();
    auto run = [&](auto bc) {
        constexpr bool BC = decltype(bc)::value;
        if (P.mode == 0) {
            bt_vcycle<D, T, BC>(Ls, P.lmin, P.ltop, sm, dc, P.nd, P.nu, P.nb, P.hom, nm, pm);
        } else {
            for (int l = P.lmin; l <= P.top; ++l) {
                const BottomLevel &L = Ls[l - P.lmin];
                for (int c = threadIdx.x; c < L.cells; c += blockDim.x) {
                    int i, j, k;
                    cell_of<D>(L.M, L.lg, c, i, j, k);
                    const int p = pad_idx<D>(L.M, i, j, k);
                    sm[L.ov + p] = sm[L.ou + p];
                }
                __syncthreads();
                if (l > P.lmin) {
                    // the FMG correction uses the copy stored at the start of step l-1
                    const int li = l - P.lmin;
                    bt_correct<D, T, BC>(L, Ls[li - 1], sm, dc, nm, pm);
                }
                bt_vcycle<D, T, BC>(Ls, P.lmin, l, sm, dc, P.nd, P.nu, P.nb, P.hom, nm, pm);
            }
        }
    };
    // all-Dirichlet trees take the plain instance (uniform per CTA)
    if (nm | pm) run(std::true_type{});
    else run(std::false_type{});
    // write back
    for (int li = 0; li < nl; ++li) {
        const BottomLevel &L = Ls[li];
        for (int c = threadIdx.x; c < L.cells; c += blockDim.x) {
            int i, j, k;
            cell_of<D>(L.M, L.lg, c, i, j, k);
            const long long g = bt_gcell<D>(A, L, kb, t, N, lgN, i, j, k);
            u[g] = sm[L.ou + pad_idx<D>(L.M, i, j, k)];
            vold[g] = sm[L.ov + pad_idx<D>(L.M, i, j, k)];
            rho[g] = sm[L.orho + c];
        }
    }
}

// shared memory of k_bottom for grids of 2 .. top_m cells per side
template <int D, typename T>
inline size_t bottom_smem(int top_m) {
    size_t n = 0;
    for (int M = 2; M <= top_m; M *= 2) {
        const size_t cells = D == 2 ? M * M : M * M * M;
        const size_t padded = D == 2 ? (M + 2) * (M + 2) : (M + 2) * (M + 2) * (M + 2);
        n += 2 * padded + cells + 2 * D * (D == 2 ? M : M * M);
    }
    const size_t h = top_m / 2 + 2;
    n += D == 2 ? h * h : h * h * h;  // correction scratch
    return n * sizeof(T);
}

}  // namespace afg
