// The bottom of the multigrid hierarchy in one launch: levels 1 (the root
// box) and below (boxes of N/2, ..., 2 cells; arXiv:1701.04329 Sec. 3.2)
// hold exactly one box per tree, and all their sides are domain boundaries.
// One CTA per tree stages those boxes in shared memory (solution and copy v'
// with a ghost layer, source term, Dirichlet face data) and runs the part of
// the FAS V-cycle below the root -- red-black Gauss-Seidel (Sec. 3.1),
// residual and averaging restriction, the coarse right-hand side
// (Eq. coarse-rhs), the 2-1-1 / 1-1-1-1 correction (Eq. coarse-corr) --
// with block barriers between the steps, then writes the boxes back.  The
// arithmetic is that of the per-level kernels, step for step.
//
// mode 0: one V-cycle from level ltop (<= 1) down to the coarsest grid and
//         back up to ltop.
// mode 1: the FMG steps l = lmin..1: store v'_l, correct from l-1 (l > lmin),
//         V-cycle from l.
#pragma once
#include <type_traits>

#include "kernels.cuh"

namespace afg {

struct BottomLevel {
    int M, cells, padded, faces;  // faces = 2D * M^(D-1)
    int ou, ov, orho, obc;        // shared-memory offsets (elements)
};

// 0-based red-black storage index for a runtime box size
__device__ __forceinline__ int rbi_rt(int D, int M, int i, int j, int k) {
    const int H = (D == 2 ? M * M : M * M * M) / 2;
    return ((i + j + k + D) & 1) * H + (k * M + j) * (M / 2) + (i >> 1);
}

template <int D>
__device__ __forceinline__ int pad_idx(int M, int i, int j, int k) {  // i,j,k in [-1, M]
    return D == 2 ? (j + 1) * (M + 2) + (i + 1) : ((k + 1) * (M + 2) + (j + 1)) * (M + 2) + (i + 1);
}

template <int D>
__device__ __forceinline__ void cell_of(int M, int c, int &i, int &j, int &k) {
    i = c % M;
    j = (c / M) % M;
    k = D == 3 ? c / (M * M) : 0;
}

// c-th cell of colour col (c < M^D / 2), box size known at compile time
template <int D, int M>
__device__ __forceinline__ void bt_cell(int c, int col, int &i, int &j, int &k) {
    constexpr int MH = M / 2;
    const int h = c % MH, row = c / MH;
    j = row % M;
    k = D == 3 ? row / M : 0;
    i = 2 * h + ((col + j + k + D) & 1);
}

// Every side of a bottom box is a domain boundary, so a neighbour outside
// the box is the ghost whose inner cell u_1 is the cell itself: Dirichlet
// g = 2b - u_1, Neumann (bit s of nm) g = u_1 + h b with h = 1/M (a bottom
// box spans the domain); b = 0 for homogeneous data.  Face data: side s,
// face cell t2 * M + t1 with (t1, t2) the tangential coordinates, x first.
template <int D, int M, typename T, bool BC>
__device__ __forceinline__ T bt_ghost(const T *bc, bool zero_b, int nm, int s, int t1, int t2, T self) {
    constexpr int F = D == 2 ? M : M * M;
    const T b = zero_b ? T(0) : bc[s * F + t2 * M + t1];
    // g = a b + c u_1: (2, -1) Dirichlet, (h, 1) Neumann (2b and -u_1 are exact)
    const bool neu = BC && ((nm >> s) & 1);
    return fma(neu ? T(1) / T(M) : T(2), b, neu ? self : -self);
}

// ((x- + x+) + (y- + y+)) + (z- + z+) around interior cell (i,j,k), ghosts
// folded in; on a periodic axis (bit a of pm) the box is its own neighbour,
// so the value across the side is the cell at the other end of the row
template <int D, int M, typename T, bool BC>
__device__ __forceinline__ T bt_sum(const T *v, const T *bc, bool zero_b, int nm, int pm, int i, int j, int k,
                                    T self) {
    const T xm = i > 0 ? v[pad_idx<D>(M, i - 1, j, k)]
                       : (BC && (pm & 1)) ? v[pad_idx<D>(M, M - 1, j, k)] : bt_ghost<D, M, T, BC>(bc, zero_b, nm, 0, j, k, self);
    const T xp = i < M - 1 ? v[pad_idx<D>(M, i + 1, j, k)]
                           : (BC && (pm & 1)) ? v[pad_idx<D>(M, 0, j, k)] : bt_ghost<D, M, T, BC>(bc, zero_b, nm, 1, j, k, self);
    const T ym = j > 0 ? v[pad_idx<D>(M, i, j - 1, k)]
                       : (BC && (pm & 2)) ? v[pad_idx<D>(M, i, M - 1, k)] : bt_ghost<D, M, T, BC>(bc, zero_b, nm, 2, i, k, self);
    const T yp = j < M - 1 ? v[pad_idx<D>(M, i, j + 1, k)]
                           : (BC && (pm & 2)) ? v[pad_idx<D>(M, i, 0, k)] : bt_ghost<D, M, T, BC>(bc, zero_b, nm, 3, i, k, self);
    T s = (xm + xp) + (ym + yp);
    if (D == 3) {
        const T zm = k > 0 ? v[pad_idx<D>(M, i, j, k - 1)]
                           : (BC && (pm & 4)) ? v[pad_idx<D>(M, i, j, M - 1)] : bt_ghost<D, M, T, BC>(bc, zero_b, nm, 4, i, j, self);
        const T zp = k < M - 1 ? v[pad_idx<D>(M, i, j, k + 1)]
                               : (BC && (pm & 4)) ? v[pad_idx<D>(M, i, j, 0)] : bt_ghost<D, M, T, BC>(bc, zero_b, nm, 5, i, j, self);
        s += zm + zp;
    }
    return s;
}

// one barrier per half-sweep: the colour-c cells read only colour 1-c cells
// and their own ghosts
template <int D, int M, typename T, bool BC>
__device__ void bt_smooth(const BottomLevel &L, T *sm, int steps, int hom, int nm, int pm) {
    constexpr int H = (D == 2 ? M * M : M * M * M) / 2;
    T *u = sm + L.ou;
    const T *rho = sm + L.orho, *bc = sm + L.obc;
    const T h2 = T(1) / (T(M) * T(M)), inv = T(1) / T(2 * D);
    for (int it = 0; it < steps; ++it)
        for (int col = 0; col < 2; ++col) {
            for (int c = threadIdx.x; c < H; c += blockDim.x) {
                int i, j, k;
                bt_cell<D, M>(c, col, i, j, k);
                const int p = pad_idx<D>(M, i, j, k);
                const T sum = bt_sum<D, M, T, BC>(u, bc, hom, nm, pm, i, j, k, u[p]);
                u[p] = (sum - h2 * rho[(k * M + j) * M + i]) * inv;
            }
            __syncthreads();
        }
}

// residual of level L (box size M), restricted into the coarse level C (M/2,
// same domain), then the coarse right-hand side
template <int D, int M, typename T, bool BC>
__device__ void bt_down(const BottomLevel &L, const BottomLevel &C, T *sm, int hom, int nm, int pm) {
    constexpr int MC = M / 2, CC = D == 2 ? MC * MC : MC * MC * MC;
    const T *u = sm + L.ou, *bcf = sm + L.obc;
    const T *rho = sm + L.orho;
    T *uc = sm + C.ou, *vc = sm + C.ov, *rc = sm + C.orho;
    const T ih2 = T(M) * T(M), ihc2 = T(MC) * T(MC), w = T(1) / T(1 << D);
    for (int c = threadIdx.x; c < CC; c += blockDim.x) {
        int X, Y, Z;
        cell_of<D>(MC, c, X, Y, Z);
        T su = T(0), sro = T(0), sout = T(0);
        for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int i = 2 * X + dx, j = 2 * Y + dy, k = D == 3 ? 2 * Z + dz : 0;
                    const T uu = u[pad_idx<D>(M, i, j, k)];
                    su += uu;
                    sro += rho[(k * M + j) * M + i];
                    const int io = i + (dx ? 1 : -1), jo = j + (dy ? 1 : -1), ko = k + (dz ? 1 : -1);
                    const int iw = (io + M) % M, jw = (jo + M) % M, kw = (ko + M) % M;  // periodic wrap
                    sout += (io >= 0 && io < M) ? u[pad_idx<D>(M, io, j, k)]
                            : (BC && (pm & 1)) ? u[pad_idx<D>(M, iw, j, k)] : bt_ghost<D, M, T, BC>(bcf, hom, nm, dx, j, k, uu);
                    sout += (jo >= 0 && jo < M) ? u[pad_idx<D>(M, i, jo, k)]
                            : (BC && (pm & 2)) ? u[pad_idx<D>(M, i, jw, k)] : bt_ghost<D, M, T, BC>(bcf, hom, nm, 2 + dy, i, k, uu);
                    if (D == 3)
                        sout += (ko >= 0 && ko < M) ? u[pad_idx<D>(M, i, j, ko)]
                                : (BC && (pm & 4)) ? u[pad_idx<D>(M, i, j, kw)] : bt_ghost<D, M, T, BC>(bcf, hom, nm, 4 + dz, i, j, uu);
                }
        const T mu = su * w;
        uc[pad_idx<D>(MC, X, Y, Z)] = mu;
        vc[pad_idx<D>(MC, X, Y, Z)] = mu;
        rc[c] = fma(-ih2, fma(T(-D), su, sout), sro) * w;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < CC; c += blockDim.x) {
        int i, j, k;
        cell_of<D>(MC, c, i, j, k);
        const T uu = uc[pad_idx<D>(MC, i, j, k)];
        rc[c] = fma(ihc2, fma(T(-2 * D), uu, bt_sum<D, MC, T, BC>(uc, sm + C.obc, hom, nm, pm, i, j, k, uu)), rc[c]);
    }
    __syncthreads();
}

// u_L += I (u_C - v'_C), 2-1-1 (2D) / 1-1-1-1 (3D); outside the box the
// difference is the homogeneous ghost of the cell inside: -d across a
// Dirichlet side, d across a Neumann side; across a periodic side it is the
// difference at the other end of the row.
// dc: scratch for the difference (padded, coarse size)
template <int D, int M, typename T, bool BC>
__device__ void bt_correct(const BottomLevel &L, const BottomLevel &C, T *sm, T *dc, int nm, int pm) {
    constexpr int MC = M / 2, CC = D == 2 ? MC * MC : MC * MC * MC, CL = D == 2 ? M * M : M * M * M;
    T *u = sm + L.ou;
    const T *uc = sm + C.ou, *vc = sm + C.ov;
    for (int c = threadIdx.x; c < CC; c += blockDim.x) {
        int i, j, k;
        cell_of<D>(MC, c, i, j, k);
        const int p = pad_idx<D>(MC, i, j, k);
        dc[p] = uc[p] - vc[p];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < CL; c += blockDim.x) {
        int i, j, k;
        cell_of<D>(M, c, i, j, k);
        const int X = i >> 1, Y = j >> 1, Z = k >> 1;
        const int xs = X + ((i & 1) ? 1 : -1), ys = Y + ((j & 1) ? 1 : -1), zs = Z + ((k & 1) ? 1 : -1);
        const T d0 = dc[pad_idx<D>(MC, X, Y, Z)];
        auto outside = [&](int s) { return (BC && ((nm >> s) & 1)) ? d0 : -d0; };
        const T dx = (xs >= 0 && xs < MC) ? dc[pad_idx<D>(MC, xs, Y, Z)]
                     : (BC && (pm & 1)) ? dc[pad_idx<D>(MC, (xs + MC) % MC, Y, Z)] : outside(xs < 0 ? 0 : 1);
        const T dy = (ys >= 0 && ys < MC) ? dc[pad_idx<D>(MC, X, ys, Z)]
                     : (BC && (pm & 2)) ? dc[pad_idx<D>(MC, X, (ys + MC) % MC, Z)] : outside(ys < 0 ? 2 : 3);
        const int q = pad_idx<D>(M, i, j, k);
        if (D == 2) {
            u[q] = fma(T(0.25), dx + dy, fma(T(0.5), d0, u[q]));
        } else {
            const T dz = (zs >= 0 && zs < MC) ? dc[pad_idx<D>(MC, X, Y, zs)]
                         : (BC && (pm & 4)) ? dc[pad_idx<D>(MC, X, Y, (zs + MC) % MC)] : outside(zs < 0 ? 4 : 5);
            u[q] = fma(T(0.25), ((d0 + dx) + dy) + dz, u[q]);
        }
    }
    __syncthreads();
}

// dispatch on the box size of level index li (M = 2 << li)
#define AFG_BT_M(li, CALL)                                  \
    switch (li) {                                           \
        case 0: { constexpr int MB = 2; CALL; break; }      \
        case 1: { constexpr int MB = 4; CALL; break; }      \
        case 2: { constexpr int MB = 8; CALL; break; }      \
        default: { constexpr int MB = 16; CALL; break; }    \
    }

template <int D, typename T, bool BC>
__device__ void bt_vcycle(const BottomLevel *Ls, int lmin, int ltop, T *sm, T *dc, int nd, int nu, int nb, int hom,
                          int nm, int pm) {
    for (int l = ltop; l > lmin; --l) {
        const int li = l - lmin;
        AFG_BT_M(li, (bt_smooth<D, MB, T, BC>(Ls[li], sm, nd, hom, nm, pm)));
        AFG_BT_M(li, (bt_down<D, MB, T, BC>(Ls[li], Ls[li - 1], sm, hom, nm, pm)));
    }
    bt_smooth<D, 2, T, BC>(Ls[0], sm, nb, hom, nm, pm);
    for (int l = lmin + 1; l <= ltop; ++l) {
        const int li = l - lmin;
        AFG_BT_M(li, (bt_correct<D, MB, T, BC>(Ls[li], Ls[li - 1], sm, dc, nm, pm)));
        AFG_BT_M(li, (bt_smooth<D, MB, T, BC>(Ls[li], sm, nu, hom, nm, pm)));
    }
}

constexpr int kBottomMaxLevels = 4;  // box sizes 16, 8, 4, 2

// lvl_b0[li]: first box of level lmin + li (one box per tree, tree order)
template <int D, typename T>
__global__ void __launch_bounds__(kThreads) k_bottom(BoxMeta A, int ntrees, int N, int lmin, int ltop, int mode,
                                                     T *u, T *rho, T *vold, int nd, int nu, int nb, int hom,
                                                     int4 lvl_b0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int t = blockIdx.x;
    BottomLevel Ls[kBottomMaxLevels];
    const int nl = 2 - lmin;
    int off = 0;
    for (int li = 0; li < nl; ++li) {
        BottomLevel &L = Ls[li];
        L.M = 2 << li;
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
    }
    T *dc = sm + off;  // correction scratch: (N/2 + 2)^D values
    const int b0s[4] = {lvl_b0.x, lvl_b0.y, lvl_b0.z, lvl_b0.w};
    pdl_trigger();
    pdl_wait();
    if (A.active && !A.active[t]) return;  // uniform per CTA: no barrier has been passed yet
    const int nm = A.nmask[b0s[nl - 1] + t];  // Neumann sides (the same for every box below the root)
    int pm = 0;  // periodic axes: the root box is its own neighbour there
    for (int a = 0; a < D; ++a) pm |= (A.nb[(b0s[nl - 1] + t) * 2 * D + 2 * a] >= 0) << a;
    // stage
    for (int li = 0; li < nl; ++li) {
        const BottomLevel &L = Ls[li];
        const int b = b0s[li] + t;
        const long long cb = A.coff[b];
        for (int c = threadIdx.x; c < L.cells; c += blockDim.x) {
            int i, j, k;
            cell_of<D>(L.M, c, i, j, k);
            const int q = rbi_rt(D, L.M, i, j, k);
            sm[L.ou + pad_idx<D>(L.M, i, j, k)] = u[cb + q];
            sm[L.ov + pad_idx<D>(L.M, i, j, k)] = vold[cb + q];
            sm[L.orho + c] = rho[cb + q];
        }
        const int F = D == 2 ? L.M : L.M * L.M;
        for (int x = threadIdx.x; x < L.faces; x += blockDim.x) {
            const int s = x / F, f = x % F;
            // face data exists on domain-boundary sides only (a periodic side's offset is a cell offset)
            const bool phys = A.nb[b * 2 * D + s] == -1;
            sm[L.obc + x] = (hom || !phys) ? T(0) : T(A.bc[A.nbase[b * 2 * D + s] + f]);
        }
    }
    __syncthreads();
    auto run = [&](auto bc) {
        constexpr bool BC = decltype(bc)::value;
        if (mode == 0) {
            bt_vcycle<D, T, BC>(Ls, lmin, ltop, sm, dc, nd, nu, nb, hom, nm, pm);
        } else {
            for (int l = lmin; l <= 1; ++l) {
                const BottomLevel &L = Ls[l - lmin];
                for (int c = threadIdx.x; c < L.cells; c += blockDim.x) {
                    int i, j, k;
                    cell_of<D>(L.M, c, i, j, k);
                    const int p = pad_idx<D>(L.M, i, j, k);
                    sm[L.ov + p] = sm[L.ou + p];
                }
                __syncthreads();
                if (l > lmin) {
                    // the FMG correction uses the copy stored at the start of step l-1
                    const int li = l - lmin;
                    AFG_BT_M(li, (bt_correct<D, MB, T, BC>(L, Ls[li - 1], sm, dc, nm, pm)));
                }
                bt_vcycle<D, T, BC>(Ls, lmin, l, sm, dc, nd, nu, nb, hom, nm, pm);
            }
        }
    };
    // all-Dirichlet trees take the plain instance (uniform per CTA)
    if (nm | pm) run(std::true_type{});
    else run(std::false_type{});
    // write back
    for (int li = 0; li < nl; ++li) {
        const BottomLevel &L = Ls[li];
        const int b = b0s[li] + t;
        const long long cb = A.coff[b];
        for (int c = threadIdx.x; c < L.cells; c += blockDim.x) {
            int i, j, k;
            cell_of<D>(L.M, c, i, j, k);
            const int q = rbi_rt(D, L.M, i, j, k);
            u[cb + q] = sm[L.ou + pad_idx<D>(L.M, i, j, k)];
            vold[cb + q] = sm[L.ov + pad_idx<D>(L.M, i, j, k)];
            rho[cb + q] = sm[L.orho + c];
        }
    }
}

template <int D, typename T>
inline size_t bottom_smem(int N) {
    size_t n = 0;
    for (int M = 2; M <= N; M *= 2) {
        const size_t cells = D == 2 ? M * M : M * M * M;
        const size_t padded = D == 2 ? (M + 2) * (M + 2) : (M + 2) * (M + 2) * (M + 2);
        n += 2 * padded + cells + 2 * D * (D == 2 ? M : M * M);
    }
    const size_t h = N / 2 + 2;
    n += D == 2 ? h * h : h * h * h;  // correction scratch
    return n * sizeof(T);
}

}  // namespace afg
