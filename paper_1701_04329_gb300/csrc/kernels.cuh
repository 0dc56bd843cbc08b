// Per-box multigrid kernels for quadtree/octree grids (sm_103a).
//
// Method: Teunissen & Ebert, arXiv:1701.04329 -- ghost cells (Sec. 2.4,
// 3.3), prolongation/restriction (Sec. 2.5), red-black Gauss-Seidel
// (Sec. 3.1) and the FAS V-cycle / FMG cycle (Sec. 3.2).
//
// Data layout.  Every box holds only its M^D interior cells; no ghost layer
// is stored.  Within a box the cells are split by colour (red = cells whose
// 1-based indices sum to an even number, i.e. (i+j+k+D) even for 0-based
// indices): first the red half, then the black half, each ordered
// (k, j, i>>1) with i>>1 fastest.  A half-sweep therefore streams exactly
// one colour of rho and u.  A group of threads stages one box, plus the side
// ghost values it needs, in a shared-memory tile of (M+2)^D values; ghost
// values are assembled there from the neighbours' faces (same level), from
// the Dirichlet data, or from the coarse neighbour with the paper's
// conservative two-point scheme.  Corner/edge ghosts are never formed: the
// (2D+1)-point operator, that scheme and the 2-1-1 / 1-1-1-1 prolongation
// do not read them.
//
// Box metadata (device, one entry per box, boxes ordered level by level):
//   nb[b*2D+s]   side s (-x,+x,-y,+y,-z,+z): >= 0 same-level box, -1 domain
//                boundary, <= -2 refinement boundary with coarse box -2-nb
//   parent[b]    box holding this box's restriction (-1 at the bottom)
//   poff[b]      offset of this box's region in the parent, 8 bits per axis
//   coff[b]      first cell of the box in every field array
//   bcoff[b*2D+s] first Dirichlet value of side s (domain boundary sides)
//   bflag[b]     bit 0: refined (values are FAS coarse values); bit 1: has a
//                side that is not a same-level neighbour
//   tree[b]      tree of the box (batched forests); active[tree] masks trees
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace afg {

constexpr int kThreads = 256;
constexpr unsigned char BF_REFINED = 1, BF_SPECIAL = 2;

struct BoxMeta {
    const int *nb;
    const int *parent;
    const int *poff;
    const long long *coff;
    const int *bcoff;
    const unsigned char *bflag;
    const int *tree;
    const int *active;  // may be null
    const double *bc;
    const double *hb;   // cell size of every box
};

template <int D, int M>
struct Geo {
    static constexpr int C = D == 2 ? M * M : M * M * M;  // cells
    static constexpr int H = C / 2;                       // cells per colour
    static constexpr int P = M + 2;                       // padded extent
    static constexpr int PC = D == 2 ? P * P : P * P * P; // padded cells
    static constexpr int F = D == 2 ? M : M * M;          // cells per face
    static constexpr int G = (C / 2) < kThreads ? (C / 2) : kThreads;  // threads per box
    static constexpr int BPC = kThreads / G;              // boxes per CTA
};

template <int D, int M>
__device__ __forceinline__ int colour_of(int i, int j, int k) { return (i + j + k + D) & 1; }

// storage index of interior cell (i,j,k) (0-based)
template <int D, int M>
__device__ __forceinline__ int rbi(int i, int j, int k) {
    return colour_of<D, M>(i, j, k) * Geo<D, M>::H + (k * M + j) * (M / 2) + (i >> 1);
}

// storage index -> (i,j,k)
template <int D, int M>
__device__ __forceinline__ void rb_cell(int q, int &i, int &j, int &k) {
    constexpr int H = Geo<D, M>::H;
    const int c = q >= H ? 1 : 0;
    const int r = q - c * H;
    const int hx = r % (M / 2), row = r / (M / 2);
    j = row % M;
    k = D == 2 ? 0 : row / M;
    i = 2 * hx + ((c + j + k + D) & 1);
}

// tile index, i,j,k in [-1, M]
template <int D, int M>
__device__ __forceinline__ int ti(int i, int j, int k) {
    constexpr int P = M + 2;
    return D == 2 ? (j + 1) * P + (i + 1) : ((k + 1) * P + (j + 1)) * P + (i + 1);
}

// position on side s: coordinate `pos` along the normal axis, (t1,t2) tangential
__device__ __forceinline__ void face_pos(int D, int s, int pos, int t1, int t2, int &i, int &j, int &k) {
    const int a = s >> 1;
    if (a == 0) { i = pos; j = t1; k = D == 3 ? t2 : 0; }
    else if (a == 1) { i = t1; j = pos; k = D == 3 ? t2 : 0; }
    else { i = t1; j = t2; k = pos; }
}

__device__ __forceinline__ int unpack_off(int p, int a) { return (p >> (8 * a)) & 0xff; }

// ---------------------------------------------------------------------------
// Ghost assembly.  Phase A (global reads only) stores the same-level ghost,
// the Dirichlet value b (domain boundary) or the coarse value u_H
// (refinement boundary) into the ghost slot; phase B, after a barrier,
// turns the last two into ghost values with the box's own cells:
//   Dirichlet:           g = 2 b - u_1
//   refinement boundary: 2D g = u_H/2 + u_1 - (u_t + u_2)/4
//                        3D g = u_H/2 + 5/4 u_1 - (u_2 + u_t1 + u_t2)/4
// (Sec. 2.4 and the default scheme of Sec. 3.3).  `only` < 0: all side
// ghosts; otherwise only ghosts next to interior cells of colour `only`.
// ---------------------------------------------------------------------------
template <int D, int M, typename T>
__device__ __forceinline__ void ghosts_phase_a(const BoxMeta &A, int b, const T *__restrict__ u, T *tile,
                                               int lt, int nthr, int only, int hom) {
    constexpr int F = Geo<D, M>::F;
    const int nf = only < 0 ? F : F / 2;
    for (int s = 0; s < 2 * D; ++s) {
        const int code = A.nb[b * 2 * D + s];
        const int hi = s & 1, a = s >> 1;
        const int pin = hi ? M - 1 : 0, pg = hi ? M : -1;
        for (int f = lt; f < nf; f += nthr) {
            int t1, t2;
            if (only < 0) { t1 = f % M; t2 = D == 3 ? f / M : 0; }
            else {
                t2 = D == 3 ? f / (M / 2) : 0;
                const int h1 = D == 3 ? f % (M / 2) : f;
                t1 = 2 * h1 + ((only + pin + t2 + D) & 1);
            }
            int i, j, k;
            face_pos(D, s, pg, t1, t2, i, j, k);
            T v;
            if (code >= 0) {
                int mi, mj, mk;
                face_pos(D, s, hi ? 0 : M - 1, t1, t2, mi, mj, mk);
                v = u[A.coff[code] + rbi<D, M>(mi, mj, mk)];
            } else if (code == -1) {
                v = hom ? T(0) : T(A.bc[A.bcoff[b * 2 * D + s] + t2 * M + t1]);
            } else {
                const int cb = -2 - code;
                const int po = A.poff[b];
                int ci, cj, ck;
                int c1 = 0, c2 = 0;
                // tangential axes in increasing order
                const int ta1 = a == 0 ? 1 : 0, ta2 = a == 2 ? 1 : 2;
                c1 = unpack_off(po, ta1) + (t1 >> 1);
                c2 = D == 3 ? unpack_off(po, ta2) + (t2 >> 1) : 0;
                face_pos(D, s, hi ? 0 : M - 1, c1, c2, ci, cj, ck);
                v = u[A.coff[cb] + rbi<D, M>(ci, cj, ck)];
            }
            tile[ti<D, M>(i, j, k)] = v;
        }
    }
}

template <int D, int M, typename T>
__device__ __forceinline__ void ghosts_phase_b(const BoxMeta &A, int b, T *tile, int lt, int nthr, int only) {
    constexpr int F = Geo<D, M>::F;
    const int nf = only < 0 ? F : F / 2;
    for (int s = 0; s < 2 * D; ++s) {
        const int code = A.nb[b * 2 * D + s];
        if (code >= 0) continue;
        const int hi = s & 1;
        const int pin = hi ? M - 1 : 0, pg = hi ? M : -1, p2 = hi ? M - 2 : 1;
        for (int f = lt; f < nf; f += nthr) {
            int t1, t2;
            if (only < 0) { t1 = f % M; t2 = D == 3 ? f / M : 0; }
            else {
                t2 = D == 3 ? f / (M / 2) : 0;
                const int h1 = D == 3 ? f % (M / 2) : f;
                t1 = 2 * h1 + ((only + pin + t2 + D) & 1);
            }
            int i, j, k;
            face_pos(D, s, pg, t1, t2, i, j, k);
            const int gidx = ti<D, M>(i, j, k);
            face_pos(D, s, pin, t1, t2, i, j, k);
            const T u1 = tile[ti<D, M>(i, j, k)];
            if (code == -1) {
                tile[gidx] = T(2) * tile[gidx] - u1;
            } else {
                const T uH = tile[gidx];
                face_pos(D, s, p2, t1, t2, i, j, k);
                const T u2 = tile[ti<D, M>(i, j, k)];
                face_pos(D, s, pin, t1 ^ 1, t2, i, j, k);
                const T ut1 = tile[ti<D, M>(i, j, k)];
                if (D == 2) {
                    tile[gidx] = T(0.5) * uH + u1 - T(0.25) * (ut1 + u2);
                } else {
                    face_pos(D, s, pin, t1, t2 ^ 1, i, j, k);
                    const T ut2 = tile[ti<D, M>(i, j, k)];
                    tile[gidx] = T(0.5) * uH + T(1.25) * u1 - T(0.25) * ((u2 + ut1) + ut2);
                }
            }
        }
    }
}

template <int D, int M, typename T>
__device__ __forceinline__ T nb_sum(const T *tile, int i, int j, int k) {
    T s = (tile[ti<D, M>(i - 1, j, k)] + tile[ti<D, M>(i + 1, j, k)]) +
          (tile[ti<D, M>(i, j - 1, k)] + tile[ti<D, M>(i, j + 1, k)]);
    if (D == 3) s += tile[ti<D, M>(i, j, k - 1)] + tile[ti<D, M>(i, j, k + 1)];
    return s;
}

template <int D, int M>
__device__ __forceinline__ int resolve_box(const BoxMeta &A, int idx, int n, int b0, const int *list) {
    if (idx >= n) return -1;
    const int b = list ? list[idx] : b0 + idx;
    if (A.active && !A.active[A.tree[b]]) return -1;
    return b;
}

// load the full box (both colours) into the tile
template <int D, int M, typename T>
__device__ __forceinline__ void load_box(const T *__restrict__ u, long long cb, T *tile, int lt, int q0, int q1) {
    constexpr int G = Geo<D, M>::G;
    for (int q = q0 + lt; q < q1; q += G) {
        int i, j, k;
        rb_cell<D, M>(q, i, j, k);
        tile[ti<D, M>(i, j, k)] = u[cb + q];
    }
}

// ---------------------------------------------------------------------------
// Red-black Gauss-Seidel half-sweep on every box of a level (Sec. 3.1):
// cells of colour `colour` get u = (sum of the 2D neighbours - h^2 rho)/(2D).
// Cross-box reads touch only cells of the other colour, which this launch
// never writes, so one launch per half-sweep is race free.
// ---------------------------------------------------------------------------
template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_smooth(BoxMeta A, int b0, int n, const int *list, T *u,
                                                     const T *__restrict__ rho, T h2, int colour, int hom) {
    using Gm = Geo<D, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw) + (threadIdx.x / Gm::G) * Gm::PC;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    const T inv = T(1) / T(2 * D);
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int b = resolve_box<D, M>(A, base + g, n, b0, list);
        bool special = false;
        long long cb = 0;
        if (b >= 0) {
            cb = A.coff[b];
            special = A.bflag[b] & BF_SPECIAL;
            const int q0 = special ? 0 : (1 - colour) * Gm::H, q1 = special ? Gm::C : (2 - colour) * Gm::H;
            load_box<D, M, T>(u, cb, tile, lt, q0, q1);
            ghosts_phase_a<D, M, T>(A, b, u, tile, lt, Gm::G, colour, hom);
        }
        __syncthreads();
        if (b >= 0 && special) ghosts_phase_b<D, M, T>(A, b, tile, lt, Gm::G, colour);
        __syncthreads();
        if (b >= 0) {
            for (int q = colour * Gm::H + lt; q < (colour + 1) * Gm::H; q += Gm::G) {
                int i, j, k;
                rb_cell<D, M>(q, i, j, k);
                const T s = nb_sum<D, M, T>(tile, i, j, k);
                u[cb + q] = (s - h2 * rho[cb + q]) * inv;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Fused residual + restriction (Eq. residual, Sec. 2.5): for every box of
// level l, r = rho - A_h(u) on its cells; the parent region receives
// u_H = mean(u), v'_H = u_H and rho_H = mean(r) (the coarse right-hand side
// is completed by k_fas, Eq. coarse-rhs).
// ---------------------------------------------------------------------------
template <int D, int M, int MP, typename T>
__global__ void __launch_bounds__(kThreads) k_resid_restrict(BoxMeta A, int b0, int n, T *u, T *rho, T *vold,
                                                             T ih2, int hom) {
    using Gm = Geo<D, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw) + (threadIdx.x / Gm::G) * Gm::PC;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    constexpr int MH = M / 2;
    constexpr int NCO = D == 2 ? MH * MH : MH * MH * MH;
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int b = resolve_box<D, M>(A, base + g, n, b0, nullptr);
        bool special = false;
        if (b >= 0) {
            special = A.bflag[b] & BF_SPECIAL;
            load_box<D, M, T>(u, A.coff[b], tile, lt, 0, Gm::C);
            ghosts_phase_a<D, M, T>(A, b, u, tile, lt, Gm::G, -1, hom);
        }
        __syncthreads();
        if (b >= 0 && special) ghosts_phase_b<D, M, T>(A, b, tile, lt, Gm::G, -1);
        __syncthreads();
        if (b >= 0) {
            const long long cb = A.coff[b];
            const int p = A.parent[b];
            const long long cp = A.coff[p];
            const int po = A.poff[b];
            for (int c = lt; c < NCO; c += Gm::G) {
                const int I = c % MH, J = (c / MH) % MH, K = D == 3 ? c / (MH * MH) : 0;
                T su = T(0), sr = T(0);
#pragma unroll
                for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) {
                            const int i = 2 * I + dx, j = 2 * J + dy, k = D == 3 ? 2 * K + dz : 0;
                            const T uc = tile[ti<D, M>(i, j, k)];
                            const T lap = (nb_sum<D, M, T>(tile, i, j, k) - T(2 * D) * uc) * ih2;
                            su += uc;
                            sr += rho[cb + rbi<D, M>(i, j, k)] - lap;
                        }
                const T w = T(1) / T(1 << D);
                const int pi = unpack_off(po, 0) + I, pj = unpack_off(po, 1) + J, pk = D == 3 ? unpack_off(po, 2) + K : 0;
                const long long q = cp + rbi<D, MP>(pi, pj, pk);
                const T mu = su * w;
                u[q] = mu;
                vold[q] = mu;
                rho[q] = sr * w;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FAS coarse right-hand side (Eq. coarse-rhs) on the refined boxes of a level
// (rho_H already holds the restricted residual): rho_H += A_H(v_H).  Leaves
// of the level store their copy v' = v.
// ---------------------------------------------------------------------------
template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_fas(BoxMeta A, int b0, int n, const T *u, T *rho, T *vold, T ih2,
                                                  int hom) {
    using Gm = Geo<D, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw) + (threadIdx.x / Gm::G) * Gm::PC;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int b = resolve_box<D, M>(A, base + g, n, b0, nullptr);
        bool refined = false, special = false;
        if (b >= 0) {
            refined = A.bflag[b] & BF_REFINED;
            special = A.bflag[b] & BF_SPECIAL;
            const long long cb = A.coff[b];
            if (refined) {
                load_box<D, M, T>(u, cb, tile, lt, 0, Gm::C);
                ghosts_phase_a<D, M, T>(A, b, u, tile, lt, Gm::G, -1, hom);
            } else {
                for (int q = lt; q < Gm::C; q += Gm::G) vold[cb + q] = u[cb + q];
            }
        }
        __syncthreads();
        if (b >= 0 && refined && special) ghosts_phase_b<D, M, T>(A, b, tile, lt, Gm::G, -1);
        __syncthreads();
        if (b >= 0 && refined) {
            const long long cb = A.coff[b];
            for (int q = lt; q < Gm::C; q += Gm::G) {
                int i, j, k;
                rb_cell<D, M>(q, i, j, k);
                const T uc = tile[ti<D, M>(i, j, k)];
                rho[cb + q] += (nb_sum<D, M, T>(tile, i, j, k) - T(2 * D) * uc) * ih2;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Coarse-grid correction u_h += I_H^h (v_H - v'_H) (Eq. coarse-corr) with the
// 2-1-1 (2D) / 1-1-1-1 (3D) prolongation (Sec. 2.5) on every box of level l.
// The difference is staged for the box's parent region plus one layer;
// outside the parent it comes from the parent's same-level neighbour, or is
// -d at the domain boundary (homogeneous Dirichlet ghost of a correction).
// ---------------------------------------------------------------------------
template <int D, int M, int MP, typename T>
__global__ void __launch_bounds__(kThreads) k_correct(BoxMeta A, int b0, int n, T *u, const T *__restrict__ vold) {
    using Gm = Geo<D, M>;
    constexpr int MH = M / 2, Q = MH + 2;
    constexpr int QC = D == 2 ? Q * Q : Q * Q * Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *dt = reinterpret_cast<T *>(smem_raw) + (threadIdx.x / Gm::G) * QC;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    auto di = [](int x, int y, int z) { return D == 2 ? (y + 1) * Q + (x + 1) : ((z + 1) * Q + (y + 1)) * Q + (x + 1); };
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int b = resolve_box<D, M>(A, base + g, n, b0, nullptr);
        if (b >= 0) {
            const int p = A.parent[b], po = A.poff[b];
            const long long cp = A.coff[p];
            const int o[3] = {unpack_off(po, 0), unpack_off(po, 1), D == 3 ? unpack_off(po, 2) : 0};
            for (int c = lt; c < QC; c += Gm::G) {
                const int x = c % Q - 1, y = (c / Q) % Q - 1, z = D == 3 ? c / (Q * Q) - 1 : 0;
                const int out = (x < 0 || x >= MH) + (y < 0 || y >= MH) + (D == 3 && (z < 0 || z >= MH));
                if (out > 1) continue;  // corners/edges are not used
                int pc[3] = {o[0] + x, o[1] + y, o[2] + z};
                int side = -1;
                for (int a = 0; a < D; ++a) {
                    if (pc[a] < 0) side = 2 * a;
                    else if (pc[a] >= MP) side = 2 * a + 1;
                }
                T d;
                if (side < 0) {
                    const long long q = cp + rbi<D, MP>(pc[0], pc[1], pc[2]);
                    d = u[q] - vold[q];
                } else {
                    const int code = A.nb[p * 2 * D + side];
                    const int a = side >> 1;
                    if (code >= 0) {
                        pc[a] = (side & 1) ? 0 : MP - 1;
                        const long long q = A.coff[code] + rbi<D, MP>(pc[0], pc[1], pc[2]);
                        d = u[q] - vold[q];
                    } else {
                        pc[a] = (side & 1) ? MP - 1 : 0;
                        const long long q = cp + rbi<D, MP>(pc[0], pc[1], pc[2]);
                        d = -(u[q] - vold[q]);
                    }
                }
                dt[di(x, y, z)] = d;
            }
        }
        __syncthreads();
        if (b >= 0) {
            const long long cb = A.coff[b];
            for (int q = lt; q < Gm::C; q += Gm::G) {
                int i, j, k;
                rb_cell<D, M>(q, i, j, k);
                const int X = i >> 1, Y = j >> 1, Z = k >> 1;
                const int sx = (i & 1) ? 1 : -1, sy = (j & 1) ? 1 : -1, sz = (k & 1) ? 1 : -1;
                const T d0 = dt[di(X, Y, Z)], dx = dt[di(X + sx, Y, Z)], dy = dt[di(X, Y + sy, Z)];
                T add;
                if (D == 2) add = T(0.5) * d0 + T(0.25) * (dx + dy);
                else add = T(0.25) * (((d0 + dx) + dy) + dt[di(X, Y, Z + sz)]);
                u[cb + q] += add;
            }
        }
        __syncthreads();
    }
}

// Restriction of u alone (FMG start, composite residual): parent region = mean of the children.
template <int D, int M, int MP, typename T>
__global__ void __launch_bounds__(kThreads) k_restrict_u(BoxMeta A, int b0, int n, T *u) {
    using Gm = Geo<D, M>;
    constexpr int MH = M / 2;
    constexpr int NCO = D == 2 ? MH * MH : MH * MH * MH;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int b = resolve_box<D, M>(A, base + g, n, b0, nullptr);
        if (b < 0) continue;
        const long long cb = A.coff[b], cp = A.coff[A.parent[b]];
        const int po = A.poff[b];
        for (int c = lt; c < NCO; c += Gm::G) {
            const int I = c % MH, J = (c / MH) % MH, K = D == 3 ? c / (MH * MH) : 0;
            T s = T(0);
            for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx)
                        s += u[cb + rbi<D, M>(2 * I + dx, 2 * J + dy, D == 3 ? 2 * K + dz : 0)];
            const int pi = unpack_off(po, 0) + I, pj = unpack_off(po, 1) + J, pk = D == 3 ? unpack_off(po, 2) + K : 0;
            u[cp + rbi<D, MP>(pi, pj, pk)] = s * (T(1) / T(1 << D));
        }
    }
}

// max of a non-negative double through its bit pattern (monotone for x >= 0)
__device__ __forceinline__ void atomic_max_pos(unsigned long long *p, double v) {
    atomicMax(p, static_cast<unsigned long long>(__double_as_longlong(v)));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
// Residual norm on leaf boxes (list): max |rho - A u| and max |rho| per tree,
// warp-shuffle reductions + one atomic per warp.  Optionally stores the
// residual, cast to R, into rout (the mixed-precision defect correction).
// ---------------------------------------------------------------------------
template <int D, int M, typename T, typename R>
__global__ void __launch_bounds__(kThreads) k_leaf_residual(BoxMeta A, const int *list, int n, const T *u,
                                                            const T *__restrict__ rho, int hom,
                                                            unsigned long long *rmax, unsigned long long *pmax,
                                                            R *rout) {
    using Gm = Geo<D, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw) + (threadIdx.x / Gm::G) * Gm::PC;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int b = resolve_box<D, M>(A, base + g, n, 0, list);
        bool special = false;
        if (b >= 0) {
            special = A.bflag[b] & BF_SPECIAL;
            load_box<D, M, T>(u, A.coff[b], tile, lt, 0, Gm::C);
            ghosts_phase_a<D, M, T>(A, b, u, tile, lt, Gm::G, -1, hom);
        }
        __syncthreads();
        if (b >= 0 && special) ghosts_phase_b<D, M, T>(A, b, tile, lt, Gm::G, -1);
        __syncthreads();
        double rm = 0.0, pm = 0.0;
        int tr = 0;
        if (b >= 0) {
            const long long cb = A.coff[b];
            tr = A.tree[b];
            const T ih2 = T(1.0 / (A.hb[b] * A.hb[b]));
            for (int q = lt; q < Gm::C; q += Gm::G) {
                int i, j, k;
                rb_cell<D, M>(q, i, j, k);
                const T uc = tile[ti<D, M>(i, j, k)];
                const T rr = rho[cb + q] - (nb_sum<D, M, T>(tile, i, j, k) - T(2 * D) * uc) * ih2;
                if (rout) rout[cb + q] = R(rr);
                rm = fmax(rm, fabs(double(rr)));
                pm = fmax(pm, fabs(double(rho[cb + q])));
            }
        }
        // groups never straddle a warp boundary unless G >= 32, so a warp holds one tree
        // when G >= 32; for smaller groups reduce per thread
        if (Gm::G >= 32) {
            rm = warp_max(rm);
            pm = warp_max(pm);
            if ((threadIdx.x & 31) == 0 && b >= 0) {
                atomic_max_pos(rmax + tr, rm);
                if (pmax) atomic_max_pos(pmax + tr, pm);
            }
        } else if (b >= 0) {
            atomic_max_pos(rmax + tr, rm);
            if (pmax) atomic_max_pos(pmax + tr, pm);
        }
        __syncthreads();
    }
}

}  // namespace afg
