// Variable-coefficient operators (arXiv:1701.04329 Sec. 3.4-3.5):
// div(eps grad u) = rho with eps per cell, in Cartesian coordinates (op 1)
// or in 2D (r,z) coordinates with r = x (op 2).
//
// The flux through the face between cells of coefficients e1 and e2 is the
// harmonic mean 2 e1 e2 / (e1 + e2) times the difference quotient (Sec. 3.4:
// the local reconstruction of a jump of eps at the face); in (r,z) the
// r-faces are also weighted by r_face / r_cell, so the face on the axis
// r = 0 carries no flux (Sec. 3.5).  With c_s the coefficient of side s of a
// cell:  h^2 (A u) = sum_s c_s u_s - (sum_s c_s) u, both sums in side order
// -x, +x, -y, +y(, -z, +z), and the red-black local solve is
// u = (sum_s c_s u_s - h^2 rho) / sum_s c_s.
//
// eps lives in the same red-black box layout as u, on every level: leaves
// hold the user's values, parents the restriction of their children (the
// mean; in (r,z) the mean weighted by the children's volumes, proportional
// to r at their centres, which every (r,z) restriction uses).  Its ghost
// values are copied from the same-level neighbour, taken from the coarse
// cell across a refinement boundary, and mirrored at the domain boundary
// (a boundary face takes its cell's coefficient).  The ghost values of u
// follow the Laplacian's rules (Sec. 2.4, 3.3), staged by gather/finalize.
//
// These kernels are table-driven: a thread group stages one box (u and eps
// with all side ghosts, and rho where needed) in shared memory and walks
// the box's cells.
#pragma once
#include "kernels.cuh"

namespace afg {

// per box: u tile, eps tile (ghosts included) and rho in storage order
template <int D, int M, typename T>
struct VarCfg {
    static constexpr int G = Geo<D, M>::G, BPC = Geo<D, M>::BPC;
    static constexpr int PC = Geo<D, M>::PC, C = Geo<D, M>::C;
    static constexpr int BOX = 2 * PC + C;
    static constexpr size_t smem() { return sizeof(T) * BOX * BPC + 2 * sizeof(BoxInfo) * BPC + Tables<D, M>::bytes(); }
};

// eps of the box and its side ghosts into the tile (tables built with only = -1)
template <int D, int M, typename T, int G>
__device__ __forceinline__ void gather_eps(const BoxInfo &I, const T *__restrict__ eps, T *tile, int lt,
                                           const short *tix, const short *gt, const short *gs) {
    constexpr int C = Geo<D, M>::C, F = Geo<D, M>::F;
    for (int q = lt; q < C; q += G) tile[tix[q]] = eps[I.coff + q];
    for (int item = lt; item < 2 * D * F; item += G) {
        const int s = item / F, f = item - s * F;
        const int code = I.code[s];
        T v;
        if (code >= 0) {
            v = eps[I.base[s] + gs[item]];
        } else {
            const int hi = s & 1, a = s >> 1;
            const int t1 = f % M, t2 = D == 3 ? f / M : 0;
            int i, j, k;
            if (code == -1) {  // mirrored: the cell's own coefficient
                face_pos(D, s, hi ? M - 1 : 0, t1, t2, i, j, k);
                v = eps[I.coff + rbi<D, M>(i, j, k)];
            } else {  // the coarse cell across the refinement boundary
                const int ta1 = a == 0 ? 1 : 0, ta2 = a == 2 ? 1 : 2;
                const int c1 = unpack_off(I.poff, ta1) + (t1 >> 1);
                const int c2 = D == 3 ? unpack_off(I.poff, ta2) + (t2 >> 1) : 0;
                face_pos(D, s, hi ? 0 : M - 1, c1, c2, i, j, k);
                v = eps[I.base[s] + rbi<D, M>(i, j, k)];
            }
        }
        tile[gt[item]] = v;
    }
}

// face coefficients c[s] of the cell at tile slot t (0-based x index i) of a
// box with cell size h and lower x coordinate x0
template <int D, int M, typename T>
__device__ __forceinline__ void var_coef(const T *E, int t, int i, T h, T x0, int op, T (&c)[2 * D]) {
    constexpr int P = M + 2;
    const T e0 = E[t];
#pragma unroll
    for (int s = 0; s < 2 * D; ++s) {
        const int o = s == 0 ? -1 : s == 1 ? 1 : s == 2 ? -P : s == 3 ? P : s == 4 ? -P * P : P * P;
        const T en = E[t + o];
        c[s] = T(2) * e0 * en / (e0 + en);
    }
    if (op == 2) {
        const T rc = x0 + (T(i) + T(0.5)) * h;
        c[0] *= (x0 + T(i) * h) / rc;
        c[1] *= (x0 + T(i + 1) * h) / rc;
    }
}

// sum_s c_s u_s and sum_s c_s for the cell at tile slot t, in side order
template <int D, int M, typename T>
__device__ __forceinline__ void var_sums(const T *U, const T *E, int t, int i, T h, T x0, int op, T &sv, T &sc) {
    constexpr int P = M + 2;
    T c[2 * D];
    var_coef<D, M, T>(E, t, i, h, x0, op, c);
    T a = T(0), b = T(0);
#pragma unroll
    for (int s = 0; s < 2 * D; ++s) {
        const int o = s == 0 ? -1 : s == 1 ? 1 : s == 2 ? -P : s == 3 ? P : s == 4 ? -P * P : P * P;
        a += c[s] * U[t + o];
        b += c[s];
    }
    sv = a;
    sc = b;
}

// The box walk shared by the kernels below: per box, u and eps (with
// their side ghosts) and rho (when want_r) are staged, the ghosts of u
// completed, then body(I, U, E, R, lt, tix) runs in the box's thread group
// and post(I, lt) in every thread of the block (I.b < 0: no box).  In a
// half-sweep the staged ghosts next to cells of the colour being updated
// come from cells of the other colour, which the launch does not write; the
// other ghosts are staged too but not read.
template <int D, int M, typename T, typename Body, typename Post>
__device__ __forceinline__ void var_walk(const BoxMeta &A, int b0, int n, const int *list, const T *u,
                                         const T *eps, const T *rho, int hom, bool want_r, Body body, Post post) {
    using S = VarCfg<D, M, T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / S::G, lt = threadIdx.x % S::G;
    T *U = reinterpret_cast<T *>(smem_raw) + g * S::BOX;
    T *E = U + S::PC, *R = E + S::PC;
    BoxInfo *info;
    short *tix, *gt, *gs;
    carve<D, M>(smem_raw, sizeof(T) * S::BOX * S::BPC, S::BPC, info, tix, gt, gs);
    build_tables<D, M>(tix, gt, gs, -1);
    const int stride = gridDim.x * S::BPC;
    int base = blockIdx.x * S::BPC, buf = 0;
    info_load<D>(A, base + g, n, b0, list, info[g], lt, S::G, false);
    pdl_wait();
    info_mask<D>(A, info[g], lt, S::G);
    __syncthreads();
    for (; base < n; base += stride) {
        const BoxInfo &I = info[buf * S::BPC + g];
        const int b = I.b;
        const bool special = b >= 0 && (I.flag & BF_SPECIAL);
        if (b >= 0) {
            gather<D, M, T, S::G>(I, u, A.bc, U, lt, -1, true, hom, tix, gt, gs);
            gather_eps<D, M, T, S::G>(I, eps, E, lt, tix, gt, gs);
            if (want_r)
                for (int q = lt; q < S::C; q += S::G) R[q] = rho[I.coff + q];
        }
        info_load<D>(A, base + stride + g, n, b0, list, info[(buf ^ 1) * S::BPC + g], lt, S::G);
        __syncthreads();
        if (special) finalize<D, M, T, S::G>(I, U, lt, -1, A.hb);
        __syncthreads();
        if (b >= 0) body(I, U, E, R, lt, tix);
        post(I, lt);  // every thread, also without a box
        buf ^= 1;
        __syncthreads();
    }
}

struct VarNoPost {
    __device__ void operator()(const BoxInfo &, int) const {}
};

// Red-black half-sweep of colour `colour` on every box of a level.
template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_var_smooth(BoxMeta A, int b0, int n, T *u, const T *rho,
                                                         const T *eps, int colour, int hom, int op) {
    using S = VarCfg<D, M, T>;
    constexpr int H = Geo<D, M>::H;
    pdl_trigger();
    auto body = [&](const BoxInfo &I, const T *U, const T *E, const T *R, int lt, const short *tix) {
        const T h = T(A.hb[I.b]), x0 = T(A.x0[I.b]), h2 = h * h;
        for (int q = colour * H + lt; q < (colour + 1) * H; q += S::G) {
            int i, j, k;
            rb_cell<D, M>(q, i, j, k);
            T sv, sc;
            var_sums<D, M, T>(U, E, tix[q], i, h, x0, op, sv, sc);
            u[I.coff + q] = (sv - h2 * R[q]) / sc;
        }
    };
    var_walk<D, M, T>(A, b0, n, nullptr, u, eps, rho, hom, true, body, VarNoPost());
}

// weights of the children of a coarse cell in a restriction: 1 (plain mean)
// or, in (r,z), the children's r at their centres
template <typename T>
__device__ __forceinline__ T var_weight(int op, T x0, T h, int ichild) {
    return op == 2 ? x0 + (T(ichild) + T(0.5)) * h : T(1);
}

// Residual and restriction: r = rho - A u on every cell of the level's boxes;
// the parent region receives u_H = I u, v'_H = u_H and rho_H = I r (the FAS
// right-hand side is completed by k_var_fas).  I is the mean of the 2^D
// children, weighted by r in (r,z).
template <int D, int M, int MP, typename T>
__global__ void __launch_bounds__(kThreads) k_var_resid_restrict(BoxMeta A, int b0, int n, T *u, T *rho, T *vold,
                                                                 const T *eps, int hom, int op) {
    using S = VarCfg<D, M, T>;
    constexpr int MH = M / 2, P = M + 2;
    constexpr int NCO = D == 2 ? MH * MH : MH * MH * MH;
    pdl_trigger();
    auto body = [&](const BoxInfo &I, const T *U, const T *E, const T *R, int lt, const short *tix) {
        const T h = T(A.hb[I.b]), x0 = T(A.x0[I.b]), ih2 = T(1) / (h * h);
        const long long cp = A.coff[I.parent];
        for (int c = lt; c < NCO; c += S::G) {
            const int X = c % MH, Y = (c / MH) % MH, Z = D == 3 ? c / (MH * MH) : 0;
            T su = T(0), sr = T(0), sw = T(0);
            for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                        const int i = 2 * X + dx, j = 2 * Y + dy, k = D == 3 ? 2 * Z + dz : 0;
                        const int t = ti<D, M>(i, j, k);
                        T sv, sc;
                        var_sums<D, M, T>(U, E, t, i, h, x0, op, sv, sc);
                        const T r = R[rbi<D, M>(i, j, k)] - (sv - sc * U[t]) * ih2;
                        const T w = var_weight<T>(op, x0, h, i);
                        su += w * U[t];
                        sr += w * r;
                        sw += w;
                    }
            (void)P;
            const int pi = unpack_off(I.poff, 0) + X, pj = unpack_off(I.poff, 1) + Y;
            const int pk = D == 3 ? unpack_off(I.poff, 2) + Z : 0;
            const long long q = cp + rbi<D, MP>(pi, pj, pk);
            const T mu = su / sw;
            u[q] = mu;
            vold[q] = mu;
            rho[q] = sr / sw;
        }
    };
    var_walk<D, M, T>(A, b0, n, nullptr, u, eps, rho, hom, true, body, VarNoPost());
}

// FAS right-hand side on the refined boxes of a level: rho_H += A_H(v_H);
// leaves store v' = v.
template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_var_fas(BoxMeta A, int b0, int n, const T *u, T *rho, T *vold,
                                                      const T *eps, int hom, int op) {
    using S = VarCfg<D, M, T>;
    pdl_trigger();
    auto body = [&](const BoxInfo &I, const T *U, const T *E, const T *R, int lt, const short *tix) {
        if (!(I.flag & BF_REFINED)) {
            for (int q = lt; q < S::C; q += S::G) vold[I.coff + q] = U[tix[q]];
            return;
        }
        const T h = T(A.hb[I.b]), x0 = T(A.x0[I.b]), ih2 = T(1) / (h * h);
        for (int q = lt; q < S::C; q += S::G) {
            int i, j, k;
            rb_cell<D, M>(q, i, j, k);
            const int t = tix[q];
            T sv, sc;
            var_sums<D, M, T>(U, E, t, i, h, x0, op, sv, sc);
            rho[I.coff + q] = R[q] + (sv - sc * U[t]) * ih2;
        }
    };
    var_walk<D, M, T>(A, b0, n, nullptr, u, eps, rho, hom, true, body, VarNoPost());
}

// Composite residual on the leaf boxes of a list: per tree the maxima of |r|
// and |rho| (non-negative doubles reduced as bit patterns), and r (cast to
// R) in rout when it is not null.
template <int D, int M, typename T, typename Ro>
__global__ void __launch_bounds__(kThreads) k_var_leaf_residual(BoxMeta A, const int *list, int n, const T *u,
                                                                const T *rho, const T *eps, int hom, int op,
                                                                unsigned long long *rmax, unsigned long long *pmax,
                                                                Ro *rout) {
    using S = VarCfg<D, M, T>;
    pdl_trigger();
    __shared__ double red[2 * kThreads / 32];
    double rm = 0.0, pm = 0.0;
    auto body = [&](const BoxInfo &I, const T *U, const T *E, const T *R, int lt, const short *tix) {
        const T h = T(A.hb[I.b]), x0 = T(A.x0[I.b]), ih2 = T(1) / (h * h);
        for (int q = lt; q < S::C; q += S::G) {
            int i, j, k;
            rb_cell<D, M>(q, i, j, k);
            const int t = tix[q];
            T sv, sc;
            var_sums<D, M, T>(U, E, t, i, h, x0, op, sv, sc);
            const T r = R[q] - (sv - sc * U[t]) * ih2;
            if (rout) rout[I.coff + q] = Ro(r);
            rm = fmax(rm, fabs(double(r)));
            pm = fmax(pm, fabs(double(R[q])));
        }
    };
    // per box: maxima over its thread group (shuffles within a warp, then
    // shared memory across the group's warps), one atomic per box and norm
    auto post = [&](const BoxInfo &I, int lt) {
        constexpr int W = S::G < 32 ? S::G : 32;
        for (int off = W / 2; off > 0; off >>= 1) {
            rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, off));
            pm = fmax(pm, __shfl_xor_sync(0xffffffffu, pm, off));
        }
        if constexpr (S::G > 32) {
            const int w = threadIdx.x / 32;
            if ((threadIdx.x & 31) == 0) { red[2 * w] = rm; red[2 * w + 1] = pm; }
            __syncthreads();
            if (lt == 0)
                for (int x = 1; x < S::G / 32; ++x) { rm = fmax(rm, red[2 * (w + x)]); pm = fmax(pm, red[2 * (w + x) + 1]); }
        }
        if (lt == 0 && I.b >= 0) {
            const int tr = A.tree[I.b];
            atomicMax(rmax + tr, (unsigned long long)__double_as_longlong(rm));
            atomicMax(pmax + tr, (unsigned long long)__double_as_longlong(pm));
        }
        rm = 0.0;
        pm = 0.0;
    };
    var_walk<D, M, T>(A, 0, n, list, u, eps, rho, hom, true, body, post);
}

// Restriction of a field (u or eps) from the boxes of a level (or a list of
// boxes) into their parents: the mean of the 2^D children, weighted by r in
// (r,z) (op 2).
template <int D, int M, int MP, typename T>
__global__ void __launch_bounds__(kThreads) k_var_restrict(BoxMeta A, int b0, int n, const int *list, T *v, int op) {
    constexpr int MH = M / 2;
    constexpr int NCO = D == 2 ? MH * MH : MH * MH * MH;
    pdl_trigger();
    pdl_wait();
    const long long total = (long long)n * NCO;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int idx = (int)(e / NCO), c = (int)(e - (long long)idx * NCO);
        const int b = list ? list[idx] : b0 + idx;
        if (A.active && !A.active[A.tree[b]]) continue;
        const int X = c % MH, Y = (c / MH) % MH, Z = D == 3 ? c / (MH * MH) : 0;
        const long long cb = A.coff[b];
        const T h = T(A.hb[b]), x0 = T(A.x0[b]);
        T s = T(0), sw = T(0);
        for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int i = 2 * X + dx, j = 2 * Y + dy, k = D == 3 ? 2 * Z + dz : 0;
                    const T w = var_weight<T>(op, x0, h, i);
                    s += w * v[cb + rbi<D, M>(i, j, k)];
                    sw += w;
                }
        const int po = A.poff[b];
        const int pi = unpack_off(po, 0) + X, pj = unpack_off(po, 1) + Y;
        const int pk = D == 3 ? unpack_off(po, 2) + Z : 0;
        v[A.coff[A.parent[b]] + rbi<D, MP>(pi, pj, pk)] = s / sw;
    }
}

}  // namespace afg
