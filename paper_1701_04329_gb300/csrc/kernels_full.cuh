// Whole-box staging with cp.async, for the kernels that apply the full
// 2D+1-point operator to every cell of a box (both colours): the fused
// residual + restriction (Eq. residual, Sec. 2.5) and the FAS coarse
// right-hand side (Eq. coarse-rhs).
//
// Shared-memory image of a box ("colour planes"): for colour col, the
// half-rows Q[col][row(j,k)][h] hold the cells (i, j, k) of that colour,
// i = 2h + ((col + j + k + D) & 1), for rows j, k in [-1, M] (the rows
// j or k = -1, M are the y/z ghost layers), and X[side][row] holds the x-side
// ghost of each row.  Cell (i, j, k), i in [0, M), is at
// Q[(i + j + k + D) & 1][row(j,k)][i >> 1]; a colour half of a box in global
// memory is exactly the interior of one plane, so every interior half-row
// and every same-level y/z ghost half-row arrives as 16-byte cp.async copies
// (x ghosts as scalars).  Ghosts of domain-boundary and refinement-boundary
// faces are staged as the adjacent inner value u_1 and completed after the
// wait (Sec. 2.4 and the default scheme of Sec. 3.3):
//   Dirichlet:           g = 2 b - u_1
//   refinement boundary: g = u_H/2 + c1 u_1 - (u_2 + u_t1 [+ u_t2])/4,
//                        c1 = 1 (2D), 5/4 (3D).
// Boxes are staged one box ahead of the one being computed (two-stage ring).
#pragma once
#include "kernels_smooth.cuh"

namespace afg {

template <int D, int M, typename T, int GT = Geo<D, M>::G>
struct FpCfg {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int MH = M / 2;
    static constexpr int ROWS = D == 2 ? (M + 2) : (M + 2) * (M + 2);
    static constexpr int PT = ROWS * MH;   // one colour plane
    static constexpr int XT = 2 * ROWS;    // x-side ghosts [side][row]
    static constexpr int UB = 2 * PT + XT; // u with its ghost layer
    static constexpr int H = Geo<D, M>::H, C = 2 * H;
    static constexpr int NVR = MH / VEC;   // vectors per half-row
    static constexpr int FR = D == 2 ? 1 : M;
    static constexpr int NV = C / VEC;     // interior vectors, both colours
    static constexpr int G = GT;           // threads per box
    static constexpr int BPC = kThreads / G;
    static constexpr int NXR = D == 2 ? M : M * M;  // rows per x side
    static constexpr int NXI = 2 * NXR;
    static constexpr int NYI = (2 * D - 2) * FR * 2 * NVR;
    static constexpr int NGI = NXI + NYI;
    static constexpr int NST = 2;
    static constexpr bool ok = MH >= VEC;
    // u image + a flat copy of C more values (rho, or u for a plain copy)
    static constexpr int BOX = UB + C;
    static constexpr size_t smem() { return sizeof(T) * BOX * BPC * NST + sizeof(BoxInfo) * BPC * (NST + 1); }
};

// slot of cell (i, j, k), i in [0, M), j and k in [-1, M]
template <int D, int M, typename T>
__device__ __forceinline__ int fp_slot(int i, int j, int k) {
    using F = FpCfg<D, M, T>;
    return ((i + j + k + D) & 1) * F::PT + sp_row<D, M>(j, k) * F::MH + (i >> 1);
}

// x-side ghost item -> side, row (all rows)
template <int D, int M>
__device__ __forceinline__ void fp_xitem(int item, int &s, int &j, int &k) {
    constexpr int NXR = D == 2 ? M : M * M;
    s = item / NXR;
    const int r = item % NXR;
    j = r % M;
    k = D == 2 ? 0 : r / M;
}

// y/z-side ghost item -> side, colour plane, vector start, ghost / inner / mirror rows
template <int D, int M, typename T>
__device__ __forceinline__ void fp_yzitem(int it2, int &s, int &col, int &h0, int &jg, int &kg, int &jin, int &kin,
                                          int &jm, int &km) {
    using F = FpCfg<D, M, T>;
    constexpr int PER = F::FR * F::NVR;
    s = 2 + it2 / (2 * PER);
    const int rem = it2 % (2 * PER);
    col = rem / PER;
    const int r2 = rem % PER;
    const int fr = r2 / F::NVR;
    h0 = (r2 % F::NVR) * F::VEC;
    const int hi = s & 1;
    if ((s >> 1) == 1) { kg = kin = km = D == 3 ? fr : 0; jg = hi ? M : -1; jin = hi ? M - 1 : 0; jm = hi ? 0 : M - 1; }
    else { jg = jin = jm = fr; kg = hi ? M : -1; kin = hi ? M - 1 : 0; km = hi ? 0 : M - 1; }
}

// Issues the copies of box I into its stage: the u image with ghosts, and C
// values from `flat` (the box's rho, or null) into the flat area.
template <int D, int M, typename T, int GT>
__device__ __forceinline__ void fp_issue(const BoxInfo &I, const T *u, const T *flat, T *st, int lt, bool image) {
    using F = FpCfg<D, M, T, GT>;
    constexpr int VEC = F::VEC, MH = F::MH, H = F::H, NVH = H / VEC;
    const T *ub = u + I.coff;
    T *fl = st + F::UB;
    for (int v = lt; v < F::NV; v += F::G) {
        if (image) {
            const int col = v / NVH, w = v % NVH;
            const int row = w / F::NVR, h0 = (w % F::NVR) * VEC;
            const int j = row % M, k = D == 2 ? 0 : row / M;
            cp_async<16>(st + col * F::PT + sp_row<D, M>(j, k) * MH + h0, ub + v * VEC);
        }
        if (flat) cp_async<16>(fl + v * VEC, flat + I.coff + v * VEC);
    }
    if (!image) return;
    for (int item = lt; item < F::NGI; item += F::G) {
        if (item < F::NXI) {
            int s, j, k;
            fp_xitem<D, M>(item, s, j, k);
            const int colg = ((s ? M : -1) + j + k + D) & 1;  // colour of the ghost cell
            const T *src = I.code[s] >= 0 ? u + I.base[s] + colg * H + hrow<D, M>(j, k) + (s ? 0 : MH - 1)
                                          : ub + (1 - colg) * H + hrow<D, M>(j, k) + (s ? MH - 1 : 0);
            cp_async<(int)sizeof(T)>(st + 2 * F::PT + s * F::ROWS + sp_row<D, M>(j, k), src);
        } else {
            int s, col, h0, jg, kg, jin, kin, jm, km;
            fp_yzitem<D, M, T>(item - F::NXI, s, col, h0, jg, kg, jin, kin, jm, km);
            const T *src = I.code[s] >= 0 ? u + I.base[s] + col * H + hrow<D, M>(jm, km) + h0
                                          : ub + (1 - col) * H + hrow<D, M>(jin, kin) + h0;
            cp_async<16>(st + col * F::PT + sp_row<D, M>(jg, kg) * MH + h0, src);
        }
    }
}

// Per-thread copy plan of fp_issue, the same for every box of a launch: for
// each ghost item of the thread, the destination in the stage, the side,
// whether it is a scalar (x side), the source offsets relative to the
// neighbour box (same-level copy) and to the box itself (the mirror u_1),
// and the item's first boundary-data offset (stride 2 along a y/z item).
template <int D, int M, typename T, int GT>
struct FpPlan {
    using F = FpCfg<D, M, T, GT>;
    static constexpr int NIV = (F::NV + F::G - 1) / F::G;
    static constexpr int NQ = (F::NGI + F::G - 1) / F::G;
    int vdst[NIV];
    int gdst[NQ], gsrc[NQ], gbc[NQ];  // dst | side << 16 | scalar << 19 ; copy | mirror << 16
    __device__ __forceinline__ void init(int lt) {
        constexpr int VEC = F::VEC, MH = F::MH, H = F::H, NVH = H / VEC;
#pragma unroll
        for (int it = 0; it < NIV; ++it) {
            const int v = lt + it * F::G;
            const int col = v / NVH, w = v % NVH;
            const int row = w / F::NVR, h0 = (w % F::NVR) * VEC;
            const int j = row % M, k = D == 2 ? 0 : row / M;
            vdst[it] = v < F::NV ? col * F::PT + sp_row<D, M>(j, k) * MH + h0 : -1;
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int item = lt + q * F::G;
            gdst[q] = -1;
            gsrc[q] = gbc[q] = 0;
            if (item >= F::NGI) continue;
            if (item < F::NXI) {
                int s, j, k;
                fp_xitem<D, M>(item, s, j, k);
                const int colg = ((s ? M : -1) + j + k + D) & 1;  // colour of the ghost cell
                gdst[q] = (2 * F::PT + s * F::ROWS + sp_row<D, M>(j, k)) | (s << 16) | (1 << 19);
                gsrc[q] = (colg * H + hrow<D, M>(j, k) + (s ? 0 : MH - 1)) |
                          (((1 - colg) * H + hrow<D, M>(j, k) + (s ? MH - 1 : 0)) << 16);
                gbc[q] = k * M + j;
            } else {
                int s, col, h0, jg, kg, jin, kin, jm, km;
                fp_yzitem<D, M, T>(item - F::NXI, s, col, h0, jg, kg, jin, kin, jm, km);
                gdst[q] = (col * F::PT + sp_row<D, M>(jg, kg) * MH + h0) | (s << 16);
                gsrc[q] = (col * H + hrow<D, M>(jm, km) + h0) | (((1 - col) * H + hrow<D, M>(jin, kin) + h0) << 16);
                const int rg = (col + jg + kg + D) & 1;
                gbc[q] = ((s >> 1) == 1 ? kin : jin) * M + 2 * h0 + rg;
            }
        }
    }
};

// fp_issue through the plan
template <int D, int M, typename T, int GT>
__device__ __forceinline__ void fp_issue_plan(const FpPlan<D, M, T, GT> &pl, const BoxInfo &I, const T *u,
                                              const T *flat, T *st, int lt, bool image) {
    using F = FpCfg<D, M, T, GT>;
    constexpr int VEC = F::VEC;
    const T *ub = u + I.coff;
    T *fl = st + F::UB;
#pragma unroll
    for (int it = 0; it < FpPlan<D, M, T, GT>::NIV; ++it) {
        const int v = lt + it * F::G;
        if (pl.vdst[it] < 0) continue;
        if (image) cp_async<16>(st + pl.vdst[it], ub + v * VEC);
        if (flat) cp_async<16>(fl + v * VEC, flat + I.coff + v * VEC);
    }
    if (!image) return;
#pragma unroll
    for (int q = 0; q < FpPlan<D, M, T, GT>::NQ; ++q) {
        const int dst = pl.gdst[q];
        if (dst < 0) continue;
        const int sd = (dst >> 16) & 7;
        const T *src = I.code[sd] >= 0 ? u + I.base[sd] + (pl.gsrc[q] & 0xffff) : ub + (pl.gsrc[q] >> 16);
        if (dst & (1 << 19)) cp_async<(int)sizeof(T)>(st + (dst & 0xffff), src);
        else cp_async<16>(st + (dst & 0xffff), src);
    }
}

// fp_fix_own through the plan
template <int D, int M, typename T, int GT>
__device__ __forceinline__ void fp_fix_own_plan(const FpPlan<D, M, T, GT> &pl, const BoxInfo &I, const BoxMeta &A,
                                                T *st, int hom) {
    using F = FpCfg<D, M, T, GT>;
    constexpr int VEC = F::VEC;
#pragma unroll
    for (int q = 0; q < FpPlan<D, M, T, GT>::NQ; ++q) {
        const int dst = pl.gdst[q];
        if (dst < 0) continue;
        const int sd = (dst >> 16) & 7;
        if (I.code[sd] != -1) continue;
        const bool neu = (I.nmask >> sd) & 1;
        const T hbox = neu ? T(A.hb[I.b]) : T(0);
        const double *bc = A.bc + I.base[sd] + pl.gbc[q];
        T *gv = st + (dst & 0xffff);
        if (dst & (1 << 19)) {
            const T bv = hom ? T(0) : T(bc[0]);
            gv[0] = neu ? fma(hbox, bv, gv[0]) : T(2) * bv - gv[0];
        } else {
#pragma unroll
            for (int x = 0; x < VEC; ++x) {
                const T bv = hom ? T(0) : T(bc[2 * x]);
                gv[x] = neu ? fma(hbox, bv, gv[x]) : T(2) * bv - gv[x];
            }
        }
    }
}

// Completes the domain-side ghosts among this thread's own items (the ones
// fp_issue gave it) from the u_1 it staged there: 2 b - u_1 (Dirichlet) or
// u_1 + h b (Neumann).  Its own copies are visible to it after its wait, so
// this needs no barrier.
template <int D, int M, typename T, int GT>
__device__ __forceinline__ void fp_fix_own(const BoxInfo &I, const BoxMeta &A, T *st, int lt, int hom) {
    using F = FpCfg<D, M, T, GT>;
    constexpr int VEC = F::VEC, MH = F::MH;
    for (int item = lt; item < F::NGI; item += F::G) {
        if (item < F::NXI) {
            int s, j, k;
            fp_xitem<D, M>(item, s, j, k);
            if (I.code[s] != -1) continue;
            T &gv = st[2 * F::PT + s * F::ROWS + sp_row<D, M>(j, k)];
            const T bv = hom ? T(0) : T(A.bc[I.base[s] + k * M + j]);
            gv = ((I.nmask >> s) & 1) ? fma(T(A.hb[I.b]), bv, gv) : T(2) * bv - gv;
        } else {
            int s, col, h0, jg, kg, jin, kin, jm, km;
            fp_yzitem<D, M, T>(item - F::NXI, s, col, h0, jg, kg, jin, kin, jm, km);
            if (I.code[s] != -1) continue;
            T *gv = st + col * F::PT + sp_row<D, M>(jg, kg) * MH + h0;
            const int rg = (col + jg + kg + D) & 1;
            const int t2 = (s >> 1) == 1 ? kin : jin;
            const bool neu = (I.nmask >> s) & 1;
#pragma unroll
            for (int x = 0; x < VEC; ++x) {
                const T bv = hom ? T(0) : T(A.bc[I.base[s] + t2 * M + 2 * (h0 + x) + rg]);
                gv[x] = neu ? fma(T(A.hb[I.b]), bv, gv[x]) : T(2) * bv - gv[x];
            }
        }
    }
}

// Completes the ghosts of non-copy faces from the staged u_1 (after the wait;
// cf_only: the refinement-boundary faces only, fp_fix_own doing the domain sides).
template <int D, int M, typename T, int GT>
__device__ __forceinline__ void fp_fix(const BoxInfo &I, const BoxMeta &A, const T *u, T *st, int lt, int hom,
                                       bool cf_only = false) {
    using F = FpCfg<D, M, T, GT>;
    constexpr int VEC = F::VEC, MH = F::MH;
    const T c1 = D == 2 ? T(1) : T(1.25);
    auto at = [&](int i, int j, int k) -> T { return st[fp_slot<D, M, T>(i, j, k)]; };
    for (int item = lt; item < F::NGI; item += F::G) {
        if (item < F::NXI) {
            int s, j, k;
            fp_xitem<D, M>(item, s, j, k);
            const int code = I.code[s];
            if (code >= 0 || (cf_only && code == -1)) continue;
            T &gv = st[2 * F::PT + s * F::ROWS + sp_row<D, M>(j, k)];
            const T u1 = gv;
            if (code == -1) {
                const T bv = hom ? T(0) : T(A.bc[I.base[s] + k * M + j]);
                gv = ((I.nmask >> s) & 1) ? fma(T(A.hb[I.b]), bv, u1) : T(2) * bv - u1;
            } else {
                const int iin = s ? M - 1 : 0, p2 = s ? M - 2 : 1;
                const int cj = unpack_off(I.poff, 1) + (j >> 1);
                const int ck = D == 3 ? unpack_off(I.poff, 2) + (k >> 1) : 0;
                const T uH = u[I.base[s] + rbi<D, M>(s ? 0 : M - 1, cj, ck)];
                T acc = at(p2, j, k) + at(iin, j ^ 1, k);
                if (D == 3) acc += at(iin, j, k ^ 1);
                gv = T(0.5) * uH + c1 * u1 - T(0.25) * acc;
            }
        } else {
            int s, col, h0, jg, kg, jin, kin, jm, km;
            fp_yzitem<D, M, T>(item - F::NXI, s, col, h0, jg, kg, jin, kin, jm, km);
            const int code = I.code[s];
            if (code >= 0 || (cf_only && code == -1)) continue;
            const int hi = s & 1, a = s >> 1;
            T *gv = st + col * F::PT + sp_row<D, M>(jg, kg) * MH + h0;
            const int rg = (col + jg + kg + D) & 1;  // i-parity of the plane's cells in the ghost row
            const int p2 = hi ? M - 2 : 1;
#pragma unroll
            for (int x = 0; x < VEC; ++x) {
                const int i = 2 * (h0 + x) + rg;
                const T u1 = gv[x];
                if (code == -1) {
                    const int t2 = a == 1 ? kin : jin;
                    const T bv = hom ? T(0) : T(A.bc[I.base[s] + t2 * M + i]);
                    gv[x] = ((I.nmask >> s) & 1) ? fma(T(A.hb[I.b]), bv, u1) : T(2) * bv - u1;
                } else {
                    const int ci = unpack_off(I.poff, 0) + (i >> 1);
                    int cj, ck;
                    T acc;
                    if (a == 1) {
                        cj = hi ? 0 : M - 1;
                        ck = D == 3 ? unpack_off(I.poff, 2) + (kin >> 1) : 0;
                        acc = at(i, p2, kin) + at(i ^ 1, jin, kin);
                        if (D == 3) acc += at(i, jin, kin ^ 1);
                    } else {
                        cj = unpack_off(I.poff, 1) + (jin >> 1);
                        ck = hi ? 0 : M - 1;
                        acc = at(i, jin, p2) + at(i ^ 1, jin, kin);
                        acc += at(i, jin ^ 1, kin);
                    }
                    const T uH = u[I.base[s] + rbi<D, M>(ci, cj, ck)];
                    gv[x] = T(0.5) * uH + c1 * u1 - T(0.25) * acc;
                }
            }
        }
    }
}

// For the VEC cells of colour col at half-row (j,k), h0..h0+VEC-1: the sums
// of their 2D neighbours less 2D times their own values (h^2 A u, Eq. 5).
template <int D, int M, typename T, bool FX = true>
__device__ __forceinline__ void fp_lap_vec(const T *st, int col, int j, int k, int h0, T *lap) {
    using F = FpCfg<D, M, T>;
    constexpr int VEC = F::VEC, MH = F::MH;
    const int rowi = sp_row<D, M>(j, k);
    const int r = (col + j + k + D) & 1;  // cells at i = 2h + r; neighbours in the other plane
    const T *po = st + (1 - col) * F::PT + rowi * MH + h0;
    const T *X = st + 2 * F::PT;
    T self[VEC], xv[VEC], ym[VEC], yp[VEC], zm[VEC], zp[VEC];
    ldv<T, VEC>(st + col * F::PT + rowi * MH + h0, self);
    ldv<T, VEC>(po, xv);
    T extra;
    if (r) extra = h0 + VEC < MH ? po[VEC] : X[F::ROWS + rowi];
    else extra = h0 > 0 ? po[-1] : X[rowi];
    ldv<T, VEC>(po - MH, ym);
    ldv<T, VEC>(po + MH, yp);
    if (D == 3) {
        ldv<T, VEC>(po - (M + 2) * MH, zm);
        ldv<T, VEC>(po + (M + 2) * MH, zp);
    }
#pragma unroll
    for (int x = 0; x < VEC; ++x) {
        const T xl = r ? xv[x] : (x ? xv[x - 1] : extra);
        const T xr = r ? (x + 1 < VEC ? xv[x + 1] : extra) : xv[x];
        lap[x] = nb_lap6<D, T, FX>(self[x], xl, xr, ym[x], yp[x], D == 3 ? zm[x] : T(0), D == 3 ? zp[x] : T(0));
    }
}

// Prologue and ring walk shared by the kernels below.  body(I, st, lt) is
// called once per staged box after its ghosts are complete; want(I) says
// whether a box needs the u image, flat(I) which array goes to the flat area
// (or null).  pre(slots) and post(slots) run in every thread of the block
// before and after the bodies of one step, with the metadata of the step's
// boxes (one per group).
// OWN: the issuing threads complete the domain-side ghosts before the box's
// barrier (fp_fix_own) and only refinement-boundary boxes take the extra
// barrier; otherwise every box with a non-copy side takes it (fewer registers).
// PLAN: copies and domain-side fixes through a per-thread plan (FpPlan), no
// per-box decoding of the items (more registers).
template <int D, int M, typename T, int GT, bool OWN = true, bool PLAN = false, typename Want, typename Flat,
          typename Body, typename Pre, typename Post>
__device__ __forceinline__ void fp_walk(const BoxMeta &A, int b0, int n, const int *list, const T *u, int hom,
                                        Want want, Flat flat, Body body, Pre pre, Post post) {
    using F = FpCfg<D, M, T, GT>;
    constexpr int NST = F::NST, NI = NST + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / F::G, lt = threadIdx.x % F::G;
    T *stages = reinterpret_cast<T *>(smem_raw);
    BoxInfo *info = reinterpret_cast<BoxInfo *>(smem_raw + sizeof(T) * F::BOX * F::BPC * NST);
    const int stride = gridDim.x * F::BPC;
    const int first = blockIdx.x * F::BPC;
    for (int q = 0; q < NST; ++q)  // static metadata: before the wait
        info_load<D>(A, first + q * stride + g, n, b0, list, info[q * F::BPC + g], lt, F::G, false);
    pdl_wait();
    for (int q = 0; q < NST; ++q) info_mask<D>(A, info[q * F::BPC + g], lt, F::G);
    __syncthreads();
    FpPlan<D, M, T, GT> pl;
    if constexpr (PLAN) pl.init(lt);
    auto issue = [&](int q) {
        const BoxInfo &In = info[(q % NI) * F::BPC + g];
        T *dst = stages + ((q % NST) * F::BPC + g) * F::BOX;
        if (In.b >= 0) {
            if constexpr (PLAN) fp_issue_plan<D, M, T, GT>(pl, In, u, flat(In), dst, lt, want(In));
            else fp_issue<D, M, T, GT>(In, u, flat(In), dst, lt, want(In));
        }
        cp_commit();
    };
    for (int q = 0; q < NST - 1; ++q) issue(q);
    int it = 0;
    for (int base = first; base < n; base += stride, ++it) {
        cp_wait<NST - 2>();
        const BoxInfo &I = info[(it % NI) * F::BPC + g];
        const bool special = I.b >= 0 && want(I) && (I.flag & BF_SPECIAL);
        const bool cf = special && (!OWN || (I.flag & BF_CF));
        T *st = stages + ((it % NST) * F::BPC + g) * F::BOX;
        if (OWN && special) {  // domain sides: this thread's own items
            if constexpr (PLAN) fp_fix_own_plan<D, M, T, GT>(pl, I, A, st, hom);
            else fp_fix_own<D, M, T, GT>(I, A, st, lt, hom);
        }
        const int any_cf = __syncthreads_or(cf);  // previous stage and metadata slot are free now
        issue(it + NST - 1);
        info_load<D>(A, base + NST * stride + g, n, b0, list, info[((it + NST) % NI) * F::BPC + g], lt, F::G);
        pre(&info[(it % NI) * F::BPC]);
        if (any_cf) {  // refinement-boundary ghosts read cells other threads staged
            if (cf) fp_fix<D, M, T, GT>(I, A, u, st, lt, hom, OWN);
            __syncthreads();
        }
        if (I.b >= 0) body(I, st, lt);
        post(&info[(it % NI) * F::BPC]);
    }
    cp_wait<0>();
}

// threads per box of the restriction: one per coarse cell, at least a warp
// (FP32); FP64 boxes take the whole block (their stages are twice as large)
template <int D, int M, typename T>
constexpr int rr_threads() {
    constexpr int NCO = D == 2 ? (M / 2) * (M / 2) : (M / 2) * (M / 2) * (M / 2);
    return sizeof(T) == 8 ? Geo<D, M>::G : (NCO < 32 ? 32 : (NCO > kThreads ? kThreads : NCO));
}

// threads per box of the FAS kernel: one per interior vector, at least a warp
template <int D, int M, typename T>
constexpr int fas_threads() {
    constexpr int NV = Geo<D, M>::C * (int)sizeof(T) / 16;
    return NV < 32 ? 32 : (NV > kThreads ? kThreads : NV);
}

// threads per box of the leaf residual: as the FAS kernel, but FP64 boxes take
// at most 64 threads where the several boxes per block that this gives fit in
// 100 KB of shared memory, two blocks per SM (measured 0.288 instead of
// 0.297 ms on a 256^3 level of 8^3 boxes)
template <int D, int M, typename T>
constexpr int leaf_threads() {
    return (sizeof(T) == 8 && fas_threads<D, M, T>() > 64 && FpCfg<D, M, T, 64>::smem() <= 100 * 1024)
               ? 64
               : fas_threads<D, M, T>();
}

// Fused residual + restriction, staged version of k_resid_restrict (same
// arithmetic and summation order).
template <int D, int M, int MP, typename T>
__global__ void __launch_bounds__(kThreads) k_resid_restrict_p(BoxMeta A, int b0, int n, T *u, T *rho, T *vold,
                                                               T ih2, int hom) {
    constexpr int GT = rr_threads<D, M, T>();
    using F = FpCfg<D, M, T, GT>;
    constexpr int MH = M / 2;
    constexpr int NCO = D == 2 ? MH * MH : MH * MH * MH;
    pdl_trigger();
    auto want = [](const BoxInfo &) { return true; };
    auto flat = [&](const BoxInfo &) -> const T * { return rho; };
    auto body = [&](const BoxInfo &I, const T *st, int lt) {
        const T *X = st + 2 * F::PT, *R = st + F::UB;
        const long long cp = A.coff[I.parent];
        for (int c = lt; c < NCO; c += F::G) {
            const int Xc = c % MH, Y = (c / MH) % MH, Z = D == 3 ? c / (MH * MH) : 0;
            // sum_c (A u)_c = (sum_outside - D sum_c u) / h^2 over the 2^D children
            T su = T(0), sro = T(0), sout = T(0);
#pragma unroll
            for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        const int i = 2 * Xc + dx, j = 2 * Y + dy, k = D == 3 ? 2 * Z + dz : 0;
                        su += st[fp_slot<D, M, T>(i, j, k)];
                        sro += R[rbi<D, M>(i, j, k)];
                        const int rowi = sp_row<D, M>(j, k);
                        T xo;
                        if (dx) xo = Xc + 1 < MH ? st[fp_slot<D, M, T>(i + 1, j, k)] : X[F::ROWS + rowi];
                        else xo = Xc > 0 ? st[fp_slot<D, M, T>(i - 1, j, k)] : X[rowi];
                        sout += xo;
                        sout += st[fp_slot<D, M, T>(i, dy ? j + 1 : j - 1, k)];
                        if (D == 3) sout += st[fp_slot<D, M, T>(i, j, dz ? k + 1 : k - 1)];
                    }
            const T w = T(1) / T(1 << D);
            const T sr = fma(-ih2, fma(T(-D), su, sout), sro);
            const int pi = unpack_off(I.poff, 0) + Xc, pj = unpack_off(I.poff, 1) + Y;
            const int pk = D == 3 ? unpack_off(I.poff, 2) + Z : 0;
            const long long q = cp + rbi<D, MP>(pi, pj, pk);
            const T mu = su * w;
            u[q] = mu;
            vold[q] = mu;
            rho[q] = sr * w;
        }
    };
    auto none = [](const BoxInfo *) {};
    fp_walk<D, M, T, GT, true, sizeof(T) == 4>(A, b0, n, nullptr, u, hom, want, flat, body, none, none);
}

// FAS coarse right-hand side, staged version of k_fas: refined boxes get
// rho_H += A_H(v_H) (and rho_hat = chat rho_H when rhoh is set); leaves copy
// v' = v.
template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_fas_p(BoxMeta A, int b0, int n, const T *u, T *rho, T *vold, T ih2,
                                                    int hom, T *rhoh, T chat) {
    constexpr int GT = fas_threads<D, M, T>();
    using F = FpCfg<D, M, T, GT>;
    constexpr int VEC = F::VEC, NVH = F::H / VEC;
    pdl_trigger();
    auto want = [](const BoxInfo &I) { return (I.flag & BF_REFINED) != 0; };
    auto flat = [&](const BoxInfo &I) -> const T * { return (I.flag & BF_REFINED) ? rho : u; };
    auto body = [&](const BoxInfo &I, const T *st, int lt) {
        const T *FL = st + F::UB;
        if (!(I.flag & BF_REFINED)) {
            for (int v = lt; v < F::NV; v += F::G) {
                T e[VEC];
                ldv<T, VEC>(FL + v * VEC, e);
                stv<T, VEC>(vold + I.coff + (long long)v * VEC, e);
            }
            return;
        }
        for (int v = lt; v < F::NV; v += F::G) {
            const int col = v / NVH, w = v % NVH;
            const int row = w / F::NVR, h0 = (w % F::NVR) * VEC;
            const int j = row % M, k = D == 2 ? 0 : row / M;
            T lap[VEC], rv[VEC], out[VEC];
            fp_lap_vec<D, M, T, false>(st, col, j, k, h0, lap);  // FP64 adds: the integer path costs registers here
            ldv<T, VEC>(FL + v * VEC, rv);
#pragma unroll
            for (int x = 0; x < VEC; ++x) out[x] = fma(ih2, lap[x], rv[x]);
            stv<T, VEC>(rho + I.coff + (long long)v * VEC, out);
            if (rhoh) {
#pragma unroll
                for (int x = 0; x < VEC; ++x) out[x] *= chat;
                stv<T, VEC>(rhoh + I.coff + (long long)v * VEC, out);
            }
        }
    };
    auto none = [](const BoxInfo *) {};
    fp_walk<D, M, T, GT>(A, b0, n, nullptr, u, hom, want, flat, body, none, none);
}

// Composite residual on the leaves (Eq. residual with the ghost rules of
// Secs. 2.4 and 3.3), staged version of k_leaf_residual: per tree, the
// maxima of |r| and |rho| over the leaf cells (as bit patterns, reduced per
// block and committed with one atomic per block when the block moves to
// another tree, and at the end), and optionally r cast to R in rout.
template <int D, int M, typename T, typename R>
__global__ void __launch_bounds__(kThreads) k_leaf_residual_p(BoxMeta A, const int *list, int n, const T *u,
                                                              const T *__restrict__ rho, int hom,
                                                              unsigned long long *rmax, unsigned long long *pmax,
                                                              R *rout) {
    constexpr int GT = leaf_threads<D, M, T>();
    using F = FpCfg<D, M, T, GT>;
    constexpr int VEC = F::VEC, NVH = F::H / VEC;
    __shared__ unsigned long long red[64];
    pdl_trigger();
    const int g = threadIdx.x / F::G;
    unsigned long long rm = 0, pm = 0;
    int cur = -1, tr = -1;  // tree of the running maxima, tree of this step's boxes (uniform in the block)
    bool mixed = false;
    auto want = [](const BoxInfo &) { return true; };
    auto flat = [&](const BoxInfo &) -> const T * { return rho; };
    auto pre = [&](const BoxInfo *slot) {
        tr = -1;
        mixed = false;
        for (int x = 0; x < F::BPC; ++x) {
            if (slot[x].b < 0) continue;
            const int t = A.tree[slot[x].b];
            if (tr < 0) tr = t;
            else if (t != tr) mixed = true;
        }
        if (mixed || (tr >= 0 && cur >= 0 && tr != cur)) {
            flush_max(rm, pm, cur, cur >= 0, rmax, pmax, red);
            rm = pm = 0;
            cur = -1;
        }
    };
    auto body = [&](const BoxInfo &I, const T *st, int lt) {
        const T ih2 = T(A.ih2[I.b]);
        const T *FL = st + F::UB;
        for (int v = lt; v < F::NV; v += F::G) {
            const int col = v / NVH, w = v % NVH;
            const int row = w / F::NVR, h0 = (w % F::NVR) * VEC;
            const int j = row % M, k = D == 2 ? 0 : row / M;
            T lap[VEC], rv[VEC];
            fp_lap_vec<D, M, T>(st, col, j, k, h0, lap);
            ldv<T, VEC>(FL + v * VEC, rv);
            R out[VEC];
#pragma unroll
            for (int x = 0; x < VEC; ++x) {
                // r = rho - (sum - 2D u) / h^2; |.| on the bit patterns
                const T rr = fma(-ih2, lap[x], rv[x]);
                out[x] = R(rr);
                rm = max(rm, abs_bits(rr));
                pm = max(pm, abs_bits(rv[x]));
            }
            if (rout) {
#pragma unroll
                for (int x = 0; x < VEC; ++x) rout[I.coff + (long long)v * VEC + x] = out[x];
            }
        }
    };
    auto post = [&](const BoxInfo *slot) {
        if (mixed) {  // boxes of several trees in this step: commit each box's maxima now
            for (int x = 0; x < F::BPC; ++x) {
                const int t = slot[x].b >= 0 ? A.tree[slot[x].b] : -1;
                flush_max(g == x ? rm : 0ull, g == x ? pm : 0ull, t, t >= 0, rmax, pmax, red);
            }
            rm = pm = 0;
        } else if (tr >= 0) {
            cur = tr;
        }
    };
    fp_walk<D, M, T, GT, false>(A, 0, n, list, u, hom, want, flat, body, pre, post);  // register-bound: no own-thread fix
    flush_max(rm, pm, cur, cur >= 0, rmax, pmax, red);
}

// ---------------------------------------------------------------------------
// Coarse-grid correction u_h += I_H^h (v_H - v'_H) (Eq. coarse-corr), staged
// version of k_correct: a box's own values (16-byte copies) and the parent's
// v_H and v'_H over the box's parent region plus one layer (scalar copies;
// outside the parent from its same-level neighbour, or mirrored inside it at
// the domain boundary, where the difference changes sign on Dirichlet sides
// and keeps it on Neumann sides) arrive by cp.async
// one box ahead; d = v_H - v'_H is formed once per staged value, then the
// 2-1-1 / 1-1-1-1 prolongation (Sec. 2.5) is added.  In 3D the prolongation
// of child (sx,sy,sz) is (1/4)((d0 + d_x(sx)) + (d_y(sy) + d_z(sz))): the two
// x-pair and four yz-pair sums of a coarse cell are formed once for its 8
// children (2.75 instead of 4 additions per fine cell; it matters for FP64,
// whose arithmetic bounds this kernel).
// ---------------------------------------------------------------------------
template <int D, int M, typename T>
struct CpCfg {
    static constexpr int MH = M / 2, Q = MH + 2;
    static constexpr int QC = D == 2 ? Q * Q : Q * Q * Q;
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int QCP = (QC + VEC - 1) / VEC * VEC;  // keeps 16-byte alignment
    static constexpr int C = Geo<D, M>::C;
    static constexpr int NV = C / VEC;
    static constexpr int G = NV < kThreads ? NV : kThreads;
    static constexpr int BPC = kThreads / G;
    static constexpr int NIT = (NV + G - 1) / G;
    // 3D: the pair sums of each coarse cell, shared by its 8 children
    static constexpr int N3 = MH * MH * MH;
    static constexpr int PSZ = D == 3 ? (6 * N3 + VEC - 1) / VEC * VEC : 0;
    static constexpr int BOX = C + 2 * QCP + PSZ;
    static constexpr int NST = 2;
    static constexpr bool ok = MH >= VEC;  // a vector stays inside one half-row
    static constexpr size_t smem() { return sizeof(T) * BOX * BPC * NST + sizeof(BoxInfo) * BPC * (NST + 1); }
};

// padded parent-region slot c -> (x, y, z) in [-1, MH], side of the parent it
// lies beyond (-1: inside), and whether it is used (corners/edges are not)
template <int D, int M>
__device__ __forceinline__ bool cp_slot(int c, int &x, int &y, int &z) {
    constexpr int Q = M / 2 + 2, MH = M / 2;
    x = c % Q - 1;
    y = (c / Q) % Q - 1;
    z = D == 3 ? c / (Q * Q) - 1 : 0;
    const int out = (x < 0 || x >= MH) + (y < 0 || y >= MH) + (D == 3 && (z < 0 || z >= MH));
    return out <= 1;
}

// Per-thread staging plan of the parent region, the same for every box of a
// launch.  With MP = M the parent-relative offset poff is 0 or M/2 per axis
// (even), so a slot (x, y, z) of the region maps to the parent's storage
// index rbi(poff + (x, y, z)) = rel(x, y, z) + rbi-offset(poff), colour
// included; rel is per slot, the poff part per box.  A slot outside the
// region's interior along axis a lies inside the parent unless poff puts it
// beyond the parent's side; then it is read from the parent's neighbour at
// the wrapped coordinate (offset rel + nbd, colour unchanged since M is even)
// or, at the domain boundary, mirrored to the slot one step inward (offset
// mir, the other colour).
template <int D, int M, typename T>
struct CpPlan {
    using S = CpCfg<D, M, T>;
    static constexpr int NQ = (S::QC + S::G - 1) / S::G;
    // meta: bit 0 valid, bits 1-2 axis (3: inside along every axis), bit 3 high side
    int rel[NQ], nbd[NQ], mir[NQ], meta[NQ];
    static __device__ __forceinline__ int rel_of(int x, int y, int z) {
        constexpr int MH = M / 2;
        return ((x + y + z + D) & 1) * Geo<D, M>::H + (z * M + y) * MH + (x >> 1);
    }
    __device__ __forceinline__ void init(int lt) {
        constexpr int MH = M / 2;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int c = lt + q * S::G;
            int x = 0, y = 0, z = 0;
            meta[q] = 0;
            rel[q] = nbd[q] = mir[q] = 0;
            if (c >= S::QC || !cp_slot<D, M>(c, x, y, z)) continue;
            int a = 3, hi = 0;
            if (x < 0 || x >= MH) { a = 0; hi = x >= MH; }
            if (y < 0 || y >= MH) { a = 1; hi = y >= MH; }
            if (D == 3 && (z < 0 || z >= MH)) { a = 2; hi = z >= MH; }
            meta[q] = 1 | (a << 1) | (hi << 3);
            rel[q] = rel_of(x, y, z);
            if (a < 3) {
                // wrapping pc_a by -+M moves (pc_x >> 1) by -+M/2, or pc_a * stride by -+M * stride
                const int wrap = a == 0 ? MH : (a == 1 ? M * MH : M * M * MH);
                nbd[q] = hi ? -wrap : wrap;
                const int st = hi ? -1 : 1;  // one step inward
                mir[q] = rel_of(x + (a == 0 ? st : 0), y + (a == 1 ? st : 0), z + (a == 2 ? st : 0));
            }
        }
    }
};

// Issues the copies of box I into its stage with the plan: the box's own
// values (vectors) and, per region slot, the parent's u and v' -- swapped
// across a Dirichlet domain side, so that DU - DV is the difference with the
// homogeneous ghost rule (-d Dirichlet, d Neumann) in every slot.
template <int D, int M, int MP, typename T>
__device__ __forceinline__ void cp_issue(const CpPlan<D, M, T> &pl, const BoxInfo &I, const T *u, const T *vold,
                                         T *st, int lt) {
    static_assert(MP == M, "the staged correction serves levels whose parents have the same box size");
    using S = CpCfg<D, M, T>;
    constexpr int MH = M / 2;
    T *U = st, *DU = st + S::C, *DV = DU + S::QCP;
    for (int v = lt; v < S::NV; v += S::G) cp_async<16>(U + v * S::VEC, u + I.coff + (long long)v * S::VEC);
    const int px = unpack_off(I.poff, 0), py = unpack_off(I.poff, 1), pz = D == 3 ? unpack_off(I.poff, 2) : 0;
    const int poffs = (pz * M + py) * MH + (px >> 1);
#pragma unroll
    for (int q = 0; q < CpPlan<D, M, T>::NQ; ++q) {
        const int m = pl.meta[q];
        if (!(m & 1)) continue;
        const int c = lt + q * S::G, a = (m >> 1) & 3, hi = (m >> 3) & 1;
        long long src = I.pcoff + poffs + pl.rel[q];
        bool swap = false;
        if (a < 3) {
            const int pa = a == 0 ? px : (a == 1 ? py : pz);
            if (pa == (hi ? MH : 0)) {  // beyond the parent's side
                const int side = 2 * a + hi;
                if (I.code[side] >= 0) {
                    src = I.base[side] + poffs + pl.rel[q] + pl.nbd[q];
                } else {
                    src = I.pcoff + poffs + pl.mir[q];
                    swap = !((I.nmask >> side) & 1);
                }
            }
        }
        cp_async<(int)sizeof(T)>((swap ? DV : DU) + c, u + src);
        cp_async<(int)sizeof(T)>((swap ? DU : DV) + c, vold + src);
    }
}

template <int D, int M, int MP, typename T>
__global__ void __launch_bounds__(kThreads) k_correct_p(BoxMeta A, int b0, int n, T *u, const T *__restrict__ vold) {
    using S = CpCfg<D, M, T>;
    constexpr int NST = S::NST, NI = NST + 1, Q = S::Q, VEC = S::VEC, MH = S::MH;
    constexpr int NVH = Geo<D, M>::H / VEC, NVR = MH / VEC > 0 ? MH / VEC : 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / S::G, lt = threadIdx.x % S::G;
    T *stages = reinterpret_cast<T *>(smem_raw);
    BoxInfo *info = reinterpret_cast<BoxInfo *>(smem_raw + sizeof(T) * S::BOX * S::BPC * NST);
    const int stride = gridDim.x * S::BPC;
    const int first = blockIdx.x * S::BPC;
    CpPlan<D, M, T> pl;
    pl.init(lt);
    pdl_trigger();
    for (int q = 0; q < NST; ++q)  // static metadata: before the wait
        pinfo_load<D>(A, first + q * stride + g, n, b0, info[q * S::BPC + g], lt, S::G, false);
    pdl_wait();
    for (int q = 0; q < NST; ++q) info_mask<D>(A, info[q * S::BPC + g], lt, S::G);
    __syncthreads();
    auto issue = [&](int q) {
        const BoxInfo &In = info[(q % NI) * S::BPC + g];
        if (In.b >= 0) cp_issue<D, M, MP, T>(pl, In, u, vold, stages + ((q % NST) * S::BPC + g) * S::BOX, lt);
        cp_commit();
    };
    for (int q = 0; q < NST - 1; ++q) issue(q);
    int it = 0;
    for (int base = first; base < n; base += stride, ++it) {
        cp_wait<NST - 2>();
        const BoxInfo &I = info[(it % NI) * S::BPC + g];
        T *st = stages + ((it % NST) * S::BPC + g) * S::BOX;
        T *U = st, *DU = st + S::C;
        const T *DV = DU + S::QCP;
        if (I.b >= 0) {  // d = v_H - v'_H in the slots this thread staged (its own copies have landed)
#pragma unroll
            for (int q = 0; q < CpPlan<D, M, T>::NQ; ++q) {
                const int c = lt + q * S::G;
                if (pl.meta[q] & 1) DU[c] -= DV[c];
            }
        }
        __syncthreads();  // the differences are visible; the previous stage and metadata slot are free
        issue(it + NST - 1);
        pinfo_load<D>(A, base + NST * stride + g, n, b0, info[((it + NST) % NI) * S::BPC + g], lt, S::G, true);
        // 3D: a child (sx,sy,sz) of coarse cell X gets (1/4)((d0 + d_x(sx)) + (d_y(sy) + d_z(sz))):
        // the 2 x-pair and 4 yz-pair sums of a coarse cell are formed once for its 8 children
        T *PS = st + S::C + 2 * S::QCP;
        if constexpr (D == 3) {
            if (I.b >= 0) {
                for (int c = lt; c < S::N3; c += S::G) {
                    const int X = c % MH, Y = (c / MH) % MH, Z = c / (MH * MH);
                    const int b = ((Z + 1) * Q + (Y + 1)) * Q + (X + 1);
                    const T d0 = DU[b], dym = DU[b - Q], dyp = DU[b + Q], dzm = DU[b - Q * Q], dzp = DU[b + Q * Q];
                    PS[c] = d0 + DU[b - 1];
                    PS[S::N3 + c] = d0 + DU[b + 1];
                    PS[2 * S::N3 + c] = dym + dzm;
                    PS[3 * S::N3 + c] = dym + dzp;
                    PS[4 * S::N3 + c] = dyp + dzm;
                    PS[5 * S::N3 + c] = dyp + dzp;
                }
            }
            __syncthreads();
        }
        if (I.b >= 0) {
#pragma unroll
            for (int itv = 0; itv < S::NIT; ++itv) {
                const int v = lt + itv * S::G;
                if (v >= S::NV) continue;
                // the VEC cells of a half-row vector: colour col, row (j,k), i = 2h + r for
                // h = h0..h0+VEC-1; their coarse cells (h, j/2, k/2) and offsets are shared
                const int col = v / NVH, w = v % NVH;
                const int row = w / NVR, h0 = (w % NVR) * VEC;
                const int j = row % M, k = D == 2 ? 0 : row / M;
                const int r = (col + j + k + D) & 1;
                const int ox = r ? 1 : -1, oy = (j & 1) ? Q : -Q;
                const int b = D == 2 ? ((j >> 1) + 1) * Q + (h0 + 1) : (((k >> 1) + 1) * Q + ((j >> 1) + 1)) * Q + (h0 + 1);
                T uv[VEC], res[VEC];
                ldv<T, VEC>(U + v * VEC, uv);
                if constexpr (D == 3) {
                    const int c0 = ((k >> 1) * MH + (j >> 1)) * MH + h0;
                    const T *px = PS + (r ? S::N3 : 0) + c0;
                    const T *qyz = PS + (2 + 2 * (j & 1) + (k & 1)) * S::N3 + c0;
#pragma unroll
                    for (int e = 0; e < VEC; ++e) res[e] = fma(T(0.25), px[e] + qyz[e], uv[e]);
                    (void)b;
                    (void)ox;
                    (void)oy;
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        const T d0 = DU[b + e], dx = DU[b + e + ox], dy = DU[b + e + oy];
                        res[e] = fma(T(0.25), dx + dy, fma(T(0.5), d0, uv[e]));
                    }
                }
                stv<T, VEC>(u + I.coff + (long long)v * VEC, res);
            }
        }
    }
    cp_wait<0>();
}

// Coarse-grid correction by parent: the 2^D children of a parent are
// consecutive in a level's box range, so one CTA stages the parent P once --
// its u and v' images with their side ghosts, as the whole-box kernels stage
// a box (fp_issue; across a domain side the mirrored inner value) -- forms
// d = v_H - v'_H on the image (negated across a Dirichlet side, the
// homogeneous rule of the correction), in 3D the pair sums of every parent
// cell, and updates all children's cells with the 2-1-1 / 1-1-1-1 scheme
// (the same arithmetic as k_correct_p).  Parents are staged one ahead
// (two-stage ring).
template <int D, int M, typename T>
struct PpCfg {
    using F = FpCfg<D, M, T, kThreads>;
    static constexpr int NC = 1 << D, C = Geo<D, M>::C, VEC = F::VEC, NV = C / VEC;
    static constexpr int IMG = F::UB;                  // one image (u or v') with its ghosts
    static constexpr int PSZ = D == 3 ? 6 * C : 0;     // pair sums of the parent's cells
    static constexpr int NST = 2;
    static constexpr size_t smem() {
        return sizeof(T) * (2 * IMG * NST + PSZ) + sizeof(BoxInfo) * (NST + 1) + sizeof(long long) * NC * (NST + 1);
    }
    // a vector stays inside one half-row, and at least two CTAs fit an SM
    // (3D boxes of 16^3 cells take the per-child kernel)
    static constexpr bool ok = F::ok && smem() <= 113 * 1024;
};

// metadata of parent group q: the parent of boxes b0 + NC q .. b0 + NC q + NC - 1
// and its children's cell offsets
template <int D, int M, typename T>
__device__ __forceinline__ void pp_info_load(const BoxMeta &A, int q, int np, int b0, BoxInfo &I, long long *ccoff,
                                             bool mask) {
    using S = PpCfg<D, M, T>;
    const int lt = threadIdx.x;
    const int b = q < np ? A.parent[b0 + S::NC * q] : -1;
    bool on = b >= 0;
    if (on && mask && A.active && !A.active[A.tree[b]]) on = false;
    if (lt < 2 * D) {
        if (on) {
            I.code[lt] = A.nb[b * 2 * D + lt];
            I.base[lt] = A.nbase[b * 2 * D + lt];
        }
    } else if (lt == 2 * D) {
        I.b = on ? b : -1;
        if (on) {
            I.coff = A.coff[b];
            I.flag = A.bflag[b];
            I.nmask = (I.flag >> BF_NSHIFT) & 0x3f;
        }
    } else if (lt >= 32 && lt < 32 + S::NC) {
        if (on) ccoff[lt - 32] = A.coff[b0 + S::NC * q + (lt - 32)];
    }
}

template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_correct_pp(BoxMeta A, int b0, int n, T *u, const T *__restrict__ vold) {
    using S = PpCfg<D, M, T>;
    using F = typename S::F;
    constexpr int NST = S::NST, NI = NST + 1, MH = M / 2, VEC = S::VEC, NVH = Geo<D, M>::H / VEC, NVR = F::NVR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *stages = reinterpret_cast<T *>(smem_raw);
    T *PS = stages + 2 * S::IMG * NST;
    BoxInfo *info = reinterpret_cast<BoxInfo *>(smem_raw + sizeof(T) * (2 * S::IMG * NST + S::PSZ));
    long long *ccoff = reinterpret_cast<long long *>(info + NI);
    const int lt = threadIdx.x;
    const int np = n / S::NC;
    pdl_trigger();
    for (int q = 0; q < NST; ++q)  // static metadata: before the wait
        pp_info_load<D, M, T>(A, blockIdx.x + q * gridDim.x, np, b0, info[q], ccoff + q * S::NC, false);
    pdl_wait();
    __syncthreads();
    if (lt == 2 * D)
        for (int q = 0; q < NST; ++q)
            if (info[q].b >= 0 && A.active && !A.active[A.tree[info[q].b]]) info[q].b = -1;
    __syncthreads();
    auto issue = [&](int q) {
        const BoxInfo &In = info[q % NI];
        if (In.b >= 0) {
            T *st = stages + (q % NST) * 2 * S::IMG;
            fp_issue<D, M, T, kThreads>(In, u, nullptr, st, lt, true);
            fp_issue<D, M, T, kThreads>(In, vold, nullptr, st + S::IMG, lt, true);
        }
        cp_commit();
    };
    for (int q = 0; q < NST - 1; ++q) issue(q);
    int it = 0;
    for (int base = blockIdx.x; base < np; base += gridDim.x, ++it) {
        cp_wait<NST - 2>();
        __syncthreads();  // the parent's images have landed; the previous stage and slots are free
        const BoxInfo &I = info[it % NI];
        const long long *cc = ccoff + (it % NI) * S::NC;
        T *Dd = stages + (it % NST) * 2 * S::IMG;
        const T *V = Dd + S::IMG;
        issue(it + NST - 1);
        pp_info_load<D, M, T>(A, base + NST * gridDim.x, np, b0, info[(it + NST) % NI], ccoff + ((it + NST) % NI) * S::NC,
                              true);
        const bool on = I.b >= 0;
        if (on)
            for (int e = lt; e < S::IMG; e += kThreads) Dd[e] = Dd[e] - V[e];
        if (on && (I.flag & BF_SPECIAL)) {  // a Dirichlet side: the difference enters as -d
            __syncthreads();
            for (int item = lt; item < F::NGI; item += kThreads) {
                int sd, slot;
                if (item < F::NXI) {
                    int j, k;
                    fp_xitem<D, M>(item, sd, j, k);
                    slot = 2 * F::PT + sd * F::ROWS + sp_row<D, M>(j, k);
                    if (I.code[sd] == -1 && !((I.nmask >> sd) & 1)) Dd[slot] = -Dd[slot];
                } else {
                    int col, h0, jg, kg, jin, kin, jm, km;
                    fp_yzitem<D, M, T>(item - F::NXI, sd, col, h0, jg, kg, jin, kin, jm, km);
                    slot = col * F::PT + sp_row<D, M>(jg, kg) * MH + h0;
                    if (I.code[sd] == -1 && !((I.nmask >> sd) & 1))
#pragma unroll
                        for (int x = 0; x < VEC; ++x) Dd[slot + x] = -Dd[slot + x];
                }
            }
        }
        __syncthreads();
        // d of parent cell (i, j, k), i in [-1, M]: the planes, or the x ghosts
        auto dat = [&](int i, int j, int k) -> T {
            if (i < 0) return Dd[2 * F::PT + sp_row<D, M>(j, k)];
            if (i >= M) return Dd[2 * F::PT + F::ROWS + sp_row<D, M>(j, k)];
            return Dd[fp_slot<D, M, T>(i, j, k)];
        };
        if constexpr (D == 3) {
            if (on)
                for (int c = lt; c < S::C; c += kThreads) {
                    const int X = c % M, Y = (c / M) % M, Z = c / (M * M);
                    const T d0 = dat(X, Y, Z), dym = dat(X, Y - 1, Z), dyp = dat(X, Y + 1, Z);
                    const T dzm = dat(X, Y, Z - 1), dzp = dat(X, Y, Z + 1);
                    PS[c] = d0 + dat(X - 1, Y, Z);
                    PS[S::C + c] = d0 + dat(X + 1, Y, Z);
                    PS[2 * S::C + c] = dym + dzm;
                    PS[3 * S::C + c] = dym + dzp;
                    PS[4 * S::C + c] = dyp + dzm;
                    PS[5 * S::C + c] = dyp + dzp;
                }
            __syncthreads();
        }
        if (on) {
            for (int t = lt; t < S::NC * S::NV; t += kThreads) {
                const int ch = t / S::NV, v = t % S::NV;
                // the child's offset in the parent: bit a of ch is its half along axis a
                const int px = (ch & 1) * MH, py = ((ch >> 1) & 1) * MH, pz = D == 3 ? ((ch >> 2) & 1) * MH : 0;
                const int col = v / NVH, w = v % NVH;
                const int row = w / NVR, h0 = (w % NVR) * VEC;
                const int j = row % M, k = D == 2 ? 0 : row / M;
                const int r = (col + j + k + D) & 1;
                T uv[VEC], res[VEC];
                T *gu = u + cc[ch] + (long long)v * VEC;
                ldv<T, VEC>(gu, uv);
                const int Y = py + (j >> 1), Z = pz + (k >> 1), X0 = px + h0;
                if constexpr (D == 3) {
                    const int c0 = (Z * M + Y) * M + X0;
                    const T *pxs = PS + (r ? S::C : 0) + c0;
                    const T *qyz = PS + (2 + 2 * (j & 1) + (k & 1)) * S::C + c0;
#pragma unroll
                    for (int e = 0; e < VEC; ++e) res[e] = fma(T(0.25), pxs[e] + qyz[e], uv[e]);
                } else {
                    const int sy = (j & 1) ? 1 : -1, sx = r ? 1 : -1;
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        const int X = X0 + e;
                        const T d0 = dat(X, Y, 0), dx = dat(X + sx, Y, 0), dy = dat(X, Y + sy, 0);
                        res[e] = fma(T(0.25), dx + dy, fma(T(0.5), d0, uv[e]));
                    }
                }
                stv<T, VEC>(gu, res);
            }
        }
    }
    cp_wait<0>();
}

}  // namespace afg
