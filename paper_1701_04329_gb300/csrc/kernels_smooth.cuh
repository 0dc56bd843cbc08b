// Red-black Gauss-Seidel half-sweep (Sec. 3.1 of arXiv:1701.04329) with a
// half-row shared-memory layout and cp.async staging, for boxes whose colour
// half-rows hold at least one 16-byte vector (M/2 >= 16/sizeof(T)).  Used for
// FP32 data; FP64 keeps the table-driven k_smooth, whose FP64 arithmetic is
// the limit there.
//
// A half-sweep of colour c reads only cells of colour 1-c.  In a row (j,k)
// the cells of one colour sit at i = 2h + r with r fixed per row, so the
// colour 1-c cells of a box plus the ghost cells a colour-c update reads form
// an array of half-rows P[k+1][j+1][h], h in [0, M/2), rows j, k in [-1, M],
// plus the x-side ghosts X[side][row].  For the VEC colour-c cells
// h0..h0+VEC-1 of row (j,k), with r = (c+j+k+D) & 1:
//   y and z neighbours: half-rows (j+-1,k), (j,k+-1) at h0..h0+VEC-1 (in those
//   rows the colour 1-c cells sit at the same i);
//   x neighbours: half-row (j,k) at h0+r-1 .. h0+r+VEC-1 (one vector and one
//   scalar, the scalar from X at the ends of the row).
//
// The colour 1-c half-rows, the colour-c source values and the ghost layer of
// a box are copied global -> shared with cp.async into a ring of NST stages,
// so the copies of the next box of a group are in flight while the current
// one is relaxed.  Same-level ghosts are plain copies of the neighbour's
// half-rows (y, z sides) or values (x sides).  Ghosts of domain-boundary and
// refinement-boundary faces are staged as the adjacent inner value u_1 and
// completed after the wait: g = 2b - u_1 (Dirichlet) or
// g = u_H/2 + c1 u_1 - (u_2 + u_t1 [+ u_t2])/4 (Sec. 3.3).  Within a colour-c
// half-sweep no box writes what another box's copies read (colour 1-c
// halves, coarse data, the box's own colour-c half before its own update),
// so staging ahead is safe.
#pragma once
#include "kernels.cuh"

namespace afg {

// storage offset, inside a colour half, of the half-row (j,k)
template <int D, int M>
__device__ __forceinline__ int hrow(int j, int k) { return (k * M + j) * (M / 2); }

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES)
                     : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// VPT: 16-byte vectors of a box's colour half per thread (1: one thread per
// vector; 2: half as many threads per box, twice the boxes per CTA)
template <int D, int M, typename T, int VPT = 1>
struct SpCfg {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int MH = M / 2;
    static constexpr int ROWS = D == 2 ? (M + 2) : (M + 2) * (M + 2);
    static constexpr int PT = ROWS * MH;     // colour 1-c half-rows, interior and y/z ghost rows
    static constexpr int XT = 2 * ROWS;      // x-side ghosts [side][row]
    static constexpr int H = Geo<D, M>::H;
    static constexpr int BOX = PT + XT + H;  // + colour-c source values
    static constexpr int NVR = MH / VEC;
    static constexpr int FR = D == 2 ? 1 : M;
    static constexpr int NV = H / VEC;
    static constexpr int G = (NV / VPT > 0 ? NV / VPT : 1) < kThreads ? (NV / VPT > 0 ? NV / VPT : 1) : kThreads;
    static constexpr int BPC = kThreads / G;
    static constexpr int NIT = (NV + G - 1) / G;
    static constexpr int NXI = (D == 2 ? M : M * M) / 2;
    static constexpr int NGI = 2 * NXI + (2 * D - 2) * FR * NVR;
    static constexpr int NST = 2;  // more stages cost resident CTAs and measured slower
    static constexpr size_t smem() { return sizeof(T) * BOX * BPC * NST + sizeof(BoxInfo) * BPC * (NST + 1); }
    static constexpr bool ok = MH >= VEC;
};

// padded row of (j,k), ghost rows included
template <int D, int M>
__device__ __forceinline__ int sp_row(int j, int k) { return D == 2 ? (j + 1) : (k + 1) * (M + 2) + (j + 1); }

// x-side ghost item -> side and row (rows whose colour-c cell touches side s)
template <int D, int M>
__device__ __forceinline__ void sp_xitem(int item, int c, int &s, int &j, int &k) {
    constexpr int MH = M / 2, NXI = (D == 2 ? M : M * M) / 2;
    s = item / NXI;
    const int ri = item % NXI;
    if (D == 2) { k = 0; j = 2 * ri + ((s + c + D) & 1); }
    else { k = ri / MH; j = 2 * (ri % MH) + ((s + c + k + D) & 1); }
}

// y/z-side ghost item -> side, vector start, ghost row, inner row, mirror row in the neighbour
template <int D, int M, typename T>
__device__ __forceinline__ void sp_yzitem(int it2, int &s, int &h0, int &jg, int &kg, int &jin, int &kin, int &jm,
                                          int &km) {
    using S = SpCfg<D, M, T>;
    s = 2 + it2 / (S::FR * S::NVR);
    const int rem = it2 % (S::FR * S::NVR);
    const int fr = rem / S::NVR;
    h0 = (rem % S::NVR) * S::VEC;
    const int hi = s & 1;
    if ((s >> 1) == 1) { kg = kin = km = D == 3 ? fr : 0; jg = hi ? M : -1; jin = hi ? M - 1 : 0; jm = hi ? 0 : M - 1; }
    else { jg = jin = jm = fr; kg = hi ? M : -1; kin = hi ? M - 1 : 0; km = hi ? 0 : M - 1; }
}

// Per-thread copy plan, the same for every box of a launch (fixed colour):
// for each ghost item of the thread, the destination in the box's stage, the
// side, whether it is a scalar (x side), and the source offsets relative to
// the neighbour box (same-level copy) and to the box's own colour-c half (u_1).
template <int D, int M, typename T, int VPT = 1>
struct SpPlan {
    using S = SpCfg<D, M, T, VPT>;
    static constexpr int NQ = (S::NGI + S::G - 1) / S::G;
    int gdst[NQ], gsrc[NQ];  // dst | side << 16 | scalar << 19 ; nb offset | u1 offset << 16
    int gbc[NQ];             // boundary data of the item's first face (stride 2 along a y/z item's vector)
    int vdst[S::NIT], vsrc[S::NIT];
    __device__ __forceinline__ void init(int lt, int c) {
        constexpr int MH = S::MH, H = S::H;
#pragma unroll
        for (int it = 0; it < S::NIT; ++it) {
            const int v = lt + it * S::G;
            const int row = v / S::NVR, h0 = (v % S::NVR) * S::VEC;
            const int j = row % M, k = D == 2 ? 0 : row / M;
            vdst[it] = sp_row<D, M>(j, k) * MH + h0;
            vsrc[it] = hrow<D, M>(j, k) + h0;
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int item = lt + q * S::G;
            gdst[q] = -1;
            gsrc[q] = 0;
            gbc[q] = 0;
            if (item >= S::NGI) continue;
            if (item < 2 * S::NXI) {
                int sd, j, k;
                sp_xitem<D, M>(item, c, sd, j, k);
                gbc[q] = k * M + j;
                gdst[q] = (S::PT + sd * S::ROWS + sp_row<D, M>(j, k)) | (sd << 16) | (1 << 19);
                gsrc[q] = ((1 - c) * H + hrow<D, M>(j, k) + (sd ? 0 : MH - 1)) | ((hrow<D, M>(j, k) + (sd ? MH - 1 : 0)) << 16);
            } else {
                int sd, h0, jg, kg, jin, kin, jm, km;
                sp_yzitem<D, M, T>(item - 2 * S::NXI, sd, h0, jg, kg, jin, kin, jm, km);
                const int rg = (c + jin + kin + D) & 1;  // i-parity of the colour-c cells of the inner row
                gbc[q] = ((sd >> 1) == 1 ? kin : jin) * M + 2 * h0 + rg;
                gdst[q] = (sp_row<D, M>(jg, kg) * MH + h0) | (sd << 16);
                gsrc[q] = ((1 - c) * H + hrow<D, M>(jm, km) + h0) | ((hrow<D, M>(jin, kin) + h0) << 16);
            }
        }
    }
};

template <int D, int M, typename T, int VPT>
__device__ __forceinline__ void sp_issue(const SpPlan<D, M, T, VPT> &pl, const BoxInfo &I, const T *u, const T *rho,
                                         T *box, int lt, int c) {
    using S = SpCfg<D, M, T, VPT>;
    constexpr int VEC = S::VEC, H = S::H;
    const T *uo = u + I.coff + (1 - c) * H, *uc = u + I.coff + c * H;
    T *R = box + S::PT + S::XT;
#pragma unroll
    for (int it = 0; it < S::NIT; ++it) {
        const int v = lt + it * S::G;
        if (v >= S::NV) continue;
        cp_async<16>(box + pl.vdst[it], uo + pl.vsrc[it]);
        cp_async<16>(R + v * VEC, rho + I.coff + c * H + v * VEC);
    }
#pragma unroll
    for (int q = 0; q < SpPlan<D, M, T, VPT>::NQ; ++q) {
        const int dst = pl.gdst[q];
        if (dst < 0) continue;
        const int sd = (dst >> 16) & 7;
        const T *src = I.code[sd] >= 0 ? u + I.base[sd] + (pl.gsrc[q] & 0xffff) : uc + (pl.gsrc[q] >> 16);
        if (dst & (1 << 19)) cp_async<(int)sizeof(T)>(box + (dst & 0xffff), src);
        else cp_async<16>(box + (dst & 0xffff), src);
    }
}

// Completes the domain-side ghosts among this thread's own items from the
// u_1 it staged there (visible to it after its own wait, before the box's
// barrier): 2 b - u_1 (Dirichlet) or u_1 + h b (Neumann).
template <int D, int M, typename T, int VPT>
__device__ __forceinline__ void sp_fix_own(const SpPlan<D, M, T, VPT> &pl, const BoxInfo &I, const BoxMeta &A, T *box,
                                           int hom) {
    using S = SpCfg<D, M, T, VPT>;
    constexpr int VEC = S::VEC;
#pragma unroll
    for (int q = 0; q < SpPlan<D, M, T, VPT>::NQ; ++q) {
        const int dst = pl.gdst[q];
        if (dst < 0) continue;
        const int sd = (dst >> 16) & 7;
        if (I.code[sd] != -1) continue;
        const bool neu = (I.nmask >> sd) & 1;
        const T hbox = neu ? T(A.hb[I.b]) : T(0);
        const double *bc = A.bc + I.base[sd] + pl.gbc[q];
        T *gv = box + (dst & 0xffff);
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

// completes the ghosts of non-copy faces from the staged u_1 (cf_only: the
// refinement-boundary faces only, the domain sides being done by sp_fix_own)
template <int D, int M, typename T, int VPT = 1>
__device__ __forceinline__ void sp_fix(const BoxInfo &I, const BoxMeta &A, const T *u, T *box, int lt, int c,
                                       int hom, bool cf_only = false) {
    using S = SpCfg<D, M, T, VPT>;
    constexpr int VEC = S::VEC, MH = S::MH;
    T *P = box, *X = box + S::PT;
    const T c1 = D == 2 ? T(1) : T(1.25);
    // interior cell (i,j,k) of colour 1-c
    auto at = [&](int i, int j, int k) -> T { return P[sp_row<D, M>(j, k) * MH + (i >> 1)]; };
    for (int item = lt; item < S::NGI; item += S::G) {
        if (item < 2 * S::NXI) {
            int s, j, k;
            sp_xitem<D, M>(item, c, s, j, k);
            const int code = I.code[s];
            if (code >= 0 || (cf_only && code == -1)) continue;
            T &gv = X[s * S::ROWS + sp_row<D, M>(j, k)];
            const T u1 = gv;
            if (code == -1) {
                if ((I.nmask >> s) & 1) continue;  // Neumann: the pass below
                const T bv = hom ? T(0) : T(A.bc[I.base[s] + k * M + j]);
                gv = T(2) * bv - u1;
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
            int s, h0, jg, kg, jin, kin, jm, km;
            sp_yzitem<D, M, T>(item - 2 * S::NXI, s, h0, jg, kg, jin, kin, jm, km);
            const int code = I.code[s];
            if (code >= 0 || (cf_only && code == -1)) continue;
            const int hi = s & 1, a = s >> 1;
            T *gv = P + sp_row<D, M>(jg, kg) * MH + h0;
            const int rg = (c + jin + kin + D) & 1;  // i-parity of the colour-c cells of the inner row
            const int p2 = hi ? M - 2 : 1;
#pragma unroll
            for (int x = 0; x < VEC; ++x) {
                const int i = 2 * (h0 + x) + rg;
                const T u1 = gv[x];
                if (code == -1) {
                    const int t2 = a == 1 ? kin : jin;
                    if ((I.nmask >> s) & 1) continue;  // Neumann: the pass below
                    const T bv = hom ? T(0) : T(A.bc[I.base[s] + t2 * M + i]);
                    gv[x] = T(2) * bv - u1;
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
    if (!I.nmask || cf_only) return;
    // Neumann domain sides: g = u_1 + h b (a separate pass keeps the common path lean)
    const T hbox = T(A.hb[I.b]);
    for (int item = lt; item < S::NGI; item += S::G) {
        if (item < 2 * S::NXI) {
            int s, j, k;
            sp_xitem<D, M>(item, c, s, j, k);
            if (I.code[s] != -1 || !((I.nmask >> s) & 1)) continue;
            T &gv = X[s * S::ROWS + sp_row<D, M>(j, k)];
            const T bv = hom ? T(0) : T(A.bc[I.base[s] + k * M + j]);
            gv = fma(hbox, bv, gv);
        } else {
            int s, h0, jg, kg, jin, kin, jm, km;
            sp_yzitem<D, M, T>(item - 2 * S::NXI, s, h0, jg, kg, jin, kin, jm, km);
            if (I.code[s] != -1 || !((I.nmask >> s) & 1)) continue;
            T *gv = P + sp_row<D, M>(jg, kg) * MH + h0;
            const int rg = (c + jin + kin + D) & 1;
            const int t2 = (s >> 1) == 1 ? kin : jin;
#pragma unroll
            for (int x = 0; x < VEC; ++x) {
                const int i = 2 * (h0 + x) + rg;
                const T bv = hom ? T(0) : T(A.bc[I.base[s] + t2 * M + i]);
                gv[x] = fma(hbox, bv, gv[x]);
            }
        }
    }
}

// resident blocks per SM the register allocation must allow (FP32 / FP64)
constexpr int kSmoothMinBlocks32 = 6, kSmoothMinBlocks64 = 5;

// scaled = 1: rho holds -h^2 rho / (2D) and the update is u = sum/(2D) + rho
template <int D, int M, typename T, int VPT = 1>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? kSmoothMinBlocks32 : kSmoothMinBlocks64) k_smooth_p(BoxMeta A, int b0, int n, const int *list, T *u,
                                                       const T *__restrict__ rho, T h2, int colour, int hom,
                                                       int scaled) {
    using S = SpCfg<D, M, T, VPT>;
    constexpr int VEC = S::VEC, MH = S::MH, H = S::H, NST = S::NST, NI = NST + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / S::G, lt = threadIdx.x % S::G;
    T *stages = reinterpret_cast<T *>(smem_raw);
    BoxInfo *info = reinterpret_cast<BoxInfo *>(smem_raw + sizeof(T) * S::BOX * S::BPC * NST);
    const int c = colour;
    const T inv = T(1) / T(2 * D);
    const int stride = gridDim.x * S::BPC;
    const int first = blockIdx.x * S::BPC;
    SpPlan<D, M, T, VPT> pl;
    pl.init(lt, c);
    // per vector of this thread, the same for every box: the stage offset of
    // the x neighbour past the vector (half-row or x ghost) and the parity of
    // its row (the vector's own half-row is at pl.vdst)
    int cxoff[S::NIT];
    bool cr[S::NIT];
#pragma unroll
    for (int itv = 0; itv < S::NIT; ++itv) {
        const int v = lt + itv * S::G;
        const int row = v / S::NVR, h0 = (v % S::NVR) * VEC;
        const int j = row % M, k = D == 2 ? 0 : row / M;
        const int r = (c + j + k + D) & 1;
        const int pr_row = sp_row<D, M>(j, k);
        if (r) cxoff[itv] = h0 + VEC < MH ? pr_row * MH + h0 + VEC : S::PT + S::ROWS + pr_row;
        else cxoff[itv] = h0 > 0 ? pr_row * MH + h0 - 1 : S::PT + pr_row;
        cr[itv] = r;
    }
    pdl_trigger();
    for (int q = 0; q < NST; ++q)  // static metadata: before the wait
        info_load<D>(A, first + q * stride + g, n, b0, list, info[q * S::BPC + g], lt, S::G, false);
    pdl_wait();
    for (int q = 0; q < NST; ++q) info_mask<D>(A, info[q * S::BPC + g], lt, S::G);
    __syncthreads();
    for (int q = 0; q < NST - 1; ++q) {
        const BoxInfo &In = info[q * S::BPC + g];
        if (In.b >= 0) sp_issue<D, M, T, VPT>(pl, In, u, rho, stages + (q * S::BPC + g) * S::BOX, lt, c);
        cp_commit();
    }
    int it = 0;
    for (int base = first; base < n; base += stride, ++it) {
        cp_wait<NST - 2>();  // this box's copies (issued NST-1 boxes ago) have landed
        const BoxInfo &I = info[(it % NI) * S::BPC + g];
        const int b = I.b;
        const bool special = b >= 0 && (I.flag & BF_SPECIAL);
        const bool cf = b >= 0 && (I.flag & BF_CF);
        T *box = stages + ((it % NST) * S::BPC + g) * S::BOX;
        if (special) sp_fix_own<D, M, T, VPT>(pl, I, A, box, hom);  // domain sides: this thread's own items
        // one barrier per box: the stage and metadata slot of the previous box are free after it
        const int any_cf = __syncthreads_or(cf);
        {
            const int q = it + NST - 1;
            const BoxInfo &In = info[(q % NI) * S::BPC + g];
            if (In.b >= 0) sp_issue<D, M, T, VPT>(pl, In, u, rho, stages + ((q % NST) * S::BPC + g) * S::BOX, lt, c);
            cp_commit();
        }
        info_load<D>(A, base + NST * stride + g, n, b0, list, info[((it + NST) % NI) * S::BPC + g], lt, S::G);
        if (any_cf) {  // refinement-boundary ghosts read cells other threads staged
            if (cf) sp_fix<D, M, T, VPT>(I, A, u, box, lt, c, hom, true);
            __syncthreads();
        }
        if (b >= 0) {
            const T *R = box + S::PT + S::XT;
#pragma unroll
            for (int itv = 0; itv < S::NIT; ++itv) {
                if (lt + itv * S::G >= S::NV) continue;
                const T *pr = box + pl.vdst[itv];  // the vector's colour 1-c half-row
                T xv[VEC], ym[VEC], yp[VEC], zm[VEC], zp[VEC], rv[VEC];
                ldv<T, VEC>(pr, xv);
                const T extra = box[cxoff[itv]];
                ldv<T, VEC>(pr - MH, ym);
                ldv<T, VEC>(pr + MH, yp);
                if (D == 3) {
                    ldv<T, VEC>(pr - (M + 2) * MH, zm);
                    ldv<T, VEC>(pr + (M + 2) * MH, zp);
                }
                ldv<T, VEC>(R + (lt + itv * S::G) * VEC, rv);
                const bool r = cr[itv];
                T out[VEC];
#pragma unroll
                for (int x = 0; x < VEC; ++x) {
                    // the x neighbours: the cell's own half-row entry and the one beside it
                    // (towards +x for r = 1, towards -x for r = 0; `extra` past the vector)
                    const T side = r ? (x + 1 < VEC ? xv[x + 1] : extra) : (x ? xv[x - 1] : extra);
                    const T sum = nb_sum6<D, T>(xv[x], side, ym[x], yp[x], D == 3 ? zm[x] : T(0), D == 3 ? zp[x] : T(0));
                    out[x] = scaled ? fma(sum, inv, rv[x]) : (sum - h2 * rv[x]) * inv;
                }
                stv<T, VEC>(u + I.coff + c * H + (lt + itv * S::G) * VEC, out);
            }
        }
    }
    cp_wait<0>();
}

}  // namespace afg
