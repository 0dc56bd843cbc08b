// Red-black Gauss-Seidel half-sweep with a half-row shared-memory layout
// (Sec. 3.1 of arXiv:1701.04329), for boxes whose colour half-rows hold at
// least one 16-byte vector (M/2 >= 16/sizeof(T)).
//
// A half-sweep of colour c reads only cells of colour 1-c.  In a row (j,k)
// the cells of one colour sit at i = 2h + r with r fixed per row, so the
// colour 1-c cells of a box plus the ghost cells a colour-c update reads form
// a padded array of half-rows: P[k+1][j+1][A0 + h], h in [-1, M/2], rows
// j, k in [-1, M].  For the VEC colour-c cells h0..h0+VEC-1 of row (j,k),
// with r = (c+j+k+D) & 1:
//   y and z neighbours: half-rows (j+-1,k), (j,k+-1) at h0..h0+VEC-1 (aligned
//   vectors: in those rows the colour 1-c cells sit at the same i);
//   x neighbours: P[h0+r-1 .. h0+r+VEC-1] of row (j,k) (one aligned vector and
//   one scalar).
// Face ghosts arrive as whole half-rows of the same-level neighbour (y, z
// sides) or one value per row (x sides).  Domain-boundary ghosts
// g = 2b - u_1 are completed while gathering (u_1 is read from the box's own
// colour-c half, not yet written); refinement-boundary ghosts
// g = u_H/2 + c1 u_1 - (u_2 + u_t...)/4 (Sec. 3.3) get their u_H/2 + c1 u_1
// part there and the rest after the barrier, from the tile.
#pragma once
#include "kernels.cuh"

namespace afg {

template <int D, int M, typename T>
struct SvCfg {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int MH = M / 2;
    static constexpr int A0 = VEC;                      // aligned start of a half-row
    static constexpr int RS = A0 + MH + VEC;            // half-row stride (elements)
    static constexpr int ROWS = D == 2 ? (M + 2) : (M + 2) * (M + 2);
    static constexpr int TILE = ROWS * RS;              // elements per box
    static constexpr int NVR = MH / VEC;                // vectors per half-row
    static constexpr int FR = D == 2 ? 1 : M;           // half-rows per y/z face
    static constexpr int H = Geo<D, M>::H;
    static constexpr int NV = H / VEC;                  // vectors per colour half
    static constexpr int G = NV < kThreads ? NV : kThreads;
    static constexpr int BPC = kThreads / G;
    static constexpr int NIT = (NV + G - 1) / G;
    static constexpr int NXI = (D == 2 ? M : M * M) / 2;   // x-ghost items per x side
    static constexpr int NGI = 2 * NXI + (2 * D - 2) * FR * NVR;  // ghost items per box
    static constexpr size_t smem() { return sizeof(T) * TILE * BPC + 2 * sizeof(BoxInfo) * BPC; }
    static constexpr bool ok = MH >= VEC;
};

// tile slot of cell (i,j,k) of the tile's colour, ghosts included (i >> 1 is
// the half-row index for either parity; -1 >> 1 = -1)
template <int D, int M, typename T>
__device__ __forceinline__ int sv_idx(int i, int j, int k) {
    using S = SvCfg<D, M, T>;
    const int row = D == 2 ? (j + 1) : (k + 1) * (M + 2) + (j + 1);
    return row * S::RS + S::A0 + (i >> 1);
}

// storage offset, inside a colour half, of the half-row (j,k)
template <int D, int M>
__device__ __forceinline__ int hrow(int j, int k) { return (k * M + j) * (M / 2); }

template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_smooth_v(BoxMeta A, int b0, int n, const int *list, T *u,
                                                       const T *__restrict__ rho, T h2, int colour, int hom) {
    using S = SvCfg<D, M, T>;
    constexpr int VEC = S::VEC, MH = S::MH, H = S::H;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / S::G, lt = threadIdx.x % S::G;
    T *P = reinterpret_cast<T *>(smem_raw) + g * S::TILE;
    BoxInfo *info = reinterpret_cast<BoxInfo *>(smem_raw + sizeof(T) * S::TILE * S::BPC);
    const int c = colour, oc = 1 - colour;
    const T inv = T(1) / T(2 * D);
    const T c1 = D == 2 ? T(1) : T(1.25);
    const int stride = gridDim.x * S::BPC;
    int base = blockIdx.x * S::BPC, buf = 0;
    pdl_trigger();
    info_load<D>(A, base + g, n, b0, list, info[g], lt, S::G, false);  // static metadata: before the wait
    pdl_wait();
    info_mask<D>(A, info[g], lt, S::G);
    __syncthreads();
    for (; base < n; base += stride) {
        const BoxInfo &I = info[buf * S::BPC + g];
        const int b = I.b;
        const bool special = b >= 0 && (I.flag & BF_SPECIAL);
        T rv[S::NIT][VEC];
        if (b >= 0) {
            const T *uo = u + I.coff + oc * H;  // this box's colour 1-c half
            const T *uc = u + I.coff + c * H;   // this box's colour c half (read only for ghosts)
            // interior half-rows of colour 1-c
            for (int v = lt; v < S::NV; v += S::G) {
                const int row = v / S::NVR, h0 = (v % S::NVR) * VEC;
                const int j = row % M, k = D == 2 ? 0 : row / M;
                T e[VEC];
                ldv<T, VEC>(uo + hrow<D, M>(j, k) + h0, e);
                stv<T, VEC>(P + sv_idx<D, M, T>(2 * h0, j, k), e);
            }
#pragma unroll
            for (int it = 0; it < S::NIT; ++it) {
                const int v = lt + it * S::G;
                if (v < S::NV) ldv<T, VEC>(rho + I.coff + c * H + v * VEC, rv[it]);
            }
            // ghosts
            for (int item = lt; item < S::NGI; item += S::G) {
                if (item < 2 * S::NXI) {  // x sides: one value per row
                    const int s = item / S::NXI, ri = item % S::NXI;
                    const int want_r = s;  // -x: rows whose colour-c cell is at i = 0; +x: at i = M-1
                    int j, k;
                    if (D == 2) { k = 0; j = 2 * ri + ((want_r + c + D) & 1); }
                    else { k = ri / MH; j = 2 * (ri % MH) + ((want_r + c + k + D) & 1); }
                    const int code = I.code[s];
                    const int ig = s ? M : -1, iin = s ? M - 1 : 0;
                    T val;
                    if (code >= 0) {
                        val = u[I.base[s] + oc * H + hrow<D, M>(j, k) + (s ? 0 : MH - 1)];
                    } else {
                        const T u1 = uc[hrow<D, M>(j, k) + (iin >> 1)];
                        if (code == -1) {
                            const T bv = hom ? T(0) : T(A.bc[I.base[s] + k * M + j]);
                            val = T(2) * bv - u1;
                        } else {
                            const int cj = unpack_off(I.poff, 1) + (j >> 1);
                            const int ck = D == 3 ? unpack_off(I.poff, 2) + (k >> 1) : 0;
                            const T uH = u[I.base[s] + rbi<D, M>(s ? 0 : M - 1, cj, ck)];
                            val = T(0.5) * uH + c1 * u1;
                        }
                    }
                    P[sv_idx<D, M, T>(ig, j, k)] = val;
                } else {  // y/z sides: whole half-rows
                    const int it2 = item - 2 * S::NXI;
                    const int s = 2 + it2 / (S::FR * S::NVR);
                    const int rem = it2 % (S::FR * S::NVR);
                    const int fr = rem / S::NVR, h0 = (rem % S::NVR) * VEC;
                    const int code = I.code[s];
                    const int hi = s & 1, a = s >> 1;
                    int jg, kg, jin, kin, jm, km;  // ghost row, inner row, mirror row in the neighbour
                    if (a == 1) { kg = kin = km = D == 3 ? fr : 0; jg = hi ? M : -1; jin = hi ? M - 1 : 0; jm = hi ? 0 : M - 1; }
                    else { jg = jin = jm = fr; kg = hi ? M : -1; kin = hi ? M - 1 : 0; km = hi ? 0 : M - 1; }
                    T e[VEC];
                    if (code >= 0) {
                        ldv<T, VEC>(u + I.base[s] + oc * H + hrow<D, M>(jm, km) + h0, e);
                    } else {
                        T u1v[VEC];
                        ldv<T, VEC>(uc + hrow<D, M>(jin, kin) + h0, u1v);
                        const int rg = (c + jin + kin + D) & 1;  // i-parity of the colour-c cells of the inner row
#pragma unroll
                        for (int x = 0; x < VEC; ++x) {
                            const int i = 2 * (h0 + x) + rg;
                            if (code == -1) {
                                const int t2 = a == 1 ? kin : jin;  // tangential coordinates (x first)
                                const T bv = hom ? T(0) : T(A.bc[I.base[s] + t2 * M + i]);
                                e[x] = T(2) * bv - u1v[x];
                            } else {
                                const int ci = unpack_off(I.poff, 0) + (i >> 1);
                                int cj, ck;
                                if (a == 1) { cj = hi ? 0 : M - 1; ck = D == 3 ? unpack_off(I.poff, 2) + (kin >> 1) : 0; }
                                else { cj = unpack_off(I.poff, 1) + (jin >> 1); ck = hi ? 0 : M - 1; }
                                const T uH = u[I.base[s] + rbi<D, M>(ci, cj, ck)];
                                e[x] = T(0.5) * uH + c1 * u1v[x];
                            }
                        }
                    }
                    stv<T, VEC>(P + sv_idx<D, M, T>(2 * h0, jg, kg), e);
                }
            }
        }
        info_load<D>(A, base + stride + g, n, b0, list, info[(buf ^ 1) * S::BPC + g], lt, S::G);
        __syncthreads();
        // refinement-boundary ghosts: subtract (u_2 + u_t1 [+ u_t2]) / 4 from the tile
        if (special) {
            for (int s = 0; s < 2 * D; ++s) {
                if (I.code[s] > -2) continue;
                const int hi = s & 1, a = s >> 1;
                const int pin = hi ? M - 1 : 0, pg = hi ? M : -1, p2 = hi ? M - 2 : 1;
                for (int f = lt; f < Geo<D, M>::F / 2; f += S::G) {
                    int t1, t2;
                    face_cell<D, M>(f, c, pin, t1, t2);
                    int i, j, k;
                    face_pos(D, s, pg, t1, t2, i, j, k);
                    const int gidx = sv_idx<D, M, T>(i, j, k);
                    face_pos(D, s, p2, t1, t2, i, j, k);
                    T acc = P[sv_idx<D, M, T>(i, j, k)];
                    face_pos(D, s, pin, t1 ^ 1, t2, i, j, k);
                    acc += P[sv_idx<D, M, T>(i, j, k)];
                    if (D == 3) {
                        face_pos(D, s, pin, t1, t2 ^ 1, i, j, k);
                        acc += P[sv_idx<D, M, T>(i, j, k)];
                    }
                    P[gidx] -= T(0.25) * acc;
                    (void)a;
                }
            }
        }
        __syncthreads();
        if (b >= 0) {
#pragma unroll
            for (int it = 0; it < S::NIT; ++it) {
                const int v = lt + it * S::G;
                if (v >= S::NV) continue;
                const int row = v / S::NVR, h0 = (v % S::NVR) * VEC;
                const int j = row % M, k = D == 2 ? 0 : row / M;
                const int r = (c + j + k + D) & 1;
                const T *pr = P + sv_idx<D, M, T>(2 * h0, j, k);
                T xv[VEC], ym[VEC], yp[VEC], zm[VEC], zp[VEC];
                ldv<T, VEC>(pr, xv);
                const T extra = r ? pr[VEC] : pr[-1];
                ldv<T, VEC>(pr - S::RS, ym);
                ldv<T, VEC>(pr + S::RS, yp);
                if (D == 3) {
                    ldv<T, VEC>(pr - (M + 2) * S::RS, zm);
                    ldv<T, VEC>(pr + (M + 2) * S::RS, zp);
                }
                T out[VEC];
#pragma unroll
                for (int x = 0; x < VEC; ++x) {
                    const T xl = r ? xv[x] : (x ? xv[x - 1] : extra);
                    const T xr = r ? (x + 1 < VEC ? xv[x + 1] : extra) : xv[x];
                    T s = (xl + xr) + (ym[x] + yp[x]);
                    if (D == 3) s += zm[x] + zp[x];
                    out[x] = (s - h2 * rv[it][x]) * inv;
                }
                stv<T, VEC>(u + I.coff + c * H + v * VEC, out);
            }
        }
        buf ^= 1;
        __syncthreads();
    }
}

}  // namespace afg
