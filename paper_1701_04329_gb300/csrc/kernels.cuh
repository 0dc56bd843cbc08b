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
//   bflag[b]     bits 2..7: Neumann domain sides (bit 2 + s)
//   bflag[b]     bit 0: refined (values are FAS coarse values); bit 1: has a
//                side that is not a same-level neighbour
//   tree[b]      tree of the box (batched forests); active[tree] masks trees
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "fxsum.cuh"

namespace afg {

constexpr int kThreads = 256;

// Programmatic dependent launch: every kernel lets the next launch start
// early (pdl_trigger) and waits for its predecessors to finish and their
// memory to be visible (pdl_wait) before reading anything a kernel wrote.
// Box metadata is written only by host uploads, so prologues may read it.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
constexpr unsigned char BF_REFINED = 1, BF_SPECIAL = 2;
constexpr int BF_NSHIFT = 2;  // flag bits 2..7: Neumann domain sides (bit 2 + s)
// BoxInfo::flag bits 8..13 (not in the per-box byte): refinement-boundary sides (bit 8 + s)
constexpr int BF_CF = 0x3f00;

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
    const long long *nbase;  // per side: cells of the neighbour / coarse box, or Dirichlet data offset
    const double *ih2;       // 1/h^2 of every box (an FP64 division costs ~11 FP64-pipe instructions)
    const unsigned char *nmask;  // bit s: side s is a Neumann domain boundary (ghost u + h b, not 2 b - u)
    const double *x0;        // lower x coordinate of every box (the radius in (r,z) coordinates)
    const unsigned char *cfmask;  // bit s: side s is a refinement boundary (a coarser neighbour)
};

// Metadata of one box, prefetched into shared memory one box ahead.
struct BoxInfo {
    long long coff;
    long long base[6];
    int code[6];
    int b, flag, poff, parent;
    long long pcoff;  // cells of the parent (k_correct)
    int nmask;        // Neumann domain sides (of the parent in k_correct)
};

// The activity mask is written by kernels: after pdl_wait, drop a prefetched
// box whose tree is masked out.
// (run by the thread that wrote I.b in info_load, so no barrier is needed)
template <int D>
__device__ __forceinline__ void info_mask(const BoxMeta &A, BoxInfo &I, int lt, int G) {
    if (lt == (2 * D) % G && A.active && I.b >= 0 && !A.active[A.tree[I.b]]) I.b = -1;
}

// Loads the metadata of entry `idx` of a level range (b0 + idx) or list.
// Threads lt, lt+G, ... of the box's group share the work; b = -1 marks an
// empty slot (past the end, or a masked tree).
template <int D>
__device__ __forceinline__ void info_load(const BoxMeta &A, int idx, int n, int b0, const int *list, BoxInfo &I,
                                          int lt, int G, bool mask = true) {
    for (int x = lt; x <= 2 * D; x += G) {
        int b = -1;
        if (idx < n) b = list ? list[idx] : b0 + idx;
        if (x < 2 * D) {
            if (b >= 0) {
                I.code[x] = A.nb[b * 2 * D + x];
                I.base[x] = A.nbase[b * 2 * D + x];
            }
        } else {
            if (mask && b >= 0 && A.active && !A.active[A.tree[b]]) b = -1;
            I.b = b;
            if (b >= 0) {
                I.coff = A.coff[b];
                I.flag = A.bflag[b] | (A.cfmask[b] << 8);
                I.poff = A.poff[b];
                I.parent = A.parent[b];
                I.nmask = (I.flag >> BF_NSHIFT) & 0x3f;
            }
        }
    }
}

template <typename T, int VEC>
struct VecT;
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<float, 2> { using type = float2; };
template <> struct VecT<float, 1> { using type = float; };
template <> struct VecT<double, 2> { using type = double2; };
template <> struct VecT<double, 1> { using type = double; };

template <typename T, int VEC>
__device__ __forceinline__ void ldv(const T *__restrict__ p, T *out) {
    using V = typename VecT<T, VEC>::type;
    const V v = *reinterpret_cast<const V *>(p);
    const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
    for (int i = 0; i < VEC; ++i) out[i] = e[i];
}

template <typename T, int VEC>
__device__ __forceinline__ void stv(T *p, const T *in) {
    using V = typename VecT<T, VEC>::type;
    V v;
    T *e = reinterpret_cast<T *>(&v);
#pragma unroll
    for (int i = 0; i < VEC; ++i) e[i] = in[i];
    *reinterpret_cast<V *>(p) = v;
}

template <typename T, int H>
constexpr int vec_of() { return (16 / (int)sizeof(T)) < H ? 16 / (int)sizeof(T) : H; }

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

// face cell f of a side: all cells (only < 0) or the half whose interior
// neighbour has colour `only` (a checkerboard of the face)
template <int D, int M>
__device__ __forceinline__ void face_cell(int f, int only, int pin, int &t1, int &t2) {
    if (only < 0) {
        t1 = f % M;
        t2 = D == 3 ? f / M : 0;
    } else {
        t2 = D == 3 ? f / (M / 2) : 0;
        const int h1 = D == 3 ? f % (M / 2) : f;
        t1 = 2 * h1 + ((only + pin + t2 + D) & 1);
    }
}

// ---------------------------------------------------------------------------
// Box staging.  gather() issues every global load of a box at once: the
// interior colour halves as 16-byte vectors, and the side ghosts of all
// sides together -- the neighbour's face cell (same level), the Dirichlet
// value b (domain boundary) or the coarse value u_H (refinement boundary).
// finalize(), after a barrier, turns the last two into ghost values with
// the box's own cells (Sec. 2.4 and the default scheme of Sec. 3.3):
//   Dirichlet:           g = 2 b - u_1
//   refinement boundary: 2D g = u_H/2 + u_1 - (u_t + u_2)/4
//                        3D g = u_H/2 + 5/4 u_1 - (u_2 + u_t1 + u_t2)/4
// `only` < 0: all side ghosts; otherwise only the ghosts next to interior
// cells of colour `only` (all a half-sweep of that colour reads).
// ---------------------------------------------------------------------------
// Index tables of a CTA (built once per launch in shared memory):
//   tix[q]      tile index of storage position q (both colours)
//   gt[item]    tile slot of ghost item (side s, face cell f) for the launch's `only`
//   gs[item]    storage index, in the same-level neighbour, of that ghost's source cell
template <int D, int M>
struct Tables {
    static constexpr int C = Geo<D, M>::C, F = Geo<D, M>::F;
    static constexpr size_t bytes() { return sizeof(short) * (C + 2 * 2 * D * F); }
};

template <int D, int M>
__device__ __forceinline__ void build_tables(short *tix, short *gt, short *gs, int only) {
    constexpr int C = Geo<D, M>::C, F = Geo<D, M>::F;
    for (int q = threadIdx.x; q < C; q += blockDim.x) {
        int i, j, k;
        rb_cell<D, M>(q, i, j, k);
        tix[q] = (short)ti<D, M>(i, j, k);
    }
    const int nf = only < 0 ? F : F / 2;
    for (int item = threadIdx.x; item < 2 * D * nf; item += blockDim.x) {
        const int s = item / nf, f = item - s * nf;
        const int hi = s & 1;
        int t1, t2;
        face_cell<D, M>(f, only, hi ? M - 1 : 0, t1, t2);
        int i, j, k;
        face_pos(D, s, hi ? M : -1, t1, t2, i, j, k);
        gt[item] = (short)ti<D, M>(i, j, k);
        face_pos(D, s, hi ? 0 : M - 1, t1, t2, i, j, k);
        gs[item] = (short)rbi<D, M>(i, j, k);
    }
}

// ---------------------------------------------------------------------------
// Box staging.  gather() issues every global load of a box at once: the
// interior colour halves as 16-byte vectors, and the side ghosts of all
// sides together -- the neighbour's face cell (same level), the Dirichlet
// value b (domain boundary) or the coarse value u_H (refinement boundary).
// finalize(), after a barrier, turns the last two into ghost values with
// the box's own cells (Sec. 2.4 and the default scheme of Sec. 3.3):
//   Dirichlet:           g = 2 b - u_1
//   refinement boundary: 2D g = u_H/2 + u_1 - (u_t + u_2)/4
//                        3D g = u_H/2 + 5/4 u_1 - (u_2 + u_t1 + u_t2)/4
// `only` < 0: all side ghosts; otherwise only the ghosts next to interior
// cells of colour `only` (all a half-sweep of that colour reads).
// ---------------------------------------------------------------------------
template <int D, int M, typename T, int G>
__device__ __forceinline__ void gather(const BoxInfo &I, const T *__restrict__ u, const double *__restrict__ bc,
                                       T *tile, int lt, int only, bool own, int hom, const short *tix,
                                       const short *gt, const short *gs) {
    constexpr int C = Geo<D, M>::C, H = Geo<D, M>::H, F = Geo<D, M>::F;
    constexpr int VEC = vec_of<T, H>();
    const int q0 = (only < 0 || own) ? 0 : (1 - only) * H;
    const int q1 = (only < 0 || own) ? C : (2 - only) * H;
    for (int v = q0 / VEC + lt; v < q1 / VEC; v += G) {
        T e[VEC];
        ldv<T, VEC>(u + I.coff + (long long)v * VEC, e);
#pragma unroll
        for (int x = 0; x < VEC; ++x) tile[tix[v * VEC + x]] = e[x];
    }
    const int nf = only < 0 ? F : F / 2;
    for (int item = lt; item < 2 * D * nf; item += G) {
        const int s = item / nf;
        const int code = I.code[s];
        const long long base = I.base[s];
        T v;
        if (code >= 0) {
            v = u[base + gs[item]];
        } else {
            const int f = item - s * nf;
            const int hi = s & 1, a = s >> 1;
            int t1, t2;
            face_cell<D, M>(f, only, hi ? M - 1 : 0, t1, t2);
            if (code == -1) {
                v = hom ? T(0) : T(bc[base + t2 * M + t1]);
            } else {
                const int ta1 = a == 0 ? 1 : 0, ta2 = a == 2 ? 1 : 2;
                const int c1 = unpack_off(I.poff, ta1) + (t1 >> 1);
                const int c2 = D == 3 ? unpack_off(I.poff, ta2) + (t2 >> 1) : 0;
                int ci, cj, ck;
                face_pos(D, s, hi ? 0 : M - 1, c1, c2, ci, cj, ck);
                v = u[base + rbi<D, M>(ci, cj, ck)];
            }
        }
        tile[gt[item]] = v;
    }
}

template <int D, int M, typename T, int G>
__device__ __forceinline__ void finalize(const BoxInfo &I, T *tile, int lt, int only, const double *hb) {
    constexpr int F = Geo<D, M>::F;
    const int nf = only < 0 ? F : F / 2;
    for (int item = lt; item < 2 * D * nf; item += G) {
        const int s = item / nf, f = item - s * nf;
        const int code = I.code[s];
        if (code >= 0) continue;
        const int hi = s & 1;
        const int pin = hi ? M - 1 : 0, pg = hi ? M : -1, p2 = hi ? M - 2 : 1;
        int t1, t2;
        face_cell<D, M>(f, only, pin, t1, t2);
        int i, j, k;
        face_pos(D, s, pg, t1, t2, i, j, k);
        const int gidx = ti<D, M>(i, j, k);
        face_pos(D, s, pin, t1, t2, i, j, k);
        const T u1 = tile[ti<D, M>(i, j, k)];
        if (code == -1) {  // the slot holds b: Dirichlet 2b - u_1, Neumann u_1 + h b
            tile[gidx] = ((I.nmask >> s) & 1) ? fma(T(hb[I.b]), tile[gidx], u1) : T(2) * tile[gidx] - u1;
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

// load the full box (both colours) into the tile (scalar; used off the hot path)
template <int D, int M, typename T>
__device__ __forceinline__ void load_box(const T *__restrict__ u, long long cb, T *tile, int lt, int q0, int q1) {
    constexpr int G = Geo<D, M>::G;
    for (int q = q0 + lt; q < q1; q += G) {
        int i, j, k;
        rb_cell<D, M>(q, i, j, k);
        tile[ti<D, M>(i, j, k)] = u[cb + q];
    }
}

// vector copy of a box's C values (rb order) into shared memory
template <int D, int M, typename T, int G>
__device__ __forceinline__ void stage_flat(const T *__restrict__ src, T *dst, int lt) {
    constexpr int C = Geo<D, M>::C;
    constexpr int VEC = vec_of<T, Geo<D, M>::H>();
    for (int v = lt; v < C / VEC; v += G) {
        T e[VEC];
        ldv<T, VEC>(src + (long long)v * VEC, e);
#pragma unroll
        for (int x = 0; x < VEC; ++x) dst[v * VEC + x] = e[x];
    }
}

// vector copy of a box's C values into a padded tile through tix
template <int D, int M, typename T, int G>
__device__ __forceinline__ void stage_tile(const T *__restrict__ src, T *dst, int lt, const short *tix) {
    constexpr int C = Geo<D, M>::C;
    constexpr int VEC = vec_of<T, Geo<D, M>::H>();
    for (int v = lt; v < C / VEC; v += G) {
        T e[VEC];
        ldv<T, VEC>(src + (long long)v * VEC, e);
#pragma unroll
        for (int x = 0; x < VEC; ++x) dst[tix[v * VEC + x]] = e[x];
    }
}

// Launch geometry of the half-sweep: one thread per 16-byte vector of a
// colour half (capped at the CTA size).
template <int D, int M, typename T>
struct SmCfg {
    static constexpr int H = Geo<D, M>::H;
    static constexpr int VEC = vec_of<T, H>();
    static constexpr int NV = H / VEC;
    static constexpr int G = NV < kThreads ? NV : kThreads;
    static constexpr int BPC = kThreads / G;
    static constexpr int NIT = (NV + G - 1) / G;
    static constexpr size_t smem() {
        return sizeof(T) * Geo<D, M>::PC * BPC + 2 * sizeof(BoxInfo) * BPC + Tables<D, M>::bytes();
    }
};

// Launch geometry of the full-box kernels (residual, FAS): a tile plus the
// box's rho in shared memory.
template <int D, int M, typename T>
struct FullCfg {
    static constexpr int G = Geo<D, M>::G;
    static constexpr int BPC = Geo<D, M>::BPC;
    static constexpr size_t smem() {
        return sizeof(T) * 2 * Geo<D, M>::PC * BPC + 2 * sizeof(BoxInfo) * BPC + Tables<D, M>::bytes();
    }
};

// FP64 neighbour sums: the first kFxTerms terms of ((x-+x+)+(y-+y+))+(z-+z+)
// are summed exactly on the integer pipe (fxsum.cuh, one rounding), the others
// are added to that partial sum in FP64.  GB300's integer ALU pipe is not
// free either, so the split balances it against the FP64 pipe; every split is
// at least as accurate as FP64 addition throughout.  FP32 sums use the FP32
// adders.
constexpr int kFxTerms = 4;

template <int D, typename T>
__device__ __forceinline__ T nb_sum_fp(const T (&x)[2 * D]) {
    T s = (x[0] + x[1]) + (x[2] + x[3]);
    if (D == 3) s += x[4] + x[5];
    return s;
}

// sum of the 2D face neighbours x[0..2D-1] (order -x,+x,-y,+y,-z,+z); FX =
// false keeps FP64 adds (for kernels where the integer path costs registers)
template <int D, typename T, bool FX = true>
__device__ __forceinline__ T nb_sum_x(const T (&x)[2 * D]) {
    constexpr int K = !FX ? 0 : kFxTerms < 2 * D ? kFxTerms : 2 * D;
    if constexpr (K > 0 && sizeof(T) == 8) {
        double p;
        if (fx_sum<K>(x, 0.0, p)) {
#pragma unroll
            for (int k = K; k < 2 * D; ++k) p += x[k];
            return p;
        }
    }
    return nb_sum_fp<D, T>(x);
}

// the same less 2D times the centre value c: h^2 times the operator of Eq. 5
// (FP64: -2D c joins the exact sum of the first kFxTerms neighbours, so the
// FP64 pipe adds only the remaining neighbours)
template <int D, typename T, bool FX = true>
__device__ __forceinline__ T nb_lap_x(T c, const T (&x)[2 * D]) {
    if constexpr (FX && sizeof(T) == 8) {
        constexpr int K = kFxTerms < 2 * D ? kFxTerms : 2 * D;
        double s;
        if (fx_sum<K, 2 * D>(x, c, s)) {
#pragma unroll
            for (int k = K; k < 2 * D; ++k) s += x[k];
            return s;
        }
    }
    return fma(T(-2 * D), c, nb_sum_x<D, T, FX>(x));
}

template <int D, typename T>
__device__ __forceinline__ T nb_sum6(T xm, T xp, T ym, T yp, T zm, T zp) {
    T x[2 * D];
    x[0] = xm; x[1] = xp; x[2] = ym; x[3] = yp;
    if constexpr (D == 3) { x[4] = zm; x[5] = zp; }
    return nb_sum_x<D, T>(x);
}

template <int D, typename T, bool FX = true>
__device__ __forceinline__ T nb_lap6(T c, T xm, T xp, T ym, T yp, T zm, T zp) {
    T x[2 * D];
    x[0] = xm; x[1] = xp; x[2] = ym; x[3] = yp;
    if constexpr (D == 3) { x[4] = zm; x[5] = zp; }
    return nb_lap_x<D, T, FX>(c, x);
}

// sum of the 2D face neighbours of tile slot t
template <int D, int M, typename T>
__device__ __forceinline__ T nb_sum_t(const T *tile, int t) {
    constexpr int P = M + 2;
    return nb_sum6<D, T>(tile[t - 1], tile[t + 1], tile[t - P], tile[t + P], D == 3 ? tile[t - P * P] : T(0),
                         D == 3 ? tile[t + P * P] : T(0));
}

// the same less 2D times the value of slot t
template <int D, int M, typename T>
__device__ __forceinline__ T nb_lap_t(const T *tile, int t) {
    constexpr int P = M + 2;
    return nb_lap6<D, T>(tile[t], tile[t - 1], tile[t + 1], tile[t - P], tile[t + P],
                         D == 3 ? tile[t - P * P] : T(0), D == 3 ? tile[t + P * P] : T(0));
}

// shared-memory carve-up: tiles, then the double-buffered BoxInfo, then tables
template <int D, int M>
__device__ __forceinline__ void carve(unsigned char *raw, size_t tiles_bytes, int bpc, BoxInfo *&info, short *&tix,
                                      short *&gt, short *&gs) {
    info = reinterpret_cast<BoxInfo *>(raw + tiles_bytes);
    tix = reinterpret_cast<short *>(raw + tiles_bytes + 2 * sizeof(BoxInfo) * bpc);
    gt = tix + Geo<D, M>::C;
    gs = gt + 2 * D * Geo<D, M>::F;
}

// ---------------------------------------------------------------------------
// Red-black Gauss-Seidel half-sweep on every box of a level (Sec. 3.1):
// cells of colour `colour` get u = (sum of the 2D neighbours - h^2 rho)/(2D).
// Cross-box reads touch only cells of the other colour, which this launch
// never writes, so one launch per half-sweep is race free.  Persistent CTAs
// walk the level; each box's metadata is prefetched one box ahead.
// ---------------------------------------------------------------------------
// rho_or_hat: the source term, or (scaled = 1) the pre-scaled source
// rho_hat = -h^2 rho / (2D), for which the update is one FMA: u = sum/(2D) + rho_hat
template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_smooth(BoxMeta A, int b0, int n, const int *list, T *u,
                                                     const T *__restrict__ rho, T h2, int colour, int hom,
                                                     int scaled) {
    using S = SmCfg<D, M, T>;
    using Gm = Geo<D, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / S::G, lt = threadIdx.x % S::G;
    T *tile = reinterpret_cast<T *>(smem_raw) + g * Gm::PC;
    BoxInfo *info;
    short *tix, *gt, *gs;
    carve<D, M>(smem_raw, sizeof(T) * Gm::PC * S::BPC, S::BPC, info, tix, gt, gs);
    pdl_trigger();
    build_tables<D, M>(tix, gt, gs, colour);
    const T inv = T(1) / T(2 * D);
    const int stride = gridDim.x * S::BPC;
    int base = blockIdx.x * S::BPC, buf = 0;
    info_load<D>(A, base + g, n, b0, list, info[g], lt, S::G, false);  // static metadata: before the wait
    pdl_wait();
    info_mask<D>(A, info[g], lt, S::G);
    __syncthreads();
    for (; base < n; base += stride) {
        const BoxInfo &I = info[buf * S::BPC + g];
        const int b = I.b;
        const bool special = b >= 0 && (I.flag & BF_SPECIAL);
        T rv[S::NIT][S::VEC];
        if (b >= 0) {
            gather<D, M, T, S::G>(I, u, A.bc, tile, lt, colour, special, hom, tix, gt, gs);
#pragma unroll
            for (int it = 0; it < S::NIT; ++it) {
                const int v = lt + it * S::G;
                if (v < S::NV) ldv<T, S::VEC>(rho + I.coff + colour * S::H + v * S::VEC, rv[it]);
            }
        }
        info_load<D>(A, base + stride + g, n, b0, list, info[(buf ^ 1) * S::BPC + g], lt, S::G);
        __syncthreads();
        if (special) finalize<D, M, T, S::G>(I, tile, lt, colour, A.hb);
        __syncthreads();
        if (b >= 0) {
#pragma unroll
            for (int it = 0; it < S::NIT; ++it) {
                const int v = lt + it * S::G;
                if (v < S::NV) {
                    T out[S::VEC];
#pragma unroll
                    for (int x = 0; x < S::VEC; ++x) {
                        const int t = tix[colour * S::H + v * S::VEC + x];
                        const T sum = nb_sum_t<D, M, T>(tile, t);
                        out[x] = scaled ? fma(sum, inv, rv[it][x]) : (sum - h2 * rv[it][x]) * inv;
                    }
                    stv<T, S::VEC>(u + I.coff + colour * S::H + v * S::VEC, out);
                }
            }
        }
        buf ^= 1;
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
    using S = FullCfg<D, M, T>;
    using Gm = Geo<D, M>;
    constexpr int P = M + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / S::G, lt = threadIdx.x % S::G;
    T *tile = reinterpret_cast<T *>(smem_raw) + g * 2 * Gm::PC;
    T *R = tile + Gm::PC;
    BoxInfo *info;
    short *tix, *gt, *gs;
    carve<D, M>(smem_raw, sizeof(T) * 2 * Gm::PC * S::BPC, S::BPC, info, tix, gt, gs);
    pdl_trigger();
    build_tables<D, M>(tix, gt, gs, -1);
    constexpr int MH = M / 2;
    constexpr int NCO = D == 2 ? MH * MH : MH * MH * MH;
    const int stride = gridDim.x * S::BPC;
    int base = blockIdx.x * S::BPC, buf = 0;
    info_load<D>(A, base + g, n, b0, nullptr, info[g], lt, S::G, false);  // static metadata: before the wait
    pdl_wait();
    info_mask<D>(A, info[g], lt, S::G);
    __syncthreads();
    for (; base < n; base += stride) {
        const BoxInfo &I = info[buf * S::BPC + g];
        const int b = I.b;
        const bool special = b >= 0 && (I.flag & BF_SPECIAL);
        if (b >= 0) {
            gather<D, M, T, S::G>(I, u, A.bc, tile, lt, -1, true, hom, tix, gt, gs);
            stage_tile<D, M, T, S::G>(rho + I.coff, R, lt, tix);
        }
        info_load<D>(A, base + stride + g, n, b0, nullptr, info[(buf ^ 1) * S::BPC + g], lt, S::G);
        __syncthreads();
        if (special) finalize<D, M, T, S::G>(I, tile, lt, -1, A.hb);
        __syncthreads();
        if (b >= 0) {
            const long long cp = A.coff[I.parent];
            for (int c = lt; c < NCO; c += S::G) {
                const int X = c % MH, Y = (c / MH) % MH, Z = D == 3 ? c / (MH * MH) : 0;
                const int t0 = ti<D, M>(2 * X, 2 * Y, D == 3 ? 2 * Z : 0);
                // Sum of the children's residuals: each child sees D siblings and D
                // cells outside the 2^D block, so sum_c (A u)_c = (sum_outside - D sum_c u) / h^2.
                T su = T(0), sro = T(0), sout = T(0);
#pragma unroll
                for (int dz = 0; dz < (D == 3 ? 2 : 1); ++dz)
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) {
                            const int t = t0 + dx + dy * P + dz * P * P;
                            su += tile[t];
                            sro += R[t];
                            // the outside neighbour of this child along each axis
                            sout += tile[t + (dx ? 1 : -1)];
                            sout += tile[t + (dy ? P : -P)];
                            if (D == 3) sout += tile[t + (dz ? P * P : -P * P)];
                        }
                const T w = T(1) / T(1 << D);
                const T sr = fma(-ih2, fma(T(-D), su, sout), sro);
                const int pi = unpack_off(I.poff, 0) + X, pj = unpack_off(I.poff, 1) + Y;
                const int pk = D == 3 ? unpack_off(I.poff, 2) + Z : 0;
                const long long q = cp + rbi<D, MP>(pi, pj, pk);
                const T mu = su * w;
                u[q] = mu;
                vold[q] = mu;
                rho[q] = sr * w;
            }
        }
        buf ^= 1;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FAS coarse right-hand side (Eq. coarse-rhs) on the refined boxes of a level
// (rho_H already holds the restricted residual): rho_H += A_H(v_H).  Leaves
// of the level store their copy v' = v.
// ---------------------------------------------------------------------------
// rhoh (may be null): also store rho_hat = chat * rho_H for the scaled smoother
template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_fas(BoxMeta A, int b0, int n, const T *u, T *rho, T *vold, T ih2,
                                                  int hom, T *rhoh, T chat) {
    using S = FullCfg<D, M, T>;
    using Gm = Geo<D, M>;
    constexpr int VEC = vec_of<T, Gm::H>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / S::G, lt = threadIdx.x % S::G;
    T *tile = reinterpret_cast<T *>(smem_raw) + g * 2 * Gm::PC;
    T *R = tile + Gm::PC;
    BoxInfo *info;
    short *tix, *gt, *gs;
    carve<D, M>(smem_raw, sizeof(T) * 2 * Gm::PC * S::BPC, S::BPC, info, tix, gt, gs);
    pdl_trigger();
    build_tables<D, M>(tix, gt, gs, -1);
    const int stride = gridDim.x * S::BPC;
    int base = blockIdx.x * S::BPC, buf = 0;
    info_load<D>(A, base + g, n, b0, nullptr, info[g], lt, S::G, false);  // static metadata: before the wait
    pdl_wait();
    info_mask<D>(A, info[g], lt, S::G);
    __syncthreads();
    for (; base < n; base += stride) {
        const BoxInfo &I = info[buf * S::BPC + g];
        const int b = I.b;
        const bool refined = b >= 0 && (I.flag & BF_REFINED);
        const bool special = refined && (I.flag & BF_SPECIAL);
        if (refined) {
            gather<D, M, T, S::G>(I, u, A.bc, tile, lt, -1, true, hom, tix, gt, gs);
            stage_flat<D, M, T, S::G>(rho + I.coff, R, lt);
        } else if (b >= 0) {
            for (int v = lt; v < Gm::C / VEC; v += S::G) {
                T e[VEC];
                ldv<T, VEC>(u + I.coff + (long long)v * VEC, e);
                stv<T, VEC>(vold + I.coff + (long long)v * VEC, e);
            }
        }
        info_load<D>(A, base + stride + g, n, b0, nullptr, info[(buf ^ 1) * S::BPC + g], lt, S::G);
        __syncthreads();
        if (special) finalize<D, M, T, S::G>(I, tile, lt, -1, A.hb);
        __syncthreads();
        if (refined) {
            for (int v = lt; v < Gm::C / VEC; v += S::G) {
                T out[VEC];
#pragma unroll
                for (int x = 0; x < VEC; ++x) {
                    const int q = v * VEC + x;
                    const int t = tix[q];
                    out[x] = fma(ih2, nb_lap_t<D, M, T>(tile, t), R[q]);
                }
                stv<T, VEC>(rho + I.coff + (long long)v * VEC, out);
                if (rhoh) {
#pragma unroll
                    for (int x = 0; x < VEC; ++x) out[x] *= chat;
                    stv<T, VEC>(rhoh + I.coff + (long long)v * VEC, out);
                }
            }
        }
        buf ^= 1;
        __syncthreads();
    }
}

// Metadata for the correction: the box, its parent, and the parent's side
// codes / neighbour offsets (the correction reads the parent's neighbours).
template <int D>
__device__ __forceinline__ void pinfo_load(const BoxMeta &A, int idx, int n, int b0, BoxInfo &I, int lt, int G,
                                           bool mask) {
    for (int x = lt; x <= 2 * D; x += G) {
        int b = idx < n ? b0 + idx : -1;
        if (x < 2 * D) {
            if (b >= 0) {
                const int p = A.parent[b];
                I.code[x] = A.nb[p * 2 * D + x];
                I.base[x] = A.nbase[p * 2 * D + x];
            }
        } else {
            if (mask && b >= 0 && A.active && !A.active[A.tree[b]]) b = -1;
            I.b = b;
            if (b >= 0) {
                I.coff = A.coff[b];
                I.poff = A.poff[b];
                I.parent = A.parent[b];
                I.pcoff = A.coff[I.parent];
                I.nmask = A.nmask[I.parent];
            }
        }
    }
}

template <int D, int M>
struct CorrCfg {
    static constexpr int MH = M / 2, Q = MH + 2;
    static constexpr int QC = D == 2 ? Q * Q : Q * Q * Q;
    static constexpr int G = Geo<D, M>::G, BPC = Geo<D, M>::BPC;
    template <typename T>
    static constexpr size_t smem() { return sizeof(T) * QC * BPC + 2 * sizeof(BoxInfo) * BPC; }
};

// ---------------------------------------------------------------------------
// Coarse-grid correction u_h += I_H^h (v_H - v'_H) (Eq. coarse-corr) with the
// 2-1-1 (2D) / 1-1-1-1 (3D) prolongation (Sec. 2.5) on every box of level l.
// The difference is staged for the box's parent region plus one layer;
// outside the parent it comes from the parent's same-level neighbour, or is
// -d at the domain boundary (homogeneous Dirichlet ghost of a correction).
// The box's own values are fetched (as vectors) together with the staging.
// ---------------------------------------------------------------------------
template <int D, int M, int MP, typename T>
__global__ void __launch_bounds__(kThreads) k_correct(BoxMeta A, int b0, int n, T *u, const T *__restrict__ vold) {
    using Gm = Geo<D, M>;
    using S = CorrCfg<D, M>;
    constexpr int MH = S::MH, Q = S::Q, QC = S::QC;
    constexpr int VEC = vec_of<T, Gm::H>();
    constexpr int NV = Gm::C / VEC;
    constexpr int NIT = (NV + S::G - 1) / S::G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lt = threadIdx.x % S::G, g = threadIdx.x / S::G;
    T *dt = reinterpret_cast<T *>(smem_raw) + g * QC;
    BoxInfo *info = reinterpret_cast<BoxInfo *>(smem_raw + sizeof(T) * QC * S::BPC);
    auto di = [](int x, int y, int z) { return D == 2 ? (y + 1) * Q + (x + 1) : ((z + 1) * Q + (y + 1)) * Q + (x + 1); };
    const int stride = gridDim.x * S::BPC;
    int base = blockIdx.x * S::BPC, buf = 0;
    pdl_trigger();
    pinfo_load<D>(A, base + g, n, b0, info[g], lt, S::G, false);
    pdl_wait();
    info_mask<D>(A, info[g], lt, S::G);
    __syncthreads();
    for (; base < n; base += stride) {
        const BoxInfo &I = info[buf * S::BPC + g];
        const int b = I.b;
        T uv[NIT][VEC];
        if (b >= 0) {
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                const int v = lt + it * S::G;
                if (v < NV) ldv<T, VEC>(u + I.coff + (long long)v * VEC, uv[it]);
            }
            const int o[3] = {unpack_off(I.poff, 0), unpack_off(I.poff, 1), D == 3 ? unpack_off(I.poff, 2) : 0};
            for (int c = lt; c < QC; c += S::G) {
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
                    const long long q = I.pcoff + rbi<D, MP>(pc[0], pc[1], pc[2]);
                    d = u[q] - vold[q];
                } else {
                    const int code = I.code[side];
                    const int a = side >> 1;
                    if (code >= 0) {
                        pc[a] = (side & 1) ? 0 : MP - 1;
                        const long long q = I.base[side] + rbi<D, MP>(pc[0], pc[1], pc[2]);
                        d = u[q] - vold[q];
                    } else {  // domain boundary: homogeneous ghost of the difference, -d (Dirichlet) or d (Neumann)
                        pc[a] = (side & 1) ? MP - 1 : 0;
                        const long long q = I.pcoff + rbi<D, MP>(pc[0], pc[1], pc[2]);
                        d = ((I.nmask >> side) & 1) ? u[q] - vold[q] : -(u[q] - vold[q]);
                    }
                }
                dt[di(x, y, z)] = d;
            }
        }
        pinfo_load<D>(A, base + stride + g, n, b0, info[(buf ^ 1) * S::BPC + g], lt, S::G, true);
        __syncthreads();
        if (b >= 0) {
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                const int v = lt + it * S::G;
                if (v >= NV) continue;
                T res[VEC];
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    int i, j, k;
                    rb_cell<D, M>(v * VEC + e, i, j, k);
                    const int X = i >> 1, Y = j >> 1, Z = k >> 1;
                    const int sx = (i & 1) ? 1 : -1, sy = (j & 1) ? 1 : -1, sz = (k & 1) ? 1 : -1;
                    const T d0 = dt[di(X, Y, Z)], dx = dt[di(X + sx, Y, Z)], dy = dt[di(X, Y + sy, Z)];
                    if (D == 2) res[e] = fma(T(0.25), dx + dy, fma(T(0.5), d0, uv[it][e]));
                    else res[e] = fma(T(0.25), ((d0 + dx) + dy) + dt[di(X, Y, Z + sz)], uv[it][e]);
                }
                stv<T, VEC>(u + I.coff + (long long)v * VEC, res);
            }
        }
        buf ^= 1;
        __syncthreads();
    }
}

// rho_hat = -h^2 rho / (2D) on a list of boxes (after the source term changed)
template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_rho_hat(BoxMeta A, const int *list, int n, const T *rho, T *rhoh) {
    using Gm = Geo<D, M>;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    pdl_trigger();
    pdl_wait();
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int idx = base + g;
        if (idx >= n) continue;
        const int b = list[idx];
        const long long cb = A.coff[b];
        const T c = T(-A.hb[b] * A.hb[b] / (2 * D));
        constexpr int VEC = 16 / (int)sizeof(T);  // a box is a whole number of 16-byte vectors
        for (int q = lt; q < Gm::C / VEC; q += Gm::G) {
            T v[VEC];
            ldv<T, VEC>(rho + cb + q * VEC, v);
#pragma unroll
            for (int x = 0; x < VEC; ++x) v[x] *= c;
            stv<T, VEC>(rhoh + cb + q * VEC, v);
        }
    }
}

// Restriction of u alone (FMG start, composite residual): parent region =
// mean of the children, for the boxes b0..b0+n-1 or the n boxes of list.
template <int D, int M, int MP, typename T>
__global__ void __launch_bounds__(kThreads) k_restrict_u(BoxMeta A, int b0, int n, const int *list, T *u) {
    using Gm = Geo<D, M>;
    constexpr int MH = M / 2;
    constexpr int NCO = D == 2 ? MH * MH : MH * MH * MH;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    pdl_trigger();
    pdl_wait();
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int b = resolve_box<D, M>(A, base + g, n, b0, list);
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

// |x| as an ordered unsigned bit pattern (sign bit cleared; integer ops only)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long abs_bits(float x) { return abs_bits(double(x)); }

// Block-wide max of per-thread values for the tree `tr` (uniform in the
// block), then one atomic per block.  Non-negative doubles compare like their
// bit patterns, so the maxima run on the integer pipe.
__device__ __forceinline__ void flush_max(unsigned long long rm, unsigned long long pm, int tr, bool valid,
                                          unsigned long long *rmax, unsigned long long *pmax,
                                          unsigned long long *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rm = max(rm, __shfl_xor_sync(0xffffffffu, rm, o));
        pm = max(pm, __shfl_xor_sync(0xffffffffu, pm, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[w] = rm;
        red[32 + w] = pm;
    }
    __syncthreads();
    if (threadIdx.x == 0 && valid) {
        unsigned long long a = 0, c = 0;
        for (int i = 0; i < kThreads / 32; ++i) {
            a = max(a, red[i]);
            c = max(c, red[32 + i]);
        }
        atomicMax(rmax + tr, a);
        if (pmax) atomicMax(pmax + tr, c);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Residual norm on leaf boxes (list): max |rho - A u| and max |rho| per tree.
// Each thread keeps running maxima over the boxes it visits; they are
// reduced over the block and committed with one atomic per block whenever
// the block moves to another tree, and at the end.  Optionally stores the
// residual, cast to R, into rout (the mixed-precision defect correction).
// ---------------------------------------------------------------------------
template <int D, int M, typename T, typename R>
__global__ void __launch_bounds__(kThreads) k_leaf_residual(BoxMeta A, const int *list, int n, const T *u,
                                                            const T *__restrict__ rho, int hom,
                                                            unsigned long long *rmax, unsigned long long *pmax,
                                                            R *rout) {
    using S = FullCfg<D, M, T>;
    using Gm = Geo<D, M>;
    constexpr int VEC = vec_of<T, Gm::H>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long red[64];
    __shared__ int blk_tree[Geo<D, M>::BPC];
    const int g = threadIdx.x / S::G, lt = threadIdx.x % S::G;
    T *tile = reinterpret_cast<T *>(smem_raw) + g * 2 * Gm::PC;
    T *RH = tile + Gm::PC;
    BoxInfo *info;
    short *tix, *gt, *gs;
    carve<D, M>(smem_raw, sizeof(T) * 2 * Gm::PC * S::BPC, S::BPC, info, tix, gt, gs);
    pdl_trigger();
    build_tables<D, M>(tix, gt, gs, -1);
    const int stride = gridDim.x * S::BPC;
    int base = blockIdx.x * S::BPC, buf = 0;
    info_load<D>(A, base + g, n, 0, list, info[g], lt, S::G, false);  // static metadata: before the wait
    pdl_wait();
    info_mask<D>(A, info[g], lt, S::G);
    __syncthreads();
    unsigned long long rm = 0, pm = 0;
    int cur = -1;  // tree of the running maxima (uniform in the block)
    for (; base < n; base += stride) {
        const BoxInfo &I = info[buf * S::BPC + g];
        const int b = I.b;
        const bool special = b >= 0 && (I.flag & BF_SPECIAL);
        double ihb = 0.0;
        if (b >= 0) {
            gather<D, M, T, S::G>(I, u, A.bc, tile, lt, -1, true, hom, tix, gt, gs);
            stage_flat<D, M, T, S::G>(rho + I.coff, RH, lt);
            ihb = A.ih2[b];
        }
        if (lt == 0) blk_tree[g] = b >= 0 ? A.tree[b] : -1;
        info_load<D>(A, base + stride + g, n, 0, list, info[(buf ^ 1) * S::BPC + g], lt, S::G);
        __syncthreads();
        // the block's boxes all belong to one tree unless the tree changes here
        int tr = -1;
        bool mixed = false;
        for (int x = 0; x < S::BPC; ++x) {
            const int t = blk_tree[x];
            if (t < 0) continue;
            if (tr < 0) tr = t;
            else if (t != tr) mixed = true;
        }
        if (mixed || (tr >= 0 && cur >= 0 && tr != cur)) {
            flush_max(rm, pm, cur, cur >= 0, rmax, pmax, red);
            rm = pm = 0;
            cur = -1;
        }
        if (special) finalize<D, M, T, S::G>(I, tile, lt, -1, A.hb);
        __syncthreads();
        if (b >= 0) {
            const T ih2 = T(ihb);
            for (int v = lt; v < Gm::C / VEC; v += S::G) {
                R out[VEC];
#pragma unroll
                for (int x = 0; x < VEC; ++x) {
                    const int q = v * VEC + x;
                    const int t = tix[q];
                    // r = rho - (sum - 2D u) / h^2 as two FMAs; |.| on the bit patterns
                    // (integer pipe), so the FP64 pipe only sees the stencil
                    const T lap = nb_lap_t<D, M, T>(tile, t);
                    const T rr = fma(-ih2, lap, RH[q]);
                    out[x] = R(rr);
                    rm = max(rm, abs_bits(rr));
                    pm = max(pm, abs_bits(RH[q]));
                }
                if (rout) {
#pragma unroll
                    for (int x = 0; x < VEC; ++x) rout[I.coff + (long long)v * VEC + x] = out[x];
                }
            }
        }
        if (mixed) {  // boxes of several trees in this block: commit each box's maxima now
            for (int x = 0; x < S::BPC; ++x) {
                const int t = blk_tree[x];
                flush_max(g == x ? rm : 0ull, g == x ? pm : 0ull, t, t >= 0, rmax, pmax, red);
            }
            rm = pm = 0;
        } else if (tr >= 0) {
            cur = tr;
        }
        buf ^= 1;
        __syncthreads();
    }
    flush_max(rm, pm, cur, cur >= 0, rmax, pmax, red);
}

}  // namespace afg
