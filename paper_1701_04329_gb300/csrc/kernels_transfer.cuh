// Field transfer on mesh adaptation (arXiv:1701.04329 Sec. 2.3: with
// prolongation and restriction given, they are applied when the mesh
// changes).  A leaf of the adapted tree that existed before keeps its values
// (a parent whose children were removed holds their mean, the restriction
// of Sec. 2.5, written into it before the change); a new child of a refined
// leaf is prolonged from that leaf with one of the schemes of Sec. 2.5 --
// linear 2-1-1 / 1-1-1-1 (0), bi/trilinear (1) or zeroth order (2) -- whose
// ghost values are filled as in the solver: same-level copy, the stored
// boundary data (2 b - u_1 Dirichlet, u_1 + h b Neumann), the refinement-
// boundary scheme of Sec. 3.3, and for the bi/trilinear scheme the edge and
// corner ghosts of Sec. 2.4 (the diagonal same-level neighbour's value, else
// f(p) = f(p + u) + f(p + w) - f(p + u + w), edges before corners).
//
// One thread group per new leaf box, following a per-box plan built on the
// host: the old box to copy, or the old leaf to prolong from with the new
// box's offset in it.
#pragma once
#include "kernels.cuh"

namespace afg {

template <int D, int M>
struct TrCfg {
    static constexpr int G = Geo<D, M>::G, BPC = Geo<D, M>::BPC, PC = Geo<D, M>::PC;
    static constexpr int ND = D == 2 ? 8 : 26;
    template <typename T>
    static constexpr size_t smem() { return sizeof(T) * PC * BPC + 2 * sizeof(BoxInfo) * BPC + Tables<D, M>::bytes(); }
};

// edge (2D: corner) ghost slot e -> position with two coordinates outside [0, M)
template <int D, int M>
__device__ __forceinline__ void tr_edge(int e, int (&p)[3], int &a0, int &a1) {
    if (D == 2) {
        p[0] = (e & 1) ? M : -1;
        p[1] = (e & 2) ? M : -1;
        p[2] = 0;
        a0 = 0;
        a1 = 1;
        return;
    }
    const int pair = e / (4 * M), r = e % (4 * M), cnr = r / M, t = r % M;
    a0 = pair == 2 ? 1 : 0;
    a1 = pair == 0 ? 1 : 2;
    const int fa = 3 - a0 - a1;  // the axis along the edge
    p[a0] = (cnr & 1) ? M : -1;
    p[a1] = (cnr & 2) ? M : -1;
    p[fa] = t;
}

__device__ __forceinline__ int tr_in(int x, int M) { return x < 0 ? 0 : M - 1; }

// the diagonal same-level neighbour's value at p (wrapped into it), if that box exists
template <int D, int M, typename T>
__device__ __forceinline__ bool tr_diag(const BoxMeta &A, const int *nball, int P, const int (&p)[3], const T *u,
                                        T &v) {
    int o[3] = {0, 0, 0}, q[3] = {p[0], p[1], p[2]};
    for (int a = 0; a < D; ++a) {
        o[a] = p[a] < 0 ? -1 : (p[a] >= M ? 1 : 0);
        q[a] = p[a] < 0 ? M - 1 : (p[a] >= M ? 0 : p[a]);
    }
    const int c = D == 2 ? 4 : 13;
    int d = D == 2 ? (o[1] + 1) * 3 + (o[0] + 1) : ((o[2] + 1) * 3 + (o[1] + 1)) * 3 + (o[0] + 1);
    d = d > c ? d - 1 : d;
    const int Q = nball[P * TrCfg<D, M>::ND + d];
    if (Q < 0) return false;
    v = u[A.coff[Q] + rbi<D, M>(q[0], q[1], q[2])];
    return true;
}

template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_transfer(BoxMeta Ao, const T *uo, const int *nball_o, BoxMeta An,
                                                       T *un, const int *new_leaves, const int *src,
                                                       const int *poff, int n, int scheme) {
    using S = TrCfg<D, M>;
    constexpr int C = Geo<D, M>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / S::G, lt = threadIdx.x % S::G;
    T *tile = reinterpret_cast<T *>(smem_raw) + g * S::PC;
    BoxInfo *info;
    short *tix, *gt, *gs;
    carve<D, M>(smem_raw, sizeof(T) * S::PC * S::BPC, S::BPC, info, tix, gt, gs);
    pdl_trigger();
    build_tables<D, M>(tix, gt, gs, -1);
    pdl_wait();
    for (int base = blockIdx.x * S::BPC; base < n; base += gridDim.x * S::BPC) {
        const int li = base + g;
        const bool on = li < n;
        const int sb = on ? src[li] : -1, po = on ? poff[li] : -1;
        const bool pro = on && po >= 0;
        BoxInfo &I = info[g];
        if (pro) info_load<D>(Ao, 0, 1, sb, nullptr, I, lt, S::G, false);
        __syncthreads();
        if (pro) gather<D, M, T, S::G>(I, uo, Ao.bc, tile, lt, -1, true, 0, tix, gt, gs);
        __syncthreads();
        if (pro && (I.flag & BF_SPECIAL)) finalize<D, M, T, S::G>(I, tile, lt, -1, Ao.hb);
        __syncthreads();
        if (pro && scheme == 1) {  // edge (2D: corner) ghosts
            for (int e = lt; e < (D == 2 ? 4 : 12 * M); e += S::G) {
                int p[3], a0, a1;
                tr_edge<D, M>(e, p, a0, a1);
                T v;
                if (!tr_diag<D, M, T>(Ao, nball_o, sb, p, uo, v)) {
                    int pu[3] = {p[0], p[1], p[2]}, pw[3] = {p[0], p[1], p[2]}, pa[3] = {p[0], p[1], p[2]};
                    pu[a0] = tr_in(p[a0], M);
                    pw[a1] = tr_in(p[a1], M);
                    pa[a0] = pu[a0];
                    pa[a1] = pw[a1];
                    v = tile[ti<D, M>(pu[0], pu[1], pu[2])] + tile[ti<D, M>(pw[0], pw[1], pw[2])] -
                        tile[ti<D, M>(pa[0], pa[1], pa[2])];
                }
                tile[ti<D, M>(p[0], p[1], p[2])] = v;
            }
        }
        __syncthreads();
        if (pro && scheme == 1 && D == 3) {  // corner ghosts, from the edge ghosts
            for (int e = lt; e < 8; e += S::G) {
                const int p[3] = {(e & 1) ? M : -1, (e & 2) ? M : -1, (e & 4) ? M : -1};
                T v;
                if (!tr_diag<D, M, T>(Ao, nball_o, sb, p, uo, v)) {
                    const int ix = tr_in(p[0], M), iy = tr_in(p[1], M), iz = tr_in(p[2], M);
                    v = tile[ti<D, M>(ix, p[1], p[2])] + tile[ti<D, M>(p[0], iy, iz)] - tile[ti<D, M>(ix, iy, iz)];
                }
                tile[ti<D, M>(p[0], p[1], p[2])] = v;
            }
        }
        __syncthreads();
        if (on) {
            const long long db = An.coff[new_leaves[li]];
            if (!pro) {
                const long long sbase = Ao.coff[sb];
                for (int q = lt; q < C; q += S::G) un[db + q] = uo[sbase + q];
            } else {
                const int ox = unpack_off(po, 0), oy = unpack_off(po, 1), oz = D == 3 ? unpack_off(po, 2) : 0;
                for (int q = lt; q < C; q += S::G) {
                    int i, j, k;
                    rb_cell<D, M>(q, i, j, k);
                    // coarse cell and the side of the neighbours each fine cell leans to
                    const int X = ox + (i >> 1), Y = oy + (j >> 1), Z = D == 3 ? oz + (k >> 1) : 0;
                    const int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
                    const T d0 = tile[ti<D, M>(X, Y, Z)];
                    T v;
                    if (scheme == 2) {
                        v = d0;
                    } else if (scheme == 1) {
                        v = T(0);
#pragma unroll
                        for (int cc = 0; cc < (1 << D); ++cc) {
                            T w = T(1);
                            int qx = X, qy = Y, qz = Z;
                            if (cc & 1) { qx += si; w *= T(0.25); } else { w *= T(0.75); }
                            if (cc & 2) { qy += sj; w *= T(0.25); } else { w *= T(0.75); }
                            if (D == 3) {
                                if (cc & 4) { qz += sk; w *= T(0.25); } else { w *= T(0.75); }
                            }
                            v += w * tile[ti<D, M>(qx, qy, qz)];
                        }
                    } else {
                        const T dx = tile[ti<D, M>(X + si, Y, Z)], dy = tile[ti<D, M>(X, Y + sj, Z)];
                        if (D == 2) {
                            v = T(0.5) * d0 + T(0.25) * (dx + dy);
                        } else {
                            const T dz = tile[ti<D, M>(X, Y, Z + sk)];
                            v = T(0.25) * (((d0 + dx) + dy) + dz);
                        }
                    }
                    un[db + q] = v;
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace afg
