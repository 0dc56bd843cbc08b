// Coarse-grid correction with the other prolongation schemes of Sec. 2.5
// (arXiv:1701.04329): bi/trilinear (scheme 1) and zeroth order (scheme 2);
// the linear 2-1-1 / 1-1-1-1 scheme is k_correct / k_correct_p.
//
// u_h += I(v_H - v'_H) on every box of a level.  The difference d = v_H - v'_H
// is read from the parent P's padded array: its cells, its side ghosts
// (the same-level neighbour's d, or -d / d of the mirrored cell at a
// Dirichlet / Neumann domain side, the homogeneous rule of the correction)
// and -- for the bi/trilinear scheme -- its edge and corner ghosts (Sec.
// 2.4): the diagonal same-level neighbour's d when that box exists, else
// the linear extrapolation f(p) = f(p + u) + f(p + w) - f(p + u + w), with u
// the unit step into P along the first axis on which p lies outside P and
// w the steps along the others (in 2D the corner ghost b + c - a; in 3D an
// edge ghost from its two side ghosts and the edge cell, a corner ghost from
// the edge ghost next to it along x, the side ghost next to it along y-z and
// the corner cell).
//
// A thread group stages, per child box, the (M/2 + 2)^D values of d its
// region needs (its part of P with a layer around it, edges and corners
// included) in shared memory, then updates the box's cells:
//   bi/trilinear: the 2^D nearest coarse cells, weight 3/4 per axis for the
//                 nearer one, 1/4 for the farther one;
//   zeroth order: the coarse cell's d.
#pragma once
#include "kernels.cuh"

namespace afg {

template <int D>
struct NbAll {
    static constexpr int ND = D == 2 ? 8 : 26;
    // direction of the offsets (ox, oy, oz) in {-1, 0, 1}: lexicographic
    // (z, y, x) with x fastest, the centre skipped
    static __device__ __forceinline__ int dir(int ox, int oy, int oz) {
        const int c = D == 2 ? 4 : 13;
        const int i = D == 2 ? (oy + 1) * 3 + (ox + 1) : ((oz + 1) * 3 + (oy + 1)) * 3 + (ox + 1);
        return i > c ? i - 1 : i;
    }
};

// d = u - v' of cell p (inside box Q, box size MP)
template <int D, int MP, typename T>
__device__ __forceinline__ T pd_cell(const BoxMeta &A, int Q, const int (&p)[3], const T *u, const T *vold) {
    const long long q = A.coff[Q] + rbi<D, MP>(p[0], p[1], p[2]);
    return u[q] - vold[q];
}

// side ghost of P at p, outside P along axis a only
template <int D, int MP, typename T>
__device__ __forceinline__ T pd_face(const BoxMeta &A, int P, const int (&p)[3], int a, const T *u, const T *vold) {
    const int hi = p[a] >= MP, s = 2 * a + hi;
    const int code = A.nb[P * 2 * D + s];
    int q[3] = {p[0], p[1], p[2]};
    if (code >= 0) {
        q[a] = hi ? 0 : MP - 1;
        return pd_cell<D, MP, T>(A, code, q, u, vold);
    }
    q[a] = hi ? MP - 1 : 0;  // domain side: the mirrored cell, -d (Dirichlet) or d (Neumann)
    const T dm = pd_cell<D, MP, T>(A, P, q, u, vold);
    return ((A.nmask[P] >> s) & 1) ? dm : -dm;
}

// the diagonal same-level neighbour of P holding p (outside P along the axes
// ax[0..n-1]), or -1
template <int D, int MP>
__device__ __forceinline__ int pd_diag(const int *nball, int P, const int (&p)[3]) {
    int o[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) o[a] = p[a] < 0 ? -1 : (p[a] >= MP ? 1 : 0);
    return nball[P * NbAll<D>::ND + NbAll<D>::dir(o[0], o[1], o[2])];
}

template <int D, int MP, typename T>
__device__ __forceinline__ T pd_wrap(const BoxMeta &A, int Q, const int (&p)[3], const T *u, const T *vold) {
    int q[3] = {p[0], p[1], p[2]};
    for (int a = 0; a < D; ++a) q[a] = p[a] < 0 ? MP - 1 : (p[a] >= MP ? 0 : p[a]);
    return pd_cell<D, MP, T>(A, Q, q, u, vold);
}

__device__ __forceinline__ int step_in(int x, int MP) { return x < 0 ? 0 : MP - 1; }

// edge ghost (outside P along axes a0 < a1 only)
template <int D, int MP, typename T>
__device__ __forceinline__ T pd_edge(const BoxMeta &A, const int *nball, int P, const int (&p)[3], int a0, int a1,
                                     const T *u, const T *vold) {
    const int Q = pd_diag<D, MP>(nball, P, p);
    if (Q >= 0) return pd_wrap<D, MP, T>(A, Q, p, u, vold);
    int pu[3] = {p[0], p[1], p[2]}, pw[3] = {p[0], p[1], p[2]}, pa[3] = {p[0], p[1], p[2]};
    pu[a0] = step_in(p[a0], MP);
    pw[a1] = step_in(p[a1], MP);
    pa[a0] = pu[a0];
    pa[a1] = pw[a1];
    return pd_face<D, MP, T>(A, P, pu, a1, u, vold) + pd_face<D, MP, T>(A, P, pw, a0, u, vold) -
           pd_cell<D, MP, T>(A, P, pa, u, vold);
}

// d of P's padded array at p (0-based, each coordinate in [-1, MP])
template <int D, int MP, typename T>
__device__ __forceinline__ T pd_any(const BoxMeta &A, const int *nball, int P, const int (&p)[3], const T *u,
                                    const T *vold) {
    int ax[3], n = 0;
    for (int a = 0; a < D; ++a)
        if (p[a] < 0 || p[a] >= MP) ax[n++] = a;
    if (n == 0) return pd_cell<D, MP, T>(A, P, p, u, vold);
    if (n == 1) return pd_face<D, MP, T>(A, P, p, ax[0], u, vold);
    if (n == 2) return pd_edge<D, MP, T>(A, nball, P, p, ax[0], ax[1], u, vold);
    // 3D corner
    const int Q = pd_diag<D, MP>(nball, P, p);
    if (Q >= 0) return pd_wrap<D, MP, T>(A, Q, p, u, vold);
    int pu[3] = {p[0], p[1], p[2]}, pw[3] = {p[0], p[1], p[2]}, pa[3];
    pu[0] = step_in(p[0], MP);           // into P along x: the edge ghost along y-z
    pw[1] = step_in(p[1], MP);           // into P along y and z: the side ghost along x
    pw[2] = step_in(p[2], MP);
    pa[0] = pu[0];
    pa[1] = pw[1];
    pa[2] = pw[2];
    return pd_edge<D, MP, T>(A, nball, P, pu, 1, 2, u, vold) + pd_face<D, MP, T>(A, P, pw, 0, u, vold) -
           pd_cell<D, MP, T>(A, P, pa, u, vold);
}

template <int D, int M>
struct PxCfg {
    static constexpr int MH = M / 2, Q = MH + 2;
    static constexpr int QC = D == 2 ? Q * Q : Q * Q * Q;
    static constexpr int G = Geo<D, M>::G, BPC = Geo<D, M>::BPC;
    template <typename T>
    static constexpr size_t smem() { return sizeof(T) * QC * BPC; }
};

template <int D, int M, int MP, typename T>
__global__ void __launch_bounds__(kThreads) k_correct_x(BoxMeta A, int b0, int n, T *u, const T *vold,
                                                        const int *nball, int scheme) {
    using S = PxCfg<D, M>;
    constexpr int MH = S::MH, Q = S::Q, C = Geo<D, M>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = threadIdx.x / S::G, lt = threadIdx.x % S::G;
    T *R = reinterpret_cast<T *>(smem_raw) + g * S::QC;
    pdl_trigger();
    pdl_wait();
    for (int base = blockIdx.x * S::BPC; base < n; base += gridDim.x * S::BPC) {
        const int idx = base + g;
        const int b = idx < n ? b0 + idx : -1;
        const bool on = b >= 0 && !(A.active && !A.active[A.tree[b]]);
        if (on) {
            const int P = A.parent[b], po = A.poff[b];
            for (int c = lt; c < S::QC; c += S::G) {
                const int x = c % Q - 1, y = (c / Q) % Q - 1, z = D == 3 ? c / (Q * Q) - 1 : 0;
                const int p[3] = {unpack_off(po, 0) + x, unpack_off(po, 1) + y, D == 3 ? unpack_off(po, 2) + z : 0};
                // only the bi/trilinear scheme reads edges and corners; the zeroth order only the region itself
                int out = (x < 0 || x >= MH) + (y < 0 || y >= MH) + (D == 3 && (z < 0 || z >= MH));
                if (scheme == 2 && out) continue;
                R[c] = pd_any<D, MP, T>(A, nball, P, p, u, vold);
            }
        }
        __syncthreads();
        if (on) {
            const long long cb = A.coff[b];
            for (int q = lt; q < C; q += S::G) {
                int i, j, k;
                rb_cell<D, M>(q, i, j, k);
                const int X = i >> 1, Y = j >> 1, Z = D == 3 ? k >> 1 : 0;
                const int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
                const int c0 = D == 2 ? (Y + 1) * Q + (X + 1) : ((Z + 1) * Q + (Y + 1)) * Q + (X + 1);
                T add;
                if (scheme == 2) {
                    add = R[c0];
                } else {
                    add = T(0);
#pragma unroll
                    for (int cc = 0; cc < (1 << D); ++cc) {
                        T w = T(1);
                        int o = c0;
                        if (cc & 1) { o += si; w *= T(0.25); } else { w *= T(0.75); }
                        if (cc & 2) { o += sj * Q; w *= T(0.25); } else { w *= T(0.75); }
                        if (D == 3) {
                            if (cc & 4) { o += sk * Q * Q; w *= T(0.25); } else { w *= T(0.75); }
                        }
                        add += w * R[o];
                    }
                }
                u[cb + q] += add;
            }
        }
        __syncthreads();
    }
}

}  // namespace afg
