// Leaf-data, boundary-data, mixed-precision and adjoint kernels
// (arXiv:1701.04329 method; the adjoint and mixed precision are additions).
#pragma once
#include "kernels.cuh"

namespace afg {

// canonical leaf cells (x fastest) <-> red-black box storage
template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_leaf_set(BoxMeta A, const int *list, int n, const double *src, T *dst) {
    using Gm = Geo<D, M>;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    pdl_trigger();
    pdl_wait();
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int li = base + g;
        if (li >= n) continue;
        const long long cb = A.coff[list[li]];
        for (int c = lt; c < Gm::C; c += Gm::G) {
            const int i = c % M, j = (c / M) % M, k = D == 3 ? c / (M * M) : 0;
            dst[cb + rbi<D, M>(i, j, k)] = T(src[(long long)li * Gm::C + c]);
        }
    }
}

template <int D, int M, typename T>
__global__ void __launch_bounds__(kThreads) k_leaf_get(BoxMeta A, const int *list, int n, const T *src, double *dst) {
    using Gm = Geo<D, M>;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    pdl_trigger();
    pdl_wait();
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int li = base + g;
        if (li >= n) continue;
        const long long cb = A.coff[list[li]];
        for (int c = lt; c < Gm::C; c += Gm::G) {
            const int i = c % M, j = (c / M) % M, k = D == 3 ? c / (M * M) : 0;
            dst[(long long)li * Gm::C + c] = double(src[cb + rbi<D, M>(i, j, k)]);
        }
    }
}

// Dirichlet data of coarse boxes: the mean of the 2^(D-1) finer faces they cover.
template <int D, int M, int MP>
__global__ void __launch_bounds__(kThreads) k_bc_restrict(BoxMeta A, int b0, int n, double *bc) {
    using Gm = Geo<D, M>;
    constexpr int MH = M / 2;
    constexpr int NF = D == 2 ? MH : MH * MH;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    pdl_trigger();
    pdl_wait();
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int idx = base + g;
        if (idx >= n) continue;
        const int b = b0 + idx, p = A.parent[b], po = A.poff[b];
        for (int s = 0; s < 2 * D; ++s) {
            if (A.nb[b * 2 * D + s] != -1) continue;
            const int a = s >> 1;
            const int ta1 = a == 0 ? 1 : 0, ta2 = a == 2 ? 1 : 2;
            const double *fb = bc + A.bcoff[b * 2 * D + s];
            double *pb = bc + A.bcoff[p * 2 * D + s];
            for (int f = lt; f < NF; f += Gm::G) {
                const int T1 = f % MH, T2 = D == 3 ? f / MH : 0;
                double sum = 0.0;
                for (int e2 = 0; e2 < (D == 3 ? 2 : 1); ++e2)
                    for (int e1 = 0; e1 < 2; ++e1) sum += fb[(2 * T2 + e2) * M + 2 * T1 + e1];
                const int P1 = unpack_off(po, ta1) + T1, P2 = D == 3 ? unpack_off(po, ta2) + T2 : 0;
                pb[P2 * MP + P1] = sum / double(1 << (D - 1));
            }
        }
    }
}

template <int D, int M>
__global__ void __launch_bounds__(kThreads) k_mixed_update(BoxMeta A, const int *list, int n, double *x, const float *e) {
    using Gm = Geo<D, M>;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    pdl_trigger();
    pdl_wait();
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int b = resolve_box<D, M>(A, base + g, n, 0, list);
        if (b < 0) continue;
        const long long cb = A.coff[b];
        for (int q = lt; q < Gm::C; q += Gm::G) x[cb + q] += double(e[cb + q]);
    }
}

// ---------------------------------------------------------------------------
// Transposed composite operator, out = K^T lam, on leaf boxes (FP64).
// K is the leaf system the FAS multigrid converges to: same-level leaf
// neighbours couple with 1/h^2; a face towards a refined same-level box sees
// the mean of the 2^D fine cells; a Dirichlet face adds -1/h^2 on the
// diagonal; a face towards a coarser leaf uses the conservative two-point
// ghost (coarse value 1/2, own cell 1 (2D) or 5/4 (3D), next inward and
// tangential partner(s) -1/4).  Its transpose is gathered per cell:
//   * ghost slots carry the symmetric part: same-level leaf lam; 2 * sum of
//     the 2^(D-1) adjacent fine lam for a refined neighbour; -lam (Dirichlet),
//     +lam (Neumann); c1 * lam (refinement boundary);
//   * at a refinement-boundary side the two cell layers next to it add
//     lam_C / 2^(D+2) (the coarse leaf's equation averages them), the first
//     layer adds -1/4 lam of its tangential partner(s), the second layer
//     -1/4 lam of the first-layer cell outside it.
// ---------------------------------------------------------------------------
template <int D, int M>
__global__ void __launch_bounds__(kThreads) k_adjoint_apply(BoxMeta A, const int *child, const double *hb,
                                                            const int *list, int n, const double *lam, double *out) {
    using Gm = Geo<D, M>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *tile = reinterpret_cast<double *>(smem_raw) + (threadIdx.x / Gm::G) * Gm::PC;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    pdl_trigger();
    pdl_wait();
    const double c1 = D == 2 ? 1.0 : 1.25;
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int b = resolve_box<D, M>(A, base + g, n, 0, list);
        if (b >= 0) {
            load_box<D, M, double>(lam, A.coff[b], tile, lt, 0, Gm::C);
        }
        __syncthreads();
        if (b >= 0) {
            for (int s = 0; s < 2 * D; ++s) {
                const int code = A.nb[b * 2 * D + s];
                const int hi = s & 1, a = s >> 1;
                const int pin = hi ? M - 1 : 0, pg = hi ? M : -1;
                for (int f = lt; f < Gm::F; f += Gm::G) {
                    const int t1 = f % M, t2 = D == 3 ? f / M : 0;
                    int i, j, k;
                    face_pos(D, s, pg, t1, t2, i, j, k);
                    const int gidx = ti<D, M>(i, j, k);
                    face_pos(D, s, pin, t1, t2, i, j, k);
                    const double self = tile[ti<D, M>(i, j, k)];
                    double v;
                    if (code >= 0 && !(A.bflag[code] & BF_REFINED)) {
                        int mi, mj, mk;
                        face_pos(D, s, hi ? 0 : M - 1, t1, t2, mi, mj, mk);
                        v = lam[A.coff[code] + rbi<D, M>(mi, mj, mk)];
                    } else if (code >= 0) {
                        // fine cells next to the face, in the children of the refined neighbour
                        const int ta1 = a == 0 ? 1 : 0, ta2 = a == 2 ? 1 : 2;
                        double sum = 0.0;
                        for (int e2 = 0; e2 < (D == 3 ? 2 : 1); ++e2)
                            for (int e1 = 0; e1 < 2; ++e1) {
                                int fc[3];
                                fc[a] = hi ? 0 : 2 * M - 1;
                                fc[ta1] = 2 * t1 + e1;
                                if (D == 3) fc[ta2] = 2 * t2 + e2;
                                int cidx = 0;
                                for (int e = 0; e < D; ++e) cidx |= (fc[e] / M) << e;
                                const int cbx = child[code * (1 << D) + cidx];
                                sum += lam[A.coff[cbx] + rbi<D, M>(fc[0] % M, fc[1] % M, D == 3 ? fc[2] % M : 0)];
                            }
                        v = 2.0 * sum;
                    } else if (code == -1) {  // the ghost's own-cell weight: -1 (2b - u) or +1 (u + h b)
                        v = ((A.nmask[b] >> s) & 1) ? self : -self;
                    } else {
                        v = c1 * self;
                    }
                    tile[gidx] = v;
                }
            }
        }
        __syncthreads();
        if (b >= 0) {
            const long long cb = A.coff[b];
            const double ih2 = A.ih2[b];
            const int po = A.poff[b];
            for (int q = lt; q < Gm::C; q += Gm::G) {
                int i, j, k;
                rb_cell<D, M>(q, i, j, k);
                const double lc = tile[ti<D, M>(i, j, k)];
                double acc = nb_sum<D, M, double>(tile, i, j, k) - double(2 * D) * lc;
                const int pc[3] = {i, j, k};
                for (int s = 0; s < 2 * D; ++s) {
                    const int code = A.nb[b * 2 * D + s];
                    if (code > -2) continue;
                    const int a = s >> 1, hi = s & 1;
                    const int pin = hi ? M - 1 : 0, p2 = hi ? M - 2 : 1;
                    if (pc[a] != pin && pc[a] != p2) continue;
                    const int ta1 = a == 0 ? 1 : 0, ta2 = a == 2 ? 1 : 2;
                    const int t1 = pc[ta1], t2 = D == 3 ? pc[ta2] : 0;
                    // coarse leaf across this side
                    int ci, cj, ck;
                    const int cc1 = unpack_off(po, ta1) + (t1 >> 1), cc2 = D == 3 ? unpack_off(po, ta2) + (t2 >> 1) : 0;
                    face_pos(D, s, hi ? 0 : M - 1, cc1, cc2, ci, cj, ck);
                    double extra = lam[A.coff[-2 - code] + rbi<D, M>(ci, cj, ck)] / double(1 << (D + 2));
                    int xi, xj, xk;
                    if (pc[a] == pin) {
                        face_pos(D, s, pin, t1 ^ 1, t2, xi, xj, xk);
                        double part = tile[ti<D, M>(xi, xj, xk)];
                        if (D == 3) {
                            face_pos(D, s, pin, t1, t2 ^ 1, xi, xj, xk);
                            part += tile[ti<D, M>(xi, xj, xk)];
                        }
                        extra -= 0.25 * part;
                    } else {
                        face_pos(D, s, pin, t1, t2, xi, xj, xk);
                        extra -= 0.25 * tile[ti<D, M>(xi, xj, xk)];
                    }
                    acc += extra;
                }
                out[cb + q] = acc * ih2;
            }
        }
        __syncthreads();
    }
}

template <int D, int M>
__global__ void __launch_bounds__(kThreads) k_adjoint_db(BoxMeta A, const double *hb, const int *list, int n,
                                                         const double *lam, double *db) {
    using Gm = Geo<D, M>;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    pdl_trigger();
    pdl_wait();
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int idx = base + g;
        if (idx >= n) continue;
        const int b = list[idx];
        const double h = hb[b];
        for (int s = 0; s < 2 * D; ++s) {
            if (A.nb[b * 2 * D + s] != -1) continue;
            const int pin = (s & 1) ? M - 1 : 0;
            for (int f = lt; f < Gm::F; f += Gm::G) {
                const int t1 = f % M, t2 = D == 3 ? f / M : 0;
                int i, j, k;
                face_pos(D, s, pin, t1, t2, i, j, k);
                // dA/db: 2/h^2 (Dirichlet ghost 2b - u) or 1/h (Neumann ghost u + h b)
                const double w = ((A.nmask[b] >> s) & 1) ? 1.0 / h : 2.0 / (h * h);
                db[A.bcoff[b * 2 * D + s] + f] = -w * lam[A.coff[b] + rbi<D, M>(i, j, k)];
            }
        }
    }
}

// ---- leaf vectors (double), one thread group per leaf box -----------------
template <int D, int M>
__global__ void __launch_bounds__(kThreads) k_leaf_axpbypcz(BoxMeta A, const int *list, int n, double *out,
                                                            double a, const double *x, double b, const double *y,
                                                            double c, const double *z) {
    using Gm = Geo<D, M>;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    pdl_trigger();
    pdl_wait();
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int bi = resolve_box<D, M>(A, base + g, n, 0, list);
        if (bi < 0) continue;
        const long long cb = A.coff[bi];
        for (int q = lt; q < Gm::C; q += Gm::G) {
            double v = a * x[cb + q];
            if (y) v += b * y[cb + q];
            if (z) v += c * z[cb + q];
            out[cb + q] = v;
        }
    }
}

template <int D, int M>
__global__ void __launch_bounds__(kThreads) k_leaf_scale(BoxMeta A, const double *hb, const int *list, int n,
                                                         double *out, const double *x, int power) {
    using Gm = Geo<D, M>;
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    pdl_trigger();
    pdl_wait();
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int bi = resolve_box<D, M>(A, base + g, n, 0, list);
        if (bi < 0) continue;
        const long long cb = A.coff[bi];
        double w = hb[bi] * hb[bi];
        if (D == 3) w *= hb[bi];
        if (power < 0) w = 1.0 / w;
        for (int q = lt; q < Gm::C; q += Gm::G) out[cb + q] = x[cb + q] * w;
    }
}

// per-CTA partial sums (mode 0: dot, 1: max |x|), fixed grid -> deterministic
template <int D, int M>
__global__ void __launch_bounds__(kThreads) k_leaf_reduce(BoxMeta A, const int *list, int n, const double *x,
                                                          const double *y, int mode, double *partials) {
    using Gm = Geo<D, M>;
    __shared__ double red[kThreads];
    const int lt = threadIdx.x % Gm::G, g = threadIdx.x / Gm::G;
    pdl_trigger();
    pdl_wait();
    double acc = 0.0;
    for (int base = blockIdx.x * Gm::BPC; base < n; base += gridDim.x * Gm::BPC) {
        const int bi = resolve_box<D, M>(A, base + g, n, 0, list);
        if (bi < 0) continue;
        const long long cb = A.coff[bi];
        for (int q = lt; q < Gm::C; q += Gm::G) {
            if (mode == 0) acc += x[cb + q] * y[cb + q];
            else acc = fmax(acc, fabs(x[cb + q]));
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = mode == 0 ? red[threadIdx.x] + red[threadIdx.x + o]
                                                          : fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

static __global__ void __launch_bounds__(kThreads) k_reduce_final(const double *partials, int n, int mode, double *result) {
    __shared__ double red[kThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) acc = mode == 0 ? acc + partials[i] : fmax(acc, partials[i]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = mode == 0 ? red[threadIdx.x] + red[threadIdx.x + o]
                                                          : fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *result = red[0];
}

}  // namespace afg
