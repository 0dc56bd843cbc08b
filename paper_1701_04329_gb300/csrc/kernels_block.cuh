// The bottom of the multigrid hierarchy for a tree whose level 1 is a block
// of r_x x r_y (x r_z) root boxes (arXiv:1701.04329 Sec. 2.2; Sec. 3.2: the
// coarse grids of a non-square domain hold several boxes, relaxed together).
// One CTA per tree stages its level-1 boxes (solution, copy v', source term,
// domain face data) into one rectangular grid per level in shared memory --
// level 1 and the grids of N/2, ..., 2 cells per root below it, which exist
// only here -- runs the part of the cycle at and below level 1 with the steps
// of block_bottom.cuh separated by block barriers, and writes level 1 back.
//
// mode 0: one V-cycle from level 1 down to the coarsest grid and back.
// mode 1: the FMG cycle below level 2: level-1 values restricted down, the
//         coarse right-hand sides formed, then for l = coarsest .. 1: v'_l =
//         u_l, correction from l-1 (l above the coarsest), V-cycle from l;
//         level 1's v' is written back for the FMG correction of level 2.
//
// The steps reproduce the oracle's cycle bit for bit on the host; the
// kernel is what the cycle drivers call at level 1 for such trees.
#pragma once
#include "block_bottom.cuh"
#include "kernels.cuh"

namespace afg {

// one tree whose level 1 is a block of root boxes
struct BlockTree {
    int nroot[3];          // root boxes per axis (1 along z in 2D)
    int bct[6];            // side types: 0 Dirichlet, 1 Neumann, 2 periodic
    const int *root_box;   // box id of root (ri, rj, rk): index ri + nroot0 (rj + nroot1 rk)
};

constexpr int kBlockMaxLevels = 4;  // box sizes 2 .. 16

// shared memory of k_bottom_block: per level u, rho, v' and a work array
// (residual, then the correction's difference) with ghost layers, and the
// face data of the non-periodic sides
template <int D, typename T>
inline size_t block_bottom_smem(int N, const BlockTree &B) {
    size_t n = 0;
    for (int M = 2; M <= N; M *= 2) {
        const BlkLevel L = blk_level(D, B.nroot, M);
        n += 4 * (size_t)L.padded;
        for (int s = 0; s < 2 * D; ++s) {
            int t1, t2;
            if (B.bct[s] != 2) n += (size_t)blk_faces(L, s, t1, t2);
        }
    }
    return n * sizeof(T);
}

template <int D, typename T>
__global__ void __launch_bounds__(kThreads) k_bottom_block(BoxMeta A, BlockTree B, int N, int mode, T *u, T *rho,
                                                           T *vold, int nd, int nu, int nb, int hom) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x, nth = blockDim.x;
    BlkLevel L[kBlockMaxLevels];
    T *fu[kBlockMaxLevels], *frho[kBlockMaxLevels], *fv[kBlockMaxLevels], *fw[kBlockMaxLevels];
    const T *fbc[kBlockMaxLevels][6];
    T *wbc[kBlockMaxLevels][6];
    int nl = 0;
    size_t off = 0;
    for (int M = 2; M <= N && nl < kBlockMaxLevels; M *= 2, ++nl) {
        L[nl] = blk_level(D, B.nroot, M);
        fu[nl] = sm + off;
        off += L[nl].padded;
        frho[nl] = sm + off;
        off += L[nl].padded;
        fv[nl] = sm + off;
        off += L[nl].padded;
        fw[nl] = sm + off;
        off += L[nl].padded;
        for (int s = 0; s < 6; ++s) {
            wbc[nl][s] = nullptr;
            int t1, t2;
            if (s < 2 * D && B.bct[s] != 2) {
                wbc[nl][s] = sm + off;
                off += blk_faces(L[nl], s, t1, t2);
            }
            fbc[nl][s] = wbc[nl][s];
        }
    }
    const int top = nl - 1;  // level 1
    const BlkLevel &LT = L[top];
    pdl_trigger();
    pdl_wait();
    for (size_t g = tid; g < off; g += nth) sm[g] = T(0);
    __syncthreads();
    // stage level 1: cell (i,j,k) of the block lies in root ((i-1)/N, ...)
    for (long long c = tid; c < LT.cells; c += nth) {
        int i, j, k;
        blk_cell(LT, c, i, j, k);
        int root, q;
        blk_cell_home(D, N, B.nroot, i, j, k, root, q);
        const long long src = A.coff[B.root_box[root]] + q;
        const long long g = blk_at(LT, i, j, k);
        fu[top][g] = u[src];
        frho[top][g] = rho[src];
        fv[top][g] = vold[src];
    }
    for (int s = 0; s < 2 * D; ++s) {
        if (B.bct[s] == 2) continue;
        int t1, t2;
        const int nf = blk_faces(LT, s, t1, t2);
        for (int f = tid; f < nf; f += nth) {
            int root, lf;
            blk_face_home(LT, N, B.nroot, s, f, root, lf);
            const int b = B.root_box[root];
            wbc[top][s][f] = hom ? T(0) : T(A.bc[A.nbase[b * 2 * D + s] + lf]);
        }
    }
    __syncthreads();
    for (int li = top; li > 0; --li) {
        for (int s = 0; s < 2 * D; ++s)
            if (B.bct[s] != 2) blk_bc_restrict(L[li], L[li - 1], s, fbc[li][s], wbc[li - 1][s], tid, nth);
        __syncthreads();
    }
    // the steps of the cycle, as in the oracle's sequence
    auto ghosts = [&](int li, T *v, bool zero_b) {
        blk_fill_ghosts(L[li], v, fbc[li], B.bct, zero_b || hom, tid, nth);
        __syncthreads();
    };
    auto smooth = [&](int li, int n) {
        for (int it = 0; it < n; ++it)
            for (int c = 0; c < 2; ++c) {
                ghosts(li, fu[li], false);
                blk_gsrb(L[li], fu[li], frho[li], c, tid, nth);
                __syncthreads();
            }
    };
    auto fas_coarse = [&](int li) {  // rr is in frho: rho = rr + A(u) in place
        ghosts(li, fu[li], false);
        blk_copy(L[li], fv[li], fu[li], tid, nth);
        blk_fas(L[li], fu[li], frho[li], frho[li], tid, nth);
        __syncthreads();
    };
    auto down = [&](int li) {
        ghosts(li, fu[li], false);
        blk_residual(L[li], fu[li], frho[li], fw[li], tid, nth);
        __syncthreads();
        blk_restrict(L[li], L[li - 1], fu[li], fu[li - 1], tid, nth);
        blk_restrict(L[li], L[li - 1], fw[li], frho[li - 1], tid, nth);
        __syncthreads();
        fas_coarse(li - 1);
    };
    auto correct = [&](int li) {
        blk_diff(L[li - 1], fw[li - 1], fu[li - 1], fv[li - 1], tid, nth);
        __syncthreads();
        ghosts(li - 1, fw[li - 1], true);
        blk_correct(L[li], L[li - 1], fu[li], fw[li - 1], tid, nth);
        __syncthreads();
    };
    auto vcycle_from = [&](int t) {
        for (int li = t; li > 0; --li) {
            smooth(li, nd);
            down(li);
        }
        smooth(0, nb);
        for (int li = 1; li <= t; ++li) {
            correct(li);
            smooth(li, nu);
        }
    };
    if (mode == 0) {
        vcycle_from(top);
    } else {
        for (int li = top; li > 0; --li) {
            blk_restrict(L[li], L[li - 1], fu[li], fu[li - 1], tid, nth);
            __syncthreads();
        }
        for (int li = top; li > 0; --li) {
            ghosts(li, fu[li], false);
            blk_residual(L[li], fu[li], frho[li], fw[li], tid, nth);
            __syncthreads();
            blk_restrict(L[li], L[li - 1], fw[li], frho[li - 1], tid, nth);
            __syncthreads();
            fas_coarse(li - 1);
        }
        for (int li = 0; li <= top; ++li) {
            blk_copy(L[li], fv[li], fu[li], tid, nth);
            __syncthreads();
            if (li > 0) correct(li);
            vcycle_from(li);
        }
    }
    // write level 1 back (u; v' as well, set by the FMG steps)
    for (long long c = tid; c < LT.cells; c += nth) {
        int i, j, k;
        blk_cell(LT, c, i, j, k);
        int root, q;
        blk_cell_home(D, N, B.nroot, i, j, k, root, q);
        const long long dst = A.coff[B.root_box[root]] + q;
        const long long g = blk_at(LT, i, j, k);
        u[dst] = fu[top][g];
        if (mode == 1) vold[dst] = fv[top][g];
    }
}

}  // namespace afg
