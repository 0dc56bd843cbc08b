// Host harness for csrc/block_bottom.cuh: the part of the multigrid cycle at
// and below level 1 of a tree whose level 1 is a block of root boxes, run
// with one thread.  Input (binary, doubles unless noted): int32 header
// D, N, nr[3], bct[6], mode (0 one V-cycle, 1 one FMG cycle), nd, nu, nb, op
// (0 Laplacian, 1 div(eps grad), 2 the same in (r,z)); then level-1 rho, u
// and eps (rectangle order with ghosts dropped: n0 x n1 (x n2), x fastest)
// and the face data of every non-periodic side (f1 + n[t1] f2).
// Output: level-1 u in the same order.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_1701_04329_gb300/csrc/block_bottom.cuh"

using namespace afg;
typedef std::vector<double> Vec;

struct Lev {
    BlkLevel L;
    Vec u, rho, vold, r, rr, d, eps;
    int M;
    Vec bc[6];
};

static int D, N, nr[3], bct[6], mode, nd, nu, nb, op;
static std::vector<Lev> lv;  // index 0 = coarsest (M = 2), last = level 1 (M = N)

static const double *const *bcp(Lev &l, const double **buf) {
    for (int s = 0; s < 6; ++s) buf[s] = l.bc[s].empty() ? nullptr : l.bc[s].data();
    return buf;
}
static void ghosts(Lev &l, Vec &v, bool zero_b) {
    const double *buf[6];
    blk_fill_ghosts(l.L, v.data(), bcp(l, buf), bct, zero_b, 0, 1);
}
static void smooth(int li, int n) {
    for (int it = 0; it < n; ++it)
        for (int c = 0; c < 2; ++c) {
            ghosts(lv[li], lv[li].u, false);
            if (op) blk_gsrb_v(lv[li].L, lv[li].M, op, lv[li].eps.data(), lv[li].u.data(), lv[li].rho.data(), c, 0, 1);
            else blk_gsrb(lv[li].L, lv[li].u.data(), lv[li].rho.data(), c, 0, 1);
        }
}
static void fas_coarse(int li) {
    Lev &c = lv[li];
    ghosts(c, c.u, false);
    blk_copy(c.L, c.vold.data(), c.u.data(), 0, 1);
    if (op) blk_fas_v(c.L, c.M, op, c.eps.data(), c.u.data(), c.rr.data(), c.rho.data(), 0, 1);
    else blk_fas(c.L, c.u.data(), c.rr.data(), c.rho.data(), 0, 1);
}
static void correct(int li) {  // fine level li from li - 1
    Lev &c = lv[li - 1], &f = lv[li];
    blk_diff(c.L, c.d.data(), c.u.data(), c.vold.data(), 0, 1);
    ghosts(c, c.d, true);
    blk_correct(f.L, c.L, f.u.data(), c.d.data(), 0, 1);
}
static void residual(Lev &f) {
    if (op) blk_residual_v(f.L, f.M, op, f.eps.data(), f.u.data(), f.rho.data(), f.r.data(), 0, 1);
    else blk_residual(f.L, f.u.data(), f.rho.data(), f.r.data(), 0, 1);
}
static void restrict_to(Lev &f, Lev &c, const Vec &vf, Vec &vc) {
    blk_restrict_v(f.L, c.L, f.M, op, vf.data(), vc.data(), 0, 1);
}
static void down(int li) {  // residual of li restricted into li - 1, coarse rhs
    Lev &f = lv[li], &c = lv[li - 1];
    ghosts(f, f.u, false);
    residual(f);
    restrict_to(f, c, f.u, c.u);
    restrict_to(f, c, f.r, c.rr);
    fas_coarse(li - 1);
}
static void vcycle_from(int top) {
    for (int li = top; li > 0; --li) {
        smooth(li, nd);
        down(li);
    }
    smooth(0, nb);
    for (int li = 1; li <= top; ++li) {
        correct(li);
        smooth(li, nu);
    }
}

int main(int argc, char **argv) {
    if (argc != 3) return 2;
    FILE *in = fopen(argv[1], "rb");
    if (!in) return 3;
    int hdr[16];
    if (fread(hdr, sizeof(int), 16, in) != 16) return 4;
    D = hdr[0]; N = hdr[1];
    for (int a = 0; a < 3; ++a) nr[a] = hdr[2 + a];
    for (int s = 0; s < 6; ++s) bct[s] = hdr[5 + s];
    mode = hdr[11]; nd = hdr[12]; nu = hdr[13]; nb = hdr[14]; op = hdr[15];
    for (int M = 2; M <= N; M *= 2) {
        Lev l;
        l.L = blk_level(D, nr, M);
        l.M = M;
        for (Vec *v : {&l.u, &l.rho, &l.vold, &l.r, &l.rr, &l.d}) v->assign(l.L.padded, 0.0);
        l.eps.assign(l.L.padded, 1.0);
        lv.push_back(l);
    }
    Lev &top = lv.back();
    const int nl = (int)lv.size();
    for (Vec *v : {&top.rho, &top.u, &top.eps})
        for (long long c = 0; c < top.L.cells; ++c) {
            int i, j, k;
            blk_cell(top.L, c, i, j, k);
            if (fread(&(*v)[blk_at(top.L, i, j, k)], 8, 1, in) != 1) return 5;
        }
    for (int li = nl - 1; li >= 0; --li)
        for (int s = 0; s < 2 * D; ++s) {
            if (bct[s] == 2) continue;
            int t1, t2;
            lv[li].bc[s].assign(blk_faces(lv[li].L, s, t1, t2), 0.0);
            if (li == nl - 1) {
                if (fread(lv[li].bc[s].data(), 8, lv[li].bc[s].size(), in) != lv[li].bc[s].size()) return 6;
            } else {
                blk_bc_restrict(lv[li + 1].L, lv[li].L, s, lv[li + 1].bc[s].data(), lv[li].bc[s].data(), 0, 1);
            }
        }
    fclose(in);
    // the coefficient on every level: restricted down, then its ghosts
    for (int li = nl - 1; li > 0; --li) restrict_to(lv[li], lv[li - 1], lv[li].eps, lv[li - 1].eps);
    for (int li = 0; li < nl; ++li) blk_fill_eps_ghosts(lv[li].L, lv[li].eps.data(), bct, 0, 1);
    if (mode == 0) {
        vcycle_from(nl - 1);
    } else {  // FMG: restrict u down, coarse right-hand sides, then up level by level
        for (int li = nl - 1; li > 0; --li) restrict_to(lv[li], lv[li - 1], lv[li].u, lv[li - 1].u);
        for (int li = nl - 1; li > 0; --li) {
            Lev &f = lv[li], &c = lv[li - 1];
            ghosts(f, f.u, false);
            residual(f);
            restrict_to(f, c, f.r, c.rr);
            fas_coarse(li - 1);
        }
        for (int li = 0; li < nl; ++li) {
            blk_copy(lv[li].L, lv[li].vold.data(), lv[li].u.data(), 0, 1);
            if (li > 0) correct(li);
            vcycle_from(li);
        }
    }
    FILE *out = fopen(argv[2], "wb");
    if (!out) return 7;
    for (long long c = 0; c < top.L.cells; ++c) {
        int i, j, k;
        blk_cell(top.L, c, i, j, k);
        fwrite(&top.u[blk_at(top.L, i, j, k)], 8, 1, out);
    }
    fclose(out);
    return 0;
}
