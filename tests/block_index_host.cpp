// Host harness for the index helpers of csrc/block_bottom.cuh: for a block of
// root boxes (argv: D N nr0 nr1 nr2) prints, per block cell in rectangle order,
// its root and red-black index, then per side and face cell its root and the
// face cell within the box side.
#include <cstdio>
#include <cstdlib>

#include "../paper_1701_04329_gb300/csrc/block_bottom.cuh"

using namespace afg;

int main(int argc, char **argv) {
    if (argc != 6) return 2;
    const int D = atoi(argv[1]), N = atoi(argv[2]);
    const int nr[3] = {atoi(argv[3]), atoi(argv[4]), atoi(argv[5])};
    const BlkLevel L = blk_level(D, nr, N);
    for (long long c = 0; c < L.cells; ++c) {
        int i, j, k, root, q;
        blk_cell(L, c, i, j, k);
        blk_cell_home(D, N, nr, i, j, k, root, q);
        printf("c %d %d\n", root, q);
    }
    for (int s = 0; s < 2 * D; ++s) {
        int t1, t2;
        const int nf = blk_faces(L, s, t1, t2);
        for (int f = 0; f < nf; ++f) {
            int root, lf;
            blk_face_home(L, N, nr, s, f, root, lf);
            printf("f %d %d %d\n", s, root, lf);
        }
    }
    return 0;
}
