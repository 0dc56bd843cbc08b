// Host tree construction and mesh adaptation (arXiv:1701.04329, Sec. 2.1-2.3).
#include "host_tree.h"

#include <algorithm>

namespace afg {

namespace {
// spread the low 21 bits of v so that bit b lands on bit D*b
uint64_t spread(uint64_t v, int D) {
    uint64_t out = 0;
    for (int b = 0; v; ++b, v >>= 1)
        if (v & 1) out |= uint64_t(1) << (D * b);
    return out;
}
int pow3(int D) { return D == 2 ? 9 : 27; }
}  // namespace

uint64_t morton_key(int D, const int idx[3]) {
    uint64_t k = 0;
    for (int a = 0; a < D; ++a) k |= spread(uint64_t(idx[a] - 1), D) << a;
    return k;
}

HostTree::HostTree(int dim, int box_n, int maxl, const int *nroot) : D(dim), N(box_n), max_level(maxl) {
    if (nroot)
        for (int a = 0; a < D; ++a) nr[a] = nroot[a];
    std::vector<HBox> pos;
    for (int k = 1; k <= nr[2]; ++k)
        for (int j = 1; j <= nr[1]; ++j)
            for (int i = 1; i <= nr[0]; ++i) {
                HBox root{};
                root.level = 1;
                root.idx[0] = i;
                root.idx[1] = j;
                root.idx[2] = k;
                pos.push_back(root);
            }
    rebuild(std::move(pos));
}

int HostTree::ndir() const { return pow3(D) - 1; }

// Directions are numbered lexicographically over (dz, dy, dx) with dx
// fastest, skipping (0,0,0).
void HostTree::dir_offset(int d, int off[3]) const {
    int centre = (pow3(D) - 1) / 2;
    int full = d >= centre ? d + 1 : d;
    off[0] = off[1] = off[2] = 0;
    for (int a = 0; a < D; ++a) {
        off[a] = full % 3 - 1;
        full /= 3;
    }
}

int HostTree::side_dir(int s) const {
    int full = 0, m = 1;
    for (int a = 0; a < D; ++a) {
        int o = (a == s / 2) ? ((s & 1) ? 1 : -1) : 0;
        full += (o + 1) * m;
        m *= 3;
    }
    int centre = (pow3(D) - 1) / 2;
    return full > centre ? full - 1 : full;
}

int HostTree::find(int level, const int idx[3]) const {
    if (level < 1 || level > L) return -1;
    for (int a = 0; a < D; ++a)
        if (idx[a] < 1 || idx[a] > side_of(a, level)) return -1;
    const auto &m = lookup_[level];
    auto it = m.find(morton_key(D, idx));
    return it == m.end() ? -1 : it->second;
}

int HostTree::nfaces_of_leaf(int b) const {
    int n = 0, per = (D == 2) ? N : N * N;
    for (int s = 0; s < 2 * D; ++s)
        if (boxes[b].nb[side_dir(s)] == -2) n += per;
    return n;
}

int HostTree::wrap(int a, int q, int side) const {
    if (bct[2 * a] != 2) return q;
    return ((q - 1) % side + side) % side + 1;
}

int HostTree::set_boundary_types(const int *types, std::string &err) {
    bool any_dirichlet = false, change = false;
    for (int s = 0; s < 2 * D; ++s) {
        if (types[s] < 0 || types[s] > 2) { err = "unknown boundary type"; return -1; }
        if ((types[s] == 2) != (types[s ^ 1] == 2)) { err = "periodic sides come in pairs (both sides of an axis)"; return -1; }
        any_dirichlet |= types[s] == 0;
        change |= (types[s] == 2) != (bct[s] == 2);
    }
    (void)any_dirichlet;  // without a Dirichlet side the problem is singular; the solver handles it
    if (change && (int)boxes.size() != nroots()) { err = "periodic sides can only be switched while the tree is its root boxes"; return -1; }
    bool same = true;
    for (int s = 0; s < 2 * D; ++s) same &= bct[s] == types[s];
    if (same) return 0;
    for (int s = 0; s < 2 * D; ++s) bct[s] = types[s];
    std::vector<HBox> pos = boxes;
    rebuild(std::move(pos));  // neighbours (and the version) change
    return 0;
}

void HostTree::rebuild(std::vector<HBox> &&pos) {
    for (auto &p : pos) {
        if (D == 2) p.idx[2] = 1;
        p.key = morton_key(D, p.idx);
    }
    std::sort(pos.begin(), pos.end(), [](const HBox &a, const HBox &b) {
        return a.level != b.level ? a.level < b.level : a.key < b.key;
    });
    boxes = std::move(pos);
    L = boxes.empty() ? 0 : boxes.back().level;
    lstart.assign(L + 2, 0);
    lcount.assign(L + 2, 0);
    lookup_.assign(L + 2, {});
    for (int i = 0; i < (int)boxes.size(); ++i) {
        int l = boxes[i].level;
        if (lcount[l] == 0) lstart[l] = i;
        lcount[l]++;
        lookup_[l].emplace(boxes[i].key, i);
    }
    const int nc = 1 << D, nd = ndir();
    for (auto &b : boxes) {
        int p[3] = {1, 1, 1};
        for (int a = 0; a < D; ++a) p[a] = (b.idx[a] + 1) >> 1;
        b.parent = b.level > 1 ? find(b.level - 1, p) : -1;
        for (int c = 0; c < 8; ++c) b.child[c] = -1;
        for (int c = 0; c < nc; ++c) {
            int q[3] = {1, 1, 1};
            for (int a = 0; a < D; ++a) q[a] = 2 * b.idx[a] - 1 + ((c >> a) & 1);
            b.child[c] = find(b.level + 1, q);
        }
        for (int d = 0; d < 26; ++d) b.nb[d] = -1;
        for (int d = 0; d < nd; ++d) {
            int off[3], q[3] = {1, 1, 1};
            dir_offset(d, off);
            bool inside = true;
            for (int a = 0; a < D; ++a) {
                const int side = side_of(a, b.level);
                q[a] = wrap(a, b.idx[a] + off[a], side);
                inside = inside && q[a] >= 1 && q[a] <= side;
            }
            b.nb[d] = inside ? find(b.level, q) : -2;
        }
    }
    leaves.clear();
    leaf_cell0.clear();
    leaf_face0.clear();
    long long cells = 0, faces = 0, per = (D == 2) ? N * N : N * N * N;
    for (int i = 0; i < (int)boxes.size(); ++i) {
        if (!boxes[i].leaf()) continue;
        leaves.push_back(i);
        leaf_cell0.push_back(cells);
        leaf_face0.push_back(faces);
        cells += per;
        faces += nfaces_of_leaf(i);
    }
    n_leaf_cells = cells;
    n_bfaces = faces;
    ++version;
}

int HostTree::refine_uniform(int level, std::string &err) {
    if (level < 1 || level > max_level) {
        err = "refine_uniform: level outside [1, max_level]";
        return -1;
    }
    while (true) {
        std::vector<HBox> pos(boxes.begin(), boxes.end());
        bool any = false;
        for (int b : leaves) {
            if (boxes[b].level >= level) continue;
            any = true;
            for (int c = 0; c < (1 << D); ++c) {
                HBox k{};
                k.level = boxes[b].level + 1;
                for (int a = 0; a < 3; ++a) k.idx[a] = a < D ? 2 * boxes[b].idx[a] - 1 + ((c >> a) & 1) : 1;
                pos.push_back(k);
            }
        }
        if (!any) return 0;
        rebuild(std::move(pos));
    }
}

int HostTree::adapt(const int8_t *flags, int n_buf, int *n_added, int *n_removed, std::string &err) {
    if (n_buf < 0 || n_buf > N) {
        err = "adapt: n_buf outside [0, box_n]";
        return -1;
    }
    const int nb = (int)boxes.size(), nd = ndir(), nc = 1 << D;
    const long long ncell = (D == 2) ? N * N : N * N * N;
    std::vector<char> refine(nb, 0), remove(nb, 0);
    std::vector<int> leaf_of(nb, -1);
    for (int i = 0; i < (int)leaves.size(); ++i) leaf_of[leaves[i]] = i;

    // cell flags -> box flags, with the buffer zone of n_buf cells
    for (int i = 0; i < (int)leaves.size(); ++i) {
        const int b = leaves[i];
        if (boxes[b].level >= max_level) continue;
        const int8_t *f = flags + (long long)i * ncell;
        for (long long c = 0; c < ncell; ++c) {
            if (f[c] <= 0) {
                if (f[c] < -1) { err = "adapt: flag out of range"; return -1; }
                continue;
            }
            if (f[c] != 1) { err = "adapt: flag out of range"; return -1; }
            refine[b] = 1;
            int ci[3] = {int(c % N), int((c / N) % N), int(c / (N * N))};
            for (int d = 0; d < nd; ++d) {
                int off[3];
                dir_offset(d, off);
                bool close = true;
                for (int a = 0; a < D && close; ++a) {
                    if (off[a] < 0) close = ci[a] < n_buf;
                    else if (off[a] > 0) close = ci[a] >= N - n_buf;
                }
                const int q = boxes[b].nb[d];
                if (close && q >= 0 && boxes[q].leaf()) refine[q] = 1;
            }
        }
    }
    for (int i = 0; i < (int)leaves.size(); ++i) {  // validate the remaining flags
        const int8_t *f = flags + (long long)i * ncell;
        for (long long c = 0; c < ncell; ++c)
            if (f[c] < -1 || f[c] > 1) { err = "adapt: flag out of range"; return -1; }
    }
    // 2:1 balance: finest level first, so that induced refinements cascade
    for (int l = L; l >= 2; --l) {
        for (int b = lstart[l]; b < lstart[l] + lcount[l]; ++b) {
            if (!refine[b]) continue;
            for (int d = 0; d < nd; ++d) {
                if (boxes[b].nb[d] != -1) continue;
                int off[3], q[3] = {1, 1, 1};
                dir_offset(d, off);
                for (int a = 0; a < D; ++a) q[a] = (wrap(a, boxes[b].idx[a] + off[a], side_of(a, l)) + 1) >> 1;
                const int c = find(l - 1, q);
                if (c < 0 || !boxes[c].leaf()) { err = "adapt: tree not 2:1 balanced"; return -4; }
                refine[c] = 1;
            }
        }
    }
    // derefinement of parents whose children are all removable leaves
    int removed = 0;
    for (int p = 0; p < nb; ++p) {
        if (boxes[p].leaf()) continue;
        bool ok = true;
        for (int c = 0; c < nc && ok; ++c) {
            const int k = boxes[p].child[c];
            if (!boxes[k].leaf() || refine[k]) { ok = false; break; }
            const int8_t *f = flags + (long long)leaf_of[k] * ncell;
            for (long long q = 0; q < ncell; ++q)
                if (f[q] != -1) { ok = false; break; }
        }
        for (int d = 0; d < nd && ok; ++d) {
            const int q = boxes[p].nb[d];
            if (q < 0 || boxes[q].leaf()) continue;
            for (int c = 0; c < nc; ++c) {
                const int k = boxes[q].child[c];
                if (!boxes[k].leaf() || refine[k]) { ok = false; break; }
            }
        }
        if (ok) {
            for (int c = 0; c < nc; ++c) remove[boxes[p].child[c]] = 1;
            removed += nc;
        }
    }
    std::vector<HBox> pos;
    pos.reserve(nb + nc * nb);
    int added = 0;
    for (int b = 0; b < nb; ++b) {
        if (remove[b]) continue;
        pos.push_back(boxes[b]);
        if (!refine[b]) continue;
        for (int c = 0; c < nc; ++c) {
            HBox k{};
            k.level = boxes[b].level + 1;
            for (int a = 0; a < 3; ++a) k.idx[a] = a < D ? 2 * boxes[b].idx[a] - 1 + ((c >> a) & 1) : 1;
            pos.push_back(k);
            ++added;
        }
    }
    if (n_added) *n_added = added;
    if (n_removed) *n_removed = removed;
    if (added || removed) rebuild(std::move(pos));
    return 0;
}

}  // namespace afg
