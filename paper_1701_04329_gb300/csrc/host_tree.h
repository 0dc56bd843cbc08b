// Host-side quadtree/octree: boxes, per-level lists and connectivity
// (Teunissen & Ebert, arXiv:1701.04329, Sec. 2.1-2.3).  The tree is rebuilt
// from its set of box positions after every change and kept in canonical
// order (level ascending, Morton order within a level), so that box ids are
// reproducible.  Position lookups go through one hash map per level.
#pragma once
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

namespace afg {

struct HBox {
    int level;        // 1 = root
    int idx[3];       // 1-based spatial index
    uint64_t key;     // Morton key of idx-1 (x in the lowest bit)
    int parent;       // -1 for the root
    int child[8];     // -1 when a leaf
    int nb[26];       // same-level neighbour, -1 none, -2 domain boundary
    bool leaf() const { return child[0] < 0; }
};

class HostTree {
  public:
    // nroot: root boxes per axis (null = one); the domain is the block of
    // nroot[0] x nroot[1] (x nroot[2]) unit root boxes (Sec. 2.2)
    HostTree(int dim, int box_n, int max_level, const int *nroot = nullptr);

    int D, N, max_level;
    int nr[3] = {1, 1, 1};             // root boxes per axis
    std::vector<HBox> boxes;           // canonical order
    std::vector<int> lstart, lcount;   // per level (index = level)
    int L = 0;                         // highest level present
    std::vector<int> leaves;           // leaf box ids, canonical order
    std::vector<long long> leaf_cell0; // first canonical leaf cell of leaf i
    std::vector<long long> leaf_face0; // first canonical boundary face of leaf i
    long long n_leaf_cells = 0, n_bfaces = 0;
    int version = 0;                   // bumped on every change
    int bct[6] = {0, 0, 0, 0, 0, 0};   // per domain side (-x,+x,-y,+y,-z,+z): 0 Dirichlet, 1 Neumann, 2 periodic

    int ndir() const;                  // 3^D - 1
    int nroots() const { return nr[0] * nr[1] * nr[2]; }
    int side_of(int a, int level) const { return nr[a] << (level - 1); }  // boxes per axis
    int side_dir(int s) const;         // face side (-x,+x,-y,...) -> direction index
    void dir_offset(int d, int off[3]) const;
    int find(int level, const int idx[3]) const;  // box id or -1
    int nfaces_of_leaf(int b) const;

    int refine_uniform(int level, std::string &err);
    // side types; periodicity (both sides of an axis) changes the connectivity and is
    // accepted only while the tree is its root boxes alone
    int set_boundary_types(const int *types, std::string &err);
    int wrap(int a, int q, int side) const;  // index q on axis a, wrapped on a periodic axis
    int adapt(const int8_t *flags, int n_buf, int *n_added, int *n_removed, std::string &err);

  private:
    std::vector<std::unordered_map<uint64_t, int>> lookup_;
    void rebuild(std::vector<HBox> &&pos);
};

uint64_t morton_key(int D, const int idx[3]);

}  // namespace afg
