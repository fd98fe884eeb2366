// Host-side adaptive quadtree and interaction lists of the fast multipole method
// that evaluates the smooth-quadrature point sum. The paper treats the FMM as a
// black box (Sec. 1 synopsis; Sec. 4, paragraph after Eq. nsrcs); the tree and
// list definitions here are the standard adaptive ones (U: adjacent leaves,
// V: well-separated children of the parent's neighbours, W/X: the mixed-level
// pairs of an adaptive tree).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace vp {

constexpr int kCoordBits = 28;  // integer coordinate bits per axis; also the level cap + 1

struct TreeOptions {
    int leaf = 64;
    int max_level = 24;
    double root[3] = {0.0, 0.0, 0.0};  // (x0, y0, side); side <= 0 -> derived
};

struct Tree {
    double x0 = 0.0, y0 = 0.0, side = 1.0;
    int n_levels = 0;                    // deepest level + 1
    int64_t n_src = 0, n_tgt = 0;
    // per box (boxes are stored level by level; children of one box are contiguous)
    std::vector<int32_t> level, ix, iy, parent, child;  // child: 4 per box, -1 if absent
    std::vector<int32_t> is_leaf;
    std::vector<int32_t> src_begin, src_end, tgt_begin, tgt_end;
    std::vector<int32_t> level_start;    // [n_levels + 1]
    std::vector<int32_t> src_perm, tgt_perm;  // sorted position -> caller index
    // interaction lists in CSR form over boxes
    std::vector<int32_t> u_ptr, u_idx;   // leaf B: leaves adjacent to B (B included)
    std::vector<int32_t> v_ptr, v_idx;   // box B: children of parent's colleagues, not adjacent
    std::vector<int32_t> w_ptr, w_idx;   // leaf B: boxes D, D not adjacent to B, parent(D) adjacent
    std::vector<int32_t> x_ptr, x_idx;   // box B: leaves C with B in W(C)

    int64_t n_boxes() const { return (int64_t)level.size(); }
    double box_side(int b) const { return side / (double)(1LL << level[b]); }
    double box_cx(int b) const { return x0 + ((double)ix[b] + 0.5) * box_side(b); }
    double box_cy(int b) const { return y0 + ((double)iy[b] + 0.5) * box_side(b); }
};

// Builds the tree over all sources and targets. Returns "" on success, else a
// message (invalid input). Points are interleaved (x, y).
std::string build_tree(int64_t n_src, const double* src_xy, int64_t n_tgt, const double* tgt_xy,
                       const TreeOptions& opt, Tree& t);

bool boxes_adjacent(const Tree& t, int a, int b);

}  // namespace vp
