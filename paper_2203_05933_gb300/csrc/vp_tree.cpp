// Host construction of the adaptive quadtree and the U/V/W/X interaction lists.
// See vp_tree.h. Points are Morton-ordered on 28-bit integer coordinates inside
// the root square; a box splits while it holds more than `leaf` sources or more
// than `leaf` targets, up to max_level. Empty children are not created.
#include "vp_tree.h"

#include <algorithm>
#include <cmath>
#include <unordered_map>

namespace vp {
namespace {

inline uint64_t spread_bits(uint64_t v)
{
    // spread the low 32 bits of v to the even bit positions
    v &= 0xffffffffULL;
    v = (v | (v << 16)) & 0x0000ffff0000ffffULL;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffULL;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0fULL;
    v = (v | (v << 2)) & 0x3333333333333333ULL;
    v = (v | (v << 1)) & 0x5555555555555555ULL;
    return v;
}

inline uint64_t morton(uint32_t ix, uint32_t iy) { return spread_bits(ix) | (spread_bits(iy) << 1); }

struct Keyed {
    uint64_t key;
    int32_t idx;
};

std::string quantise(int64_t n, const double* xy, double x0, double y0, double side, bool clamp,
                     std::vector<Keyed>& out)
{
    const double scale = (double)(1u << kCoordBits) / side;
    const int64_t maxc = (1LL << kCoordBits) - 1;
    out.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const double x = xy[2 * i], y = xy[2 * i + 1];
        if (!std::isfinite(x) || !std::isfinite(y)) return "non-finite point coordinate";
        int64_t cx = (int64_t)std::floor((x - x0) * scale);
        int64_t cy = (int64_t)std::floor((y - y0) * scale);
        if (clamp) {
            cx = std::min<int64_t>(std::max<int64_t>(cx, 0), maxc);
            cy = std::min<int64_t>(std::max<int64_t>(cy, 0), maxc);
        } else if (cx < 0 || cy < 0 || cx > maxc || cy > maxc) {
            return "point outside the root box";
        }
        out[(size_t)i] = Keyed{morton((uint32_t)cx, (uint32_t)cy), (int32_t)i};
    }
    std::sort(out.begin(), out.end(), [](const Keyed& a, const Keyed& b) {
        return a.key < b.key || (a.key == b.key && a.idx < b.idx);
    });
    return "";
}

// first position in [lo, hi) whose key >= k
inline int32_t lower(const std::vector<Keyed>& v, int32_t lo, int32_t hi, uint64_t k)
{
    auto it = std::lower_bound(v.begin() + lo, v.begin() + hi, k,
                               [](const Keyed& a, uint64_t kk) { return a.key < kk; });
    return (int32_t)(it - v.begin());
}

inline uint64_t hash_key(int level, int32_t ix, int32_t iy)
{
    return ((uint64_t)level << 56) | ((uint64_t)(uint32_t)ix << 28) | (uint64_t)(uint32_t)iy;
}

void to_csr(const std::vector<std::vector<int32_t>>& lists, std::vector<int32_t>& ptr,
            std::vector<int32_t>& idx)
{
    ptr.assign(lists.size() + 1, 0);
    size_t total = 0;
    for (size_t b = 0; b < lists.size(); ++b) {
        total += lists[b].size();
        ptr[b + 1] = (int32_t)total;
    }
    idx.clear();
    idx.reserve(total);
    for (auto& l : lists) idx.insert(idx.end(), l.begin(), l.end());
}

}  // namespace

bool boxes_adjacent(const Tree& t, int a, int b)
{
    const int L = std::max(t.level[a], t.level[b]);
    const int64_t sa = 1LL << (L - t.level[a]);
    const int64_t sb = 1LL << (L - t.level[b]);
    const int64_t ax0 = (int64_t)t.ix[a] * sa, ax1 = ax0 + sa;
    const int64_t ay0 = (int64_t)t.iy[a] * sa, ay1 = ay0 + sa;
    const int64_t bx0 = (int64_t)t.ix[b] * sb, bx1 = bx0 + sb;
    const int64_t by0 = (int64_t)t.iy[b] * sb, by1 = by0 + sb;
    return ax0 <= bx1 && bx0 <= ax1 && ay0 <= by1 && by0 <= ay1;
}

std::string build_tree(int64_t n_src, const double* src_xy, int64_t n_tgt, const double* tgt_xy,
                       const TreeOptions& opt, Tree& t)
{
    if (n_src < 0 || n_tgt < 0) return "negative point count";
    if (n_src > INT32_MAX / 2 || n_tgt > INT32_MAX / 2) return "too many points";
    if (opt.leaf < 1 || opt.leaf > 4096) return "leaf size outside [1, 4096]";
    if (opt.max_level < 0 || opt.max_level >= kCoordBits) return "max_level outside [0, 27]";
    t = Tree();
    t.n_src = n_src;
    t.n_tgt = n_tgt;

    // root square
    bool clamp = false;
    if (opt.root[2] > 0.0) {
        if (!std::isfinite(opt.root[0]) || !std::isfinite(opt.root[1]) || !std::isfinite(opt.root[2]))
            return "non-finite root box";
        t.x0 = opt.root[0];
        t.y0 = opt.root[1];
        t.side = opt.root[2];
    } else {
        double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
        auto scan = [&](int64_t n, const double* xy) {
            for (int64_t i = 0; i < n; ++i) {
                xmin = std::min(xmin, xy[2 * i]);
                xmax = std::max(xmax, xy[2 * i]);
                ymin = std::min(ymin, xy[2 * i + 1]);
                ymax = std::max(ymax, xy[2 * i + 1]);
            }
        };
        scan(n_src, src_xy);
        scan(n_tgt, tgt_xy);
        if (n_src + n_tgt == 0) {
            xmin = ymin = 0.0;
            xmax = ymax = 1.0;
        }
        if (!std::isfinite(xmin) || !std::isfinite(xmax) || !std::isfinite(ymin) || !std::isfinite(ymax))
            return "non-finite point coordinate";
        double side = std::max(xmax - xmin, ymax - ymin);
        if (!(side > 0.0)) side = 1.0;
        side *= 1.0 + 1.0 / 1048576.0;
        t.side = side;
        t.x0 = 0.5 * (xmin + xmax) - 0.5 * side;
        t.y0 = 0.5 * (ymin + ymax) - 0.5 * side;
        clamp = true;
    }

    std::vector<Keyed> ks, kt;
    std::string err = quantise(n_src, src_xy, t.x0, t.y0, t.side, clamp, ks);
    if (!err.empty()) return err;
    err = quantise(n_tgt, tgt_xy, t.x0, t.y0, t.side, clamp, kt);
    if (!err.empty()) return err;
    t.src_perm.resize((size_t)n_src);
    t.tgt_perm.resize((size_t)n_tgt);
    for (int64_t i = 0; i < n_src; ++i) t.src_perm[(size_t)i] = ks[(size_t)i].idx;
    for (int64_t i = 0; i < n_tgt; ++i) t.tgt_perm[(size_t)i] = kt[(size_t)i].idx;

    // breadth-first splitting; boxes end up stored level by level
    auto push_box = [&](int lvl, int32_t bx, int32_t by, int32_t par, int32_t s0, int32_t s1, int32_t t0,
                        int32_t t1) {
        t.level.push_back(lvl);
        t.ix.push_back(bx);
        t.iy.push_back(by);
        t.parent.push_back(par);
        for (int c = 0; c < 4; ++c) t.child.push_back(-1);
        t.is_leaf.push_back(1);
        t.src_begin.push_back(s0);
        t.src_end.push_back(s1);
        t.tgt_begin.push_back(t0);
        t.tgt_end.push_back(t1);
        return (int32_t)(t.level.size() - 1);
    };
    push_box(0, 0, 0, -1, 0, (int32_t)n_src, 0, (int32_t)n_tgt);
    t.level_start.push_back(0);
    int32_t lvl_begin = 0, lvl_end = 1;
    for (int lvl = 0;; ++lvl) {
        t.level_start.push_back(lvl_end);
        if (lvl >= opt.max_level) break;
        for (int32_t b = lvl_begin; b < lvl_end; ++b) {
            const int32_t ns = t.src_end[b] - t.src_begin[b];
            const int32_t nt = t.tgt_end[b] - t.tgt_begin[b];
            if (ns <= opt.leaf && nt <= opt.leaf) continue;
            const int shift = 2 * (kCoordBits - lvl - 1);
            const uint64_t prefix = morton((uint32_t)t.ix[b], (uint32_t)t.iy[b]);
            int32_t s_cur = t.src_begin[b], t_cur = t.tgt_begin[b];
            for (int c = 0; c < 4; ++c) {
                const uint64_t hi = ((prefix << 2) | (uint64_t)c) + 1;
                const int32_t s_next = lower(ks, s_cur, t.src_end[b], hi << shift);
                const int32_t t_next = lower(kt, t_cur, t.tgt_end[b], hi << shift);
                if (s_next > s_cur || t_next > t_cur) {
                    const int32_t cb = push_box(lvl + 1, 2 * t.ix[b] + (c & 1), 2 * t.iy[b] + (c >> 1), b,
                                                s_cur, s_next, t_cur, t_next);
                    t.child[(size_t)b * 4 + c] = cb;
                    t.is_leaf[b] = 0;
                }
                s_cur = s_next;
                t_cur = t_next;
            }
        }
        const int32_t next_end = (int32_t)t.level.size();
        if (next_end == lvl_end) break;
        lvl_begin = lvl_end;
        lvl_end = next_end;
    }
    t.n_levels = (int)t.level_start.size() - 1;
    const int32_t nb = (int32_t)t.level.size();

    // colleague lookup
    std::unordered_map<uint64_t, int32_t> where;
    where.reserve((size_t)nb * 2);
    for (int32_t b = 0; b < nb; ++b) where[hash_key(t.level[b], t.ix[b], t.iy[b])] = b;
    auto colleagues = [&](int32_t b, std::vector<int32_t>& out) {
        out.clear();
        const int lvl = t.level[b];
        const int32_t lim = (int32_t)(1LL << lvl);
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int32_t cx = t.ix[b] + dx, cy = t.iy[b] + dy;
                if (cx < 0 || cy < 0 || cx >= lim || cy >= lim) continue;
                auto it = where.find(hash_key(lvl, cx, cy));
                if (it != where.end()) out.push_back(it->second);
            }
    };

    std::vector<std::vector<int32_t>> U(nb), V(nb), W(nb), X(nb);
    std::vector<int32_t> col, pcol, stack;
    for (int32_t b = 0; b < nb; ++b) {
        // V: children of the parent's colleagues that are not adjacent to b
        if (t.level[b] >= 2) {
            colleagues(t.parent[b], pcol);
            for (int32_t q : pcol) {
                for (int c = 0; c < 4; ++c) {
                    const int32_t ch = t.child[(size_t)q * 4 + c];
                    if (ch < 0) continue;
                    if (std::abs(t.ix[ch] - t.ix[b]) > 1 || std::abs(t.iy[ch] - t.iy[b]) > 1) V[b].push_back(ch);
                }
            }
        }
        if (!t.is_leaf[b]) continue;
        // U and W of a leaf
        U[b].push_back(b);
        colleagues(b, col);
        stack.clear();
        for (int32_t c : col)
            if (c != b) stack.push_back(c);
        while (!stack.empty()) {
            const int32_t c = stack.back();
            stack.pop_back();
            if (t.is_leaf[c]) {
                U[b].push_back(c);
                continue;
            }
            for (int k = 0; k < 4; ++k) {
                const int32_t d = t.child[(size_t)c * 4 + k];
                if (d < 0) continue;
                if (boxes_adjacent(t, d, b))
                    stack.push_back(d);
                else
                    W[b].push_back(d);
            }
        }
        // coarser adjacent leaves: leaf colleagues of an ancestor that touch b
        for (int32_t a = t.parent[b]; a >= 0; a = t.parent[a]) {
            colleagues(a, pcol);
            for (int32_t q : pcol)
                if (q != a && t.is_leaf[q] && boxes_adjacent(t, q, b)) U[b].push_back(q);
        }
    }
    for (int32_t b = 0; b < nb; ++b)
        for (int32_t d : W[b]) X[d].push_back(b);
    for (int32_t b = 0; b < nb; ++b) {
        std::sort(U[b].begin(), U[b].end());
        std::sort(V[b].begin(), V[b].end());
        std::sort(W[b].begin(), W[b].end());
        std::sort(X[b].begin(), X[b].end());
    }
    to_csr(U, t.u_ptr, t.u_idx);
    to_csr(V, t.v_ptr, t.v_idx);
    to_csr(W, t.w_ptr, t.w_idx);
    to_csr(X, t.x_ptr, t.x_idx);
    return "";
}

}  // namespace vp
