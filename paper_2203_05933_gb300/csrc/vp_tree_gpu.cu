// Adaptive quadtree and interaction lists built on the GPU (plan time). The
// result is the tree the host build (vp_tree.cpp) makes for the same points and
// options, bit for bit: the same Morton keys on 28-bit coordinates, the same
// stable order of equal keys (caller index ascending), the same breadth-first
// box numbering, the same U/V/W/X lists in ascending box order. The paper
// treats the FMM as a black box (Sec. 1 synopsis; Sec. 4, paragraph after
// Eq. nsrcs); the list definitions are the standard adaptive ones.
//
// Steps: bounding square (a min/max reduction, when the caller gives none);
// Morton keys (quantisation with the host's rounding: (x - x0) * scale without
// contraction, floor); a stable least-significant-digit radix sort of the
// (key, index) pairs, 8 bits per pass, ranks within a block from warp match
// masks so that equal digits keep their order; splitting level by level (each
// box of a level finds its children's ranges by binary search in the sorted
// keys; the host turns the counts into offsets); the lists per box (colleagues
// by binary search in the level's Morton-ordered boxes, a per-thread stack for
// the finer adjacent leaves and the W list, ancestors' colleagues for the
// coarser adjacent leaves), counted, then filled and sorted; X as W transposed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "vp_internal.h"

namespace vp {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                           // items per thread per tile
constexpr int kSortTile = kSortThreads * kSortItems;     // 4096
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

__device__ __forceinline__ uint64_t spread_bits_d(uint64_t v)
{
    v &= 0xffffffffULL;
    v = (v | (v << 16)) & 0x0000ffff0000ffffULL;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffULL;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0fULL;
    v = (v | (v << 2)) & 0x3333333333333333ULL;
    v = (v | (v << 1)) & 0x5555555555555555ULL;
    return v;
}

__device__ __forceinline__ uint64_t morton_d(uint32_t ix, uint32_t iy)
{
    return spread_bits_d(ix) | (spread_bits_d(iy) << 1);
}

// per block: min x, max x, min y, max y of its points; bad |= non-finite
__global__ void k_bbox(int64_t n, const double* __restrict__ xy, double* __restrict__ part, int* __restrict__ bad)
{
    double mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
    int nf = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = xy[2 * i], y = xy[2 * i + 1];
        if (!isfinite(x) || !isfinite(y)) nf = 1;
        mnx = fmin(mnx, x);
        mxx = fmax(mxx, x);
        mny = fmin(mny, y);
        mxy = fmax(mxy, y);
    }
    __shared__ double s[4][256];
    s[0][threadIdx.x] = mnx;
    s[1][threadIdx.x] = mxx;
    s[2][threadIdx.x] = mny;
    s[3][threadIdx.x] = mxy;
    nf = __syncthreads_or(nf);
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s[0][threadIdx.x] = fmin(s[0][threadIdx.x], s[0][threadIdx.x + o]);
            s[1][threadIdx.x] = fmax(s[1][threadIdx.x], s[1][threadIdx.x + o]);
            s[2][threadIdx.x] = fmin(s[2][threadIdx.x], s[2][threadIdx.x + o]);
            s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) part[4 * blockIdx.x + k] = s[k][0];
        if (nf) atomicOr(bad, 1);
    }
}

// key[i] = Morton key of point i on the 28-bit grid of the root square, val[i] = i.
// bad bit 1: non-finite coordinate; bit 2: outside the root square (no clamping)
__global__ void k_morton(int64_t n, const double* __restrict__ xy, double x0, double y0, double scale, int clamp,
                         uint64_t* __restrict__ key, int32_t* __restrict__ val, int* __restrict__ bad)
{
    const int64_t maxc = (1LL << kCoordBits) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = xy[2 * i], y = xy[2 * i + 1];
        int64_t cx = 0, cy = 0;
        if (!isfinite(x) || !isfinite(y)) {
            atomicOr(bad, 1);
        } else {
            cx = (int64_t)floor(__dmul_rn(__dsub_rn(x, x0), scale));
            cy = (int64_t)floor(__dmul_rn(__dsub_rn(y, y0), scale));
            if (clamp) {
                cx = min(max(cx, (int64_t)0), maxc);
                cy = min(max(cy, (int64_t)0), maxc);
            } else if (cx < 0 || cy < 0 || cx > maxc || cy > maxc) {
                atomicOr(bad, 2);
                cx = cy = 0;
            }
        }
        key[i] = morton_d((uint32_t)cx, (uint32_t)cy);
        val[i] = (int32_t)i;
    }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, val), 8 bits per pass.
// counts[d * nblocks + b] = items of tile b with digit d
__global__ void __launch_bounds__(kSortThreads)
    k_radix_count(int64_t n, const uint64_t* __restrict__ key, int shift, int nblocks, uint32_t* __restrict__ counts)
{
    __shared__ uint32_t h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        const int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) counts[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

// exclusive scan of counts (digit-major), one block: each thread scans a
// contiguous segment, then the segment totals are scanned
__global__ void __launch_bounds__(1024) k_scan_u32(int64_t n, uint32_t* __restrict__ a)
{
    __shared__ uint32_t tot[1024];
    const int64_t seg = (n + blockDim.x - 1) / blockDim.x;
    const int64_t lo = threadIdx.x * seg, hi = min(n, lo + seg);
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += a[i];
    tot[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const uint32_t v = tot[t];
            tot[t] = run;
            run += v;
        }
    }
    __syncthreads();
    uint32_t run = tot[threadIdx.x];
    for (int64_t i = lo; i < hi; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

// scatter of one tile in order: 16 rounds of 256 consecutive items; within a
// round an item's rank among the block's equal digits = items of earlier warps
// (per-warp digit counts, prefix over warps) + earlier lanes of its warp (match mask)
__global__ void __launch_bounds__(kSortThreads)
    k_radix_scatter(int64_t n, const uint64_t* __restrict__ key, const int32_t* __restrict__ val, int shift,
                    int nblocks, const uint32_t* __restrict__ offs, uint64_t* __restrict__ okey,
                    int32_t* __restrict__ oval)
{
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t base[kRadix];              // next free position of each digit for this tile
    __shared__ uint16_t wcount[kWarps][kRadix];    // items of each digit per warp in the current round
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) base[d] = offs[(int64_t)d * nblocks + blockIdx.x];
    const int64_t tbase = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        for (int i = threadIdx.x; i < kWarps * kRadix; i += blockDim.x) (&wcount[0][0])[i] = 0;
        __syncthreads();
        const int64_t i = tbase + (int64_t)r * kSortThreads + threadIdx.x;
        const bool live = i < n;
        const uint64_t k = live ? key[i] : 0;
        const int d = live ? (int)((k >> shift) & (kRadix - 1)) : -1;  // -1: no digit
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (live && rank == 0) wcount[warp][d] = (uint16_t)__popc(peers);
        __syncthreads();
        if (live) {
            uint32_t before = 0;
            for (int w = 0; w < warp; ++w) before += wcount[w][d];
            const uint32_t pos = base[d] + before + (uint32_t)rank;
            okey[pos] = k;
            oval[pos] = val[i];
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < kRadix; dd += blockDim.x) {
            uint32_t s = 0;
            for (int w = 0; w < kWarps; ++w) s += wcount[w][dd];
            base[dd] += s;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Splitting. Boxes of one level: level-local arrays in breadth-first order.
struct DevBoxes {
    int32_t* ix = nullptr;
    int32_t* iy = nullptr;
    int32_t* parent = nullptr;
    int32_t* child = nullptr;   // [4] per box
    int32_t* is_leaf = nullptr;
    int32_t* sb = nullptr;      // source begin / end, target begin / end
    int32_t* se = nullptr;
    int32_t* tb = nullptr;
    int32_t* te = nullptr;
};

// first position in [lo, hi) with key >= k
__device__ __forceinline__ int32_t lower_d(const uint64_t* __restrict__ key, int32_t lo, int32_t hi, uint64_t k)
{
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (key[mid] < k)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// per box b of the level [b0, b1): children's ranges (cr [b][4][4]) and count (cnt[b - b0])
__global__ void k_split(DevBoxes B, int32_t b0, int32_t b1, int lvl, int leaf, int max_level,
                        const uint64_t* __restrict__ ks, const uint64_t* __restrict__ kt, int32_t* __restrict__ cr,
                        int32_t* __restrict__ cnt)
{
    for (int32_t b = b0 + blockIdx.x * blockDim.x + threadIdx.x; b < b1; b += gridDim.x * blockDim.x) {
        const int32_t s0 = B.sb[b], s1 = B.se[b], t0 = B.tb[b], t1 = B.te[b];
        int n = 0;
        if (lvl < max_level && (s1 - s0 > leaf || t1 - t0 > leaf)) {
            const int shift = 2 * (kCoordBits - lvl - 1);
            const uint64_t prefix = morton_d((uint32_t)B.ix[b], (uint32_t)B.iy[b]);
            int32_t sc = s0, tc = t0;
            for (int c = 0; c < 4; ++c) {
                const uint64_t hi = (((prefix << 2) | (uint64_t)c) + 1) << shift;
                const int32_t sn = lower_d(ks, sc, s1, hi);
                const int32_t tn = lower_d(kt, tc, t1, hi);
                int32_t* r = cr + ((int64_t)(b - b0) * 4 + c) * 4;
                r[0] = sc;
                r[1] = sn;
                r[2] = tc;
                r[3] = tn;
                if (sn > sc || tn > tc) ++n;
                sc = sn;
                tc = tn;
            }
        }
        cnt[b - b0] = n;
    }
}

// children of the level's boxes at next + off[b - b0] (off: exclusive scan of cnt)
__global__ void k_emit(DevBoxes B, int32_t b0, int32_t b1, const int32_t* __restrict__ cr,
                       const int32_t* __restrict__ cnt, const int32_t* __restrict__ off, int32_t next)
{
    for (int32_t b = b0 + blockIdx.x * blockDim.x + threadIdx.x; b < b1; b += gridDim.x * blockDim.x) {
        for (int c = 0; c < 4; ++c) B.child[4 * (int64_t)b + c] = -1;
        if (cnt[b - b0] == 0) {
            B.is_leaf[b] = 1;
            continue;
        }
        B.is_leaf[b] = 0;
        int32_t o = next + off[b - b0];
        for (int c = 0; c < 4; ++c) {
            const int32_t* r = cr + ((int64_t)(b - b0) * 4 + c) * 4;
            if (!(r[1] > r[0] || r[3] > r[2])) continue;
            B.ix[o] = 2 * B.ix[b] + (c & 1);
            B.iy[o] = 2 * B.iy[b] + (c >> 1);
            B.parent[o] = b;
            B.sb[o] = r[0];
            B.se[o] = r[1];
            B.tb[o] = r[2];
            B.te[o] = r[3];
            B.is_leaf[o] = 1;  // until its own level is split
            for (int k = 0; k < 4; ++k) B.child[4 * (int64_t)o + k] = -1;
            B.child[4 * (int64_t)b + c] = o;
            ++o;
        }
    }
}

// ---------------------------------------------------------------------------
// Lists. lkey[b] = Morton key of (ix, iy) at the box's level; the boxes of a
// level are in Morton order (children are emitted in quadrant order, parents in
// level order), so a colleague is found by binary search in its level's range.
struct DevLevels {
    const int32_t* lvl_of = nullptr;    // [nb] level of each box
    const int32_t* level_start = nullptr;
    const uint64_t* lkey = nullptr;
};

__device__ __forceinline__ int32_t find_box(const DevLevels& L, int lvl, int32_t x, int32_t y)
{
    const int32_t lim = (int32_t)(1LL << lvl);
    if (x < 0 || y < 0 || x >= lim || y >= lim) return -1;
    const uint64_t k = morton_d((uint32_t)x, (uint32_t)y);
    int32_t lo = L.level_start[lvl], hi = L.level_start[lvl + 1];
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (L.lkey[mid] < k)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < L.level_start[lvl + 1] && L.lkey[lo] == k) ? lo : -1;
}

__device__ __forceinline__ bool adjacent_d(const DevBoxes& B, const DevLevels& L, int32_t a, int32_t b)
{
    const int la = L.lvl_of[a], lb = L.lvl_of[b];
    const int Lm = max(la, lb);
    const int64_t sa = 1LL << (Lm - la), sb = 1LL << (Lm - lb);
    const int64_t ax0 = (int64_t)B.ix[a] * sa, ax1 = ax0 + sa, ay0 = (int64_t)B.iy[a] * sa, ay1 = ay0 + sa;
    const int64_t bx0 = (int64_t)B.ix[b] * sb, bx1 = bx0 + sb, by0 = (int64_t)B.iy[b] * sb, by1 = by0 + sb;
    return ax0 <= bx1 && bx0 <= ax1 && ay0 <= by1 && by0 <= ay1;
}

__global__ void k_lkey(int32_t nb, DevBoxes B, uint64_t* __restrict__ lkey)
{
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        lkey[b] = morton_d((uint32_t)B.ix[b], (uint32_t)B.iy[b]);
}

// Insertion sort of a short list in place.
__device__ __forceinline__ void sort_small(int32_t* a, int n)
{
    for (int i = 1; i < n; ++i) {
        const int32_t v = a[i];
        int j = i - 1;
        while (j >= 0 && a[j] > v) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = v;
    }
}

constexpr int kStack = 256;  // DFS stack of the finer adjacent boxes (3 per level at most, plus 8 colleagues)

// One thread per box. FILL = false: counts into uc, vc, wc. FILL = true: the lists
// at their offsets (uo, vo, wo: exclusive scans of the counts), each sorted.
// A stack overflow (never for kStack >= 8 + 3 * 27) sets *bad.
template <bool FILL>
__global__ void k_lists(int32_t nb, DevBoxes B, DevLevels L, int32_t* __restrict__ uc, int32_t* __restrict__ vc,
                        int32_t* __restrict__ wc, const int32_t* __restrict__ uo, const int32_t* __restrict__ vo,
                        const int32_t* __restrict__ wo, int32_t* __restrict__ ui, int32_t* __restrict__ vi,
                        int32_t* __restrict__ wi, int* __restrict__ bad)
{
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int lvl = L.lvl_of[b];
        int nv = 0, nu = 0, nw = 0;
        int32_t* vout = FILL ? vi + vo[b] : nullptr;
        int32_t* uout = FILL ? ui + uo[b] : nullptr;
        int32_t* wout = FILL ? wi + wo[b] : nullptr;
        // V: children of the parent's colleagues that are not adjacent to b
        if (lvl >= 2) {
            const int32_t p = B.parent[b];
            const int lp = lvl - 1;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int32_t q = find_box(L, lp, B.ix[p] + dx, B.iy[p] + dy);
                    if (q < 0) continue;
                    for (int c = 0; c < 4; ++c) {
                        const int32_t ch = B.child[4 * (int64_t)q + c];
                        if (ch < 0) continue;
                        if (abs(B.ix[ch] - B.ix[b]) > 1 || abs(B.iy[ch] - B.iy[b]) > 1) {
                            if (FILL) vout[nv] = ch;
                            ++nv;
                        }
                    }
                }
        }
        if (B.is_leaf[b]) {
            if (FILL) uout[nu] = b;
            ++nu;
            int32_t stack[kStack];
            int sp = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int32_t c = find_box(L, lvl, B.ix[b] + dx, B.iy[b] + dy);
                    if (c >= 0 && c != b) stack[sp++] = c;
                }
            while (sp > 0) {
                const int32_t c = stack[--sp];
                if (B.is_leaf[c]) {
                    if (FILL) uout[nu] = c;
                    ++nu;
                    continue;
                }
                for (int k = 0; k < 4; ++k) {
                    const int32_t d = B.child[4 * (int64_t)c + k];
                    if (d < 0) continue;
                    if (adjacent_d(B, L, d, b)) {
                        if (sp < kStack)
                            stack[sp++] = d;
                        else
                            atomicOr(bad, 4);
                    } else {
                        if (FILL) wout[nw] = d;
                        ++nw;
                    }
                }
            }
            // coarser adjacent leaves: leaf colleagues of an ancestor that touch b
            for (int32_t a = B.parent[b]; a >= 0; a = B.parent[a]) {
                const int la = L.lvl_of[a];
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int32_t q = find_box(L, la, B.ix[a] + dx, B.iy[a] + dy);
                        if (q < 0 || q == a || !B.is_leaf[q] || !adjacent_d(B, L, q, b)) continue;
                        if (FILL) uout[nu] = q;
                        ++nu;
                    }
            }
        }
        if (FILL) {
            sort_small(vout, nv);
            sort_small(uout, nu);
            sort_small(wout, nw);
        } else {
            uc[b] = nu;
            vc[b] = nv;
            wc[b] = nw;
        }
    }
}

// X = W transposed: for each b and each d in W(b), x[d] receives b (order fixed by the sort after)
__global__ void k_x_count(int32_t nb, const int32_t* __restrict__ wo, const int32_t* __restrict__ wi,
                          int32_t* __restrict__ xc)
{
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        for (int32_t e = wo[b]; e < wo[b + 1]; ++e) atomicAdd(&xc[wi[e]], 1);
}

__global__ void k_x_fill(int32_t nb, const int32_t* __restrict__ wo, const int32_t* __restrict__ wi,
                         int32_t* __restrict__ xcur, int32_t* __restrict__ xi)
{
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        for (int32_t e = wo[b]; e < wo[b + 1]; ++e) xi[atomicAdd(&xcur[wi[e]], 1)] = b;
}

__global__ void k_sort_lists(int32_t nb, const int32_t* __restrict__ ptr, int32_t* __restrict__ idx)
{
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        sort_small(idx + ptr[b], ptr[b + 1] - ptr[b]);
}

// device allocations of one build, freed on exit
struct DevMem {
    std::vector<void*> ptrs;
    ~DevMem()
    {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    T* get(size_t n)
    {
        void* p = nullptr;
        if (cudaMalloc(&p, (n ? n : 1) * sizeof(T)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return (T*)p;
    }
    void release(void* p)
    {
        for (auto& q : ptrs)
            if (q == p) {
                cudaFree(q);
                q = nullptr;
            }
    }
};

int grid_of(int64_t n, int threads)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 32));
}

// stable sort of (key, val) by key: 7 passes of 8 bits (keys below 2^56)
cudaError_t radix_sort(int64_t n, uint64_t*& key, int32_t*& val, uint64_t* key2, int32_t* val2, uint32_t* counts,
                       cudaStream_t s)
{
    if (n <= 1) return cudaSuccess;
    const int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    for (int shift = 0; shift < 2 * kCoordBits; shift += kRadixBits) {
        k_radix_count<<<nblocks, kSortThreads, 0, s>>>(n, key, shift, nblocks, counts);
        k_scan_u32<<<1, 1024, 0, s>>>((int64_t)kRadix * nblocks, counts);
        k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(n, key, val, shift, nblocks, counts, key2, val2);
        std::swap(key, key2);
        std::swap(val, val2);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t to_host(std::vector<T>& h, const T* d, size_t n, cudaStream_t s)
{
    h.resize(n);
    if (n == 0) return cudaSuccess;
    return cudaMemcpyAsync(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost, s);
}

// exclusive scan on the host: out[0] = 0, out[i + 1] = out[i] + in[i]
void host_scan(const std::vector<int32_t>& in, std::vector<int32_t>& out)
{
    out.assign(in.size() + 1, 0);
    for (size_t i = 0; i < in.size(); ++i) out[i + 1] = out[i] + in[i];
}

}  // namespace

#define VPT_CUDA(x)                                                    \
    do {                                                               \
        const cudaError_t e_ = (x);                                    \
        if (e_ != cudaSuccess) return std::string("CUDA: ") + cudaGetErrorString(e_); \
    } while (0)

std::string build_tree_gpu(int64_t n_src, const double* src_xy, int64_t n_tgt, const double* tgt_xy,
                           const TreeOptions& opt, Tree& t, cudaStream_t s)
{
    if (n_src < 0 || n_tgt < 0) return "negative point count";
    if (n_src > INT32_MAX / 2 || n_tgt > INT32_MAX / 2) return "too many points";
    if (opt.leaf < 1 || opt.leaf > 4096) return "leaf size outside [1, 4096]";
    if (opt.max_level < 0 || opt.max_level >= kCoordBits) return "max_level outside [0, 27]";
    t = Tree();
    t.n_src = n_src;
    t.n_tgt = n_tgt;
    DevMem mem;
    int* d_bad = mem.get<int>(1);
    if (!d_bad) return "device allocation failed";
    VPT_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), s));

    // root square (the host build's rules)
    bool clamp = false;
    if (opt.root[2] > 0.0) {
        if (!std::isfinite(opt.root[0]) || !std::isfinite(opt.root[1]) || !std::isfinite(opt.root[2]))
            return "non-finite root box";
        t.x0 = opt.root[0];
        t.y0 = opt.root[1];
        t.side = opt.root[2];
    } else {
        double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
        for (int pass = 0; pass < 2; ++pass) {
            const int64_t n = pass ? n_tgt : n_src;
            if (n == 0) continue;
            const int nb = (int)std::min<int64_t>(1024, (n + 255) / 256);
            double* part = mem.get<double>((size_t)4 * nb);
            if (!part) return "device allocation failed";
            k_bbox<<<nb, 256, 0, s>>>(n, pass ? tgt_xy : src_xy, part, d_bad);
            std::vector<double> hp;
            VPT_CUDA(to_host(hp, part, (size_t)4 * nb, s));
            VPT_CUDA(cudaStreamSynchronize(s));
            for (int b = 0; b < nb; ++b) {
                xmin = std::min(xmin, hp[4 * (size_t)b]);
                xmax = std::max(xmax, hp[4 * (size_t)b + 1]);
                ymin = std::min(ymin, hp[4 * (size_t)b + 2]);
                ymax = std::max(ymax, hp[4 * (size_t)b + 3]);
            }
        }
        int bad = 0;
        VPT_CUDA(cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost));
        if (n_src + n_tgt == 0) {
            xmin = ymin = 0.0;
            xmax = ymax = 1.0;
        }
        if (bad || !std::isfinite(xmin) || !std::isfinite(xmax) || !std::isfinite(ymin) || !std::isfinite(ymax))
            return "non-finite point coordinate";
        double side = std::max(xmax - xmin, ymax - ymin);
        if (!(side > 0.0)) side = 1.0;
        side *= 1.0 + 1.0 / 1048576.0;
        t.side = side;
        t.x0 = 0.5 * (xmin + xmax) - 0.5 * side;
        t.y0 = 0.5 * (ymin + ymax) - 0.5 * side;
        clamp = true;
    }
    const double scale = (double)(1u << kCoordBits) / t.side;

    // Morton keys and their stable sort, sources and targets
    uint64_t* keys[2] = {nullptr, nullptr};
    int32_t* perms[2] = {nullptr, nullptr};
    const int64_t nmax = std::max<int64_t>(std::max(n_src, n_tgt), 1);
    uint64_t* k2 = mem.get<uint64_t>((size_t)nmax);
    int32_t* v2 = mem.get<int32_t>((size_t)nmax);
    uint32_t* counts = mem.get<uint32_t>((size_t)kRadix * ((nmax + kSortTile - 1) / kSortTile));
    if (!k2 || !v2 || !counts) return "device allocation failed";
    std::vector<uint64_t*> kbuf;
    for (int pass = 0; pass < 2; ++pass) {
        const int64_t n = pass ? n_tgt : n_src;
        uint64_t* k = mem.get<uint64_t>((size_t)std::max<int64_t>(n, 1));
        int32_t* v = mem.get<int32_t>((size_t)std::max<int64_t>(n, 1));
        if (!k || !v) return "device allocation failed";
        if (n > 0) k_morton<<<grid_of(n, 256), 256, 0, s>>>(n, pass ? tgt_xy : src_xy, t.x0, t.y0, scale, clamp ? 1 : 0,
                                                            k, v, d_bad);
        uint64_t* kk = k;
        int32_t* vv = v;
        // the sort ping-pongs between (k, v) and the shared (k2, v2); keep the result
        // in this pass's own buffers
        VPT_CUDA(radix_sort(n, kk, vv, k2, v2, counts, s));
        if (kk != k) {
            VPT_CUDA(cudaMemcpyAsync(k, kk, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
            VPT_CUDA(cudaMemcpyAsync(v, vv, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        }
        keys[pass] = k;
        perms[pass] = v;
    }
    {
        int bad = 0;
        VPT_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        VPT_CUDA(cudaStreamSynchronize(s));
        if (bad & 1) return "non-finite point coordinate";
        if (bad & 2) return "point outside the root box";
    }
    VPT_CUDA(to_host(t.src_perm, perms[0], (size_t)n_src, s));
    VPT_CUDA(to_host(t.tgt_perm, perms[1], (size_t)n_tgt, s));

    // breadth-first splitting, one level at a time
    int64_t cap = std::max<int64_t>(1024, 8 * (n_src + n_tgt) / opt.leaf + 64);
    DevBoxes B;
    auto alloc_boxes = [&](DevBoxes& X, int64_t c) -> bool {
        X.ix = mem.get<int32_t>((size_t)c);
        X.iy = mem.get<int32_t>((size_t)c);
        X.parent = mem.get<int32_t>((size_t)c);
        X.child = mem.get<int32_t>((size_t)c * 4);
        X.is_leaf = mem.get<int32_t>((size_t)c);
        X.sb = mem.get<int32_t>((size_t)c);
        X.se = mem.get<int32_t>((size_t)c);
        X.tb = mem.get<int32_t>((size_t)c);
        X.te = mem.get<int32_t>((size_t)c);
        return X.ix && X.iy && X.parent && X.child && X.is_leaf && X.sb && X.se && X.tb && X.te;
    };
    if (!alloc_boxes(B, cap)) return "device allocation failed";
    {
        const int32_t root[9] = {0, 0, -1, 1, 0, (int32_t)n_src, 0, (int32_t)n_tgt, 0};
        int32_t* dst[8] = {B.ix, B.iy, B.parent, B.is_leaf, B.sb, B.se, B.tb, B.te};
        for (int k = 0; k < 8; ++k) VPT_CUDA(cudaMemcpyAsync(dst[k], &root[k], sizeof(int32_t), cudaMemcpyHostToDevice, s));
        VPT_CUDA(cudaMemsetAsync(B.child, 0xff, 4 * sizeof(int32_t), s));
        VPT_CUDA(cudaStreamSynchronize(s));  // the root values live on this stack frame
    }
    t.level_start.push_back(0);
    int32_t lvl_begin = 0, lvl_end = 1;
    std::vector<int32_t> cnt, off;
    for (int lvl = 0;; ++lvl) {
        t.level_start.push_back(lvl_end);
        if (lvl >= opt.max_level) break;
        const int32_t nl = lvl_end - lvl_begin;
        int32_t* d_cr = mem.get<int32_t>((size_t)nl * 16);
        int32_t* d_cnt = mem.get<int32_t>((size_t)nl);
        int32_t* d_off = mem.get<int32_t>((size_t)nl + 1);
        if (!d_cr || !d_cnt || !d_off) return "device allocation failed";
        k_split<<<grid_of(nl, 256), 256, 0, s>>>(B, lvl_begin, lvl_end, lvl, opt.leaf, opt.max_level, keys[0], keys[1],
                                                  d_cr, d_cnt);
        VPT_CUDA(to_host(cnt, d_cnt, (size_t)nl, s));
        VPT_CUDA(cudaStreamSynchronize(s));
        host_scan(cnt, off);
        const int32_t total = off.back();
        if ((int64_t)lvl_end + total > cap) {  // grow the box arrays
            int64_t ncap = std::max<int64_t>(2 * cap, (int64_t)lvl_end + total);
            DevBoxes N;
            if (!alloc_boxes(N, ncap)) return "device allocation failed";
            int32_t* from[9] = {B.ix, B.iy, B.parent, B.child, B.is_leaf, B.sb, B.se, B.tb, B.te};
            int32_t* to[9] = {N.ix, N.iy, N.parent, N.child, N.is_leaf, N.sb, N.se, N.tb, N.te};
            for (int k = 0; k < 9; ++k) {
                VPT_CUDA(cudaMemcpyAsync(to[k], from[k], (size_t)lvl_end * (k == 3 ? 4 : 1) * sizeof(int32_t),
                                         cudaMemcpyDeviceToDevice, s));
            }
            VPT_CUDA(cudaStreamSynchronize(s));
            for (int k = 0; k < 9; ++k) mem.release(from[k]);
            B = N;
            cap = ncap;
        }
        VPT_CUDA(cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        k_emit<<<grid_of(nl, 256), 256, 0, s>>>(B, lvl_begin, lvl_end, d_cr, d_cnt, d_off, lvl_end);
        VPT_CUDA(cudaStreamSynchronize(s));  // before off and cnt change
        mem.release(d_cr);
        mem.release(d_cnt);
        mem.release(d_off);
        if (total == 0) break;
        lvl_begin = lvl_end;
        lvl_end += total;
    }
    t.n_levels = (int)t.level_start.size() - 1;
    const int32_t nb = lvl_end;
    // boxes of the last level were emitted as leaves by their parents (or are the root)

    // lists
    std::vector<int32_t> lvl_of((size_t)nb);
    for (int l = 0; l < t.n_levels; ++l)
        for (int32_t b = t.level_start[(size_t)l]; b < t.level_start[(size_t)l + 1]; ++b) lvl_of[(size_t)b] = l;
    int32_t* d_lvl = mem.get<int32_t>((size_t)nb);
    int32_t* d_ls = mem.get<int32_t>(t.level_start.size());
    uint64_t* d_lkey = mem.get<uint64_t>((size_t)nb);
    int32_t* d_uc = mem.get<int32_t>((size_t)nb);
    int32_t* d_vc = mem.get<int32_t>((size_t)nb);
    int32_t* d_wc = mem.get<int32_t>((size_t)nb);
    if (!d_lvl || !d_ls || !d_lkey || !d_uc || !d_vc || !d_wc) return "device allocation failed";
    VPT_CUDA(cudaMemcpyAsync(d_lvl, lvl_of.data(), (size_t)nb * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    VPT_CUDA(cudaMemcpyAsync(d_ls, t.level_start.data(), t.level_start.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s));
    k_lkey<<<grid_of(nb, 256), 256, 0, s>>>(nb, B, d_lkey);
    DevLevels L;
    L.lvl_of = d_lvl;
    L.level_start = d_ls;
    L.lkey = d_lkey;
    k_lists<false><<<grid_of(nb, 128), 128, 0, s>>>(nb, B, L, d_uc, d_vc, d_wc, nullptr, nullptr, nullptr, nullptr,
                                                    nullptr, nullptr, d_bad);
    std::vector<int32_t> uc, vc, wc;
    VPT_CUDA(to_host(uc, d_uc, (size_t)nb, s));
    VPT_CUDA(to_host(vc, d_vc, (size_t)nb, s));
    VPT_CUDA(to_host(wc, d_wc, (size_t)nb, s));
    VPT_CUDA(cudaStreamSynchronize(s));
    host_scan(uc, t.u_ptr);
    host_scan(vc, t.v_ptr);
    host_scan(wc, t.w_ptr);
    int32_t* d_uo = mem.get<int32_t>((size_t)nb + 1);
    int32_t* d_vo = mem.get<int32_t>((size_t)nb + 1);
    int32_t* d_wo = mem.get<int32_t>((size_t)nb + 1);
    int32_t* d_ui = mem.get<int32_t>((size_t)t.u_ptr.back());
    int32_t* d_vi = mem.get<int32_t>((size_t)t.v_ptr.back());
    int32_t* d_wi = mem.get<int32_t>((size_t)t.w_ptr.back());
    int32_t* d_xc = mem.get<int32_t>((size_t)nb);
    if (!d_uo || !d_vo || !d_wo || !d_ui || !d_vi || !d_wi || !d_xc) return "device allocation failed";
    VPT_CUDA(cudaMemcpyAsync(d_uo, t.u_ptr.data(), t.u_ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    VPT_CUDA(cudaMemcpyAsync(d_vo, t.v_ptr.data(), t.v_ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    VPT_CUDA(cudaMemcpyAsync(d_wo, t.w_ptr.data(), t.w_ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_lists<true><<<grid_of(nb, 128), 128, 0, s>>>(nb, B, L, nullptr, nullptr, nullptr, d_uo, d_vo, d_wo, d_ui, d_vi,
                                                   d_wi, d_bad);
    VPT_CUDA(cudaMemsetAsync(d_xc, 0, (size_t)nb * sizeof(int32_t), s));
    k_x_count<<<grid_of(nb, 256), 256, 0, s>>>(nb, d_wo, d_wi, d_xc);
    std::vector<int32_t> xc;
    VPT_CUDA(to_host(xc, d_xc, (size_t)nb, s));
    VPT_CUDA(cudaStreamSynchronize(s));
    host_scan(xc, t.x_ptr);
    int32_t* d_xo = mem.get<int32_t>((size_t)nb + 1);
    int32_t* d_xi = mem.get<int32_t>((size_t)t.x_ptr.back());
    if (!d_xo || !d_xi) return "device allocation failed";
    VPT_CUDA(cudaMemcpyAsync(d_xo, t.x_ptr.data(), t.x_ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    VPT_CUDA(cudaMemcpyAsync(d_xc, t.x_ptr.data(), (size_t)nb * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_x_fill<<<grid_of(nb, 256), 256, 0, s>>>(nb, d_wo, d_wi, d_xc, d_xi);
    k_sort_lists<<<grid_of(nb, 256), 256, 0, s>>>(nb, d_xo, d_xi);
    {
        int bad = 0;
        VPT_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        VPT_CUDA(cudaStreamSynchronize(s));
        if (bad & 4) return "internal error: list stack overflow";
    }

    // boxes and lists to the host structure
    t.level = lvl_of;
    VPT_CUDA(to_host(t.ix, B.ix, (size_t)nb, s));
    VPT_CUDA(to_host(t.iy, B.iy, (size_t)nb, s));
    VPT_CUDA(to_host(t.parent, B.parent, (size_t)nb, s));
    VPT_CUDA(to_host(t.child, B.child, (size_t)nb * 4, s));
    VPT_CUDA(to_host(t.is_leaf, B.is_leaf, (size_t)nb, s));
    VPT_CUDA(to_host(t.src_begin, B.sb, (size_t)nb, s));
    VPT_CUDA(to_host(t.src_end, B.se, (size_t)nb, s));
    VPT_CUDA(to_host(t.tgt_begin, B.tb, (size_t)nb, s));
    VPT_CUDA(to_host(t.tgt_end, B.te, (size_t)nb, s));
    VPT_CUDA(to_host(t.u_idx, d_ui, (size_t)t.u_ptr.back(), s));
    VPT_CUDA(to_host(t.v_idx, d_vi, (size_t)t.v_ptr.back(), s));
    VPT_CUDA(to_host(t.w_idx, d_wi, (size_t)t.w_ptr.back(), s));
    VPT_CUDA(to_host(t.x_idx, d_xi, (size_t)t.x_ptr.back(), s));
    VPT_CUDA(cudaStreamSynchronize(s));
    return "";
}

}  // namespace vp
