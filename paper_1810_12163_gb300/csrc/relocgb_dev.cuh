// Device-side access to the leaf mode store: M(u), the union over the trees
// in use of the first k_top modes of the leaf each tree maps pixel u to
// (tree order, then mode rank).
#pragma once
#include "internal.h"

namespace rl {

__device__ __forceinline__ int mode_count(const ModeView &mv, const uint16_t *lv, int hw_max, int p,
                                          int n_trees, int k_top) {
    int total = 0;
    for (int t = 0; t < n_trees; ++t) {
        const uint16_t leaf = lv[(size_t)t * hw_max + p];
        if (leaf == 0xFFFF) return 0;
        const int nm = mv.nmodes[t * mv.leaves_per_tree + leaf];
        total += nm < k_top ? nm : k_top;
    }
    return total;
}

// m-th element of M(u) -> (global leaf, rank within the leaf).
__device__ __forceinline__ void mode_at(const ModeView &mv, const uint16_t *lv, int hw_max, int p,
                                        int n_trees, int k_top, int m, uint32_t *L, int *rank) {
    for (int t = 0; t < n_trees; ++t) {
        const uint32_t l = (uint32_t)(t * mv.leaves_per_tree + lv[(size_t)t * hw_max + p]);
        int nm = mv.nmodes[l];
        nm = nm < k_top ? nm : k_top;
        if (m < nm) {
            *L = l;
            *rank = m;
            return;
        }
        m -= nm;
    }
    *L = 0;
    *rank = 0;
}

// Per-pixel record for forests of at most kRecTrees trees: the leaf reached
// in each tree (uint16) and that leaf's min(modes, k_top) (uint8), so M(u)
// is enumerated from one 16-byte load.

__device__ __forceinline__ int rec_leaf(const uint4 &r, int t) {
    const uint32_t w = t < 2 ? r.x : (t < 4 ? r.y : r.z);
    return (t & 1) ? (int)(w >> 16) : (int)(w & 0xFFFFu);
}

__device__ __forceinline__ int rec_count(const uint4 &r, int t) {
    // counts of trees 0..3 in r.w, tree 4 in the high half of r.z
    return t < 4 ? (int)((r.w >> (8 * t)) & 255u) : (int)((r.z >> 16) & 255u);
}

// |M(u)| of pixel p: the sum of its record's per-tree counts when there are
// records (the relocaliser then writes no separate count map), else the
// count map's entry.
__device__ __forceinline__ int pixel_modes(const uint16_t *mc, const uint4 *pr, int p, int n_trees) {
    if (!pr) return mc[p];
    const uint4 r = pr[p];
    int s = 0;
    for (int t = 0; t < n_trees; ++t) s += rec_count(r, t);
    return s;
}

__device__ __forceinline__ uint4 make_rec(const int leaf[kRecTrees], const int cnt[kRecTrees], int T) {
    uint4 r = make_uint4(0, 0, 0, 0);
    for (int t = 0; t < T; ++t) {
        const uint32_t l = (uint32_t)leaf[t] & 0xFFFFu;
        if (t == 0) r.x |= l;
        if (t == 1) r.x |= l << 16;
        if (t == 2) r.y |= l;
        if (t == 3) r.y |= l << 16;
        if (t == 4) r.z |= l;
        const uint32_t c = (uint32_t)cnt[t] & 255u;
        if (t < 4) r.w |= c << (8 * t);
        else r.z |= c << 16;
    }
    return r;
}

// m-th element of M(u) from the pixel record -> (global leaf, rank).
__device__ __forceinline__ void mode_at_rec(const uint4 &rec, int n_trees, int leaves_per_tree, int m,
                                            uint32_t *L, int *rank) {
    for (int t = 0; t < n_trees; ++t) {
        const int nm = rec_count(rec, t);
        if (m < nm) {
            *L = (uint32_t)(t * leaves_per_tree + rec_leaf(rec, t));
            *rank = m;
            return;
        }
        m -= nm;
    }
    *L = 0;
    *rank = 0;
}

// Decoded mode position: FP32 leaf centroid + FP16 offset (FP32 add), or
// the stored FP32 position.
__device__ __forceinline__ float3 mode_pos(const ModeView &mv, uint32_t L, int rank) {
    const size_t e = (size_t)L * mv.m_max + rank;
    if (mv.mpos_h) {
        const ushort4 h = mv.mpos_h[e];
        const float4 c = mv.centroid[L];
        return make_float3(__fadd_rn(c.x, __half2float(__ushort_as_half(h.x))),
                           __fadd_rn(c.y, __half2float(__ushort_as_half(h.y))),
                           __fadd_rn(c.z, __half2float(__ushort_as_half(h.z))));
    }
    const float4 f = mv.mpos_f[e];
    return make_float3(f.x, f.y, f.z);
}

}  // namespace rl
