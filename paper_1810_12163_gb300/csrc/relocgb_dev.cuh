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
