// Device helpers shared by hypothesis generation and the pose kernel: the
// Philox draws of an attempt, the M(u) lookup and the back-projection.  All
// arithmetic here is integer or explicitly rounded FP32, so it is exact
// whatever the compiler's contraction setting.
#pragma once
#include "internal.h"
#include "relocgb_dev.cuh"

namespace rl {

struct HypArgs {
    const Frame *frames;
    const uint16_t *leaves;  // [B][T][hw_max]
    const uint16_t *mcount;  // [B][hw_max] |M(u)|
    const uint4 *prec;       // [B][hw_max] pixel records (<= 5 trees) or null
    const uint2 *pcm;        // [B][hw_max] colour-check masks and |M(u)|, or null
    int hw_max;
    ModeView mv;
    RParams p;
    double *hyp_pose;        // [B][N][12]
    int32_t *hyp_iter;       // [B][N]
    unsigned long long *work;  // profiling counters or null
    const uint32_t *pbits;   // [B][hw_max / 32 + 1] non-empty-M(u) bitmap (with pcm), or null
};

__device__ __forceinline__ float3 backproject_d(const Frame &fr, int p, float d) {
    const int u = p % fr.W, v = p / fr.W;
    return make_float3(__fdiv_rn(__fmul_rn(__fsub_rn((float)u, fr.cx), d), fr.fx),
                       __fdiv_rn(__fmul_rn(__fsub_rn((float)v, fr.cy), d), fr.fy), d);
}

__device__ __forceinline__ float3 backproject(const Frame &fr, int p) { return backproject_d(fr, p, fr.depth[p]); }

// The draws of iteration `it` of `slot`: three pixels, the colour-check pair
// and the three mode indices into M(u).
struct Draw {
    int pix[3];
    uint32_t m[3];
    int j;
};

// With p.redraw (reading R8b) a pixel that `usable` rejects (no depth or an
// empty M(u)) is redrawn within the iteration, up to batch_attempts draws in
// all: draw at >= 1 of pixel i takes word 0 of the Philox block with counter
// (slot, TAG_REDRAW << 16 | level, it, 4 at + i).  Kept out of line: the
// default reading never calls it.
template <class Usable>
__device__ __noinline__ int3 redraw_pixels(const HypArgs &a, const Frame &fr, int slot, int it, Usable usable,
                                           int3 pix) {
    const uint32_t WH = (uint32_t)(fr.W * fr.H);
    const uint32_t ctr2 = (TAG_REDRAW << 16) | (uint32_t)a.p.level;
    auto fix = [&](int q, int i) {
        for (int at = 1; at < a.p.batch_attempts && !usable(q); ++at)
            q = (int)draw_below(philox(make_uint4(slot, ctr2, it, 4u * at + i), fr.key0, fr.key1).x, WH);
        return q;
    };
    return make_int3(fix(pix.x, 0), fix(pix.y, 1), fix(pix.z, 2));
}

template <class Usable, int REDRAW = -1>
__device__ __forceinline__ Draw draw(const HypArgs &a, const Frame &fr, int slot, int it, Usable usable) {
    const uint32_t ctr1 = (TAG_HYP << 16) | (uint32_t)a.p.level;
    const uint4 r0 = philox(make_uint4(slot, ctr1, it, 0), fr.key0, fr.key1);
    const uint32_t WH = (uint32_t)(fr.W * fr.H);
    Draw d;
    d.pix[0] = (int)draw_below(r0.x, WH);
    d.pix[1] = (int)draw_below(r0.y, WH);
    d.pix[2] = (int)draw_below(r0.z, WH);
    d.j = (int)draw_below(r0.w, 3);
    // REDRAW: the reading fixed at compile time (0 or 1), or -1: a.p.redraw
    if (REDRAW == 1 || (REDRAW < 0 && a.p.redraw)) {
        const int3 q = redraw_pixels(a, fr, slot, it, usable, make_int3(d.pix[0], d.pix[1], d.pix[2]));
        d.pix[0] = q.x;
        d.pix[1] = q.y;
        d.pix[2] = q.z;
    }
    return d;
}

// M(u) element through the pixel record when there is one.
__device__ __forceinline__ void lookup(const HypArgs &a, const uint16_t *lv, const uint4 *pr, int p, int m,
                                       uint32_t *L, int *rank) {
    if (pr)
        mode_at_rec(pr[p], a.p.n_trees, a.mv.leaves_per_tree, m, L, rank);
    else
        mode_at(a.mv, lv, a.hw_max, p, a.p.n_trees, a.p.k_top, m, L, rank);
}

}  // namespace rl
