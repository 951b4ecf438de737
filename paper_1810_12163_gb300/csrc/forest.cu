// Random forest factory (Sec. 4.5), split features and forest walk
// (Eq. 1-3), and deterministic online reservoir adaptation (Sec. 3.2.2).
//
// Compiled with --fmad=false: the FP32 feature arithmetic and the FP64
// back-projection are plain IEEE operations in a fixed order, so leaves and
// reservoir contents are exactly reproducible.
#include "internal.h"
#include "relocgb_dev.cuh"

namespace rl {

__device__ __forceinline__ float unit24(uint32_t u) {
    return __fmul_rn((float)(u >> 8), 1.0f / 16777216.0f);
}

// One thread per branch node.  Two Philox blocks per node: (type draw, dx,
// dy, channel) and (tau).
__global__ void k_forest_random(float4 *nodes, int n_trees, int n_branch, float p_depth,
                                float dlo, float dhi, float tdlo, float tdhi, float trlo,
                                float trhi, int tau_zero, uint32_t k0, uint32_t k1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_trees * n_branch) return;
    const int t = i / n_branch, n = i % n_branch;
    const uint4 r0 = philox(make_uint4(t, TAG_FOREST << 16, n, 0), k0, k1);
    const uint4 r1 = philox(make_uint4(t, TAG_FOREST << 16, n, 1), k0, k1);
    const bool is_depth = (double)r0.x < (double)p_depth * 4294967296.0;
    const float span = __fsub_rn(dhi, dlo);
    float4 nd;
    nd.x = __fadd_rn(dlo, __fmul_rn(span, unit24(r0.y)));
    nd.y = __fadd_rn(dlo, __fmul_rn(span, unit24(r0.z)));
    float tau = 0.0f;
    if (!tau_zero) {
        const float lo = is_depth ? tdlo : trlo, hi = is_depth ? tdhi : trhi;
        tau = __fadd_rn(lo, __fmul_rn(__fsub_rn(hi, lo), unit24(r1.x)));
    }
    nd.z = tau;
    const uint32_t meta = is_depth ? 0u : (1u | (draw_below(r0.w, 3) << 8));
    nd.w = __uint_as_float(meta);
    nodes[i] = nd;
}

rl_status launch_forest_random(rl_forest *f, cudaStream_t s) {
    const rl_forest_params &p = f->p;
    const int n = p.n_trees * f->n_branch;
    k_forest_random<<<(n + 255) / 256, 256, 0, s>>>(
        f->nodes, p.n_trees, f->n_branch, p.p_depth, p.delta_lo, p.delta_hi, p.tau_depth_lo,
        p.tau_depth_hi, p.tau_rgb_lo, p.tau_rgb_hi, p.tau_zero, (uint32_t)f->seed,
        (uint32_t)(f->seed >> 32));
    RL_LAUNCH_CK();
    return RL_OK;
}

// ---------------------------------------------------------------------------
// Eq. 1-3.  Probe q = p + delta * (fx / 585) / D(p), rounded to the nearest
// pixel and clamped to the image; a Depth split compares D(p) - D(q), a
// DA-RGB split C(p,c) - C(q,c), against tau; true goes right (2n+2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int probe_coord(int p, float off, int extent) {
    const float v = __fadd_rn(__fadd_rn((float)p, off), 0.5f);
    // floor to an integer (saturating beyond the int range, 0 for NaN), then
    // clamp: the same as clamping floor(v) in FP32 and converting
    return min(max(__float2int_rd(v), 0), extent - 1);
}

__device__ __forceinline__ int walk_tree(const float4 *__restrict__ nodes, int depth,
                                         const float *__restrict__ D, const uint8_t *__restrict__ C,
                                         int W, int H, float s, int x, int y, float d, float inv) {
    int n = 0;
    const int p = y * W + x;
    for (int level = 0; level < depth; ++level) {
        const float4 nd = __ldg(&nodes[n]);
        const uint32_t meta = __float_as_uint(nd.w);
        const float ox = __fmul_rn(__fmul_rn(nd.x, s), inv);
        const float oy = __fmul_rn(__fmul_rn(nd.y, s), inv);
        const int qx = probe_coord(x, ox, W);
        const int qy = probe_coord(y, oy, H);
        const int q = qy * W + qx;
        float f;
        if ((meta & 255u) == 0u) {
            const float dq = __ldg(&D[q]);
            f = __fsub_rn(d, dq > 0.0f ? dq : 0.0f);
        } else {
            const int c = (int)(meta >> 8);
            f = __fsub_rn((float)__ldg(&C[p * 3 + c]), (float)__ldg(&C[q * 3 + c]));
        }
        n = (f >= nd.z) ? 2 * n + 2 : 2 * n + 1;
    }
    return n - ((1 << depth) - 1);
}

// All T trees of one pixel walked level by level, interleaved: T
// independent chains of dependent node and probe loads in flight at once.
// PRE: the nodes' offsets are already multiplied by s (k_scale_nodes).
template <int T, bool PRE>
__device__ __forceinline__ void walk_trees(const float4 *__restrict__ nodes, int n_branch, int depth,
                                           const float *__restrict__ D, const uint8_t *__restrict__ C,
                                           int W, int H, float s, int x, int y, float d, float inv,
                                           int leaf[T]) {
    int n[T];
#pragma unroll
    for (int t = 0; t < T; ++t) n[t] = 0;
    const int p = y * W + x;
    for (int level = 0; level < depth; ++level) {
        float4 nd[T];
#pragma unroll
        for (int t = 0; t < T; ++t) nd[t] = __ldg(&nodes[(size_t)t * n_branch + n[t]]);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint32_t meta = __float_as_uint(nd[t].w);
            const float ox = __fmul_rn(PRE ? nd[t].x : __fmul_rn(nd[t].x, s), inv);
            const float oy = __fmul_rn(PRE ? nd[t].y : __fmul_rn(nd[t].y, s), inv);
            const int q = probe_coord(y, oy, H) * W + probe_coord(x, ox, W);
            float f;
            if ((meta & 255u) == 0u) {
                const float dq = __ldg(&D[q]);
                f = __fsub_rn(d, dq > 0.0f ? dq : 0.0f);
            } else {
                const int c = (int)(meta >> 8);
                f = __fsub_rn((float)__ldg(&C[p * 3 + c]), (float)__ldg(&C[q * 3 + c]));
            }
            n[t] = (f >= nd[t].z) ? 2 * n[t] + 2 : 2 * n[t] + 1;
        }
    }
#pragma unroll
    for (int t = 0; t < T; ++t) leaf[t] = n[t] - ((1 << depth) - 1);
}

template <int T, bool PRE>
__device__ __forceinline__ int walk_and_store(const float4 *nodes, int n_branch, int depth, const Frame &fr,
                                              float s, int x, int y, float d, float inv, uint16_t *o,
                                              int hw_max, const uint8_t *nmodes, int lpt, int k_top,
                                              bool count, uint4 *rec) {
    int leaf[kRecTrees], cnt[kRecTrees];
    walk_trees<T, PRE>(nodes, n_branch, depth, fr.depth, fr.rgb, fr.W, fr.H, s, x, y, d, inv, leaf);
    int total = 0;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        if (o) o[(size_t)t * hw_max] = (uint16_t)leaf[t];
        cnt[t] = count ? min((int)__ldg(&nmodes[t * lpt + leaf[t]]), k_top) : 0;
        total += cnt[t];
    }
    if (rec) *rec = make_rec(leaf, cnt, T);
    return total;
}

// out: uint16 [frame][tree][hw_max] (null: not written); one thread per
// pixel walks every tree.
// When `mcount` is given it also receives |M(u)| = sum over the trees of
// min(modes of the reached leaf, k_top) per pixel (0 without depth); the
// pixel records `prec` (at most kRecTrees trees) hold the per-tree counts.
// nodes_s: the nodes scaled for focal length fx_s (k_scale_nodes), used for
// the frames of that focal length, or null.
__global__ void k_leaves(const float4 *__restrict__ nodes, int n_branch, int depth, int n_trees,
                         const Frame *__restrict__ frames, int hw_max, uint16_t *__restrict__ out,
                         const uint8_t *__restrict__ nmodes, int leaves_per_tree, int k_top,
                         uint16_t *__restrict__ mcount, uint4 *__restrict__ prec,
                         const float4 *__restrict__ nodes_s, float fx_s) {
    const Frame fr = frames[blockIdx.y];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= fr.W * fr.H) return;
    const int x = p % fr.W, y = p / fr.W;
    const float d = __ldg(&fr.depth[p]);
    uint16_t *o = out ? out + (size_t)blockIdx.y * n_trees * hw_max + p : nullptr;  // null: no leaf map
    uint4 *rec = prec ? prec + (size_t)blockIdx.y * hw_max + p : nullptr;
    if (!(d > 0.0f)) {
        if (o)
            for (int t = 0; t < n_trees; ++t) o[(size_t)t * hw_max] = 0xFFFF;
        if (mcount) mcount[(size_t)blockIdx.y * hw_max + p] = 0;
        if (rec) *rec = make_uint4(0, 0, 0, 0);
        return;
    }
    const float s = __fdiv_rn(fr.fx, 585.0f);
    const float inv = __frcp_rn(d);
    int total = 0;
    const bool cnt = mcount != nullptr || prec != nullptr;  // per-tree counts wanted
    const bool pre = nodes_s != nullptr && fr.fx == fx_s;  // the same for the whole block (one frame)
#define RL_WALK(T)                                                                                          \
    total = pre ? walk_and_store<T, true>(nodes_s, n_branch, depth, fr, s, x, y, d, inv, o, hw_max, nmodes, \
                                          leaves_per_tree, k_top, cnt, rec)                                  \
                : walk_and_store<T, false>(nodes, n_branch, depth, fr, s, x, y, d, inv, o, hw_max, nmodes,  \
                                           leaves_per_tree, k_top, cnt, rec)
    switch (n_trees) {
    case 1: RL_WALK(1); break;
    case 2: RL_WALK(2); break;
    case 3: RL_WALK(3); break;
    case 4: RL_WALK(4); break;
    case 5: RL_WALK(5); break;
#undef RL_WALK
    default:
        for (int t = 0; t < n_trees; ++t) {
            const int leaf = walk_tree(nodes + (size_t)t * n_branch, depth, fr.depth, fr.rgb, fr.W, fr.H,
                                       s, x, y, d, inv);
            if (o) o[(size_t)t * hw_max] = (uint16_t)leaf;
            if (cnt) total += min((int)__ldg(&nmodes[t * leaves_per_tree + leaf]), k_top);
        }
    }
    if (mcount) mcount[(size_t)blockIdx.y * hw_max + p] = (uint16_t)total;
}

rl_status launch_leaves(const rl_forest *f, const Frame *frames_dev, int n_frames, int n_trees,
                        int hw_max, uint16_t *out, int max_w, int max_h, cudaStream_t s,
                        int k_top, uint16_t *mcount, uint4 *prec, int threads, const float4 *nodes_s,
                        float fx_s) {
    const int npx = max_w * max_h;
    dim3 grid((npx + threads - 1) / threads, n_frames);
    k_leaves<<<grid, threads, 0, s>>>(f->nodes, f->n_branch, f->p.depth, n_trees, frames_dev, hw_max, out,
                                  f->nmodes, f->leaves_per_tree, k_top, mcount,
                                  n_trees <= kRecTrees ? prec : nullptr, nodes_s, fx_s);
    RL_LAUNCH_CK();
    return RL_OK;
}

// The split nodes with their offsets multiplied by s = fx / 585 (Eq. 1-3's
// depth-normalised probe offset), rounded as the walk rounds its own first
// product: the walk then needs one product per coordinate.
__global__ void k_scale_nodes(const float4 *__restrict__ nodes, float4 *__restrict__ out, int count, float fx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float s = __fdiv_rn(fx, 585.0f);
    const float4 v = nodes[i];
    out[i] = make_float4(__fmul_rn(v.x, s), __fmul_rn(v.y, s), v.z, v.w);
}

rl_status launch_scale_nodes(const rl_forest *f, int n_trees, float4 *out, float fx, cudaStream_t s) {
    const int count = n_trees * f->n_branch;
    k_scale_nodes<<<(count + 255) / 256, 256, 0, s>>>(f->nodes, out, count, fx);
    RL_LAUNCH_CK();
    return RL_OK;
}

// ---------------------------------------------------------------------------
// Reservoir adaptation (Sec. 3.2.2), deterministic Algorithm R.
//
// For one frame: (1) every grid pixel with depth is back-projected, moved to
// world space and walked down every tree; per-leaf arrival counts are taken.
// (2) The rank of each example among the frame's examples of the same leaf
// (in pixel order) gives its count c = count_before_frame + rank.  (3) The
// Algorithm R decision for count c is a pure function of (leaf, c); an
// example writes its slot unless a later example of the same leaf in this
// frame draws the same slot.  (4) Counts are committed.
// ---------------------------------------------------------------------------
struct Pose12 {
    double m[12];
};

__global__ void k_adapt_examples(const float4 *__restrict__ nodes, int n_branch, int depth,
                                 int n_trees, int leaves_per_tree, const float *__restrict__ D,
                                 const uint8_t *__restrict__ C, int W, int H, float fx, float fy,
                                 float cx, float cy, Pose12 T, int gw, int gh, int step, int origin,
                                 uint32_t *__restrict__ ex_leaf, float4 *__restrict__ ex_pt,
                                 uint32_t *__restrict__ frame_cnt) {
    const int P = gw * gh;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P) return;
    const int x = origin + (g % gw) * step, y = origin + (g / gw) * step;
    const int p = y * W + x;
    const float d = D[p];
    if (!(d > 0.0f)) {
        for (int t = 0; t < n_trees; ++t) ex_leaf[(size_t)t * P + g] = 0xFFFFFFFFu;
        return;
    }
    const float xc = __fdiv_rn(__fmul_rn(__fsub_rn((float)x, cx), d), fx);
    const float yc = __fdiv_rn(__fmul_rn(__fsub_rn((float)y, cy), d), fy);
    const float zc = d;
    float w[3];
    for (int r = 0; r < 3; ++r) {
        const double a = __dmul_rn(T.m[4 * r + 0], (double)xc);
        const double b = __dmul_rn(T.m[4 * r + 1], (double)yc);
        const double c = __dmul_rn(T.m[4 * r + 2], (double)zc);
        w[r] = (float)__dadd_rn(__dadd_rn(__dadd_rn(a, b), c), T.m[4 * r + 3]);
    }
    const uint32_t rgb = (uint32_t)C[3 * p] | ((uint32_t)C[3 * p + 1] << 8) | ((uint32_t)C[3 * p + 2] << 16);
    ex_pt[g] = make_float4(w[0], w[1], w[2], __uint_as_float(rgb));
    const float s = __fdiv_rn(fx, 585.0f);
    const float inv = __frcp_rn(d);
    for (int t = 0; t < n_trees; ++t) {
        const int leaf = walk_tree(nodes + (size_t)t * n_branch, depth, D, C, W, H, s, x, y, d, inv);
        const uint32_t L = (uint32_t)(t * leaves_per_tree + leaf);
        ex_leaf[(size_t)t * P + g] = L;
        atomicAdd(&frame_cnt[L], 1u);
    }
}

// rank of example (t, g) among examples (t, g' < g) with the same leaf.
__global__ void k_adapt_rank(const uint32_t *__restrict__ ex_leaf, int P,
                             uint32_t *__restrict__ ex_rank) {
    __shared__ uint32_t tile[256];
    const int t = blockIdx.y;
    const uint32_t *row = ex_leaf + (size_t)t * P;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t mine = g < P ? row[g] : 0xFFFFFFFFu;
    const int last = min(P, (int)((blockIdx.x + 1) * blockDim.x));
    uint32_t rank = 0;
    for (int base = 0; base < last; base += 256) {
        const int j = base + threadIdx.x;
        tile[threadIdx.x] = j < P ? row[j] : 0xFFFFFFFEu;
        __syncthreads();
        const int lim = min(256, g - base);
        if (mine != 0xFFFFFFFFu)
            for (int k = 0; k < lim; ++k) rank += (tile[k] == mine);
        __syncthreads();
    }
    if (g < P) ex_rank[(size_t)t * P + g] = rank;
}

__device__ __forceinline__ int64_t reservoir_slot(uint32_t L, uint32_t c, int kappa, uint32_t k0,
                                                  uint32_t k1) {
    if (c < (uint32_t)kappa) return c;
    const uint4 r = philox(make_uint4(L, TAG_RESERVOIR << 16, c, 0), k0, k1);
    const uint64_t j = ((uint64_t)r.x * ((uint64_t)c + 1)) >> 32;
    return j < (uint64_t)kappa ? (int64_t)j : -1;
}

__global__ void k_adapt_insert(const uint32_t *__restrict__ ex_leaf,
                               const uint32_t *__restrict__ ex_rank, const float4 *__restrict__ ex_pt,
                               int P, int n_trees, const uint32_t *__restrict__ res_count,
                               const uint32_t *__restrict__ frame_cnt, int kappa, uint32_t k0,
                               uint32_t k1, float4 *__restrict__ res) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P * n_trees) return;
    const uint32_t L = ex_leaf[e];
    if (L == 0xFFFFFFFFu) return;
    const uint32_t base = res_count[L];
    const uint32_t c = base + ex_rank[e];
    const int64_t slot = reservoir_slot(L, c, kappa, k0, k1);
    if (slot < 0) return;
    const uint32_t end = base + frame_cnt[L];
    const uint32_t from = max(c + 1, (uint32_t)kappa);
    for (uint32_t c2 = from; c2 < end; ++c2)
        if (reservoir_slot(L, c2, kappa, k0, k1) == slot) return;  // overwritten later
    res[(size_t)L * kappa + slot] = ex_pt[e % P];
}

__global__ void k_adapt_commit(uint32_t *__restrict__ res_count, uint32_t *__restrict__ frame_cnt,
                               int L) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    const uint32_t n = frame_cnt[l];
    if (n) {
        res_count[l] += n;
        frame_cnt[l] = 0;
    }
}

rl_status adapt_frame(rl_forest *f, const float *depth, const uint8_t *rgb,
                      const rl_intrinsics *K, const double T[16], cudaStream_t s) {
    const rl_forest_params &p = f->p;
    const int o = p.grid_origin, st = p.grid_step;
    const int gw = K->width > o ? (K->width - o + st - 1) / st : 0;
    const int gh = K->height > o ? (K->height - o + st - 1) / st : 0;
    const int P = gw * gh;
    if (P == 0) return RL_OK;
    if (f->ex_capacity < P) {
        arena_free(f->ctx, f->ex_leaf);
        arena_free(f->ctx, f->ex_pt);
        arena_free(f->ctx, f->ex_rank);
        f->ex_leaf = nullptr;
        f->ex_pt = nullptr;
        f->ex_rank = nullptr;
        f->ex_capacity = 0;
        RL_TRY(alloc_n(f->ctx, (uint64_t)P * p.n_trees, &f->ex_leaf));
        RL_TRY(alloc_n(f->ctx, (uint64_t)P, &f->ex_pt));
        RL_TRY(alloc_n(f->ctx, (uint64_t)P * p.n_trees, &f->ex_rank));
        f->ex_capacity = P;
    }
    Pose12 pose;
    for (int i = 0; i < 12; ++i) pose.m[i] = T[i];
    const uint32_t k0 = (uint32_t)f->seed, k1 = (uint32_t)(f->seed >> 32);
    k_adapt_examples<<<(P + 127) / 128, 128, 0, s>>>(
        f->nodes, f->n_branch, p.depth, p.n_trees, f->leaves_per_tree, depth, rgb, K->width,
        K->height, K->fx, K->fy, K->cx, K->cy, pose, gw, gh, st, o, f->ex_leaf, f->ex_pt,
        f->frame_cnt);
    RL_LAUNCH_CK();
    k_adapt_rank<<<dim3((P + 255) / 256, p.n_trees), 256, 0, s>>>(f->ex_leaf, P, f->ex_rank);
    RL_LAUNCH_CK();
    const int E = P * p.n_trees;
    k_adapt_insert<<<(E + 255) / 256, 256, 0, s>>>(f->ex_leaf, f->ex_rank, f->ex_pt, P, p.n_trees,
                                                   f->res_count, f->frame_cnt, p.kappa, k0, k1,
                                                   f->res);
    RL_LAUNCH_CK();
    k_adapt_commit<<<(f->n_leaves + 255) / 256, 256, 0, s>>>(f->res_count, f->frame_cnt, f->n_leaves);
    RL_LAUNCH_CK();
    return RL_OK;
}

rl_status reset_leaves(rl_forest *f, cudaStream_t s) {
    RL_CK(cudaMemsetAsync(f->res_count, 0, sizeof(uint32_t) * f->n_leaves, s));
    RL_CK(cudaMemsetAsync(f->frame_cnt, 0, sizeof(uint32_t) * f->n_leaves, s));
    RL_CK(cudaMemsetAsync(f->nmodes, 0, f->n_leaves, s));
    RL_CK(cudaMemsetAsync(f->centroid, 0, sizeof(float4) * f->n_leaves, s));
    f->cursor = 0;
    return RL_OK;
}

}  // namespace rl
