// Hypothesis generation (Sec. 3.2.3): the first iteration of each slot whose
// triple of pixel-to-mode correspondences passes the three checks, one warp
// per hypothesis slot (the pose of that triple is fitted by a separate
// kernel); compaction of the successful slots; pixel batches of the
// preemptive RANSAC.
//
// Compiled with --fmad=false: back-projection (FP32) and the three checks
// (FP64 from FP32 inputs) are plain IEEE operations in a fixed order, so
// every accept/reject decision, and therefore the winning iteration of each
// slot, is exactly reproducible.
#include "hypgen_dev.cuh"
#include "kernels.h"

namespace rl {

__device__ __forceinline__ double dist2_64(float3 a, float3 b) {
    const double e0 = (double)a.x - (double)b.x, e1 = (double)a.y - (double)b.y;
    const double e2 = (double)a.z - (double)b.z;
    return (e0 * e0 + e1 * e1) + e2 * e2;
}

__device__ __forceinline__ float dist2_32(float3 a, float3 b) {
    const float e0 = __fsub_rn(a.x, b.x), e1 = __fsub_rn(a.y, b.y), e2 = __fsub_rn(a.z, b.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(e0, e0), __fmul_rn(e1, e1)), __fmul_rn(e2, e2));
}

// Thresholds of the FP32 pre-tests: the squared spread threshold widened by
// 2e-5 relative and rounded outwards, and the rigidity tolerance.
struct CheckThr {
    float sq_lo, sq_hi, tol;
};

// A generation attempt is evaluated in two stages, cheapest rejection first
// (the outcome does not depend on the order).  Stage 1: the draws, a
// non-empty M(u) at every pixel (|M(u)| is 0 without depth) and the colour
// of the checked pair.  Stage 2: the modes of the other pairs, spread and
// rigidity.  The spread and rigidity tests run in FP32 (errors below 1e-6
// relative) and are re-evaluated in FP64 whenever the FP32 value lies within
// 2e-5 relative of the threshold, so each decision equals the FP64 decision
// while the narrow FP64 pipe is almost never used.
template <int REDRAW>
__device__ __forceinline__ bool stage1(const HypArgs &a, const Frame &fr, const uint16_t *lv,
                                       const uint16_t *mc, const uint4 *pr, int slot, int it,
                                       Draw &d) {
    const int T = a.p.n_trees;
    auto usable = [&](int q) { return pixel_modes(mc, pr, q, T) != 0; };
    d = draw<decltype(usable), REDRAW>(a, fr, slot, it, usable);
    const int c0 = pixel_modes(mc, pr, d.pix[0], T), c1 = pixel_modes(mc, pr, d.pix[1], T),
              c2 = pixel_modes(mc, pr, d.pix[2], T);
    if (c0 == 0 || c1 == 0 || c2 == 0) return false;
    const uint32_t ctr1 = (TAG_HYP << 16) | (uint32_t)a.p.level;
    const uint4 r1 = philox(make_uint4(slot, ctr1, it, 1), fr.key0, fr.key1);
    d.m[0] = draw_below(r1.x, (uint32_t)c0);
    d.m[1] = draw_below(r1.y, (uint32_t)c1);
    d.m[2] = draw_below(r1.z, (uint32_t)c2);
    // check 1: colour of pair j
    const int j = d.j;
    const int pj = j == 0 ? d.pix[0] : (j == 1 ? d.pix[1] : d.pix[2]);
    const int mj = (int)(j == 0 ? d.m[0] : (j == 1 ? d.m[1] : d.m[2]));
    uint32_t L;
    int rank;
    lookup(a, lv, pr, pj, mj, &L, &rank);
    const uchar4 mcol = a.mv.mrgb[(size_t)L * a.mv.m_max + rank];
    const uint8_t *pc = fr.rgb + (size_t)pj * 3;
    const int dr = abs((int)pc[0] - (int)mcol.x), dg = abs((int)pc[1] - (int)mcol.y),
              db = abs((int)pc[2] - (int)mcol.z);
    return max(dr, max(dg, db)) <= a.p.colour_thresh;
}

// Stage 1 from the colour-check masks: per attempt three independent 8-byte
// loads give every |M(u)| and the colour decision of each mode of the
// checked pixel.  Two attempts run together, with every load issued before
// the second Philox block of either attempt, which then hides the latency.
// Draws are valid pixel indices for any counter, so the loads need no guard.
__device__ __forceinline__ bool mask_decide(const uint2 w0, const uint2 w1, const uint2 w2, const uint4 r1,
                                            Draw &d) {
    const uint32_t c0 = w0.y >> 24, c1 = w1.y >> 24, c2 = w2.y >> 24;
    if (c0 == 0 || c1 == 0 || c2 == 0) return false;
    d.m[0] = draw_below(r1.x, c0);
    d.m[1] = draw_below(r1.y, c1);
    d.m[2] = draw_below(r1.z, c2);
    const uint2 wj = d.j == 0 ? w0 : (d.j == 1 ? w1 : w2);
    const uint32_t mj = d.j == 0 ? d.m[0] : (d.j == 1 ? d.m[1] : d.m[2]);
    const uint32_t bits = mj < 32 ? wj.x >> mj : wj.y >> (mj - 32);
    return (bits & 1u) != 0;
}

template <int REDRAW>
__device__ __forceinline__ void stage1_mask2(const HypArgs &a, const Frame &fr, const uint2 *cm, int slot,
                                             int itA, int itB, Draw &dA, Draw &dB, bool &sA, bool &sB) {
    auto usable = [&](int q) { return (cm[q].y >> 24) != 0; };
    dA = draw<decltype(usable), REDRAW>(a, fr, slot, itA, usable);
    dB = draw<decltype(usable), REDRAW>(a, fr, slot, itB, usable);
    const uint2 a0 = cm[dA.pix[0]], a1 = cm[dA.pix[1]], a2 = cm[dA.pix[2]];
    const uint2 b0 = cm[dB.pix[0]], b1 = cm[dB.pix[1]], b2 = cm[dB.pix[2]];
    const uint32_t ctr1 = (TAG_HYP << 16) | (uint32_t)a.p.level;
    const uint4 rA = philox(make_uint4(slot, ctr1, itA, 1), fr.key0, fr.key1);
    const uint4 rB = philox(make_uint4(slot, ctr1, itB, 1), fr.key0, fr.key1);
    sA = mask_decide(a0, a1, a2, rA, dA);
    sB = mask_decide(b0, b1, b2, rB, dB);
}

// Stage 1 from the non-empty-M(u) bitmap (staged in shared memory) and the
// colour-check masks: the three draws must have a non-empty M(u) (three
// bit tests), and only the checked pixel j's mask word is gathered, for its
// |M(u)| and colour bits; the mode indices of the other two pixels are drawn
// in stage 2.  The decision is the same as mask_decide's.
__device__ __forceinline__ bool bit_set(const uint32_t *bits, int p) { return (bits[p >> 5] >> (p & 31)) & 1u; }

template <int REDRAW>
__device__ __forceinline__ void stage1_bits2(const HypArgs &a, const Frame &fr, const uint2 *cm,
                                             const uint32_t *s_bits, int slot, int itA, int itB, Draw &dA,
                                             Draw &dB, bool &sA, bool &sB) {
    auto usable = [&](int q) { return bit_set(s_bits, q); };
    dA = draw<decltype(usable), REDRAW>(a, fr, slot, itA, usable);
    dB = draw<decltype(usable), REDRAW>(a, fr, slot, itB, usable);
    const int pjA = dA.j == 0 ? dA.pix[0] : (dA.j == 1 ? dA.pix[1] : dA.pix[2]);
    const int pjB = dB.j == 0 ? dB.pix[0] : (dB.j == 1 ? dB.pix[1] : dB.pix[2]);
    const uint2 wA = cm[pjA], wB = cm[pjB];
    const bool okA = bit_set(s_bits, dA.pix[0]) && bit_set(s_bits, dA.pix[1]) && bit_set(s_bits, dA.pix[2]);
    const bool okB = bit_set(s_bits, dB.pix[0]) && bit_set(s_bits, dB.pix[1]) && bit_set(s_bits, dB.pix[2]);
    const uint32_t ctr1 = (TAG_HYP << 16) | (uint32_t)a.p.level;
    const uint4 rA = philox(make_uint4(slot, ctr1, itA, 1), fr.key0, fr.key1);
    const uint4 rB = philox(make_uint4(slot, ctr1, itB, 1), fr.key0, fr.key1);
    auto decide = [](bool ok, uint2 w, uint4 r, const Draw &d) {
        if (!ok) return false;
        const uint32_t rj = d.j == 0 ? r.x : (d.j == 1 ? r.y : r.z);
        const uint32_t mj = draw_below(rj, w.y >> 24);
        const uint32_t bits = mj < 32 ? w.x >> mj : w.y >> (mj - 32);
        return (bits & 1u) != 0;
    };
    sA = decide(okA, wA, rA, dA);
    sB = decide(okB, wB, rB, dB);
}

// rec, dep: the three pixels' records and depths when already gathered
// (else read here).
__device__ __forceinline__ bool stage2(const HypArgs &a, const CheckThr &ct, const Frame &fr,
                                       const uint16_t *lv, const uint4 *pr, const int pix[3],
                                       const int m[3], const uint4 *rec = nullptr, const float *dep = nullptr) {
    float3 xw[3];
    for (int i = 0; i < 3; ++i) {
        uint32_t L;
        int rank;
        if (rec)
            mode_at_rec(rec[i], a.p.n_trees, a.mv.leaves_per_tree, m[i], &L, &rank);
        else
            lookup(a, lv, pr, pix[i], m[i], &L, &rank);
        xw[i] = mode_pos(a.mv, L, rank);
    }
    // check 2: scene points pairwise at least sqrt(min_sq_dist) apart
    const int PA[3] = {0, 0, 1}, PB[3] = {1, 2, 2};
    float dW2f[3];
    for (int k = 0; k < 3; ++k) {
        dW2f[k] = dist2_32(xw[PA[k]], xw[PB[k]]);
        if (dW2f[k] < ct.sq_lo) return false;
        if (!(dW2f[k] > ct.sq_hi) && dist2_64(xw[PA[k]], xw[PB[k]]) < a.p.min_sq_dist) return false;
    }
    // check 3: rigidity, |d_W - d_C| <= max_trans_err for every pair
    float3 xc[3];
    for (int i = 0; i < 3; ++i) xc[i] = dep ? backproject_d(fr, pix[i], dep[i]) : backproject(fr, pix[i]);
    for (int k = 0; k < 3; ++k) {
        const float dw = sqrtf(dW2f[k]), dc = sqrtf(dist2_32(xc[PA[k]], xc[PB[k]]));
        const float diff = fabsf(__fsub_rn(dw, dc));
        const float margin = __fadd_rn(__fmul_rn(2e-5f, __fadd_rn(dw, dc)), 2e-6f);
        if (diff > __fadd_rn(ct.tol, margin)) return false;
        if (diff >= __fsub_rn(ct.tol, margin)) {
            const double e = fabs(sqrt(dist2_64(xw[PA[k]], xw[PB[k]])) -
                                  sqrt(dist2_64(xc[PA[k]], xc[PB[k]])));
            if (e > a.p.max_trans_err) return false;
        }
    }
    return true;
}

// Warp per (frame, slot).  The 32 lanes run stage 1 on 64 (with masks) or
// 32 consecutive iterations and append the survivors, in iteration order, to
// a ring in shared memory; whenever it holds 32 of them, the lanes run
// stage 2 on the 32 oldest.  The first success in a drained group is the lowest successful
// iteration, exactly as a sequential loop would find it: every lower
// iteration failed stage 1 or was drained earlier.  Compaction keeps the
// lanes converged on the rarely reached stage 2.
constexpr int HG_RING = 128;  // < 32 pending after a drain + 64 appended

// WARPS slots per block; registers stay capped at 64 (32 warps per SM).
template <int WARPS, int REDRAW>
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS) k_hypgen(HypArgs a) {
    constexpr int HG_WARPS = WARPS;
    __shared__ int4 s_ring[HG_WARPS][HG_RING];   // it | j << 30, pixels of the triple
    __shared__ uint2 s_mode[HG_WARPS][HG_RING];  // mode indices m0 | m1 << 16, m2 (without the bitmap)
    extern __shared__ uint32_t s_bits[];         // the frame's non-empty-M(u) bitmap (with pbits)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int slot = blockIdx.x * HG_WARPS + w;
    const int b = blockIdx.y;
    const Frame fr = a.frames[b];
    const bool use_bits = a.pbits != nullptr && a.pcm != nullptr;
    if (use_bits) {  // every thread of the block stages the bitmap, before any may leave
        const int nw = (fr.W * fr.H + 31) >> 5;
        const uint32_t *src = a.pbits + (size_t)b * (a.hw_max / 32 + 1);
        for (int k = threadIdx.x; k < nw; k += blockDim.x) s_bits[k] = src[k];
        __syncthreads();
    }
    if (slot >= a.p.n_hyp) return;
    int32_t *iter_out = a.hyp_iter + (size_t)b * a.p.n_hyp + slot;
    if (fr.W * fr.H == 0) {  // empty frame (e.g. accepted by an earlier cascade level)
        if (lane == 0) *iter_out = -1;
        return;
    }
    const uint16_t *lv = a.leaves + (size_t)b * a.p.n_trees * a.hw_max;
    const uint16_t *mc = a.mcount + (size_t)b * a.hw_max;
    const uint4 *pr = a.prec ? a.prec + (size_t)b * a.hw_max : nullptr;
    const uint2 *cm = a.pcm ? a.pcm + (size_t)b * a.hw_max : nullptr;
    CheckThr ct;
    ct.sq_lo = __double2float_rd(a.p.min_sq_dist * (1.0 - 2e-5));
    ct.sq_hi = __double2float_ru(a.p.min_sq_dist * (1.0 + 2e-5));
    ct.tol = (float)a.p.max_trans_err;
    int4 *ring = s_ring[w];
    uint2 *rmode = s_mode[w];
    unsigned head = 0, tail = 0;  // warp-uniform ring counters
    const unsigned lt = (1u << lane) - 1u;
    // Stage 2 on the pending entries head .. head + n - 1 (n <= 32); the
    // winning lane stores its iteration.
    unsigned n_att = 0, n_s2 = 0;  // stage-1 attempts and stage-2 evaluations (profiling)
    auto count = [&]() {
        if (a.work && lane == 0) {
            atomicAdd(&a.work[W_HYP_ATTEMPTS], (unsigned long long)n_att);
            atomicAdd(&a.work[W_HYP_STAGE2], (unsigned long long)n_s2);
        }
    };
    auto drain = [&](unsigned n) -> bool {
        n_s2 += n;
        bool ok = false;
        int it = 0;
        if ((unsigned)lane < n) {
            const unsigned e = (head + lane) % HG_RING;
            const int4 r = ring[e];
            const int pix[3] = {r.y, r.z, r.w};
            it = r.x & 0x3fffffff;
            int m[3];
            if (use_bits && pr) {
                // every gather that depends on the pixels alone, issued
                // together: |M(u)|, the pixel records and the depths; then
                // the mode draws of the attempt from its second Philox block
                uint32_t c3[3];
                uint4 rec[3];
                float dep[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    c3[i] = cm[pix[i]].y >> 24;
                    rec[i] = pr[pix[i]];
                    dep[i] = fr.depth[pix[i]];
                }
                const uint32_t ctr1 = (TAG_HYP << 16) | (uint32_t)a.p.level;
                const uint4 r1 = philox(make_uint4(slot, ctr1, it, 1), fr.key0, fr.key1);
                m[0] = (int)draw_below(r1.x, c3[0]);
                m[1] = (int)draw_below(r1.y, c3[1]);
                m[2] = (int)draw_below(r1.z, c3[2]);
                ok = stage2(a, ct, fr, lv, pr, pix, m, rec, dep);
            } else {
                if (use_bits) {
                    const uint32_t ctr1 = (TAG_HYP << 16) | (uint32_t)a.p.level;
                    const uint4 r1 = philox(make_uint4(slot, ctr1, it, 1), fr.key0, fr.key1);
                    m[0] = (int)draw_below(r1.x, cm[pix[0]].y >> 24);
                    m[1] = (int)draw_below(r1.y, cm[pix[1]].y >> 24);
                    m[2] = (int)draw_below(r1.z, cm[pix[2]].y >> 24);
                } else {
                    const uint2 mm = rmode[e];
                    m[0] = (int)(mm.x & 0xffffu);
                    m[1] = (int)(mm.x >> 16);
                    m[2] = (int)mm.y;
                }
                ok = stage2(a, ct, fr, lv, pr, pix, m);
            }
        }
        const unsigned win = __ballot_sync(0xffffffffu, ok);
        if (win && lane == __ffs(win) - 1) *iter_out = it;
        head += n;
        return win != 0;
    };
    auto append = [&](bool s1, int it, const Draw &d) {
        const unsigned mask = __ballot_sync(0xffffffffu, s1);
        if (s1) {
            const unsigned e = (tail + __popc(mask & lt)) % HG_RING;
            ring[e] = make_int4(it | (d.j << 30), d.pix[0], d.pix[1], d.pix[2]);
            if (!use_bits) rmode[e] = make_uint2(d.m[0] | (d.m[1] << 16), d.m[2]);
        }
        tail += __popc(mask);
    };
    // iterations in groups of 64 (masks: two per lane) or 32; survivors are
    // appended in iteration order
    const int step = cm ? 64 : 32;
    for (int base = 0; base < a.p.max_iter; base += step) {
        if (cm) {
            Draw dA, dB;
            bool sA, sB;
            const int itA = base + lane, itB = base + 32 + lane;
            if (use_bits)
                stage1_bits2<REDRAW>(a, fr, cm, s_bits, slot, itA, itB, dA, dB, sA, sB);
            else
                stage1_mask2<REDRAW>(a, fr, cm, slot, itA, itB, dA, dB, sA, sB);
            append(sA && itA < a.p.max_iter, itA, dA);
            append(sB && itB < a.p.max_iter, itB, dB);
        } else {
            const int it = base + lane;
            Draw d;
            const bool s1 = it < a.p.max_iter && stage1<REDRAW>(a, fr, lv, mc, pr, slot, it, d);
            append(s1, it, d);
        }
        n_att += (unsigned)min(step, a.p.max_iter - base);
        __syncwarp();
        while (tail - head >= 32) {
            if (drain(32)) {
                count();
                return;
            }
            __syncwarp();
        }
    }
    if (!(tail - head > 0 && drain(tail - head)) && lane == 0) *iter_out = -1;
    count();
}

// Colour-check masks (Sec. 3.2.3, check 1 precomputed): bit m of pixel u is
// set iff the m-th mode of M(u) passes the colour check against u's RGB;
// |M(u)| (<= kMaskModes) sits in the top byte.  The same integer test as the
// per-attempt check, so every decision is unchanged.
__global__ void __launch_bounds__(256) k_colour_mask(const Frame *__restrict__ frames,
                                                     const uint16_t *__restrict__ mcount,
                                                     const uint4 *__restrict__ prec, int hw_max, ModeView mv,
                                                     RParams p, uint2 *__restrict__ pcm,
                                                     uint32_t *__restrict__ pbits) {
    const int b = blockIdx.y;
    const Frame fr = frames[b];
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = px < fr.W * fr.H;
    const size_t o = (size_t)b * hw_max + px;
    const uint4 rec = in ? prec[o] : make_uint4(0, 0, 0, 0);  // masks exist only with pixel records
    int cnt = 0;
    for (int t = 0; t < p.n_trees; ++t) cnt += rec_count(rec, t);  // |M(u)|
    // bit px of the non-empty-M(u) bitmap: a warp covers one 32-pixel word
    const unsigned word = __ballot_sync(0xffffffffu, cnt > 0);
    if (in && (threadIdx.x & 31) == 0) pbits[(size_t)b * (hw_max / 32 + 1) + (px >> 5)] = word;
    if (!in) return;
    uint32_t lo = 0, hi = 0;
    if (cnt > 0) {
        const uint8_t *pc = fr.rgb + (size_t)px * 3;
        const int pr = pc[0], pg = pc[1], pb = pc[2];
        int m = 0;
        for (int t = 0; t < p.n_trees; ++t) {
            const int nm = rec_count(rec, t);
            const uchar4 *col = mv.mrgb + (size_t)(t * mv.leaves_per_tree + rec_leaf(rec, t)) * mv.m_max;
            for (int r = 0; r < nm; ++r, ++m) {
                const uchar4 c = col[r];
                const int dl = max(abs(pr - (int)c.x), max(abs(pg - (int)c.y), abs(pb - (int)c.z)));
                if (dl <= p.colour_thresh) {
                    if (m < 32) lo |= 1u << m;
                    else hi |= 1u << (m - 32);
                }
            }
        }
    }
    pcm[o] = make_uint2(lo, hi | ((uint32_t)cnt << 24));
}

rl_status launch_colour_mask(const Frame *frames, const uint16_t *mcount, const uint4 *prec, int hw_max,
                             ModeView mv, const RParams &p, uint2 *pcm, uint32_t *pbits, int n, int max_hw,
                             cudaStream_t s, int threads) {
    dim3 grid((max_hw + threads - 1) / threads, n);
    k_colour_mask<<<grid, threads, 0, s>>>(frames, mcount, prec, hw_max, mv, p, pcm, pbits);
    RL_LAUNCH_CK();
    return RL_OK;
}

// Successful slots in slot order (block per frame).
__global__ void __launch_bounds__(1024) k_compact(const int32_t *__restrict__ hyp_iter, int N,
                                                  int32_t *__restrict__ hyp_list,
                                                  int32_t *__restrict__ n_hyp) {
    __shared__ int warp_tot[32];
    __shared__ int running;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int32_t *it = hyp_iter + (size_t)b * N;
    int32_t *out = hyp_list + (size_t)b * N;
    if (tid == 0) running = 0;
    __syncthreads();
    for (int base = 0; base < N; base += blockDim.x) {
        const int s = base + tid;
        const bool v = s < N && it[s] >= 0;
        const unsigned m = __ballot_sync(0xffffffffu, v);
        if (lane == 0) warp_tot[w] = __popc(m);
        __syncthreads();
        int off = running;
        for (int k = 0; k < w; ++k) off += warp_tot[k];
        if (v) out[off + __popc(m & ((1u << lane) - 1))] = s;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += warp_tot[k];
            running += t;
        }
        __syncthreads();
    }
    if (tid == 0) n_hyp[b] = running;
}

// Pixel batch `batch`: eta draws, each redrawn up to batch_attempts times
// until its pixel has a non-empty M(u) (which implies depth); skipped (-1)
// otherwise.
__global__ void k_sample_batch(const Frame *__restrict__ frames, const uint16_t *__restrict__ mcount,
                               const uint4 *__restrict__ prec, int hw_max, RParams p, int batch,
                               int32_t *__restrict__ pix_out, float4 *__restrict__ xc_out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (j >= p.eta) return;
    const Frame fr = frames[b];
    const uint16_t *mc = mcount + (size_t)b * hw_max;
    const uint4 *pr = prec ? prec + (size_t)b * hw_max : nullptr;
    const uint32_t WH = (uint32_t)(fr.W * fr.H);
    int pix = -1;
    for (int at = 0; at < p.batch_attempts && WH > 0; ++at) {
        const uint4 r = philox(make_uint4(batch, (TAG_BATCH << 16) | (uint32_t)p.level, j, at),
                               fr.key0, fr.key1);
        const int q = (int)draw_below(r.x, WH);
        if (pixel_modes(mc, pr, q, p.n_trees) == 0) continue;
        pix = q;
        break;
    }
    const size_t o = (size_t)b * p.max_pix + (size_t)batch * p.eta + j;
    pix_out[o] = pix;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pix >= 0) {
        const float3 c = backproject(fr, pix);
        x = make_float4(c.x, c.y, c.z, 0.f);
    }
    xc_out[o] = x;
}

template <int REDRAW>
static void launch_hypgen_shape(const HypArgs &a, int warps, int n, size_t sm, cudaStream_t s) {
    const int N = a.p.n_hyp;
    switch (warps) {
    case 2: k_hypgen<2, REDRAW><<<dim3((N + 1) / 2, n), 64, sm, s>>>(a); break;
    case 8: k_hypgen<8, REDRAW><<<dim3((N + 7) / 8, n), 256, sm, s>>>(a); break;
    case 16: k_hypgen<16, REDRAW><<<dim3((N + 15) / 16, n), 512, sm, s>>>(a); break;
    default: k_hypgen<4, REDRAW><<<dim3((N + 3) / 4, n), 128, sm, s>>>(a); break;
    }
}

rl_status launch_hypgen(const Frame *frames, const uint16_t *leaves, const uint16_t *mcount,
                        const uint4 *prec, const uint2 *pcm, const uint32_t *pbits, int hw_max, ModeView mv,
                        const RParams &p, double *hyp_pose, int32_t *hyp_iter, unsigned long long *work, int n,
                        cudaStream_t s, int warps) {
    // the bitmap path needs the frame's bitmap in shared memory
    const size_t bits_smem = (size_t)(hw_max / 32 + 1) * 4;
    const bool bits = pcm && pbits && bits_smem <= kHypBitsSmemMax;
    HypArgs a{frames, leaves, mcount, prec, pcm, hw_max, mv, p, hyp_pose, hyp_iter, work, bits ? pbits : nullptr};
    const size_t sm = bits ? bits_smem : 0;
    if (p.redraw)
        launch_hypgen_shape<1>(a, warps, n, sm, s);
    else
        launch_hypgen_shape<0>(a, warps, n, sm, s);
    RL_LAUNCH_CK();
    return RL_OK;
}

template <int REDRAW>
static rl_status prepare_hypgen_reading() {
    const int sm = (int)kHypBitsSmemMax;
    RL_CK(cudaFuncSetAttribute(k_hypgen<2, REDRAW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    RL_CK(cudaFuncSetAttribute(k_hypgen<4, REDRAW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    RL_CK(cudaFuncSetAttribute(k_hypgen<8, REDRAW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    RL_CK(cudaFuncSetAttribute(k_hypgen<16, REDRAW>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    return RL_OK;
}

rl_status prepare_hypgen() {
    RL_TRY(prepare_hypgen_reading<0>());
    return prepare_hypgen_reading<1>();
}

rl_status launch_compact(const int32_t *hyp_iter, int N, int32_t *hyp_list, int32_t *n_hyp, int n,
                         cudaStream_t s) {
    k_compact<<<n, 1024, 0, s>>>(hyp_iter, N, hyp_list, n_hyp);
    RL_LAUNCH_CK();
    return RL_OK;
}

rl_status launch_sample_batch(const Frame *frames, const uint16_t *mcount, const uint4 *prec, int hw_max,
                              const RParams &p, int batch, int32_t *pix, float4 *xc, int n,
                              cudaStream_t s) {
    dim3 grid((p.eta + 127) / 128, n);
    k_sample_batch<<<grid, 128, 0, s>>>(frames, mcount, prec, hw_max, p, batch, pix, xc);
    RL_LAUNCH_CK();
    return RL_OK;
}

}  // namespace rl
