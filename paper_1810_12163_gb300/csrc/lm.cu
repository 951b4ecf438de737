// Levenberg-Marquardt refinement of a preemptive round (Sec. 3.2.3) with one
// thread-block cluster per frame.
//
// The CTAS CTAs of a cluster share the frame's surviving hypotheses
// (n <= 64) and split its pixel set by tiles of LMC_P pixels: CTA c takes
// tiles c, c + CTAS, ...  The first round (most hypotheses, fewest pixels)
// uses clusters of 4.  Later rounds have few hypotheses and up to 3.5x the
// pixels; a frame's LM there is a chain of passes whose length is set by its
// slowest hypothesis, so they use clusters of 8 to shorten each pass.  The
// cluster size is a function of the round alone, so a frame's results do not
// depend on the batch it runs in.
//
// A pass streams the CTA's tiles of the mode table (rows of decoded M(u))
// into shared memory with bulk asynchronous copies on an mbarrier pipeline.
// It covers the hypotheses still iterating, listed in increasing order:
// thread t works for list entry t % HB on pixel group t / HB (HB = next power
// of two >= their count), so the lanes of a warp mostly read the same staged
// row (broadcast) and share control flow, and once most hypotheses have
// stopped the few remaining ones are spread over all lanes.  Per
// (hypothesis, pixel) a pass finds the nearest mode under the pixel's
// Mahalanobis metric, keeps it if within the inlier radius and adds its
// terms to FP32 normal equations.
//
// The iterations of the method (normal equations at H, damped solve, cost
// of the step on the same correspondences, accept iff it decreases) are
// regrouped so that each iteration needs one pass: the pass at the trial
// pose Hn evaluates the step's cost on the current correspondences (read
// from the staged tile) and, in the same sweep, the correspondences and
// normal equations at Hn, which become those of the next iteration if the
// step is accepted; after a rejection the pose, and so its normal
// equations, are unchanged.  Correspondences are double-buffered per
// hypothesis (int16).  The arithmetic and its order are those of the plain
// sequence, so the results are the same.
//
// Sums are reduced over the CTA in group order and over the cluster through
// distributed shared memory in rank order, so every CTA holds bit-identical
// values; each CTA solves every hypothesis's 6x6 system in FP64 and takes
// the same decisions, with one cluster barrier per iteration.
//
// Every wait on a copy is bounded: a wait that gives up marks the frame in
// dev_err, the CTA skips the rest of its work while keeping step with the
// cluster barriers, and waits (bounded again) for its copies in flight
// before it exits.
#include <cooperative_groups.h>

#include "internal.h"
#include "kernels.h"
#include "lm_dev.cuh"

namespace rl {

namespace cg = cooperative_groups;

constexpr int LMC_CTAS_FIRST = 4;  // cluster size of the first preemptive round
constexpr int LMC_CTAS_LATER = 8;  // and of the later rounds
constexpr int LMC_THREADS = 256;
constexpr int LMC_P = 16;        // pixels per tile (max_pix is a multiple)
constexpr int LMC_STAGES = 2;
constexpr int LMC_HMAX = 64;
constexpr int LMC_NV = 31;       // 21 J^T J + 6 J^T r + cost, inlier count, trial cost, Eq. 5 energy
constexpr int LMC_PS = 33;       // odd stride of the per-thread partials (no bank conflicts)
constexpr uint32_t kWaitLimit = kLmWaitLimit;
constexpr int LMC_KP = 4;                       // pixels of a thread per tile (staged) or chunk (direct)
constexpr int LMC_LIST = LMC_THREADS * LMC_KP;  // full-search list capacity of a tile or chunk
constexpr int LMC_SB = 8;                       // lanes per full nearest-mode search
constexpr int LMC_DIRECT = 8;                   // at most this many hypotheses: rows read from global memory
constexpr int LMC_COOP = LMC_THREADS / 16;      // at most this many hypotheses: one half-warp per solve

struct LmcLayout {
    uint32_t t0, t1, t2, xc, cnt, stage, tx;
    uint32_t H, Hn, Pf, lambda, tot, nw, loc, state, cbuf, act, list, flag, bar, total;
};

__host__ __device__ inline uint32_t lmc_a16(uint32_t x) { return (x + 15u) & ~15u; }

// Shared-memory layout for rows of `stride` modes.  Region 0 holds the
// staged tiles during the pixel pass and the per-thread partial sums during
// the reductions (never both at once).
__host__ __device__ inline LmcLayout lmc_layout(int stride, bool cov) {
    LmcLayout L;
    const uint32_t rows = (uint32_t)LMC_P * (uint32_t)stride;
    uint32_t o = 0;
    L.t0 = o; o += rows * 16;
    L.t1 = o; if (cov) o += rows * 16;
    L.t2 = o; if (cov) o += lmc_a16(rows * 4);
    L.xc = o; o += LMC_P * 16;
    L.cnt = o; o += lmc_a16(LMC_P * 2);
    L.stage = o;
    L.tx = rows * 16 + (cov ? rows * 20 : 0) + LMC_P * 16 + LMC_P * 2;
    const uint32_t stages = LMC_STAGES * L.stage;
    const uint32_t partials = LMC_THREADS * LMC_PS * 4;
    o = lmc_a16(stages > partials ? stages : partials);
    L.H = o; o += LMC_HMAX * 12 * 8;
    L.Hn = o; o += LMC_HMAX * 12 * 8;
    L.Pf = o; o += LMC_HMAX * 12 * 4;
    L.lambda = o; o += LMC_HMAX * 8;
    L.tot = o; o += LMC_HMAX * LMC_NV * 4;
    L.nw = o; o += LMC_HMAX * LMC_NV * 4;
    L.loc = o; o += 2 * LMC_HMAX * LMC_NV * 4;
    L.state = o; o += LMC_HMAX * 4;
    L.cbuf = o; o += LMC_HMAX * 4;
    L.act = o; o += LMC_HMAX * 4 + 16;  // list, then its length
    L.list = o; o += LMC_LIST * 4;      // pairs to search in full (int16) and their nearest modes (int16)
    L.flag = o; o += 16;
    L.bar = o; o += LMC_STAGES * 8;
    L.total = lmc_a16(o);
    return L;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t limit = kWaitLimit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// One pass over this CTA's tiles at pose P (per hypothesis, FP32 copy in
// registers): nearest mode, inlier test and normal-equation terms for every
// (hypothesis, pixel), correspondences written to buffer `wbuf`; with
// `trial`, also the cost of the correspondences in buffer `rbuf` at P.
struct LmcPass {
    float acc[28];
    int nin;
    float trial;
    float energy;  // Eq. 5 at the pass's pose: sum over the pixels of the nearest mode's distance
};

// The damped step of one hypothesis by one lane: T its sums (21 J^T J upper
// triangle, 6 J^T r, cost, inlier count), the FP64 solve, and either the new
// pose (Hn, FP32 copy Pf) or *state = 0 when the step stops it.  Both solve
// variants stay out of line, so that their registers do not weigh on the
// pixel passes.
__device__ __noinline__ void lm_solve_lane(const float *T, double lambda, const double *H, double lm_stop,
                                           int *state, double *Hn, float *Pf) {
    bool stop = T[28] < 3.f;
    double step[6];
    if (!stop) {
        double A[36], rhs[6];
        int k = 0;
        for (int r = 0; r < 6; ++r)
            for (int c = r; c < 6; ++c, ++k) A[6 * r + c] = A[6 * c + r] = (double)T[k];
        for (int r = 0; r < 6; ++r) {
            A[6 * r + r] += lambda * (double)T[r * 6 - r * (r - 1) / 2];
            rhs[r] = -(double)T[21 + r];
        }
        if (!chol_solve6(A, rhs, step)) {
            stop = true;
        } else {
            double sn = 0.0;
            for (int r = 0; r < 6; ++r) sn += step[r] * step[r];
            stop = sqrt(sn) < lm_stop;
        }
    }
    if (stop) {
        *state = 0;
    } else {
        double N[12];
        for (int i = 0; i < 12; ++i) N[i] = H[i];
        se3_left(step, N);
        for (int i = 0; i < 12; ++i) {
            Hn[i] = N[i];
            Pf[i] = (float)N[i];
        }
    }
}

// The same by the 16 lanes q of a half-warp (every lane of the warp calls
// it); mine: the half-warp's hypothesis is still iterating.
__device__ __noinline__ void lm_solve_half(const float *T, double lambda, const double *H, double lm_stop, int q,
                                           bool mine, int *state, double *Hn, float *Pf) {
    double Nq = 0.0;
    const bool stop = lm_step_half(T, lambda, H, lm_stop, q, Nq) || T[28] < 3.f;
    if (!mine) return;
    if (stop) {
        if (q == 0) *state = 0;
    } else if (q < 12) {
        Hn[q] = Nq;
        Pf[q] = (float)Nq;
    }
}

template <int CTAS>
__global__ void __cluster_dims__(CTAS, 1, 1) __launch_bounds__(LMC_THREADS, 2) k_lm_cluster(LmArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = (int)cluster.block_rank();
    const int b = blockIdx.y;
    const int n = a.q.n_cur[b];
    if (!round_active(n, a.p)) return;  // same n in every CTA of the cluster
    const bool cov = a.p.use_cov;
    const int stride = a.p.mpad;
    const LmcLayout L = lmc_layout(stride, cov);
    const int t = threadIdx.x;

    float *s_acc = (float *)smem;
    double(*s_H)[12] = (double(*)[12])(smem + L.H);
    double(*s_Hn)[12] = (double(*)[12])(smem + L.Hn);
    float(*s_Pf)[12] = (float(*)[12])(smem + L.Pf);  // FP32 copy of the pose of the next pass
    double *s_lambda = (double *)(smem + L.lambda);
    float(*s_tot)[LMC_NV] = (float(*)[LMC_NV])(smem + L.tot);
    float(*s_new)[LMC_NV] = (float(*)[LMC_NV])(smem + L.nw);
    float *s_loc = (float *)(smem + L.loc);  // two buffers of [LMC_HMAX][LMC_NV]
    int *s_state = (int *)(smem + L.state);
    int *s_cbuf = (int *)(smem + L.cbuf);
    int *s_act = (int *)(smem + L.act);  // hypotheses of the next pass, increasing
    int *s_nact = s_act + LMC_HMAX;      // and their count
    volatile int *s_abort = (volatile int *)(smem + L.flag);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t bar0 = sbase + L.bar;

    const int NC = a.p.n_cull;
    const size_t row0 = (size_t)b * a.p.max_pix;
    const float4 *g_t0 = a.q.tab0 + row0 * stride;
    const float4 *g_t1 = a.q.tab1 + row0 * stride;
    const float *g_t2 = a.q.tab2 + row0 * stride;
    const float4 *g_xc = a.q.xc + row0;
    const int16_t *g_cnt = a.q.tab_cnt + row0;
    // correspondences: two int16 buffers of [pixel][n] in the frame's slice
    int16_t *corr0 = (int16_t *)(a.q.corr + (size_t)b * NC * a.p.max_pix);
    const size_t cstride = (size_t)NC * a.p.max_pix;
    const int n_tiles = (a.n_pix + LMC_P - 1) / LMC_P;
    const int my_tiles = crank < n_tiles ? (n_tiles - crank + CTAS - 1) / CTAS : 0;
    const float thr2 = (float)(a.p.lm_inlier_thresh * a.p.lm_inlier_thresh);
    // direct passes after the first: at most LMC_DIRECT hypotheses, and the
    // CTA's local pixel indices fit the list entries' 10 bits (the same
    // decision in every CTA of the cluster)
    const bool dir_ok = n <= LMC_DIRECT && (n_tiles + CTAS - 1) / CTAS * LMC_P <= 1024;

    // Lane roles of a pass over the k hypotheses listed in s_act: list entry
    // hs = (t / S) % HB on pixel group g = (t / S) / HB.  With fewer than 16
    // hypotheses a tile has fewer (hypothesis, pixel) pairs than threads: S
    // adjacent lanes then share a pair and split its mode scan (every S-th
    // mode), and the nearest mode is found by a shuffle reduction (ties: lower
    // index, as a sequential scan finds it).  hl: the hypothesis served.
    int HB = 1, S = 1, Gp = 1, sub = 0, hs = 0, g = 0, hl = 0, k_act = 0;
    bool mine = false;
    auto roles = [&](int k, bool direct) {
        k_act = k;
        HB = 1;
        while (HB < k) HB <<= 1;
        const int G = LMC_THREADS / HB;
        S = !direct && G > LMC_P ? G / LMC_P : 1;
        Gp = G / S;  // pixel groups
        sub = t % S;
        hs = (t / S) % HB;
        g = (t / S) / HB;
        mine = hs < k;
        hl = mine ? s_act[hs] : 0;
    };

    for (int i = t; i < n * 12; i += LMC_THREADS) {
        const double v = a.q.cur_pose[((size_t)b * NC + i / 12) * 12 + i % 12];
        s_H[i / 12][i % 12] = v;
        s_Pf[i / 12][i % 12] = (float)v;
    }
    for (int i = t; i < n; i += LMC_THREADS) {
        s_lambda[i] = a.p.lm_lambda0;
        s_state[i] = 1;
        s_act[i] = i;
        s_cbuf[i] = 0;
    }
    if (t == 0) {
        *s_abort = 0;
        for (int s = 0; s < LMC_STAGES; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // thread 0 is the producer: my j-th tile into stage s
    // per stage: copies issued (thread 0), phases consumed, phases seen complete
    uint32_t issued[LMC_STAGES] = {}, waited[LMC_STAGES] = {}, landed[LMC_STAGES] = {};
    auto issue = [&](int j, int s) {
        const uint32_t bar = bar0 + 8 * s;
        const uint32_t st = sbase + s * L.stage;
        const size_t r = (size_t)(crank + j * CTAS) * LMC_P;  // first row of the tile
        const uint32_t rows = (uint32_t)LMC_P * stride;
        mbar_expect_tx(bar, L.tx);
        bulk_g2s(st + L.t0, g_t0 + r * stride, rows * 16, bar);
        if (cov) {
            bulk_g2s(st + L.t1, g_t1 + r * stride, rows * 16, bar);
            bulk_g2s(st + L.t2, g_t2 + r * stride, rows * 4, bar);
        }
        bulk_g2s(st + L.xc, g_xc + r, LMC_P * 16, bar);
        bulk_g2s(st + L.cnt, g_cnt + r, LMC_P * 2, bar);
        ++issued[s];
    };

    unsigned w_pairs = 0, w_modes = 0, w_in = 0, w_trial = 0, w_evals = 0;

    // Nearest-mode anchors.  Each (hypothesis, pixel) pair keeps, from its
    // last full nearest-mode search, the transformed point y there, the
    // nearest mode b and a slack.  d_m(y) = |U_m (y - mu_m)| moves by at
    // most L |dy| when y moves by dy (L >= the largest |U_m|_2 of the pixel's
    // modes; the table holds the largest Frobenius norm), so while
    // |y - y_anchor| <= (d_2 - d_b - margin) / 2L, with d_2 the second-nearest
    // distance at the anchor, b is still the strict nearest mode; the margin
    // covers the FP32 rounding of the four distances involved.  Such a pair
    // reads only b's record.  The other pairs go to a list that LMC_SB lanes
    // per pair search in full (nearest and second-nearest, ties to the lower
    // index), re-anchoring them.  The nearest mode used is therefore always
    // the one a full FP32 search finds.  A pass either streams the CTA's
    // tiles of the mode table into shared memory (many hypotheses share each
    // row) or, for frames with at most LMC_DIRECT hypotheses, reads the rows
    // from global memory (few share a row, and the anchors spare most reads).
    uint16_t *s_list = (uint16_t *)(smem + L.list);           // [LMC_LIST] local pixel << 6 | list entry
    int16_t *s_res = (int16_t *)(smem + L.list) + LMC_LIST;   // [LMC_LIST] nearest mode of the entry
    int *s_nl = (int *)(smem + L.flag) + 1;                   // two list counters, by tile parity
    float4 *g_anc = a.q.lm_anc + (size_t)b * cstride;
    // squared distance (Eq. 5 form) of y to the record m of a row
    auto q_at = [&](const float4 *r0, const float4 *r1, const float *r2, int m, float y0, float y1, float y2) {
        const float4 m0 = r0[m];
        const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
        if (cov) {
            const float4 m1 = r1[m];
            const float w0 = fmaf(m0.w, v0, fmaf(m1.x, v1, m1.y * v2));
            const float w1 = fmaf(m1.z, v1, m1.w * v2);
            const float w2 = r2[m] * v2;
            return fmaf(w0, w0, fmaf(w1, w1, w2 * w2));
        }
        return fmaf(v0, v0, fmaf(v1, v1, v2 * v2));
    };
    // inlier test and normal-equation terms of a pair whose nearest mode is
    // bm, the trial cost of its previous correspondence, its new one
    auto finish = [&](const float4 *r0, const float4 *r1, const float *r2, size_t ci, float y0, float y1,
                      float y2, int bm, bool trial, const int16_t *cr, int16_t *cw, LmcPass &o) {
        const int m_old = trial ? (int)cr[ci] : -1;
        int best_m = bm;
        if (bm >= 0) {
            o.energy += sqrtf(q_at(r0, r1, r2, bm, y0, y1, y2));
            const float4 m0 = r0[bm];
            const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
            if (fmaf(v0, v0, fmaf(v1, v1, v2 * v2)) <= thr2) {
                ++o.nin;
                ++w_in;
                if (cov) {
                    const float4 m1 = r1[bm];
                    lm_accumulate(y0, y1, y2, v0, v1, v2, m0.w, m1.x, m1.y, m1.z, m1.w, r2[bm], o.acc);
                } else {
                    lm_accumulate(y0, y1, y2, v0, v1, v2, 1.f, 0.f, 0.f, 1.f, 0.f, 1.f, o.acc);
                }
            } else {
                best_m = -1;
            }
        }
        if (m_old >= 0) {  // the previous correspondence at the trial pose
            ++w_trial;
            if (cov) {
                o.trial += q_at(r0, r1, r2, m_old, y0, y1, y2);
            } else {
                const float4 m0 = r0[m_old];
                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                o.trial = fmaf(v0, v0, fmaf(v1, v1, fmaf(v2, v2, o.trial)));
            }
        }
        cw[ci] = (int16_t)best_m;  // local mode index in the row, -1: none
    };
    // Running maxima over a row's modes for the anchor's bound: |U|_F^2 and
    // |mu|^2 of record m.
    auto row_maxima = [&](const float4 *r0, const float4 *r1, const float *r2, int m, float &fro2, float &mu2) {
        const float4 m0 = r0[m];
        mu2 = fmaxf(mu2, fmaf(m0.x, m0.x, fmaf(m0.y, m0.y, m0.z * m0.z)));
        if (cov) {
            const float4 m1 = r1[m];
            const float u22 = r2[m];
            fro2 = fmaxf(fro2, fmaf(m0.w, m0.w, fmaf(m1.x, m1.x, fmaf(m1.y, m1.y, fmaf(m1.z, m1.z,
                                                                             fmaf(m1.w, m1.w, u22 * u22))))));
        }
    };
    // Anchor of pair ci from a full search at y: nearest and second-nearest
    // squared distances, the nearest mode, and over the row's modes the
    // largest squared Frobenius norm of U and the largest |mu|^2.
    auto anchor = [&](size_t ci, float y0, float y1, float y2, float best, float second, int best_m, float fro2,
                      float mu2) {
        float slack2 = -1.f;
        if (best_m >= 0) {
            if (!(second < INFINITY)) {
                slack2 = 0.25f;  // a single mode stays the nearest (bounded to 0.5 m)
            } else {
                const float Lf = (cov ? sqrtf(fro2) : 1.f) * 1.00001f;
                const float db = sqrtf(best), d2 = sqrtf(second);
                const float ny = sqrtf(fmaf(y0, y0, fmaf(y1, y1, y2 * y2)));
                const float margin = 4e-6f * (Lf * (ny + 0.5f + sqrtf(mu2)) + d2 + 1.f);
                const float sl = fminf(0.5f, (d2 - db - margin) / (2.f * Lf));
                if (sl > 0.f) slack2 = sl * sl * 0.99999f;
            }
        }
        // the nearest mode rides in the low 8 bits of slack^2, which is first
        // shrunk by 1e-4 relative so that the packed value stays below it
        slack2 = slack2 > 0.f ? slack2 * 0.9999f : -1.f;
        const int packed = (__float_as_int(slack2) & ~0xFF) | (best_m >= 0 ? best_m : 0);
        g_anc[ci] = make_float4(y0, y1, y2, __int_as_float(packed));
    };
    // Full search of one listed pair by the LMC_SB lanes of a group (every
    // lane of the warp calls it; `on` marks a real entry); lane 0 of the
    // group re-anchors the pair.  Returns the nearest mode (-1: none).
    auto search = [&](bool on, const float4 *r0, const float4 *r1, const float *r2, int cnt, int i, size_t ci,
                      float y0, float y1, float y2) {
        const int sub = t % LMC_SB;
        float best = INFINITY, second = INFINITY, fro2 = 0.f, mu2 = 0.f;
        int best_m = -1;
        for (int m = sub; m < cnt; m += LMC_SB) {
            const float qm = q_at(r0, r1, r2, m, y0, y1, y2);
            if (qm < best) {
                second = best;
                best = qm;
                best_m = m;
            } else {
                second = fminf(second, qm);
            }
            row_maxima(r0, r1, r2, m, fro2, mu2);
        }
#pragma unroll
        for (int off = 1; off < LMC_SB; off <<= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, off);
            const float os = __shfl_xor_sync(0xffffffffu, second, off);
            const int om = __shfl_xor_sync(0xffffffffu, best_m, off);
            if (om >= 0 && (best_m < 0 || ob < best || (ob == best && om < best_m))) {
                second = fminf(best, fminf(second, os));
                best = ob;
                best_m = om;
            } else {
                second = fminf(second, fminf(ob, os));
            }
            fro2 = fmaxf(fro2, __shfl_xor_sync(0xffffffffu, fro2, off));
            mu2 = fmaxf(mu2, __shfl_xor_sync(0xffffffffu, mu2, off));
        }
        if (on && sub == 0) {
            w_evals += cnt;
            anchor(ci, y0, y1, y2, best, second, best_m, fro2, mu2);
        }
        return best_m;
    };
    // The certified case of a pair: true (and the pair finished) when its
    // anchor still settles the nearest mode.
    auto anchored = [&](const float4 *r0, const float4 *r1, const float *r2, size_t ci, float y0, float y1, float y2,
                        bool trial, const int16_t *cr, int16_t *cw, LmcPass &o) {
        const float4 an = g_anc[ci];
        const float e0 = y0 - an.x, e1 = y1 - an.y, e2 = y2 - an.z;
        if (!(fmaf(e0, e0, fmaf(e1, e1, e2 * e2)) <= an.w)) return false;
        ++w_evals;
        finish(r0, r1, r2, ci, y0, y1, y2, __float_as_int(an.w) & 0xFF, trial, cr, cw, o);
        return true;
    };

    // One tile of a pass with S > 1: pixel g of the tile for hypothesis hl,
    // modes sub, sub + S, ... on this lane; every lane reaches the shuffles.
    auto split_tile = [&](bool live, int s, int j, bool trial, bool rec, const int16_t *cr, int16_t *cw, LmcPass &o,
                          float r00, float r01, float r02, float tx, float r10, float r11, float r12, float ty,
                          float r20, float r21, float r22, float tz) {
        const uint8_t *st = smem + s * L.stage;
        const float4 *s_t0 = (const float4 *)(st + L.t0);
        const float4 *s_t1 = (const float4 *)(st + L.t1);
        const float *s_t2 = (const float *)(st + L.t2);
        const float4 *s_xc = (const float4 *)(st + L.xc);
        const int16_t *s_cnt = (const int16_t *)(st + L.cnt);
        const int i0 = (crank + j * CTAS) * LMC_P;
        const int il = g;
        const bool on = live && il < min(LMC_P, a.n_pix - i0);
        const int cnt = on ? (int)s_cnt[il] : 0;
        const int base = il * stride;
        float y0 = 0.f, y1 = 0.f, y2 = 0.f;
        if (cnt > 0) {
            const float4 x = s_xc[il];
            y0 = fmaf(r00, x.x, fmaf(r01, x.y, fmaf(r02, x.z, tx)));
            y1 = fmaf(r10, x.x, fmaf(r11, x.y, fmaf(r12, x.z, ty)));
            y2 = fmaf(r20, x.x, fmaf(r21, x.y, fmaf(r22, x.z, tz)));
        }
        float best = INFINITY, second = INFINITY;  // second: for the anchor (direct passes follow)
        float fro2 = 0.f, mu2 = 0.f;
        int best_m = -1;
        if (rec)
            for (int m = sub; m < cnt; m += S) row_maxima(s_t0 + base, s_t1 + base, s_t2 + base, m, fro2, mu2);
        if (cov) {
            auto d2of = [&](int m) {
                const float4 m0 = s_t0[base + m], m1 = s_t1[base + m];
                const float u22 = s_t2[base + m];
                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                const float w0 = fmaf(m0.w, v0, fmaf(m1.x, v1, m1.y * v2));
                const float w1 = fmaf(m1.z, v1, m1.w * v2);
                const float w2 = u22 * v2;
                return fmaf(w0, w0, fmaf(w1, w1, w2 * w2));
            };
            int m = sub;
            for (; m + S < cnt; m += 2 * S) {
                const float da = d2of(m), db = d2of(m + S);
                if (da < best) { second = best; best = da; best_m = m; } else { second = fminf(second, da); }
                if (db < best) { second = best; best = db; best_m = m + S; } else { second = fminf(second, db); }
            }
            if (m < cnt) {
                const float da = d2of(m);
                if (da < best) { second = best; best = da; best_m = m; } else { second = fminf(second, da); }
            }
        } else {
            auto d2of = [&](int m) {
                const float4 m0 = s_t0[base + m];
                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                return fmaf(v0, v0, fmaf(v1, v1, v2 * v2));
            };
            int m = sub;
            for (; m + S < cnt; m += 2 * S) {
                const float da = d2of(m), db = d2of(m + S);
                if (da < best) { second = best; best = da; best_m = m; } else { second = fminf(second, da); }
                if (db < best) { second = best; best = db; best_m = m + S; } else { second = fminf(second, db); }
            }
            if (m < cnt) {
                const float da = d2of(m);
                if (da < best) { second = best; best = da; best_m = m; } else { second = fminf(second, da); }
            }
        }
        for (int off = 1; off < S; off <<= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, off);
            const float os = __shfl_xor_sync(0xffffffffu, second, off);
            const int om = __shfl_xor_sync(0xffffffffu, best_m, off);
            if (om >= 0 && (best_m < 0 || ob < best || (ob == best && om < best_m))) {
                second = fminf(best, fminf(second, os));
                best = ob;
                best_m = om;
            } else {
                second = fminf(second, fminf(ob, os));
            }
            fro2 = fmaxf(fro2, __shfl_xor_sync(0xffffffffu, fro2, off));
            mu2 = fmaxf(mu2, __shfl_xor_sync(0xffffffffu, mu2, off));
        }
        if (sub != 0 || !on) return;
        const size_t ci = (size_t)(i0 + il) * n + hl;
        if (rec && cnt > 0) anchor(ci, y0, y1, y2, best, second, best_m, fro2, mu2);
        const int m_old = trial ? (int)cr[ci] : -1;
        if (cnt > 0) {
            ++w_pairs;
            w_modes += cnt;
            w_evals += cnt;
            o.energy += sqrtf(best);
            if (best_m >= 0) {
                const float4 m0 = s_t0[base + best_m];
                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                if (fmaf(v0, v0, fmaf(v1, v1, v2 * v2)) <= thr2) {
                    ++o.nin;
                    ++w_in;
                    if (cov) {
                        const float4 m1 = s_t1[base + best_m];
                        lm_accumulate(y0, y1, y2, v0, v1, v2, m0.w, m1.x, m1.y, m1.z, m1.w, s_t2[base + best_m],
                                      o.acc);
                    } else {
                        lm_accumulate(y0, y1, y2, v0, v1, v2, 1.f, 0.f, 0.f, 1.f, 0.f, 1.f, o.acc);
                    }
                } else {
                    best_m = -1;
                }
            }
            if (m_old >= 0) {  // the previous correspondence at the trial pose
                ++w_trial;
                const float4 m0 = s_t0[base + m_old];
                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                if (cov) {
                    const float4 m1 = s_t1[base + m_old];
                    const float q0 = fmaf(m0.w, v0, fmaf(m1.x, v1, m1.y * v2));
                    const float q1 = fmaf(m1.z, v1, m1.w * v2);
                    const float q2 = s_t2[base + m_old] * v2;
                    o.trial = fmaf(q0, q0, fmaf(q1, q1, fmaf(q2, q2, o.trial)));
                } else {
                    o.trial = fmaf(v0, v0, fmaf(v1, v1, fmaf(v2, v2, o.trial)));
                }
            }
        } else {
            best_m = -1;
        }
        cw[ci] = (int16_t)best_m;  // local mode index in the row, -1: none
    };
    // The pass; act: this thread's hypothesis takes part, P: its pose;
    // first: the round's first pass.  Frames with at most LMC_DIRECT
    // hypotheses stream their tiles in the first pass, which anchors every
    // pair, and read the table from global memory in the later passes.
    auto pass = [&](bool act, const float *P, bool trial, int rbuf, int wbuf, bool first) {
        LmcPass o;
#pragma unroll
        for (int k = 0; k < 28; ++k) o.acc[k] = 0.f;
        o.nin = 0;
        o.trial = 0.f;
        o.energy = 0.f;
        float r00 = 0.f, r01 = 0.f, r02 = 0.f, tx = 0.f, r10 = 0.f, r11 = 0.f, r12 = 0.f, ty = 0.f;
        float r20 = 0.f, r21 = 0.f, r22 = 0.f, tz = 0.f;
        if (act) {
            r00 = P[0]; r01 = P[1]; r02 = P[2]; tx = P[3];
            r10 = P[4]; r11 = P[5]; r12 = P[6]; ty = P[7];
            r20 = P[8]; r21 = P[9]; r22 = P[10]; tz = P[11];
        }
        const int16_t *cr = corr0 + (size_t)rbuf * cstride;
        int16_t *cw = corr0 + (size_t)wbuf * cstride;
        // region 0 was last written by threads (partials): order those writes
        // before the copies that overwrite it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (t == 0) s_nl[0] = s_nl[1] = 0;
        __syncthreads();
        if (dir_ok && !first) {
            // rows from global memory; chunks of Gp * LMC_KP of the CTA's
            // pixels (local pixel j is pixel j % 16 of tile crank + (j / 16) * CTAS)
            const int n_local = my_tiles * LMC_P;
            const int lane = t & 31;
            auto pixel_of = [&](int j) { return (crank + (j / LMC_P) * CTAS) * LMC_P + j % LMC_P; };
            int c = 0;
            for (int c0 = 0; c0 < n_local; c0 += Gp * LMC_KP, c ^= 1) {
                int pend[LMC_KP];
#pragma unroll
                for (int k = 0; k < LMC_KP; ++k) {
                    pend[k] = -1;
                    bool need = false;
                    const int j = c0 + g + k * Gp;
                    const int i = j < n_local ? pixel_of(j) : a.n_pix;
                    if (act && i < a.n_pix) {
                        const size_t ci = (size_t)i * n + hl;
                        const int cnt = g_cnt[i];
                        if (cnt == 0) {
                            cw[ci] = -1;
                        } else {
                            ++w_pairs;
                            w_modes += cnt;
                            const float4 x = g_xc[i];
                            const float y0 = fmaf(r00, x.x, fmaf(r01, x.y, fmaf(r02, x.z, tx)));
                            const float y1 = fmaf(r10, x.x, fmaf(r11, x.y, fmaf(r12, x.z, ty)));
                            const float y2 = fmaf(r20, x.x, fmaf(r21, x.y, fmaf(r22, x.z, tz)));
                            const size_t rb = (size_t)i * stride;
                            need = !anchored(g_t0 + rb, g_t1 + rb, g_t2 + rb, ci, y0, y1, y2, trial, cr, cw, o);
                        }
                    }
                    // one list append per warp
                    const unsigned mk = __ballot_sync(0xffffffffu, need);
                    int base = 0;
                    if (lane == 0 && mk) base = atomicAdd(&s_nl[c], __popc(mk));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (need) {
                        pend[k] = base + __popc(mk & ((1u << lane) - 1u));
                        s_list[pend[k]] = (uint16_t)((j << 6) | hs);
                    }
                }
                __syncthreads();
                if (t == 0) s_nl[c ^ 1] = 0;
                const int nl = s_nl[c];
                for (int e0 = 0; e0 < nl; e0 += LMC_THREADS / LMC_SB) {
                    const int e = e0 + t / LMC_SB;
                    const bool on = e < nl;
                    int i = 0, cnt = 0, h = 0;
                    float y0 = 0.f, y1 = 0.f, y2 = 0.f;
                    if (on) {
                        const int v = s_list[e];
                        i = pixel_of(v >> 6);
                        h = s_act[v & 63];
                        cnt = g_cnt[i];
                        const float4 x = g_xc[i];
                        const float *Q = s_Pf[h];
                        y0 = fmaf(Q[0], x.x, fmaf(Q[1], x.y, fmaf(Q[2], x.z, Q[3])));
                        y1 = fmaf(Q[4], x.x, fmaf(Q[5], x.y, fmaf(Q[6], x.z, Q[7])));
                        y2 = fmaf(Q[8], x.x, fmaf(Q[9], x.y, fmaf(Q[10], x.z, Q[11])));
                    }
                    const size_t rb = (size_t)i * stride;
                    const int bm = search(on, g_t0 + rb, g_t1 + rb, g_t2 + rb, cnt, i, (size_t)i * n + h, y0, y1, y2);
                    if (on && t % LMC_SB == 0) s_res[e] = (int16_t)bm;
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < LMC_KP; ++k) {
                    if (pend[k] < 0) continue;
                    const int i = pixel_of(c0 + g + k * Gp);
                    const float4 x = g_xc[i];
                    const float y0 = fmaf(r00, x.x, fmaf(r01, x.y, fmaf(r02, x.z, tx)));
                    const float y1 = fmaf(r10, x.x, fmaf(r11, x.y, fmaf(r12, x.z, ty)));
                    const float y2 = fmaf(r20, x.x, fmaf(r21, x.y, fmaf(r22, x.z, tz)));
                    const size_t rb = (size_t)i * stride;
                    finish(g_t0 + rb, g_t1 + rb, g_t2 + rb, (size_t)i * n + hl, y0, y1, y2, (int)s_res[pend[k]],
                           trial, cr, cw, o);
                }
                __syncthreads();  // the list is rewritten two chunks later
            }
            return o;
        }
        const bool rec = dir_ok && first;  // anchor every pair for the direct passes that follow
        if (t == 0 && !*s_abort)
            for (int j = 0; j < LMC_STAGES && j < my_tiles; ++j) issue(j, j);
        for (int j = 0; j < my_tiles; ++j) {
            const int s = j % LMC_STAGES;
            const uint32_t parity = waited[s] & 1u;
            ++waited[s];
            if (!*s_abort) {
                if (mbar_wait_bounded(bar0 + 8 * s, parity, a.wait_limit)) {
                    ++landed[s];
                } else {
                    *s_abort = 1;
                    a.q.dev_err[b] = 1;
                }
            }
            if (S > 1) {
                split_tile(act && !*s_abort, s, j, trial, rec, cr, cw, o, r00, r01, r02, tx, r10, r11, r12, ty, r20,
                           r21, r22, tz);
            } else if (act && !*s_abort) {
                // one lane per pair: at least 16 hypotheses, so never a frame
                // whose pairs need anchors (rec implies S > 1)
                const uint8_t *st = smem + s * L.stage;
                const float4 *s_t0 = (const float4 *)(st + L.t0);
                const float4 *s_t1 = (const float4 *)(st + L.t1);
                const float *s_t2 = (const float *)(st + L.t2);
                const float4 *s_xc = (const float4 *)(st + L.xc);
                const int16_t *s_cnt = (const int16_t *)(st + L.cnt);
                const int i0 = (crank + j * CTAS) * LMC_P;
                const int np = min(LMC_P, a.n_pix - i0);
                for (int il = g; il < np; il += Gp) {
                    const size_t ci = (size_t)(i0 + il) * n + hl;
                    const int m_old = trial ? (int)cr[ci] : -1;
                    const int cnt = s_cnt[il];
                    int best_m = -1;
                    if (cnt > 0) {
                        ++w_pairs;
                        w_modes += cnt;
                        w_evals += cnt;
                        const float4 x = s_xc[il];
                        const float y0 = fmaf(r00, x.x, fmaf(r01, x.y, fmaf(r02, x.z, tx)));
                        const float y1 = fmaf(r10, x.x, fmaf(r11, x.y, fmaf(r12, x.z, ty)));
                        const float y2 = fmaf(r20, x.x, fmaf(r21, x.y, fmaf(r22, x.z, tz)));
                        const int base = il * stride;
                        float best = INFINITY;
                        // two modes per step (independent chains), compared in mode order
                        if (cov) {
                            auto d2of = [&](int m) {
                                const float4 m0 = s_t0[base + m], m1 = s_t1[base + m];
                                const float u22 = s_t2[base + m];
                                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                                const float w0 = fmaf(m0.w, v0, fmaf(m1.x, v1, m1.y * v2));
                                const float w1 = fmaf(m1.z, v1, m1.w * v2);
                                const float w2 = u22 * v2;
                                return fmaf(w0, w0, fmaf(w1, w1, w2 * w2));
                            };
                            int m = 0;
                            for (; m + 1 < cnt; m += 2) {
                                const float da = d2of(m), db = d2of(m + 1);
                                if (da < best) { best = da; best_m = m; }
                                if (db < best) { best = db; best_m = m + 1; }
                            }
                            if (m < cnt) {
                                const float da = d2of(m);
                                if (da < best) { best = da; best_m = m; }
                            }
                        } else {
                            auto d2of = [&](int m) {
                                const float4 m0 = s_t0[base + m];
                                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                                return fmaf(v0, v0, fmaf(v1, v1, v2 * v2));
                            };
                            int m = 0;
                            for (; m + 1 < cnt; m += 2) {
                                const float da = d2of(m), db = d2of(m + 1);
                                if (da < best) { best = da; best_m = m; }
                                if (db < best) { best = db; best_m = m + 1; }
                            }
                            if (m < cnt) {
                                const float da = d2of(m);
                                if (da < best) { best = da; best_m = m; }
                            }
                        }
                        o.energy += sqrtf(best);
                        if (best_m >= 0) {
                            const float4 m0 = s_t0[base + best_m];
                            const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                            if (fmaf(v0, v0, fmaf(v1, v1, v2 * v2)) <= thr2) {
                                ++o.nin;
                                ++w_in;
                                if (cov) {
                                    const float4 m1 = s_t1[base + best_m];
                                    lm_accumulate(y0, y1, y2, v0, v1, v2, m0.w, m1.x, m1.y, m1.z, m1.w,
                                                  s_t2[base + best_m], o.acc);
                                } else {
                                    lm_accumulate(y0, y1, y2, v0, v1, v2, 1.f, 0.f, 0.f, 1.f, 0.f, 1.f, o.acc);
                                }
                            } else {
                                best_m = -1;
                            }
                        }
                        if (m_old >= 0) {  // the previous correspondence at the trial pose
                            ++w_trial;
                            const float4 m0 = s_t0[base + m_old];
                            const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                            if (cov) {
                                const float4 m1 = s_t1[base + m_old];
                                const float q0 = fmaf(m0.w, v0, fmaf(m1.x, v1, m1.y * v2));
                                const float q1 = fmaf(m1.z, v1, m1.w * v2);
                                const float q2 = s_t2[base + m_old] * v2;
                                o.trial = fmaf(q0, q0, fmaf(q1, q1, fmaf(q2, q2, o.trial)));
                            } else {
                                o.trial = fmaf(v0, v0, fmaf(v1, v1, fmaf(v2, v2, o.trial)));
                            }
                        }
                    }
                    cw[ci] = (int16_t)best_m;  // local mode index in the row, -1: none
                }
            }
            __syncthreads();  // stage s consumed by every thread
            if (t == 0 && !*s_abort && j + LMC_STAGES < my_tiles) issue(j + LMC_STAGES, s);
        }
        return o;
    };
    // Sums of this CTA's pass over groups (fixed order) into loc buffer lb,
    // then over the cluster's CTAs (rank order) into dst.
    auto reduce = [&](const LmcPass &o, int lb, float (*dst)[LMC_NV]) {
        float *mypart = s_acc + t * LMC_PS;
#pragma unroll
        for (int k = 0; k < 28; ++k) mypart[k] = o.acc[k];
        mypart[28] = (float)o.nin;
        mypart[29] = o.trial;
        mypart[30] = o.energy;
        __syncthreads();
        float *loc = s_loc + lb * (LMC_HMAX * LMC_NV);
        for (int e = t; e < k_act * LMC_NV; e += LMC_THREADS) {
            const int j = e / LMC_NV, k = e % LMC_NV;
            float v = 0.f;
            // the lanes holding list entry j's partials, in group order
            for (int gg = 0; gg < Gp; ++gg) v += s_acc[(S * (gg * HB + j)) * LMC_PS + k];
            loc[s_act[j] * LMC_NV + k] = v;
        }
        // Double-buffered loc: a CTA rewrites buffer lb two reductions later,
        // after the next barrier, which every CTA reaches only after reading
        // buffer lb here; one barrier per reduction suffices.
        cluster.sync();
        for (int e = t; e < k_act * LMC_NV; e += LMC_THREADS) {
            const int h = s_act[e / LMC_NV], k = e % LMC_NV;
            float v = 0.f;
            for (int r = 0; r < CTAS; ++r) v += cluster.map_shared_rank(loc, r)[h * LMC_NV + k];
            dst[h][k] = v;
        }
        __syncthreads();
    };

    // normal equations and correspondences at the initial poses
    {
        roles(n, false);
        const LmcPass o = pass(mine, s_Pf[hl], false, 0, 0, true);
        reduce(o, 0, s_tot);
    }
    for (int it = 0; it < a.p.lm_max_iter; ++it) {
        // damped FP64 solve.  Each SM sub-partition has its own narrow FP64
        // pipe, which a warp instruction holds for the same time whatever its
        // active lanes.  Up to LMC_COOP hypotheses: one per half-warp, its
        // solve spread over the 16 lanes (at most two warps per
        // sub-partition).  More: hypothesis h on lane h / 4 of warp h % 4,
        // one warp on each sub-partition.
        if (n <= LMC_COOP) {
            const int h = t >> 4;
            const bool mine = h < n && s_state[h];
            if (__any_sync(0xffffffffu, mine))  // both half-warps take part in the shuffles
                lm_solve_half(s_tot[h], s_lambda[h], s_H[h], a.p.lm_stop, t & 15, mine, s_state + h, s_Hn[h], s_Pf[h]);
        } else {
            const int h = (t & 31) * 4 + (t >> 5);
            if (t < 128 && (t & 31) < LMC_HMAX / 4 && h < n && s_state[h])
                lm_solve_lane(s_tot[h], s_lambda[h], s_H[h], a.p.lm_stop, s_state + h, s_Hn[h], s_Pf[h]);
        }
        // The stop flags were just written by the solving threads: the
        // predicate below is evaluated before its barrier, so it must see them
        // through one of its own.  Every CTA then takes the same exit decision
        // and the cluster barriers stay paired (a CTA that left the loop alone
        // would be read through distributed shared memory after it exits).
        __syncthreads();
        if (!__syncthreads_or(t < n && s_state[t])) break;  // identical in every CTA
        // list the hypotheses still iterating (the same list in every CTA)
        if (t < 32) {
            const bool on0 = t < n && s_state[t], on1 = t + 32 < n && s_state[t + 32];
            const unsigned m0 = __ballot_sync(0xffffffffu, on0), m1 = __ballot_sync(0xffffffffu, on1);
            const unsigned below = (1u << t) - 1u;
            if (on0) s_act[__popc(m0 & below)] = t;
            if (on1) s_act[__popc(m0) + __popc(m1 & below)] = t + 32;
            if (t == 0) *s_nact = __popc(m0) + __popc(m1);
        }
        __syncthreads();
        roles(*s_nact, dir_ok);
        // trial cost of the step on the current correspondences, and the
        // normal equations at the trial pose (used if the step is accepted)
        const int ob = mine ? s_cbuf[hl] : 0;
        const LmcPass o = pass(mine, s_Pf[hl], true, ob, ob ^ 1, false);
        reduce(o, (it + 1) & 1, s_new);
        for (int h = t; h < n; h += LMC_THREADS) {
            if (!s_state[h]) continue;
            if (s_new[h][29] < s_tot[h][27]) {
                for (int i = 0; i < 12; ++i) s_H[h][i] = s_Hn[h][i];
                for (int k = 0; k < 29; ++k) s_tot[h][k] = s_new[h][k];
                s_tot[h][30] = s_new[h][30];  // the energy at the accepted pose
                s_cbuf[h] ^= 1;
                s_lambda[h] /= 10.0;
            } else {
                s_lambda[h] *= 10.0;
            }
        }
        __syncthreads();
    }
    __syncthreads();  // the last accept/reject updates of s_H before other threads write them out
    if (crank == 0) {
        for (int i = t; i < n * 12; i += LMC_THREADS)
            a.q.cur_pose[((size_t)b * NC + i / 12) * 12 + i % 12] = s_H[i / 12][i % 12];
        // Eq. 5 over the round's pixel set at each refined pose, from the pass
        // that evaluated that pose: the round needs no separate energy launch
        for (int h = t; h < n; h += LMC_THREADS) a.q.cur_energy[(size_t)b * NC + h] = s_tot[h][30];
    }
    if (a.work && (w_pairs | w_modes | w_in | w_trial | w_evals)) {
        atomicAdd(&a.work[W_LM_PAIRS], (unsigned long long)w_pairs);
        atomicAdd(&a.work[W_LM_MODES], (unsigned long long)w_modes);
        atomicAdd(&a.work[W_LM_INLIERS], (unsigned long long)w_in);
        atomicAdd(&a.work[W_LM_TRIAL], (unsigned long long)w_trial);
        atomicAdd(&a.work[W_LM_EVALS], (unsigned long long)w_evals);
    }
    if (t == 0 && *s_abort)  // copies still in flight must land before the CTA exits
        for (int s = 0; s < LMC_STAGES; ++s)
            while (landed[s] < issued[s] && mbar_wait_bounded(bar0 + 8 * s, landed[s] & 1u)) ++landed[s];
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

size_t lm_cluster_smem(int mpad, bool cov) { return lmc_layout(mpad, cov).total; }

rl_status launch_lm_cluster(const LmArgs &a, int n, cudaStream_t s) {
    const size_t sm = lm_cluster_smem(a.p.mpad, a.p.use_cov);
    const bool first = a.n_pix <= 2 * a.p.eta;  // round r refines on eta * (r + 2) pixels
    if (first) {
        k_lm_cluster<LMC_CTAS_FIRST><<<dim3(LMC_CTAS_FIRST, n), LMC_THREADS, sm, s>>>(a);
    } else {
        k_lm_cluster<LMC_CTAS_LATER><<<dim3(LMC_CTAS_LATER, n), LMC_THREADS, sm, s>>>(a);
    }
    RL_LAUNCH_CK();
    return RL_OK;
}

rl_status prepare_lm_cluster() {
    RL_CK(cudaFuncSetAttribute(k_lm_cluster<LMC_CTAS_FIRST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kLmClusterSmemMax));
    RL_CK(cudaFuncSetAttribute(k_lm_cluster<LMC_CTAS_LATER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kLmClusterSmemMax));
    if (LMC_CTAS_LATER > 8)  // clusters above 8 CTAs are not portable and must be allowed explicitly
        RL_CK(cudaFuncSetAttribute(k_lm_cluster<LMC_CTAS_LATER>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return RL_OK;
}

}  // namespace rl
