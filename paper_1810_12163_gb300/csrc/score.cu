// Scoring kernels of the relocaliser: the energy of Eq. 5 on growing pixel
// sets, cull / halving selection, Levenberg-Marquardt refinement in se(3)
// (Sec. 3.2.3) and model-based ranking by depth raycast (Eq. 6-8).
//
// FP32 arithmetic with fused multiply-adds; FP64 only for poses, the 6x6
// normal-equation solve and the SE(3) update.  Every reduction has a fixed
// shape, so results do not depend on how many frames share a launch.
#include <math.h>

#include "internal.h"
#include "relocgb_dev.cuh"
#include "kernels.h"
#include "lm_dev.cuh"

namespace rl {

// ---------------------------------------------------------------------------
// Eq. 5 partial energies.  Block = HT hypotheses of one frame (one per
// thread) x one chunk of the pixel set; the chunk's pixels and their modes
// (decoded to FP32) are staged in shared memory and read by broadcast.
// ---------------------------------------------------------------------------

// Partial energy with S lanes per hypothesis (S a power of two <= 32): lane
// t serves hypothesis h0 + t / S and scans modes t % S, t % S + S, ...  Every
// lane runs every pixel, so the shuffles see the whole warp.
__device__ __noinline__ void energy_split(const EnergyArgs &a, int b, int h0, int nb, int S, int np,
                                          const float4 *s_xc, const float4 *s_m0, const float4 *s_m1,
                                          const float *s_m2, const int *s_cnt) {
    const int hl = threadIdx.x / S, sub = threadIdx.x % S;
    const bool act = hl < nb;
    float r00 = 0.f, r01 = 0.f, r02 = 0.f, t0 = 0.f, r10 = 0.f, r11 = 0.f, r12 = 0.f, t1 = 0.f;
    float r20 = 0.f, r21 = 0.f, r22 = 0.f, t2 = 0.f;
    if (act) {
        const int h = h0 + hl;
        const int id = a.idx ? a.idx[(size_t)b * a.idx_stride + h] : h;
        const double *P = a.pose + ((size_t)b * a.pose_stride + id) * 12;
        r00 = (float)P[0]; r01 = (float)P[1]; r02 = (float)P[2]; t0 = (float)P[3];
        r10 = (float)P[4]; r11 = (float)P[5]; r12 = (float)P[6]; t1 = (float)P[7];
        r20 = (float)P[8]; r21 = (float)P[9]; r22 = (float)P[10]; t2 = (float)P[11];
    }
    float acc = 0.f;
    for (int i = 0; i < np; ++i) {
        const int cnt = s_cnt[i];
        if (cnt == 0) continue;  // the same for every lane
        const float4 x = s_xc[i];
        const float y0 = fmaf(r00, x.x, fmaf(r01, x.y, fmaf(r02, x.z, t0)));
        const float y1 = fmaf(r10, x.x, fmaf(r11, x.y, fmaf(r12, x.z, t1)));
        const float y2 = fmaf(r20, x.x, fmaf(r21, x.y, fmaf(r22, x.z, t2)));
        const int base = i * a.maxm;
        float best = INFINITY;
        if (a.p.use_cov) {
            for (int m = sub; m < cnt; m += S) {
                const float4 m0 = s_m0[base + m], m1 = s_m1[base + m];
                const float u22 = s_m2[base + m];
                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                const float w0 = fmaf(m0.w, v0, fmaf(m1.x, v1, m1.y * v2));
                const float w1 = fmaf(m1.z, v1, m1.w * v2);
                const float w2 = u22 * v2;
                best = fminf(best, fmaf(w0, w0, fmaf(w1, w1, w2 * w2)));
            }
        } else {
            for (int m = sub; m < cnt; m += S) {
                const float4 m0 = s_m0[base + m];
                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                best = fminf(best, fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
            }
        }
        for (int off = 1; off < S; off <<= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, off));
        acc += sqrtf(best);
    }
    if (act && sub == 0) a.part[((size_t)b * a.part_h + h0 + hl) * a.n_chunks + blockIdx.y] = acc;
}

__global__ void __launch_bounds__(256) k_energy(EnergyArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    float4 *s_xc = (float4 *)smem;                         // [chunk]
    float4 *s_m0 = s_xc + a.chunk;                         // [chunk*maxm] mu.xyz, U00
    float4 *s_m1 = s_m0 + a.chunk * a.maxm;                // [chunk*maxm] U01 U02 U11 U12
    float *s_m2 = (float *)(s_m1 + a.chunk * a.maxm);      // [chunk*maxm] U22
    int *s_cnt = (int *)(s_m2 + a.chunk * a.maxm);         // [chunk]

    const int b = blockIdx.z;
    const int n = a.count[b];
    if (a.round_gate && !round_active(n, a.p)) return;
    const int h0 = blockIdx.x * blockDim.x;
    if (h0 >= n) return;
    const int p0 = blockIdx.y * a.chunk;
    if (p0 >= a.n_pix) return;
    const int np = min(a.chunk, a.n_pix - p0);
    const float4 *xc = a.xc + (size_t)b * a.max_pix + p0;
    const size_t row0 = (size_t)b * a.max_pix + p0;   // first table row of the chunk
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        s_xc[i] = xc[i];
        s_cnt[i] = a.q_tab_cnt[row0 + i];
    }
    // the chunk's rows of the mode table are contiguous: coalesced copy
    const int mpad = a.p.mpad;
    const float4 *tb0 = a.q_tab0 + row0 * mpad;
    const float4 *tb1 = a.q_tab1 + row0 * mpad;
    const float *tb2 = a.q_tab2 + row0 * mpad;
    for (int e = threadIdx.x; e < np * mpad; e += blockDim.x) {
        s_m0[e] = tb0[e];
        if (a.p.use_cov) {
            s_m1[e] = tb1[e];
            s_m2[e] = tb2[e];
        }
    }
    __syncthreads();
    if (a.work && threadIdx.x == 0) {
        unsigned long long pairs = 0, modes = 0;
        for (int i = 0; i < np; ++i)
            if (s_cnt[i] > 0) {
                ++pairs;
                modes += (unsigned long long)s_cnt[i];
            }
        const unsigned long long nh = (unsigned long long)min((int)blockDim.x, n - h0);
        atomicAdd(&a.work[W_E_PAIRS], nh * pairs);
        atomicAdd(&a.work[W_E_MODES], nh * modes);
    }
    // With fewer hypotheses than threads, S adjacent lanes share one and
    // split each pixel's mode scan (every S-th mode); the minimum is exact in
    // any order, so the partial energy is the same as with one lane.
    const int nb = min((int)blockDim.x, n - h0);
    int hb = 1;
    while (hb < nb) hb <<= 1;
    const int S = min(32, (int)blockDim.x / hb);
    if (S > 1) {
        energy_split(a, b, h0, nb, S, np, s_xc, s_m0, s_m1, s_m2, s_cnt);
        return;
    }
    const int h = h0 + threadIdx.x;
    if (h >= n) return;
    const int id = a.idx ? a.idx[(size_t)b * a.idx_stride + h] : h;
    const double *P = a.pose + ((size_t)b * a.pose_stride + id) * 12;
    const float r00 = (float)P[0], r01 = (float)P[1], r02 = (float)P[2], t0 = (float)P[3];
    const float r10 = (float)P[4], r11 = (float)P[5], r12 = (float)P[6], t1 = (float)P[7];
    const float r20 = (float)P[8], r21 = (float)P[9], r22 = (float)P[10], t2 = (float)P[11];
    float acc = 0.f;
    for (int i = 0; i < np; ++i) {
        const int cnt = s_cnt[i];
        if (cnt == 0) continue;
        const float4 x = s_xc[i];
        const float y0 = fmaf(r00, x.x, fmaf(r01, x.y, fmaf(r02, x.z, t0)));
        const float y1 = fmaf(r10, x.x, fmaf(r11, x.y, fmaf(r12, x.z, t1)));
        const float y2 = fmaf(r20, x.x, fmaf(r21, x.y, fmaf(r22, x.z, t2)));
        const int base = i * a.maxm;
        float best = INFINITY;
        if (a.p.use_cov) {
            for (int m = 0; m < cnt; ++m) {
                const float4 m0 = s_m0[base + m], m1 = s_m1[base + m];
                const float u22 = s_m2[base + m];
                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                const float w0 = fmaf(m0.w, v0, fmaf(m1.x, v1, m1.y * v2));
                const float w1 = fmaf(m1.z, v1, m1.w * v2);
                const float w2 = u22 * v2;
                best = fminf(best, fmaf(w0, w0, fmaf(w1, w1, w2 * w2)));
            }
        } else {
            for (int m = 0; m < cnt; ++m) {
                const float4 m0 = s_m0[base + m];
                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                best = fminf(best, fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
            }
        }
        acc += sqrtf(best);
    }
    a.part[((size_t)b * a.part_h + h) * a.n_chunks + blockIdx.y] = acc;
}

// ---------------------------------------------------------------------------
// Cull (phase 0) and halving rounds (phase 1): sum the partial energies in
// chunk order, rank by (E, slot), keep the best min(n, N_cull) or ceil(n/2).
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(1024) k_select(SelectArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    float *sE = (float *)smem;                       // [n]
    int *sS = (int *)(sE + a.p.n_hyp);               // [n]
    double *sP = (double *)(sS + a.p.n_hyp);         // [n_cull][12]
    float *sKE = (float *)(sP + a.p.n_cull * 12);    // [n_cull]
    int *sKS = (int *)(sKE + a.p.n_cull);            // [n_cull]
    const int b = blockIdx.x, tid = threadIdx.x;
    const int n = a.count[b];
    if (a.phase == 1 && !round_active(n, a.p)) return;
    const int N = a.p.n_hyp, NC = a.p.n_cull;
    for (int i = tid; i < n; i += blockDim.x) {
        float e = 0.f;
        if (a.phase == 1 && a.energy_from_lm) {
            e = a.q.cur_energy[(size_t)b * NC + i];
        } else {
            const float *pp = a.part + ((size_t)b * a.part_h + i) * a.n_chunks;
            for (int c = 0; c < a.n_chunks_used; ++c) e += pp[c];
        }
        if (isnan(e)) e = INFINITY;
        sE[i] = e;
        sS[i] = a.phase == 0 ? a.hyp_list[(size_t)b * N + i] : a.q.cur_slot[(size_t)b * NC + i];
    }
    __syncthreads();
    const int keep = a.phase == 0 ? min(n, NC) : (n + 1) / 2;
    for (int i = tid; i < n; i += blockDim.x) {
        const float e = sE[i];
        const int s = sS[i];
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            const float f = sE[j];
            rank += (f < e) || (f == e && sS[j] < s);
        }
        if (rank < keep) {
            const double *src = a.phase == 0 ? a.hyp_pose + ((size_t)b * N + s) * 12
                                             : a.q.cur_pose + ((size_t)b * NC + i) * 12;
            for (int k = 0; k < 12; ++k) sP[rank * 12 + k] = src[k];
            sKE[rank] = e;
            sKS[rank] = s;
        }
    }
    __syncthreads();
    for (int i = tid; i < keep; i += blockDim.x) {
        for (int k = 0; k < 12; ++k) a.q.cur_pose[((size_t)b * NC + i) * 12 + k] = sP[i * 12 + k];
        a.q.cur_energy[(size_t)b * NC + i] = sKE[i];
        a.q.cur_slot[(size_t)b * NC + i] = sKS[i];
    }
    if (a.phase == 0)
        for (int i = tid; i < keep; i += blockDim.x) {
            a.q.cull_slot[(size_t)b * NC + i] = sKS[i];
            a.q.cull_energy[(size_t)b * NC + i] = sKE[i];
        }
    const bool take = a.q.n_chosen[b] < 0 && keep <= a.p.k_out;
    if (take)
        for (int i = tid; i < keep; i += blockDim.x) {
            for (int k = 0; k < 12; ++k)
                a.q.chosen_pose[((size_t)b * 16 + i) * 12 + k] = sP[i * 12 + k];
            a.q.chosen_energy[(size_t)b * 16 + i] = sKE[i];
            a.q.chosen_slot[(size_t)b * 16 + i] = sKS[i];
        }
    if (a.phase == 1 && a.round < 16)
        for (int i = tid; i < keep; i += blockDim.x) {
            const size_t o = ((size_t)b * 16 + a.round) * NC + i;
            a.q.round_slot[o] = sKS[i];
            a.q.round_energy[o] = sKE[i];
            for (int k = 0; k < 12; ++k) a.q.round_pose[o * 12 + k] = sP[i * 12 + k];
        }
    __syncthreads();
    if (tid == 0) {
        a.q.n_cur[b] = keep;
        a.q.n_pix[b] = a.n_pix;
        if (take) {
            a.q.n_chosen[b] = keep;
            a.q.chosen_npix[b] = a.n_pix;
        }
        if (a.phase == 1) {
            if (a.round < 16) a.q.round_count[(size_t)b * 16 + a.round] = keep;
            a.q.n_rounds[b] = a.round + 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Levenberg-Marquardt in se(3) (Sec. 3.2.3) for rows of the mode table too
// long for the cluster kernel's staged tiles (lm.cu).
// ---------------------------------------------------------------------------

// LM, hypotheses spread over threads.  A round's n hypotheses of a frame are
// split over up to LM3_BPQ blocks; inside a block, thread t works for
// hypothesis h = t % HB on the pixels g, g + G, ... (g = t / HB, G = 256/HB,
// HB = the next power of two >= the block's hypothesis count).  As rounds
// halve n, each hypothesis gets more threads.  Partial normal equations are
// tree-reduced over the G groups in shared memory (fixed shape), the 6x6
// system of each hypothesis is solved in FP64 by one thread, and the trial
// cost with the same correspondences is reduced the same way.
constexpr int LM3_THREADS = 256;
constexpr int LM3_BPQ = 4;

__global__ void __launch_bounds__(LM3_THREADS, 2) k_lm_spread(LmArgs a) {
    __shared__ float s_red[LM3_THREADS * 8];         // 8 partial values per thread per pass
    __shared__ double s_H[64][12];                    // current pose per local hypothesis
    __shared__ double s_Hn[64][12];                   // trial pose
    __shared__ double s_lambda[64];
    __shared__ float s_tot[64][28];
    __shared__ int s_state[64];                       // 1 active, 0 stopped
    __shared__ int s_nin[64];
    const int b = blockIdx.y;
    const int n = a.q.n_cur[b];
    if (!round_active(n, a.p)) return;
    // hypotheses of this block: [h0, h0 + nb)
    const int per = (n + LM3_BPQ - 1) / LM3_BPQ;
    const int h0 = blockIdx.x * per;
    const int nb = min(per, n - h0);
    if (nb <= 0) return;
    int HB = 1;
    while (HB < nb) HB <<= 1;
    const int G = LM3_THREADS / HB;
    const int t = threadIdx.x;
    const int hl = t % HB, g = t / HB;
    const bool mine = hl < nb;
    const int NC = a.p.n_cull;
    const size_t row0 = (size_t)b * a.p.max_pix;
    const int stride = a.p.mpad;
    const float4 *xcs = a.q.xc + row0;
    const float4 *t0 = a.q.tab0 + row0 * stride;
    const float4 *t1 = a.q.tab1 + row0 * stride;
    const float *t2 = a.q.tab2 + row0 * stride;
    const int16_t *tcnt = a.q.tab_cnt + row0;
    // correspondences [pixel][nb] of this block's hypotheses (local mode index, -1 none)
    int32_t *corr = a.q.corr + ((size_t)b * NC + h0) * a.p.max_pix;
    const float thr2 = (float)(a.p.lm_inlier_thresh * a.p.lm_inlier_thresh);
    const bool cov = a.p.use_cov;
    for (int i = t; i < nb * 12; i += LM3_THREADS) s_H[i / 12][i % 12] = a.q.cur_pose[((size_t)b * NC + h0 + i / 12) * 12 + i % 12];
    for (int i = t; i < nb; i += LM3_THREADS) {
        s_lambda[i] = a.p.lm_lambda0;
        s_state[i] = 1;
    }
    __syncthreads();
    unsigned w_pairs = 0, w_modes = 0, w_in = 0, w_trial = 0;
    for (int it = 0; it < a.p.lm_max_iter; ++it) {
        const bool act = mine && s_state[hl];
        if (!__syncthreads_or(act)) break;
        float acc[28];
#pragma unroll
        for (int k = 0; k < 28; ++k) acc[k] = 0.f;
        int nin = 0;
        if (act) {
            const float r00 = (float)s_H[hl][0], r01 = (float)s_H[hl][1], r02 = (float)s_H[hl][2], tx = (float)s_H[hl][3];
            const float r10 = (float)s_H[hl][4], r11 = (float)s_H[hl][5], r12 = (float)s_H[hl][6], ty = (float)s_H[hl][7];
            const float r20 = (float)s_H[hl][8], r21 = (float)s_H[hl][9], r22 = (float)s_H[hl][10], tz = (float)s_H[hl][11];
            for (int i = g; i < a.n_pix; i += G) {
                const int cnt = tcnt[i];
                int best_m = -1;
                if (cnt > 0) {
                    ++w_pairs;
                    w_modes += cnt;
                    const float4 x = xcs[i];
                    const float y0 = fmaf(r00, x.x, fmaf(r01, x.y, fmaf(r02, x.z, tx)));
                    const float y1 = fmaf(r10, x.x, fmaf(r11, x.y, fmaf(r12, x.z, ty)));
                    const float y2 = fmaf(r20, x.x, fmaf(r21, x.y, fmaf(r22, x.z, tz)));
                    const size_t base = (size_t)i * stride;
                    float best = INFINITY;
                    if (cov) {
                        for (int m = 0; m < cnt; ++m) {
                            const float4 m0 = __ldg(&t0[base + m]), m1 = __ldg(&t1[base + m]);
                            const float u22 = __ldg(&t2[base + m]);
                            const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                            const float w0 = fmaf(m0.w, v0, fmaf(m1.x, v1, m1.y * v2));
                            const float w1 = fmaf(m1.z, v1, m1.w * v2);
                            const float w2 = u22 * v2;
                            const float d2 = fmaf(w0, w0, fmaf(w1, w1, w2 * w2));
                            if (d2 < best) {
                                best = d2;
                                best_m = m;
                            }
                        }
                    } else {
                        for (int m = 0; m < cnt; ++m) {
                            const float4 m0 = __ldg(&t0[base + m]);
                            const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                            const float d2 = fmaf(v0, v0, fmaf(v1, v1, v2 * v2));
                            if (d2 < best) {
                                best = d2;
                                best_m = m;
                            }
                        }
                    }
                    if (best_m >= 0) {
                        const float4 m0 = __ldg(&t0[base + best_m]);
                        const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                        if (fmaf(v0, v0, fmaf(v1, v1, v2 * v2)) <= thr2) {
                            ++nin;
                            ++w_in;
                            if (cov) {
                                const float4 m1 = __ldg(&t1[base + best_m]);
                                lm_accumulate(y0, y1, y2, v0, v1, v2, m0.w, m1.x, m1.y, m1.z, m1.w,
                                               __ldg(&t2[base + best_m]), acc);
                            } else {
                                lm_accumulate(y0, y1, y2, v0, v1, v2, 1.f, 0.f, 0.f, 1.f, 0.f, 1.f, acc);
                            }
                        } else {
                            best_m = -1;
                        }
                    }
                }
                corr[(size_t)i * nb + hl] = best_m;
            }
        }
        // tree reduction of the 28 sums and the inlier count over the groups
        for (int part = 0; part < 4; ++part) {
            for (int k = 0; k < 7; ++k) s_red[t * 8 + k] = acc[part * 7 + k];
            if (part == 0) s_red[t * 8 + 7] = __int_as_float(nin);
            __syncthreads();
            for (int s = G >> 1; s > 0; s >>= 1) {
                if (g < s)
                    for (int k = 0; k < 8; ++k) {
                        if (k == 7 && part != 0) continue;
                        const int o1 = t * 8 + k, o2 = (t + s * HB) * 8 + k;
                        if (k == 7)
                            s_red[o1] = __int_as_float(__float_as_int(s_red[o1]) + __float_as_int(s_red[o2]));
                        else
                            s_red[o1] += s_red[o2];
                    }
                __syncthreads();
            }
            if (g == 0 && mine) {
                for (int k = 0; k < 7; ++k) s_tot[hl][part * 7 + k] = s_red[t * 8 + k];
                if (part == 0) s_nin[hl] = __float_as_int(s_red[t * 8 + 7]);
            }
            __syncthreads();
        }
        // FP64 solve per active hypothesis
        if (g == 0 && act) {
            int status = s_nin[hl] < 3 ? 1 : 0;
            double step[6];
            if (!status) {
                double A[36], rhs[6];
                int k = 0;
                for (int r = 0; r < 6; ++r)
                    for (int c = r; c < 6; ++c, ++k) A[6 * r + c] = A[6 * c + r] = (double)s_tot[hl][k];
                for (int r = 0; r < 6; ++r) {
                    A[6 * r + r] += s_lambda[hl] * (double)s_tot[hl][r * 6 - r * (r - 1) / 2];
                    rhs[r] = -(double)s_tot[hl][21 + r];
                }
                if (!chol_solve6(A, rhs, step)) {
                    status = 1;
                } else {
                    double sn = 0.0;
                    for (int r = 0; r < 6; ++r) sn += step[r] * step[r];
                    if (sqrt(sn) < a.p.lm_stop) status = 1;
                }
            }
            if (status) {
                s_state[hl] = 0;
            } else {
                double Hn[12];
                for (int i = 0; i < 12; ++i) Hn[i] = s_H[hl][i];
                se3_left(step, Hn);
                for (int i = 0; i < 12; ++i) s_Hn[hl][i] = Hn[i];
            }
        }
        __syncthreads();
        // trial cost with the same correspondences
        const bool act2 = mine && s_state[hl];
        float trial = 0.f;
        if (act2) {
            const float s00 = (float)s_Hn[hl][0], s01 = (float)s_Hn[hl][1], s02 = (float)s_Hn[hl][2], u0t = (float)s_Hn[hl][3];
            const float s10 = (float)s_Hn[hl][4], s11 = (float)s_Hn[hl][5], s12 = (float)s_Hn[hl][6], u1t = (float)s_Hn[hl][7];
            const float s20 = (float)s_Hn[hl][8], s21 = (float)s_Hn[hl][9], s22 = (float)s_Hn[hl][10], u2t = (float)s_Hn[hl][11];
            for (int i = g; i < a.n_pix; i += G) {
                const int m = corr[(size_t)i * nb + hl];
                if (m < 0) continue;
                ++w_trial;
                const float4 x = xcs[i];
                const size_t e = (size_t)i * stride + m;
                const float4 m0 = __ldg(&t0[e]);
                const float y0 = fmaf(s00, x.x, fmaf(s01, x.y, fmaf(s02, x.z, u0t)));
                const float y1 = fmaf(s10, x.x, fmaf(s11, x.y, fmaf(s12, x.z, u1t)));
                const float y2 = fmaf(s20, x.x, fmaf(s21, x.y, fmaf(s22, x.z, u2t)));
                const float v0 = y0 - m0.x, v1 = y1 - m0.y, v2 = y2 - m0.z;
                if (cov) {
                    const float4 m1 = __ldg(&t1[e]);
                    const float r0 = fmaf(m0.w, v0, fmaf(m1.x, v1, m1.y * v2));
                    const float r1 = fmaf(m1.z, v1, m1.w * v2);
                    const float r2 = __ldg(&t2[e]) * v2;
                    trial = fmaf(r0, r0, fmaf(r1, r1, fmaf(r2, r2, trial)));
                } else {
                    trial = fmaf(v0, v0, fmaf(v1, v1, fmaf(v2, v2, trial)));
                }
            }
        }
        s_red[t * 8] = trial;
        __syncthreads();
        for (int s = G >> 1; s > 0; s >>= 1) {
            if (g < s) s_red[t * 8] += s_red[(t + s * HB) * 8];
            __syncthreads();
        }
        if (g == 0 && act2) {
            if (s_red[t * 8] < s_tot[hl][27]) {
                for (int i = 0; i < 12; ++i) s_H[hl][i] = s_Hn[hl][i];
                s_lambda[hl] /= 10.0;
            } else {
                s_lambda[hl] *= 10.0;
            }
        }
        __syncthreads();
    }
    for (int i = t; i < nb * 12; i += LM3_THREADS)
        a.q.cur_pose[((size_t)b * NC + h0 + i / 12) * 12 + i % 12] = s_H[i / 12][i % 12];
    if (a.work && mine) {
        atomicAdd(&a.work[W_LM_PAIRS], (unsigned long long)w_pairs);
        atomicAdd(&a.work[W_LM_MODES], (unsigned long long)w_modes);
        atomicAdd(&a.work[W_LM_INLIERS], (unsigned long long)w_in);
        atomicAdd(&a.work[W_LM_TRIAL], (unsigned long long)w_trial);
    }
}

// Mode table of batch `batch`: for each drawn pixel, M(u) decoded to FP32
// (position, Cholesky factor) into one row of mpad records.
__global__ void k_build_table(QueryState q, int hw_max, ModeView mv, RParams p, int batch) {
    const int b = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.eta * p.mpad) return;
    const int i = batch * p.eta + e / p.mpad, m = e % p.mpad;
    const size_t row = (size_t)b * p.max_pix + i;
    const int pix = q.pix[row];
    const int cnt = pix < 0 ? 0
                            : pixel_modes(q.mcount + (size_t)b * hw_max,
                                          q.prec ? q.prec + (size_t)b * hw_max : nullptr, pix, p.n_trees);
    if (m == 0) q.tab_cnt[row] = (int16_t)cnt;
    if (m >= cnt) return;
    uint32_t L;
    int rank;
    if (q.prec)
        mode_at_rec(q.prec[(size_t)b * hw_max + pix], p.n_trees, mv.leaves_per_tree, m, &L, &rank);
    else
        mode_at(mv, q.leaves + (size_t)b * p.n_trees * hw_max, hw_max, pix, p.n_trees, p.k_top, m, &L, &rank);
    const float3 mp = mode_pos(mv, L, rank);
    const size_t me = (size_t)L * mv.m_max + rank;
    const size_t o = row * p.mpad + m;
    if (p.use_cov) {
        const float4 u0 = mv.mU[2 * me], u1 = mv.mU[2 * me + 1];
        q.tab0[o] = make_float4(mp.x, mp.y, mp.z, u0.x);
        q.tab1[o] = make_float4(u0.y, u0.z, u0.w, u1.x);
        q.tab2[o] = u1.y;
    } else {
        q.tab0[o] = make_float4(mp.x, mp.y, mp.z, 1.f);
    }
}

rl_status launch_build_table(const QueryState &q, int hw_max, ModeView mv, const RParams &p, int batch,
                             int n, cudaStream_t s) {
    dim3 grid((p.eta * p.mpad + 255) / 256, n);
    k_build_table<<<grid, 256, 0, s>>>(q, hw_max, mv, p, batch);
    RL_LAUNCH_CK();
    return RL_OK;
}

// z-depth of the first box face hit by the ray of pixel (u, v) (exit point
// from inside the box, entry point from outside), in FP64.
__device__ bool ray_depth64(const double *P, int u, int v, float fx, float fy, float cx, float cy,
                            const double lo[3], const double hi[3], double *depth) {
    const double dc0 = ((double)u - (double)cx) / (double)fx;
    const double dc1 = ((double)v - (double)cy) / (double)fy;
    double tn = -INFINITY, tf = INFINITY;
    for (int ax = 0; ax < 3; ++ax) {
        const double d = P[4 * ax] * dc0 + P[4 * ax + 1] * dc1 + P[4 * ax + 2];
        const double o = P[4 * ax + 3];
        if (d == 0.0) {
            if (o < lo[ax] || o > hi[ax]) return false;
            continue;
        }
        const double t1 = (lo[ax] - o) / d, t2 = (hi[ax] - o) / d;
        tn = fmax(tn, fmin(t1, t2));
        tf = fmin(tf, fmax(t1, t2));
    }
    if (tn > tf) return false;
    if (tn > 0.0) { *depth = tn; return true; }
    if (tf > 0.0) { *depth = tf; return true; }
    return false;
}

// The FP64 re-evaluation of one ray, kept out of line so that none of its
// FP64 work is scheduled into the FP32 loop that rarely needs it.
__device__ __noinline__ bool ray_depth_fp64(const double *P, int u, int v, float fx, float fy, float cx, float cy,
                                            const double lo[3], const double hi[3], float *depth) {
    double dd = 0.0;
    const bool ok = ray_depth64(P, u, v, fx, fy, cx, cy, lo, hi, &dd);
    *depth = (float)dd;
    return ok;
}

// Each thread owns RC_PIX pixels of an RC_TILE-pixel tile and runs all poses
// of the frame over them in turn (poses staged in shared memory, RC_CHUNK at a
// time), so each pixel's live depth and viewing direction are read once.  The
// hit test runs in FP32; a ray whose decision lies within a relative margin
// of 1e-4 of changing (near-parallel faces, grazing edges, a face through the
// camera) is re-evaluated in FP64, so the valid mask of Eq. 7 is the FP64
// one.  Per pose the tile's sums are reduced over the thread's pixels in
// order, then over lanes, then over warps in order, one partial per (pose,
// tile).
constexpr int RC_CHUNK = 16;

__global__ void __launch_bounds__(256) k_raycast_score(RaycastArgs a) {
    __shared__ float sPf[RC_CHUNK][12];
    __shared__ float s_sum[RC_CHUNK][8];
    __shared__ int s_syn[RC_CHUNK][8], s_both[RC_CHUNK][8];
    const int b = blockIdx.y;
    const int n_poses = a.n_poses_of(b);
    if (n_poses <= 0) return;
    const Frame fr = a.frames[b];
    const int npx = fr.W * fr.H;
    int u[RC_PIX], v[RC_PIX];
    float dc0[RC_PIX], dc1[RC_PIX], dl[RC_PIX];
    bool in[RC_PIX];
#pragma unroll
    for (int q = 0; q < RC_PIX; ++q) {
        const int p = blockIdx.x * RC_TILE + q * 256 + threadIdx.x;
        in[q] = p < npx;
        u[q] = 0; v[q] = 0;
        dc0[q] = 0.f; dc1[q] = 0.f; dl[q] = 0.f;
        if (in[q]) {
            u[q] = p % fr.W;
            v[q] = p / fr.W;
            // fast approximate divisions: their few-ulp error is far inside
            // the margin that sends a ray to the FP64 path
            dc0[q] = __fdividef((float)u[q] - fr.cx, fr.fx);
            dc1[q] = __fdividef((float)v[q] - fr.cy, fr.fy);
            dl[q] = fr.depth[p];
        }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned n64 = 0;  // rays re-evaluated in FP64 (profiling counter)
    for (int c0 = 0; c0 < n_poses; c0 += RC_CHUNK) {
        const int cnt = min(RC_CHUNK, n_poses - c0);
        __syncthreads();  // the previous chunk's poses and partials are consumed
        for (int e = threadIdx.x; e < cnt * 12; e += blockDim.x) sPf[e / 12][e % 12] = (float)a.pose_of(b, c0 + e / 12)[e % 12];
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const float *P = sPf[k];
            float sum = 0.f;
            int syn = 0, both = 0;
            // A camera more than 1 mm inside the box: every ray leaves the
            // box exactly once, at the nearest exit plane; with t_ax = (bound
            // - o) / d, bound = hi for d >= +0 and lo for d <= -0 (a zero
            // component then gives +inf), the depth is min_ax t_ax, a
            // continuous function of the ray with no hit/miss decision to
            // certify.  Same value as the slab test below up to FP32 rounding.
            // The approximate reciprocal (within 2 ulp) maps +-0 to +-inf.
            const float ox = P[3], oy = P[7], oz = P[11];
            const bool inside = ox - a.lo[0] > 1e-3f && a.hi[0] - ox > 1e-3f && oy - a.lo[1] > 1e-3f &&
                                a.hi[1] - oy > 1e-3f && oz - a.lo[2] > 1e-3f && a.hi[2] - oz > 1e-3f;
            if (inside) {
                const float lx = a.lo[0] - ox, hx = a.hi[0] - ox, ly = a.lo[1] - oy, hy = a.hi[1] - oy;
                const float lz = a.lo[2] - oz, hz = a.hi[2] - oz;
#pragma unroll
                for (int q = 0; q < RC_PIX; ++q) {
                    if (!in[q]) continue;
                    const float d0 = fmaf(P[0], dc0[q], fmaf(P[1], dc1[q], P[2]));
                    const float d1 = fmaf(P[4], dc0[q], fmaf(P[5], dc1[q], P[6]));
                    const float d2 = fmaf(P[8], dc0[q], fmaf(P[9], dc1[q], P[10]));
                    const float t0 = (signbit(d0) ? lx : hx) * __fdividef(1.0f, d0);
                    const float t1 = (signbit(d1) ? ly : hy) * __fdividef(1.0f, d1);
                    const float t2 = (signbit(d2) ? lz : hz) * __fdividef(1.0f, d2);
                    const float depth = fminf(t0, fminf(t1, t2));
                    ++syn;
                    if (dl[q] > 0.f) {
                        ++both;
                        sum += fabsf(dl[q] - depth);
                    }
                }
            } else {
#pragma unroll
            for (int q = 0; q < RC_PIX; ++q) {
                if (!in[q]) continue;
                float d[3], o[3];
                for (int r = 0; r < 3; ++r) {
                    d[r] = fmaf(P[4 * r], dc0[q], fmaf(P[4 * r + 1], dc1[q], P[4 * r + 2]));
                    o[r] = P[4 * r + 3];
                }
                const float dn = fabsf(d[0]) + fabsf(d[1]) + fabsf(d[2]);
                float tn = -INFINITY, tf = INFINITY;
                bool ok = true, unsure = false;
                for (int ax = 0; ax < 3; ++ax) {
                    if (fabsf(d[ax]) <= 1e-5f * dn) {
                        unsure = true;
                        continue;
                    }
                    const float inv = __fdividef(1.0f, d[ax]);
                    const float ta = (a.lo[ax] - o[ax]) * inv, tb = (a.hi[ax] - o[ax]) * inv;
                    tn = fmaxf(tn, fminf(ta, tb));
                    tf = fminf(tf, fmaxf(ta, tb));
                }
                float depth = 0.f;
                if (!unsure) {
                    const float scale = fmaxf(fabsf(tn), fabsf(tf));
                    if (fabsf(tf - tn) <= 1e-4f * scale || fabsf(tn) <= 1e-4f * scale ||
                        fabsf(tf) <= 1e-4f * scale)
                        unsure = true;
                }
                if (unsure) {
                    ++n64;
                    ok = ray_depth_fp64(a.pose_of(b, c0 + k), u[q], v[q], fr.fx, fr.fy, fr.cx, fr.cy, a.lo64,
                                        a.hi64, &depth);
                } else if (tn <= tf && tn > 0.f) {
                    depth = tn;
                } else if (tn <= tf && tf > 0.f) {
                    depth = tf;
                } else {
                    ok = false;
                }
                if (ok) {
                    ++syn;
                    if (dl[q] > 0.f) {
                        ++both;
                        sum += fabsf(dl[q] - depth);
                    }
                }
            }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
            syn = __reduce_add_sync(0xffffffffu, syn);
            both = __reduce_add_sync(0xffffffffu, both);
            if (lane == 0) {
                s_sum[k][w] = sum;
                s_syn[k][w] = syn;
                s_both[k][w] = both;
            }
        }
        __syncthreads();
        if (threadIdx.x < cnt) {
            const int k = threadIdx.x;
            float ts = 0.f;
            int tsyn = 0, tb = 0;
            for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) {
                ts += s_sum[k][ww];
                tsyn += s_syn[k][ww];
                tb += s_both[k][ww];
            }
            const size_t o = ((size_t)b * a.pose_cap + c0 + k) * a.n_tiles + blockIdx.x;
            a.part_sum[o] = (double)ts;
            a.part_cnt[2 * o] = tsyn;
            a.part_cnt[2 * o + 1] = tb;
        }
    }
    if (a.work) {
        if (threadIdx.x == 0)
            atomicAdd(&a.work[W_RAYS], (unsigned long long)n_poses *
                                           (unsigned long long)min(RC_TILE, npx - (int)(blockIdx.x * RC_TILE)));
        if (n64) atomicAdd(&a.work[W_RAY64], (unsigned long long)n64);
    }
}

// Eq. 7 from the tile partials of one (frame, pose): FP64 sums in tile order.
__device__ float score_from_tiles(const double *part_sum, const int32_t *part_cnt, size_t base,
                                  int n_tiles, double npx, float *valid_frac) {
    double sum = 0.0;
    long syn = 0, both = 0;
    for (int t = 0; t < n_tiles; ++t) {
        sum += part_sum[base + t];
        syn += part_cnt[2 * (base + t)];
        both += part_cnt[2 * (base + t) + 1];
    }
    const double frac = (double)syn / npx;
    if (valid_frac) *valid_frac = (float)frac;
    return (frac >= 0.1 && both > 0) ? (float)(sum / (double)both) : INFINITY;
}

// Eq. 7-8 per frame, then the frame's result record.
__global__ void __launch_bounds__(256) k_finalize(QueryState q, RParams p, int n_tiles, int ranked) {
    __shared__ double s_sum[8];
    __shared__ long long s_syn[8], s_both[8];
    const int b = blockIdx.x;
    const Frame fr = q.frames[b];
    if (ranked && q.n_hyp[b] > 0) {
        // Eq. 7 for each chosen pose: tile partials summed by a fixed-shape
        // block reduction (FP64 sums, integer counts)
        const double npx = (double)fr.W * (double)fr.H;
        for (int c = 0; c < q.n_chosen[b]; ++c) {
            const size_t base = ((size_t)b * 16 + c) * n_tiles;
            double sum = 0.0;
            long long syn = 0, both = 0;
            for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) {
                sum += q.score_part[base + t];
                syn += q.score_cnt[2 * (base + t)];
                both += q.score_cnt[2 * (base + t) + 1];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sum += __shfl_down_sync(0xffffffffu, sum, o);
                syn += __shfl_down_sync(0xffffffffu, syn, o);
                both += __shfl_down_sync(0xffffffffu, both, o);
            }
            if ((threadIdx.x & 31) == 0) {
                s_sum[threadIdx.x >> 5] = sum;
                s_syn[threadIdx.x >> 5] = syn;
                s_both[threadIdx.x >> 5] = both;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double ts = 0.0;
                long long tsyn = 0, tb = 0;
                for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                    ts += s_sum[k];
                    tsyn += s_syn[k];
                    tb += s_both[k];
                }
                const double frac = (double)tsyn / npx;
                // a pose whose ICP failed is discarded (Sec. 3.2.4)
                const bool kept = !p.icp || q.icp_ok[(size_t)b * 16 + c];
                q.chosen_score[(size_t)b * 16 + c] =
                    (kept && frac >= 0.1 && tb > 0) ? (float)(ts / (double)tb) : INFINITY;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x != 0) return;
    DevResult *out = (DevResult *)q.result_blob + b;
    out->err = q.dev_err[b];
    out->n_hypotheses = q.n_hyp[b];
    out->n_chosen = q.n_hyp[b] > 0 ? q.n_chosen[b] : 0;
    out->n_pixels = q.n_pix[b];
    out->score = INFINITY;
    out->best = -1;
    out->icp_mask = 0;
    if (p.icp && q.n_hyp[b] > 0) {
        const int n_icp = ranked ? q.n_chosen[b] : 1;
        for (int c = 0; c < n_icp; ++c)
            if (q.icp_ok[(size_t)b * 16 + c]) out->icp_mask |= 1 << c;
    }
    if (q.n_hyp[b] == 0) {
        out->status = RL_NO_POSE;
        for (int k = 0; k < 12; ++k) out->pose[k] = (k % 5 == 0) ? 1.0 : 0.0;
        out->energy = INFINITY;
        out->energy_per_pixel = INFINITY;
        return;
    }
    out->status = RL_POSE_FOUND;
    const int NC = p.n_cull;
    int best = -1;
    float bs = INFINITY;
    if (ranked) {
        for (int c = 0; c < q.n_chosen[b]; ++c) {
            const float s = q.chosen_score[(size_t)b * 16 + c];
            if (s < bs) {
                bs = s;
                best = c;
            }
        }
        if (best < 0) best = 0;
        out->score = bs;
        out->best = best;
        for (int k = 0; k < 12; ++k) out->pose[k] = q.chosen_pose[((size_t)b * 16 + best) * 12 + k];
        out->energy = q.chosen_energy[(size_t)b * 16 + best];
        out->energy_per_pixel = out->energy / (float)q.chosen_npix[b];
    } else {
        for (int c = 0; c < q.n_chosen[b]; ++c) q.chosen_score[(size_t)b * 16 + c] = INFINITY;
        for (int k = 0; k < 12; ++k) out->pose[k] = q.cur_pose[((size_t)b * NC) * 12 + k];
        out->energy = q.cur_energy[(size_t)b * NC];
        out->energy_per_pixel = out->energy / (float)q.n_pix[b];
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
rl_status launch_energy(const EnergyArgs &a0, int max_count, int n, cudaStream_t s, int max_threads) {
    EnergyArgs a = a0;
    int ht = 32;  // hypotheses per block: the smallest power of two covering them, capped
    while (ht < max_count && ht < max_threads) ht <<= 1;
    const size_t sm = (size_t)a.chunk * sizeof(float4) + (size_t)a.chunk * a.maxm * (2 * sizeof(float4) + sizeof(float)) +
                      (size_t)a.chunk * sizeof(int);
    dim3 grid((max_count + ht - 1) / ht, (a.n_pix + a.chunk - 1) / a.chunk, n);
    k_energy<<<grid, ht, sm, s>>>(a);
    RL_LAUNCH_CK();
    return RL_OK;
}

size_t energy_smem(int chunk, int maxm) {
    return (size_t)chunk * sizeof(float4) + (size_t)chunk * maxm * (2 * sizeof(float4) + sizeof(float)) +
           (size_t)chunk * sizeof(int);
}

rl_status launch_select(const SelectArgs &a, int n, cudaStream_t s) {
    const size_t sm = (size_t)a.p.n_hyp * (sizeof(float) + sizeof(int)) +
                      (size_t)a.p.n_cull * (12 * sizeof(double) + sizeof(float) + sizeof(int)) + 64;
    k_select<<<n, 1024, sm, s>>>(a);
    RL_LAUNCH_CK();
    return RL_OK;
}

bool lm_uses_cluster(const RParams &p) {
    return p.n_cull <= 64 && lm_cluster_smem(p.mpad, p.use_cov) <= kLmClusterSmemMax;
}

// The cluster kernel, or (rows too long for its staged tiles) the spread
// kernel; n_cull <= 64 (checked when the relocaliser is created).
rl_status launch_lm(const LmArgs &a, int n, cudaStream_t s) {
    if (lm_uses_cluster(a.p)) return launch_lm_cluster(a, n, s);
    dim3 grid(LM3_BPQ, n);
    k_lm_spread<<<grid, LM3_THREADS, 0, s>>>(a);
    RL_LAUNCH_CK();
    return RL_OK;
}

// Kernel attributes set once, outside any stream capture.
rl_status prepare_kernels() {
    static bool done = false;
    static std::mutex mu;
    std::lock_guard<std::mutex> g(mu);
    if (done) return RL_OK;
    RL_TRY(prepare_lm_cluster());
    RL_TRY(prepare_hypgen());
    done = true;
    return RL_OK;
}

rl_status launch_raycast(const RaycastArgs &a, int n, int max_hw, cudaStream_t s) {
    dim3 grid(a.n_tiles, n);
    k_raycast_score<<<grid, 256, 0, s>>>(a);
    RL_LAUNCH_CK();
    return RL_OK;
}

rl_status launch_finalize(const QueryState &q, const RParams &p, int n_tiles, int ranked, int n,
                          cudaStream_t s) {
    k_finalize<<<n, 256, 0, s>>>(q, p, n_tiles, ranked);
    RL_LAUNCH_CK();
    return RL_OK;
}

}  // namespace rl

namespace rl {
// Standalone Eq. 6-7 scorer: poses [n][12] against one live depth frame.
__global__ void k_scores_final(const double *part_sum, const int32_t *part_cnt, int n_tiles,
                               int n, double npx, float *scores, float *valid_frac) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    float vf;
    scores[c] = score_from_tiles(part_sum, part_cnt, (size_t)c * n_tiles, n_tiles, npx, &vf);
    valid_frac[c] = vf;
}

rl_status launch_score_poses(const RaycastArgs &a, int n_poses, int npx, float *scores,
                             float *valid_frac, cudaStream_t s) {
    dim3 grid(a.n_tiles, 1);
    k_raycast_score<<<grid, 256, 0, s>>>(a);
    RL_LAUNCH_CK();
    k_scores_final<<<(n_poses + 63) / 64, 64, 0, s>>>(a.part_sum, a.part_cnt, a.n_tiles, n_poses,
                                                      (double)npx, scores, valid_frac);
    RL_LAUNCH_CK();
    return RL_OK;
}
}  // namespace rl
