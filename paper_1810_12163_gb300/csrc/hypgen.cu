// Hypothesis generation (Sec. 3.2.3): Kabsch on checked triples of
// pixel-to-mode correspondences, one warp per hypothesis slot; compaction of
// the successful slots; pixel batches of the preemptive RANSAC.
//
// Compiled with --fmad=false: back-projection (FP32) and the three checks
// (FP64 from FP32 inputs) are plain IEEE operations in a fixed order, so
// every accept/reject decision, and therefore the winning iteration of each
// slot, is exactly reproducible.
#include "internal.h"
#include "kernels.h"
#include "relocgb_dev.cuh"

namespace rl {

// Largest-eigenvalue eigenvector of a symmetric 4x4 matrix by cyclic Jacobi.
__device__ void jacobi4_max_eigvec(double A[4][4], double q[4]) {
    double V[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int i = 0; i < 4; ++i) {
            dg += A[i][i] * A[i][i];
            for (int j = i + 1; j < 4; ++j) off += A[i][j] * A[i][j];
        }
        if (off <= 1e-32 * dg || off == 0.0) break;
        for (int p = 0; p < 3; ++p)
            for (int r = p + 1; r < 4; ++r) {
                const double apr = A[p][r];
                if (apr == 0.0) continue;
                const double theta = (A[r][r] - A[p][p]) / (2.0 * apr);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 4; ++k) {
                    if (k == p || k == r) continue;
                    const double akp = A[k][p], akr = A[k][r];
                    A[k][p] = A[p][k] = c * akp - s * akr;
                    A[k][r] = A[r][k] = s * akp + c * akr;
                }
                A[p][p] -= t * apr;
                A[r][r] += t * apr;
                A[p][r] = A[r][p] = 0.0;
                for (int k = 0; k < 4; ++k) {
                    const double vkp = V[k][p], vkr = V[k][r];
                    V[k][p] = c * vkp - s * vkr;
                    V[k][r] = s * vkp + c * vkr;
                }
            }
    }
    int best = 0;
    for (int i = 1; i < 4; ++i)
        if (A[i][i] > A[best][best]) best = i;
    for (int i = 0; i < 4; ++i) q[i] = V[i][best];
}

// Rigid transform (camera -> world) of three pairs by Horn's closed form
// (unit quaternion of the largest eigenvalue), which solves the same least
// squares problem as Kabsch's SVD construction.
__device__ __noinline__ void kabsch3_horn(const double a[3][3], const double b[3][3], double H[12]) {
    double ca[3], cb[3];
    for (int k = 0; k < 3; ++k) {
        ca[k] = (a[0][k] + a[1][k] + a[2][k]) / 3.0;
        cb[k] = (b[0][k] + b[1][k] + b[2][k]) / 3.0;
    }
    double S[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < 3; ++i)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) S[r][c] += (a[i][r] - ca[r]) * (b[i][c] - cb[c]);
    const double Sxx = S[0][0], Sxy = S[0][1], Sxz = S[0][2];
    const double Syx = S[1][0], Syy = S[1][1], Syz = S[1][2];
    const double Szx = S[2][0], Szy = S[2][1], Szz = S[2][2];
    double N[4][4] = {{Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx},
                      {Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz},
                      {Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy},
                      {Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz}};
    double q[4];
    jacobi4_max_eigvec(N, q);
    const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const double q0 = q[0] / nq, q1 = q[1] / nq, q2 = q[2] / nq, q3 = q[3] / nq;
    const double R[3][3] = {
        {q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3, 2 * (q1 * q2 - q0 * q3), 2 * (q1 * q3 + q0 * q2)},
        {2 * (q1 * q2 + q0 * q3), q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3, 2 * (q2 * q3 - q0 * q1)},
        {2 * (q1 * q3 - q0 * q2), 2 * (q2 * q3 + q0 * q1), q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3}};
    for (int r = 0; r < 3; ++r) {
        H[4 * r + 0] = R[r][0];
        H[4 * r + 1] = R[r][1];
        H[4 * r + 2] = R[r][2];
        H[4 * r + 3] = cb[r] - (R[r][0] * ca[0] + R[r][1] * ca[1] + R[r][2] * ca[2]);
    }
}

struct HypArgs {
    const Frame *frames;
    const uint16_t *leaves;  // [B][T][hw_max]
    const uint16_t *mcount;  // [B][hw_max] |M(u)|
    const uint4 *prec;       // [B][hw_max] pixel records (<= 5 trees) or null
    int hw_max;
    ModeView mv;
    RParams p;
    double *hyp_pose;        // [B][N][12]
    int32_t *hyp_iter;       // [B][N]
};

__device__ __forceinline__ float3 backproject(const Frame &fr, int p) {
    const float d = fr.depth[p];
    const int u = p % fr.W, v = p / fr.W;
    return make_float3(__fdiv_rn(__fmul_rn(__fsub_rn((float)u, fr.cx), d), fr.fx),
                       __fdiv_rn(__fmul_rn(__fsub_rn((float)v, fr.cy), d), fr.fy), d);
}

__device__ __forceinline__ double dist2_64(float3 a, float3 b) {
    const double e0 = (double)a.x - (double)b.x, e1 = (double)a.y - (double)b.y;
    const double e2 = (double)a.z - (double)b.z;
    return (e0 * e0 + e1 * e1) + e2 * e2;
}

__device__ __forceinline__ float dist2_32(float3 a, float3 b) {
    const float e0 = __fsub_rn(a.x, b.x), e1 = __fsub_rn(a.y, b.y), e2 = __fsub_rn(a.z, b.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(e0, e0), __fmul_rn(e1, e1)), __fmul_rn(e2, e2));
}

// The draws of iteration `it` of `slot`: three pixels, the colour-check pair
// and the three mode indices into M(u).
struct Draw {
    int pix[3];
    uint32_t m[3];
    int j;
};

__device__ __forceinline__ Draw draw(const HypArgs &a, const Frame &fr, int slot, int it) {
    const uint32_t ctr1 = (TAG_HYP << 16) | (uint32_t)a.p.level;
    const uint4 r0 = philox(make_uint4(slot, ctr1, it, 0), fr.key0, fr.key1);
    const uint32_t WH = (uint32_t)(fr.W * fr.H);
    Draw d;
    d.pix[0] = (int)draw_below(r0.x, WH);
    d.pix[1] = (int)draw_below(r0.y, WH);
    d.pix[2] = (int)draw_below(r0.z, WH);
    d.j = (int)draw_below(r0.w, 3);
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

// One generation attempt, evaluated cheapest-rejection first (the outcome
// does not depend on the order): every pixel needs a non-empty M(u) (|M(u)|
// is 0 without depth), then the colour of the checked pair, then the modes
// of the other pairs, spread and rigidity.  The spread and rigidity tests
// run in FP32 and are re-evaluated in FP64 whenever the FP32 value lies
// within a margin of the threshold far wider than its rounding error, so
// each decision equals the FP64 decision.
__device__ bool attempt(const HypArgs &a, const Frame &fr, const uint16_t *lv, const uint16_t *mc,
                        const uint4 *pr, int slot, int it) {
    Draw d = draw(a, fr, slot, it);
    int cnt[3];
    for (int i = 0; i < 3; ++i) {
        cnt[i] = mc[d.pix[i]];
        if (cnt[i] == 0) return false;
    }
    const uint32_t ctr1 = (TAG_HYP << 16) | (uint32_t)a.p.level;
    const uint4 r1 = philox(make_uint4(slot, ctr1, it, 1), fr.key0, fr.key1);
    const uint32_t u1[3] = {r1.x, r1.y, r1.z};
    // check 1: colour of pair j
    uint32_t L[3];
    int rank[3];
    {
        const int j = d.j;
        lookup(a, lv, pr, d.pix[j], (int)draw_below(u1[j], (uint32_t)cnt[j]), &L[j], &rank[j]);
        const uchar4 mcol = a.mv.mrgb[(size_t)L[j] * a.mv.m_max + rank[j]];
        const uint8_t *pc = fr.rgb + (size_t)d.pix[j] * 3;
        const int dr = abs((int)pc[0] - (int)mcol.x), dg = abs((int)pc[1] - (int)mcol.y),
                  db = abs((int)pc[2] - (int)mcol.z);
        if (max(dr, max(dg, db)) > a.p.colour_thresh) return false;
    }
    for (int i = 0; i < 3; ++i)
        if (i != d.j)
            lookup(a, lv, pr, d.pix[i], (int)draw_below(u1[i], (uint32_t)cnt[i]), &L[i], &rank[i]);
    float3 xw[3];
    for (int i = 0; i < 3; ++i) xw[i] = mode_pos(a.mv, L[i], rank[i]);
    // check 2: scene points pairwise at least sqrt(min_sq_dist) apart
    const int PA[3] = {0, 0, 1}, PB[3] = {1, 2, 2};
    const double thr = a.p.min_sq_dist;
    float dW2f[3];
    for (int k = 0; k < 3; ++k) {
        dW2f[k] = dist2_32(xw[PA[k]], xw[PB[k]]);
        const double f = (double)dW2f[k];
        if (f < thr * (1.0 - 1e-5)) return false;
        if (!(f > thr * (1.0 + 1e-5)) && dist2_64(xw[PA[k]], xw[PB[k]]) < thr) return false;
    }
    // check 3: rigidity, |d_W - d_C| <= max_trans_err for every pair
    float3 xc[3];
    for (int i = 0; i < 3; ++i) xc[i] = backproject(fr, d.pix[i]);
    const double tol = a.p.max_trans_err;
    for (int k = 0; k < 3; ++k) {
        const float dw = sqrtf(dW2f[k]), dc = sqrtf(dist2_32(xc[PA[k]], xc[PB[k]]));
        const double diff = fabs((double)dw - (double)dc);
        const double margin = 1e-5 * ((double)dw + (double)dc) + 1e-6;
        if (diff > tol + margin) return false;
        if (diff >= tol - margin) {
            const double e = fabs(sqrt(dist2_64(xw[PA[k]], xw[PB[k]])) -
                                  sqrt(dist2_64(xc[PA[k]], xc[PB[k]])));
            if (e > tol) return false;
        }
    }
    return true;
}

// The accepted triple of (slot, it), re-derived exactly, and its pose.
__device__ __noinline__ void accept_triple(const HypArgs &a, const Frame &fr, const uint16_t *lv,
                                           const uint16_t *mc, const uint4 *pr, int slot, int it, double H[12]) {
    const Draw d = draw(a, fr, slot, it);
    const uint32_t ctr1 = (TAG_HYP << 16) | (uint32_t)a.p.level;
    const uint4 r1 = philox(make_uint4(slot, ctr1, it, 1), fr.key0, fr.key1);
    const uint32_t u1[3] = {r1.x, r1.y, r1.z};
    double xc[3][3], xw[3][3];
    for (int i = 0; i < 3; ++i) {
        uint32_t L;
        int rank;
        lookup(a, lv, pr, d.pix[i], (int)draw_below(u1[i], (uint32_t)mc[d.pix[i]]), &L, &rank);
        const float3 c = backproject(fr, d.pix[i]);
        const float3 w = mode_pos(a.mv, L, rank);
        xc[i][0] = c.x; xc[i][1] = c.y; xc[i][2] = c.z;
        xw[i][0] = w.x; xw[i][1] = w.y; xw[i][2] = w.z;
    }
    kabsch3_horn(xc, xw, H);
}

// Warp per (frame, slot): the 32 lanes try 32 consecutive iterations; the
// lowest successful iteration wins, exactly as a sequential loop would.
// The attempt loop is latency bound (scattered loads of leaves and modes):
// registers are capped at 64 so that 32 warps per SM hide that latency.
__global__ void __launch_bounds__(128, 8) k_hypgen(HypArgs a) {
    const int lane = threadIdx.x & 31;
    const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int b = blockIdx.y;
    if (slot >= a.p.n_hyp) return;
    const Frame fr = a.frames[b];
    int32_t *iter_fail = a.hyp_iter + (size_t)b * a.p.n_hyp + slot;
    if (fr.W * fr.H == 0) {  // empty frame (e.g. accepted by an earlier cascade level)
        if (lane == 0) *iter_fail = -1;
        return;
    }
    const uint16_t *lv = a.leaves + (size_t)b * a.p.n_trees * a.hw_max;
    const uint16_t *mc = a.mcount + (size_t)b * a.hw_max;
    const uint4 *pr = a.prec ? a.prec + (size_t)b * a.hw_max : nullptr;
    int32_t *iter_out = a.hyp_iter + (size_t)b * a.p.n_hyp + slot;
    double *pose_out = a.hyp_pose + ((size_t)b * a.p.n_hyp + slot) * 12;
    for (int base = 0; base < a.p.max_iter; base += 32) {
        const int it = base + lane;
        const bool ok = it < a.p.max_iter && attempt(a, fr, lv, mc, pr, slot, it);
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (mask) {
            if (lane == __ffs(mask) - 1) {
                double H[12];
                accept_triple(a, fr, lv, mc, pr, slot, it, H);
                for (int k = 0; k < 12; ++k) pose_out[k] = H[k];
                *iter_out = it;
            }
            return;
        }
    }
    if (lane == 0) *iter_out = -1;
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
                               int hw_max, RParams p, int batch, int32_t *__restrict__ pix_out,
                               float4 *__restrict__ xc_out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (j >= p.eta) return;
    const Frame fr = frames[b];
    const uint16_t *mc = mcount + (size_t)b * hw_max;
    const uint32_t WH = (uint32_t)(fr.W * fr.H);
    int pix = -1;
    for (int at = 0; at < p.batch_attempts && WH > 0; ++at) {
        const uint4 r = philox(make_uint4(batch, (TAG_BATCH << 16) | (uint32_t)p.level, j, at),
                               fr.key0, fr.key1);
        const int q = (int)draw_below(r.x, WH);
        if (mc[q] == 0) continue;
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

rl_status launch_hypgen(const Frame *frames, const uint16_t *leaves, const uint16_t *mcount,
                        const uint4 *prec, int hw_max, ModeView mv, const RParams &p,
                        double *hyp_pose, int32_t *hyp_iter, int n, cudaStream_t s) {
    HypArgs a{frames, leaves, mcount, prec, hw_max, mv, p, hyp_pose, hyp_iter};
    dim3 grid((p.n_hyp + 3) / 4, n);
    k_hypgen<<<grid, 128, 0, s>>>(a);
    RL_LAUNCH_CK();
    return RL_OK;
}

rl_status launch_compact(const int32_t *hyp_iter, int N, int32_t *hyp_list, int32_t *n_hyp, int n,
                         cudaStream_t s) {
    k_compact<<<n, 1024, 0, s>>>(hyp_iter, N, hyp_list, n_hyp);
    RL_LAUNCH_CK();
    return RL_OK;
}

rl_status launch_sample_batch(const Frame *frames, const uint16_t *mcount, int hw_max,
                              const RParams &p, int batch, int32_t *pix, float4 *xc, int n,
                              cudaStream_t s) {
    dim3 grid((p.eta + 127) / 128, n);
    k_sample_batch<<<grid, 128, 0, s>>>(frames, mcount, hw_max, p, batch, pix, xc);
    RL_LAUNCH_CK();
    return RL_OK;
}

}  // namespace rl
