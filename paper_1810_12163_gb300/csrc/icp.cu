// ICP of a camera pose against the scene model before ranking (Sec. 3.2.4).
// The paper refines each chosen pose by ICP and drops the pose when ICP
// fails; the ICP variant is its host system's.  Here: point-to-plane ICP
// against the analytic room box with projective association, Gauss-Newton
// on a camera-frame update H exp(xi), coarse to fine over pixel strides (the
// rules are stated with rl_icp_params in the public header).
//
// One thread block owns one (frame, pose) for all iterations: its threads
// stride over the level's pixels accumulating the 27 normal-equation sums
// in FP32 registers, the sums are reduced across lanes by shuffles and
// across warps in warp order in FP64, and one thread solves the ridged 6x6
// system in FP64 and composes the update.  The frame's depth image stays in
// L2 across the poses and iterations that read it.
#include "kernels.h"
#include "lm_dev.cuh"

namespace rl {

constexpr int ICP_THREADS = 256;
constexpr int ICP_WARPS = ICP_THREADS / 32;
constexpr int ICP_NS = 27;  // upper triangle of J^T J (21, row-major), then J^T r (6)

__global__ void __launch_bounds__(ICP_THREADS) k_icp(IcpArgs a) {
    const int b = blockIdx.y, c = blockIdx.x;
    if (a.gate && a.gate[b] <= 0) return;
    const int cnt = a.counts ? a.counts[b] : a.cap;
    if (c >= cnt) return;
    const Frame fr = a.frames[b];
    double *P = a.poses + ((size_t)b * a.pose_stride + c) * 12;
    __shared__ double sH[12];
    __shared__ float s_part[ICP_WARPS][ICP_NS];
    __shared__ int s_cnt[ICP_WARPS][2];
    __shared__ double s_tot[ICP_NS];
    __shared__ int s_n[2];  // inliers, valid pixels of the last iteration
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid < 12) sH[tid] = P[tid];
    if (tid == 0) {
        s_fail = 0;
        s_n[0] = s_n[1] = 0;
    }
    const float ifx = 1.0f / fr.fx, ify = 1.0f / fr.fy;
    unsigned long long visited = 0;
    bool stop = false;
    for (int l = 0; l < a.ip.levels && !stop; ++l) {
        const int st = a.ip.stride[l];
        const int nu = (fr.W + st - 1) / st, nl = nu * ((fr.H + st - 1) / st);
        const float dist2 = a.ip.dist[l] * a.ip.dist[l];
        for (int it = 0; it < a.ip.iters[l] && !stop; ++it) {
            __syncthreads();  // sH holds the current pose
            float R[9], t[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
#pragma unroll
                for (int k = 0; k < 3; ++k) R[3 * r + k] = (float)sH[4 * r + k];
                t[r] = (float)sH[4 * r + 3];
            }
            float acc[ICP_NS];
#pragma unroll
            for (int k = 0; k < ICP_NS; ++k) acc[k] = 0.f;
            int n_in = 0, n_valid = 0;
            for (int p = tid; p < nl; p += ICP_THREADS) {
                const int u = (p % nu) * st, v = (p / nu) * st;
                const float d = fr.depth[(size_t)v * fr.W + u];
                if (!(d > 0.f) || isinf(d)) continue;
                ++n_valid;
                const float c0 = ((float)u - fr.cx) * ifx, c1 = ((float)v - fr.cy) * ify;
                float dir[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) dir[r] = fmaf(R[3 * r], c0, fmaf(R[3 * r + 1], c1, R[3 * r + 2]));
                // first face hit by t + s dir: exit from inside, entry from outside
                float tn = -INFINITY, tf = INFINITY;
                int an = 0, af = 0;
                bool hit = true;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    if (dir[ax] == 0.f) {
                        hit = hit && t[ax] >= a.lo[ax] && t[ax] <= a.hi[ax];
                        continue;
                    }
                    const float inv = 1.0f / dir[ax];
                    const float t1 = (a.lo[ax] - t[ax]) * inv, t2 = (a.hi[ax] - t[ax]) * inv;
                    const float tmin = fminf(t1, t2), tmax = fmaxf(t1, t2);
                    if (tmin > tn) { tn = tmin; an = ax; }
                    if (tmax < tf) { tf = tmax; af = ax; }
                }
                if (!hit || tn > tf || !(tf > 0.f)) continue;
                const float sh = tn > 0.f ? tn : tf;
                const int ax = tn > 0.f ? an : af;
                const float gap = d - sh;
                const float dd2 = fmaf(dir[0], dir[0], fmaf(dir[1], dir[1], dir[2] * dir[2]));
                if (gap * gap * dd2 > dist2) continue;
                // face normal n = e_ax; m = R^T n (row ax of R); x = d c(u)
                const float m0 = ax == 0 ? R[0] : (ax == 1 ? R[3] : R[6]);
                const float m1 = ax == 0 ? R[1] : (ax == 1 ? R[4] : R[7]);
                const float m2 = ax == 0 ? R[2] : (ax == 1 ? R[5] : R[8]);
                const float res = gap * (ax == 0 ? dir[0] : (ax == 1 ? dir[1] : dir[2]));
                const float x0 = d * c0, x1 = d * c1, x2 = d;
                const float J[6] = {m0, m1, m2, x1 * m2 - x2 * m1, x2 * m0 - x0 * m2, x0 * m1 - x1 * m0};
                int k = 0;
#pragma unroll
                for (int r = 0; r < 6; ++r)
#pragma unroll
                    for (int q = r; q < 6; ++q) {
                        acc[k] = fmaf(J[r], J[q], acc[k]);
                        ++k;
                    }
#pragma unroll
                for (int r = 0; r < 6; ++r) acc[21 + r] = fmaf(J[r], res, acc[21 + r]);
                ++n_in;
            }
            visited += (unsigned long long)n_valid;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int k = 0; k < ICP_NS; ++k) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
                n_in += __shfl_down_sync(0xffffffffu, n_in, o);
                n_valid += __shfl_down_sync(0xffffffffu, n_valid, o);
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < ICP_NS; ++k) s_part[w][k] = acc[k];
                s_cnt[w][0] = n_in;
                s_cnt[w][1] = n_valid;
            }
            __syncthreads();
            if (tid < ICP_NS) {
                double sum = 0.0;
                for (int ww = 0; ww < ICP_WARPS; ++ww) sum += (double)s_part[ww][tid];
                s_tot[tid] = sum;
            } else if (tid < ICP_NS + 2) {
                int sum = 0;
                for (int ww = 0; ww < ICP_WARPS; ++ww) sum += s_cnt[ww][tid - ICP_NS];
                s_n[tid - ICP_NS] = sum;
            }
            __syncthreads();
            if (tid == 0) {
                if (s_n[0] < 6) {
                    s_fail = 1;
                } else {
                    double A[36], g[6], xi[6];
                    int k = 0;
                    for (int r = 0; r < 6; ++r)
                        for (int q = r; q < 6; ++q) {
                            A[6 * r + q] = A[6 * q + r] = s_tot[k];
                            ++k;
                        }
                    const double lam = a.ip.ridge * (A[0] + A[7] + A[14] + A[21] + A[28] + A[35]) / 6.0;
                    for (int r = 0; r < 6; ++r) {
                        A[7 * r] += lam;
                        g[r] = -s_tot[21 + r];
                    }
                    if (!chol_solve6(A, g, xi)) {
                        s_fail = 1;
                    } else {
                        // H <- H exp(xi): exp(xi) as the left update of the identity
                        double E[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0}, N[12];
                        se3_left(xi, E);
                        for (int r = 0; r < 3; ++r)
                            for (int q = 0; q < 4; ++q)
                                N[4 * r + q] = sH[4 * r] * E[q] + sH[4 * r + 1] * E[4 + q] + sH[4 * r + 2] * E[8 + q] +
                                               (q == 3 ? sH[4 * r + 3] : 0.0);
                        for (int q = 0; q < 12; ++q) sH[q] = N[q];
                    }
                }
            }
            __syncthreads();
            stop = s_fail != 0;
        }
    }
    if (a.work && visited) atomicAdd(&a.work[W_ICP_PIX], visited);
    if (tid == 0) {
        const int nin = s_n[0], nval = s_n[1];
        const bool ok = !s_fail && nval > 0 && (double)nin >= a.ip.min_frac * (double)nval;
        const size_t o = (size_t)b * a.out_stride + c;
        a.ok[o] = ok ? 1 : 0;
        a.frac[o] = nval > 0 ? (float)((double)nin / (double)nval) : 0.f;
        if (ok)
            for (int q = 0; q < 12; ++q) P[q] = sH[q];
    }
}

rl_status launch_icp(const IcpArgs &a, int n, cudaStream_t s) {
    if (n <= 0 || a.cap <= 0) return RL_OK;
    dim3 grid(a.cap, n);
    k_icp<<<grid, ICP_THREADS, 0, s>>>(a);
    RL_LAUNCH_CK();
    return RL_OK;
}

}  // namespace rl
