// ICP of a camera pose against the scene model before ranking (Sec. 3.2.4).
// The paper refines each chosen pose by ICP and drops the pose when ICP
// fails; the ICP variant is its host system's.  Here: point-to-plane ICP
// against the analytic room box with projective association, Gauss-Newton
// on a camera-frame update H exp(xi), coarse to fine over pixel strides (the
// rules are stated with rl_icp_params in the public header).
//
// One thread block owns one (frame, pose) for all iterations: its threads
// stride over the level's pixels accumulating the normal equations in FP32
// registers, the sums are reduced across lanes by shuffles and across warps
// in warp order in FP64, and one thread solves the ridged 6x6 system in FP64
// and composes the update.  The frame's depth image stays in L2 across the
// poses and iterations that read it.
//
// The camera-frame Jacobian J = (m, x x m), m = R^T n, equals B J_w with
// B = diag(R^T, R^T) and the world-frame J_w = (n, q' x n), q' = R x = d dir.
// With n = e_a a face axis, J_w has three nonzero entries, so each pixel adds
// 9 terms to the sums of its face axis (27 in all) instead of 27 terms of a
// dense J.  B is orthogonal: the ridged system is solved in the world frame
// (same trace, same ridge) and the step is rotated back, xi = B xi_w.
#include "kernels.h"
#include "lm_dev.cuh"

namespace rl {

constexpr int ICP_THREADS = 256;
constexpr int ICP_WARPS = ICP_THREADS / 32;
// Sums per face axis a (i1 = a+1, i2 = a+2 mod 3; the rotational entries of
// J_w are P1 = q'[i2] at w[i1] and P2 = -q'[i1] at w[i2]): count, P1, P2,
// P1^2, P2^2, P1 P2, r, P1 r, P2 r.
constexpr int ICP_NS = 27;

template <int O>
__device__ __forceinline__ void icp_add(float acc[ICP_NS], float P1, float P2, float r) {
    acc[O] += 1.f;
    acc[O + 1] += P1;
    acc[O + 2] += P2;
    acc[O + 3] = fmaf(P1, P1, acc[O + 3]);
    acc[O + 4] = fmaf(P2, P2, acc[O + 4]);
    acc[O + 5] = fmaf(P1, P2, acc[O + 5]);
    acc[O + 6] += r;
    acc[O + 7] = fmaf(P1, r, acc[O + 7]);
    acc[O + 8] = fmaf(P2, r, acc[O + 8]);
}

// One live pixel (u, v) against the pose (R, t): adds its point-to-plane
// terms to acc when it has a model point within sqrt(dist2).  INSIDE: the
// camera centre lies strictly inside the box (known per pose), so the first
// face hit is the exit face, s = min over axes of the distance to the face
// the ray heads for; otherwise the general slab test (exit from inside,
// entry from outside).  exit_num[ax] = (hi - t, t - lo) for the two ray
// directions.
template <bool INSIDE>
__device__ __forceinline__ void icp_pixel(const IcpArgs &a, float d, int u, int v, float cx, float cy, float ifx,
                                          float ify, const float R[9], const float t[3], const float exit_hi[3],
                                          const float exit_lo[3], float dist2, float acc[ICP_NS], int &n_in,
                                          int &n_valid) {
    if (!(d > 0.f) || isinf(d)) return;
    ++n_valid;
    const float c0 = ((float)u - cx) * ifx, c1 = ((float)v - cy) * ify;
    float dir[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) dir[r] = fmaf(R[3 * r], c0, fmaf(R[3 * r + 1], c1, R[3 * r + 2]));
    float sh;
    int ax;
    if (INSIDE) {
        // exit distance along axis k: e_k / |dir_k| (e_k > 0); the smallest is
        // found by cross-multiplication (a zero |dir_k| never wins), then one
        // division
        float na = dir[0] > 0.f ? exit_hi[0] : exit_lo[0], da = fabsf(dir[0]);
        ax = 0;
#pragma unroll
        for (int k = 1; k < 3; ++k) {
            const float nk = dir[k] > 0.f ? exit_hi[k] : exit_lo[k], dk = fabsf(dir[k]);
            if (nk * da < na * dk) { na = nk; da = dk; ax = k; }
        }
        sh = __fdividef(na, da);
    } else {
        float tn = -INFINITY, tf = INFINITY;
        int an = 0, af = 0;
        bool hit = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (dir[k] == 0.f) {
                hit = hit && t[k] >= a.lo[k] && t[k] <= a.hi[k];
                continue;
            }
            const float inv = __fdividef(1.0f, dir[k]);
            const float t1 = (a.lo[k] - t[k]) * inv, t2 = (a.hi[k] - t[k]) * inv;
            const float tmin = fminf(t1, t2), tmax = fmaxf(t1, t2);
            if (tmin > tn) { tn = tmin; an = k; }
            if (tmax < tf) { tf = tmax; af = k; }
        }
        if (!hit || tn > tf || !(tf > 0.f)) return;
        sh = tn > 0.f ? tn : tf;
        ax = tn > 0.f ? an : af;
    }
    const float gap = d - sh;
    const float dd2 = fmaf(dir[0], dir[0], fmaf(dir[1], dir[1], dir[2] * dir[2]));
    if (gap * gap * dd2 > dist2) return;
    // q' = d dir (the camera point rotated into the world frame); residual
    // r = n . (q - p) = gap dir[ax]
    const float q0 = d * dir[0], q1 = d * dir[1], q2 = d * dir[2];
    // neighbouring pixels of a warp mostly share a face, so the branch on
    // the axis rarely diverges; constant offsets keep acc in registers
    if (ax == 0)
        icp_add<0>(acc, q2, -q1, gap * dir[0]);
    else if (ax == 1)
        icp_add<9>(acc, q0, -q2, gap * dir[1]);
    else
        icp_add<18>(acc, q1, -q0, gap * dir[2]);
    ++n_in;
}

// The thread's pixels of one level: grid cells (iu, iv) ICP_THREADS apart
// in row-major order, stepped without divisions; ICP_LOADS depths are loaded
// before any is used, so that their latencies overlap.
constexpr int ICP_LOADS = 4;

template <bool INSIDE>
__device__ __forceinline__ void icp_sweep(const Frame &fr, const IcpArgs &a, int iu, int iv, int du, int dv, int nu,
                                          int nv, int st, float ifx, float ify, const float R[9], const float t[3],
                                          const float exit_hi[3], const float exit_lo[3], float dist2,
                                          float acc[ICP_NS], int &n_in, int &n_valid) {
    while (iv < nv) {
        float dk[ICP_LOADS];
        int uk[ICP_LOADS], vk[ICP_LOADS];
#pragma unroll
        for (int j = 0; j < ICP_LOADS; ++j) {
            uk[j] = iu * st;
            vk[j] = iv * st;
            dk[j] = iv < nv ? fr.depth[(size_t)vk[j] * fr.W + uk[j]] : 0.f;  // 0: no pixel
            iu += du;
            iv += dv;
            if (iu >= nu) {
                iu -= nu;
                ++iv;
            }
        }
#pragma unroll
        for (int j = 0; j < ICP_LOADS; ++j)
            icp_pixel<INSIDE>(a, dk[j], uk[j], vk[j], fr.cx, fr.cy, ifx, ify, R, t, exit_hi, exit_lo, dist2, acc,
                              n_in, n_valid);
    }
}

// One Gauss-Newton step from the reduced per-axis sums (thread 0 only; kept
// out of line so that its FP64 temporaries do not raise the pixel loop's
// register count): assembles the world-frame system, solves (A_w + lambda I)
// xi_w = -g_w with lambda = ridge * trace / 6, rotates the step into the
// camera frame and sets H <- H exp(xi).  False when there are fewer than 6
// inliers or the system is not positive definite.
__device__ __noinline__ bool icp_step(double *sH, const double *s_tot, double ridge) {
    double A[36], g[6], xi[6];
    for (int k = 0; k < 36; ++k) A[k] = 0.0;
    for (int k = 0; k < 6; ++k) g[k] = 0.0;
    double n_in = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double *S = s_tot + 9 * a;
        const int w1 = 3 + (a + 1) % 3, w2 = 3 + (a + 2) % 3;
        n_in += S[0];
        A[7 * a] += S[0];
        A[6 * a + w1] += S[1]; A[6 * w1 + a] += S[1];
        A[6 * a + w2] += S[2]; A[6 * w2 + a] += S[2];
        A[7 * w1] += S[3];
        A[7 * w2] += S[4];
        A[6 * w1 + w2] += S[5]; A[6 * w2 + w1] += S[5];
        g[a] -= S[6];
        g[w1] -= S[7];
        g[w2] -= S[8];
    }
    if (n_in < 6.0) return false;
    const double lam = ridge * (A[0] + A[7] + A[14] + A[21] + A[28] + A[35]) / 6.0;
    for (int r = 0; r < 6; ++r) A[7 * r] += lam;
    double xw[6];
    if (!chol_solve6(A, g, xw)) return false;
    // xi = diag(R^T, R^T) xi_w
    for (int r = 0; r < 3; ++r) {
        xi[r] = sH[r] * xw[0] + sH[4 + r] * xw[1] + sH[8 + r] * xw[2];
        xi[3 + r] = sH[r] * xw[3] + sH[4 + r] * xw[4] + sH[8 + r] * xw[5];
    }
    // H <- H exp(xi): exp(xi) as the left update of the identity
    double E[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0}, N[12];
    se3_left(xi, E);
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 4; ++q)
            N[4 * r + q] = sH[4 * r] * E[q] + sH[4 * r + 1] * E[4 + q] + sH[4 * r + 2] * E[8 + q] +
                           (q == 3 ? sH[4 * r + 3] : 0.0);
    for (int q = 0; q < 12; ++q) sH[q] = N[q];
    return true;
}

__global__ void __launch_bounds__(ICP_THREADS, 3) k_icp(IcpArgs a) {
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
        const int nu = (fr.W + st - 1) / st, nv = (fr.H + st - 1) / st;
        const float dist2 = a.ip.dist[l] * a.ip.dist[l];
        // the level's pixels (column iu, row iv of the strided grid) visited
        // ICP_THREADS apart in row-major order, stepped without divisions
        const int du = nu > 0 ? ICP_THREADS % nu : 0, dv = nu > 0 ? ICP_THREADS / nu : 0;
        const int iu0 = nu > 0 ? tid % nu : 0, iv0 = nu > 0 ? tid / nu : nv;
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
            float exit_hi[3], exit_lo[3];
            bool inside = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                exit_hi[k] = a.hi[k] - t[k];
                exit_lo[k] = t[k] - a.lo[k];
                inside = inside && exit_hi[k] > 0.f && exit_lo[k] > 0.f;
            }
            if (inside)  // the same for every thread of the block
                icp_sweep<true>(fr, a, iu0, iv0, du, dv, nu, nv, st, ifx, ify, R, t, exit_hi, exit_lo, dist2, acc,
                                n_in, n_valid);
            else
                icp_sweep<false>(fr, a, iu0, iv0, du, dv, nu, nv, st, ifx, ify, R, t, exit_hi, exit_lo, dist2, acc,
                                 n_in, n_valid);
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
            if (tid == 0 && !icp_step(sH, s_tot, a.ip.ridge)) s_fail = 1;
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
