// Really Quick Shift clustering of leaf reservoirs and the leaf mode store
// (Sec. 3.2.2, step 3).  One block per leaf; the leaf's reservoir is staged
// in shared memory.  Compiled with --fmad=false.
//
// The clustering decisions (density order, parent within tau_c, nearest
// parent) are those of the FP64 definition: densities summed in index order
// from FP64 exp, squared distances in FP64.  GB300 runs FP64 at about 1/64 of
// its FP32 rate, so the O(n^2) loops run in FP32 with a certified error bound
// and fall back to the FP64 value only where the bound cannot decide:
//  - densities: FP32 expf of an FP32 argument x, each row summed with
//    Kahan compensation; with t = exp(x), S = sum of t |x| (summed alongside)
//    and rho the density, |rho32 - rho64| <= 9.6e-7 S + 1.32e-6 rho: expf
//    within 4 ulp (4.8e-7 relative) and x within 8 ulp relative (4.8e-7 |x|,
//    so 4.8e-7 t |x| per term), the compensated sum within 2 ulp of rho and
//    the final rounding to float within 0.5 ulp, all doubled;
//  - a density comparison whose difference lies within the two bounds marks
//    both points; their FP64 densities are then computed exactly as the
//    definition does and the parents of the affected points are recomputed;
//  - squared distances in FP32 are within 5e-7 relative of the FP64 value;
//    tests against tau_c^2 or against the current nearest candidate closer
//    than 1e-6 relative are redone in FP64.
// Cluster statistics and the covariance factor are FP64, members in index
// order, so the modes are identical to the FP64 definition's.
#include "internal.h"

namespace rl {

struct RqsArgs {
    const float4 *res;
    const uint32_t *res_count;
    int kappa, m_max, min_cluster_size, n_leaves, fp16;
    double inv2s2, tau2, cov_eps;
    int64_t begin;
    uint8_t *nmodes;
    float4 *centroid;
    ushort4 *mpos_h;
    float4 *mpos_f;
    uchar4 *mrgb;
    float4 *mU;
    int32_t *msize;
};

// Upper Cholesky factor U (U^T U = S) of S = (cov + eps I)^-1.
__device__ void inverse_cov_factor(const double cv[6], double eps, double U[6]) {
    const double a = cv[0] + eps, b = cv[1], c = cv[2];
    const double d = cv[3] + eps, e = cv[4], f = cv[5] + eps;
    const double A = d * f - e * e, B = c * e - b * f, C = b * e - c * d;
    const double det = a * A + b * B + c * C;
    const double s00 = A / det, s01 = B / det, s02 = C / det;
    const double s11 = (a * f - c * c) / det, s12 = (b * c - a * e) / det;
    const double s22 = (a * d - b * b) / det;
    const double l00 = sqrt(s00);
    const double l10 = s01 / l00, l20 = s02 / l00;
    const double l11 = sqrt(s11 - l10 * l10);
    const double l21 = (s12 - l20 * l10) / l11;
    const double l22 = sqrt(s22 - l20 * l20 - l21 * l21);
    U[0] = l00; U[1] = l10; U[2] = l20; U[3] = l11; U[4] = l21; U[5] = l22;
}

__device__ __forceinline__ double dist2(const float4 a, const float4 b) {
    const double ex = (double)a.x - (double)b.x;
    const double ey = (double)a.y - (double)b.y;
    const double ez = (double)a.z - (double)b.z;
    return (ex * ex + ey * ey) + ez * ez;
}

__device__ __forceinline__ float dist2f(const float4 a, const float4 b) {
    const float ex = a.x - b.x, ey = a.y - b.y, ez = a.z - b.z;
    return (ex * ex + ey * ey) + ez * ez;
}

// Parent of point i: the nearest point j of higher density (equal density:
// lower index) with squared distance <= tau2.  Densities come with error
// bounds err (0 for exact FP64 values): a pair the bounds cannot order is
// decided exactly when both points have FP64 densities (exact != null marks
// them), otherwise both points are marked in need64 and *any64 is set.
__device__ int rqs_parent(const RqsArgs &a, const float4 *pts, const double *rho, const float *rhof,
                          const float *err, int *need64, const int *exact, int n, int i, int *any64) {
    const float4 pi = pts[i];
    const float ri = rhof[i], ei = err[i];
    const float tau2f = (float)a.tau2;
    int best = -1;
    float bd = 0.f;
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        // FP32 density order: err covers the FP32 sum and its rounding to
        // float; the factor covers the FP32 subtraction and addition
        const float rj = rhof[j];
        bool higher;
        if (fabsf(rj - ri) > (ei + err[j]) * 1.0001f) {
            higher = rj > ri;
        } else if (exact && exact[j]) {
            higher = rho[j] > rho[i] || (rho[j] == rho[i] && j < i);
        } else {
            need64[i] = 1;
            need64[j] = 1;
            if (any64) *any64 = 1;
            continue;
        }
        if (!higher) continue;
        const float d2 = dist2f(pi, pts[j]);
        // FP32 squared distances are within 5e-7 relative of FP64
        if (fabsf(d2 - tau2f) <= 1e-6f * tau2f) {
            if (dist2(pi, pts[j]) > a.tau2) continue;
        } else if (d2 > tau2f) {
            continue;
        }
        if (best < 0 || d2 < bd * (1.f - 1e-6f)) {
            best = j;
            bd = d2;
        } else if (d2 <= bd * (1.f + 1e-6f) && dist2(pi, pts[j]) < dist2(pi, pts[best])) {
            best = j;
            bd = d2;
        }
    }
    return best;
}

// Shared memory: pts[kappa] float4, rho[kappa] double, parent/root/csize/
// crank/need64[kappa] int, err/rhof[kappa] float, cl_root[64], mu[64][3]
// double.
__global__ void __launch_bounds__(256) k_rqs(RqsArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int K = a.kappa;
    float4 *pts = (float4 *)smem;
    double *rho = (double *)(pts + K);
    int *parent = (int *)(rho + K);
    int *root = parent + K;
    int *csize = root + K;
    int *crank = csize + K;
    int *need64 = crank + K;
    float *err = (float *)(need64 + K);
    float *rhof = err + K;
    int *cl_root = (int *)(rhof + K + (K & 1));  // [64]; keeps mu 8-byte aligned for odd kappa
    double *mu = (double *)(cl_root + 64);  // [64][3]
    __shared__ int n_qual, any64;

    const int L = (int)((a.begin + blockIdx.x) % a.n_leaves);
    const uint32_t cnt = a.res_count[L];
    const int n = cnt < (uint32_t)K ? (int)cnt : K;
    const int tid = threadIdx.x, nt = blockDim.x;

    for (int i = tid; i < n; i += nt) {
        pts[i] = a.res[(size_t)L * K + i];
        csize[i] = 0;
    }
    if (tid == 0) n_qual = 0;
    __syncthreads();
    // Parzen density in FP32 with its error bound (see the file comment).
    const float c32 = (float)a.inv2s2;
    for (int i = tid; i < n; i += nt) {
        const float4 pi = pts[i];
        float sum = 0.f, comp = 0.f, sx = 0.f;  // Kahan sum of t, plain sum of t |x|
        for (int j = 0; j < n; ++j) {
            const float x = dist2f(pi, pts[j]) * c32;
            const float t = expf(-x);
            sx += t * x;
            const float yk = t - comp;
            const float tk = sum + yk;
            comp = (tk - sum) - yk;
            sum = tk;
        }
        rho[i] = (double)sum;
        rhof[i] = sum;
        err[i] = 9.6e-7f * sx + 1.32e-6f * sum + 1e-30f * (float)n;
        need64[i] = 0;
    }
    if (tid == 0) any64 = 0;
    __syncthreads();
    // Parent: nearest point of higher density within tau_c (ties: lower
    // index).  Density pairs the bounds cannot order are left to the FP64
    // pass below.
    for (int i = tid; i < n; i += nt) parent[i] = rqs_parent(a, pts, rho, rhof, err, need64, nullptr, n, i, &any64);
    __syncthreads();
    if (any64) {
        // exact FP64 densities of the marked points, as the definition sums them
        for (int i = tid; i < n; i += nt) {
            if (!need64[i]) continue;
            const float4 pi = pts[i];
            double r = 0.0;
            for (int j = 0; j < n; ++j) r += exp(-(dist2(pi, pts[j]) * a.inv2s2));
            rho[i] = r;
            rhof[i] = (float)r;
            err[i] = (float)(1.2e-7 * r);  // the rounding to float only
        }
        __syncthreads();
        // parents of the points that took part in an undecided comparison
        for (int i = tid; i < n; i += nt)
            if (need64[i]) parent[i] = rqs_parent(a, pts, rho, rhof, err, need64, need64, n, i, nullptr);
        __syncthreads();
    }
    for (int i = tid; i < n; i += nt) {
        int r = i;
        while (parent[r] >= 0) r = parent[r];
        root[i] = r;
        atomicAdd(&csize[r], 1);
    }
    __syncthreads();
    // Rank the qualifying clusters by (size desc, root asc).
    for (int r = tid; r < n; r += nt) {
        crank[r] = -1;
        if (parent[r] >= 0 || csize[r] < a.min_cluster_size) continue;
        const int sr = csize[r];
        int rank = 0;
        for (int q = 0; q < n; ++q)
            if (parent[q] < 0 && csize[q] >= a.min_cluster_size &&
                (csize[q] > sr || (csize[q] == sr && q < r)))
                ++rank;
        crank[r] = rank;
        atomicAdd(&n_qual, 1);
        if (rank < a.m_max) cl_root[rank] = r;
    }
    __syncthreads();
    const int kept = min(n_qual, a.m_max);
    // Per-cluster statistics, members summed in index order.
    if (tid < kept) {
        const int k = tid, r = cl_root[k];
        double sx = 0, sy = 0, sz = 0;
        long sr = 0, sg = 0, sb = 0;
        int c = 0;
        for (int i = 0; i < n; ++i) {
            if (root[i] != r) continue;
            const float4 p = pts[i];
            sx += (double)p.x;
            sy += (double)p.y;
            sz += (double)p.z;
            const uint32_t rgb = __float_as_uint(p.w);
            sr += rgb & 255;
            sg += (rgb >> 8) & 255;
            sb += (rgb >> 16) & 255;
            ++c;
        }
        const double m0 = sx / c, m1 = sy / c, m2 = sz / c;
        double cv[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            if (root[i] != r) continue;
            const float4 p = pts[i];
            const double e0 = (double)p.x - m0, e1 = (double)p.y - m1, e2 = (double)p.z - m2;
            cv[0] += e0 * e0; cv[1] += e0 * e1; cv[2] += e0 * e2;
            cv[3] += e1 * e1; cv[4] += e1 * e2; cv[5] += e2 * e2;
        }
        for (int q = 0; q < 6; ++q) cv[q] = c > 1 ? cv[q] / (double)(c - 1) : 0.0;
        mu[3 * k + 0] = m0;
        mu[3 * k + 1] = m1;
        mu[3 * k + 2] = m2;
        double U[6];
        inverse_cov_factor(cv, a.cov_eps, U);
        const size_t e = (size_t)L * a.m_max + k;
        a.mU[2 * e] = make_float4((float)U[0], (float)U[1], (float)U[2], (float)U[3]);
        a.mU[2 * e + 1] = make_float4((float)U[4], (float)U[5], 0.f, 0.f);
        a.mrgb[e] = make_uchar4((uint8_t)((sr + c / 2) / c), (uint8_t)((sg + c / 2) / c),
                                (uint8_t)((sb + c / 2) / c), 0);
        a.msize[e] = c;
    }
    __syncthreads();
    // Per-leaf FP32 centroid of the kept modes; positions as FP16 offsets.
    __shared__ float cen[3];
    if (tid == 0) {
        double c0 = 0, c1 = 0, c2 = 0;
        for (int k = 0; k < kept; ++k) {
            c0 += mu[3 * k];
            c1 += mu[3 * k + 1];
            c2 += mu[3 * k + 2];
        }
        cen[0] = kept > 0 ? (float)(c0 / kept) : 0.f;
        cen[1] = kept > 0 ? (float)(c1 / kept) : 0.f;
        cen[2] = kept > 0 ? (float)(c2 / kept) : 0.f;
        a.centroid[L] = make_float4(cen[0], cen[1], cen[2], 0.f);
        a.nmodes[L] = (uint8_t)kept;
    }
    __syncthreads();
    for (int k = tid; k < a.m_max; k += nt) {
        const size_t e = (size_t)L * a.m_max + k;
        if (k >= kept) {
            if (a.fp16) a.mpos_h[e] = make_ushort4(0, 0, 0, 0);
            else a.mpos_f[e] = make_float4(0, 0, 0, 0);
            a.mrgb[e] = make_uchar4(0, 0, 0, 0);
            a.mU[2 * e] = make_float4(0, 0, 0, 0);
            a.mU[2 * e + 1] = make_float4(0, 0, 0, 0);
            a.msize[e] = 0;
            continue;
        }
        if (a.fp16) {
            const __half hx = __double2half(mu[3 * k + 0] - (double)cen[0]);
            const __half hy = __double2half(mu[3 * k + 1] - (double)cen[1]);
            const __half hz = __double2half(mu[3 * k + 2] - (double)cen[2]);
            a.mpos_h[e] = make_ushort4(__half_as_ushort(hx), __half_as_ushort(hy),
                                       __half_as_ushort(hz), 0);
        } else {
            a.mpos_f[e] = make_float4((float)mu[3 * k], (float)mu[3 * k + 1], (float)mu[3 * k + 2], 0.f);
        }
    }
}

static size_t rqs_smem(int kappa) {
    return (size_t)kappa * (sizeof(float4) + sizeof(double) + 5 * sizeof(int) + 2 * sizeof(float)) +
           (size_t)(kappa & 1) * sizeof(float) + 64 * sizeof(int) +
           64 * 3 * sizeof(double);
}

rl_status update_modes(rl_forest *f, int64_t begin, int64_t count, cudaStream_t s) {
    if (count <= 0) return RL_OK;
    const rl_forest_params &p = f->p;
    RqsArgs a;
    a.res = f->res;
    a.res_count = f->res_count;
    a.kappa = p.kappa;
    a.m_max = p.m_max;
    a.min_cluster_size = p.min_cluster_size;
    a.n_leaves = f->n_leaves;
    a.fp16 = p.mode_precision == RL_MODES_FP16_OFFSET;
    const double sg = (double)p.sigma, tc = (double)p.tau_c;
    a.inv2s2 = 1.0 / (2.0 * sg * sg);
    a.tau2 = tc * tc;
    a.cov_eps = (double)p.cov_eps;
    a.begin = begin;
    a.nmodes = f->nmodes;
    a.centroid = f->centroid;
    a.mpos_h = f->mpos_h;
    a.mpos_f = f->mpos_f;
    a.mrgb = f->mrgb;
    a.mU = f->mU;
    a.msize = f->msize;
    const size_t sm = rqs_smem(p.kappa);
    RL_CK(cudaFuncSetAttribute(k_rqs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    // Grid dimension x is limited to 2^31-1; leaves per launch are chunked.
    for (int64_t off = 0; off < count; off += (1 << 30)) {
        const int64_t n = count - off < (1 << 30) ? count - off : (1 << 30);
        a.begin = begin + off;
        k_rqs<<<(unsigned)n, 256, sm, s>>>(a);
        RL_LAUNCH_CK();
    }
    return RL_OK;
}

}  // namespace rl
