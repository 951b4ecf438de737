// Pose of every successful hypothesis slot (Sec. 3.2.3): the accepted triple
// is re-derived from its Philox counters and the camera-to-world transform
// is fitted by Kabsch's least-squares criterion in FP64, one thread per slot
// so that every lane of the narrow FP64 pipe does useful work.
#include "hypgen_dev.cuh"
#include "kernels.h"

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

// Cofactor (I, J) of a 4x4 matrix.
template <int I, int J>
__device__ __forceinline__ double cofactor4(const double (&M)[4][4]) {
    constexpr int r0 = I == 0 ? 1 : 0, r1 = I <= 1 ? 2 : 1, r2 = I <= 2 ? 3 : 2;
    constexpr int c0 = J == 0 ? 1 : 0, c1 = J <= 1 ? 2 : 1, c2 = J <= 2 ? 3 : 2;
    const double d = M[r0][c0] * (M[r1][c1] * M[r2][c2] - M[r1][c2] * M[r2][c1]) -
                     M[r0][c1] * (M[r1][c0] * M[r2][c2] - M[r1][c2] * M[r2][c0]) +
                     M[r0][c2] * (M[r1][c0] * M[r2][c1] - M[r1][c1] * M[r2][c0]);
    return ((I + J) & 1) ? -d : d;
}

// Largest-eigenvalue eigenvector of Horn's traceless symmetric 4x4 matrix
// without iterating on the matrix: the eigenvalue is the largest root of the
// characteristic polynomial l^4 - (p2/2) l^2 - (p3/3) l + det N (Newton's
// identities with power sums p_k = tr N^k and tr N = 0), reached by Newton's
// method from the upper bound (E_A + E_B)/2; the eigenvector is a column of
// the adjugate of N - l I, which is proportional to q q^T for a simple
// eigenvalue.  Returns false when the eigenvalue is too close to the next one
// for the adjugate to be accurate (product of the gaps below 2e-3 |N|^3,
// i.e. a nearly collinear triple); the caller then uses Jacobi.
__device__ bool horn_max_eigvec_poly(const double (&N)[4][4], double bound, double q[4]) {
    double p2 = 0.0, p3 = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            p2 += N[i][j] * N[i][j];
            double nij2 = 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) nij2 += N[i][k] * N[k][j];
            p3 += nij2 * N[j][i];
        }
    const double detN = N[0][0] * cofactor4<0, 0>(N) + N[0][1] * cofactor4<0, 1>(N) +
                        N[0][2] * cofactor4<0, 2>(N) + N[0][3] * cofactor4<0, 3>(N);
    const double c2 = -0.5 * p2, c1 = -p3 / 3.0, c0 = detN;
    const double sN = sqrt(p2);
    if (!(sN > 0.0)) return false;
    double lam = fmin(bound, sN);
    for (int k = 0; k < 60; ++k) {
        const double f = ((lam * lam + c2) * lam + c1) * lam + c0;
        const double fp = (4.0 * lam * lam + 2.0 * c2) * lam + c1;
        if (!(fp > 0.0)) break;
        const double d = f / fp;
        lam -= d;
        if (fabs(d) <= 1e-15 * sN) break;
    }
    double M[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) M[i][j] = N[i][j] - (i == j ? lam : 0.0);
    const double d0 = cofactor4<0, 0>(M), d1 = cofactor4<1, 1>(M), d2 = cofactor4<2, 2>(M),
                 d3 = cofactor4<3, 3>(M);
    // adj(M) = (product of the negative gaps) q q^T: the diagonal is <= 0
    if (!(-(d0 + d1 + d2 + d3) >= 2e-3 * sN * sN * sN)) return false;
    int i = 0;
    double dm = d0;
    if (d1 < dm) { dm = d1; i = 1; }
    if (d2 < dm) { dm = d2; i = 2; }
    if (d3 < dm) { dm = d3; i = 3; }
    if (i == 0) { q[0] = d0; q[1] = cofactor4<0, 1>(M); q[2] = cofactor4<0, 2>(M); q[3] = cofactor4<0, 3>(M); }
    else if (i == 1) { q[0] = cofactor4<1, 0>(M); q[1] = d1; q[2] = cofactor4<1, 2>(M); q[3] = cofactor4<1, 3>(M); }
    else if (i == 2) { q[0] = cofactor4<2, 0>(M); q[1] = cofactor4<2, 1>(M); q[2] = d2; q[3] = cofactor4<2, 3>(M); }
    else { q[0] = cofactor4<3, 0>(M); q[1] = cofactor4<3, 1>(M); q[2] = cofactor4<3, 2>(M); q[3] = d3; }
    return true;
}

// Rigid transform (camera -> world) of three pairs by Horn's closed form
// (unit quaternion of the largest eigenvalue), which solves the same least
// squares problem as Kabsch's SVD construction.  Since the cross-covariance
// of three pairs has rank 2, the two largest eigenvalues of N differ by twice
// its smaller singular value.
__device__ void kabsch3_horn(const double a[3][3], const double b[3][3], double H[12]) {
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
    double ea = 0.0, eb = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            ea += (a[i][k] - ca[k]) * (a[i][k] - ca[k]);
            eb += (b[i][k] - cb[k]) * (b[i][k] - cb[k]);
        }
    double q[4];
    if (!horn_max_eigvec_poly(N, 0.5 * (ea + eb), q)) jacobi4_max_eigvec(N, q);
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

// The accepted triple of (slot, it), re-derived exactly, and its pose.
__device__ __forceinline__ void accept_triple(const HypArgs &a, const Frame &fr, const uint16_t *lv,
                                           const uint16_t *mc, const uint4 *pr, int slot, int it, double H[12]) {
    const int T = a.p.n_trees;
    const Draw d = draw(a, fr, slot, it, [&](int q) { return pixel_modes(mc, pr, q, T) != 0; });
    const uint32_t ctr1 = (TAG_HYP << 16) | (uint32_t)a.p.level;
    const uint4 r1 = philox(make_uint4(slot, ctr1, it, 1), fr.key0, fr.key1);
    const uint32_t u1[3] = {r1.x, r1.y, r1.z};
    double xc[3][3], xw[3][3];
    for (int i = 0; i < 3; ++i) {
        uint32_t L;
        int rank;
        lookup(a, lv, pr, d.pix[i], (int)draw_below(u1[i], (uint32_t)pixel_modes(mc, pr, d.pix[i], T)), &L, &rank);
        const float3 c = backproject(fr, d.pix[i]);
        const float3 w = mode_pos(a.mv, L, rank);
        xc[i][0] = c.x; xc[i][1] = c.y; xc[i][2] = c.z;
        xw[i][0] = w.x; xw[i][1] = w.y; xw[i][2] = w.z;
    }
    kabsch3_horn(xc, xw, H);
}


__global__ void __launch_bounds__(128) k_hyppose(HypArgs a) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (slot >= a.p.n_hyp) return;
    const int it = a.hyp_iter[(size_t)b * a.p.n_hyp + slot];
    if (it < 0) return;
    const Frame fr = a.frames[b];
    const uint16_t *lv = a.leaves + (size_t)b * a.p.n_trees * a.hw_max;
    const uint16_t *mc = a.mcount + (size_t)b * a.hw_max;
    const uint4 *pr = a.prec ? a.prec + (size_t)b * a.hw_max : nullptr;
    double H[12];
    accept_triple(a, fr, lv, mc, pr, slot, it, H);
    double *out = a.hyp_pose + ((size_t)b * a.p.n_hyp + slot) * 12;
    for (int k = 0; k < 12; ++k) out[k] = H[k];
}

rl_status launch_hyppose(const Frame *frames, const uint16_t *leaves, const uint16_t *mcount,
                         const uint4 *prec, int hw_max, ModeView mv, const RParams &p,
                         double *hyp_pose, int32_t *hyp_iter, int n, cudaStream_t s) {
    HypArgs a{frames, leaves, mcount, prec, nullptr, hw_max, mv, p, hyp_pose, hyp_iter, nullptr};
    dim3 grid((p.n_hyp + 127) / 128, n);
    k_hyppose<<<grid, 128, 0, s>>>(a);
    RL_LAUNCH_CK();
    return RL_OK;
}

}  // namespace rl
