// Device helpers of the Levenberg-Marquardt refinement (Sec. 3.2.3): the
// normal-equation terms of one correspondence, the damped 6x6 solve and the
// SE(3) update, both in FP64.
#pragma once
#include <math.h>

#include "internal.h"

namespace rl {

// A preemptive round runs while more than k_out hypotheses remain (or more
// than one when halving continues to a single hypothesis).
__device__ __forceinline__ bool round_active(int n, const RParams &p) {
    return n > p.k_out || (p.halve_to_one && n > 1);
}

// Adds one correspondence to the normal equations: residual r = U (y - mu)
// with y = H x the transformed camera point, mu the mode mean and U the
// upper Cholesky factor of its precision (U = I without covariances); the
// Jacobian of r with respect to a left perturbation exp(xi^) H, xi =
// (t, w), is U [I | -[y]x].  acc: 21 entries of the upper triangle of J^T J
// (row-major), 6 of J^T r, then the cost r^T r.
__device__ __forceinline__ void lm_accumulate(float y0, float y1, float y2, float v0, float v1, float v2,
                                              float U00, float U01, float U02, float U11, float U12,
                                              float U22, float acc[28]) {
    const float j0[6] = {U00, U01, U02, U02 * y1 - U01 * y2, U00 * y2 - U02 * y0, U01 * y0 - U00 * y1};
    const float j1[6] = {0.f, U11, U12, U12 * y1 - U11 * y2, -U12 * y0, U11 * y0};
    const float j2[6] = {0.f, 0.f, U22, U22 * y1, -U22 * y0, 0.f};
    const float rr0 = fmaf(U00, v0, fmaf(U01, v1, U02 * v2));
    const float rr1 = fmaf(U11, v1, U12 * v2);
    const float rr2 = U22 * v2;
    int k = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c, ++k)
            acc[k] = fmaf(j0[r], j0[c], fmaf(j1[r], j1[c], fmaf(j2[r], j2[c], acc[k])));
#pragma unroll
    for (int r = 0; r < 6; ++r) acc[21 + r] = fmaf(j0[r], rr0, fmaf(j1[r], rr1, fmaf(j2[r], rr2, acc[21 + r])));
    acc[27] = fmaf(rr0, rr0, fmaf(rr1, rr1, fmaf(rr2, rr2, acc[27])));
}

// Solves A x = b for symmetric positive definite A (row-major 6x6) by
// Cholesky.  One reciprocal square root per pivot gives both the pivot
// (s / sqrt s) and its reciprocal, so no entry needs a division.
__device__ __forceinline__ bool chol_solve6(const double A[36], const double b[6], double x[6]) {
    double L[36], inv[6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            double s = A[6 * i + j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                const double rs = rsqrt(s);
                L[6 * i + i] = s * rs;
                inv[i] = rs;
            } else {
                L[6 * i + j] = s * inv[j];
            }
        }
    double y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double s = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
        y[i] = s * inv[i];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
        x[i] = s * inv[i];
    }
    return true;
}

// H <- exp(xi^) H with xi = (t, w): R = I + A K + B K^2, V = I + B K + C K^2
// (K = [w]x, th = |w|, A = sin th / th, B = (1 - cos th) / th^2,
// C = (th - sin th) / th^3).  For th < 1/4 the three coefficients come from
// their Taylor series in th^2 (seven terms: truncation below 1e-17), which
// spares the FP64 sine and cosine on the usual small LM steps.
__device__ __forceinline__ void se3_left(const double xi[6], double H[12]) {
    const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double A, B, C;
    if (th2 < 0.0625) {
        // coefficients x^k / (2k+1)!, x^k / (2k+2)!, x^k / (2k+3)! with alternating signs
        A = 1.0 + th2 * (-1.0 / 6 + th2 * (1.0 / 120 + th2 * (-1.0 / 5040 + th2 * (1.0 / 362880 +
            th2 * (-1.0 / 39916800 + th2 * (1.0 / 6227020800.0))))));
        B = 0.5 + th2 * (-1.0 / 24 + th2 * (1.0 / 720 + th2 * (-1.0 / 40320 + th2 * (1.0 / 3628800 +
            th2 * (-1.0 / 479001600 + th2 * (1.0 / 87178291200.0))))));
        C = 1.0 / 6 + th2 * (-1.0 / 120 + th2 * (1.0 / 5040 + th2 * (-1.0 / 362880 + th2 * (1.0 / 39916800 +
            th2 * (-1.0 / 6227020800.0 + th2 * (1.0 / 1307674368000.0))))));
    } else {
        const double th = sqrt(th2);
        double s, c;
        sincos(th, &s, &c);
        A = s / th;
        B = (1.0 - c) / th2;
        C = (th - s) / (th2 * th);
    }
    const double K[9] = {0, -w2, w1, w2, 0, -w0, -w1, w0, 0};
    double K2[9], Rd[9], Vd[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double I = (i % 4 == 0) ? 1.0 : 0.0;
        Rd[i] = I + A * K[i] + B * K2[i];
        Vd[i] = I + B * K[i] + C * K2[i];
    }
    double N[12];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const double td = Vd[3 * r] * xi[0] + Vd[3 * r + 1] * xi[1] + Vd[3 * r + 2] * xi[2];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            N[4 * r + c] = Rd[3 * r] * H[c] + Rd[3 * r + 1] * H[4 + c] + Rd[3 * r + 2] * H[8 + c];
        N[4 * r + 3] = Rd[3 * r] * H[3] + Rd[3 * r + 1] * H[7] + Rd[3 * r + 2] * H[11] + td;
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) H[i] = N[i];
}

// The same damped step computed by the 16 lanes of a half-warp for one
// hypothesis (q = lane % 16; every lane of the warp must call it, since it
// shuffles across the whole warp).  A warp instruction holds the narrow FP64
// pipe for the same time whatever its active lanes, so spreading one
// hypothesis's solve over lanes shortens it by the parallel width of each
// step: the Cholesky factorisation goes column by column (lane q holds
// column 0's entry (q, 0) in c0 and one entry of the trailing 5x5 block in
// a), the two triangular solves column by column too, and the SE(3) update
// has one lane per entry of R, V and the new pose.
//
// T: the hypothesis's sums (21 J^T J upper triangle, 6 J^T r, ...), lambda
// its damping, H its pose (row-major 3x4).  Returns, on every lane of the
// half-warp, whether the step stops the hypothesis (factorisation failed or
// step norm below lm_stop); otherwise lanes q < 12 return the new pose's
// entry q in Nq.
__device__ __forceinline__ double shfl16(double v, int src) { return __shfl_sync(0xffffffffu, v, src, 16); }

// position of entry (i, j), 1 <= j <= i <= 5, in the trailing block, column by column
__device__ __forceinline__ int tri_idx(int i, int j) { return (j - 1) * 6 - (j - 1) * j / 2 + (i - j); }

__device__ __forceinline__ bool lm_step_half(const float *T, double lambda, const double *H, double lm_stop, int q,
                                             double &Nq) {
    // the trailing-block entry (ai, aj) of this lane (lane 15 repeats (5, 5))
    int ai = 5, aj = 5;
    {
        int r = q;
#pragma unroll
        for (int j = 1; j <= 5; ++j) {
            if (r >= 0 && r < 6 - j) {
                aj = j;
                ai = j + r;
            }
            r -= 6 - j;
        }
    }
    // damped normal equations: A = J^T J + lambda diag(J^T J), b = -J^T r
    double c0 = 0.0, yb = 0.0;
    if (q < 6) {
        c0 = (double)T[q];  // A(q, 0) = upper-triangle entry (0, q)
        if (q == 0) c0 += lambda * c0;
        yb = -(double)T[21 + q];
    }
    double a = (double)T[aj * 6 - aj * (aj - 1) / 2 + (ai - aj)];
    if (ai == aj) a += lambda * a;

    // Cholesky A = L L^T, right-looking
    bool ok = true;
    double inv_q = 0.0;  // 1 / L(q, q) on lanes q < 6
    {
        const double d = shfl16(c0, 0);
        ok = ok && d > 0.0;
        const double rs = rsqrt(d);
        c0 *= rs;
        if (q == 0) inv_q = rs;
        const double li = shfl16(c0, ai), lj = shfl16(c0, aj);
        a = fma(-li, lj, a);
    }
#pragma unroll
    for (int k = 1; k < 6; ++k) {
        const double d = shfl16(a, tri_idx(k, k));
        ok = ok && d > 0.0;
        const double rs = rsqrt(d);
        if (q == k) inv_q = rs;
        if (aj == k) a *= rs;
        if (k < 5) {
            const bool upd = aj > k;
            const double li = shfl16(a, upd ? tri_idx(ai, k) : 0);
            const double lj = shfl16(a, upd ? tri_idx(aj, k) : 0);
            if (upd) a = fma(-li, lj, a);
        }
    }
    // L y = b (lane i < 6 holds b_i, then y_i)
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (q == k) yb *= inv_q;
        const double yk = shfl16(yb, k);
        const bool upd = q > k && q < 6;
        const double lik = k == 0 ? shfl16(c0, q) : shfl16(a, upd ? tri_idx(q, k) : 0);
        if (upd) yb = fma(-lik, yk, yb);
    }
    // L^T x = y (lane i < 6 then holds x_i)
#pragma unroll
    for (int k = 5; k >= 0; --k) {
        if (q == k) yb *= inv_q;
        if (k > 0) {
            const double xk = shfl16(yb, k);
            const double l0 = shfl16(c0, k);
            const double l1 = shfl16(a, q >= 1 && q < k ? tri_idx(k, q) : 0);
            if (q < k) yb = fma(-(q == 0 ? l0 : l1), xk, yb);
        }
    }
    double xi[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) xi[r] = shfl16(yb, r);
    double sn = 0.0;
#pragma unroll
    for (int r = 0; r < 6; ++r) sn += xi[r] * xi[r];
    // (no early return: the two half-warps may decide differently, and the
    // shuffles below need the whole warp)
    const bool stop = !ok || sqrt(sn) < lm_stop;

    // H <- exp(xi^) H: A, B, C on lanes 0, 1, 2 (Taylor series below th = 1/4)
    const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    const int sel = q % 3;
    double p;
    if (th2 < 0.0625) {
        constexpr double cA[7] = {1.0, -1.0 / 6, 1.0 / 120, -1.0 / 5040, 1.0 / 362880, -1.0 / 39916800,
                                  1.0 / 6227020800.0};
        constexpr double cB[7] = {0.5, -1.0 / 24, 1.0 / 720, -1.0 / 40320, 1.0 / 3628800, -1.0 / 479001600,
                                  1.0 / 87178291200.0};
        constexpr double cC[7] = {1.0 / 6, -1.0 / 120, 1.0 / 5040, -1.0 / 362880, 1.0 / 39916800,
                                  -1.0 / 6227020800.0, 1.0 / 1307674368000.0};
        p = sel == 0 ? cA[6] : sel == 1 ? cB[6] : cC[6];
#pragma unroll
        for (int k = 5; k >= 0; --k) p = fma(p, th2, sel == 0 ? cA[k] : sel == 1 ? cB[k] : cC[k]);
    } else {
        const double th = sqrt(th2);
        double sv, cv;
        sincos(th, &sv, &cv);
        p = sel == 0 ? sv / th : sel == 1 ? (1.0 - cv) / th2 : (th - sv) / (th2 * th);
    }
    const double cfA = shfl16(p, 0), cfB = shfl16(p, 1), cfC = shfl16(p, 2);
    // R = I + A K + B K^2 and V = I + B K + C K^2 (K = [w]x, K^2 = w w^T - th2 I):
    // entry (q / 3, q % 3) on lanes q < 9
    double Rd, Vd;
    {
        const int r = q / 3 < 3 ? q / 3 : 2, c = sel;
        const double wr = r == 0 ? w0 : r == 1 ? w1 : w2;
        const double wc = c == 0 ? w0 : c == 1 ? w1 : w2;
        // K(r, c): 0 on the diagonal, +-w_k off it (k the third index)
        const int k3 = 3 - r - c;
        const double wk = k3 == 0 ? w0 : k3 == 1 ? w1 : w2;
        const bool pos = (c - r == 1 || c - r == -2);
        const double Kv = r == c ? 0.0 : (pos ? -wk : wk);
        const double I = r == c ? 1.0 : 0.0;
        const double K2 = fma(wr, wc, r == c ? -th2 : 0.0);
        Rd = fma(cfB, K2, fma(cfA, Kv, I));
        Vd = fma(cfC, K2, fma(cfB, Kv, I));
    }
    // new pose entry (q / 4, q % 4) on lanes q < 12
    {
        const int r = q / 4 < 3 ? q / 4 : 2, c = q % 4;
        const double R0 = shfl16(Rd, 3 * r), R1 = shfl16(Rd, 3 * r + 1), R2 = shfl16(Rd, 3 * r + 2);
        const double V0 = shfl16(Vd, 3 * r), V1 = shfl16(Vd, 3 * r + 1), V2 = shfl16(Vd, 3 * r + 2);
        double N = R0 * H[c] + R1 * H[4 + c] + R2 * H[8 + c];
        if (c == 3) N += V0 * xi[0] + V1 * xi[1] + V2 * xi[2];
        Nq = N;
    }
    return stop;
}

}  // namespace rl
