/*
 * CPU oracle, part 3: camera pose estimation (Sec. 3.2.3), model-based
 * hypothesis ranking (Sec. 3.2.4, Eq. 6-8) and the relocalisation cascade
 * (Sec. 3.2.5).  Readings R7-R18 are listed in oracle.c.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static uint32_t below(uint32_t u, uint32_t n)
{
    return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* ---------------------------------------------------------------------- */
/* Small dense linear algebra in FP64.                                    */
/* ---------------------------------------------------------------------- */

/* Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix: on return
 * w holds the eigenvalues (descending) and V the eigenvectors as columns. */
static void jacobi_eig3(const double M[9], double w[3], double V[9])
{
    double A[9];
    memcpy(A, M, sizeof(A));
    for (int i = 0; i < 9; ++i)
        V[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        double diag = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off <= 1e-34 * diag || off == 0.0)
            break;
        static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (int k = 0; k < 3; ++k) {
            const int p = P[k][0], q = P[k][1];
            const double apq = A[3 * p + q];
            if (apq == 0.0)
                continue;
            const double theta = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            /* J = identity with J[p][p]=c, J[p][q]=s, J[q][p]=-s, J[q][q]=c */
            double J[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
            J[3 * p + p] = c; J[3 * p + q] = s; J[3 * q + p] = -s; J[3 * q + q] = c;
            double T[9], B[9], NV[9];
            for (int i = 0; i < 3; ++i)          /* T = A J */
                for (int j = 0; j < 3; ++j)
                    T[3 * i + j] = A[3 * i + 0] * J[0 + j] + A[3 * i + 1] * J[3 + j] + A[3 * i + 2] * J[6 + j];
            for (int i = 0; i < 3; ++i)          /* B = J^T T */
                for (int j = 0; j < 3; ++j)
                    B[3 * i + j] = J[0 + i] * T[0 + j] + J[3 + i] * T[3 + j] + J[6 + i] * T[6 + j];
            for (int i = 0; i < 3; ++i)          /* V = V J */
                for (int j = 0; j < 3; ++j)
                    NV[3 * i + j] = V[3 * i + 0] * J[0 + j] + V[3 * i + 1] * J[3 + j] + V[3 * i + 2] * J[6 + j];
            memcpy(A, B, sizeof(A));
            A[3 * p + q] = A[3 * q + p] = 0.0;
            memcpy(V, NV, sizeof(NV));
        }
    }
    double e[3] = {A[0], A[4], A[8]};
    int idx[3] = {0, 1, 2};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (e[idx[b]] > e[idx[a]]) { int t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
    double W[9];
    for (int c = 0; c < 3; ++c) {
        w[c] = e[idx[c]];
        for (int r = 0; r < 3; ++r)
            W[3 * r + c] = V[3 * r + idx[c]];
    }
    memcpy(V, W, sizeof(W));
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double norm3(const double a[3]) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* Kabsch (1976), reading R10: SVD of the cross-covariance A = sum a' b'^T
 * through the eigen-decomposition of A^T A. */
void orc_kabsch(const double *a, const double *b, int n, double R[9], double t[3])
{
    double ca[3] = {0, 0, 0}, cb[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            ca[k] += a[3 * i + k];
            cb[k] += b[3 * i + k];
        }
    for (int k = 0; k < 3; ++k) {
        ca[k] /= n;
        cb[k] /= n;
    }
    double A[9] = {0};
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                A[3 * r + c] += (a[3 * i + r] - ca[r]) * (b[3 * i + c] - cb[c]);
    double AtA[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            AtA[3 * r + c] = A[0 + r] * A[0 + c] + A[3 + r] * A[3 + c] + A[6 + r] * A[6 + c];
    double w[3], V[9];
    jacobi_eig3(AtA, w, V);
    /* left singular vectors: u_i = A v_i / sigma_i, u3 = u1 x u2 */
    double v1[3] = {V[0], V[3], V[6]}, v2[3] = {V[1], V[4], V[7]};
    double u1[3], u2[3], u3[3];
    for (int r = 0; r < 3; ++r) {
        u1[r] = A[3 * r + 0] * v1[0] + A[3 * r + 1] * v1[1] + A[3 * r + 2] * v1[2];
        u2[r] = A[3 * r + 0] * v2[0] + A[3 * r + 1] * v2[1] + A[3 * r + 2] * v2[2];
    }
    double n1 = norm3(u1);
    for (int r = 0; r < 3; ++r) u1[r] /= n1;
    double d12 = u1[0] * u2[0] + u1[1] * u2[1] + u1[2] * u2[2];
    for (int r = 0; r < 3; ++r) u2[r] -= d12 * u1[r];
    double n2 = norm3(u2);
    if (n2 < 1e-300) { /* collinear: any unit vector orthogonal to u1 */
        double e[3] = {fabs(u1[0]) < 0.9 ? 1.0 : 0.0, fabs(u1[0]) < 0.9 ? 0.0 : 1.0, 0.0};
        double d = e[0] * u1[0] + e[1] * u1[1];
        for (int r = 0; r < 3; ++r) u2[r] = e[r] - d * u1[r];
        n2 = norm3(u2);
    }
    for (int r = 0; r < 3; ++r) u2[r] /= n2;
    cross3(u1, u2, u3);
    double U[9] = {u1[0], u2[0], u3[0], u1[1], u2[1], u3[1], u1[2], u2[2], u3[2]};
    /* d = sign det(V U^T) = det(V) since det(U) = +1 */
    double detV = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6])
                + V[2] * (V[3] * V[7] - V[4] * V[6]);
    double D[3] = {1.0, 1.0, detV < 0 ? -1.0 : 1.0};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            R[3 * r + c] = V[3 * r + 0] * D[0] * U[3 * c + 0] + V[3 * r + 1] * D[1] * U[3 * c + 1]
                         + V[3 * r + 2] * D[2] * U[3 * c + 2];
    for (int r = 0; r < 3; ++r)
        t[r] = cb[r] - (R[3 * r + 0] * ca[0] + R[3 * r + 1] * ca[1] + R[3 * r + 2] * ca[2]);
}

/* Cholesky solve of a symmetric positive-definite 6x6 system; 0 on failure. */
int orc_chol_solve6(const double A[36], const double b[6], double x[6])
{
    double L[36] = {0};
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[6 * i + j];
            for (int k = 0; k < j; ++k)
                s -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                if (!(s > 0.0))
                    return 0;
                L[6 * i + i] = sqrt(s);
            } else {
                L[6 * i + j] = s / L[6 * j + j];
            }
        }
    }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k)
            s -= L[6 * i + k] * y[k];
        y[i] = s / L[6 * i + i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k)
            s -= L[6 * k + i] * x[k];
        x[i] = s / L[6 * i + i];
    }
    return 1;
}

/* SE(3) exponential of xi = (v, w) applied on the left: H <- exp(xi^) H. */
void orc_se3_left_update(const double xi[6], double H[12])
{
    const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2, th = sqrt(th2);
    double A, B, C;
    if (th < 1e-8) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
        C = 1.0 / 6.0 - th2 / 120.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
        C = (th - sin(th)) / (th2 * th);
    }
    const double K[9] = {0, -w2, w1, w2, 0, -w0, -w1, w0, 0};
    double K2[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            K2[3 * r + c] = K[3 * r + 0] * K[0 + c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
    double Rd[9], Vd[9];
    for (int i = 0; i < 9; ++i) {
        const double I = (i % 4 == 0) ? 1.0 : 0.0;
        Rd[i] = I + A * K[i] + B * K2[i];
        Vd[i] = I + B * K[i] + C * K2[i];
    }
    double td[3];
    for (int r = 0; r < 3; ++r)
        td[r] = Vd[3 * r + 0] * xi[0] + Vd[3 * r + 1] * xi[1] + Vd[3 * r + 2] * xi[2];
    double N[12];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c)
            N[4 * r + c] = Rd[3 * r + 0] * H[0 + c] + Rd[3 * r + 1] * H[4 + c] + Rd[3 * r + 2] * H[8 + c];
        N[4 * r + 3] = Rd[3 * r + 0] * H[3] + Rd[3 * r + 1] * H[7] + Rd[3 * r + 2] * H[11] + td[r];
    }
    memcpy(H, N, sizeof(N));
}

/* ---------------------------------------------------------------------- */
/* Frame helpers.                                                         */
/* ---------------------------------------------------------------------- */

/* x_C = D(u) K^-1 u, in FP32 with a fixed operation order (R9). */
static void backproject(const float *depth_img, int W, float fx, float fy, float cx, float cy,
                        int pix, double xc[3])
{
    const int u = pix % W, v = pix / W;
    const float d = depth_img[pix];
    xc[0] = (double)((((float)u - cx) * d) / fx);
    xc[1] = (double)((((float)v - cy) * d) / fy);
    xc[2] = (double)d;
}

/* |M(u)| (R7) */
static int mode_count(int pix, int WH, const uint16_t *leaves, int n_trees_used,
                      int leaves_per_tree, const uint8_t *nmodes, int k_top)
{
    int total = 0;
    for (int t = 0; t < n_trees_used; ++t) {
        const uint16_t leaf = leaves[(size_t)t * WH + pix];
        if (leaf == 0xFFFF)
            return 0;
        int nm = nmodes[(size_t)t * leaves_per_tree + leaf];
        total += nm < k_top ? nm : k_top;
    }
    return total;
}

/* The m-th element of M(u): global mode record index. */
static size_t mode_at(int pix, int WH, int m, const uint16_t *leaves, int n_trees_used,
                      int leaves_per_tree, const uint8_t *nmodes, int k_top, int m_max)
{
    for (int t = 0; t < n_trees_used; ++t) {
        const size_t L = (size_t)t * leaves_per_tree + leaves[(size_t)t * WH + pix];
        int nm = nmodes[L] < k_top ? nmodes[L] : k_top;
        if (m < nm)
            return L * (size_t)m_max + (size_t)m;
        m -= nm;
    }
    return (size_t)-1;
}

static void apply_pose(const double H[12], const double x[3], double y[3])
{
    for (int r = 0; r < 3; ++r)
        y[r] = H[4 * r + 0] * x[0] + H[4 * r + 1] * x[1] + H[4 * r + 2] * x[2] + H[4 * r + 3];
}

/* squared Eq. 5 distance of y to mode e (Mahalanobis via U, or Euclidean) */
static double mode_dist2(const double y[3], size_t e, const float *mpos, const float *mU, int use_cov,
                         double r_out[3])
{
    const double v0 = y[0] - (double)mpos[3 * e + 0];
    const double v1 = y[1] - (double)mpos[3 * e + 1];
    const double v2 = y[2] - (double)mpos[3 * e + 2];
    double r0 = v0, r1 = v1, r2 = v2;
    if (use_cov) {
        const float *U = mU + 6 * e;
        r0 = (double)U[0] * v0 + (double)U[1] * v1 + (double)U[2] * v2;
        r1 = (double)U[3] * v1 + (double)U[4] * v2;
        r2 = (double)U[5] * v2;
    }
    if (r_out) { r_out[0] = r0; r_out[1] = r1; r_out[2] = r2; }
    return r0 * r0 + r1 * r1 + r2 * r2;
}

/* ---------------------------------------------------------------------- */
/* Eq. 5: E(H) = sum_i min_{(mu,Sigma) in M(u_i)} |Sigma^-1/2 (H x_i - mu)| */
/* ---------------------------------------------------------------------- */
double orc_energy(const double H[12], const int32_t *pix, int n_pix,
                  const float *depth_img, int W, int Himg, float fx, float fy, float cx, float cy,
                  const uint16_t *leaves, int n_trees_used, int leaves_per_tree,
                  const uint8_t *nmodes, const float *mpos, const float *mU, int m_max,
                  int k_top, int use_cov)
{
    const int WH = W * Himg;
    double E = 0.0;
    for (int i = 0; i < n_pix; ++i) {
        if (pix[i] < 0)
            continue;
        double xc[3], y[3];
        backproject(depth_img, W, fx, fy, cx, cy, pix[i], xc);
        apply_pose(H, xc, y);
        const int nm = mode_count(pix[i], WH, leaves, n_trees_used, leaves_per_tree, nmodes, k_top);
        double best = INFINITY;
        for (int m = 0; m < nm; ++m) {
            size_t e = mode_at(pix[i], WH, m, leaves, n_trees_used, leaves_per_tree, nmodes, k_top, m_max);
            double q = mode_dist2(y, e, mpos, mU, use_cov, NULL);
            if (q < best)
                best = q;
        }
        E += sqrt(best);
    }
    return E;
}

/* ---------------------------------------------------------------------- */
/* Levenberg-Marquardt refinement in se(3) (Sec. 3.2.3, reading R15).     */
/* ---------------------------------------------------------------------- */
int orc_lm_refine(double H[12], const int32_t *pix, int n_pix,
                  const float *depth_img, int W, int Himg, float fx, float fy, float cx, float cy,
                  const uint16_t *leaves, int n_trees_used, int leaves_per_tree,
                  const uint8_t *nmodes, const float *mpos, const float *mU, int m_max,
                  int k_top, int use_cov, int max_iter, double lambda0,
                  double inlier_thresh, double stop)
{
    const int WH = W * Himg;
    size_t *corr = (size_t *)malloc(sizeof(size_t) * (size_t)(n_pix > 0 ? n_pix : 1));
    double lambda = lambda0;
    int it = 0;
    for (; it < max_iter; ++it) {
        /* correspondences at the current pose: nearest mode, inlier test */
        double JtJ[36] = {0}, g[6] = {0}, cost = 0.0;
        int n_in = 0;
        for (int i = 0; i < n_pix; ++i) {
            corr[i] = (size_t)-1;
            if (pix[i] < 0)
                continue;
            double xc[3], y[3];
            backproject(depth_img, W, fx, fy, cx, cy, pix[i], xc);
            apply_pose(H, xc, y);
            const int nm = mode_count(pix[i], WH, leaves, n_trees_used, leaves_per_tree, nmodes, k_top);
            double best = INFINITY;
            size_t be = (size_t)-1;
            for (int m = 0; m < nm; ++m) {
                size_t e = mode_at(pix[i], WH, m, leaves, n_trees_used, leaves_per_tree, nmodes, k_top, m_max);
                double q = mode_dist2(y, e, mpos, mU, use_cov, NULL);
                if (q < best) {
                    best = q;
                    be = e;
                }
            }
            if (be == (size_t)-1)
                continue;
            double eu = mode_dist2(y, be, mpos, mU, 0, NULL);
            if (eu > inlier_thresh * inlier_thresh)
                continue;
            corr[i] = be;
            ++n_in;
            double r[3];
            cost += mode_dist2(y, be, mpos, mU, use_cov, r);
            /* J = U [I | -[y]x] */
            double Jp[18] = {1, 0, 0, 0, y[2], -y[1],
                             0, 1, 0, -y[2], 0, y[0],
                             0, 0, 1, y[1], -y[0], 0};
            double J[18];
            if (use_cov) {
                const float *U = mU + 6 * be;
                for (int c = 0; c < 6; ++c) {
                    J[0 + c] = (double)U[0] * Jp[c] + (double)U[1] * Jp[6 + c] + (double)U[2] * Jp[12 + c];
                    J[6 + c] = (double)U[3] * Jp[6 + c] + (double)U[4] * Jp[12 + c];
                    J[12 + c] = (double)U[5] * Jp[12 + c];
                }
            } else {
                memcpy(J, Jp, sizeof(J));
            }
            for (int a = 0; a < 6; ++a) {
                for (int b = 0; b < 6; ++b)
                    JtJ[6 * a + b] += J[a] * J[b] + J[6 + a] * J[6 + b] + J[12 + a] * J[12 + b];
                g[a] += J[a] * r[0] + J[6 + a] * r[1] + J[12 + a] * r[2];
            }
        }
        if (n_in < 3)
            break;
        double A[36], rhs[6], step[6];
        memcpy(A, JtJ, sizeof(A));
        for (int a = 0; a < 6; ++a) {
            A[6 * a + a] += lambda * JtJ[6 * a + a];
            rhs[a] = -g[a];
        }
        if (!orc_chol_solve6(A, rhs, step))
            break;
        double sn = 0.0;
        for (int a = 0; a < 6; ++a)
            sn += step[a] * step[a];
        if (sqrt(sn) < stop)
            break;
        double Hn[12];
        memcpy(Hn, H, sizeof(Hn));
        orc_se3_left_update(step, Hn);
        /* cost at the trial pose with the same correspondences */
        double trial = 0.0;
        for (int i = 0; i < n_pix; ++i) {
            if (corr[i] == (size_t)-1)
                continue;
            double xc[3], y[3];
            backproject(depth_img, W, fx, fy, cx, cy, pix[i], xc);
            apply_pose(Hn, xc, y);
            trial += mode_dist2(y, corr[i], mpos, mU, use_cov, NULL);
        }
        if (trial < cost) {
            memcpy(H, Hn, sizeof(Hn));
            lambda /= 10.0;
        } else {
            lambda *= 10.0;
        }
    }
    free(corr);
    return it;
}

/* ---------------------------------------------------------------------- */
/* Eq. 6-7 with an analytic box scene model (reading R16).                */
/* ---------------------------------------------------------------------- */
static double ray_box_depth(const double o[3], const double d[3], const double lo[3], const double hi[3])
{
    double tn = -INFINITY, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < lo[a] || o[a] > hi[a])
                return NAN;
            continue;
        }
        double t1 = (lo[a] - o[a]) / d[a], t2 = (hi[a] - o[a]) / d[a];
        double tmin = t1 < t2 ? t1 : t2, tmax = t1 < t2 ? t2 : t1;
        if (tmin > tn) tn = tmin;
        if (tmax < tf) tf = tmax;
    }
    if (tn > tf)
        return NAN;
    if (tn > 0.0)
        return tn; /* camera outside: entry point */
    if (tf > 0.0)
        return tf; /* camera inside: exit point (first inner wall) */
    return NAN;
}

void orc_raycast_box(const double H[12], int W, int Himg, float fx, float fy, float cx, float cy,
                     const double lo[3], const double hi[3], double *out)
{
    const double o[3] = {H[3], H[7], H[11]};
    for (int v = 0; v < Himg; ++v)
        for (int u = 0; u < W; ++u) {
            const double dc[3] = {((double)u - (double)cx) / (double)fx,
                                  ((double)v - (double)cy) / (double)fy, 1.0};
            double dw[3];
            for (int r = 0; r < 3; ++r)
                dw[r] = H[4 * r + 0] * dc[0] + H[4 * r + 1] * dc[1] + H[4 * r + 2] * dc[2];
            /* the camera-frame ray has unit z, so its parameter is z-depth */
            out[(size_t)v * W + u] = ray_box_depth(o, dw, lo, hi);
        }
}

double orc_depth_score(const double H[12], const float *depth_img, int W, int Himg,
                       float fx, float fy, float cx, float cy,
                       const double lo[3], const double hi[3],
                       double *mean_abs, double *valid_frac)
{
    double *syn = (double *)malloc(sizeof(double) * (size_t)W * Himg);
    orc_raycast_box(H, W, Himg, fx, fy, cx, cy, lo, hi, syn);
    double sum = 0.0;
    long n_syn = 0, n_both = 0;
    for (long i = 0; i < (long)W * Himg; ++i) {
        if (isnan(syn[i]))
            continue;
        ++n_syn;
        if (depth_img[i] > 0.0f) {
            sum += fabs((double)depth_img[i] - syn[i]);
            ++n_both;
        }
    }
    free(syn);
    const double mu = n_both > 0 ? sum / (double)n_both : INFINITY;
    const double frac = (double)n_syn / ((double)W * Himg);
    if (mean_abs) *mean_abs = mu;
    if (valid_frac) *valid_frac = frac;
    return (frac >= 0.1 && n_both > 0) ? mu : INFINITY;
}

/* ---------------------------------------------------------------------- */
/* Sec. 3.2.3: hypothesis generation, preemptive RANSAC; Sec. 3.2.4.      */
/* ---------------------------------------------------------------------- */
typedef struct {
    double H[12];
    double E;
    int slot;
} hyp_t;

static int hyp_cmp(const void *a, const void *b)
{
    const hyp_t *x = (const hyp_t *)a, *y = (const hyp_t *)b;
    if (x->E < y->E) return -1;
    if (x->E > y->E) return 1;
    return (x->slot > y->slot) - (x->slot < y->slot);
}

/* One generation attempt (R8, R9); returns 1 and fills H on success. */
static int try_hypothesis(const orc_params *p, const uint32_t key[2], int slot, int it,
                          const float *depth_img, const uint8_t *rgb, int W, int Himg,
                          float fx, float fy, float cx, float cy,
                          const uint16_t *leaves, int leaves_per_tree,
                          const uint8_t *nmodes, const float *mpos, const uint8_t *mrgb,
                          int m_max, double H[12])
{
    const int WH = W * Himg;
    uint32_t c0[4] = {(uint32_t)slot, (3u << 16) | (uint32_t)p->level, (uint32_t)it, 0u};
    uint32_t c1[4] = {(uint32_t)slot, (3u << 16) | (uint32_t)p->level, (uint32_t)it, 1u};
    uint32_t r0[4], r1[4];
    orc_philox4x32_10(c0, key, r0);
    orc_philox4x32_10(c1, key, r1);
    int pix[3];
    size_t mode[3];
    double xc[3][3], xw[3][3];
    for (int i = 0; i < 3; ++i) {
        pix[i] = (int)below(r0[i], (uint32_t)WH);
        /* R8: a pixel without depth or with an empty M(u) fails the
         * iteration.  R8b (redraw): it is redrawn within the iteration, as
         * the batch sampler of R12 does, up to batch_attempts draws in all;
         * draw a >= 1 of pixel i takes word 0 of the Philox block with
         * counter (slot, 5 << 16 | level, it, 4a + i). */
        for (int a = 1; p->redraw && a < p->batch_attempts; ++a) {
            if (depth_img[pix[i]] > 0.0f &&
                mode_count(pix[i], WH, leaves, p->n_trees_used, leaves_per_tree, nmodes, p->k_top) > 0)
                break;
            uint32_t c2[4] = {(uint32_t)slot, (5u << 16) | (uint32_t)p->level, (uint32_t)it, 4u * (uint32_t)a + (uint32_t)i};
            uint32_t r2[4];
            orc_philox4x32_10(c2, key, r2);
            pix[i] = (int)below(r2[0], (uint32_t)WH);
        }
        if (!(depth_img[pix[i]] > 0.0f))
            return 0;
        const int nm = mode_count(pix[i], WH, leaves, p->n_trees_used, leaves_per_tree, nmodes, p->k_top);
        if (nm == 0)
            return 0;
        const int m = (int)below(r1[i], (uint32_t)nm);
        mode[i] = mode_at(pix[i], WH, m, leaves, p->n_trees_used, leaves_per_tree, nmodes, p->k_top, m_max);
        backproject(depth_img, W, fx, fy, cx, cy, pix[i], xc[i]);
        for (int a = 0; a < 3; ++a)
            xw[i][a] = (double)mpos[3 * mode[i] + a];
    }
    /* check 1: colour of one randomly chosen pair */
    const int j = (int)below(r0[3], 3);
    int linf = 0;
    for (int c = 0; c < 3; ++c) {
        int d = (int)rgb[(size_t)pix[j] * 3 + c] - (int)mrgb[3 * mode[j] + c];
        if (d < 0) d = -d;
        if (d > linf) linf = d;
    }
    if (linf > p->colour_thresh)
        return 0;
    /* check 2: scene points far enough apart; check 3: rigidity */
    static const int PA[3] = {0, 0, 1}, PB[3] = {1, 2, 2};
    double dW2[3], dC2[3];
    for (int k = 0; k < 3; ++k) {
        const int a = PA[k], b = PB[k];
        double e0 = xw[a][0] - xw[b][0], e1 = xw[a][1] - xw[b][1], e2 = xw[a][2] - xw[b][2];
        dW2[k] = (e0 * e0 + e1 * e1) + e2 * e2;
        double f0 = xc[a][0] - xc[b][0], f1 = xc[a][1] - xc[b][1], f2 = xc[a][2] - xc[b][2];
        dC2[k] = (f0 * f0 + f1 * f1) + f2 * f2;
    }
    for (int k = 0; k < 3; ++k)
        if (dW2[k] < p->min_sq_dist)
            return 0;
    for (int k = 0; k < 3; ++k)
        if (fabs(sqrt(dW2[k]) - sqrt(dC2[k])) > p->max_trans_err)
            return 0;
    double a[9], b[9], R[9], t[3];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            a[3 * i + k] = xc[i][k];
            b[3 * i + k] = xw[i][k];
        }
    orc_kabsch(a, b, 3, R, t);
    for (int r = 0; r < 3; ++r) {
        H[4 * r + 0] = R[3 * r + 0];
        H[4 * r + 1] = R[3 * r + 1];
        H[4 * r + 2] = R[3 * r + 2];
        H[4 * r + 3] = t[r];
    }
    return 1;
}

/* Pixel batch b (R12). */
static void sample_batch(const orc_params *p, const uint32_t key[2], int b,
                         const float *depth_img, int WH, const uint16_t *leaves, int leaves_per_tree,
                         const uint8_t *nmodes, int32_t *out)
{
    for (int j = 0; j < p->eta; ++j) {
        out[j] = -1;
        for (int a = 0; a < p->batch_attempts; ++a) {
            uint32_t c[4] = {(uint32_t)b, (4u << 16) | (uint32_t)p->level, (uint32_t)j, (uint32_t)a};
            uint32_t r[4];
            orc_philox4x32_10(c, key, r);
            const int pix = (int)below(r[0], (uint32_t)WH);
            if (!(depth_img[pix] > 0.0f))
                continue;
            if (mode_count(pix, WH, leaves, p->n_trees_used, leaves_per_tree, nmodes, p->k_top) == 0)
                continue;
            out[j] = pix;
            break;
        }
    }
}

/* State handed in at a stage boundary (orc_relocalise_from): the survivor
 * set replaces the oracle's own, and each survivor's Eq. 5 energy is
 * recomputed in FP64 on the pixel set of that point before the usual
 * stable sort by (E, slot). */
static const orc_resume *handin_at(const orc_resume *rs, int n_rs, int stage)
{
    for (int k = 0; k < n_rs; ++k)
        if (rs[k].stage == stage)
            return &rs[k];
    return NULL;
}

static void replace_survivors(const orc_resume *rs, hyp_t *hyp, int *n, const int32_t *I, int nI,
                              const float *depth_img, int W, int Himg, float fx, float fy,
                              float cx, float cy, const uint16_t *leaves, const orc_params *p,
                              int leaves_per_tree, const uint8_t *nmodes, const float *mpos,
                              const float *mU, int m_max)
{
    *n = rs->n;
    for (int h = 0; h < rs->n; ++h) {
        hyp[h].slot = rs->slot[h];
        memcpy(hyp[h].H, rs->pose + 12 * (size_t)h, sizeof(hyp[h].H));
        hyp[h].E = orc_energy(hyp[h].H, I, nI, depth_img, W, Himg, fx, fy, cx, cy, leaves,
                              p->n_trees_used, leaves_per_tree, nmodes, mpos, mU, m_max,
                              p->k_top, p->use_cov);
    }
    qsort(hyp, (size_t)*n, sizeof(hyp_t), hyp_cmp);
}

void orc_relocalise(const orc_params *p,
                    const float *depth_img, const uint8_t *rgb, int W, int Himg,
                    float fx, float fy, float cx, float cy,
                    const uint16_t *leaves, int n_trees_forest, int leaves_per_tree,
                    const uint8_t *nmodes, const float *mpos, const uint8_t *mrgb,
                    const float *mU, int m_max,
                    const double box_lo[3], const double box_hi[3],
                    uint64_t query_seed, orc_result *out, orc_debug *dbg)
{
    orc_relocalise_from(p, depth_img, rgb, W, Himg, fx, fy, cx, cy, leaves, n_trees_forest,
                        leaves_per_tree, nmodes, mpos, mrgb, mU, m_max, box_lo, box_hi,
                        query_seed, NULL, 0, out, dbg);
}

void orc_relocalise_from(const orc_params *p,
                         const float *depth_img, const uint8_t *rgb, int W, int Himg,
                         float fx, float fy, float cx, float cy,
                         const uint16_t *leaves, int n_trees_forest, int leaves_per_tree,
                         const uint8_t *nmodes, const float *mpos, const uint8_t *mrgb,
                         const float *mU, int m_max,
                         const double box_lo[3], const double box_hi[3],
                         uint64_t query_seed, const orc_resume *rs, int n_rs, orc_result *out,
                         orc_debug *dbg)
{
    (void)n_trees_forest;
    const orc_resume *hand;
    const int WH = W * Himg;
    const uint32_t key[2] = {(uint32_t)query_seed, (uint32_t)(query_seed >> 32)};
    memset(out, 0, sizeof(*out));
    out->score = INFINITY;
    out->best = -1;
    for (int i = 0; i < 16; ++i) {
        out->pose[i] = (i % 5 == 0) ? 1.0 : 0.0;
        out->chosen_icp_frac[i] = -1.0;
    }

    /* 1. hypothesis generation: one independent attempt loop per slot */
    hyp_t *hyp = (hyp_t *)malloc(sizeof(hyp_t) * (size_t)p->n_hyp);
    int n = 0;
    for (int s = 0; s < p->n_hyp; ++s) {
        int found = -1;
        double H[12];
        for (int it = 0; it < p->max_iter; ++it) {
            if (try_hypothesis(p, key, s, it, depth_img, rgb, W, Himg, fx, fy, cx, cy,
                               leaves, leaves_per_tree, nmodes, mpos, mrgb, m_max, H)) {
                found = it;
                break;
            }
        }
        if (dbg && dbg->hyp_iter)
            dbg->hyp_iter[s] = found;
        if (dbg && dbg->hyp_pose)
            for (int k = 0; k < 12; ++k)
                dbg->hyp_pose[12 * s + k] = found >= 0 ? H[k] : 0.0;
        if (found >= 0) {
            memcpy(hyp[n].H, H, sizeof(H));
            hyp[n].slot = s;
            hyp[n].E = 0.0;
            ++n;
        }
    }
    out->n_hypotheses = n;
    if (n == 0) {
        out->status = 1;
        free(hyp);
        return;
    }

    /* 2. initial cull on I_0 */
    int max_batches = 1;
    {
        int m = n < p->n_cull ? n : p->n_cull;
        while (m > 1) { m = (m + 1) / 2; ++max_batches; }
    }
    int32_t *I = (int32_t *)malloc(sizeof(int32_t) * (size_t)p->eta * (size_t)(max_batches + 1));
    int nI = 0;
    sample_batch(p, key, 0, depth_img, WH, leaves, leaves_per_tree, nmodes, I);
    if (dbg && dbg->batch_pix)
        memcpy(dbg->batch_pix, I, sizeof(int32_t) * (size_t)p->eta);
    nI = p->eta;
    for (int h = 0; h < n; ++h)
        hyp[h].E = orc_energy(hyp[h].H, I, nI, depth_img, W, Himg, fx, fy, cx, cy, leaves,
                              p->n_trees_used, leaves_per_tree, nmodes, mpos, mU, m_max,
                              p->k_top, p->use_cov);
    qsort(hyp, (size_t)n, sizeof(hyp_t), hyp_cmp);
    if (n > p->n_cull)
        n = p->n_cull;
    if ((hand = handin_at(rs, n_rs, 0)) != NULL)
        replace_survivors(hand, hyp, &n, I, nI, depth_img, W, Himg, fx, fy, cx, cy, leaves, p,
                          leaves_per_tree, nmodes, mpos, mU, m_max);
    if (dbg && dbg->cull_slot)
        for (int h = 0; h < n; ++h) {
            dbg->cull_slot[h] = hyp[h].slot;
            if (dbg->cull_energy) dbg->cull_energy[h] = hyp[h].E;
        }

    hyp_t chosen[16];
    int n_chosen = -1;
    int chosen_nI = nI;
    if (n <= p->k_out) {
        n_chosen = n;
        memcpy(chosen, hyp, sizeof(hyp_t) * (size_t)n);
    }

    /* 3. preemptive rounds: grow I, refine, re-score, keep the better half */
    int b = 1, round_off = 0, n_rounds = 0;
    while (n > p->k_out || (p->halve_to_one && n > 1)) {
        sample_batch(p, key, b, depth_img, WH, leaves, leaves_per_tree, nmodes, I + nI);
        if (dbg && dbg->batch_pix && b < 16)
            memcpy(dbg->batch_pix + (size_t)b * p->eta, I + nI, sizeof(int32_t) * (size_t)p->eta);
        nI += p->eta;
        ++b;
        for (int h = 0; h < n; ++h) {
            if (p->pose_update)
                orc_lm_refine(hyp[h].H, I, nI, depth_img, W, Himg, fx, fy, cx, cy, leaves,
                              p->n_trees_used, leaves_per_tree, nmodes, mpos, mU, m_max,
                              p->k_top, p->use_cov, p->lm_max_iter, p->lm_lambda0,
                              p->lm_inlier_thresh, p->lm_stop);
            hyp[h].E = orc_energy(hyp[h].H, I, nI, depth_img, W, Himg, fx, fy, cx, cy, leaves,
                                  p->n_trees_used, leaves_per_tree, nmodes, mpos, mU, m_max,
                                  p->k_top, p->use_cov);
        }
        qsort(hyp, (size_t)n, sizeof(hyp_t), hyp_cmp);
        n = (n + 1) / 2;
        if ((hand = handin_at(rs, n_rs, n_rounds + 1)) != NULL)
            replace_survivors(hand, hyp, &n, I, nI, depth_img, W, Himg, fx, fy, cx, cy, leaves, p,
                              leaves_per_tree, nmodes, mpos, mU, m_max);
        if (dbg && n_rounds < 16) {
            if (dbg->round_count) dbg->round_count[n_rounds] = n;
            for (int h = 0; h < n; ++h) {
                if (dbg->round_slot) dbg->round_slot[round_off + h] = hyp[h].slot;
                if (dbg->round_energy) dbg->round_energy[round_off + h] = hyp[h].E;
                if (dbg->round_pose)
                    memcpy(dbg->round_pose + 12 * (size_t)(round_off + h), hyp[h].H, sizeof(double) * 12);
            }
            round_off += n;
        }
        ++n_rounds;
        if (n_chosen < 0 && n <= p->k_out) {
            n_chosen = n;
            chosen_nI = nI;
            memcpy(chosen, hyp, sizeof(hyp_t) * (size_t)n);
        }
    }
    if (dbg) dbg->n_rounds = n_rounds;
    out->n_pixels = nI;
    out->n_chosen = n_chosen;
    for (int c = 0; c < n_chosen; ++c) {
        for (int k = 0; k < 16; ++k)
            out->chosen_pose[c][k] = k < 12 ? chosen[c].H[k] : (k == 15 ? 1.0 : 0.0);
        out->chosen_energy[c] = chosen[c].E;
        out->chosen_slot[c] = chosen[c].slot;
        out->chosen_score[c] = INFINITY;
    }

    /* 4. ICP against the model (R21): each chosen pose when ranking, else the
     * output pose; a pose is replaced by its refinement only when ICP
     * succeeds, and a chosen pose whose ICP failed is not ranked. */
    int icp_ok[16] = {0};
    if (p->icp) {
        const int n_icp = p->rank ? n_chosen : 1;
        for (int c = 0; c < n_icp; ++c) {
            double Hc[12], frac;
            memcpy(Hc, p->rank ? chosen[c].H : hyp[0].H, sizeof(Hc));
            icp_ok[c] = orc_icp_refine(Hc, depth_img, W, Himg, fx, fy, cx, cy, box_lo, box_hi, &p->icp_p, &frac);
            out->chosen_icp_frac[c] = frac;
            if (icp_ok[c]) {
                out->icp_mask |= 1 << c;
                memcpy(p->rank ? chosen[c].H : hyp[0].H, Hc, sizeof(Hc));
                if (p->rank)
                    for (int k = 0; k < 12; ++k)
                        out->chosen_pose[c][k] = Hc[k];
            }
        }
    }

    /* 5. model-based ranking of the chosen set (Eq. 6-8) */
    int best = 0;
    double best_E = hyp[0].E;
    const double *best_H = hyp[0].H;
    int best_nI = nI;
    if (p->rank) {
        double bs = INFINITY;
        int bi = -1;
        for (int c = 0; c < n_chosen; ++c) {
            if (p->icp && !icp_ok[c])
                continue; /* discarded: score stays +inf */
            out->chosen_score[c] = orc_depth_score(chosen[c].H, depth_img, W, Himg, fx, fy, cx, cy,
                                                   box_lo, box_hi, NULL, NULL);
            if (out->chosen_score[c] < bs) {
                bs = out->chosen_score[c];
                bi = c;
            }
        }
        if (bi < 0)
            bi = 0;
        best = bi;
        out->score = bs;
        best_E = chosen[bi].E;
        best_H = chosen[bi].H;
        best_nI = chosen_nI;
        out->best = bi;
    }
    for (int k = 0; k < 12; ++k)
        out->pose[k] = best_H[k];
    out->pose[12] = out->pose[13] = out->pose[14] = 0.0;
    out->pose[15] = 1.0;
    out->energy = best_E;
    out->energy_per_pixel = best_E / (double)best_nI;
    out->status = 0;
    (void)best;
    free(I);
    free(hyp);
}

/* Sec. 3.2.5: run the levels in order, falling back iff score > tau_l. */
int orc_cascade(int n_levels, const orc_params *levels, const double *thresholds,
                const float *const *depth_imgs, const uint8_t *const *rgbs,
                const int *Ws, const int *Hs, const float *fxs, const float *fys,
                const float *cxs, const float *cys, const uint16_t *const *leaf_maps,
                int n_trees_forest, int leaves_per_tree,
                const uint8_t *nmodes, const float *mpos, const uint8_t *mrgb,
                const float *mU, int m_max, const double box_lo[3], const double box_hi[3],
                uint64_t query_seed, orc_result *out)
{
    for (int l = 0; l < n_levels; ++l) {
        orc_relocalise(&levels[l], depth_imgs[l], rgbs[l], Ws[l], Hs[l], fxs[l], fys[l], cxs[l], cys[l],
                       leaf_maps[l], n_trees_forest, leaves_per_tree, nmodes, mpos, mrgb, mU, m_max,
                       box_lo, box_hi, query_seed, out, NULL);
        if (l == n_levels - 1 || (out->status == 0 && out->score <= thresholds[l]))
            return l;
    }
    return n_levels - 1;
}
