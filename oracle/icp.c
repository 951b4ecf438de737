/*
 * CPU oracle, part 4: ICP refinement of a camera pose against the scene
 * model before ranking (Sec. 3.2.4, reading R21).  TEST INFRASTRUCTURE ONLY
 * (see oracle.h).
 *
 * The paper refines every chosen pose by ICP against the 3D model and drops
 * the pose when ICP fails; the ICP variant itself is left to the host
 * reconstruction system.  Reading R21, written out plainly here:
 *
 *  - Model: the analytic room box [lo, hi] (as for the ranking raycast, R16).
 *  - Data association is projective: live pixel u with depth d has camera
 *    ray c(u) = ((u - cx)/fx, (v - cy)/fy, 1); under the current pose
 *    H = [R | t] its point is q = t + d R c(u), and its model point p is the
 *    first box face hit by the same ray t + s R c(u) (exit point from inside
 *    the box, entry point from outside), with that face's axis normal n.
 *  - The residual is point-to-plane, r = n . (q - p); a pair with
 *    |q - p| > dist_l is an outlier and does not enter the sums.
 *  - Gauss-Newton on a camera-frame update H exp(xi) with xi = (v, w), so a
 *    rotation turns about the camera centre: with x = d c(u) the camera
 *    point and m = R^T n the face normal in the camera frame, the Jacobian
 *    of r is J = (m, x x m); the step solves (sum J J^T + lambda I) xi =
 *    -sum J r with lambda = ridge * trace(sum J J^T) / 6.  Directions the
 *    visible faces leave unconstrained (a wall seen alone: the two
 *    translations along it and the turn about its normal) then keep their
 *    value instead of drifting.
 *  - Coarse to fine: level l uses the pixels whose column and row are both
 *    multiples of stride_l, for iters_l iterations with inlier distance
 *    dist_l.
 *  - ICP fails when an iteration has fewer than 6 inliers or its system is
 *    not positive definite, or when the last iteration's inliers are fewer
 *    than min_frac of its valid pixels (depth > 0 and finite).
 */
#include "oracle.h"

#include <math.h>
#include <string.h>

/* First box face hit by o + s d, s > 0: parameter s and face axis. */
static int ray_box_face(const double o[3], const double d[3], const double lo[3], const double hi[3],
                        double *s_out, int *axis_out)
{
    double tn = -INFINITY, tf = INFINITY;
    int an = -1, af = -1;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < lo[a] || o[a] > hi[a])
                return 0;
            continue;
        }
        const double t1 = (lo[a] - o[a]) / d[a], t2 = (hi[a] - o[a]) / d[a];
        const double tmin = t1 < t2 ? t1 : t2, tmax = t1 < t2 ? t2 : t1;
        if (tmin > tn) { tn = tmin; an = a; }
        if (tmax < tf) { tf = tmax; af = a; }
    }
    if (tn > tf)
        return 0;
    if (tn > 0.0) { *s_out = tn; *axis_out = an; return 1; }
    if (tf > 0.0) { *s_out = tf; *axis_out = af; return 1; }
    return 0;
}

/* Normal equations of one ICP iteration over the pixels of one level. */
typedef struct {
    double A[36], g[6];
    long n_in, n_valid;
} icp_sums;

static void icp_accumulate(const double H[12], const float *depth_img, int W, int Himg,
                           float fx, float fy, float cx, float cy, const double lo[3], const double hi[3],
                           int stride, double dist, icp_sums *S)
{
    memset(S, 0, sizeof(*S));
    const double o[3] = {H[3], H[7], H[11]};
    for (int v = 0; v < Himg; v += stride)
        for (int u = 0; u < W; u += stride) {
            const float df = depth_img[(size_t)v * W + u];
            if (!(df > 0.0f) || isinf(df))
                continue;
            S->n_valid++;
            const double d = (double)df;
            const double c[3] = {((double)u - (double)cx) / (double)fx, ((double)v - (double)cy) / (double)fy, 1.0};
            double dir[3];
            for (int r = 0; r < 3; ++r)
                dir[r] = H[4 * r + 0] * c[0] + H[4 * r + 1] * c[1] + H[4 * r + 2] * c[2];
            double s;
            int a;
            if (!ray_box_face(o, dir, lo, hi, &s, &a))
                continue;
            double e[3];
            for (int r = 0; r < 3; ++r)
                e[r] = (o[r] + d * dir[r]) - (o[r] + s * dir[r]);
            if (e[0] * e[0] + e[1] * e[1] + e[2] * e[2] > dist * dist)
                continue;
            /* n = e_a; m = R^T n is row a of R; x = d c(u) */
            const double m[3] = {H[4 * a + 0], H[4 * a + 1], H[4 * a + 2]};
            const double x[3] = {d * c[0], d * c[1], d * c[2]};
            const double res = e[a];
            /* J = (m, x x m) */
            const double J[6] = {m[0], m[1], m[2],
                                 x[1] * m[2] - x[2] * m[1],
                                 x[2] * m[0] - x[0] * m[2],
                                 x[0] * m[1] - x[1] * m[0]};
            for (int i = 0; i < 6; ++i) {
                S->g[i] += J[i] * res;
                for (int j = 0; j < 6; ++j)
                    S->A[6 * i + j] += J[i] * J[j];
            }
            S->n_in++;
        }
}

int orc_icp_refine(double H[12], const float *depth_img, int W, int Himg,
                   float fx, float fy, float cx, float cy,
                   const double lo[3], const double hi[3], const orc_icp_params *ip,
                   double *frac_out)
{
    icp_sums S;
    memset(&S, 0, sizeof(S));
    if (frac_out)
        *frac_out = 0.0;
    for (int l = 0; l < ip->levels; ++l)
        for (int it = 0; it < ip->iters[l]; ++it) {
            icp_accumulate(H, depth_img, W, Himg, fx, fy, cx, cy, lo, hi, ip->stride[l], ip->dist[l], &S);
            if (frac_out)
                *frac_out = S.n_valid > 0 ? (double)S.n_in / (double)S.n_valid : 0.0;
            if (S.n_in < 6)
                return 0;
            double A[36], b[6], xi[6];
            const double tr = S.A[0] + S.A[7] + S.A[14] + S.A[21] + S.A[28] + S.A[35];
            memcpy(A, S.A, sizeof(A));
            for (int i = 0; i < 6; ++i) {
                A[6 * i + i] += ip->ridge * tr / 6.0;
                b[i] = -S.g[i];
            }
            if (!orc_chol_solve6(A, b, xi))
                return 0;
            /* H <- H exp(xi): E = exp(xi) as the left update of the identity */
            double E[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0}, N[12];
            orc_se3_left_update(xi, E);
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 4; ++k)
                    N[4 * r + k] = H[4 * r + 0] * E[k] + H[4 * r + 1] * E[4 + k] + H[4 * r + 2] * E[8 + k] +
                                   (k == 3 ? H[4 * r + 3] : 0.0);
            memcpy(H, N, sizeof(N));
        }
    return S.n_valid > 0 && (double)S.n_in >= ip->min_frac * (double)S.n_valid;
}
