/*
 * CPU oracle, part 2: Really Quick Shift clustering of leaf reservoirs and
 * the leaf mode store (Sec. 3.2.2, step 3; readings R6 and R7 in oracle.c).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Really Quick Shift (Fulkerson & Soatto 2010) on the n points of a leaf. */
int orc_rqs_leaf(const float *pos, const uint8_t *rgb, int n,
                 float sigma, float tau_c, int min_cluster_size, int m_max,
                 double *mu, uint8_t *colour, double *cov, int32_t *size,
                 int32_t *parent, int32_t *root, double *density)
{
    if (n <= 0)
        return 0;
    const double sgm = (double)sigma, tc = (double)tau_c;
    const double inv2s2 = 1.0 / (2.0 * sgm * sgm);
    const double tau2 = tc * tc;
    /* Parzen density of every point (Gaussian kernel, all points). */
    for (int i = 0; i < n; ++i) {
        double rho = 0.0;
        for (int j = 0; j < n; ++j) {
            double ex = (double)pos[3 * i + 0] - (double)pos[3 * j + 0];
            double ey = (double)pos[3 * i + 1] - (double)pos[3 * j + 1];
            double ez = (double)pos[3 * i + 2] - (double)pos[3 * j + 2];
            double d2 = (ex * ex + ey * ey) + ez * ez;
            rho += exp(-(d2 * inv2s2));
        }
        density[i] = rho;
    }
    /* Parent: nearest point of higher density within tau_c. */
    for (int i = 0; i < n; ++i) {
        int best = -1;
        double best_d2 = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i)
                continue;
            int higher = density[j] > density[i] || (density[j] == density[i] && j < i);
            if (!higher)
                continue;
            double ex = (double)pos[3 * i + 0] - (double)pos[3 * j + 0];
            double ey = (double)pos[3 * i + 1] - (double)pos[3 * j + 1];
            double ez = (double)pos[3 * i + 2] - (double)pos[3 * j + 2];
            double d2 = (ex * ex + ey * ey) + ez * ez;
            if (d2 > tau2)
                continue;
            if (best < 0 || d2 < best_d2) {
                best = j;
                best_d2 = d2;
            }
        }
        parent[i] = best;
    }
    /* Roots: follow parents (density increases along a chain, no cycles). */
    int32_t *csize = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    for (int i = 0; i < n; ++i) {
        int r = i;
        while (parent[r] >= 0)
            r = parent[r];
        root[i] = r;
        csize[r] += 1;
    }
    /* Clusters above the size floor, sorted by (size desc, root asc). */
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int n_cl = 0;
    for (int r = 0; r < n; ++r)
        if (parent[r] < 0 && csize[r] >= min_cluster_size)
            order[n_cl++] = r;
    for (int a = 1; a < n_cl; ++a) { /* insertion sort, stable */
        int32_t v = order[a];
        int b = a - 1;
        while (b >= 0 && csize[order[b]] < csize[v]) {
            order[b + 1] = order[b];
            --b;
        }
        order[b + 1] = v;
    }
    const int kept = n_cl < m_max ? n_cl : m_max;
    for (int k = 0; k < kept; ++k) {
        const int r = order[k];
        double sx = 0, sy = 0, sz = 0;
        long sr = 0, sg = 0, sb = 0;
        int cnt = 0;
        for (int i = 0; i < n; ++i) {
            if (root[i] != r)
                continue;
            sx += (double)pos[3 * i + 0];
            sy += (double)pos[3 * i + 1];
            sz += (double)pos[3 * i + 2];
            sr += rgb[3 * i + 0];
            sg += rgb[3 * i + 1];
            sb += rgb[3 * i + 2];
            ++cnt;
        }
        const double m[3] = {sx / cnt, sy / cnt, sz / cnt};
        double c[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            if (root[i] != r)
                continue;
            double e0 = (double)pos[3 * i + 0] - m[0];
            double e1 = (double)pos[3 * i + 1] - m[1];
            double e2 = (double)pos[3 * i + 2] - m[2];
            c[0] += e0 * e0; c[1] += e0 * e1; c[2] += e0 * e2;
            c[3] += e1 * e1; c[4] += e1 * e2; c[5] += e2 * e2;
        }
        for (int q = 0; q < 6; ++q)
            cov[6 * k + q] = cnt > 1 ? c[q] / (double)(cnt - 1) : 0.0;
        mu[3 * k + 0] = m[0];
        mu[3 * k + 1] = m[1];
        mu[3 * k + 2] = m[2];
        colour[3 * k + 0] = (uint8_t)((sr + cnt / 2) / cnt);
        colour[3 * k + 1] = (uint8_t)((sg + cnt / 2) / cnt);
        colour[3 * k + 2] = (uint8_t)((sb + cnt / 2) / cnt);
        size[k] = cnt;
    }
    free(order);
    free(csize);
    return kept;
}

/* IEEE binary16 from binary64, round to nearest even (from the format's
 * definition: 1 sign bit, 5 exponent bits with bias 15, 10 fraction bits). */
static uint16_t half_from_double(double x)
{
    uint16_t sign = signbit(x) ? 0x8000u : 0u;
    double a = fabs(x);
    if (isnan(x))
        return 0x7E00u;
    if (a >= 65520.0) /* rounds past the largest finite half, 65504 */
        return sign | 0x7C00u;
    if (a < ldexp(1.0, -14)) { /* subnormal range: units of 2^-24 */
        double q = nearbyint(ldexp(a, 24));
        return sign | (uint16_t)q; /* q == 1024 is the smallest normal */
    }
    int e;
    frexp(a, &e); /* a = f * 2^e, f in [0.5, 1) */
    int E = e - 1; /* a in [2^E, 2^(E+1)) */
    double q = nearbyint(ldexp(a, 10 - E)); /* in [1024, 2048] */
    if (q >= 2048.0) {
        q = 1024.0;
        E += 1;
    }
    if (E + 15 >= 31)
        return sign | 0x7C00u;
    return sign | (uint16_t)(((E + 15) << 10) | ((int)q - 1024));
}

static double half_to_double(uint16_t h)
{
    int s = (h >> 15) & 1, E = (h >> 10) & 31, m = h & 1023;
    double v;
    if (E == 0)
        v = ldexp((double)m, -24);
    else if (E == 31)
        v = m ? NAN : INFINITY;
    else
        v = ldexp((double)(1024 + m), E - 25);
    return s ? -v : v;
}

/* Upper Cholesky factor U (U^T U = S) of the inverse of the regularised
 * covariance: Mahalanobis |S^1/2 v| of Eq. 5 equals |U v|. */
static void inverse_cov_factor(const double cov[6], double eps, double U[6])
{
    const double a = cov[0] + eps, b = cov[1], c = cov[2];
    const double d = cov[3] + eps, e = cov[4], f = cov[5] + eps;
    /* symmetric [[a b c][b d e][c e f]]: inverse by cofactors */
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

void orc_update_modes(const float *res_pos, const uint8_t *res_rgb, const uint32_t *res_count,
                      int kappa, int leaf_begin, int leaf_count, int n_leaves_total,
                      float sigma, float tau_c, int min_cluster_size, int m_max,
                      float cov_eps, int fp16_offsets,
                      uint8_t *nmodes, float *centroid, float *mpos, uint8_t *mrgb,
                      float *mU, int32_t *msize)
{
    /* Leaves are independent: the arithmetic of each leaf is unchanged by
     * running several leaves at once. */
#pragma omp parallel for schedule(dynamic, 16)
    for (int q = 0; q < leaf_count; ++q) {
        double mu[3 * 64], cov[6 * 64];
        uint8_t col[3 * 64];
        int32_t sz[64];
        int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)kappa);
        int32_t *rt = (int32_t *)malloc(sizeof(int32_t) * (size_t)kappa);
        double *den = (double *)malloc(sizeof(double) * (size_t)kappa);
        const int L = (leaf_begin + q) % n_leaves_total;
        const uint32_t c = res_count[L];
        const int n = c < (uint32_t)kappa ? (int)c : kappa;
        const int k = orc_rqs_leaf(res_pos + (size_t)L * kappa * 3, res_rgb + (size_t)L * kappa * 3,
                                   n, sigma, tau_c, min_cluster_size, m_max,
                                   mu, col, cov, sz, par, rt, den);
        nmodes[L] = (uint8_t)k;
        /* per-leaf FP32 centroid: mean of the kept modal centroids */
        double cs[3] = {0, 0, 0};
        for (int m = 0; m < k; ++m)
            for (int a = 0; a < 3; ++a)
                cs[a] += mu[3 * m + a];
        float cf[3];
        for (int a = 0; a < 3; ++a) {
            cf[a] = k > 0 ? (float)(cs[a] / k) : 0.0f;
            centroid[(size_t)L * 3 + a] = cf[a];
        }
        for (int m = 0; m < m_max; ++m) {
            const size_t e = (size_t)L * m_max + m;
            if (m >= k) {
                for (int a = 0; a < 3; ++a) { mpos[e * 3 + a] = 0.0f; mrgb[e * 3 + a] = 0; }
                for (int a = 0; a < 6; ++a) mU[e * 6 + a] = 0.0f;
                msize[e] = 0;
                continue;
            }
            for (int a = 0; a < 3; ++a) {
                if (fp16_offsets) {
                    uint16_t h = half_from_double(mu[3 * m + a] - (double)cf[a]);
                    mpos[e * 3 + a] = cf[a] + (float)half_to_double(h);
                } else {
                    mpos[e * 3 + a] = (float)mu[3 * m + a];
                }
                mrgb[e * 3 + a] = col[3 * m + a];
            }
            double U[6];
            inverse_cov_factor(cov + 6 * m, (double)cov_eps, U);
            for (int a = 0; a < 6; ++a)
                mU[e * 6 + a] = (float)U[a];
            msize[e] = sz[m];
        }
        free(par); free(rt); free(den);
    }
}

/* Mode positions written back into a store (Sec. 3.2.2 mode layout): FP32
 * as given, or as FP16 offsets from the leaf's FP32 centroid, i.e. the half
 * (round to nearest even) of the FP64 difference, decoded as centroid +
 * offset in FP32 -- the same encoding orc_update_modes applies to the modal
 * centroids.  Entries at ranks >= nmodes[leaf] are left untouched. */
void orc_set_mode_positions(const float *pos, const uint8_t *nmodes, const float *centroid,
                            int n_leaves, int m_max, int fp16_offsets, float *mpos)
{
    for (int L = 0; L < n_leaves; ++L)
        for (int m = 0; m < nmodes[L] && m < m_max; ++m) {
            const size_t e = (size_t)L * m_max + m;
            for (int a = 0; a < 3; ++a) {
                const float x = pos[e * 3 + a];
                if (fp16_offsets) {
                    const float c = centroid[(size_t)L * 3 + a];
                    const uint16_t h = half_from_double((double)x - (double)c);
                    mpos[e * 3 + a] = c + (float)half_to_double(h);
                } else {
                    mpos[e * 3 + a] = x;
                }
            }
        }
}
