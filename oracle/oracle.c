/*
 * CPU oracle, part 1: random streams, random forest factory, split
 * features and forest walk.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings of the paper used throughout the oracle.  Where the paper fixes
 * a step, the step is followed as written; where it is silent, this is the
 * reading taken (the CUDA library documents the same readings).
 *
 *  R1  Probe position (Eq. 1-2).  delta is in pixel*metres at a reference
 *      focal length f_ref = 585; at focal length fx the offset is scaled by
 *      s = fx / 585 (FP32).  With inv = 1/D(p) (FP32),
 *      q_x = floor(((float)p_x + (delta_x * s) * inv) + 0.5), clamped to
 *      [0, W-1] before conversion to int; likewise for y.  A probe whose
 *      depth is 0 reads 0.  Colour channels are read as floats 0..255.
 *      Pixels with D(p) <= 0 reach no leaf (0xFFFF).
 *  R2  Split parameters of the random forest (Sec. 4.5): per branch node,
 *      Depth with probability p else DA-RGB with channel uniform in {R,G,B};
 *      delta_x, delta_y uniform in [delta_lo, delta_hi); tau either 0 (as in
 *      the paper) or uniform in a per-feature range.
 *  R3  Node indexing: complete binary tree in heap order, root 0, children
 *      2n+1 (test false, left) and 2n+2 (test true, right, Eq. 3);
 *      leaf index = n - (2^depth - 1).
 *  R4  Training grid (Sec. 3.2.2, step 1): pixels (o + 4i, o + 4j), i,j >= 0,
 *      with origin o = 0 by default (the paper's N+ is read as a slip).
 *  R5  Reservoirs: Vitter's Algorithm R.  The c-th example (0-based) offered
 *      to a leaf goes to slot c if c < kappa, else r = U[0, c] (Philox) and
 *      slot r is replaced iff r < kappa.  Examples are offered in the order
 *      (frame, grid pixel row-major, tree).
 *  R6  Really Quick Shift: Gaussian Parzen density with bandwidth sigma
 *      (clustererSigma) on Euclidean 3D distance, summed over all points of
 *      the leaf; parent = nearest point of strictly higher density (equal
 *      density: lower index) within distance tau_c (clustererTau, metres).
 *      Clusters smaller than minClusterSize are dropped, the rest sorted by
 *      size (descending, ties by lower root index) and the first M_max kept.
 *      Per cluster: mean position, mean colour rounded half up, unbiased
 *      covariance; the covariance is regularised by eps*I (eps = 1e-4 m^2).
 *  R7  M(u) is the union over the trees in use of the first K_top modes of
 *      the leaf the pixel reaches in each tree (in tree order, then rank).
 *  R8  Hypothesis sampling: three pixels uniform over H*W; the iteration
 *      fails if a pixel has no depth or an empty M(u); the scene point is a
 *      mode drawn uniformly from M(u); the colour-check pair uniform in 0..2.
 *  R9  Checks in order: colour (L-inf > threshold rejects), spread (any
 *      squared pairwise scene distance < minSquaredDistanceBetweenSampled-
 *      Modes rejects), rigidity (any pair with |d_W - d_C| > maxTranslation-
 *      ErrorForCorrectPose rejects), then Kabsch.  x_C is computed in FP32:
 *      ((u - cx) * D) / fx, ((v - cy) * D) / fy, D.
 *  R10 Kabsch: R = V diag(1,1,sign det(V U^T)) U^T from the SVD of the
 *      cross-covariance; t = c_W - R c_C.
 *  R11 Successful slots are kept in slot order.
 *  R12 Pixel batches: eta draws with replacement; an invalid draw (no depth
 *      or empty M(u)) is redrawn up to `batch_attempts` times, then skipped.
 *  R13 Energy (Eq. 5): Mahalanobis with the regularised mode covariance if
 *      usePredictionCovariance..., else Euclidean; min over M(u) taken on the
 *      squared form; E summed over the whole current set I.
 *  R14 Cull keeps min(N_cull, n), stable by (E, slot); each round keeps
 *      ceil(n/2); the chosen set Xi is the survivor set the first time
 *      n <= k; with halve_to_one the rounds continue to a single pose.
 *  R15 LM: residual U*(exp(xi)H x - mu) for inliers (nearest-mode Euclidean
 *      distance <= 0.1 m), left perturbation, Marquardt damping
 *      (lambda0 1e-3, /10 on accept, *10 on reject), step accepted iff the
 *      cost with the same correspondences decreases, stop when |step| <
 *      1e-6 or after 10 iterations, no update with fewer than 3 inliers.
 *  R16 Raycast: z-depth of the first intersection of each pixel ray with the
 *      room box (exit point when the camera is inside, entry point when
 *      outside); no hit is invalid.  Live depth is valid iff > 0.
 *  R17 Cascade inputs: level subsample s keeps pixel (s*u', s*v') and
 *      divides the intrinsics by s.
 *  R18 Random streams: Philox4x32-10 keyed by a 64-bit seed; counters
 *      (entity, tag<<16 | level, index, sub-index); a 32-bit draw u maps to
 *      [0, n) by (u * n) >> 32.
 *  R19 Success: |t - t_gt| <= 5 cm and rotation angle <= 5 degrees.
 */
#include "oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#include <math.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* Philox4x32-10, from the description in Salmon et al., SC'11.           */
/* ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t below(uint32_t u, uint32_t n) /* R18: u -> [0, n) */
{
    return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

static float unit24(uint32_t u) /* exact FP32 in [0,1) from the top 24 bits */
{
    return (float)(u >> 8) * (1.0f / 16777216.0f);
}

/* ---------------------------------------------------------------------- */
/* Random forest factory (Sec. 4.5, reading R2).                          */
/* ---------------------------------------------------------------------- */
void orc_forest_random(int n_trees, int depth, float p_depth,
                       float delta_lo, float delta_hi,
                       float tau_depth_lo, float tau_depth_hi,
                       float tau_rgb_lo, float tau_rgb_hi, int tau_zero,
                       uint64_t seed,
                       float *dx, float *dy, float *tau, uint8_t *type, uint8_t *channel)
{
    const int n_branch = (1 << depth) - 1;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int t = 0; t < n_trees; ++t) {
        for (int n = 0; n < n_branch; ++n) {
            uint32_t c0[4] = {(uint32_t)t, 1u << 16, (uint32_t)n, 0u};
            uint32_t c1[4] = {(uint32_t)t, 1u << 16, (uint32_t)n, 1u};
            uint32_t r0[4], r1[4];
            orc_philox4x32_10(c0, key, r0);
            orc_philox4x32_10(c1, key, r1);
            const int is_depth = (double)r0[0] < (double)p_depth * 4294967296.0;
            const size_t i = (size_t)t * n_branch + n;
            float span = delta_hi - delta_lo;
            dx[i] = delta_lo + span * unit24(r0[1]);
            dy[i] = delta_lo + span * unit24(r0[2]);
            type[i] = is_depth ? 0 : 1;
            channel[i] = is_depth ? 0 : (uint8_t)below(r0[3], 3);
            if (tau_zero) {
                tau[i] = 0.0f;
            } else if (is_depth) {
                float s = tau_depth_hi - tau_depth_lo;
                tau[i] = tau_depth_lo + s * unit24(r1[0]);
            } else {
                float s = tau_rgb_hi - tau_rgb_lo;
                tau[i] = tau_rgb_lo + s * unit24(r1[0]);
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Eq. 1 (Depth) and Eq. 2 (DA-RGB) at pixel p for one split node (R1).   */
/* ---------------------------------------------------------------------- */
static int probe_coord(int p, float off, int extent)
{
    float v = ((float)p + off) + 0.5f;
    float f = floorf(v);
    f = fminf(fmaxf(f, 0.0f), (float)(extent - 1));
    return (int)f;
}

float orc_feature(float ndx, float ndy, int ntype, int nchannel,
                  const float *depth_img, const uint8_t *rgb, int W, int H, float fx,
                  int x, int y)
{
    const float s = fx / 585.0f;
    const float d = depth_img[(size_t)y * W + x];
    const float inv = 1.0f / d;
    const float ox = (ndx * s) * inv;
    const float oy = (ndy * s) * inv;
    const int qx = probe_coord(x, ox, W);
    const int qy = probe_coord(y, oy, H);
    const size_t q = (size_t)qy * W + qx;
    if (ntype == 0) {
        const float dq = depth_img[q] > 0.0f ? depth_img[q] : 0.0f;
        return d - dq;
    }
    const float cp = (float)rgb[((size_t)y * W + x) * 3 + nchannel];
    const float cq = (float)rgb[q * 3 + nchannel];
    return cp - cq;
}

/* Walk one tree from the root to a leaf (Eq. 3, reading R3). */
static int walk_tree(const float *dx, const float *dy, const float *tau,
                     const uint8_t *type, const uint8_t *channel, int depth,
                     const float *depth_img, const uint8_t *rgb, int W, int H, float fx,
                     int x, int y)
{
    int n = 0;
    for (int level = 0; level < depth; ++level) {
        const float f = orc_feature(dx[n], dy[n], type[n], channel[n],
                                    depth_img, rgb, W, H, fx, x, y);
        n = (f >= tau[n]) ? 2 * n + 2 : 2 * n + 1;
    }
    return n - ((1 << depth) - 1);
}

void orc_forest_leaves(const float *dx, const float *dy, const float *tau,
                       const uint8_t *type, const uint8_t *channel,
                       int n_trees, int depth,
                       const float *depth_img, const uint8_t *rgb, int W, int H, float fx,
                       uint16_t *leaves)
{
    const int n_branch = (1 << depth) - 1;
    for (int t = 0; t < n_trees; ++t) {
        const size_t o = (size_t)t * n_branch;
        /* pixels are independent; rows may run concurrently */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < H; ++y) {
            for (int x = 0; x < W; ++x) {
                const size_t p = (size_t)y * W + x;
                uint16_t leaf = 0xFFFF;
                if (depth_img[p] > 0.0f)
                    leaf = (uint16_t)walk_tree(dx + o, dy + o, tau + o, type + o, channel + o,
                                               depth, depth_img, rgb, W, H, fx, x, y);
                leaves[(size_t)t * W * H + p] = leaf;
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Sec. 3.2.2: add one posed frame to the leaf reservoirs (R4, R5).       */
/* ---------------------------------------------------------------------- */
void orc_reservoir_add_frame(const float *dx, const float *dy, const float *tau,
                             const uint8_t *type, const uint8_t *channel,
                             int n_trees, int depth,
                             const float *depth_img, const uint8_t *rgb, int W, int H,
                             float fx, float fy, float cx, float cy,
                             const double T[16], int grid_step, int grid_origin,
                             int kappa, uint64_t forest_seed,
                             float *res_pos, uint8_t *res_rgb, uint32_t *res_count)
{
    const int n_branch = (1 << depth) - 1;
    const int n_leaves = 1 << depth;
    const uint32_t key[2] = {(uint32_t)forest_seed, (uint32_t)(forest_seed >> 32)};
    for (int y = grid_origin; y < H; y += grid_step) {
        for (int x = grid_origin; x < W; x += grid_step) {
            const size_t p = (size_t)y * W + x;
            const float d = depth_img[p];
            if (!(d > 0.0f))
                continue;
            /* back-projection x_C = D(u) K^-1 u (FP32, fixed order) */
            const float xc = (((float)x - cx) * d) / fx;
            const float yc = (((float)y - cy) * d) / fy;
            const float zc = d;
            /* world point with the given camera->world pose (FP64) */
            float xw[3];
            for (int r = 0; r < 3; ++r)
                xw[r] = (float)(((T[4 * r + 0] * (double)xc + T[4 * r + 1] * (double)yc)
                                 + T[4 * r + 2] * (double)zc) + T[4 * r + 3]);
            for (int t = 0; t < n_trees; ++t) {
                const size_t o = (size_t)t * n_branch;
                const int leaf = walk_tree(dx + o, dy + o, tau + o, type + o, channel + o,
                                           depth, depth_img, rgb, W, H, fx, x, y);
                const uint32_t L = (uint32_t)(t * n_leaves + leaf);
                const uint32_t c = res_count[L];
                int64_t slot = -1;
                if (c < (uint32_t)kappa) {
                    slot = c;
                } else {
                    uint32_t ctr[4] = {L, 2u << 16, c, 0u};
                    uint32_t r[4];
                    orc_philox4x32_10(ctr, key, r);
                    uint64_t j = ((uint64_t)r[0] * ((uint64_t)c + 1)) >> 32; /* U[0, c] */
                    if (j < (uint64_t)kappa)
                        slot = (int64_t)j;
                }
                if (slot >= 0) {
                    const size_t e = (size_t)L * kappa + (size_t)slot;
                    res_pos[e * 3 + 0] = xw[0];
                    res_pos[e * 3 + 1] = xw[1];
                    res_pos[e * 3 + 2] = xw[2];
                    res_rgb[e * 3 + 0] = rgb[p * 3 + 0];
                    res_rgb[e * 3 + 1] = rgb[p * 3 + 1];
                    res_rgb[e * 3 + 2] = rgb[p * 3 + 2];
                }
                res_count[L] = c + 1;
            }
        }
    }
}

/* Threads of the OpenMP loops (pixel rows, leaves); the arithmetic does not
 * depend on it.  Test and timing infrastructure only. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

