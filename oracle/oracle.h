/*
 * CPU oracle for the RGB-D relocaliser of Cavallari et al., "Real-Time
 * RGB-D Camera Pose Estimation in Novel Scenes using a Relocalisation
 * Cascade" (TPAMI 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct CPU
 * implementation used to check the CUDA path.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Precision: FP64 everywhere except the split-feature arithmetic (Eq. 1-3),
 * which is FP32 with a fixed operation order and no contraction (compiled
 * with -ffp-contract=off) so that forest leaves are exactly reproducible.
 *
 * Every function cites the section / equation of the paper it follows.
 * Points where the paper is silent are resolved by the readings listed at
 * the top of oracle.c (R1..R19); the same readings are documented for users
 * of the library.
 */
#ifndef RELOC_ORACLE_H
#define RELOC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Philox4x32-10 (Salmon, Moraru, Dror, Shaw, SC'11) ---------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- random forest factory (Sec. 4.5) --------------------------------- */
/* Arrays have n_trees * (2^depth - 1) entries, tree-major, heap order. */
void orc_forest_random(int n_trees, int depth, float p_depth,
                       float delta_lo, float delta_hi,
                       float tau_depth_lo, float tau_depth_hi,
                       float tau_rgb_lo, float tau_rgb_hi, int tau_zero,
                       uint64_t seed,
                       float *dx, float *dy, float *tau, uint8_t *type, uint8_t *channel);

/* ---- Eq. 1-3: features and forest walk -------------------------------- */
/* leaves: uint16 [n_trees][H][W]; 0xFFFF for pixels with no valid depth. */
void orc_forest_leaves(const float *dx, const float *dy, const float *tau,
                       const uint8_t *type, const uint8_t *channel,
                       int n_trees, int depth,
                       const float *depth_img, const uint8_t *rgb, int W, int H, float fx,
                       uint16_t *leaves);
/* The two raw features (Eq. 1 and Eq. 2) of one pixel for one split node. */
float orc_feature(float ndx, float ndy, int ntype, int nchannel,
                  const float *depth_img, const uint8_t *rgb, int W, int H, float fx,
                  int x, int y);

/* ---- Sec. 3.2.2: leaf reservoirs ------------------------------------- */
/* Reservoir store: pos float[L][kappa][3], rgb uint8[L][kappa][3],
 * count uint32[L] (examples ever offered to the leaf). */
void orc_reservoir_add_frame(const float *dx, const float *dy, const float *tau,
                             const uint8_t *type, const uint8_t *channel,
                             int n_trees, int depth,
                             const float *depth_img, const uint8_t *rgb, int W, int H,
                             float fx, float fy, float cx, float cy,
                             const double cam_to_world[16], int grid_step, int grid_origin,
                             int kappa, uint64_t forest_seed,
                             float *res_pos, uint8_t *res_rgb, uint32_t *res_count);

/* ---- Sec. 3.2.2: Really Quick Shift clustering of one leaf ------------- */
/* Outputs (arrays sized m_max): number of kept clusters; per cluster the
 * FP64 3D centroid, mean colour (rounded), FP64 covariance (6 unique: xx xy
 * xz yy yz zz), size.  parent/root (sized n) are returned for inspection. */
int orc_rqs_leaf(const float *pos, const uint8_t *rgb, int n,
                 float sigma, float tau_c, int min_cluster_size, int m_max,
                 double *mu, uint8_t *colour, double *cov, int32_t *size,
                 int32_t *parent, int32_t *root, double *density);

/* Mode store of a forest (FP32, as used by the relocaliser):
 *   nmodes uint8[L], centroid float[L][3],
 *   mpos float[L][m_max][3] (decoded), mrgb uint8[L][m_max][3],
 *   mU float[L][m_max][6] (upper Cholesky factor of the regularised inverse
 *   covariance, order U00 U01 U02 U11 U12 U22), msize int32[L][m_max]. */
void orc_update_modes(const float *res_pos, const uint8_t *res_rgb, const uint32_t *res_count,
                      int kappa, int leaf_begin, int leaf_count, int n_leaves_total,
                      float sigma, float tau_c, int min_cluster_size, int m_max,
                      float cov_eps, int fp16_offsets,
                      uint8_t *nmodes, float *centroid, float *mpos, uint8_t *mrgb,
                      float *mU, int32_t *msize);

/* Writes positions pos[L][m_max][3] into the store's mpos in its precision
 * (FP32, or FP16 offsets from the leaf's FP32 centroid as orc_update_modes
 * encodes them); ranks >= nmodes[L] are untouched. */
void orc_set_mode_positions(const float *pos, const uint8_t *nmodes, const float *centroid,
                            int n_leaves, int m_max, int fp16_offsets, float *mpos);

/* ---- Kabsch (Sec. 3.2.3), Eq. 5, LM and ranking ----------------------- */
/* Rigid transform (R,t) minimising sum |R a_i + t - b_i|^2 over 3D pairs. */
void orc_kabsch(const double *a, const double *b, int n, double R[9], double t[3]);

/* ICP refinement against the box model (Sec. 3.2.4, reading R21). */
typedef struct {
    int32_t levels;           /* coarse-to-fine levels, 1..3 */
    int32_t stride[3];        /* pixel stride of each level */
    int32_t iters[3];         /* Gauss-Newton iterations of each level */
    int32_t pad;
    double  dist[3];          /* inlier distance |q - p| of each level, m */
    double  min_frac;         /* success: last-iteration inliers >= min_frac x valid pixels */
    double  ridge;            /* lambda = ridge * trace(J^T J) / 6 */
} orc_icp_params;

typedef struct {
    int32_t n_hyp;            /* N_max */
    int32_t max_iter;         /* maxCandidateGenerationIterations */
    int32_t n_cull;           /* N_cull */
    int32_t eta;              /* ransacInliersPerIteration */
    int32_t k_out;            /* maxRelocalisationsToOutput */
    int32_t pose_update;      /* poseUpdate */
    int32_t use_cov;          /* usePredictionCovarianceForPoseOptimization */
    int32_t colour_thresh;    /* L-inf colour check threshold (0..255) */
    double  min_sq_dist;      /* minSquaredDistanceBetweenSampledModes */
    double  max_trans_err;    /* maxTranslationErrorForCorrectPose */
    int32_t k_top;            /* modes per leaf used at inference */
    int32_t n_trees_used;     /* first n trees of the forest */
    int32_t lm_max_iter;
    int32_t batch_attempts;
    double  lm_lambda0;
    double  lm_inlier_thresh;
    double  lm_stop;
    int32_t rank;             /* model-based ranking of the chosen set */
    int32_t halve_to_one;     /* keep halving to 1 after the chosen set */
    int32_t level;            /* cascade level, part of the random stream */
    int32_t icp;              /* ICP of the chosen set (ranked) or output pose (R21) */
    int32_t redraw;           /* R8b: an invalid pixel draw is redrawn within its iteration */
    orc_icp_params icp_p;
} orc_params;

typedef struct {
    double pose[16];          /* camera->world, row major */
    double energy;            /* Eq. 5 of the output pose on the final set I */
    double energy_per_pixel;
    double score;             /* s(xi*) of Eq. 7, +inf if unranked/failed */
    int32_t n_hypotheses;     /* hypotheses that passed generation */
    int32_t n_chosen;         /* |Xi| */
    int32_t n_pixels;         /* final |I| */
    int32_t status;           /* 0 pose found, 1 no pose */
    double chosen_pose[16][16];
    double chosen_energy[16];
    double chosen_score[16];
    int32_t chosen_slot[16];
    int32_t best;             /* index into chosen of xi* */
    int32_t icp_mask;         /* bit c: ICP refined chosen pose c (ranked) / the output (bit 0, unranked) */
    double chosen_icp_frac[16]; /* last-iteration inlier fraction of each ICP run, -1 if not run */
} orc_result;

/* Optional diagnostics; any pointer may be NULL.  hyp_*: per slot of the
 * generation step; cull_*: survivors of the initial cull (slot ids and
 * energies, in rank order); round_*: survivors after each halving round,
 * flattened. */
typedef struct {
    double  *hyp_pose;        /* [n_hyp][12] row-major 3x4 */
    int32_t *hyp_iter;        /* [n_hyp], -1 if the slot failed */
    int32_t *cull_slot;       /* [n_cull] */
    double  *cull_energy;     /* [n_cull] */
    int32_t *round_slot;      /* [sum of survivors over rounds] */
    double  *round_energy;
    double  *round_pose;      /* [..][12] */
    int32_t *round_count;     /* [16] survivors after each round */
    int32_t *batch_pix;       /* [16][eta] pixel ids of each batch, -1 skipped */
    int32_t n_rounds;
    int32_t pad;
} orc_debug;

/* Full relocaliser of Sec. 3.2.3-3.2.4 on one frame. `leaves` is the
 * uint16 [n_trees][H][W] leaf map of this frame; the mode store is as
 * produced by orc_update_modes.  box_lo/hi define the analytic scene model
 * used by the ranking step. */
void orc_relocalise(const orc_params *p,
                    const float *depth_img, const uint8_t *rgb, int W, int H,
                    float fx, float fy, float cx, float cy,
                    const uint16_t *leaves, int n_trees_forest, int leaves_per_tree,
                    const uint8_t *nmodes, const float *mpos, const uint8_t *mrgb,
                    const float *mU, int m_max,
                    const double box_lo[3], const double box_hi[3],
                    uint64_t query_seed, orc_result *out, orc_debug *dbg);

/* Survivor set handed to orc_relocalise_from at a stage boundary of the
 * preemptive loop (Sec. 3.2.3): stage 0 = straight after the initial cull,
 * stage r + 1 = after the halving of preemptive round r.  The n survivors
 * (generation slot ids and 3x4 row-major poses) replace the oracle's own
 * set at that point; their energies are recomputed in FP64 on the pixel set
 * of that point and the set is re-sorted by (E, slot).  Everything after it
 * (later rounds, the chosen set, ICP, ranking) runs as in orc_relocalise.
 * Several hand-ins (distinct stages) apply in stage order.  The tests use
 * them to keep comparing a query whose survivor set or LM trajectory
 * legitimately left the oracle's. */
typedef struct {
    int32_t stage;
    int32_t n;
    const int32_t *slot;      /* [n] */
    const double *pose;       /* [n][12] */
} orc_resume;

/* orc_relocalise with n_rs survivor sets handed in (rs may be NULL if 0). */
void orc_relocalise_from(const orc_params *p,
                         const float *depth_img, const uint8_t *rgb, int W, int H,
                         float fx, float fy, float cx, float cy,
                         const uint16_t *leaves, int n_trees_forest, int leaves_per_tree,
                         const uint8_t *nmodes, const float *mpos, const uint8_t *mrgb,
                         const float *mU, int m_max,
                         const double box_lo[3], const double box_hi[3],
                         uint64_t query_seed, const orc_resume *rs, int n_rs, orc_result *out,
                         orc_debug *dbg);

/* Eq. 5 energy of one pose on a pixel set (pixel ids into the frame). */
double orc_energy(const double pose12[12], const int32_t *pix, int n_pix,
                  const float *depth_img, int W, int H, float fx, float fy, float cx, float cy,
                  const uint16_t *leaves, int n_trees_used, int leaves_per_tree,
                  const uint8_t *nmodes, const float *mpos, const float *mU, int m_max,
                  int k_top, int use_cov);

/* LM refinement (Sec. 3.2.3) of one pose on a pixel set; returns iterations. */
int orc_lm_refine(double pose12[12], const int32_t *pix, int n_pix,
                  const float *depth_img, int W, int H, float fx, float fy, float cx, float cy,
                  const uint16_t *leaves, int n_trees_used, int leaves_per_tree,
                  const uint8_t *nmodes, const float *mpos, const float *mU, int m_max,
                  int k_top, int use_cov, int max_iter, double lambda0,
                  double inlier_thresh, double stop);

/* Eq. 6-7: synthetic z-depth of the box seen from `pose` and the score. */
void orc_raycast_box(const double pose12[12], int W, int H, float fx, float fy, float cx, float cy,
                     const double box_lo[3], const double box_hi[3], double *out_depth);
double orc_depth_score(const double pose12[12], const float *depth_img, int W, int H,
                       float fx, float fy, float cx, float cy,
                       const double box_lo[3], const double box_hi[3],
                       double *mean_abs, double *valid_frac);

/* ICP of one pose against the box (R21); H is updated in place.  Returns 1
 * on success, 0 on failure; *frac_out = inliers / valid pixels of the last
 * iteration run. */
int orc_icp_refine(double pose12[12], const float *depth_img, int W, int H,
                   float fx, float fy, float cx, float cy,
                   const double box_lo[3], const double box_hi[3], const orc_icp_params *ip,
                   double *frac_out);

/* Oracle-internal FP64 helpers shared by the LM and ICP parts. */
int orc_chol_solve6(const double A[36], const double b[6], double x[6]);
void orc_se3_left_update(const double xi[6], double H[12]);

/* Sec. 3.2.5: cascade.  levels[l] describes level l; level_depth[l] etc.
 * are that level's (possibly subsampled) inputs and leaf maps.  Returns the
 * level that produced the output. */
int orc_cascade(int n_levels, const orc_params *levels, const double *thresholds,
                const float *const *depth_imgs, const uint8_t *const *rgbs,
                const int *Ws, const int *Hs, const float *fxs, const float *fys,
                const float *cxs, const float *cys, const uint16_t *const *leaf_maps,
                int n_trees_forest, int leaves_per_tree,
                const uint8_t *nmodes, const float *mpos, const uint8_t *mrgb,
                const float *mU, int m_max, const double box_lo[3], const double box_hi[3],
                uint64_t query_seed, orc_result *out);

#ifdef __cplusplus
}
#endif
void orc_set_threads(int n);

#endif
