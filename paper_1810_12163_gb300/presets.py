"""Parameter sets of the paper's parameter table (Appendix B): the default
relocaliser and the Fast / Intermediate / Slow relocalisers tuned for the
cascades.  Values the paper does not give use this library's readings
(colour threshold 30, K_top 10, LM 10 iterations / 0.1 m inliers / damping
1e-3, 32 batch redraws, covariance regulariser 1e-4 m^2).
"""

FOREST_DEFAULT = dict(
    n_trees=5, depth=15, p_depth=0.4, delta_lo=-130.0, delta_hi=130.0, tau_depth_lo=-0.2,
    tau_depth_hi=0.2, tau_rgb_lo=-50.0, tau_rgb_hi=50.0, tau_zero=0, kappa=1024, m_max=50,
    min_cluster_size=20, sigma=0.1, tau_c=0.05, cov_eps=1e-4, mode_precision=1, grid_step=4,
    grid_origin=0,
)
# clustererTau 0.2, minClusterSize 5, reservoirCapacity 2048 for the cascade relocalisers
FOREST_CASCADE = dict(FOREST_DEFAULT, kappa=2048, min_cluster_size=5, tau_c=0.2)

# ICP before ranking (Sec. 3.2.4; this library's reading of an ICP the paper
# leaves to its host system): off by default; strides, iterations and inlier
# distances per coarse-to-fine level, success threshold, relative ridge.
ICP_DEFAULT = dict(icp=0, icp_levels=3, icp_stride=(4, 2, 1), icp_iters=(6, 3, 2),
                   icp_dist=(0.1, 0.05, 0.025), icp_min_frac=0.5, icp_ridge=1e-4)

_COMMON = dict(colour_thresh=30, k_top=10, n_trees_used=5, lm_max_iter=10, batch_attempts=32,
               lm_lambda0=1e-3, lm_inlier_thresh=0.1, lm_stop=1e-6, rank=1, halve_to_one=0,
               **ICP_DEFAULT)

DEFAULT = dict(_COMMON, n_hyp=1024, max_iter=6000, n_cull=64, max_trans_err=0.05,
               min_sq_dist=0.09, pose_update=1, eta=512, use_cov=1, k_out=16)
FAST = dict(_COMMON, n_hyp=2048, max_iter=500, n_cull=64, max_trans_err=0.05, min_sq_dist=0.0,
            pose_update=0, eta=256, use_cov=0, k_out=1)
INTERMEDIATE = dict(_COMMON, n_hyp=2048, max_iter=1000, n_cull=64, max_trans_err=0.1,
                    min_sq_dist=0.09, pose_update=1, eta=256, use_cov=0, k_out=1)
SLOW = dict(_COMMON, n_hyp=2048, max_iter=250, n_cull=64, max_trans_err=0.1, min_sq_dist=0.0225,
            pose_update=1, eta=256, use_cov=0, k_out=16)

# cascade fall-back thresholds found by the paper's tuning (metres)
THRESH_FAST_TO_INTERMEDIATE = 0.05
THRESH_INTERMEDIATE_TO_SLOW = 0.075
