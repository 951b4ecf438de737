/*
 * relocgb -- RGB-D camera relocalisation on GB300 (sm_103a).
 *
 * C ABI of the library.  It implements the per-frame relocaliser of
 * Cavallari, Golodetz, Lord, Valentin, Prisacariu, Di Stefano and Torr,
 * "Real-Time RGB-D Camera Pose Estimation in Novel Scenes using a
 * Relocalisation Cascade" (TPAMI 2019):
 *
 *   forest factory ....... Sec. 4.5 (random complete trees)
 *   online adaptation .... Sec. 3.2.2 (leaf reservoirs, Really Quick Shift)
 *   pose estimation ...... Sec. 3.2.3 (Kabsch hypotheses on triples, checks,
 *                          preemptive RANSAC with the energy of Eq. 5, LM)
 *   hypothesis ranking ... Sec. 3.2.4 (Eq. 6-8, depth raycast of the model)
 *   cascade .............. Sec. 3.2.5
 *
 * Conventions shared by every call:
 *  - Every function returns rl_status; outputs are written only on RL_OK.
 *    A frame for which no pose hypothesis survives is NOT an error: the
 *    result carries status RL_NO_POSE and score +inf.
 *  - No call traps the device, throws across the ABI, or allocates device
 *    memory after rl_context_create: all device state lives in the
 *    caller-owned arena handed to the context.
 *  - Streams are passed as `void *` holding a cudaStream_t (NULL = legacy
 *    default stream).  Calls that return results to the host synchronise
 *    that stream before returning.
 *  - Images: depth float32 [H][W] in metres (<= 0 or NaN = invalid), colour
 *    uint8 [H][W][3] (RGB) registered to depth.  Poses: row-major 4x4 FP64,
 *    camera -> world (x right, y down, z forward in the camera).
 *  - rl_mem says where image pointers live (host memory is copied in on the
 *    given stream; device pointers must stay valid until the stream work
 *    completes).
 *  - Handles are opaque and owned by the library; release them with the
 *    matching *_destroy.  Handles are not thread-safe: one thread at a time
 *    per handle.
 */
#ifndef RELOCGB_H
#define RELOCGB_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RL_OK = 0,
    RL_ERR_INVALID_ARG = 1, /* bad pointer, size or parameter */
    RL_ERR_OOM = 2,         /* arena exhausted */
    RL_ERR_ADMISSION = 3,   /* serving: request refused by the memory budget */
    RL_ERR_CUDA = 4,        /* a CUDA runtime call failed (see rl_last_error) */
    RL_ERR_TIMEOUT = 5,     /* a bounded wait ran out */
    RL_ERR_BUSY = 6,        /* handle still referenced by another handle */
    RL_ERR_IO = 7,          /* file could not be read or written */
    RL_ERR_INTERNAL = 8     /* device-side consistency check failed */
} rl_status;

typedef enum { RL_HOST = 0, RL_DEVICE = 1 } rl_mem;
typedef enum { RL_POSE_FOUND = 0, RL_NO_POSE = 1 } rl_pose_status;
typedef enum { RL_MODES_FP32 = 0, RL_MODES_FP16_OFFSET = 1 } rl_mode_precision;

typedef struct rl_ctx rl_ctx;
typedef struct rl_forest rl_forest;
typedef struct rl_scene rl_scene;
typedef struct rl_reloc rl_reloc;
typedef struct rl_cascade rl_cascade;

typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
} rl_intrinsics;

/* Forest and adaptation parameters (Sec. 3.2.2, Sec. 4.5 and the parameter
 * table of Appendix B). */
typedef struct {
    int32_t n_trees;          /* trees in the forest (paper: 5) */
    int32_t depth;            /* split levels per tree, 1..15 (paper: 15 / 14) */
    float p_depth;            /* probability of a Depth split (paper: 0.4) */
    float delta_lo, delta_hi; /* probe offset range, pixel*metres at f = 585 */
    float tau_depth_lo, tau_depth_hi; /* threshold range of Depth splits (m) */
    float tau_rgb_lo, tau_rgb_hi;     /* threshold range of DA-RGB splits */
    int32_t tau_zero;         /* 1: every threshold is 0, as in Sec. 4.5 */
    int32_t kappa;            /* reservoirCapacity */
    int32_t m_max;            /* maxClusterCount (<= 64) */
    int32_t min_cluster_size; /* minClusterSize */
    float sigma;              /* clustererSigma, metres */
    float tau_c;              /* clustererTau, metres */
    float cov_eps;            /* covariance regulariser, m^2 (not in the paper) */
    int32_t mode_precision;   /* rl_mode_precision */
    int32_t grid_step;        /* training-pixel grid spacing (paper: 4) */
    int32_t grid_origin;      /* first grid row/column (0) */
} rl_forest_params;

/* ICP refinement against the scene model before ranking (Sec. 3.2.4: the
 * paper refines each chosen pose by ICP and drops it when ICP fails, with
 * the ICP of its host reconstruction system).  Point-to-plane ICP with
 * projective association: pixel u's live point under the current pose
 * against the first model face hit by the same pixel ray; pairs farther
 * apart than dist[l] are outliers.  Gauss-Newton on a camera-frame update
 * H exp(xi), xi = (v, w), with a ridge lambda = ridge * trace(J^T J) / 6 on
 * the normal equations, so that directions the visible faces leave
 * unconstrained keep their value.  Level l uses the pixels whose column and
 * row are multiples of stride[l], for iters[l] iterations.  ICP fails when
 * an iteration has fewer than 6 inliers or a system that is not positive
 * definite, or when the last iteration's inliers are fewer than
 * min_frac x its valid pixels.  Sums are FP32 per thread, FP64 across
 * threads; the solve and the pose are FP64. */
typedef struct {
    int32_t levels;           /* coarse-to-fine levels, 1..3 */
    int32_t stride[3];        /* pixel stride of each level, 1..16 */
    int32_t iters[3];         /* Gauss-Newton iterations of each level, 1..50 */
    int32_t pad;
    double dist[3];           /* inlier distance of each level, metres, > 0 */
    double min_frac;          /* success threshold on the inlier fraction, 0..1 */
    double ridge;             /* relative ridge, >= 0 */
} rl_icp_params;

/* Relocaliser parameters (Sec. 3.2.3-3.2.4; names follow the parameter
 * table of Appendix B). */
typedef struct {
    int32_t n_hyp;            /* maxPoseCandidates, N_max (<= 4096) */
    int32_t max_iter;         /* maxCandidateGenerationIterations, 1 .. 2^30 - 64 */
    int32_t n_cull;           /* maxPoseCandidatesAfterCull, N_cull (<= 64) */
    int32_t eta;              /* ransacInliersPerIteration (<= 1024) */
    int32_t k_out;            /* maxRelocalisationsToOutput (<= 16) */
    int32_t pose_update;      /* poseUpdate: LM refinement on/off */
    int32_t use_cov;          /* usePredictionCovarianceForPoseOptimization */
    int32_t colour_thresh;    /* L-inf colour check threshold, 0..255 */
    double min_sq_dist;       /* minSquaredDistanceBetweenSampledModes, m^2 */
    double max_trans_err;     /* maxTranslationErrorForCorrectPose, m */
    int32_t k_top;            /* modes per leaf used at inference */
    int32_t n_trees_used;     /* use the first n trees of the forest */
    int32_t lm_max_iter;      /* LM iterations per refinement */
    int32_t batch_attempts;   /* redraws of an invalid batch pixel */
    double lm_lambda0;        /* initial Marquardt damping */
    double lm_inlier_thresh;  /* LM inlier radius, m */
    double lm_stop;           /* LM stops when |step| < lm_stop */
    int32_t rank;             /* score the chosen set by Eq. 6-8 */
    int32_t halve_to_one;     /* keep halving after the chosen set is taken */
    int32_t icp;              /* 1: ICP before ranking (each chosen pose; the
                                 output pose alone when rank == 0); needs a scene */
    int32_t redraw;           /* 0: a generation draw of a pixel without depth or
                                 with an empty M(u) fails its iteration (the
                                 default reading); 1: it is redrawn within the
                                 iteration, up to batch_attempts draws in all
                                 (the paper does not say which it does) */
    rl_icp_params icp_p;
} rl_ransac_params;

#define RL_MAX_CHOSEN 16

typedef struct {
    double pose[16];          /* output camera->world pose (xi* if ranked) */
    float energy;             /* Eq. 5 energy of the output pose */
    float energy_per_pixel;   /* energy / |I| */
    float score;              /* s(xi*) of Eq. 7 (+inf if not ranked) */
    int32_t level;            /* cascade level that produced the pose */
    int32_t n_hypotheses;     /* hypotheses that passed generation */
    int32_t n_chosen;         /* |Xi| */
    int32_t n_pixels;         /* final |I| */
    int32_t status;           /* rl_pose_status */
    double chosen_pose[RL_MAX_CHOSEN][16];
    float chosen_energy[RL_MAX_CHOSEN];
    float chosen_score[RL_MAX_CHOSEN];
    int32_t chosen_slot[RL_MAX_CHOSEN];
    int32_t best;             /* index of xi* in chosen_pose */
    int32_t icp_mask;         /* ICP on: bit c set iff ICP refined chosen pose c
                                 (ranked) / the output pose (bit 0, unranked);
                                 chosen_pose holds the refined poses, a failed
                                 pose stays as RANSAC left it with score +inf */
    float chosen_icp_frac[RL_MAX_CHOSEN]; /* last-iteration inlier fraction, -1 if ICP did not run */
} rl_result;

/* ---- context --------------------------------------------------------- */
/* Creates a context on `device` over a caller-owned device buffer of
 * `arena_bytes` bytes (256-byte aligned) that must outlive the context.
 * Errors: RL_ERR_INVALID_ARG (null/misaligned arena), RL_ERR_CUDA. */
rl_status rl_context_create(int32_t device, void *arena_dev_ptr, uint64_t arena_bytes,
                            rl_ctx **out);
rl_status rl_context_destroy(rl_ctx *ctx);
/* Bytes of the arena in use / high-water mark. */
rl_status rl_context_usage(const rl_ctx *ctx, uint64_t *used, uint64_t *peak);
/* Message of the last failed call on this thread ("" if none). */
const char *rl_last_error(void);

/* ---- forest (Sec. 4.5 factory, Sec. 3.2.2 adaptation) ---------------- */
/* Random forest of complete trees (Sec. 4.5): per branch node a Depth split
 * with probability p_depth, else a DA-RGB split on a uniform channel;
 * offsets and thresholds uniform in the given ranges.  Nodes are in heap
 * order (children 2n+1 = test false, 2n+2 = test true, Eq. 3).  Draws use
 * Philox4x32-10 keyed by `seed`; the same seed gives the same forest.
 * Allocates nodes, reservoirs and the mode store from the arena
 * (RL_ERR_OOM if it does not fit).  Reservoirs start empty. */
rl_status rl_forest_create_random(rl_ctx *ctx, const rl_forest_params *p, uint64_t seed,
                                  rl_forest **out);
/* RL_ERR_BUSY while a relocaliser still uses the forest. */
rl_status rl_forest_destroy(rl_forest *f);
/* Empties every reservoir and mode list (the leaf reset of Sec. 3.2.1). */
rl_status rl_forest_reset_leaves(rl_forest *f, void *stream);
/* Sec. 3.2.2 steps 1-2: the pixels of a regular grid (spacing grid_step)
 * with valid depth are back-projected with `cam_to_world`, passed down
 * every tree, and offered to the reached leaf's reservoir by Algorithm R
 * (Vitter 1985) in the order (pixel row-major, tree).  Deterministic. */
rl_status rl_forest_adapt(rl_forest *f, const float *depth, const uint8_t *rgb,
                          const rl_intrinsics *K, const double cam_to_world[16], rl_mem mem,
                          void *stream);
/* Sec. 3.2.2 step 3: Really Quick Shift on the next `n_leaves` leaves in
 * round-robin order (n_leaves < 0: every leaf); keeps the largest M_max
 * clusters per leaf with centroid, colour, covariance.  Ordered by CUDA
 * events against relocalisation on other streams (the serving loop's
 * included): the update waits on `stream` for launches already enqueued
 * that read the modes, and launches enqueued after this call wait for the
 * update.  rl_forest_reset_leaves is ordered the same way. */
rl_status rl_forest_update_modes(rl_forest *f, int32_t n_leaves, void *stream);
/* Streaming adaptation (Sec. 3.2.2: leaves are re-clustered a few hundred
 * per frame while the relocaliser keeps running): enable = 1 gives the
 * forest a second mode store.  Relocalisation launches then read a complete
 * snapshot, the front store, while rl_forest_update_modes writes the back
 * store on its own stream and swaps the two.  Each launch sees the modes
 * after the last update enqueued (in host order) before it, never a leaf
 * halfway through re-clustering.
 *   Ordering is by CUDA events, with no host waits: a launch waits on its
 * stream for the last update; an update waits on its stream for every
 * launch that read the store it overwrites.  rl_forest_adapt writes only the
 * reservoirs, which relocalisation never reads, so it needs no ordering
 * against launches.  Enqueueing from several host threads is safe (the
 * forest serialises its bookkeeping); export, save, set_mode_positions and
 * reset_leaves act on the front store and belong between updates.
 *   Costs: a second mode store (L x M_max x 34 bytes + L x 17 bytes) and,
 * per update, a device copy of the previous update's leaves.  Must be set
 * before any relocaliser of the forest exists (RL_ERR_BUSY otherwise).
 * enable = 0 frees the second store. */
rl_status rl_forest_set_streaming(rl_forest *f, int32_t enable);
/* Eq. 1-3 for every pixel: out_leaves is a DEVICE uint16 [n_trees][H][W]
 * buffer (0xFFFF where depth is invalid).  Bit-exact FP32 arithmetic. */
rl_status rl_forest_leaves(rl_forest *f, const float *depth, const uint8_t *rgb,
                           const rl_intrinsics *K, int32_t n_trees, uint16_t *out_leaves,
                           rl_mem mem, void *stream);
/* Copies forest state to HOST buffers (any may be NULL).  Sizes: nodes
 * T*(2^d-1); reservoirs L*kappa with L = T*2^d; modes L*m_max.
 * node_meta = type (0 Depth, 1 DA-RGB) | channel << 8.  Mode positions are
 * decoded to FP32; mode_U holds the upper Cholesky factor of the inverse
 * regularised covariance (U00 U01 U02 U11 U12 U22). */
rl_status rl_forest_export(rl_forest *f, float *node_dx, float *node_dy, float *node_tau,
                           int32_t *node_meta, float *res_pos /* L*kappa*3 */,
                           uint8_t *res_rgb /* L*kappa*3 */, uint32_t *res_count /* L */,
                           uint8_t *nmodes /* L */, float *mode_pos /* L*m_max*3 */,
                           uint8_t *mode_rgb /* L*m_max*3 */, float *mode_U /* L*m_max*6 */,
                           int32_t *mode_size /* L*m_max */);
/* Overwrites the positions of the stored modes (HOST float [L][m_max][3];
 * ranks at or beyond a leaf's mode count are ignored), re-encoded in the
 * forest's precision: FP16 offsets from the leaf's FP32 centroid (which is
 * kept; the difference is rounded once to half) or FP32.  The paper has no
 * counterpart: it injects outlier modes for precision and stress studies.
 * Synchronises the device. */
rl_status rl_forest_set_mode_positions(rl_forest *f, const float *mode_pos);
/* Binary checkpoint of nodes, reservoirs, modes and the round-robin cursor. */
rl_status rl_forest_save(rl_forest *f, const char *path);
rl_status rl_forest_load(rl_ctx *ctx, const char *path, rl_forest **out);

/* ---- scene model (stands in for the fused model of Sec. 3.2.4) -------- */
/* Axis-aligned box room [lo, hi] (metres) rendered analytically by the
 * ranking step's depth raycast. */
rl_status rl_scene_box(rl_ctx *ctx, const double lo[3], const double hi[3], rl_scene **out);
rl_status rl_scene_destroy(rl_scene *s);
/* Eq. 6-7 for n given camera->world poses (HOST [n][16] row-major) against
 * one live depth frame: the box is raycast at each pose (z-depth of the
 * first face hit; exit point from inside, entry point from outside), the
 * masked mean |D_live - D_synth| is taken over pixels valid in both, and
 * the score is +inf when fewer than 10% of the synthetic pixels are valid.
 * scores / valid_frac are HOST [n] (valid_frac may be NULL).  Scratch comes
 * from the context arena (RL_ERR_OOM if it does not fit).  Synchronises
 * `stream`. */
rl_status rl_score_poses(rl_scene *s, const float *depth, const rl_intrinsics *K,
                         const double *poses, int32_t n, rl_mem mem, void *stream,
                         float *scores, float *valid_frac);

/* ICP of n given camera->world poses (HOST [n][16] row-major) against one
 * live depth frame and the box model, with the rl_icp_params rules above.
 * refined: HOST [n][16], the refined pose, or the input pose where ICP
 * failed; ok: HOST [n] 1/0; frac: HOST [n] last-iteration inlier fraction
 * (may be NULL).  Scratch comes from the context arena (RL_ERR_OOM if it
 * does not fit).  Synchronises `stream`. */
rl_status rl_icp_poses(rl_scene *s, const float *depth, const rl_intrinsics *K,
                       const double *poses, int32_t n, const rl_icp_params *p, rl_mem mem,
                       void *stream, double *refined, int32_t *ok, float *frac);

/* Same score as rl_score_poses, for callers that cannot allocate device
 * memory (a real-time loop whose memory is fixed at start-up, a host
 * framework that owns all device memory, code that must not trigger the
 * implicit synchronisation of cudaMalloc/cudaFree).  It allocates nothing:
 * no context or scene handle, no cudaMalloc/cudaFree, no allocating library
 * routine.  The paper has no counterpart of this call.
 *   box_lo/box_hi: HOST double[3], the room box.
 *   depth: DEVICE float [H][W]; poses: DEVICE double [n][16] row-major
 *   camera->world; scores: DEVICE float [n]; valid_frac: DEVICE float [n] or
 *   NULL.  The call only enqueues work on `stream` and returns.
 * Its partial sums live in a fixed 1 MiB device array inside the library
 * (65536 records of one 1024-pixel tile per pose): n * ceil(W*H/1024) must
 * not exceed 65536 (e.g. n <= 218 at 640x480) and n must not exceed 65535,
 * else RL_ERR_INVALID_ARG with the limit in rl_last_error().  Every GPU that
 * loads the library holds the array until the process exits.  All calls
 * share it and it keeps the last call's contents; nothing in it needs to
 * start at zero.  Calls that overlap on the GPU (unordered streams) race on
 * it.  The first call on a device looks up the array's device address with
 * that device current; make that first call before any stream capture.  The
 * address is remembered with the CUDA context it belongs to and looked up
 * again when the device's current context changes (after cudaDeviceReset):
 * the first call after such a reset must likewise come before any capture. */
rl_status rl_score_poses_noalloc(const double box_lo[3], const double box_hi[3],
                                 const float *depth, const rl_intrinsics *K,
                                 const double *poses, int32_t n, void *stream,
                                 float *scores, float *valid_frac);

/* ---- relocaliser (Sec. 3.2.3-3.2.4) ---------------------------------- */
/* Allocates per-query state for up to `max_batch` frames of at most
 * max_width x max_height from the arena.  `scene` may be NULL when
 * p->rank == 0. */
rl_status rl_reloc_create(rl_forest *f, rl_scene *scene, const rl_ransac_params *p,
                          int32_t max_width, int32_t max_height, int32_t max_batch,
                          rl_reloc **out);
rl_status rl_reloc_destroy(rl_reloc *r);
/* Relocalises one frame: Eq. 1-3 leaves for every pixel, N_max hypotheses
 * by Kabsch on checked triples, cull to N_cull by Eq. 5 on eta pixels,
 * preemptive rounds (grow I by eta, LM, re-score, keep the better half),
 * then Eq. 6-8 ranking of the chosen set.  `query_seed` keys every random
 * draw.  Synchronises `stream`; writes *out on RL_OK. */
rl_status rl_relocalise(rl_reloc *r, const float *depth, const uint8_t *rgb,
                        const rl_intrinsics *K, uint64_t query_seed, rl_mem mem, void *stream,
                        rl_result *out);
/* Batched form: n frames of the same size, contiguous ([n][H][W] depth,
 * [n][H][W][3] colour), all work of all frames in the same launches.  Each
 * frame's result is identical to relocalising it alone. */
rl_status rl_relocalise_batch(rl_reloc *r, int32_t n, const float *depth, const uint8_t *rgb,
                              const rl_intrinsics *K, const uint64_t *query_seeds, rl_mem mem,
                              void *stream, rl_result *out);
/* Asynchronous batched form for serving loops: inputs must be DEVICE
 * pointers; nothing is copied back until rl_reloc_fetch. */
rl_status rl_relocalise_batch_async(rl_reloc *r, int32_t n, const float *depth,
                                    const uint8_t *rgb, const rl_intrinsics *K,
                                    const uint64_t *query_seeds, void *stream);
rl_status rl_reloc_fetch(rl_reloc *r, int32_t n, void *stream, rl_result *out);
/* The launch sequence of a call depends only on the batch size and the
 * cascade level; by default it is captured once into a CUDA graph (on a
 * private stream) and replayed on the caller's stream.  enable = 0 launches
 * kernels one by one.  Results are identical either way.  The first call
 * of a given batch size performs the capture and must not itself run under
 * the caller's stream capture. */
rl_status rl_reloc_set_graphs(rl_reloc *r, int32_t enable);
/* Kernel launches in the captured graph of an n-frame call at level 0 (all
 * its sub-batches), in *out; -1 when no such graph is captured (yet, or
 * graphs are off).  A call replaying it launches exactly these kernels. */
rl_status rl_reloc_graph_kernels(rl_reloc *r, int32_t n, int32_t *out);
/* Failure injection for tests of the device-side failure path (the paper
 * has no counterpart).  The LM kernel waits, with a bound, for the bulk
 * copies that stage its mode-table tiles; a wait that runs out marks the
 * frame, the kernel skips the rest of that frame's work, drains its copies
 * in flight (always with the full bound) and the call returns
 * RL_ERR_TIMEOUT.  `probes` sets how many times a tile wait probes before it
 * gives up (0: at once); a negative value restores the default (2^22).
 * Synchronises the device and drops the relocaliser's captured graphs,
 * which hold the limit; a cascade's graphs keep the limit they were captured
 * with. */
rl_status rl_reloc_set_wait_limit(rl_reloc *r, int64_t probes);

/* Intermediate results of frame `q` of the last call (HOST buffers, any may
 * be NULL): per generation slot the 3x4 pose and the iteration that
 * succeeded (-1 failed); the cull survivors (slot, energy) in rank order;
 * the survivors after each preemptive round; the pixel ids of each batch. */
rl_status rl_reloc_debug(rl_reloc *r, int32_t q, double *hyp_pose /* n_hyp*12 */,
                         int32_t *hyp_iter /* n_hyp */, int32_t *cull_slot /* n_cull */,
                         float *cull_energy /* n_cull */, int32_t *round_count /* 16 */,
                         int32_t *round_slot /* 16*n_cull */, float *round_energy /* 16*n_cull */,
                         double *round_pose /* 16*n_cull*12 */, int32_t *batch_pix /* 16*eta */,
                         int32_t *n_rounds);

/* ---- launch-shape tuning ---------------------------------------------- */
/* Launch shapes of the relocaliser's kernels that do not change any result
 * (every kernel computes the same values in the same order for each of
 * them).  Defaults: {16, 128, 128, 256, 8}. */
typedef struct {
    int32_t hypgen_warps;     /* warps (slots) per block of generation: 2, 4, 8 or 16 */
    int32_t energy_threads;   /* at most this many hypotheses per block of Eq. 5: 32, 64, 128 or 256 */
    int32_t leaves_threads;   /* pixels per block of the forest walk: 64, 128, 256 or 512 */
    int32_t mask_threads;     /* pixels per block of the colour-check masks: 64, 128 or 256 */
    int32_t streams;          /* sub-batches of a call run concurrently on this many streams: 1, 2,
                               * 4 or 8 (at most one per 8 frames; a call with profiling on runs as
                               * one batch).  The frames are independent, so every result is the
                               * same as in one batch. */
} rl_tuning;

rl_status rl_reloc_get_tuning(rl_reloc *r, rl_tuning *out);
/* RL_ERR_INVALID_ARG for a value outside the lists above.  Drops the
 * relocaliser's captured CUDA graphs (they hold the old launch shapes). */
rl_status rl_reloc_set_tuning(rl_reloc *r, const rl_tuning *t);
/* Autotuner.  If cache_path (may be NULL) holds an entry for this
 * relocaliser's key (rl_tuning_key), applies it.  Otherwise times every
 * candidate of each knob in turn on n given frames (calls of
 * rl_relocalise_batch with per-kernel CUDA-event timing, two per
 * candidate), keeps the fastest (ties: the current value), applies the
 * result and, with a cache_path, records it there.  *out (may be NULL)
 * receives the tuning in use.  The paper has no counterpart. */
rl_status rl_reloc_autotune(rl_reloc *r, int32_t n, const float *depth, const uint8_t *rgb,
                            const rl_intrinsics *K, const uint64_t *seeds, rl_mem mem, void *stream,
                            const char *cache_path, rl_tuning *out);
/* Cache key of a relocaliser: device name and SM count, maximum frame size
 * and batch, and the parameters that shape its kernels.  RL_ERR_INVALID_ARG
 * if buf (len bytes) is too small. */
rl_status rl_tuning_key(rl_reloc *r, char *buf, int32_t len);
/* Tuning cache (text file, one "key = w e l m" line per key).  Host only.
 * read: *found = 0 if the file or the key is absent (RL_OK).  write:
 * replaces the key's line or appends it; RL_ERR_IO on file errors. */
rl_status rl_tuning_cache_read(const char *path, const char *key, rl_tuning *out, int32_t *found);
rl_status rl_tuning_cache_write(const char *path, const char *key, const rl_tuning *t);

/* ---- tracing ---------------------------------------------------------- */
/* Per-kernel timing of a relocaliser: when enabled, every kernel launch of
 * its calls is bracketed by CUDA events on the caller's stream; durations
 * and launch counts accumulate per kernel (ids 0..RL_N_KERNELS-1, names
 * from rl_kernel_name), and the kernels count their work units (uint64
 * [RL_N_WORK]: energy (H,px) pairs, energy (H,px,mode) triples, LM (H,px)
 * nearest-mode searches, LM (H,px,mode) triples, LM inlier accumulations,
 * LM trial evaluations, rays cast, generation attempts (stage 1: draws and
 * colour check), generation stage-2 evaluations (spread and rigidity), ICP
 * pixel evaluations (valid pixels visited, over all iterations), ranking rays
 * re-evaluated in FP64 (hit decision within the FP32 margin), LM
 * (H,px,mode) distances actually evaluated (below the LM triples where a
 * certified bound settled the nearest mode without a full search)).
 * Enabling resets all counters.  The
 * paper has no counterpart; its Sec. A.1 timing breakdown is per stage. */
#define RL_N_KERNELS 12
#define RL_N_WORK 12
rl_status rl_reloc_profile(rl_reloc *r, int32_t enable);
rl_status rl_reloc_profile_read(rl_reloc *r, double *ms /* [RL_N_KERNELS] */,
                                int64_t *launches /* [RL_N_KERNELS] */,
                                uint64_t *work /* [RL_N_WORK] */);
const char *rl_kernel_name(int32_t kernel_id);

/* ---- cascade (Sec. 3.2.5) -------------------------------------------- */
/* Levels run in order on the same frame; level l works on the frame
 * subsampled by subsample[l] (pixel (s*u, s*v), intrinsics / s) and falls
 * back to level l+1 iff its score exceeds thresholds[l].  The levels must
 * share one forest, be distinct relocalisers, and the last level works at
 * full resolution (subsample 1).  All levels of a call are enqueued at once
 * (one CUDA graph per batch size): the fall-back decision is taken on the
 * device, frames accepted early become empty frames for later levels, and
 * results come back in one copy.  The cascade keeps pointers to the levels
 * (RL_ERR_BUSY on destroying a level first). */
rl_status rl_cascade_create(rl_reloc *const *levels, const double *thresholds,
                            const int32_t *subsample, int32_t n_levels, rl_cascade **out);
rl_status rl_cascade_destroy(rl_cascade *c);
rl_status rl_cascade_relocalise(rl_cascade *c, const float *depth, const uint8_t *rgb,
                                const rl_intrinsics *K, uint64_t query_seed, rl_mem mem,
                                void *stream, rl_result *out);
/* Batched cascade: each frame falls back independently; all frames of a
 * level run in the same launches. */
rl_status rl_cascade_relocalise_batch(rl_cascade *c, int32_t n, const float *depth,
                                      const uint8_t *rgb, const rl_intrinsics *K,
                                      const uint64_t *query_seeds, rl_mem mem, void *stream,
                                      rl_result *out);

/* ---- serving loop ---------------------------------------------------- */
/* A server relocalises requests from many camera streams against several
 * models (one forest + scene + relocaliser parameters each, e.g. one per
 * room), with frames of any size up to the model's maximum.  Each model has
 * a worker thread and two device slots of max_batch frames: while one batch
 * runs, everything that arrived meanwhile is staged into the other (batches
 * form continuously from the queue; models overlap on separate streams).
 * Admission: a request's staged bytes (W*H*7) count against memory_budget
 * until its result is fetched; over budget, submit returns RL_ERR_ADMISSION
 * unless queue_when_full, in which case the request waits on the host.  A
 * frame's result is identical whatever batch it joins.  The paper has no
 * counterpart (it relocalises one frame at a time). */
typedef struct rl_server rl_server;

typedef struct {
    int32_t max_batch;        /* frames per device slot */
    int32_t queue_when_full;  /* 1: queue over-budget requests, 0: refuse them */
    uint64_t memory_budget;   /* bytes of admitted frame data */
} rl_server_params;

typedef struct {
    uint64_t submitted, completed, refused;
    uint64_t peak_admitted_bytes;
    double p50_ms, p99_ms, mean_ms;  /* submit -> result available */
    double frames_per_s;             /* completed / (last completion - first submit) */
} rl_server_stats;

rl_status rl_server_create(rl_ctx *ctx, const rl_server_params *p, rl_server **out);
/* Adds a model; allocates two relocalisers of max_batch frames from the
 * context arena and starts its worker thread. */
rl_status rl_server_add_model(rl_server *s, rl_forest *f, rl_scene *scene,
                              const rl_ransac_params *p, int32_t max_width, int32_t max_height,
                              int32_t *model_id);
/* Adds a cascade model (Sec. 3.2.5): per slot, one relocaliser per level
 * (levels[l] parameters, input subsampled by subsample[l], the last level at
 * full resolution) chained as by rl_cascade_create with thresholds [L-1];
 * requests to it return the cascade's result (level = the accepting level). */
rl_status rl_server_add_cascade_model(rl_server *s, rl_forest *f, rl_scene *scene,
                                      const rl_ransac_params *levels, const int32_t *subsample,
                                      const double *thresholds, int32_t n_levels, int32_t max_width,
                                      int32_t max_height, int32_t *model_id);
/* Copies the HOST frame and enqueues it; *ticket identifies the request. */
rl_status rl_server_submit(rl_server *s, int32_t model, const float *depth, const uint8_t *rgb,
                           const rl_intrinsics *K, uint64_t query_seed, uint64_t *ticket);
/* *done = 1 and *out filled (ticket released) once the result is ready. */
rl_status rl_server_poll(rl_server *s, uint64_t ticket, int32_t *done, rl_result *out);
/* Waits at most timeout_ms; RL_ERR_TIMEOUT if the result is not ready
 * (the ticket stays valid). */
rl_status rl_server_wait(rl_server *s, uint64_t ticket, uint32_t timeout_ms, rl_result *out);
rl_status rl_server_get_stats(rl_server *s, rl_server_stats *out);
/* Clears the counters and latencies of rl_server_get_stats (requests in
 * flight and tickets are unaffected), e.g. after a warm-up. */
rl_status rl_server_reset_stats(rl_server *s);
/* Finishes queued work, stops the workers and releases the models. */
rl_status rl_server_destroy(rl_server *s);

#ifdef __cplusplus
}
#endif
#endif
