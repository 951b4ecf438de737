// Internal declarations of the relocgb library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/relocgb.h"

// ---------------------------------------------------------------------------
// Error plumbing: every ABI entry point returns rl_status; the message of the
// last failure is kept per thread.
// ---------------------------------------------------------------------------
namespace rl {
void set_error(const std::string &msg);
rl_status fail(rl_status s, const std::string &msg);
rl_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);
}  // namespace rl

#define RL_CK(call)                                                               \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) return rl::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define RL_TRY(call)                         \
    do {                                     \
        rl_status s_ = (call);               \
        if (s_ != RL_OK) return s_;          \
    } while (0)

#define RL_LAUNCH_CK() RL_CK(cudaGetLastError())

// ---------------------------------------------------------------------------
// Arena: first-fit sub-allocator over the caller's device buffer.  Host-side
// bookkeeping only; no device allocation ever happens after context creation.
// ---------------------------------------------------------------------------
struct rl_ctx {
    int device = 0;
    uint8_t *base = nullptr;
    uint64_t bytes = 0;
    uint64_t used = 0, peak = 0;
    std::map<uint64_t, uint64_t> live;  // offset -> size
    std::mutex mu;
    int sm_count = 0;
};

namespace rl {
rl_status arena_alloc(rl_ctx *c, uint64_t bytes, void **out);
void arena_free(rl_ctx *c, void *p);
template <class T>
rl_status alloc_n(rl_ctx *c, uint64_t n, T **out) {
    void *p = nullptr;
    rl_status s = arena_alloc(c, n * sizeof(T), &p);
    *out = static_cast<T *>(p);
    return s;
}
}  // namespace rl

// ---------------------------------------------------------------------------
// Forest and its leaf models.
// ---------------------------------------------------------------------------
// The arrays of one mode store (a streaming forest keeps two of them).
struct ModeStore {
    uint8_t *nmodes = nullptr;
    float4 *centroid = nullptr;
    ushort4 *mpos_h = nullptr;
    float4 *mpos_f = nullptr;
    uchar4 *mrgb = nullptr;
    float4 *mU = nullptr;
    int32_t *msize = nullptr;
};

struct rl_reloc;

struct rl_forest {
    rl_ctx *ctx = nullptr;
    rl_forest_params p{};
    uint64_t seed = 0;
    int n_branch = 0;          // per tree, 2^d - 1
    int leaves_per_tree = 0;   // 2^d
    int n_leaves = 0;          // T * 2^d
    // split nodes [T][n_branch]: (dx, dy, tau, meta) with meta = type | channel << 8
    float4 *nodes = nullptr;
    // reservoirs [L][kappa]: (x, y, z, rgb packed into the low 24 bits)
    float4 *res = nullptr;
    uint32_t *res_count = nullptr;  // [L]
    // modes [L][m_max]
    uint8_t *nmodes = nullptr;      // [L]
    float4 *centroid = nullptr;     // [L]
    ushort4 *mpos_h = nullptr;      // FP16 offsets from centroid
    float4 *mpos_f = nullptr;       // FP32 positions
    uchar4 *mrgb = nullptr;
    float4 *mU = nullptr;           // [L][m_max][2]: U00 U01 U02 U11 | U12 U22 0 0
    int32_t *msize = nullptr;
    // adaptation scratch
    uint32_t *ex_leaf = nullptr;    // [T][grid pixels]
    float4 *ex_pt = nullptr;        // [grid pixels]
    uint32_t *ex_rank = nullptr;    // [T][grid pixels]
    uint32_t *frame_cnt = nullptr;  // [L]
    int ex_capacity = 0;
    float *stage_depth = nullptr;
    uint8_t *stage_rgb = nullptr;
    int stage_pixels = 0;
    int64_t cursor = 0;             // round-robin mode update
    int refcount = 0;
    // Streaming adaptation: the mode arrays above are the front store that
    // relocalisers read; `alt` is the back store that the next mode update
    // writes before the two are swapped (see rl_forest_set_streaming).
    bool streaming = false;
    ModeStore alt{};
    int mode_buf = 0;                          // id of the front store (0/1): part of graph keys
    int64_t last_begin = 0, last_count = 0;    // leaves the back store lacks (written by the last update)
    cudaEvent_t ready = nullptr;               // recorded after the last update on its stream
    std::vector<rl_reloc *> readers;           // relocalisers of this forest
    std::mutex mu;                             // front/back bookkeeping against concurrent launches
};

struct rl_scene {
    rl_ctx *ctx = nullptr;
    double lo[3], hi[3];
};

// Relocalisers using at most this many trees keep a 16-byte per-pixel record
// (leaf ids and per-tree mode counts) next to the leaf maps.
constexpr int kRecTrees = 5;

// Device-side view of the mode store used by the relocaliser kernels.
struct ModeView {
    const uint8_t *nmodes;
    const float4 *centroid;
    const ushort4 *mpos_h;  // null when FP32
    const float4 *mpos_f;   // null when FP16
    const uchar4 *mrgb;
    const float4 *mU;
    int m_max;
    int leaves_per_tree;
};

// ICP settings of Sec. 3.2.4 (see rl_icp_params), as the kernels read them.
struct IcpParams {
    int levels, stride[3], iters[3];
    float dist[3];
    double min_frac, ridge;
};

// Relocaliser parameters as passed to kernels.
struct RParams {
    int n_hyp, max_iter, n_cull, eta, k_out, pose_update, use_cov, colour_thresh;
    double min_sq_dist, max_trans_err;
    int k_top, n_trees, lm_max_iter, batch_attempts;
    double lm_lambda0, lm_inlier_thresh, lm_stop;
    int rank, halve_to_one;
    int level;        // cascade level, part of every random counter
    int max_rounds;   // preemptive rounds for this configuration
    int max_pix;      // eta * (max_rounds + 1)
    int maxm;         // bound on |M(u)|: trees x min(k_top, m_max)
    int mpad;         // maxm rounded up to an odd count (mode-table row stride)
    int icp;          // ICP before ranking (or of the output pose when unranked)
    int redraw;       // generation redraws an unusable pixel within its iteration
    IcpParams icp_p;
};

// Per-frame description used by batched kernels.
struct Frame {
    const float *depth;
    const uint8_t *rgb;
    float fx, fy, cx, cy;
    int W, H;
    uint32_t key0, key1;
};

// Probes of the LM kernel's bounded waits on its own bulk copies.
constexpr uint32_t kLmWaitLimit = 1u << 22;

// Device-resident per-query RANSAC state (arrays sized for max_batch).
struct QueryState {
    uint16_t *leaves;        // [B][T][HWmax]
    uint16_t *mcount;        // [B][HWmax] |M(u)| per pixel
    uint4 *prec;             // [B][HWmax] per-pixel leaves + counts (<= 5 trees), else null
    uint2 *pcm;              // [B][HWmax] colour-check bits of M(u) | |M(u)| << 56 (|M(u)| <= 56), else null
    uint32_t *pbits;         // [B][HWmax / 32 + 1] bit p: M(u) of pixel p is non-empty (with pcm)
    double *hyp_pose;        // [B][N][12]
    int32_t *hyp_iter;       // [B][N]
    int32_t *hyp_list;       // [B][N] slots of successful hypotheses
    int32_t *n_hyp;          // [B]
    int32_t *pix;            // [B][max_pix] pixel ids (-1 skipped)
    float4 *xc;              // [B][max_pix] camera points
    // Mode table of the pixel set: M(u) of every pixel of I decoded once
    // when its batch is drawn, rows of mpad records
    float4 *tab0;            // [B][max_pix][mpad] mu.xyz, U00
    float4 *tab1;            // [B][max_pix][mpad] U01 U02 U11 U12
    float *tab2;             // [B][max_pix][mpad] U22
    int16_t *tab_cnt;        // [B][max_pix] |M(u)| (0 for a skipped draw)
    float4 *lm_anc;          // [B][n_cull][max_pix] LM nearest-mode anchors: y, slack^2 with
                             // the nearest mode in its low 8 bits
    int32_t *n_pix;          // [B]
    double *cur_pose;        // [B][n_cull][12]
    int32_t *cur_slot;       // [B][n_cull]
    float *cur_energy;       // [B][n_cull]
    int32_t *n_cur;          // [B]
    int32_t *cull_slot;      // [B][n_cull] survivors of the initial cull
    float *cull_energy;      // [B][n_cull]
    float *energy_part;      // [B][max(N, n_cull)][n_chunks]
    float *cand_energy;      // [B][N] (cull) energies
    int32_t *corr;           // [B][n_cull][max_pix] LM correspondences
    double *chosen_pose;     // [B][16][12]
    float *chosen_energy;    // [B][16]
    int32_t *chosen_slot;    // [B][16]
    int32_t *chosen_npix;    // [B]
    int32_t *n_chosen;       // [B]
    double *score_part;      // [B][16][n_score_tiles][2] sum, counts
    int32_t *score_cnt;      // [B][16][n_score_tiles][2]
    float *chosen_score;     // [B][16]
    int32_t *icp_ok;         // [B][16] ICP succeeded (ranked: chosen pose c; unranked: slot 0)
    float *icp_frac;         // [B][16] last-iteration inlier fraction, -1 if ICP did not run
    int32_t *round_count;    // [B][16]
    int32_t *round_slot;     // [B][16][n_cull]
    float *round_energy;     // [B][16][n_cull]
    double *round_pose;      // [B][16][n_cull][12]
    int32_t *n_rounds;       // [B]
    Frame *frames;           // [B]
    uint8_t *result_blob;    // [B] device results (DevResult)
    int32_t *dev_err;        // [B] nonzero: a bounded device-side wait gave up
};

struct DevResult {
    double pose[12];
    float energy, energy_per_pixel, score;
    int32_t n_hypotheses, n_chosen, n_pixels, status, best, err, icp_mask, pad;
};

// Per-kernel timing with CUDA events recorded on the launching stream, plus
// device-side work counters of the scoring kernels (off unless enabled).
enum KernelId {
    K_LEAVES = 0, K_HYPGEN, K_COMPACT, K_SAMPLE, K_ENERGY, K_SELECT, K_LM, K_RAYCAST, K_FINALIZE,
    K_HYPPOSE, K_CMASK, K_ICP, K_COUNT
};
// work counters: energy (H,px) pairs, energy (H,px,mode) triples, LM pass-1
// (H,px) evaluations, LM (H,px,mode) triples of the nearest-mode searches
// the method defines, LM inlier accumulations, LM pass-2 evaluations,
// raycast rays, generation attempts and stage-2 evaluations, ICP
// valid-pixel evaluations, raycast rays re-evaluated in FP64, LM
// (H,px,mode) distances actually evaluated (fewer than the method's triples
// where a certified bound settles the nearest mode)
enum WorkId {
    W_E_PAIRS = 0, W_E_MODES, W_LM_PAIRS, W_LM_MODES, W_LM_INLIERS, W_LM_TRIAL, W_RAYS, W_HYP_ATTEMPTS,
    W_HYP_STAGE2, W_ICP_PIX, W_RAY64, W_LM_EVALS, W_COUNT
};

struct Profiler {
    bool on = false;
    struct Pending {
        int kid;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[K_COUNT] = {};
    int64_t launches[K_COUNT] = {};
    unsigned long long *work = nullptr;  // device [W_COUNT]
};

struct rl_reloc {
    rl_forest *forest = nullptr;
    rl_scene *scene = nullptr;
    rl_ransac_params p{};
    RParams rp{};
    int max_w = 0, max_h = 0, max_batch = 0;
    int n_chunks = 0;        // energy partial-sum chunks per hypothesis
    int n_score_tiles = 0;
    QueryState q{};
    float *stage_depth = nullptr;
    uint8_t *stage_rgb = nullptr;
    std::vector<void *> allocs;
    Frame *host_frames = nullptr;  // pinned mirror of q.frames
    DevResult *host_results = nullptr;
    int last_batch = 0;
    int refcount = 0;
    Profiler prof;
    // Captured launch sequences keyed by (batch size, cascade level, front
    // mode store of the forest).
    struct Graph {
        int n, level, buf;
        cudaGraphExec_t exec;
        uint64_t last_use;
        int kernels;  // kernel nodes of the graph
    };
    std::vector<Graph> graphs;
    cudaStream_t capture_stream = nullptr;
    bool use_graphs = true;
    uint64_t calls = 0;
    rl_tuning tune{16, 128, 128, 256, 8};  // launch shapes (results do not depend on them)
    uint64_t tune_gen = 0;                    // bumped by every rl_reloc_set_tuning
    float4 *nodes_s = nullptr;                // split nodes scaled for the call's focal length
    // per array of q: byte offset of its pointer in QueryState and bytes per frame
    std::vector<std::pair<size_t, size_t>> q_layout;
    // sub-batches of a call (tune.streams): private streams and fork/join events
    cudaStream_t side[7] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[7] = {};
    uint32_t lm_wait_limit = kLmWaitLimit;  // probes of the LM kernel's waits for staged tiles
    // streaming forests: recorded after the last launch that read mode store b
    cudaEvent_t read_done[2] = {nullptr, nullptr};
    bool read_valid[2] = {false, false};
};

// Per-frame output of a cascade, written on the device by each level's
// fall-back decision.
struct CascadeOut {
    DevResult *res;          // [B]
    double *chosen_pose;     // [B][16][12]
    float *chosen_energy;    // [B][16]
    float *chosen_score;     // [B][16]
    float *icp_frac;         // [B][16] ICP inlier fractions of the level that produced the result
    int32_t *chosen_slot;    // [B][16]
    int32_t *level;          // [B]
    int32_t *done;           // [B] accepted by some level
};

struct rl_cascade {
    std::vector<rl_reloc *> levels;
    std::vector<double> thresholds;
    std::vector<int32_t> subsample;
    rl_ctx *ctx = nullptr;
    int max_batch = 0;
    CascadeOut out{};
    Frame *full_dev = nullptr;            // [B] full-resolution frames
    std::vector<void *> allocs;
    struct Graph {
        int n, buf;
        uint64_t tune_gen;  // sum of the levels' tune_gen at capture
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    // sub-batches of a call (the first level's tune.streams): private streams and fork/join events
    cudaStream_t side[7] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[7] = {};
    cudaStream_t capture_stream = nullptr;
    bool use_graphs = true;
};

// ---------------------------------------------------------------------------
// Device helpers shared by the kernels of this library.
// ---------------------------------------------------------------------------
namespace rl {

enum : uint32_t { TAG_FOREST = 1, TAG_RESERVOIR = 2, TAG_HYP = 3, TAG_BATCH = 4, TAG_REDRAW = 5 };

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the multiply-xor round
// with Weyl-sequence key schedule.
__host__ __device__ inline uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    }
    return c;
}

// 32-bit draw -> [0, n) by multiply-shift.
__host__ __device__ inline uint32_t draw_below(uint32_t u, uint32_t n) {
    return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

}  // namespace rl

// Launch helpers (defined in the .cu files).
namespace rl {
rl_status launch_forest_random(rl_forest *f, cudaStream_t s);
rl_status launch_leaves(const rl_forest *f, const Frame *frames_dev, int n_frames, int n_trees,
                        int hw_max, uint16_t *out, int max_w, int max_h, cudaStream_t s,
                        int k_top = 0, uint16_t *mcount = nullptr, uint4 *prec = nullptr,
                        int threads = 128, const float4 *nodes_s = nullptr, float fx_s = 0.f);
// The first n_trees trees' split nodes with offsets premultiplied by fx / 585
// into out (read by launch_leaves for frames of that focal length).
rl_status launch_scale_nodes(const rl_forest *f, int n_trees, float4 *out, float fx, cudaStream_t s);
rl_status adapt_frame(rl_forest *f, const float *depth, const uint8_t *rgb,
                      const rl_intrinsics *K, const double T[16], cudaStream_t s);
rl_status update_modes(rl_forest *f, int64_t begin, int64_t count, cudaStream_t s);
rl_status reset_leaves(rl_forest *f, cudaStream_t s);
ModeView mode_view(const rl_forest *f);
// The launch sequence of n frames whose query state is q (r->q, or a slice
// of it for a sub-batch: query_slice).
rl_status run_relocalise(rl_reloc *r, const QueryState &q, int n, int level, cudaStream_t s);
// q for the frames b0, b0 + 1, ... of r's batch.
QueryState query_slice(const rl_reloc *r, int b0);
// Batch of n frames whose descriptors (device pointers, per-frame sizes and
// intrinsics, keys) are given on the host: descriptors are copied and the
// launch sequence is enqueued on s (graph replay when enabled).
rl_status reloc_enqueue_frames(rl_reloc *r, int n, const Frame *frames, cudaStream_t s);
// Copies the results of the last n frames back and waits for s.
// Cascade counterparts: frames in the last level's host_frames.
rl_status cascade_enqueue_frames(rl_cascade *c, int n, cudaStream_t s);
rl_status cascade_fetch_results(rl_cascade *c, int n, cudaStream_t s, rl_result *out);
rl_status reloc_fetch_results(rl_reloc *r, int n, cudaStream_t s, rl_result *out);
}  // namespace rl
