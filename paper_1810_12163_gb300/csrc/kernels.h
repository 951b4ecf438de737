// Argument blocks and launchers of the relocaliser kernels.
#pragma once
#include "internal.h"

namespace rl {

struct EnergyArgs {
    const double *pose;        // pose (12 doubles) of hypothesis i of frame b:
    int pose_stride;           //   pose[(b*pose_stride + idx) * 12]
    const int32_t *idx;        // idx[b*idx_stride + i] or i when null
    int idx_stride;
    const int32_t *count;      // hypotheses of frame b
    const int32_t *pix;        // [B][max_pix]
    const float4 *xc;          // [B][max_pix]
    int max_pix, n_pix;
    const uint16_t *leaves;
    int hw_max;
    ModeView mv;
    RParams p;
    int chunk, maxm;
    float *part;               // [B][part_h][n_chunks]
    int part_h, n_chunks;
    int round_gate;            // skip frames whose round is inactive
    unsigned long long *work;  // profiling counters or null
    const uint16_t *mcount;    // [B][hw_max] |M(u)|
    const uint4 *prec;         // [B][hw_max] pixel records or null
    const float4 *q_tab0;      // mode table of the pixel set (rows of p.mpad)
    const float4 *q_tab1;
    const float *q_tab2;
    const int16_t *q_tab_cnt;
};

// Mode table of pixel batch `batch` (decoded M(u) of each drawn pixel).
rl_status launch_build_table(const QueryState &q, int hw_max, ModeView mv, const RParams &p, int batch,
                             int n, cudaStream_t s);

struct SelectArgs {
    int phase, round;
    const float *part;
    int part_h, n_chunks_used, n_chunks;
    const int32_t *count;        // n_hyp (cull) or n_cur (round)
    const double *hyp_pose;      // cull source [B][N][12]
    const int32_t *hyp_list;     // cull source slots [B][N]
    QueryState q;
    RParams p;
    int n_pix;                   // |I| after this phase
    int energy_from_lm;          // rounds: the LM kernel left each survivor's energy in q.cur_energy
};

struct LmArgs {
    QueryState q;
    const uint16_t *leaves;
    int hw_max;
    ModeView mv;
    RParams p;
    int n_pix;
    unsigned long long *work;  // profiling counters or null
    int maxm;                  // |M(u)| bound: trees x min(k_top, m_max)
    int maxm_pad;              // maxm rounded up to an odd count (shared-memory rows)
    uint32_t wait_limit;       // probes of a wait for a staged tile before it gives up
};

rl_status prepare_kernels();

// LM with one thread-block cluster per frame (at most 64 hypotheses); its
// shared memory grows with the padded row length, and above
// kLmClusterSmemMax the other LM kernels are used.
constexpr size_t kLmClusterSmemMax = 200 * 1024;
size_t lm_cluster_smem(int mpad, bool cov);
rl_status launch_lm_cluster(const LmArgs &a, int n, cudaStream_t s);
// True when a round's LM runs in the cluster kernel (which also leaves each
// refined pose's Eq. 5 energy in q.cur_energy).
bool lm_uses_cluster(const RParams &p);
rl_status prepare_lm_cluster();

// Ranking raycast tiles: 256 threads x RC_PIX pixels; one partial record
// per (frame, pose, tile).
constexpr int RC_PIX = 2;
constexpr int RC_TILE = 256 * RC_PIX;

struct RaycastArgs {
    const Frame *frames;
    const double *poses;       // [B][pose_cap][12]
    const int32_t *n_poses;    // poses per frame, or null: pose_cap for every frame
    int pose_cap;
    float lo[3], hi[3];
    double lo64[3], hi64[3];
    double *part_sum;          // [B][pose_cap][n_tiles]
    int32_t *part_cnt;         // [B][pose_cap][n_tiles][2]
    int n_tiles;
    unsigned long long *work;  // profiling counters or null
    __device__ int n_poses_of(int b) const { return n_poses ? n_poses[b] : pose_cap; }
    __device__ const double *pose_of(int b, int c) const {
        return poses + ((size_t)b * pose_cap + c) * 12;
    }
};

// ICP of Sec. 3.2.4 (one thread block per pose): pose c of frame b is
// poses[(b * pose_stride + c) * 12], refined in place when ICP succeeds.
struct IcpArgs {
    const Frame *frames;
    double *poses;             // [B][pose_stride][12]
    int pose_stride;
    const int32_t *counts;     // poses per frame, or null: `cap` for every frame
    const int32_t *gate;       // frames with gate[b] <= 0 are skipped, or null
    int cap;                   // poses per frame when counts is null / grid width
    int32_t *ok;               // [B][out_stride]
    float *frac;               // [B][out_stride]
    int out_stride;
    float lo[3], hi[3];
    IcpParams ip;
    unsigned long long *work;  // profiling counters or null
};
rl_status launch_icp(const IcpArgs &a, int n, cudaStream_t s);

size_t energy_smem(int chunk, int maxm);
rl_status launch_energy(const EnergyArgs &a, int max_count, int n, cudaStream_t s, int max_threads = 128);
rl_status launch_select(const SelectArgs &a, int n, cudaStream_t s);
rl_status launch_lm(const LmArgs &a, int n, cudaStream_t s);
rl_status launch_raycast(const RaycastArgs &a, int n, int max_hw, cudaStream_t s);
rl_status launch_score_poses(const RaycastArgs &a, int n_poses, int npx, float *scores,
                             float *valid_frac, cudaStream_t s);
rl_status launch_finalize(const QueryState &q, const RParams &p, int n_tiles, int ranked, int n,
                          cudaStream_t s);
rl_status launch_hypgen(const Frame *frames, const uint16_t *leaves, const uint16_t *mcount,
                        const uint4 *prec, const uint2 *pcm, const uint32_t *pbits, int hw_max, ModeView mv,
                        const RParams &p, double *hyp_pose, int32_t *hyp_iter, unsigned long long *work, int n,
                        cudaStream_t s, int warps = 16);
// Generation stages the frame's non-empty-M(u) bitmap (W*H/8 bytes) in shared
// memory when it fits this bound (640x480: 38.4 KB).
constexpr size_t kHypBitsSmemMax = 64 * 1024;
rl_status prepare_hypgen();
// Largest |M(u)| the colour-check masks cover.
constexpr int kMaskModes = 56;
rl_status launch_colour_mask(const Frame *frames, const uint16_t *mcount, const uint4 *prec, int hw_max,
                             ModeView mv, const RParams &p, uint2 *pcm, uint32_t *pbits, int n, int max_hw,
                             cudaStream_t s, int threads = 256);
rl_status launch_hyppose(const Frame *frames, const uint16_t *leaves, const uint16_t *mcount,
                         const uint4 *prec, int hw_max, ModeView mv, const RParams &p,
                         double *hyp_pose, int32_t *hyp_iter, int n, cudaStream_t s);
rl_status launch_compact(const int32_t *hyp_iter, int N, int32_t *hyp_list, int32_t *n_hyp, int n,
                         cudaStream_t s);
rl_status launch_sample_batch(const Frame *frames, const uint16_t *mcount, const uint4 *prec, int hw_max,
                              const RParams &p, int batch, int32_t *pix, float4 *xc, int n,
                              cudaStream_t s);
rl_status launch_subsample(const Frame *src, Frame *dst_desc, float *dst_depth, uint8_t *dst_rgb,
                           int s_factor, int n, int max_w, int max_h, cudaStream_t s);

}  // namespace rl
