// Relocaliser and cascade handles: per-query device state, the launch
// sequence of one relocalisation (Sec. 3.2.3-3.2.4), results and the
// cascade's fall-back rule (Sec. 3.2.5).
#include <math.h>
#include <string.h>

#include <stddef.h>

#include <algorithm>
#include <chrono>
#include <memory>

#include "kernels.h"

namespace rl {

static int rounds_for(int n_cull, int k_out, int halve_to_one) {
    int m = n_cull, r = 0;
    while (m > k_out || (halve_to_one && m > 1)) {
        m = (m + 1) / 2;
        ++r;
    }
    return r;
}

static rl_status check_ransac(const rl_ransac_params *p, const rl_forest *f) {
    if (!p) return fail(RL_ERR_INVALID_ARG, "null relocaliser params");
    if (p->n_hyp < 1 || p->n_hyp > 4096) return fail(RL_ERR_INVALID_ARG, "n_hyp must be 1..4096");
    if (p->max_iter < 1 || p->max_iter > (1 << 30) - 64)
        return fail(RL_ERR_INVALID_ARG, "max_iter must be in [1, 2^30 - 64]");
    if (p->n_cull < 1 || p->n_cull > 64) return fail(RL_ERR_INVALID_ARG, "n_cull must be 1..64");
    if (p->eta < 1 || p->eta > 4096) return fail(RL_ERR_INVALID_ARG, "eta must be 1..4096");
    if (p->k_out < 1 || p->k_out > RL_MAX_CHOSEN) return fail(RL_ERR_INVALID_ARG, "k_out must be 1..16");
    if (p->k_top < 1) return fail(RL_ERR_INVALID_ARG, "k_top must be >= 1");
    if (p->n_trees_used < 1 || p->n_trees_used > f->p.n_trees)
        return fail(RL_ERR_INVALID_ARG, "n_trees_used must be 1..forest trees");
    if (p->batch_attempts < 1) return fail(RL_ERR_INVALID_ARG, "batch_attempts must be >= 1");
    if (p->lm_max_iter < 0) return fail(RL_ERR_INVALID_ARG, "lm_max_iter must be >= 0");
    if (p->colour_thresh < 0) return fail(RL_ERR_INVALID_ARG, "colour_thresh must be >= 0");
    if (p->icp != 0 && p->icp != 1) return fail(RL_ERR_INVALID_ARG, "icp must be 0 or 1");
    if (p->redraw != 0 && p->redraw != 1) return fail(RL_ERR_INVALID_ARG, "redraw must be 0 or 1");
    return RL_OK;
}

static rl_status check_icp(const rl_icp_params *ip) {
    if (!ip) return fail(RL_ERR_INVALID_ARG, "null ICP params");
    if (ip->levels < 1 || ip->levels > 3) return fail(RL_ERR_INVALID_ARG, "icp levels must be 1..3");
    for (int l = 0; l < ip->levels; ++l) {
        if (ip->stride[l] < 1 || ip->stride[l] > 16) return fail(RL_ERR_INVALID_ARG, "icp stride must be 1..16");
        if (ip->iters[l] < 1 || ip->iters[l] > 50) return fail(RL_ERR_INVALID_ARG, "icp iters must be 1..50");
        if (!(ip->dist[l] > 0.0) || !(ip->dist[l] < 1e6)) return fail(RL_ERR_INVALID_ARG, "icp dist must be > 0");
    }
    if (!(ip->min_frac >= 0.0 && ip->min_frac <= 1.0)) return fail(RL_ERR_INVALID_ARG, "icp min_frac must be 0..1");
    if (!(ip->ridge >= 0.0 && ip->ridge < 1e6)) return fail(RL_ERR_INVALID_ARG, "icp ridge must be >= 0");
    return RL_OK;
}

static IcpParams icp_device_params(const rl_icp_params &ip) {
    IcpParams d{};
    d.levels = ip.levels;
    for (int l = 0; l < 3; ++l) {
        d.stride[l] = ip.stride[l];
        d.iters[l] = ip.iters[l];
        d.dist[l] = (float)ip.dist[l];
    }
    d.min_frac = ip.min_frac;
    d.ridge = ip.ridge;
    return d;
}

template <class T>
static rl_status ralloc(rl_reloc *r, uint64_t n, T **out) {
    RL_TRY(alloc_n(r->forest->ctx, n, out));
    r->allocs.push_back(*out);
    return RL_OK;
}

static void prof_free(rl_reloc *r);
static void graphs_free(rl_reloc *r);

static void reloc_release(rl_reloc *r) {
    prof_free(r);
    graphs_free(r);
    for (int i = 0; i < 7; ++i) {
        if (r->side[i]) cudaStreamDestroy(r->side[i]);
        if (r->join_ev[i]) cudaEventDestroy(r->join_ev[i]);
        r->side[i] = nullptr;
        r->join_ev[i] = nullptr;
    }
    if (r->fork_ev) cudaEventDestroy(r->fork_ev);
    r->fork_ev = nullptr;
    for (void *p : r->allocs) arena_free(r->forest->ctx, p);
    r->allocs.clear();
    if (r->host_frames) cudaFreeHost(r->host_frames);
    if (r->host_results) cudaFreeHost(r->host_results);
    r->host_frames = nullptr;
    r->host_results = nullptr;
}

// Host mirrors of the per-query outputs copied back after each call.
struct HostOut {
    DevResult res;
};

static rl_status set_frames(rl_reloc *r, int n, const float *depth, const uint8_t *rgb,
                            const rl_intrinsics *K, const uint64_t *seeds, cudaStream_t s) {
    const size_t hw = (size_t)K->width * K->height;
    for (int i = 0; i < n; ++i) {
        Frame &f = r->host_frames[i];
        f.depth = depth + hw * i;
        f.rgb = rgb + hw * 3 * i;
        f.fx = K->fx; f.fy = K->fy; f.cx = K->cx; f.cy = K->cy;
        f.W = K->width; f.H = K->height;
        f.key0 = (uint32_t)seeds[i];
        f.key1 = (uint32_t)(seeds[i] >> 32);
    }
    RL_CK(cudaMemcpyAsync(r->q.frames, r->host_frames, sizeof(Frame) * n, cudaMemcpyHostToDevice, s));
    return RL_OK;
}

// Event pair around one launch when profiling is on.
struct ProfScope {
    rl_reloc *r;
    int kid;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    ProfScope(rl_reloc *r_, int kid_, cudaStream_t s_) : r(r_), kid(kid_), s(s_) {
        if (r->prof.on) {
            a = take_event(r);
            cudaEventRecord(a, s);
        }
    }
    ~ProfScope() {
        if (!a) return;
        cudaEvent_t b = take_event(r);
        cudaEventRecord(b, s);
        r->prof.pending.push_back({kid, a, b});
    }
    static cudaEvent_t take_event(rl_reloc *r) {
        if (r->prof.pool.empty()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = r->prof.pool.back();
        r->prof.pool.pop_back();
        return e;
    }
};

static void prof_resolve(rl_reloc *r) {
    for (auto &p : r->prof.pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            r->prof.ms[p.kid] += ms;
            r->prof.launches[p.kid] += 1;
        }
        r->prof.pool.push_back(p.a);
        r->prof.pool.push_back(p.b);
    }
    r->prof.pending.clear();
}

#define PROF(kid) ProfScope prof_scope_##kid##__LINE__(r, kid, s)

rl_status run_relocalise(rl_reloc *r, const QueryState &q, int n, int level, cudaStream_t s) {
    rl_forest *f = r->forest;
    RParams p = r->rp;
    p.level = level;
    const int hw_max = r->max_w * r->max_h;
    const ModeView mv = mode_view(f);
    const int N = p.n_hyp, NC = p.n_cull;
    RL_CK(cudaMemsetAsync(q.n_chosen, 0xFF, sizeof(int32_t) * n, s));
    RL_CK(cudaMemsetAsync(q.n_rounds, 0, sizeof(int32_t) * n, s));
    RL_CK(cudaMemsetAsync(q.round_count, 0, sizeof(int32_t) * 16 * n, s));
    RL_CK(cudaMemsetAsync(q.dev_err, 0, sizeof(int32_t) * n, s));
    unsigned long long *work = r->prof.on ? r->prof.work : nullptr;
    // with pixel records (at most kRecTrees trees) every consumer reads the
    // leaves and |M(u)| from them, so neither the per-tree leaf map nor the
    // count map is written
    { PROF(K_LEAVES); RL_TRY(launch_leaves(f, q.frames, n, p.n_trees, hw_max, q.prec ? nullptr : q.leaves, r->max_w, r->max_h, s, p.k_top, q.prec ? nullptr : q.mcount, q.prec, r->tune.leaves_threads, r->nodes_s, r->host_frames[0].fx)); }
    if (q.pcm) { PROF(K_CMASK); RL_TRY(launch_colour_mask(q.frames, q.mcount, q.prec, hw_max, mv, p, q.pcm, q.pbits, n, hw_max, s, r->tune.mask_threads)); }
    { PROF(K_HYPGEN); RL_TRY(launch_hypgen(q.frames, q.leaves, q.mcount, q.prec, q.pcm, q.pbits, hw_max, mv, p, q.hyp_pose, q.hyp_iter, work, n, s, r->tune.hypgen_warps)); }
    { PROF(K_HYPPOSE); RL_TRY(launch_hyppose(q.frames, q.leaves, q.mcount, q.prec, hw_max, mv, p, q.hyp_pose, q.hyp_iter, n, s)); }
    { PROF(K_COMPACT); RL_TRY(launch_compact(q.hyp_iter, N, q.hyp_list, q.n_hyp, n, s)); }
    { PROF(K_SAMPLE); RL_TRY(launch_sample_batch(q.frames, q.mcount, q.prec, hw_max, p, 0, q.pix, q.xc, n, s));
      RL_TRY(launch_build_table(q, hw_max, mv, p, 0, n, s)); }

    const int maxm = p.maxm;
    int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(32, 40960 / (p.mpad * 36)));
    EnergyArgs ea{};
    ea.mcount = q.mcount;
    ea.prec = q.prec;
    ea.pix = q.pix;
    ea.xc = q.xc;
    ea.max_pix = p.max_pix;
    ea.leaves = q.leaves;
    ea.hw_max = hw_max;
    ea.mv = mv;
    ea.p = p;
    ea.chunk = chunk;
    ea.maxm = p.mpad;  // shared-memory row stride of the staged table
    ea.q_tab0 = q.tab0;
    ea.q_tab1 = q.tab1;
    ea.q_tab2 = q.tab2;
    ea.q_tab_cnt = q.tab_cnt;
    ea.part = q.energy_part;
    ea.part_h = std::max(N, NC);
    ea.n_chunks = r->n_chunks;
    // initial cull on I_0
    ea.pose = q.hyp_pose;
    ea.pose_stride = N;
    ea.idx = q.hyp_list;
    ea.idx_stride = N;
    ea.count = q.n_hyp;
    ea.n_pix = p.eta;
    ea.round_gate = 0;
    ea.work = work;
    { PROF(K_ENERGY); RL_TRY(launch_energy(ea, N, n, s, r->tune.energy_threads)); }
    SelectArgs sa{};
    sa.phase = 0;
    sa.round = 0;
    sa.part = q.energy_part;
    sa.part_h = ea.part_h;
    sa.n_chunks = r->n_chunks;
    sa.n_chunks_used = (p.eta + chunk - 1) / chunk;
    sa.count = q.n_hyp;
    sa.hyp_pose = q.hyp_pose;
    sa.hyp_list = q.hyp_list;
    sa.q = q;
    sa.p = p;
    sa.n_pix = p.eta;
    { PROF(K_SELECT); RL_TRY(launch_select(sa, n, s)); }
    // preemptive rounds
    for (int round = 0; round < p.max_rounds; ++round) {
        const int n_pix = p.eta * (round + 2);
        { PROF(K_SAMPLE); RL_TRY(launch_sample_batch(q.frames, q.mcount, q.prec, hw_max, p, round + 1, q.pix, q.xc, n, s));
          RL_TRY(launch_build_table(q, hw_max, mv, p, round + 1, n, s)); }
        const bool lm = p.pose_update && p.lm_max_iter > 0;
        if (lm) {
            LmArgs la{q, q.leaves, hw_max, mv, p, n_pix, work, maxm, maxm | 1, r->lm_wait_limit};
            PROF(K_LM);
            RL_TRY(launch_lm(la, n, s));
        }
        // the cluster LM kernel leaves each refined pose's energy on the
        // round's pixel set; otherwise the energies are computed here
        sa.energy_from_lm = lm && lm_uses_cluster(p);
        if (!sa.energy_from_lm) {
            ea.pose = q.cur_pose;
            ea.pose_stride = NC;
            ea.idx = nullptr;
            ea.idx_stride = 0;
            ea.count = q.n_cur;
            ea.n_pix = n_pix;
            ea.round_gate = 1;
            PROF(K_ENERGY);
            RL_TRY(launch_energy(ea, NC, n, s, r->tune.energy_threads));
        }
        sa.phase = 1;
        sa.round = round;
        sa.count = q.n_cur;
        sa.n_chunks_used = (n_pix + chunk - 1) / chunk;
        sa.n_pix = n_pix;
        { PROF(K_SELECT); RL_TRY(launch_select(sa, n, s)); }
    }
    const int ranked = p.rank && r->scene != nullptr;
    if (p.icp && r->scene) {
        // ICP before ranking: each chosen pose, or the output pose when unranked
        IcpArgs ia{};
        ia.frames = q.frames;
        ia.poses = ranked ? q.chosen_pose : q.cur_pose;
        ia.pose_stride = ranked ? 16 : NC;
        ia.counts = ranked ? q.n_chosen : nullptr;
        ia.gate = q.n_hyp;
        ia.cap = ranked ? p.k_out : 1;
        ia.ok = q.icp_ok;
        ia.frac = q.icp_frac;
        ia.out_stride = 16;
        for (int a = 0; a < 3; ++a) {
            ia.lo[a] = (float)r->scene->lo[a];
            ia.hi[a] = (float)r->scene->hi[a];
        }
        ia.ip = p.icp_p;
        ia.work = work;
        PROF(K_ICP);
        RL_TRY(launch_icp(ia, n, s));
    }
    if (ranked) {
        RaycastArgs ra{};
        ra.frames = q.frames;
        ra.poses = q.chosen_pose;
        ra.n_poses = q.n_chosen;
        ra.pose_cap = 16;
        for (int a = 0; a < 3; ++a) {
            ra.lo[a] = (float)r->scene->lo[a];
            ra.hi[a] = (float)r->scene->hi[a];
            ra.lo64[a] = r->scene->lo[a];
            ra.hi64[a] = r->scene->hi[a];
        }
        ra.part_sum = q.score_part;
        ra.part_cnt = q.score_cnt;
        ra.n_tiles = r->n_score_tiles;
        ra.work = work;
        PROF(K_RAYCAST);
        RL_TRY(launch_raycast(ra, n, hw_max, s));
    }
    { PROF(K_FINALIZE); RL_TRY(launch_finalize(q, p, r->n_score_tiles, ranked, n, s)); }
    return RL_OK;
}

// The launch sequence depends only on (n, level) and the relocaliser's
// fixed buffers, so it is captured once into a CUDA graph on a private
// stream and replayed on the caller's stream.  Profiling bypasses graphs
// (it needs events around individual launches).
static const size_t kMaxGraphs = 8;

static void graphs_free(rl_reloc *r) {
    for (auto &g : r->graphs) cudaGraphExecDestroy(g.exec);
    r->graphs.clear();
    if (r->capture_stream) cudaStreamDestroy(r->capture_stream);
    r->capture_stream = nullptr;
}

// Reader side of a forest's mode store: under the forest's lock, the launch
// waits for the last mode update (on whatever stream it was enqueued) and
// records, after its own work, the event that the next update of the store
// it read waits for.  A streaming forest (see rl_forest_set_streaming) has
// two stores; the others have one, which updates overwrite in place.
struct ModeReadScope {
    rl_forest *f;
    std::unique_lock<std::mutex> lk;
    int buf = 0;
    ModeReadScope(rl_forest *forest, cudaStream_t s, rl_status *st) : f(forest), lk(forest->mu) {
        buf = f->mode_buf;
        *st = RL_OK;
        if (f->ready && cudaStreamWaitEvent(s, f->ready, 0) != cudaSuccess)
            *st = fail(RL_ERR_CUDA, "waiting for the mode snapshot failed");
    }
    rl_status done(rl_reloc *r, cudaStream_t s) {
        if (!r->read_done[buf]) RL_CK(cudaEventCreateWithFlags(&r->read_done[buf], cudaEventDisableTiming));
        RL_CK(cudaEventRecord(r->read_done[buf], s));
        r->read_valid[buf] = true;
        return RL_OK;
    }
};

QueryState query_slice(const rl_reloc *r, int b0) {
    QueryState o = r->q;
    for (const auto &e : r->q_layout) {
        char *ptr;
        memcpy(&ptr, (char *)&o + e.first, sizeof(ptr));
        if (ptr) ptr += (size_t)b0 * e.second;
        memcpy((char *)&o + e.first, &ptr, sizeof(ptr));
    }
    return o;
}

// Frames per sub-batch below which a call is not split.
constexpr int kMinPart = 8;

// The call's frames as tune.streams sub-batches on as many streams (the
// caller's and private ones), forked from and joined back into s.  The
// frames are independent, so each sub-batch computes what the whole batch
// would for its frames; their kernels overlap wherever one sub-batch leaves
// SMs idle (the tails of the preemptive rounds, whose launches last as long
// as their slowest frame).  Inside a stream capture the fork and join bring
// the private streams into the same graph.
static rl_status run_relocalise_parts(rl_reloc *r, int n, int level, cudaStream_t s) {
    // nodes scaled for the call's focal length (frames of another one, in a
    // replayed graph, walk the unscaled nodes)
    RL_TRY(launch_scale_nodes(r->forest, r->rp.n_trees, r->nodes_s, r->host_frames[0].fx, s));
    const int parts = r->prof.on ? 1 : std::max(1, std::min(r->tune.streams, n / kMinPart));
    if (parts <= 1) return run_relocalise(r, r->q, n, level, s);
    for (int i = 0; i < parts - 1; ++i) {
        if (!r->side[i]) RL_CK(cudaStreamCreateWithFlags(&r->side[i], cudaStreamNonBlocking));
        if (!r->join_ev[i]) RL_CK(cudaEventCreateWithFlags(&r->join_ev[i], cudaEventDisableTiming));
    }
    if (!r->fork_ev) RL_CK(cudaEventCreateWithFlags(&r->fork_ev, cudaEventDisableTiming));
    RL_CK(cudaEventRecord(r->fork_ev, s));
    int b0 = 0;
    for (int i = 0; i < parts; ++i) {
        const int nb = n / parts + (i < n % parts ? 1 : 0);
        cudaStream_t si = i == 0 ? s : r->side[i - 1];
        if (i > 0) RL_CK(cudaStreamWaitEvent(si, r->fork_ev, 0));
        RL_TRY(run_relocalise(r, query_slice(r, b0), nb, level, si));
        if (i > 0) RL_CK(cudaEventRecord(r->join_ev[i - 1], si));
        b0 += nb;
    }
    for (int i = 0; i < parts - 1; ++i) RL_CK(cudaStreamWaitEvent(s, r->join_ev[i], 0));
    return RL_OK;
}

static rl_status launch_relocalise_snapshot(rl_reloc *r, int n, int level, int buf, cudaStream_t s);

rl_status launch_relocalise(rl_reloc *r, int n, int level, cudaStream_t s) {
    rl_status st;
    ModeReadScope scope(r->forest, s, &st);
    RL_TRY(st);
    RL_TRY(launch_relocalise_snapshot(r, n, level, scope.buf, s));
    return scope.done(r, s);
}

static rl_status launch_relocalise_snapshot(rl_reloc *r, int n, int level, int buf, cudaStream_t s) {
    ++r->calls;
    if (r->prof.on || !r->use_graphs) return run_relocalise_parts(r, n, level, s);
    for (auto &g : r->graphs)
        if (g.n == n && g.level == level && g.buf == buf) {
            g.last_use = r->calls;
            RL_CK(cudaGraphLaunch(g.exec, s));
            return RL_OK;
        }
    if (!r->capture_stream) RL_CK(cudaStreamCreateWithFlags(&r->capture_stream, cudaStreamNonBlocking));
    // inputs staged on `s` must be visible to the captured work: the graph
    // is launched on `s`, so only the capture itself runs on the private stream
    RL_CK(cudaStreamBeginCapture(r->capture_stream, cudaStreamCaptureModeThreadLocal));
    rl_status st = run_relocalise_parts(r, n, level, r->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(r->capture_stream, &g);
    if (st != RL_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    int kernels = 0;
    {
        size_t nn = 0;
        if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
            std::vector<cudaGraphNode_t> nodes(nn);
            if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
                for (size_t i = 0; i < nn; ++i) {
                    cudaGraphNodeType t;
                    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
                }
        }
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    if (r->graphs.size() >= kMaxGraphs) {  // evict the least recently used
        size_t lru = 0;
        for (size_t i = 1; i < r->graphs.size(); ++i)
            if (r->graphs[i].last_use < r->graphs[lru].last_use) lru = i;
        cudaGraphExecDestroy(r->graphs[lru].exec);
        r->graphs.erase(r->graphs.begin() + lru);
    }
    r->graphs.push_back({n, level, buf, exec, r->calls, kernels});
    RL_CK(cudaGraphLaunch(exec, s));
    return RL_OK;
}

// ICP outputs of one result: the mask, and each ICP run's inlier fraction
// (-1 where ICP did not run).
static void fill_icp(rl_result &o, const DevResult &d, const rl_reloc *r, const float *frac16) {
    o.icp_mask = d.icp_mask;
    for (int c = 0; c < RL_MAX_CHOSEN; ++c) o.chosen_icp_frac[c] = -1.f;
    if (!frac16 || !r->rp.icp || d.n_hypotheses <= 0) return;
    const int ranked = r->rp.rank && r->scene != nullptr;
    const int n_icp = ranked ? std::max(0, d.n_chosen) : 1;
    for (int c = 0; c < n_icp && c < RL_MAX_CHOSEN; ++c) o.chosen_icp_frac[c] = frac16[c];
}

static rl_status fetch_results(rl_reloc *r, int n, cudaStream_t s, rl_result *out, int level) {
    QueryState &q = r->q;
    std::vector<double> cp((size_t)n * 16 * 12);
    std::vector<float> ce((size_t)n * 16), cs((size_t)n * 16);
    std::vector<int32_t> cslot((size_t)n * 16);
    std::vector<float> icpf(r->rp.icp ? (size_t)n * 16 : 0);
    RL_CK(cudaMemcpyAsync(r->host_results, q.result_blob, sizeof(DevResult) * n, cudaMemcpyDeviceToHost, s));
    if (r->rp.icp) RL_CK(cudaMemcpyAsync(icpf.data(), q.icp_frac, icpf.size() * 4, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaMemcpyAsync(cp.data(), q.chosen_pose, cp.size() * 8, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaMemcpyAsync(ce.data(), q.chosen_energy, ce.size() * 4, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaMemcpyAsync(cs.data(), q.chosen_score, cs.size() * 4, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaMemcpyAsync(cslot.data(), q.chosen_slot, cslot.size() * 4, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaStreamSynchronize(s));
    if (!r->prof.pending.empty()) prof_resolve(r);
    for (int i = 0; i < n; ++i) {
        const DevResult &d = r->host_results[i];
        rl_result &o = out[i];
        memset(&o, 0, sizeof(o));
        for (int k = 0; k < 12; ++k) o.pose[k] = d.pose[k];
        o.pose[15] = 1.0;
        o.energy = d.energy;
        o.energy_per_pixel = d.energy_per_pixel;
        o.score = d.score;
        o.level = level;
        o.n_hypotheses = d.n_hypotheses;
        o.n_chosen = std::max(0, d.n_chosen);
        o.n_pixels = d.n_pixels;
        o.status = d.status;
        o.best = d.best;
        fill_icp(o, d, r, icpf.empty() ? nullptr : &icpf[(size_t)i * 16]);
        for (int c = 0; c < o.n_chosen && c < RL_MAX_CHOSEN; ++c) {
            for (int k = 0; k < 12; ++k) o.chosen_pose[c][k] = cp[((size_t)i * 16 + c) * 12 + k];
            o.chosen_pose[c][15] = 1.0;
            o.chosen_energy[c] = ce[(size_t)i * 16 + c];
            o.chosen_score[c] = cs[(size_t)i * 16 + c];
            o.chosen_slot[c] = cslot[(size_t)i * 16 + c];
        }
    }
    for (int i = 0; i < n; ++i)
        if (r->host_results[i].err)
            return fail(RL_ERR_TIMEOUT, "a bounded device-side wait gave up; the results of this call are invalid");
    return RL_OK;
}

// Copies n host frames into the staging area (or points at device frames)
// and fills the frame descriptors.
static rl_status stage_inputs(rl_reloc *r, int n, const float *depth, const uint8_t *rgb,
                              const rl_intrinsics *K, const uint64_t *seeds, rl_mem mem,
                              cudaStream_t s) {
    const size_t hw = (size_t)K->width * K->height;
    if (mem == RL_HOST) {
        RL_CK(cudaMemcpyAsync(r->stage_depth, depth, sizeof(float) * hw * n, cudaMemcpyHostToDevice, s));
        RL_CK(cudaMemcpyAsync(r->stage_rgb, rgb, hw * 3 * n, cudaMemcpyHostToDevice, s));
        return set_frames(r, n, r->stage_depth, r->stage_rgb, K, seeds, s);
    }
    if (mem != RL_DEVICE) return fail(RL_ERR_INVALID_ARG, "bad rl_mem");
    return set_frames(r, n, depth, rgb, K, seeds, s);
}

static rl_status check_call(rl_reloc *r, int n, const float *depth, const uint8_t *rgb,
                            const rl_intrinsics *K, const uint64_t *seeds) {
    if (!r || !depth || !rgb || !K || !seeds) return fail(RL_ERR_INVALID_ARG, "null argument");
    if (n < 1 || n > r->max_batch) return fail(RL_ERR_INVALID_ARG, "batch size outside 1..max_batch");
    if (K->width < 1 || K->height < 1 || K->width > r->max_w || K->height > r->max_h)
        return fail(RL_ERR_INVALID_ARG, "frame larger than the relocaliser's maximum size");
    if (!(K->fx > 0) || !(K->fy > 0)) return fail(RL_ERR_INVALID_ARG, "focal lengths must be > 0");
    return RL_OK;
}

rl_status reloc_enqueue_frames(rl_reloc *r, int n, const Frame *frames, cudaStream_t s) {
    if (n < 1 || n > r->max_batch) return fail(RL_ERR_INVALID_ARG, "batch size outside 1..max_batch");
    for (int i = 0; i < n; ++i) {
        if (frames[i].W > r->max_w || frames[i].H > r->max_h)
            return fail(RL_ERR_INVALID_ARG, "frame larger than the relocaliser's maximum size");
        r->host_frames[i] = frames[i];
    }
    RL_CK(cudaMemcpyAsync(r->q.frames, r->host_frames, sizeof(Frame) * n, cudaMemcpyHostToDevice, s));
    RL_TRY(launch_relocalise(r, n, 0, s));
    r->last_batch = n;
    return RL_OK;
}

rl_status reloc_fetch_results(rl_reloc *r, int n, cudaStream_t s, rl_result *out) {
    return fetch_results(r, n, s, out, 0);
}

}  // namespace rl

using namespace rl;

extern "C" rl_status rl_reloc_create(rl_forest *f, rl_scene *scene, const rl_ransac_params *p,
                                     int32_t max_w, int32_t max_h, int32_t max_batch,
                                     rl_reloc **out) {
    if (!f || !out) return fail(RL_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    RL_TRY(check_ransac(p, f));
    if (max_w < 1 || max_h < 1 || max_w > 8192 || max_h > 8192 || (int64_t)max_w * max_h > (1 << 26))
        return fail(RL_ERR_INVALID_ARG, "bad maximum frame size");
    if (max_batch < 1 || max_batch > 65535) return fail(RL_ERR_INVALID_ARG, "max_batch must be 1..65535");
    if (p->rank && !scene) return fail(RL_ERR_INVALID_ARG, "ranking needs a scene model");
    if (p->icp && !scene) return fail(RL_ERR_INVALID_ARG, "ICP needs a scene model");
    if (p->icp) RL_TRY(check_icp(&p->icp_p));
    RL_CK(cudaSetDevice(f->ctx->device));
    RL_TRY(prepare_kernels());
    rl_reloc *r = new rl_reloc();
    r->forest = f;
    r->scene = scene;
    r->p = *p;
    r->max_w = max_w;
    r->max_h = max_h;
    r->max_batch = max_batch;
    RParams &rp = r->rp;
    rp.n_hyp = p->n_hyp; rp.max_iter = p->max_iter; rp.n_cull = p->n_cull; rp.eta = p->eta;
    rp.k_out = p->k_out; rp.pose_update = p->pose_update; rp.use_cov = p->use_cov;
    rp.colour_thresh = p->colour_thresh; rp.min_sq_dist = p->min_sq_dist;
    rp.max_trans_err = p->max_trans_err; rp.k_top = p->k_top; rp.n_trees = p->n_trees_used;
    rp.lm_max_iter = p->lm_max_iter; rp.batch_attempts = p->batch_attempts;
    rp.lm_lambda0 = p->lm_lambda0; rp.lm_inlier_thresh = p->lm_inlier_thresh; rp.lm_stop = p->lm_stop;
    rp.rank = p->rank; rp.halve_to_one = p->halve_to_one; rp.level = 0;
    rp.icp = p->icp;
    rp.redraw = p->redraw;
    if (p->icp) rp.icp_p = icp_device_params(p->icp_p);
    rp.max_rounds = rounds_for(p->n_cull, p->k_out, p->halve_to_one);
    // rows of whole 16-pixel tiles: the LM kernel stages tiles with bulk copies
    rp.max_pix = (p->eta * (rp.max_rounds + 1) + 15) / 16 * 16;
    const int maxm = p->n_trees_used * std::min(p->k_top, f->p.m_max);
    rp.maxm = maxm;
    rp.mpad = maxm | 1;
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(32, 40960 / (rp.mpad * 36)));
    r->n_chunks = (rp.max_pix + chunk - 1) / chunk;
    const size_t hw = (size_t)max_w * max_h;
    r->n_score_tiles = (int)((hw + RC_TILE - 1) / RC_TILE);
    const uint64_t B = max_batch, N = p->n_hyp, NC = p->n_cull, MP = rp.max_pix;
    QueryState &q = r->q;
    rl_status s = RL_OK;
#define A(field, count)                                                                            \
    if (s == RL_OK) {                                                                              \
        s = ralloc(r, (uint64_t)(count), &q.field);                                                \
        r->q_layout.push_back({offsetof(QueryState, field), (size_t)((count) / B) * sizeof(*q.field)}); \
    }
    A(leaves, B * p->n_trees_used * hw);
    A(mcount, B * hw);
    if (p->n_trees_used <= kRecTrees) A(prec, B * hw);
    if (p->n_trees_used <= kRecTrees && maxm <= kMaskModes) A(pcm, B * hw);
    if (q.pcm) A(pbits, B * (hw / 32 + 1));
    A(hyp_pose, B * N * 12);
    A(hyp_iter, B * N);
    A(hyp_list, B * N);
    A(n_hyp, B);
    A(pix, B * MP);
    A(xc, B * MP);
    A(tab0, B * MP * (uint64_t)rp.mpad);
    A(tab1, B * MP * (uint64_t)rp.mpad);
    A(tab2, B * MP * (uint64_t)rp.mpad);
    A(tab_cnt, B * MP);
    A(lm_anc, B * NC * MP);
    A(n_pix, B);
    A(cur_pose, B * NC * 12);
    A(cur_slot, B * NC);
    A(cur_energy, B * NC);
    A(n_cur, B);
    A(cull_slot, B * NC);
    A(cull_energy, B * NC);
    A(energy_part, B * std::max(N, NC) * (uint64_t)r->n_chunks);
    A(corr, B * NC * MP);
    A(chosen_pose, B * 16 * 12);
    A(chosen_energy, B * 16);
    A(chosen_slot, B * 16);
    A(chosen_npix, B);
    A(n_chosen, B);
    A(score_part, B * 16 * (uint64_t)r->n_score_tiles);
    A(score_cnt, B * 16 * 2 * (uint64_t)r->n_score_tiles);
    A(chosen_score, B * 16);
    A(icp_ok, B * 16);
    A(icp_frac, B * 16);
    A(round_count, B * 16);
    A(round_slot, B * 16 * NC);
    A(round_energy, B * 16 * NC);
    A(round_pose, B * 16 * NC * 12);
    A(n_rounds, B);
    A(frames, B);
    A(result_blob, B * sizeof(DevResult));
    A(dev_err, B);
#undef A
    if (s == RL_OK) s = ralloc(r, (uint64_t)p->n_trees_used * f->n_branch, &r->nodes_s);
    if (s == RL_OK) s = ralloc(r, B * hw, &r->stage_depth);
    if (s == RL_OK) s = ralloc(r, B * hw * 3, &r->stage_rgb);
    if (s == RL_OK && cudaMallocHost(&r->host_frames, sizeof(Frame) * B) != cudaSuccess)
        s = fail(RL_ERR_CUDA, "pinned host allocation failed");
    if (s == RL_OK && cudaMallocHost(&r->host_results, sizeof(DevResult) * B) != cudaSuccess)
        s = fail(RL_ERR_CUDA, "pinned host allocation failed");
    if (s == RL_OK) {
        const size_t sm_sel = (size_t)N * 8 + NC * (12 * 8 + 8) + 64;
        const size_t sm_en = energy_smem(chunk, rp.mpad);
        if (sm_sel > 200 * 1024 || sm_en > 200 * 1024) s = fail(RL_ERR_INVALID_ARG, "configuration needs too much shared memory");
    }
    if (s != RL_OK) {
        reloc_release(r);
        delete r;
        return s;
    }
    f->refcount++;
    {
        std::lock_guard<std::mutex> g(f->mu);
        f->readers.push_back(r);
    }
    *out = r;
    return RL_OK;
}

extern "C" rl_status rl_reloc_destroy(rl_reloc *r) {
    if (!r) return fail(RL_ERR_INVALID_ARG, "null relocaliser");
    if (r->refcount > 0) return fail(RL_ERR_BUSY, "relocaliser still used by a cascade");
    cudaSetDevice(r->forest->ctx->device);
    cudaDeviceSynchronize();
    r->forest->refcount--;
    {
        rl_forest *f = r->forest;
        std::lock_guard<std::mutex> g(f->mu);
        for (size_t i = 0; i < f->readers.size(); ++i)
            if (f->readers[i] == r) {
                f->readers.erase(f->readers.begin() + i);
                break;
            }
    }
    for (cudaEvent_t &e : r->read_done)
        if (e) cudaEventDestroy(e);
    reloc_release(r);
    delete r;
    return RL_OK;
}

extern "C" rl_status rl_relocalise_batch(rl_reloc *r, int32_t n, const float *depth, const uint8_t *rgb,
                                         const rl_intrinsics *K, const uint64_t *seeds, rl_mem mem,
                                         void *stream, rl_result *out) {
    RL_TRY(check_call(r, n, depth, rgb, K, seeds));
    if (!out) return fail(RL_ERR_INVALID_ARG, "null output");
    RL_CK(cudaSetDevice(r->forest->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RL_TRY(stage_inputs(r, n, depth, rgb, K, seeds, mem, s));
    RL_TRY(launch_relocalise(r, n, 0, s));
    r->last_batch = n;
    return fetch_results(r, n, s, out, 0);
}

extern "C" rl_status rl_relocalise(rl_reloc *r, const float *depth, const uint8_t *rgb,
                                   const rl_intrinsics *K, uint64_t seed, rl_mem mem, void *stream,
                                   rl_result *out) {
    return rl_relocalise_batch(r, 1, depth, rgb, K, &seed, mem, stream, out);
}

extern "C" rl_status rl_relocalise_batch_async(rl_reloc *r, int32_t n, const float *depth,
                                               const uint8_t *rgb, const rl_intrinsics *K,
                                               const uint64_t *seeds, void *stream) {
    RL_TRY(check_call(r, n, depth, rgb, K, seeds));
    RL_CK(cudaSetDevice(r->forest->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    RL_TRY(stage_inputs(r, n, depth, rgb, K, seeds, RL_DEVICE, s));
    RL_TRY(launch_relocalise(r, n, 0, s));
    r->last_batch = n;
    return RL_OK;
}

extern "C" rl_status rl_reloc_fetch(rl_reloc *r, int32_t n, void *stream, rl_result *out) {
    if (!r || !out) return fail(RL_ERR_INVALID_ARG, "null argument");
    if (n < 1 || n > r->last_batch) return fail(RL_ERR_INVALID_ARG, "n exceeds the last batch");
    RL_CK(cudaSetDevice(r->forest->ctx->device));
    return fetch_results(r, n, (cudaStream_t)stream, out, 0);
}

extern "C" rl_status rl_reloc_debug(rl_reloc *r, int32_t qi, double *hyp_pose, int32_t *hyp_iter,
                                    int32_t *cull_slot, float *cull_energy, int32_t *round_count,
                                    int32_t *round_slot, float *round_energy, double *round_pose,
                                    int32_t *batch_pix, int32_t *n_rounds) {
    if (!r) return fail(RL_ERR_INVALID_ARG, "null relocaliser");
    if (qi < 0 || qi >= r->last_batch) return fail(RL_ERR_INVALID_ARG, "query index outside the last batch");
    RL_CK(cudaSetDevice(r->forest->ctx->device));
    RL_CK(cudaDeviceSynchronize());
    const QueryState &q = r->q;
    const size_t N = r->rp.n_hyp, NC = r->rp.n_cull, MP = r->rp.max_pix;
    if (hyp_pose) RL_CK(cudaMemcpy(hyp_pose, q.hyp_pose + qi * N * 12, N * 12 * 8, cudaMemcpyDeviceToHost));
    if (hyp_iter) RL_CK(cudaMemcpy(hyp_iter, q.hyp_iter + qi * N, N * 4, cudaMemcpyDeviceToHost));
    if (cull_slot) RL_CK(cudaMemcpy(cull_slot, q.cull_slot + qi * NC, NC * 4, cudaMemcpyDeviceToHost));
    if (cull_energy) RL_CK(cudaMemcpy(cull_energy, q.cull_energy + qi * NC, NC * 4, cudaMemcpyDeviceToHost));
    if (round_count) RL_CK(cudaMemcpy(round_count, q.round_count + qi * 16, 16 * 4, cudaMemcpyDeviceToHost));
    if (round_slot) RL_CK(cudaMemcpy(round_slot, q.round_slot + qi * 16 * NC, 16 * NC * 4, cudaMemcpyDeviceToHost));
    if (round_energy) RL_CK(cudaMemcpy(round_energy, q.round_energy + qi * 16 * NC, 16 * NC * 4, cudaMemcpyDeviceToHost));
    if (round_pose) RL_CK(cudaMemcpy(round_pose, q.round_pose + qi * 16 * NC * 12, 16 * NC * 12 * 8, cudaMemcpyDeviceToHost));
    if (batch_pix) {
        const size_t nb = std::min<size_t>(16, (size_t)r->rp.max_rounds + 1);
        for (size_t i = 0; i < 16 * (size_t)r->rp.eta; ++i) batch_pix[i] = -1;
        RL_CK(cudaMemcpy(batch_pix, q.pix + qi * MP, nb * r->rp.eta * 4, cudaMemcpyDeviceToHost));
    }
    if (n_rounds) RL_CK(cudaMemcpy(n_rounds, q.n_rounds + qi, 4, cudaMemcpyDeviceToHost));
    return RL_OK;
}

// ---------------------------------------------------------------------------
// Cascade (Sec. 3.2.5).  All levels of all frames are enqueued together
// (one CUDA graph per batch size): level l runs on every frame; its
// decision kernel copies each still-open frame's result to the cascade
// output and, when the frame's score is within tau_l (or l is the last
// level), closes it by turning its descriptors of every later level into
// an empty 0x0 frame, on which later levels do no work.  No host round trip
// happens between levels.
// ---------------------------------------------------------------------------
namespace rl {

struct LaterFrames {
    Frame *f[8];
    int n;
};

__global__ void k_subsample_all(const Frame *__restrict__ full, const int32_t *__restrict__ done,
                                int s_factor, float *dd, uint8_t *dc, int max_hw) {
    const int b = blockIdx.y;
    if (done[b]) return;
    const Frame f = full[b];
    const int W2 = (f.W + s_factor - 1) / s_factor, H2 = (f.H + s_factor - 1) / s_factor;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= W2 * H2) return;
    const int sp = ((p / W2) * s_factor) * f.W + (p % W2) * s_factor;
    dd[(size_t)b * max_hw + p] = f.depth[sp];
    uint8_t *o = dc + ((size_t)b * max_hw + p) * 3;
    o[0] = f.rgb[sp * 3 + 0];
    o[1] = f.rgb[sp * 3 + 1];
    o[2] = f.rgb[sp * 3 + 2];
}

__global__ void k_cascade_decide(QueryState lq, CascadeOut co, LaterFrames later, float tau, int level,
                                 int last, int n) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n || co.done[b]) return;
    const DevResult r = ((const DevResult *)lq.result_blob)[b];
    const int32_t earlier_err = level > 0 ? co.res[b].err : 0;  // sticky over the levels
    co.res[b] = r;
    co.res[b].err |= earlier_err;
    co.level[b] = level;
    const int nc = r.n_chosen > 0 ? r.n_chosen : 0;
    for (int c = 0; c < nc; ++c) {
        for (int k = 0; k < 12; ++k)
            co.chosen_pose[((size_t)b * 16 + c) * 12 + k] = lq.chosen_pose[((size_t)b * 16 + c) * 12 + k];
        co.chosen_energy[(size_t)b * 16 + c] = lq.chosen_energy[(size_t)b * 16 + c];
        co.chosen_score[(size_t)b * 16 + c] = lq.chosen_score[(size_t)b * 16 + c];
        co.chosen_slot[(size_t)b * 16 + c] = lq.chosen_slot[(size_t)b * 16 + c];
    }
    for (int c = 0; c < 16; ++c) co.icp_frac[(size_t)b * 16 + c] = lq.icp_frac[(size_t)b * 16 + c];
    // fall back iff the output pose's score exceeds tau (Sec. 3.2.5)
    const bool accept = last || (r.status == RL_POSE_FOUND && r.score <= tau);
    if (!accept) return;
    co.done[b] = 1;
    for (int k = 0; k < later.n; ++k) {
        later.f[k][b].W = 0;
        later.f[k][b].H = 0;
    }
}

// The cascade outputs of frames b0, b0 + 1, ...
static CascadeOut cascade_out_slice(const CascadeOut &o, int b0) {
    const size_t b = (size_t)b0;
    CascadeOut s = o;
    s.res += b;
    s.chosen_pose += b * 16 * 12;
    s.chosen_energy += b * 16;
    s.chosen_score += b * 16;
    s.icp_frac += b * 16;
    s.chosen_slot += b * 16;
    s.level += b;
    s.done += b;
    return s;
}

// All levels for the nb frames b0, b0 + 1, ... of the call.
static rl_status cascade_enqueue_part(rl_cascade *c, int b0, int nb, cudaStream_t s) {
    const int L = (int)c->levels.size();
    const CascadeOut out = cascade_out_slice(c->out, b0);
    RL_CK(cudaMemsetAsync(out.done, 0, sizeof(int32_t) * nb, s));
    for (int l = 0; l < L; ++l) {
        rl_reloc *r = c->levels[l];
        const QueryState q = query_slice(r, b0);
        const int sf = c->subsample[l];
        if (sf > 1) {
            const int hw = r->max_w * r->max_h;
            dim3 grid((hw + 255) / 256, nb);
            k_subsample_all<<<grid, 256, 0, s>>>(c->full_dev + b0, out.done, sf, r->stage_depth + (size_t)b0 * hw,
                                                 r->stage_rgb + (size_t)b0 * hw * 3, hw);
            RL_LAUNCH_CK();
        }
        RL_TRY(run_relocalise(r, q, nb, l, s));
        LaterFrames later{};
        for (int k = l + 1; k < L && later.n < 8; ++k) later.f[later.n++] = c->levels[k]->q.frames + b0;
        const float tau = l < L - 1 ? (float)c->thresholds[l] : INFINITY;
        k_cascade_decide<<<(nb + 127) / 128, 128, 0, s>>>(q, out, later, tau, l, l == L - 1, nb);
        RL_LAUNCH_CK();
    }
    return RL_OK;
}

// A cascade call as sub-batches on concurrent streams, as for one level
// (run_relocalise_parts): each sub-batch runs every level for its frames.
static rl_status cascade_enqueue(rl_cascade *c, int n, cudaStream_t s) {
    bool prof = false;
    for (rl_reloc *r : c->levels) prof = prof || r->prof.on;
    for (rl_reloc *r : c->levels)  // each level's nodes scaled for its focal length
        RL_TRY(launch_scale_nodes(r->forest, r->rp.n_trees, r->nodes_s, r->host_frames[0].fx, s));
    const int parts = prof ? 1 : std::max(1, std::min(c->levels[0]->tune.streams, n / kMinPart));
    if (parts <= 1) return cascade_enqueue_part(c, 0, n, s);
    for (int i = 0; i < parts - 1; ++i) {
        if (!c->side[i]) RL_CK(cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking));
        if (!c->join_ev[i]) RL_CK(cudaEventCreateWithFlags(&c->join_ev[i], cudaEventDisableTiming));
    }
    if (!c->fork_ev) RL_CK(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
    RL_CK(cudaEventRecord(c->fork_ev, s));
    int b0 = 0;
    for (int i = 0; i < parts; ++i) {
        const int nb = n / parts + (i < n % parts ? 1 : 0);
        cudaStream_t si = i == 0 ? s : c->side[i - 1];
        if (i > 0) RL_CK(cudaStreamWaitEvent(si, c->fork_ev, 0));
        RL_TRY(cascade_enqueue_part(c, b0, nb, si));
        if (i > 0) RL_CK(cudaEventRecord(c->join_ev[i - 1], si));
        b0 += nb;
    }
    for (int i = 0; i < parts - 1; ++i) RL_CK(cudaStreamWaitEvent(s, c->join_ev[i], 0));
    return RL_OK;
}

static rl_status cascade_launch_snapshot(rl_cascade *c, int n, int buf, cudaStream_t s);

// The levels' forests are read under the reader protocol of launch_relocalise
// (each distinct forest locked, in address order); the graph cache is keyed
// by the forests' front stores.
static rl_status cascade_launch(rl_cascade *c, int n, cudaStream_t s) {
    std::vector<rl_forest *> fs;
    for (rl_reloc *r : c->levels)
        if (std::find(fs.begin(), fs.end(), r->forest) == fs.end()) fs.push_back(r->forest);
    std::sort(fs.begin(), fs.end());
    std::vector<std::unique_ptr<ModeReadScope>> scopes;
    int buf = 0;
    for (size_t k = 0; k < fs.size(); ++k) {
        rl_status st;
        scopes.emplace_back(new ModeReadScope(fs[k], s, &st));
        RL_TRY(st);
        buf |= scopes.back()->buf << k;
    }
    RL_TRY(cascade_launch_snapshot(c, n, buf, s));
    for (rl_reloc *r : c->levels)
        for (auto &sc : scopes)
            if (sc->f == r->forest) RL_TRY(sc->done(r, s));
    return RL_OK;
}

// Changes with the tuning of any level (a captured graph holds the levels'
// launch shapes and sub-batches).
static uint64_t cascade_tune_gen(const rl_cascade *c) {
    uint64_t g = 0;
    for (const rl_reloc *r : c->levels) g += r->tune_gen;
    return g;
}

static rl_status cascade_launch_snapshot(rl_cascade *c, int n, int buf, cudaStream_t s) {
    bool prof = false;
    for (rl_reloc *r : c->levels) prof = prof || r->prof.on;
    if (prof || !c->use_graphs) return cascade_enqueue(c, n, s);
    const uint64_t gen = cascade_tune_gen(c);
    for (size_t i = 0; i < c->graphs.size();)  // captured under another tuning of some level
        if (c->graphs[i].tune_gen != gen) {
            cudaGraphExecDestroy(c->graphs[i].exec);
            c->graphs.erase(c->graphs.begin() + i);
        } else {
            ++i;
        }
    for (auto &g : c->graphs)
        if (g.n == n && g.buf == buf) {
            RL_CK(cudaGraphLaunch(g.exec, s));
            return RL_OK;
        }
    if (!c->capture_stream) RL_CK(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    RL_CK(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
    rl_status st = cascade_enqueue(c, n, c->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->capture_stream, &g);
    if (st != RL_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    if (c->graphs.size() >= 8) {
        cudaGraphExecDestroy(c->graphs.front().exec);
        c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back({n, buf, gen, exec});
    RL_CK(cudaGraphLaunch(exec, s));
    return RL_OK;
}

static rl_status cascade_fetch(rl_cascade *c, int n, cudaStream_t s, rl_result *out) {
    std::vector<DevResult> res(n);
    std::vector<double> cp((size_t)n * 16 * 12);
    std::vector<float> ce((size_t)n * 16), cs((size_t)n * 16);
    std::vector<int32_t> cslot((size_t)n * 16), lvl(n);
    std::vector<float> icpf((size_t)n * 16);
    RL_CK(cudaMemcpyAsync(res.data(), c->out.res, sizeof(DevResult) * n, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaMemcpyAsync(icpf.data(), c->out.icp_frac, icpf.size() * 4, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaMemcpyAsync(cp.data(), c->out.chosen_pose, cp.size() * 8, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaMemcpyAsync(ce.data(), c->out.chosen_energy, ce.size() * 4, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaMemcpyAsync(cs.data(), c->out.chosen_score, cs.size() * 4, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaMemcpyAsync(cslot.data(), c->out.chosen_slot, cslot.size() * 4, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaMemcpyAsync(lvl.data(), c->out.level, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    RL_CK(cudaStreamSynchronize(s));
    for (rl_reloc *r : c->levels)
        if (!r->prof.pending.empty()) prof_resolve(r);
    for (int i = 0; i < n; ++i) {
        const DevResult &d = res[i];
        rl_result &o = out[i];
        memset(&o, 0, sizeof(o));
        for (int k = 0; k < 12; ++k) o.pose[k] = d.pose[k];
        o.pose[15] = 1.0;
        o.energy = d.energy;
        o.energy_per_pixel = d.energy_per_pixel;
        o.score = d.score;
        o.level = lvl[i];
        o.n_hypotheses = d.n_hypotheses;
        o.n_chosen = std::max(0, d.n_chosen);
        o.n_pixels = d.n_pixels;
        o.status = d.status;
        o.best = d.best;
        fill_icp(o, d, c->levels[lvl[i]], &icpf[(size_t)i * 16]);
        for (int k = 0; k < o.n_chosen && k < RL_MAX_CHOSEN; ++k) {
            for (int j = 0; j < 12; ++j) o.chosen_pose[k][j] = cp[((size_t)i * 16 + k) * 12 + j];
            o.chosen_pose[k][15] = 1.0;
            o.chosen_energy[k] = ce[(size_t)i * 16 + k];
            o.chosen_score[k] = cs[(size_t)i * 16 + k];
            o.chosen_slot[k] = cslot[(size_t)i * 16 + k];
        }
    }
    for (int i = 0; i < n; ++i)
        if (res[i].err)
            return fail(RL_ERR_TIMEOUT, "a bounded device-side wait gave up; the results of this call are invalid");
    return RL_OK;
}

static void cascade_release(rl_cascade *c) {
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    c->capture_stream = nullptr;
    for (int i = 0; i < 7; ++i) {
        if (c->side[i]) cudaStreamDestroy(c->side[i]);
        if (c->join_ev[i]) cudaEventDestroy(c->join_ev[i]);
        c->side[i] = nullptr;
        c->join_ev[i] = nullptr;
    }
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    c->fork_ev = nullptr;
    for (void *p : c->allocs) arena_free(c->ctx, p);
    c->allocs.clear();
}

}  // namespace rl

extern "C" rl_status rl_cascade_create(rl_reloc *const *levels, const double *thresholds,
                                       const int32_t *subsample, int32_t n_levels,
                                       rl_cascade **out) {
    if (!levels || !out || n_levels < 1 || n_levels > 8) return fail(RL_ERR_INVALID_ARG, "bad cascade");
    if (n_levels > 1 && !thresholds) return fail(RL_ERR_INVALID_ARG, "thresholds needed");
    *out = nullptr;
    for (int l = 0; l < n_levels; ++l) {
        if (!levels[l]) return fail(RL_ERR_INVALID_ARG, "null level");
        if (levels[l]->forest != levels[0]->forest)
            return fail(RL_ERR_INVALID_ARG, "cascade levels must share one forest");
        if (subsample && subsample[l] < 1) return fail(RL_ERR_INVALID_ARG, "subsample must be >= 1");
        for (int k = 0; k < l; ++k)
            if (levels[k] == levels[l]) return fail(RL_ERR_INVALID_ARG, "each level needs its own relocaliser");
    }
    if (subsample && subsample[n_levels - 1] != 1)
        return fail(RL_ERR_INVALID_ARG, "the last level works at full resolution (subsample 1)");
    rl_cascade *c = new rl_cascade();
    c->ctx = levels[0]->forest->ctx;
    c->max_batch = levels[0]->max_batch;
    for (int l = 0; l < n_levels; ++l) {
        c->levels.push_back(levels[l]);
        c->subsample.push_back(subsample ? subsample[l] : 1);
        if (l < n_levels - 1) c->thresholds.push_back(thresholds[l]);
        c->max_batch = std::min(c->max_batch, levels[l]->max_batch);
    }
    const uint64_t B = c->max_batch;
    rl_status s = RL_OK;
    auto A = [&](auto **ptr, uint64_t cnt) {
        if (s == RL_OK) s = alloc_n(c->ctx, cnt, ptr);
        if (s == RL_OK) c->allocs.push_back(*ptr);
    };
    A(&c->out.res, B);
    A(&c->out.chosen_pose, B * 16 * 12);
    A(&c->out.chosen_energy, B * 16);
    A(&c->out.chosen_score, B * 16);
    A(&c->out.icp_frac, B * 16);
    A(&c->out.chosen_slot, B * 16);
    A(&c->out.level, B);
    A(&c->out.done, B);
    A(&c->full_dev, B);
    if (s != RL_OK) {
        cascade_release(c);
        delete c;
        return s;
    }
    for (int l = 0; l < n_levels; ++l) levels[l]->refcount++;
    *out = c;
    return RL_OK;
}

extern "C" rl_status rl_cascade_destroy(rl_cascade *c) {
    if (!c) return fail(RL_ERR_INVALID_ARG, "null cascade");
    cudaSetDevice(c->ctx->device);
    cudaDeviceSynchronize();
    for (rl_reloc *r : c->levels) r->refcount--;
    cascade_release(c);
    delete c;
    return RL_OK;
}

namespace rl {

// Enqueues a cascade call on n full-resolution frames whose descriptors are
// in the last level's host_frames (images already on the device): each
// earlier level gets its subsampled copy of every frame (its own size and
// intrinsics / s), then all levels run as one graph.
rl_status cascade_enqueue_frames(rl_cascade *c, int n, cudaStream_t s) {
    rl_reloc *top = c->levels.back();
    const Frame *full = top->host_frames;
    RL_CK(cudaMemcpyAsync(top->q.frames, full, sizeof(Frame) * n, cudaMemcpyHostToDevice, s));
    RL_CK(cudaMemcpyAsync(c->full_dev, full, sizeof(Frame) * n, cudaMemcpyHostToDevice, s));
    const int L = (int)c->levels.size();
    for (int l = 0; l < L - 1; ++l) {
        rl_reloc *r = c->levels[l];
        const int sf = c->subsample[l];
        const int hw = r->max_w * r->max_h;
        for (int i = 0; i < n; ++i) {
            Frame &f = r->host_frames[i];
            f = full[i];
            if (sf > 1) {
                const int W = (full[i].W + sf - 1) / sf, H = (full[i].H + sf - 1) / sf;
                if (W > r->max_w || H > r->max_h)
                    return fail(RL_ERR_INVALID_ARG, "level input larger than the level's maximum size");
                f.depth = r->stage_depth + (size_t)hw * i;
                f.rgb = r->stage_rgb + (size_t)hw * 3 * i;
                f.fx = (float)((double)full[i].fx / sf);
                f.fy = (float)((double)full[i].fy / sf);
                f.cx = (float)((double)full[i].cx / sf);
                f.cy = (float)((double)full[i].cy / sf);
                f.W = W;
                f.H = H;
            }
        }
        RL_CK(cudaMemcpyAsync(r->q.frames, r->host_frames, sizeof(Frame) * n, cudaMemcpyHostToDevice, s));
    }
    RL_TRY(cascade_launch(c, n, s));
    for (rl_reloc *r : c->levels) r->last_batch = n;
    return RL_OK;
}

rl_status cascade_fetch_results(rl_cascade *c, int n, cudaStream_t s, rl_result *out) {
    return cascade_fetch(c, n, s, out);
}

}  // namespace rl

using namespace rl;

extern "C" rl_status rl_cascade_relocalise_batch(rl_cascade *c, int32_t n, const float *depth,
                                                 const uint8_t *rgb, const rl_intrinsics *K,
                                                 const uint64_t *seeds, rl_mem mem, void *stream,
                                                 rl_result *out) {
    if (!c || !out) return fail(RL_ERR_INVALID_ARG, "null argument");
    rl_reloc *top = c->levels.back();
    RL_TRY(check_call(top, n, depth, rgb, K, seeds));
    if (n > c->max_batch) return fail(RL_ERR_INVALID_ARG, "batch larger than a level's max_batch");
    RL_CK(cudaSetDevice(c->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    // full-resolution frames: staged into (or pointing at) the last level's inputs
    RL_TRY(stage_inputs(top, n, depth, rgb, K, seeds, mem, s));
    RL_TRY(cascade_enqueue_frames(c, n, s));
    return cascade_fetch(c, n, s, out);
}

extern "C" rl_status rl_cascade_relocalise(rl_cascade *c, const float *depth, const uint8_t *rgb,
                                           const rl_intrinsics *K, uint64_t seed, rl_mem mem,
                                           void *stream, rl_result *out) {
    return rl_cascade_relocalise_batch(c, 1, depth, rgb, K, &seed, mem, stream, out);
}

// ---------------------------------------------------------------------------
// Kernel profiler (tracing): CUDA events per launch on the caller's stream.
// ---------------------------------------------------------------------------
namespace rl {
static void prof_free(rl_reloc *r) {
    prof_resolve(r);
    for (cudaEvent_t e : r->prof.pool) cudaEventDestroy(e);
    r->prof.pool.clear();
}
}  // namespace rl

static const char *kKernelNames[K_COUNT] = {"leaves",  "hypgen", "compact", "sample_batch", "energy",
                                             "select", "lm",     "raycast_score", "finalize", "hyppose",
                                             "colour_mask", "icp"};
static_assert(K_COUNT == RL_N_KERNELS, "kernel ids and the public count differ");
static_assert(W_COUNT == RL_N_WORK, "work counters and the public count differ");

extern "C" const char *rl_kernel_name(int32_t kid) {
    return (kid >= 0 && kid < K_COUNT) ? kKernelNames[kid] : "";
}

extern "C" rl_status rl_reloc_set_graphs(rl_reloc *r, int32_t enable) {
    if (!r) return fail(RL_ERR_INVALID_ARG, "null relocaliser");
    r->use_graphs = enable != 0;
    return RL_OK;
}

extern "C" rl_status rl_reloc_graph_kernels(rl_reloc *r, int32_t n, int32_t *out) {
    if (!r || !out) return fail(RL_ERR_INVALID_ARG, "null argument");
    *out = -1;
    for (const auto &g : r->graphs)
        if (g.n == n && g.level == 0) *out = g.kernels;
    return RL_OK;
}

extern "C" rl_status rl_reloc_set_wait_limit(rl_reloc *r, int64_t probes) {
    if (!r) return fail(RL_ERR_INVALID_ARG, "null relocaliser");
    if (probes > (int64_t)UINT32_MAX) return fail(RL_ERR_INVALID_ARG, "probe limit beyond 2^32 - 1");
    RL_CK(cudaSetDevice(r->forest->ctx->device));
    RL_CK(cudaDeviceSynchronize());
    r->lm_wait_limit = probes < 0 ? kLmWaitLimit : (uint32_t)probes;
    graphs_free(r);  // captured launches hold the old limit
    return RL_OK;
}

extern "C" rl_status rl_reloc_profile(rl_reloc *r, int32_t enable) {
    if (!r) return fail(RL_ERR_INVALID_ARG, "null relocaliser");
    RL_CK(cudaSetDevice(r->forest->ctx->device));
    RL_CK(cudaDeviceSynchronize());
    prof_resolve(r);
    for (int k = 0; k < K_COUNT; ++k) {
        r->prof.ms[k] = 0.0;
        r->prof.launches[k] = 0;
    }
    if (!r->prof.work) RL_TRY(ralloc(r, W_COUNT, &r->prof.work));
    RL_CK(cudaMemset(r->prof.work, 0, sizeof(unsigned long long) * W_COUNT));
    r->prof.on = enable != 0;
    return RL_OK;
}

extern "C" rl_status rl_reloc_profile_read(rl_reloc *r, double *ms, int64_t *launches, uint64_t *work) {
    if (!r) return fail(RL_ERR_INVALID_ARG, "null relocaliser");
    RL_CK(cudaSetDevice(r->forest->ctx->device));
    RL_CK(cudaDeviceSynchronize());
    prof_resolve(r);
    for (int k = 0; k < K_COUNT; ++k) {
        if (ms) ms[k] = r->prof.ms[k];
        if (launches) launches[k] = r->prof.launches[k];
    }
    if (work) {
        if (r->prof.work)
            RL_CK(cudaMemcpy(work, r->prof.work, sizeof(unsigned long long) * W_COUNT, cudaMemcpyDeviceToHost));
        else
            for (int k = 0; k < W_COUNT; ++k) work[k] = 0;
    }
    return RL_OK;
}

// ---------------------------------------------------------------------------
// Standalone ranking score (Eq. 6-7) of given poses.
// ---------------------------------------------------------------------------
extern "C" rl_status rl_score_poses(rl_scene *sc, const float *depth, const rl_intrinsics *K,
                                    const double *poses, int32_t n, rl_mem mem, void *stream,
                                    float *scores, float *valid_frac) {
    if (!sc || !depth || !K || !poses || !scores) return fail(RL_ERR_INVALID_ARG, "null argument");
    if (n < 1 || n > 65535) return fail(RL_ERR_INVALID_ARG, "n must be 1..65535");
    if (K->width < 1 || K->height < 1 || K->width > 8192 || K->height > 8192 || !(K->fx > 0) || !(K->fy > 0))
        return fail(RL_ERR_INVALID_ARG, "bad intrinsics");
    if (mem != RL_HOST && mem != RL_DEVICE) return fail(RL_ERR_INVALID_ARG, "bad rl_mem");
    rl_ctx *ctx = sc->ctx;
    RL_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int npx = K->width * K->height;
    const int tiles = (npx + RC_TILE - 1) / RC_TILE;
    Frame *fr = nullptr;
    double *pd = nullptr, *psum = nullptr;
    int32_t *pcnt = nullptr;
    float *sd = nullptr, *vd = nullptr, *dd = nullptr;
    rl_status st = alloc_n(ctx, 1, &fr);
    if (st == RL_OK) st = alloc_n(ctx, (uint64_t)n * 12, &pd);
    if (st == RL_OK) st = alloc_n(ctx, (uint64_t)n * tiles, &psum);
    if (st == RL_OK) st = alloc_n(ctx, (uint64_t)n * tiles * 2, &pcnt);
    if (st == RL_OK) st = alloc_n(ctx, (uint64_t)n * 2, &sd);
    if (st == RL_OK && mem == RL_HOST) st = alloc_n(ctx, (uint64_t)npx, &dd);
    std::vector<double> p12((size_t)n * 12);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 12; ++k) p12[(size_t)i * 12 + k] = poses[(size_t)i * 16 + k];
    Frame h{};
    h.depth = mem == RL_HOST ? dd : depth;
    h.rgb = nullptr;
    h.fx = K->fx; h.fy = K->fy; h.cx = K->cx; h.cy = K->cy;
    h.W = K->width; h.H = K->height;
    std::vector<float> hs((size_t)n * 2);
    if (st == RL_OK && mem == RL_HOST &&
        cudaMemcpyAsync(dd, depth, sizeof(float) * npx, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = fail(RL_ERR_CUDA, "depth copy failed");
    if (st == RL_OK && cudaMemcpyAsync(fr, &h, sizeof(Frame), cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = fail(RL_ERR_CUDA, "frame copy failed");
    if (st == RL_OK && cudaMemcpyAsync(pd, p12.data(), p12.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = fail(RL_ERR_CUDA, "pose copy failed");
    if (st == RL_OK) {
        vd = sd + n;
        RaycastArgs ra{};
        ra.frames = fr;
        ra.poses = pd;
        ra.n_poses = nullptr;
        ra.pose_cap = n;
        for (int a = 0; a < 3; ++a) {
            ra.lo[a] = (float)sc->lo[a];
            ra.hi[a] = (float)sc->hi[a];
            ra.lo64[a] = sc->lo[a];
            ra.hi64[a] = sc->hi[a];
        }
        ra.part_sum = psum;
        ra.part_cnt = pcnt;
        ra.n_tiles = tiles;
        st = launch_score_poses(ra, n, npx, sd, vd, s);
    }
    if (st == RL_OK && cudaMemcpyAsync(hs.data(), sd, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = fail(RL_ERR_CUDA, "score copy failed");
    if (st == RL_OK && cudaStreamSynchronize(s) != cudaSuccess) st = fail(RL_ERR_CUDA, "scoring failed");
    if (st == RL_OK)
        for (int i = 0; i < n; ++i) {
            scores[i] = hs[i];
            if (valid_frac) valid_frac[i] = hs[n + i];
        }
    void *ptrs[] = {fr, pd, psum, pcnt, sd, dd};
    for (void *p : ptrs) arena_free(ctx, p);
    return st;
}

// ---------------------------------------------------------------------------
// Standalone ICP (Sec. 3.2.4) of given poses against the box model.
// ---------------------------------------------------------------------------
extern "C" rl_status rl_icp_poses(rl_scene *sc, const float *depth, const rl_intrinsics *K,
                                  const double *poses, int32_t n, const rl_icp_params *ip, rl_mem mem,
                                  void *stream, double *refined, int32_t *ok, float *frac) {
    if (!sc || !depth || !K || !poses || !ip || !refined || !ok) return fail(RL_ERR_INVALID_ARG, "null argument");
    if (n < 1 || n > 65535) return fail(RL_ERR_INVALID_ARG, "n must be 1..65535");
    if (K->width < 1 || K->height < 1 || K->width > 8192 || K->height > 8192 || !(K->fx > 0) || !(K->fy > 0))
        return fail(RL_ERR_INVALID_ARG, "bad intrinsics");
    if (mem != RL_HOST && mem != RL_DEVICE) return fail(RL_ERR_INVALID_ARG, "bad rl_mem");
    RL_TRY(check_icp(ip));
    rl_ctx *ctx = sc->ctx;
    RL_CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int npx = K->width * K->height;
    Frame *fr = nullptr;
    double *pd = nullptr;
    int32_t *okd = nullptr;
    float *fd = nullptr, *dd = nullptr;
    rl_status st = alloc_n(ctx, 1, &fr);
    if (st == RL_OK) st = alloc_n(ctx, (uint64_t)n * 12, &pd);
    if (st == RL_OK) st = alloc_n(ctx, (uint64_t)n, &okd);
    if (st == RL_OK) st = alloc_n(ctx, (uint64_t)n, &fd);
    if (st == RL_OK && mem == RL_HOST) st = alloc_n(ctx, (uint64_t)npx, &dd);
    std::vector<double> p12((size_t)n * 12);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 12; ++k) p12[(size_t)i * 12 + k] = poses[(size_t)i * 16 + k];
    Frame h{};
    h.depth = mem == RL_HOST ? dd : depth;
    h.rgb = nullptr;
    h.fx = K->fx; h.fy = K->fy; h.cx = K->cx; h.cy = K->cy;
    h.W = K->width; h.H = K->height;
    std::vector<int32_t> hok(n);
    std::vector<float> hfrac(n);
    if (st == RL_OK && mem == RL_HOST &&
        cudaMemcpyAsync(dd, depth, sizeof(float) * npx, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = fail(RL_ERR_CUDA, "depth copy failed");
    if (st == RL_OK && cudaMemcpyAsync(fr, &h, sizeof(Frame), cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = fail(RL_ERR_CUDA, "frame copy failed");
    if (st == RL_OK && cudaMemcpyAsync(pd, p12.data(), p12.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = fail(RL_ERR_CUDA, "pose copy failed");
    if (st == RL_OK) {
        IcpArgs ia{};
        ia.frames = fr;
        ia.poses = pd;
        ia.pose_stride = n;
        ia.cap = n;
        ia.ok = okd;
        ia.frac = fd;
        ia.out_stride = n;
        for (int a = 0; a < 3; ++a) {
            ia.lo[a] = (float)sc->lo[a];
            ia.hi[a] = (float)sc->hi[a];
        }
        ia.ip = icp_device_params(*ip);
        st = launch_icp(ia, 1, s);
    }
    if (st == RL_OK && (cudaMemcpyAsync(p12.data(), pd, p12.size() * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaMemcpyAsync(hok.data(), okd, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaMemcpyAsync(hfrac.data(), fd, sizeof(float) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess))
        st = fail(RL_ERR_CUDA, "result copy failed");
    if (st == RL_OK && cudaStreamSynchronize(s) != cudaSuccess) st = fail(RL_ERR_CUDA, "ICP failed");
    if (st == RL_OK)
        for (int i = 0; i < n; ++i) {
            for (int k = 0; k < 16; ++k) refined[(size_t)i * 16 + k] = k < 12 ? p12[(size_t)i * 12 + k] : (k == 15 ? 1.0 : 0.0);
            ok[i] = hok[i];
            if (frac) frac[i] = hfrac[i];
        }
    void *ptrs[] = {fr, pd, okd, fd, dd};
    for (void *p : ptrs) arena_free(ctx, p);
    return st;
}

// ---------------------------------------------------------------------------
// Launch-shape tuning and the autotuner.  Every tunable shape leaves each
// kernel's arithmetic and its order unchanged, so tuning never changes a
// result; only the time to get it.
// ---------------------------------------------------------------------------
namespace rl {

static bool one_of(int v, std::initializer_list<int> l) {
    for (int x : l)
        if (v == x) return true;
    return false;
}

static bool valid_tuning(const rl_tuning &t) {
    return one_of(t.hypgen_warps, {2, 4, 8, 16}) && one_of(t.energy_threads, {32, 64, 128, 256}) &&
           one_of(t.leaves_threads, {64, 128, 256, 512}) && one_of(t.mask_threads, {64, 128, 256}) &&
           one_of(t.streams, {1, 2, 4, 8});
}

static std::string trim(const std::string &x) {
    size_t a = x.find_first_not_of(" \t\r\n"), b = x.find_last_not_of(" \t\r\n");
    return a == std::string::npos ? std::string() : x.substr(a, b - a + 1);
}

}  // namespace rl

extern "C" rl_status rl_reloc_get_tuning(rl_reloc *r, rl_tuning *out) {
    if (!r || !out) return fail(RL_ERR_INVALID_ARG, "null argument");
    *out = r->tune;
    return RL_OK;
}

extern "C" rl_status rl_reloc_set_tuning(rl_reloc *r, const rl_tuning *t) {
    if (!r || !t) return fail(RL_ERR_INVALID_ARG, "null argument");
    if (!valid_tuning(*t)) return fail(RL_ERR_INVALID_ARG, "tuning value outside its list");
    RL_CK(cudaSetDevice(r->forest->ctx->device));
    RL_CK(cudaDeviceSynchronize());
    graphs_free(r);
    r->tune = *t;
    ++r->tune_gen;
    return RL_OK;
}

extern "C" rl_status rl_tuning_key(rl_reloc *r, char *buf, int32_t len) {
    if (!r || !buf || len < 1) return fail(RL_ERR_INVALID_ARG, "null argument");
    cudaDeviceProp prop;
    RL_CK(cudaGetDeviceProperties(&prop, r->forest->ctx->device));
    std::string name = prop.name;
    for (char &ch : name)
        if (ch == ' ' || ch == '=' || ch == '\t') ch = '_';
    const RParams &p = r->rp;
    char tmp[512];
    const int w = snprintf(tmp, sizeof(tmp), "%s|sm%d|%dx%d|b%d|T%d|d%d|ktop%d|mpad%d|N%d|C%d|eta%d|cov%d|mask%d",
                           name.c_str(), prop.multiProcessorCount, r->max_w, r->max_h, r->max_batch, p.n_trees,
                           r->forest->p.depth, p.k_top, p.mpad, p.n_hyp, p.n_cull, p.eta, p.use_cov ? 1 : 0,
                           r->q.pcm ? 1 : 0);
    if (w < 0 || w >= len) return fail(RL_ERR_INVALID_ARG, "key buffer too small");
    memcpy(buf, tmp, (size_t)w + 1);
    return RL_OK;
}

extern "C" rl_status rl_tuning_cache_read(const char *path, const char *key, rl_tuning *out, int32_t *found) {
    if (!path || !key || !out || !found) return fail(RL_ERR_INVALID_ARG, "null argument");
    *found = 0;
    FILE *fp = fopen(path, "r");
    if (!fp) return RL_OK;
    char line[1024];
    while (fgets(line, sizeof(line), fp)) {
        std::string l(line);
        const size_t eq = l.find('=');
        if (eq == std::string::npos || trim(l.substr(0, eq)) != key) continue;
        rl_tuning t{};
        t.streams = 1;  // entries written before the streams knob hold four values
        const int got = sscanf(l.c_str() + eq + 1, "%d %d %d %d %d", &t.hypgen_warps, &t.energy_threads,
                               &t.leaves_threads, &t.mask_threads, &t.streams);
        if ((got == 4 || got == 5) && valid_tuning(t)) {
            *out = t;
            *found = 1;
        }
    }
    fclose(fp);
    return RL_OK;
}

extern "C" rl_status rl_tuning_cache_write(const char *path, const char *key, const rl_tuning *t) {
    if (!path || !key || !t) return fail(RL_ERR_INVALID_ARG, "null argument");
    if (!valid_tuning(*t)) return fail(RL_ERR_INVALID_ARG, "tuning value outside its list");
    std::vector<std::string> lines;
    if (FILE *fp = fopen(path, "r")) {
        char line[1024];
        while (fgets(line, sizeof(line), fp)) {
            std::string l(line);
            const size_t eq = l.find('=');
            if (eq != std::string::npos && trim(l.substr(0, eq)) == key) continue;  // replaced below
            if (!trim(l).empty()) lines.push_back(trim(l));
        }
        fclose(fp);
    }
    char entry[1100];
    snprintf(entry, sizeof(entry), "%s = %d %d %d %d %d", key, t->hypgen_warps, t->energy_threads,
             t->leaves_threads, t->mask_threads, t->streams);
    lines.push_back(entry);
    const std::string tmp = std::string(path) + ".tmp";
    FILE *fp = fopen(tmp.c_str(), "w");
    if (!fp) return fail(RL_ERR_IO, "cannot write the tuning cache");
    bool ok = true;
    for (auto &l : lines) ok = ok && fprintf(fp, "%s\n", l.c_str()) > 0;
    ok = (fclose(fp) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) return fail(RL_ERR_IO, "cannot write the tuning cache");
    return RL_OK;
}

extern "C" rl_status rl_reloc_autotune(rl_reloc *r, int32_t n, const float *depth, const uint8_t *rgb,
                                       const rl_intrinsics *K, const uint64_t *seeds, rl_mem mem, void *stream,
                                       const char *cache_path, rl_tuning *out) {
    if (!r) return fail(RL_ERR_INVALID_ARG, "null relocaliser");
    char key[512];
    RL_TRY(rl_tuning_key(r, key, (int32_t)sizeof(key)));
    if (cache_path) {
        rl_tuning t{};
        int32_t found = 0;
        RL_TRY(rl_tuning_cache_read(cache_path, key, &t, &found));
        if (found) {
            RL_TRY(rl_reloc_set_tuning(r, &t));
            if (out) *out = t;
            return RL_OK;
        }
    }
    RL_TRY(check_call(r, n, depth, rgb, K, seeds));
    const bool was_on = r->prof.on;
    std::vector<rl_result> res((size_t)n);
    struct Knob {
        int32_t rl_tuning::*field;
        std::vector<int> values;
        int kid;
    };
    std::vector<Knob> knobs = {{&rl_tuning::hypgen_warps, {4, 8, 16}, K_HYPGEN},
                               {&rl_tuning::energy_threads, {32, 64, 128, 256}, K_ENERGY},
                               {&rl_tuning::leaves_threads, {64, 128, 256, 512}, K_LEAVES}};
    if (r->q.pcm) knobs.push_back({&rl_tuning::mask_threads, {64, 128, 256}, K_CMASK});
    rl_tuning t = r->tune;
    rl_status st = RL_OK;
    for (const Knob &k : knobs) {
        int best = t.*k.field;
        double best_ms = INFINITY, cur_ms = INFINITY;
        for (int v : k.values) {
            rl_tuning c = t;
            c.*k.field = v;
            r->tune = c;
            double ms[RL_N_KERNELS];
            if ((st = rl_reloc_profile(r, 1)) != RL_OK) break;      // resets the counters; launches bypass graphs
            for (int rep = 0; rep < 2 && st == RL_OK; ++rep)
                st = rl_relocalise_batch(r, n, depth, rgb, K, seeds, mem, stream, res.data());
            if (st == RL_OK) st = rl_reloc_profile_read(r, ms, nullptr, nullptr);
            if (st != RL_OK) break;
            if (v == t.*k.field) cur_ms = ms[k.kid];
            if (ms[k.kid] < best_ms) {
                best_ms = ms[k.kid];
                best = v;
            }
        }
        if (st != RL_OK) break;
        // keep the current value unless another is at least 2% faster
        t.*k.field = best_ms < 0.98 * cur_ms ? best : t.*k.field;
    }
    rl_reloc_profile(r, was_on ? 1 : 0);
    // sub-batches: whole calls on the captured-graph path, timed on the host
    // (per-kernel times cannot see kernels of different streams overlap)
    if (st == RL_OK && !was_on && r->use_graphs && n >= 2 * kMinPart) {
        int best = t.streams;
        double best_ms = INFINITY, cur_ms = INFINITY;
        for (int v : {1, 2, 4, 8}) {
            if (v > 1 && n / kMinPart < v) break;  // would run as fewer sub-batches
            rl_tuning c = t;
            c.streams = v;
            if ((st = rl_reloc_set_tuning(r, &c)) != RL_OK) break;  // drops the captured graphs
            if ((st = rl_relocalise_batch(r, n, depth, rgb, K, seeds, mem, stream, res.data())) != RL_OK) break;
            double ms = INFINITY;
            for (int rep = 0; rep < 3 && st == RL_OK; ++rep) {
                const auto t0 = std::chrono::steady_clock::now();
                st = rl_relocalise_batch(r, n, depth, rgb, K, seeds, mem, stream, res.data());
                ms = std::min(ms, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                                      .count());
            }
            if (st != RL_OK) break;
            if (v == t.streams) cur_ms = ms;
            if (ms < best_ms) {
                best_ms = ms;
                best = v;
            }
        }
        if (st == RL_OK) t.streams = best_ms < 0.98 * cur_ms ? best : t.streams;
    }
    if (st != RL_OK) {
        r->tune = t;
        return st;
    }
    RL_TRY(rl_reloc_set_tuning(r, &t));
    if (cache_path) RL_TRY(rl_tuning_cache_write(cache_path, key, &t));
    if (out) *out = t;
    return RL_OK;
}
