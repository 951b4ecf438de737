// Context, arena allocator, error plumbing, forest and scene handles.
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include <cuda_fp16.h>

#include "internal.h"

namespace rl {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

rl_status fail(rl_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

rl_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_last_error = buf;
    return RL_ERR_CUDA;
}

static const uint64_t kAlign = 256;

rl_status arena_alloc(rl_ctx *c, uint64_t bytes, void **out) {
    *out = nullptr;
    if (bytes == 0) bytes = kAlign;
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    std::lock_guard<std::mutex> g(c->mu);
    uint64_t cursor = 0;
    for (auto &kv : c->live) {  // first fit between live blocks
        if (kv.first - cursor >= bytes) break;
        cursor = kv.first + kv.second;
    }
    if (cursor + bytes > c->bytes) {
        char buf[160];
        snprintf(buf, sizeof(buf), "arena exhausted: need %llu bytes, %llu of %llu in use",
                 (unsigned long long)bytes, (unsigned long long)c->used,
                 (unsigned long long)c->bytes);
        return fail(RL_ERR_OOM, buf);
    }
    c->live[cursor] = bytes;
    c->used += bytes;
    c->peak = std::max(c->peak, c->used);
    *out = c->base + cursor;
    return RL_OK;
}

void arena_free(rl_ctx *c, void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(c->mu);
    uint64_t off = (uint64_t)((uint8_t *)p - c->base);
    auto it = c->live.find(off);
    if (it == c->live.end()) return;
    c->used -= it->second;
    c->live.erase(it);
}

ModeView mode_view(const rl_forest *f) {
    ModeView v;
    v.nmodes = f->nmodes;
    v.centroid = f->centroid;
    v.mpos_h = f->p.mode_precision == RL_MODES_FP16_OFFSET ? f->mpos_h : nullptr;
    v.mpos_f = f->p.mode_precision == RL_MODES_FP16_OFFSET ? nullptr : f->mpos_f;
    v.mrgb = f->mrgb;
    v.mU = f->mU;
    v.m_max = f->p.m_max;
    v.leaves_per_tree = f->leaves_per_tree;
    return v;
}

// ---------------------------------------------------------------------------
// Streaming adaptation: two mode stores.  Relocalisers read the front store
// (the forest's mode arrays); a mode update first waits for every launch
// that read the back store, swaps the two, brings the new front up to date
// on the leaves the previous update wrote (a device copy of that range from
// the old front), clusters its own range into it and records `ready`, which
// later relocalisation launches wait for.  A launch thus sees one complete
// snapshot: the modes after the last update enqueued before it.
// ---------------------------------------------------------------------------
static ModeStore front_store(const rl_forest *f) {
    ModeStore m;
    m.nmodes = f->nmodes;
    m.centroid = f->centroid;
    m.mpos_h = f->mpos_h;
    m.mpos_f = f->mpos_f;
    m.mrgb = f->mrgb;
    m.mU = f->mU;
    m.msize = f->msize;
    return m;
}

static void set_front_store(rl_forest *f, const ModeStore &m) {
    f->nmodes = m.nmodes;
    f->centroid = m.centroid;
    f->mpos_h = m.mpos_h;
    f->mpos_f = m.mpos_f;
    f->mrgb = m.mrgb;
    f->mU = m.mU;
    f->msize = m.msize;
}

void free_store(rl_ctx *c, ModeStore &m) {
    void *ptrs[] = {m.nmodes, m.centroid, m.mpos_h, m.mpos_f, m.mrgb, m.mU, m.msize};
    for (void *p : ptrs) arena_free(c, p);
    m = ModeStore{};
}

static rl_status alloc_store(rl_forest *f, ModeStore &m) {
    const uint64_t L = (uint64_t)f->n_leaves, M = (uint64_t)f->p.m_max;
    rl_status s = alloc_n(f->ctx, L, &m.nmodes);
    if (s == RL_OK) s = alloc_n(f->ctx, L, &m.centroid);
    if (s == RL_OK && f->p.mode_precision == RL_MODES_FP16_OFFSET) s = alloc_n(f->ctx, L * M, &m.mpos_h);
    if (s == RL_OK && f->p.mode_precision == RL_MODES_FP32) s = alloc_n(f->ctx, L * M, &m.mpos_f);
    if (s == RL_OK) s = alloc_n(f->ctx, L * M, &m.mrgb);
    if (s == RL_OK) s = alloc_n(f->ctx, L * M * 2, &m.mU);
    if (s == RL_OK) s = alloc_n(f->ctx, L * M, &m.msize);
    if (s != RL_OK) free_store(f->ctx, m);
    return s;
}

template <class T>
static rl_status copy_rows(T *dst, const T *src, int64_t row, int64_t b, int64_t n, cudaStream_t s) {
    if (!dst || !src || n <= 0) return RL_OK;
    RL_CK(cudaMemcpyAsync(dst + b * row, src + b * row, sizeof(T) * (size_t)(n * row), cudaMemcpyDeviceToDevice, s));
    return RL_OK;
}

// Leaves [begin, begin + count) mod L of every mode array, src -> dst.
static rl_status copy_store_range(const rl_forest *f, const ModeStore &src, const ModeStore &dst, int64_t begin,
                                  int64_t count, cudaStream_t s) {
    const int64_t L = f->n_leaves, M = f->p.m_max;
    count = std::min<int64_t>(count, L);
    const int64_t b0 = begin % L, n0 = std::min<int64_t>(count, L - b0), n1 = count - n0;
    const int64_t segs[2][2] = {{b0, n0}, {0, n1}};
    for (const auto &g : segs) {
        RL_TRY(copy_rows(dst.nmodes, src.nmodes, 1, g[0], g[1], s));
        RL_TRY(copy_rows(dst.centroid, src.centroid, 1, g[0], g[1], s));
        RL_TRY(copy_rows(dst.mpos_h, src.mpos_h, M, g[0], g[1], s));
        RL_TRY(copy_rows(dst.mpos_f, src.mpos_f, M, g[0], g[1], s));
        RL_TRY(copy_rows(dst.mrgb, src.mrgb, M, g[0], g[1], s));
        RL_TRY(copy_rows(dst.mU, src.mU, 2 * M, g[0], g[1], s));
        RL_TRY(copy_rows(dst.msize, src.msize, M, g[0], g[1], s));
    }
    return RL_OK;
}

// Stream s waits for every launch that read mode store b.
static rl_status wait_readers(rl_forest *f, int b, cudaStream_t s) {
    for (rl_reloc *r : f->readers)
        if (r->read_valid[b]) RL_CK(cudaStreamWaitEvent(s, r->read_done[b], 0));
    return RL_OK;
}

// An in-place update of a one-store forest's modes, enqueued on s: it waits
// for the launches that read the store, and launches enqueued after it (on
// any stream) wait for `ready`, recorded after it.
template <class F>
static rl_status in_place_update(rl_forest *f, cudaStream_t s, F &&update) {
    std::lock_guard<std::mutex> g(f->mu);
    RL_TRY(wait_readers(f, 0, s));
    RL_TRY(update());
    if (!f->ready) RL_CK(cudaEventCreateWithFlags(&f->ready, cudaEventDisableTiming));
    RL_CK(cudaEventRecord(f->ready, s));
    return RL_OK;
}

static rl_status streaming_update(rl_forest *f, int64_t begin, int64_t count, cudaStream_t s) {
    std::lock_guard<std::mutex> g(f->mu);
    const int back = 1 - f->mode_buf;
    RL_TRY(wait_readers(f, back, s));
    const ModeStore old_front = front_store(f), old_back = f->alt;
    set_front_store(f, old_back);  // the back store becomes the front
    f->alt = old_front;
    rl_status st = copy_store_range(f, old_front, old_back, f->last_begin, f->last_count, s);
    if (st == RL_OK) st = update_modes(f, begin, count, s);
    if (st == RL_OK && cudaEventRecord(f->ready, s) != cudaSuccess) st = fail(RL_ERR_CUDA, "event record failed");
    if (st != RL_OK) {  // keep the previous snapshot in front
        set_front_store(f, old_front);
        f->alt = old_back;
        return st;
    }
    f->mode_buf = back;
    f->last_begin = begin;
    f->last_count = count;
    return RL_OK;
}

}  // namespace rl

using namespace rl;

extern "C" const char *rl_last_error(void) { return g_last_error.c_str(); }

extern "C" rl_status rl_context_create(int32_t device, void *arena, uint64_t bytes, rl_ctx **out) {
    if (!out) return fail(RL_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!arena || bytes < (1u << 20)) return fail(RL_ERR_INVALID_ARG, "arena null or < 1 MiB");
    if ((uintptr_t)arena % 256 != 0) return fail(RL_ERR_INVALID_ARG, "arena not 256-byte aligned");
    int n = 0;
    RL_CK(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(RL_ERR_INVALID_ARG, "bad device index");
    RL_CK(cudaSetDevice(device));
    cudaPointerAttributes attr;
    RL_CK(cudaPointerGetAttributes(&attr, arena));
    if (attr.type != cudaMemoryTypeDevice || attr.device != device)
        return fail(RL_ERR_INVALID_ARG, "arena is not device memory of this device");
    rl_ctx *c = new rl_ctx();
    c->device = device;
    c->base = (uint8_t *)arena;
    c->bytes = bytes;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    *out = c;
    return RL_OK;
}

extern "C" rl_status rl_context_destroy(rl_ctx *c) {
    if (!c) return fail(RL_ERR_INVALID_ARG, "null context");
    delete c;
    return RL_OK;
}

extern "C" rl_status rl_context_usage(const rl_ctx *c, uint64_t *used, uint64_t *peak) {
    if (!c) return fail(RL_ERR_INVALID_ARG, "null context");
    if (used) *used = c->used;
    if (peak) *peak = c->peak;
    return RL_OK;
}

// ---------------------------------------------------------------------------
// Forest
// ---------------------------------------------------------------------------
static rl_status check_forest_params(const rl_forest_params *p) {
    if (!p) return fail(RL_ERR_INVALID_ARG, "null forest params");
    if (p->n_trees < 1 || p->n_trees > 16) return fail(RL_ERR_INVALID_ARG, "n_trees must be 1..16");
    if (p->depth < 1 || p->depth > 15) return fail(RL_ERR_INVALID_ARG, "depth must be 1..15");
    if (p->kappa < 1 || p->kappa > 4096) return fail(RL_ERR_INVALID_ARG, "kappa must be 1..4096");
    if (p->m_max < 1 || p->m_max > 64) return fail(RL_ERR_INVALID_ARG, "m_max must be 1..64");
    if (p->min_cluster_size < 1) return fail(RL_ERR_INVALID_ARG, "min_cluster_size must be >= 1");
    if (!(p->sigma > 0) || !(p->tau_c >= 0)) return fail(RL_ERR_INVALID_ARG, "bad sigma/tau_c");
    if (p->grid_step < 1 || p->grid_origin < 0) return fail(RL_ERR_INVALID_ARG, "bad grid");
    if (p->mode_precision != RL_MODES_FP32 && p->mode_precision != RL_MODES_FP16_OFFSET)
        return fail(RL_ERR_INVALID_ARG, "bad mode_precision");
    if (!(p->p_depth >= 0 && p->p_depth <= 1)) return fail(RL_ERR_INVALID_ARG, "bad p_depth");
    return RL_OK;
}

static void forest_release(rl_forest *f) {
    rl_ctx *c = f->ctx;
    void *ptrs[] = {f->nodes, f->res, f->res_count, f->nmodes, f->centroid, f->mpos_h, f->mpos_f,
                    f->mrgb, f->mU, f->msize, f->ex_leaf, f->ex_pt, f->ex_rank, f->frame_cnt,
                    f->stage_depth, f->stage_rgb};
    for (void *p : ptrs) arena_free(c, p);
    free_store(c, f->alt);
    if (f->ready) cudaEventDestroy(f->ready);
    f->ready = nullptr;
}

static rl_status forest_alloc(rl_ctx *ctx, const rl_forest_params *p, uint64_t seed,
                              rl_forest **out) {
    RL_TRY(check_forest_params(p));
    rl_forest *f = new rl_forest();
    f->ctx = ctx;
    f->p = *p;
    f->seed = seed;
    f->n_branch = (1 << p->depth) - 1;
    f->leaves_per_tree = 1 << p->depth;
    f->n_leaves = p->n_trees << p->depth;
    const uint64_t L = (uint64_t)f->n_leaves, M = (uint64_t)p->m_max;
    rl_status s = RL_OK;
    if (s == RL_OK) s = alloc_n(ctx, (uint64_t)p->n_trees * f->n_branch, &f->nodes);
    if (s == RL_OK) s = alloc_n(ctx, L * p->kappa, &f->res);
    if (s == RL_OK) s = alloc_n(ctx, L, &f->res_count);
    if (s == RL_OK) s = alloc_n(ctx, L, &f->nmodes);
    if (s == RL_OK) s = alloc_n(ctx, L, &f->centroid);
    if (s == RL_OK && p->mode_precision == RL_MODES_FP16_OFFSET) s = alloc_n(ctx, L * M, &f->mpos_h);
    if (s == RL_OK && p->mode_precision == RL_MODES_FP32) s = alloc_n(ctx, L * M, &f->mpos_f);
    if (s == RL_OK) s = alloc_n(ctx, L * M, &f->mrgb);
    if (s == RL_OK) s = alloc_n(ctx, L * M * 2, &f->mU);
    if (s == RL_OK) s = alloc_n(ctx, L * M, &f->msize);
    if (s == RL_OK) s = alloc_n(ctx, L, &f->frame_cnt);
    if (s != RL_OK) {
        forest_release(f);
        delete f;
        return s;
    }
    *out = f;
    return RL_OK;
}

extern "C" rl_status rl_forest_create_random(rl_ctx *ctx, const rl_forest_params *p, uint64_t seed,
                                             rl_forest **out) {
    if (!ctx || !out) return fail(RL_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    RL_CK(cudaSetDevice(ctx->device));
    rl_forest *f = nullptr;
    RL_TRY(forest_alloc(ctx, p, seed, &f));
    rl_status s = launch_forest_random(f, 0);
    if (s == RL_OK) s = reset_leaves(f, 0);
    if (s == RL_OK) {
        cudaError_t e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) s = cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    }
    if (s != RL_OK) {
        forest_release(f);
        delete f;
        return s;
    }
    *out = f;
    return RL_OK;
}

extern "C" rl_status rl_forest_destroy(rl_forest *f) {
    if (!f) return fail(RL_ERR_INVALID_ARG, "null forest");
    if (f->refcount > 0) return fail(RL_ERR_BUSY, "forest still used by a relocaliser");
    cudaSetDevice(f->ctx->device);
    cudaDeviceSynchronize();
    forest_release(f);
    delete f;
    return RL_OK;
}

extern "C" rl_status rl_forest_reset_leaves(rl_forest *f, void *stream) {
    if (!f) return fail(RL_ERR_INVALID_ARG, "null forest");
    RL_CK(cudaSetDevice(f->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (!f->streaming) return in_place_update(f, s, [&] { return reset_leaves(f, s); });
    // both stores emptied once no launch reads either
    std::lock_guard<std::mutex> g(f->mu);
    RL_TRY(wait_readers(f, 0, s));
    RL_TRY(wait_readers(f, 1, s));
    RL_TRY(reset_leaves(f, s));
    RL_CK(cudaMemsetAsync(f->alt.nmodes, 0, f->n_leaves, s));
    RL_CK(cudaMemsetAsync(f->alt.centroid, 0, sizeof(float4) * f->n_leaves, s));
    RL_CK(cudaEventRecord(f->ready, s));
    f->last_count = 0;
    return RL_OK;
}

static rl_status check_intrinsics(const rl_intrinsics *K) {
    if (!K) return fail(RL_ERR_INVALID_ARG, "null intrinsics");
    if (K->width < 1 || K->height < 1 || K->width > 8192 || K->height > 8192)
        return fail(RL_ERR_INVALID_ARG, "image size must be 1..8192");
    if (!(K->fx > 0) || !(K->fy > 0)) return fail(RL_ERR_INVALID_ARG, "focal lengths must be > 0");
    return RL_OK;
}

extern "C" rl_status rl_forest_adapt(rl_forest *f, const float *depth, const uint8_t *rgb,
                                     const rl_intrinsics *K, const double T[16], rl_mem mem,
                                     void *stream) {
    if (!f || !depth || !rgb || !T) return fail(RL_ERR_INVALID_ARG, "null argument");
    RL_TRY(check_intrinsics(K));
    RL_CK(cudaSetDevice(f->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int npx = K->width * K->height;
    if (mem == RL_HOST) {
        if (f->stage_pixels < npx) {
            arena_free(f->ctx, f->stage_depth);
            arena_free(f->ctx, f->stage_rgb);
            f->stage_depth = nullptr;
            f->stage_rgb = nullptr;
            f->stage_pixels = 0;
            RL_TRY(alloc_n(f->ctx, (uint64_t)npx, &f->stage_depth));
            RL_TRY(alloc_n(f->ctx, (uint64_t)npx * 3, &f->stage_rgb));
            f->stage_pixels = npx;
        }
        RL_CK(cudaMemcpyAsync(f->stage_depth, depth, sizeof(float) * npx, cudaMemcpyHostToDevice, s));
        RL_CK(cudaMemcpyAsync(f->stage_rgb, rgb, (size_t)npx * 3, cudaMemcpyHostToDevice, s));
        depth = f->stage_depth;
        rgb = f->stage_rgb;
    } else if (mem != RL_DEVICE) {
        return fail(RL_ERR_INVALID_ARG, "bad rl_mem");
    }
    RL_TRY(adapt_frame(f, depth, rgb, K, T, s));
    if (mem == RL_HOST) RL_CK(cudaStreamSynchronize(s));  // staging reused next call
    return RL_OK;
}

extern "C" rl_status rl_forest_update_modes(rl_forest *f, int32_t n_leaves, void *stream) {
    if (!f) return fail(RL_ERR_INVALID_ARG, "null forest");
    RL_CK(cudaSetDevice(f->ctx->device));
    int64_t count = n_leaves < 0 ? f->n_leaves : std::min<int64_t>(n_leaves, f->n_leaves);
    int64_t begin = n_leaves < 0 ? 0 : f->cursor;
    cudaStream_t s = (cudaStream_t)stream;
    if (f->streaming)
        RL_TRY(streaming_update(f, begin, count, s));
    else
        RL_TRY(in_place_update(f, s, [&] { return update_modes(f, begin, count, s); }));
    if (n_leaves >= 0) f->cursor = (f->cursor + count) % f->n_leaves;
    return RL_OK;
}

extern "C" rl_status rl_forest_set_streaming(rl_forest *f, int32_t enable) {
    if (!f) return fail(RL_ERR_INVALID_ARG, "null forest");
    if (enable != 0 && enable != 1) return fail(RL_ERR_INVALID_ARG, "enable must be 0 or 1");
    if ((enable != 0) == f->streaming) return RL_OK;
    if (f->refcount > 0) return fail(RL_ERR_BUSY, "set streaming before creating relocalisers of the forest");
    RL_CK(cudaSetDevice(f->ctx->device));
    RL_CK(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> g(f->mu);
    if (enable) {
        RL_TRY(alloc_store(f, f->alt));
        rl_status s = copy_store_range(f, front_store(f), f->alt, 0, f->n_leaves, 0);
        if (s == RL_OK && cudaEventCreateWithFlags(&f->ready, cudaEventDisableTiming) != cudaSuccess)
            s = fail(RL_ERR_CUDA, "event creation failed");
        if (s == RL_OK && (cudaEventRecord(f->ready, 0) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess))
            s = fail(RL_ERR_CUDA, "initial mode copy failed");
        if (s != RL_OK) {
            free_store(f->ctx, f->alt);
            if (f->ready) cudaEventDestroy(f->ready);
            f->ready = nullptr;
            return s;
        }
        f->last_count = 0;
        f->streaming = true;
    } else {
        free_store(f->ctx, f->alt);
        cudaEventDestroy(f->ready);
        f->ready = nullptr;
        f->streaming = false;
    }
    return RL_OK;
}

extern "C" rl_status rl_forest_leaves(rl_forest *f, const float *depth, const uint8_t *rgb,
                                      const rl_intrinsics *K, int32_t n_trees,
                                      uint16_t *out_leaves, rl_mem mem, void *stream) {
    if (!f || !depth || !rgb || !out_leaves) return fail(RL_ERR_INVALID_ARG, "null argument");
    RL_TRY(check_intrinsics(K));
    if (n_trees < 1 || n_trees > f->p.n_trees) return fail(RL_ERR_INVALID_ARG, "bad n_trees");
    RL_CK(cudaSetDevice(f->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int npx = K->width * K->height;
    float *d = nullptr;
    uint8_t *c = nullptr;
    Frame *fr = nullptr;
    RL_TRY(alloc_n(f->ctx, 1, &fr));
    rl_status st = RL_OK;
    if (mem == RL_HOST) {
        st = alloc_n(f->ctx, (uint64_t)npx, &d);
        if (st == RL_OK) st = alloc_n(f->ctx, (uint64_t)npx * 3, &c);
        if (st == RL_OK && cudaMemcpyAsync(d, depth, sizeof(float) * npx, cudaMemcpyHostToDevice, s) != cudaSuccess)
            st = fail(RL_ERR_CUDA, "copy of depth failed");
        if (st == RL_OK && cudaMemcpyAsync(c, rgb, (size_t)npx * 3, cudaMemcpyHostToDevice, s) != cudaSuccess)
            st = fail(RL_ERR_CUDA, "copy of colour failed");
    }
    if (st == RL_OK) {
        Frame h;
        h.depth = mem == RL_HOST ? d : depth;
        h.rgb = mem == RL_HOST ? c : rgb;
        h.fx = K->fx; h.fy = K->fy; h.cx = K->cx; h.cy = K->cy;
        h.W = K->width; h.H = K->height;
        h.key0 = h.key1 = 0;
        if (cudaMemcpyAsync(fr, &h, sizeof(Frame), cudaMemcpyHostToDevice, s) != cudaSuccess)
            st = fail(RL_ERR_CUDA, "copy of frame descriptor failed");
        if (st == RL_OK) st = launch_leaves(f, fr, 1, n_trees, npx, out_leaves, K->width, K->height, s);
        if (st == RL_OK && cudaStreamSynchronize(s) != cudaSuccess)
            st = fail(RL_ERR_CUDA, "leaf kernel failed");
    }
    arena_free(f->ctx, fr);
    arena_free(f->ctx, d);
    arena_free(f->ctx, c);
    return st;
}

// Decodes the mode store to host buffers.
// Re-encodes the positions of leaves [l0, l0 + n): FP16 offsets from the
// stored FP32 centroid (difference exact in FP64, one rounding to half) or
// FP32 positions.  Ranks at or beyond the leaf's mode count are untouched.
__global__ void k_set_mode_positions(const float *__restrict__ pos, int l0, int n, int m_max,
                                     const uint8_t *__restrict__ nmodes, const float4 *__restrict__ centroid,
                                     ushort4 *mpos_h, float4 *mpos_f) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * m_max) return;
    const int l = l0 + e / m_max, r = e % m_max;
    if (r >= nmodes[l]) return;
    const float x = pos[3 * e], y = pos[3 * e + 1], z = pos[3 * e + 2];
    const size_t o = (size_t)l * m_max + r;
    if (mpos_h) {
        const float4 c = centroid[l];
        mpos_h[o] = make_ushort4(__half_as_ushort(__double2half((double)x - (double)c.x)),
                                 __half_as_ushort(__double2half((double)y - (double)c.y)),
                                 __half_as_ushort(__double2half((double)z - (double)c.z)), 0);
    } else {
        mpos_f[o] = make_float4(x, y, z, 0.f);
    }
}

extern "C" rl_status rl_forest_set_mode_positions(rl_forest *f, const float *mode_pos) {
    if (!f || !mode_pos) return fail(RL_ERR_INVALID_ARG, "null argument");
    RL_CK(cudaSetDevice(f->ctx->device));
    RL_CK(cudaDeviceSynchronize());
    const int M = f->p.m_max;
    const int chunk = std::max(1, (1 << 20) / (M * 3));  // leaves per staged chunk (<= 12 MB)
    float *stage = nullptr;
    RL_TRY(alloc_n(f->ctx, (uint64_t)chunk * M * 3, &stage));
    rl_status st = RL_OK;
    for (int l0 = 0; l0 < f->n_leaves && st == RL_OK; l0 += chunk) {
        const int n = std::min(chunk, f->n_leaves - l0);
        cudaError_t e = cudaMemcpy(stage, mode_pos + (size_t)l0 * M * 3, sizeof(float) * n * M * 3,
                                   cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "cudaMemcpy", __FILE__, __LINE__);
            break;
        }
        k_set_mode_positions<<<(n * M + 255) / 256, 256>>>(stage, l0, n, M, f->nmodes, f->centroid,
                                                           f->mpos_h, f->mpos_f);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(e, "k_set_mode_positions", __FILE__, __LINE__);
    }
    arena_free(f->ctx, stage);
    if (f->streaming) {  // the back store lacks the new positions everywhere
        f->last_begin = 0;
        f->last_count = f->n_leaves;
    }
    return st;
}

extern "C" rl_status rl_forest_export(rl_forest *f, float *node_dx, float *node_dy,
                                      float *node_tau, int32_t *node_meta, float *res_pos,
                                      uint8_t *res_rgb, uint32_t *res_count, uint8_t *nmodes,
                                      float *mode_pos, uint8_t *mode_rgb, float *mode_U,
                                      int32_t *mode_size) {
    if (!f) return fail(RL_ERR_INVALID_ARG, "null forest");
    RL_CK(cudaSetDevice(f->ctx->device));
    RL_CK(cudaDeviceSynchronize());
    const uint64_t NB = (uint64_t)f->p.n_trees * f->n_branch, L = f->n_leaves;
    const uint64_t K = f->p.kappa, M = f->p.m_max;
    if (node_dx || node_dy || node_tau || node_meta) {
        std::vector<float4> n(NB);
        RL_CK(cudaMemcpy(n.data(), f->nodes, NB * sizeof(float4), cudaMemcpyDeviceToHost));
        for (uint64_t i = 0; i < NB; ++i) {
            if (node_dx) node_dx[i] = n[i].x;
            if (node_dy) node_dy[i] = n[i].y;
            if (node_tau) node_tau[i] = n[i].z;
            if (node_meta) memcpy(&node_meta[i], &n[i].w, 4);
        }
    }
    if (res_pos || res_rgb) {
        std::vector<float4> r(L * K);
        RL_CK(cudaMemcpy(r.data(), f->res, L * K * sizeof(float4), cudaMemcpyDeviceToHost));
        for (uint64_t i = 0; i < L * K; ++i) {
            if (res_pos) { res_pos[3 * i] = r[i].x; res_pos[3 * i + 1] = r[i].y; res_pos[3 * i + 2] = r[i].z; }
            uint32_t c;
            memcpy(&c, &r[i].w, 4);
            if (res_rgb) { res_rgb[3 * i] = c & 255; res_rgb[3 * i + 1] = (c >> 8) & 255; res_rgb[3 * i + 2] = (c >> 16) & 255; }
        }
    }
    if (res_count) RL_CK(cudaMemcpy(res_count, f->res_count, L * 4, cudaMemcpyDeviceToHost));
    std::vector<uint8_t> nm(L);
    RL_CK(cudaMemcpy(nm.data(), f->nmodes, L, cudaMemcpyDeviceToHost));
    if (nmodes) memcpy(nmodes, nm.data(), L);
    if (mode_pos) {
        std::vector<float4> cen(L);
        RL_CK(cudaMemcpy(cen.data(), f->centroid, L * sizeof(float4), cudaMemcpyDeviceToHost));
        if (f->p.mode_precision == RL_MODES_FP16_OFFSET) {
            std::vector<ushort4> h(L * M);
            RL_CK(cudaMemcpy(h.data(), f->mpos_h, L * M * sizeof(ushort4), cudaMemcpyDeviceToHost));
            for (uint64_t l = 0; l < L; ++l)
                for (uint64_t m = 0; m < M; ++m) {
                    const ushort4 v = h[l * M + m];
                    const uint64_t e = l * M + m;
                    if (m >= nm[l]) { mode_pos[3 * e] = mode_pos[3 * e + 1] = mode_pos[3 * e + 2] = 0.f; continue; }
                    __half_raw hx, hy, hz;
                    hx.x = v.x; hy.x = v.y; hz.x = v.z;
                    mode_pos[3 * e + 0] = cen[l].x + __half2float(__half(hx));
                    mode_pos[3 * e + 1] = cen[l].y + __half2float(__half(hy));
                    mode_pos[3 * e + 2] = cen[l].z + __half2float(__half(hz));
                }
        } else {
            std::vector<float4> pf(L * M);
            RL_CK(cudaMemcpy(pf.data(), f->mpos_f, L * M * sizeof(float4), cudaMemcpyDeviceToHost));
            for (uint64_t e = 0; e < L * M; ++e) {
                mode_pos[3 * e] = pf[e].x; mode_pos[3 * e + 1] = pf[e].y; mode_pos[3 * e + 2] = pf[e].z;
            }
        }
    }
    if (mode_rgb) {
        std::vector<uchar4> c(L * M);
        RL_CK(cudaMemcpy(c.data(), f->mrgb, L * M * sizeof(uchar4), cudaMemcpyDeviceToHost));
        for (uint64_t e = 0; e < L * M; ++e) {
            mode_rgb[3 * e] = c[e].x; mode_rgb[3 * e + 1] = c[e].y; mode_rgb[3 * e + 2] = c[e].z;
        }
    }
    if (mode_U) {
        std::vector<float4> u(L * M * 2);
        RL_CK(cudaMemcpy(u.data(), f->mU, L * M * 2 * sizeof(float4), cudaMemcpyDeviceToHost));
        for (uint64_t e = 0; e < L * M; ++e) {
            const float4 a = u[2 * e], b = u[2 * e + 1];
            float *o = mode_U + 6 * e;
            o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y;
        }
    }
    if (mode_size) RL_CK(cudaMemcpy(mode_size, f->msize, L * M * 4, cudaMemcpyDeviceToHost));
    return RL_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint: header + raw device arrays.
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t pad;
    rl_forest_params p;
    uint64_t seed;
    int64_t cursor;
};

rl_status dump(FILE *fp, const void *dev, uint64_t bytes) {
    std::vector<uint8_t> h(bytes);
    if (bytes && cudaMemcpy(h.data(), dev, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(RL_ERR_CUDA, "device read failed");
    if (bytes && fwrite(h.data(), 1, bytes, fp) != bytes) return fail(RL_ERR_IO, "write failed");
    return RL_OK;
}

rl_status load(FILE *fp, void *dev, uint64_t bytes) {
    std::vector<uint8_t> h(bytes);
    if (bytes && fread(h.data(), 1, bytes, fp) != bytes) return fail(RL_ERR_IO, "truncated checkpoint");
    if (bytes && cudaMemcpy(dev, h.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(RL_ERR_CUDA, "device write failed");
    return RL_OK;
}

struct Blob {
    void *ptr;
    uint64_t bytes;
};

std::vector<Blob> forest_blobs(rl_forest *f) {
    const uint64_t L = f->n_leaves, M = f->p.m_max;
    std::vector<Blob> b = {
        {f->nodes, (uint64_t)f->p.n_trees * f->n_branch * sizeof(float4)},
        {f->res, L * f->p.kappa * sizeof(float4)},
        {f->res_count, L * 4},
        {f->nmodes, L},
        {f->centroid, L * sizeof(float4)},
        {f->mrgb, L * M * sizeof(uchar4)},
        {f->mU, L * M * 2 * sizeof(float4)},
        {f->msize, L * M * 4},
    };
    if (f->mpos_h) b.push_back({f->mpos_h, L * M * sizeof(ushort4)});
    if (f->mpos_f) b.push_back({f->mpos_f, L * M * sizeof(float4)});
    return b;
}
}  // namespace

extern "C" rl_status rl_forest_save(rl_forest *f, const char *path) {
    if (!f || !path) return fail(RL_ERR_INVALID_ARG, "null argument");
    RL_CK(cudaSetDevice(f->ctx->device));
    RL_CK(cudaDeviceSynchronize());
    FILE *fp = fopen(path, "wb");
    if (!fp) return fail(RL_ERR_IO, std::string("cannot open ") + path);
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "RLGBFRST", 8);
    h.version = 1;
    h.p = f->p;
    h.seed = f->seed;
    h.cursor = f->cursor;
    rl_status s = fwrite(&h, sizeof(h), 1, fp) == 1 ? RL_OK : fail(RL_ERR_IO, "write failed");
    for (const Blob &b : forest_blobs(f))
        if (s == RL_OK) s = dump(fp, b.ptr, b.bytes);
    if (fclose(fp) != 0 && s == RL_OK) s = fail(RL_ERR_IO, "close failed");
    return s;
}

extern "C" rl_status rl_forest_load(rl_ctx *ctx, const char *path, rl_forest **out) {
    if (!ctx || !path || !out) return fail(RL_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    RL_CK(cudaSetDevice(ctx->device));
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(RL_ERR_IO, std::string("cannot open ") + path);
    CkptHeader h;
    if (fread(&h, sizeof(h), 1, fp) != 1 || memcmp(h.magic, "RLGBFRST", 8) != 0 || h.version != 1) {
        fclose(fp);
        return fail(RL_ERR_IO, "not a relocgb forest checkpoint");
    }
    rl_forest *f = nullptr;
    rl_status s = forest_alloc(ctx, &h.p, h.seed, &f);
    if (s != RL_OK) {
        fclose(fp);
        return s;
    }
    for (const Blob &b : forest_blobs(f))
        if (s == RL_OK) s = load(fp, b.ptr, b.bytes);
    fclose(fp);
    if (s != RL_OK) {
        forest_release(f);
        delete f;
        return s;
    }
    f->cursor = h.cursor;
    *out = f;
    return RL_OK;
}

// ---------------------------------------------------------------------------
// Scene
// ---------------------------------------------------------------------------
extern "C" rl_status rl_scene_box(rl_ctx *ctx, const double lo[3], const double hi[3], rl_scene **out) {
    if (!ctx || !lo || !hi || !out) return fail(RL_ERR_INVALID_ARG, "null argument");
    for (int a = 0; a < 3; ++a)
        if (!(hi[a] > lo[a])) return fail(RL_ERR_INVALID_ARG, "box must have hi > lo");
    rl_scene *s = new rl_scene();
    s->ctx = ctx;
    for (int a = 0; a < 3; ++a) { s->lo[a] = lo[a]; s->hi[a] = hi[a]; }
    *out = s;
    return RL_OK;
}

extern "C" rl_status rl_scene_destroy(rl_scene *s) {
    if (!s) return fail(RL_ERR_INVALID_ARG, "null scene");
    delete s;
    return RL_OK;
}
