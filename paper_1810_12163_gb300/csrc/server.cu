// Serving loop: relocalisation requests from many camera streams, several
// rooms (models) and mixed resolutions, batched continuously on the GPU.
//
// Each model owns two relocaliser instances ("slots" of max_batch frames)
// and one worker thread.  While one instance's batch runs on the GPU the
// worker stages the next batch from everything that arrived meanwhile into
// the other; models run on separate streams, so their work overlaps on the
// device.  Requests are admitted against a byte budget of staged frame data;
// forests, modes and per-query RANSAC state stay resident in device memory.
// A frame's result does not depend on the batch it joins (every kernel works
// per frame with fixed-shape reductions).
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "internal.h"

namespace rl {
namespace {

using Clock = std::chrono::steady_clock;

double now_ms() {
    return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket;
    rl_intrinsics K;
    uint64_t seed;
    std::vector<float> depth;
    std::vector<uint8_t> rgb;
    uint64_t bytes;
    double t_submit;
};

struct Ticket {
    bool done = false;
    rl_status status = RL_OK;
    rl_result result{};
};

struct Slot {
    rl_reloc *r = nullptr;          // single relocaliser, or
    rl_cascade *c = nullptr;        // a cascade over `levels`
    std::vector<rl_reloc *> levels;
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    float *pin_depth = nullptr;     // pinned staging [max_batch][hw]
    uint8_t *pin_rgb = nullptr;
    std::vector<Request> batch;     // requests in flight
    bool busy = false;
};

struct Model {
    int id = 0;
    int max_w = 0, max_h = 0;
    Slot slot[2];
    std::deque<Request> queue;      // admitted, waiting for a slot
    std::thread worker;
};

}  // namespace
}  // namespace rl

struct rl_server {
    rl_ctx *ctx = nullptr;
    rl_server_params p{};
    std::vector<rl::Model *> models;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, rl::Ticket> tickets;
    std::deque<std::pair<int, rl::Request>> pending;  // over budget, waiting for admission
    uint64_t next_ticket = 1;
    uint64_t bytes_admitted = 0, peak_bytes = 0;
    uint64_t submitted = 0, completed = 0, refused = 0;
    std::vector<double> latencies;
    double t_first = -1.0, t_last = -1.0;
    bool stop = false;
};

namespace rl {
namespace {

// Moves pending requests into model queues while the byte budget allows.
void admit_locked(rl_server *s) {
    while (!s->pending.empty()) {
        auto &front = s->pending.front();
        if (s->bytes_admitted + front.second.bytes > s->p.memory_budget && s->bytes_admitted > 0) break;
        s->bytes_admitted += front.second.bytes;
        s->peak_bytes = std::max(s->peak_bytes, s->bytes_admitted);
        s->models[front.first]->queue.push_back(std::move(front.second));
        s->pending.pop_front();
    }
}

rl_status launch_slot(Model *m, Slot &sl) {
    const int hw = m->max_w * m->max_h;
    const int n = (int)sl.batch.size();
    std::vector<Frame> fr(n);
    for (int i = 0; i < n; ++i) {
        const Request &rq = sl.batch[i];
        const size_t px = (size_t)rq.K.width * rq.K.height;
        memcpy(sl.pin_depth + (size_t)hw * i, rq.depth.data(), px * sizeof(float));
        memcpy(sl.pin_rgb + (size_t)hw * 3 * i, rq.rgb.data(), px * 3);
        rl_reloc *owner = sl.c ? sl.c->levels.back() : sl.r;  // full-resolution inputs
        float *dd = owner->stage_depth + (size_t)hw * i;
        uint8_t *dc = owner->stage_rgb + (size_t)hw * 3 * i;
        RL_CK(cudaMemcpyAsync(dd, sl.pin_depth + (size_t)hw * i, px * sizeof(float), cudaMemcpyHostToDevice, sl.stream));
        RL_CK(cudaMemcpyAsync(dc, sl.pin_rgb + (size_t)hw * 3 * i, px * 3, cudaMemcpyHostToDevice, sl.stream));
        Frame &f = fr[i];
        f.depth = dd;
        f.rgb = dc;
        f.fx = rq.K.fx; f.fy = rq.K.fy; f.cx = rq.K.cx; f.cy = rq.K.cy;
        f.W = rq.K.width; f.H = rq.K.height;
        f.key0 = (uint32_t)rq.seed;
        f.key1 = (uint32_t)(rq.seed >> 32);
    }
    if (sl.c) {
        rl_reloc *top = sl.c->levels.back();
        for (int i = 0; i < n; ++i) top->host_frames[i] = fr[i];
        RL_TRY(cascade_enqueue_frames(sl.c, n, sl.stream));
    } else {
        RL_TRY(reloc_enqueue_frames(sl.r, n, fr.data(), sl.stream));
    }
    RL_CK(cudaEventRecord(sl.done_ev, sl.stream));
    sl.busy = true;
    return RL_OK;
}

void complete_slot(rl_server *s, Model *m, Slot &sl) {
    const int n = (int)sl.batch.size();
    std::vector<rl_result> res(n);
    const rl_status st = sl.c ? cascade_fetch_results(sl.c, n, sl.stream, res.data())
                              : reloc_fetch_results(sl.r, n, sl.stream, res.data());
    const double t = now_ms();
    std::lock_guard<std::mutex> g(s->mu);
    for (int i = 0; i < n; ++i) {
        Ticket &tk = s->tickets[sl.batch[i].ticket];
        tk.done = true;
        tk.status = st;
        tk.result = res[i];
        s->bytes_admitted -= sl.batch[i].bytes;
        if (st == RL_OK) {
            s->latencies.push_back(t - sl.batch[i].t_submit);
            ++s->completed;
        }
    }
    s->t_last = t;
    sl.batch.clear();
    sl.busy = false;
    admit_locked(s);
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    (void)m;
}

void worker(rl_server *s, Model *m) {
    cudaSetDevice(s->ctx->device);
    const int B = s->p.max_batch;
    uint64_t seq = 0, slot_seq[2] = {0, 0};
    while (true) {
        int to_launch = -1;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            const bool any_busy = m->slot[0].busy || m->slot[1].busy;
            if (!any_busy) s->cv_work.wait(lk, [&] { return s->stop || !m->queue.empty(); });
            if (s->stop && m->queue.empty() && !any_busy) return;
            const int free_slot = !m->slot[0].busy ? 0 : (!m->slot[1].busy ? 1 : -1);
            if (free_slot >= 0 && !m->queue.empty()) {
                Slot &sl = m->slot[free_slot];
                while (!m->queue.empty() && (int)sl.batch.size() < B) {
                    sl.batch.push_back(std::move(m->queue.front()));
                    m->queue.pop_front();
                }
                to_launch = free_slot;
            }
        }
        if (to_launch >= 0) {
            Slot &sl = m->slot[to_launch];
            if (launch_slot(m, sl) != RL_OK) {
                std::lock_guard<std::mutex> g(s->mu);
                for (auto &rq : sl.batch) {
                    Ticket &tk = s->tickets[rq.ticket];
                    tk.done = true;
                    tk.status = RL_ERR_CUDA;
                    s->bytes_admitted -= rq.bytes;
                }
                sl.batch.clear();
                sl.busy = false;
                s->cv_done.notify_all();
            } else {
                slot_seq[to_launch] = ++seq;
            }
            continue;  // stage more while a slot is free
        }
        int oldest = -1;
        for (int k = 0; k < 2; ++k)
            if (m->slot[k].busy && (oldest < 0 || slot_seq[k] < slot_seq[oldest])) oldest = k;
        if (oldest < 0) continue;
        Slot &sl = m->slot[oldest];
        if (cudaEventQuery(sl.done_ev) == cudaSuccess) {
            complete_slot(s, m, sl);
        } else if (m->slot[0].busy && m->slot[1].busy) {
            cudaEventSynchronize(sl.done_ev);  // no free slot to stage into
            complete_slot(s, m, sl);
        } else {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait_for(lk, std::chrono::microseconds(200),
                                [&] { return s->stop || !m->queue.empty(); });
        }
    }
}

}  // namespace
}  // namespace rl

using namespace rl;

extern "C" rl_status rl_server_create(rl_ctx *ctx, const rl_server_params *p, rl_server **out) {
    if (!ctx || !p || !out) return fail(RL_ERR_INVALID_ARG, "null argument");
    if (p->max_batch < 1 || p->max_batch > 1024) return fail(RL_ERR_INVALID_ARG, "max_batch must be 1..1024");
    if (p->memory_budget == 0) return fail(RL_ERR_INVALID_ARG, "memory_budget must be > 0");
    rl_server *s = new rl_server();
    s->ctx = ctx;
    s->p = *p;
    *out = s;
    return RL_OK;
}

namespace rl {
namespace {

struct CascadeSpec {
    const rl_ransac_params *levels;
    const int32_t *subsample;
    const double *thresholds;
    int n;
};

void release_slot(Slot &sl) {
    if (sl.c) rl_cascade_destroy(sl.c);
    for (rl_reloc *r : sl.levels) rl_reloc_destroy(r);
    if (sl.r) rl_reloc_destroy(sl.r);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done_ev) cudaEventDestroy(sl.done_ev);
    if (sl.pin_depth) cudaFreeHost(sl.pin_depth);
    if (sl.pin_rgb) cudaFreeHost(sl.pin_rgb);
    sl = Slot();
}

// Two slots (relocaliser or cascade, stream, event, pinned staging) and the
// model's worker thread.
rl_status add_model(rl_server *s, rl_forest *f, rl_scene *scene, const rl_ransac_params *rp,
                    const CascadeSpec *cs, int32_t max_w, int32_t max_h, int32_t *model_id) {
    RL_CK(cudaSetDevice(s->ctx->device));
    Model *m = new Model();
    m->max_w = max_w;
    m->max_h = max_h;
    const size_t hw = (size_t)max_w * max_h;
    const int B = s->p.max_batch;
    rl_status st = RL_OK;
    for (int k = 0; k < 2 && st == RL_OK; ++k) {
        Slot &sl = m->slot[k];
        if (!cs) {
            st = rl_reloc_create(f, scene, rp, max_w, max_h, B, &sl.r);
        } else {
            for (int l = 0; l < cs->n && st == RL_OK; ++l) {
                const int sf = cs->subsample[l];
                rl_reloc *r = nullptr;
                st = rl_reloc_create(f, scene, &cs->levels[l], (max_w + sf - 1) / sf, (max_h + sf - 1) / sf, B, &r);
                if (st == RL_OK) sl.levels.push_back(r);
            }
            if (st == RL_OK)
                st = rl_cascade_create(sl.levels.data(), cs->thresholds, cs->subsample, cs->n, &sl.c);
        }
        if (st == RL_OK && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess)
            st = fail(RL_ERR_CUDA, "stream creation failed");
        if (st == RL_OK && cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming) != cudaSuccess)
            st = fail(RL_ERR_CUDA, "event creation failed");
        if (st == RL_OK && cudaMallocHost(&sl.pin_depth, hw * B * sizeof(float)) != cudaSuccess)
            st = fail(RL_ERR_CUDA, "pinned allocation failed");
        if (st == RL_OK && cudaMallocHost(&sl.pin_rgb, hw * 3 * B) != cudaSuccess)
            st = fail(RL_ERR_CUDA, "pinned allocation failed");
    }
    if (st != RL_OK) {
        for (auto &sl : m->slot) release_slot(sl);
        delete m;
        return st;
    }
    std::lock_guard<std::mutex> g(s->mu);
    m->id = (int)s->models.size();
    s->models.push_back(m);
    m->worker = std::thread(worker, s, m);
    *model_id = m->id;
    return RL_OK;
}

}  // namespace
}  // namespace rl

extern "C" rl_status rl_server_add_model(rl_server *s, rl_forest *f, rl_scene *scene,
                                         const rl_ransac_params *rp, int32_t max_w, int32_t max_h,
                                         int32_t *model_id) {
    if (!s || !f || !rp || !model_id) return fail(RL_ERR_INVALID_ARG, "null argument");
    return add_model(s, f, scene, rp, nullptr, max_w, max_h, model_id);
}

extern "C" rl_status rl_server_add_cascade_model(rl_server *s, rl_forest *f, rl_scene *scene,
                                                 const rl_ransac_params *levels, const int32_t *subsample,
                                                 const double *thresholds, int32_t n_levels, int32_t max_w,
                                                 int32_t max_h, int32_t *model_id) {
    if (!s || !f || !levels || !subsample || !model_id || (n_levels > 1 && !thresholds))
        return fail(RL_ERR_INVALID_ARG, "null argument");
    if (n_levels < 1 || n_levels > 8) return fail(RL_ERR_INVALID_ARG, "n_levels must be 1..8");
    if (subsample[n_levels - 1] != 1) return fail(RL_ERR_INVALID_ARG, "the last level must run at full resolution");
    const CascadeSpec cs{levels, subsample, thresholds, n_levels};
    return add_model(s, f, scene, nullptr, &cs, max_w, max_h, model_id);
}

extern "C" rl_status rl_server_submit(rl_server *s, int32_t model, const float *depth, const uint8_t *rgb,
                                      const rl_intrinsics *K, uint64_t seed, uint64_t *ticket) {
    if (!s || !depth || !rgb || !K || !ticket) return fail(RL_ERR_INVALID_ARG, "null argument");
    if (model < 0 || model >= (int)s->models.size()) return fail(RL_ERR_INVALID_ARG, "unknown model");
    Model *m = s->models[model];
    if (K->width < 1 || K->height < 1 || K->width > m->max_w || K->height > m->max_h || !(K->fx > 0) || !(K->fy > 0))
        return fail(RL_ERR_INVALID_ARG, "frame size or intrinsics not accepted by this model");
    Request rq;
    rq.K = *K;
    rq.seed = seed;
    const size_t px = (size_t)K->width * K->height;
    rq.bytes = px * (sizeof(float) + 3);
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop) return fail(RL_ERR_INVALID_ARG, "server is shutting down");
    const bool fits = s->bytes_admitted + rq.bytes <= s->p.memory_budget || s->bytes_admitted == 0;
    if (!fits && !s->p.queue_when_full) {
        ++s->refused;
        return fail(RL_ERR_ADMISSION, "request refused: device memory budget exhausted");
    }
    rq.ticket = s->next_ticket++;
    lk.unlock();
    rq.depth.assign(depth, depth + px);
    rq.rgb.assign(rgb, rgb + px * 3);
    rq.t_submit = now_ms();
    lk.lock();
    *ticket = rq.ticket;
    s->tickets[rq.ticket] = Ticket{};
    ++s->submitted;
    if (s->t_first < 0) s->t_first = rq.t_submit;
    s->pending.emplace_back(model, std::move(rq));
    admit_locked(s);
    s->cv_work.notify_all();
    return RL_OK;
}

extern "C" rl_status rl_server_poll(rl_server *s, uint64_t ticket, int32_t *done, rl_result *out) {
    if (!s || !done) return fail(RL_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(RL_ERR_INVALID_ARG, "unknown ticket");
    *done = it->second.done ? 1 : 0;
    if (!it->second.done) return RL_OK;
    const rl_status st = it->second.status;
    if (out) *out = it->second.result;
    s->tickets.erase(it);
    if (st != RL_OK) return fail(st, "request failed on the device");
    return RL_OK;
}

extern "C" rl_status rl_server_wait(rl_server *s, uint64_t ticket, uint32_t timeout_ms, rl_result *out) {
    if (!s) return fail(RL_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(RL_ERR_INVALID_ARG, "unknown ticket");
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        auto jt = s->tickets.find(ticket);
        return jt != s->tickets.end() && jt->second.done;
    });
    if (!ok) return fail(RL_ERR_TIMEOUT, "request not finished within the timeout");
    it = s->tickets.find(ticket);
    const rl_status st = it->second.status;
    if (out) *out = it->second.result;
    s->tickets.erase(it);
    if (st != RL_OK) return fail(st, "request failed on the device");
    return RL_OK;
}

extern "C" rl_status rl_server_get_stats(rl_server *s, rl_server_stats *out) {
    if (!s || !out) return fail(RL_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> g(s->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->refused = s->refused;
    out->peak_admitted_bytes = s->peak_bytes;
    std::vector<double> l = s->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) { return l[std::min(l.size() - 1, (size_t)(q * (l.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.5);
        out->p99_ms = pct(0.99);
        double sum = 0.0;
        for (double v : l) sum += v;
        out->mean_ms = sum / l.size();
        if (s->t_last > s->t_first) out->frames_per_s = 1000.0 * l.size() / (s->t_last - s->t_first);
    }
    return RL_OK;
}

extern "C" rl_status rl_server_reset_stats(rl_server *s) {
    if (!s) return fail(RL_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> g(s->mu);
    s->submitted = s->completed = s->refused = 0;
    s->peak_bytes = s->bytes_admitted;
    s->latencies.clear();
    s->t_first = s->t_last = -1.0;
    return RL_OK;
}

extern "C" rl_status rl_server_destroy(rl_server *s) {
    if (!s) return fail(RL_ERR_INVALID_ARG, "null server");
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (Model *m : s->models)
        if (m->worker.joinable()) m->worker.join();
    cudaSetDevice(s->ctx->device);
    for (Model *m : s->models) {
        for (auto &sl : m->slot) {
            if (sl.stream) cudaStreamSynchronize(sl.stream);
            release_slot(sl);
        }
        delete m;
    }
    delete s;
    return RL_OK;
}
