// Depth-raycast ranking score (Eq. 6-7) of given poses, with no device
// allocation at all: the per-tile partial sums live in a fixed array that is
// part of the library image on every GPU that loads it.
//
// Who needs this: callers that cannot call cudaMalloc -- a real-time loop
// whose device memory is fixed when it starts, a host framework that owns
// every byte of device memory and forbids other allocators, or code that
// must never trigger the implicit device-wide synchronisation that
// cudaMalloc / cudaFree can cause.  Such callers pass device inputs and
// device outputs; everything else the kernel needs is already resident.
#include <math.h>
#include <stdio.h>

#include <cuda.h>

#include <mutex>

#include "internal.h"

namespace rl {
namespace {

// One partial record per (pose, 1024-pixel tile): FP64 sum of |D_l - D_s|,
// count of valid synthetic pixels, count valid in both.
struct Partial {
    double sum;
    int32_t syn, both;
};

constexpr int kTilePixels = 1024;             // 256 threads x 4 pixels
constexpr int kMaxPartials = 65536;           // 65536 x 16 B = 1 MiB per device
constexpr int kMaxPoses = 65535;              // poses run on the grid's y dimension

// The scratch itself.  Every GPU that loads the library holds these 1 MiB
// until the process exits.  Calls share it: a call overwrites what the last
// call left, and two calls that overlap on the GPU (different streams, no
// ordering between them) race on it.
static __device__ __align__(256) Partial g_score_scratch[kMaxPartials];

// Device address of g_score_scratch per device, looked up with that device
// current (host code may not use the symbol's own name as a device address).
// The address belongs to the CUDA context it was looked up in, so each
// entry remembers that context and is looked up again when the device's
// current context is another one (after cudaDeviceReset, or when the primary
// context was released and created anew).
constexpr int kMaxDevices = 64;
struct ScratchEntry {
    CUcontext ctx;
    Partial *ptr;
};
ScratchEntry g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mu;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);

// cuCtxGetCurrent through the runtime's driver entry-point query, so the
// library needs no link against the driver library; null if unavailable.
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(f);
    }();
    return fn;
}

CUcontext current_context() {
    CUcontext c = nullptr;
    if (CtxGetCurrentFn f = ctx_get_current())
        if (f(&c) != CUDA_SUCCESS) c = nullptr;
    return c;
}

rl_status scratch_for_current_device(Partial **out) {
    int dev = -1;
    RL_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(RL_ERR_INVALID_ARG, "device index beyond 63");
    std::lock_guard<std::mutex> g(g_scratch_mu);
    ScratchEntry &e = g_scratch[dev];
    const CUcontext now = current_context();
    if (!e.ptr || (now && now != e.ctx)) {
        void *p = nullptr;
        cudaError_t err = cudaGetSymbolAddress(&p, g_score_scratch);
        if (err != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress(g_score_scratch)", __FILE__, __LINE__);
        e.ptr = static_cast<Partial *>(p);
        e.ctx = current_context();  // the lookup made the device's context current if it was not
    }
    *out = e.ptr;
    return RL_OK;
}

struct StaticArgs {
    const float *depth;
    const double *poses;  // [n][16] row-major camera->world
    float fx, fy, cx, cy;
    int W, H, n, tiles;
    float lo[3], hi[3];
    double lo64[3], hi64[3];
    Partial *part;        // [n][tiles]
};

__device__ bool ray_hit64(const double *P, int u, int v, const StaticArgs &a, double *depth) {
    const double dc0 = ((double)u - (double)a.cx) / (double)a.fx;
    const double dc1 = ((double)v - (double)a.cy) / (double)a.fy;
    double tn = -INFINITY, tf = INFINITY;
    for (int ax = 0; ax < 3; ++ax) {
        const double d = P[4 * ax] * dc0 + P[4 * ax + 1] * dc1 + P[4 * ax + 2];
        const double o = P[4 * ax + 3];
        if (d == 0.0) {
            if (o < a.lo64[ax] || o > a.hi64[ax]) return false;
            continue;
        }
        const double t1 = (a.lo64[ax] - o) / d, t2 = (a.hi64[ax] - o) / d;
        tn = fmax(tn, fmin(t1, t2));
        tf = fmin(tf, fmax(t1, t2));
    }
    if (tn > tf) return false;
    if (tn > 0.0) { *depth = tn; return true; }
    if (tf > 0.0) { *depth = tf; return true; }
    return false;
}

// Same arithmetic as the relocaliser's ranking kernel: FP32 slab test,
// FP64 re-evaluation of rays within a 1e-4 relative margin of their
// hit/miss decision.
__device__ void ray_term(const double *P, int p, const StaticArgs &a, float *sum, int *syn, int *both) {
    const int u = p % a.W, v = p / a.W;
    const float dc0 = ((float)u - a.cx) / a.fx, dc1 = ((float)v - a.cy) / a.fy;
    float d[3], o[3];
    for (int r = 0; r < 3; ++r) {
        d[r] = fmaf((float)P[4 * r], dc0, fmaf((float)P[4 * r + 1], dc1, (float)P[4 * r + 2]));
        o[r] = (float)P[4 * r + 3];
    }
    const float dn = fabsf(d[0]) + fabsf(d[1]) + fabsf(d[2]);
    float tn = -INFINITY, tf = INFINITY;
    bool ok = true, unsure = false;
    for (int ax = 0; ax < 3; ++ax) {
        if (fabsf(d[ax]) <= 1e-5f * dn) {
            unsure = true;
            continue;
        }
        const float inv = 1.0f / d[ax];
        const float ta = (a.lo[ax] - o[ax]) * inv, tb = (a.hi[ax] - o[ax]) * inv;
        tn = fmaxf(tn, fminf(ta, tb));
        tf = fminf(tf, fmaxf(ta, tb));
    }
    float depth = 0.f;
    if (!unsure) {
        const float scale = fmaxf(fabsf(tn), fabsf(tf));
        if (fabsf(tf - tn) <= 1e-4f * scale || fabsf(tn) <= 1e-4f * scale || fabsf(tf) <= 1e-4f * scale)
            unsure = true;
    }
    if (unsure) {
        double dd;
        ok = ray_hit64(P, u, v, a, &dd);
        depth = (float)dd;
    } else if (tn <= tf && tn > 0.f) {
        depth = tn;
    } else if (tn <= tf && tf > 0.f) {
        depth = tf;
    } else {
        ok = false;
    }
    if (!ok) return;
    *syn += 1;
    const float dl = a.depth[p];
    if (dl > 0.f) {
        *both += 1;
        *sum += fabsf(dl - depth);
    }
}

__global__ void __launch_bounds__(256) k_score_static(StaticArgs a) {
    __shared__ float s_sum[8];
    __shared__ int s_syn[8], s_both[8];
    const int c = blockIdx.y;
    const double *P = a.poses + (size_t)c * 16;
    float sum = 0.f;
    int syn = 0, both = 0;
    const int base = blockIdx.x * kTilePixels;
    for (int k = 0; k < kTilePixels / 256; ++k) {
        const int p = base + k * 256 + threadIdx.x;
        if (p < a.W * a.H) ray_term(P, p, a, &sum, &syn, &both);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        syn += __shfl_down_sync(0xffffffffu, syn, o);
        both += __shfl_down_sync(0xffffffffu, both, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_sum[w] = sum;
        s_syn[w] = syn;
        s_both[w] = both;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Partial r{0.0, 0, 0};
        for (int k = 0; k < 8; ++k) {
            r.sum += (double)s_sum[k];
            r.syn += s_syn[k];
            r.both += s_both[k];
        }
        a.part[(size_t)c * a.tiles + blockIdx.x] = r;  // every record read below is written here
    }
}

__global__ void k_score_static_final(StaticArgs a, float *scores, float *valid_frac) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.n) return;
    double sum = 0.0;
    long syn = 0, both = 0;
    for (int t = 0; t < a.tiles; ++t) {
        const Partial r = a.part[(size_t)c * a.tiles + t];
        sum += r.sum;
        syn += r.syn;
        both += r.both;
    }
    const double frac = (double)syn / ((double)a.W * (double)a.H);
    scores[c] = (frac >= 0.1 && both > 0) ? (float)(sum / (double)both) : INFINITY;
    if (valid_frac) valid_frac[c] = (float)frac;
}

}  // namespace
}  // namespace rl

using namespace rl;

extern "C" rl_status rl_score_poses_noalloc(const double box_lo[3], const double box_hi[3],
                                            const float *depth, const rl_intrinsics *K,
                                            const double *poses, int32_t n, void *stream,
                                            float *scores, float *valid_frac) {
    if (!box_lo || !box_hi || !depth || !K || !poses || !scores)
        return fail(RL_ERR_INVALID_ARG, "null argument");
    for (int ax = 0; ax < 3; ++ax)
        if (!(box_hi[ax] > box_lo[ax])) return fail(RL_ERR_INVALID_ARG, "box must have hi > lo");
    if (K->width < 1 || K->height < 1 || K->width > 8192 || K->height > 8192 || !(K->fx > 0) || !(K->fy > 0))
        return fail(RL_ERR_INVALID_ARG, "bad intrinsics");
    if (n < 1) return fail(RL_ERR_INVALID_ARG, "n must be >= 1");
    if (n > kMaxPoses) {
        char buf[128];
        snprintf(buf, sizeof(buf), "n = %d exceeds the limit of %d poses per call", n, kMaxPoses);
        return fail(RL_ERR_INVALID_ARG, buf);
    }
    const int64_t tiles = ((int64_t)K->width * K->height + kTilePixels - 1) / kTilePixels;
    if ((int64_t)n * tiles > kMaxPartials) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "n * ceil(W*H / %d) = %lld exceeds the fixed scratch of %d records; "
                 "score at most %lld poses of this size per call",
                 kTilePixels, (long long)(n * tiles), kMaxPartials, (long long)(kMaxPartials / tiles));
        return fail(RL_ERR_INVALID_ARG, buf);
    }
    Partial *part = nullptr;
    RL_TRY(scratch_for_current_device(&part));
    StaticArgs a;
    a.depth = depth;
    a.poses = poses;
    a.fx = K->fx; a.fy = K->fy; a.cx = K->cx; a.cy = K->cy;
    a.W = K->width; a.H = K->height; a.n = n; a.tiles = (int)tiles;
    for (int ax = 0; ax < 3; ++ax) {
        a.lo[ax] = (float)box_lo[ax];
        a.hi[ax] = (float)box_hi[ax];
        a.lo64[ax] = box_lo[ax];
        a.hi64[ax] = box_hi[ax];
    }
    a.part = part;
    cudaStream_t s = (cudaStream_t)stream;
    k_score_static<<<dim3((unsigned)tiles, (unsigned)n), 256, 0, s>>>(a);
    RL_LAUNCH_CK();
    k_score_static_final<<<(n + 63) / 64, 64, 0, s>>>(a, scores, valid_frac);
    RL_LAUNCH_CK();
    return RL_OK;
}
