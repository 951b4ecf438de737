"""relocgb: GB300-native RGB-D camera relocalisation (Cavallari et al.,
TPAMI 2019) -- Python layer over the C ABI of librelocgb.

The relocaliser runs entirely in the CUDA library; this module marshals
arguments, owns the device arena (a PyTorch tensor) and picks streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding, presets  # noqa: F401
from .binding import RL_N_KERNELS as N_KERNELS
from .binding import RL_N_WORK as N_WORK
from .binding import (RL_DEVICE, RL_HOST, RL_NO_POSE, RL_POSE_FOUND,  # noqa: F401
                      ForestParams, IcpParams, Intrinsics, RansacParams, RelocError, Result, call, lib)

__all__ = ["Context", "Forest", "Scene", "Relocaliser", "Cascade", "intrinsics", "presets",
           "RelocError", "lib"]


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    if stream is None:
        return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def intrinsics(K) -> Intrinsics:
    if isinstance(K, Intrinsics):
        return K
    return Intrinsics(float(K.fx), float(K.fy), float(K.cx), float(K.cy), int(K.width), int(K.height))


def _struct(cls, d: dict):
    s = cls()
    names = {f[0] for f in cls._fields_}
    for k, v in d.items():
        if k in names:
            setattr(s, k, v)
    return s


def icp_struct(d: dict) -> IcpParams:
    """rl_icp_params from icp_* keys (missing keys take presets.ICP_DEFAULT)."""
    d = dict(presets.ICP_DEFAULT, **{k: v for k, v in d.items() if k.startswith("icp_")})
    ip = IcpParams()
    ip.levels = int(d["icp_levels"])
    for l in range(3):
        ip.stride[l] = int(d["icp_stride"][l]) if l < len(d["icp_stride"]) else 1
        ip.iters[l] = int(d["icp_iters"][l]) if l < len(d["icp_iters"]) else 1
        ip.dist[l] = float(d["icp_dist"][l]) if l < len(d["icp_dist"]) else 1.0
    ip.min_frac = float(d["icp_min_frac"])
    ip.ridge = float(d["icp_ridge"])
    return ip


def ransac_struct(d: dict) -> RansacParams:
    s = _struct(RansacParams, {k: v for k, v in d.items() if not k.startswith("icp_")})
    s.icp_p = icp_struct(d)
    return s


class _Image:
    """Pointer + memory kind of an image argument (numpy = host, torch = device)."""

    def __init__(self, a, dtype):
        torch = _torch()
        if isinstance(a, torch.Tensor):
            if not a.is_cuda:
                a = a.numpy()
            else:
                if a.dtype != {np.float32: torch.float32, np.uint8: torch.uint8}[dtype]:
                    raise TypeError(f"expected {dtype} tensor")
                self.keep = a.contiguous()
                self.ptr = ctypes.c_void_p(self.keep.data_ptr())
                self.mem = RL_DEVICE
                return
        self.keep = np.ascontiguousarray(a, dtype=dtype)
        self.ptr = self.keep.ctypes.data_as(ctypes.c_void_p)
        self.mem = RL_HOST


class Context:
    """Device context over a caller-owned arena (a uint8 CUDA tensor)."""

    def __init__(self, device: int = 0, arena_bytes: int = 4 << 30):
        torch = _torch()
        lib()
        self.device = device
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=f"cuda:{device}")
        self.h = ctypes.c_void_p()
        call("rl_context_create", device, ctypes.c_void_p(self.arena.data_ptr()), arena_bytes,
             ctypes.byref(self.h))

    def usage(self):
        used, peak = ctypes.c_uint64(), ctypes.c_uint64()
        call("rl_context_usage", self.h, ctypes.byref(used), ctypes.byref(peak))
        return used.value, peak.value

    def close(self):
        if self.h:
            call("rl_context_destroy", self.h)
            self.h = ctypes.c_void_p()


class Forest:
    def __init__(self, ctx: Context, handle, params: dict):
        self.ctx = ctx
        self.h = handle
        self.params = dict(params)
        self.n_trees = params["n_trees"]
        self.depth = params["depth"]
        self.n_leaves = self.n_trees << self.depth

    @classmethod
    def random(cls, ctx: Context, params: dict, seed: int):
        full = dict(presets.FOREST_DEFAULT, **params)
        h = ctypes.c_void_p()
        call("rl_forest_create_random", ctx.h, ctypes.byref(_struct(ForestParams, full)), seed,
             ctypes.byref(h))
        return cls(ctx, h, full)

    @classmethod
    def load(cls, ctx: Context, path: str, params: dict):
        h = ctypes.c_void_p()
        call("rl_forest_load", ctx.h, path.encode(), ctypes.byref(h))
        return cls(ctx, h, params)

    def save(self, path: str):
        call("rl_forest_save", self.h, path.encode())

    def reset_leaves(self, stream=None):
        call("rl_forest_reset_leaves", self.h, _stream_ptr(stream))

    def adapt(self, depth, rgb, K, cam_to_world, stream=None):
        d = _Image(depth, np.float32)
        c = _Image(rgb, np.uint8)
        if d.mem != c.mem:
            raise ValueError("depth and colour must live in the same memory")
        T = np.ascontiguousarray(np.asarray(cam_to_world, np.float64).reshape(16))
        Ki = intrinsics(K)
        call("rl_forest_adapt", self.h, d.ptr, c.ptr, ctypes.byref(Ki),
             T.ctypes.data_as(ctypes.c_void_p), d.mem, _stream_ptr(stream))

    def update_modes(self, n_leaves: int = -1, stream=None):
        call("rl_forest_update_modes", self.h, n_leaves, _stream_ptr(stream))

    def set_streaming(self, enable: bool = True):
        """Double-buffered modes: relocalisation reads a complete snapshot
        while update_modes re-clusters leaves on another stream (call before
        creating relocalisers of this forest)."""
        call("rl_forest_set_streaming", self.h, int(enable))

    def leaves(self, depth, rgb, K, n_trees=None, stream=None):
        torch = _torch()
        Ki = intrinsics(K)
        T = self.n_trees if n_trees is None else n_trees
        out = torch.empty((T, Ki.height, Ki.width), dtype=torch.int16, device=f"cuda:{self.ctx.device}")
        d = _Image(depth, np.float32)
        c = _Image(rgb, np.uint8)
        call("rl_forest_leaves", self.h, d.ptr, c.ptr, ctypes.byref(Ki), T,
             ctypes.c_void_p(out.data_ptr()), d.mem, _stream_ptr(stream))
        return out.cpu().numpy().view(np.uint16)

    def export(self, reservoirs=False):
        p = self.params
        NB = self.n_trees * ((1 << self.depth) - 1)
        L, M, K = self.n_leaves, p["m_max"], p["kappa"]
        out = dict(dx=np.zeros(NB, np.float32), dy=np.zeros(NB, np.float32),
                   tau=np.zeros(NB, np.float32), meta=np.zeros(NB, np.int32),
                   res_count=np.zeros(L, np.uint32), nmodes=np.zeros(L, np.uint8),
                   mode_pos=np.zeros((L, M, 3), np.float32), mode_rgb=np.zeros((L, M, 3), np.uint8),
                   mode_U=np.zeros((L, M, 6), np.float32), mode_size=np.zeros((L, M), np.int32))
        if reservoirs:
            out["res_pos"] = np.zeros((L, K, 3), np.float32)
            out["res_rgb"] = np.zeros((L, K, 3), np.uint8)
        ptr = lambda k: out[k].ctypes.data_as(ctypes.c_void_p) if k in out else None
        call("rl_forest_export", self.h, ptr("dx"), ptr("dy"), ptr("tau"), ptr("meta"),
             ptr("res_pos"), ptr("res_rgb"), ptr("res_count"), ptr("nmodes"), ptr("mode_pos"),
             ptr("mode_rgb"), ptr("mode_U"), ptr("mode_size"))
        out["type"] = (out["meta"] & 255).astype(np.uint8)
        out["channel"] = (out["meta"] >> 8).astype(np.uint8)
        return out

    def set_mode_positions(self, mode_pos):
        """Overwrites the stored modes' positions ([L][m_max][3] FP32), re-encoded
        in the forest's precision (see rl_forest_set_mode_positions)."""
        pos = np.ascontiguousarray(mode_pos, np.float32)
        if pos.shape != (self.n_leaves, self.params["m_max"], 3):
            raise ValueError(f"mode_pos must have shape {(self.n_leaves, self.params['m_max'], 3)}")
        call("rl_forest_set_mode_positions", self.h, pos.ctypes.data_as(ctypes.c_void_p))

    def close(self):
        if self.h:
            call("rl_forest_destroy", self.h)
            self.h = ctypes.c_void_p()


class Scene:
    def __init__(self, ctx: Context, lo, hi):
        lo = np.ascontiguousarray(lo, np.float64)
        hi = np.ascontiguousarray(hi, np.float64)
        self.h = ctypes.c_void_p()
        call("rl_scene_box", ctx.h, lo.ctypes.data_as(ctypes.c_void_p),
             hi.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self.h))

    def score_poses(self, depth, K, poses, stream=None):
        """Eq. 6-7 scores of the given camera->world poses against `depth`."""
        d = _Image(depth, np.float32)
        P = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(-1, 16))
        n = P.shape[0]
        scores = np.zeros(n, np.float32)
        frac = np.zeros(n, np.float32)
        call("rl_score_poses", self.h, d.ptr, ctypes.byref(intrinsics(K)),
             P.ctypes.data_as(ctypes.c_void_p), n, d.mem, _stream_ptr(stream),
             scores.ctypes.data_as(ctypes.c_void_p), frac.ctypes.data_as(ctypes.c_void_p))
        return scores, frac

    def icp_poses(self, depth, K, poses, stream=None, **icp):
        """ICP (Sec. 3.2.4) of the given camera->world poses against `depth`
        and the box: (refined [n][4][4], ok [n] bool, inlier fraction [n]).
        Keyword arguments: icp_levels, icp_stride, icp_iters, icp_dist,
        icp_min_frac, icp_ridge (defaults: presets.ICP_DEFAULT)."""
        d = _Image(depth, np.float32)
        P = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(-1, 16))
        n = P.shape[0]
        out = np.zeros((n, 16), np.float64)
        ok = np.zeros(n, np.int32)
        frac = np.zeros(n, np.float32)
        ip = icp_struct(icp)
        call("rl_icp_poses", self.h, d.ptr, ctypes.byref(intrinsics(K)),
             P.ctypes.data_as(ctypes.c_void_p), n, ctypes.byref(ip), d.mem, _stream_ptr(stream),
             out.ctypes.data_as(ctypes.c_void_p), ok.ctypes.data_as(ctypes.c_void_p),
             frac.ctypes.data_as(ctypes.c_void_p))
        return out.reshape(n, 4, 4), ok.astype(bool), frac

    def close(self):
        if self.h:
            call("rl_scene_destroy", self.h)
            self.h = ctypes.c_void_p()


def result_dict(r: Result) -> dict:
    nc = max(0, r.n_chosen)
    return dict(
        pose=np.array(r.pose).reshape(4, 4), energy=r.energy, energy_per_pixel=r.energy_per_pixel,
        score=r.score, level=r.level, n_hypotheses=r.n_hypotheses, n_chosen=r.n_chosen,
        n_pixels=r.n_pixels, status=r.status, best=r.best,
        chosen_pose=np.array([np.array(r.chosen_pose[i]).reshape(4, 4) for i in range(nc)]),
        chosen_energy=np.array(r.chosen_energy[:nc]), chosen_score=np.array(r.chosen_score[:nc]),
        chosen_slot=np.array(r.chosen_slot[:nc]), icp_mask=r.icp_mask,
        chosen_icp_frac=np.array(r.chosen_icp_frac[:max(nc, 1)]),
    )


class Relocaliser:
    def __init__(self, forest: Forest, scene: Scene | None, params: dict, max_w: int, max_h: int,
                 max_batch: int = 1):
        self.forest = forest
        self.params = dict(presets.DEFAULT, **params)
        self.max_batch = max_batch
        self.h = ctypes.c_void_p()
        call("rl_reloc_create", forest.h, scene.h if scene else None,
             ctypes.byref(ransac_struct(self.params)), max_w, max_h, max_batch,
             ctypes.byref(self.h))

    def relocalise_batch(self, depth, rgb, K, seeds, stream=None, raw=False):
        d = _Image(depth, np.float32)
        c = _Image(rgb, np.uint8)
        seeds = np.ascontiguousarray(seeds, np.uint64)
        n = len(seeds)
        out = (Result * n)()
        call("rl_relocalise_batch", self.h, n, d.ptr, c.ptr, ctypes.byref(intrinsics(K)),
             seeds.ctypes.data_as(ctypes.c_void_p), d.mem, _stream_ptr(stream), out)
        return out if raw else [result_dict(out[i]) for i in range(n)]

    def relocalise(self, depth, rgb, K, seed, stream=None):
        return self.relocalise_batch(depth, rgb, K, [seed], stream)[0]

    def relocalise_batch_async(self, depth, rgb, K, seeds, stream=None):
        """Enqueues a batch (inputs in device memory) and returns at once;
        fetch() waits for the stream and returns the results."""
        d = _Image(depth, np.float32)
        c = _Image(rgb, np.uint8)
        if d.mem != RL_DEVICE or c.mem != RL_DEVICE:
            raise ValueError("relocalise_batch_async takes device tensors")
        seeds = np.ascontiguousarray(seeds, np.uint64)
        call("rl_relocalise_batch_async", self.h, len(seeds), d.ptr, c.ptr, ctypes.byref(intrinsics(K)),
             seeds.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream))
        self._pending = len(seeds)

    def fetch(self, stream=None, raw=False):
        n = self._pending
        out = (Result * n)()
        call("rl_reloc_fetch", self.h, n, _stream_ptr(stream), out)
        return out if raw else [result_dict(out[i]) for i in range(n)]

    @property
    def tuning(self) -> dict:
        """Launch shapes in use (they never change a result)."""
        t = binding.Tuning()
        call("rl_reloc_get_tuning", self.h, ctypes.byref(t))
        return {f: getattr(t, f) for f, _ in binding.Tuning._fields_}

    def set_tuning(self, tuning: dict):
        t = binding.Tuning(**dict(self.tuning, **tuning))
        call("rl_reloc_set_tuning", self.h, ctypes.byref(t))

    def tuning_key(self) -> str:
        buf = ctypes.create_string_buffer(512)
        call("rl_tuning_key", self.h, buf, 512)
        return buf.value.decode()

    def autotune(self, depth, rgb, K, seeds, cache_path=None, stream=None) -> dict:
        """Times the candidate launch shapes on these frames (or takes them from
        cache_path) and applies the fastest; returns the tuning in use."""
        d = _Image(depth, np.float32)
        c = _Image(rgb, np.uint8)
        seeds = np.ascontiguousarray(seeds, np.uint64)
        t = binding.Tuning()
        call("rl_reloc_autotune", self.h, len(seeds), d.ptr, c.ptr, ctypes.byref(intrinsics(K)),
             seeds.ctypes.data_as(ctypes.c_void_p), d.mem, _stream_ptr(stream),
             cache_path.encode() if cache_path else None, ctypes.byref(t))
        return {f: getattr(t, f) for f, _ in binding.Tuning._fields_}

    def set_graphs(self, enable: bool = True):
        """Replay captured CUDA graphs (default) or launch kernels one by one."""
        call("rl_reloc_set_graphs", self.h, int(enable))

    def graph_kernels(self, n: int) -> int:
        """Kernel launches of the captured graph of an n-frame call (-1: none
        captured)."""
        k = ctypes.c_int32()
        call("rl_reloc_graph_kernels", self.h, int(n), ctypes.byref(k))
        return k.value

    def set_wait_limit(self, probes: int = -1):
        """Failure injection: probes of the LM kernel's waits for staged tiles
        before they give up (0: at once, negative: the default); see
        rl_reloc_set_wait_limit."""
        call("rl_reloc_set_wait_limit", self.h, int(probes))

    def profile(self, enable: bool = True):
        """Turn per-kernel event timing and work counters on/off (resets them)."""
        call("rl_reloc_profile", self.h, int(enable))

    def profile_read(self):
        ms = np.zeros(N_KERNELS)
        launches = np.zeros(N_KERNELS, np.int64)
        work = np.zeros(N_WORK, np.uint64)
        call("rl_reloc_profile_read", self.h, ms.ctypes.data_as(ctypes.c_void_p),
             launches.ctypes.data_as(ctypes.c_void_p), work.ctypes.data_as(ctypes.c_void_p))
        names = [lib().rl_kernel_name(i).decode() for i in range(N_KERNELS)]
        kernels = {names[i]: dict(ms=float(ms[i]), launches=int(launches[i])) for i in range(N_KERNELS)}
        keys = ["energy_pairs", "energy_modes", "lm_pairs", "lm_modes", "lm_inliers", "lm_trial", "rays",
                "hyp_attempts", "hyp_stage2", "icp_pixels", "rays_fp64", "lm_evals"]
        return kernels, {k: int(v) for k, v in zip(keys, work)}

    def debug(self, q: int = 0):
        p = self.params
        N, NC, eta = p["n_hyp"], p["n_cull"], p["eta"]
        d = dict(hyp_pose=np.zeros((N, 12)), hyp_iter=np.zeros(N, np.int32),
                 cull_slot=np.zeros(NC, np.int32), cull_energy=np.zeros(NC, np.float32),
                 round_count=np.zeros(16, np.int32), round_slot=np.zeros((16, NC), np.int32),
                 round_energy=np.zeros((16, NC), np.float32), round_pose=np.zeros((16, NC, 12)),
                 batch_pix=np.zeros((16, eta), np.int32), n_rounds=np.zeros(1, np.int32))
        ptr = lambda k: d[k].ctypes.data_as(ctypes.c_void_p)
        call("rl_reloc_debug", self.h, q, ptr("hyp_pose"), ptr("hyp_iter"), ptr("cull_slot"),
             ptr("cull_energy"), ptr("round_count"), ptr("round_slot"), ptr("round_energy"),
             ptr("round_pose"), ptr("batch_pix"), ptr("n_rounds"))
        d["n_rounds"] = int(d["n_rounds"][0])
        return d

    def close(self):
        if self.h:
            call("rl_reloc_destroy", self.h)
            self.h = ctypes.c_void_p()


class Cascade:
    def __init__(self, levels: list, thresholds, subsample):
        self.levels = levels
        n = len(levels)
        arr = (ctypes.c_void_p * n)(*[lv.h.value for lv in levels])
        th = np.ascontiguousarray(list(thresholds) + [0.0], np.float64)
        ss = np.ascontiguousarray(subsample, np.int32)
        self.h = ctypes.c_void_p()
        call("rl_cascade_create", arr, th.ctypes.data_as(ctypes.c_void_p),
             ss.ctypes.data_as(ctypes.c_void_p), n, ctypes.byref(self.h))

    def relocalise_batch(self, depth, rgb, K, seeds, stream=None):
        d = _Image(depth, np.float32)
        c = _Image(rgb, np.uint8)
        seeds = np.ascontiguousarray(seeds, np.uint64)
        n = len(seeds)
        out = (Result * n)()
        call("rl_cascade_relocalise_batch", self.h, n, d.ptr, c.ptr, ctypes.byref(intrinsics(K)),
             seeds.ctypes.data_as(ctypes.c_void_p), d.mem, _stream_ptr(stream), out)
        return [result_dict(out[i]) for i in range(n)]

    def close(self):
        if self.h:
            call("rl_cascade_destroy", self.h)
            self.h = ctypes.c_void_p()


class Server:
    """Serving loop over several models (rooms / parameter sets): requests
    from host frames of any size up to the model's maximum are batched
    continuously on the GPU (see rl_server_* in include/relocgb.h)."""

    def __init__(self, ctx: Context, max_batch: int = 16, memory_budget: int = 1 << 30,
                 queue_when_full: bool = True):
        from .binding import ServerParams
        self.ctx = ctx
        self.h = ctypes.c_void_p()
        p = ServerParams(max_batch, int(queue_when_full), memory_budget)
        call("rl_server_create", ctx.h, ctypes.byref(p), ctypes.byref(self.h))
        self._keep = []

    def add_model(self, forest: Forest, scene: Scene | None, params: dict, max_w: int, max_h: int) -> int:
        mid = ctypes.c_int32()
        full = dict(presets.DEFAULT, **params)
        call("rl_server_add_model", self.h, forest.h, scene.h if scene else None,
             ctypes.byref(ransac_struct(full)), max_w, max_h, ctypes.byref(mid))
        return mid.value

    def add_cascade_model(self, forest: Forest, scene: Scene | None, levels: list, subsample,
                          thresholds, max_w: int, max_h: int) -> int:
        """A cascade (Sec. 3.2.5) served like a single relocaliser: levels are
        parameter dicts, subsample[l] the level's input subsampling (last 1)."""
        mid = ctypes.c_int32()
        L = len(levels)
        arr = (RansacParams * L)(*[ransac_struct(dict(presets.DEFAULT, **p)) for p in levels])
        ss = np.ascontiguousarray(subsample, np.int32)
        th = np.ascontiguousarray(list(thresholds) + [0.0], np.float64)
        call("rl_server_add_cascade_model", self.h, forest.h, scene.h if scene else None,
             ctypes.cast(arr, ctypes.c_void_p), ss.ctypes.data_as(ctypes.c_void_p),
             th.ctypes.data_as(ctypes.c_void_p), L, max_w, max_h, ctypes.byref(mid))
        return mid.value

    def submit(self, model: int, depth, rgb, K, seed: int) -> int:
        d = np.ascontiguousarray(depth, np.float32)
        c = np.ascontiguousarray(rgb, np.uint8)
        t = ctypes.c_uint64()
        call("rl_server_submit", self.h, model, d.ctypes.data_as(ctypes.c_void_p),
             c.ctypes.data_as(ctypes.c_void_p), ctypes.byref(intrinsics(K)), seed, ctypes.byref(t))
        return t.value

    def poll(self, ticket: int):
        done = ctypes.c_int32()
        r = Result()
        call("rl_server_poll", self.h, ticket, ctypes.byref(done), ctypes.byref(r))
        return result_dict(r) if done.value else None

    def wait(self, ticket: int, timeout_ms: int = 60_000):
        r = Result()
        call("rl_server_wait", self.h, ticket, timeout_ms, ctypes.byref(r))
        return result_dict(r)

    def reset_stats(self):
        call("rl_server_reset_stats", self.h)

    def stats(self) -> dict:
        from .binding import ServerStats
        st = ServerStats()
        call("rl_server_get_stats", self.h, ctypes.byref(st))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            call("rl_server_destroy", self.h)
            self.h = ctypes.c_void_p()


def tuning_cache_read(path: str, key: str):
    """Tuning recorded under key in the cache file, or None."""
    t = binding.Tuning()
    found = ctypes.c_int32()
    call("rl_tuning_cache_read", path.encode(), key.encode(), ctypes.byref(t), ctypes.byref(found))
    return {f: getattr(t, f) for f, _ in binding.Tuning._fields_} if found.value else None


def tuning_cache_write(path: str, key: str, tuning: dict):
    """Records tuning under key (streams defaults to 1)."""
    t = binding.Tuning(**dict(dict(streams=1), **tuning))
    call("rl_tuning_cache_write", path.encode(), key.encode(), ctypes.byref(t))

