"""ctypes binding of librelocgb (include/relocgb.h).

Argument marshalling only: every step of the relocaliser runs in the CUDA
library.  PyTorch supplies the device arena and streams.  There is no CPU
fallback: if the library is not built, `lib()` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librelocgb.so")
_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I32 = ctypes.c_int32
U64 = ctypes.c_uint64


class RelocError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


STATUS_NAMES = {0: "RL_OK", 1: "RL_ERR_INVALID_ARG", 2: "RL_ERR_OOM", 3: "RL_ERR_ADMISSION",
                4: "RL_ERR_CUDA", 5: "RL_ERR_TIMEOUT", 6: "RL_ERR_BUSY", 7: "RL_ERR_IO",
                8: "RL_ERR_INTERNAL"}
RL_HOST, RL_DEVICE = 0, 1
RL_POSE_FOUND, RL_NO_POSE = 0, 1
RL_MODES_FP32, RL_MODES_FP16_OFFSET = 0, 1
RL_N_KERNELS = 12  # kernels the profiler reports (RL_N_KERNELS of the header)
RL_N_WORK = 12     # work counters (RL_N_WORK of the header)


class Intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("width", I32), ("height", I32)]


class ForestParams(ctypes.Structure):
    _fields_ = [("n_trees", I32), ("depth", I32), ("p_depth", ctypes.c_float),
                ("delta_lo", ctypes.c_float), ("delta_hi", ctypes.c_float),
                ("tau_depth_lo", ctypes.c_float), ("tau_depth_hi", ctypes.c_float),
                ("tau_rgb_lo", ctypes.c_float), ("tau_rgb_hi", ctypes.c_float),
                ("tau_zero", I32), ("kappa", I32), ("m_max", I32), ("min_cluster_size", I32),
                ("sigma", ctypes.c_float), ("tau_c", ctypes.c_float), ("cov_eps", ctypes.c_float),
                ("mode_precision", I32), ("grid_step", I32), ("grid_origin", I32)]


class IcpParams(ctypes.Structure):
    _fields_ = [("levels", I32), ("stride", I32 * 3), ("iters", I32 * 3), ("pad", I32),
                ("dist", ctypes.c_double * 3), ("min_frac", ctypes.c_double), ("ridge", ctypes.c_double)]


class RansacParams(ctypes.Structure):
    _fields_ = [("n_hyp", I32), ("max_iter", I32), ("n_cull", I32), ("eta", I32), ("k_out", I32),
                ("pose_update", I32), ("use_cov", I32), ("colour_thresh", I32),
                ("min_sq_dist", ctypes.c_double), ("max_trans_err", ctypes.c_double),
                ("k_top", I32), ("n_trees_used", I32), ("lm_max_iter", I32),
                ("batch_attempts", I32), ("lm_lambda0", ctypes.c_double),
                ("lm_inlier_thresh", ctypes.c_double), ("lm_stop", ctypes.c_double),
                ("rank", I32), ("halve_to_one", I32), ("icp", I32), ("redraw", I32),
                ("icp_p", IcpParams)]


class ServerParams(ctypes.Structure):
    _fields_ = [("max_batch", I32), ("queue_when_full", I32), ("memory_budget", U64)]


class Tuning(ctypes.Structure):
    _fields_ = [("hypgen_warps", ctypes.c_int32), ("energy_threads", ctypes.c_int32),
                ("leaves_threads", ctypes.c_int32), ("mask_threads", ctypes.c_int32),
                ("streams", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", U64), ("completed", U64), ("refused", U64),
                ("peak_admitted_bytes", U64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("frames_per_s", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("pose", ctypes.c_double * 16), ("energy", ctypes.c_float),
                ("energy_per_pixel", ctypes.c_float), ("score", ctypes.c_float), ("level", I32),
                ("n_hypotheses", I32), ("n_chosen", I32), ("n_pixels", I32), ("status", I32),
                ("chosen_pose", (ctypes.c_double * 16) * 16), ("chosen_energy", ctypes.c_float * 16),
                ("chosen_score", ctypes.c_float * 16), ("chosen_slot", I32 * 16), ("best", I32),
                ("icp_mask", I32), ("chosen_icp_frac", ctypes.c_float * 16)]


_SIGS = {
    "rl_context_create": [I32, P, U64, P],
    "rl_context_destroy": [P],
    "rl_context_usage": [P, P, P],
    "rl_forest_create_random": [P, P, U64, P],
    "rl_forest_destroy": [P],
    "rl_forest_reset_leaves": [P, P],
    "rl_forest_adapt": [P, P, P, P, P, I32, P],
    "rl_forest_update_modes": [P, I32, P],
    "rl_forest_set_streaming": [P, I32],
    "rl_forest_leaves": [P, P, P, P, I32, P, I32, P],
    "rl_forest_export": [P] + [P] * 12,
    "rl_forest_set_mode_positions": [P, P],
    "rl_forest_save": [P, ctypes.c_char_p],
    "rl_forest_load": [P, ctypes.c_char_p, P],
    "rl_scene_box": [P, P, P, P],
    "rl_scene_destroy": [P],
    "rl_score_poses": [P, P, P, P, I32, I32, P, P, P],
    "rl_score_poses_noalloc": [P, P, P, P, P, I32, P, P, P],
    "rl_icp_poses": [P, P, P, P, I32, P, I32, P, P, P, P],
    "rl_reloc_create": [P, P, P, I32, I32, I32, P],
    "rl_reloc_destroy": [P],
    "rl_relocalise": [P, P, P, P, U64, I32, P, P],
    "rl_relocalise_batch": [P, I32, P, P, P, P, I32, P, P],
    "rl_relocalise_batch_async": [P, I32, P, P, P, P, P],
    "rl_reloc_fetch": [P, I32, P, P],
    "rl_reloc_debug": [P, I32] + [P] * 10,
    "rl_reloc_profile": [P, I32],
    "rl_reloc_set_graphs": [P, I32],
    "rl_reloc_graph_kernels": [P, I32, P],
    "rl_reloc_set_wait_limit": [P, ctypes.c_int64],
    "rl_reloc_profile_read": [P, P, P, P],
    "rl_cascade_create": [P, P, P, I32, P],
    "rl_cascade_destroy": [P],
    "rl_cascade_relocalise": [P, P, P, P, U64, I32, P, P],
    "rl_cascade_relocalise_batch": [P, I32, P, P, P, P, I32, P, P],
    "rl_server_create": [P, P, P],
    "rl_server_add_model": [P, P, P, P, I32, I32, P],
    "rl_server_add_cascade_model": [P, P, P, P, P, P, I32, I32, I32, P],
    "rl_server_reset_stats": [P],
    "rl_reloc_get_tuning": [P, P],
    "rl_reloc_set_tuning": [P, P],
    "rl_reloc_autotune": [P, I32, P, P, P, P, I32, P, ctypes.c_char_p, P],
    "rl_tuning_key": [P, ctypes.c_char_p, I32],
    "rl_tuning_cache_read": [ctypes.c_char_p, ctypes.c_char_p, P, P],
    "rl_tuning_cache_write": [ctypes.c_char_p, ctypes.c_char_p, P],
    "rl_server_submit": [P, I32, P, P, P, U64, P],
    "rl_server_poll": [P, U64, P, P],
    "rl_server_wait": [P, U64, ctypes.c_uint32, P],
    "rl_server_get_stats": [P, P],
    "rl_server_destroy": [P],
}


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"librelocgb.so is not built ({LIB_PATH}); run "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.rl_last_error.argtypes = []
            L.rl_last_error.restype = ctypes.c_char_p
            L.rl_kernel_name.argtypes = [I32]
            L.rl_kernel_name.restype = ctypes.c_char_p
            _lib = L
    return _lib


def check(status):
    if status != 0:
        msg = lib().rl_last_error()
        raise RelocError(status, msg.decode() if msg else "")


def call(name, *args):
    check(getattr(lib(), name)(*args))


def exported_symbols():
    return sorted(_SIGS) + ["rl_last_error", "rl_kernel_name"]
