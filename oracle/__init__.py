"""Python handle on the CPU oracle (plain C, FP64; see oracle.h).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The CUDA library never imports this
package and this package never imports the library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["oracle.c", "adapt.c", "ransac.c", "icp.c"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off keeps FP32 feature
    arithmetic free of fused multiply-adds on every host ISA)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_LIB_PATH):
        if os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(s) for s in srcs):
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp",
           "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


P = ctypes.c_void_p
I32 = ctypes.c_int
F32 = ctypes.c_float
F64 = ctypes.c_double
U64 = ctypes.c_uint64


class IcpParams(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int32), ("stride", ctypes.c_int32 * 3), ("iters", ctypes.c_int32 * 3),
        ("pad", ctypes.c_int32), ("dist", F64 * 3), ("min_frac", F64), ("ridge", F64),
    ]


class Params(ctypes.Structure):
    _fields_ = [
        ("n_hyp", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("n_cull", ctypes.c_int32),
        ("eta", ctypes.c_int32), ("k_out", ctypes.c_int32), ("pose_update", ctypes.c_int32),
        ("use_cov", ctypes.c_int32), ("colour_thresh", ctypes.c_int32),
        ("min_sq_dist", F64), ("max_trans_err", F64),
        ("k_top", ctypes.c_int32), ("n_trees_used", ctypes.c_int32),
        ("lm_max_iter", ctypes.c_int32), ("batch_attempts", ctypes.c_int32),
        ("lm_lambda0", F64), ("lm_inlier_thresh", F64), ("lm_stop", F64),
        ("rank", ctypes.c_int32), ("halve_to_one", ctypes.c_int32), ("level", ctypes.c_int32),
        ("icp", ctypes.c_int32), ("redraw", ctypes.c_int32), ("icp_p", IcpParams),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("pose", F64 * 16), ("energy", F64), ("energy_per_pixel", F64), ("score", F64),
        ("n_hypotheses", ctypes.c_int32), ("n_chosen", ctypes.c_int32),
        ("n_pixels", ctypes.c_int32), ("status", ctypes.c_int32),
        ("chosen_pose", (F64 * 16) * 16), ("chosen_energy", F64 * 16),
        ("chosen_score", F64 * 16), ("chosen_slot", ctypes.c_int32 * 16),
        ("best", ctypes.c_int32), ("icp_mask", ctypes.c_int32), ("chosen_icp_frac", F64 * 16),
    ]


class Resume(ctypes.Structure):
    _fields_ = [("stage", ctypes.c_int32), ("n", ctypes.c_int32), ("slot", P), ("pose", P)]


class Debug(ctypes.Structure):
    _fields_ = [
        ("hyp_pose", P), ("hyp_iter", P), ("cull_slot", P), ("cull_energy", P),
        ("round_slot", P), ("round_energy", P), ("round_pose", P), ("round_count", P),
        ("batch_pix", P), ("n_rounds", ctypes.c_int32), ("pad", ctypes.c_int32),
    ]


def _declare(L):
    L.orc_philox4x32_10.argtypes = [P, P, P]
    L.orc_set_threads.argtypes = [I32]
    L.orc_set_threads.restype = None
    L.orc_forest_random.argtypes = [I32, I32, F32, F32, F32, F32, F32, F32, F32, I32, U64,
                                    P, P, P, P, P]
    L.orc_forest_leaves.argtypes = [P, P, P, P, P, I32, I32, P, P, I32, I32, F32, P]
    L.orc_feature.argtypes = [F32, F32, I32, I32, P, P, I32, I32, F32, I32, I32]
    L.orc_feature.restype = F32
    L.orc_reservoir_add_frame.argtypes = [P, P, P, P, P, I32, I32, P, P, I32, I32,
                                          F32, F32, F32, F32, P, I32, I32, I32, U64, P, P, P]
    L.orc_rqs_leaf.argtypes = [P, P, I32, F32, F32, I32, I32, P, P, P, P, P, P, P]
    L.orc_rqs_leaf.restype = I32
    L.orc_update_modes.argtypes = [P, P, P, I32, I32, I32, I32, F32, F32, I32, I32, F32, I32,
                                   P, P, P, P, P, P]
    L.orc_set_mode_positions.argtypes = [P, P, P, I32, I32, I32, P]
    L.orc_set_mode_positions.restype = None
    L.orc_kabsch.argtypes = [P, P, I32, P, P]
    L.orc_chol_solve6.argtypes = [P, P, P]
    L.orc_chol_solve6.restype = I32
    L.orc_se3_left_update.argtypes = [P, P]
    L.orc_se3_left_update.restype = None
    L.orc_energy.argtypes = [P, P, I32, P, I32, I32, F32, F32, F32, F32, P, I32, I32,
                             P, P, P, I32, I32, I32]
    L.orc_energy.restype = F64
    L.orc_lm_refine.argtypes = [P, P, I32, P, I32, I32, F32, F32, F32, F32, P, I32, I32,
                                P, P, P, I32, I32, I32, I32, F64, F64, F64]
    L.orc_lm_refine.restype = I32
    L.orc_raycast_box.argtypes = [P, I32, I32, F32, F32, F32, F32, P, P, P]
    L.orc_depth_score.argtypes = [P, P, I32, I32, F32, F32, F32, F32, P, P, P, P]
    L.orc_depth_score.restype = F64
    L.orc_relocalise.argtypes = [ctypes.POINTER(Params), P, P, I32, I32, F32, F32, F32, F32,
                                 P, I32, I32, P, P, P, P, I32, P, P, U64,
                                 ctypes.POINTER(Result), ctypes.POINTER(Debug)]
    L.orc_relocalise_from.argtypes = [ctypes.POINTER(Params), P, P, I32, I32, F32, F32, F32, F32,
                                      P, I32, I32, P, P, P, P, I32, P, P, U64,
                                      ctypes.POINTER(Resume), I32, ctypes.POINTER(Result),
                                      ctypes.POINTER(Debug)]
    L.orc_cascade.argtypes = [I32, ctypes.POINTER(Params), P, P, P, P, P, P, P, P, P, P,
                              I32, I32, P, P, P, P, I32, P, P, U64, ctypes.POINTER(Result)]
    L.orc_cascade.restype = I32
    L.orc_icp_refine.argtypes = [P, P, I32, I32, F32, F32, F32, F32, P, P, ctypes.POINTER(IcpParams), P]
    L.orc_icp_refine.restype = I32


def _p(a):
    return a.ctypes.data_as(P) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------
def philox(ctr, key):
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def forest_random(n_trees, depth, p_depth=0.4, delta=(-130.0, 130.0), tau_depth=(-0.2, 0.2),
                  tau_rgb=(-50.0, 50.0), tau_zero=False, seed=2):
    nb = (1 << depth) - 1
    f = {
        "dx": np.zeros(n_trees * nb, np.float32), "dy": np.zeros(n_trees * nb, np.float32),
        "tau": np.zeros(n_trees * nb, np.float32), "type": np.zeros(n_trees * nb, np.uint8),
        "channel": np.zeros(n_trees * nb, np.uint8), "n_trees": n_trees, "depth": depth,
    }
    lib().orc_forest_random(n_trees, depth, p_depth, delta[0], delta[1], tau_depth[0], tau_depth[1],
                            tau_rgb[0], tau_rgb[1], int(tau_zero), seed,
                            _p(f["dx"]), _p(f["dy"]), _p(f["tau"]), _p(f["type"]), _p(f["channel"]))
    return f


def _fargs(f):
    return [_p(f["dx"]), _p(f["dy"]), _p(f["tau"]), _p(f["type"]), _p(f["channel"])]


def forest_leaves(f, depth_img, rgb, fx, n_trees=None):
    d = _c(depth_img, np.float32)
    c = _c(rgb, np.uint8)
    H, W = d.shape
    T = f["n_trees"] if n_trees is None else n_trees
    out = np.zeros((T, H, W), np.uint16)
    lib().orc_forest_leaves(*_fargs(f), T, f["depth"], _p(d), _p(c), W, H, fx, _p(out))
    return out


def feature(dx, dy, ftype, channel, depth_img, rgb, fx, x, y):
    d = _c(depth_img, np.float32)
    c = _c(rgb, np.uint8)
    H, W = d.shape
    return lib().orc_feature(dx, dy, ftype, channel, _p(d), _p(c), W, H, fx, x, y)


class Reservoirs:
    """Leaf reservoirs of a forest (Sec. 3.2.2)."""

    def __init__(self, forest, kappa, seed):
        self.forest = forest
        self.kappa = kappa
        self.seed = seed
        L = forest["n_trees"] << forest["depth"]
        self.n_leaves = L
        self.pos = np.zeros((L, kappa, 3), np.float32)
        self.rgb = np.zeros((L, kappa, 3), np.uint8)
        self.count = np.zeros(L, np.uint32)

    def add_frame(self, depth_img, rgb, K, cam_to_world, grid_step=4, grid_origin=0):
        d = _c(depth_img, np.float32)
        c = _c(rgb, np.uint8)
        H, W = d.shape
        T = _c(cam_to_world, np.float64)
        f = self.forest
        lib().orc_reservoir_add_frame(*_fargs(f), f["n_trees"], f["depth"], _p(d), _p(c), W, H,
                                      K.fx, K.fy, K.cx, K.cy, _p(T), grid_step, grid_origin,
                                      self.kappa, self.seed, _p(self.pos), _p(self.rgb),
                                      _p(self.count))


def rqs_leaf(pos, rgb, sigma, tau_c, min_cluster_size, m_max):
    pos = _c(pos, np.float32)
    rgb = _c(rgb, np.uint8)
    n = pos.shape[0]
    mu = np.zeros((m_max, 3)); col = np.zeros((m_max, 3), np.uint8)
    cov = np.zeros((m_max, 6)); size = np.zeros(m_max, np.int32)
    par = np.zeros(max(n, 1), np.int32); root = np.zeros(max(n, 1), np.int32)
    den = np.zeros(max(n, 1))
    k = lib().orc_rqs_leaf(_p(pos), _p(rgb), n, sigma, tau_c, min_cluster_size, m_max,
                           _p(mu), _p(col), _p(cov), _p(size), _p(par), _p(root), _p(den))
    return dict(k=k, mu=mu[:k], colour=col[:k], cov=cov[:k], size=size[:k],
                parent=par[:n], root=root[:n], density=den[:n])


class Modes:
    """Leaf mode store (decoded FP32) of a forest."""

    def __init__(self, n_leaves, m_max):
        self.m_max = m_max
        self.nmodes = np.zeros(n_leaves, np.uint8)
        self.centroid = np.zeros((n_leaves, 3), np.float32)
        self.pos = np.zeros((n_leaves, m_max, 3), np.float32)
        self.rgb = np.zeros((n_leaves, m_max, 3), np.uint8)
        self.U = np.zeros((n_leaves, m_max, 6), np.float32)
        self.size = np.zeros((n_leaves, m_max), np.int32)


def update_modes(res: Reservoirs, modes: Modes, sigma, tau_c, min_cluster_size,
                 leaf_begin=0, leaf_count=None, cov_eps=1e-4, fp16_offsets=True):
    L = res.n_leaves
    if leaf_count is None:
        leaf_count = L
    lib().orc_update_modes(_p(res.pos), _p(res.rgb), _p(res.count), res.kappa, leaf_begin,
                           leaf_count, L, sigma, tau_c, min_cluster_size, modes.m_max, cov_eps,
                           int(fp16_offsets), _p(modes.nmodes), _p(modes.centroid), _p(modes.pos),
                           _p(modes.rgb), _p(modes.U), _p(modes.size))
    return modes


def set_mode_positions(modes: Modes, pos, fp16_offsets: bool):
    """Writes positions ([L][m_max][3] FP32) into the stored modes in the
    store's precision: FP32, or FP16 offsets from the leaf's FP32 centroid
    (Sec. 3.2.2 mode layout); ranks beyond a leaf's mode count are untouched."""
    pos = _c(pos, np.float32)
    assert pos.shape == modes.pos.shape
    lib().orc_set_mode_positions(_p(pos), _p(modes.nmodes), _p(modes.centroid), modes.pos.shape[0],
                                 modes.m_max, int(fp16_offsets), _p(modes.pos))
    return modes


def set_threads(n: int):
    """Threads of the oracle's OpenMP loops (results do not depend on it)."""
    lib().orc_set_threads(int(n))


def kabsch(a, b):
    a = _c(a, np.float64)
    b = _c(b, np.float64)
    R = np.zeros(9)
    t = np.zeros(3)
    lib().orc_kabsch(_p(a), _p(b), a.shape[0], _p(R), _p(t))
    return R.reshape(3, 3), t


def chol_solve6(A, b):
    """Solves A x = b for a symmetric positive-definite 6x6 A (the damped
    normal equations of the LM step, Sec. 3.2.3); None when A is not positive
    definite."""
    A = _c(A, np.float64)
    b = _c(b, np.float64)
    x = np.zeros(6)
    return x if lib().orc_chol_solve6(_p(A), _p(b), _p(x)) else None


def se3_left_update(xi, pose):
    """exp(xi^) H for xi = (v, w) in se(3), the LM pose update of Sec. 3.2.3;
    pose is 4x4 (or 3x4) camera->world, the result 4x4."""
    H = np.array(np.asarray(pose, np.float64)[:3, :4], dtype=np.float64, order="C", copy=True)
    xi = _c(xi, np.float64)
    lib().orc_se3_left_update(_p(xi), _p(H))
    return np.vstack([H, [0.0, 0.0, 0.0, 1.0]])


PARAM_DEFAULTS = dict(
    n_hyp=1024, max_iter=6000, n_cull=64, eta=512, k_out=16, pose_update=1, use_cov=1,
    colour_thresh=30, min_sq_dist=0.09, max_trans_err=0.05, k_top=10, n_trees_used=5,
    lm_max_iter=10, batch_attempts=32, lm_lambda0=1e-3, lm_inlier_thresh=0.1, lm_stop=1e-6,
    rank=1, halve_to_one=0, level=0, redraw=0,
    icp=0, icp_levels=3, icp_stride=(4, 2, 1), icp_iters=(6, 3, 2), icp_dist=(0.1, 0.05, 0.025),
    icp_min_frac=0.5, icp_ridge=1e-4,
)


def make_icp_params(levels=3, stride=(4, 2, 1), iters=(6, 3, 2), dist=(0.1, 0.05, 0.025),
                    min_frac=0.5, ridge=1e-4):
    ip = IcpParams()
    ip.levels = levels
    for i in range(3):
        ip.stride[i] = stride[i] if i < len(stride) else 1
        ip.iters[i] = iters[i] if i < len(iters) else 0
        ip.dist[i] = dist[i] if i < len(dist) else 0.0
    ip.min_frac = min_frac
    ip.ridge = ridge
    return ip


def make_params(**kw):
    d = dict(PARAM_DEFAULTS)
    for k, v in kw.items():
        if k in d:
            d[k] = v
    p = Params()
    for k, v in d.items():
        if not k.startswith("icp_"):
            setattr(p, k, v)
    p.icp_p = make_icp_params(d["icp_levels"], d["icp_stride"], d["icp_iters"], d["icp_dist"],
                              d["icp_min_frac"], d["icp_ridge"])
    return p


def icp_refine(pose, depth_img, K, lo, hi, **icp):
    """ICP of one pose against the box (R21): (refined 4x4, ok, last-iteration
    inlier fraction).  Keyword arguments as make_icp_params."""
    H12 = _pose12(pose).copy()
    d = _c(depth_img, np.float32)
    H, W = d.shape
    lo = _c(lo, np.float64); hi = _c(hi, np.float64)
    ip = make_icp_params(**icp)
    frac = ctypes.c_double()
    ok = lib().orc_icp_refine(_p(H12), _p(d), W, H, K.fx, K.fy, K.cx, K.cy, _p(lo), _p(hi),
                              ctypes.byref(ip), ctypes.byref(frac))
    out = np.eye(4)
    out[:3, :4] = H12.reshape(3, 4)
    return out, bool(ok), frac.value


def _pose12(pose):
    return _c(np.asarray(pose, np.float64)[:3, :4].reshape(12) if np.ndim(pose) == 2
              else np.asarray(pose, np.float64)[:12], np.float64)


def energy(pose, pix, depth_img, K, leaves, modes: Modes, k_top, use_cov, leaves_per_tree,
           n_trees_used=None):
    H12 = _pose12(pose)
    pix = _c(pix, np.int32)
    d = _c(depth_img, np.float32)
    H, W = d.shape
    lv = _c(leaves, np.uint16)
    T = lv.shape[0] if n_trees_used is None else n_trees_used
    return lib().orc_energy(_p(H12), _p(pix), pix.shape[0], _p(d), W, H, K.fx, K.fy, K.cx, K.cy,
                            _p(lv), T, leaves_per_tree, _p(modes.nmodes), _p(modes.pos),
                            _p(modes.U), modes.m_max, k_top, int(use_cov))


def lm_refine(pose, pix, depth_img, K, leaves, modes: Modes, k_top, use_cov, leaves_per_tree,
              max_iter=10, lambda0=1e-3, inlier_thresh=0.1, stop=1e-6):
    H12 = _pose12(pose).copy()
    pix = _c(pix, np.int32)
    d = _c(depth_img, np.float32)
    H, W = d.shape
    lv = _c(leaves, np.uint16)
    it = lib().orc_lm_refine(_p(H12), _p(pix), pix.shape[0], _p(d), W, H, K.fx, K.fy, K.cx, K.cy,
                             _p(lv), lv.shape[0], leaves_per_tree, _p(modes.nmodes), _p(modes.pos),
                             _p(modes.U), modes.m_max, k_top, int(use_cov), max_iter, lambda0,
                             inlier_thresh, stop)
    out = np.eye(4)
    out[:3, :4] = H12.reshape(3, 4)
    return out, it


def raycast_box(pose, K, lo, hi):
    H12 = _pose12(pose)
    out = np.zeros((K.height, K.width))
    lo = _c(lo, np.float64); hi = _c(hi, np.float64)
    lib().orc_raycast_box(_p(H12), K.width, K.height, K.fx, K.fy, K.cx, K.cy, _p(lo), _p(hi), _p(out))
    return out


def depth_score(pose, depth_img, K, lo, hi):
    H12 = _pose12(pose)
    d = _c(depth_img, np.float32)
    lo = _c(lo, np.float64); hi = _c(hi, np.float64)
    mu = ctypes.c_double(); frac = ctypes.c_double()
    s = lib().orc_depth_score(_p(H12), _p(d), K.width, K.height, K.fx, K.fy, K.cx, K.cy,
                              _p(lo), _p(hi), ctypes.byref(mu), ctypes.byref(frac))
    return s, mu.value, frac.value


def _result_dict(r: Result):
    nc = r.n_chosen if r.n_chosen > 0 else 0
    return dict(
        pose=np.array(r.pose).reshape(4, 4), energy=r.energy, energy_per_pixel=r.energy_per_pixel,
        score=r.score, n_hypotheses=r.n_hypotheses, n_chosen=r.n_chosen, n_pixels=r.n_pixels,
        status=r.status, best=r.best,
        chosen_pose=np.array([np.array(r.chosen_pose[i]).reshape(4, 4) for i in range(nc)]),
        chosen_energy=np.array(r.chosen_energy[:nc]), chosen_score=np.array(r.chosen_score[:nc]),
        chosen_slot=np.array(r.chosen_slot[:nc]), icp_mask=r.icp_mask,
        chosen_icp_frac=np.array(r.chosen_icp_frac[:max(nc, 1)]),
    )


def relocalise(params: dict, depth_img, rgb, K, leaves, modes: Modes, box_lo, box_hi, seed,
               leaves_per_tree, debug=False, resume=None):
    """One relocalisation (Sec. 3.2.3-3.2.4).  resume = a list of
    (stage, slots, poses [n][12]) hands survivor sets in at stage boundaries
    of the preemptive loop (stage 0: after the cull; r + 1: after round r),
    at most one per stage; see orc_resume in oracle.h."""
    p = make_params(**params)
    d = _c(depth_img, np.float32)
    c = _c(rgb, np.uint8)
    H, W = d.shape
    lv = _c(leaves, np.uint16)
    lo = _c(box_lo, np.float64); hi = _c(box_hi, np.float64)
    res = Result()
    dbg = Debug()
    arrays = {}
    if debug:
        arrays = dict(
            hyp_pose=np.zeros((p.n_hyp, 12)), hyp_iter=np.zeros(p.n_hyp, np.int32),
            cull_slot=np.full(p.n_cull, -1, np.int32), cull_energy=np.zeros(p.n_cull),
            round_slot=np.full(4 * p.n_cull + 64, -1, np.int32),
            round_energy=np.zeros(4 * p.n_cull + 64),
            round_pose=np.zeros((4 * p.n_cull + 64, 12)), round_count=np.zeros(16, np.int32),
            batch_pix=np.full((16, p.eta), -1, np.int32),
        )
        for k, a in arrays.items():
            setattr(dbg, k, _p(a))
    rs, keep = None, []
    if resume:
        stages = [int(st) for st, _, _ in resume]
        assert len(set(stages)) == len(stages), "one hand-in per stage"
        rs = (Resume * len(resume))()
        for k, (stage, slots, poses) in enumerate(resume):
            rs_slot = _c(slots, np.int32)
            rs_pose = _c(np.asarray(poses, np.float64).reshape(-1, 12), np.float64)
            assert rs_slot.shape[0] == rs_pose.shape[0]
            keep += [rs_slot, rs_pose]
            rs[k] = Resume(int(stage), int(rs_slot.shape[0]), _p(rs_slot), _p(rs_pose))
    lib().orc_relocalise_from(ctypes.byref(p), _p(d), _p(c), W, H, K.fx, K.fy, K.cx, K.cy, _p(lv),
                              lv.shape[0], leaves_per_tree, _p(modes.nmodes), _p(modes.pos),
                              _p(modes.rgb), _p(modes.U), modes.m_max, _p(lo), _p(hi), seed,
                              rs, len(resume) if resume else 0,
                              ctypes.byref(res), ctypes.byref(dbg) if debug else None)
    out = _result_dict(res)
    if debug:
        arrays["n_rounds"] = dbg.n_rounds
        out["debug"] = arrays
    return out


def cascade(levels: list, thresholds, frames: list, leaf_maps: list, modes: Modes, box_lo, box_hi,
            seed, leaves_per_tree):
    """levels: list of param dicts; frames: list of (depth, rgb, K) per level."""
    nl = len(levels)
    P_arr = (Params * nl)(*[make_params(**lv) for lv in levels])
    th = _c(list(thresholds) + [np.inf] * (nl - len(thresholds)), np.float64)
    ds = [_c(f[0], np.float32) for f in frames]
    cs = [_c(f[1], np.uint8) for f in frames]
    lvs = [_c(x, np.uint16) for x in leaf_maps]
    ptr = lambda arrs: (P * nl)(*[a.ctypes.data for a in arrs])
    Ws = _c([f[2].width for f in frames], np.int32)
    Hs = _c([f[2].height for f in frames], np.int32)
    fx = _c([f[2].fx for f in frames], np.float32)
    fy = _c([f[2].fy for f in frames], np.float32)
    cx = _c([f[2].cx for f in frames], np.float32)
    cy = _c([f[2].cy for f in frames], np.float32)
    lo = _c(box_lo, np.float64); hi = _c(box_hi, np.float64)
    res = Result()
    n_trees_forest = max(x.shape[0] for x in lvs)
    lvl = lib().orc_cascade(nl, P_arr, _p(th), ptr(ds), ptr(cs), _p(Ws), _p(Hs), _p(fx), _p(fy),
                            _p(cx), _p(cy), ptr(lvs), n_trees_forest, leaves_per_tree,
                            _p(modes.nmodes), _p(modes.pos), _p(modes.rgb), _p(modes.U),
                            modes.m_max, _p(lo), _p(hi), seed, ctypes.byref(res))
    out = _result_dict(res)
    out["level"] = lvl
    return out
