"""rl_score_poses_noalloc: the depth-raycast ranking score for callers that
cannot allocate device memory (fixed-budget real-time loops, host frameworks
that own all device memory, code that must avoid the implicit
synchronisation of cudaMalloc/cudaFree).

The entry point is called through the C ABI with device inputs and outputs
only, twice in a row (the second call reuses the library's fixed scratch
array), and each result is checked against the allocating entry point
rl_score_poses on the same poses and against the FP64 oracle's score
(Eq. 6-7) of every pose."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from synth import rooms, workloads

pytestmark = pytest.mark.gpu


def _poses(seed, n_inside, n_outside):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inside):
        out.append(rooms.look_pose(rng.uniform([0.5, 0.5, 0.5], [3.5, 2.5, 2.0]), rng.uniform(0, 6.3),
                                   rng.uniform(-0.6, 0.6), rng.uniform(-0.3, 0.3)))
    for _ in range(n_outside):
        c = np.array([2.0, 1.5, 1.25]) + rng.normal(size=3) * 3.0
        c[0] = -abs(c[0]) - 0.5
        yaw = math.atan2(1.5 - c[1], 2.0 - c[0]) + rng.uniform(-0.4, 0.4)
        out.append(rooms.look_pose(c, yaw, rng.uniform(-0.3, 0.3)))
    out.append(rooms.look_pose([-1.0, 1.5, 1.25], math.pi, 0.0))  # facing away: +inf
    return np.stack(out)


def test_noalloc_scores_match_allocating_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_12163_gb300 as rg
    from paper_1810_12163_gb300 import binding

    L = binding.lib()
    w = workloads.CONFIG2
    room = w.room()
    depth, _ = rooms.render(room, w.K, rooms.look_pose([2.0, 1.4, 1.3], 2.0, -0.1), noise_seed=2)
    depth = rooms.mask_depth(depth, 0.25, seed=9)
    K = rg.intrinsics(w.K)
    lo = np.ascontiguousarray(room.lo, np.float64)
    hi = np.ascontiguousarray(room.hi, np.float64)
    ctx = rg.Context(0, arena_bytes=256 << 20)
    scene = rg.Scene(ctx, lo, hi)
    d_dev = torch.from_numpy(depth).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call_no, poses in enumerate((_poses(1, 12, 8), _poses(2, 30, 17))):
        n = poses.shape[0]
        p_dev = torch.from_numpy(poses.reshape(n, 16).copy()).cuda()
        s_dev = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
        f_dev = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
        st = L.rl_score_poses_noalloc(lo.ctypes.data_as(ctypes.c_void_p), hi.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.c_void_p(d_dev.data_ptr()), ctypes.byref(K),
                                      ctypes.c_void_p(p_dev.data_ptr()), n, stream,
                                      ctypes.c_void_p(s_dev.data_ptr()), ctypes.c_void_p(f_dev.data_ptr()))
        assert st == 0, L.rl_last_error()
        torch.cuda.synchronize()
        s = s_dev.cpu().numpy()
        f = f_dev.cpu().numpy()
        ref_s, ref_f = scene.score_poses(depth, w.K, poses)
        assert np.array_equal(np.isinf(s), np.isinf(ref_s)), (call_no, s, ref_s)
        fin = np.isfinite(ref_s)
        np.testing.assert_allclose(s[fin], ref_s[fin], rtol=1e-4)
        np.testing.assert_allclose(f, ref_f, atol=1e-6)
        assert np.isinf(s[-1]) and fin.sum() >= 10
        # the FP64 oracle: same finite/infinite split, scores within 1e-4
        # relative (FP32 ray arithmetic, FP64 partial sums), valid fractions
        # within a few rays of the FP64 decision
        for i in range(n):
            o_s, _, o_f = oracle.depth_score(poses[i], depth, w.K, room.lo, room.hi)
            assert np.isinf(s[i]) == np.isinf(o_s), (call_no, i, s[i], o_s)
            if np.isfinite(o_s):
                assert abs(s[i] - o_s) <= 1e-4 * o_s, (call_no, i, s[i], o_s)
            assert abs(f[i] - o_f) <= 1e-5, (call_no, i, f[i], o_f)
    # a request beyond the fixed scratch is refused with the limit spelled out
    n = 300
    p_dev = torch.zeros((n, 16), dtype=torch.float64, device="cuda")
    s_dev = torch.zeros(n, dtype=torch.float32, device="cuda")
    st = L.rl_score_poses_noalloc(lo.ctypes.data_as(ctypes.c_void_p), hi.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_void_p(d_dev.data_ptr()), ctypes.byref(K),
                                  ctypes.c_void_p(p_dev.data_ptr()), n, stream,
                                  ctypes.c_void_p(s_dev.data_ptr()), None)
    assert st == 1  # RL_ERR_INVALID_ARG
    assert b"at most 218 poses" in L.rl_last_error()
    # more poses than the launch grid takes, even where the scratch would
    # fit them (frames of at most 1024 pixels need one record per pose)
    K1 = rg.intrinsics(rooms.Intrinsics(20.0, 20.0, 16.0, 16.0, 32, 32))
    st = L.rl_score_poses_noalloc(lo.ctypes.data_as(ctypes.c_void_p), hi.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_void_p(d_dev.data_ptr()), ctypes.byref(K1),
                                  ctypes.c_void_p(p_dev.data_ptr()), 65536, stream,
                                  ctypes.c_void_p(s_dev.data_ptr()), None)
    assert st == 1 and b"limit of 65535 poses" in L.rl_last_error()
    scene.close()
