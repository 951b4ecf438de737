"""CUDA path vs the CPU oracle, stage by stage, through the C ABI.

Bit-exact: forest nodes, leaf maps (Eq. 1-3), reservoirs (Algorithm R),
mode membership, generation iterations (every Philox choice and check
outcome), pixel batches.  Tolerances: poses 1 mm / 0.05 deg, FP32 energies
1e-4 relative of the FP64 oracle, cull survivors equal up to swaps of
energies within 1e-5 relative.
"""
import math

import numpy as np
import pytest

import oracle
from synth import rooms, workloads
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_12163_gb300 as rg
    rg.lib()
    return rg


@pytest.fixture(scope="module")
def ctx(rg):
    return rg.Context(0, arena_bytes=12 << 30)


@pytest.fixture(scope="module")
def small(rg, ctx):
    w = H.WORKLOADS[H.SMALL]
    return w, H.gpu_model(ctx, w)


def test_forest_nodes_bitexact(rg, ctx):
    for w in (H.WORKLOADS[H.SMALL], workloads.CONFIG2):
        g = rg.Forest.random(ctx, w.forest, w.forest_seed)
        e = g.export()
        o = H.oracle_forest_nodes(w)
        for k in ("dx", "dy", "tau"):
            assert np.array_equal(e[k].view(np.uint32), o[k].view(np.uint32)), k
        assert np.array_equal(e["type"], o["type"])
        assert np.array_equal(e["channel"], o["channel"])
        g.close()


@pytest.mark.parametrize("size", [(96, 72), (97, 71), (160, 120), (640, 480), (33, 257)])
def test_leaves_bitexact(rg, ctx, size):
    w = H.WORKLOADS[H.SMALL]
    g = rg.Forest.random(ctx, dict(w.forest, n_trees=3, depth=12), 11)
    o = oracle.forest_random(3, 12, 0.4, (-130.0, 130.0), (-0.2, 0.2), (-50.0, 50.0), False, 11)
    W, Hh = size
    K = rooms.intrinsics_for(W, Hh) if (W, Hh) in [(96, 72), (160, 120), (640, 480)] else \
        rooms.Intrinsics(0.9 * W, 0.9 * W, W / 2 + 0.3, Hh / 2 - 0.2, W, Hh)
    room = w.room()
    d, c = rooms.render(room, K, rooms.look_pose([1.0, 0.8, 1.1], 0.6, 0.2), noise_seed=3)
    d = rooms.mask_depth(d, 0.2, seed=4)          # invalid pixels and probes reading 0
    d[:, :3] = -1.0                               # negative depth is invalid too
    lg = g.leaves(d, c, K)
    lo = oracle.forest_leaves(o, d, c, K.fx)
    assert np.array_equal(lg, lo)
    assert (lg == 0xFFFF).any() and (lg != 0xFFFF).any()
    g.close()


def test_reservoirs_and_modes_bitexact(rg, small):
    w, g = small
    f, res, modes = H.oracle_model(w.name)
    e = g.export(reservoirs=True)
    assert np.array_equal(e["res_count"], res.count)
    kappa = w.forest["kappa"]
    n = np.minimum(res.count, kappa)
    mask = np.arange(kappa)[None, :] < n[:, None]
    assert np.array_equal(e["res_pos"][mask].view(np.uint32), res.pos[mask].view(np.uint32))
    assert np.array_equal(e["res_rgb"][mask], res.rgb[mask])
    assert (n > 0).sum() > 10
    # Really Quick Shift: identical membership -> identical counts/sizes/colours
    assert np.array_equal(e["nmodes"], modes.nmodes)
    mm = np.arange(w.forest["m_max"])[None, :] < modes.nmodes[:, None]
    assert np.array_equal(e["mode_size"][mm], modes.size[mm])
    assert np.array_equal(e["mode_rgb"][mm], modes.rgb[mm])
    assert np.array_equal(e["mode_pos"][mm].view(np.uint32), modes.pos[mm].view(np.uint32))
    np.testing.assert_allclose(e["mode_U"][mm], modes.U[mm], rtol=2e-7, atol=0)
    assert modes.nmodes.sum() > 20


def _compare_query(rg, rel, w, q, params):
    d, c, T, seed = w.query(q)
    gr = rel.relocalise(d, c, w.K, seed)
    orun, _ = H.oracle_query(w.name, q, params)
    return H.compare_results(rg, gr, rel.debug(0), orun, params, f"q{q}")


def test_relocalise_parity_small(rg, ctx, small):
    w, g = small
    scene = rg.Scene(ctx, w.room().lo, w.room().hi)
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 1)
    for q in range(w.n_queries):
        _compare_query(rg, rel, w, q, w.ransac)
    rel.close()


def test_relocalise_parity_small_variants(rg, ctx, small):
    """Euclidean energy, no LM, plain (unranked) output, k = 1."""
    w, g = small
    scene = rg.Scene(ctx, w.room().lo, w.room().hi)
    for extra in (dict(use_cov=0), dict(pose_update=0), dict(rank=0, k_out=1, halve_to_one=0)):
        p = dict(w.ransac, **extra)
        rel = rg.Relocaliser(g, scene, p, w.width, w.height, 1)
        for q in range(2):
            _compare_query(rg, rel, w, q, p)
        rel.close()


def test_relocalise_parity_six_trees(rg, ctx):
    """Six trees, one more than a pixel record holds: the walk writes the
    per-tree leaf map and the |M(u)| map, generation checks colours per
    attempt (no colour-check masks), and every consumer reads the maps."""
    w = workloads.small_case(n_trees=6)
    g = H.gpu_model(ctx, w)
    scene = rg.Scene(ctx, w.room().lo, w.room().hi)
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 1)
    n_hyp = 0
    for q in range(3):
        d, c, T, seed = w.query(q)
        gr = rel.relocalise(d, c, w.K, seed)
        n_hyp += gr["n_hypotheses"]
        orun, _ = H.oracle_query(w.name, q, w.ransac)
        H.compare_results(rg, gr, rel.debug(0), orun, w.ransac, f"six trees q{q}")
    assert n_hyp > 0
    rel.close()
    scene.close()
    g.close()


def test_batch_invariance(rg, ctx, small):
    """Each frame's result is identical alone and inside a batch."""
    w, g = small
    scene = rg.Scene(ctx, w.room().lo, w.room().hi)
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 4)
    qs = [w.query(q) for q in range(4)]
    D = np.stack([q[0] for q in qs])
    C = np.stack([q[1] for q in qs])
    seeds = [q[3] for q in qs]
    batch = rel.relocalise_batch(D, C, w.K, seeds)
    for i in range(4):
        alone = rel.relocalise(D[i], C[i], w.K, seeds[i])
        assert np.array_equal(alone["pose"], batch[i]["pose"])
        assert alone["energy"] == batch[i]["energy"] and alone["n_hypotheses"] == batch[i]["n_hypotheses"]
        assert (alone["score"] == batch[i]["score"]) or (np.isinf(alone["score"]) and np.isinf(batch[i]["score"]))
    rel.close()


def test_graph_replay_matches_direct_launches(rg, ctx, small):
    """Captured-graph replay (default) and kernel-by-kernel launches give
    bit-identical results, across batch sizes that need new captures."""
    w, g = small
    scene = rg.Scene(ctx, w.room().lo, w.room().hi)
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 3)
    qs = [w.query(q) for q in range(3)]
    D = np.stack([q[0] for q in qs])
    C = np.stack([q[1] for q in qs])
    seeds = [q[3] for q in qs]
    for n in (3, 1, 3):
        rel.set_graphs(True)
        a = rel.relocalise_batch(D[:n], C[:n], w.K, seeds[:n])
        rel.set_graphs(False)
        b = rel.relocalise_batch(D[:n], C[:n], w.K, seeds[:n])
        for x, y in zip(a, b):
            assert np.array_equal(x["pose"], y["pose"]) and x["energy"] == y["energy"]
            assert np.array_equal(x["chosen_score"], y["chosen_score"])
    rel.close()


def test_no_depth_gives_no_pose(rg, ctx, small):
    w, g = small
    rel = rg.Relocaliser(g, None, dict(w.ransac, rank=0), w.width, w.height, 1)
    d = np.zeros((w.height, w.width), np.float32)
    c = np.zeros((w.height, w.width, 3), np.uint8)
    r = rel.relocalise(d, c, w.K, 1)
    assert r["status"] == rg.RL_NO_POSE and r["n_hypotheses"] == 0 and np.isinf(r["score"])
    rel.close()


def test_invalid_arguments(rg, ctx, small):
    w, g = small
    with pytest.raises(rg.RelocError) as e:
        rg.Relocaliser(g, None, dict(w.ransac, n_cull=0), w.width, w.height, 1)
    assert e.value.status == 1
    with pytest.raises(rg.RelocError):
        rg.Relocaliser(g, None, dict(w.ransac, rank=1), w.width, w.height, 1)  # rank needs a scene
    rel = rg.Relocaliser(g, None, dict(w.ransac, rank=0), w.width, w.height, 1)
    d, c, T, seed = w.query(0)
    big = rooms.Intrinsics(100, 100, 50, 50, w.width + 1, w.height)
    with pytest.raises(rg.RelocError):
        rel.relocalise(np.zeros((w.height, w.width + 1), np.float32),
                       np.zeros((w.height, w.width + 1, 3), np.uint8), big, 1)
    with pytest.raises(rg.RelocError) as e:
        g.close()                                  # still used by `rel`
    assert e.value.status == 6
    rel.close()


def test_relocalise_parity_config1(rg, ctx):
    w = workloads.CONFIG1
    g = H.gpu_model(ctx, w)
    f, res, modes = H.oracle_model(w.name)
    e = g.export()
    assert np.array_equal(e["nmodes"], modes.nmodes)
    scene = rg.Scene(ctx, w.room().lo, w.room().hi)
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 1)
    for q in range(w.n_queries):
        _compare_query(rg, rel, w, q, w.ransac)
    rel.close()
    g.close()


def test_score_poses_parity(rg, ctx):
    """Eq. 6-7 on poses from the input generator: inside the room, partly
    outside (silhouettes), outside facing away (+inf), missing live depth."""
    w = workloads.CONFIG2
    room = w.room()
    scene = rg.Scene(ctx, room.lo, room.hi)
    rng = np.random.default_rng(12)
    gt = rooms.look_pose([2.0, 1.4, 1.3], 2.0, -0.1)
    d, _ = rooms.render(room, w.K, gt, noise_seed=2)
    d = rooms.mask_depth(d, 0.3, seed=5)
    poses = [gt]
    for _ in range(12):                                   # inside, perturbed
        poses.append(rooms.look_pose(rng.uniform([0.5, 0.5, 0.5], [3.5, 2.5, 2.0]),
                                     rng.uniform(0, 6.3), rng.uniform(-0.6, 0.6), rng.uniform(-0.3, 0.3)))
    for _ in range(12):                                   # outside the box, looking at it
        c = np.array([2.0, 1.5, 1.25]) + rng.normal(size=3) * 3.0
        c[0] = -abs(c[0]) - 0.5
        yaw = math.atan2(1.5 - c[1], 2.0 - c[0]) + rng.uniform(-0.4, 0.4)
        poses.append(rooms.look_pose(c, yaw, rng.uniform(-0.3, 0.3)))
    poses.append(rooms.look_pose([-1.0, 1.5, 1.25], math.pi, 0.0))   # facing away
    s_g, f_g = scene.score_poses(d, w.K, np.stack(poses))
    for i, P in enumerate(poses):
        s_o, mu_o, f_o = oracle.depth_score(P, d, w.K, room.lo, room.hi)
        assert abs(f_g[i] - f_o) < 1e-6, (i, f_g[i], f_o)
        if math.isinf(s_o):
            assert math.isinf(s_g[i]), i
        else:
            assert abs(s_g[i] - s_o) <= 1e-4 * s_o, (i, s_g[i], s_o)
    assert math.isinf(s_g[-1]) and sum(0.1 < f < 1.0 for f in f_g) >= 3
    scene.close()
