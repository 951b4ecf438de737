"""Streaming adaptation concurrent with relocalisation (Sec. 3.2.2: leaves
are re-clustered round-robin, a few per frame, while relocalisation runs).

A streaming forest (two mode stores) adapts and re-clusters on one CUDA
stream while relocalisations run on another.  Every relocalisation must
equal, bit for bit, what a single-store forest gives when the same steps
run one after the other in host order: a launch sees the modes after the
last update enqueued before it and nothing of a later one.  The
round-robin modes themselves match the FP64 oracle's leaf-range updates
(wrapping around the leaf array) bit for bit."""
import numpy as np
import pytest

import oracle
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
    return rg.Context(0, arena_bytes=8 << 30)


def _same(a, b):
    return (np.array_equal(a["pose"], b["pose"]) and a["energy"] == b["energy"]
            and a["n_hypotheses"] == b["n_hypotheses"]
            and (a["score"] == b["score"] or (np.isinf(a["score"]) and np.isinf(b["score"]))))


def test_streaming_snapshots_equal_the_serial_schedule(rg, ctx):
    import torch
    w = H.WORKLOADS[H.SMALL]
    frames = list(w.training_frames())
    n0, step_leaves = 6, 200                      # 512 leaves: the round robin wraps
    forests = []
    for streaming in (True, False):
        g = rg.Forest.random(ctx, w.forest, w.forest_seed)
        for d, c, T in frames[:n0]:
            g.adapt(d, c, w.K, T)
        g.update_modes(-1)
        if streaming:
            g.set_streaming(True)
        forests.append(g)
    A, B = forests
    room = w.room()
    scene = rg.Scene(ctx, room.lo, room.hi)
    relA = rg.Relocaliser(A, scene, w.ransac, w.width, w.height, 4)
    relB = rg.Relocaliser(B, scene, w.ransac, w.width, w.height, 4)
    qs = [w.query(q) for q in range(4)]
    D = torch.from_numpy(np.stack([q[0] for q in qs])).cuda()
    C = torch.from_numpy(np.stack([q[1] for q in qs])).cuda()
    sR, sT = torch.cuda.Stream(), torch.cuda.Stream()
    dev = [(torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda(), T) for d, c, T in frames[n0:]]
    torch.cuda.synchronize()
    changed = 0
    for k, (dd, cc, T) in enumerate(dev):
        seeds = [100 * k + i for i in range(4)]
        # streaming: relocalise on sR, then adapt and re-cluster on sT, no host wait between
        relA.relocalise_batch_async(D, C, w.K, seeds, stream=sR)
        A.adapt(dd, cc, w.K, T, stream=sT)
        A.update_modes(step_leaves, stream=sT)
        resA = relA.fetch(stream=sR)
        # serial: relocalise, then adapt and re-cluster
        resB = relB.relocalise_batch(D, C, w.K, seeds)
        B.adapt(dd, cc, w.K, T)
        B.update_modes(step_leaves)
        for a, b in zip(resA, resB):
            assert _same(a, b), k
        # a launch enqueued after the update sees it
        resA2 = relA.relocalise_batch(D, C, w.K, seeds, stream=sR)
        resB2 = relB.relocalise_batch(D, C, w.K, seeds)
        for a, b in zip(resA2, resB2):
            assert _same(a, b), k
        changed += any(not _same(a, b) for a, b in zip(resA, resA2))
    torch.cuda.synchronize()
    assert changed > 0   # the updates did change what relocalisation sees
    ea, eb = A.export(), B.export()
    for key in ("nmodes", "mode_pos", "mode_rgb", "mode_size"):
        assert np.array_equal(ea[key], eb[key]), key

    # the round-robin modes against the oracle's leaf-range updates
    f = H.oracle_forest_nodes(w)
    res = oracle.Reservoirs(f, w.forest["kappa"], w.forest_seed)
    modes = oracle.Modes(res.n_leaves, w.forest["m_max"])
    kw = dict(cov_eps=w.forest["cov_eps"], fp16_offsets=bool(w.forest["mode_precision"]))
    for d, c, T in frames[:n0]:
        res.add_frame(d, c, w.K, T, w.forest["grid_step"], w.forest["grid_origin"])
    oracle.update_modes(res, modes, w.forest["sigma"], w.forest["tau_c"], w.forest["min_cluster_size"], **kw)
    cursor = 0
    for d, c, T in frames[n0:]:
        res.add_frame(d, c, w.K, T, w.forest["grid_step"], w.forest["grid_origin"])
        oracle.update_modes(res, modes, w.forest["sigma"], w.forest["tau_c"], w.forest["min_cluster_size"],
                            leaf_begin=cursor, leaf_count=step_leaves, **kw)
        cursor = (cursor + step_leaves) % res.n_leaves
    assert np.array_equal(ea["nmodes"], modes.nmodes)
    mm = np.arange(w.forest["m_max"])[None, :] < modes.nmodes[:, None]
    assert np.array_equal(ea["mode_pos"][mm].view(np.uint32), modes.pos[mm].view(np.uint32))
    relA.close()
    relB.close()
    scene.close()
    A.close()
    B.close()


def test_streaming_must_be_set_before_relocalisers(rg, ctx):
    w = H.WORKLOADS[H.SMALL]
    g = rg.Forest.random(ctx, w.forest, w.forest_seed)
    rel = rg.Relocaliser(g, None, dict(w.ransac, rank=0), w.width, w.height, 1)
    with pytest.raises(rg.RelocError):
        g.set_streaming(True)
    rel.close()
    g.set_streaming(True)
    g.set_streaming(False)
    g.close()


def test_tracking_loss_protocol_parity(rg, ctx):
    """Tracking-loss recovery (Sec. 4): from empty leaves, frame t is
    relocalised with the forest adapted from frames < t (round-robin modes),
    then frame t is added with its true pose.  Each relocalisation against
    the oracle run on the same forest state."""
    import torch
    w = H.WORKLOADS[H.SMALL]
    frames = list(w.training_frames())[:8]
    step_leaves = 200
    g = rg.Forest.random(ctx, w.forest, w.forest_seed)
    g.set_streaming(True)
    room = w.room()
    scene = rg.Scene(ctx, room.lo, room.hi)
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 1)
    f = H.oracle_forest_nodes(w)
    res = oracle.Reservoirs(f, w.forest["kappa"], w.forest_seed)
    modes = oracle.Modes(res.n_leaves, w.forest["m_max"])
    kw = dict(cov_eps=w.forest["cov_eps"], fp16_offsets=bool(w.forest["mode_precision"]))
    sR, sT = torch.cuda.Stream(), torch.cuda.Stream()
    cursor, found = 0, 0
    for t, (d, c, T) in enumerate(frames):
        dd, cc = torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda()
        if t >= 1:
            seed = 7000 + t
            rel.relocalise_batch_async(dd[None], cc[None], w.K, [seed], stream=sR)
        g.adapt(dd, cc, w.K, T, stream=sT)
        g.update_modes(step_leaves, stream=sT)
        if t >= 1:
            gr = rel.fetch(stream=sR)[0]
            lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=w.ransac["n_trees_used"])
            orr = H.OracleRun(w.ransac, d, c, w.K, lv, modes, room.lo, room.hi, seed,
                                    1 << w.forest["depth"])
            H.compare_results(rg, gr, rel.debug(0), orr, w.ransac, f"tracking loss frame {t}")
            found += gr["status"] == rg.RL_POSE_FOUND
        res.add_frame(d, c, w.K, T, w.forest["grid_step"], w.forest["grid_origin"])
        oracle.update_modes(res, modes, w.forest["sigma"], w.forest["tau_c"], w.forest["min_cluster_size"],
                            leaf_begin=cursor, leaf_count=step_leaves, **kw)
        cursor = (cursor + step_leaves) % res.n_leaves
    assert found >= 3
    rel.close()
    scene.close()
    g.close()


def test_tracking_loss_step_config2(rg, ctx):
    """Paper-sized tracking-loss step: a five-tree depth-15 forest from
    empty leaves adapts three frames of a fresh trajectory (65,536 leaves
    re-clustered per frame, double-buffered), then relocalises the fourth;
    modes and the relocalisation against the oracle on the same state."""
    import math
    import torch
    from synth import rooms, workloads
    w = workloads.CONFIG2
    room = w.room()
    poses = rooms.training_trajectory(room, 4, seed=21)
    frames = [rooms.render(room, w.K, T, w.noise_sigma, noise_seed=60000 + t) + (T,) for t, T in enumerate(poses)]
    step = 65536
    g = rg.Forest.random(ctx, w.forest, w.forest_seed)
    g.set_streaming(True)
    scene = rg.Scene(ctx, room.lo, room.hi)
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 1)
    f = H.oracle_forest_nodes(w)
    res = oracle.Reservoirs(f, w.forest["kappa"], w.forest_seed)
    modes = oracle.Modes(res.n_leaves, w.forest["m_max"])
    kw = dict(cov_eps=w.forest["cov_eps"], fp16_offsets=bool(w.forest["mode_precision"]))
    sT = torch.cuda.Stream()
    cursor = 0
    for d, c, T in frames[:3]:
        g.adapt(torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda(), w.K, T, stream=sT)
        g.update_modes(step, stream=sT)
        res.add_frame(d, c, w.K, T, w.forest["grid_step"], w.forest["grid_origin"])
        oracle.update_modes(res, modes, w.forest["sigma"], w.forest["tau_c"], w.forest["min_cluster_size"],
                            leaf_begin=cursor, leaf_count=step, **kw)
        cursor = (cursor + step) % res.n_leaves
    torch.cuda.synchronize()
    e = g.export()
    assert np.array_equal(e["nmodes"], modes.nmodes)
    mm = np.arange(w.forest["m_max"])[None, :] < modes.nmodes[:, None]
    assert np.array_equal(e["mode_pos"][mm].view(np.uint32), modes.pos[mm].view(np.uint32))
    d, c, T = frames[3]
    seed = 123457
    gr = rel.relocalise(d, c, w.K, seed)
    lv = oracle.forest_leaves(f, d, c, w.K.fx)
    orr = H.OracleRun(w.ransac, d, c, w.K, lv, modes, room.lo, room.hi, seed, 1 << w.forest["depth"])
    H.compare_results(rg, gr, rel.debug(0), orr, w.ransac, "config2 tracking-loss frame 3")
    rel.close()
    scene.close()
    g.close()
