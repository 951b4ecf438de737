"""Serving loop: requests from several camera streams over two models and
two resolutions arrive from concurrent threads; each result equals the
result of relocalising the frame alone; admission and bounded waits."""
import threading

import numpy as np
import pytest

from synth import rooms, workloads
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_12163_gb300 as rg
    ctx = rg.Context(0, arena_bytes=4 << 30)
    w = H.WORKLOADS[H.SMALL]
    g = H.gpu_model(ctx, w)
    scene = rg.Scene(ctx, w.room().lo, w.room().hi)
    return rg, ctx, w, g, scene


def _frames(w):
    out = []
    for q in range(6):
        d, c, T, seed = w.query(q)
        out.append((d, c, w.K, seed))
        ds, cs, Ks = rooms.subsample(d, c, w.K, 2)           # a second, smaller stream
        out.append((ds, cs, Ks, seed + 7))
    return out


def test_mixed_streams_match_alone(setup):
    rg, ctx, w, g, scene = setup
    params = [w.ransac, dict(w.ransac, use_cov=0, n_hyp=64)]
    srv = rg.Server(ctx, max_batch=4, memory_budget=1 << 26)
    models = [srv.add_model(g, scene, p, w.width, w.height) for p in params]
    frames = _frames(w)
    jobs = [(m, f) for m in models for f in frames]
    tickets = [None] * len(jobs)

    def producer(k):
        for i in range(k, len(jobs), 3):
            m, (d, c, K, seed) = jobs[i]
            tickets[i] = srv.submit(m, d, c, K, seed)

    th = [threading.Thread(target=producer, args=(k,)) for k in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    got = [srv.wait(t, 60_000) for t in tickets]
    st = srv.stats()
    assert st["completed"] == len(jobs) and st["refused"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0 and st["frames_per_s"] > 0
    srv.close()
    # the same frames relocalised one at a time
    for p_i, p in enumerate(params):
        rel = rg.Relocaliser(g, scene, p, w.width, w.height, 1)
        for f_i, (d, c, K, seed) in enumerate(frames):
            alone = rel.relocalise(d, c, K, seed)
            r = got[p_i * len(frames) + f_i]
            assert np.array_equal(alone["pose"], r["pose"]), (p_i, f_i)
            assert alone["energy"] == r["energy"] and alone["n_hypotheses"] == r["n_hypotheses"]
            assert (alone["score"] == r["score"]) or (np.isinf(alone["score"]) and np.isinf(r["score"]))
        rel.close()


def test_admission_refusal_and_bounded_wait(setup):
    rg, ctx, w, g, scene = setup
    d, c, T, seed = w.query(0)
    one = d.size * 7
    srv = rg.Server(ctx, max_batch=2, memory_budget=one, queue_when_full=False)
    m = srv.add_model(g, scene, w.ransac, w.width, w.height)
    accepted, refused = [], 0
    for i in range(8):
        try:
            accepted.append(srv.submit(m, d, c, w.K, seed + i))
        except rg.RelocError as e:
            assert e.status == 3                               # RL_ERR_ADMISSION
            refused += 1
    assert refused >= 1 and accepted
    for t in accepted:
        assert srv.wait(t, 60_000)["n_hypotheses"] >= 0
    with pytest.raises(rg.RelocError):
        srv.wait(accepted[0], 10)                              # released ticket
    assert srv.stats()["refused"] == refused
    srv.close()


def test_wait_times_out_then_completes(setup):
    rg, ctx, w, g, scene = setup
    d, c, T, seed = w.query(1)
    srv = rg.Server(ctx, max_batch=1, memory_budget=1 << 30)
    m = srv.add_model(g, scene, w.ransac, w.width, w.height)
    tickets = [srv.submit(m, d, c, w.K, seed + i) for i in range(12)]
    with pytest.raises(rg.RelocError) as e:
        srv.wait(tickets[-1], 0)                               # 11 batches ahead of it
    assert e.value.status == 5                                 # RL_ERR_TIMEOUT, ticket kept
    results = [srv.wait(t, 60_000) for t in tickets]
    assert len(results) == 12
    srv.close()


def test_cascade_model_matches_the_cascade_alone(setup):
    """A cascade served among other requests (two resolutions) returns what
    the same cascade returns for the frame alone."""
    rg, ctx, w, g, scene = setup
    levels = [dict(w.ransac, n_hyp=48, n_trees_used=1, k_out=1), dict(w.ransac)]
    subsample, thresholds = [2, 1], [0.06]
    srv = rg.Server(ctx, max_batch=4, memory_budget=1 << 26)
    mc = srv.add_cascade_model(g, scene, levels, subsample, thresholds, w.width, w.height)
    mp = srv.add_model(g, scene, w.ransac, w.width, w.height)
    frames = _frames(w)
    tickets = [(srv.submit(mc, d, c, K, seed), srv.submit(mp, d, c, K, seed + 1)) for d, c, K, seed in frames]
    got = [srv.wait(tc, 60_000) for tc, _ in tickets]
    for _, tp in tickets:
        srv.wait(tp, 60_000)
    srv.close()
    used = set()
    for (d, c, K, seed), r in zip(frames, got):
        lv = [rg.Relocaliser(g, scene, p, (K.width + s - 1) // s, (K.height + s - 1) // s, 1)
              for p, s in zip(levels, subsample)]
        cas = rg.Cascade(lv, thresholds, subsample)
        alone = cas.relocalise_batch(d[None], c[None], K, [seed])[0]
        cas.close()
        for x in lv:
            x.close()
        used.add(alone["level"])
        assert r["level"] == alone["level"]
        assert np.array_equal(alone["pose"], r["pose"])
        assert alone["energy"] == r["energy"] and alone["n_hypotheses"] == r["n_hypotheses"]
        assert (alone["score"] == r["score"]) or (np.isinf(alone["score"]) and np.isinf(r["score"]))
    assert used  # at least one level produced the results


def _oracle_room(w):
    """The oracle's forest nodes and modes of a serving room's workload."""
    import oracle
    f = H.oracle_forest_nodes(w)
    res = oracle.Reservoirs(f, w.forest["kappa"], w.forest_seed)
    for d, c, T in w.training_frames():
        res.add_frame(d, c, w.K, T, w.forest["grid_step"], w.forest["grid_origin"])
    modes = oracle.Modes(res.n_leaves, w.forest["m_max"])
    oracle.update_modes(res, modes, w.forest["sigma"], w.forest["tau_c"], w.forest["min_cluster_size"],
                        cov_eps=w.forest["cov_eps"], fp16_offsets=bool(w.forest["mode_precision"]))
    return f, modes


def test_config4_rooms_served_against_the_oracle():
    """Config 4 through the serving loop: the 6x5x3 m and 10x8x3 m rooms,
    each with its own five-tree depth-15 forest trained on its 200-frame
    trajectory, served as the config-3 cascade; a 640x480 query and a
    320x240 query (the same view at half resolution, K / 2) per room,
    submitted together, each compared with the FP64 oracle's cascade and
    with the same cascade run alone.  The second room's forest trains on
    the default stream while the first room's requests run on the serving
    loop's streams, and its own requests follow its last mode update at
    once: the library must order both by itself."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_1810_12163_gb300 as rg
    ctx = rg.Context(0, arena_bytes=16 << 30)
    th = workloads.cascade_thresholds()
    subsample = [s for s, _ in workloads.CASCADE_LEVELS]
    levels = [p for _, p in workloads.CASCADE_LEVELS]
    srv = rg.Server(ctx, max_batch=4, memory_budget=1 << 30)
    jobs = []
    keep = []
    models, g_of, scene_of = {}, {}, {}
    for w in workloads.SERVING_ROOMS[1:]:
        g = H.gpu_model(ctx, w)
        scene = rg.Scene(ctx, w.room().lo, w.room().hi)
        keep += [g, scene]
        g_of[w.name], scene_of[w.name] = g, scene
        # the room's forest and modes equal the oracle's
        f, modes = models[w.name] = _oracle_room(w)
        e = g.export()
        assert np.array_equal(e["nmodes"], modes.nmodes), w.name
        mm = np.arange(w.forest["m_max"])[None, :] < modes.nmodes[:, None]
        assert np.array_equal(e["mode_pos"][mm].view(np.uint32), modes.pos[mm].view(np.uint32)), w.name
        m = srv.add_cascade_model(g, scene, levels, subsample, th, w.width, w.height)
        d, c, T, seed = w.query(2)
        ds, cs, Ks = rooms.subsample(d, c, w.K, 2)
        for dd, cc, KK, sd in ((d, c, w.K, seed), (ds, cs, Ks, seed + 1)):
            jobs.append((w, dd, cc, KK, sd, srv.submit(m, dd, cc, KK, sd)))
    got = [srv.wait(tk, 120_000) for *_, tk in jobs]
    srv.close()
    lpt = 1 << workloads.FOREST_DEFAULT["depth"]
    for (w, d, c, K, seed, _), r in zip(jobs, got):
        f, modes = models[w.name]
        frames, maps, params = [], [], []
        for lvl, (s, p) in enumerate(workloads.CASCADE_LEVELS):
            ds, cs, Ks = rooms.subsample(d, c, K, s) if s > 1 else (d, c, K)
            frames.append((ds, cs, Ks))
            maps.append(oracle.forest_leaves(f, ds, cs, Ks.fx, n_trees=p["n_trees_used"]))
            params.append(dict(p, level=lvl))
        o = oracle.cascade(params, th, frames, maps, modes, w.room().lo, w.room().hi, seed, lpt)
        what = f"{w.name} {K.width}x{K.height} level {r['level']}/{o['level']}"
        # the same cascade run on its own
        lv = [rg.Relocaliser(g_of[w.name], scene_of[w.name], p, (K.width + s - 1) // s, (K.height + s - 1) // s, 1)
              for s, p in workloads.CASCADE_LEVELS]
        cas = rg.Cascade(lv, th, subsample)
        alone = cas.relocalise_batch(d[None], c[None], K, [seed])[0]
        cas.close()
        for x in lv:
            x.close()
        # served in a batch with the other resolution: bit-identical to alone
        assert r["level"] == alone["level"] and r["n_hypotheses"] == alone["n_hypotheses"], what
        assert np.array_equal(r["pose"], alone["pose"]), what
        assert r["n_hypotheses"] >= 0
        if r["level"] != o["level"]:
            # a fall-back decision on a score within its tolerance of tau
            lvl = min(r["level"], o["level"])
            assert abs(min(r["score"], o["score"]) - th[lvl]) <= 1e-4 + 1e-3 * th[lvl], what
            continue
        assert r["n_hypotheses"] == o["n_hypotheses"], what
        dt, dr = H.pose_err(r["pose"], o["pose"])
        assert dt <= H.POSE_T_TOL and dr <= H.POSE_R_TOL, (what, dt, dr)
        tol = H.score_tolerances([r["pose"]], [o["pose"]], [o["score"]])
        H.check_scores([r["score"]], [o["score"]], tol, what)
    for x in keep:
        x.close()
    ctx.close()
