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
