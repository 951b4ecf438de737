"""Autotuner: tuned and extreme launch shapes give bit-identical results
(each kernel computes the same values in the same order), the tuning is
recorded in and reused from the cache, and bad values are refused."""
import numpy as np
import pytest

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


def _run(rel, qs, w):
    D = np.stack([q[0] for q in qs])
    C = np.stack([q[1] for q in qs])
    return rel.relocalise_batch(D, C, w.K, [q[3] for q in qs])


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x["pose"], y["pose"]) and x["energy"] == y["energy"]
        assert x["n_hypotheses"] == y["n_hypotheses"] and x["best"] == y["best"]
        assert np.array_equal(x["chosen_score"], y["chosen_score"])


def test_tuning_never_changes_results(setup, tmp_path):
    rg, ctx, w, g, scene = setup
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 4)
    qs = [w.query(q) for q in range(4)]
    base = _run(rel, qs, w)
    for t in (dict(hypgen_warps=2, energy_threads=32, leaves_threads=64, mask_threads=64, streams=1),
              dict(hypgen_warps=8, energy_threads=256, leaves_threads=512, mask_threads=256, streams=4)):
        rel.set_tuning(t)
        assert rel.tuning == t
        _same(_run(rel, qs, w), base)
    cache = str(tmp_path / "tuning.txt")
    tuned = rel.autotune(np.stack([q[0] for q in qs]), np.stack([q[1] for q in qs]), w.K,
                         [q[3] for q in qs], cache_path=cache)
    assert rel.tuning == tuned
    _same(_run(rel, qs, w), base)
    assert rg.tuning_cache_read(cache, rel.tuning_key()) == tuned
    # a second relocaliser of the same shape takes the cached tuning without timing
    rel2 = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 4)
    assert rel2.tuning_key() == rel.tuning_key()
    rg.tuning_cache_write(cache, rel2.tuning_key(), dict(hypgen_warps=2, energy_threads=64,
                                                         leaves_threads=256, mask_threads=128, streams=2))
    got = rel2.autotune(np.stack([q[0] for q in qs]), np.stack([q[1] for q in qs]), w.K,
                        [q[3] for q in qs], cache_path=cache)
    assert got == dict(hypgen_warps=2, energy_threads=64, leaves_threads=256, mask_threads=128, streams=2)
    _same(_run(rel2, qs, w), base)
    with pytest.raises(rg.RelocError):
        rel.set_tuning(dict(hypgen_warps=5))
    rel.close()
    rel2.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_sub_batches_on_streams_give_the_batch_results(setup, graphs):
    """A call of 20 frames split into 2 sub-batches (streams 2, and streams 4,
    which 20 frames cap at 2 of at least 8 frames) on concurrent streams, on
    the captured-graph path and launched kernel by kernel: every frame's
    result is bit-identical to the one-stream batch."""
    rg, ctx, w, g, scene = setup
    n = 20
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, n)
    rel.set_graphs(graphs)
    qs = [w.query(q % 6) for q in range(n)]
    qs = [(d, c, T, 1000 + i) for i, (d, c, T, _) in enumerate(qs)]
    base = _run(rel, qs, w)
    assert sum(r["n_hypotheses"] > 0 for r in base) >= n // 2
    kernels = {}
    for streams in (2, 4, 1):
        rel.set_tuning(dict(streams=streams))
        _same(_run(rel, qs, w), base)
        _same(_run(rel, qs, w), base)  # the second call replays the captured graph
        kernels[streams] = rel.graph_kernels(n)
    if graphs:
        # each sub-batch launches the whole sequence; 20 frames make two of at
        # least 8; one kernel (the split nodes scaled for the call's focal
        # length) runs once per call, before the fork
        assert kernels[1] > 20 and kernels[2] == kernels[4] == 2 * (kernels[1] - 1) + 1, kernels
    else:
        assert set(kernels.values()) == {-1}
    rel.close()


def test_frames_of_another_focal_length_walk_the_unscaled_nodes(setup):
    """A call reads split nodes premultiplied by its first frame's fx / 585.
    A graph captured for one focal length and replayed for another keeps the
    old scaled nodes, and its frames then walk the unscaled ones: the
    results equal those of a relocaliser that only saw the second focal
    length (whose own graph walks the nodes scaled for it)."""
    from synth import rooms
    rg, ctx, w, g, scene = setup
    K2 = rooms.Intrinsics(w.K.fx * 1.05, w.K.fy * 1.05, w.K.cx, w.K.cy, w.K.width, w.K.height)
    qs = [w.query(q) for q in range(4)]
    D = np.stack([q[0] for q in qs])
    C = np.stack([q[1] for q in qs])
    seeds = [q[3] for q in qs]
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 4)
    rel.relocalise_batch(D, C, w.K, seeds)             # captures the graph for w.K
    replayed = rel.relocalise_batch(D, C, K2, seeds)   # replays it for K2
    fresh = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 4)
    _same(replayed, fresh.relocalise_batch(D, C, K2, seeds))
    assert sum(r["n_hypotheses"] > 0 for r in replayed) >= 2
    rel.close()
    fresh.close()
