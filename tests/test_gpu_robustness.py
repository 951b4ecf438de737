"""Robustness inputs (missing depth and depth-dependent noise, reading R22:
every depth image corrupted, training frames and queries) through the CUDA
path against the FP64 oracle: the forest adapted from corrupted frames
(reservoirs and modes bit-exact) and corrupted queries, with and without
ICP, at the usual parity bars."""
import numpy as np
import pytest

import oracle
from synth import workloads
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


@pytest.mark.parametrize("kind,level", [("missing", 0.9), ("noise", 0.05)])
def test_parity_on_corrupted_inputs(rg, ctx, kind, level):
    w = H.WORKLOADS[H.SMALL]
    frames = [(workloads.corrupt(d, kind, level, i), c, T) for i, (d, c, T) in enumerate(w.training_frames())]
    g = rg.Forest.random(ctx, w.forest, w.forest_seed)
    for d, c, T in frames:
        g.adapt(d, c, w.K, T)
    g.update_modes(-1)
    f = H.oracle_forest_nodes(w)
    res = oracle.Reservoirs(f, w.forest["kappa"], w.forest_seed)
    for d, c, T in frames:
        res.add_frame(d, c, w.K, T, w.forest["grid_step"], w.forest["grid_origin"])
    modes = oracle.Modes(res.n_leaves, w.forest["m_max"])
    oracle.update_modes(res, modes, w.forest["sigma"], w.forest["tau_c"], w.forest["min_cluster_size"],
                        cov_eps=w.forest["cov_eps"], fp16_offsets=bool(w.forest["mode_precision"]))
    e = g.export(reservoirs=True)
    assert np.array_equal(e["res_count"], res.count)
    assert np.array_equal(e["nmodes"], modes.nmodes)
    mm = np.arange(w.forest["m_max"])[None, :] < modes.nmodes[:, None]
    assert np.array_equal(e["mode_pos"][mm].view(np.uint32), modes.pos[mm].view(np.uint32))
    room = w.room()
    scene = rg.Scene(ctx, room.lo, room.hi)
    for params in (w.ransac, dict(w.ransac, **workloads.ICP_ON)):
        rel = rg.Relocaliser(g, scene, params, w.width, w.height, 1)
        for q in range(3):
            d, c, T, seed = w.query(q)
            d = workloads.corrupt(d, kind, level, 10000 + q)
            gr = rel.relocalise(d, c, w.K, seed)
            lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=params["n_trees_used"])
            orr = H.OracleRun(params, d, c, w.K, lv, modes, room.lo, room.hi, seed,
                                    1 << w.forest["depth"])
            H.compare_results(rg, gr, rel.debug(0), orr, params, f"{kind} {level} q{q} icp={params.get('icp', 0)}")
        rel.close()
    scene.close()
    g.close()


def test_config2_query_with_90_percent_missing_depth(rg, ctx):
    """A paper-sized query with 90% of its depth masked, against the clean
    config-2 forest: generation mostly draws invalid pixels, the rest of the
    path sees a sparse image."""
    w = workloads.CONFIG2
    g = H.gpu_model(ctx, w)
    f, res, modes = H.oracle_model(w.name)
    room = w.room()
    scene = rg.Scene(ctx, room.lo, room.hi)
    rel = rg.Relocaliser(g, scene, w.ransac, w.width, w.height, 1)
    d, c, T, seed = w.query(3)
    d = workloads.corrupt(d, "missing", 0.9, 10003)
    gr = rel.relocalise(d, c, w.K, seed)
    lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=w.ransac["n_trees_used"])
    orr = H.OracleRun(w.ransac, d, c, w.K, lv, modes, room.lo, room.hi, seed, 1 << w.forest["depth"])
    H.compare_results(rg, gr, rel.debug(0), orr, w.ransac, "config2 missing 0.9")
    rel.close()
    scene.close()
    g.close()


@pytest.mark.parametrize("level", [0.7, 0.9])
def test_redraw_reading_parity(rg, ctx, level):
    """Reading R8b (an unusable generation draw is redrawn within its
    iteration): queries with missing depth against the clean small-case
    forest, every stage compared with the oracle run with the same reading;
    the reading keeps far more hypotheses than R8."""
    w = H.WORKLOADS[H.SMALL]
    g = H.gpu_model(ctx, w)
    f, res, modes = H.oracle_model(w.name)
    room = w.room()
    scene = rg.Scene(ctx, room.lo, room.hi)
    p = dict(w.ransac, redraw=1)
    rel = rg.Relocaliser(g, scene, p, w.width, w.height, 1)
    more = 0
    for q in range(3):
        d, c, T, seed = w.query(q)
        d = workloads.corrupt(d, "missing", level, 10000 + q)
        gr = rel.relocalise(d, c, w.K, seed)
        lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=p["n_trees_used"])
        orr = H.OracleRun(p, d, c, w.K, lv, modes, room.lo, room.hi, seed, 1 << w.forest["depth"])
        H.compare_results(rg, gr, rel.debug(0), orr, p, f"redraw missing {level} q{q}")
        r8 = oracle.relocalise(dict(p, redraw=0), d, c, w.K, lv, modes, room.lo, room.hi, seed,
                               1 << w.forest["depth"])
        more += gr["n_hypotheses"] > 2 * max(1, r8["n_hypotheses"])
    assert more >= 2
    rel.close()
    scene.close()
    g.close()
