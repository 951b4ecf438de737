"""Precision and stress (config 5): the config-2 room and forest training,
4096 hypotheses per query, every stored mode of a leaf used (K_top = M_max =
50), 60% of the stored modes moved to points uniform in the room volume, and
leaf modes stored as FP16 offsets from FP32 centroids versus all FP32.

The oracle builds its own mode store: its reservoirs and Really Quick Shift
modes of the config-2 training, the same outlier draw (synth.outliers) on
its own decoded positions, written back in the store's precision by the
oracle.  The library's decoded positions must equal the oracle's bit for
bit, and parity keeps the usual bars; the 5 cm / 5 degree success rate over
200 seeded queries is measured for both storage precisions."""
import numpy as np
import pytest

import oracle
from synth import outliers, workloads
from tests import helpers as H

pytestmark = pytest.mark.gpu
N_ORACLE = 2        # queries recomputed by the FP64 oracle per precision
N_SUCCESS = 200     # queries of the success rate
SUCCESS = {}


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
    return rg.Context(0, arena_bytes=24 << 30)


@pytest.fixture(scope="module")
def queries():
    w = workloads.config5(1)
    return [w.query(q) for q in range(N_SUCCESS)]


@pytest.fixture(scope="module")
def nodes():
    return H.oracle_forest_nodes(workloads.CONFIG2)


def _oracle_modes(w):
    """The oracle's config-5 mode store: config-2 reservoirs clustered in
    the workload's storage precision, 60% of the stored modes moved by the
    outlier draw, positions written back in that precision."""
    f, res, _ = H.oracle_model(workloads.CONFIG2.name)
    fp = w.forest
    modes = oracle.Modes(res.n_leaves, fp["m_max"])
    oracle.update_modes(res, modes, fp["sigma"], fp["tau_c"], fp["min_cluster_size"],
                        cov_eps=fp["cov_eps"], fp16_offsets=bool(fp["mode_precision"]))
    room = w.room()
    pos, hit = outliers.replace_modes(modes.pos, modes.nmodes, room.lo, room.hi,
                                      workloads.CONFIG5_OUTLIER_FRACTION, workloads.CONFIG5_OUTLIER_SEED)
    oracle.set_mode_positions(modes, pos, bool(fp["mode_precision"]))
    return modes


def _success(pose, truth):
    dt, dr = H.pose_err(pose, truth)
    return dt <= 0.05 and dr <= 5.0


@pytest.mark.parametrize("precision", [1, 0], ids=["fp16_offsets", "fp32"])
def test_config5_outlier_modes(rg, ctx, queries, nodes, precision):
    w = workloads.config5(precision)
    room = w.room()
    forest = H.gpu_model(ctx, w)
    ex = forest.export()
    M = w.forest["m_max"]
    stored = np.arange(M)[None, :] < ex["nmodes"][:, None]
    pos, hit = outliers.replace_modes(ex["mode_pos"], ex["nmodes"], room.lo, room.hi,
                                      workloads.CONFIG5_OUTLIER_FRACTION, workloads.CONFIG5_OUTLIER_SEED)
    assert abs(hit.sum() / stored.sum() - 0.6) < 0.01
    forest.set_mode_positions(pos)
    ex2 = forest.export()
    err = np.abs(ex2["mode_pos"] - pos)[stored]
    if precision == 0:
        assert err.max() == 0.0
    else:
        # offsets from the centroid stay below 8 m in a 4 x 3 x 2.5 m room:
        # half an FP16 ulp there is 2^-9 m
        assert err.max() <= 2.0 ** -9
    untouched = stored & ~hit
    assert np.array_equal(ex2["mode_pos"][untouched], ex["mode_pos"][untouched])

    scene = rg.Scene(ctx, room.lo, room.hi)
    # success rate over 200 queries in launches of 64
    rel = rg.Relocaliser(forest, scene, w.ransac, w.width, w.height, 64)
    ok = 0
    for b0 in range(0, N_SUCCESS, 64):
        qs = queries[b0:b0 + 64]
        out = rel.relocalise_batch(np.stack([q[0] for q in qs]), np.stack([q[1] for q in qs]), w.K,
                                   [q[3] for q in qs])
        ok += sum(_success(r["pose"], q[2]) for r, q in zip(out, qs))
    rel.close()
    SUCCESS[precision] = ok / N_SUCCESS
    print(f"config 5 {w.name}: success {ok}/{N_SUCCESS}")

    # the oracle's own store: same modes, same decoded outlier positions
    modes = _oracle_modes(w)
    assert np.array_equal(ex2["nmodes"], modes.nmodes)
    assert np.array_equal(ex2["mode_pos"][stored].view(np.uint32), modes.pos[stored].view(np.uint32))
    assert np.array_equal(ex2["mode_rgb"][stored], modes.rgb[stored])
    np.testing.assert_allclose(ex2["mode_U"][stored], modes.U[stored], rtol=2e-7, atol=0)
    rel1 = rg.Relocaliser(forest, scene, w.ransac, w.width, w.height, 1)
    for q in range(N_ORACLE):
        d, c, T, seed = queries[q]
        gr = rel1.relocalise(d, c, w.K, seed)
        lv = oracle.forest_leaves(nodes, d, c, w.K.fx, n_trees=w.ransac["n_trees_used"])
        orr = H.OracleRun(w.ransac, d, c, w.K, lv, modes, room.lo, room.hi, seed, 1 << w.forest["depth"])
        H.compare_results(rg, gr, rel1.debug(0), orr, w.ransac, f"config5 {w.name} q{q}")
    rel1.close()
    forest.close()


def test_config5_storage_precision_does_not_change_success():
    if len(SUCCESS) < 2:
        pytest.skip("needs both precisions")
    assert abs(SUCCESS[1] - SUCCESS[0]) <= 0.05, SUCCESS
