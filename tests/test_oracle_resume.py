"""Pins of the oracle's survivor hand-in (orc_relocalise_from) and of its
mode-position writer, which the parity tests use to keep comparing a query
after a legitimate divergence and to build the outlier-mode store of the
precision workload from the oracle's own modes (Sec. 3.2.2-3.2.3)."""
import numpy as np
import pytest

import oracle
from tests import helpers as H
from tests.test_oracle_pins import _brute_energy


@pytest.fixture(scope="module")
def run():
    w = H.WORKLOADS[H.SMALL]
    f, res, modes = H.oracle_model(w.name)
    d, c, T, seed = w.query(0)
    lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=w.ransac["n_trees_used"])
    args = (w.ransac, d, c, w.K, lv, modes, w.room().lo, w.room().hi, seed, 1 << w.forest["depth"])
    r = oracle.relocalise(*args, debug=True)
    assert r["n_hypotheses"] > w.ransac["n_cull"] and r["debug"]["n_rounds"] >= 3
    return w, modes, lv, d, args, r


def _stage_state(dbg, stage):
    """(slots, poses) of the survivor set at a stage boundary of a run."""
    if stage == 0:
        n = int((dbg["cull_slot"] >= 0).sum())
        slots = dbg["cull_slot"][:n]
        return slots, dbg["hyp_pose"][slots]
    off = int(dbg["round_count"][: stage - 1].sum())
    k = int(dbg["round_count"][stage - 1])
    return dbg["round_slot"][off:off + k], dbg["round_pose"][off:off + k]


def test_hand_in_of_own_state_reproduces_the_run(run):
    """Handing the oracle its own survivor set at any stage boundary changes
    nothing: same rounds, chosen set, scores and output."""
    w, modes, lv, d, args, r = run
    dbg = r["debug"]
    for stage in range(dbg["n_rounds"] + 1):
        r2 = oracle.relocalise(*args, debug=True, resume=[(stage,) + _stage_state(dbg, stage)])
        for k in ("pose", "energy", "score", "n_chosen", "best", "chosen_pose", "chosen_score",
                  "chosen_slot", "n_pixels"):
            assert np.array_equal(r[k], r2[k]), (stage, k)
        for k in ("cull_slot", "cull_energy", "round_slot", "round_energy", "round_pose", "round_count"):
            assert np.array_equal(dbg[k], r2["debug"][k]), (stage, k)
    # every stage handed in at once: the same again
    r3 = oracle.relocalise(*args, debug=True,
                           resume=[(st,) + _stage_state(dbg, st) for st in range(dbg["n_rounds"] + 1)])
    assert np.array_equal(r["pose"], r3["pose"]) and np.array_equal(r["chosen_slot"], r3["chosen_slot"])
    assert np.array_equal(dbg["round_pose"], r3["debug"]["round_pose"])


def test_hand_in_replaces_the_survivor_set(run):
    """A survivor set with one member exchanged for a culled hypothesis: the
    oracle continues from exactly that set, ordered by brute-force Eq. 5
    energies on the first batch, and its later rounds keep subsets of it."""
    w, modes, lv, d, args, r = run
    dbg = r["debug"]
    p = dict(oracle.PARAM_DEFAULTS, **w.ransac)
    slots, poses = _stage_state(dbg, 0)
    culled = [s for s in np.nonzero(dbg["hyp_iter"] >= 0)[0] if s not in set(slots)]
    slots = np.array(list(slots[:-1]) + [culled[0]], np.int32)
    poses = dbg["hyp_pose"][slots]
    r2 = oracle.relocalise(*args, debug=True, resume=[(0, slots, poses)])
    d2 = r2["debug"]
    n = len(slots)
    assert sorted(d2["cull_slot"][:n]) == sorted(slots)
    lpt = 1 << w.forest["depth"]
    S_all = np.einsum("...ki,...kj->...ij", _U_full(modes), _U_full(modes))
    pix0 = d2["batch_pix"][0]
    E = np.array([_brute_energy(H.as44(dbg["hyp_pose"][s]), pix0, d, w.K, lv, modes, S_all,
                                p["k_top"], p["use_cov"], lpt) for s in slots])
    order = slots[np.lexsort((slots, E))]
    assert list(d2["cull_slot"][:n]) == list(order)
    np.testing.assert_allclose(d2["cull_energy"][:n], np.sort(E), rtol=1e-12)
    k = d2["round_count"][0]
    assert set(d2["round_slot"][:k]) <= set(slots) and culled[0] in set(d2["cull_slot"][:n])
    # a later hand-in keeps the earlier one: the modified run's own round-1
    # survivors handed in on top reproduce the modified run
    hand = [(0, slots, poses), (2,) + _stage_state(d2, 2)]
    r3 = oracle.relocalise(*args, debug=True, resume=hand)
    assert np.array_equal(r3["pose"], r2["pose"]) and np.array_equal(r3["chosen_slot"], r2["chosen_slot"])
    assert np.array_equal(r3["debug"]["cull_slot"], d2["cull_slot"])


def _U_full(modes):
    u = modes.U.astype(np.float64)
    U = np.zeros(u.shape[:-1] + (3, 3))
    U[..., 0, 0], U[..., 0, 1], U[..., 0, 2] = u[..., 0], u[..., 1], u[..., 2]
    U[..., 1, 1], U[..., 1, 2], U[..., 2, 2] = u[..., 3], u[..., 4], u[..., 5]
    return U


def test_set_mode_positions_encoding():
    """FP32 stores take positions as given; FP16-offset stores keep
    centroid + half(x - centroid) with numpy's IEEE half rounding; ranks
    beyond a leaf's mode count stay untouched."""
    rng = np.random.default_rng(21)
    L, M = 40, 6
    m = oracle.Modes(L, M)
    m.nmodes[:] = rng.integers(0, M + 1, size=L)
    m.centroid[:] = rng.uniform(0, 4, size=(L, 3)).astype(np.float32)
    m.pos[:] = -7.0
    pos = rng.uniform(-1, 11, size=(L, M, 3)).astype(np.float32)
    stored = np.arange(M)[None, :] < m.nmodes[:, None].astype(int)
    for fp16 in (False, True):
        mm = oracle.Modes(L, M)
        mm.nmodes[:] = m.nmodes
        mm.centroid[:] = m.centroid
        mm.pos[:] = -7.0
        oracle.set_mode_positions(mm, pos, fp16)
        c = np.broadcast_to(m.centroid[:, None, :], pos.shape)
        if fp16:
            want = c + np.float16(pos.astype(np.float64) - c.astype(np.float64)).astype(np.float32)
            assert np.abs(want - pos)[stored].max() <= 2.0 ** -8   # offsets below 16 m
        else:
            want = pos
        assert np.array_equal(mm.pos[stored], want[stored])
        assert (mm.pos[~stored] == -7.0).all()
