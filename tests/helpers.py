"""Shared test helpers: run a workload through the CPU oracle and through the
CUDA library, and compare results with the tolerances of the matching rules
(bit-exact integer work; poses 1 mm / 0.05 deg; FP32 energies 1e-4 relative
of FP64; cull survivors equal up to swaps of energies within 1e-5)."""
from __future__ import annotations

import functools
import math

import numpy as np

import oracle
from synth import workloads

POSE_T_TOL = 1e-3                 # metres
POSE_R_TOL = 0.05                 # degrees
ENERGY_RTOL = 1e-4
SWAP_RTOL = 1e-5


def pose_err(A, B):
    A = np.asarray(A)
    B = np.asarray(B)
    dt = float(np.linalg.norm(A[:3, 3] - B[:3, 3]))
    c = (np.trace(A[:3, :3].T @ B[:3, :3]) - 1.0) / 2.0
    return dt, math.degrees(math.acos(min(1.0, max(-1.0, c))))


def as44(p12):
    T = np.eye(4)
    T[:3, :4] = np.asarray(p12).reshape(3, 4)
    return T


def oracle_forest_nodes(w: workloads.Workload):
    f = w.forest
    return oracle.forest_random(f["n_trees"], f["depth"], f["p_depth"], (f["delta_lo"], f["delta_hi"]),
                                (f["tau_depth_lo"], f["tau_depth_hi"]),
                                (f["tau_rgb_lo"], f["tau_rgb_hi"]), bool(f["tau_zero"]),
                                w.forest_seed)


@functools.lru_cache(maxsize=4)
def oracle_model(w_name: str, n_train: int | None = None):
    """Oracle forest, reservoirs and modes of a workload (cached)."""
    w = WORKLOADS[w_name]
    f = oracle_forest_nodes(w)
    res = oracle.Reservoirs(f, w.forest["kappa"], w.forest_seed)
    for i, (d, c, T) in enumerate(w.training_frames()):
        if n_train is not None and i >= n_train:
            break
        res.add_frame(d, c, w.K, T, w.forest["grid_step"], w.forest["grid_origin"])
    modes = oracle.Modes(res.n_leaves, w.forest["m_max"])
    oracle.update_modes(res, modes, w.forest["sigma"], w.forest["tau_c"],
                        w.forest["min_cluster_size"], cov_eps=w.forest["cov_eps"],
                        fp16_offsets=bool(w.forest["mode_precision"]))
    return f, res, modes


def oracle_query(w_name: str, q: int, params=None):
    """(OracleRun of query q of a workload, ground-truth pose)."""
    w = WORKLOADS[w_name]
    f, res, modes = oracle_model(w_name)
    d, c, T, seed = w.query(q)
    p = dict(w.ransac if params is None else params)
    lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=p["n_trees_used"])
    return OracleRun(p, d, c, w.K, lv, modes, w.room().lo, w.room().hi, seed, 1 << w.forest["depth"]), T


WORKLOADS = {w.name: w for w in [workloads.CONFIG1, workloads.CONFIG2, workloads.small_case(),
                                  workloads.small_case(n_trees=6)]}
SMALL = workloads.small_case().name


def gpu_model(ctx, w: workloads.Workload, n_train=None):
    import paper_1810_12163_gb300 as rg
    forest = rg.Forest.random(ctx, w.forest, w.forest_seed)
    for i, (d, c, T) in enumerate(w.training_frames()):
        if n_train is not None and i >= n_train:
            break
        forest.adapt(d, c, w.K, T)
    forest.update_modes(-1)
    return forest


# Per-session counts of the comparisons (printed at the end of a pytest run
# by tests/conftest.py): queries compared, queries compared down to their
# output, survivor sets handed back to the oracle after a legitimate
# divergence, LM trajectories that separated, ICP decisions taken at their
# threshold.
SESSION = dict(queries=0, to_output=0, resumes=0, separations=0, icp_threshold=0, sep_max_energy_gap=0.0)


class OracleRun:
    """The oracle's run of one query together with its inputs, so that a
    comparison can hand the oracle the GPU's survivor set and poses after a
    legitimate divergence and keep comparing what follows (oracle.relocalise
    with resume)."""

    def __init__(self, params, d, c, K, lv, modes, lo, hi, seed, lpt):
        self.args = (params, d, c, K, lv, modes, lo, hi, seed, lpt)
        self.p = dict(oracle.PARAM_DEFAULTS, **params)
        self.d, self.K, self.lv, self.modes, self.lpt = d, K, lv, modes, lpt
        self.handins = []
        self.result = oracle.relocalise(*self.args, debug=True)

    def resume(self, stage, slots, poses):
        """Re-runs the oracle with this survivor set handed in at `stage`,
        on top of every earlier hand-in of this query."""
        self.handins.append((stage, np.array(slots, np.int32), np.array(poses, np.float64)))
        return oracle.relocalise(*self.args, debug=True, resume=self.handins)

    def energy(self, pose12, pix):
        p = self.p
        return oracle.energy(pose12, pix, self.d, self.K, self.lv, self.modes, p["k_top"], p["use_cov"],
                             self.lpt, p["n_trees_used"])


def score_tolerances(gpu_poses, ora_poses, ora_scores, max_range=6.0, incidence=10.0):
    """Tolerance of each Eq. 6 score given how far the two sides' poses are
    apart.  The masked mean |D_l - D_synth| is 1-Lipschitz in D_synth, and a
    rigid motion (dt, dtheta) moves a synthetic z-depth by at most
    (dt + range * dtheta) / cos(incidence); the factor 10 covers incidence
    angles up to 84 degrees.  On top: FP32 summation, 1e-4 relative."""
    tol = []
    for Pg, Po, s in zip(gpu_poses, ora_poses, ora_scores):
        dt, dr = pose_err(Pg, Po)
        pose_term = incidence * (dt + max_range * math.radians(dr))
        tol.append(ENERGY_RTOL * (abs(s) if np.isfinite(s) else 0.0) + pose_term)
    return np.array(tol)


def check_scores(gpu_scores, ora_scores, tol, what):
    g = np.asarray(gpu_scores, np.float64)
    o = np.asarray(ora_scores, np.float64)
    assert np.array_equal(np.isfinite(g), np.isfinite(o)), (what, g, o)
    f = np.isfinite(o)
    assert (np.abs(g[f] - o[f]) <= tol[f]).all(), (what, g, o, tol)


def _energy_close(e_g, e_o):
    return abs(e_g - e_o) <= ENERGY_RTOL * max(abs(e_o), 1e-30) + 1e-6


def compare_survivors(gpu_slots, gpu_E, ora_slots, ora_E, what):
    """Equal survivor sets, allowing swaps between energies within SWAP_RTOL
    of the cut; energies rank by rank within 1e-4 relative.  Returns True
    when the sets are identical."""
    gs, os_ = list(gpu_slots), list(ora_slots)
    assert len(gs) == len(os_), f"{what}: {len(gs)} vs {len(os_)} survivors"
    for e_g, e_o in zip(gpu_E, ora_E):
        assert _energy_close(e_g, e_o), f"{what}: energy {e_g} vs {e_o}"
    if set(gs) == set(os_):
        return True
    cut = max(ora_E)
    for s in set(gs) ^ set(os_):
        e = gpu_E[gs.index(s)] if s in gs else ora_E[os_.index(s)]
        assert abs(e - cut) <= SWAP_RTOL * abs(cut) + 1e-6, f"{what}: survivor {s} differs, E={e} cut={cut}"
    return False


def _by_slot_energies(gpu_slots, gpu_E, ora_slots, ora_E, what):
    """Identical survivor sets; each survivor's energy within 1e-4 relative
    of the oracle's FP64 energy of the same hypothesis."""
    o = {int(s): e for s, e in zip(ora_slots, ora_E)}
    assert set(o) == {int(s) for s in gpu_slots}, (what, sorted(o), sorted(gpu_slots))
    for s, e in zip(gpu_slots, gpu_E):
        assert _energy_close(e, o[int(s)]), f"{what}: slot {s} energy {e} vs {o[int(s)]}"


def compare_results(rg, gr, dbg, orun, params, what):
    """GPU result and debug record of one query against the oracle's
    (an OracleRun), stage by stage, down to the output pose.

    Bars: bit-exact winning iterations and pixel batches; hypothesis poses
    1e-6 m / 1e-4 deg; energies 1e-4 relative; survivor sets equal up to
    swaps of energies within 1e-5 relative of the cut; refined and output
    poses 1 mm / 0.05 deg.  After a legitimate divergence -- a swap at the
    cut, or an LM trajectory that separated along a flat valley of Eq. 5
    after an accept/reject decision fell within FP32 rounding of its
    threshold -- the oracle is handed the GPU's survivor set and poses at
    that stage boundary and the comparison continues at the same bars
    against its re-run.  A separated hypothesis's GPU energy must be within
    1e-4 of the FP64 energy of the GPU's own pose; the gap between the two
    sides' energies is recorded (their end points are different LM outcomes,
    not one pose), and separations may occur in at most one query in ten.
    Returns the counts of this query (also added to SESSION)."""
    assert isinstance(orun, OracleRun)
    rep = dict(resumes=0, separations=0, icp_threshold=0)
    orr = orun.result
    od = orr["debug"]
    SESSION["queries"] += 1
    # generation: identical winning iteration for every slot (bit-exact choices)
    assert np.array_equal(dbg["hyp_iter"], od["hyp_iter"]), what
    for s in np.nonzero(dbg["hyp_iter"] >= 0)[0]:
        dt, dr = pose_err(as44(dbg["hyp_pose"][s]), as44(od["hyp_pose"][s]))
        assert dt < 1e-6 and dr < 1e-4, (what, s, dt, dr)
    assert gr["n_hypotheses"] == orr["n_hypotheses"], what
    if orr["n_hypotheses"] == 0:
        assert gr["status"] == rg.RL_NO_POSE and orr["status"] == 1, what
        SESSION["to_output"] += 1
        return rep
    # pixel batches: bit-exact
    nb = min(16, dbg["n_rounds"] + 1)
    assert np.array_equal(dbg["batch_pix"][:nb], od["batch_pix"][:nb]), what
    # initial cull
    nc = min(params["n_cull"], orr["n_hypotheses"])
    gs, ge = dbg["cull_slot"][:nc], dbg["cull_energy"][:nc]
    if not compare_survivors(gs, ge, od["cull_slot"][:nc], od["cull_energy"][:nc], f"{what} cull"):
        orr = orun.resume(0, gs, od["hyp_pose"][gs])
        od = orr["debug"]
        rep["resumes"] += 1
        _by_slot_energies(gs, ge, od["cull_slot"][:nc], od["cull_energy"][:nc], f"{what} cull (handed in)")
    # preemptive rounds
    assert dbg["n_rounds"] == od["n_rounds"], what
    off = 0
    for r in range(dbg["n_rounds"]):
        k = int(od["round_count"][r])
        assert dbg["round_count"][r] == k, what
        gs, ge, gp = dbg["round_slot"][r][:k], dbg["round_energy"][r][:k], dbg["round_pose"][r][:k]
        os_, oe, op = od["round_slot"][off:off + k], od["round_energy"][off:off + k], od["round_pose"][off:off + k]
        oi = {int(s): i for i, s in enumerate(os_)}
        separated = []
        for i, s in enumerate(gs):
            if int(s) not in oi:
                continue
            j = oi[int(s)]
            dt, dr = pose_err(as44(gp[i]), as44(op[j]))
            if dt > POSE_T_TOL or dr > POSE_R_TOL:
                gap = abs(ge[i] - oe[j]) / abs(oe[j])
                SESSION["sep_max_energy_gap"] = max(SESSION["sep_max_energy_gap"], float(gap))
                separated.append((int(s), dt, dr))
        diverged = bool(separated)
        if not diverged:
            diverged = not compare_survivors(gs, ge, os_, oe, f"{what} round {r}")
        if diverged:
            orr = orun.resume(r + 1, gs, gp)
            od = orr["debug"]
            rep["resumes"] += 1
            rep["separations"] += len(separated)
            _by_slot_energies(gs, ge, od["round_slot"][off:off + k], od["round_energy"][off:off + k],
                              f"{what} round {r} (handed in)")
        off += k
    # the chosen set, matched by generation slot
    assert gr["n_chosen"] == orr["n_chosen"], what
    nch = gr["n_chosen"]
    g_slots = [int(s) for s in gr["chosen_slot"][:nch]]
    o_slots = [int(s) for s in orr["chosen_slot"][:nch]]
    assert sorted(g_slots) == sorted(o_slots), (what, g_slots, o_slots)
    om = [o_slots.index(s) for s in g_slots]          # oracle index of GPU chosen c
    for c, o in enumerate(om):
        assert _energy_close(gr["chosen_energy"][c], orr["chosen_energy"][o]), (what, c)
    icp_same = [True] * nch
    if params.get("icp"):
        mf = dict(oracle.PARAM_DEFAULTS, **params)["icp_min_frac"]
        if params["rank"]:
            for c, o in enumerate(om):
                icp_same[c] = check_icp_one(bool(gr["icp_mask"] >> c & 1), gr["chosen_icp_frac"][c],
                                            gr["chosen_pose"][c], bool(orr["icp_mask"] >> o & 1),
                                            orr["chosen_icp_frac"][o], orr["chosen_pose"][o], mf,
                                            f"{what} chosen {c}")
        else:
            icp_same[0] = check_icp_one(bool(gr["icp_mask"] & 1), gr["chosen_icp_frac"][0], gr["pose"],
                                        bool(orr["icp_mask"] & 1), orr["chosen_icp_frac"][0], orr["pose"],
                                        mf, f"{what} output")
        rep["icp_threshold"] += icp_same.count(False)
    if params["rank"]:
        for c, o in enumerate(om):
            if not icp_same[c]:
                continue
            dt, dr = pose_err(gr["chosen_pose"][c], orr["chosen_pose"][o])
            assert dt <= POSE_T_TOL and dr <= POSE_R_TOL, (what, "chosen", c, dt, dr)
        keep = [c for c in range(nch) if icp_same[c]]
        gsc = np.array([gr["chosen_score"][c] for c in keep])
        osc = np.array([orr["chosen_score"][om[c]] for c in keep])
        tol = score_tolerances([gr["chosen_pose"][c] for c in keep],
                               [orr["chosen_pose"][om[c]] for c in keep], osc)
        check_scores(gsc, osc, tol, what)
        gb, ob = gr["best"], orr["best"]
        if g_slots[gb] != o_slots[ob]:
            # argmin between near-tied scores (or a pose whose ICP decision
            # fell at its threshold): either choice is valid
            a, b = om[gb], ob
            if icp_same[gb] and icp_same[om.index(ob)]:
                ta = tol[keep.index(gb)]
                tb = tol[keep.index(om.index(ob))]
                assert abs(orr["chosen_score"][a] - orr["chosen_score"][b]) <= ta + tb, (what, a, b)
        # the output is the GPU's chosen pose xi* and its RANSAC energy
        assert np.array_equal(gr["pose"], gr["chosen_pose"][gb]), what
        o_out_pose, o_out_E = orr["chosen_pose"][om[gb]], orr["chosen_energy"][om[gb]]
        out_same = icp_same[gb]
    else:
        o_out_pose, o_out_E = orr["pose"], orr["energy"]
        out_same = icp_same[0] if params.get("icp") else True
    np.testing.assert_allclose(gr["energy"], o_out_E, rtol=ENERGY_RTOL, err_msg=what)
    if out_same:
        dt, dr = pose_err(gr["pose"], o_out_pose)
        assert dt <= POSE_T_TOL and dr <= POSE_R_TOL, (what, "output", dt, dr)
    SESSION["to_output"] += 1
    for k in ("resumes", "separations", "icp_threshold"):
        SESSION[k] += rep[k]
    # separations stay rare: at most one query in ten (and three per session
    # below thirty queries)
    assert SESSION["separations"] <= max(3, SESSION["queries"] // 10), SESSION
    return rep


ICP_FRAC_TOL = 1e-3   # inlier fractions: a few pixels at the inlier radius flip in FP32


def oracle_icp_kwargs(p: dict) -> dict:
    """oracle.icp_refine keywords from icp_* parameters."""
    d = dict(oracle.PARAM_DEFAULTS, **p)
    return dict(levels=d["icp_levels"], stride=d["icp_stride"], iters=d["icp_iters"],
                dist=d["icp_dist"], min_frac=d["icp_min_frac"], ridge=d["icp_ridge"])


def check_icp_one(ok_g, frac_g, P_g, ok_o, frac_o, P_o, min_frac, what):
    """One ICP run, GPU vs oracle: inlier fractions within ICP_FRAC_TOL; the
    success decision equal unless the oracle's fraction lies within that
    tolerance of the threshold; refined poses within 1 mm / 0.05 deg.
    Returns True when both sides took the same decision."""
    assert abs(frac_g - frac_o) <= ICP_FRAC_TOL, (what, frac_g, frac_o)
    if ok_g != ok_o:
        assert abs(frac_o - min_frac) <= ICP_FRAC_TOL, (what, ok_g, ok_o, frac_o)
        return False
    dt, dr = pose_err(P_g, P_o)
    assert dt <= POSE_T_TOL and dr <= POSE_R_TOL, (what, dt, dr)
    return True
