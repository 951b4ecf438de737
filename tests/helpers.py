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


def oracle_query(w_name: str, q: int, params=None, debug=True):
    w = WORKLOADS[w_name]
    f, res, modes = oracle_model(w_name)
    d, c, T, seed = w.query(q)
    p = dict(w.ransac if params is None else params)
    lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=p["n_trees_used"])
    r = oracle.relocalise(p, d, c, w.K, lv, modes, w.room().lo, w.room().hi, seed,
                          1 << w.forest["depth"], debug=debug)
    return r, T


WORKLOADS = {w.name: w for w in [workloads.CONFIG1, workloads.CONFIG2, workloads.small_case()]}
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


LM_SEPARATIONS = []


def check_refined_pose(dt, dr, e_gpu, e_ora, what):
    """Poses after LM agree within 1 mm / 0.05 deg.  LM is iterative and
    non-smooth (inlier set and accept/reject decisions): when such a decision
    falls within FP32 rounding of its threshold, the FP32-accumulated GPU
    trajectory and the FP64 oracle trajectory of a hypothesis with few
    inliers can separate along a flat direction of Eq. 5.  Then the pose is
    not unique and the test checks what is: both poses have the same energy
    (1e-4 relative), and such separations stay rare."""
    if dt <= POSE_T_TOL and dr <= POSE_R_TOL:
        return
    assert abs(e_gpu - e_ora) <= ENERGY_RTOL * abs(e_ora), (what, dt, dr, e_gpu, e_ora)
    LM_SEPARATIONS.append((what, dt, dr))
    assert len(LM_SEPARATIONS) <= 3, LM_SEPARATIONS


SEP_ENERGY_RTOL = 1e-3


def lm_separated(gpu_poses, ora_poses, gpu_slots, ora_slots, gpu_E, ora_E, what):
    """True when a survivor's LM trajectory separated from the oracle's: the
    same hypothesis at the same rank ends more than 1 mm / 0.05 deg away.
    After an accept/reject decision falls within FP32 rounding of its
    threshold, the two trajectories continue from different points of a flat
    valley of Eq. 5 and end at different poses, so their energies are no
    longer those of one pose: they must agree within SEP_ENERGY_RTOL, the
    separation counts toward the session's limit and the comparison of this
    query stops (what follows from it differs legitimately)."""
    for i, (sg, so) in enumerate(zip(gpu_slots, ora_slots)):
        if sg != so:
            continue
        dt, dr = pose_err(as44(gpu_poses[i]), as44(ora_poses[i]))
        if dt <= POSE_T_TOL and dr <= POSE_R_TOL:
            continue
        assert abs(gpu_E[i] - ora_E[i]) <= SEP_ENERGY_RTOL * abs(ora_E[i]), (what, i, dt, dr, gpu_E[i], ora_E[i])
        LM_SEPARATIONS.append((what, dt, dr))
        assert len(LM_SEPARATIONS) <= 3, LM_SEPARATIONS
        return True
    return False


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


def compare_survivors(gpu_slots, gpu_E, ora_slots, ora_E, what):
    """Equal survivor sets, allowing swaps between energies within SWAP_RTOL
    of the cut.  Returns True when the sets are identical."""
    gs, os_ = list(gpu_slots), list(ora_slots)
    assert len(gs) == len(os_), f"{what}: {len(gs)} vs {len(os_)} survivors"
    for e_g, e_o in zip(gpu_E, ora_E):
        assert abs(e_g - e_o) <= ENERGY_RTOL * max(abs(e_o), 1e-30) + 1e-6, \
            f"{what}: energy {e_g} vs {e_o}"
    if set(gs) == set(os_):
        return True
    cut = max(ora_E)
    for s in set(gs) ^ set(os_):
        e = gpu_E[gs.index(s)] if s in gs else ora_E[os_.index(s)]
        assert abs(e - cut) <= SWAP_RTOL * abs(cut) + 1e-6, f"{what}: survivor {s} differs, E={e} cut={cut}"
    return False


def compare_results(rg, gr, dbg, orr, params, what):
    """GPU result and debug record of one query against the oracle's, with
    the bars stated in the module docstring."""
    od = orr["debug"]
    # generation: identical winning iteration for every slot (bit-exact choices)
    assert np.array_equal(dbg["hyp_iter"], od["hyp_iter"])
    ok = dbg["hyp_iter"] >= 0
    for s in np.nonzero(ok)[0]:
        dt, dr = pose_err(as44(dbg["hyp_pose"][s]), as44(od["hyp_pose"][s]))
        assert dt < 1e-6 and dr < 1e-4, (what, s, dt, dr)
    assert gr["n_hypotheses"] == orr["n_hypotheses"]
    if orr["n_hypotheses"] == 0:
        assert gr["status"] == rg.RL_NO_POSE and orr["status"] == 1
        return
    # batch pixels: bit-exact
    nb = min(16, dbg["n_rounds"] + 1)
    assert np.array_equal(dbg["batch_pix"][:nb], od["batch_pix"][:nb])
    # cull survivors
    nc = min(params["n_cull"], orr["n_hypotheses"])
    same = compare_survivors(dbg["cull_slot"][:nc], dbg["cull_energy"][:nc],
                             od["cull_slot"][:nc], od["cull_energy"][:nc], f"{what} cull")
    if not same:
        return
    # preemptive rounds
    assert dbg["n_rounds"] == od["n_rounds"]
    off = 0
    for r in range(dbg["n_rounds"]):
        k = od["round_count"][r]
        assert dbg["round_count"][r] == k
        gs, ge = dbg["round_slot"][r][:k], dbg["round_energy"][r][:k]
        os_, oe = od["round_slot"][off:off + k], od["round_energy"][off:off + k]
        if lm_separated(dbg["round_pose"][r][:k], od["round_pose"][off:off + k], gs, os_, ge, oe,
                        f"{what} round {r}"):
            return
        if not compare_survivors(gs, ge, os_, oe, f"{what} round {r}"):
            return
        for i in range(k):
            dt, dr = pose_err(as44(dbg["round_pose"][r][i]), as44(od["round_pose"][off + i]))
            check_refined_pose(dt, dr, ge[i], oe[i], f"{what} round {r} survivor {i}")
        off += k
    # ranking scores of the chosen set, then the output pose
    assert gr["n_chosen"] == orr["n_chosen"]
    if params.get("icp") and not check_icp(gr, orr, params, what):
        return
    if params["rank"]:
        tol = score_tolerances(gr["chosen_pose"], orr["chosen_pose"], orr["chosen_score"])
        check_scores(gr["chosen_score"], orr["chosen_score"], tol, what)
        if gr["best"] != orr["best"]:
            # argmin between near-tied scores: either choice is valid
            a, b = gr["best"], orr["best"]
            assert abs(orr["chosen_score"][a] - orr["chosen_score"][b]) <= tol[a] + tol[b], (what, a, b)
            return
    dt, dr = pose_err(gr["pose"], orr["pose"])
    np.testing.assert_allclose(gr["energy"], orr["energy"], rtol=ENERGY_RTOL)
    check_refined_pose(dt, dr, gr["energy"], orr["energy"], f"{what} output")


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


def check_icp(gr, orr, params, what):
    """ICP outputs of a relocalisation (ranked: every chosen pose;
    unranked: the output pose).  False when a success decision differs at
    the threshold (what follows from it then differs legitimately)."""
    mf = dict(oracle.PARAM_DEFAULTS, **params)["icp_min_frac"]
    if params["rank"]:
        same = True
        for c in range(gr["n_chosen"]):
            same &= check_icp_one(bool(gr["icp_mask"] >> c & 1), gr["chosen_icp_frac"][c], gr["chosen_pose"][c],
                                  bool(orr["icp_mask"] >> c & 1), orr["chosen_icp_frac"][c], orr["chosen_pose"][c],
                                  mf, f"{what} chosen {c}")
        return same
    return check_icp_one(bool(gr["icp_mask"] & 1), gr["chosen_icp_frac"][0], gr["pose"],
                         bool(orr["icp_mask"] & 1), orr["chosen_icp_frac"][0], orr["pose"], mf, f"{what} output")


def oracle_modes_from_export(ex, m_max):
    """Oracle mode store holding exactly the library's decoded modes (both
    sides then score the same mode positions)."""
    L = ex["nmodes"].shape[0]
    m = oracle.Modes(L, m_max)
    m.nmodes[:] = ex["nmodes"]
    m.pos[:] = ex["mode_pos"]
    m.rgb[:] = ex["mode_rgb"]
    m.U[:] = ex["mode_U"]
    m.size[:] = ex["mode_size"]
    return m
