"""Pins of the CPU oracle to facts outside itself: published known-answer
vectors, hand-computed fixtures, closed forms, independent numpy
re-derivations (Horn's quaternion method, brute-force energies, a numpy
renderer), statistical properties (Algorithm R's unbiasedness) and
invariants of the method (cull keeps the lowest energies, halving, argmin
ranking, the cascade's fall-back rule).  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
from synth import rooms, workloads
from tests import helpers as H
from tests import philox_ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]
        assert list(philox_ref.philox4x32_10(v[0:4], v[4:6])) == v[6:10]


# ---------------------------------------------------------------- forest factory
def test_forest_random_distribution():
    f = oracle.forest_random(5, 12, 0.4, (-130.0, 130.0), (-0.2, 0.2), (-50.0, 50.0), False, 2)
    n = f["type"].size
    frac = (f["type"] == 0).mean()
    assert abs(frac - 0.4) < 4 * math.sqrt(0.24 / n)           # Depth with probability p
    assert f["dx"].min() >= -130 and f["dx"].max() < 130
    for a in (f["dx"], f["dy"]):                                 # uniform offsets
        h, _ = np.histogram(a, bins=10, range=(-130, 130))
        chi2 = ((h - n / 10) ** 2 / (n / 10)).sum()
        assert chi2 < 30
    rgb = f["type"] == 1
    h = np.bincount(f["channel"][rgb], minlength=3)
    assert h.size == 3 and ((h - rgb.sum() / 3) ** 2 / (rgb.sum() / 3)).sum() < 15
    assert (f["channel"][~rgb] == 0).all()
    td = f["tau"][~rgb]
    tr = f["tau"][rgb]
    assert td.min() >= -0.2 and td.max() < 0.2 and tr.min() >= -50 and tr.max() < 50
    assert abs(np.corrcoef(f["dx"], f["dy"])[0, 1]) < 0.05         # independent offsets
    z = oracle.forest_random(1, 6, 0.4, tau_zero=True, seed=9)
    assert (z["tau"] == 0).all()
    # all-depth and all-colour forests
    assert (oracle.forest_random(1, 8, 1.0, seed=1)["type"] == 0).all()
    assert (oracle.forest_random(1, 8, 0.0, seed=1)["type"] == 1).all()


def test_forest_nodes_rederived_with_independent_philox():
    """Reading R2 node by node: node n of tree t draws Philox blocks at
    counters (t, 1 << 16, n, 0) and (t, 1 << 16, n, 1); Depth iff
    r0[0] < p 2^32; dx, dy from r0[1], r0[2] and the channel from r0[3]; tau
    from r1[0]; uniforms are the top 24 bits scaled to [0, 1) in FP32."""
    lo, hi, tlo, thi, clo, chi = -130.0, 130.0, -0.2, 0.2, -50.0, 50.0
    seed = 0x1234_5678_9ABC
    f = oracle.forest_random(3, 7, 0.4, (lo, hi), (tlo, thi), (clo, chi), False, seed)
    key = philox_ref.key_of(seed)
    f32 = np.float32

    def uni(u):
        return f32((int(u) >> 8) * 2.0 ** -24)

    nb = (1 << 7) - 1
    for t in range(3):
        for n in range(0, nb, 5):
            r0 = philox_ref.philox4x32_10((t, 1 << 16, n, 0), key)
            r1 = philox_ref.philox4x32_10((t, 1 << 16, n, 1), key)
            i = t * nb + n
            depth = r0[0] < 0.4 * 4294967296.0
            assert f["type"][i] == (0 if depth else 1)
            span = f32(hi) - f32(lo)
            assert f["dx"][i] == f32(lo) + span * uni(r0[1]) and f["dy"][i] == f32(lo) + span * uni(r0[2])
            assert f["channel"][i] == (0 if depth else philox_ref.below(r0[3], 3))
            a, b = (tlo, thi) if depth else (clo, chi)
            assert f["tau"][i] == f32(a) + (f32(b) - f32(a)) * uni(r1[0])


# ---------------------------------------------------------------- Eq. 1-3
def _probe_image():
    D = np.array([[1, 1, 1, 1], [1, 2, 2, 1], [1, 2, 2, 0], [1, 1, 1, 1]], np.float32)
    C = np.zeros((4, 4, 3), np.uint8)
    for y in range(4):
        for x in range(4):
            for c in range(3):
                C[y, x, c] = 10 * y + x + 100 * c
    return D, C


def test_feature_golden():
    D, C = _probe_image()
    rows = [l.split("#")[0].split() for l in open(os.path.join(GOLDEN, "feature_probes.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 8
    for r in rows:
        fx, x, y, dx, dy, t, ch = float(r[0]), int(r[1]), int(r[2]), float(r[3]), float(r[4]), int(r[5]), int(r[6])
        want = float(r[9])
        assert oracle.feature(dx, dy, t, ch, D, C, fx, x, y) == want, r


def test_forest_walk_golden():
    """Depth-2 tree: root Depth split, children DA-RGB splits (heap order,
    true -> 2n+2).  Hand-computed leaves for three pixels."""
    D, C = _probe_image()
    f = dict(dx=np.array([4.0, 0.0, 2.0], np.float32), dy=np.array([4.0, 0.0, 0.0], np.float32),
             tau=np.array([0.5, 0.0, -5.0], np.float32), type=np.array([0, 1, 1], np.uint8),
             channel=np.array([0, 0, 2], np.uint8), n_trees=1, depth=2)
    lv = oracle.forest_leaves(f, D, C, 585.0)[0]
    # p=(1,1): root f = 2 - D(3,3)=1 = 1 >= 0.5 -> node 2; node 2 probe x:
    # floor(1 + 2*0.5 + 0.5) = 2 -> C(1,1,2)=211 - C(2,1,2)=212 = -1 >= -5 -> node 6 -> leaf 3
    assert lv[1, 1] == 3
    # p=(0,0): D=1, root probe (4,4)->clamped (3,3): 1-1 = 0 < 0.5 -> node 1;
    # node 1: offset 0 -> f = 0 >= 0 -> node 4 -> leaf 1
    assert lv[0, 0] == 1
    # p=(3,2): no depth -> no leaf
    assert lv[2, 3] == 0xFFFF


# ---------------------------------------------------------------- Kabsch
def _horn(a, b):
    ac, bc = a - a.mean(0), b - b.mean(0)
    S = ac.T @ bc
    Sxx, Sxy, Sxz = S[0]; Syx, Syy, Syz = S[1]; Szx, Szy, Szz = S[2]
    N = np.array([[Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx],
                  [Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz],
                  [Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy],
                  [Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz]])
    q = np.linalg.eigh(N)[1][:, -1]
    q0, q1, q2, q3 = q / np.linalg.norm(q)
    R = np.array([[q0*q0+q1*q1-q2*q2-q3*q3, 2*(q1*q2-q0*q3), 2*(q1*q3+q0*q2)],
                  [2*(q1*q2+q0*q3), q0*q0-q1*q1+q2*q2-q3*q3, 2*(q2*q3-q0*q1)],
                  [2*(q1*q3-q0*q2), 2*(q2*q3+q0*q1), q0*q0-q1*q1-q2*q2+q3*q3]])
    return R, b.mean(0) - R @ a.mean(0)


def test_kabsch_exact_recovery():
    rng = np.random.default_rng(0)
    for n in (3, 4, 10):
        for _ in range(50):
            R = _rot(rng.normal(size=3), rng.uniform(0, math.pi))
            t = rng.normal(size=3)
            a = rng.normal(size=(n, 3))
            b = a @ R.T + t
            Re, te = oracle.kabsch(a, b)
            assert np.abs(Re - R).max() < 1e-12 and np.abs(te - t).max() < 1e-12


def test_kabsch_matches_horn_on_noisy_pairs():
    rng = np.random.default_rng(1)
    for n in (3, 5, 20):
        for _ in range(50):
            R = _rot(rng.normal(size=3), rng.uniform(0, math.pi))
            a = rng.normal(size=(n, 3))
            b = a @ R.T + rng.normal(size=3) + 0.05 * rng.normal(size=(n, 3))
            Re, te = oracle.kabsch(a, b)
            Rh, th = _horn(a, b)
            assert abs(np.linalg.det(Re) - 1) < 1e-12
            assert np.abs(Re - Rh).max() < 1e-9 and np.abs(te - th).max() < 1e-9


def test_kabsch_reflection_is_rejected():
    """Mirror-image point sets: the least-squares rotation (det +1), never
    the reflection, must come out."""
    rng = np.random.default_rng(2)
    a = rng.normal(size=(6, 3))
    b = a * np.array([1, 1, -1.0])
    Re, te = oracle.kabsch(a, b)
    Rh, th = _horn(a, b)
    assert abs(np.linalg.det(Re) - 1) < 1e-12
    assert np.abs(Re - Rh).max() < 1e-8


# ---------------------------------------------------------------- Eq. 5
def _tiny_model(rng, W=8, Hh=6, T=2, lpt=16, m_max=5, k_top=3):
    depth = rng.uniform(0.8, 3.0, size=(Hh, W)).astype(np.float32)
    depth[0, 0] = 0.0
    leaves = rng.integers(0, lpt, size=(T, Hh, W)).astype(np.uint16)
    leaves[:, 0, 0] = 0xFFFF
    modes = oracle.Modes(T * lpt, m_max)
    modes.nmodes[:] = rng.integers(0, m_max + 1, size=T * lpt)
    modes.pos[:] = rng.uniform(-1, 4, size=modes.pos.shape).astype(np.float32)
    S_all = np.zeros((T * lpt, m_max, 3, 3))
    for L in range(T * lpt):
        for m in range(m_max):
            A = rng.normal(size=(3, 3)) * 0.05
            cov = A @ A.T + 1e-3 * np.eye(3)
            S = np.linalg.inv(cov)
            U = np.linalg.cholesky(S).T                      # U^T U = S
            modes.U[L, m] = [U[0, 0], U[0, 1], U[0, 2], U[1, 1], U[1, 2], U[2, 2]]
            Uf = modes.U[L, m].astype(np.float64)
            Uq = np.array([[Uf[0], Uf[1], Uf[2]], [0, Uf[3], Uf[4]], [0, 0, Uf[5]]])
            S_all[L, m] = Uq.T @ Uq                           # exactly what is stored
    return depth, leaves, modes, S_all


def _brute_energy(H4, pix, depth, K, leaves, modes, S_all, k_top, use_cov, lpt):
    W = depth.shape[1]
    E = 0.0
    for p in pix:
        if p < 0:
            continue
        u, v = p % W, p // W
        d = np.float32(depth.flat[p])
        xc = np.array([np.float32((np.float32(u) - np.float32(K.cx)) * d) / np.float32(K.fx),
                       np.float32((np.float32(v) - np.float32(K.cy)) * d) / np.float32(K.fy), d], np.float64)
        y = H4[:3, :3] @ xc + H4[:3, 3]
        best = np.inf
        for t in range(leaves.shape[0]):
            L = t * lpt + int(leaves[t].flat[p])
            for m in range(min(int(modes.nmodes[L]), k_top)):
                v_ = y - modes.pos[L, m].astype(np.float64)
                q = v_ @ S_all[L, m] @ v_ if use_cov else v_ @ v_
                best = min(best, q)
        E += math.sqrt(best)
    return E


def _twist(xi):
    v, w = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    X = np.zeros((4, 4))
    X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    X[:3, 3] = v
    return X


@pytest.mark.parametrize("theta", [0.0, 1e-9, 1e-3, 0.3, 2.5])
def test_se3_left_update_is_the_matrix_exponential(theta):
    """The LM update exp(xi^) H of Sec. 3.2.3 against scipy's matrix
    exponential of the 4x4 twist: a non-identity H tells a left update from a
    right one, distinct v and w tell their order, and the angles span the
    small-angle branch and the closed form."""
    expm = pytest.importorskip("scipy.linalg").expm
    rng = np.random.default_rng(7)
    H0 = np.eye(4)
    H0[:3, :3] = _rot(rng.normal(size=3), 0.7)
    H0[:3, 3] = [1.5, -0.4, 2.0]
    axis = rng.normal(size=3)
    xi = np.concatenate([[0.03, -0.02, 0.05], theta * axis / np.linalg.norm(axis)])
    got = oracle.se3_left_update(xi, H0)
    want = expm(_twist(xi)) @ H0
    assert np.abs(got - want).max() < 1e-12
    np.testing.assert_allclose(got[:3, :3] @ got[:3, :3].T, np.eye(3), atol=1e-12)


def test_cholesky_solve_matches_numpy_and_rejects_indefinite():
    rng = np.random.default_rng(11)
    for _ in range(20):
        M = rng.normal(size=(6, 6))
        A = M @ M.T + 0.1 * np.eye(6)
        b = rng.normal(size=6)
        x = oracle.chol_solve6(A, b)
        np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)
    A = np.diag([1.0, 2.0, 3.0, -1e-3, 5.0, 6.0])
    assert oracle.chol_solve6(A, np.ones(6)) is None
    assert oracle.chol_solve6(np.zeros((6, 6)), np.ones(6)) is None


def test_energy_brute_force():
    rng = np.random.default_rng(3)
    depth, leaves, modes, S_all = _tiny_model(rng)
    K = rooms.Intrinsics(5.0, 5.5, 3.7, 2.4, 8, 6)
    valid = [p for p in range(48) if depth.flat[p] > 0 and
             sum(min(int(modes.nmodes[t * 16 + int(leaves[t].flat[p])]), 3) for t in range(2)) > 0]
    pix = np.array(valid[:30] + [-1], np.int32)
    for trial in range(5):
        H4 = np.eye(4)
        H4[:3, :3] = _rot(rng.normal(size=3), rng.uniform(0, 3))
        H4[:3, 3] = rng.normal(size=3)
        for use_cov in (0, 1):
            e = oracle.energy(H4, pix, depth, K, leaves, modes, 3, use_cov, 16)
            b = _brute_energy(H4, pix, depth, K, leaves, modes, S_all, 3, use_cov, 16)
            assert abs(e - b) <= 1e-9 * max(1.0, b), (use_cov, e, b)


def _exact_room_model(w, pose, n_pix=64, extra_modes=3, seed=0):
    """Modes that contain the exact world point of each pixel (plus
    distractors), built directly from a noise-free render."""
    rng = np.random.default_rng(seed)
    K = w.K
    d, c = rooms.render(w.room(), K, pose, noise_sigma=0.0)
    Hh, W = d.shape
    pix = rng.choice(Hh * W, size=n_pix, replace=False).astype(np.int32)
    leaves = np.zeros((1, Hh, W), np.uint16)
    modes = oracle.Modes(n_pix, 1 + extra_modes)
    for i, p in enumerate(pix):
        leaves[0].flat[p] = i
        u, v = p % W, p // W
        dd = np.float32(d.flat[p])
        xc = np.array([np.float32((np.float32(u) - np.float32(K.cx)) * dd) / np.float32(K.fx),
                       np.float32((np.float32(v) - np.float32(K.cy)) * dd) / np.float32(K.fy), dd])
        xw = pose[:3, :3] @ xc + pose[:3, 3]
        modes.nmodes[i] = 1 + extra_modes
        modes.pos[i, 0] = xw
        modes.pos[i, 1:] = xw + rng.normal(size=(extra_modes, 3)) * 0.5
        modes.U[i] = [20.0, 0, 0, 20.0, 0, 20.0]
    return d, c, leaves, modes, pix


def test_ground_truth_is_energy_minimum_and_lm_converges():
    w = workloads.CONFIG1
    rng = np.random.default_rng(4)
    gt = rooms.look_pose([1.7, 1.4, 1.2], 0.4, 0.1)
    d, c, leaves, modes, pix = _exact_room_model(w, gt)
    for use_cov in (0, 1):
        e0 = oracle.energy(gt, pix, d, w.K, leaves, modes, 4, use_cov, leaves_per_tree=pix.size)
        assert e0 < 1e-4 * pix.size                            # exact modes (FP32 rounding only)
        for _ in range(10):
            xi = rng.normal(size=6) * np.array([0.01, 0.01, 0.01, 0.01, 0.01, 0.01])
            P = np.eye(4)
            P[:3, :3] = _rot(xi[3:], np.linalg.norm(xi[3:])) @ gt[:3, :3]
            P[:3, 3] = gt[:3, 3] + xi[:3]
            assert oracle.energy(P, pix, d, w.K, leaves, modes, 4, use_cov, pix.size) > e0
            Pr, it = oracle.lm_refine(P, pix, d, w.K, leaves, modes, 4, use_cov, pix.size,
                                      max_iter=20)
            dt, dr = H.pose_err(Pr, gt)
            assert dt < 1e-5 and dr < 1e-3, (use_cov, dt, dr, it)


def _noisy_lm_case():
    """64 pixels of a noise-free render, one mode each at the exact world
    point plus 1 cm noise, anisotropic precision factors U; the camera points
    X, means MU, factors Um (3x3) and a start pose 6 mm / 0.23 deg away."""
    w = workloads.CONFIG1
    rng = np.random.default_rng(21)
    gt = rooms.look_pose([1.7, 1.4, 1.2], 0.4, 0.1)
    d, c, leaves, modes, pix = _exact_room_model(w, gt, n_pix=64, extra_modes=0)
    modes.pos[:, 0] += (rng.normal(size=(pix.size, 3)) * 0.01).astype(np.float32)
    U = np.zeros((pix.size, 6), np.float32)
    U[:, [0, 3, 5]] = rng.uniform(10.0, 40.0, size=(pix.size, 3))
    U[:, [1, 2, 4]] = rng.uniform(-5.0, 5.0, size=(pix.size, 3))
    modes.U[:, 0] = U
    K = w.K
    Hh, W = d.shape
    xs = []
    for p in pix:
        u, v, dd = p % W, p // W, np.float32(d.flat[p])
        xs.append([np.float32((np.float32(u) - np.float32(K.cx)) * dd) / np.float32(K.fx),
                   np.float32((np.float32(v) - np.float32(K.cy)) * dd) / np.float32(K.fy), dd])
    X = np.array(xs, np.float64)
    MU = modes.pos[:, 0].astype(np.float64)
    Um = np.zeros((pix.size, 3, 3))
    Um[:, 0, :] = U[:, 0:3]
    Um[:, 1, 1:] = U[:, 3:5]
    Um[:, 2, 2] = U[:, 5]
    P0 = np.eye(4)
    P0[:3, :3] = _rot([0.3, -0.5, 0.8], 0.004) @ gt[:3, :3]
    P0[:3, 3] = gt[:3, 3] + [0.006, -0.004, 0.005]
    return d, K, leaves, modes, pix, X, MU, Um, P0


def test_lm_reaches_the_weighted_least_squares_optimum():
    """LM (Sec. 3.2.3) on noisy modes with anisotropic precision factors U:
    its end point is the minimiser of sum |U (H x - mu)|^2 found by scipy's
    trust-region least squares (pose update through scipy's expm).  The two
    optima with and without U differ, so a wrong weighting, Jacobian or
    update fails."""
    so = pytest.importorskip("scipy.optimize")
    expm = pytest.importorskip("scipy.linalg").expm
    d, K, leaves, modes, pix, X, MU, Um, P0 = _noisy_lm_case()

    def optimum(weighted):
        def res(xi):
            Pn = expm(_twist(xi)) @ P0
            e = X @ Pn[:3, :3].T + Pn[:3, 3] - MU
            return (np.einsum("nij,nj->ni", Um, e) if weighted else e).ravel()
        r = so.least_squares(res, np.zeros(6), method="trf", x_scale="jac", xtol=1e-15, ftol=1e-15, gtol=1e-15)
        return expm(_twist(r.x)) @ P0

    P_w, P_u = optimum(True), optimum(False)
    dt, dr = H.pose_err(P_w, P_u)
    assert dt > 2e-4                      # the weighting moves the optimum
    P_lm, it = oracle.lm_refine(P0, pix, d, K, leaves, modes, 1, 1, pix.size, max_iter=50, stop=1e-12)
    dt, dr = H.pose_err(P_lm, P_w)
    assert dt < 1e-7 and dr < 1e-5, (dt, dr, it)
    P_lm0, _ = oracle.lm_refine(P0, pix, d, K, leaves, modes, 1, 0, pix.size, max_iter=50, stop=1e-12)
    dt, dr = H.pose_err(P_lm0, P_u)
    assert dt < 1e-7 and dr < 1e-5, (dt, dr)


def test_lm_first_step_is_the_marquardt_damped_step():
    """One LM iteration from P0: xi solves (A + lambda diag(A)) xi = -g with
    A = sum J^T J, g = sum J^T r, r = U (y - mu), J = U [I | -[y]x] (left
    perturbation, y = H x), and the accepted pose is exp(xi^) P0.  Written
    here from the definitions; lambda = 1 makes the damping form matter."""
    expm = pytest.importorskip("scipy.linalg").expm
    d, K, leaves, modes, pix, X, MU, Um, P0 = _noisy_lm_case()
    Y = X @ P0[:3, :3].T + P0[:3, 3]
    r = np.einsum("nij,nj->ni", Um, Y - MU)
    Jp = np.zeros((len(Y), 3, 6))
    Jp[:, :, :3] = np.eye(3)
    Jp[:, 0, 4], Jp[:, 0, 5] = Y[:, 2], -Y[:, 1]
    Jp[:, 1, 3], Jp[:, 1, 5] = -Y[:, 2], Y[:, 0]
    Jp[:, 2, 3], Jp[:, 2, 4] = Y[:, 1], -Y[:, 0]
    J = np.einsum("nij,njk->nik", Um, Jp)
    A = np.einsum("nij,nik->jk", J, J)
    g = np.einsum("nij,ni->j", J, r)
    lam = 1.0
    xi = np.linalg.solve(A + lam * np.diag(np.diag(A)), -g)
    P1 = expm(_twist(xi)) @ P0
    r1 = np.einsum("nij,nj->ni", Um, X @ P1[:3, :3].T + P1[:3, 3] - MU)
    assert (r1 ** 2).sum() < (r ** 2).sum()          # the step is accepted
    xi_lev = np.linalg.solve(A + lam * np.eye(6), -g)
    assert np.abs(xi_lev - xi).max() > 1e-4          # the damping form matters here
    P_lm, it = oracle.lm_refine(P0, pix, d, K, leaves, modes, 1, 1, pix.size, max_iter=1, lambda0=lam,
                                stop=1e-15)
    assert np.abs(P_lm - P1).max() < 1e-12


def test_lm_needs_three_inliers():
    w = workloads.CONFIG1
    gt = rooms.look_pose([1.7, 1.4, 1.2], 0.4, 0.1)
    d, c, leaves, modes, pix = _exact_room_model(w, gt, n_pix=2, extra_modes=0)
    P = gt.copy()
    P[:3, 3] += 0.01
    Pr, it = oracle.lm_refine(P, pix, d, w.K, leaves, modes, 1, 0, pix.size)
    assert np.array_equal(Pr, P) and it == 0


# ---------------------------------------------------------------- reservoirs
def _single_leaf_forest():
    # offset 0 -> feature D(p)-D(p) = 0 < tau=1 -> every pixel to leaf 0
    return dict(dx=np.zeros(1, np.float32), dy=np.zeros(1, np.float32),
                tau=np.ones(1, np.float32), type=np.zeros(1, np.uint8),
                channel=np.zeros(1, np.uint8), n_trees=1, depth=1)


def test_reservoir_is_unbiased():
    """Algorithm R keeps every one of n offered examples with probability
    kappa/n (Vitter 1985): chi-square over seeds."""
    f = _single_leaf_forest()
    K = rooms.Intrinsics(16.0, 16.0, 8.0, 8.0, 16, 16)
    d = np.ones((16, 16), np.float32)
    c = np.zeros((16, 16, 3), np.uint8)
    frames = 3
    n_ex = 16 * frames
    kappa = 4
    counts = np.zeros(n_ex)
    trials = 3000
    for s in range(trials):
        res = oracle.Reservoirs(f, kappa, seed=1000 + s)
        for fr in range(frames):
            T = np.eye(4)
            T[0, 3] = 100.0 * fr                           # tag the frame in x
            res.add_frame(d, c, K, T)
        assert res.count[0] == n_ex
        for e in range(kappa):
            x, y = res.pos[0, e, 0], res.pos[0, e, 1]
            fr = int(round(x / 100.0))
            u = int(round((x - 100.0 * fr) * 16 + 8))
            v = int(round(y * 16 + 8))
            counts[fr * 16 + (v // 4) * 4 + u // 4] += 1
    exp = trials * kappa / n_ex
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 90, chi2      # 47 dof: p(chi2 > 90) < 1e-4
    assert counts.sum() == trials * kappa


def test_reservoir_fills_in_order_below_capacity():
    f = _single_leaf_forest()
    K = rooms.Intrinsics(16.0, 16.0, 8.0, 8.0, 16, 16)
    d = np.ones((16, 16), np.float32)
    d[4, 4] = 0.0                                           # invalid grid pixel is skipped
    res = oracle.Reservoirs(f, 32, seed=5)
    res.add_frame(d, np.zeros((16, 16, 3), np.uint8), K, np.eye(4))
    assert res.count[0] == 15
    xs = [(res.pos[0, e, 0], res.pos[0, e, 1]) for e in range(15)]
    grid = [((u - 8) / 16, (v - 8) / 16) for v in range(0, 16, 4) for u in range(0, 16, 4) if (u, v) != (4, 4)]
    assert np.allclose(xs, grid)
    # the grid's origin is a parameter (reading R4 takes 0); origin 2 shifts it
    res = oracle.Reservoirs(f, 32, seed=5)
    res.add_frame(d, np.zeros((16, 16, 3), np.uint8), K, np.eye(4), grid_step=4, grid_origin=2)
    grid = [((u - 8) / 16, (v - 8) / 16) for v in range(2, 16, 4) for u in range(2, 16, 4)]
    assert res.count[0] == len(grid) == 16
    assert np.allclose([(res.pos[0, e, 0], res.pos[0, e, 1]) for e in range(16)], grid)


# ---------------------------------------------------------------- RQS + modes
def _blobs(rng, sizes, centres, spread=0.01):
    pts = np.concatenate([c + spread * rng.normal(size=(n, 3)) for n, c in zip(sizes, centres)])
    cols = np.concatenate([np.full((n, 3), 40 * (i + 1)) for i, n in enumerate(sizes)])
    perm = rng.permutation(len(pts))
    return pts[perm].astype(np.float32), cols[perm].astype(np.uint8)


def test_rqs_separated_blobs():
    rng = np.random.default_rng(6)
    centres = [np.array([0, 0, 0.0]), np.array([1, 0, 0.0]), np.array([0, 1.5, 0.3]), np.array([3, 3, 3.0])]
    sizes = [50, 30, 12, 3]
    pts, cols = _blobs(rng, sizes, centres)
    r = oracle.rqs_leaf(pts, cols, 0.1, 0.05, 5, 10)
    assert r["k"] == 3                                       # the 3-point blob is below minClusterSize
    assert list(r["size"]) == [50, 30, 12]
    for k in range(3):
        members = pts[np.linalg.norm(pts - centres[k], axis=1) < 0.2].astype(np.float64)
        assert np.allclose(r["mu"][k], members.mean(0), atol=1e-12)
        cov = np.cov(members.T)
        assert np.allclose(r["cov"][k], cov[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]], atol=1e-12)
        assert (r["colour"][k] == 40 * (k + 1)).all()
    r2 = oracle.rqs_leaf(pts, cols, 0.1, 0.05, 5, 2)
    assert r2["k"] == 2 and list(r2["size"]) == [50, 30]     # M_max truncation keeps the largest


def test_rqs_parent_is_nearest_denser_point():
    # 1-D chain: the densest point in the middle; parents point inwards.
    pts = np.array([[0, 0, 0], [0.03, 0, 0], [0.06, 0, 0], [0.09, 0, 0], [0.12, 0, 0]], np.float32)
    r = oracle.rqs_leaf(pts, np.zeros((5, 3), np.uint8), 0.1, 0.05, 1, 5)
    assert r["density"].argmax() == 2
    assert list(r["parent"]) == [1, 2, -1, 2, 3]
    assert list(r["root"]) == [2, 2, 2, 2, 2]
    r = oracle.rqs_leaf(pts, np.zeros((5, 3), np.uint8), 0.1, 0.02, 1, 5)  # links too long
    assert list(r["parent"]) == [-1] * 5 and r["k"] == 5


def test_rqs_densities_are_the_parzen_sums():
    """rho_i = sum_j exp(-|x_i - x_j|^2 / (2 sigma^2)) over all points of
    the leaf (Sec. 3.2.2), recomputed in numpy."""
    rng = np.random.default_rng(5)
    pts = (rng.normal(size=(40, 3)) * 0.08 + [1.0, 2.0, 0.5]).astype(np.float32)
    for sigma in (0.05, 0.1, 0.3):
        r = oracle.rqs_leaf(pts, np.zeros((40, 3), np.uint8), sigma, 0.05, 1, 10)
        X = pts.astype(np.float64)
        d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
        np.testing.assert_allclose(r["density"], np.exp(-d2 / (2.0 * float(np.float32(sigma)) ** 2)).sum(1),
                                   rtol=1e-12)


def test_rqs_mode_colour_is_the_rounded_mean():
    """A mode's colour is the mean of its members' colours per channel,
    rounded to the nearest integer with halves up (reading of "colour
    centroid" for 8-bit colours)."""
    pts = np.array([[0, 0, 0], [0.01, 0, 0], [0.0, 0.01, 0]], np.float32)
    cols = np.array([[10, 200, 7], [11, 201, 8], [11, 201, 8]], np.uint8)   # means 10.67, 200.67, 7.67
    r = oracle.rqs_leaf(pts, cols, 0.1, 0.05, 1, 5)
    assert r["k"] == 1 and list(r["colour"][0]) == [11, 201, 8]
    r = oracle.rqs_leaf(pts[:2], cols[:2], 0.1, 0.05, 1, 5)                # means 10.5, 200.5, 7.5
    assert r["k"] == 1 and list(r["colour"][0]) == [11, 201, 8]


def test_rqs_equal_densities_link_to_the_lower_index():
    """Reading of the parent rule at equal densities: the point of lower
    index counts as denser, so of two mirror-image points the second links
    to the first, which is the root."""
    pts = np.array([[0, 0, 0], [0.03, 0, 0]], np.float32)
    r = oracle.rqs_leaf(pts, np.zeros((2, 3), np.uint8), 0.1, 0.05, 1, 5)
    assert r["density"][0] == r["density"][1]
    assert list(r["parent"]) == [-1, 0] and list(r["root"]) == [0, 0] and r["k"] == 1
    pts = np.array([[0.03, 0, 0], [0, 0, 0], [0.06, 0, 0]], np.float32)  # middle first
    r = oracle.rqs_leaf(pts, np.zeros((3, 3), np.uint8), 0.1, 0.05, 1, 5)
    assert r["density"][1] == r["density"][2] and r["density"][0] > r["density"][1]
    assert list(r["parent"]) == [-1, 0, 0]


def test_mode_store_encoding():
    """FP16 offsets from an FP32 leaf centroid (numpy's IEEE half rounding),
    colour rounding and U^T U = (cov + eps I)^-1."""
    rng = np.random.default_rng(8)
    f = _single_leaf_forest()
    res = oracle.Reservoirs(f, 256, seed=1)
    centres = [np.array([1.2, 0.4, 2.0]), np.array([2.9, 1.1, 0.7]), np.array([0.3, 2.5, 1.9])]
    pts, cols = _blobs(rng, [60, 40, 25], centres, spread=0.02)
    res.pos[0, :125] = pts
    res.rgb[0, :125] = cols
    res.count[0] = 125
    for fp16 in (True, False):
        m = oracle.Modes(res.n_leaves, 4)
        oracle.update_modes(res, m, 0.1, 0.05, 5, cov_eps=1e-4, fp16_offsets=fp16)
        r = oracle.rqs_leaf(pts, cols, 0.1, 0.05, 5, 4)
        assert m.nmodes[0] == 3
        cen = (r["mu"].sum(0) / 3).astype(np.float32)
        assert np.array_equal(m.centroid[0], cen)
        for k in range(3):
            if fp16:
                want = cen + np.float16(r["mu"][k] - cen.astype(np.float64)).astype(np.float32)
            else:
                want = r["mu"][k].astype(np.float32)
            assert np.array_equal(m.pos[0, k], want)
            u = m.U[0, k].astype(np.float64)
            U = np.array([[u[0], u[1], u[2]], [0, u[3], u[4]], [0, 0, u[5]]])
            cov = r["cov"][k]
            C = np.array([[cov[0], cov[1], cov[2]], [cov[1], cov[3], cov[4]], [cov[2], cov[4], cov[5]]])
            S = np.linalg.inv(C + 1e-4 * np.eye(3))
            assert np.allclose(U.T @ U, S, rtol=2e-6, atol=1e-6 * np.abs(S).max())
            assert m.size[0, k] == r["size"][k]


# ---------------------------------------------------------------- Eq. 6-7
def test_raycast_matches_independent_render():
    w = workloads.CONFIG1
    room = w.room()
    rng = np.random.default_rng(9)
    for _ in range(5):
        pos = rng.uniform([0.5, 0.5, 0.5], [3.5, 2.5, 2.0])
        T = rooms.look_pose(pos, rng.uniform(0, 6.28), rng.uniform(-0.5, 0.5), rng.uniform(-0.3, 0.3))
        d_ref, _ = rooms.render(room, w.K, T, noise_sigma=0.0)
        d = oracle.raycast_box(T, w.K, room.lo, room.hi)
        assert np.abs(d - d_ref.astype(np.float64)).max() < 1e-5


def test_raycast_closed_forms_and_outside_camera():
    K = rooms.Intrinsics(100.0, 100.0, 50.0, 40.0, 101, 81)
    lo, hi = np.zeros(3), np.array([4.0, 3.0, 2.5])
    T = rooms.look_pose([1.0, 1.5, 1.25], 0.0, 0.0)          # looking +x at the wall x=4
    d = oracle.raycast_box(T, K, lo, hi)
    assert abs(d[40, 50] - 3.0) < 1e-12                      # fronto-parallel wall: constant z-depth
    assert np.allclose(d[30:50, 40:60], 3.0)
    T = rooms.look_pose([-1.0, 1.5, 1.25], 0.0, 0.0)         # outside, facing the box
    d = oracle.raycast_box(T, K, lo, hi)
    assert abs(d[40, 50] - 1.0) < 1e-12                      # entry face at distance 1
    T = rooms.look_pose([-1.0, 1.5, 1.25], math.pi, 0.0)     # outside, facing away
    assert np.isnan(oracle.raycast_box(T, K, lo, hi)).all()
    s, mu, frac = oracle.depth_score(T, np.ones((81, 101), np.float32), K, lo, hi)
    assert math.isinf(s) and frac == 0.0


def test_depth_score_of_ground_truth_is_noise_mean():
    w = workloads.CONFIG2
    room = w.room()
    T = rooms.look_pose([2.0, 1.4, 1.3], 2.0, -0.1)
    sigma = 0.002
    d, _ = rooms.render(room, w.K, T, noise_sigma=sigma, noise_seed=1)
    s, mu, frac = oracle.depth_score(T, d, w.K, room.lo, room.hi)
    assert frac == 1.0
    assert abs(s - sigma * math.sqrt(2 / math.pi)) < 0.03 * sigma   # E|N(0, s^2)|
    d2 = d.copy()
    d2[:, : w.width // 2] = 0                                # missing live depth is masked out
    s2, _, _ = oracle.depth_score(T, d2, w.K, room.lo, room.hi)
    assert abs(s2 - sigma * math.sqrt(2 / math.pi)) < 0.05 * sigma


# ---------------------------------------------------------------- ICP before ranking (R21)
_ICP_K = rooms.Intrinsics(292.5, 292.5, 160.0, 120.0, 320, 240)
_ICP_ROOM = rooms.Room((4.0, 3.0, 2.5), 5)


def _rot_deg(axis, deg):
    return rooms._rodrigues(axis, math.radians(deg))


def _corner_view():
    """Camera near one corner looking at the opposite lower corner: two walls
    and the floor in view, so every pose direction is constrained."""
    pos = np.array([1.0, 0.8, 1.6])
    tgt = np.array([4.0, 3.0, 0.0]) - pos
    return rooms.look_pose(pos, math.atan2(tgt[1], tgt[0]), math.atan2(tgt[2], math.hypot(tgt[0], tgt[1])))


def test_depth_score_needs_a_tenth_of_the_rays_on_the_model():
    """Eq. 8: the score is the masked mean depth difference when at least a
    tenth of the synthetic depth image is valid, else infinite.  Cameras
    outside the box see it with 36% and 6% of their rays (counted here with
    the numpy renderer)."""
    w = workloads.CONFIG1
    room = w.room()
    d, _ = rooms.render(room, w.K, rooms.look_pose([1.7, 1.4, 1.2], 0.4, 0.1), noise_sigma=0.0)
    for yaw_deg, finite in ((-100.0, True), (-83.0, False)):
        P = rooms.look_pose([room.hi[0] + 0.5, 0.5 * (room.lo[1] + room.hi[1]), 1.2], math.radians(yaw_deg), 0.0)
        syn = _numpy_box_depth(P, w.K, room.lo, room.hi)
        frac_np = np.isfinite(syn).mean()
        assert (frac_np > 0.3) if finite else (0.02 < frac_np < 0.08)
        s, mu, frac = oracle.depth_score(P, d, w.K, room.lo, room.hi)
        assert abs(frac - frac_np) <= 2.0 / d.size
        m = np.isfinite(syn) & (d > 0)
        np.testing.assert_allclose(mu, np.abs(d[m] - syn[m]).mean(), rtol=1e-6)
        assert (s == mu) if finite else math.isinf(s)


def test_icp_recovers_exact_pose_of_corner_view():
    """Noise-free depth: the true pose zeroes every residual, so ICP started a
    few cm / degrees away must land on it (a wrong sign, index or transposed
    Jacobian block would not converge there), and started on it stays."""
    T = _corner_view()
    d, _ = rooms.render(_ICP_ROOM, _ICP_K, T, noise_sigma=0.0)
    rng = np.random.default_rng(1)
    for _ in range(4):
        P = T.copy()
        P[:3, :3] = _rot_deg(rng.normal(size=3), 2.5) @ T[:3, :3]
        P[:3, 3] += rng.normal(size=3) * 0.03
        R, ok, frac = oracle.icp_refine(P, d, _ICP_K, _ICP_ROOM.lo, _ICP_ROOM.hi)
        dt, dr = H.pose_err(R, T)
        assert ok and frac == 1.0
        assert dt < 1e-6 and dr < 1e-4, (dt, dr)
    R, ok, _ = oracle.icp_refine(T, d, _ICP_K, _ICP_ROOM.lo, _ICP_ROOM.hi)
    assert ok and H.pose_err(R, T)[0] < 1e-6
    # pure rotation and pure translation errors separately
    for P in (T @ np.block([[_rot_deg([1, 0, 0], 3.0), np.zeros((3, 1))], [np.zeros((1, 3)), np.ones((1, 1))]]),
              T + np.block([[np.zeros((3, 3)), np.array([[0.04], [-0.03], [0.02]])], [np.zeros((1, 4))]])):
        R, ok, _ = oracle.icp_refine(P, d, _ICP_K, _ICP_ROOM.lo, _ICP_ROOM.hi)
        assert ok and H.pose_err(R, T)[0] < 1e-6 and H.pose_err(R, T)[1] < 1e-4


def test_icp_first_step_is_the_ridge_damped_point_to_plane_step():
    """One ICP iteration (reading R21) re-derived in numpy from its
    definition: projective association with the first box face along each
    pixel ray, residual n . (q - p), inliers within the radius, camera-frame
    Jacobian (m, x x m) with m = R^T n, step (A + ridge tr(A)/6 I) xi = -g,
    pose H exp(xi^).  A large ridge makes its scaling matter."""
    expm = pytest.importorskip("scipy.linalg").expm
    T = _corner_view()
    d, _ = rooms.render(_ICP_ROOM, _ICP_K, T, noise_sigma=0.0)
    P = T.copy()
    P[:3, :3] = _rot_deg([0.2, 1.0, -0.4], 1.5) @ T[:3, :3]
    P[:3, 3] += [0.02, -0.015, 0.01]
    stride, dist, ridge = 4, 0.1, 0.05
    K = _ICP_K
    lo, hi = np.asarray(_ICP_ROOM.lo, float), np.asarray(_ICP_ROOM.hi, float)
    R0, o = P[:3, :3], P[:3, 3]
    A = np.zeros((6, 6))
    g = np.zeros(6)
    for v in range(0, K.height, stride):
        for u in range(0, K.width, stride):
            dep = float(d[v, u])
            if not dep > 0:
                continue
            c = np.array([(u - K.cx) / K.fx, (v - K.cy) / K.fy, 1.0])
            w_ = R0 @ c
            with np.errstate(divide="ignore", invalid="ignore"):
                t1, t2 = (lo - o) / w_, (hi - o) / w_
            tmin, tmax = np.minimum(t1, t2), np.maximum(t1, t2)
            tn, an, tf, af = tmin.max(), int(tmin.argmax()), tmax.min(), int(tmax.argmin())
            if tn > tf:
                continue
            sh, ax = (tn, an) if tn > 0 else (tf, af)
            if not sh > 0:
                continue
            e = (dep - sh) * w_
            if e @ e > dist * dist:
                continue
            m = R0[ax]
            x = dep * c
            J = np.concatenate([m, np.cross(x, m)])
            A += np.outer(J, J)
            g += J * e[ax]
    xi = np.linalg.solve(A + ridge * np.trace(A) / 6.0 * np.eye(6), -g)
    want = P @ expm(_twist(xi))
    got, ok, _ = oracle.icp_refine(P, d, K, _ICP_ROOM.lo, _ICP_ROOM.hi, levels=1, stride=(stride,), iters=(1,),
                                   dist=(dist,), ridge=ridge, min_frac=0.0)
    assert ok
    assert np.abs(got - want).max() < 1e-10
    xi_abs = np.linalg.solve(A + ridge * np.eye(6), -g)
    assert np.abs(xi_abs - xi).max() > 1e-4          # the ridge scaling matters here


def test_icp_single_wall_keeps_unconstrained_directions():
    """A wall seen alone fixes only the distance to it and the two tilts.
    ICP must correct those exactly and leave the camera centre's offset along
    the wall and the turn about the wall normal where they started."""
    T = rooms.look_pose([2.5, 1.5, 1.25], 0.0, 0.0)          # 1.5 m from the wall x = 4
    d, _ = rooms.render(_ICP_ROOM, _ICP_K, T, noise_sigma=0.0)
    P = T.copy()
    P[:3, :3] = _rot_deg([0, 0, 1], 1.5) @ _rot_deg([0, 1, 0], -1.0) @ _rot_deg([1, 0, 0], 2.0) @ T[:3, :3]
    P[:3, 3] += [0.04, 0.05, 0.03]
    R, ok, frac = oracle.icp_refine(P, d, _ICP_K, _ICP_ROOM.lo, _ICP_ROOM.hi)
    assert ok and frac == 1.0
    assert abs(R[0, 3] - T[0, 3]) < 1e-6                      # distance to the wall
    assert np.abs(R[:3, 2] - np.array([1.0, 0.0, 0.0])).max() < 1e-6   # view direction = wall normal
    # offset along the wall kept: only a second-order coupling remains (the
    # first steps move along the still-tilted normal: 4 cm x 2 deg ~ 1.4 mm),
    # where a turn about any point but the camera centre would shift it by
    # distance x angle (1.5 m x 2 deg ~ 5 cm)
    assert np.abs(R[1:3, 3] - P[1:3, 3]).max() < 2e-3
    roll = lambda M: math.degrees(math.atan2(M[2, 0], -M[1, 0]))       # turn about the normal
    assert abs(roll(R) - roll(P)) < 0.02, (roll(R), roll(P))


def test_icp_failure_cases():
    T = _corner_view()
    d, _ = rooms.render(_ICP_ROOM, _ICP_K, T, noise_sigma=0.0)
    lo, hi = _ICP_ROOM.lo, _ICP_ROOM.hi
    R, ok, frac = oracle.icp_refine(T, np.zeros_like(d), _ICP_K, lo, hi)       # no valid depth
    assert not ok and frac == 0.0 and np.array_equal(R, T)
    Tout = rooms.look_pose([-1.0, 1.5, 1.25], math.pi, 0.0)                     # outside, facing away
    assert not oracle.icp_refine(Tout, d, _ICP_K, lo, hi)[1]
    P = T.copy()
    P[:3, 3] += T[:3, 2] * 0.3                                 # 30 cm along the view: no pair within 10 cm
    R, ok, frac = oracle.icp_refine(P, d, _ICP_K, lo, hi)
    assert not ok and frac == 0.0
    # the inlier-fraction rule: half the image without a model counterpart
    d2 = d.copy()
    d2[(np.arange(d.shape[0]) // 4) % 2 == 0] += 0.5    # every other band of 4 rows
    _, ok, frac = oracle.icp_refine(T, d2, _ICP_K, lo, hi, min_frac=0.6)
    assert not ok and abs(frac - 0.5) < 0.01
    _, ok, frac = oracle.icp_refine(T, d2, _ICP_K, lo, hi, min_frac=0.4)
    assert ok and abs(frac - 0.5) < 0.01


def _numpy_box_depth(P, K, lo, hi):
    """Vectorised slab test: z-depth of the exit point from inside the box,
    of the entry point from outside, NaN when the ray misses."""
    uu, vv = np.meshgrid(np.arange(K.width, dtype=float), np.arange(K.height, dtype=float))
    dc = np.stack([(uu - K.cx) / K.fx, (vv - K.cy) / K.fy, np.ones_like(uu)], -1)
    dw = dc @ np.asarray(P)[:3, :3].T
    o = np.asarray(P)[:3, 3]
    with np.errstate(divide="ignore", invalid="ignore"):
        t1, t2 = (lo - o) / dw, (hi - o) / dw
    tmin = np.where(dw == 0, np.where((o >= lo) & (o <= hi), -np.inf, np.nan), np.minimum(t1, t2))
    tmax = np.where(dw == 0, np.where((o >= lo) & (o <= hi), np.inf, np.nan), np.maximum(t1, t2))
    tn, tf = np.max(tmin, -1), np.min(tmax, -1)
    out = np.where(tn > 0, tn, np.where(tf > 0, tf, np.nan))
    return np.where(tn <= tf, out, np.nan)


# ---------------------------------------------------------------- RANSAC invariants
def _numpy_attempt(w, p, d, c, lv, modes, key, slot, it):
    """Re-derives one generation attempt with the Python Philox; returns
    the three (x_C, x_W) pairs or None if a check rejects it."""
    Hh, W = d.shape
    WH = W * Hh
    r0 = philox_ref.philox4x32_10((slot, (3 << 16) | p["level"], it, 0), key)
    r1 = philox_ref.philox4x32_10((slot, (3 << 16) | p["level"], it, 1), key)
    lpt = 1 << w.forest["depth"]

    def modes_of(q):
        ms = []
        for t in range(p["n_trees_used"]):
            L = t * lpt + int(lv[t].flat[q])
            ms += [(L, m) for m in range(min(int(modes.nmodes[L]), p["k_top"]))]
        return ms

    xs, xw, pix, me = [], [], [], []
    for i in range(3):
        q = philox_ref.below(r0[i], WH)
        # reading R8b: an unusable pixel is redrawn within the iteration
        for a in range(1, p["batch_attempts"] if p.get("redraw") else 1):
            if d.flat[q] > 0 and modes_of(q):
                break
            r2 = philox_ref.philox4x32_10((slot, (5 << 16) | p["level"], it, 4 * a + i), key)
            q = philox_ref.below(r2[0], WH)
        if not d.flat[q] > 0:
            return None
        ms = modes_of(q)
        if not ms:
            return None
        L, m = ms[philox_ref.below(r1[i], len(ms))]
        u, v = q % W, q // W
        dd = np.float32(d.flat[q])
        xs.append(np.array([np.float32((np.float32(u) - np.float32(w.K.cx)) * dd) / np.float32(w.K.fx),
                            np.float32((np.float32(v) - np.float32(w.K.cy)) * dd) / np.float32(w.K.fy), dd],
                           np.float64))
        xw.append(modes.pos[L, m].astype(np.float64))
        pix.append(q)
        me.append((L, m))
    j = philox_ref.below(r0[3], 3)
    if np.abs(c.reshape(-1, 3)[pix[j]].astype(int) - modes.rgb[me[j]].astype(int)).max() > p["colour_thresh"]:
        return None
    for a, b in ((0, 1), (0, 2), (1, 2)):
        dw2 = float(((xw[a] - xw[b]) ** 2).sum())
        if dw2 < p["min_sq_dist"]:
            return None
    for a, b in ((0, 1), (0, 2), (1, 2)):
        dw = math.sqrt(((xw[a] - xw[b]) ** 2).sum())
        dc = math.sqrt(((xs[a] - xs[b]) ** 2).sum())
        if abs(dw - dc) > p["max_trans_err"]:
            return None
    return np.array(xs), np.array(xw)


def test_generation_redraw_reading_rederived():
    """Reading R8b (redraw within the iteration) on a query with 70% of its
    depth missing: each slot's winning iteration is the first accepted one
    of the numpy re-derivation with redraws, the accepted triple gives the
    oracle's pose, and redrawing keeps far more hypotheses than R8."""
    w = H.WORKLOADS[H.SMALL]
    f, res, modes = H.oracle_model(w.name)
    d, c, T, seed = w.query(1)
    d = rooms.mask_depth(d, 0.7, seed=17)
    lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=w.ransac["n_trees_used"])
    args = (d, c, w.K, lv, modes, w.room().lo, w.room().hi, seed, 1 << w.forest["depth"])
    p = dict(oracle.PARAM_DEFAULTS, **w.ransac, redraw=1)
    r = oracle.relocalise(p, *args, debug=True)
    r8 = oracle.relocalise(dict(p, redraw=0), *args, debug=True)
    assert r["n_hypotheses"] >= 3 * max(1, r8["n_hypotheses"]), (r["n_hypotheses"], r8["n_hypotheses"])
    key = philox_ref.key_of(seed)
    it = r["debug"]["hyp_iter"]
    for slot in range(0, p["n_hyp"], 11):
        last = it[slot] if it[slot] >= 0 else p["max_iter"]
        for k in range(min(last, 40)):
            assert _numpy_attempt(w, p, d, c, lv, modes, key, slot, k) is None
        if it[slot] >= 0:
            pair = _numpy_attempt(w, p, d, c, lv, modes, key, slot, it[slot])
            assert pair is not None
            Rh, th = _horn(*pair)
            P = r["debug"]["hyp_pose"][slot].reshape(3, 4)
            assert np.abs(P[:, :3] - Rh).max() < 1e-9 and np.abs(P[:, 3] - th).max() < 1e-9
    # without missing depth every first draw is usable: the readings agree
    d0, c0, _, _ = w.query(1)
    lv0 = oracle.forest_leaves(f, d0, c0, w.K.fx, n_trees=w.ransac["n_trees_used"])
    a0 = (d0, c0, w.K, lv0, modes, w.room().lo, w.room().hi, seed, 1 << w.forest["depth"])
    ra = oracle.relocalise(p, *a0, debug=True)
    rb = oracle.relocalise(dict(p, redraw=0), *a0, debug=True)
    if (d0 > 0).all() and all((modes.nmodes[t * (1 << w.forest["depth"]) + lv0[t].astype(int)] > 0).all()
                              for t in range(p["n_trees_used"])):
        assert np.array_equal(ra["debug"]["hyp_iter"], rb["debug"]["hyp_iter"])


@pytest.fixture(scope="module")
def small_run():
    w = H.WORKLOADS[H.SMALL]
    f, res, modes = H.oracle_model(w.name)
    out = []
    for q in range(2):
        d, c, T, seed = w.query(q)
        lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=w.ransac["n_trees_used"])
        r = oracle.relocalise(w.ransac, d, c, w.K, lv, modes, w.room().lo, w.room().hi, seed,
                              1 << w.forest["depth"], debug=True)
        out.append((d, c, T, seed, lv, r))
    return w, f, modes, out


def test_generation_rederived_with_independent_philox(small_run):
    """Every slot stops at its first accepted iteration; the accepted triple
    re-derived in numpy gives the same Kabsch pose (Horn's method)."""
    w, f, modes, runs = small_run
    p = dict(oracle.PARAM_DEFAULTS, **w.ransac)
    d, c, T, seed, lv, r = runs[0]
    key = philox_ref.key_of(seed)
    it = r["debug"]["hyp_iter"]
    assert (it >= 0).sum() == r["n_hypotheses"] > 10
    for slot in range(0, p["n_hyp"], 7):
        last = it[slot] if it[slot] >= 0 else p["max_iter"]
        for k in range(min(last, 60)):                   # earlier iterations all rejected
            assert _numpy_attempt(w, p, d, c, lv, modes, key, slot, k) is None
        if it[slot] >= 0:
            pair = _numpy_attempt(w, p, d, c, lv, modes, key, slot, it[slot])
            assert pair is not None
            Rh, th = _horn(*pair)
            P = r["debug"]["hyp_pose"][slot].reshape(3, 4)
            assert np.abs(P[:, :3] - Rh).max() < 1e-8 and np.abs(P[:, 3] - th).max() < 1e-8


def test_batch_pixels_rederived_with_independent_philox(small_run):
    """Reading R12: pixel j of batch b is the first of up to batch_attempts
    Philox draws (counter (b, 4 << 16 | level, j, a)) with depth and a
    non-empty M(u), or none; re-derived here with the Python Philox."""
    w, f, modes, runs = small_run
    p = dict(oracle.PARAM_DEFAULTS, **w.ransac)
    lpt = 1 << w.forest["depth"]
    for d, c, T, seed, lv, r in runs:
        key = philox_ref.key_of(seed)
        WH = d.size
        bp = r["debug"]["batch_pix"]
        n_batches = r["debug"]["n_rounds"] + 1
        assert n_batches >= 2
        skipped = 0
        for b in range(n_batches):
            for j in range(p["eta"]):
                want = -1
                for a in range(p["batch_attempts"]):
                    q = philox_ref.below(philox_ref.philox4x32_10((b, (4 << 16) | p["level"], j, a), key)[0], WH)
                    if not d.flat[q] > 0:
                        continue
                    cnt = sum(min(int(modes.nmodes[t * lpt + int(lv[t].flat[q])]), p["k_top"])
                              for t in range(p["n_trees_used"]))
                    if cnt == 0:
                        continue
                    want = q
                    break
                skipped += want < 0
                assert bp[b][j] == want, (b, j)
        assert skipped < n_batches * p["eta"]


def test_generation_rederived_at_the_paper_colour_threshold():
    """The re-derivation of the generation test with check 1 at its
    configured strength (colour 30 instead of the parity case's loosened
    120), so the colour test (L-infinity over RGB) decides most attempts."""
    w = H.WORKLOADS[H.SMALL]
    f, res, modes = H.oracle_model(w.name)
    p = dict(oracle.PARAM_DEFAULTS, **dict(w.ransac, colour_thresh=30))
    d, c, T, seed = w.query(0)
    lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=p["n_trees_used"])
    r = oracle.relocalise(p, d, c, w.K, lv, modes, w.room().lo, w.room().hi, seed, 1 << w.forest["depth"],
                          debug=True)
    key = philox_ref.key_of(seed)
    it = r["debug"]["hyp_iter"]
    assert 0 < (it >= 0).sum() < p["n_hyp"]
    for slot in range(0, p["n_hyp"], 5):
        last = it[slot] if it[slot] >= 0 else p["max_iter"]
        for k in range(min(last, 150)):
            assert _numpy_attempt(w, p, d, c, lv, modes, key, slot, k) is None, (slot, k)
        if it[slot] >= 0:
            assert _numpy_attempt(w, p, d, c, lv, modes, key, slot, it[slot]) is not None


@pytest.mark.parametrize("offset, passes", [((20, 20, 20), True), ((30, 0, 0), True), ((0, -31, 0), False)])
def test_colour_check_is_the_largest_channel_difference(offset, passes):
    """Check 1 (Sec. 3.2.3) accepts a pair iff max over R, G, B of the
    absolute difference between the pixel's colour and the mode's colour
    centroid is at most the threshold: uniform frame colour 100, every mode
    coloured 100 + offset, checks 2 and 3 opened, colour threshold 30."""
    w = H.WORKLOADS[H.SMALL]
    f, res, modes0 = H.oracle_model(w.name)
    modes = oracle.Modes(modes0.nmodes.size, modes0.m_max)
    for k in ("nmodes", "centroid", "pos", "U", "size"):
        getattr(modes, k)[:] = getattr(modes0, k)
    modes.rgb[:] = np.array([100, 100, 100]) + np.array(offset)
    p = dict(oracle.PARAM_DEFAULTS, **dict(w.ransac, colour_thresh=30, min_sq_dist=1e-6, max_trans_err=1e9,
                                           pose_update=0, rank=0))
    d, c, T, seed = w.query(0)
    c = np.full_like(c, 100)
    lv = oracle.forest_leaves(f, d, w.query(0)[1], w.K.fx, n_trees=p["n_trees_used"])
    r = oracle.relocalise(p, d, c, w.K, lv, modes, w.room().lo, w.room().hi, seed, 1 << w.forest["depth"],
                          debug=True)
    it = r["debug"]["hyp_iter"]
    if passes:
        assert (it >= 0).all() and np.median(it) <= 1
    else:
        assert (it < 0).all() and r["n_hypotheses"] == 0


def test_cull_keeps_lowest_brute_force_energies(small_run):
    w, f, modes, runs = small_run
    p = dict(oracle.PARAM_DEFAULTS, **w.ransac)
    d, c, T, seed, lv, r = runs[0]
    dbg = r["debug"]
    lpt = 1 << w.forest["depth"]
    S_all = np.zeros(modes.U.shape[:2] + (3, 3))
    for L in np.nonzero(modes.nmodes)[0]:
        for m in range(modes.nmodes[L]):
            u = modes.U[L, m].astype(np.float64)
            U = np.array([[u[0], u[1], u[2]], [0, u[3], u[4]], [0, 0, u[5]]])
            S_all[L, m] = U.T @ U
    pix0 = dbg["batch_pix"][0]
    slots = np.nonzero(dbg["hyp_iter"] >= 0)[0]
    E = np.array([_brute_energy(H.as44(dbg["hyp_pose"][s]), pix0, d, w.K, lv, modes, S_all,
                                p["k_top"], p["use_cov"], lpt) for s in slots])
    order = slots[np.lexsort((slots, E))][: p["n_cull"]]
    assert list(dbg["cull_slot"][: len(order)]) == list(order)
    np.testing.assert_allclose(dbg["cull_energy"][: len(order)], np.sort(E)[: len(order)], rtol=1e-12)


def test_halving_and_chosen_set(small_run):
    w, f, modes, runs = small_run
    p = dict(oracle.PARAM_DEFAULTS, **w.ransac)
    for d, c, T, seed, lv, r in runs:
        dbg = r["debug"]
        n = min(r["n_hypotheses"], p["n_cull"])
        counts = []
        while n > p["k_out"] or (p["halve_to_one"] and n > 1):
            n = (n + 1) // 2
            counts.append(n)
        assert list(dbg["round_count"][: len(counts)]) == counts
        assert dbg["n_rounds"] == len(counts)
        assert r["n_pixels"] == p["eta"] * (len(counts) + 1)
        # each round's survivors are the better half of the previous round's
        off = 0
        prev = list(dbg["cull_slot"][: min(r["n_hypotheses"], p["n_cull"])])
        for k in counts:
            cur = list(dbg["round_slot"][off: off + k])
            assert set(cur) <= set(prev)
            e = dbg["round_energy"][off: off + k]
            assert (np.diff(e) >= 0).all()
            prev = cur
            off += k
        # the chosen set is the first survivor set of at most k_out hypotheses
        seq = [min(r["n_hypotheses"], p["n_cull"])] + counts
        first = next(i for i, k in enumerate(seq) if k <= p["k_out"])
        assert r["n_chosen"] == seq[first]
        if first == 0:
            want = dbg["cull_slot"][: seq[0]]
        else:
            o = sum(counts[: first - 1])
            want = dbg["round_slot"][o: o + seq[first]]
        assert list(r["chosen_slot"]) == list(want)
        # ranking returns the argmin of the chosen scores, recomputed here
        room = w.room()
        sc = []
        for P in r["chosen_pose"]:
            syn = _numpy_box_depth(P, w.K, room.lo, room.hi)
            m = (d > 0) & np.isfinite(syn)
            frac = np.isfinite(syn).mean()
            sc.append(np.abs(d[m] - syn[m]).mean() if frac >= 0.1 and m.any() else np.inf)
        np.testing.assert_allclose(r["chosen_score"], sc, rtol=1e-6)
        assert r["best"] == int(np.argmin(sc))
        assert np.array_equal(r["pose"], r["chosen_pose"][r["best"]])


def test_icp_in_relocaliser_refines_and_discards(small_run):
    """With ICP on, the chosen set is the one RANSAC gives without it; each
    chosen pose is replaced by its ICP result iff ICP succeeds, a failed pose
    is not ranked (score +inf), and the output is the argmin over the
    rest.  Unranked, ICP refines the output pose alone."""
    w, f, modes, runs = small_run
    room = w.room()
    for d, c, T, seed, lv, r in runs:
        p = dict(w.ransac, icp=1)
        ri = oracle.relocalise(p, d, c, w.K, lv, modes, room.lo, room.hi, seed, 1 << w.forest["depth"])
        assert ri["n_chosen"] == r["n_chosen"]
        assert np.array_equal(ri["chosen_slot"], r["chosen_slot"])
        scores = []
        for k, P0 in enumerate(r["chosen_pose"]):
            Pk, ok, frac = oracle.icp_refine(P0, d, w.K, room.lo, room.hi)
            assert bool(ri["icp_mask"] >> k & 1) == ok
            assert ri["chosen_icp_frac"][k] == frac
            assert np.array_equal(ri["chosen_pose"][k], Pk if ok else P0)
            scores.append(oracle.depth_score(Pk, d, w.K, room.lo, room.hi)[0] if ok else np.inf)
        assert np.array_equal(ri["chosen_score"], scores)
        if np.isfinite(scores).any():
            assert ri["best"] == int(np.argmin(scores))
        assert np.array_equal(ri["pose"], ri["chosen_pose"][ri["best"]])
        # unranked: the output pose alone
        pu = dict(w.ransac, icp=1, rank=0)
        r0 = oracle.relocalise(dict(pu, icp=0), d, c, w.K, lv, modes, room.lo, room.hi, seed,
                               1 << w.forest["depth"])
        ru = oracle.relocalise(pu, d, c, w.K, lv, modes, room.lo, room.hi, seed, 1 << w.forest["depth"])
        Pk, ok, frac = oracle.icp_refine(r0["pose"], d, w.K, room.lo, room.hi)
        assert ru["icp_mask"] == int(ok) and ru["chosen_icp_frac"][0] == frac
        assert np.array_equal(ru["pose"], Pk if ok else r0["pose"])


def test_cascade_fall_back_rule():
    w = H.WORKLOADS[H.SMALL]
    f, res, modes = H.oracle_model(w.name)
    d, c, T, seed = w.query(3)
    lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=w.ransac["n_trees_used"])
    frames = [(d, c, w.K), (d, c, w.K)]
    levels = [dict(w.ransac, level=0), dict(w.ransac, level=1, n_hyp=64)]
    lpt = 1 << w.forest["depth"]
    r = oracle.cascade(levels, [np.inf], frames, [lv, lv], modes, w.room().lo, w.room().hi, seed, lpt)
    assert r["level"] == 0                                    # tau = +inf always accepts
    r = oracle.cascade(levels, [-np.inf], frames, [lv, lv], modes, w.room().lo, w.room().hi, seed, lpt)
    assert r["level"] == 1                                    # tau = -inf always falls back
    single = oracle.relocalise(levels[1], d, c, w.K, lv, modes, w.room().lo, w.room().hi, seed, lpt)
    assert np.array_equal(single["pose"], r["pose"])
    r0 = oracle.relocalise(levels[0], d, c, w.K, lv, modes, w.room().lo, w.room().hi, seed, lpt)
    thr = r0["score"]
    r = oracle.cascade(levels, [thr], frames, [lv, lv], modes, w.room().lo, w.room().hi, seed, lpt)
    assert r["level"] == 0                                    # score <= tau accepts
    r = oracle.cascade(levels, [np.nextafter(thr, -np.inf)], frames, [lv, lv], modes, w.room().lo,
                       w.room().hi, seed, lpt)
    assert r["level"] == 1                                    # score > tau falls back


def test_no_depth_frame_has_no_pose():
    w = H.WORKLOADS[H.SMALL]
    f, res, modes = H.oracle_model(w.name)
    d = np.zeros((w.height, w.width), np.float32)
    c = np.zeros((w.height, w.width, 3), np.uint8)
    lv = oracle.forest_leaves(f, d, c, w.K.fx)
    assert (lv == 0xFFFF).all()
    r = oracle.relocalise(w.ransac, d, c, w.K, lv, modes, w.room().lo, w.room().hi, 1,
                          1 << w.forest["depth"])
    assert r["status"] == 1 and r["n_hypotheses"] == 0 and math.isinf(r["score"])


def test_oracle_results_do_not_depend_on_its_thread_count():
    """The oracle's OpenMP loops split independent leaves and pixel rows
    only: modes, leaf maps and a relocalisation are bit-identical with one
    thread and with four."""
    w = H.WORKLOADS[H.SMALL]
    out = []
    for n in (1, 4):
        oracle.set_threads(n)
        try:
            f, res, modes = H.oracle_model.__wrapped__(w.name)      # not the cached model
            d, c, T, seed = w.query(1)
            lv = oracle.forest_leaves(f, d, c, w.K.fx, n_trees=w.ransac["n_trees_used"])
            r = oracle.relocalise(w.ransac, d, c, w.K, lv, modes, w.room().lo, w.room().hi, seed,
                                  1 << w.forest["depth"])
        finally:
            oracle.set_threads(1)
        out.append((modes, lv, r))
    (m1, l1, r1), (m4, l4, r4) = out
    for k in ("nmodes", "pos", "rgb", "U", "size"):
        assert np.array_equal(getattr(m1, k), getattr(m4, k)), k
    assert np.array_equal(l1, l4)
    assert np.array_equal(r1["pose"], r4["pose"]) and r1["score"] == r4["score"]
