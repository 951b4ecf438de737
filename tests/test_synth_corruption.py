"""The depth corruptions of the robustness sweeps follow the paper's rules
(Sec. 4, robustness to missing and noisy depth): a pixel is zeroed iff its
uniform draw r satisfies r <= p; noisy depth is d + n d with n ~ N(0, s^2)
per pixel.  Checked against the rules and the distributions they imply."""
import numpy as np

from synth import rooms, workloads


def _depth():
    w = workloads.CONFIG2
    d, _ = rooms.render(w.room(), w.K, w.query(0)[2], noise_sigma=0.002, noise_seed=1)
    return d


def test_missing_depth_rule():
    d = _depth()
    n = d.size
    for p in (0.1, 0.5, 0.9, 0.95):
        out = rooms.mask_depth(d, p, seed=5)
        r = np.random.default_rng(5).uniform(0.0, 1.0, size=d.shape)
        assert np.array_equal(out == 0, (r <= p) | (d == 0))        # zero iff r <= p
        assert np.array_equal(out[r > p], d[r > p])                  # the rest untouched
        frac = (r <= p).mean()
        assert abs(frac - p) < 5 * np.sqrt(p * (1 - p) / n)          # binomial
    assert np.array_equal(rooms.mask_depth(d, 0.0, seed=5), d)
    assert (rooms.mask_depth(d, 1.0, seed=5) == 0).all()


def test_noisy_depth_rule_and_distribution():
    d = _depth().astype(np.float64)
    for s in (0.025, 0.1):
        out = rooms.noisy_depth(d, s, seed=7).astype(np.float64)
        rel = (out - d) / d
        m = d > 0
        assert abs(rel[m].mean()) < 5 * s / np.sqrt(m.sum())         # zero mean
        assert abs(rel[m].std() / s - 1) < 0.02                        # n ~ N(0, s^2)
        n = np.random.default_rng(7).normal(0.0, s, size=d.shape)
        np.testing.assert_allclose(out[m], (d + n * d)[m], rtol=1e-6)  # d + n d
        # depth-dependent: the absolute spread grows with depth
        near, far = m & (d < np.percentile(d[m], 30)), m & (d > np.percentile(d[m], 70))
        assert (out - d)[far].std() > (out - d)[near].std() * np.mean(d[far]) / np.mean(d[near]) * 0.9
    zero = np.zeros((4, 4), np.float32)
    assert (rooms.noisy_depth(zero, 0.1, seed=1) == 0).all()         # missing stays missing


def test_sweep_corruption_is_seeded_per_image():
    d = _depth()
    a = workloads.corrupt(d, "missing", 0.5, 3)
    assert np.array_equal(a, workloads.corrupt(d, "missing", 0.5, 3))
    assert not np.array_equal(a, workloads.corrupt(d, "missing", 0.5, 4))
    assert workloads.corrupt(d, "noise", 0.0, 3) is d
