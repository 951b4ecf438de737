"""Mutation check of the oracle's pins (test infrastructure, run by hand).

Plants one plausible mistake at a time (a dropped term, a wrong sign,
index, threshold or rule) in a scratch copy of oracle/ under a temporary
directory, runs the CPU pins (tests/test_oracle_pins.py and
tests/test_synth_corruption.py) against that copy, and reports whether a
pin failed.  Every mistake listed should be caught.

    python -m tests.oracle_mutations [name filter ...]
"""
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MUT = tempfile.mkdtemp(prefix="oracle_mutation_")
M = [
 ("energy squared", "ransac.c", "        E += sqrt(best);", "        E += best;"),
 ("U transposed", "ransac.c",
  """        r0 = (double)U[0] * v0 + (double)U[1] * v1 + (double)U[2] * v2;
        r1 = (double)U[3] * v1 + (double)U[4] * v2;
        r2 = (double)U[5] * v2;""",
  """        r0 = (double)U[0] * v0;
        r1 = (double)U[1] * v0 + (double)U[3] * v1;
        r2 = (double)U[2] * v0 + (double)U[4] * v1 + (double)U[5] * v2;"""),
 ("LM Levenberg damping", "ransac.c", "            A[6 * a + a] += lambda * JtJ[6 * a + a];", "            A[6 * a + a] += lambda;"),
 ("LM lambda on accept", "ransac.c", "            lambda /= 10.0;", "            lambda *= 10.0;"),
 ("LM inlier test Mahalanobis", "ransac.c", "            double eu = mode_dist2(y, be, mpos, mU, 0, NULL);", "            double eu = mode_dist2(y, be, mpos, mU, use_cov, NULL);"),
 ("score valid fraction 0.5", "ransac.c", "    return (frac >= 0.1 && n_both > 0) ? mu : INFINITY;", "    return (frac >= 0.5 && n_both > 0) ? mu : INFINITY;"),
 ("score mean over synthetic pixels", "ransac.c", "    const double mu = n_both > 0 ? sum / (double)n_both : INFINITY;", "    const double mu = n_both > 0 ? sum / (double)n_syn : INFINITY;"),
 ("raycast range not z", "ransac.c", "            out[(size_t)v * W + u] = ray_box_depth(o, dw, lo, hi);", "            out[(size_t)v * W + u] = ray_box_depth(o, dw, lo, hi) * sqrt(dc[0] * dc[0] + dc[1] * dc[1] + 1.0);"),
 ("colour L1", "ransac.c", "        if (d > linf) linf = d;", "        linf += d;"),
 ("spread on camera points", "ransac.c", "        if (dW2[k] < p->min_sq_dist)", "        if (dC2[k] < p->min_sq_dist)"),
 ("rigidity 2x", "ransac.c", "        if (fabs(sqrt(dW2[k]) - sqrt(dC2[k])) > p->max_trans_err)", "        if (fabs(sqrt(dW2[k]) - sqrt(dC2[k])) > 2.0 * p->max_trans_err)"),
 ("halving floor", "ransac.c", "        n = (n + 1) / 2;", "        n = n / 2;"),
 ("chosen = last set", "ransac.c", "        if (n_chosen < 0 && n <= p->k_out) {", "        if (n <= p->k_out) {"),
 ("batch keeps pixels without modes", "ransac.c",
  """            if (mode_count(pix, WH, leaves, p->n_trees_used, leaves_per_tree, nmodes, p->k_top) == 0)
                continue;
""", ""),
 ("mode draw wrong word", "ransac.c", "        const int m = (int)below(r1[i], (uint32_t)nm);", "        const int m = (int)below(r1[(i + 1) % 3], (uint32_t)nm);"),
 ("backproject fx for y", "ransac.c", "    xc[1] = (double)((((float)v - cy) * d) / fy);", "    xc[1] = (double)((((float)v - cy) * d) / fx);"),
 ("Kabsch no reflection fix", "ransac.c", "    double D[3] = {1.0, 1.0, detV < 0 ? -1.0 : 1.0};", "    double D[3] = {1.0, 1.0, 1.0};"),
 ("RQS kernel 1/s2", "adapt.c", "    const double inv2s2 = 1.0 / (2.0 * sgm * sgm);", "    const double inv2s2 = 1.0 / (sgm * sgm);"),
 ("RQS tie order", "adapt.c", "            int higher = density[j] > density[i] || (density[j] == density[i] && j < i);", "            int higher = density[j] > density[i] || (density[j] == density[i] && j > i);"),
 ("RQS parent radius not squared", "adapt.c", "    const double tau2 = tc * tc;", "    const double tau2 = tc;"),
 ("probe truncation", "oracle.c", "    float v = ((float)p + off) + 0.5f;", "    float v = ((float)p + off);"),
 ("walk left/right swapped", "oracle.c", "        n = (f >= tau[n]) ? 2 * n + 2 : 2 * n + 1;", "        n = (f >= tau[n]) ? 2 * n + 1 : 2 * n + 2;"),
 ("DA-RGB channel of p", "oracle.c", "    const float cq = (float)rgb[q * 3 + nchannel];", "    const float cq = (float)rgb[q * 3 + 0];"),
 ("ICP inlier radius 2x", "icp.c", "            if (e[0] * e[0] + e[1] * e[1] + e[2] * e[2] > dist * dist)", "            if (e[0] * e[0] + e[1] * e[1] + e[2] * e[2] > 4.0 * dist * dist)"),
 ("ICP ridge not scaled", "icp.c", "                A[6 * i + i] += ip->ridge * tr / 6.0;", "                A[6 * i + i] += ip->ridge;"),
 ("ICP min_frac ignored", "icp.c", "    return S.n_valid > 0 && (double)S.n_in >= ip->min_frac * (double)S.n_valid;", "    return S.n_valid > 0;"),
 ("reservoir draw U[0, c-1]", "oracle.c", "                    uint64_t j = ((uint64_t)r[0] * ((uint64_t)c + 1)) >> 32; /* U[0, c] */",
  "                    uint64_t j = ((uint64_t)r[0] * ((uint64_t)c)) >> 32;"),
 ("reservoir grid from 0", "oracle.c", "    for (int y = grid_origin; y < H; y += grid_step) {", "    for (int y = 0; y < H; y += grid_step) {"),
 ("forest p_depth inverted", "oracle.c", "            const int is_depth = (double)r0[0] < (double)p_depth * 4294967296.0;",
  "            const int is_depth = (double)r0[0] >= (double)p_depth * 4294967296.0;"),
 ("cluster size floor strict", "adapt.c", "        if (parent[r] < 0 && csize[r] >= min_cluster_size)", "        if (parent[r] < 0 && csize[r] > min_cluster_size)"),
 ("clusters ascending", "adapt.c", "        while (b >= 0 && csize[order[b]] < csize[v]) {", "        while (b >= 0 && csize[order[b]] > csize[v]) {"),
 ("covariance biased", "adapt.c", "            cov[6 * k + q] = cnt > 1 ? c[q] / (double)(cnt - 1) : 0.0;", "            cov[6 * k + q] = cnt > 1 ? c[q] / (double)cnt : 0.0;"),
 ("colour centroid truncated", "adapt.c", "        colour[3 * k + 0] = (uint8_t)((sr + cnt / 2) / cnt);", "        colour[3 * k + 0] = (uint8_t)(sr / cnt);"),
 ("eps on one diagonal only", "adapt.c", "    const double d = cov[3] + eps, e = cov[4], f = cov[5] + eps;", "    const double d = cov[3], e = cov[4], f = cov[5];"),
 ("cascade strict threshold", "ransac.c", "        if (l == n_levels - 1 || (out->status == 0 && out->score <= thresholds[l]))",
  "        if (l == n_levels - 1 || (out->status == 0 && out->score < thresholds[l]))"),
 ("ICP rotation Jacobian m x x", "icp.c", "                                 x[1] * m[2] - x[2] * m[1],", "                                 x[2] * m[1] - x[1] * m[2],"),
 ("half rounding truncates", "adapt.c", "    double q = nearbyint(ldexp(a, 10 - E)); /* in [1024, 2048] */",
  "    double q = floor(ldexp(a, 10 - E));"),
 ("forest dy from the dx word", "oracle.c", "            dy[i] = delta_lo + span * unit24(r0[2]);", "            dy[i] = delta_lo + span * unit24(r0[1]);"),
 ("batch draws share the generation tag", "ransac.c", "            uint32_t c[4] = {(uint32_t)b, (4u << 16) | (uint32_t)p->level, (uint32_t)j, (uint32_t)a};",
  "            uint32_t c[4] = {(uint32_t)b, (3u << 16) | (uint32_t)p->level, (uint32_t)j, (uint32_t)a};"),
]
RUNNER = r'''
import sys
sys.path.insert(0, %r)
import oracle
assert oracle.__file__.startswith(%r)
sys.path.insert(1, %r)
import pytest
sys.exit(pytest.main(["tests/test_oracle_pins.py", "tests/test_synth_corruption.py", "-x", "-q", "-p", "no:cacheprovider"]))
''' % (MUT, MUT, ROOT)


def main(only):
    missed = 0
    try:
        for name, f, old, new in M:
            if only and not any(o in name for o in only):
                continue
            dst = os.path.join(MUT, "oracle")
            if os.path.exists(dst):
                shutil.rmtree(dst)
            shutil.copytree(os.path.join(ROOT, "oracle"), dst, ignore=shutil.ignore_patterns("_build", "__pycache__"))
            p = os.path.join(dst, f)
            with open(p) as fh:
                s = fh.read()
            assert s.count(old) == 1, (name, s.count(old))
            with open(p, "w") as fh:
                fh.write(s.replace(old, new))
            r = subprocess.run([sys.executable, "-c", RUNNER], cwd=ROOT, capture_output=True, text=True,
                               timeout=900)
            caught = r.returncode != 0
            missed += not caught
            last = [ln for ln in r.stdout.splitlines() if "FAILED" in ln or "passed" in ln or "failed" in ln][-2:]
            print(f"{'CAUGHT' if caught else 'MISSED'}  {name}: {' | '.join(last)[:160]}", flush=True)
    finally:
        shutil.rmtree(MUT, ignore_errors=True)
    return missed


if __name__ == "__main__":
    sys.exit(1 if main(sys.argv[1:]) else 0)
