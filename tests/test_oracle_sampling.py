"""Pins of the sampling oracle (Sec. 5.2, Fig. sampleNDF) against facts that
do not come from the oracle's own descent: the NDF image from point queries
(Eq. 4), the product form of a rank-1 material, a hand-worked choice, and the
statistics of many samples."""
import numpy as np
import pytest

import synth
from oracle import sampling as osm


def _material(N, L, B, R, seed, signed=False):
    mat = {}
    for i, (k, n) in enumerate((("fx", N), ("fy", N), ("flw", L), ("fs", B), ("ft", B))):
        u = synth.uniform(seed, 60 + i, n * R).reshape(n, R)
        mat[k] = 2 * u - 1 if signed else u
    return mat


@pytest.mark.parametrize("B,R", [(2, 1), (8, 3), (16, 5), (32, 2)])
def test_bin_probabilities_are_the_normalised_ndf_image(B, R):
    # telescoping: a quad's average times its area is the sum of its bins, so
    # the product of the step probabilities along a path is bin / image sum
    mat = _material(16, 5, B, R, 7 + B)
    pmf = osm.bin_pmf(mat, 3, 9, 2.6)
    img = osm.ndf_image(mat, 3, 9, 2.6)
    assert np.allclose(pmf, img / img.sum(), rtol=1e-12, atol=1e-15)


def test_rank_one_material_samples_s_and_t_independently():
    mat = _material(8, 4, 16, 1, 3)
    pmf = osm.bin_pmf(mat, 1, 2, 1.0)
    ps = mat["fs"][:, 0] / mat["fs"][:, 0].sum()
    pt = mat["ft"][:, 0] / mat["ft"][:, 0].sum()
    assert np.allclose(pmf, np.outer(ps, pt), rtol=1e-12, atol=1e-15)


def test_choice_rule_hand_worked():
    q4 = np.array([1.0, 2.0, 3.0, 4.0])  # cumulative 1, 3, 6, 10
    for u, k in ((0.05, 0), (0.1, 1), (0.15, 1), (0.35, 2), (0.6, 3), (0.65, 3), (0.999, 3)):
        assert osm.choose(q4, u)[0] == k, (u, k)
    assert osm.choose(q4, 0.35)[1] == pytest.approx(0.3)
    # a negative average is clamped to 0 and can never be chosen
    neg = np.array([-1.0, 2.0, 0.0, 2.0])
    assert [osm.choose(neg, u)[0] for u in (0.0, 0.49, 0.5, 0.99)] == [1, 1, 3, 3]
    # all clamped to 0: uniform over the four quads
    assert [osm.choose(np.array([-1.0, -2.0, 0.0, -3.0]), u)[0] for u in (0.1, 0.3, 0.6, 0.9)] == [0, 1, 2, 3]


def test_signed_material_gives_a_distribution():
    mat = _material(8, 4, 16, 6, 11, signed=True)
    pmf = osm.bin_pmf(mat, 5, 1, 3.0)
    assert np.all(pmf >= 0.0)
    assert pmf.sum() == pytest.approx(1.0, abs=1e-12)
    img = osm.ndf_image(mat, 5, 1, 3.0)
    assert np.any(img < 0) and img.sum() > 0  # the case exercises the clamping
    # a bin with a negative value is never reached: its own clamped probability
    # is 0, or an ancestor's average is <= 0 and that ancestor's probability is 0
    assert np.all(pmf[img < 0] == 0.0)
    u = synth.sample_uniforms(5, 4000).astype(np.float64)
    for i in range(4000):
        s, t, p, v, _ = osm.sample(mat, 5, 1, 3.0, u[i])
        assert v >= 0.0 and p > 0.0


def test_samples_follow_the_pmf_and_stay_in_their_bin():
    B = 8
    mat = _material(16, 5, B, 3, 21)
    pmf = osm.bin_pmf(mat, 7, 2, 1.5)
    img = osm.ndf_image(mat, 7, 2, 1.5)
    n = 30_000
    u = synth.sample_uniforms(9, n).astype(np.float64)
    cnt = np.zeros((B, B))
    for i in range(n):
        s, t, p, v, _ = osm.sample(mat, 7, 2, 1.5, u[i])
        b_s, b_t = int(np.floor(s)), int(np.floor(t))
        assert s - b_s == pytest.approx(u[i, 6]) and t - b_t == pytest.approx(u[i, 7])
        assert p == pytest.approx(pmf[b_s, b_t], rel=1e-12)
        assert v == pytest.approx(img[b_s, b_t], rel=1e-12)
        cnt[b_s, b_t] += 1
    exp = n * pmf
    chi2 = float(((cnt - exp) ** 2 / exp).sum())
    dof = B * B - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), chi2
