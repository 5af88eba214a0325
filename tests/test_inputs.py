"""The seeded input generators (paper_2410_00233_gb300/inputs.py) follow their stated recipe:
reproducible counter-based streams, PSFs normalised, odd and centred, separable PSFs of
Kronecker rank 1 and non-separable ones of higher rank, piecewise-constant images in [0, 1]
on a zero background, the noise scaled to exactly eta ||b_true|| (Sec. 5.3.2), and the
workload mixes (medium: n = 128, 31 x 31, reflexive, 1 %/5 % noise, automatic rank; batched:
n cycling 64..384, odd s in [15, 63], k in [5, 20], p = max(2, (k + 3) // 4), boundary, TV
type and PSF family alternating independently of n)."""
import numpy as np
import pytest

from paper_2410_00233_gb300 import inputs as I


def test_streams_are_reproducible_and_distinct():
    a = I.gaussian(1000, I.rng(7))
    assert np.array_equal(a, I.gaussian(1000, I.rng(7)))
    assert not np.array_equal(a, I.gaussian(1000, I.rng(8)))
    assert abs(a.mean()) < 0.15 and abs(a.std() - 1.0) < 0.1


@pytest.mark.parametrize("make", [
    lambda g: I.psf_gaussian(9, 1.5, 3.0, 30.0),
    lambda g: I.psf_gaussian_mixture(31, g),
    lambda g: I.psf_turbulence(63, g),
    lambda g: I.psf_separable(15, g),
    lambda g: I.psf_random(7, g),
])
def test_psfs_are_normalised_positive_odd(make):
    p = make(I.rng(3))
    assert p.shape[0] == p.shape[1] and p.shape[0] % 2 == 1
    assert np.all(p > 0.0)
    assert abs(p.sum() - 1.0) < 1e-12


def test_gaussian_psf_peaks_at_the_centre_and_is_point_symmetric():
    p = I.psf_gaussian(11, 1.2, 2.5, 40.0)
    c = 11 // 2
    assert np.unravel_index(np.argmax(p), p.shape) == (c, c)
    assert np.allclose(p, p[::-1, ::-1], rtol=0, atol=1e-15)


def test_separable_psf_has_rank_one_and_speckle_psf_does_not():
    g = I.rng(11)
    sv = np.linalg.svd(I.psf_separable(15, g), compute_uv=False)
    assert sv[1] < 1e-13 * sv[0]
    sv = np.linalg.svd(I.psf_turbulence(31, g), compute_uv=False)
    assert np.sum(sv > 1e-3 * sv[0]) >= 8  # slowly decaying Kronecker spectrum


def test_images_are_piecewise_constant_on_zero_background():
    x = I.image_piecewise_constant(64, I.rng(5))
    assert x.shape == (64, 64) and x.min() >= 0.0 and x.max() <= 1.0
    assert np.mean(x == 0.0) > 0.05  # background left
    assert 1 < len(np.unique(x)) <= 3 + 64 // 16 + 1  # one value per shape, plus zero


def test_noise_has_exactly_the_stated_relative_norm():
    g = I.rng(2)
    b = g.uniform(size=(20, 20))
    for eta in (0.01, 0.05, 0.07):
        e = I.noise_vector(b, eta, I.gaussian((20, 20), g))
        assert abs(np.linalg.norm(e) / np.linalg.norm(b) - eta) < 1e-14


def test_medium_workload_recipe():
    for i in range(4):
        pr = I.problem_medium(i)
        assert pr.n == 128 and pr.psf.shape == (31, 31) and pr.bc == I.BC_REFLEXIVE
        assert pr.eta == (0.01 if i % 2 == 0 else 0.05)
        assert pr.tau == 1e-3 and pr.k == 30 and pr.iso
        assert pr.zeta.shape == (128, 128) and pr.start.shape == (128 * 128,)
    assert not np.array_equal(I.problem_medium(0).psf, I.problem_medium(1).psf)


def test_batched_workload_recipe():
    probs = [I.problem_batched(i) for i in range(16)]
    assert [p.n for p in probs[:4]] == [64, 128, 256, 384]
    for i, p in enumerate(probs):
        s = p.psf.shape[0]
        assert s % 2 == 1 and 15 <= s <= 63 and s <= p.n
        assert 5 <= p.k <= 20 and p.p == max(2, (p.k + 3) // 4)
        assert 0.01 <= p.eta <= 0.05
        assert p.bc == (i // 4) % 2 and p.iso == bool((i // 8) % 2)
    full = [I.problem_batched(i) for i in range(96)]
    for n in (64, 128, 256, 384):  # every size carries every boundary / TV combination
        assert {(p.bc, p.iso) for p in full if p.n == n} == {(0, False), (0, True), (1, False), (1, True)}
