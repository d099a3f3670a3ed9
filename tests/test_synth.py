"""The seeded input generators against the distributions they state: the Plummer and NFW
enclosed-mass profiles, the halo mass function, the box, the masses and the seeds.  They hold no
arithmetic of the method; both the oracle and the CUDA path take their output as input."""
import numpy as np
import pytest

from paper_1609_08621_gb300 import synth

stats = pytest.importorskip("scipy.stats")


def test_plummer_radii_follow_the_plummer_mass_profile():
    a = 0.02
    r = synth._plummer_radius(np.random.default_rng(1), a, 20000)
    cdf = lambda x: x ** 3 / (x * x + a * a) ** 1.5  # M(<r) / M
    assert stats.kstest(r, cdf).pvalue > 1e-3
    # the test has the power to see a 10% error in the scale radius
    assert stats.kstest(r, lambda x: x ** 3 / (x * x + (1.1 * a) ** 2) ** 1.5).pvalue < 1e-6


@pytest.mark.parametrize("c", [5.0, 15.0])
def test_nfw_radii_follow_the_nfw_mass_profile(c):
    rvir = 0.05
    r = synth._nfw_radius(np.random.default_rng(2), c, rvir, 20000)
    mu = lambda x: np.log1p(x) - x / (1.0 + x)
    assert np.all((r >= 0) & (r <= rvir))
    assert stats.kstest(r, lambda x: mu(np.minimum(x, rvir) * c / rvir) / mu(c)).pvalue > 1e-3
    assert stats.kstest(r, lambda x: mu(np.minimum(x, rvir) * 1.2 * c / rvir) / mu(1.2 * c)).pvalue < 1e-6


def test_isotropic_directions():
    rng = np.random.default_rng(3)
    p = synth._isotropic(rng, np.ones(40000))
    assert np.allclose(np.linalg.norm(p, axis=0), 1.0)
    for q in range(3):  # each component of a uniform direction is uniform on [-1, 1]
        assert stats.kstest(p[q], "uniform", args=(-1, 2)).pvalue > 1e-3


@pytest.mark.parametrize("gen", ["clustered_plummer", "clustered_nfw", "uniform_box"])
def test_generators_are_seeded_in_the_box_with_equal_masses(gen):
    f = getattr(synth, gen)
    pos, m = f(30000, 7)
    assert pos.shape == (3, 30000) and pos.dtype == np.float64 and m.dtype == np.float32
    assert np.all((pos >= 0.0) & (pos < 1.0))
    assert np.all(m == m[0]) and abs(float(m.astype(np.float64).sum()) - 1.0) < 1e-4
    pos2, _ = f(30000, 7)
    assert np.array_equal(pos, pos2)
    pos3, _ = f(30000, 8)
    assert not np.array_equal(pos, pos3)


def test_clustered_sets_are_clustered():
    """Half (Plummer) or 70% (NFW) of the particles sit in small structures: the densest
    1/1000 of a 32^3 grid holds far more than the uniform share."""
    for f, frac in ((synth.clustered_plummer, 0.5), (synth.clustered_nfw, 0.7)):
        pos, _ = f(50000, 9)
        cells = np.floor(pos * 32).astype(np.int64)
        occ = np.bincount(cells[0] * 1024 + cells[1] * 32 + cells[2], minlength=32 ** 3)
        top = np.sort(occ)[::-1][: 32 ** 3 // 1000]
        assert top.sum() > 0.25 * frac * 50000  # uniform: ~0.1% of the particles


def test_batch_box_sizes():
    boxes, off = synth.batch_boxes(6, 3, n_lo=1000, n_hi=3000)
    ns = np.diff(off)
    assert off[0] == 0 and len(boxes) == 6 and np.all((ns >= 1000) & (ns <= 3000))
    assert all(b[1].size == k for b, k in zip(boxes, ns))


def test_paper_softening_scale():
    # 1/50 of the mean separation n^(-1/3)
    assert synth.paper_softening(128 ** 3) == pytest.approx(1.0 / 6400.0, rel=1e-15)
