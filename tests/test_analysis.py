"""Post-processing of the validation observables (host arithmetic, no GPU):
the tanh interface fit of Eq. tanh and the g(r) normalisation."""
import math

import numpy as np
import pytest

from paper_2510_21230_gb300 import analysis, synth


def _two_interface_profile(L, nb, zc, right, left):
    z = (np.arange(nb) + 0.5) * L / nb
    u = (z - zc + 0.5 * L) % L - 0.5 * L
    rho = np.where(u >= 0.0,
                   analysis.tanh_profile(u, right[0], right[1], right[2], right[3]),
                   analysis.tanh_profile(-u, left[0], left[1], left[2], left[3]))
    return z, rho


@pytest.mark.parametrize("zc", [37.5, 60.0, 110.0])
def test_fit_recovers_exact_tanh_interfaces(zc):
    """A profile made of two Eq. tanh halves (different widths and positions,
    slab centre anywhere, even across the periodic boundary) is fitted back."""
    L, nb = 120.0, 600
    z, rho = _two_interface_profile(L, nb, zc, (0.70, 0.02, 15.0, 2.5), (0.70, 0.02, 14.0, 3.0))
    f = analysis.fit_interfaces(z, rho, L)
    assert f["right"]["rho_l"] == pytest.approx(0.70, abs=1e-4)
    assert f["right"]["rho_g"] == pytest.approx(0.02, abs=1e-4)
    assert f["right"]["d"] == pytest.approx(2.5, rel=1e-3)
    assert f["left"]["d"] == pytest.approx(3.0, rel=1e-3)
    # circular distance of the fitted interface positions from the true ones
    for side, off in (("right", zc + 15.0), ("left", zc - 14.0)):
        dz = (f[side]["z0"] - off + 0.5 * L) % L - 0.5 * L
        assert abs(dz) < 0.05, side


def test_fit_tolerates_counting_noise():
    L, nb = 75.0, 600
    z, rho = _two_interface_profile(L, nb, 40.0, (0.73, 0.018, 12.0, 2.2), (0.73, 0.018, 12.0, 2.2))
    rng = np.random.default_rng(81)
    noisy = rho + rng.normal(0.0, 0.01, size=rho.shape)
    f = analysis.fit_interfaces(z, noisy, L)
    for side in ("right", "left"):
        assert f[side]["rho_l"] == pytest.approx(0.73, abs=0.01)
        assert f[side]["rho_g"] == pytest.approx(0.018, abs=0.01)
        assert f[side]["d"] == pytest.approx(2.2, rel=0.15)
        assert f[side]["rms"] < 0.02


def test_slab_start_profile_fits_its_recipe():
    """The synthetic slab start (liquid 0.73, vapour 0.02, 30 sigma thick,
    centred in a 120-sigma box) fits to those densities and a sharp interface."""
    cfg = synth.slab()
    L = cfg["box"]
    nb = 600
    counts = np.bincount(np.minimum((cfg["x"][2] / (L[2] / nb)).astype(int), nb - 1), minlength=nb)
    z, rho = analysis.density_profile(counts, 1, L)
    f = analysis.fit_interfaces(z, rho, L[2])
    assert f["centre"] == pytest.approx(60.0, abs=0.5)
    for side in ("right", "left"):
        assert f[side]["rho_l"] == pytest.approx(0.73, rel=0.05)
        assert f[side]["rho_g"] == pytest.approx(0.02, abs=0.01)
    assert (f["right"]["z0"] - f["left"]["z0"]) == pytest.approx(30.0, abs=1.5)


def test_rdf_normalisation_of_uniform_pairs():
    """Counts proportional to the shell volumes with the ideal-gas total give g = 1."""
    n, V, r_max, nb = 1000, 1250.0, 2.5, 25
    edges = np.linspace(0.0, r_max, nb + 1)
    shell = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    counts = 0.5 * n * (n / V) * shell * 7
    r, g = analysis.rdf(counts, 7, n, V, r_max)
    assert np.allclose(g, 1.0)
    assert r[0] == pytest.approx(0.05)
