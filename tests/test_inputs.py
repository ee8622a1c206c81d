"""The seeded input recipe: reproducible per seed, independent streams, and the distributions it
states (checked by sample statistics on large draws)."""
import numpy as np
import pytest

from paper_2005_00331_gb300 import inputs


def test_reproducible_and_seed_dependent():
    a = inputs.displacement_noise(1000, 2, 7)
    np.testing.assert_array_equal(a, inputs.displacement_noise(1000, 2, 7))
    assert not np.array_equal(a, inputs.displacement_noise(1000, 2, 8))
    # generators draw from separate streams: same seed, different sequences
    assert not np.allclose(inputs.normal_vector(1000, 7), inputs.displacement_noise(1000, 1, 7) / 1e-3)


def test_stated_distributions():
    n = 200_000
    u = inputs.displacement_noise(n, 1, 0)
    assert abs(u.mean()) < 5 * 1e-3 / np.sqrt(n) and u.std() == pytest.approx(1e-3, rel=0.01)
    phi = inputs.uniform_phase(n, 0)
    assert phi.min() >= 0.9 and phi.max() < 1.0 and phi.mean() == pytest.approx(0.95, abs=1e-3)
    po = inputs.phi_old_above(phi, 0)
    d = po - phi
    assert d.min() >= 0.0 and d.max() <= 2e-8 and np.all(po <= 1.0)
    g = inputs.lognormal_field(n, 0)
    # lognormal with E[X] = 2.7e-3 and sigma 0.2 of the underlying normal
    assert g.mean() == pytest.approx(2.7e-3, rel=0.005)
    assert np.log(g).std() == pytest.approx(0.2, rel=0.01)
    assert np.median(g) == pytest.approx(2.7e-3 * np.exp(-0.02), rel=0.005)
