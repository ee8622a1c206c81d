"""Seeded synthetic inputs for the notched-specimen workloads.

This module draws random numbers only; it holds none of the method's arithmetic (no mesh,
no basis, no constitutive law), so the oracle side and the CUDA side can both be fed from it.
Every generator takes an integer seed and uses NumPy's PCG64 through ``default_rng``.
"""
import numpy as np

__all__ = ["displacement_noise", "uniform_phase", "phi_old_above", "lognormal_field", "normal_vector"]


def _rng(seed, stream):
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(stream)]))


def displacement_noise(n_nodes, dim, seed, std=1e-3):
    """dim * n_nodes independent N(0, std^2) values (component blocked)."""
    return _rng(seed, 1).normal(0.0, std, dim * n_nodes)


def uniform_phase(n_nodes, seed, lo=0.9, hi=1.0):
    """n_nodes independent U(lo, hi) values."""
    return _rng(seed, 2).uniform(lo, hi, n_nodes)


def phi_old_above(phi, seed, width=2e-8):
    """min(1, phi + U(0, width)): a previous phase field a little above phi."""
    return np.minimum(1.0, phi + _rng(seed, 3).uniform(0.0, width, len(phi)))


def lognormal_field(n_nodes, seed, mean=2.7e-3, sigma=0.2):
    """Lognormal values with E[X] = mean: underlying normal N(ln(mean) - sigma^2/2, sigma^2)."""
    return np.exp(_rng(seed, 4).normal(np.log(mean) - 0.5 * sigma ** 2, sigma, n_nodes))


def normal_vector(n, seed, stream=5):
    """n independent N(0, 1) values (test directions, right-hand sides)."""
    return _rng(seed, stream).normal(0.0, 1.0, n)
