"""Pins of the oracle's pointwise laws: split identities, Alg. 2, tangents against finite differences."""
import numpy as np
import pytest

from oracle import material as mat

LAM, MU = 121.15, 80.77


def rand_sym(rng, d, n, away_from_kinks=False):
    a = rng.normal(size=(4 * n if away_from_kinks else n, d, d))
    a = 0.5 * (a + np.swapaxes(a, 1, 2))
    if away_from_kinks:
        # finite differences straddling a kink of x -> max(x, 0) are not derivatives
        lam = np.linalg.eigvalsh(a)
        ok = (np.abs(lam).min(axis=1) > 0.05) & (np.abs(np.trace(a, axis1=1, axis2=2)) > 0.05)
        a = a[ok][:n]
    return a


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_split_identities(d, split):
    rng = np.random.default_rng(1)
    e = rand_sym(rng, d, 200, away_from_kinks=True)
    sp, sm, Esp, Es = mat.stress_energy(e, LAM, MU, split)
    sig = LAM * np.trace(e, axis1=1, axis2=2)[:, None, None] * np.eye(d) + 2 * MU * e
    np.testing.assert_allclose(sp + sm, sig, rtol=1e-13, atol=1e-12)
    # E_s^+ <= E_s and both parts non-negative
    assert np.all(Esp >= -1e-14) and np.all(Es - Esp >= -1e-12)
    # Euler: E_s^+ is homogeneous of degree 2, so sigma^+ : e = 2 E_s^+
    np.testing.assert_allclose(np.einsum("nij,nij->n", sp, e), 2 * Esp, rtol=1e-12)
    # sigma^+ = d E_s^+ / d e (central differences of the energy; eigh round-off limits h)
    h = 1e-5
    for (i, j) in [(0, 0), (0, 1), (d - 1, d - 1)]:
        E = np.zeros((d, d))
        E[i, j] += 0.5
        E[j, i] += 0.5
        fd = (mat.stress_energy(e + h * E, LAM, MU, split)[2] - mat.stress_energy(e - h * E, LAM, MU, split)[2]) / (2 * h)
        np.testing.assert_allclose(fd, np.einsum("nij,ij->n", sp, E), rtol=1e-6, atol=1e-6)


def test_positive_part_2d_closed_form():
    # 2x2 symmetric: eigenvalues m +- r, m = tr/2, r = sqrt(((a-c)/2)^2 + b^2)
    rng = np.random.default_rng(2)
    e = rand_sym(rng, 2, 100)
    a, b, c = e[:, 0, 0], e[:, 0, 1], e[:, 1, 1]
    m, r = (a + c) / 2, np.sqrt(((a - c) / 2) ** 2 + b ** 2)
    l1, l2 = m + r, m - r
    # e_+ = l1^+ P1 + l2^+ P2 with projector P1 = (e - l2 I)/(l1 - l2)
    P1 = (e - l2[:, None, None] * np.eye(2)) / (l1 - l2)[:, None, None]
    P2 = np.eye(2) - P1
    ref = np.maximum(l1, 0)[:, None, None] * P1 + np.maximum(l2, 0)[:, None, None] * P2
    np.testing.assert_allclose(mat.positive_part(e), ref, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_alg2_matches_finite_differences_and_divided_differences(d):
    rng = np.random.default_rng(3)
    for _ in range(50):
        A = rand_sym(rng, d, 1, away_from_kinks=True)[0]
        dA = rand_sym(rng, d, 1)[0]
        a2 = mat.alg2_dplus(A, dA)
        h = 1e-6
        fd = (mat.positive_part(A + h * dA) - mat.positive_part(A - h * dA)) / (2 * h)
        np.testing.assert_allclose(a2, fd, atol=1e-7)
        np.testing.assert_allclose(mat.dplus(A[None], dA[None])[0], a2, atol=1e-12)


def test_dplus_repeated_eigenvalues():
    # at A = 0 every eigenvalue is 0 (repeated): Theta = H(0) = 1, d(A_+) = identity map
    for d in (2, 3):
        dA = rand_sym(np.random.default_rng(4), d, 1)[0]
        np.testing.assert_allclose(mat.dplus(np.zeros((1, d, d)), dA[None])[0], dA, atol=1e-15)
        # A = -I: all negative, repeated -> d(A_+) = 0
        np.testing.assert_allclose(mat.dplus(-np.eye(d)[None], dA[None])[0], 0 * dA, atol=1e-15)
        # A = diag(1, 1, ...) positive repeated -> identity map
        np.testing.assert_allclose(mat.dplus(np.eye(d)[None], dA[None])[0], dA, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_dstress_finite_differences(d, split):
    rng = np.random.default_rng(5)
    e = rand_sym(rng, d, 100, away_from_kinks=True)
    de = rand_sym(rng, d, 100)
    dp, dm = mat.dstress(e, de, LAM, MU, split)
    h = 1e-6
    sp1, sm1, _, _ = mat.stress_energy(e + h * de, LAM, MU, split)
    sp0, sm0, _, _ = mat.stress_energy(e - h * de, LAM, MU, split)
    np.testing.assert_allclose(dp, (sp1 - sp0) / (2 * h), rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(dm, (sm1 - sm0) / (2 * h), rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("d", [2, 3])
def test_tangent_at_zero_strain_is_isotropic(d):
    # e = 0: tr e = 0 >= 0 and all eigenvalues 0 -> sigma^+ part carries the whole C; g=1 gives C
    T = mat.tangent4(np.zeros((1, d, d)), LAM, MU, 1.0, mat.SPLIT_MIEHE)[0]
    I = np.eye(d)
    C = LAM * np.einsum("kj,lm->kjlm", I, I) + MU * (np.einsum("kl,jm->kjlm", I, I) + np.einsum("km,jl->kjlm", I, I))
    np.testing.assert_allclose(T, C, atol=1e-12)
    # with degradation g: g * C (everything counted as tensile)
    T2 = mat.tangent4(np.zeros((1, d, d)), LAM, MU, 0.25, mat.SPLIT_MIEHE)[0]
    np.testing.assert_allclose(T2, 0.25 * C, atol=1e-12)


def test_degradation():
    k = 1e-10
    phi = np.linspace(0, 1, 11)
    np.testing.assert_allclose(mat.g(phi, k), (1 - k) * phi ** 2 + k)
    h = 1e-6
    np.testing.assert_allclose(mat.dg(phi, k), (mat.g(phi + h, k) - mat.g(phi - h, k)) / (2 * h), atol=1e-9)
    assert mat.g(0.0, k) == k and abs(mat.g(1.0, k) - 1.0) < 1e-16


@pytest.mark.parametrize("d", [2, 3])
def test_noise_eigenvalues_are_zero(d):
    """An eigenvalue at rounding-noise level (relative 1e-17) of either sign gives the tangent of an
    exact zero eigenvalue (H(0) = 1), and the trace switch likewise."""
    base = np.zeros((1, d, d))
    base[0, d - 1, d - 1] = 1e-3
    Tz = mat.tangent4(base, LAM, MU, 0.3, mat.SPLIT_MIEHE)
    for s in (1.0, -1.0):
        e = base.copy()
        e[0, 0, 0] = s * 1e-20
        np.testing.assert_allclose(mat.tangent4(e, LAM, MU, 0.3, mat.SPLIT_MIEHE), Tz, rtol=1e-12, atol=1e-9)
    # without the snap the negative noise eigenvalue would switch H: check the switch is real
    e = base.copy()
    e[0, 0, 0] = -1e-6
    assert np.abs(mat.tangent4(e, LAM, MU, 0.3, mat.SPLIT_MIEHE) - Tz).max() > 1.0
