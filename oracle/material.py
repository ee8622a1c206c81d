"""Pointwise constitutive laws of the AT2 phase-field model (oracle; test infrastructure only).

Sec. 2.1 of the paper:
* degradation g(phi) = (1 - kappa) phi^2 + kappa;
* strain e = (grad u + grad u^T) / 2, solid energy E_s = lambda/2 tr(e)^2 + mu e:e;
* Miehe split: E_s^+ = lambda/2 <tr e>_+^2 + mu tr(e_+^2), e_+ = sum_i lambda_i^+ v_i v_i^T,
  sigma^+ = lambda <tr e>_+ I + 2 mu e_+; E_s^- = E_s - E_s^+, sigma^- = sigma - sigma^+;
* "isotropic" runs (no split, Sec. 5): E_s^+ = E_s, sigma^+ = sigma, sigma^- = 0.

Sec. 3.5: derivative of e_+ by the linearised eigen-system, Eqs. (lin_lambda), (lin_v) and
Alg. 2, and the derivative of sigma^+ (the formula below Alg. 2's introduction).

Readings taken where the paper is silent or garbled (all documented in the design notes):
* Alg. 2 divides by lambda_j - lambda_i, which is 0 for repeated eigenvalues. For the tangent the
  oracle uses the divided-difference form of the same derivative,
  d(e_+)[dA] = V (Theta o (V^T dA V)) V^T, Theta_ij = (l_i^+ - l_j^+)/(l_i - l_j) for l_i != l_j and
  Theta_ij = H(l_i) for l_i == l_j, with H(x) = 1 for x >= 0 (Alg. 2 takes d lambda^+ = d lambda at
  lambda = 0). ``alg2_dplus`` is Alg. 2 itself; the tests check both agree for distinct eigenvalues.
* The trace switch of d sigma^+ uses tr(e) < 0 -> 0, else 1 (as printed).
* Eigenvalues and the trace whose magnitude is at most ZERO_TOL times the largest eigenvalue
  magnitude are taken as exactly 0 before any switch or positive part is evaluated: where a strain
  component is rounding noise (e.g. a displacement constant along a direction), the sign of such an
  eigenvalue is noise and would flip H and the tangent.
"""
import numpy as np

SPLIT_NONE = 0
SPLIT_MIEHE = 1
ZERO_TOL = 1e-12


def g(phi, kappa):
    return (1.0 - kappa) * phi ** 2 + kappa


def dg(phi, kappa):
    return 2.0 * (1.0 - kappa) * phi


def ddg(phi, kappa):
    return 2.0 * (1.0 - kappa) * np.ones_like(np.asarray(phi, dtype=np.float64))


def heaviside(x):
    """H(x) = 1 for x >= 0, else 0."""
    return (np.asarray(x) >= 0.0).astype(np.float64)


def sym(a):
    return 0.5 * (a + np.swapaxes(a, -1, -2))


def trace(a):
    return np.trace(a, axis1=-2, axis2=-1)


def eye_like(a):
    d = a.shape[-1]
    return np.broadcast_to(np.eye(d), a.shape)


def eig_snapped(e):
    """numpy.linalg.eigh with eigenvalues of magnitude <= ZERO_TOL * max|lambda| set to 0."""
    lam, V = np.linalg.eigh(e)
    scale = np.max(np.abs(lam), axis=-1, keepdims=True)
    return np.where(np.abs(lam) <= ZERO_TOL * scale, 0.0, lam), V


def snapped_trace(e):
    """tr(e), set to 0 when its magnitude is at most ZERO_TOL * max|lambda|."""
    tr = trace(e)
    scale = np.max(np.abs(np.linalg.eigvalsh(e)), axis=-1)
    return np.where(np.abs(tr) <= ZERO_TOL * scale, 0.0, tr)


def positive_part(e):
    """e_+ = sum_i max(0, lambda_i) v_i v_i^T (eigen-decomposition by numpy.linalg.eigh)."""
    lam, V = eig_snapped(e)
    return np.einsum("...ik,...k,...jk->...ij", V, np.maximum(lam, 0.0), V)


def stress_energy(e, lam, mu, split):
    """Returns (sigma^+, sigma^-, E_s^+, E_s) at strain e (..., d, d); lam, mu broadcast over (...)."""
    lam = np.asarray(lam, dtype=np.float64)[..., None, None]
    mu = np.asarray(mu, dtype=np.float64)[..., None, None]
    tr = trace(e)[..., None, None]
    I = eye_like(e)
    sig = lam * tr * I + 2.0 * mu * e
    Es = (0.5 * lam * tr ** 2 + mu * np.einsum("...ij,...ij->...", e, e)[..., None, None])[..., 0, 0]
    if split == SPLIT_NONE:
        return sig, np.zeros_like(sig), Es, Es
    ep = positive_part(e)
    trp = np.maximum(snapped_trace(e), 0.0)[..., None, None]
    sigp = lam * trp * I + 2.0 * mu * ep
    Esp = (0.5 * lam * trp ** 2)[..., 0, 0] + mu[..., 0, 0] * np.einsum("...ij,...ij->...", ep, ep)
    return sigp, sig - sigp, Esp, Es


def alg2_dplus(A, dA):
    """Derivative of A_+ at A in direction dA, following Alg. 2 step by step (single matrix).

    Requires pairwise distinct eigenvalues (Alg. 2 divides by lambda_j - lambda_i).
    """
    A = np.asarray(A, dtype=np.float64)
    d = A.shape[0]
    lam, V = np.linalg.eigh(A)  # decompose A = V D V^T
    dV = np.zeros((d, d))
    dlam_plus = np.zeros(d)
    for i in range(d):
        # L = A - lambda_i I has pseudo-inverse V Ddag V^T, Ddag = diag(1/(lambda_j - lambda_i)), 0 at j = i
        Ddag = np.zeros(d)
        for j in range(d):
            if j != i:
                Ddag[j] = 1.0 / (lam[j] - lam[i])
        Ldag = V @ np.diag(Ddag) @ V.T
        dV[:, i] = -Ldag @ dA @ V[:, i]          # Eq. (lin_v)
        dlam = V[:, i] @ dA @ V[:, i]            # Eq. (lin_lambda)
        dlam_plus[i] = dlam if lam[i] >= 0.0 else 0.0
    Dp = np.diag(np.maximum(lam, 0.0))
    return dV @ Dp @ V.T + V @ np.diag(dlam_plus) @ V.T + V @ Dp @ dV.T


def theta_matrix(lam):
    """Divided differences of x -> max(x, 0) at the eigenvalues (..., d) -> (..., d, d)."""
    li = lam[..., :, None]
    lj = lam[..., None, :]
    num = np.maximum(li, 0.0) - np.maximum(lj, 0.0)
    den = li - lj
    same = den == 0.0
    safe = np.where(same, 1.0, den)
    H = np.broadcast_to(heaviside(li), num.shape)
    return np.where(same, H, num / safe)


def dplus(e, de):
    """d(e_+)[de] in divided-difference form (equal to Alg. 2 for distinct eigenvalues)."""
    lam, V = eig_snapped(e)
    Th = theta_matrix(lam)
    W = np.einsum("...ki,...kl,...lj->...ij", V, de, V)
    return np.einsum("...ik,...kl,...jl->...ij", V, Th * W, V)


def dstress(e, de, lam, mu, split):
    """(d sigma^+[de], d sigma^-[de]) at strain e, direction de (both symmetric)."""
    lam = np.asarray(lam, dtype=np.float64)[..., None, None]
    mu = np.asarray(mu, dtype=np.float64)[..., None, None]
    I = eye_like(e)
    trd = trace(de)[..., None, None]
    dsig = lam * trd * I + 2.0 * mu * de
    if split == SPLIT_NONE:
        return dsig, np.zeros_like(dsig)
    Ht = heaviside(snapped_trace(e))[..., None, None]
    dsigp = lam * Ht * trd * I + 2.0 * mu * dplus(e, de)
    return dsigp, dsig - dsigp


def tangent4(e, lam, mu, gt, split):
    """Fourth-order tangent T[k, j, l, m] = (g(phi~) d sigma^+ + d sigma^-)[sym(E_lm)]_{kj}.

    Contracting T with the displacement gradient of a direction gives the u-test coefficient of
    the first two terms of Eq. (G)."""
    d = e.shape[-1]
    out = np.zeros(e.shape[:-2] + (d, d, d, d))
    gt = np.asarray(gt, dtype=np.float64)[..., None, None]
    for l in range(d):
        for m in range(d):
            E = np.zeros((d, d))
            E[l, m] += 0.5
            E[m, l] += 0.5
            de = np.broadcast_to(E, e.shape)
            dp, dm = dstress(e, de, lam, mu, split)
            out[..., :, :, l, m] = gt * dp + dm
    return out
