"""1D bases for Q_p elements (oracle; test infrastructure only).

The paper uses continuous Q_p elements (Sec. 3.1) and refers to the standard matrix-free
setting of Kronbichler and Kormann for the operator evaluation (Sec. 3.4). The paper does
not name the node set or the quadrature; this oracle takes Lagrange polynomials on the
Gauss-Lobatto-Legendre (GLL) nodes and (p+1) Gauss-Legendre points per direction.

All points and nodes live on the unit interval [0, 1].
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0, 1]: (points, weights), weights sum to 1."""
    x, w = npleg.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def gll_nodes(p):
    """p+1 Gauss-Lobatto-Legendre nodes on [0, 1]: the end points and the roots of P_p'."""
    if p < 1:
        raise ValueError("degree must be >= 1")
    if p == 1:
        xi = np.array([-1.0, 1.0])
    else:
        inner = npleg.Legendre.basis(p).deriv().roots()
        xi = np.concatenate([[-1.0], np.sort(np.real(inner)), [1.0]])
    return 0.5 * (xi + 1.0)


def gll_weights(p):
    """GLL quadrature weights on [0, 1]: w_k = 1 / (p (p+1) P_p(xi_k)^2) on [-1, 1], halved."""
    xi = 2.0 * gll_nodes(p) - 1.0
    Pp = npleg.Legendre.basis(p)(xi)
    return 0.5 * 2.0 / (p * (p + 1) * Pp ** 2)


def lagrange(nodes, x):
    """Values and first derivatives of the Lagrange polynomials on ``nodes`` at points ``x``.

    Returns (L, dL), both of shape (len(x), len(nodes)), with
    L[i, k] = prod_{m != k} (x_i - x_m) / (x_k - x_m) and dL its derivative in x.
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nn = len(nodes)
    L = np.ones((len(x), nn))
    dL = np.zeros((len(x), nn))
    for k in range(nn):
        for m in range(nn):
            if m != k:
                L[:, k] *= (x - nodes[m]) / (nodes[k] - nodes[m])
        for j in range(nn):
            if j == k:
                continue
            term = np.full(len(x), 1.0 / (nodes[k] - nodes[j]))
            for m in range(nn):
                if m != k and m != j:
                    term *= (x - nodes[m]) / (nodes[k] - nodes[m])
            dL[:, k] += term
    return L, dL
