"""Pins of the oracle's 1D bases and meshes against closed forms and the paper's printed DoF counts."""
import os

import numpy as np
import pytest

from oracle import basis, mesh as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gll_nodes_closed_forms():
    # GLL nodes on [-1, 1]: p=2 {0}, p=3 {+-1/sqrt5}, p=4 {0, +-sqrt(3/7)} plus the end points
    np.testing.assert_allclose(basis.gll_nodes(1), [0.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(basis.gll_nodes(2), [0.0, 0.5, 1.0], atol=1e-15)
    s = 1 / np.sqrt(5)
    np.testing.assert_allclose(basis.gll_nodes(3), [0, (1 - s) / 2, (1 + s) / 2, 1], atol=1e-15)
    s = np.sqrt(3 / 7)
    np.testing.assert_allclose(basis.gll_nodes(4), [0, (1 - s) / 2, 0.5, (1 + s) / 2, 1], atol=1e-15)


def test_gll_weights_closed_forms():
    np.testing.assert_allclose(basis.gll_weights(1), [0.5, 0.5], atol=1e-15)
    np.testing.assert_allclose(basis.gll_weights(2), [1 / 6, 2 / 3, 1 / 6], atol=1e-15)
    np.testing.assert_allclose(basis.gll_weights(3), [1 / 12, 5 / 12, 5 / 12, 1 / 12], atol=1e-15)
    np.testing.assert_allclose(basis.gll_weights(4), [1 / 20, 49 / 180, 32 / 90, 49 / 180, 1 / 20], atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_gauss_exact_for_degree_2n_minus_1(n):
    x, w = basis.gauss_legendre(n)
    for k in range(2 * n):
        assert abs(w @ x ** k - 1.0 / (k + 1)) < 1e-15
    # and not exact one degree higher (checks that the rule really has n points)
    assert abs(w @ x ** (2 * n) - 1.0 / (2 * n + 1)) > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_cardinal_and_derivative(p):
    nodes = basis.gll_nodes(p)
    L, dL = basis.lagrange(nodes, nodes)
    np.testing.assert_allclose(L, np.eye(p + 1), atol=1e-14)
    # reproduce every monomial of degree <= p and its derivative
    x = np.linspace(0, 1, 7)
    Lx, dLx = basis.lagrange(nodes, x)
    for k in range(p + 1):
        np.testing.assert_allclose(Lx @ nodes ** k, x ** k, atol=1e-13)
        np.testing.assert_allclose(dLx @ nodes ** k, k * x ** max(k - 1, 0) if k else 0 * x, atol=1e-12)


def test_paper_dof_counts_with_duplicated_slit():
    """Table tab:slit:dofs:p: counts of the paper's specimen (slit cut into the mesh)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "dof_counts_slit.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 8
    for lvl, p, dofs in rows:
        m = M.Mesh(2, int(p), 2 ** int(lvl))
        assert m.n_dofs_duplicated_slit() == int(dofs)


@pytest.mark.parametrize("dim,p,N,expected", [
    (2, 1, 32, 3267), (2, 1, 256, 198147), (2, 2, 256, 789507), (2, 3, 256, 1774083),
    (2, 4, 256, 3151875), (2, 2, 128, 198147), (3, 2, 64, 8586756), (3, 3, 48, 12194500)])
def test_dof_counts_without_duplication(dim, p, N, expected):
    # (d+1)(pN+1)^d, computed from the node set (not the formula)
    n1 = p * N + 1
    assert (dim + 1) * n1 ** dim == expected
    if n1 ** dim < 3e5:
        m = M.Mesh(dim, p, N)
        assert m.n_dofs == expected and len(np.unique(m.cell_nodes)) == m.n_nodes


def test_level_sizes():
    assert M.level_sizes(32) == [32, 16, 8, 4]
    assert M.level_sizes(48) == [48, 24, 12, 6, 3]
    assert M.level_sizes(256) == [256, 128, 64, 32, 16, 8, 4]
    assert M.level_sizes(64) == [64, 32, 16, 8, 4]


@pytest.mark.parametrize("dim,p,N", [(2, 1, 4), (2, 3, 4), (3, 2, 2)])
def test_mesh_structure(dim, p, N):
    m = M.Mesh(dim, p, N)
    # every cell's nodes span a box of edge h, and node coordinates are inside [0, 1]
    c = m.coords[m.cell_nodes]
    ext = c.max(axis=1) - c.min(axis=1)
    np.testing.assert_allclose(ext, m.h, atol=1e-14)
    assert m.coords.min() == 0.0 and abs(m.coords.max() - 1.0) < 1e-15
    # each interior vertex is shared by 2^d cells
    cnt = np.bincount(m.cell_nodes.ravel(), minlength=m.n_nodes)
    assert cnt.max() == 2 ** dim
    # Dirichlet: every displacement component on bottom and top faces
    nb = (p * N + 1) ** (dim - 1)
    assert m.dirichlet_mask().sum() == 2 * dim * nb
    # slit: pN/2 + 1 nodes per line on the mid line / plane
    assert len(m.slit_nodes()) == (p * N // 2 + 1) * (p * N + 1) ** (dim - 2)
