"""Pins of the oracle's mesh with the slit cut into it (Sec. 5.1: the slit's nodes duplicated, the
tip shared): the DoF counts the paper prints, the identity that a field continuous across the slit
sees the uncut mesh, the Jacobian as the derivative of the residual, and a slit that opens under
tension."""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fe, material as mat, mesh as M, solvers as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
LAM, MU, GC, KAPPA = 121.15, 80.77, 2.7e-3, 1e-10


def test_cut_mesh_has_the_papers_dof_counts():
    """Table tab:slit:dofs:p, counted on the cut mesh itself (level 9 only for p = 1: the larger
    meshes take minutes to build here)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "dof_counts_slit.txt")) if l.strip() and l[0] != "#"]
    for lvl, p, dofs in rows:
        lvl, p, dofs = int(lvl), int(p), int(dofs)
        if lvl == 9 and p > 1:
            continue
        assert M.Mesh(2, p, 2 ** lvl, slit="duplicate").n_dofs == dofs


def expansion(m):
    """P: uncut layout -> cut layout (duplicates copy their grid node), for all n_comp blocks."""
    ng, nn = m.n_grid_nodes, m.n_nodes
    cols = np.concatenate([np.arange(ng), m.dup_of])
    blocks = [sp.csr_matrix((np.ones(nn), (np.arange(nn), cols)), shape=(nn, ng))] * m.n_comp
    return sp.block_diag(blocks).tocsr()


def random_state(m, rng):
    d, nn = m.dim, m.n_nodes
    U = np.zeros(m.n_dofs)
    U[:d * nn] = rng.normal(0, 1e-2, d * nn)
    U[d * nn:] = rng.uniform(0.6, 1.0, nn)
    return U, np.clip(U[d * nn:] + rng.normal(0, 0.02, nn), 0, 1)


@pytest.mark.parametrize("dim,p,N", [(2, 1, 4), (2, 2, 2), (2, 3, 2), (3, 1, 2)])
@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_continuous_fields_see_the_uncut_mesh(dim, p, N, split):
    """A field equal on both copies of every slit node is a field of the uncut mesh, so the cut mesh's
    residual and Jacobian sum back to the uncut ones: P^T R_cut(P U) = R(U), P^T G_cut P = G."""
    mg, mc = M.Mesh(dim, p, N), M.Mesh(dim, p, N, slit="duplicate")
    assert len(mc.dup_of) == (p * N // 2) * (p * N + 1 if dim == 3 else 1)
    prm = fe.Params(LAM, MU, GC, 0.3, KAPPA, split)
    U, phit = random_state(mg, np.random.default_rng(21))
    P = expansion(mc)
    Rg = fe.residual(mg, prm, U, phit, zero_dirichlet=False)
    Rc = fe.residual(mc, prm, P @ U, mc.expand(phit, 1), zero_dirichlet=False)
    assert np.abs(P.T @ Rc - Rg).max() <= 1e-13 * np.abs(Rg).max()
    Gg = fe.assemble(mg, prm, U, phit)
    Gc = fe.assemble(mc, prm, P @ U, mc.expand(phit, 1))
    assert abs(P.T @ Gc @ P - Gg).max() <= 1e-12 * abs(Gg).max()


@pytest.mark.parametrize("dim,p,N", [(2, 2, 2), (3, 1, 2)])
def test_cut_mesh_jacobian_is_residual_derivative(dim, p, N):
    """Central differences of the residual along a direction that jumps across the slit."""
    m = M.Mesh(dim, p, N, slit="duplicate")
    prm = fe.Params(LAM, MU, GC, 0.3, KAPPA, mat.SPLIT_MIEHE)
    rng = np.random.default_rng(22)
    U, phit = random_state(m, rng)
    v = rng.normal(size=m.n_dofs)
    h = 1e-6
    fd = (fe.residual(m, prm, U + h * v, phit, zero_dirichlet=False) -
          fe.residual(m, prm, U - h * v, phit, zero_dirichlet=False)) / (2 * h)
    Gv = fe.assemble(m, prm, U, phit) @ v
    assert np.linalg.norm(fd - Gv) <= 1e-6 * np.linalg.norm(Gv)


def test_slit_opens_under_tension():
    """Linear elasticity (phi = phi~ = 1, no split) of the cut specimen with the top pulled: the upper
    copy of every slit node moves up relative to the lower copy, most at the mouth (x = 0), least next
    to the shared tip; on the uncut mesh the same solve has no opening by construction."""
    m = M.Mesh(2, 2, 8, slit="duplicate")
    prm = fe.Params(LAM, MU, GC, 0.25, KAPPA, mat.SPLIT_NONE)
    U = m.dirichlet_values(1e-3)
    U[2 * m.n_nodes:] = 1.0
    one = np.ones(m.n_nodes)
    nu = 2 * m.n_nodes
    mask = m.dirichlet_mask()[:nu]
    G = fe.masked(fe.assemble(m, prm, U, one)[:nu, :nu], mask)
    R = fe.residual(m, prm, U, one)[:nu]
    U[:nu] += spla.spsolve(G.tocsc(), np.where(mask, 0.0, -R))
    assert np.abs(fe.residual(m, prm, U, one)[:nu]).max() <= 1e-12 * np.abs(R).max()
    uy = U[m.n_nodes:nu]
    order = np.argsort(m.coords[m.dup_of, 0])
    opening = (uy[m.dup_of] - uy[m.n_grid_nodes:])[order]
    assert np.all(opening > 0)
    assert np.all(np.diff(opening) < 0)
