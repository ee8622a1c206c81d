"""GPU parity of the mesh flags, the residual and the matrix-free Jacobian against the oracle.

Tolerances: FP64 applies and residuals within 1e-12 relative l2 (relative to the largest of the
two norms); FP32 applies within 2e-5 relative l2 (single-precision arithmetic through sum
factorisation: a few hundred rounded operations per output, each 6e-8 relative)."""
import numpy as np
import pytest

from oracle import fe
from problems import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(2, 1, 5), (2, 2, 9), (2, 3, 6), (2, 4, 5), (3, 1, 5), (3, 2, 3), (3, 3, 3), (3, 4, 2)]
FP64_TOL = 1e-12
FP32_TOL = 2e-5


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(a), np.linalg.norm(b), 1e-300)


def cuda(a, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


@pytest.mark.parametrize("dim,p,N", [(2, 1, 8), (2, 3, 6), (3, 2, 4)])
def test_node_flags_bit_exact(dim, p, N):
    pr = Problem(dim, p, N)
    ctx = pr.context()
    fl = ctx.node_flags().cpu().numpy()
    m = pr.mesh
    nn = m.n_nodes
    dmask = m.dirichlet_mask()
    for c in range(dim):
        np.testing.assert_array_equal((fl >> c) & 1, dmask[c * nn:(c + 1) * nn].astype(np.uint8))
    slit = np.zeros(nn, dtype=np.uint8)
    slit[m.slit_nodes()] = 1
    np.testing.assert_array_equal((fl >> 6) & 1, slit)
    top = np.zeros(nn, dtype=np.uint8)
    top[m.top_nodes()] = 1
    np.testing.assert_array_equal((fl >> 4) & 1, top)


@pytest.mark.parametrize("dim,p,N", CASES)
@pytest.mark.parametrize("split", [0, 1])
def test_residual_fp64(dim, p, N, split):
    pr = Problem(dim, p, N, split=split, seed=dim * 10 + p)
    ctx = pr.context()
    r = ctx.residual().cpu().numpy()
    assert rel(r, pr.residual()) <= FP64_TOL


@pytest.mark.parametrize("dim,p,N", CASES)
@pytest.mark.parametrize("split", [0, 1])
def test_apply_modes_fp64(dim, p, N, split):
    pr = Problem(dim, p, N, split=split, seed=dim * 10 + p + 1, active_frac=0.3)
    ctx = pr.context()
    x = np.random.default_rng(p).normal(size=pr.mesh.n_dofs)
    xd = cuda(x)
    from paper_2005_00331_gb300 import PFF_MASK_ADJOINT, PFF_MASK_RAW, PFF_MODE_BLOCKDIAG, PFF_MODE_TRANSPOSE
    G = pr.G()
    # masked full operator
    y = ctx.apply_jacobian(xd).cpu().numpy()
    assert rel(y, fe.masked(G, pr.mask) @ x) <= FP64_TOL
    # raw (no masking)
    y = ctx.apply_jacobian(xd, mode=PFF_MASK_RAW).cpu().numpy()
    assert rel(y, G @ x) <= FP64_TOL
    # block diagonal, masked
    Gb = pr.G(fe.MODE_BLOCKDIAG)
    y = ctx.apply_jacobian(xd, mode=PFF_MODE_BLOCKDIAG).cpu().numpy()
    assert rel(y, fe.masked(Gb, pr.mask) @ x) <= FP64_TOL
    # transpose, masked and adjoint of the residual (Dirichlet rows of x removed, output raw)
    y = ctx.apply_jacobian(xd, mode=PFF_MODE_TRANSPOSE).cpu().numpy()
    assert rel(y, fe.masked(G.T.tocsr(), pr.mask) @ x) <= FP64_TOL
    dmask = pr.mesh.dirichlet_mask()
    y = ctx.apply_jacobian(xd, mode=PFF_MODE_TRANSPOSE | PFF_MASK_ADJOINT).cpu().numpy()
    assert rel(y, G.T @ np.where(dmask, 0.0, x)) <= FP64_TOL


@pytest.mark.parametrize("dim,p,N", CASES)
@pytest.mark.parametrize("split", [0, 1])
def test_apply_fp32(dim, p, N, split):
    pr = Problem(dim, p, N, split=split, seed=dim * 10 + p + 2, active_frac=0.2)
    ctx = pr.context()
    x = np.random.default_rng(p + 7).normal(size=pr.mesh.n_dofs)
    y = ctx.apply_jacobian(cuda(x, np.float32)).cpu().numpy()
    ref = fe.masked(pr.G(), pr.mask) @ x.astype(np.float32).astype(np.float64)
    assert rel(y, ref) <= FP32_TOL


def test_apply_fields_and_ragged_tiles():
    """Nodal material fields, and N not a multiple of the tile edge (partial tiles)."""
    for dim, p, N in [(2, 2, 11), (3, 1, 7), (3, 3, 3)]:
        pr = Problem(dim, p, N, split=1, seed=5, fields=True, active_frac=0.1)
        ctx = pr.context()
        x = np.random.default_rng(1).normal(size=pr.mesh.n_dofs)
        y = ctx.apply_jacobian(cuda(x)).cpu().numpy()
        assert rel(y, fe.masked(pr.G(), pr.mask) @ x) <= FP64_TOL
        assert rel(ctx.residual().cpu().numpy(), pr.residual()) <= FP64_TOL


def test_zero_strain_state_miehe():
    """u = 0 except the lifted load: many points have e = 0 exactly (repeated eigenvalues 0)."""
    pr = Problem(2, 2, 8, split=1, zero_u=True)
    ctx = pr.context()
    x = np.random.default_rng(3).normal(size=pr.mesh.n_dofs)
    y = ctx.apply_jacobian(cuda(x)).cpu().numpy()
    assert rel(y, fe.masked(pr.G(), pr.mask) @ x) <= FP64_TOL
    assert rel(ctx.residual().cpu().numpy(), pr.residual()) <= FP64_TOL


@pytest.mark.parametrize("dim,p,N", [(2, 1, 9), (2, 2, 9), (2, 3, 6), (2, 4, 5), (3, 1, 5), (3, 2, 3), (3, 3, 3),
                                     (3, 4, 2)])
@pytest.mark.parametrize("split", [0, 1])
def test_apply_float_float_fp64(dim, p, N, split):
    """fp64_mode = 1: the FP64 Jacobian in double-word arithmetic on the FP32 pipe, all modes;
    same 1e-12 tolerance as native FP64."""
    from paper_2005_00331_gb300 import PFF_MASK_ADJOINT, PFF_MASK_RAW, PFF_MODE_BLOCKDIAG, PFF_MODE_TRANSPOSE
    pr = Problem(dim, p, N, split=split, seed=40 + p, active_frac=0.3)
    ctx = pr.context(fp64_mode=1)
    x = np.random.default_rng(p + 40).normal(size=pr.mesh.n_dofs)
    xd = cuda(x)
    G = pr.G()
    assert rel(ctx.apply_jacobian(xd).cpu().numpy(), fe.masked(G, pr.mask) @ x) <= FP64_TOL
    assert rel(ctx.apply_jacobian(xd, mode=PFF_MASK_RAW).cpu().numpy(), G @ x) <= FP64_TOL
    Gb = pr.G(fe.MODE_BLOCKDIAG)
    assert rel(ctx.apply_jacobian(xd, mode=PFF_MODE_BLOCKDIAG).cpu().numpy(), fe.masked(Gb, pr.mask) @ x) <= FP64_TOL
    dmask = pr.mesh.dirichlet_mask()
    y = ctx.apply_jacobian(xd, mode=PFF_MODE_TRANSPOSE | PFF_MASK_ADJOINT).cpu().numpy()
    assert rel(y, G.T @ np.where(dmask, 0.0, x)) <= FP64_TOL


@pytest.mark.parametrize("dim,p,N", [(2, 1, 9), (2, 2, 9), (2, 3, 6), (2, 4, 5)])
@pytest.mark.parametrize("split", [0, 1])
def test_apply_fp32_recomputed_tangent(dim, p, N, split):
    """fp32_tangent = 1: the FP32 Jacobian recomputed at the Gauss points from the nodal state (no stored
    per-point data) in every mode and masking, against the oracle within the FP32 tolerance; also the
    tension state from rest, whose points mostly have e = 0 (repeated eigenvalues 0, H(0) = 1)."""
    from paper_2005_00331_gb300 import PFF_MASK_ADJOINT, PFF_MASK_RAW, PFF_MODE_BLOCKDIAG, PFF_MODE_TRANSPOSE
    for zero_u in (False, True):
        pr = Problem(dim, p, N, split=split, seed=60 + p, active_frac=0.2, zero_u=zero_u)
        ctx = pr.context(fp32_tangent=1)
        x = np.random.default_rng(p + 61).normal(size=pr.mesh.n_dofs)
        x32 = x.astype(np.float32).astype(np.float64)
        xd = cuda(x, np.float32)
        G, Gb = pr.G(), pr.G(fe.MODE_BLOCKDIAG)
        dmask = pr.mesh.dirichlet_mask()
        for mode, ref in ((0, fe.masked(G, pr.mask) @ x32), (PFF_MASK_RAW, G @ x32),
                          (PFF_MODE_BLOCKDIAG, fe.masked(Gb, pr.mask) @ x32),
                          (PFF_MODE_TRANSPOSE, fe.masked(G.T.tocsr(), pr.mask) @ x32),
                          (PFF_MODE_TRANSPOSE | PFF_MASK_ADJOINT, G.T @ np.where(dmask, 0.0, x32))):
            y = ctx.apply_jacobian(xd, mode=mode).cpu().numpy()
            assert rel(y, ref) <= FP32_TOL, (mode, zero_u)
