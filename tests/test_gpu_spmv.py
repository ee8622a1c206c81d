"""GPU parity of the assembled-matrix comparator (Sec. 6.3, fig. compare:vmult): the CSR matrix
that pff_csr_assemble probes out of the matrix-free operator against the oracle's assembled,
masked Jacobian of Eq. (G), entry by entry, and cuSPARSE's y = A x against the oracle's product and
the matrix-free apply; at the comparator's size (2D, 128^2 cells, p = 1..4) against the
matrix-free apply, which holds at any size."""
import numpy as np
import pytest
import scipy.sparse as sp

from problems import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(a), np.linalg.norm(b), 1e-300)


def cuda(a, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def need_cusparse():
    from paper_2005_00331_gb300 import load_library
    if load_library().pff_csr_spmv_available() != 1:
        pytest.skip("cuSPARSE cannot be loaded on this machine (the assembled matrix is still tested)")


@pytest.mark.parametrize("dim,p,N,split", [(2, 1, 12, 1), (2, 2, 8, 0), (2, 3, 5, 1), (2, 4, 4, 1), (3, 1, 5, 1),
                                           (3, 2, 3, 0)])
def test_assembled_matrix_against_oracle(dim, p, N, split):
    from oracle import fe
    pr = Problem(dim, p, N, split=split, seed=6, active_frac=0.25, fields=(dim == 2 and p == 2))
    with pr.context() as ctx:
        nnz = ctx.csr_assemble()
        rowptr, col, val = (t.cpu().numpy() for t in ctx.csr_export())
    n = pr.mesh.n_dofs
    assert len(col) == nnz and rowptr[-1] == nnz
    A = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    G = fe.masked(pr.G(), pr.mask)
    assert abs(A - G).max() <= 1e-12 * abs(G).max()


@pytest.mark.parametrize("dim,p,N,split", [(2, 2, 8, 1), (3, 2, 3, 0)])
def test_spmv_against_oracle(dim, p, N, split):
    need_cusparse()
    from oracle import fe
    pr = Problem(dim, p, N, split=split, seed=6, active_frac=0.25)
    x = np.random.default_rng(7).normal(size=pr.mesh.n_dofs)
    with pr.context() as ctx:
        ctx.csr_assemble()
        y_sp = ctx.csr_spmv(cuda(x)).cpu().numpy()
        y_mf = ctx.apply_jacobian(cuda(x)).cpu().numpy()
    G = fe.masked(pr.G(), pr.mask)
    assert rel(y_sp, G @ x) <= 1e-12
    assert rel(y_sp, y_mf) <= 1e-12


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_spmv_equals_matrix_free_at_comparator_size(p):
    need_cusparse()
    pr = Problem(2, p, 128, split=1, seed=8, active_frac=0.3)
    x = cuda(np.random.default_rng(9).normal(size=pr.mesh.n_dofs))
    with pr.context() as ctx:
        ctx.csr_assemble()
        y_sp = ctx.csr_spmv(x).cpu().numpy()
        y_mf = ctx.apply_jacobian(x).cpu().numpy()
    assert rel(y_sp, y_mf) <= 1e-12


def test_spmv_argument_checks():
    from paper_2005_00331_gb300 import PFFError
    pr = Problem(2, 1, 8, split=1, seed=1)
    x = cuda(np.ones(pr.mesh.n_dofs))
    with pr.context() as ctx:
        with pytest.raises(PFFError):
            ctx.csr_spmv(x)  # nothing assembled
        with pytest.raises(PFFError):
            ctx.csr_export()  # nothing assembled
        ctx.csr_assemble()
        with pytest.raises(PFFError):
            ctx.csr_spmv(x, x)  # aliased
