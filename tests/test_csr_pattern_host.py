"""The CSR pattern of the assembled comparator matrix (host code of libpff, no GPU) against the
definition it states -- DoFs couple when their nodes share a cell, G_uphi = 0, masked rows hold
their diagonal, masked columns are empty -- computed here from the oracle mesh's cell lists, and
against the nonzeros of the oracle's assembled, masked Jacobian of Eq. (G)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fe, material as mat, mesh as M
from paper_2005_00331_gb300 import csr_pattern

CASES = [(2, 1, 4), (2, 2, 3), (2, 3, 2), (2, 4, 2), (3, 1, 2), (3, 2, 2)]


def flags_of(m, seed):
    """Dirichlet bits of the tension test (bits 0..d-1) and a random active set (bit d)."""
    d, nn = m.dim, m.n_nodes
    mask = m.dirichlet_mask()
    fl = np.zeros(nn, dtype=np.uint8)
    for c in range(d):
        fl |= (mask[c * nn:(c + 1) * nn].astype(np.uint8) << c)
    act = np.random.default_rng(seed).uniform(size=nn) < 0.3
    fl |= act.astype(np.uint8) << d
    return fl


def expected_rows(m, fl):
    d, nn = m.dim, m.n_nodes
    nbr = [set() for _ in range(nn)]
    for cell in m.cell_nodes:
        for a in cell:
            nbr[a].update(cell.tolist())
    rows = []
    for g in range(d + 1):
        for i in range(nn):
            r = g * nn + i
            if (fl[i] >> g) & 1:
                rows.append([r])
                continue
            comps = range(d) if g < d else range(d + 1)
            rows.append(sorted(f * nn + j for f in comps for j in nbr[i] if not (fl[j] >> f) & 1))
    return rows


@pytest.mark.parametrize("dim,p,N", CASES)
def test_pattern_is_cell_coupling(dim, p, N):
    m = M.Mesh(dim, p, N)
    fl = flags_of(m, 3)
    rowptr, col = csr_pattern(dim, p, N, fl)
    assert rowptr[0] == 0 and rowptr[-1] == len(col) and np.all(np.diff(rowptr) >= 1)
    got = [col[rowptr[r]:rowptr[r + 1]].tolist() for r in range(m.n_dofs)]
    assert got == expected_rows(m, fl)  # includes: columns ascending


@pytest.mark.parametrize("dim,p,N", CASES)
@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_pattern_holds_the_masked_jacobian(dim, p, N, split):
    """Every nonzero of Z G Z + (I - Z) lies in the pattern, and at a random state nearly every
    pattern entry is a nonzero (the pattern is not padded)."""
    m = M.Mesh(dim, p, N)
    fl = flags_of(m, 4)
    d, nn = dim, m.n_nodes
    mask = np.zeros(m.n_dofs, dtype=bool)
    for c in range(d + 1):
        mask[c * nn:(c + 1) * nn] = (fl >> c) & 1
    rng = np.random.default_rng(5)
    U = np.zeros(m.n_dofs)
    U[:d * nn] = rng.normal(0, 1e-2, d * nn)
    U[d * nn:] = rng.uniform(0.5, 1.0, nn)
    G = fe.masked(fe.assemble(m, fe.Params(eps=0.2, split=split), U, U[d * nn:].copy()), mask).tocsr()
    G.eliminate_zeros()
    rowptr, col = csr_pattern(dim, p, N, fl)
    pat = set()
    for r in range(m.n_dofs):
        pat.update((r, int(c)) for c in col[rowptr[r]:rowptr[r + 1]])
    nz = set(zip(*G.nonzero()))
    assert nz <= pat
    assert len(nz) >= 0.9 * len(pat)


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        csr_pattern(2, 1, 4, np.zeros(10, dtype=np.uint8))
    from paper_2005_00331_gb300 import PFFError
    with pytest.raises(PFFError):
        csr_pattern(4, 1, 1, np.zeros(16, dtype=np.uint8))


@pytest.mark.parametrize("dim,p,N", CASES)
def test_probing_fills_every_entry_once(dim, p, N):
    """The assembly's probing plan (host code of libpff): over all (component, colour) probes, the
    columns it fills in each row are exactly the row's pattern, each once; and emulating the probes
    with the oracle's masked Jacobian (y = A x for the indicator x of the probe) rebuilds A exactly."""
    from paper_2005_00331_gb300 import csr_probe_targets
    m = M.Mesh(dim, p, N)
    fl = flags_of(m, 6)
    rowptr, col = csr_pattern(dim, p, N, fl)
    d, nn, n = dim, m.n_nodes, m.n_dofs
    mask = np.zeros(n, dtype=bool)
    for c in range(d + 1):
        mask[c * nn:(c + 1) * nn] = (fl >> c) & 1
    rng = np.random.default_rng(7)
    U = np.zeros(n)
    U[:d * nn] = rng.normal(0, 1e-2, d * nn)
    U[d * nn:] = rng.uniform(0.5, 1.0, nn)
    A = fe.masked(fe.assemble(m, fe.Params(eps=0.2, split=mat.SPLIT_MIEHE), U, U[d * nn:].copy()), mask).tocsr()
    mm = 2 * p + 1
    ijk = m.node_ijk
    colour = sum((ijk[:, t] % mm) * mm ** t for t in range(dim))
    hits = np.zeros(len(col), dtype=int)
    val = np.zeros(len(col))
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    for f in range(d + 1):
        for c in range(mm ** dim):
            x = np.zeros(n)
            x[f * nn:(f + 1) * nn] = colour == c
            y = A @ x
            t = csr_probe_targets(dim, p, N, f, c)
            ok = col == t[rows]
            hits += ok
            val[ok] = y[rows[ok]]
    assert np.all(hits == 1)
    B = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    assert abs(B - A).max() == 0.0


def test_cusparse_entry_points_resolve():
    """The comparator's SpMV library loads and every entry point it calls resolves (no GPU work)."""
    from paper_2005_00331_gb300 import load_library
    assert load_library().pff_csr_spmv_available() == 1


@pytest.mark.parametrize("dim,p,N", [(2, 1, 64), (2, 2, 32), (2, 3, 32), (2, 4, 32), (3, 1, 8), (3, 2, 4),
                                     (3, 4, 3)])
def test_pattern_size_closed_form(dim, p, N):
    """Nothing masked: per direction, an index shares cells with p + 1 indices at the two ends and off
    the cell vertices, and with 2p + 1 at the N - 1 inner vertices, so sum_i |window_i| =
    2(p+1) + (N-1)(2p+1) + N(p-1)(p+1) =: S, and the nodes' windows hold S^d entries; displacement
    rows see d components, phase-field rows d + 1: nnz = (d^2 + d + 1) S^d. Everything masked: the
    diagonal, nnz = n_dofs."""
    n1 = p * N + 1
    S = 2 * (p + 1) + (N - 1) * (2 * p + 1) + N * (p - 1) * (p + 1)
    rowptr, col = csr_pattern(dim, p, N, np.zeros(n1 ** dim, dtype=np.uint8))
    assert len(col) == (dim * dim + dim + 1) * S ** dim
    rowptr, col = csr_pattern(dim, p, N, np.full(n1 ** dim, (1 << (dim + 1)) - 1, dtype=np.uint8))
    assert np.array_equal(col, np.arange((dim + 1) * n1 ** dim))
