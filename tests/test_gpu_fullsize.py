"""Parity at the full sizes of the benchmark configurations, on sampled outputs.

The oracle computes a sampled output exactly from the cells that touch its node (element matrices
of Eq. (G) and element residuals of Eq. (residual), no sum factorisation); the GPU computes the
whole vector in the launch configuration the benchmark times. Sizes:
* 2D Q2 256 x 256 (789,507 DoFs), state u ~ N(0, 1e-6), phi ~ U(0.9, 1), phi_old = phi (every
  phase-field DoF active by the configured rule phi_old - phi < 1e-8) and a mixed variant;
* 3D Q2 64^3 (8,586,756 DoFs) and 3D Q3 48^3 (12,194,500 DoFs), notched cube;
* 2D Q2 128 x 128 (198,147 DoFs) with a lognormal nodal G_c field: adjoint and parameter gradients.
"""
import numpy as np
import pytest

from oracle import fe, mesh as M
from paper_2005_00331_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM, MU, GC, KAPPA = 121.15, 80.77, 2.7e-3, 1e-10


def cuda(a, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def cells_of_nodes(m, nodes):
    """All cells containing any of the given nodes."""
    p, N = m.p, m.N
    out = set()
    for nd in nodes:
        ijk = m.node_ijk[nd]
        ranges = []
        for t in range(m.dim):
            i = ijk[t]
            lo = i // p - (1 if i % p == 0 else 0)
            hi = min(i // p, N - 1)
            ranges.append([c for c in range(max(lo, 0), hi + 1)])
        for c in np.array(np.meshgrid(*ranges, indexing="ij")).reshape(m.dim, -1).T:
            out.add(int(sum(int(c[t]) * N ** t for t in range(m.dim))))
    return np.array(sorted(out))


class Big:
    def __init__(self, dim, p, N, split=1, seed=0, mixed=False, fields=False):
        m = M.Mesh(dim, p, N)
        self.m, self.dim = m, dim
        nn = m.n_nodes
        self.prm = fe.Params(LAM, MU, GC, 2.0 / N, KAPPA, split)
        U = m.dirichlet_values(1e-3)
        U[:dim * nn] += np.where(m.dirichlet_mask()[:dim * nn], 0.0, inputs.displacement_noise(nn, dim, seed))
        phi = inputs.uniform_phase(nn, seed)
        phi[m.slit_nodes()] = 0.0
        U[dim * nn:] = phi
        self.U = U
        self.phi_old = inputs.phi_old_above(phi, seed) if mixed else phi.copy()
        self.active = (self.phi_old - phi) < 1e-8
        self.mask = m.dirichlet_mask()
        self.mask[dim * nn:] |= self.active
        self.fields = {}
        if fields:
            self.fields = dict(gc_field=inputs.lognormal_field(nn, seed))

    def context(self, **kw):
        from paper_2005_00331_gb300 import setup_mesh
        m = self.m
        ctx = setup_mesh(dim=self.dim, degree=m.p, n_cells_1d=m.N, split=self.prm.split, eps=self.prm.eps, **kw)
        ctx.set_state(cuda(self.U), cuda(self.phi_old), cuda(self.phi_old), cuda(self.active, np.uint8),
                      cuda(self.fields["gc_field"]) if self.fields else None)
        return ctx

    def sample(self, k, seed=1):
        rng = np.random.default_rng(seed)
        return np.sort(rng.choice(self.m.n_dofs, size=k, replace=False))

    def rows_apply(self, dofs, x, mode=fe.MODE_FULL):
        m = self.m
        nodes = dofs % m.n_nodes
        cells = cells_of_nodes(m, nodes)
        xm = np.where(self.mask, 0.0, x)
        y = fe.apply_ebe(m, self.prm, self.U, self.phi_old, xm, mode=mode, cells=cells, **self.fields)
        y = np.where(self.mask, x, y)
        return y[dofs]

    def rows_apply_many(self, dofs, xs):
        """rows_apply for several inputs, with the element matrices of the sampled cells built once."""
        m = self.m
        cells = cells_of_nodes(m, dofs % m.n_nodes)
        T = fe.Tables(m)
        cd = m.cell_dofs()[cells]
        K = np.concatenate([fe.element_matrices(m, self.prm, self.U, self.phi_old, cells[s:s + 256], T, **self.fields)
                            for s in range(0, len(cells), 256)])
        out = []
        for x in xs:
            xm = np.where(self.mask, 0.0, x)
            y = np.zeros(m.n_dofs)
            np.add.at(y, cd, np.einsum("cij,cj->ci", K, xm[cd]))
            out.append(np.where(self.mask, x, y)[dofs])
        return out

    def rows_residual(self, dofs):
        m = self.m
        cells = cells_of_nodes(m, dofs % m.n_nodes)
        R = fe.residual(m, self.prm, self.U, self.phi_old, cells=cells, **self.fields)
        return R[dofs]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(a), np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("mixed", [False, True])
def test_c2_apply_and_residual_sampled(mixed):
    big = Big(2, 2, 256, mixed=mixed)
    x = inputs.normal_vector(big.m.n_dofs, 3)
    dofs = big.sample(300)
    ref = big.rows_apply(dofs, x)
    for kw, prec, tol in (({"fp64_mode": 0}, 64, 1e-12), ({"fp64_mode": 1}, 64, 1e-12), ({}, 32, 2e-5)):
        ctx = big.context(**kw)
        xd = cuda(x, np.float32 if prec == 32 else np.float64)
        y = ctx.apply_jacobian(xd).cpu().numpy().astype(np.float64)
        if prec == 32:
            ref32 = big.rows_apply(dofs, x.astype(np.float32).astype(np.float64))
            assert rel(y[dofs], ref32) <= tol
        else:
            assert rel(y[dofs], ref) <= tol
        ctx.close()
    ctx = big.context()
    r = ctx.residual().cpu().numpy()
    assert rel(r[dofs], big.rows_residual(dofs)) <= 1e-12


def _apply_all_precisions(big, x, dofs):
    """Sampled rows of the masked apply in FP64 (double-word and native arithmetic, 1e-12) and in FP32
    (2e-5 against the oracle applied to the FP32-rounded input), each in the launch configuration of a
    context on the full mesh."""
    ref, ref32 = big.rows_apply_many(dofs, [x, x.astype(np.float32).astype(np.float64)])
    for kw, prec, tol, r in (({"fp64_mode": 1}, 64, 1e-12, ref), ({"fp64_mode": 0}, 64, 1e-12, ref),
                             ({}, 32, 2e-5, ref32)):
        ctx = big.context(**kw)
        xd = cuda(x, np.float32 if prec == 32 else np.float64)
        y = ctx.apply_jacobian(xd).cpu().numpy().astype(np.float64)
        assert rel(y[dofs], r) <= tol, (kw, prec)
        ctx.close()
        del ctx


def test_c3_apply_sampled():
    """3D Q2 64^3 notched cube (8.6 M DoFs)."""
    big = Big(3, 2, 64, seed=2, mixed=True)
    _apply_all_precisions(big, inputs.normal_vector(big.m.n_dofs, 4), big.sample(120, seed=5))


def test_c5_apply_and_residual_sampled():
    """3D Q3 48^3 notched cube (12.2 M DoFs), the size of the load-step configuration: applies in all
    precisions and the FP64 residual on sampled rows."""
    big = Big(3, 3, 48, seed=3, mixed=True)
    dofs = big.sample(40, seed=6)
    _apply_all_precisions(big, inputs.normal_vector(big.m.n_dofs, 5), dofs)
    ctx = big.context()
    r = ctx.residual().cpu().numpy()
    assert rel(r[dofs], big.rows_residual(dofs)) <= 1e-12


def test_c4_adjoint_sampled():
    """2D Q2 128 x 128, lognormal G_c: dR/dU^T v and dR/dG_c^T v on sampled entries, and a central
    finite difference of <v, R> along a random direction (1e-6 relative)."""
    from paper_2005_00331_gb300 import PFF_MASK_ADJOINT, PFF_MODE_TRANSPOSE
    big = Big(2, 2, 128, seed=7, fields=True)
    m = big.m
    big.active[:] = False
    big.mask = m.dirichlet_mask()
    ctx = big.context()
    v = inputs.normal_vector(m.n_dofs, 8)
    vm = np.where(m.dirichlet_mask(), 0.0, v)
    gU = ctx.apply_jacobian(cuda(v), mode=PFF_MODE_TRANSPOSE | PFF_MASK_ADJOINT).cpu().numpy()
    g_gc = ctx.param_grad(cuda(v))[0].cpu().numpy()
    # oracle: transpose of the element matrices of the cells around sampled nodes
    nodes = np.random.default_rng(9).choice(m.n_nodes, 80, replace=False)
    cells = cells_of_nodes(m, nodes)
    yT = fe.apply_ebe(m, big.prm, big.U, big.phi_old, vm, mode=fe.MODE_TRANSPOSE, cells=cells, **big.fields)
    dofs = np.concatenate([nodes + c * m.n_nodes for c in range(3)])
    assert rel(gU[dofs], yT[dofs]) <= 1e-12
    # parameter gradient (oracle over the whole mesh) at the sampled nodes
    sub = fe.param_grad(m, big.prm, big.U, big.phi_old, vm, **big.fields)
    assert rel(g_gc[nodes], sub[0][nodes]) <= 1e-12
    # finite differences of <v, R> on the GPU. R is linear in phi and in G_c, so central differences
    # along a phi direction and along a G_c direction are exact up to rounding; in u the Miehe split
    # has kinks (an eigenvalue or the trace changing sign at a Gauss point), so the u direction takes
    # a step small enough that no point of this random state crosses one.
    act = torch.zeros(m.n_nodes, dtype=torch.uint8, device="cuda")
    po = cuda(big.phi_old)
    gcf = big.fields["gc_field"]
    vd = cuda(v)

    def vr(U, gc):
        ctx.set_state(cuda(U), po, po, act, cuda(gc))
        return float(vd @ ctx.residual())

    nn = m.n_nodes
    free = ~m.dirichlet_mask()
    d = np.where(free, inputs.normal_vector(m.n_dofs, 10), 0.0)
    d_phi = np.where(np.arange(m.n_dofs) >= 2 * nn, d, 0.0)
    d_u = d - d_phi
    for dd, rel_h, tol in ((d_phi, 1e-6, 1e-6), (d_u, 1e-9, 1e-5)):
        h = rel_h * np.linalg.norm(big.U) / np.linalg.norm(dd)
        fd = (vr(big.U + h * dd, gcf) - vr(big.U - h * dd, gcf)) / (2 * h)
        an = float(gU @ dd)
        assert abs(fd - an) <= tol * abs(an)
    # linear in G_c: a large step keeps the rounding of <v, R> (whose G_c part is small) out of the quotient
    dg = inputs.normal_vector(nn, 11) * gcf
    h = 0.1
    fd = (vr(big.U, gcf + h * dg) - vr(big.U, gcf - h * dg)) / (2 * h)
    an = float(g_gc @ dg)
    assert abs(fd - an) <= 1e-6 * abs(an)
