"""The slit cut into the mesh (Sec. 5.1: the slit's nodes duplicated, the tip shared) on the GPU, against
the oracle's cut mesh (`Mesh(..., slit="duplicate")`): sizes (the paper's DoF counts), node flags, the
lumped mass seen through the active-set rule, the Jacobian in every mode and precision, the residual, and
one Newton step (FGMRES with the multigrid, whose coarse levels are uncut) against the oracle's direct
step."""
import os

import numpy as np
import pytest

from oracle import fe, mesh as M, solvers as S
from paper_2005_00331_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM, MU, GC, KAPPA = 121.15, 80.77, 2.7e-3, 1e-10
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# (dim, p, N): N / 2 a multiple of the tile height along the last axis
CASES = [(2, 1, 32), (2, 2, 16), (2, 3, 8), (2, 4, 8), (3, 1, 4), (3, 2, 4), (3, 3, 4), (3, 4, 2)]
FAST = CASES[:6]  # the oracle assembles 3D Q3 and Q4 slowly: those run in full mode only


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(a), np.linalg.norm(b), 1e-300)


def cuda(a, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


class Cut:
    """A seeded state on the cut mesh: u ~ N(0, 1e-6) on free DoFs plus the lifted load, phi ~ U(0.9, 1)
    (the cut itself is the crack), phi_old a little above phi, a random active set (copies included)."""

    def __init__(self, dim, p, N, split=1, seed=0, active_frac=0.2, load=1e-3):
        m = M.Mesh(dim, p, N, slit="duplicate")
        self.m, self.dim, self.p, self.N = m, dim, p, N
        nn = m.n_nodes
        self.prm = fe.Params(LAM, MU, GC, 2.0 / N, KAPPA, split)
        U = m.dirichlet_values(load)
        dm = m.dirichlet_mask()[:dim * nn]
        U[:dim * nn] += np.where(dm, 0.0, inputs.displacement_noise(nn, dim, seed))
        U[dim * nn:] = inputs.uniform_phase(nn, seed)
        self.U = U
        self.phi_old = np.minimum(1.0, U[dim * nn:] + 1e-3 * np.abs(inputs.normal_vector(nn, seed, 7)))
        self.phi_tilde = np.clip(U[dim * nn:] + 0.01 * inputs.normal_vector(nn, seed, 8), 0.0, 1.0)
        self.active = inputs.uniform_phase(nn, seed + 100, 0.0, 1.0) < active_frac
        self.mask = m.dirichlet_mask()
        self.mask[dim * nn:] |= self.active

    def context(self, **kw):
        from paper_2005_00331_gb300 import setup_mesh
        ctx = setup_mesh(dim=self.dim, degree=self.p, n_cells_1d=self.N, split=self.prm.split, eps=self.prm.eps,
                         slit_cut=1, **kw)
        ctx.set_state(cuda(self.U), cuda(self.phi_old), cuda(self.phi_tilde), cuda(self.active, np.uint8))
        return ctx


def test_sizes_are_the_papers_slit_dof_counts():
    """pff_sizes of a context with the slit cut equals every row of Table tab:slit:dofs:p."""
    from paper_2005_00331_gb300 import setup_mesh
    rows = [l.split() for l in open(os.path.join(GOLDEN, "dof_counts_slit.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 8
    for lvl, p, dofs in rows:
        lvl, p, dofs = int(lvl), int(p), int(dofs)
        with setup_mesh(dim=2, degree=p, n_cells_1d=2 ** lvl, eps=2.0 ** (1 - lvl), slit_cut=1) as ctx:
            assert ctx.n_dofs == dofs


@pytest.mark.parametrize("dim,p,N", CASES)
def test_flags_and_active_set_rule(dim, p, N):
    """Node flags (Dirichlet, slit, copy) match the oracle's cut mesh; the active set computed by the
    library with the rule of Alg. 1 (lumped mass of the cut mesh, halved on both sides of the slit)
    matches the oracle's bit for bit."""
    from paper_2005_00331_gb300 import PFF_FLAG_COPY, PFF_FLAG_SLIT
    c = Cut(dim, p, N, seed=1)
    m = c.m
    with c.context() as ctx:
        fl = ctx.node_flags().cpu().numpy()
        assert len(fl) == m.n_nodes
        dm = m.dirichlet_mask()
        for k in range(dim):
            np.testing.assert_array_equal((fl >> k) & 1, dm[k * m.n_nodes:(k + 1) * m.n_nodes])
        copy = np.zeros(m.n_nodes, dtype=bool)
        copy[m.n_grid_nodes:] = True
        np.testing.assert_array_equal((fl & PFF_FLAG_COPY) != 0, copy)
        slit = np.zeros(m.n_nodes, dtype=bool)
        slit[m.slit_nodes()] = True
        np.testing.assert_array_equal((fl & PFF_FLAG_SLIT) != 0, slit)
        # active set from the library's own rule (set_state with active = None)
        ctx.set_state(cuda(c.U), cuda(c.phi_old), cuda(c.phi_tilde), None)
        got = ctx.get_active().cpu().numpy().astype(bool)
    R = fe.residual(m, c.prm, c.U, c.phi_tilde)
    ref = S.active_set(m, R, c.U[dim * m.n_nodes:], c.phi_old)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("split,modes", [(0, "all"), (1, "all")])
@pytest.mark.parametrize("dim,p,N", FAST)
def test_apply_and_residual(dim, p, N, split, modes):
    """Masked Jacobian in full, block-diagonal and transpose mode (FP64 native and double-word at 1e-12,
    FP32 at 2e-5) and the FP64 residual, against the oracle's assembly on the cut mesh."""
    _apply_and_residual(dim, p, N, split, modes)


@pytest.mark.parametrize("dim,p,N", CASES[6:])
def test_apply_and_residual_3d_high_degree(dim, p, N):
    _apply_and_residual(dim, p, N, 1, "full")


def _apply_and_residual(dim, p, N, split, modes):
    from paper_2005_00331_gb300 import PFF_MODE_BLOCKDIAG, PFF_MODE_FULL, PFF_MODE_TRANSPOSE
    c = Cut(dim, p, N, split=split, seed=2 + p)
    m = c.m
    x = inputs.normal_vector(m.n_dofs, 3)
    todo = ((PFF_MODE_FULL, fe.MODE_FULL), (PFF_MODE_BLOCKDIAG, fe.MODE_BLOCKDIAG),
            (PFF_MODE_TRANSPOSE, fe.MODE_TRANSPOSE))
    for mode, fm in (todo if modes == "all" else todo[:1]):
        G = fe.assemble(m, c.prm, c.U, c.phi_tilde, mode=fm)
        ref = fe.apply_masked(G, c.mask, x)
        ref32 = fe.apply_masked(G, c.mask, x.astype(np.float32).astype(np.float64))
        for fp64_mode in (0, 1):
            with c.context(fp64_mode=fp64_mode) as ctx:
                assert rel(ctx.apply_jacobian(cuda(x), mode=mode).cpu().numpy(), ref) <= 1e-12
        with c.context() as ctx:
            y = ctx.apply_jacobian(cuda(x, np.float32), mode=mode).cpu().numpy().astype(np.float64)
            assert rel(y, ref32) <= 2e-5
    with c.context() as ctx:
        assert rel(ctx.residual().cpu().numpy(), fe.residual(m, c.prm, c.U, c.phi_tilde)) <= 1e-12


@pytest.mark.parametrize("mg", [32, 64])
@pytest.mark.parametrize("dim,p,N", [(2, 2, 16), (2, 1, 32), (3, 2, 4)])
def test_newton_step_on_cut_mesh(dim, p, N, mg):
    """One step of Alg. 1 on the tension test with the slit cut into the mesh: the library's step (FGMRES
    to 1e-10 with the monolithic multigrid, cut finest level, uncut coarse levels) against the oracle's
    step with a sparse direct solve; the slit opens (the copies move down, the grid nodes up). The state
    is u = 0 with the top load lifted and phi ~ U(0.9, 1), phi_old a little above: the active-set rule
    decides with a margin (from rest with phi = phi_old = 1, R_phi is 0 up to rounding wherever the
    strain is 0, and the strict inequality of Alg. 1 then follows the rounding)."""
    m = M.Mesh(dim, p, N, slit="duplicate")
    prm = fe.Params(LAM, MU, GC, 2.0 / N, KAPPA, 1)
    nn = m.n_nodes
    U = m.dirichlet_values(1e-3)
    U[dim * nn:] = inputs.uniform_phase(nn, 4)
    phi = np.minimum(1.0, U[dim * nn:] + 1e-3 * np.abs(inputs.normal_vector(nn, 4, 7)))
    U_ref, act_ref, _, _ = S.pdas_step(m, prm, U, phi, phi)
    assert 0 < act_ref.sum() < nn
    from paper_2005_00331_gb300 import setup_mesh
    with setup_mesh(dim=dim, degree=p, n_cells_1d=N, split=1, eps=2.0 / N, slit_cut=1, mg_precision=mg,
                    lin_rtol=1e-10) as ctx:
        ctx.set_state(cuda(U), cuda(phi), cuda(phi), None)
        rep = ctx.solve_newton_step()
        Ug = ctx.get_state().cpu().numpy()
        act = ctx.get_active().cpu().numpy().astype(bool)
    np.testing.assert_array_equal(act, act_ref)
    assert rep["gmres_rel"] <= 1e-10 and rep["gmres_iters"] < 80
    assert rel(Ug - U, U_ref - U) <= 1e-7
    uz = Ug[(dim - 1) * nn:dim * nn]
    assert np.all(uz[m.n_grid_nodes:] < uz[m.dup_of])  # the slit opens under tension


def test_load_steps_and_resume_on_cut_mesh(tmp_path):
    """Three quasi-static load steps of the tension test on the cut 2D Q2 16 x 16 mesh (Miehe split):
    every step converges on both sides and the GPU states equal the oracle's load steps (direct solves);
    a checkpoint after the second step, resumed in a fresh context, continues to the same third state."""
    from paper_2005_00331_gb300 import checkpoint, setup_mesh
    m = M.Mesh(2, 2, 16, slit="duplicate")
    prm = fe.Params(LAM, MU, GC, 2.0 / 16, KAPPA, 1)
    U = m.dirichlet_values(0.0)
    phi = np.ones(m.n_nodes)
    U[2 * m.n_nodes:] = phi
    loads = [1e-3, 2e-3, 3e-3]
    stats = []
    ref = S.load_steps(m, prm, U, loads, stats=stats)
    assert all(conv for _, conv in stats)
    kw = dict(dim=2, degree=2, n_cells_1d=16, split=1, eps=2.0 / 16, slit_cut=1, mg_precision=32, lin_rtol=1e-10)
    path = str(tmp_path / "cut_step2.npz")
    with setup_mesh(**kw) as ctx:
        ctx.set_state(cuda(U), cuda(phi), cuda(phi), None)
        for k, load in enumerate(loads):
            st, reps = ctx.solve_load_step(load, check=False)
            assert st == 0
            assert rel(ctx.get_state().cpu().numpy(), ref[k]) <= 1e-6
            if k == 1:
                checkpoint.save(path, ctx.checkpoint(load))
        U_run = ctx.get_state().cpu().numpy()
    ck = checkpoint.load(path)
    assert ck.slit_cut == 1
    with setup_mesh(**kw) as ctx:
        ctx.resume(ck)
        ctx.solve_load_step(loads[2])
        assert rel(ctx.get_state().cpu().numpy(), U_run) <= 1e-7
