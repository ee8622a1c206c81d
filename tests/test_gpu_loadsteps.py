"""GPU parity of the load-displacement output (the force on the loaded face of the tension test,
Sec. 5.1, and of the shear test, Sec. 5.2) and of the shear test's load steps (Sec. 3.2, Alg. 1)."""
import numpy as np
import pytest

from oracle import fe, mesh as M, solvers as S
from problems import GC, KAPPA, LAM, MU, Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(a), np.linalg.norm(b), 1e-300)


def cuda(a, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


@pytest.mark.parametrize("dim,p,N,split", [(2, 1, 16, 1), (2, 2, 8, 0), (2, 3, 5, 1), (2, 4, 3, 1), (3, 1, 6, 1),
                                           (3, 2, 3, 0)])
def test_reaction_force_against_oracle(dim, p, N, split):
    """FP64: the sum of the top-face u_d rows of the full residual, against the oracle's, relative to
    the sum of their magnitudes (several tiles and a ragged tail in 2D)."""
    pr = Problem(dim, p, N, split=split, seed=5, active_frac=0.2, fields=(dim == 2 and p == 2))
    with pr.context() as ctx:
        F = ctx.reaction_force()
    ref = fe.reaction_force(pr.mesh, pr.prm, pr.U, pr.phi_tilde, **pr.fields)
    R = fe.residual(pr.mesh, pr.prm, pr.U, pr.phi_tilde, zero_dirichlet=False, **pr.fields)
    scale = np.abs(R[pr.mesh.dof(dim - 1, pr.mesh.top_nodes())]).sum()
    assert abs(F - ref) <= 1e-12 * scale


@pytest.mark.parametrize("dim,p,N,split,load", [(2, 2, 8, 1, 2e-3), (2, 2, 8, 1, -2e-3), (2, 3, 6, 0, 2e-3),
                                                (3, 2, 4, 1, 2e-3), (3, 1, 4, 0, -2e-3)])
def test_reaction_force_uniaxial_strain(dim, p, N, split, load):
    """Closed form: u_d = load x_d, phi = phi~ = c give sigma_dd = (lambda + 2 mu) load on the unit top
    face, degraded by g(c) unless the Miehe split sees compression."""
    from paper_2005_00331_gb300 import setup_mesh
    c = 0.7
    m = M.Mesh(dim, p, N)
    U = np.zeros(m.n_dofs)
    U[(dim - 1) * m.n_nodes:dim * m.n_nodes] = load * m.coords[:, dim - 1]
    U[dim * m.n_nodes:] = c
    phi = np.full(m.n_nodes, c)
    with setup_mesh(dim=dim, degree=p, n_cells_1d=N, split=split, eps=0.2) as ctx:
        ctx.set_state(cuda(U), cuda(phi), cuda(phi), cuda(np.zeros(m.n_nodes), np.uint8))
        F = ctx.reaction_force()
    g = (1.0 - KAPPA) * c * c + KAPPA
    expect = (LAM + 2 * MU) * load * (g if (split == 0 or load > 0) else 1.0)
    assert abs(F - expect) <= 1e-12 * abs(expect)


def _specimen(split=1):
    m = M.Mesh(2, 1, 16)
    prm = fe.Params(LAM, MU, GC, 2.0 / 16, KAPPA, split)
    U = m.dirichlet_values(0.0)
    phi = np.ones(m.n_nodes)
    phi[m.slit_nodes()] = 0.0
    U[2 * m.n_nodes:] = phi
    return m, prm, U, phi


@pytest.mark.parametrize("split", [0, 1])
def test_shear_load_steps_against_oracle(split):
    """Shear test (Sec. 5.2): the top face moved to the right in three load steps, with (Miehe) and
    without (isotropic) split: states and x forces on the top face against the oracle's."""
    from paper_2005_00331_gb300 import setup_mesh
    m, prm, U, phi = _specimen(split)
    loads = [4e-3, 8e-3, 1.2e-2]
    ref, phits = S.load_steps(m, prm, U, loads, comp=0, return_phit=True)
    with setup_mesh(dim=2, degree=1, n_cells_1d=16, split=split, eps=2.0 / 16, mg_precision=32,
                    lin_rtol=1e-10) as ctx:
        ctx.set_load_component(0)
        ctx.set_state(cuda(U), cuda(phi), cuda(phi), None)
        for k, load in enumerate(loads):
            ctx.solve_load_step(load)
            assert rel(ctx.get_state().cpu().numpy(), ref[k]) <= 1e-6
            F_ref = fe.reaction_force(m, prm, ref[k], phits[k], comp=0)
            assert F_ref > 0 and abs(ctx.reaction_force() - F_ref) <= 1e-4 * F_ref


@pytest.mark.parametrize("dim,p,N,split", [(2, 2, 8, 1), (2, 3, 5, 0), (3, 2, 3, 1)])
def test_reaction_force_shear_component(dim, p, N, split):
    """The x force on the top face (load component 0) at a random state against the oracle, and the
    simple-shear closed form (1 + g(c)) mu gamma / 2 (Miehe) or g(c) mu gamma (no split)."""
    from paper_2005_00331_gb300 import setup_mesh
    pr = Problem(dim, p, N, split=split, seed=9, active_frac=0.2)
    with pr.context() as ctx:
        ctx.set_load_component(0)
        F = ctx.reaction_force()
    ref = fe.reaction_force(pr.mesh, pr.prm, pr.U, pr.phi_tilde, comp=0)
    R = fe.residual(pr.mesh, pr.prm, pr.U, pr.phi_tilde, zero_dirichlet=False)
    assert abs(F - ref) <= 1e-12 * np.abs(R[pr.mesh.dof(0, pr.mesh.top_nodes())]).sum()
    c, gamma = 0.7, 2e-3
    m = pr.mesh
    U = np.zeros(m.n_dofs)
    U[:m.n_nodes] = gamma * m.coords[:, dim - 1]
    U[dim * m.n_nodes:] = c
    phi = np.full(m.n_nodes, c)
    with setup_mesh(dim=dim, degree=p, n_cells_1d=N, split=split, eps=0.2) as ctx:
        ctx.set_load_component(0)
        ctx.set_state(cuda(U), cuda(phi), cuda(phi), cuda(np.zeros(m.n_nodes), np.uint8))
        F = ctx.reaction_force()
    g = (1.0 - KAPPA) * c * c + KAPPA
    expect = MU * gamma * (g if split == 0 else 0.5 * (1.0 + g))
    assert abs(F - expect) <= 1e-12 * abs(expect)


def test_history_argument_checks():
    """pff_set_history rejects n_hist outside 0..2, a missing array, and a context without state."""
    from paper_2005_00331_gb300 import PFFError, load_library, setup_mesh
    import ctypes
    lib = load_library()
    m, prm, U, phi = _specimen()
    with setup_mesh(dim=2, degree=1, n_cells_1d=16, split=1, eps=2.0 / 16) as ctx:
        with pytest.raises(PFFError):
            ctx.set_history(cuda(phi))  # no state yet
        ctx.set_state(cuda(U), cuda(phi), cuda(phi), None)
        ctx.set_history(cuda(phi))
        assert ctx.get_history()[0] == 1
        t = cuda(phi)
        p = ctypes.c_void_p(t.data_ptr())
        assert lib.pff_set_history(ctx._h, p, None, 2) == -1
        assert lib.pff_set_history(ctx._h, p, p, 3) == -1
        assert lib.pff_set_history(ctx._h, None, None, 1) == -1
        assert lib.pff_set_load_component(ctx._h, 2) == -1
        assert lib.pff_set_load_component(ctx._h, -1) == -1
