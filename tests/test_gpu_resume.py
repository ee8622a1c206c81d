"""Checkpoint / resume of the quasi-static load-step loop (Sec. 3.2, Alg. 1) on the GPU: the force
after each load step against the oracle's, and a run resumed from a checkpoint file against the
uninterrupted run."""
import numpy as np
import pytest

from oracle import fe, mesh as M, solvers as S
from problems import GC, KAPPA, LAM, MU

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(a), np.linalg.norm(b), 1e-300)


def cuda(a, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _specimen(split=1):
    m = M.Mesh(2, 1, 16)
    prm = fe.Params(LAM, MU, GC, 2.0 / 16, KAPPA, split)
    U = m.dirichlet_values(0.0)
    phi = np.ones(m.n_nodes)
    phi[m.slit_nodes()] = 0.0
    U[2 * m.n_nodes:] = phi
    return m, prm, U, phi


def test_load_displacement_and_resume(tmp_path):
    """Three load steps of the notched specimen (2D Q1 16 x 16, Miehe split, mixed multigrid): the
    force after each step against the oracle's at its own converged states; then a checkpoint after
    the second step, written to disk, read back into a fresh context, continues with the third step
    to the state of the uninterrupted run."""
    from paper_2005_00331_gb300 import checkpoint, setup_mesh
    m, prm, U, phi = _specimen()
    loads = [4e-3, 8e-3, 1.2e-2]
    ref, phits = S.load_steps(m, prm, U, loads, return_phit=True)
    kw = dict(dim=2, degree=1, n_cells_1d=16, split=1, eps=2.0 / 16, mg_precision=32, lin_rtol=1e-10)
    path = str(tmp_path / "step2.npz")
    with setup_mesh(**kw) as ctx:
        ctx.set_state(cuda(U), cuda(phi), cuda(phi), None)
        assert ctx.get_history()[0] == 0
        for k, load in enumerate(loads):
            ctx.solve_load_step(load)
            F = ctx.reaction_force()
            F_ref = fe.reaction_force(m, prm, ref[k], phits[k])  # with the phi~ the step solved with
            assert F > 0 and abs(F - F_ref) <= 1e-4 * abs(F_ref)
            if k == 1:
                ck = ctx.checkpoint(load)
                assert ck.n_hist == 2
                checkpoint.save(path, ck)
        U_run = ctx.get_state().cpu().numpy()
        n, phi1, _ = ctx.get_history()
        assert n == 2 and np.array_equal(phi1.cpu().numpy(), U_run[2 * m.n_nodes:])
    ck = checkpoint.load(path)
    assert ck.load == loads[1]
    with setup_mesh(**kw) as ctx:
        ctx.resume(ck)
        n, phi1, phi2 = ctx.get_history()
        assert n == 2 and np.array_equal(phi1.cpu().numpy(), ck.phi1) and np.array_equal(phi2.cpu().numpy(), ck.phi2)
        ctx.solve_load_step(loads[2])
        U_res = ctx.get_state().cpu().numpy()
    assert rel(U_res, U_run) <= 1e-7
    assert rel(U_res, ref[2]) <= 1e-6
