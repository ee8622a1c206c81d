"""Failure detection without a GPU fault: a non-finite state, an FGMRES iteration cap and the
active-set loop's cap come back as status codes (PFF_ERR_NAN, PFF_ERR_NOT_CONVERGED), and the
context keeps working afterwards. NaN arithmetic does not trap, and every device loop has a fixed
trip count or a fixed bound, so none of these cases can hang or fault the GPU. Also the device
memory accounting that these diagnostics report with."""
import ctypes

import numpy as np
import pytest

from problems import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cuda(a, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def test_nan_state_is_reported_and_the_context_recovers():
    from paper_2005_00331_gb300 import PFF_ERR_NAN
    pr = Problem(2, 2, 8, split=1, seed=2, active_frac=0.1)
    nn = pr.mesh.n_nodes
    idx = int(np.nonzero(~pr.mask[:nn])[0][nn // 4])  # an unmasked u_x DoF
    U_bad = pr.U.copy()
    U_bad[idx] = np.nan
    act = cuda(pr.active.astype(np.uint8), np.uint8)
    with pr.context() as ctx:
        ctx.set_state(cuda(U_bad), cuda(pr.phi_old), cuda(pr.phi_tilde), act)
        rep = ctx.solve_newton_step(check=False)
        assert rep["status"] == PFF_ERR_NAN
        assert np.isnan(ctx.get_state().cpu().numpy()[idx])  # no update was applied
        ctx.set_state(cuda(pr.U), cuda(pr.phi_old), cuda(pr.phi_tilde), act)
        rep = ctx.solve_newton_step()  # raises on any error status
        assert rep["status"] == 0 and np.all(np.isfinite(ctx.get_state().cpu().numpy()))


def test_iteration_caps_are_reported():
    from paper_2005_00331_gb300 import PFF_ERR_NOT_CONVERGED, load_library
    pr = Problem(2, 2, 8, split=1, seed=3, active_frac=0.2)
    lib = load_library()
    with pr.context(mg_precision=32, gmres_max_iters=1, lin_rtol=1e-12) as ctx:
        b = cuda(np.where(pr.mask, 0.0, np.random.default_rng(4).normal(size=pr.mesh.n_dofs)))
        x = torch.empty_like(b)
        its, rel = ctypes.c_int(), ctypes.c_double()
        st = lib.pff_solve_linear(ctx._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                  ctypes.byref(its), ctypes.byref(rel))
        assert st == PFF_ERR_NOT_CONVERGED and its.value == 1 and rel.value > 1e-12
        U0 = ctx.get_state().cpu().numpy()
        rep = ctx.solve_newton_step(check=False)
        assert rep["status"] == PFF_ERR_NOT_CONVERGED and rep["gmres_iters"] == 1
        assert not np.array_equal(ctx.get_state().cpu().numpy(), U0)  # the capped correction is applied
    with pr.context(mg_precision=32) as ctx:
        st, reps = ctx.solve_pdas(max_iters=1, check=False)
        assert st == PFF_ERR_NOT_CONVERGED and len(reps) == 1  # Alg. 1 needs two steps to see A settle


def test_memory_accounting():
    """pff_memory: the FGMRES basis to the byte, levels decreasing with the mesh, parts summing to the
    total, and the comparator matrix and the lazily allocated multigrid work vectors counted once
    they exist."""
    pr = Problem(2, 2, 16, split=1, seed=1)
    nd, m = pr.mesh.n_dofs, 50
    with pr.context() as ctx:
        m0 = ctx.memory()
        # basis V, directions Z, work vector, Hessenberg scalars, y; plus the CGS2 pass counter (4 bytes)
        assert m0["krylov"] == 8 * ((m + 1) * nd + m * nd + nd + 3 * (m + 1) + 4 + m + 1) + 4
        lv = m0["levels"]
        assert len(lv) == ctx.n_levels and all(a > b > 0 for a, b in zip(lv, lv[1:]))
        assert m0["total"] == sum(lv) + m0["krylov"] + m0["coarse"] + m0["other"] and m0["coarse"] > 0
        nnz = ctx.csr_assemble()
        m1 = ctx.memory()
        assert m1["other"] - m0["other"] == 12 * nnz + 4 * (nd + 1)
        ctx.solve_newton_step()
        m2 = ctx.memory()
        assert all(b >= a for a, b in zip(m1["levels"], m2["levels"])) and m2["levels"][0] > m1["levels"][0]
