"""GPU parity of the multigrid pieces (Sec. 3.3) and of the Newton step (Alg. 1) against the oracle.

Level data, transfers and the diagonal are FP64 computations compared at 1e-12. Pieces that
depend on the CG-Lanczos eigenvalue estimate (smoother, V-cycle) are compared at 1e-9: the
estimate itself is a 15-step Krylov process whose rounding differs between the two summation
orders. Solves are compared through their FP64 residuals (linear tolerance 1e-6 of Sec. 6.2)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fe, solvers as S
from problems import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(a), np.linalg.norm(b), 1e-300)


def cuda(a, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


MG_CASES = [(2, 1, 16, 0), (2, 2, 8, 1), (2, 3, 8, 1), (2, 4, 4, 0), (3, 1, 8, 1), (3, 2, 4, 0)]


def oracle_levels(pr, cheb_degree=5):
    return S.build_levels(pr.dim, pr.p, pr.N, pr.prm, pr.U, pr.phi_tilde, pr.active, cheb_degree=cheb_degree,
                          eig_iters=15, eig_seed=0, coarse_min=3, **pr.fields)


@pytest.mark.parametrize("dim,p,N,split", MG_CASES)
def test_fp32_multigrid_diagonal(dim, p, N, split):
    """With the FP32 multigrid the Jacobi diagonal is computed in FP32 from the FP32 per-point data;
    the FP64 diagonal is still available on request."""
    pr = Problem(dim, p, N, split=split, seed=3, active_frac=0.25)
    lv = oracle_levels(pr)
    ctx = pr.context(mg_precision=32)
    for l, L in enumerate(lv):
        assert rel(ctx.diagonal(l, precision=32).cpu().numpy().astype(np.float64), L.diag) <= 2e-6
        assert rel(ctx.diagonal(l).cpu().numpy(), L.diag) <= 1e-12


@pytest.mark.parametrize("dim,p,N,split", MG_CASES)
def test_levels_diagonal_transfers(dim, p, N, split):
    pr = Problem(dim, p, N, split=split, seed=3, active_frac=0.25)
    lv = oracle_levels(pr)
    ctx = pr.context()
    assert ctx.n_levels == len(lv)
    for l, L in enumerate(lv):
        # state carried to the level, active bits, masked diagonal
        assert rel(ctx.level_state(l).cpu().numpy(), L.U) <= 1e-13
        fl = ctx.node_flags(l).cpu().numpy()
        np.testing.assert_array_equal(((fl >> dim) & 1).astype(bool), L.active)
        assert rel(ctx.diagonal(l).cpu().numpy(), L.diag) <= 1e-12
        if l + 1 < len(lv):
            Lc = lv[l + 1]
            nnc, nnf = Lc.mesh.n_nodes, L.mesh.n_nodes
            xc = np.random.default_rng(l).normal(size=Lc.mesh.n_dofs)
            ref = np.concatenate([Lc.P @ xc[c * nnc:(c + 1) * nnc] for c in range(dim + 1)])
            ref[L.mask] = 0.0
            assert rel(ctx.prolongate(l, cuda(xc)).cpu().numpy(), ref) <= 1e-13
            xf = np.random.default_rng(l + 50).normal(size=L.mesh.n_dofs)
            xfm = np.where(L.mask, 0.0, xf)
            ref = np.concatenate([Lc.P.T @ xfm[c * nnf:(c + 1) * nnf] for c in range(dim + 1)])
            ref[Lc.mask] = 0.0
            assert rel(ctx.restrict(l, cuda(xf)).cpu().numpy(), ref) <= 1e-13
            # FP32 transfers
            assert rel(ctx.restrict(l, cuda(xf, np.float32), precision=32).cpu().numpy(), ref) <= 1e-6


@pytest.mark.parametrize("dim,p,N,split", MG_CASES)
def test_level_operators(dim, p, N, split):
    pr = Problem(dim, p, N, split=split, seed=4, active_frac=0.2)
    lv = oracle_levels(pr)
    ctx = pr.context()
    for l in range(1, len(lv)):
        x = np.random.default_rng(l).normal(size=lv[l].mesh.n_dofs)
        y = ctx.apply_jacobian(cuda(x), level=l).cpu().numpy()
        assert rel(y, lv[l].G @ x) <= 1e-12


@pytest.mark.parametrize("dim,p,N,split", MG_CASES)
def test_eigen_smoother_coarse_vcycle_fp64(dim, p, N, split):
    pr = Problem(dim, p, N, split=split, seed=5, active_frac=0.2)
    lv = oracle_levels(pr, cheb_degree=5)
    ctx = pr.context(mg_precision=64)
    for l in range(len(lv) - 1):
        lam = ctx.lambda_max(l)
        assert abs(lam[0] - lv[l].lam_max[0]) <= 1e-9 * lv[l].lam_max[0]
        assert abs(lam[1] - lv[l].lam_max[1]) <= 1e-9 * lv[l].lam_max[1]
        f = np.where(lv[l].mask, 0.0, np.random.default_rng(l).normal(size=lv[l].mesh.n_dofs))
        assert rel(ctx.smooth(l, cuda(f)).cpu().numpy(), S.smooth(lv[l], f)) <= 1e-9
    Lc = lv[-1]
    r = np.where(Lc.mask, 0.0, np.random.default_rng(9).normal(size=Lc.mesh.n_dofs))
    assert rel(ctx.coarse_solve(cuda(r)).cpu().numpy(), spla.spsolve(Lc.G.tocsc(), r)) <= 1e-10
    r = np.where(lv[0].mask, 0.0, np.random.default_rng(10).normal(size=pr.mesh.n_dofs))
    z = ctx.vcycle(cuda(r)).cpu().numpy()
    assert rel(z, S.vcycle(lv, r)) <= 1e-9


@pytest.mark.parametrize("dim,p,N,split", MG_CASES)
def test_coarse_solve_precision(dim, p, N, split):
    """The FP32 multigrid's coarse solve is FP64 by default (dense FP64 inverses): the direct solve of the
    oracle's coarse operator to 1e-10. The FP32 variant (coarse_precision 32) only to FP32 accuracy."""
    pr = Problem(dim, p, N, split=split, seed=5, active_frac=0.2)
    Lc = oracle_levels(pr)[-1]
    r = np.where(Lc.mask, 0.0, np.random.default_rng(9).normal(size=Lc.mesh.n_dofs))
    ref = spla.spsolve(Lc.G.tocsc(), r)
    with pr.context(mg_precision=32) as ctx:
        assert rel(ctx.coarse_solve(cuda(r)).cpu().numpy(), ref) <= 1e-10
    with pr.context(mg_precision=32, coarse_precision=32) as ctx:
        err = rel(ctx.coarse_solve(cuda(r)).cpu().numpy(), ref)
        assert 1e-10 < err <= 1e-3


@pytest.mark.parametrize("dim,p,N,split", MG_CASES)
def test_smoother_fp32(dim, p, N, split):
    """The FP32 smoother of every smoothed level against the oracle's FP64 smoother with the same
    eigenvalue estimate: the FP32 multigrid's own lambda_max agrees with the oracle's to 1e-5 and one
    degree-5 application to 2e-5 (rounding of a few dozen FP32 operations per entry, amplified by at
    most the Chebyshev polynomial's growth on the spectrum)."""
    pr = Problem(dim, p, N, split=split, seed=5, active_frac=0.2)
    lv = oracle_levels(pr, cheb_degree=5)
    with pr.context(mg_precision=32) as ctx:
        for l in range(len(lv) - 1):
            lam = ctx.lambda_max(l)
            for b in range(2):
                assert abs(lam[b] - lv[l].lam_max[b]) <= 1e-5 * lv[l].lam_max[b]
            f = np.where(lv[l].mask, 0.0, np.random.default_rng(l).normal(size=lv[l].mesh.n_dofs))
            x = ctx.smooth(l, cuda(f, np.float32), precision=32).cpu().numpy().astype(np.float64)
            assert rel(x, S.smooth(lv[l], f)) <= 2e-5


@pytest.mark.parametrize("dim,p,N,split,cmin", [(2, 1, 32, 1, 3), (2, 2, 32, 1, 3), (3, 1, 16, 0, 2)])
def test_vcycle_fp32_four_levels(dim, p, N, split, cmin):
    """The FP32 V-cycle (FP64 coarse solve) on four levels against the oracle's FP64 cycle."""
    pr = Problem(dim, p, N, split=split, seed=6, active_frac=0.2)
    lv = S.build_levels(pr.dim, pr.p, pr.N, pr.prm, pr.U, pr.phi_tilde, pr.active, cheb_degree=5,
                        eig_iters=15, eig_seed=0, coarse_min=cmin)
    assert len(lv) >= 4
    with pr.context(mg_precision=32, coarse_min=cmin) as ctx:
        assert ctx.n_levels == len(lv)
        r = np.where(lv[0].mask, 0.0, np.random.default_rng(11).normal(size=pr.mesh.n_dofs))
        assert rel(ctx.vcycle(cuda(r)).cpu().numpy(), S.vcycle(lv, r)) <= 1e-3


@pytest.mark.parametrize("dim,p,N,split,tangent", [(2, 2, 8, 1, 0), (2, 2, 8, 1, 1), (3, 1, 8, 0, 0)])
def test_vcycle_fp32(dim, p, N, split, tangent):
    """Mixed precision: FP32 levels, smoothers and transfers, FP64 coarse solve; agrees with the FP64
    cycle to FP32 accuracy, with stored per-point values and with the recomputed FP32 tangent."""
    pr = Problem(dim, p, N, split=split, seed=6, active_frac=0.2)
    lv = oracle_levels(pr)
    ctx = pr.context(mg_precision=32, fp32_tangent=tangent)
    r = np.where(lv[0].mask, 0.0, np.random.default_rng(11).normal(size=pr.mesh.n_dofs))
    z = ctx.vcycle(cuda(r)).cpu().numpy()
    assert rel(z, S.vcycle(lv, r)) <= 1e-3


@pytest.mark.parametrize("dim,p,N", [(2, 2, 64), (3, 2, 8)])
def test_fp32_run_to_run_variation(dim, p, N, capsys):
    """Tile seams are summed with atomics, so the order of the FP32 sums, and with it the last bits of
    an FP32 apply and of the FP32 V-cycle, may change from run to run. Ten repetitions on several tiles:
    the largest relative difference from the first run stays at FP32 rounding (recorded in the output),
    and the FP64 applies are reproducible to 1e-15."""
    pr = Problem(dim, p, N, split=1, seed=12, active_frac=0.2)
    ctx = pr.context(mg_precision=32)
    x = cuda(np.random.default_rng(13).normal(size=pr.mesh.n_dofs))
    r = cuda(np.where(pr.mask, 0.0, np.random.default_rng(14).normal(size=pr.mesh.n_dofs)))
    y0 = ctx.apply_jacobian(x.float(), precision=32).double()
    z0 = ctx.vcycle(r)
    yd0 = ctx.apply_jacobian(x)
    dy = dz = dd = 0.0
    for _ in range(10):
        dy = max(dy, float((ctx.apply_jacobian(x.float(), precision=32).double() - y0).norm() / y0.norm()))
        dz = max(dz, float((ctx.vcycle(r) - z0).norm() / z0.norm()))
        dd = max(dd, float((ctx.apply_jacobian(x) - yd0).norm() / yd0.norm()))
    with capsys.disabled():
        print("\nrun-to-run variation %dD Q%d %d^%d: FP32 apply %.2e, FP32 V-cycle %.2e, FP64 apply %.2e"
              % (dim, p, N, dim, dy, dz, dd))
    assert dy <= 1e-6 and dz <= 1e-5 and dd <= 1e-15


@pytest.mark.parametrize("prec,fp64_mode", [(64, 0), (32, 0), (32, 1)])
@pytest.mark.parametrize("dim,p,N,split", [(2, 2, 16, 1), (3, 2, 4, 1)])
def test_fgmres_solve(prec, fp64_mode, dim, p, N, split):
    pr = Problem(dim, p, N, split=split, seed=7, active_frac=0.1)
    ctx = pr.context(mg_precision=prec, fp64_mode=fp64_mode)
    Gm = fe.masked(pr.G(), pr.mask)
    b = np.where(pr.mask, 0.0, np.random.default_rng(12).normal(size=pr.mesh.n_dofs))
    x, its, relres = ctx.solve_linear(cuda(b))
    x = x.cpu().numpy()
    assert np.linalg.norm(Gm @ x - b) <= 1.01e-6 * np.linalg.norm(b)
    assert its < 60
    xd = spla.spsolve(Gm.tocsc(), b)
    assert rel(x, xd) <= 1e-3


def test_fgmres_beyond_sixteen_basis_vectors():
    """FGMRES whose Krylov basis grows past 16 vectors in one cycle. There, CGS2 leaves its fused
    passes (one instantiation per basis size up to 16) for the separate multi-dot and update kernels.
    A one-step smoother and a tight tolerance force the iterations. The solution must match the
    direct solve, and the true residual must meet the tolerance."""
    pr = Problem(2, 2, 8, split=1, seed=7, active_frac=0.1)
    ctx = pr.context(mg_precision=64, cheb_degree=1, lin_rtol=1e-11, gmres_restart=30)
    Gm = fe.masked(pr.G(), pr.mask)
    b = np.where(pr.mask, 0.0, np.random.default_rng(13).normal(size=pr.mesh.n_dofs))
    x, its, relres = ctx.solve_linear(cuda(b))
    x = x.cpu().numpy()
    assert its > 16 and relres <= 1e-11
    assert np.linalg.norm(Gm @ x - b) <= 1e-8 * np.linalg.norm(b)
    xd = spla.spsolve(Gm.tocsc(), b)
    assert rel(x, xd) <= 1e-6


@pytest.mark.parametrize("split", [0, 1])
def test_newton_step_c1(split):
    """The tension test of the paper at 32 x 32 Q1 (3267 DoFs): one primal-dual active-set step with
    GMG-preconditioned FGMRES against the oracle's step with a direct solve."""
    from oracle import mesh as M
    m = M.Mesh(2, 1, 32)
    prm = fe.Params(121.15, 80.77, 2.7e-3, 2.0 / 32, 1e-10, split)
    U = m.dirichlet_values(1e-3)
    phi = np.ones(m.n_nodes)
    phi[m.slit_nodes()] = 0.0
    U[2 * m.n_nodes:] = phi
    from paper_2005_00331_gb300 import setup_mesh
    for prec in (64, 32):
        ctx = setup_mesh(dim=2, degree=1, n_cells_1d=32, split=split, eps=2.0 / 32, mg_precision=prec)
        ctx.set_state(cuda(U), cuda(phi), cuda(phi), None)
        Uo, act, rn, _ = S.pdas_step(m, prm, U, phi, phi)
        rep = ctx.solve_newton_step()
        np.testing.assert_array_equal(ctx.get_active().cpu().numpy().astype(bool), act)
        assert abs(rep["res_norm"] - rn) <= 1e-12 * rn
        Ug = ctx.get_state().cpu().numpy()
        assert np.linalg.norm(Ug - Uo) <= 1e-4 * np.linalg.norm(Uo - U)
        assert rep["gmres_rel"] <= 1e-6


def test_pdas_loop_reaches_newton_tolerance():
    """Alg. 1 repeated on the GPU until the active set is unchanged and ||R~|| <= 1e-8 ||R~_0||; the final
    residual is re-checked by the oracle in FP64."""
    from oracle import mesh as M
    from paper_2005_00331_gb300 import setup_mesh
    m = M.Mesh(2, 1, 16)
    prm = fe.Params(121.15, 80.77, 2.7e-3, 2.0 / 16, 1e-10, 1)
    U = m.dirichlet_values(1e-3)
    phi = np.ones(m.n_nodes)
    phi[m.slit_nodes()] = 0.0
    U[2 * m.n_nodes:] = phi
    ctx = setup_mesh(dim=2, degree=1, n_cells_1d=16, split=1, eps=2.0 / 16, mg_precision=32, lin_rtol=1e-10)
    ctx.set_state(cuda(U), cuda(phi), cuda(phi), None)
    st, reps = ctx.solve_pdas(max_iters=15, newton_rtol=1e-8)
    norms = [r["res_norm"] for r in reps]
    assert st == 0 and norms[-1] <= 1e-8 * norms[0] and reps[-1]["n_changed"] == 0
    Ug = ctx.get_state().cpu().numpy()
    R = fe.residual(m, prm, Ug, phi)
    act = ctx.get_active().cpu().numpy().astype(bool)
    mask = S.newton_mask(m, act)
    assert np.linalg.norm(np.where(mask, 0, R)) <= 1e-7 * norms[0]


@pytest.mark.parametrize("dim,p,N,split", [(2, 2, 6, 1), (3, 1, 4, 0), (2, 3, 4, 0)])
def test_param_grad_and_adjoint(dim, p, N, split):
    pr = Problem(dim, p, N, split=split, seed=8, fields=True)
    ctx = pr.context()
    v = np.random.default_rng(13).normal(size=pr.mesh.n_dofs)
    vm = np.where(pr.mesh.dirichlet_mask(), 0.0, v)
    g = [t.cpu().numpy() for t in ctx.param_grad(cuda(v))]
    ref = fe.param_grad(pr.mesh, pr.prm, pr.U, pr.phi_tilde, vm, **pr.fields)
    for a, b in zip(g, ref):
        assert rel(a, b) <= 1e-12
    from paper_2005_00331_gb300 import PFF_MASK_ADJOINT, PFF_MODE_TRANSPOSE
    gU = ctx.apply_jacobian(cuda(v), mode=PFF_MODE_TRANSPOSE | PFF_MASK_ADJOINT).cpu().numpy()
    assert rel(gU, pr.G().T @ vm) <= 1e-12


@pytest.mark.parametrize("dim,p,N,loads", [(2, 1, 16, [4e-3, 8e-3, 1.2e-2]), (2, 2, 8, [1e-4, 2e-4, 3e-4]),
                                             (3, 1, 4, [1e-4, 2e-4, 3e-4])])
def test_load_steps_against_oracle(dim, p, N, loads):
    """Three quasi-static load steps with the extrapolated phase field, Miehe split: GPU (FGMRES + mixed
    GMG) against the oracle (direct solves). Every step converges on both sides (status and the
    oracle's own test), in the same number of Newton iterations up to one, to the same state. The 2D Q2
    and 3D Q1 cases are ones whose second step never converged when phi~ was extrapolated from the
    initial phase field."""
    from oracle import mesh as M
    from paper_2005_00331_gb300 import setup_mesh
    m = M.Mesh(dim, p, N)
    prm = fe.Params(121.15, 80.77, 2.7e-3, 2.0 / N, 1e-10, 1)
    U = m.dirichlet_values(0.0)
    phi = np.ones(m.n_nodes)
    phi[m.slit_nodes()] = 0.0
    U[dim * m.n_nodes:] = phi
    stats = []
    ref = S.load_steps(m, prm, U, loads, stats=stats)
    assert all(conv for _, conv in stats)
    ctx = setup_mesh(dim=dim, degree=p, n_cells_1d=N, split=1, eps=2.0 / N, mg_precision=32, lin_rtol=1e-10)
    ctx.set_state(cuda(U), cuda(phi), cuda(phi), None)
    for k, load in enumerate(loads):
        st, reps = ctx.solve_load_step(load, check=False)
        assert st == 0
        assert abs(len(reps) - stats[k][0]) <= 1
        Ug = ctx.get_state().cpu().numpy()
        assert rel(Ug, ref[k]) <= 1e-6
        assert ctx.get_history()[0] == min(k + 1, 2)
