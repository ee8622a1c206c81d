"""Pins of the oracle's transfers, Chebyshev smoother, eigenvalue estimate, FGMRES, V-cycle and
primal-dual active-set step (Alg. 1)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fe, material as mat, mesh as M, solvers as S

LAM, MU, GC, KAPPA = 121.15, 80.77, 2.7e-3, 1e-10


def test_splitmix64_published_vector():
    # first outputs of the reference SplitMix64 generator seeded with 1234567
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
           16408922859458223821]
    assert [S.splitmix64(1234567, i) for i in range(5)] == ref
    v = S.start_vector(1000, 0)
    assert v.min() >= -0.5 and v.max() < 0.5 and abs(v.mean()) < 0.05


def qp_poly(coords, p, rng):
    """A random polynomial of degree <= p in every coordinate (an element of Q_p)."""
    d = coords.shape[1]
    cf = rng.normal(size=(p + 1,) * d)
    out = np.zeros(len(coords))
    for idx in np.ndindex(*cf.shape):
        out += cf[idx] * np.prod([coords[:, t] ** idx[t] for t in range(d)], axis=0)
    return out


@pytest.mark.parametrize("dim,p,Nc", [(2, 1, 2), (2, 2, 3), (2, 3, 2), (2, 4, 2), (3, 2, 2), (3, 3, 1)])
def test_transfers_reproduce_polynomials(dim, p, Nc):
    """P10: prolongation reproduces every coarse Q_p function at the fine nodes; the state
    interpolation (fine -> coarse) reproduces fine Q_p functions at the coarse nodes."""
    rng = np.random.default_rng(20)
    mc, mf = M.Mesh(dim, p, Nc), M.Mesh(dim, p, 2 * Nc)
    P = S.prolongation(dim, p, Nc, 2 * Nc)
    T = S.state_interpolation(dim, p, 2 * Nc, Nc)
    for _ in range(3):
        np.testing.assert_allclose(P @ qp_poly(mc.coords, p, np.random.default_rng(_)),
                                   qp_poly(mf.coords, p, np.random.default_rng(_)), atol=1e-12)
        np.testing.assert_allclose(T @ qp_poly(mf.coords, p, np.random.default_rng(_)),
                                   qp_poly(mc.coords, p, np.random.default_rng(_)), atol=1e-12)
    # partition of unity and interpolation property
    np.testing.assert_allclose(P @ np.ones(mc.n_nodes), 1.0, atol=1e-14)
    np.testing.assert_allclose((T @ P).toarray(), np.eye(mc.n_nodes), atol=1e-13)


def test_colocated_nodes():
    # p = 2: every coarse node coincides with a fine vertex; p = 3: only coarse vertices do
    assert np.all(S.colocated_1d(4, 8, 2) == 2 * np.arange(9))
    c3 = S.colocated_1d(2, 4, 3)
    assert list(np.nonzero(c3 >= 0)[0]) == [0, 3, 6] and list(c3[[0, 3, 6]]) == [0, 6, 12]
    c4 = S.colocated_1d(2, 4, 4)
    assert list(np.nonzero(c4 >= 0)[0]) == [0, 2, 4, 6, 8]


@pytest.mark.parametrize("degree", [1, 2, 3, 5])
def test_chebyshev_closed_form_on_diagonal(degree):
    """P11: on A = diag(a), D = I the error after s steps is p_s(A) e_0 with the shifted and
    scaled Chebyshev polynomial p_s(t) = T_s((theta - t)/delta) / T_s(theta/delta)."""
    rng = np.random.default_rng(21)
    a = np.sort(rng.uniform(0.01, 2.0, 50))
    f = rng.normal(size=50)
    lam_max = a.max()
    x = S.chebyshev(lambda v: a * v, np.ones(50), f, degree, lam_max)
    lo, hi = 0.24 * lam_max, 1.2 * lam_max
    theta, delta = (lo + hi) / 2, (hi - lo) / 2

    def Tn(n, z):
        z = np.asarray(z, dtype=np.float64)
        return np.where(np.abs(z) <= 1, np.cos(n * np.arccos(np.clip(z, -1, 1))),
                        np.cosh(n * np.arccosh(np.maximum(np.abs(z), 1))) * np.sign(z) ** n)

    ps = Tn(degree, (theta - a) / delta) / Tn(degree, theta / delta)
    np.testing.assert_allclose(x, (1 - ps) * f / a, rtol=1e-11, atol=1e-12)


def test_cg_lanczos_exact_after_n_steps():
    rng = np.random.default_rng(22)
    n = 12
    B = rng.normal(size=(n, n))
    A = B @ B.T + n * np.eye(n)
    dinv = 1 / np.diag(A)
    ev = S.cg_lanczos(lambda v: A @ v, dinv, rng.normal(size=n), n)
    Ds = np.diag(np.sqrt(dinv))
    ref = np.linalg.eigvalsh(Ds @ A @ Ds)
    assert abs(ev.max() - ref.max()) < 1e-8 * ref.max()
    assert abs(ev.min() - ref.min()) < 1e-8 * ref.max()
    # few steps: the estimate is a lower bound of lambda_max (Ritz value)
    ev5 = S.cg_lanczos(lambda v: A @ v, dinv, rng.normal(size=n), 5)
    assert ev5.max() <= ref.max() * (1 + 1e-12)


def test_fgmres_against_direct_solve():
    rng = np.random.default_rng(23)
    n = 80
    A = sp.random(n, n, density=0.1, random_state=1) + 4 * sp.eye(n)
    b = rng.normal(size=n)
    x, its, rel = S.fgmres(lambda v: A @ v, b, lambda v: v, tol=1e-10, restart=15)
    ref = spla.spsolve(A.tocsc(), b)
    assert rel <= 1e-10 and np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b) * 1.01
    np.testing.assert_allclose(x, ref, rtol=1e-8, atol=1e-9)
    # exact preconditioner: one iteration
    Ainv = spla.factorized(A.tocsc())
    _, its1, _ = S.fgmres(lambda v: A @ v, b, Ainv, tol=1e-10)
    assert its1 == 1


def c1_state(m, load=1e-3):
    """Tension-test state: u = 0 with the top load lifted, phi = 1 except 0 on the slit."""
    U = m.dirichlet_values(load)
    phi = np.ones(m.n_nodes)
    phi[m.slit_nodes()] = 0.0
    U[m.dim * m.n_nodes:] = phi
    return U, phi


def test_active_set_rule():
    """Alg. 1 with r = -R: phi DoFs where -R/m + c (phi - phi_old) > 0 (strict), phi DoFs only."""
    m = M.Mesh(2, 1, 2)
    nn = m.n_nodes
    R = np.zeros(m.n_dofs)
    mass = fe.lumped_mass(m)
    phi = np.full(nn, 0.5)
    phi_old = np.full(nn, 0.5)
    R[2 * nn:] = np.linspace(-1, 1, nn) * mass   # -R/m = -linspace
    R[:2 * nn] = -1e9                            # displacement rows never count
    act = S.active_set(m, R, phi, phi_old, c=1.0)
    np.testing.assert_array_equal(act, np.linspace(-1, 1, nn) < 0)
    # a tie (exactly zero) is inactive; a violated bound phi > phi_old makes a DoF active
    R[2 * nn:] = 0.0
    assert not S.active_set(m, R, phi, phi_old).any()
    assert S.active_set(m, R, phi + 1e-3, phi_old).all()


@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_gmg_fgmres_step_matches_direct_step(split):
    """One PDAS step of the tension test (C1-like, 16x16 Q1): the FGMRES + GMG solution equals the
    direct solution within the linear tolerance, and the V-cycle contracts."""
    m = M.Mesh(2, 1, 16)
    prm = fe.Params(LAM, MU, GC, 2.0 / 16, KAPPA, split)
    U, phi = c1_state(m)
    U1, act1, r1, _ = S.pdas_step(m, prm, U, phi, phi, solve="direct")
    U2, act2, r2, info = S.pdas_step(m, prm, U, phi, phi, solve="gmg", levels_kw=dict(cheb_degree=3))
    np.testing.assert_array_equal(act1, act2)
    assert info["gmres_rel"] <= 1e-6
    dU = U1 - U
    assert np.linalg.norm(U2 - U1) <= 1e-5 * np.linalg.norm(dU)
    # slit phi DoFs heal under R -> active, reset to phi_old = 0 and kept there
    assert act1[m.slit_nodes()].all()
    np.testing.assert_array_equal(U1[2 * m.n_nodes:][m.slit_nodes()], 0.0)


def test_vcycle_contracts():
    m = M.Mesh(2, 2, 8)
    prm = fe.Params(LAM, MU, GC, 2.0 / 8, KAPPA, mat.SPLIT_MIEHE)
    rng = np.random.default_rng(24)
    U = m.dirichlet_values(1e-3)
    U[:2 * m.n_nodes] += np.where(m.dirichlet_mask()[:2 * m.n_nodes], 0, rng.normal(0, 1e-4, 2 * m.n_nodes))
    U[2 * m.n_nodes:] = rng.uniform(0.9, 1, m.n_nodes)
    act = np.zeros(m.n_nodes, dtype=bool)
    lv = S.build_levels(2, 2, 8, prm, U, U[2 * m.n_nodes:], act, cheb_degree=3)
    G = lv[0].G
    e = rng.normal(size=m.n_dofs)
    e[lv[0].mask] = 0
    # error propagation of one V-cycle as a stationary iteration: e <- e - M^{-1} G e. G is block
    # lower triangular, so the first cycle moves displacement error into the phase field (its
    # Euclidean norm can grow once); the asymptotic rate (spectral radius) is what must be < 1.
    e0 = np.linalg.norm(e)
    ratios = []
    for _ in range(10):
        e_new = e - S.vcycle(lv, G @ e)
        ratios.append(np.linalg.norm(e_new) / np.linalg.norm(e))
        e = e_new
    assert max(ratios[3:]) < 0.5
    assert np.linalg.norm(e) < 1e-2 * e0


def test_pdas_loop_converges_tension_test():
    """Alg. 1 repeated: active sets settle and the reduced residual drops below 1e-8 relative."""
    m = M.Mesh(2, 1, 8)
    prm = fe.Params(LAM, MU, GC, 2.0 / 8, KAPPA, mat.SPLIT_MIEHE)
    U, phi_old = c1_state(m)
    norms, acts = [], []
    for k in range(12):
        U, act, rn, _ = S.pdas_step(m, prm, U, phi_old, phi_old)
        norms.append(rn)
        acts.append(act)
        if k > 0 and np.array_equal(acts[-1], acts[-2]) and rn <= 1e-8 * norms[0]:
            break
    assert norms[-1] <= 1e-8 * norms[0]
    # irreversibility: phi never exceeds phi_old
    assert np.all(U[2 * m.n_nodes:] <= phi_old + 1e-12)


def _cheb_smoother_dense(A, d, degree, lam_max, lo=0.24, hi=1.2):
    """x = S f of a Chebyshev-Jacobi smoother with zero initial guess, as a dense matrix from its
    error polynomial (Saad, Sec. 12.3): A^{-1} f - x = T_s((theta - M)/delta) / T_s(theta/delta) A^{-1} f
    with M = D^{-1} A, evaluated through the eigen-decomposition of D^{-1/2} A D^{-1/2} instead of the
    three-term recurrence."""
    a, b = lo * lam_max, hi * lam_max
    theta, delta = 0.5 * (a + b), 0.5 * (b - a)
    Ts = np.polynomial.chebyshev.Chebyshev.basis(degree)
    sq = np.sqrt(d)
    w, Q = np.linalg.eigh(A / np.outer(sq, sq))
    R = (Q * (Ts((theta - w) / delta) / Ts(theta / delta))) @ Q.T
    R = R / sq[:, None] * sq[None, :]  # D^{-1/2} R_sym D^{1/2}
    return (np.eye(len(d)) - R) @ np.linalg.inv(A)


@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_vcycle_equals_dense_two_grid(split):
    """The V-cycle as a composition: on two levels it equals e = S r, e += P Gc^{-1} P^T (r - G e)
    (masked as stated in the readings), e += S (r - G e), with the smoother built from its closed-form
    error polynomial and the coarse operator inverted densely."""
    dim, p, N = 2, 1, 8
    m = M.Mesh(dim, p, N)
    prm = fe.Params(LAM, MU, GC, 2.0 / N, KAPPA, split)
    rng = np.random.default_rng(31)
    U = m.dirichlet_values(1e-3)
    U[:dim * m.n_nodes] += np.where(m.dirichlet_mask()[:dim * m.n_nodes], 0, rng.normal(0, 1e-4, dim * m.n_nodes))
    U[dim * m.n_nodes:] = rng.uniform(0.9, 1, m.n_nodes)
    act = rng.uniform(size=m.n_nodes) < 0.2
    lv = S.build_levels(dim, p, N, prm, U, U[dim * m.n_nodes:], act, cheb_degree=4)
    assert len(lv) == 2
    L0, L1 = lv
    r = np.where(L0.mask, 0.0, rng.normal(size=m.n_dofs))
    e_oracle = S.vcycle(lv, r)

    G = L0.G.toarray()
    nu = L0.nu
    Sm = np.zeros_like(G)
    Sm[:nu, :nu] = _cheb_smoother_dense(L0.Guu.toarray(), L0.diag[:nu], 4, L0.lam_max[0])
    Sm[nu:, nu:] = _cheb_smoother_dense(L0.Gpp.toarray(), L0.diag[nu:], 4, L0.lam_max[1])
    P1 = L1.P.toarray()
    P = np.kron(np.eye(dim + 1), P1)  # component-blocked vectors
    Gc_inv = np.linalg.inv(L1.G.toarray())
    e = Sm @ r
    rc = P.T @ (r - G @ e)
    rc[L1.mask] = 0.0
    pe = P @ (Gc_inv @ rc)
    pe[L0.mask] = 0.0
    e = e + pe
    e = e + Sm @ (r - G @ e)
    assert np.linalg.norm(e - e_oracle) <= 1e-10 * np.linalg.norm(e_oracle)
