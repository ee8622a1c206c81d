"""Pins of the oracle's residual (Eq. residual), Jacobian (Eq. G) and energy (Sec. 2.1).

Independent references: exact symbolic integration of textbook element matrices (sympy),
finite differences of the residual and of the energy, the constant-strain patch test and the
phi = 1 limit, in which the displacement block is plain linear elasticity.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import basis, fe, material as mat, mesh as M

sympy = pytest.importorskip("sympy")

LAM, MU, GC, KAPPA = 121.15, 80.77, 2.7e-3, 1e-10


def sym_element(dim, p, h, eps):
    """Exact textbook element matrices on [0,h]^dim: mass, Laplace, isotropic elasticity.

    The Q_p shape functions are tensor products, so every integral is a product of exact 1D
    integrals I_sr[a, b] = int_0^h l_a^(s) l_b^(r) dx (s, r = derivative orders), done in sympy."""
    x = sympy.symbols("x")
    nodes = [sympy.Rational(k, p) for k in range(p + 1)]  # GLL nodes = equidistant for p <= 2
    assert p <= 2
    hh = sympy.Rational(1) / sympy.Rational(round(1 / h))

    def lag(k):
        out = sympy.Integer(1)
        for m in range(p + 1):
            if m != k:
                out *= (x / hh - nodes[m]) / (nodes[k] - nodes[m])
        return out

    L = [lag(k) for k in range(p + 1)]
    dL = [sympy.diff(f, x) for f in L]
    I = {}
    for s_, A in ((0, L), (1, dL)):
        for r_, B in ((0, L), (1, dL)):
            I[s_, r_] = np.array([[float(sympy.integrate(A[a] * B[b], (x, 0, hh))) for b in range(p + 1)]
                                  for a in range(p + 1)])
    import itertools
    locs = [tuple(reversed(t)) for t in itertools.product(range(p + 1), repeat=dim)]  # x fastest
    na = len(locs)

    def prod(da, db):
        """int d^{da} N_a d^{db} N_b with da, db = derivative direction or None."""
        out = np.ones((na, na))
        for a in range(na):
            for b in range(na):
                for t in range(dim):
                    out[a, b] *= I[int(da == t), int(db == t)][locs[a][t], locs[b][t]]
        return out

    Mm = prod(None, None)
    Kl = sum(prod(t, t) for t in range(dim))
    # sigma(du) : e(w), w = N_a e_k, du = N_b e_l
    Ke = np.zeros((dim, na, dim, na))
    for k in range(dim):
        for l in range(dim):
            Ke[k, :, l, :] = LAM * prod(k, l) + MU * prod(l, k)
            if k == l:
                Ke[k, :, l, :] += MU * Kl
    return Mm, Kl, Ke.reshape(dim * na, dim * na)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_single_cell_closed_forms(dim, p, split):
    """P2: one cell, u = 0, phi = phi~ = 1: G_uu = elasticity K, G_phiphi = G_c (M/eps + eps K_lap)."""
    N = 1
    m = M.Mesh(dim, p, N)
    eps = 0.3
    prm = fe.Params(LAM, MU, GC, eps, KAPPA, split)
    U = np.zeros(m.n_dofs)
    U[dim * m.n_nodes:] = 1.0
    G = fe.assemble(m, prm, U, np.ones(m.n_nodes)).toarray()
    Mm, Kl, Ke = sym_element(dim, p, m.h, eps)
    nu = dim * m.n_nodes
    np.testing.assert_allclose(G[:nu, :nu], Ke, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(G[nu:, nu:], GC * (Mm / eps + eps * Kl), rtol=1e-12, atol=1e-16)
    assert np.abs(G[nu:, :nu]).max() == 0.0 and np.abs(G[:nu, nu:]).max() == 0.0


def random_state(m, rng, phi_lo=0.9):
    U = np.zeros(m.n_dofs)
    nn, d = m.n_nodes, m.dim
    U[:d * nn] = rng.normal(0, 1e-2, d * nn)
    U[d * nn:] = rng.uniform(phi_lo, 1.0, nn)
    pt = np.clip(U[d * nn:] + rng.normal(0, 0.02, nn), 0, 1)
    return U, pt


CASES = [(2, 1, 3), (2, 2, 2), (2, 3, 2), (2, 4, 1), (3, 1, 2), (3, 2, 1)]


@pytest.mark.parametrize("dim,p,N", CASES)
@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_jacobian_is_derivative_of_residual(dim, p, N, split):
    """P4: G = dR/dU with phi~ frozen (central differences along random directions)."""
    m = M.Mesh(dim, p, N)
    rng = np.random.default_rng(10 + p)
    prm = fe.Params(LAM, MU, GC, 0.2, KAPPA, split)
    U, pt = random_state(m, rng)
    G = fe.assemble(m, prm, U, pt)
    for _ in range(2):
        v = rng.normal(size=m.n_dofs)
        h = 1e-6 * np.linalg.norm(U) / np.linalg.norm(v)
        fd = (fe.residual(m, prm, U + h * v, pt, zero_dirichlet=False)
              - fe.residual(m, prm, U - h * v, pt, zero_dirichlet=False)) / (2 * h)
        gv = G @ v
        assert np.linalg.norm(fd - gv) <= 1e-6 * np.linalg.norm(gv)


@pytest.mark.parametrize("dim,p,N", [(2, 2, 2), (3, 1, 2)])
@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_residual_is_energy_gradient(dim, p, N, split):
    """P5: with phi~ = phi the residual is the gradient of the discrete energy."""
    m = M.Mesh(dim, p, N)
    rng = np.random.default_rng(7)
    prm = fe.Params(LAM, MU, GC, 0.2, KAPPA, split)
    U, _ = random_state(m, rng)
    phi = U[dim * m.n_nodes:]
    R = fe.residual(m, prm, U, phi, zero_dirichlet=False)
    for _ in range(3):
        v = rng.normal(size=m.n_dofs)
        h = 1e-6 * np.linalg.norm(U) / np.linalg.norm(v)
        fd = (fe.energy(m, prm, U + h * v) - fe.energy(m, prm, U - h * v)) / (2 * h)
        assert abs(fd - R @ v) <= 1e-6 * max(abs(R @ v), 1e-12)


@pytest.mark.parametrize("dim,p,N", [(2, 1, 4), (2, 3, 3), (3, 2, 2)])
@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_patch_test(dim, p, N, split):
    """P7: u = A x + b, phi = 1: R_u = 0 at interior DoFs; R_phi = g'(1) E_s^+(A) int psi."""
    m = M.Mesh(dim, p, N)
    rng = np.random.default_rng(8)
    A = rng.normal(0, 1e-3, (dim, dim))
    b = rng.normal(0, 1e-3, dim)
    U = np.zeros(m.n_dofs)
    for k in range(dim):
        U[k * m.n_nodes:(k + 1) * m.n_nodes] = m.coords @ A[k] + b[k]
    U[dim * m.n_nodes:] = 1.0
    prm = fe.Params(LAM, MU, GC, 0.2, KAPPA, split)
    R = fe.residual(m, prm, U, np.ones(m.n_nodes), zero_dirichlet=False)
    interior = np.all((m.node_ijk > 0) & (m.node_ijk < m.n1 - 1), axis=1)
    ru = R[:dim * m.n_nodes].reshape(dim, -1)[:, interior]
    assert np.abs(ru).max() < 1e-13
    e = 0.5 * (A + A.T)
    Esp = mat.stress_energy(e[None], LAM, MU, split)[2][0]
    np.testing.assert_allclose(R[dim * m.n_nodes:], mat.dg(1.0, KAPPA) * Esp * fe.lumped_mass(m), rtol=1e-11)


@pytest.mark.parametrize("dim,p,N", [(2, 2, 2), (3, 1, 2)])
def test_phi_one_limit_is_linear_elasticity(dim, p, N):
    """P8: phi = phi~ = 1 -> G_uu is the isotropic elasticity matrix for both splits, and
    G_phiu = g'(1) sigma : e(du) psi."""
    m = M.Mesh(dim, p, N)
    rng = np.random.default_rng(9)
    U, _ = random_state(m, rng)
    U[dim * m.n_nodes:] = 1.0
    one = np.ones(m.n_nodes)
    Gn = fe.assemble(m, fe.Params(LAM, MU, GC, 0.2, KAPPA, mat.SPLIT_NONE), U, one)
    Gm = fe.assemble(m, fe.Params(LAM, MU, GC, 0.2, KAPPA, mat.SPLIT_MIEHE), U, one)
    nu = dim * m.n_nodes
    d_uu = abs(Gn[:nu, :nu] - Gm[:nu, :nu]).max()
    assert d_uu <= 1e-12 * abs(Gn[:nu, :nu]).max()
    # G_uu with the state-independent elasticity matrix of a zero state
    G0 = fe.assemble(m, fe.Params(LAM, MU, GC, 0.2, KAPPA, mat.SPLIT_NONE), np.where(np.arange(m.n_dofs) < nu, 0.0, 1.0), one)
    assert abs(G0[:nu, :nu] - Gn[:nu, :nu]).max() <= 1e-12 * abs(Gn[:nu, :nu]).max()


@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_structure(split):
    """P9: G_uphi = 0 (R_u does not depend on phi), G_uu and G_phiphi symmetric, masked rows identity,
    transpose mode is the transpose, element-by-element product equals the assembled one (P3)."""
    m = M.Mesh(2, 2, 3)
    rng = np.random.default_rng(11)
    prm = fe.Params(LAM, MU, GC, 0.2, KAPPA, split)
    U, pt = random_state(m, rng)
    G = fe.assemble(m, prm, U, pt)
    nu = 2 * m.n_nodes
    # d R_u / d phi by finite differences of the residual (phi~ held fixed) is zero
    v = np.zeros(m.n_dofs)
    v[nu:] = rng.normal(size=m.n_nodes)
    Rp = fe.residual(m, prm, U + 1e-3 * v, pt, zero_dirichlet=False)
    Rm = fe.residual(m, prm, U - 1e-3 * v, pt, zero_dirichlet=False)
    assert np.abs((Rp - Rm)[:nu]).max() == 0.0
    assert abs(G[:nu, :nu] - G[:nu, :nu].T).max() <= 1e-12 * abs(G[:nu, :nu]).max()
    assert abs(G[nu:, nu:] - G[nu:, nu:].T).max() <= 1e-12 * abs(G[nu:, nu:]).max()
    Gt = fe.assemble(m, prm, U, pt, mode=fe.MODE_TRANSPOSE)
    assert abs(Gt - G.T).max() <= 1e-14 * abs(G).max()
    Gb = fe.assemble(m, prm, U, pt, mode=fe.MODE_BLOCKDIAG)
    assert abs(Gb[nu:, :nu]).max() == 0.0 and abs(Gb[nu:, nu:] - G[nu:, nu:]).max() == 0.0
    x = rng.normal(size=m.n_dofs)
    np.testing.assert_allclose(fe.apply_ebe(m, prm, U, pt, x), G @ x, rtol=1e-13, atol=1e-13 * np.abs(G @ x).max())
    mask = m.dirichlet_mask()
    Gm = fe.masked(G, mask)
    np.testing.assert_allclose(Gm @ x, fe.apply_masked(G, mask, x), rtol=1e-14, atol=1e-14)
    np.testing.assert_array_equal((Gm @ x)[mask], x[mask])


@pytest.mark.parametrize("dim,p,N", [(2, 1, 3), (2, 3, 2), (3, 2, 2)])
def test_lumped_mass_is_gll_weight_product(dim, p, N):
    m = M.Mesh(dim, p, N)
    w = basis.gll_weights(p)
    # int psi_i = h^d prod_t (sum of the GLL weights of the 1D node over the cells sharing it)
    w1 = np.zeros(m.n1)
    for c in range(N):
        w1[c * p:c * p + p + 1] += w * m.h
    ref = np.prod(w1[m.node_ijk], axis=1)
    np.testing.assert_allclose(fe.lumped_mass(m), ref, rtol=1e-13)
    assert abs(fe.lumped_mass(m).sum() - 1.0) < 1e-13


@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_param_grad_finite_differences(split):
    """(dR/d field)^T v for nodal G_c, lambda, mu fields against central differences of R."""
    m = M.Mesh(2, 2, 2)
    rng = np.random.default_rng(12)
    prm = fe.Params(LAM, MU, GC, 0.2, KAPPA, split)
    U, pt = random_state(m, rng)
    fields = dict(gc_field=GC * np.exp(rng.normal(0, 0.2, m.n_nodes)),
                  lam_field=LAM * (1 + 0.1 * rng.normal(size=m.n_nodes)),
                  mu_field=MU * (1 + 0.1 * rng.normal(size=m.n_nodes)))
    v = rng.normal(size=m.n_dofs)
    v[m.dirichlet_mask()] = 0.0
    grads = fe.param_grad(m, prm, U, pt, v, **fields)
    for gi, key in enumerate(("gc_field", "lam_field", "mu_field")):
        dirv = rng.normal(size=m.n_nodes)
        h = 1e-6 * np.linalg.norm(fields[key]) / np.linalg.norm(dirv)
        fp = dict(fields)
        fm = dict(fields)
        fp[key] = fields[key] + h * dirv
        fm[key] = fields[key] - h * dirv
        fd = (fe.residual(m, prm, U, pt, **fp) - fe.residual(m, prm, U, pt, **fm)) @ v / (2 * h)
        assert abs(fd - grads[gi] @ dirv) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("dim,p,N", [(2, 1, 4), (2, 3, 3), (3, 2, 2)])
@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
@pytest.mark.parametrize("load", [2e-3, -2e-3])
def test_reaction_force_uniaxial_strain(dim, p, N, split, load):
    """Load-displacement ordinate in closed form: u_d = load x_d (top face moved by `load`, bottom
    fixed, no lateral motion) and phi = phi~ = c give a uniform stress with sigma_dd = (lambda + 2 mu)
    load on the unit top face. Without a split all of it is degraded by g(c); with the Miehe split a
    stretched specimen (load > 0) is degraded and a compressed one is not."""
    c = 0.7
    m = M.Mesh(dim, p, N)
    U = np.zeros(m.n_dofs)
    U[(dim - 1) * m.n_nodes:dim * m.n_nodes] = load * m.coords[:, dim - 1]
    U[dim * m.n_nodes:] = c
    F = fe.reaction_force(m, fe.Params(LAM, MU, GC, 0.2, KAPPA, split), U, np.full(m.n_nodes, c))
    degraded = split == mat.SPLIT_NONE or load > 0
    expect = (LAM + 2 * MU) * load * (mat.g(c, KAPPA) if degraded else 1.0)
    assert abs(F - expect) <= 1e-13 * abs(expect)


def test_reaction_force_balance():
    """The basis functions sum to one and a rigid translation has no strain, so every u-component of
    the residual (Dirichlet rows kept) sums to zero over all nodes for any state; at a converged load
    step (residual with the phi~ the step solved with) the interior u-rows vanish as well, and the top
    reaction equals minus the bottom one."""
    from oracle import solvers as S
    m = M.Mesh(2, 1, 8)
    prm = fe.Params(LAM, MU, GC, 2.0 / 8, KAPPA, mat.SPLIT_MIEHE)
    rng = np.random.default_rng(12)
    U, phit = random_state(m, rng)
    R = fe.residual(m, prm, U, phit, zero_dirichlet=False)
    for k in range(2):
        assert abs(R[k * m.n_nodes:(k + 1) * m.n_nodes].sum()) <= 1e-14 * np.abs(R).sum()
    U = m.dirichlet_values(0.0)
    phi = np.ones(m.n_nodes)
    phi[m.slit_nodes()] = 0.0
    U[2 * m.n_nodes:] = phi
    for Uk, phit in zip(*S.load_steps(m, prm, U, [4e-3, 8e-3], return_phit=True)):
        top = fe.reaction_force(m, prm, Uk, phit)
        R = fe.residual(m, prm, Uk, phit, zero_dirichlet=False)
        bottom = R[m.dof(1, m.bottom_nodes())].sum()
        assert top > 0 and abs(top + bottom) <= 1e-10 * top


@pytest.mark.parametrize("dim,p,N", [(2, 1, 4), (2, 2, 3), (3, 2, 2)])
@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
@pytest.mark.parametrize("gamma", [2e-3, -2e-3])
def test_reaction_force_simple_shear(dim, p, N, split, gamma):
    """Shear test (Sec. 5.2) in closed form: u_x = gamma x_d (top face moved sideways by gamma), phi =
    phi~ = c: the strain has eigenvalues +-gamma/2 (and 0 in 3D) and no trace, so sigma_xd = mu gamma;
    without a split it is degraded by g(c), with the Miehe split only its tensile half is, which
    leaves (1 + g(c)) mu gamma / 2 on the unit top face in the x direction."""
    c = 0.7
    m = M.Mesh(dim, p, N)
    U = np.zeros(m.n_dofs)
    U[:m.n_nodes] = gamma * m.coords[:, dim - 1]
    U[dim * m.n_nodes:] = c
    F = fe.reaction_force(m, fe.Params(LAM, MU, GC, 0.2, KAPPA, split), U, np.full(m.n_nodes, c), comp=0)
    g = mat.g(c, KAPPA)
    expect = MU * gamma * (g if split == mat.SPLIT_NONE else 0.5 * (1.0 + g))
    assert abs(F - expect) <= 1e-13 * abs(expect)


@pytest.mark.parametrize("split", [mat.SPLIT_NONE, mat.SPLIT_MIEHE])
def test_shear_load_steps_balance(split):
    """Shear load steps of the notched specimen converge to states whose x reaction on the top face
    equals minus that on the bottom face and is positive for a rightward load."""
    from oracle import solvers as S
    m = M.Mesh(2, 1, 8)
    prm = fe.Params(LAM, MU, GC, 2.0 / 8, KAPPA, split)
    U = m.dirichlet_values(0.0, comp=0)
    phi = np.ones(m.n_nodes)
    phi[m.slit_nodes()] = 0.0
    U[2 * m.n_nodes:] = phi
    for Uk, phit in zip(*S.load_steps(m, prm, U, [4e-3, 8e-3], comp=0, return_phit=True)):
        assert np.all(Uk[m.dof(0, m.top_nodes())] == Uk[m.dof(0, m.top_nodes())][0])
        assert np.all(Uk[m.dof(1, m.top_nodes())] == 0.0)
        top = fe.reaction_force(m, prm, Uk, phit, comp=0)
        R = fe.residual(m, prm, Uk, phit, zero_dirichlet=False)
        bottom = R[m.dof(0, m.bottom_nodes())].sum()
        assert top > 0 and abs(top + bottom) <= 1e-10 * top
