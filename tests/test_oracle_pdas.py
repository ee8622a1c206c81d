"""Pins of the oracle's primal-dual active-set loop (Alg. 1) and of its load stepping (Sec. 3.2, 5.1)
against what the mathematics fixes, not against the oracle itself.

* With split none, u = 0 and no load, E_s^+ = 0 and the phase-field equation is the linear obstacle
  problem  min 1/2 phi^T A phi - b^T phi  s.t.  phi <= psi,  A = G_c (M / eps + eps K),  b = (G_c / eps) M 1.
  On a uniform Q1 mesh with eps = 2h every off-diagonal entry of A is <= 0, so A is a Stieltjes matrix.
  For such A the primal-dual active-set iteration (Hintermueller, Ito, Kunisch, SIAM J. Optim. 13, 2002)
  has, whatever the start: phi_{k+1} <= phi_k from the second iterate on, phi_k feasible from the second
  iterate on, nested active sets from the third on, and it stops at the unique KKT point. Derivation, with
  d = phi_{k+1} - phi_k and I, A the new inactive and active sets: on A, d = 0 (node stayed) or
  d = psi - phi_k < 0 (violated node entered); on I, (A d)_I = m lambda_k <= 0, and A_II^{-1} >= 0,
  A_IA <= 0 give d_I <= 0.
* Brute force: on a 3 x 3 Q1 mesh every one of the 2^16 active sets is tried; exactly one satisfies the
  KKT conditions, and it is the set the loop stops on.
* Load steps: every step converges, and the converged state solves the discrete variational inequality
  of Problem (Euler-Lagrange) (block-triangular, each block strictly convex, so the KKT point is unique):
  R_u = 0 on free rows, phi <= phi_old, R_phi = 0 where phi < phi_old, -R_phi / m >= 0 where phi = phi_old.
  The two cases (2D Q2 8^2, 3D Q1 4^3, Miehe split) are ones whose second step did not converge within 30
  iterations when phi~ was extrapolated from the initial phase field.
"""
import numpy as np
import pytest

from oracle import fe, material as mat, mesh as M, solvers as S

LAM, MU, GC, KAPPA = 121.15, 80.77, 2.7e-3, 1e-10


def _obstacle(N, amp, width):
    """Q1 mesh, split none, u = 0, obstacle psi = 1 - amp * exp(-|x - c|^2 / width) below the
    unconstrained minimiser phi = 1."""
    m = M.Mesh(2, 1, N)
    prm = fe.Params(LAM, MU, GC, 2.0 / N, KAPPA, mat.SPLIT_NONE)
    x, y = m.coords[:, 0], m.coords[:, 1]
    psi = 1.0 - amp * np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / width)
    return m, prm, psi


def _run_pdas(m, prm, psi, phi0, max_iters=60):
    nn = m.n_nodes
    U = m.dirichlet_values(0.0)
    U[2 * nn:] = phi0
    phis, acts = [], []
    for k in range(max_iters):
        U, act, _, _ = S.pdas_step(m, prm, U, psi, psi)
        assert np.all(U[:2 * nn] == 0.0)           # no load, no strain: u stays 0
        phis.append(U[2 * nn:].copy())
        acts.append(act)
        if k > 0 and np.array_equal(acts[-1], acts[-2]):
            return phis, acts
    raise AssertionError("no termination within %d iterations" % max_iters)


def _lcp_data(m, prm, psi):
    nn = m.n_nodes
    U0 = np.zeros(3 * nn)
    A = fe.assemble(m, prm, U0, psi)[2 * nn:, 2 * nn:].toarray()
    b = -fe.residual(m, prm, U0, psi)[2 * nn:]    # R_phi(phi = 0) = -b
    return A, b, fe.lumped_mass(m)


@pytest.mark.parametrize("amp,width,shift", [(0.3, 0.05, 0.1), (0.5, 0.1, 0.3)])
def test_stieltjes_obstacle_monotone_and_finite(amp, width, shift):
    m, prm, psi = _obstacle(16, amp, width)
    A, b, mass = _lcp_data(m, prm, psi)
    off = A - np.diag(np.diag(A))
    assert off.max() <= 0.0 and np.all(np.linalg.eigvalsh(A) > 0)   # the theorem's premise
    phis, acts = _run_pdas(m, prm, psi, psi - shift)                 # feasible start far below psi
    assert len(phis) <= m.n_nodes + 2
    tol = 1e-14
    for k in range(1, len(phis)):
        assert np.all(phis[k] <= phis[k - 1] + tol)                  # monotone from the 2nd iterate
        assert np.all(phis[k] <= psi + tol)                          # feasible from the 2nd iterate
    for k in range(2, len(acts) - 1):
        assert not np.any(acts[k + 1] & ~acts[k])                    # nested from the 3rd set
    # the start overshoots (the first solve ignores the obstacle almost everywhere), so the loop has
    # work to do: the second active set is larger than the final one
    assert acts[1].sum() > acts[-1].sum() > 0
    # the limit is the KKT point
    phi = phis[-1]
    lam = -(A @ phi - b) / mass
    act = acts[-1]
    assert np.all(phi[act] == psi[act]) and np.all(lam[act] > 0)
    assert np.abs(lam[~act]).max() <= 1e-10 * np.abs(lam).max()


def test_obstacle_brute_force_unique_kkt_point():
    m, prm, psi = _obstacle(3, 0.5, 0.1)
    nn = m.n_nodes
    A, b, mass = _lcp_data(m, prm, psi)
    kkt_sets = []
    for code in range(1 << nn):
        act = ((code >> np.arange(nn)) & 1).astype(bool)
        ina = ~act
        phi = psi.copy()
        if ina.any():
            phi[ina] = np.linalg.solve(A[np.ix_(ina, ina)], b[ina] - A[np.ix_(ina, act)] @ psi[act])
        if np.any(phi > psi + 1e-13):
            continue
        if np.all(-(A @ phi - b)[act] / mass[act] >= -1e-13):
            kkt_sets.append((act, phi))
    assert len(kkt_sets) == 1
    act_bf, phi_bf = kkt_sets[0]
    assert 0 < act_bf.sum() < nn
    phis, acts = _run_pdas(m, prm, psi, psi - 0.3)
    np.testing.assert_array_equal(acts[-1], act_bf)
    assert np.abs(phis[-1] - phi_bf).max() <= 1e-13


def _kkt(m, prm, U, phi_old, phit):
    d, nn = m.dim, m.n_nodes
    R = fe.residual(m, prm, U, phit)
    Rfull = fe.residual(m, prm, U, phit, zero_dirichlet=False)
    phi = U[d * nn:]
    lam = -R[d * nn:] / fe.lumped_mass(m)
    on = phi == phi_old
    return dict(ru=np.abs(R[:d * nn]).max() / np.abs(Rfull[:d * nn]).max(),
                violation=(phi - phi_old).max(),
                lam_active_min=lam[on].min() / np.abs(lam).max(),
                r_inactive=np.abs(lam[~on]).max() / np.abs(lam).max(),
                n_active=int(on.sum()))


@pytest.mark.parametrize("dim,p,N", [(2, 2, 8), (3, 1, 4)])
def test_load_steps_converge_to_kkt_points(dim, p, N):
    m = M.Mesh(dim, p, N)
    prm = fe.Params(LAM, MU, GC, 2.0 / N, KAPPA, mat.SPLIT_MIEHE)
    U = m.dirichlet_values(0.0)
    phi0 = np.ones(m.n_nodes)
    phi0[m.slit_nodes()] = 0.0
    U[dim * m.n_nodes:] = phi0
    stats = []
    out, phits = S.load_steps(m, prm, U, [1e-4, 2e-4, 3e-4], return_phit=True, stats=stats)
    assert all(conv for _, conv in stats) and max(it for it, _ in stats) <= 12
    prev = phi0
    for Uk, pt in zip(out, phits):
        k = _kkt(m, prm, Uk, prev, pt)
        assert k["ru"] <= 1e-12 and k["violation"] <= 0.0
        assert k["lam_active_min"] > 0 and k["r_inactive"] <= 1e-12 and k["n_active"] > 0
        prev = Uk[dim * m.n_nodes:]


def test_extrapolation_from_solved_steps_only():
    """phi~ of the first two load steps is the last solved phase field (the initial one for the first),
    from the third on clamp(2 phi^{n-1} - phi^{n-2}, 0, 1) of the last two solved steps."""
    m = M.Mesh(2, 1, 4)
    prm = fe.Params(LAM, MU, GC, 0.5, KAPPA, mat.SPLIT_MIEHE)
    U = m.dirichlet_values(0.0)
    phi0 = np.ones(m.n_nodes)
    phi0[m.slit_nodes()] = 0.0
    U[2 * m.n_nodes:] = phi0
    out, phits = S.load_steps(m, prm, U, [1e-3, 2e-3, 3e-3, 4e-3], return_phit=True)
    sol = [Uk[2 * m.n_nodes:] for Uk in out]
    np.testing.assert_array_equal(phits[0], phi0)
    np.testing.assert_array_equal(phits[1], sol[0])
    np.testing.assert_array_equal(phits[2], np.clip(2 * sol[1] - sol[0], 0, 1))
    np.testing.assert_array_equal(phits[3], np.clip(2 * sol[2] - sol[1], 0, 1))
