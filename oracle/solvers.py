"""Active set, transfers, smoothers and Krylov solvers (oracle; test infrastructure only).

Paper references:
* Alg. 1 (primal-dual active set): A_k = {i ~ phi : (M^{-1} R_k)_i + c (U_k - U_old)_i > 0},
  d phi = 0 on A_k, Newton step on the complement. Reading of the garbled signs: R_k in Alg. 1
  is the right-hand side r = -R of Eq. (residual), so the step solves G dU = -R, and M is the
  lumped phase-field mass. On entering A a DoF is reset to phi_old (feasibility).
* Sec. 3.3: monolithic geometric multigrid GMG(G) whose smoother is block diagonal,
  S = diag(S(G_uu), S(G_phiphi)), each block a Chebyshev-Jacobi smoother on
  [c lambda_max, C lambda_max] with c = 0.24, C = 1.2; lambda_max estimated with CG; GMRES
  outside (here the flexible variant, because the preconditioner may vary).
* Nested spaces (Sec. 3.3): the coarse Q_p space is a subspace of the fine one, so the
  prolongation is the interpolation of the coarse function at the fine nodes and the
  restriction is its transpose.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe
from .basis import gll_nodes, lagrange
from .mesh import Mesh, level_sizes

MASK64 = (1 << 64) - 1


# --- counter-based start vectors ------------------------------------------------------------
def splitmix64(seed, i):
    """SplitMix64 (Steele, Lea, Flood 2014) output for counter i: a 64-bit integer."""
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def start_vector(n, seed):
    """Entries (z >> 11) * 2^-53 - 1/2 of SplitMix64, a deterministic vector in [-1/2, 1/2)."""
    return np.array([(splitmix64(seed, i) >> 11) * 2.0 ** -53 - 0.5 for i in range(n)])


# --- Alg. 1 -------------------------------------------------------------------------------
def active_set(mesh, R, phi, phi_old, c=1.0):
    """Boolean per node: (M_L^{-1} r)_i + c (phi_i - phi_old_i) > 0 with r = -R_phi."""
    m = fe.lumped_mass(mesh)
    r_phi = -R[mesh.dim * mesh.n_nodes:]
    return r_phi / m + c * (phi - phi_old) > 0.0


def newton_mask(mesh, active):
    mask = mesh.dirichlet_mask()
    mask[mesh.dim * mesh.n_nodes:] |= active
    return mask


# --- transfers between nested meshes -------------------------------------------------------
def _prolong_1d(Nc, Nf, p):
    """Fine nodes x coarse nodes: coarse 1D basis evaluated at the fine node coordinates."""
    mc, mf = Mesh(2, p, Nc), Mesh(2, p, Nf)
    xi = gll_nodes(p)
    P = np.zeros((mf.n1, mc.n1))
    H = 1.0 / Nc
    for i, x in enumerate(mf.x1):
        c = min(int(np.floor(x / H + 1e-12)), Nc - 1)
        L, _ = lagrange(xi, [(x - c * H) / H])
        P[i, c * p:c * p + p + 1] = L[0]
    P[np.abs(P) < 1e-15] = 0.0
    return P


def _interp_1d(Nf, Nc, p):
    """Coarse nodes x fine nodes: the fine 1D basis evaluated at the coarse node coordinates."""
    mc, mf = Mesh(2, p, Nc), Mesh(2, p, Nf)
    xi = gll_nodes(p)
    T = np.zeros((mc.n1, mf.n1))
    h = 1.0 / Nf
    for j, x in enumerate(mc.x1):
        c = min(int(np.floor(x / h + 1e-12)), Nf - 1)
        L, _ = lagrange(xi, [(x - c * h) / h])
        T[j, c * p:c * p + p + 1] = L[0]
    T[np.abs(T) < 1e-15] = 0.0
    return T


def _kron_dim(A, dim):
    M = sp.csr_matrix(A)
    out = M
    for _ in range(dim - 1):
        out = sp.kron(M, out, format="csr")  # node index x fastest: kron(P_z, P_y, P_x)
    return out


def prolongation(dim, p, Nc, Nf):
    """Scalar prolongation matrix (fine nodes x coarse nodes)."""
    return _kron_dim(_prolong_1d(Nc, Nf, p), dim)


def state_interpolation(dim, p, Nf, Nc):
    """Scalar fine-to-coarse interpolation (coarse nodes x fine nodes): evaluates the fine FE
    function at the coarse nodes (used to carry the state to coarse levels)."""
    return _kron_dim(_interp_1d(Nf, Nc, p), dim)


def colocated_1d(Nc, Nf, p):
    """For every coarse 1D node the fine 1D node at the same coordinate, or -1."""
    mc, mf = Mesh(2, p, Nc), Mesh(2, p, Nf)
    out = -np.ones(mc.n1, dtype=np.int64)
    for j, x in enumerate(mc.x1):
        k = np.nonzero(np.abs(mf.x1 - x) <= 1e-12)[0]
        if len(k):
            out[j] = k[0]
    return out


# --- Chebyshev-Jacobi and eigenvalue estimate ---------------------------------------------
def chebyshev(apply_A, dinv, f, degree, lam_max, lo=0.24, hi=1.2, x0=None):
    """Chebyshev iteration of the given degree for A x = f, Jacobi-preconditioned, on the
    interval [lo lam_max, hi lam_max] (Saad, Iterative Methods, Chebyshev acceleration)."""
    a, b = lo * lam_max, hi * lam_max
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    sigma = theta / delta
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = dinv * (f - apply_A(x)) if x0 is not None else dinv * f
    rho = 1.0 / sigma
    d = r / theta
    for k in range(1, degree + 1):
        x = x + d
        if k == degree:
            break
        r = dinv * (f - apply_A(x))
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return x


def cg_lanczos(apply_A, dinv, b, iters):
    """Jacobi-preconditioned CG from b; returns the eigenvalues of the Lanczos tridiagonal
    built from the CG coefficients (estimates of the spectrum of D^{-1} A)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = dinv * r
    pvec = z.copy()
    rz = r @ z
    alphas, betas = [], []
    for _ in range(iters):
        Ap = apply_A(pvec)
        pAp = pvec @ Ap
        if pAp <= 0 or rz <= 0:
            break
        alpha = rz / pAp
        x += alpha * pvec
        r -= alpha * Ap
        z = dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        rz = rz_new
        if rz <= 0:
            break
        pvec = z + beta * pvec
    k = len(alphas)
    Tm = np.zeros((k, k))
    for j in range(k):
        Tm[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            Tm[j, j + 1] = Tm[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return np.linalg.eigvalsh(Tm)


# --- multigrid -----------------------------------------------------------------------------
class Level:
    pass


def build_levels(dim, p, N, prm, U, phi_tilde, active, cheb_degree=5, eig_iters=15, eig_seed=0,
                 coarse_min=3, **fields):
    """Meshes, rediscretised masked operators, diagonals and smoother intervals of every level.

    The state (U, phi~, nodal fields) is carried to coarse levels by evaluating the fine FE
    function at the coarse nodes; a coarse phase-field DoF is active iff the fine DoF at the
    same point is active (the paper is silent on level operators of the masked problem).
    """
    sizes = level_sizes(N, coarse_min)
    levels = []
    Uc, ptc, act = U, phi_tilde, active
    fc = dict(fields)
    for li, n in enumerate(sizes):
        L = Level()
        L.mesh = Mesh(dim, p, n)
        m = L.mesh
        if li > 0:
            Nf = sizes[li - 1]
            Ts = state_interpolation(dim, p, Nf, n)
            nnf = levels[-1].mesh.n_nodes
            Uc = np.concatenate([Ts @ Uc[c * nnf:(c + 1) * nnf] for c in range(dim + 1)])
            ptc = Ts @ ptc
            fc = {k: (None if v is None else Ts @ v) for k, v in fc.items()}
            co = colocated_1d(n, Nf, p)
            idx = np.indices((m.n1,) * dim)[::-1].reshape(dim, -1).T
            fine_1d = co[idx]
            ok = np.all(fine_1d >= 0, axis=1)
            strides = levels[-1].mesh.n1 ** np.arange(dim)
            fine_node = (fine_1d * strides).sum(axis=1)
            act = np.zeros(m.n_nodes, dtype=bool)
            act[ok] = levels[-1].active[fine_node[ok]]
            L.P = prolongation(dim, p, n, Nf)
        L.U, L.phi_tilde, L.active, L.fields = Uc, ptc, act, fc
        L.mask = newton_mask(m, act)
        G = fe.assemble(m, prm, Uc, ptc, mode=fe.MODE_FULL, **fc)
        L.G = fe.masked(G, L.mask)
        L.diag = L.G.diagonal()
        nu = dim * m.n_nodes
        L.nu = nu
        L.Guu = L.G[:nu, :nu]
        L.Gpp = L.G[nu:, nu:]
        L.lam_max = []
        for Gb, db, sl in ((L.Guu, L.diag[:nu], slice(0, nu)), (L.Gpp, L.diag[nu:], slice(nu, None))):
            b0 = start_vector(m.n_dofs, eig_seed)[sl]
            b0 = np.where(L.mask[sl], 0.0, b0)
            ev = cg_lanczos(lambda v, Gb=Gb: Gb @ v, 1.0 / db, b0, eig_iters)
            L.lam_max.append(float(ev.max()))
        L.cheb_degree = cheb_degree
        levels.append(L)
    return levels


def smooth(L, f):
    nu = L.nu
    xu = chebyshev(lambda v: L.Guu @ v, 1.0 / L.diag[:nu], f[:nu], L.cheb_degree, L.lam_max[0])
    xp = chebyshev(lambda v: L.Gpp @ v, 1.0 / L.diag[nu:], f[nu:], L.cheb_degree, L.lam_max[1])
    return np.concatenate([xu, xp])


def _prolong_vec(L, Lc, ec):
    """Fine-level vector P ec; Lc.P maps the coarse level Lc to its parent L."""
    nnc = Lc.mesh.n_nodes
    return np.concatenate([Lc.P @ ec[c * nnc:(c + 1) * nnc] for c in range(L.mesh.dim + 1)])


def _restrict_vec(L, Lc, r):
    """Coarse-level vector P^T r."""
    nn = L.mesh.n_nodes
    return np.concatenate([Lc.P.T @ r[c * nn:(c + 1) * nn] for c in range(L.mesh.dim + 1)])


def vcycle(levels, r, li=0):
    """One V-cycle of GMG(G) with the block-diagonal smoother; exact coarse solve."""
    L = levels[li]
    if li == len(levels) - 1:
        return spla.spsolve(L.G.tocsc(), r)
    Lc = levels[li + 1]
    e = smooth(L, r)
    res = r - L.G @ e
    rc = _restrict_vec(L, Lc, res)
    rc[Lc.mask] = 0.0
    ec = vcycle(levels, rc, li + 1)
    pe = _prolong_vec(L, Lc, ec)
    pe[L.mask] = 0.0
    e = e + pe
    res = r - L.G @ e
    return e + smooth(L, res)


def fgmres(apply_A, b, precond, tol=1e-6, restart=50, maxiter=1000, x0=None):
    """Right-preconditioned flexible GMRES(restart) with classical Gram-Schmidt applied twice.
    Stops when ||b - A x|| <= tol ||b - A x0||. Returns (x, iterations, final relative residual)."""
    n = len(b)
    x = np.zeros(n) if x0 is None else x0.copy()
    r = b - apply_A(x)
    r0 = np.linalg.norm(r)
    if r0 == 0.0:
        return x, 0, 0.0
    its = 0
    rel = 1.0
    while its < maxiter:
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        gvec = np.zeros(restart + 1)
        gvec[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            Z[j] = precond(V[j])
            w = apply_A(Z[j])
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            H[:j + 1, j] = h + h2
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            k = j + 1
            its += 1
            rel = abs(gvec[j + 1]) / r0
            if rel <= tol or its >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), gvec[:k])
        x = x + Z[:k].T @ y
        r = b - apply_A(x)
        rel = np.linalg.norm(r) / r0
        if rel <= tol:
            break
    return x, its, rel


def pdas_step(mesh, prm, U, phi_old, phi_tilde, c=1.0, solve="direct", levels_kw=None, **fields):
    """One iteration of Alg. 1. Returns (U_new, active, ||R~||, info).

    R~ is the residual with Dirichlet and active rows removed, evaluated at the projected state
    (phi reset to phi_old on the active set) before the Newton update.
    """
    d, nn = mesh.dim, mesh.n_nodes
    U = U.copy()
    R = fe.residual(mesh, prm, U, phi_tilde, **fields)
    act = active_set(mesh, R, U[d * nn:], phi_old, c)
    U[d * nn:][act] = phi_old[act]
    R = fe.residual(mesh, prm, U, phi_tilde, **fields)
    mask = newton_mask(mesh, act)
    rhs = np.where(mask, 0.0, -R)
    G = fe.masked(fe.assemble(mesh, prm, U, phi_tilde, **fields), mask)
    info = {}
    if solve == "direct":
        dU = spla.spsolve(G.tocsc(), rhs)
    else:
        levels = build_levels(mesh.dim, mesh.p, mesh.N, prm, U, phi_tilde, act, **(levels_kw or {}),
                              **fields)
        dU, its, rel = fgmres(lambda v: G @ v, rhs, lambda v: vcycle(levels, v), tol=1e-6)
        info.update(gmres_iters=its, gmres_rel=rel)
    return U + dU, act, float(np.linalg.norm(rhs)), info


def load_steps(mesh, prm, U, loads, max_iters=30, rtol=1e-8, comp=None, return_phit=False, stats=None,
               **fields):
    """Quasi-static loading of the tension test (Sec. 5.1; comp = 0: of the shear test, Sec. 5.2, whose
    top face moves to the right). For each load: u_comp := load on the top face (comp = d-1 by
    default); phi_old := the phase field of the last solved load step (the phase field of ``U`` before
    the first); phi~ := clamp(2 phi^{n-1} - phi^{n-2}, 0, 1), the linear extrapolation of Sec. 3.2 from
    the solutions of the previous two load steps (dt = 1), or phi^{n-1} while fewer than two load steps
    have been solved: the initial phase field is not the solution of a load step, and extrapolating from
    it doubles the diffuse profile the first step forms around the slit. Then Alg. 1 is repeated until
    the active set is unchanged and ||R~|| <= rtol ||R~_0||. Returns the states (and, with return_phit,
    the phi~ each step solved with, which the u-equation of its residual uses); ``stats``, if a list,
    receives (iterations, converged) per step. A step that does not converge still becomes the
    previous step of the next one."""
    d, nn = mesh.dim, mesh.n_nodes
    U = U.copy()
    solved = []               # phase fields of the solved load steps, the last two kept
    start = U[d * nn:].copy()
    out, phits = [], []
    for load in loads:
        U[mesh.dof(d - 1 if comp is None else comp, mesh.top_nodes())] = load
        prev_phi = solved[-1] if solved else start
        phi_old = prev_phi.copy()
        phit = prev_phi.copy() if len(solved) < 2 else np.clip(2.0 * solved[-1] - solved[-2], 0.0, 1.0)
        norms, prev, conv = [], None, False
        for _ in range(max_iters):
            U, act, rn, _ = pdas_step(mesh, prm, U, phi_old, phit, **fields)
            norms.append(rn)
            if prev is not None and np.array_equal(prev, act) and rn <= rtol * norms[0]:
                conv = True
                break
            prev = act
        if stats is not None:
            stats.append((len(norms), conv))
        solved = (solved + [U[d * nn:].copy()])[-2:]
        out.append(U.copy())
        phits.append(phit)
    return (out, phits) if return_phit else out
