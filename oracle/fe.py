"""Residual, Jacobian and energy of the phase-field fracture problem (oracle; test infrastructure only).

Everything is assembled cell by cell from full tensor-product shape-function tables
(N[q, a], grad N[q, a, :]) and quadrature loops; there is no sum factorisation.

Paper references:
* energy functional with the Miehe split, Sec. 2.1;
* residual R(u, phi)(w, psi), Eq. (residual): the u-equation uses g(phi~) with phi~ the
  extrapolated phase field, the phi-equation uses phi itself;
* Jacobian G, Eq. (G): derivative of R with phi~ frozen, which makes G block lower triangular
  (Sec. 3.3);
* matrix-free product G x = sum_k C^T P_k^T G_k P_k C x (Sec. 3.4): ``apply_ebe`` is that sum
  with explicit element matrices G_k.

Material parameters lambda, mu and G_c are either constants or nodal fields interpolated with the
Q_p basis (nodal fields are not in the paper; they are needed for parameter gradients).
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import material as mat
from .basis import gauss_legendre, gll_nodes, lagrange


@dataclass
class Params:
    lam: float = 121.15
    mu: float = 80.77
    gc: float = 2.7e-3
    eps: float = 2.0 / 32
    kappa: float = 1e-10
    split: int = mat.SPLIT_NONE


class Tables:
    """Shape-function tables of one (uniform, axis-aligned) cell of edge h."""

    def __init__(self, mesh):
        d, p, h = mesh.dim, mesh.p, mesh.h
        n = p + 1
        q, w = gauss_legendre(n)
        S, D = lagrange(gll_nodes(p), q)  # S[qi, k], D[qi, k] on the unit interval
        nq = na = n ** d
        qi = np.indices((n,) * d)[::-1].reshape(d, -1).T  # (nq, d), x fastest
        ai = qi.copy()
        N = np.ones((nq, na))
        dN = np.ones((nq, na, d))
        JxW = np.ones(nq) * h ** d
        for Q in range(nq):
            for t in range(d):
                JxW[Q] *= w[qi[Q, t]]
            for a in range(na):
                for t in range(d):
                    N[Q, a] *= S[qi[Q, t], ai[a, t]]
                    for j in range(d):
                        dN[Q, a, j] *= (D if j == t else S)[qi[Q, t], ai[a, t]]
        self.N, self.dN, self.JxW = N, dN / h, JxW
        self.nq, self.na, self.dim = nq, na, d


def _fields(mesh, prm, gc_field, lam_field, mu_field, cells, T):
    """Material parameters at the quadrature points of ``cells`` (constants or nodal fields)."""
    out = []
    for f, c in ((gc_field, prm.gc), (lam_field, prm.lam), (mu_field, prm.mu)):
        if f is None:
            out.append(np.full((len(cells), T.nq), float(c)))
        else:
            out.append(np.asarray(f)[mesh.cell_nodes[cells]] @ T.N.T)
    return out


def qp_state(mesh, U, phi_tilde, cells, T):
    """grad u, phi, grad phi and phi~ at the quadrature points of ``cells``."""
    d = mesh.dim
    nn = mesh.n_nodes
    cn = mesh.cell_nodes[cells]
    ue = np.stack([U[c * nn:(c + 1) * nn][cn] for c in range(d)], axis=1)  # (nc, d, na)
    pe = U[d * nn:(d + 1) * nn][cn]
    grad_u = np.einsum("cka,qaj->cqkj", ue, T.dN)
    phi = pe @ T.N.T
    grad_phi = np.einsum("ca,qaj->cqj", pe, T.dN)
    phit = np.asarray(phi_tilde)[cn] @ T.N.T
    return grad_u, phi, grad_phi, phit


def _chunks(n, size=2048):
    for s in range(0, n, size):
        yield np.arange(s, min(n, s + size))


def residual(mesh, prm, U, phi_tilde, gc_field=None, lam_field=None, mu_field=None,
             zero_dirichlet=True, cells=None):
    """R(U)(w, psi) of Eq. (residual) for every test basis function, as a global vector.

    u-rows:   int (g(phi~) sigma^+ + sigma^-) : e(w)
    phi-rows: int g'(phi) E_s^+ psi - (G_c/eps)(1 - phi) psi + G_c eps grad phi . grad psi
    Rows of Dirichlet DoFs are set to 0 when ``zero_dirichlet``. With ``cells`` only those cells are
    summed (exact at nodes all of whose cells are listed).
    """
    T = Tables(mesh)
    d, nn = mesh.dim, mesh.n_nodes
    R = np.zeros(mesh.n_dofs)
    all_cells = np.arange(mesh.n_cells) if cells is None else np.asarray(cells)
    for s in range(0, len(all_cells), 2048):
        cells = all_cells[s:s + 2048]
        grad_u, phi, grad_phi, phit = qp_state(mesh, U, phi_tilde, cells, T)
        gc, lam, mu = _fields(mesh, prm, gc_field, lam_field, mu_field, cells, T)
        e = mat.sym(grad_u)
        sp_, sm_, Esp, _ = mat.stress_energy(e, lam, mu, prm.split)
        tau = mat.g(phit, prm.kappa)[..., None, None] * sp_ + sm_
        ru = np.einsum("q,cqkj,qaj->cka", T.JxW, tau, T.dN)
        s = mat.dg(phi, prm.kappa) * Esp - gc / prm.eps * (1.0 - phi)
        r_phi = np.einsum("q,cq,qa->ca", T.JxW, s, T.N) + \
            np.einsum("q,cq,cqj,qaj->ca", T.JxW, gc * prm.eps, grad_phi, T.dN)
        cn = mesh.cell_nodes[cells]
        for k in range(d):
            np.add.at(R, k * nn + cn, ru[:, k, :])
        np.add.at(R, d * nn + cn, r_phi)
    if zero_dirichlet:
        R[mesh.dirichlet_mask()] = 0.0
    return R


def reaction_force(mesh, prm, U, phi_tilde, gc_field=None, lam_field=None, mu_field=None, comp=None):
    """Force on the loaded (top) face in the loading direction e_comp (comp = d-1, the default: the
    tension test of Sec. 5.1; comp = 0: the shear test of Sec. 5.2), the ordinate of the
    load-displacement curve: the u_comp-rows of the residual, Dirichlet rows kept, summed over the
    top-face nodes. That sum is the u-equation tested with w = e_comp times the sum of the top-face
    basis functions, i.e. the work of the stress g(phi~) sigma^+ + sigma^- on the field that moves the
    top face by a unit amount in the loading direction (the consistent nodal reaction; for a
    homogeneous stress it equals the face integral of sigma_{comp,d})."""
    R = residual(mesh, prm, U, phi_tilde, gc_field, lam_field, mu_field, zero_dirichlet=False)
    return float(R[mesh.dof(mesh.dim - 1 if comp is None else comp, mesh.top_nodes())].sum())


def energy(mesh, prm, U, gc_field=None, lam_field=None, mu_field=None):
    """Discrete energy of Sec. 2.1 with the split, evaluated by the same Gauss rule:
    int g(phi) E_s^+ + E_s^- + G_c/2 ((1 - phi)^2/eps + eps |grad phi|^2)."""
    T = Tables(mesh)
    total = 0.0
    phi_nodes = U[mesh.dim * mesh.n_nodes:]
    for cells in _chunks(mesh.n_cells):
        grad_u, phi, grad_phi, _ = qp_state(mesh, U, phi_nodes, cells, T)
        gc, lam, mu = _fields(mesh, prm, gc_field, lam_field, mu_field, cells, T)
        e = mat.sym(grad_u)
        _, _, Esp, Es = mat.stress_energy(e, lam, mu, prm.split)
        dens = mat.g(phi, prm.kappa) * Esp + (Es - Esp) + \
            0.5 * gc * ((1.0 - phi) ** 2 / prm.eps + prm.eps * np.einsum("cqj,cqj->cq", grad_phi, grad_phi))
        total += float(np.einsum("q,cq->", T.JxW, dens))
    return total


MODE_FULL, MODE_BLOCKDIAG, MODE_TRANSPOSE = 0, 1, 2


def element_matrices(mesh, prm, U, phi_tilde, cells, T, gc_field=None, lam_field=None, mu_field=None,
                     mode=MODE_FULL):
    """Element matrices G_k of Eq. (G) for ``cells``: (nc, nloc, nloc), local order component-major.

    u-u block:   int (g(phi~) dsigma^+[e(du)] + dsigma^-[e(du)]) : e(w)
    phi-u block: int g'(phi) sigma^+ : e(du) psi          (dropped in block-diagonal mode)
    phi-phi:     int (g''(phi) E_s^+ + G_c/eps) dphi psi + G_c eps grad dphi . grad psi
    u-phi block: 0 (phi~ is frozen).
    """
    d, na = mesh.dim, T.na
    grad_u, phi, grad_phi, phit = qp_state(mesh, U, phi_tilde, cells, T)
    gc, lam, mu = _fields(mesh, prm, gc_field, lam_field, mu_field, cells, T)
    e = mat.sym(grad_u)
    sp_, _, Esp, _ = mat.stress_energy(e, lam, mu, prm.split)
    T4 = mat.tangent4(e, lam, mu, mat.g(phit, prm.kappa), prm.split)
    nc = len(cells)
    K = np.zeros((nc, (d + 1) * na, (d + 1) * na))
    Kuu = np.einsum("q,qaj,cqkjlm,qbm->ckalb", T.JxW, T.dN, T4, T.dN).reshape(nc, d * na, d * na)
    K[:, :d * na, :d * na] = Kuu
    if mode != MODE_BLOCKDIAG:
        b = mat.dg(phi, prm.kappa)[..., None, None] * sp_
        Kpu = np.einsum("q,qa,cqlm,qbm->calb", T.JxW, T.N, b, T.dN).reshape(nc, na, d * na)
        K[:, d * na:, :d * na] = Kpu
    c = mat.ddg(phi, prm.kappa) * Esp + gc / prm.eps
    Kpp = np.einsum("q,cq,qa,qb->cab", T.JxW, c, T.N, T.N) + \
        np.einsum("q,cq,qaj,qbj->cab", T.JxW, gc * prm.eps, T.dN, T.dN)
    K[:, d * na:, d * na:] = Kpp
    if mode == MODE_TRANSPOSE:
        K = np.swapaxes(K, 1, 2)
    return K


def assemble(mesh, prm, U, phi_tilde, mode=MODE_FULL, **fields):
    """Sparse global Jacobian (CSR), unmasked: the sum over cells of P_k^T G_k P_k."""
    T = Tables(mesh)
    dofs = mesh.cell_dofs()
    rows, cols, vals = [], [], []
    for cells in _chunks(mesh.n_cells, 512):
        K = element_matrices(mesh, prm, U, phi_tilde, cells, T, mode=mode, **fields)
        cd = dofs[cells]
        rows.append(np.repeat(cd, cd.shape[1], axis=1).ravel())
        cols.append(np.tile(cd, (1, cd.shape[1])).ravel())
        vals.append(K.ravel())
    G = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.n_dofs, mesh.n_dofs))
    return G.tocsr()


def apply_ebe(mesh, prm, U, phi_tilde, x, mode=MODE_FULL, cells=None, **fields):
    """Unmasked G x as the element-by-element sum of Sec. 3.4 (no global matrix)."""
    T = Tables(mesh)
    dofs = mesh.cell_dofs()
    y = np.zeros(mesh.n_dofs)
    all_cells = np.arange(mesh.n_cells) if cells is None else np.asarray(cells)
    for s in range(0, len(all_cells), 512):
        cc = all_cells[s:s + 512]
        K = element_matrices(mesh, prm, U, phi_tilde, cc, T, mode=mode, **fields)
        cd = dofs[cc]
        np.add.at(y, cd, np.einsum("cij,cj->ci", K, x[cd]))
    return y


def masked(G, mask):
    """Operator with the rows and columns of ``mask`` replaced by the identity:
    Z G Z + (I - Z), Z = diag(1 - mask). This is how constrained rows (Dirichlet DoFs,
    C in Sec. 3.4) and the active set (Alg. 1: d phi = 0 on A) enter the linear solve."""
    z = sp.diags((~mask).astype(np.float64))
    return (z @ G @ z + sp.diags(mask.astype(np.float64))).tocsr()


def apply_masked(G, mask, x):
    xz = np.where(mask, 0.0, x)
    y = G @ xz
    return np.where(mask, x, y)


def lumped_mass(mesh):
    """Diagonal of the lumped phase-field mass: m_i = int psi_i (one value per node)."""
    T = Tables(mesh)
    m = np.zeros(mesh.n_nodes)
    np.add.at(m, mesh.cell_nodes, np.broadcast_to(T.JxW @ T.N, mesh.cell_nodes.shape))
    return m


def param_grad(mesh, prm, U, phi_tilde, v, gc_field=None, lam_field=None, mu_field=None):
    """(dR/dG_c)^T v, (dR/dlambda)^T v, (dR/dmu)^T v for nodal fields, each one value per node.

    R is linear in (lambda, mu) at fixed strain and affine in G_c, so the partial derivative of
    each pointwise term is that term evaluated with unit parameters; v is a test vector in the
    layout of U (Dirichlet rows of v should be 0 when R has its Dirichlet rows zeroed).
    """
    T = Tables(mesh)
    d, nn = mesh.dim, mesh.n_nodes
    out = np.zeros((3, nn))
    for cells in _chunks(mesh.n_cells):
        grad_u, phi, grad_phi, phit = qp_state(mesh, U, phi_tilde, cells, T)
        gv, vphi, grad_vphi, _ = qp_state(mesh, v, phi_tilde, cells, T)
        e = mat.sym(grad_u)
        gt = mat.g(phit, prm.kappa)[..., None, None]
        dg_ = mat.dg(phi, prm.kappa)
        # G_c: -(1/eps)(1 - phi) psi + eps grad phi . grad psi
        s_gc = -(1.0 - phi) / prm.eps * vphi + prm.eps * np.einsum("cqj,cqj->cq", grad_phi, grad_vphi)
        terms = [s_gc]
        for lam_u, mu_u in ((1.0, 0.0), (0.0, 1.0)):
            sp_, sm_, Esp, _ = mat.stress_energy(e, lam_u, mu_u, prm.split)
            tau = gt * sp_ + sm_
            terms.append(np.einsum("cqkj,cqkj->cq", tau, gv) + dg_ * Esp * vphi)
        cn = mesh.cell_nodes[cells]
        for t, s in enumerate(terms):
            np.add.at(out[t], cn, np.einsum("q,cq,qa->ca", T.JxW, s, T.N))
    return out[0], out[1], out[2]
