"""Matched problems for the parity tests: one synthetic state, fed identically to the oracle
and to the CUDA library. The state is built with the oracle's mesh (Dirichlet lift, slit), from
the seeded generators of paper_2005_00331_gb300.inputs."""
import numpy as np

from oracle import fe, mesh as M
from paper_2005_00331_gb300 import inputs

LAM, MU, GC, KAPPA = 121.15, 80.77, 2.7e-3, 1e-10


class Problem:
    def __init__(self, dim, p, N, split=0, seed=0, load=1e-3, u_std=1e-3, active_frac=0.0, fields=False,
                 eps=None, zero_u=False):
        self.dim, self.p, self.N, self.split = dim, p, N, split
        m = M.Mesh(dim, p, N)
        self.mesh = m
        nn = m.n_nodes
        self.eps = eps if eps is not None else 2.0 / N
        self.prm = fe.Params(LAM, MU, GC, self.eps, KAPPA, split)
        U = m.dirichlet_values(load)
        if not zero_u:
            noise = inputs.displacement_noise(nn, dim, seed, std=u_std)
            dmask = m.dirichlet_mask()[:dim * nn]
            U[:dim * nn] += np.where(dmask, 0.0, noise)
        phi = inputs.uniform_phase(nn, seed)
        phi[m.slit_nodes()] = 0.0
        U[dim * nn:] = phi
        self.U = U
        self.phi_old = np.minimum(1.0, phi + np.abs(inputs.normal_vector(nn, seed, 7)) * 1e-3)
        self.phi_tilde = np.clip(phi + 0.01 * inputs.normal_vector(nn, seed, 8), 0.0, 1.0)
        act = np.zeros(nn, dtype=bool)
        if active_frac > 0:
            act = inputs.uniform_phase(nn, seed + 100, 0.0, 1.0) < active_frac
        self.active = act
        self.mask = m.dirichlet_mask()
        self.mask[dim * nn:] |= act
        self.fields = {}
        if fields:
            self.fields = dict(gc_field=inputs.lognormal_field(nn, seed),
                               lam_field=LAM * (1 + 0.1 * inputs.normal_vector(nn, seed, 9)),
                               mu_field=MU * (1 + 0.1 * inputs.normal_vector(nn, seed, 10)))

    # ---- oracle side -----------------------------------------------------------------------
    def G(self, mode=fe.MODE_FULL):
        return fe.assemble(self.mesh, self.prm, self.U, self.phi_tilde, mode=mode, **self.fields)

    def residual(self):
        return fe.residual(self.mesh, self.prm, self.U, self.phi_tilde, **self.fields)

    # ---- GPU side --------------------------------------------------------------------------
    def context(self, mg_precision=64, **kw):
        import torch
        from paper_2005_00331_gb300 import setup_mesh
        ctx = setup_mesh(dim=self.dim, degree=self.p, n_cells_1d=self.N, split=self.split, eps=self.eps,
                         mg_precision=mg_precision, **kw)
        dev = torch.device("cuda")
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        f = self.fields
        ctx.set_state(t(self.U), t(self.phi_old), t(self.phi_tilde), t(self.active.astype(np.uint8)),
                      t(f["gc_field"]) if f else None, t(f["lam_field"]) if f else None,
                      t(f["mu_field"]) if f else None)
        return ctx
