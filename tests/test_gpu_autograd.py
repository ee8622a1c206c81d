"""The residual under torch.autograd with the hand-written adjoint (transpose Jacobian apply and
parameter gradients), checked against central finite differences and against the oracle's
gradient (config: 2D Q2, lognormal nodal G_c field, FP64)."""
import numpy as np
import pytest

from oracle import fe
from problems import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("split", [0, 1])
def test_autograd_residual(split):
    from paper_2005_00331_gb300 import ResidualFunction
    pr = Problem(2, 2, 8, split=split, seed=21, fields=True)
    ctx = pr.context()
    U = cuda(pr.U).requires_grad_(True)
    gc = cuda(pr.fields["gc_field"]).requires_grad_(True)
    lam = cuda(pr.fields["lam_field"]).requires_grad_(True)
    mu = cuda(pr.fields["mu_field"]).requires_grad_(True)
    po, pt = cuda(pr.phi_old), cuda(pr.phi_tilde)
    w = cuda(np.random.default_rng(1).normal(size=pr.mesh.n_dofs))
    R = ResidualFunction.apply(ctx, U, po, pt, gc, lam, mu)
    loss = (R * w).sum()
    loss.backward()
    # oracle gradient: G^T (w with Dirichlet rows removed) and the parameter gradients
    wm = np.where(pr.mesh.dirichlet_mask(), 0.0, w.cpu().numpy())
    gU_ref = pr.G().T @ wm
    g_ref = fe.param_grad(pr.mesh, pr.prm, pr.U, pr.phi_tilde, wm, **pr.fields)
    for got, ref in [(U.grad, gU_ref), (gc.grad, g_ref[0]), (lam.grad, g_ref[1]), (mu.grad, g_ref[2])]:
        got = got.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)

    # central differences of the GPU residual along random directions: 1e-6 relative
    def L(Uv, gcv, lamv, muv):
        with torch.no_grad():
            return float((ResidualFunction.apply(ctx, Uv, po, pt, gcv, lamv, muv) * w).sum())

    rng = np.random.default_rng(2)
    for which, base, grad in [(0, U, U.grad), (1, gc, gc.grad), (2, lam, lam.grad), (3, mu, mu.grad)]:
        d = cuda(rng.normal(size=base.numel()))
        if which == 0:
            d = d * cuda((~pr.mesh.dirichlet_mask()).astype(np.float64))
        h = 1e-6 * float(base.detach().norm()) / float(d.norm())
        args_p = [U.detach(), gc.detach(), lam.detach(), mu.detach()]
        args_m = list(args_p)
        args_p[which] = args_p[which] + h * d
        args_m[which] = args_m[which] - h * d
        fd = (L(*args_p) - L(*args_m)) / (2 * h)
        an = float((grad * d).sum())
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-30), (which, fd, an)
