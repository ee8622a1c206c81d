"""The allocation-free parameter gradient (pff_param_grad_noalloc) against pff_param_grad.

Some callers of this library cannot allocate device memory at the moment they need a gradient:
code that runs while a CUDA graph is being captured (cudaMalloc is not allowed there) or a host
application that hands out all device memory through its own pool. pff_param_grad allocates its
per-point scratch lazily on its first call; pff_param_grad_noalloc instead uses a fixed array that
the library keeps in device memory, so the caller only passes inputs and outputs. This file is
named so that pytest runs it after every other test file.
"""
import numpy as np
import pytest

from problems import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_noalloc_matches_param_grad_on_two_calls():
    """Two calls in a row on a fresh context (the shared scratch keeps the previous call's contents)
    equal pff_param_grad within 1e-12 and leave the context's device memory unchanged; the ordinary
    entry point called afterwards allocates its scratch, which shows the accounting would see it."""
    pr = Problem(2, 2, 16, split=1, seed=31, fields=True)
    ctx = pr.context()
    nn = pr.mesh.n_nodes
    vs = [cuda(np.random.default_rng(100 + call).normal(size=pr.mesh.n_dofs)) for call in range(2)]
    m0 = ctx.memory()
    got = []
    for v in vs:
        outs = [torch.empty(nn, dtype=torch.float64, device="cuda") for _ in range(3)]
        got.append([g.clone() for g in ctx.param_grad_noalloc(*outs, v)])
    torch.cuda.synchronize()
    assert ctx.memory() == m0
    for v, g in zip(vs, got):
        ref = ctx.param_grad(v)
        for a, b in zip(g, ref):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
    assert ctx.memory()["total"] > m0["total"]


def test_noalloc_rejects_problems_beyond_its_scratch():
    from paper_2005_00331_gb300 import PFFError, setup_mesh
    from paper_2005_00331_gb300.pff import PFF_ERR_TOO_LARGE
    ctx = setup_mesh(dim=2, degree=1, n_cells_1d=512, split=0, eps=2.0 / 512)
    nn = ctx.n_nodes
    U = torch.zeros(ctx.n_dofs, dtype=torch.float64, device="cuda")
    U[2 * nn:] = 1.0
    one = torch.ones(nn, dtype=torch.float64, device="cuda")
    ctx.set_state(U, one, one, torch.zeros(nn, dtype=torch.uint8, device="cuda"))
    outs = [torch.empty(nn, dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(PFFError) as err:
        ctx.param_grad_noalloc(*outs, U)
    assert err.value.status == PFF_ERR_TOO_LARGE
