"""The allocation-free backward pass, through the C ABI, against the workspace-taking one.

Some callers cannot allocate device memory: a stream being captured into a CUDA graph, a
process whose allocator belongs to another framework, or a fixed device-memory budget.  They
use girih_mlp_backward_static, whose workspace is an array compiled into the library.  This file
runs last (collection order) and must pass alone in a fresh process as well as after the other
tests.
"""
import ctypes

import numpy as np
import pytest

import paper_1510_04995_gb300 as girih
from oracle import mlp

pytestmark = pytest.mark.gpu

D = girih.MLP_FEATURES


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _case(n, seed):
    import torch
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(n, D)).astype(np.float32)
    t = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2]).astype(np.float32)
    p = rng.uniform(-0.3, 0.3, mlp.n_params(D)).astype(np.float32)
    return [torch.from_numpy(a).cuda() for a in (p, X, t)], (p, X, t)


def test_static_backward_matches_workspace_backward_twice():
    import torch
    L = girih.lib()
    npar = L.girih_mlp_num_params(D)
    for call, (n, seed) in enumerate([(777, 1), (3000, 2)]):  # two calls in a row, different sizes
        (dp, dX, dt), (p, X, t) = _case(n, seed)
        g_ref = torch.zeros(npar, device="cuda")
        l_ref = torch.zeros(1, device="cuda")
        ws = torch.zeros(L.girih_mlp_workspace_floats(n), device="cuda")
        girih.check(L.girih_mlp_backward(_p(dp), _p(dX), _p(dt), n, D, _p(g_ref), _p(l_ref), _p(ws), None))
        g = torch.zeros(npar, device="cuda")
        loss = torch.zeros(1, device="cuda")
        girih.check(L.girih_mlp_backward_static(_p(dp), _p(dX), _p(dt), n, D, _p(g), _p(loss), None))
        torch.cuda.synchronize()
        gr, gs = g_ref.double().cpu().numpy(), g.double().cpu().numpy()
        # the same kernels with a fixed-order reduction on a different workspace: identical bits
        assert torch.equal(g, g_ref), call
        assert torch.equal(loss, l_ref), call
        # and, per parameter block and element by element, the FP64 oracle at the network tests'
        # tolerance
        go = mlp.backward(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
        scale = float(np.max(np.abs(go)))
        for name, gb, ob in zip(("W1", "b1", "W2", "b2", "W3", "b3"), mlp.unpack(gs, D), mlp.unpack(go, D)):
            tol = 1e-4 * float(np.max(np.abs(ob))) + 1e-6 * scale
            assert float(np.max(np.abs(gb - ob))) <= tol, (call, name)


def test_static_backward_rejects_too_many_rows():
    import torch
    L = girih.lib()
    n = girih.MLP_STATIC_MAX_ROWS + 1
    (dp, dX, dt), _ = _case(n, 3)
    g = torch.full((L.girih_mlp_num_params(D),), 7.0, device="cuda")
    assert L.girih_mlp_backward_static(_p(dp), _p(dX), _p(dt), n, D, _p(g), None, None) == 1
    torch.cuda.synchronize()
    assert bool((g == 7.0).all())  # nothing was enqueued
