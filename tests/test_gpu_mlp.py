"""The learned tuner's CUDA network kernels against the FP64 network oracle."""
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


BLOCKS = ("W1", "b1", "W2", "b2", "W3", "b3")


def assert_blockwise_close(g, go, d, rtol=1e-4, what="gradient"):
    """Element-by-element comparison per parameter block (W1, b1, W2, b2, W3, b3):
    |g - g_o| <= rtol * max|g_o(block)| + 1e-6 * max|g_o|, so that a wrong small block (a bias
    gradient next to the large W2 block) cannot hide inside a global norm."""
    scale = float(np.max(np.abs(go)))
    for name, gb, ob in zip(BLOCKS, mlp.unpack(np.asarray(g, dtype=np.float64), d), mlp.unpack(go, d)):
        tol = rtol * float(np.max(np.abs(ob))) + 1e-6 * scale
        err = np.abs(np.asarray(gb) - np.asarray(ob))
        assert float(np.max(err)) <= tol, f"{what} block {name}: max error {np.max(err):.3e} > {tol:.3e}"


def _rand(n, d, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(n, d))
    t = np.sin(X[:, 0] * 2) + 0.5 * X[:, 1] * X[:, 2] + 0.1 * X[:, 3:].sum(axis=1)
    p = rng.uniform(-0.3, 0.3, mlp.n_params(d))
    return X, t, p


def _gpu_grad(p, X, t):
    import torch
    n, d = X.shape
    L = girih.lib()
    dp, dX, dt = _dev(p), _dev(X), _dev(t)
    g = torch.zeros(L.girih_mlp_num_params(d), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ws = torch.zeros(L.girih_mlp_workspace_floats(n), dtype=torch.float32, device="cuda")
    girih.check(L.girih_mlp_backward(_p(dp), _p(dX), _p(dt), n, d, _p(g), _p(loss), _p(ws), None))
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    girih.check(L.girih_mlp_forward(_p(dp), _p(dX), n, d, _p(y), _p(ws), None))
    torch.cuda.synchronize()
    return y.double().cpu().numpy(), g.double().cpu().numpy(), float(loss.item())


@pytest.mark.parametrize("n", [1, 7, 300, 2049])
def test_forward_and_gradient_match_oracle(n):
    X, t, p = _rand(n, D, n)
    y, g, loss = _gpu_grad(p, X, t)
    yo, _ = mlp.forward(p, X)
    go = mlp.backward(p, X, t)
    assert np.max(np.abs(y - yo)) <= 1e-4 * max(1.0, np.max(np.abs(yo)))
    assert_blockwise_close(g, go, D)
    assert abs(loss - mlp.loss(p, X, t)) <= 1e-4 * mlp.loss(p, X, t)


def test_sgd_and_adam_steps_match_oracle():
    import torch
    L = girih.lib()
    rng = np.random.default_rng(1)
    p = rng.normal(size=500)
    g = rng.normal(size=500)
    dp, dg = _dev(p), _dev(g)
    girih.check(L.girih_mlp_sgd(_p(dp), _p(dg), 500, ctypes.c_float(0.05), None))
    assert np.allclose(dp.double().cpu().numpy(), mlp.sgd_step(p, g, 0.05), rtol=1e-6, atol=1e-6)
    dp = _dev(p)
    m = torch.zeros(500, device="cuda")
    v = torch.zeros(500, device="cuda")
    mo, vo, po = np.zeros(500), np.zeros(500), p.copy()
    for step in range(1, 4):
        g = rng.normal(size=500)
        girih.check(L.girih_mlp_adam(_p(dp), _p(_dev(g)), _p(m), _p(v), 500, step, ctypes.c_float(1e-2),
                                     ctypes.c_float(0.9), ctypes.c_float(0.999), ctypes.c_float(1e-8), None))
        po, mo, vo = mlp.adam_step(po, g, mo, vo, step, 1e-2)
    torch.cuda.synchronize()
    assert np.allclose(dp.double().cpu().numpy(), po, rtol=1e-5, atol=1e-6)
    # SGD and Adam on a full parameter vector of the network, compared block by block
    npar = mlp.n_params(D)
    p = rng.normal(size=npar)
    g = rng.normal(size=npar)
    dp = _dev(p)
    girih.check(L.girih_mlp_sgd(_p(dp), _p(_dev(g)), npar, ctypes.c_float(0.05), None))
    torch.cuda.synchronize()
    assert_blockwise_close(dp.double().cpu().numpy(), mlp.sgd_step(p, g, 0.05), D, rtol=1e-6, what="SGD step")
    dp = _dev(p)
    m = torch.zeros(npar, device="cuda")
    v = torch.zeros(npar, device="cuda")
    mo, vo, po = np.zeros(npar), np.zeros(npar), p.copy()
    for step in range(1, 4):
        g = rng.normal(size=npar)
        girih.check(L.girih_mlp_adam(_p(dp), _p(_dev(g)), _p(m), _p(v), npar, step, ctypes.c_float(1e-2),
                                     ctypes.c_float(0.9), ctypes.c_float(0.999), ctypes.c_float(1e-8), None))
        po, mo, vo = mlp.adam_step(po, g, mo, vo, step, 1e-2)
    torch.cuda.synchronize()
    assert_blockwise_close(dp.double().cpu().numpy(), po, D, rtol=1e-5, what="Adam step")


def test_gpu_training_reduces_loss_like_oracle():
    """Adam training with the CUDA kernels tracks the FP64 oracle's training curve."""
    import torch
    L = girih.lib()
    n = 512
    X, t, p = _rand(n, D, 42)
    dp, dX, dt = _dev(p), _dev(X), _dev(t)
    npar = L.girih_mlp_num_params(D)
    g = torch.zeros(npar, device="cuda")
    m = torch.zeros(npar, device="cuda")
    v = torch.zeros(npar, device="cuda")
    loss = torch.zeros(1, device="cuda")
    ws = torch.zeros(L.girih_mlp_workspace_floats(n), device="cuda")
    po, mo, vo = p.copy(), np.zeros(npar), np.zeros(npar)
    l0 = mlp.loss(p, X, t)
    for step in range(1, 301):
        girih.check(L.girih_mlp_backward(_p(dp), _p(dX), _p(dt), n, D, _p(g), _p(loss), _p(ws), None))
        girih.check(L.girih_mlp_adam(_p(dp), _p(g), _p(m), _p(v), npar, step, ctypes.c_float(3e-3),
                                     ctypes.c_float(0.9), ctypes.c_float(0.999), ctypes.c_float(1e-8), None))
        if step <= 20:
            po, mo, vo = mlp.adam_step(po, mlp.backward(po, X, t), mo, vo, step, 3e-3)
    torch.cuda.synchronize()
    p20 = None
    lg = mlp.loss(dp.double().cpu().numpy(), X, t)
    assert lg < 0.1 * l0
    assert mlp.loss(po, X, t) < l0  # the oracle's first steps also descend


def test_bad_arguments():
    L = girih.lib()
    assert L.girih_mlp_forward(None, None, 0, D, None, None, None) == 1
    assert L.girih_mlp_sgd(None, None, 0, ctypes.c_float(0.1), None) == 1
