"""The C-ABI library without a GPU: it loads, exports every symbol the header declares, its model
functions reproduce the paper's worked examples, and argument errors are reported."""
import ctypes

import pytest

import paper_1510_04995_gb300 as girih
from paper_1510_04995_gb300 import build as gbuild

MiB = 1024.0 * 1024.0


@pytest.fixture(scope="module")
def L():
    gbuild.build()
    return girih.lib()


def test_exports_every_declared_symbol(L):
    names = girih.header_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n


def test_cache_block_model_eq2_worked_example(L):
    # Sect. 3.3: D_w = 8, N_F = 1, 7-point constant (N_D = 2) -> C_S = 94 * N_xb bytes
    assert girih.model_cache_block(1.0, 8, 1, 1, 2) == pytest.approx(94.0)
    assert girih.model_cache_block(1000.0, 8, 1, 1, 2) == pytest.approx(94000.0)


@pytest.mark.parametrize("dw,paper_mib,tol", [(16, 3.0, 0.25), (32, 12.5, 0.2), (48, 27.0, 0.5)])
def test_cache_block_model_eq3_worked_examples(L, dw, paper_mib, tol):
    # Sect. 3.5: 25-point constant coefficient at N = 960^3 (N_xb = 960 * 8 bytes), N_D = 3, N_F = 1:
    # D_w = 16 needs ~3 MiB, D_w = 32 ~12.5 MiB, D_w = 48 ~27 MiB per thread.
    cs = girih.model_cache_block(960 * 8, dw, 1, 4, 3) / MiB
    assert abs(cs - paper_mib) <= tol


def test_code_balance_model(L):
    # Eq. 4 (R = 1, FP64): 16 [(2Dw - 2) + (N_D Dw + 2)] / Dw^2
    for dw in (4, 8, 16, 32):
        assert girih.model_code_balance(dw, 1, 2, 8) == pytest.approx(16 * ((2 * dw - 2) + (2 * dw + 2)) / dw ** 2)
    # Eq. 5 at R = 4 and the FP32 form (8R instead of 16R)
    assert girih.model_code_balance(16, 4, 2, 8) == pytest.approx(64 * (24 + 40) / 256)
    assert girih.model_code_balance(16, 4, 2, 4) == pytest.approx(0.5 * girih.model_code_balance(16, 4, 2, 8))
    # larger diamonds never cost more bytes per update
    vals = [girih.model_code_balance(d, 1, 9, 8) for d in (4, 8, 16, 32, 64)]
    assert all(a > b for a, b in zip(vals, vals[1:]))


@pytest.mark.parametrize("args", [
    (7, 8, 8, 8, 0, 0, 1),      # unknown stencil
    (0, 0, 8, 8, 0, 0, 1),      # empty grid
    (0, 8, 8, 8, 0, 5, 1),      # unknown dtype
    (0, 8, 8, 8, 0, 0, -1),     # negative T
    (2, 8, 8, 8, 10, 0, 1),     # ldx < nx + 2R
])
def test_plan_rejects_bad_arguments(L, args):
    h = ctypes.c_void_p(123)
    rc = L.girih_plan(ctypes.byref(h), *args)
    assert rc == 1 and h.value is None
    assert len(girih.last_error()) > 0


def test_null_handles_are_rejected(L):
    assert L.girih_run(None, None, None, None, None, None) == 1
    assert L.girih_plan_destroy(None) == 0
    assert L.girih_mlp_num_params(16) == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1


def test_features_encode_configuration(L):
    import numpy as np
    out = np.zeros(girih.MLP_FEATURES, dtype=np.float32)
    cfg = girih.config(girih.MWD, dw=16, nf=2, cluster=8, threads=256)
    assert L.girih_mlp_features(1, 1, 512, 256, 128, ctypes.byref(cfg), out.ctypes.data_as(ctypes.c_void_p)) == 0
    assert out[1] == 1 and out[0] == 0 and out[4] == 1 and out[8] == 1
    assert out[5] == pytest.approx(0.9) and out[6] == pytest.approx(0.8) and out[7] == pytest.approx(0.7)
