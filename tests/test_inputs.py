"""The seeded generator: known SplitMix64 outputs, numpy/torch agreement, workload recipes."""
import numpy as np
import pytest

from paper_1510_04995_gb300 import inputs


def test_splitmix64_reference_outputs():
    # SplitMix64 with state 0 (seed word 0): published first outputs of the generator.
    st = 0
    outs = []
    for _ in range(3):
        st = (st + inputs.GAMMA) & inputs.MASK64
        outs.append(inputs._mix_int(st))
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_numpy_torch_same_bits():
    torch = pytest.importorskip("torch")
    a = inputs.uniform_np(123, 5, 1000, -1.0, 1.0)
    b = inputs.uniform_torch(123, 5, 1000, -1.0, 1.0, "cpu").numpy()
    assert np.array_equal(a, b)
    assert a.min() >= -1.0 and a.max() < 1.0


def test_problem_recipes():
    u, up, co, c = inputs.make_problem(1, 5, 6, 7)
    assert u.shape == (9, 8, 7) and co.shape == (7, 9, 8, 7)
    assert np.all(u[0] == 0) and np.all(u[:, :, 0] == 0)
    inner = (slice(1, -1),) * 3
    s = co[1][inner] + co[2][inner] + co[3][inner] + co[4][inner] + co[5][inner] + co[6][inner]
    assert np.allclose(co[0][inner], 1.0 - s, atol=1e-15)
    assert np.all(co[1:][(slice(None),) + inner] <= 1.0 / 7.0)
    u, up, co, c = inputs.make_problem(3, 4, 4, 4)
    assert co.shape == (13, 12, 12, 12) and co.max() < 0.01
    assert np.array_equal(u, up)
    assert c == ()
    assert inputs.make_problem(2, 4, 4, 4)[3] == (-0.9, 0.05, 0.025, 0.0125, 0.00625)
    u, up, co, c = inputs.make_problem(4, 5, 4, 3)
    assert co.shape == (1, 11, 12, 13) and np.array_equal(u, up)
    inner = co[0][4:-4, 4:-4, 4:-4]
    assert inner.min() >= 0.5 and inner.max() < 1.0 and co[0].sum() == inner.sum()  # zero halo
    assert c == (-0.9, 0.05, 0.025, 0.0125, 0.00625)
    u, up, co, c = inputs.make_problem(5, 4, 5, 6)
    assert co is None and u.shape == (8, 7, 6) and c == (0.4, 0.05, 0.02, 0.0075)
    assert abs(c[0] + 6 * c[1] + 12 * c[2] + 8 * c[3] - 1.0) < 1e-15
