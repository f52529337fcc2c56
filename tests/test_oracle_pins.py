"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each check is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign or
index, a transposed axis, a wrong coefficient grid) fails at least one of them:
* brute force: an independent table-driven evaluator agrees bit for bit on 8^3 grids;
* closed forms: Dirichlet sine modes of the 7-point operator decay by their eigenvalue per step,
  and sine modes of the 25-point leapfrog follow their scalar recurrence inside the light cone;
* invariants: constant fields are preserved when the weights sum to one (7-point) or when the
  Laplacian part annihilates constants (25-point), linearity, impulse responses;
* special cases: uniform coefficient grids reduce the variable stencils to the constant ones,
  and a unit factor grid reduces Listing 3 as printed (25-point with the factor grid C) to the
  25-point constant stencil.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1510_04995_gb300 import inputs


def _grid(stencil, n, seed=7, ldx=None):
    return inputs.make_problem(stencil, n, n, n, seed=seed, ldx=ldx)


@pytest.mark.parametrize("stencil", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("T", [1, 2, 3])
def test_brute_force_bitwise(stencil, T):
    """Oracle loop nests == table-driven per-point evaluation on 8^3 (Listings 1-4)."""
    R = inputs.RADIUS[stencil]
    u, up, co, c = _grid(stencil, 8)
    if stencil in (2, 3, 4):  # a non-trivial u_prev so the 2V - U term is exercised
        up = up.copy()
        up[R:-R, R:-R, R:-R] *= 0.5
    bu, bup = brute.sweep(stencil, u, up, co, c, T, R)
    oracle.sweep(stencil, u, up, co, c, T, 8, 8, 8)
    assert np.array_equal(u, bu)
    assert np.array_equal(up, bup)


def _sine(n, modes, R):
    a, b, cc = modes
    i = np.arange(n + 2 * R, dtype=np.float64) - (R - 1)  # interior index 1..n at padded R..R+n-1
    sx = np.sin(a * math.pi * i / (n + 1))
    sy = np.sin(b * math.pi * i / (n + 1))
    sz = np.sin(cc * math.pi * i / (n + 1))
    u = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    out = np.zeros_like(u)
    out[R:R + n, R:R + n, R:R + n] = u[R:R + n, R:R + n, R:R + n]
    return out


@pytest.mark.parametrize("modes", [(1, 1, 1), (3, 5, 7), (16, 1, 8)])
def test_7c_dirichlet_sine_mode(modes):
    """With a zero halo at index 0 and n+1, sin modes are exact eigenvectors of Listing 1."""
    n, T = 16, 8
    c0, c1 = 0.4, 0.1
    u = _sine(n, modes, 1)
    up = u.copy()
    oracle.sweep(0, u, up, None, (c0, c1), T, n, n, n)
    mu = c0 + 2 * c1 * sum(math.cos(m * math.pi / (n + 1)) for m in modes)
    u0 = _sine(n, modes, 1)
    ref = (mu ** T) * u0
    # rounding errors are relative to the initial amplitude (the mode itself may decay fast)
    assert np.max(np.abs(u - ref)) / np.max(np.abs(u0)) < 1e-14 * T
    assert np.max(np.abs(ref)) > 1e-4 * np.max(np.abs(u0))  # the decay is still well resolved
    ref1 = (mu ** (T - 1)) * u0  # level T-1 is returned in u_prev
    assert np.max(np.abs(up - ref1)) / np.max(np.abs(u0)) < 1e-14 * T


def test_7c_sine_mode_value_at_64():
    """Worked number for the 64^3 workload: mode (1,1,1) decays by mu = 0.99929934 per step."""
    n = 64
    mu = 0.4 + 2 * 0.1 * 3 * math.cos(math.pi / (n + 1))
    assert abs(mu - 0.99929934) < 5e-9
    assert abs(mu ** 8 - 0.99440842) < 5e-9


@pytest.mark.parametrize("stencil", [0, 1])
def test_constant_preserved_7pt(stencil):
    """Weights summing to 1 with a constant halo keep a constant field constant."""
    n, T, cval = 10, 5, 0.75
    u, up, co, c = _grid(stencil, n)
    u[:] = cval
    up[:] = cval
    oracle.sweep(stencil, u, up, co, c, T, n, n, n)
    assert np.max(np.abs(u - cval)) <= 4 * T * np.finfo(float).eps


@pytest.mark.parametrize("stencil", [2, 3, 4])
def test_constant_preserved_25pt(stencil):
    """Leapfrog with a Laplacian part that annihilates constants keeps u = u_prev = const (with the
    factor grid: whatever the factors, since they multiply a zero bracket)."""
    n, T, cval = 12, 4, -0.3
    u, up, co, c = _grid(stencil, n)
    u[:] = cval
    up[:] = cval
    if stencil in (2, 4):
        c = (-6 * (0.05 + 0.025 + 0.0125 + 0.00625), 0.05, 0.025, 0.0125, 0.00625)
    else:
        co = co.copy()
        co[0] = -2.0 * co[1:].sum(axis=0)
    oracle.sweep(stencil, u, up, co, c, T, n, n, n)
    assert np.max(np.abs(u - cval)) < 1e-14


def test_25c_light_cone_sine_mode():
    """Inside the light cone (distance > R*T from the halo) a sine mode follows
    a_{t+1} = (2 + lam) a_t - a_{t-1}, a_0 = a_{-1} = 1, lam = c0 + 2 sum_r c_r sum_axes cos(r theta)."""
    n, T, R = 72, 6, 4
    c = (-0.9, 0.05, 0.025, 0.0125, 0.00625)
    th = (2 * math.pi / 17, 2 * math.pi / 11, 2 * math.pi / 23)
    idx = np.arange(n + 2 * R, dtype=np.float64)
    f = [np.sin(t * idx + 0.3) for t in th]
    phi = f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
    u = np.zeros_like(phi)
    u[R:-R, R:-R, R:-R] = phi[R:-R, R:-R, R:-R]
    up = u.copy()
    oracle.sweep(2, u, up, None, c, T, n, n, n)
    lam = c[0] + 2 * sum(c[r] * sum(math.cos(r * t) for t in th) for r in range(1, 5))
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    a_prev, a = Decimal(1), Decimal(1)
    L = Decimal(2) + Decimal(lam)
    for _ in range(T):
        a_prev, a = a, L * a - a_prev
    aT = float(a)
    m = R + R * T + 1
    core = (slice(m, n + 2 * R - m),) * 3
    err = np.max(np.abs(u[core] - aT * phi[core])) / np.max(np.abs(aT * phi[core]))
    assert err < 1e-12
    # outside the cone the wall is felt: the identity must NOT hold everywhere (the test has teeth)
    assert np.max(np.abs(u[R:-R, R:-R, R:-R] - aT * phi[R:-R, R:-R, R:-R])) > 1e-6


@pytest.mark.parametrize("kappa", [0.75, 0.5])
def test_25cg_light_cone_sine_mode(kappa):
    """Listing 3 as printed with a uniform factor grid C = kappa: inside the light cone a sine mode
    follows a_{t+1} = (2 + kappa*lam) a_t - a_{t-1}, a_0 = a_{-1} = 1 (the factor scales the whole
    bracket, centre term included, and not the leapfrog terms 2V - U)."""
    n, T, R = 72, 6, 4
    c = (-0.9, 0.05, 0.025, 0.0125, 0.00625)
    th = (2 * math.pi / 13, 2 * math.pi / 19, 2 * math.pi / 29)
    idx = np.arange(n + 2 * R, dtype=np.float64)
    f = [np.sin(t * idx + 0.7) for t in th]
    phi = f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
    u = np.zeros_like(phi)
    u[R:-R, R:-R, R:-R] = phi[R:-R, R:-R, R:-R]
    up = u.copy()
    co = np.zeros((1,) + u.shape)
    co[0, R:-R, R:-R, R:-R] = kappa
    oracle.sweep(4, u, up, co, c, T, n, n, n)
    lam = c[0] + 2 * sum(c[r] * sum(math.cos(r * t) for t in th) for r in range(1, 5))
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    a_prev, a = Decimal(1), Decimal(1)
    L = Decimal(2) + Decimal(kappa) * Decimal(lam)
    for _ in range(T):
        a_prev, a = a, L * a - a_prev
    aT = float(a)
    m = R + R * T + 1
    core = (slice(m, n + 2 * R - m),) * 3
    err = np.max(np.abs(u[core] - aT * phi[core])) / np.max(np.abs(aT * phi[core]))
    assert err < 1e-12
    assert np.max(np.abs(u[R:-R, R:-R, R:-R] - aT * phi[R:-R, R:-R, R:-R])) > 1e-6


def test_25cg_unit_factor_equals_25c():
    """A factor grid of ones reduces Listing 3 as printed to the 25-point constant stencil, bit for
    bit (multiplying by 1 is exact)."""
    n, T = 12, 4
    u, up, _, c = _grid(2, n)
    up = up.copy()
    up[4:-4, 4:-4, 4:-4] *= 0.25
    u2, up2 = u.copy(), up.copy()
    co = np.ones((1,) + u.shape)
    oracle.sweep(2, u, up, None, c, T, n, n, n)
    oracle.sweep(4, u2, up2, co, c, T, n, n, n)
    assert np.array_equal(u, u2) and np.array_equal(up, up2)


@pytest.mark.parametrize("modes", [(1, 1, 1), (3, 5, 7), (16, 2, 9)])
def test_27b_dirichlet_sine_mode(modes):
    """With a zero halo at index 0 and n+1, sin modes are exact eigenvectors of the 27-point box
    operator: mu = c0 + 2 c1 (cx+cy+cz) + 4 c2 (cx cy + cx cz + cy cz) + 8 c3 cx cy cz, c = cos(m pi/(n+1))."""
    n, T = 16, 6
    c = (0.4, 0.05, 0.02, 0.0075)
    u = _sine(n, modes, 1)
    up = u.copy()
    oracle.sweep(5, u, up, None, c, T, n, n, n)
    cx, cy, cz = (math.cos(m * math.pi / (n + 1)) for m in modes)
    mu = c[0] + 2 * c[1] * (cx + cy + cz) + 4 * c[2] * (cx * cy + cx * cz + cy * cz) + 8 * c[3] * cx * cy * cz
    ref = _sine(n, modes, 1) * mu ** T
    scale = max(np.max(np.abs(ref)), 1e-300)
    assert np.max(np.abs(u - ref)) <= 1e-13 * max(scale, abs(mu) ** T)
    # the same field with the 7-point operator decays differently (the corners and edges count)
    u7 = _sine(n, modes, 1)
    oracle.sweep(0, u7, u7.copy(), None, (0.4, 0.1), T, n, n, n)
    assert np.max(np.abs(u7 - ref)) > 1e-6 * np.max(np.abs(_sine(n, modes, 1)))


def test_27b_constant_preserved_and_reduces_to_7c():
    """Weights summing to one keep a constant field; with zero edge and corner weights the box
    operator is the 7-point constant one (up to the rounding of its six-term face sum)."""
    n, T, cval = 10, 4, 0.7
    u, up, _, c = _grid(5, n)
    u[1:-1, 1:-1, 1:-1] = cval
    oracle.sweep(5, u, up, None, c, T, n, n, n)
    core = u[1 + T:-1 - T, 1 + T:-1 - T, 1 + T:-1 - T]
    assert np.max(np.abs(core - cval)) <= 1e-14
    u, up, _, _ = _grid(5, n)
    u2, up2 = u.copy(), up.copy()
    oracle.sweep(5, u, up, None, (0.4, 0.1, 0.0, 0.0), T, n, n, n)
    oracle.sweep(0, u2, up2, None, (0.4, 0.1), T, n, n, n)
    assert np.max(np.abs(u - u2)) <= 4e-16 * T * np.max(np.abs(u2))


def test_rbgs_impulse_two_half_sweeps():
    """One red-black iteration (two half-sweeps) of an impulse on a black point, hand-derived:
    the red half-sweep gives its six red neighbours c1; the black half-sweep then reads those NEW
    values (Gauss-Seidel, not Jacobi): the impulse point becomes c0 + 6 c1^2, the black points two
    steps away along an axis c1^2 and the black points at face-diagonal offsets 2 c1^2."""
    n = 11
    c0, c1 = 0.25, 0.125                       # exact in binary: every product and sum below is exact
    u = np.zeros((n + 2,) * 3)
    m = 6                                      # interior coordinate 5: (5+5+5) odd -> black
    u[m, m, m] = 1.0
    up = u.copy()
    oracle.sweep(6, u, up, None, (c0, c1), 2, n, n, n)
    ref = np.zeros_like(u)
    ref[m, m, m] = c0 + 6 * c1 * c1
    for ax in range(3):
        for sg in (1, -1):
            d = [0, 0, 0]
            d[ax] = sg
            ref[m + d[0], m + d[1], m + d[2]] = c1               # red neighbours, from half-sweep 0
            d[ax] = 2 * sg
            ref[m + d[0], m + d[1], m + d[2]] = c1 * c1          # black, one red neighbour updated
    for a in range(3):
        for b in range(a + 1, 3):
            for sa in (1, -1):
                for sb in (1, -1):
                    d = [0, 0, 0]
                    d[a], d[b] = sa, sb
                    ref[m + d[0], m + d[1], m + d[2]] = 2 * c1 * c1  # black, two red neighbours
    assert np.array_equal(u, ref)
    # Jacobi on the same two steps differs (the black half-sweep would read the old red values)
    uj = np.zeros_like(ref)
    uj[m, m, m] = 1.0
    oracle.sweep(0, uj, uj.copy(), None, (c0, c1), 2, n, n, n)
    assert not np.array_equal(uj, ref)


def test_rbgs_harmonic_fixed_point_and_convergence():
    """A discrete harmonic field (linear in x, y, z, with matching Dirichlet halo) is a fixed point
    of the Laplace red-black iteration (c0 = 0, c1 = 1/6); from random interior values the
    iteration converges towards it, faster than Jacobi (the spectral radius of red-black
    Gauss-Seidel is the square of Jacobi's)."""
    n = 12
    idx = np.arange(n + 2, dtype=np.float64)
    lin = (0.5 * idx[None, None, :] + 0.25 * idx[None, :, None] + 0.125 * idx[:, None, None])
    u = lin.copy()
    oracle.sweep(6, u, u.copy(), None, (0.0, 1.0 / 6.0), 8, n, n, n)
    assert np.max(np.abs(u - lin)) <= 4e-15 * np.max(np.abs(lin))
    rnd, _, _, _ = _grid(6, n)
    u0 = lin.copy()
    u0[1:-1, 1:-1, 1:-1] += rnd[1:-1, 1:-1, 1:-1]
    ug, uj = u0.copy(), u0.copy()
    oracle.sweep(6, ug, ug.copy(), None, (0.0, 1.0 / 6.0), 40, n, n, n)     # 20 iterations
    oracle.sweep(0, uj, uj.copy(), None, (0.0, 1.0 / 6.0), 20, n, n, n)     # 20 Jacobi steps
    eg, ej = np.max(np.abs(ug - lin)), np.max(np.abs(uj - lin))
    assert eg < 0.5 * ej and eg < np.max(np.abs(u0 - lin))


def test_7v_uniform_equals_7c():
    n, T = 9, 4
    u, up, _, c = _grid(0, n)
    u2, up2 = u.copy(), up.copy()
    co = np.zeros((7,) + u.shape)
    co[0] = 0.4
    co[1:] = 0.1
    oracle.sweep(0, u, up, None, c, T, n, n, n)
    oracle.sweep(1, u2, up2, co, (), T, n, n, n)
    assert np.max(np.abs(u - u2)) <= 1e-15


def test_25v_uniform_equals_25c():
    n, T = 12, 3
    u, up, _, c = _grid(2, n)
    u2, up2 = u.copy(), up.copy()
    co = np.zeros((13,) + u.shape)
    co[0] = c[0]
    for r in range(1, 5):
        co[3 * r - 2:3 * r + 1] = c[r]
    oracle.sweep(2, u, up, None, c, T, n, n, n)
    oracle.sweep(3, u2, up2, co, (), T, n, n, n)
    assert np.max(np.abs(u - u2)) <= 1e-14 * np.max(np.abs(u))


def _impulse_pattern(stencil, co, c, R, n):
    """Expected one-step response of a unit impulse at the centre (u_prev = 0)."""
    m = n // 2 + R
    exp = {}
    if stencil == 0:
        exp[(0, 0, 0)] = c[0]
        for d in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
            exp[d] = c[1]
    elif stencil == 1:
        # the value at p + d receives C_m(p + d) times the impulse, where d is the opposite offset
        exp[(0, 0, 0)] = co[0, m, m, m]
        for g, (dx, dy, dz) in zip(range(1, 7), [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]):
            exp[(-dx, -dy, -dz)] = co[g, m - dz, m - dy, m - dx]
    elif stencil == 2:
        exp[(0, 0, 0)] = 2.0 + c[0]
        for r in range(1, 5):
            for d in [(r, 0, 0), (-r, 0, 0), (0, r, 0), (0, -r, 0), (0, 0, r), (0, 0, -r)]:
                exp[d] = c[r]
    elif stencil == 5:
        exp[(0, 0, 0)] = c[0]
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    m = (dx != 0) + (dy != 0) + (dz != 0)
                    if m:
                        exp[(dx, dy, dz)] = c[m]
    elif stencil == 4:
        # the point at p + d updates with its own factor C(p + d) times c_r (the impulse is its
        # neighbour at -d); the centre keeps 2V and gains C(p) * c0
        exp[(0, 0, 0)] = 2.0 + co[0, m, m, m] * c[0]
        for r in range(1, 5):
            for d in [(r, 0, 0), (-r, 0, 0), (0, r, 0), (0, -r, 0), (0, 0, r), (0, 0, -r)]:
                exp[d] = co[0, m + d[2], m + d[1], m + d[0]] * c[r]
    else:
        exp[(0, 0, 0)] = 2.0 + co[0, m, m, m]
        g = 1
        for r in range(1, 5):
            for ax in range(3):
                for sgn in (1, -1):
                    d = [0, 0, 0]
                    d[ax] = sgn * r
                    exp[tuple(d)] = co[g, m + d[2], m + d[1], m + d[0]]
                g += 1
    return m, exp


@pytest.mark.parametrize("stencil", [0, 1, 2, 3, 4, 5])
def test_impulse_response(stencil):
    R = inputs.RADIUS[stencil]
    n = 11
    u, up, co, c = _grid(stencil, n)
    u[:] = 0
    up[:] = 0
    m, exp = _impulse_pattern(stencil, co, c, R, n)
    u[m, m, m] = 1.0
    oracle.sweep(stencil, u, up, co, c, 1, n, n, n)
    ref = np.zeros_like(u)
    for (dx, dy, dz), v in exp.items():
        ref[m + dz, m + dy, m + dx] = v
    assert np.array_equal(u, ref)


@pytest.mark.parametrize("stencil", [0, 1, 2, 3, 4, 5, 6])
def test_linearity(stencil):
    n, T = 10, 3
    u1, up1, co, c = _grid(stencil, n, seed=1)
    u2, up2, _, _ = _grid(stencil, n, seed=2)
    al, be = 0.37, -1.9
    u3, up3 = al * u1 + be * u2, al * up1 + be * up2
    for u, up in ((u1, up1), (u2, up2), (u3, up3)):
        oracle.sweep(stencil, u, up, co, c, T, n, n, n)
    comb = al * u1 + be * u2
    assert np.max(np.abs(u3 - comb)) <= 1e-13 * max(1.0, np.max(np.abs(comb)))


def test_padded_leading_dimension_matches_dense():
    """A padded x pitch (ldx > nx + 2R) changes nothing in the interior."""
    n, T = 9, 4
    for stencil in range(7):
        u, up, co, c = _grid(stencil, n)
        R = inputs.RADIUS[stencil]
        u2, up2, co2, _ = _grid(stencil, n, ldx=n + 2 * R + 5)
        oracle.sweep(stencil, u, up, co, c, T, n, n, n)
        oracle.sweep(stencil, u2, up2, co2, c, T, n, n, n)
        assert np.array_equal(u, u2[:, :, :n + 2 * R])


def test_openmp_threads_do_not_change_result():
    u, up, co, c = _grid(3, 14)
    u2, up2 = u.copy(), up.copy()
    oracle.sweep(3, u, up, co, c, 3, 14, 14, 14, nthreads=1)
    oracle.sweep(3, u2, up2, co, c, 3, 14, 14, 14, nthreads=4)
    assert np.array_equal(u, u2)


def test_t0_is_noop_and_odd_t_swaps():
    u, up, co, c = _grid(0, 6)
    a, b = u.copy(), up.copy()
    oracle.sweep(0, u, up, co, c, 0, 6, 6, 6)
    assert np.array_equal(u, a) and np.array_equal(up, b)
    oracle.sweep(0, u, up, co, c, 1, 6, 6, 6)
    assert np.array_equal(up, a)  # level 0 moved to u_prev


def test_oracle_rejects_bad_arguments():
    u, up, co, c = _grid(1, 6)
    with pytest.raises(ValueError):
        oracle.sweep(1, u, up, None, c, 1, 6, 6, 6)
