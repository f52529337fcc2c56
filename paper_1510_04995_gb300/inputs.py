"""Seeded synthetic inputs for the stencil sweeps (shared by the oracle tests and the CUDA path).

This module holds no stencil arithmetic.  It only turns (seed, stream, index) into numbers:

* ``splitmix64(seed, stream, n)`` -- the n-th output of a counter-based SplitMix64 generator
  (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the state
  after n steps is ``s0 + (n+1)*GAMMA`` and the output is the published 64-bit finaliser of that
  state.  ``s0`` is the finaliser applied to ``seed*GAMMA2 + stream``.  Every value depends only on
  (seed, stream, linear index), so a grid can be generated in any order, on the host with numpy
  or on the device with torch, with identical bits (both back ends are tested against each other).
* ``uniform(a, b)`` -- top 53 bits of the output as a double in [0, 1), mapped to [a, b).

Grids use the padded layout ``[nz+2R][ny+2R][ldx]`` with x fastest; halo cells are 0 (the paper's
loops skip R cells at each face and never write them; zero is the value the workloads fix).
Random values are drawn at the *padded* linear index, so the interior values do not depend on ldx
only through their position -- the index used is ``(k*(ny+2R)+j)*(nx+2R)+i`` on the dense layout.
FP32 inputs are round-to-nearest casts of the FP64 values.

Workload recipes (the configurations the sweeps are measured and tested on):
  7c  : u0 ~ U[-1,1] (stream 0); c0 = 0.4, c1 = 0.1.
  7v  : u0 ~ U[-1,1]; C1..C6 ~ U[0,1/7] (streams 2..7); C0 = 1 - (C1+...+C6) summed in that order in FP64.
  25c : u0 ~ U[-1,1]; u_prev = u0 (zero initial velocity); c0 = -0.9, c_r = 0.1/2^r.
  25v : u0 ~ U[-1,1]; u_prev = u0; C00..C12 ~ U[0,0.01] (streams 1..13).
  25cg: u0 ~ U[-1,1]; u_prev = u0; c as 25c; the per-point factor C ~ U[0.5,1] (stream 1).
  27b : u0 ~ U[-1,1]; centre 0.4, faces 0.05, edges 0.02, corners 0.0075 (weights sum to 1).
  rbgs: u0 ~ U[-1,1]; c0 = 0, c1 = 1/6 (red-black Gauss-Seidel for the 7-point Laplace equation).
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
GAMMA2 = 0xD1B54A32D192ED03
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
DEFAULT_SEED = 20151016

RADIUS = {0: 1, 1: 1, 2: 4, 3: 4, 4: 4, 5: 1, 6: 1}
NCOEF = {0: 0, 1: 7, 2: 0, 3: 13, 4: 1, 5: 0, 6: 0}
SECOND_ORDER = {0: False, 1: False, 2: True, 3: True, 4: True, 5: False, 6: False}
STENCIL_NAMES = {0: "7pt_const", 1: "7pt_var", 2: "25pt_const", 3: "25pt_var", 4: "25pt_cgrid", 5: "27pt_box",
                 6: "7pt_rbgs"}
CONST_COEFFS = {0: (0.4, 0.1), 2: (-0.9, 0.1 / 2, 0.1 / 4, 0.1 / 8, 0.1 / 16),
                4: (-0.9, 0.1 / 2, 0.1 / 4, 0.1 / 8, 0.1 / 16),
                5: (0.4, 0.05, 0.02, 0.0075), 6: (0.0, 1.0 / 6.0)}


def _mix_int(z: int) -> int:
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def stream_base(seed: int, stream: int) -> int:
    return _mix_int(((seed * GAMMA2) + stream) & MASK64)


def _mix_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
    return z ^ (z >> np.uint64(31))


def uniform_np(seed: int, stream: int, n: int, a: float, b: float) -> np.ndarray:
    """n doubles in [a, b) from (seed, stream), index 0..n-1 (numpy, host)."""
    base = np.uint64(stream_base(seed, stream))
    idx = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix_np(base + idx * np.uint64(GAMMA))
    x = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return a + (b - a) * x


def _srl(x, k: int):
    """Logical right shift of int64 tensors holding uint64 bit patterns."""
    import torch
    return (x >> k) & ((1 << (64 - k)) - 1)


def _to_i64(v: int) -> int:
    v &= MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def uniform_torch(seed: int, stream: int, n: int, a: float, b: float, device) -> "torch.Tensor":
    """Same bits as uniform_np, computed with int64 wrap-around arithmetic in torch (any device)."""
    import torch
    base = torch.tensor(_to_i64(stream_base(seed, stream)), dtype=torch.int64, device=device)
    out = torch.empty(n, dtype=torch.float64, device=device)
    chunk = 1 << 26
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = torch.arange(s + 1, e + 1, dtype=torch.int64, device=device)
        z = base + idx * _to_i64(GAMMA)
        z = (z ^ _srl(z, 30)) * _to_i64(M1)
        z = (z ^ _srl(z, 27)) * _to_i64(M2)
        z = z ^ _srl(z, 31)
        x = _srl(z, 11).to(torch.float64) * (1.0 / 9007199254740992.0)
        out[s:e] = a + (b - a) * x
    return out


def padded_shape(nx: int, ny: int, nz: int, R: int, ldx: int | None = None):
    return (nz + 2 * R, ny + 2 * R, ldx if ldx else nx + 2 * R)


def _field(seed, stream, nx, ny, nz, R, ldx, a, b, backend, device):
    """Random interior in [a,b), zero halo; values drawn at the dense padded index."""
    dense = (nz + 2 * R, ny + 2 * R, nx + 2 * R)
    n = dense[0] * dense[1] * dense[2]
    if backend == "numpy":
        v = uniform_np(seed, stream, n, a, b).reshape(dense)
        out = np.zeros(padded_shape(nx, ny, nz, R, ldx), dtype=np.float64)
        out[R:R + nz, R:R + ny, R:R + nx] = v[R:R + nz, R:R + ny, R:R + nx]
        return out
    import torch
    v = uniform_torch(seed, stream, n, a, b, device).reshape(dense)
    out = torch.zeros(padded_shape(nx, ny, nz, R, ldx), dtype=torch.float64, device=device)
    out[R:R + nz, R:R + ny, R:R + nx] = v[R:R + nz, R:R + ny, R:R + nx]
    return out


def make_problem(stencil: int, nx: int, ny: int, nz: int, seed: int = DEFAULT_SEED,
                 ldx: int | None = None, backend: str = "numpy", device=None):
    """Return (u, u_prev, coeffs, c) in FP64 for one of the seven workloads.

    u, u_prev: padded grids.  coeffs: None or an array [ncoef, *padded] (coefficient halo = 0).
    c: tuple of the constant coefficients (empty for the variable-coefficient stencils 1 and 3).
    """
    R = RADIUS[stencil]
    u = _field(seed, 0, nx, ny, nz, R, ldx, -1.0, 1.0, backend, device)
    u_prev = u.copy() if backend == "numpy" else u.clone()
    coeffs = None
    if stencil == 1:
        offs = [_field(seed, 1 + m, nx, ny, nz, R, ldx, 0.0, 1.0 / 7.0, backend, device) for m in range(1, 7)]
        s = offs[0]
        for m in range(1, 6):
            s = s + offs[m]
        c0 = 1.0 - s
        lib = np if backend == "numpy" else __import__("torch")
        c0 = c0 * _interior_mask(nx, ny, nz, R, ldx, backend, device)
        coeffs = lib.stack([c0] + offs)
    elif stencil == 3:
        grids = [_field(seed, 1 + m, nx, ny, nz, R, ldx, 0.0, 0.01, backend, device) for m in range(13)]
        lib = np if backend == "numpy" else __import__("torch")
        coeffs = lib.stack(grids)
    elif stencil == 4:
        lib = np if backend == "numpy" else __import__("torch")
        coeffs = lib.stack([_field(seed, 1, nx, ny, nz, R, ldx, 0.5, 1.0, backend, device)])
    c = CONST_COEFFS.get(stencil, ())
    return u, u_prev, coeffs, c


def _interior_mask(nx, ny, nz, R, ldx, backend, device):
    shape = padded_shape(nx, ny, nz, R, ldx)
    if backend == "numpy":
        m = np.zeros(shape)
        m[R:R + nz, R:R + ny, R:R + nx] = 1.0
        return m
    import torch
    m = torch.zeros(shape, dtype=torch.float64, device=device)
    m[R:R + nz, R:R + ny, R:R + nx] = 1.0
    return m
