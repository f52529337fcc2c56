"""Brute-force per-point evaluator -- TEST INFRASTRUCTURE ONLY.

An independent restatement of the six operators of Listings 1-4 (arXiv 1510.04995, Sect. 2.2)
as a table of terms.  Each term is (coefficient source, list of neighbour offsets (dx, dy, dz));
a point's update is the running sum, in table order, of coefficient * (sum of the neighbours in
list order).  The 25-point stencil with the factor grid (Listing 3 as printed) uses the 25-point
constant table and multiplies the sum by the point's factor before the leapfrog terms.  The
27-point box operator (Sect. 8.4) groups its 26 neighbours by class (face, edge, corner).  Red-black
Gauss-Seidel is evaluated as Sect. 8.4 states it, in place on one array (``rbgs_in_place``), which
checks the oracle's two-buffer half-step form.  Every level is recomputed point by point over the whole interior in pure Python,
so it is only meant for tiny grids (8^3, T <= 3), where it must agree bit for bit with the C loop
nests (same terms, same order, one rounding per operation).
"""
from __future__ import annotations

import numpy as np


def _axis(r):
    return [(r, 0, 0), (-r, 0, 0)], [(0, r, 0), (0, -r, 0)], [(0, 0, r), (0, 0, -r)]


def term_table(stencil: int):
    """List of (("c", index) | ("C", grid), offsets).  'c' = constant coefficient, 'C' = grid."""
    if stencil == 0:
        x, y, z = _axis(1)
        return [(("c", 0), [(0, 0, 0)]), (("c", 1), x), (("c", 1), y), (("c", 1), z)]
    if stencil == 1:
        return [(("C", 0), [(0, 0, 0)]), (("C", 1), [(1, 0, 0)]), (("C", 2), [(-1, 0, 0)]),
                (("C", 3), [(0, 1, 0)]), (("C", 4), [(0, -1, 0)]), (("C", 5), [(0, 0, 1)]),
                (("C", 6), [(0, 0, -1)])]
    if stencil == 5:
        # box: centre, then the face, edge and corner classes, offsets in (dz, dy, dx) order
        offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        tab = [(("c", 0), [(0, 0, 0)])]
        for m in (1, 2, 3):
            tab.append((("c", m), [o for o in offs if sum(v != 0 for v in o) == m]))
        return tab
    if stencil in (2, 4):
        tab = [(("c", 0), [(0, 0, 0)])]
        for r in range(1, 5):
            x, y, z = _axis(r)
            tab.append((("c", r), x + y + z))
        return tab
    tab = [(("C", 0), [(0, 0, 0)])]
    g = 1
    for r in range(1, 5):
        for pair in _axis(r):
            tab.append((("C", g), pair))
            g += 1
    return tab


def rbgs_in_place(u, c, T: int):
    """Red-black Gauss-Seidel written the way Sect. 8.4 states it: ONE array, updated in place, half
    sweep t visiting the points with (x + y + z + t) even (interior coordinates) in lexicographic
    order and replacing each by c0*u + c1*(x pair) + c1*(y pair) + c1*(z pair) of the current
    array.  Returns (array after T half-sweeps, array after T-1)."""
    a = u.copy()
    prev = u.copy()
    nz, ny, nx = (s - 2 for s in u.shape)
    for t in range(T):
        prev = a.copy()
        for k in range(1, nz + 1):
            for j in range(1, ny + 1):
                for i in range(1, nx + 1):
                    if ((i - 1) + (j - 1) + (k - 1) + t) % 2:
                        continue
                    v = float(c[0]) * float(a[k, j, i])
                    v = v + float(c[1]) * (float(a[k, j, i + 1]) + float(a[k, j, i - 1]))
                    v = v + float(c[1]) * (float(a[k, j + 1, i]) + float(a[k, j - 1, i]))
                    v = v + float(c[1]) * (float(a[k + 1, j, i]) + float(a[k - 1, j, i]))
                    a[k, j, i] = v
    return a, prev


def sweep(stencil: int, u, u_prev, coeffs, c, T: int, R: int):
    """Return (level T, level T-1) as new arrays; inputs are padded [nz+2R][ny+2R][nx+2R]."""
    if stencil == 6:
        return rbgs_in_place(u, c, T)
    a = [u.copy(), u_prev.copy()]
    nz, ny, nx = (s - 2 * R for s in u.shape)
    second = stencil in (2, 3, 4)
    tab = term_table(stencil)
    for t in range(T):
        V, U = a[t % 2], a[(t + 1) % 2]
        new = U.copy()
        for k in range(R, R + nz):
            for j in range(R, R + ny):
                for i in range(R, R + nx):
                    acc = None
                    for (kind, q), offs in tab:
                        s = None
                        for dx, dy, dz in offs:
                            v = float(V[k + dz, j + dy, i + dx])
                            s = v if s is None else s + v
                        w = float(c[q]) if kind == "c" else float(coeffs[q, k, j, i])
                        term = w * s
                        acc = term if acc is None else acc + term
                    if stencil == 4:  # Listing 3's per-point factor on the whole bracket
                        acc = float(coeffs[0, k, j, i]) * acc
                    if second:
                        acc = (2.0 * float(V[k, j, i]) - float(U[k, j, i])) + acc
                    new[k, j, i] = acc
        a[(t + 1) % 2] = new
    if T % 2 == 1:
        a = [a[1], a[0]]
    return a[0], a[1]
