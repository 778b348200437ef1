"""Exact steady state of the oracle's scheme by a sparse direct solve.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

The steady state of the march (Eq. 21-24 with the boundaries of Sec. 3.5)
is the fixed point x = S(x) of one step on the populations.  S is affine,
S(x) = A x + b with b = S(0), so the fixed point solves (I - A) x = b.
This module writes that definition out: it assembles A column by column
from the oracle's own step and hands (I - A) x = b to a sparse LU
factorisation (the library routine serving as the one step).  It reaches
the steady state of cases the march cannot finish in reasonable time, such
as O2 dissolved in the ionomer (relaxation times within 1e-5 of 1/2).

Assembly by probing: one step moves populations by at most one cell in x,
y and z, so cells whose (x, y, z) agree modulo 3 never feed the same output
entry.  One probe per (colour, population) -- 27 q probes in all -- sets
population i of every cell of one colour to 1; the output entry (j, c') of
that probe is A[(j, c'), (i, c)] for the one cell c of that colour in the
3 x 3 x 3 neighbourhood of c'.  The y and z extents must be multiples of 3
(or at most 3) so that the periodic wrap keeps same-colour cells 3 apart.
"""
from __future__ import annotations

import numpy as np


def step_matrix(o):
    """(A, b): the linear part of one step of OracleLBM `o` as a sparse CSR
    matrix over the q * nz * ny * nx populations (layout [q][z][y][x]) and
    b = S(0).  The state of `o` is left at S(0)."""
    import scipy.sparse as sp

    q = o.q
    nz, ny, nx = o.shape
    for n in (ny, nz):
        if n > 3 and n % 3:
            raise ValueError("the y and z extents must be multiples of 3 (or at most 3)")
    shape = (q, nz, ny, nx)
    N = nz * ny * nx
    o.set_populations(np.zeros(shape))
    o.step(1)
    b = o.populations().ravel().copy()
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    colour = (x % 3) + 3 * (y % 3) + 9 * (z % 3)
    cell = np.arange(N).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    for col in range(27):
        cx, cy, cz = col % 3, (col // 3) % 3, col // 9
        # for every output cell, the source cell of this colour in its neighbourhood (or none)
        src = -np.ones((nz, ny, nx), np.int64)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    sx, sy, sz = x + dx, (y + dy) % ny, (z + dz) % nz
                    ok = (sx >= 0) & (sx < nx) & (sx % 3 == cx) & (sy % 3 == cy) & (sz % 3 == cz)
                    src = np.where(ok & (src < 0), cell[sz, sy, np.clip(sx, 0, nx - 1)], src)
        mask = (colour == col).astype(np.float64)
        if not mask.any():
            continue
        for i in range(q):
            probe = np.zeros(shape)
            probe[i] = mask
            o.set_populations(probe)
            o.step(1)
            out = o.populations().reshape(q, N) - b.reshape(q, N)
            jj, cc = np.nonzero(np.abs(out) > 0)
            s = src.ravel()[cc]
            keep = s >= 0
            rows.append(jj[keep] * N + cc[keep])
            cols.append(i * N + s[keep])
            vals.append(out[jj[keep], cc[keep]])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(q * N, q * N))
    o.set_populations(b.reshape(shape))
    return A, b


def solve(o, A=None):
    """Set `o` to the exact fixed point of its step, (I - A) x = S(0), and
    return it (shape (q, nz, ny, nx)).  Inactive cells stay 0.  Pass A
    from step_matrix to reuse it when only the sources or boundary values
    changed."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import spsolve

    shape = (o.q,) + o.shape
    if A is None:
        A, b = step_matrix(o)
    else:
        o.set_populations(np.zeros(shape))
        o.step(1)
        b = o.populations().ravel().copy()
    n = A.shape[0]
    x = spsolve((sp.identity(n, format="csc") - A.tocsc()), b)
    o.set_populations(x.reshape(shape))
    return x.reshape(shape)
