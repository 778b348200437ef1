"""The seeded structure generator (Sec. 2.1.2 QSGS, Sec. 5.3 micropores, the
reactive-face sampling) checked for the properties its reading promises:
exact phase counts, growth only by adjacency, ionomer only on the solid,
micropores only in solid that touches no ionomer, faces only where a pore
cell meets solid, and results that do not depend on the thread count.
The GPU generator is compared with this one byte for byte
(tests/test_gpu_structures.py)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1410_1914_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PORE, SOLID, IONOMER, MICRO = 0, 1, 2, 3


def _neighbours(mask):
    """Number of the 6 neighbours (all axes periodic) for which mask holds."""
    n = np.zeros(mask.shape, np.int32)
    for ax in range(3):
        for sh in (1, -1):
            n += np.roll(mask, sh, axis=ax)
    return n


@pytest.mark.parametrize("shape,seed,pore,ion", [((20, 24, 28), 1, 0.45, 0.19), ((16, 16, 40), 2, 0.6, 0.12)])
def test_pt_layer_counts_and_adjacency(shape, seed, pore, ion):
    ph = inputs.pt_cl(shape, seed, pore, ion)
    N = ph.size
    assert (ph == SOLID).sum() == round((1 - pore - ion) * N)
    assert (ph == IONOMER).sum() == round(ion * N)
    assert set(np.unique(ph)) <= {PORE, SOLID, IONOMER}
    # the ionomer has no seeds (c_d = 0): every ionomer cell grew next to solid or ionomer
    grown = (ph == SOLID) | (ph == IONOMER)
    assert np.all(_neighbours(grown)[ph == IONOMER] >= 1)


def test_solid_growth_from_seeds_only():
    """With P_alpha = 0 a cell joins only with two grown neighbours (rule
    2a): from isolated seeds nothing can grow, so the phase stays at its
    seeds, each drawn with probability c_d."""
    ph = np.zeros((24, 24, 24), np.uint8)
    n = inputs.grow(ph, SOLID, allowed=[PORE], grown=[SOLID], target=ph.size, c_d=0.002, p_alpha=0.0, seed=5,
                    stream=1, max_sweeps=50)
    seeds = (ph == SOLID)
    assert n == seeds.sum() > 0
    assert abs(n - 0.002 * ph.size) < 5 * np.sqrt(0.002 * ph.size)
    # no cell has two seed neighbours (rule 2a would have taken it in the first sweep)
    assert np.all(_neighbours(seeds)[~seeds] <= 1)


def test_npmc_micropores_avoid_ionomer():
    ph = inputs.npmc_cl((24, 24, 32), 3, 0.45, inputs.EQ4_EPS045_IONOMER, 0.55)
    micro = ph == MICRO
    assert micro.sum() == round(0.10 * ph.size)
    assert np.all(_neighbours(ph == IONOMER)[micro] == 0)


def test_reactive_faces_lie_on_pore_solid_faces():
    ph = inputs.pt_cl((12, 14, 20), 4, 0.5, 0.15)
    full = inputs.reactive_faces(ph, 1.0, 0)
    # bit d: the face toward +x, -x, +y, -y, +z, -z, as (dz, dy, dx) steps
    dirs = [(0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)]
    expect = np.zeros(ph.shape, np.uint8)
    for d, (dz, dy, dx) in enumerate(dirs):
        nb = np.roll(ph, (-dz, -dy, -dx), axis=(0, 1, 2))
        ok = (ph == PORE) & (nb == SOLID)
        if dx == 1:
            ok[:, :, -1] = False   # x is not periodic
        if dx == -1:
            ok[:, :, 0] = False
        expect |= (ok.astype(np.uint8) << d)
    np.testing.assert_array_equal(full, expect)
    some = inputs.reactive_faces(ph, 0.05, 9)
    assert np.all((some & ~full) == 0)
    n_full = int(np.unpackbits(full).sum())
    n_some = int(np.unpackbits(some).sum())
    assert abs(n_some - 0.05 * n_full) < 5 * np.sqrt(0.05 * n_full)


def test_reservoir_plane():
    ph = inputs.with_reservoir(inputs.pt_cl((8, 8, 12), 6, 0.4, 0.2))
    assert np.all(ph[:, :, 0] == PORE)


def test_independent_of_thread_count():
    code = ("import sys, hashlib; sys.path.insert(0, %r)\n"
            "from paper_1410_1914_gb300 import inputs\n"
            "ph = inputs.npmc_cl((20, 22, 26), 7, 0.45, 0.19, 0.55)\n"
            "print(hashlib.sha256(ph.tobytes()).hexdigest())\n") % ROOT
    out = []
    for threads in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
        out.append(r.stdout.strip())
    assert out[0] == out[1]
