"""Catalyst-layer structures on the GPU (argument marshalling only).

The same recipes as the host generator of the ``inputs`` module -- the Pt
layer of Sec. 2.1.2 (QSGS solid, then ionomer grown on it), the NPMC layer
of Sec. 2.2 / 5.3 (micropores carved into solid that touches no ionomer) and
the reactive-face sampling -- run by the CUDA library and bit-identical to
the host results, plus the connected-phase statistics of Sec. 2.1.3.  Every
function takes and returns CUDA uint8 tensors of shape (nz, ny, nx).
"""
from __future__ import annotations

from . import _lib as L

PORE, SOLID, IONOMER, MICROPORE = 0, 1, 2, 3
PHASE_SETS = {"C/Pt": (SOLID,), "void": (PORE, MICROPORE), "ionomer": (IONOMER,)}


def _bits(codes) -> int:
    m = 0
    for c in codes:
        m |= 1 << int(c)
    return m


def pt_cl(shape, seed: int, pore: float, ionomer: float, c_d: float = 0.01, p_alpha: float = 0.01,
          device="cuda"):
    """Pt catalyst layer (same recipe and result as inputs.pt_cl)."""
    import torch
    nz, ny, nx = shape
    N = nx * ny * nz
    ph = torch.zeros(shape, dtype=torch.uint8, device=device)
    n_solid = int(round((1.0 - pore - ionomer) * N))
    n_ion = int(round(ionomer * N))
    L.cl_qsgs_grow(ph, SOLID, _bits([PORE]), _bits([SOLID]), n_solid, c_d, p_alpha, seed, 1)
    L.cl_qsgs_grow(ph, IONOMER, _bits([PORE]), _bits([SOLID, IONOMER]), n_ion, 0.0, p_alpha, seed, 2)
    return ph


def npmc_cl(shape, seed: int, base_pore: float, ionomer: float, total_pore: float, c_d: float = 0.01,
            p_alpha: float = 0.01, micro_c_d: float = 0.05, micro_p_alpha: float = 0.02, device="cuda"):
    """NPMC layer (same recipe and result as inputs.npmc_cl)."""
    import torch
    ph = pt_cl(shape, seed, base_pore, ionomer, c_d, p_alpha, device)
    region = torch.empty_like(ph)
    L.cl_qsgs_region_not_adjacent(ph, SOLID, IONOMER, region)
    n_micro = int(round((total_pore - base_pore) * ph.numel()))
    L.cl_qsgs_grow(ph, MICROPORE, _bits([SOLID]), _bits([MICROPORE]), n_micro, micro_c_d, micro_p_alpha, seed, 3,
                   region=region)
    return ph


def reactive_faces(phase, fraction: float, seed: int, from_code: int = PORE, to_code: int = SOLID):
    """Face bits on from_code cells toward to_code neighbours, each kept with `fraction`."""
    import torch
    out = torch.empty_like(phase)
    L.cl_qsgs_reactive_faces(phase, from_code, to_code, fraction, seed, out)
    return out


def connectivity(phase, neighbours: int = 26, periodic_yz: bool = False) -> dict:
    """Sec. 2.1.3 statistics of the three phases: {name: stats}."""
    return {name: L.cl_phase_connectivity(phase, codes, neighbours, periodic_yz)
            for name, codes in PHASE_SETS.items()}
