"""Seeded synthetic catalyst-layer structures (input generation only).

The structures stand in for the paper's reconstructed catalyst layers
(arXiv:1410.1914, Sec. 2): pore / solid (carbon + Pt, or the NPMC solid) /
ionomer voxels grown by QSGS (Sec. 2.1.2), with reactive faces sampled on
solid-pore interfaces (Pt layer, Sec. 2.1.2.2) or placed on every
solid-pore face (NPMC layer, Sec. 2.2), and micropores carved into the solid
away from the ionomer (Sec. 5.3).  This module holds none of the solver's
arithmetic; the CUDA path's callers and the CPU oracle's tests both read the
arrays it returns.

Phase codes: 0 pore, 1 solid, 2 ionomer, 3 micropore.  Arrays have shape
(nz, ny, nx), x fastest.  Reactive-face bytes: bit d-1 marks the face toward
x + c_d, d = 1..6 = +x, -x, +y, -y, +z, -z.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsgs.c")
_LIB = os.path.join(_HERE, "libqsgs.so")
_lock = threading.Lock()
_lib = None

PORE, SOLID, IONOMER, MICROPORE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P, I, U8, U32, U64, D, LL = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint8, ctypes.c_uint32,
                                         ctypes.c_uint64, ctypes.c_double, ctypes.c_long)
            L.qsgs_grow.restype = LL
            L.qsgs_grow.argtypes = [P, I, I, I, U8, U32, U32, P, LL, D, D, U64, U64, I]
            L.qsgs_reactive_faces.restype = LL
            L.qsgs_reactive_faces.argtypes = [P, I, I, I, U8, U8, D, U64, P]
            L.qsgs_region_not_adjacent.restype = None
            L.qsgs_region_not_adjacent.argtypes = [P, I, I, I, U8, U8, P]
            L.qsgs_hash4.restype = U64
            L.qsgs_hash4.argtypes = [U64, U64, U64, U64]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def grow(phase: np.ndarray, code: int, allowed, grown, target: int, c_d: float, p_alpha: float,
         seed: int, stream: int, region: np.ndarray | None = None, max_sweeps: int = 100000) -> int:
    """QSGS growth of `code` in place until `target` cells carry it."""
    assert phase.dtype == np.uint8 and phase.flags.c_contiguous
    nz, ny, nx = phase.shape
    am = sum(1 << a for a in allowed)
    gm = sum(1 << g for g in grown) | (1 << code)
    reg = None if region is None else np.ascontiguousarray(region, dtype=np.uint8)
    return _L().qsgs_grow(_p(phase), nx, ny, nz, code, am, gm, None if reg is None else _p(reg),
                          int(target), float(c_d), float(p_alpha), seed & (2**64 - 1),
                          stream & (2**64 - 1), max_sweeps)


def reactive_faces(phase: np.ndarray, fraction: float, seed: int, from_code: int = PORE,
                   to_code: int = SOLID) -> np.ndarray:
    """Face bits on `from_code` cells toward `to_code` neighbours, each kept with `fraction`."""
    phase = np.ascontiguousarray(phase, dtype=np.uint8)
    nz, ny, nx = phase.shape
    out = np.zeros_like(phase)
    _L().qsgs_reactive_faces(_p(phase), nx, ny, nz, from_code, to_code, float(fraction),
                             seed & (2**64 - 1), _p(out))
    return out


def hash4(seed: int, stream: int, a: int, b: int) -> int:
    return int(_L().qsgs_hash4(seed, stream, a, b))


def pt_cl(shape, seed: int, pore: float, ionomer: float, c_d: float = 0.01,
          p_alpha: float = 0.01) -> np.ndarray:
    """Pt catalyst layer: QSGS solid (carbon + Pt) then QSGS ionomer grown on it.

    `pore`, `ionomer` are volume fractions; solid = 1 - pore - ionomer.
    """
    nz, ny, nx = shape
    N = nx * ny * nz
    ph = np.zeros(shape, dtype=np.uint8)
    n_solid = int(round((1.0 - pore - ionomer) * N))
    n_ion = int(round(ionomer * N))
    grow(ph, SOLID, allowed=[PORE], grown=[SOLID], target=n_solid, c_d=c_d, p_alpha=p_alpha,
         seed=seed, stream=1)
    # ionomer: the solid cells act as the seeds (Sec. 2.1.2.3)
    grow(ph, IONOMER, allowed=[PORE], grown=[SOLID, IONOMER], target=n_ion, c_d=0.0,
         p_alpha=p_alpha, seed=seed, stream=2)
    return ph


def npmc_cl(shape, seed: int, base_pore: float, ionomer: float, total_pore: float,
            c_d: float = 0.01, p_alpha: float = 0.01, micro_c_d: float = 0.05,
            micro_p_alpha: float = 0.02) -> np.ndarray:
    """NPMC layer: the Pt-layer structure, then micropores (phase 3) carved
    into solid cells that touch no ionomer until pore + micropore = total_pore."""
    ph = pt_cl(shape, seed, base_pore, ionomer, c_d, p_alpha)
    N = ph.size
    region = np.zeros_like(ph)
    nz, ny, nx = ph.shape
    _L().qsgs_region_not_adjacent(_p(ph), nx, ny, nz, SOLID, IONOMER, _p(region))
    n_micro = int(round((total_pore - base_pore) * N))
    grow(ph, MICROPORE, allowed=[SOLID], grown=[MICROPORE], target=n_micro, c_d=micro_c_d,
         p_alpha=micro_p_alpha, seed=seed, stream=3, region=region)
    return ph


def with_reservoir(phase: np.ndarray) -> np.ndarray:
    """The gas reservoir of Sec. 3.5.2: the first x-plane made pore-only."""
    ph = phase.copy()
    ph[:, :, 0] = PORE
    return ph


# -------------------------------------------------------------- workloads
# Volume fractions of the 256^3 layer come from Eq. 4 at porosity 0.45 with
# beta_N = 0.3, theta_Pt = 0.4 and the densities of Sec. 2.1.3 (tests check
# these literals against the oracle's Eq. 4).
EQ4_EPS045_IONOMER = 0.188743
EQ4_EPS045_SOLID = 0.361257

# Eq. 4 makes the ionomer share of the non-pore volume independent of the
# porosity (beta_N = 0.3, theta_Pt = 0.4): eps_N / (1 - eps) = 0.343169
# (tests check this literal against the oracle's Eq. 4).
EQ4_IONOMER_SHARE = 0.343169

WORKLOADS = {
    # plain method, small
    "pt_cl_48": dict(shape=(48, 48, 48), seed=0, kind="pt", pore=0.50, ionomer=0.20, c_d=0.01,
                     params=dict(dx_m=2e-9, knudsen=0, T_K=353.0, p_atm=1.0, M_kgmol=0.032,
                                 bc_in=0, bc_out=0, c_in=1.0, c_out=0.0, tau_ref=1.0)),
    # Pt layer, Knudsen, 5 % reactive carbon-pore faces, k = 1e-3 m/s
    "pt_cl_256": dict(shape=(256, 256, 256), seed=1, kind="pt", pore=0.45,
                      ionomer=EQ4_EPS045_IONOMER, c_d=0.01, react_fraction=0.05,
                      params=dict(dx_m=2e-9, knudsen=1, T_K=353.0, p_atm=1.0, M_kgmol=0.032,
                                  k_ms=1e-3, bc_in=0, bc_out=1, c_in=1.0, c_out=0.0, tau_ref=1.0)),
    # NPMC layer with micropores, every solid-pore face reactive, k = 1e-5 m/s
    "npmc_cl_400": dict(shape=(400, 400, 400), seed=2, kind="npmc", pore=0.45,
                        ionomer=EQ4_EPS045_IONOMER, total_pore=0.55, c_d=0.01, react_fraction=1.0,
                        params=dict(dx_m=1e-9, knudsen=1, T_K=353.0, p_atm=1.0, M_kgmol=0.032,
                                    k_ms=1e-5, bc_in=0, bc_out=1, c_in=1.0, c_out=0.0, tau_ref=1.0)),
}


def make_workload(name: str, shape=None, seed=None, reactive: bool | None = None):
    """(phase, reactive_faces or None, params) for a named workload.

    `shape`/`seed` override the defaults (smaller instances of the same
    recipe for tests).  Reactive workloads get the reservoir plane and a
    zero-flux outlet; `reactive=False` gives the D_eff variant (Dirichlet
    at both ends, no reaction)."""
    w = WORKLOADS[name]
    shape = tuple(shape or w["shape"])
    seed = w["seed"] if seed is None else seed
    params = dict(w["params"])
    if w["kind"] == "pt":
        ph = pt_cl(shape, seed, w["pore"], w["ionomer"], w["c_d"])
    else:
        ph = npmc_cl(shape, seed, w["pore"], w["ionomer"], w["total_pore"], w["c_d"])
    is_reactive = ("react_fraction" in w) if reactive is None else reactive
    react = None
    if is_reactive:
        ph = with_reservoir(ph)
        react = reactive_faces(ph, w["react_fraction"], seed)
        params["bc_out"] = 1
    else:
        params["bc_out"] = 0
        params["k_ms"] = 0.0
    return ph, react, params


def batch_workloads(n: int = 64, seed0: int = 100, edge_range=(32, 160), eps_range=(0.35, 0.65),
                    dx_m: float = 2e-9):
    """Many small structures of uneven size (the batched-launch workload).

    Member i: a cube of edge uniform in edge_range, porosity uniform in
    eps_range, Pt layer for even i and NPMC layer (5 % of the volume carved
    as micropores) for odd i; Knudsen diffusivity at 353 K; D_eff set-up
    (fixed concentrations 1 and 0 at the x faces, no reaction).
    Returns a list of (phase, None, params)."""
    out = []
    for i in range(n):
        seed = seed0 + i
        u1 = hash4(seed, 0xBA7C, 1, 0) / 2.0**64
        u2 = hash4(seed, 0xBA7C, 2, 0) / 2.0**64
        L = edge_range[0] + int(u1 * (edge_range[1] - edge_range[0] + 1))
        eps = eps_range[0] + u2 * (eps_range[1] - eps_range[0])
        ion = (1.0 - eps) * EQ4_IONOMER_SHARE
        if i % 2 == 0:
            ph = pt_cl((L, L, L), seed, eps, ion)
        else:
            base = max(eps - 0.05, 0.05)
            ph = npmc_cl((L, L, L), seed, base, (1.0 - base) * EQ4_IONOMER_SHARE, eps)
        params = dict(dx_m=dx_m, knudsen=1, T_K=353.0, p_atm=1.0, M_kgmol=0.032, bc_in=0, bc_out=0,
                      c_in=1.0, c_out=0.0, tau_ref=1.0, k_ms=0.0)
        out.append((ph, None, params))
    return out
