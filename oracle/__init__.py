"""FP64 CPU oracle for the reactive-diffusion LBM of arXiv:1410.1914 (D3Q7 and
the paper's D3Q19 lattice).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.  It shares no
code with the CUDA path.  The arithmetic lives in ``oracle_lbm.c`` (plain C,
double precision, optionally OpenMP over cells); this module only loads it
and marshals numpy arrays.

What each function follows:
  volume_fractions     Eq. 1-4 (Sec. 2.1.1)
  pt_loading           Eq. 5
  bulk_diffusivity     Eq. 7
  knudsen_diffusivity  Eq. 8
  bosanquet            Eq. 9
  chord_counts         Sec. 2.1.3, 13-direction pore length
  active_mask          Sec. 2.1.3 connectivity, as a 6-connected flood from
                       the inlet plane
  phase_connectivity   Sec. 2.1.3 connected-phase labelling (26 or 6
                       neighbours), transport / dead portions, surface area
  OracleLBM            Eq. 21, 23, 24 on D3Q7 or D3Q19 (Eq. 22); boundaries of Sec. 3.5;
                       Eq. 19 readout; Eq. 17b/18a kinetics as a surface sink
                       (per-cell rate factor for a non-uniform potential);
                       the a_i S source term of Eq. 21 (Eq. 16)
  steady.solve         the exact steady state: the fixed point of one step,
                       (I - A) x = S(0), by a sparse direct solve
  coupled.solve        Sec. 3.3-3.4: O2 in the ionomer, protons (Eq. 16) and
                       the potential-dependent Tafel rate (Eq. 17b, 18b)

Arrays are numpy with shape (nz, ny, nx), x fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_lbm.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle_lbm.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx_m", ctypes.c_double), ("T_K", ctypes.c_double), ("p_atm", ctypes.c_double),
        ("M_kgmol", ctypes.c_double), ("D_bulk", ctypes.c_double),
        ("D_ionomer", ctypes.c_double), ("k_ms", ctypes.c_double),
        ("knudsen", ctypes.c_int), ("bc_in", ctypes.c_int), ("bc_out", ctypes.c_int),
        ("c_in", ctypes.c_double), ("c_out", ctypes.c_double), ("tau_ref", ctypes.c_double),
        ("carrier", ctypes.c_int), ("lattice", ctypes.c_int), ("ionomer_o2", ctypes.c_int),
    ]


_D = ctypes.c_double
_P = ctypes.c_void_p
_L = ctypes.c_long


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            sig = {
                "orc_volume_fractions": (None, [_D, _D, _D, _D, _D, _D, _P]),
                "orc_pt_loading": (_D, [_D, _D, _D]),
                "orc_bulk_diffusivity": (_D, [_D, _D]),
                "orc_knudsen_diffusivity": (_D, [_D, _D, _D]),
                "orc_bosanquet": (_D, [_D, _D]),
                "orc_henry_constant": (_D, [_D]),
                "orc_ionomer_o2_diffusivity": (_D, [_D]),
                "orc_chord_counts": (None, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
                "orc_pore_diameter": (None, [_P, _L, _D, _P]),
                "orc_active_mask": (_L, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
                "orc_phase_connectivity": (None, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint,
                                                  ctypes.c_int, ctypes.c_int, _P, _P]),
                "orc_lbm_new": (_P, [ctypes.POINTER(_Params), _P, _P, _P]),
                "orc_lbm_free": (None, [_P]),
                "orc_lbm_init_field": (None, [_P, _P]),
                "orc_lbm_init_linear": (None, [_P]),
                "orc_lbm_step": (None, [_P, _L]),
                "orc_lbm_concentration": (None, [_P, _P]),
                "orc_lbm_populations": (None, [_P, _P]),
                "orc_lbm_set_populations": (None, [_P, _P]),
                "orc_lbm_set_kscale": (None, [_P, _P]),
                "orc_lbm_set_source": (None, [_P, _P]),
                "orc_lbm_cell_reaction": (None, [_P, _P]),
                "orc_lbm_fluxes": (None, [_P, _P]),
                "orc_lbm_effective_diffusivity": (None, [_P, _P]),
                "orc_lbm_reaction_rate": (_D, [_P, _P, _P]),
                "orc_lbm_current_density": (_D, [_P]),
                "orc_lbm_solve": (_L, [_P, _D, _L, _L]),
                "orc_lbm_n": (_L, [_P]),
                "orc_lbm_step_count": (_L, [_P]),
                "orc_lbm_dt": (_D, [_P]),
                "orc_lbm_D_b": (_D, [_P]),
                "orc_lbm_D_max": (_D, [_P]),
                "orc_lbm_k_lu": (_D, [_P]),
                "orc_lbm_get_tau": (None, [_P, _P]),
                "orc_lbm_get_D": (None, [_P, _P]),
                "orc_lbm_get_active": (None, [_P, _P]),
                "orc_lbm_get_react": (None, [_P, _P]),
                "orc_lbm_q": (ctypes.c_int, [_P]),
                "orc_num_threads": (ctypes.c_int, []),
                "orc_set_num_threads": (ctypes.c_int, [ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> int:
    """OpenMP threads of the oracle's later loops (n > 0); returns the count."""
    return lib().orc_set_num_threads(int(n))


# ---------------------------------------------------------------- formulas
def volume_fractions(eps, beta_N=0.3, theta_Pt=0.4, rho_N=2000.0, rho_C=1800.0, rho_Pt=21450.0):
    """Eq. 4a-4c: (eps_N, eps_C, eps_Pt)."""
    out = np.zeros(3)
    lib().orc_volume_fractions(eps, beta_N, theta_Pt, rho_N, rho_C, rho_Pt, _ptr(out))
    return tuple(float(v) for v in out)


def pt_loading(eps_Pt, rho_Pt_mg_cm3, l_cm):
    """Eq. 5: gamma_Pt [mg/cm^2]."""
    return lib().orc_pt_loading(eps_Pt, rho_Pt_mg_cm3, l_cm)


def bulk_diffusivity(T_K, p_atm):
    """Eq. 7 [m^2/s]."""
    return lib().orc_bulk_diffusivity(T_K, p_atm)


def knudsen_diffusivity(d_p_m, T_K, M_kgmol=0.032):
    """Eq. 8 [m^2/s]."""
    return lib().orc_knudsen_diffusivity(d_p_m, T_K, M_kgmol)


def bosanquet(D_kn, D_b):
    """Eq. 9 [m^2/s]."""
    return lib().orc_bosanquet(D_kn, D_b)


def henry_constant(T_K):
    """Eq. 11 [Pa m^3/mol]."""
    return lib().orc_henry_constant(T_K)


def ionomer_o2_diffusivity(T_K):
    """Eq. 13 [m^2/s]."""
    return lib().orc_ionomer_o2_diffusivity(T_K)


def chord_counts(phase: np.ndarray) -> np.ndarray:
    """13-direction pore run lengths in cells, shape (nz, ny, nx, 13)."""
    phase = np.ascontiguousarray(phase, dtype=np.uint8)
    nz, ny, nx = phase.shape
    out = np.zeros((nz, ny, nx, 13), dtype=np.int32)
    lib().orc_chord_counts(_ptr(phase), nx, ny, nz, _ptr(out))
    return out


def pore_diameter(phase: np.ndarray, dx_m: float) -> np.ndarray:
    """Sec. 2.1.3 13-direction mean pore length [m] (0 for non-pore cells)."""
    counts = chord_counts(phase)
    out = np.zeros(phase.shape, dtype=np.float64)
    lib().orc_pore_diameter(_ptr(counts), out.size, dx_m, _ptr(out))
    return out


def active_mask(phase: np.ndarray, ionomer_transport: bool = False, protons: bool = False) -> np.ndarray:
    """Transport cells 6-connected to the inlet plane x = 0 (y, z periodic).
    Transport phases: pore and micropore (+ ionomer if ionomer_transport);
    ionomer alone if protons (Eq. 16)."""
    phase = np.ascontiguousarray(phase, dtype=np.uint8)
    nz, ny, nx = phase.shape
    out = np.zeros(phase.shape, dtype=np.uint8)
    mode = 2 if protons else int(bool(ionomer_transport))
    lib().orc_active_mask(_ptr(phase), nx, ny, nz, mode, _ptr(out))
    return out


STAT_KEYS = ("n_cells", "n_portions", "n_transport_portions", "n_transport_cells", "surface_faces",
             "transport_surface_faces", "largest_portion")


def phase_connectivity(phase: np.ndarray, phase_set, neighbours: int = 26, periodic_yz: bool = False):
    """Sec. 2.1.3 connected-phase labelling of the cells whose code is in
    ``phase_set`` (iterable of codes): (labels, stats).  labels (int32, shape
    of phase): the smallest cell index of the cell's portion, -1 outside the
    set.  stats: dict with STAT_KEYS (portions, "transport" portions touching
    both x end planes, their cells, surface faces to other phases, largest
    portion)."""
    phase = np.ascontiguousarray(phase, dtype=np.uint8)
    nz, ny, nx = phase.shape
    mask = 0
    for k in phase_set:
        mask |= 1 << int(k)
    labels = np.zeros(phase.shape, dtype=np.int32)
    out = np.zeros(7, dtype=np.int64)
    lib().orc_phase_connectivity(_ptr(phase), nx, ny, nz, mask, int(neighbours), int(bool(periodic_yz)),
                                 _ptr(labels), _ptr(out))
    return labels, {k: int(v) for k, v in zip(STAT_KEYS, out)}


# ---------------------------------------------------------------- solver
DEFAULTS = dict(dx_m=2e-9, T_K=353.0, p_atm=1.0, M_kgmol=0.032, D_bulk=0.0, D_ionomer=0.0,
                k_ms=0.0, knudsen=0, bc_in=0, bc_out=0, c_in=1.0, c_out=0.0, tau_ref=1.0, carrier=0,
                lattice=0, ionomer_o2=0)


class OracleLBM:
    """Double-precision BGK solver (Eq. 21-24) on D3Q7 (``lattice=0``) or the
    paper's D3Q19 (``lattice=1``, Eq. 22-23).

    ``phase`` (nz, ny, nx) uint8 codes 0 pore / 1 solid / 2 ionomer /
    3 micropore.  ``react`` (same shape, uint8): bit f marks the face toward
    x + e_f as catalytic (f = 0..5 = +x, -x, +y, -y, +z, -z).
    ``D`` (same shape, float64): per-cell diffusivity override [m^2/s].
    ``react()`` returns the derived per-link bits (uint32, bit i-1 = link
    toward x + c_i reacts).
    """

    def __init__(self, phase, react=None, D=None, **params):
        p = dict(DEFAULTS)
        p.update(params)
        self.phase = np.ascontiguousarray(phase, dtype=np.uint8)
        nz, ny, nx = self.phase.shape
        self.shape = (nz, ny, nx)
        self.params = p
        cp = _Params(nx, ny, nz, p["dx_m"], p["T_K"], p["p_atm"], p["M_kgmol"], p["D_bulk"],
                     p["D_ionomer"], p["k_ms"], int(p["knudsen"]), int(p["bc_in"]), int(p["bc_out"]),
                     p["c_in"], p["c_out"], p["tau_ref"], int(p["carrier"]), int(p["lattice"]),
                     int(p["ionomer_o2"]))
        if int(p["ionomer_o2"]) and (int(p["carrier"]) != 0 or not ionomer_o2_diffusivity(p["T_K"]) > 0):
            raise ValueError("ionomer_o2 needs the O2 carrier and T_K > 283.7 K (Eq. 13)")
        if int(p["lattice"]) not in (0, 1):
            raise ValueError("lattice must be 0 (D3Q7) or 1 (D3Q19)")
        if int(p["carrier"]) == 1 and not (p["D_ionomer"] > 0 and p["k_ms"] == 0):
            raise ValueError("protons (carrier 1) need D_ionomer > 0 (the conductivity) and k_ms = 0")
        self._react = None if react is None else np.ascontiguousarray(react, dtype=np.uint8)
        self._Dov = None if D is None else np.ascontiguousarray(D, dtype=np.float64)
        h = lib().orc_lbm_new(ctypes.byref(cp), _ptr(self.phase),
                              None if self._react is None else _ptr(self._react),
                              None if self._Dov is None else _ptr(self._Dov))
        if not h:
            raise ValueError("no transport cell is connected to the inlet plane")
        self._h = h
        self.q = lib().orc_lbm_q(h)
        self.init_linear()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_lbm_free(h)
            self._h = None

    # state
    def init_linear(self):
        lib().orc_lbm_init_linear(self._h)

    def init_field(self, C):
        C = np.ascontiguousarray(C, dtype=np.float64).reshape(self.shape)
        lib().orc_lbm_init_field(self._h, _ptr(C))

    def step(self, n: int = 1):
        lib().orc_lbm_step(self._h, int(n))

    def solve(self, tol=1e-8, check_every=100, max_steps=10_000_000):
        return lib().orc_lbm_solve(self._h, tol, int(check_every), int(max_steps))

    # readouts
    def concentration(self):
        out = np.zeros(self.shape)
        lib().orc_lbm_concentration(self._h, _ptr(out))
        return out

    def populations(self):
        out = np.zeros((self.q,) + self.shape)
        lib().orc_lbm_populations(self._h, _ptr(out))
        return out

    def set_populations(self, g):
        """Replace the pre-collision populations, shape (q, nz, ny, nx);
        entries of inactive cells are ignored (kept 0)."""
        g = np.ascontiguousarray(g, dtype=np.float64).reshape((self.q,) + self.shape)
        lib().orc_lbm_set_populations(self._h, _ptr(g))

    def set_rate_scale(self, k):
        """Per-cell factor on the rate constant k of the catalytic faces
        (Eq. 17b with a non-uniform potential); None restores uniform k."""
        if k is None:
            self._kscale = None
            lib().orc_lbm_set_kscale(self._h, None)
            return
        self._kscale = np.ascontiguousarray(k, dtype=np.float64).reshape(self.shape)
        lib().orc_lbm_set_kscale(self._h, _ptr(self._kscale))

    def set_source(self, S):
        """Per-cell amount added to C per step in lattice units (the source
        of Eq. 16, entering as w_i S after collision); None removes it."""
        if S is None:
            lib().orc_lbm_set_source(self._h, None)
            return
        S = np.ascontiguousarray(S, dtype=np.float64).reshape(self.shape)
        lib().orc_lbm_set_source(self._h, _ptr(S))

    def cell_reaction(self):
        """Amount consumed per step on each cell's reactive links (lattice units)."""
        out = np.zeros(self.shape)
        lib().orc_lbm_cell_reaction(self._h, _ptr(out))
        return out

    def fluxes(self):
        out = np.zeros(5)
        lib().orc_lbm_fluxes(self._h, _ptr(out))
        return dict(J_in=out[0], J_out=out[1], R=out[2], sum_C=out[3], n_active=int(out[4]))

    def effective_diffusivity(self):
        """Eq. 19: (D_eff [m^2/s], D_eff / D_b, D_eff in lattice units)."""
        out = np.zeros(3)
        lib().orc_lbm_effective_diffusivity(self._h, _ptr(out))
        return float(out[0]), float(out[1]), float(out[2])

    def reaction_rate(self):
        """(total [C*m^3/s], per-plane rate (nx,), per-plane mean C (nx,))."""
        nx = self.shape[2]
        pr = np.zeros(nx)
        pc = np.zeros(nx)
        tot = lib().orc_lbm_reaction_rate(self._h, _ptr(pr), _ptr(pc))
        return float(tot), pr, pc

    def current_density(self):
        """Eq. 25: i_d = 4 F R / A_cross [A/m^2]."""
        return lib().orc_lbm_current_density(self._h)

    # scalars and maps
    @property
    def steps(self):
        return lib().orc_lbm_step_count(self._h)

    @property
    def dt(self):
        return lib().orc_lbm_dt(self._h)

    @property
    def D_b(self):
        return lib().orc_lbm_D_b(self._h)

    @property
    def D_max(self):
        return lib().orc_lbm_D_max(self._h)

    @property
    def k_lu(self):
        return lib().orc_lbm_k_lu(self._h)

    def tau(self):
        out = np.zeros(self.shape)
        lib().orc_lbm_get_tau(self._h, _ptr(out))
        return out

    def D(self):
        out = np.zeros(self.shape)
        lib().orc_lbm_get_D(self._h, _ptr(out))
        return out

    def active(self):
        out = np.zeros(self.shape, dtype=np.uint8)
        lib().orc_lbm_get_active(self._h, _ptr(out))
        return out

    def react(self):
        out = np.zeros(self.shape, dtype=np.uint32)
        lib().orc_lbm_get_react(self._h, _ptr(out))
        return out
