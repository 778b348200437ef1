"""Thin ctypes binding of the C ABI in include/cl_lbm.h.

Argument marshalling only: every step of the solver runs in libcllbm.so.
Functions keep the C names.  Array arguments may be numpy arrays (host) or
torch tensors (host or CUDA); the device flag of the C call is derived from
the tensor.  A failed call raises ClError with the library's message.  If
the CUDA library is not built the import of any entry point raises: there
is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcllbm.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "cl_lbm.h")

CL_OK, CL_ERR_ARG, CL_ERR_OOM, CL_ERR_CUDA, CL_ERR_STATE = 0, 1, 2, 3, 4
CL_ERR_DIVERGED, CL_ERR_NOT_CONVERGED, CL_ERR_NO_PATH, CL_ERR_TIMEOUT = 5, 6, 7, 8
CL_BC_DIRICHLET, CL_BC_ZERO_FLUX = 0, 1
CL_STORE_FP32, CL_STORE_FP16DEV, CL_STORE_FP32POP = 0, 1, 2
CL_REACT_GIVEN, CL_REACT_ALL_PORE_SOLID, CL_REACT_IONOMER_SOLID = 0, 1, 2
CL_CARRIER_O2, CL_CARRIER_PROTON = 0, 1
CL_LATTICE_D3Q7, CL_LATTICE_D3Q19 = 0, 1

cl_alloc_fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
cl_free_fn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class cl_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx_m", ctypes.c_double), ("T_K", ctypes.c_double), ("p_atm", ctypes.c_double),
        ("M_kgmol", ctypes.c_double), ("D_bulk", ctypes.c_double), ("D_ionomer", ctypes.c_double),
        ("k_ms", ctypes.c_double),
        ("knudsen", ctypes.c_int), ("bc_in", ctypes.c_int), ("bc_out", ctypes.c_int),
        ("c_in", ctypes.c_double), ("c_out", ctypes.c_double), ("tau_ref", ctypes.c_double),
        ("storage", ctypes.c_int), ("react_rule", ctypes.c_int), ("carrier", ctypes.c_int),
        ("lattice", ctypes.c_int), ("ionomer_o2", ctypes.c_int), ("check_every", ctypes.c_int),
        ("tol_flux", ctypes.c_double), ("tol_rel", ctypes.c_double),
        ("max_steps", ctypes.c_longlong),
        ("cuda_stream", ctypes.c_void_p),
        ("alloc", cl_alloc_fn), ("free", cl_free_fn), ("alloc_ctx", ctypes.c_void_p),
    ]


class cl_structure_info(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_longlong), ("n_transport", ctypes.c_longlong),
        ("n_active", ctypes.c_longlong), ("n_wall_links", ctypes.c_longlong),
        ("n_react_links", ctypes.c_longlong),
        ("D_b", ctypes.c_double), ("D_max", ctypes.c_double), ("dt_s", ctypes.c_double),
        ("k_lu", ctypes.c_double), ("mean_pore_diameter_m", ctypes.c_double),
    ]


class cl_phase_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in (
        "n_cells", "n_portions", "n_transport_portions", "n_transport_cells", "surface_faces",
        "transport_surface_faces", "largest_portion")]


class cl_solve_info(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_longlong), ("converged", ctypes.c_int),
        ("J_in", ctypes.c_double), ("J_out", ctypes.c_double), ("R", ctypes.c_double),
        ("flux_balance", ctypes.c_double), ("rel_change", ctypes.c_double),
        ("resid", ctypes.c_double), ("seconds", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cl_coupled_params(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double), ("phi_m", ctypes.c_double), ("phi_ref", ctypes.c_double),
        ("relax", ctypes.c_double), ("tol_phi", ctypes.c_double), ("max_outer", ctypes.c_int),
        ("krylov_tol", ctypes.c_double), ("krylov_max_iter", ctypes.c_int), ("steady_solver", ctypes.c_int),
    ]


class cl_coupled_info(ctypes.Structure):
    _fields_ = [
        ("outer", ctypes.c_int), ("converged", ctypes.c_int), ("dphi", ctypes.c_double),
        ("current_o2_A", ctypes.c_double), ("current_membrane_A", ctypes.c_double),
        ("o2_iterations", ctypes.c_longlong), ("proton_iterations", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cl_steady_info(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("cycles", ctypes.c_int), ("inner_iterations", ctypes.c_longlong),
        ("residual", ctypes.c_double), ("seconds", ctypes.c_double),
        ("J_in", ctypes.c_double), ("J_out", ctypes.c_double), ("R", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I = ctypes.c_int
_S = ctypes.c_int  # cl_status
_H = ctypes.c_void_p  # cl_handle

SIGNATURES = {
    "cl_params_default": (None, [ctypes.POINTER(cl_params)]),
    "cl_lbm_create": (_S, [ctypes.POINTER(_H), ctypes.POINTER(cl_params)]),
    "cl_lbm_destroy": (None, [_H]),
    "cl_lbm_set_structure": (_S, [_H, _P, _P, _I]),
    "cl_lbm_set_diffusivity": (_S, [_H, _P, _I]),
    "cl_lbm_init": (_S, [_H, _P, _I]),
    "cl_lbm_step": (_S, [_H, ctypes.c_longlong]),
    "cl_lbm_solve": (_S, [_H, ctypes.POINTER(cl_solve_info)]),
    "cl_lbm_solve_budget": (_S, [_H, ctypes.c_longlong, ctypes.POINTER(cl_solve_info)]),
    "cl_lbm_solve_krylov": (_S, [_H, ctypes.c_double, ctypes.c_int, ctypes.c_longlong,
                                 ctypes.POINTER(cl_solve_info), ctypes.POINTER(ctypes.c_int)]),
    "cl_lbm_solve_krylov_dsa": (_S, [_H, ctypes.c_double, ctypes.c_int, ctypes.c_longlong,
                                     ctypes.POINTER(cl_solve_info), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_longlong)]),
    "cl_lbm_fluxes": (_S, [_H, _P]),
    "cl_lbm_effective_diffusivity": (_S, [_H, _P, _P]),
    "cl_lbm_reaction_rate": (_S, [_H, _P, _P, _P]),
    "cl_lbm_current_density": (_S, [_H, ctypes.POINTER(ctypes.c_double)]),
    "cl_lbm_get_field": (_S, [_H, _P, _I]),
    "cl_lbm_get_populations": (_S, [_H, _P, _I]),
    "cl_lbm_get_setup": (_S, [_H, _P, _P, _P, _P, _I]),
    "cl_lbm_get_links": (_S, [_H, _P, _P, _I]),
    "cl_lbm_get_info": (_S, [_H, ctypes.POINTER(cl_structure_info)]),
    "cl_lbm_get_step": (_S, [_H, ctypes.POINTER(ctypes.c_longlong)]),
    "cl_status_str": (ctypes.c_char_p, [_I]),
    "cl_henry_constant": (ctypes.c_double, [ctypes.c_double]),
    "cl_ionomer_o2_diffusivity": (ctypes.c_double, [ctypes.c_double]),
    "cl_ionomer_effective_diffusivity": (ctypes.c_double, [ctypes.c_double]),
    "cl_tafel_rate_constant": (ctypes.c_double, [ctypes.c_double] * 5),
    "cl_last_error_message": (ctypes.c_char_p, []),
    "cl_version": (ctypes.c_char_p, []),
    "cl_active_mask_noalloc": (_S, [_P, _I, _I, _I, _I, _P, _P]),
    "cl_phase_connectivity": (_S, [_P, _I, _I, _I, ctypes.c_uint, _I, _I, _P, ctypes.POINTER(cl_phase_stats),
                                   _I, _P]),
    "cl_qsgs_grow": (_S, [_P, _I, _I, _I, _I, ctypes.c_uint, ctypes.c_uint, _P, ctypes.c_longlong,
                          ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, _I,
                          ctypes.POINTER(ctypes.c_longlong), _P]),
    "cl_qsgs_region_not_adjacent": (_S, [_P, _I, _I, _I, _I, _I, _P, _P]),
    "cl_qsgs_reactive_faces": (_S, [_P, _I, _I, _I, _I, _I, ctypes.c_double, ctypes.c_uint64, _P,
                                    ctypes.POINTER(ctypes.c_longlong), _P]),
    "cl_batch_create": (_S, [ctypes.POINTER(_H), ctypes.POINTER(_H), _I, _I]),
    "cl_batch_destroy": (None, [_H]),
    "cl_batch_step": (_S, [_H, ctypes.c_longlong]),
    "cl_batch_solve": (_S, [_H, ctypes.c_longlong, _P, ctypes.POINTER(_I)]),
    "cl_batch_autotune": (_S, [_H, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                               ctypes.POINTER(ctypes.c_double)]),
    "cl_batch_configure": (_S, [_H, _I, _I, _I]),
    "cl_batch_info": (_S, [_H, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "cl_batch_set_wait_test": (_S, [_H, ctypes.c_longlong, _I]),
    "cl_lbm_set_wait_test": (_S, [_H, ctypes.c_longlong, _I]),
    "cl_lbm_set_tile_rows": (_S, [_H, _I, ctypes.POINTER(_I)]),
    "cl_lbm_set_rate_scale": (_S, [_H, _P, _I]),
    "cl_lbm_set_source": (_S, [_H, _P, _I]),
    "cl_lbm_cell_reaction": (_S, [_H, _P, _I]),
    "cl_lbm_solve_steady_lines": (_S, [_H, ctypes.c_double, _I, _I, ctypes.c_double,
                                       ctypes.POINTER(cl_steady_info)]),
    "cl_coupled_solve": (_S, [_H, _H, ctypes.POINTER(cl_coupled_params), _P, _I, ctypes.POINTER(cl_coupled_info)]),
}

_lock = threading.Lock()
_lib = None


class ClError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} ({msg})")


def load() -> ctypes.CDLL:
    """Load libcllbm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run __graft_entry__.build())")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def status_str(s: int) -> str:
    return load().cl_status_str(int(s)).decode()


def last_error_message() -> str:
    return load().cl_last_error_message().decode()


def version() -> str:
    return load().cl_version().decode()


def _check(status: int, where: str):
    if status != CL_OK:
        raise ClError(status, where, last_error_message())


def _arr(x, dtype, n=None, writable=False):
    """(pointer, is_device, keepalive) for a numpy array or torch tensor."""
    if x is None:
        return None, 0, None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            tdt = {np.uint8: torch.uint8, np.float32: torch.float32, np.float64: torch.float64,
                   np.int32: torch.int32, np.uint16: None}[dtype]
            if tdt is not None and x.dtype != tdt:
                raise TypeError(f"tensor dtype {x.dtype}, expected {tdt}")
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if n is not None and x.numel() < n:
                raise ValueError(f"tensor has {x.numel()} elements, need {n}")
            return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), x
    except ImportError:
        pass
    if not isinstance(x, np.ndarray):
        raise TypeError("expected a numpy array or torch tensor")
    if x.dtype != dtype:
        raise TypeError(f"array dtype {x.dtype}, expected {np.dtype(dtype)}")
    if not x.flags.c_contiguous:
        raise ValueError("array must be C-contiguous")
    if writable and not x.flags.writeable:
        raise ValueError("array must be writable")
    if n is not None and x.size < n:
        raise ValueError(f"array has {x.size} elements, need {n}")
    return x.ctypes.data_as(ctypes.c_void_p), 0, x


def cl_params_default(**overrides) -> cl_params:
    p = cl_params()
    load().cl_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def current_torch_stream() -> int:
    """cudaStream_t of torch's current stream, or 0."""
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


class TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self, device: int = 0):
        import torch
        self._torch = torch
        self.device = device

        def _alloc(nbytes, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0)))
            except Exception:  # the C side reports CL_ERR_OOM
                return None

        def _free(ptr, nbytes, stream, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = cl_alloc_fn(_alloc)
        self.free = cl_free_fn(_free)


# ------------------------------------------------------------ ABI mirrors
def cl_lbm_create(params: cl_params) -> int:
    h = ctypes.c_void_p()
    _check(load().cl_lbm_create(ctypes.byref(h), ctypes.byref(params)), "cl_lbm_create")
    return h.value


def cl_lbm_destroy(h: int) -> None:
    load().cl_lbm_destroy(h)


def cl_lbm_set_structure(h: int, phase, reactive_faces=None, n: int | None = None) -> None:
    pp, dev, _k1 = _arr(phase, np.uint8, n)
    rp, rdev, _k2 = _arr(reactive_faces, np.uint8, n)
    if reactive_faces is not None and rdev != dev:
        raise ValueError("phase and reactive_faces must both be host or both be device")
    _check(load().cl_lbm_set_structure(h, pp, rp, dev), "cl_lbm_set_structure")


def cl_lbm_set_diffusivity(h: int, D, n: int | None = None) -> None:
    p, dev, _k = _arr(D, np.float64, n)
    _check(load().cl_lbm_set_diffusivity(h, p, dev), "cl_lbm_set_diffusivity")


def cl_lbm_set_rate_scale(h: int, kscale, n: int | None = None) -> None:
    p, dev, _k = _arr(kscale, np.float64, n)
    _check(load().cl_lbm_set_rate_scale(h, p, dev), "cl_lbm_set_rate_scale")


def cl_lbm_set_source(h: int, S, n: int | None = None) -> None:
    p, dev, _k = _arr(S, np.float64, n)
    _check(load().cl_lbm_set_source(h, p, dev), "cl_lbm_set_source")


def cl_lbm_cell_reaction(h: int, out, n: int | None = None) -> None:
    p, dev, _k = _arr(out, np.float64, n, writable=True)
    _check(load().cl_lbm_cell_reaction(h, p, dev), "cl_lbm_cell_reaction")


def cl_coupled_solve(o2: int, pr: int, params: cl_coupled_params, phi_out=None, n: int | None = None):
    """(status, info); phi_out (float64, nx*ny*nz) receives the ionomer potential."""
    p, dev, _k = _arr(phi_out, np.float64, n, writable=True)
    info = cl_coupled_info()
    st = load().cl_coupled_solve(o2, pr, ctypes.byref(params), p, dev, ctypes.byref(info))
    if st not in (CL_OK, CL_ERR_NOT_CONVERGED):
        _check(st, "cl_coupled_solve")
    return st, info


def cl_lbm_solve_steady_lines(h: int, tol: float, max_iter: int, restart: int, cg_tol: float):
    """(status, cl_steady_info); raises on errors other than CL_ERR_NOT_CONVERGED."""
    info = cl_steady_info()
    st = load().cl_lbm_solve_steady_lines(h, float(tol), int(max_iter), int(restart), float(cg_tol),
                                          ctypes.byref(info))
    if st not in (CL_OK, CL_ERR_NOT_CONVERGED):
        _check(st, "cl_lbm_solve_steady_lines")
    return st, info


def cl_lbm_set_tile_rows(h: int, rows: int) -> int:
    out = ctypes.c_int(0)
    _check(load().cl_lbm_set_tile_rows(h, rows, ctypes.byref(out)), "cl_lbm_set_tile_rows")
    return out.value


def cl_lbm_init(h: int, C0=None, n: int | None = None) -> None:
    p, dev, _k = _arr(C0, np.float32, n)
    _check(load().cl_lbm_init(h, p, dev), "cl_lbm_init")


def cl_lbm_step(h: int, nsteps: int) -> None:
    _check(load().cl_lbm_step(h, int(nsteps)), "cl_lbm_step")


def cl_lbm_solve(h: int, raise_on_not_converged: bool = False) -> tuple[int, cl_solve_info]:
    info = cl_solve_info()
    s = load().cl_lbm_solve(h, ctypes.byref(info))
    if s not in (CL_OK, CL_ERR_NOT_CONVERGED) or (raise_on_not_converged and s != CL_OK):
        _check(s, "cl_lbm_solve")
    return s, info


def cl_lbm_solve_budget(h: int, max_steps: int) -> tuple[int, cl_solve_info]:
    info = cl_solve_info()
    s = load().cl_lbm_solve_budget(h, int(max_steps), ctypes.byref(info))
    if s not in (CL_OK, CL_ERR_NOT_CONVERGED):
        _check(s, "cl_lbm_solve_budget")
    return s, info


def cl_lbm_solve_krylov(h: int, tol: float, max_iter: int, max_steps: int) -> tuple[int, cl_solve_info, int]:
    info = cl_solve_info()
    it = ctypes.c_int(0)
    s = load().cl_lbm_solve_krylov(h, float(tol), int(max_iter), int(max_steps), ctypes.byref(info),
                                   ctypes.byref(it))
    if s not in (CL_OK, CL_ERR_NOT_CONVERGED):
        _check(s, "cl_lbm_solve_krylov")
    return s, info, it.value


def cl_lbm_solve_krylov_dsa(h: int, tol: float, max_iter: int, max_steps: int) -> tuple[int, cl_solve_info, int, int]:
    info = cl_solve_info()
    it = ctypes.c_int(0)
    inner = ctypes.c_longlong(0)
    s = load().cl_lbm_solve_krylov_dsa(h, float(tol), int(max_iter), int(max_steps), ctypes.byref(info),
                                       ctypes.byref(it), ctypes.byref(inner))
    if s not in (CL_OK, CL_ERR_NOT_CONVERGED):
        _check(s, "cl_lbm_solve_krylov_dsa")
    return s, info, it.value, inner.value


def cl_lbm_fluxes(h: int) -> np.ndarray:
    out = np.zeros(5)
    _check(load().cl_lbm_fluxes(h, out.ctypes.data_as(ctypes.c_void_p)), "cl_lbm_fluxes")
    return out


def cl_lbm_effective_diffusivity(h: int) -> tuple[float, float]:
    d = ctypes.c_double()
    r = ctypes.c_double()
    _check(load().cl_lbm_effective_diffusivity(h, ctypes.byref(d), ctypes.byref(r)),
           "cl_lbm_effective_diffusivity")
    return d.value, r.value


def cl_lbm_reaction_rate(h: int, nx: int) -> tuple[float, np.ndarray, np.ndarray]:
    tot = ctypes.c_double()
    pr = np.zeros(nx)
    pc = np.zeros(nx)
    _check(load().cl_lbm_reaction_rate(h, ctypes.byref(tot), pr.ctypes.data_as(ctypes.c_void_p),
                                       pc.ctypes.data_as(ctypes.c_void_p)), "cl_lbm_reaction_rate")
    return tot.value, pr, pc


def cl_lbm_current_density(h: int) -> float:
    v = ctypes.c_double()
    _check(load().cl_lbm_current_density(h, ctypes.byref(v)), "cl_lbm_current_density")
    return v.value


def cl_lbm_get_field(h: int, out) -> None:
    p, dev, _k = _arr(out, np.float32, writable=True)
    _check(load().cl_lbm_get_field(h, p, dev), "cl_lbm_get_field")


def cl_lbm_get_populations(h: int, out) -> None:
    p, dev, _k = _arr(out, np.float32, writable=True)
    _check(load().cl_lbm_get_populations(h, p, dev), "cl_lbm_get_populations")


def cl_lbm_get_setup(h: int, active=None, omega=None, chord=None, link_mask=None) -> None:
    a, d1, _k1 = _arr(active, np.uint8, writable=True)
    o, d2, _k2 = _arr(omega, np.float32, writable=True)
    c, d3, _k3 = _arr(chord, np.int32, writable=True)
    m, d4, _k4 = _arr(link_mask, np.uint16, writable=True)
    devs = {d for d, x in ((d1, active), (d2, omega), (d3, chord), (d4, link_mask)) if x is not None}
    if len(devs) > 1:
        raise ValueError("outputs must all be host or all be device")
    _check(load().cl_lbm_get_setup(h, a, o, c, m, devs.pop() if devs else 0), "cl_lbm_get_setup")


def cl_lbm_get_links(h: int, wall=None, reactive=None) -> None:
    w, d1, _k1 = _arr(wall, np.uint32, writable=True)
    r, d2, _k2 = _arr(reactive, np.uint32, writable=True)
    devs = {d for d, x in ((d1, wall), (d2, reactive)) if x is not None}
    if len(devs) > 1:
        raise ValueError("outputs must both be host or both be device")
    _check(load().cl_lbm_get_links(h, w, r, devs.pop() if devs else 0), "cl_lbm_get_links")


def cl_phase_connectivity(phase, phase_set, neighbours: int = 26, periodic_yz: bool = False, labels=None,
                          stream: int | None = None) -> dict:
    """Sec. 2.1.3 connected-phase labelling on the GPU.  phase: (nz, ny, nx)
    uint8 (numpy or torch); phase_set: iterable of codes; labels: optional
    int32 output of the same shape and side.  Returns the statistics."""
    nz, ny, nx = (int(v) for v in phase.shape)
    n = nx * ny * nz
    pp, pdev, _k1 = _arr(phase, np.uint8, n)
    lp, ldev, _k2 = _arr(labels, np.int32, n, writable=True)
    if labels is not None and ldev != pdev:
        raise ValueError("phase and labels must be on the same side")
    mask = 0
    for k in phase_set:
        mask |= 1 << int(k)
    st = current_torch_stream() if stream is None else stream
    out = cl_phase_stats()
    _check(load().cl_phase_connectivity(pp, nx, ny, nz, mask, int(neighbours), int(bool(periodic_yz)), lp,
                                        ctypes.byref(out), pdev, st), "cl_phase_connectivity")
    return {k: getattr(out, k) for k, _ in out._fields_}


def _dev_u8(x, what):
    p, dev, _k = _arr(x, np.uint8, None, writable=True)
    if not dev:
        raise ValueError(f"{what} must be a CUDA uint8 tensor")
    return p


def cl_qsgs_grow(phase, code: int, allowed_mask: int, grown_mask: int, target: int, c_d: float, p_alpha: float,
                 seed: int, stream_id: int, region=None, max_sweeps: int = 100000) -> int:
    """QSGS growth in place on a CUDA uint8 tensor (nz, ny, nx); returns the final count."""
    nz, ny, nx = (int(v) for v in phase.shape)
    out = ctypes.c_longlong(0)
    _check(load().cl_qsgs_grow(_dev_u8(phase, "phase"), nx, ny, nz, int(code), int(allowed_mask), int(grown_mask),
                               None if region is None else _dev_u8(region, "region"), int(target), float(c_d),
                               float(p_alpha), seed & (2**64 - 1), stream_id & (2**64 - 1), int(max_sweeps),
                               ctypes.byref(out), current_torch_stream()), "cl_qsgs_grow")
    return out.value


def cl_qsgs_region_not_adjacent(phase, code: int, avoid: int, region) -> None:
    nz, ny, nx = (int(v) for v in phase.shape)
    _check(load().cl_qsgs_region_not_adjacent(_dev_u8(phase, "phase"), nx, ny, nz, int(code), int(avoid),
                                              _dev_u8(region, "region"), current_torch_stream()),
           "cl_qsgs_region_not_adjacent")


def cl_qsgs_reactive_faces(phase, from_code: int, to_code: int, fraction: float, seed: int, out) -> int:
    nz, ny, nx = (int(v) for v in phase.shape)
    n = ctypes.c_longlong(0)
    _check(load().cl_qsgs_reactive_faces(_dev_u8(phase, "phase"), nx, ny, nz, int(from_code), int(to_code),
                                         float(fraction), seed & (2**64 - 1), _dev_u8(out, "out"),
                                         ctypes.byref(n), current_torch_stream()), "cl_qsgs_reactive_faces")
    return n.value


def cl_lbm_get_info(h: int) -> cl_structure_info:
    info = cl_structure_info()
    _check(load().cl_lbm_get_info(h, ctypes.byref(info)), "cl_lbm_get_info")
    return info


def _common_cuda_device(*tensors):
    """The one CUDA device that every tensor lives on; ValueError otherwise."""
    devs = set()
    for t in tensors:
        dev = getattr(t, "device", None)
        if dev is None or getattr(dev, "type", None) != "cuda":
            raise ValueError("expected CUDA tensors")
        devs.add(dev.index)
    if len(devs) != 1:
        raise ValueError(f"tensors on different CUDA devices: {sorted(devs)}")
    return devs.pop()


def cl_active_mask_noalloc(phase, active, ionomer_transport: bool = False, stream: int | None = None) -> None:
    """Inlet-connected transport cells without device allocation.  `phase`
    (uint8) and `active` (uint8, written) are CUDA tensors of shape (nz, ny, nx)
    on one device; the call runs with that device current, on its current
    torch stream unless `stream` is given."""
    import torch
    dev = _common_cuda_device(phase, active)
    nz, ny, nx = (int(v) for v in phase.shape)
    pp, _p, _k1 = _arr(phase, np.uint8, nx * ny * nz)
    ap, _a, _k2 = _arr(active, np.uint8, nx * ny * nz, writable=True)
    with torch.cuda.device(dev):
        st = int(torch.cuda.current_stream(dev).cuda_stream) if stream is None else stream
        _check(load().cl_active_mask_noalloc(pp, nx, ny, nz, int(bool(ionomer_transport)), ap, st),
               "cl_active_mask_noalloc")


def cl_lbm_get_step(h: int) -> int:
    s = ctypes.c_longlong()
    _check(load().cl_lbm_get_step(h, ctypes.byref(s)), "cl_lbm_get_step")
    return s.value


# ------------------------------------------------------------------ batches
def cl_batch_create(handles, z_chunk: int = 0) -> int:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    b = ctypes.c_void_p()
    _check(load().cl_batch_create(ctypes.byref(b), arr, len(handles), int(z_chunk)), "cl_batch_create")
    return b.value


def cl_batch_destroy(b: int) -> None:
    load().cl_batch_destroy(b)


def cl_batch_step(b: int, nsteps: int) -> None:
    _check(load().cl_batch_step(b, int(nsteps)), "cl_batch_step")


def cl_batch_solve(b: int, n: int, max_steps: int):
    infos = (cl_solve_info * n)()
    nc = ctypes.c_int()
    s = load().cl_batch_solve(b, int(max_steps), ctypes.cast(infos, ctypes.c_void_p), ctypes.byref(nc))
    if s not in (CL_OK, CL_ERR_NOT_CONVERGED):
        _check(s, "cl_batch_solve")
    return s, [infos[i].as_dict() for i in range(n)], nc.value


def cl_batch_autotune(b: int, steps_per_trial: int = 20):
    zc, pf, tr, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(load().cl_batch_autotune(b, int(steps_per_trial), ctypes.byref(zc), ctypes.byref(pf), ctypes.byref(tr),
                                    ctypes.byref(ms)), "cl_batch_autotune")
    return zc.value, pf.value, tr.value, ms.value


def cl_batch_configure(b: int, z_chunk: int, prefetch: int, tile_rows: int) -> None:
    _check(load().cl_batch_configure(b, int(z_chunk), int(prefetch), int(tile_rows)), "cl_batch_configure")


def cl_batch_info(b: int):
    g, n, u = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().cl_batch_info(b, ctypes.byref(g), ctypes.byref(n), ctypes.byref(u)), "cl_batch_info")
    return dict(grid_blocks=g.value, n_items=n.value, uses_graph=bool(u.value))
