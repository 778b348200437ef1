"""Object wrapper over one cl_lbm handle (argument marshalling only)."""
from __future__ import annotations

import numpy as np

from . import _lib as L

_STORAGE = {"fp32": L.CL_STORE_FP32, "fp16dev": L.CL_STORE_FP16DEV, "fp32pop": L.CL_STORE_FP32POP}
_LATTICE = {"d3q7": L.CL_LATTICE_D3Q7, "d3q19": L.CL_LATTICE_D3Q19}


class Solver:
    """One solver on one box.  Parameters are the cl_params fields; the
    ``lattice`` may also be given by name ("d3q7", "d3q19").

    ``shape`` is (nz, ny, nx).  ``stream``: a cudaStream_t (int); default is
    torch's current stream when torch has initialised CUDA, else the legacy
    default stream.  ``torch_alloc``: route device allocations through torch's
    caching allocator.
    """

    def __init__(self, shape, storage: str = "fp32", stream: int | None = None,
                 torch_alloc: bool = False, **params):
        nz, ny, nx = (int(v) for v in shape)
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        p = L.cl_params_default(nx=nx, ny=ny, nz=nz)
        p.storage = _STORAGE[storage]
        if isinstance(params.get("lattice"), str):
            params["lattice"] = _LATTICE[params["lattice"]]
        for k, v in params.items():
            setattr(p, k, v)
        self.q = 19 if p.lattice == L.CL_LATTICE_D3Q19 else 7
        p.cuda_stream = L.current_torch_stream() if stream is None else stream
        self._alloc = None
        if torch_alloc:
            self._alloc = L.TorchAllocator()
            p.alloc = self._alloc.alloc
            p.free = self._alloc.free
        self.params = p
        self.h = L.cl_lbm_create(p)

    def close(self):
        if getattr(self, "h", None):
            L.cl_lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ set-up
    def set_structure(self, phase, reactive_faces=None):
        L.cl_lbm_set_structure(self.h, phase, reactive_faces, self.n)

    def set_diffusivity(self, D):
        L.cl_lbm_set_diffusivity(self.h, D, self.n)

    def set_tile_rows(self, rows: int = 0) -> int:
        """Tile shape of the plane march ((C, delta) storage): rows of the
        512-cell tile per warp, 1 (64 x 8), 2 (32 x 16) or 4 (16 x 32); 0
        picks the shape with the fewest idle lanes along x.  Returns the
        shape in use."""
        return L.cl_lbm_set_tile_rows(self.h, rows)

    def set_rate_scale(self, kscale):
        """Per-cell factor on k (Eq. 17b with a non-uniform potential); None: uniform."""
        L.cl_lbm_set_rate_scale(self.h, kscale, self.n)

    def set_source(self, S):
        """Per-cell source per step, lattice units (the a_i S term of Eq. 21); None: none."""
        L.cl_lbm_set_source(self.h, S, self.n)

    def cell_reaction(self):
        """Per-cell amount consumed per step on catalytic faces (lattice units)."""
        out = np.zeros(self.shape, dtype=np.float64)
        L.cl_lbm_cell_reaction(self.h, out, self.n)
        return out

    def init(self, C0=None):
        L.cl_lbm_init(self.h, C0, self.n)

    # ------------------------------------------------------------ stepping
    def step(self, n: int = 1):
        L.cl_lbm_step(self.h, n)

    def solve(self, raise_on_not_converged: bool = False):
        status, info = L.cl_lbm_solve(self.h, raise_on_not_converged)
        d = info.as_dict()
        d["status"] = L.status_str(status)
        return d

    def solve_budget(self, max_steps: int):
        status, info = L.cl_lbm_solve_budget(self.h, max_steps)
        d = info.as_dict()
        d["status"] = L.status_str(status)
        return d

    def solve_krylov(self, tol: float = 1e-8, max_iter: int = 20000, max_steps: int | None = None):
        """Mixed-precision Krylov solve of the fixed-point equation of the
        step map (plain f32 populations only), then the stopping rule of the
        time march from its result with at most max_steps steps (default:
        the handle's max_steps).  Returns the solve info with "iterations"
        (BiCGSTAB iterations) added."""
        if max_steps is None:
            max_steps = self.params.max_steps
        status, info, it = L.cl_lbm_solve_krylov(self.h, tol, max_iter, max_steps)
        d = info.as_dict()
        d["status"] = L.status_str(status)
        d["iterations"] = it
        return d

    def solve_krylov_dsa(self, tol: float = 1e-8, max_iter: int = 20000, max_steps: int | None = None):
        """solve_krylov with flexible GMRES and the diffusion preconditioner
        (either lattice, plain f32 populations).  Adds "iterations" (step
        applications) and "inner_iterations" (conjugate-gradient
        iterations) to the solve info."""
        if max_steps is None:
            max_steps = self.params.max_steps
        status, info, it, inner = L.cl_lbm_solve_krylov_dsa(self.h, tol, max_iter, max_steps)
        d = info.as_dict()
        d["status"] = L.status_str(status)
        d["iterations"] = it
        d["inner_iterations"] = inner
        return d

    def solve_steady_lines(self, tol: float = 1e-12, max_iter: int = 4000, restart: int = 1500,
                           cg_tol: float = 1e-3):
        """Steady state as the fixed point of the line-eliminated map C = F(C)
        (D3Q7, plain f32 populations), flexible GMRES in FP64 with the
        finite-volume preconditioner.  Returns the call's info and status."""
        st, info = L.cl_lbm_solve_steady_lines(self.h, tol, max_iter, restart, cg_tol)
        d = info.as_dict()
        d["status"] = L.status_str(st)
        return d

    # ------------------------------------------------------------ readouts
    def fluxes(self):
        f = L.cl_lbm_fluxes(self.h)
        return dict(J_in=f[0], J_out=f[1], R=f[2], sum_C=f[3], n_active=int(f[4]))

    def effective_diffusivity(self):
        return L.cl_lbm_effective_diffusivity(self.h)

    def reaction_rate(self):
        return L.cl_lbm_reaction_rate(self.h, self.shape[2])

    def current_density(self):
        """Eq. 25: i_d = 4 F R / A_cross [A/m^2]."""
        return L.cl_lbm_current_density(self.h)

    def field(self):
        out = np.zeros(self.shape, dtype=np.float32)
        L.cl_lbm_get_field(self.h, out)
        return out

    def populations(self):
        out = np.zeros((self.q,) + self.shape, dtype=np.float32)
        L.cl_lbm_get_populations(self.h, out)
        return out

    def setup(self, chord: bool = False):
        active = np.zeros(self.shape, dtype=np.uint8)
        omega = np.zeros(self.shape, dtype=np.float32)
        mask = np.zeros(self.shape, dtype=np.uint16)
        ch = np.zeros(self.shape + (13,), dtype=np.int32) if chord else None
        L.cl_lbm_get_setup(self.h, active, omega, ch, mask)
        return dict(active=active, omega=omega, chord=ch, mask=mask)

    def links(self):
        """(wall, reactive) link bit sets per cell, uint32 (bit i-1: link toward x + c_i)."""
        wall = np.zeros(self.shape, dtype=np.uint32)
        react = np.zeros(self.shape, dtype=np.uint32)
        L.cl_lbm_get_links(self.h, wall, react)
        return wall, react

    def info(self):
        i = L.cl_lbm_get_info(self.h)
        return {k: getattr(i, k) for k, _ in i._fields_}

    @property
    def steps(self):
        return L.cl_lbm_get_step(self.h)
