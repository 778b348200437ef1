"""Coupled O2 / proton steady state (Sec. 3.3-3.4, Eq. 16-18) through
cl_coupled_solve: two handles (O2 with the reaction sites of Eq. 18 as
catalytic faces, protons on the x-mirrored box) and the Picard iteration on
the ionomer potential, all in the library's kernels.  Argument marshalling
only."""
from __future__ import annotations

import numpy as np

from . import _lib as L
from .solver import Solver


def solve(phase, params, sigma, phi_m, k_ref, alpha=0.61, phi_ref=None, relax=0.5, tol_phi=1e-7,
          max_outer=200, ionomer_D=None, krylov_tol=None, krylov_max_iter=20000, steady_solver=None,
          stream=None):
    """Coupled steady state on `phase` (nz, ny, nx).

    params: the O2 set-up (dx_m, T_K, knudsen, c_in in mol/m^3, bc_in,
    bc_out, ...); sigma: ionomer proton conductivity [S/m]; phi_m: membrane
    potential [V] at x = L; k_ref: rate constant [m/s] at phi_ref (default
    phi_m); ionomer_D: None carries O2 in the ionomer by Eq. 10-13
    (ionomer_o2), a value [m^2/s] gives the ionomer that diffusivity.
    steady_solver: "krylov" (population-space GMRES with the diffusion
    preconditioner) or "lines" (populations eliminated along lines; it also
    reaches the contrast of Eq. 13); default "lines" when ionomer_D is None.
    krylov_tol: residual of each steady solve (default 1e-12 for "lines",
    1e-10 for "krylov").
    Returns a dict: phi (V, 0 outside the proton-conducting ionomer), C
    (O2 field), current_A_o2, current_A_membrane, outer, converged, dphi,
    and the Krylov step applications of both carriers."""
    phase = np.ascontiguousarray(phase, dtype=np.uint8)
    shape = phase.shape
    phi_ref = phi_m if phi_ref is None else phi_ref
    o2p = dict(params, k_ms=k_ref, carrier=L.CL_CARRIER_O2, react_rule=L.CL_REACT_IONOMER_SOLID)
    if ionomer_D is None:
        o2p.update(ionomer_o2=1)
    else:
        o2p.update(ionomer_o2=0, D_ionomer=ionomer_D)
    o2 = Solver(shape, storage="fp32pop", stream=stream, **o2p)
    o2.set_structure(phase, None)
    prp = dict(dx_m=params["dx_m"], T_K=params.get("T_K", 353.0), knudsen=0, carrier=L.CL_CARRIER_PROTON,
               D_ionomer=sigma, k_ms=0.0, bc_in=L.CL_BC_DIRICHLET, bc_out=L.CL_BC_ZERO_FLUX, c_in=phi_m,
               c_out=phi_m, tau_ref=1.0)
    pr = Solver(shape, storage="fp32pop", stream=stream, **prp)
    pr.set_structure(np.ascontiguousarray(phase[:, :, ::-1]), None)
    if steady_solver is None:
        steady_solver = "lines" if ionomer_D is None else "krylov"
    if krylov_tol is None:
        # the line-eliminated residual is taken against |F(0)|: 1e-12 leaves the ionomer's slow
        # modes at about 1e-7 of C, where 1e-10 left them at 1e-5
        krylov_tol = 1e-12 if steady_solver == "lines" else 1e-10
    cp = L.cl_coupled_params(alpha=alpha, phi_m=phi_m, phi_ref=phi_ref, relax=relax, tol_phi=tol_phi,
                             max_outer=max_outer, krylov_tol=krylov_tol, krylov_max_iter=krylov_max_iter,
                             steady_solver={"krylov": 0, "lines": 1}[steady_solver])
    phi = np.zeros(shape, dtype=np.float64)
    st, info = L.cl_coupled_solve(o2.h, pr.h, cp, phi, phi.size)
    out = dict(info.as_dict())
    out.update(phi=phi, C=o2.field(), status=L.status_str(st), o2=o2, protons=pr,
               current_A_o2=info.current_o2_A, current_A_membrane=info.current_membrane_A,
               converged=bool(info.converged))
    return out
