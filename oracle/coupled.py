"""Coupled electrochemical reaction transport (Sec. 3.3-3.4, Eq. 16-18) in
the FP64 oracle.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the statement of
what a coupled solve computes, built from two ``OracleLBM`` solves.

The paper writes the full coupling -- O2 dissolved in the ionomer, proton
conduction in the ionomer, and a Tafel rate that depends on the local
ionomer potential -- but presets a uniform potential for its results
(Sec. 3.5.2).  The reading taken here:

  * O2 (Eq. 10-15): the gas-equivalent concentration C (mol/m^3) in pore,
    micropore and ionomer (``ionomer_o2 = 1``).  The reaction sites of
    Eq. 18, ionomer cells next to Pt, are the faces of ionomer cells toward
    solid cells; each is a first-order sink k(phi) C_wall, the surface form
    of Eq. 18a that the uniform-potential solver already uses (n of Eq. 18
    is the number of such faces of a cell).
  * Kinetics (Eq. 17b): k(phi) = k_ref exp(alpha F (phi - phi_ref) / (R T)),
    phi the ionomer potential of the cell that owns the face.
  * Protons (Eq. 16): div(sigma grad phi) = S_e in the ionomer, with S_e the
    current drawn per unit volume of a cell, 4 F times its O2 consumption
    (Eq. 18b, n i / Delta).  The membrane is the x = L face (phi = phi_m);
    the gas side x = 0 passes no protons.  The proton solve runs on the
    mirrored box, so that its inlet plane is the membrane.  Sites of ionomer
    cells without an ionomer path to the membrane draw no current (k = 0).
  * Outer iteration: Picard on phi with relaxation until phi changes by
    less than tol_phi (V).  Each inner solve is the exact steady state of
    the scheme (``steady.solve``: the march of the dissolved-O2 problem
    would take too long), so the y and z extents must be multiples of 3.
"""
from __future__ import annotations

import numpy as np

from . import OracleLBM, steady

F = 96485.33212
R_GAS = 8.314462618
DIRS = [(0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)]  # (dz, dy, dx) of faces +x, -x, +y, -y, +z, -z


def ionomer_solid_faces(phase: np.ndarray) -> np.ndarray:
    """Face mask (bit d: face toward x + c_d) of every ionomer cell face
    that borders a solid cell; x not periodic, y and z periodic."""
    phase = np.asarray(phase)
    out = np.zeros(phase.shape, np.uint8)
    for d, (dz, dy, dx) in enumerate(DIRS):
        nb = np.roll(phase, (-dz, -dy, -dx), axis=(0, 1, 2))
        ok = (phase == 2) & (nb == 1)
        if dx == 1:
            ok[:, :, -1] = False
        if dx == -1:
            ok[:, :, 0] = False
        out |= ok.astype(np.uint8) << d
    return out


def solve(phase, params, sigma, phi_m, k_ref, alpha=0.61, phi_ref=None, relax=0.5, tol_phi=1e-9,
          max_outer=200, ionomer_D=None):
    """Coupled O2 / proton steady state on `phase` (nz, ny, nx).

    params: the O2 set-up (dx_m, T_K, knudsen, c_in in mol/m^3, bc_in, bc_out,
    ...); sigma: ionomer proton conductivity [S/m]; phi_m: membrane
    potential [V]; k_ref: rate constant [m/s] at phi_ref (default phi_m).
    Returns a dict: phi (V, NaN outside the proton-conducting ionomer), C,
    site (cells that carry current), R_cell (mol/s per cell), current_A from
    the O2 side (4 F sum R_cell) and from the proton side (the membrane
    flux), the proton solve's source sum, the outer iterations, converged.

    ionomer_D: None carries O2 in the ionomer as Eq. 10-15 (D_e RT/H,
    ``ionomer_o2 = 1``); a value [m^2/s] gives the ionomer that diffusivity
    instead.  The coupling of Sec. 3.3-3.4 (Eq. 16-18) is the same for any
    ionomer diffusivity; a larger one keeps the O2 problem within reach of
    an iterative steady solver at the ~1e5 pore/ionomer contrast of Eq. 13."""
    phase = np.ascontiguousarray(phase, dtype=np.uint8)
    phi_ref = phi_m if phi_ref is None else phi_ref
    T = params.get("T_K", 353.0)
    faces = ionomer_solid_faces(phase)
    o2_params = dict(params, ionomer_o2=1, k_ms=k_ref, carrier=0) if ionomer_D is None else \
        dict(params, ionomer_o2=0, D_ionomer=ionomer_D, k_ms=k_ref, carrier=0)
    o2 = OracleLBM(phase, react=faces, **o2_params)
    pr_params = dict(dx_m=params["dx_m"], T_K=T, knudsen=0, carrier=1, D_ionomer=sigma, k_ms=0.0,
                     bc_in=0, bc_out=1, c_in=phi_m, c_out=phi_m, tau_ref=1.0)
    pr = OracleLBM(phase[:, :, ::-1], **pr_params)
    A_pr, _ = steady.step_matrix(pr)
    p_act = pr.active()[:, :, ::-1].astype(bool)
    site = p_act & (o2.react() != 0) & o2.active().astype(bool)
    phi = np.where(p_act, phi_m, np.nan)
    dx3 = params["dx_m"] ** 3
    dphi = np.inf
    outer = 0
    for outer in range(1, max_outer + 1):
        kscale = np.where(site, np.exp(alpha * F * (np.nan_to_num(phi, nan=phi_ref) - phi_ref) / (R_GAS * T)), 0.0)
        o2.set_rate_scale(kscale)
        steady.solve(o2)
        R_cell = o2.cell_reaction() * dx3 / o2.dt  # mol/s per cell
        S_e = 4.0 * F * R_cell / dx3                # A/m^3, Eq. 18b
        src = -(S_e * pr.dt)[:, :, ::-1]            # div(sigma grad phi) = S_e as a sink per step
        pr.set_source(src)
        steady.solve(pr, A_pr)
        phi_new = np.where(p_act, pr.concentration()[:, :, ::-1], np.nan)
        dphi = float(np.nanmax(np.abs(phi_new - phi)))
        phi = phi + relax * (phi_new - phi)
        if dphi < tol_phi:
            break
    fp = pr.fluxes()
    return dict(phi=phi, C=o2.concentration(), site=site, R_cell=R_cell,
                current_A_o2=4.0 * F * float(R_cell.sum()),
                current_A_membrane=fp["J_in"] * dx3 / pr.dt,
                source_sum_lu=float(src.sum()), membrane_flux_lu=fp["J_in"],
                outer=outer, converged=dphi < tol_phi, o2=o2, protons=pr)
