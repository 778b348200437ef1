"""The exact steady-state solve of the oracle (oracle/steady.py) and the
coupled O2 / proton problem of Sec. 3.3-3.4 (oracle/coupled.py), pinned by
closed forms, conservation and limits rather than by their own arithmetic.

* The direct solve of (I - A) x = S(0), with A assembled from the oracle's
  step, is the march's fixed point (bulk D, both lattices), and it reaches
  the Henry-law series slab at the physical pore/ionomer contrast, where
  the march would need ~1e8 steps.
* The source term (Eq. 16 with S_e, entering Eq. 21 as a_i S): a 1D
  column with a uniform source and one fixed-value face has the discrete
  parabola of the finite-volume balance (the steady 1D scheme is that
  balance at tau = 1, with the face value shifted by the source's share
  that anti-bounce-back returns), and in 3D the membrane flux equals the
  summed sources.
* The coupling: with a very large conductivity the potential stays at the
  membrane value and the reaction equals the uniform-potential solve; with
  a small one the potential falls away from the membrane (Eq. 16 with a
  positive S_e), the Tafel rate (Eq. 17b) drops with it, and the current
  drawn from O2 equals the current through the membrane.
"""
import numpy as np
import pytest

import oracle
from oracle import coupled, steady
from paper_1410_1914_gb300 import inputs

R = 8.314462618


@pytest.mark.parametrize("lattice,shape", [(0, (12, 12, 20)), (1, (9, 9, 12))])
def test_direct_steady_state_is_the_march_fixed_point(lattice, shape):
    ph, react, params = inputs.make_workload("pt_cl_48", shape=shape, seed=51)
    o = oracle.OracleLBM(ph, react=react, lattice=lattice, **params)
    x = steady.solve(o)
    o.step(1)
    assert np.abs(o.populations() - x).max() <= 1e-13
    o.set_populations(x)
    m = oracle.OracleLBM(ph, react=react, lattice=lattice, **params)
    m.solve(tol=1e-13, check_every=100, max_steps=2_000_000)
    assert o.effective_diffusivity()[1] == pytest.approx(m.effective_diffusivity()[1], rel=1e-9)


def test_direct_steady_state_reaches_the_series_slab_at_physical_contrast():
    T = 333.0
    n_p, n_i = 9, 6
    ph = np.zeros((3, 3, n_p + n_i), np.uint8)
    ph[:, :, n_p:] = 2
    o = oracle.OracleLBM(ph, dx_m=1e-8, T_K=T, ionomer_o2=1)   # D_b from Eq. 7: contrast ~1e5
    D_p = o.D_b
    assert D_p / o.D().max() < 2 and D_p / o.D()[0, 0, -1] > 5e4
    steady.solve(o)
    D_e = oracle.ionomer_o2_diffusivity(T)
    H = oracle.henry_constant(T)
    flux = 1.0 / (n_p * 1e-8 / D_p + n_i * 1e-8 * H / (R * T * D_e))
    assert o.effective_diffusivity()[0] == pytest.approx(flux * (n_p + n_i) * 1e-8, rel=1e-9)


def test_source_in_a_column_gives_the_discrete_parabola():
    """At tau = 1 every post-collision population is w_i (C + S), so the
    steady column obeys the finite-volume balance D (phi_{i-1} - 2 phi_i +
    phi_{i+1}) + S = 0 with D = 1/8, zero flux at x = L, and, at the
    fixed-value face, the anti-bounce-back -w (C_0 + S) + 2 w phi_b: the
    face value acts as phi_b - S (the bounced population carries the
    source's share back), a shift of the order of the source per cell."""
    n = 12
    ph = np.full((1, 1, n), 2, np.uint8)
    S = 1e-3
    o = oracle.OracleLBM(ph, carrier=1, D_ionomer=1.0, k_ms=0.0, bc_in=0, bc_out=1, c_in=0.6, c_out=0.6)
    o.set_source(np.full(ph.shape, S))
    steady.solve(o)
    phi = o.concentration().ravel()
    D = 0.25 * (1.0 - 0.5)   # cs^2 (tau - 1/2) at tau = 1, lattice units
    M = np.zeros((n, n))
    rhs = np.full(n, -S)
    for i in range(n):
        if i > 0:
            M[i, i - 1] += D
            M[i, i] -= D
        if i < n - 1:
            M[i, i + 1] += D
            M[i, i] -= D
    M[0, 0] -= 2 * D          # fixed value on the half-way face x = 0, seen as 0.6 - S
    rhs[0] -= 2 * D * (0.6 - S)
    np.testing.assert_allclose(phi, np.linalg.solve(M, rhs), rtol=0, atol=1e-12)
    f = o.fluxes()
    assert f["J_in"] == pytest.approx(-S * n, rel=1e-12)


def _layer(seed=2):
    ph = inputs.with_reservoir(inputs.pt_cl((9, 9, 20), seed, 0.35, 0.35))
    params = dict(dx_m=5e-9, T_K=333.0, p_atm=1.0, M_kgmol=0.032, knudsen=1, bc_in=0, bc_out=1,
                  c_in=7.7, c_out=0.0, tau_ref=1.0)
    return ph, params


def test_large_conductivity_is_the_uniform_potential_solve():
    ph, params = _layer()
    r = coupled.solve(ph, params, sigma=1e4, phi_m=0.6, k_ref=1e-2)
    assert r["converged"] and r["site"].sum() > 0
    assert np.nanmax(np.abs(r["phi"] - 0.6)) < 1e-6
    # the uncoupled solve: uniform k on the same current-carrying sites
    o = oracle.OracleLBM(ph, react=coupled.ionomer_solid_faces(ph), **dict(params, ionomer_o2=1, k_ms=1e-2))
    o.set_rate_scale(r["site"].astype(float))
    steady.solve(o)
    assert r["current_A_o2"] == pytest.approx(4 * coupled.F * o.reaction_rate()[0], rel=1e-6)


def test_coupling_conserves_current_and_lowers_the_rate():
    ph, params = _layer()
    weak = coupled.solve(ph, params, sigma=1e4, phi_m=0.6, k_ref=1e-2)
    r = coupled.solve(ph, params, sigma=1e-4, phi_m=0.6, k_ref=1e-2)
    assert r["converged"]
    # the membrane passes what the sources draw, and that is 4 F times the O2 consumed
    assert r["membrane_flux_lu"] == pytest.approx(-r["source_sum_lu"], rel=1e-10)
    assert r["current_A_membrane"] == pytest.approx(r["current_A_o2"], rel=1e-10)
    # Eq. 16 with S_e > 0 and a fixed membrane value: the potential falls away from the membrane
    phi = r["phi"]
    assert np.nanmax(phi) <= 0.6 + 1e-12 and np.nanmin(phi) < 0.6 - 1e-3
    # Eq. 17b: a lower potential means a lower rate
    assert r["current_A_o2"] < weak["current_A_o2"]


def test_given_ionomer_diffusivity_keeps_the_coupling_pins():
    """With the ionomer's O2 diffusivity given instead of Eq. 10-13 (a lower
    contrast to the pores), the same conservation holds: the membrane passes
    what the sources draw, 4 F times the O2 consumed, and the potential falls
    away from the membrane; a very large conductivity keeps phi uniform."""
    ph, params = _layer()
    r = coupled.solve(ph, params, sigma=1e-4, phi_m=0.6, k_ref=1e-2, ionomer_D=2e-7)
    assert r["converged"] and r["site"].sum() > 0
    assert r["o2"].D()[ph == 2].max() == pytest.approx(2e-7, rel=1e-12)
    assert r["membrane_flux_lu"] == pytest.approx(-r["source_sum_lu"], rel=1e-10)
    assert r["current_A_membrane"] == pytest.approx(r["current_A_o2"], rel=1e-10)
    assert np.nanmax(r["phi"]) <= 0.6 + 1e-12 and np.nanmin(r["phi"]) < 0.6 - 1e-4
    flat = coupled.solve(ph, params, sigma=1e4, phi_m=0.6, k_ref=1e-2, ionomer_D=2e-7)
    assert np.nanmax(np.abs(flat["phi"] - 0.6)) < 1e-6
    assert r["current_A_o2"] < flat["current_A_o2"]
