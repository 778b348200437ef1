"""O2 dissolved in the ionomer (Eq. 10-15), pinned by the physics of the
interface rather than by the oracle's own formula.

In real variables the pore carries the gas concentration C with D_p and the
ionomer carries the dissolved concentration C_e with D_e, and Henry's law
(Eq. 10) makes C_e = C RT/H at the interface and at a fixed-value face
inside the ionomer.  A pore layer in series with an ionomer layer therefore
passes the molar flux (C_in - C_out) / (L_p / D_p + L_i H / (R T D_e)).  The
solver works in the gas-equivalent variable of Eq. 14-15; with
ionomer_o2 = 1 its D_eff must equal that series law (the cell-wise harmonic
mean with D_e RT/H in the ionomer cells), which fails if the RT/H factor of
the interface is dropped (flux continuity).

Eq. 11 and Eq. 13 themselves are written as printed; no value of them is
printed in the paper to pin them against (parity unpinned for those two
formulas).
"""
import numpy as np
import pytest

import oracle

R = 8.314462618


@pytest.mark.parametrize("T,lattice", [(333.0, 0), (353.0, 0), (353.0, 1)])
def test_pore_ionomer_series_slab(T, lattice):
    n_p, n_i = 9, 6
    nx = n_p + n_i
    ph = np.zeros((3, 4, nx), np.uint8)
    ph[:, :, n_p:] = 2                     # ionomer behind the pore layer
    D_p = 1e-9                             # a small bulk D keeps the contrast modest for the test
    o = oracle.OracleLBM(ph, dx_m=1e-8, D_bulk=D_p, T_K=T, ionomer_o2=1, lattice=lattice)
    o.init_field(np.zeros(ph.shape))
    n = o.solve(tol=1e-14, check_every=500, max_steps=20_000_000)
    assert n > 0
    D_e = oracle.ionomer_o2_diffusivity(T)
    H = oracle.henry_constant(T)
    L_p, L_i = n_p * 1e-8, n_i * 1e-8
    flux = 1.0 / (L_p / D_p + L_i * H / (R * T * D_e))       # real molar flux per unit C_in - C_out
    d_eff, _, _ = o.effective_diffusivity()
    assert d_eff == pytest.approx(flux * nx * 1e-8, rel=1e-9)
    # without the RT/H factor the same box would pass a flux larger by H/(RT)
    wrong = 1.0 / (L_p / D_p + L_i / D_e) * nx * 1e-8
    assert abs(d_eff / wrong - 1) > 0.5


def test_ionomer_o2_needs_o2_carrier_and_positive_diffusivity():
    ph = np.zeros((2, 2, 4), np.uint8)
    with pytest.raises(ValueError):
        oracle.OracleLBM(ph, ionomer_o2=1, carrier=1, D_ionomer=1.0)
    with pytest.raises(ValueError):
        oracle.OracleLBM(ph, ionomer_o2=1, T_K=280.0)
