"""Oracle formulas (Eq. 4, 5, 7, 8, 9) against the values the paper prints
(tests/golden/paper_values.json) and against special cases fixed by the
equations' form."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1410_1914_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "paper_values.json")) as fh:
    GOLD = json.load(fh)


def test_eq4_printed_fractions():
    g = GOLD["volume_fractions_eps040"]
    eN, eC, ePt = oracle.volume_fractions(g["eps"])
    # printed to 4 decimals of the fraction; eps_C's last digit differs by one
    assert eN == pytest.approx(g["eps_N"], abs=6e-5)
    assert ePt == pytest.approx(g["eps_Pt"], abs=6e-5)
    assert eC == pytest.approx(g["eps_C"], abs=1.6e-4)
    # Eq. 2: the three solid-side phases fill the non-void volume
    assert eN + eC + ePt == pytest.approx(1 - g["eps"], abs=1e-14)


def test_eq4_weight_ratios_recovered():
    """Eq. 1a-1c: the fractions times densities give back beta_N and theta_Pt."""
    for eps in (0.3, 0.45, 0.6):
        eN, eC, ePt = oracle.volume_fractions(eps)
        mN, mC, mPt = eN * 2000.0, eC * 1800.0, ePt * 21450.0
        assert mN / (mN + mC + mPt) == pytest.approx(0.3, rel=1e-12)
        assert mPt / mC == pytest.approx(0.4, rel=1e-12)


def test_ionomer_to_carbon_ratio():
    eN, eC, ePt = oracle.volume_fractions(0.4)
    assert (eN * 2000.0) / (eC * 1800.0) == pytest.approx(GOLD["ionomer_to_carbon_ratio"]["value"], abs=5e-3)


def test_eq5_pt_loading():
    g = GOLD["pt_loading_4um"]
    _, _, ePt = oracle.volume_fractions(0.4)
    assert oracle.pt_loading(ePt, 21450.0, g["l_cm"]) == pytest.approx(g["value_mg_cm2"], abs=5e-3)
    g2 = GOLD["npmc_loading_4um"]
    _, eC, ePt = oracle.volume_fractions(0.4)
    assert oracle.pt_loading(eC + ePt, g2["rho_solid_mg_cm3"], g2["l_cm"]) == pytest.approx(
        g2["value_mg_cm2"], abs=1.5e-3)


def test_eq8_printed():
    g = GOLD["knudsen_60nm_333K"]
    assert oracle.knudsen_diffusivity(g["d_p_m"], g["T_K"]) == pytest.approx(g["D_kn"], rel=6e-4)
    # Eq. 8's own simplified form 48.5 d_p sqrt(T/32) agrees to its 3 printed digits
    assert oracle.knudsen_diffusivity(g["d_p_m"], g["T_K"]) == pytest.approx(
        48.5 * g["d_p_m"] * np.sqrt(g["T_K"] / 32.0), rel=2e-3)
    # linear in d_p, square root in T, inverse square root in M
    assert oracle.knudsen_diffusivity(2e-8, 300.0) == pytest.approx(2 * oracle.knudsen_diffusivity(1e-8, 300.0), rel=1e-14)
    assert oracle.knudsen_diffusivity(1e-8, 1200.0) == pytest.approx(2 * oracle.knudsen_diffusivity(1e-8, 300.0), rel=1e-14)
    assert oracle.knudsen_diffusivity(1e-8, 300.0, 0.128) == pytest.approx(
        0.5 * oracle.knudsen_diffusivity(1e-8, 300.0, 0.032), rel=1e-14)


def test_eq9_printed_and_limits():
    g = GOLD["bosanquet_60nm"]
    dkn = oracle.knudsen_diffusivity(6e-8, 333.0)
    assert oracle.bosanquet(dkn, g["D_b"]) == pytest.approx(g["D"], rel=1e-3)
    assert oracle.bosanquet(1.0, 1.0) == pytest.approx(0.5, rel=1e-15)
    assert oracle.bosanquet(1e30, 3e-5) == pytest.approx(3e-5, rel=1e-12)


def test_eq7_reference_point_and_scaling():
    g = GOLD["eq7_reference_point"]
    assert oracle.bulk_diffusivity(g["T_K"], g["p_atm"]) == pytest.approx(g["D_b"], rel=1e-15)
    assert oracle.bulk_diffusivity(4 * 293.2, 1.0) == pytest.approx(8 * 2.2e-5, rel=1e-14)
    assert oracle.bulk_diffusivity(293.2, 2.0) == pytest.approx(1.1e-5, rel=1e-14)


def test_workload_literals_match_eq4():
    """The 256^3 and 400^3 workloads state Eq. 4 at porosity 0.45 as literals."""
    eN, eC, ePt = oracle.volume_fractions(0.45)
    assert inputs.EQ4_EPS045_IONOMER == pytest.approx(eN, abs=1e-6)
    assert inputs.EQ4_EPS045_SOLID == pytest.approx(eC + ePt, abs=1e-6)


def test_ionomer_share_literal_matches_eq4():
    for eps in (0.35, 0.5, 0.65):
        eN, eC, ePt = oracle.volume_fractions(eps)
        assert inputs.EQ4_IONOMER_SHARE == pytest.approx(eN / (1 - eps), abs=1e-6)
