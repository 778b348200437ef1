"""Eq. 28 (Bruggeman form with tau = eps^alpha) as used by the porosity sweep:
the fit returns the exponent of an exact power law, per point and by least
squares, and the paper's convention (Gamma_eff = Gamma eps^1.5 for the
classical tau = eps^-0.5) gives alpha = -0.5."""
import math

import pytest

from paper_1410_1914_gb300.sweep import IONOMER_SHARE, bruggeman_alpha


@pytest.mark.parametrize("alpha", [-0.5, -1.48, -2.11])
def test_power_law_is_recovered(alpha):
    eps = [0.3, 0.4, 0.5, 0.6]
    ratio = [e ** (1.0 - alpha) for e in eps]
    fit = bruggeman_alpha(eps, ratio)
    assert fit["alpha_mean"] == pytest.approx(alpha, abs=1e-12)
    assert fit["alpha_lsq"] == pytest.approx(alpha, abs=1e-12)
    assert all(a == pytest.approx(alpha, abs=1e-12) for a in fit["alpha_per_point"])


def test_classical_bruggeman():
    # Gamma_eff = Gamma eps^1.5 is tau = eps^-0.5 (Sec. 5.1)
    fit = bruggeman_alpha([0.45], [0.45 ** 1.5])
    assert fit["alpha_mean"] == pytest.approx(-0.5, abs=1e-12)


def test_ionomer_share_matches_eq4():
    import oracle
    for eps in (0.3, 0.5):
        eps_N = oracle.volume_fractions(eps)[0]
        assert IONOMER_SHARE * (1 - eps) == pytest.approx(eps_N, rel=2e-6)
