"""CUDA path vs the FP64 oracle, through the C ABI (gpu).

Integer set-up products (connectivity, 13-direction lengths, link masks) must
match bit for bit; floating-point results within the FP32 bounds stated in
each test.  Sizes span several 128-wide x tiles with ragged tails.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1410_1914_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _solver(shape, **params):
    from paper_1410_1914_gb300 import Solver
    return Solver(shape, **params)


CASES = {
    # (workload recipe, shape (nz, ny, nx), seed, extra params)
    "pt_ragged": ("pt_cl_256", (13, 17, 291), 21, dict(k_ms=2e4)),
    "pt_deff": ("pt_cl_48", (19, 23, 37), 22, {}),
    "npmc": ("npmc_cl_400", (24, 20, 150), 23, dict(k_ms=5e3)),
}


def _case(name):
    wl, shape, seed, extra = CASES[name]
    ph, react, params = inputs.make_workload(wl, shape=shape, seed=seed)
    params = dict(params, **extra)
    return ph, react, params


@pytest.mark.parametrize("name", sorted(CASES))
def test_setup_bit_exact(cuda_lib, name):
    ph, react, params = _case(name)
    s = _solver(ph.shape, **params)
    s.set_structure(ph, react)
    su = s.setup(chord=True)
    o = oracle.OracleLBM(ph, react=react, **params)
    np.testing.assert_array_equal(su["active"], o.active())
    np.testing.assert_array_equal(su["chord"], oracle.chord_counts(ph))
    # reactive bits of the link mask against the oracle's reactive faces
    np.testing.assert_array_equal((su["mask"] >> 6) & 0x3F, o.react())
    tau = o.tau()
    act = o.active() > 0
    np.testing.assert_allclose(su["omega"][act], 1.0 / tau[act], rtol=1e-6)
    assert np.all(su["omega"][~act] == 0)
    info = s.info()
    assert info["n_active"] == int(act.sum())
    assert info["D_max"] == pytest.approx(o.D_max, rel=1e-12)
    assert info["dt_s"] == pytest.approx(o.dt, rel=1e-12)
    assert info["k_lu"] == pytest.approx(o.k_lu, rel=1e-12)
    s.close()


def test_react_rule_all_pore_solid(cuda_lib):
    """The all-faces rule equals an explicit mask of every pore-solid face."""
    ph, _, params = _case("npmc")
    params = dict(params)
    full = inputs.reactive_faces(ph, 1.0, 0)
    a = _solver(ph.shape, react_rule=1, **params)
    a.set_structure(ph, None)
    b = _solver(ph.shape, **params)
    b.set_structure(ph, full)
    np.testing.assert_array_equal(a.setup()["mask"], b.setup()["mask"])


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("steps", [1, 2, 10, 150])
def test_trajectory(cuda_lib, name, steps):
    ph, react, params = _case(name)
    s = _solver(ph.shape, **params)
    s.set_structure(ph, react)
    s.step(steps)
    o = oracle.OracleLBM(ph, react=react, **params)
    o.step(steps)
    C = s.field()
    ref = o.concentration()
    # FP32 storage and arithmetic: a few ulp of O(1) values per step
    np.testing.assert_allclose(C, ref, rtol=0, atol=2e-6 + 1e-7 * steps)
    fg, fo = s.fluxes(), o.fluxes()
    scale = max(abs(fo["J_in"]), 1e-30)
    assert fg["n_active"] == fo["n_active"]
    assert abs(fg["J_in"] - fo["J_in"]) <= 2e-5 * scale + 1e-6
    assert abs(fg["J_out"] - fo["J_out"]) <= 2e-5 * scale + 1e-6
    assert abs(fg["R"] - fo["R"]) <= 2e-5 * max(abs(fo["R"]), 1e-30) + 1e-6 * scale
    assert fg["sum_C"] == pytest.approx(fo["sum_C"], rel=1e-5)
    tg, pRg, pCg = s.reaction_rate()
    to, pRo, pCo = o.reaction_rate()
    assert tg == pytest.approx(to, rel=2e-5, abs=1e-30)
    np.testing.assert_allclose(pCg, pCo, atol=2e-6 + 1e-7 * steps)
    s.close()


def test_populations_layout(cuda_lib):
    """Post-collision populations, layout [7][nz][ny][nx]; sum = C."""
    ph, react, params = _case("pt_ragged")
    s = _solver(ph.shape, **params)
    s.set_structure(ph, react)
    s.step(3)
    g = s.populations()
    np.testing.assert_allclose(g.sum(axis=0), s.field(), rtol=0, atol=3e-7)
    assert s.steps == 3


def test_custom_init_and_step_counter(cuda_lib):
    ph, react, params = _case("pt_deff")
    rng = np.random.default_rng(0)
    C0 = rng.random(ph.shape).astype(np.float32)
    s = _solver(ph.shape, **params)
    s.set_structure(ph, react)
    s.init(C0)
    s.step(65)  # one 64-step graph + one single step
    o = oracle.OracleLBM(ph, react=react, **params)
    o.init_field(C0.astype(np.float64))
    o.step(65)
    np.testing.assert_allclose(s.field(), o.concentration(), atol=2e-5)
    assert s.steps == 65


def test_converged_deff_small_workload(cuda_lib):
    """48^3 plain-method workload: GPU FP32 solve vs the converged FP64 oracle
    D_eff (tests/golden/c1_deff.json); bound 1e-3 relative."""
    with open(os.path.join(HERE, "golden", "c1_deff.json")) as fh:
        gold = json.load(fh)
    ph, react, params = inputs.make_workload("pt_cl_48")
    s = _solver(ph.shape, check_every=200, tol_rel=1e-5, tol_flux=1e-4, max_steps=3_000_000, **params)
    s.set_structure(ph, react)
    info = s.solve()
    assert info["converged"] == 1, info
    d, ratio = s.effective_diffusivity()
    assert ratio == pytest.approx(gold["D_eff_over_Db"], rel=1e-3)
    assert d == pytest.approx(gold["D_eff_m2s"], rel=1e-3)
