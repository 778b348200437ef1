"""Tile shapes of the plane-marching step kernel (gpu).

A thread block of the (C, delta) step kernel marches a column of 512 cells
along z: 64 x 8, 32 x 16 or 16 x 32 cells (1, 2 or 4 tile rows per warp).
The shape is a layout choice only: every cell takes the same arithmetic on
the same operands, so the state after any number of steps must be bit for
bit the same for every shape, and each must match the FP64 oracle within
the storage's bound (tests/tolerances.py).  The fused reduction of the check
step sums the same terms in another block order, so the fluxes agree to
FP64 rounding.  Boxes with ragged x and y extents (rows of 45, 70 and 291
cells, 5 to 40 rows) put partial tiles on both edges for every shape.  A
batch of members with mixed shapes must step bit-identically to its members
stepped alone.
"""
import numpy as np
import pytest

import oracle
from paper_1410_1914_gb300 import inputs
from tolerances import field_tol, step_sampled

pytestmark = pytest.mark.gpu

CASES = {
    # (workload recipe, shape (nz, ny, nx), seed, extra params)
    "pt_ragged": ("pt_cl_256", (13, 17, 291), 71, dict(k_ms=2e4)),
    "npmc_70": ("npmc_cl_400", (9, 40, 70), 72, dict(k_ms=5e3)),
    "pt_thin": ("pt_cl_48", (21, 5, 45), 73, {}),
}
STEPS = 30


def _run(storage, ph, react, params, rows):
    from paper_1410_1914_gb300 import Solver
    s = Solver(ph.shape, storage=storage, check_every=STEPS, **params)
    s.set_structure(ph, react)
    assert s.set_tile_rows(rows) == rows
    info = s.solve_budget(STEPS)  # STEPS - 1 plain steps and the reducing step
    assert s.steps == STEPS
    return s, info


@pytest.mark.parametrize("storage", ["fp32", "fp16dev"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_shapes_bit_identical_and_against_oracle(cuda_lib, storage, name):
    wl, shape, seed, extra = CASES[name]
    ph, react, params = inputs.make_workload(wl, shape=shape, seed=seed)
    params = dict(params, **extra)
    pops, infos, fields = {}, {}, {}
    for rows in (1, 2, 4):
        s, info = _run(storage, ph, react, params, rows)
        pops[rows] = s.populations()
        fields[rows] = s.field()
        infos[rows] = info
        s.close()
    for rows in (2, 4):
        np.testing.assert_array_equal(pops[rows], pops[1], err_msg=f"rows {rows}")
        for key in ("J_in", "J_out", "R"):
            assert infos[rows][key] == pytest.approx(infos[1][key], rel=1e-12, abs=0), (rows, key)
    o = oracle.OracleLBM(ph, react=react, **params)
    dmax = step_sampled(o, STEPS)
    err = float(np.abs(fields[1] - o.concentration()).max())
    assert err <= field_tol(storage, STEPS, dmax), err
    fo = o.fluxes()
    rel = {"fp32": 1e-6, "fp16dev": 5e-4}[storage]
    # J_in is a sum over the inlet plane of differences of O(1) values: each cell's share
    # carries the storage's rounding (the full-size tests use the same floor)
    floor = {"fp32": 1e-9, "fp16dev": 2e-6}[storage] * shape[0] * shape[1] + 1e-7
    for rows in (1, 2, 4):
        assert abs(infos[rows]["J_in"] - fo["J_in"]) <= rel * abs(fo["J_in"]) + floor, rows
        if fo["R"] > 0:
            assert infos[rows]["R"] == pytest.approx(fo["R"], rel=rel, abs=0), rows


def test_default_shape_and_arguments(cuda_lib):
    from paper_1410_1914_gb300 import Solver
    from paper_1410_1914_gb300 import _lib as L
    # least modelled cost: idle lanes along x (64 rows, a multiple of every tile height), ties to the wider tile
    for nx, rows in ((256, 1), (400, 4), (96, 2), (45, 4), (128, 1), (160, 2)):
        s = Solver((4, 64, nx), storage="fp16dev", dx_m=5e-9, knudsen=0)
        assert s.set_tile_rows(0) == rows, nx
        s.close()
    s = Solver((4, 6, 70), storage="fp32", dx_m=5e-9, knudsen=0)
    for bad in (3, -1, 8):
        with pytest.raises(L.ClError) as e:
            s.set_tile_rows(bad)
        assert e.value.status == L.CL_ERR_ARG
    s.close()
    p = Solver((4, 6, 70), storage="fp32pop", dx_m=5e-9, knudsen=0)
    with pytest.raises(L.ClError) as e:
        p.set_tile_rows(2)
    assert e.value.status == L.CL_ERR_STATE
    p.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16dev"])
def test_batch_of_mixed_shapes_equals_single_steps(cuda_lib, storage):
    from paper_1410_1914_gb300 import Solver
    from paper_1410_1914_gb300.batch import Batch
    members = [("pt_cl_256", (20, 30, 70), 81, dict(k_ms=2e4), 1),
               ("npmc_cl_400", (33, 17, 45), 82, dict(k_ms=5e3), 2),
               ("pt_cl_256", (12, 40, 130), 83, dict(k_ms=1e4), 4),
               ("pt_cl_48", (24, 24, 24), 84, {}, 0)]

    def make():
        out = []
        for wl, shape, seed, extra, rows in members:
            ph, react, params = inputs.make_workload(wl, shape=shape, seed=seed)
            s = Solver(ph.shape, storage=storage, check_every=20, **dict(params, **extra))
            s.set_structure(ph, react)
            s.set_tile_rows(rows)
            out.append(s)
        return out

    alone, together = make(), make()
    for s in alone:
        s.set_tile_rows(0)  # stepped alone in the default shape
        s.step(26)
    b = Batch(together, z_chunk=8)
    b.configure(8, 0, 0)  # each member's own shape: three shapes in one launch
    b.step(13)
    b.configure(16, 2, 4)  # then every member in 16 x 32 tiles
    b.step(13)
    for sa, sb in zip(alone, together):
        np.testing.assert_array_equal(sb.populations(), sa.populations())
    b.close()
    for s in alone + together:
        s.close()
