"""Writes the oracle-derived expected values under tests/golden/.

Calls only the FP64 oracle (oracle/) and the seeded structure generator;
nothing from the CUDA path.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1410_1914_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def c1_deff(lattice=0):
    """Plain-method small workload: 48^3 Pt layer at 2 nm, bulk D only,
    Dirichlet 1 -> 0 in x, periodic y, z; converged to a relative change of
    1e-8 per 100 steps (Eq. 19 readout).  lattice 0: D3Q7, 1: D3Q19."""
    ph, react, params = inputs.make_workload("pt_cl_48")
    o = oracle.OracleLBM(ph, react=react, lattice=lattice, **params)
    t0 = time.time()
    steps = o.solve(tol=1e-8, check_every=100, max_steps=2_000_000)
    d, ratio, dlu = o.effective_diffusivity()
    f = o.fluxes()
    return dict(workload="pt_cl_48", lattice=["D3Q7", "D3Q19"][lattice], steps=int(steps), seconds=time.time() - t0, D_eff_m2s=d,
                D_eff_over_Db=ratio, D_eff_lu=dlu, J_in=f["J_in"], J_out=f["J_out"],
                n_active=f["n_active"], tol=1e-8, check_every=100, threads=oracle.num_threads())


if __name__ == "__main__":
    which = sys.argv[1:] or ["c1_deff", "c1_deff_d3q19"]
    for name in which:
        out = c1_deff(lattice=1 if name.endswith("d3q19") else 0)
        print(name, out)
        with open(os.path.join(HERE, name + ".json"), "w") as fh:
            json.dump(out, fh, indent=1)
