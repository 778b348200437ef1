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


def remaining(dq, dq_prev):
    """Geometric tail of a readout that approaches its limit: with the last
    two increments dq, dq_prev of one check interval and ratio rho = dq /
    dq_prev in (0, 1), the change still to come is |dq| rho / (1 - rho);
    no estimate (infinity) otherwise."""
    if dq_prev == 0.0:
        return 0.0 if dq == 0.0 else float("inf")
    rho = dq / dq_prev
    if not 0.0 < rho < 1.0:
        return float("inf")
    return abs(dq) * rho / (1.0 - rho)


# converged instances of the full-size settings at 64^3 (same recipes, other seeds):
#   c2_deff_64   256^3 Pt recipe, D_eff set-up (Knudsen D, Dirichlet 1 -> 0, no reaction)
#   c2_react_64  256^3 Pt recipe, reactive set-up (reservoir plane, 5 % catalytic faces, k = 1e-3 m/s,
#                zero-flux outlet)
#   c3_react_64  400^3 NPMC recipe at its 1 nm voxels (micropores, every pore-solid face catalytic,
#                k = 1e-5 m/s, zero-flux outlet)
CONVERGED = {
    "c2_deff_64": ("pt_cl_256", 41, False),
    "c2_react_64": ("pt_cl_256", 41, True),
    "c3_react_64": ("npmc_cl_400", 42, True),
}


def converged(name, edge=64, chunk=1000, rel=1e-10, max_steps=3_000_000):
    """March the FP64 oracle in chunks until the tracked readout (J_out for
    D_eff, R for reactive runs) has an estimated remaining relative change
    below `rel` and the per-step balance J_in = J_out + R holds to 1e-8, at
    two checks in a row; store the readouts and the extrapolated limit."""
    recipe, seed, reactive = CONVERGED[name]
    ph, react, params = inputs.make_workload(recipe, shape=(edge, edge, edge), seed=seed, reactive=reactive)
    o = oracle.OracleLBM(ph, react=react, **params)
    t0 = time.time()
    key = "R" if reactive else "J_out"
    hist = []
    quiet = 0
    steps = 0
    while steps < max_steps:
        o.step(chunk)
        steps += chunk
        f = o.fluxes()
        hist.append(f[key])
        bal = abs(f["J_in"] - f["J_out"] - f["R"]) / abs(f["J_in"])
        if len(hist) >= 3:
            rem = remaining(hist[-1] - hist[-2], hist[-2] - hist[-3])
            quiet = quiet + 1 if (rem < rel * abs(hist[-1]) and bal < 1e-8) else 0
            if quiet >= 2:
                break
    f = o.fluxes()
    d, ratio, dlu = o.effective_diffusivity()
    R, _, _ = o.reaction_rate()
    return dict(workload=recipe, shape=[edge, edge, edge], seed=seed, reactive=reactive, lattice="D3Q7",
                steps=steps, converged=quiet >= 2, seconds=time.time() - t0,
                D_eff_m2s=d, D_eff_over_Db=ratio, D_eff_lu=dlu, R=R, J_in=f["J_in"], J_out=f["J_out"],
                R_lu=f["R"], flux_balance=abs(f["J_in"] - f["J_out"] - f["R"]) / abs(f["J_in"]),
                n_active=f["n_active"], rule=f"remaining change of {key} < {rel} relative, balance < 1e-8, "
                f"two checks of {chunk} steps in a row", threads=oracle.num_threads())


# converged reactive instances by the oracle's exact steady state (oracle/steady.py: the
# fixed point of one step by a sparse direct solve; the march approaches it too slowly
# with a zero-flux outlet): y and z extents multiples of 3
EXACT = {
    "c2_react_48": ("pt_cl_256", 43, True),
    "c3_react_48": ("npmc_cl_400", 44, True),
}


def exact(name, edge=48):
    """The exact steady state of a reactive 48^3 instance: readouts of the
    oracle's populations at the fixed point of its step."""
    from oracle import steady
    recipe, seed, reactive = EXACT[name]
    ph, react, params = inputs.make_workload(recipe, shape=(edge, edge, edge), seed=seed, reactive=reactive)
    o = oracle.OracleLBM(ph, react=react, **params)
    t0 = time.time()
    steady.solve(o)
    f = o.fluxes()
    R, _, _ = o.reaction_rate()
    return dict(workload=recipe, shape=[edge, edge, edge], seed=seed, reactive=reactive, lattice="D3Q7",
                method="exact fixed point of the oracle's step (oracle/steady.py)", converged=True,
                seconds=time.time() - t0, R=R, J_in=f["J_in"], J_out=f["J_out"], R_lu=f["R"],
                flux_balance=abs(f["J_in"] - f["J_out"] - f["R"]) / abs(f["J_in"]), n_active=f["n_active"],
                threads=oracle.num_threads())


if __name__ == "__main__":
    which = sys.argv[1:] or ["c1_deff", "c1_deff_d3q19"]
    for name in which:
        if name in CONVERGED:
            out = converged(name)
        elif name in EXACT:
            out = exact(name)
        else:
            out = c1_deff(lattice=1 if name.endswith("d3q19") else 0)
        print(name, out)
        with open(os.path.join(HERE, name + ".json"), "w") as fh:
            json.dump(out, fh, indent=1)
