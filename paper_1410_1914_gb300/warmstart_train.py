"""Training data, training loop and evaluation of the learned warm start.

Data: seeded QSGS cubes (Pt and NPMC layers, porosity 0.35-0.65, Knudsen
diffusivity, D_eff set-up) solved to convergence by the batched LBM; the
network input comes from each solver's set-up (``cl_lbm_features``) and the
target is its converged field minus the linear ramp, times nx.

Evaluation: on held-out cubes, the number of steps until D_eff stays within
1e-3 of the converged value, from the linear ramp and from the network's
prediction, with the same solver and stopping checks.  The LBM still
computes the answer; the network only chooses where it starts.

    python -m paper_1410_1914_gb300.warmstart_train --out weights.npz
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs


def make_dataset(n: int, size: int = 48, seed0: int = 1000, storage: str = "fp32", check_every: int = 200,
                 tol_rel: float = 1e-6, max_steps: int = 4_000_000, net=None):
    """Solve n seeded cubes of edge `size` in one batch; return (features,
    targets, masks, stats).  With `net`, every solve starts from that
    network's warm start (the converged fields, hence the targets, are the
    same; only the number of steps changes)."""
    import torch

    from . import warmstart as W
    from .batch import Batch
    from .solver import Solver
    work = inputs.batch_workloads(n, seed0=seed0, edge_range=(size, size))
    solvers = []
    t0 = time.perf_counter()
    for ph, react, params in work:
        s = Solver(ph.shape, storage=storage, check_every=check_every, tol_rel=tol_rel, tol_flux=1e-4, **params)
        s.set_structure(ph, react)
        if net is not None:
            W.warm_start(net, s)
        solvers.append(s)
    b = Batch(solvers)
    status, infos, nconv = b.solve(max_steps)
    solve_s = time.perf_counter() - t0
    feats = torch.empty(n, size, size, size, W.FEATURES, dtype=torch.bfloat16, device="cuda")
    targets = torch.empty(n, size ** 3, dtype=torch.float32, device="cuda")
    masks = torch.empty(n, size ** 3, dtype=torch.uint8, device="cuda")
    for i, s in enumerate(solvers):
        feats[i] = W.features(s)[0]
        targets[i] = W.target(s)
        masks[i] = W.active_mask(s)
    b.close()
    for s in solvers:
        s.close()
    stats = dict(n=n, size=size, seed0=seed0, tol_rel=tol_rel, storage=storage, warm=net is not None,
                 status=status, converged=nconv,
                 solve_seconds=solve_s, mean_steps=float(np.mean([x["steps"] for x in infos])))
    return feats, targets, masks, stats


def _augment(rng, x, t, m, D):
    """Random y/z rolls and a y<->z transpose: the structures are periodic in
    y and z and statistically isotropic there, so the target moves with them."""
    import torch
    B = x.shape[0]
    sy, sz = int(rng.integers(D)), int(rng.integers(D))
    x = torch.roll(x, shifts=(sz, sy), dims=(1, 2))
    t = torch.roll(t.view(B, D, D, D), shifts=(sz, sy), dims=(1, 2))
    m = torch.roll(m.view(B, D, D, D), shifts=(sz, sy), dims=(1, 2))
    if rng.random() < 0.5:
        x, t, m = x.transpose(1, 2), t.transpose(1, 2), m.transpose(1, 2)
    return x.contiguous(), t.contiguous().view(-1), m.contiguous().view(-1)


def train(net, groups, steps: int, lr: float = 1e-3, seed: int = 0, log_every: int = 100):
    """groups: list of (feats, targets, masks, batch, weight); each step draws
    one group with probability proportional to its weight, then a batch of
    distinct cubes from it.  Cosine learning-rate decay."""
    import torch
    rng = np.random.default_rng(seed)
    w = np.array([g[4] for g in groups], dtype=np.float64)
    w /= w.sum()
    losses = []
    t0 = time.perf_counter()
    for it in range(1, steps + 1):
        feats, targets, masks, batch, _ = groups[int(rng.choice(len(groups), p=w))]
        n, D = feats.shape[0], feats.shape[1]
        idx = torch.from_numpy(rng.choice(n, size=min(batch, n), replace=False)).cuda()
        x, t, m = _augment(rng, feats.index_select(0, idx), targets.index_select(0, idx),
                           masks.index_select(0, idx), D)
        lr_t = lr * 0.5 * (1 + np.cos(np.pi * it / steps))
        net.forward(x, x.shape[0], D)
        net.backward(t, m)
        net.step(lr=float(lr_t))
        if it % log_every == 0 or it == steps:
            net.check()
            losses.append((it, D, net.loss_value(), time.perf_counter() - t0))
    torch.cuda.synchronize()
    return losses


def evaluate(net, size: int = 96, n: int = 4, seed0: int = 5000, storage: str = "fp32", check_every: int = 200,
             max_steps: int = 6_000_000, rel: float = 1e-3, extra_arms=(), base_warm: bool = True):
    """Steps (and seconds) to D_eff within rel, from the ramp and from the
    warm start.  The ramp run is carried on to an extrapolated relative
    change below 1e-9 and its last D_eff is the converged reference.
    extra_arms: further (storage, warm) runs scored against the same
    reference, reported as "<storage>+ramp" / "<storage>+warm"."""
    import torch

    from . import warmstart as W
    from .convergence import deff_trace, time_to_tolerance
    from .solver import Solver
    work = inputs.batch_workloads(n, seed0=seed0, edge_range=(size, size))
    rows = []
    for ph, react, params in work:
        row = {}
        for mode in ("ramp", "warm") if base_warm else ("ramp",):
            s = Solver(ph.shape, storage=storage, check_every=check_every, **params)
            s.set_structure(ph, react)
            t_inf = 0.0
            if mode == "warm":
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                W.warm_start(net, s)
                torch.cuda.synchronize()
                t_inf = time.perf_counter() - t1
            st, sec, val = deff_trace(s, max_steps, check_every, stop_rel_change=1e-9 if mode == "ramp" else 1e-8)
            s.close()
            if mode == "ramp":
                ref = float(val[-1])
                row["reference_D_eff_over_Db"] = ref
            k, secs = time_to_tolerance(st, sec, val, ref, rel)
            row[mode] = {"steps": k, "seconds": None if secs is None else secs + t_inf, "inference_s": t_inf,
                         "final_rel_err": abs(float(val[-1]) - ref) / abs(ref)}
        if "warm" in row and row["ramp"]["steps"] and row["warm"]["steps"]:
            row["steps_saved_frac"] = 1.0 - row["warm"]["steps"] / row["ramp"]["steps"]
        for st_mode, warm in extra_arms:
            s = Solver(ph.shape, storage=st_mode, check_every=check_every, **params)
            s.set_structure(ph, react)
            t_inf = 0.0
            if warm:
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                W.warm_start(net, s)
                torch.cuda.synchronize()
                t_inf = time.perf_counter() - t1
            # FP16 readouts carry ~1e-5 noise: the trace only has to outlast the band
            st, sec, val = deff_trace(s, max_steps, check_every, stop_rel_change=1e-7)
            s.close()
            k, secs = time_to_tolerance(st, sec, val, ref, rel)
            row[f"{st_mode}+{'warm' if warm else 'ramp'}"] = {
                "steps": k, "seconds": None if secs is None else secs + t_inf, "inference_s": t_inf,
                "final_rel_err": abs(float(val[-1]) - ref) / abs(ref)}
        rows.append(row)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", nargs="+", default=["48:256:4", "96:48:1"],
                    help="training groups edge:count:batch (cubes of that edge, solved, batch per step)")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--data-storage", default="fp32", choices=["fp32", "fp16dev"],
                    help="storage mode of the solves that make the training targets")
    ap.add_argument("--data-warm", default=None,
                    help="weights whose warm start speeds up the training solves (targets unchanged)")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval-size", type=int, nargs="+", default=[96])
    ap.add_argument("--n-eval", type=int, default=3)
    ap.add_argument("--out", default="warmstart_weights.npz")
    ap.add_argument("--eval-only", default=None, help="weights to evaluate (no data, no training)")
    ap.add_argument("--eval-seed0", type=int, default=5000)
    ap.add_argument("--eval-fp16", action="store_true", help="also score FP16-state runs from the ramp and warm start")
    ap.add_argument("--eval-no-fp32-warm", action="store_true", help="skip the FP32-state warm-start run")
    ap.add_argument("--eval-check-every", type=int, default=200)
    ap.add_argument("--report", default=None)
    args = ap.parse_args()
    import torch

    from .warmstart import UNet, load_pretrained
    torch.cuda.set_device(0)
    arms = (("fp16dev", False), ("fp16dev", True)) if args.eval_fp16 else ()
    if args.eval_only:
        net = load_pretrained(args.eval_only)
        rows = []
        for size in args.eval_size:
            r = evaluate(net, size, args.n_eval, seed0=args.eval_seed0, extra_arms=arms,
                         base_warm=not args.eval_no_fp32_warm, check_every=args.eval_check_every)
            for x in r:
                x["size"] = size
            print(json.dumps({"eval": r}), flush=True)
            rows += r
        if args.report:
            with open(args.report, "w") as fh:
                json.dump({"eval": rows, "config": vars(args)}, fh, indent=1)
        return
    groups, dstats = [], []
    data_net = None
    if args.data_warm:
        from .warmstart import load_pretrained
        data_net = load_pretrained(args.data_warm)
    for k, spec in enumerate(args.data):
        size, count, batch = (int(v) for v in spec.split(":"))
        f, t, m, st = make_dataset(count, size, seed0=1000 + 10000 * k, storage=args.data_storage,
                                   tol_rel=1e-6 if size <= 64 else 1e-5, net=data_net)
        print(json.dumps({"dataset": st}), flush=True)
        dstats.append(st)
        # equal voxels per draw: weight a group by its cubes' share of the data volume
        groups.append((f, t, m, batch, count * size ** 3))
    net = UNet(seed=0)
    losses = train(net, groups, args.steps, args.lr)
    print(json.dumps({"train": losses[-6:], "params": net.num_params()}), flush=True)
    np.savez_compressed(args.out, **{k: v.astype(np.float16) for k, v in net.state_dict().items()})
    rows = []
    for size in args.eval_size:
        r = evaluate(net, size, args.n_eval, seed0=args.eval_seed0, extra_arms=arms)
        for x in r:
            x["size"] = size
        print(json.dumps({"eval": r}), flush=True)
        rows += r
    rep = {"dataset": dstats, "train_losses": losses, "params": net.num_params(), "eval": rows,
           "config": vars(args)}
    if args.report:
        with open(args.report, "w") as fh:
            json.dump(rep, fh, indent=1)


if __name__ == "__main__":
    main()
