"""Learned warm start of the slip-wall solver (the paper has none).

A convolutional encoder-decoder (lbm_net_*, trained by the library's own
CUDA kernels) maps (solid mask, signed wall distance, Kn) on an H x W
lattice to the steady (rho, u) of a random-cylinder channel; the solver is
then started from those fields (lbm_set_fields: equilibrium plus
first-order non-equilibrium part) and runs to the same residual as from
rest, so the network only ever saves steps -- a poor prediction costs
steps, never accuracy.

Pipeline (all on the GPU through the C ABI):
  1. make_dataset: seeded cylinder arrays, solved together by the batched
     solver to `tol` (targets), inputs from the geometry;
  2. train: Adam on the mean squared error of the normalised fields;
  3. evaluate: held-out cases solved in a batch three times -- from rest,
     from the network's prediction, from a deliberately wrong start (noise)
     -- reporting steps and wall time to `tol`, and the prediction's error
     split into magnitude (the best single scale factor per case) and shape.

Solves use the interval residual (residual_mode 1: the mean change of u per
step over each check interval), with which FP32 solves reach the workload's
1e-8.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import cases as cases_mod
from . import lbm


@dataclasses.dataclass
class Dataset:
    cases: list
    x: np.ndarray          # (n, H, W, 3) float32 network inputs
    y: np.ndarray          # (n, H, W, 3) float32 normalised targets
    uref: np.ndarray       # (n,) velocity scale per case
    steps: np.ndarray      # steps the solver took per case
    converged: np.ndarray  # bool per case


def make_cases(n: int, seed0: int, size: int = 256, kn_range=(0.001, 0.1),
               u_ref: float = 0.01) -> list:
    """Seeded random-cylinder arrays; Kn log-uniform over kn_range, the body
    force set per case so that a H^2 / (8 nu) = u_ref (low Mach number at
    every Kn, so every case has a steady state)."""
    rng = np.random.default_rng(seed0)
    out = []
    for k in range(n):
        Kn = float(math.exp(rng.uniform(math.log(kn_range[0]), math.log(kn_range[1]))))
        c = cases_mod.cylinder_array(size, size, seed0 * 100003 + k, porosity=0.7,
                                     r_max=min(32.0, size / 8.0), Kn=Kn, ax=1.0,
                                     name=f"ws_{seed0}_{k}")
        nu = viscosity(c)
        out.append(dataclasses.replace(c, ax=u_ref * 8.0 * nu / c.H ** 2))
    return out


def viscosity(case) -> float:
    """nu = (tau_s - 1/2) / 3 with tau_s from Kn and H (Eq. tKnrela, Eq. EqViscos)."""
    p = lbm.lbm_params_default()
    _, _, info = lbm.lbm_precompute(case.Kn, case.H, p, [1], [0.5])
    return (info.tau_s - 0.5) / 3.0


def velocity_scale(case) -> float:
    """u_ref = a H^2 / (8 nu), the centre-line speed of a channel of width H."""
    return math.hypot(case.ax, case.ay) * case.H ** 2 / (8.0 * viscosity(case))


def inputs(case) -> np.ndarray:
    """(H, W, 3): solid mask, signed distance / 16, (log10 Kn + 2) / 1."""
    sdf = cases_mod.signed_distance(case) / 16.0
    kn = np.full(case.solid.shape, math.log10(case.Kn) + 2.0)
    return np.stack([case.solid.astype(np.float64), sdf, kn], axis=-1).astype(np.float32)


def encode(rho, ux, uy, uref, solid):
    """Normalised targets: (rho - 1) / uref, u / uref (zero in solids)."""
    fl = solid == 0
    return np.stack([np.where(fl, (rho - 1.0) / uref, 0.0), np.where(fl, ux / uref, 0.0),
                     np.where(fl, uy / uref, 0.0)], axis=-1).astype(np.float32)


def decode(y, uref, solid):
    fl = solid == 0
    rho = np.where(fl, 1.0 + y[..., 0].astype(np.float64) * uref, 1.0)
    ux = np.where(fl, y[..., 1].astype(np.float64) * uref, 0.0)
    uy = np.where(fl, y[..., 2].astype(np.float64) * uref, 0.0)
    return rho, ux, uy


def make_dataset(n: int, seed0: int, size: int = 256, tol: float = 1e-8, max_steps: int = 40000,
                 check_every: int = 100, kn_range=(0.001, 0.1)) -> Dataset:
    """Solve n seeded cases together; keep those that reached tol (a case
    that ran out of steps or went unstable is no target)."""
    cl = make_cases(n, seed0, size, kn_range)
    b = lbm.Batch(cl, precision="fp32", params=[{"residual_mode": 1}] * len(cl))
    steps, res, total = b.run_to(tol, max_steps, check_every)
    keep, xs, ys, urefs = [], [], [], []
    for k, c in enumerate(cl):
        if steps[k] <= 0:
            continue
        rho, ux, uy = b.fields(k)
        if not (np.isfinite(rho).all() and np.isfinite(ux).all() and np.isfinite(uy).all()):
            continue
        u = velocity_scale(c)
        keep.append(k)
        xs.append(inputs(c))
        ys.append(encode(rho, ux, uy, u, c.solid))
        urefs.append(u)
    b.close()
    keep = np.array(keep, np.int64)
    return Dataset([cl[k] for k in keep], np.stack(xs), np.stack(ys), np.array(urefs), steps[keep],
                   np.ones(len(keep), bool))


def train(net, data: Dataset, epochs: int, batch: int, lr: float, seed: int = 0, log=None):
    """Adam on shuffled mini-batches; returns the loss per epoch."""
    import torch

    rng = np.random.default_rng(seed)
    n = data.x.shape[0]
    xs = torch.tensor(data.x, device="cuda")
    ys = torch.tensor(data.y, device="cuda")
    hist = []
    for ep in range(epochs):
        order = rng.permutation(n)
        tot = 0.0
        nb = 0
        for s in range(0, n - batch + 1, batch):
            idx = torch.tensor(order[s:s + batch], device="cuda")
            xb = xs.index_select(0, idx).contiguous()
            yb = ys.index_select(0, idx).contiguous()
            tot += net.train_step(xb.data_ptr(), yb.data_ptr(), batch, lr)
            nb += 1
        hist.append(tot / max(nb, 1))
        if log:
            log(f"epoch {ep} loss {hist[-1]:.4e}")
    return hist


def predict(net, cl: list, batch: int):
    """Network fields (rho, ux, uy) for each case."""
    import torch

    out = []
    for s in range(0, len(cl), batch):
        part = cl[s:s + batch]
        x = torch.tensor(np.stack([inputs(c) for c in part]), device="cuda")
        y = torch.empty((len(part), part[0].ny, part[0].nx, 3), device="cuda")
        net.forward(x.data_ptr(), len(part), y.data_ptr())
        yh = y.cpu().numpy()
        for k, c in enumerate(part):
            out.append(decode(yh[k], velocity_scale(c), c.solid))
    return out


def evaluate(net, cl: list, tol: float = 1e-8, max_steps: int = 40000, check_every: int = 100,
             batch: int = 8, seed: int = 0, exact: bool = False) -> dict:
    """Steps and wall time to `tol` for the held-out cases from rest, from the
    network's fields, and from noise (fallback check); with exact=True also
    from the converged fields themselves (what any predictor could save)."""
    import torch

    preds = predict(net, cl, batch) if net is not None else None
    rng = np.random.default_rng(seed)
    result = {}
    modes = ["rest"] + (["network"] if net is not None else []) + ["noise"] + (["exact"] if exact else [])
    for mode in modes:
        b = lbm.Batch(cl, precision="fp32", params=[{"residual_mode": 1}] * len(cl))
        t0 = time.perf_counter()
        if mode != "rest":
            for k, c in enumerate(cl):
                if mode == "network":
                    rho, ux, uy = preds[k]
                elif mode == "exact":
                    rho, ux, uy = result["rest"]["fields"][k]
                else:
                    u = velocity_scale(c)
                    fl = c.solid == 0
                    rho = 1.0 + 0.01 * u * rng.standard_normal(c.solid.shape) * fl
                    ux = 2.0 * u * rng.standard_normal(c.solid.shape) * fl
                    uy = 2.0 * u * rng.standard_normal(c.solid.shape) * fl
                b.set_fields(k, rho, ux, uy)
        torch.cuda.synchronize()
        steps, res, total = b.run_to(tol, max_steps, check_every)
        wall = time.perf_counter() - t0
        fields = [b.fields(k) for k in range(len(cl))]
        b.close()
        result[mode] = dict(steps=steps, residual=res, total=total, wall=wall, fields=fields)
    if preds is None:
        return result
    # the network's error against the converged state (from rest): velocity
    # rel. L2; the same after the best single scale factor of the predicted
    # velocity (what remains is the error of the flow's shape); density
    # (rho - 1) rel. L2
    err, shape, dens, scale = [], [], [], []
    for k, c in enumerate(cl):
        fl = c.solid == 0
        rho, ux, uy = result["rest"]["fields"][k]
        pr, pu, pv = preds[k]
        den = np.sqrt((ux[fl] ** 2 + uy[fl] ** 2).sum())
        num = np.sqrt(((pu - ux)[fl] ** 2 + (pv - uy)[fl] ** 2).sum())
        pp = (pu[fl] ** 2 + pv[fl] ** 2).sum()
        a = ((pu * ux)[fl].sum() + (pv * uy)[fl].sum()) / pp if pp > 0 else 0.0
        num_s = np.sqrt(((a * pu - ux)[fl] ** 2 + (a * pv - uy)[fl] ** 2).sum())
        dr = np.sqrt(((rho - 1.0)[fl] ** 2).sum())
        err.append(num / den if den > 0 else np.inf)
        shape.append(num_s / den if den > 0 else np.inf)
        dens.append(np.sqrt(((pr - rho)[fl] ** 2).sum()) / dr if dr > 0 else np.inf)
        scale.append(a)
    result["network"]["prediction_error"] = np.array(err)
    result["network"]["shape_error"] = np.array(shape)
    result["network"]["density_error"] = np.array(dens)
    result["network"]["best_scale"] = np.array(scale)
    return result


def main(argv=None):
    """Train on seeded cases and report steps / wall time to tol on held-out
    seeds, from rest versus from the network (and from noise)."""
    import argparse
    import json

    import torch

    from . import build

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-steps", type=int, default=40000)
    ap.add_argument("--base", type=int, default=32)
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--kn-min", type=float, default=0.001)
    ap.add_argument("--kn-max", type=float, default=0.1)
    args = ap.parse_args(argv)
    kn = (args.kn_min, args.kn_max)
    build.build()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    data = make_dataset(args.train, 1, args.size, args.tol, args.max_steps, kn_range=kn)
    t_data = time.perf_counter() - t0
    net = lbm.Net(args.size, args.size, base=args.base, levels=args.levels, precision="bf16",
                  max_batch=args.batch, seed=0)
    t0 = time.perf_counter()
    hist = train(net, data, args.epochs, args.batch, args.lr, log=print)
    t_train = time.perf_counter() - t0
    held = make_cases(args.test, 100000, args.size, kn_range=kn)
    ev = evaluate(net, held, args.tol, args.max_steps, batch=args.batch, exact=True)
    rest, nn_, noise = ev["rest"]["steps"], ev["network"]["steps"], ev["noise"]["steps"]
    ex = ev["exact"]["steps"]
    bx = (rest > 0) & (ex > 0)
    both = (rest > 0) & (nn_ > 0)
    rep = {
        "train_cases": args.train, "test_cases": args.test, "size": args.size,
        "train_converged": len(data.cases), "data_seconds": t_data,
        "train_seconds": t_train, "epochs": args.epochs, "loss_first": hist[0], "loss_last": hist[-1],
        "tol": args.tol, "max_steps": args.max_steps,
        "converged": {"rest": int((rest > 0).sum()), "network": int((nn_ > 0).sum()),
                      "noise": int((noise > 0).sum())},
        "median_steps": {"rest": float(np.median(rest[both])) if both.any() else None,
                         "network": float(np.median(nn_[both])) if both.any() else None},
        "median_step_ratio": float(np.median(nn_[both] / rest[both])) if both.any() else None,
        "step_ratio_quartiles": ([float(v) for v in np.percentile(nn_[both] / rest[both], [25, 75])]
                                 if both.any() else None),
        "prediction_error_median": (float(np.median(ev["network"]["prediction_error"][rest > 0]))
                                    if (rest > 0).any() else None),
        "shape_error_median": (float(np.median(ev["network"]["shape_error"][rest > 0]))
                               if (rest > 0).any() else None),
        "density_error_median": (float(np.median(ev["network"]["density_error"][rest > 0]))
                                 if (rest > 0).any() else None),
        "best_scale_quartiles": ([float(v) for v in np.percentile(ev["network"]["best_scale"][rest > 0],
                                                                  [25, 50, 75])]
                                 if (rest > 0).any() else None),
        "exact_fields_median_step_ratio": float(np.median(ex[bx] / rest[bx])) if bx.any() else None,
        "params": net.n_params,
        "batch_wall_seconds": {m: ev[m]["wall"] for m in ev},
        "batch_total_steps": {m: int(ev[m]["total"]) for m in ev},
    }
    print(json.dumps(rep))
    return rep


if __name__ == "__main__":
    main()
