"""Training and use of the learned column scheduler (host driver).

The network, its features and its training steps run in libgsk's kernels
(gsk_features, gsk_mlp_train_step, gsk_mlp_forward); this module only
orchestrates: it runs the solver without a model (FIFO queue) on seeded
training systems to log (features, Lanczos steps) pairs, trains the network
on log(steps) with Adam on the GPU, and saves / loads the model.

    python -m paper_1609_08377_gb300.scheduler train --out paper_1609_08377_gb300/sched_model.json

Training systems: the C/H generators of the 1,000- and 20,000-atom
workloads at seeds 1-5 (the evaluation workloads use seed 0), with per-column
damping drawn from {0.05, 0.1, 0.2}.
"""

from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import gsk
from . import synthetic as syn

MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sched_model.json")


def _torch():
    import torch

    return torch


def collect(solver: gsk.Solver, cols: np.ndarray, eta: np.ndarray, n_shifts: int = 128,
            precision: str = "mixed_df", tol: float = 1e-8):
    """Solve the columns without a model; return (features, steps)."""
    torch = _torch()
    eps = syn.energy_grid(n_shifts)
    z = eps.astype(np.complex128) + 1j
    off = solver.pattern_offsets(cols)
    G = torch.empty(int(off[-1]) * n_shifts, dtype=torch.complex128, device="cuda")
    it, st, _ = solver.solve(z, cols, G, eta=eta, precision=precision, tol=tol, sched="fifo")
    feat = torch.empty((cols.size, gsk.MLP_IN), dtype=torch.float32, device="cuda")
    solver.features(cols, eta, feat)
    ok = st == gsk.GSK_CONVERGED
    return feat.cpu().numpy()[ok], it[ok].astype(np.float64)


def training_set(seeds=(1, 2, 3, 4, 5), n1k: int = 1000, n20k: int = 192, log=print):
    F, Y = [], []
    for seed in seeds:
        for name, n_cols in (("ch1k", n1k), ("ch20k", n20k)):
            if n_cols <= 0:
                continue
            wl = syn.WORKLOADS[name]
            s = syn.make_system(wl.n_atoms, wl.c_fraction, seed)
            solver = gsk.from_system(s)
            cols = syn.column_subset(s.M, n_cols, seed)
            eta = syn.eta_per_column(cols.size, seed)
            t0 = time.time()
            f, y = collect(solver, cols, eta)
            solver.close()
            F.append(f)
            Y.append(y)
            log(f"collected {name} seed {seed}: {len(y)} columns, steps {y.min():.0f}..{y.max():.0f} "
                f"({time.time() - t0:.1f} s)")
    return np.concatenate(F), np.concatenate(Y)


def init_params(seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases (flat layout of include/gsk.h)."""
    rng = np.random.default_rng(seed)
    nh, ni = gsk.MLP_HIDDEN, gsk.MLP_IN
    p = np.zeros(gsk.MLP_NPARAM, dtype=np.float32)
    o = 0
    lim = np.sqrt(6.0 / (ni + nh))
    p[o:o + nh * ni] = rng.uniform(-lim, lim, nh * ni)
    o += nh * ni + nh
    lim = np.sqrt(6.0 / (2 * nh))
    p[o:o + nh * nh] = rng.uniform(-lim, lim, nh * nh)
    o += nh * nh + nh
    lim = np.sqrt(6.0 / (nh + 1))
    p[o:o + nh] = rng.uniform(-lim, lim, nh)
    return p


def fit(F: np.ndarray, steps: np.ndarray, epochs: int = 3000, lr: float = 3e-3, seed: int = 0, log=print):
    """Full-batch Adam on the GPU; returns the model dict."""
    torch = _torch()
    mean = F.mean(axis=0)
    std = F.std(axis=0)
    std = np.where(std < 1e-6, 1.0, std)
    t = np.log(steps)
    t_mean, t_std = float(t.mean()), float(t.std() or 1.0)
    target = (t - t_mean) / t_std
    dev = "cuda"
    n = F.shape[0]
    Xd = torch.from_numpy(F.astype(np.float32)).to(dev)
    Td = torch.from_numpy(target.astype(np.float32)).to(dev)
    norm = torch.from_numpy(np.concatenate([mean, std]).astype(np.float32)).to(dev)
    params = torch.from_numpy(init_params(seed)).to(dev)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    work = torch.empty(gsk.mlp_workspace_bytes(n) // 4 + 1, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    hist = []
    for it in range(1, epochs + 1):
        gsk.mlp_train_step(n, Xd, norm, Td, params, m, v, it, lr, work, loss=loss)
        if it % 500 == 0 or it == 1:
            hist.append((it, float(loss.item())))
            log(f"step {it}: loss {hist[-1][1]:.4f}")
    return {"params": params.cpu().numpy().tolist(), "norm": norm.cpu().numpy().tolist(),
            "target_mean": t_mean, "target_std": t_std, "n_train": int(n), "loss_history": hist}


def predict(model: dict, F: np.ndarray) -> np.ndarray:
    """Predicted Lanczos steps from raw features (runs gsk_mlp_forward)."""
    torch = _torch()
    Xd = torch.from_numpy(np.ascontiguousarray(F, dtype=np.float32)).cuda()
    params = torch.tensor(model["params"], dtype=torch.float32, device="cuda")
    norm = torch.tensor(model["norm"], dtype=torch.float32, device="cuda")
    y = torch.empty(F.shape[0], dtype=torch.float32, device="cuda")
    gsk.mlp_forward(F.shape[0], Xd, norm, params, y)
    return np.exp(y.cpu().numpy() * model["target_std"] + model["target_mean"])


def save(model: dict, path: str = MODEL_PATH) -> None:
    with open(path, "w") as f:
        json.dump(model, f)


def load(path: str = MODEL_PATH) -> dict:
    with open(path) as f:
        return json.load(f)


def install(solver: gsk.Solver, model: dict) -> None:
    solver.set_sched_model(np.asarray(model["params"], dtype=np.float32),
                           np.asarray(model["norm"], dtype=np.float32))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train"])
    ap.add_argument("--out", default=MODEL_PATH)
    ap.add_argument("--n1k", type=int, default=1000)
    ap.add_argument("--n20k", type=int, default=192)
    ap.add_argument("--epochs", type=int, default=3000)
    args = ap.parse_args()
    F, Y = training_set(n1k=args.n1k, n20k=args.n20k)
    model = fit(F, Y, epochs=args.epochs)
    model["training"] = {"systems": "ch1k and ch20k generators, seeds 1-5, eta in {0.05, 0.1, 0.2}",
                         "columns_per_system": {"ch1k": args.n1k, "ch20k": args.n20k},
                         "solver": "gsk_solve, GSK_MIXED_DF, FIFO, tol 1e-8, 128 shifts"}
    save(model, args.out)
    print("saved", args.out, "n_train", model["n_train"])


if __name__ == "__main__":
    main()
