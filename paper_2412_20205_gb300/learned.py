"""Training pipeline of the learned post-smoother (network kernels in cnn.cu).

Data: for seeded random smooth right-hand sides on one grid, the discrete
solution u_h is computed by the solver itself (FP64, relative residual
1e-13).  Then igamg_training_pairs runs restarted RRE (Algorithm 5) from
s_0 = 0 in the library, probing every V-cycle at the iterate x_mid just
before the finest-level post-smoothing; each V-cycle yields one pair
(r, e) = (b - A x_mid, u_h - x_mid).  The network has no biases, so it is
positively homogeneous (net(c r) = c net(r) for c > 0): a pair scaled by any
positive c is an equally valid example, and each pair is scaled to unit RMS
error, which gives every V-cycle the same weight in the loss.

Training: minibatch gradients of 0.5 mean((net(r) - e)^2) by igamg_cnn_grad
and Adam steps by igamg_adam_step with a cosine learning-rate decay; PyTorch
only holds the tensors and draws the minibatch indices.

Command line (GPU):
  python -m paper_2412_20205_gb300.learned train --out W.npy
  python -m paper_2412_20205_gb300.learned eval --weights W.npy
"""
import argparse
import math
import time

import numpy as np
import torch

from . import (Solver, igamg_adam_step, igamg_cnn_grad, igamg_cnn_num_weights, igamg_cnn_workspace_bytes,
               igamg_training_pairs, igamg_training_workspace_bytes)


def _coeffs(seed, modes):
    """Seeded N(0, 1) sine-series coefficients (modes x modes)."""
    return np.random.default_rng(seed).standard_normal((modes, modes))


def generate_pairs(n=256, p=3, problems=420, k=5, seed0=0, modes=16, tol=1e-10, max_restarts=20,
                   device="cuda"):
    """Returns (R, E) float32 tensors of shape (pairs, m, m), m = n + p - 2:
    per problem the discrete solution by an FP64 solve to 1e-13, then the
    pairs of its restarted RRE run from igamg_training_pairs."""
    s = Solver(2, p, n, k=k, device=device)
    m = s.levels[-1][0]
    N = s.N
    per = (k + 1) * max_restarts                    # most pairs one problem can give
    Rb = torch.empty((per, N), dtype=torch.float32, device=device)
    Eb = torch.empty_like(Rb)
    ws = torch.empty(igamg_training_workspace_bytes(s.ctx, k), dtype=torch.uint8, device=device)
    R, E = [], []
    for i in range(problems):
        b = s.rhs_sine(_coeffs(seed0 + i, modes))
        uh = s.solve(b, tol=1e-13, method="rre", k=k, prec="fp64", max_cycles=100)["x"].clone()
        c = igamg_training_pairs(s.ctx, b, uh, k, tol, max_restarts, Rb, Eb, ws)
        R.append(Rb[:c].clone())
        E.append(Eb[:c].clone())
    s.close()
    R, E = torch.cat(R), torch.cat(E)
    return R.view(-1, m, m), E.view(-1, m, m)


def init_weights(seed=0, device="cuda"):
    """He-style initialisation, last layer scaled down (small initial corrections)."""
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal(16 * 9) * math.sqrt(2.0 / 9)
    w2 = rng.standard_normal(16 * 16 * 9) * math.sqrt(2.0 / 144)
    w3 = rng.standard_normal(16 * 9) * math.sqrt(1.0 / 144) * 0.1
    w = np.concatenate([w1, w2, w3])
    assert w.size == igamg_cnn_num_weights()
    return torch.tensor(w, dtype=torch.float32, device=device)


def train(R, E, steps=1000, batch=16, lr=2e-3, lr_min=1e-5, seed=0, w=None, log_every=0):
    """Adam on minibatches of the pairs with cosine decay lr -> lr_min;
    returns (weights, [(step, minibatch loss)])."""
    device = R.device
    P, H, W = R.shape
    w = init_weights(seed, device) if w is None else w.clone()
    m1 = torch.zeros_like(w)
    m2 = torch.zeros_like(w)
    grad = torch.empty_like(w)
    loss = torch.empty(1, dtype=torch.float32, device=device)
    ws = torch.empty(igamg_cnn_workspace_bytes(batch, H, W), dtype=torch.uint8, device=device)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    for step in range(1, steps + 1):
        idx = torch.randint(0, P, (batch,), generator=gen).to(device)
        r = R.index_select(0, idx).contiguous()
        e = E.index_select(0, idx).contiguous()
        igamg_cnn_grad(batch, H, W, r, e, w, grad, loss, ws)
        a = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * (step - 1) / max(steps - 1, 1)))
        igamg_adam_step(w, grad, m1, m2, step, a)
        if log_every and (step % log_every == 0 or step == 1):
            losses.append((step, float(loss.item())))
    return w, losses


def evaluate(w, n=1024, p=3, seeds=(10000, 10001, 10002, 10003, 10004), k=5, tol=1e-10, modes=16, reps=3,
             stall_ratio=0.95, device="cuda"):
    """Learned vs plain multigrid + RRE in FP32-IR on seeded random right-hand
    sides: cycles, time per solve (median of reps, CUDA events), and the
    relative difference of the solution from an FP64 solve to 1e-13."""
    s = Solver(2, p, n, k=k, device=device)
    s.set_smoother(w, stall_ratio)
    out = []
    for seed in seeds:
        b = s.rhs_sine(_coeffs(seed, modes))
        ref = s.solve(b, tol=1e-13, method="rre", k=k, prec="fp64", max_cycles=200)["x"].clone()
        row = {"seed": seed}
        for prec in ("fp32_ir", "fp32_ir_learned"):
            o = s.solve(b, tol=tol, method="rre", k=k, prec=prec)
            ts = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                o = s.solve(b, tol=tol, method="rre", k=k, prec=prec)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            row[prec] = {"cycles": o["cycles"], "vcycles": o["vcycles"], "ms": float(np.median(ts)),
                         "converged": bool(o["converged"]), "fell_back": o.get("fell_back", False),
                         "err_vs_fp64": float((o["x"] - ref).norm() / ref.norm())}
        out.append(row)
    s.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2412_20205_gb300.learned")
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", required=True)
    t.add_argument("--problems", type=int, default=420)
    t.add_argument("--steps", type=int, default=4000)
    t.add_argument("--batch", type=int, default=16)
    t.add_argument("--lr", type=float, default=2e-3)
    t.add_argument("--seed", type=int, default=0)
    e = sub.add_parser("eval")
    e.add_argument("--weights", required=True)
    e.add_argument("--n", type=int, default=1024)
    e.add_argument("--p", type=int, nargs="+", default=[3, 4])
    a = ap.parse_args(argv)
    if a.cmd == "train":
        t0 = time.time()
        R, E = generate_pairs(problems=a.problems)
        torch.cuda.synchronize()
        t1 = time.time()
        print(f"pairs {tuple(R.shape)}  generation {t1 - t0:.1f} s", flush=True)
        w, losses = train(R, E, steps=a.steps, batch=a.batch, lr=a.lr, seed=a.seed, log_every=max(a.steps // 20, 1))
        torch.cuda.synchronize()
        print(f"training {time.time() - t1:.1f} s  loss {[(s, round(l, 4)) for s, l in losses]}", flush=True)
        np.save(a.out, w.cpu().numpy())
    else:
        w = torch.tensor(np.load(a.weights), dtype=torch.float32, device="cuda")
        for p in a.p:
            for row in evaluate(w, n=a.n, p=p):
                print({"n": a.n, "p": p, **row}, flush=True)


if __name__ == "__main__":
    main()
