"""Training of the learned CG preconditioner with the library's own kernels.

Pairs come from the solver itself: on seeded training models (the dipping-layer recipe of
``synth.workload_esi_2d`` with other seeds) the diagonally preconditioned CG is run to a
tight tolerance for the solution q*, and to k = 1, 2, 3, 5, 8, 12, 16, 20 iterations for
iterates q_k (50 images drawn from each: 5 models x 8 x 50 = 2000 pairs);
the residual r_k = S^T d - (S^T S + beta B^2) q_k, scaled by 1 / (beta B^2) and packed, is
the network input, and the packed error q* - q_k the target (the preconditioned residual
should point along the error).  The objective is the scale-free cosine misfit of
``esi_pc_grad``; Adam updates run on the GPU.

    python -m paper_2211_06300_gb300.pc_train --out paper_2211_06300_gb300/pc_weights.npy
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import esi, synth

TRAIN_SEEDS = (100, 101, 102, 103, 104)
HELD_OUT_SEED = 900


def penalty(ctx1, shape, dx, nt, device, factor: float = 10.0, iters: int = 8) -> float:
    """beta = factor * lambda_max(S^T S) / max B^2 (lambda_max by power iterations on a
    one-shot context)."""
    import torch
    torch.manual_seed(0)
    p = torch.randn((1, nt) + tuple(shape), dtype=torch.float32, device=device)
    lam = 0.0
    for _ in range(iters):
        p = p / p.norm()
        f, _ = ctx1.adjoint(ctx1.forward(ext=p))
        lam = float((f * p).sum())
        p = f
    nz, nx = shape
    far = max(math.hypot(x, z) for x in (0.0, (nx - 1) * dx) for z in (0.0, (nz - 1) * dx))
    return factor * lam / (far + dx) ** 2


def problem(seed: int, nt: int, ns: int, device):
    """Observed data on the true model and a context on the smoothed starting model."""
    import torch
    w = synth.workload_esi_2d(nt=nt, ns=ns, seed=seed)
    vref = float(w.v_true.max())
    ct = esi.Context(torch.tensor(w.v_true, dtype=torch.float32, device=device), w.dx, w.dt, nt,
                     w.nb, w.geom, vref=vref)
    wav = torch.tensor(w.wavelets(), dtype=torch.float32, device=device)
    dobs = ct.forward(wavelet=wav)
    ct.close()
    v0 = torch.tensor(w.v_start, dtype=torch.float32, device=device)
    ctx = esi.Context(v0, w.dx, w.dt, nt, w.nb, w.geom, vref=vref)
    c1 = esi.Context(v0, w.dx, w.dt, nt, w.nb, w.geom.select([0]), vref=vref)
    beta = penalty(c1, w.shape, w.dx, nt, device)
    c1.close()
    return w, ctx, dobs, beta


def make_pairs(seed: int, nt: int, ns: int, iters=(1, 2, 3, 5, 8), per_iter: int = 80,
               device="cuda", rng=None):
    import torch
    rng = rng or np.random.default_rng(seed)
    w, ctx, dobs, beta = problem(seed, nt, ns, device)
    qs, rep = ctx.cg_solve(dobs, lam=beta, tol=1e-5, max_iter=200, precond="diag")
    b, _ = ctx.adjoint(dobs)
    X, E = [], []
    for k in iters:
        qk, _ = ctx.cg_solve(dobs, lam=beta, tol=0.0, max_iter=k, precond="diag")
        rk = ctx.normal_apply(qk, beta)
        torch.sub(b, rk, out=rk)
        xin = ctx.pc_pack(rk, lam=beta, scale=True)
        del rk
        torch.sub(qs, qk, out=qk)
        tgt = ctx.pc_pack(qk)
        del qk
        nimg = xin.shape[0]
        sel = torch.tensor(rng.choice(nimg, size=min(per_iter, nimg), replace=False), device=device)
        X.append(xin[sel].clone())
        E.append(tgt[sel].clone())
        del xin, tgt
    ctx.close()
    return torch.cat(X), torch.cat(E), {"seed": seed, "beta": beta, "iters_to_1e-5": int(max(rep["iters"]))}


def init_vector(seed: int) -> np.ndarray:
    """He-initialised weights, zero biases, zero last layer (the untrained preconditioner is
    exactly the diagonal one).  Layout of esi_pc_param_count()."""
    rng = np.random.default_rng(seed)
    layers = [(16, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 16)]
    out = []
    for li, (ci, co) in enumerate(layers):
        W = rng.standard_normal(9 * ci * co) * math.sqrt(2.0 / (9 * ci))
        if li == len(layers) - 1:
            W[:] = 0.0
        out += [W, np.zeros(co)]
    return np.concatenate(out).astype(np.float32)


def fit(X, E, epochs: int = 6, batch: int = 16, lr: float = 1e-3, seed: int = 0, log=print):
    """Adam on the cosine misfit with the library's forward / backward kernels."""
    import torch
    n, h, w_, _ = X.shape
    net = esi.PCNet(h, w_, batch)
    net.set_params(torch.tensor(init_vector(seed), device=X.device))
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        perm = rng.permutation(n)
        tot, cnt = 0.0, 0
        for i in range(0, n - batch + 1, batch):
            idx = torch.tensor(perm[i:i + batch], device=X.device)
            loss = net.train_step(X[idx].contiguous(), E[idx].contiguous(), lr)
            tot += loss
            cnt += 1
        losses.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep}: mean cosine misfit {losses[-1]:.4f}")
    params = net.get_params()
    net.close()
    return params, losses


def evaluate(params, seed: int = HELD_OUT_SEED, nt: int = 3000, ns: int = 16, tol: float = 1e-3,
             max_iter: int = 60, device="cuda"):
    """Plain, diagonal and learned CG on a held-out model: iterations and time to tol."""
    import torch
    w, ctx, dobs, beta = problem(seed, nt, ns, device)
    ctx.pc_load(params)
    out = {"seed": seed, "beta": beta}
    q = ctx.empty_field()
    for pc in ("none", "diag", "learned"):
        ctx.cg_solve(dobs, lam=beta, tol=tol, max_iter=3, precond=pc, out=q)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = ctx.cg_solve(dobs, lam=beta, tol=tol, max_iter=max_iter, precond=pc, out=q)
        torch.cuda.synchronize()
        out[pc] = {"iters": int(max(rep["iters"])), "converged": bool(rep["converged"]),
                   "time_s": time.perf_counter() - t0,
                   "rel_res": float(max(r[-1] for r in rep["rel_res"] if r.size)),
                   "ms_precond": float(rep["ms_precond"])}
    out["learned_fallbacks"] = ctx.pc_fallbacks
    ctx.close()
    return out


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--nt", type=int, default=3000)
    ap.add_argument("--ns", type=int, default=8)
    ap.add_argument("--per-iter", type=int, default=50)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--iters", default="1,2,3,5,8,12,16,20",
                    help="diagonal-PCG iteration counts whose residual / error pairs are taken")
    ap.add_argument("--eval", action="store_true")
    args = ap.parse_args()
    dev = torch.device("cuda")
    Xs, Es, meta = [], [], []
    t0 = time.perf_counter()
    for s in TRAIN_SEEDS:
        X, E, m = make_pairs(s, args.nt, args.ns, iters=tuple(int(k) for k in args.iters.split(",")),
                             per_iter=args.per_iter, device=dev)
        Xs.append(X)
        Es.append(E)
        meta.append(m)
        print(json.dumps(m), flush=True)
    X, E = torch.cat(Xs), torch.cat(Es)
    print(f"{X.shape[0]} pairs in {time.perf_counter() - t0:.1f} s", flush=True)
    t1 = time.perf_counter()
    params, losses = fit(X, E, epochs=args.epochs, lr=args.lr)
    print(f"trained in {time.perf_counter() - t1:.1f} s", flush=True)
    if args.out:
        np.save(args.out, params.cpu().numpy())
    if args.eval:
        print(json.dumps(evaluate(params)), flush=True)


if __name__ == "__main__":
    main()
