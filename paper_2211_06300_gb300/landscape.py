"""Misfit landscape in the transmission case (section "Misfit landscape in transmission case").

A 1D layered model; receivers along the surface and down two vertical lines at the model's
sides; one source at the top-left corner of that frame, on a receiver.  Starting models
m0 = (1 + eps) m_true over a grid of velocity errors eps in [-0.5, 0.5]; at each one the
objectives of classic FWI (Eq. "fwi"), WRI (Eq. "wrimisfit") and ESI (Eq. "esi") at a large
and a small penalty, each from 10 inner CG iterations as in the paper's numerical tests.
Everything runs through the library: esi_gradient's misfit (FWI), esi_wri_solve /
esi_cg_solve followed by the saddle-point esi_gradient with the observed data (WRI / ESI).

Readings (the paper gives neither sizes nor the penalty's scale): the acquisition frame sits
two cells inside the sponge; the penalty is beta = b lambda_max(S^T S) for WRI and
b lambda_max(S^T S) / max B^2 for ESI, b in {100, 0.01}, lambda_max by power iterations on
the true model; the ESI inner solve uses the diagonal preconditioner; the sponge's reference
velocity is the largest velocity of the scan (fixed over eps).
"""
from __future__ import annotations

import argparse
import json
import math
from typing import Dict, Optional, Sequence

import numpy as np

from . import synth


def layered_model(shape=(201, 201), dx: float = 10.0, seed: int = 11, nlayers: int = 5,
                  vmin: float = 1500.0, vmax: float = 3000.0) -> np.ndarray:
    """v(z): nlayers constant layers, velocities increasing with depth, interface depths drawn
    from the seed (at least 3 cells apart)."""
    nz, nx = shape
    rng = np.random.default_rng(seed)
    while True:
        cuts = np.sort(rng.integers(nz // 8, nz - nz // 8, nlayers - 1))
        if np.all(np.diff(np.concatenate([[0], cuts, [nz]])) >= 3):
            break
    vel = np.linspace(vmin, vmax, nlayers)
    v = np.empty(nz)
    edges = np.concatenate([[0], cuts, [nz]])
    for k in range(nlayers):
        v[edges[k]:edges[k + 1]] = vel[k]
    return np.repeat(v[:, None], nx, axis=1)


def acquisition(shape, dx: float, nb: int, step: int = 2) -> synth.Geometry:
    """One shot at the frame's top-left corner; receivers every `step` cells along the
    surface row and down the left and right columns of the frame (the corner receiver
    coincides with the source)."""
    nz, nx = shape
    i0, j0, j1, iz1 = nb + 2, nb + 2, nx - nb - 3, nz - nb - 3
    top = [(j * dx, 0.0, i0 * dx) for j in range(j0, j1 + 1, step)]
    left = [(j0 * dx, 0.0, i * dx) for i in range(i0 + step, iz1 + 1, step)]
    right = [(j1 * dx, 0.0, i * dx) for i in range(i0 + step, iz1 + 1, step)]
    rec = np.asarray(top + left + right, dtype=np.float64)
    src = np.asarray([[j0 * dx, 0.0, i0 * dx]])
    return synth.Geometry(src, np.array([0, rec.shape[0]], dtype=np.int64), rec)


def basin(eps: Sequence[float], J: Sequence[float]) -> Dict:
    """Shape of a sampled curve: local minima (interior samples below both neighbours, plus
    the ends when below their neighbour), the global minimiser, and the interval around it
    over which the curve decreases monotonically toward it (the sampled basin of attraction)."""
    J = np.asarray(J, dtype=np.float64)
    n = len(J)
    mins = [i for i in range(n) if (i == 0 or J[i] < J[i - 1]) and (i == n - 1 or J[i] < J[i + 1])]
    k = int(np.argmin(J))
    lo = k
    while lo > 0 and J[lo - 1] > J[lo]:
        lo -= 1
    hi = k
    while hi < n - 1 and J[hi + 1] > J[hi]:
        hi += 1
    return {"local_minima_eps": [float(eps[i]) for i in mins], "argmin_eps": float(eps[k]),
            "basin_eps": [float(eps[lo]), float(eps[hi])]}


def _power(ctx, nt, shape, device, iters: int = 8) -> float:
    """lambda_max(S^T S) by power iterations (esi_normal_apply with no penalty)."""
    import torch
    gen = torch.Generator(device="cpu").manual_seed(0)
    p = torch.randn((1, nt) + tuple(shape), generator=gen, dtype=torch.float64).to(
        device=device, dtype=ctx.dtype)
    lam = 0.0
    for _ in range(iters):
        p = p / p.norm()
        f = ctx.normal_apply(p, 0.0)
        lam = float((f * p).sum())
        p = f
    return lam


def scan(v_true: np.ndarray, dx: float, dt: float, nt: int, nb: int, f_peak: float,
         eps_grid: Sequence[float], b_values: Sequence[float] = (100.0, 0.01), n_cg: int = 10,
         dtype: str = "f32", device: str = "cuda", step: int = 2,
         betas: Optional[Dict] = None, cg_tol: float = 1e-6, log=None) -> Dict:
    """The objectives along the scan: {"eps", "fwi", "wri": {b: [...]}, "esi": {b: [...]},
    "beta", "lambda_max", "breakdowns"}.  `betas` ({"wri": {b: beta}, "esi": {b: beta}})
    replaces the penalties derived from lambda_max.  An inner solve stops after n_cg
    iterations or at cg_tol; one that meets a breakdown (p^T A p <= 0 once its residual has
    vanished in the field precision) keeps its last iterate, and the event is listed."""
    import torch
    from . import esi
    tdt = torch.float64 if dtype == "f64" else torch.float32
    shape = v_true.shape
    geom = acquisition(shape, dx, nb, step)
    vref = float(v_true.max()) * (1.0 + max(abs(float(e)) for e in eps_grid))
    vt = torch.tensor(v_true, dtype=tdt, device=device)
    ctx = esi.Context(vt, dx, dt, nt, nb, geom, vref=vref)
    wav = torch.tensor(synth.ricker(nt, dt, f_peak)[None, :], dtype=tdt, device=device)
    dobs = ctx.forward(wavelet=wav)
    if betas is None:
        lam_max = _power(ctx, nt, shape, device)
        nz, nx = shape
        xs, zs = geom.src_xyz[0, 0], geom.src_xyz[0, 2]
        bmax = max(math.hypot(x - xs, z - zs) for x in (0.0, (nx - 1) * dx)
                   for z in (0.0, (nz - 1) * dx)) + dx
        beta = {"wri": {b: b * lam_max for b in b_values},
                "esi": {b: b * lam_max / bmax ** 2 for b in b_values}}
    else:
        lam_max, beta = None, betas
        b_values = list(betas["wri"])
    out = {"eps": [float(e) for e in eps_grid], "fwi": [],
           "wri": {b: [] for b in b_values}, "esi": {b: [] for b in b_values},
           "beta": beta, "lambda_max": lam_max, "breakdowns": []}
    q = ctx.empty_field()

    def solve(tag, e, b, **kw):
        try:
            ctx.cg_solve(dobs, tol=cg_tol, max_iter=n_cg, out=q, **kw)
        except esi.EsiError as ex:
            if ex.status != esi.ESI_ERR_BREAKDOWN:
                raise
            out["breakdowns"].append({"eps": float(e), "method": tag, "b": b})
    for e in eps_grid:
        ctx.set_velocity(vt * (1.0 + float(e)))
        _, J = ctx.gradient(wavelet=wav, dobs=dobs, mode="adjoint", param="v")
        out["fwi"].append(J)
        for b in b_values:
            solve("wri", e, b, lam=beta["wri"][b], wri_wavelet=wav)
            _, J = ctx.gradient(wavelet=wav, ext=q, dobs=dobs, mode="wri", beta=beta["wri"][b])
            out["wri"][b].append(J)
            solve("esi", e, b, lam=beta["esi"][b], precond="diag")
            _, J = ctx.gradient(ext=q, dobs=dobs, mode="saddle", beta=beta["esi"][b])
            out["esi"][b].append(J)
        if log:
            print(f"eps {float(e):+.3f} fwi {out['fwi'][-1]:.6e} " +
                  " ".join(f"{m}{b:g} {out[m][b][-1]:.6e}" for m in ("wri", "esi")
                           for b in b_values), file=log, flush=True)
    ctx.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="misfit landscape of FWI, WRI and ESI")
    ap.add_argument("--n", type=int, default=201, help="grid cells per side")
    ap.add_argument("--nt", type=int, default=1200)
    ap.add_argument("--dx", type=float, default=10.0)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--nb", type=int, default=20)
    ap.add_argument("--f-peak", type=float, default=10.0)
    ap.add_argument("--n-eps", type=int, default=21)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--out", default=None, help="write the curves as JSON")
    a = ap.parse_args(argv)
    v = layered_model((a.n, a.n), a.dx)
    eps = np.linspace(-0.5, 0.5, a.n_eps)
    import sys
    r = scan(v, a.dx, a.dt, a.nt, a.nb, a.f_peak, eps, dtype=a.dtype, log=sys.stdout)
    curves = {"fwi": r["fwi"]}
    for m in ("wri", "esi"):
        for b, J in r[m].items():
            curves[f"{m}_b{b:g}"] = J
    res = {"config": vars(a), "eps": r["eps"], "curves": curves,
           "beta": {m: {f"{b:g}": x for b, x in r["beta"][m].items()} for m in ("wri", "esi")},
           "lambda_max": r["lambda_max"], "breakdowns": r["breakdowns"],
           "summary": {k: basin(eps, J) for k, J in curves.items()}}
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)
    print(json.dumps(res["summary"]))
    return res


if __name__ == "__main__":
    main()
