"""FP64 oracle of the outer loop: Algorithm "nestedloop" (variable projection between m and q).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``; it shares no code with the CUDA path.

Per outer iteration i the algorithm solves the normal equation for the extended source q
(Algorithm 1, the inner loop), builds the saddle-point gradient from u = A^{-1} q and the
adjoint field lambda = beta B^H B q, turns it into a descent direction with L-BFGS and
updates the model after a line search.  The paper leaves the L-BFGS and line-search details
and the penalty schedule open; this module takes these readings (the CUDA outer loop takes
the same ones, in its own code):

* objective: Eq. "esi", J = 1/2 ||S q - d||^2 + beta/2 ||B q||^2, summed over shots, at the
  inner solution q (WRI: Eq. "wrimisfit" with u = A^{-1}(f + q));
* parameter: the velocity v; the gradient is the saddle-point one (Algorithm 2, "gradewi";
  WRI: "gradient2") through the chain rule to v;
* L-BFGS two-loop recursion (Nocedal & Wright, Algorithm 7.4) over the newest `memory`
  pairs (s, y), initial matrix (s^T y / y^T y) I of the newest pair; a pair is kept only when
  s^T y > 1e-12 ||s|| ||y||; when the direction is not a descent direction, the memory is
  cleared and the steepest descent direction used;
* line search: projected backtracking with the Armijo test J(m_t) <= J(m) + c1 g^T (m_t - m),
  m_t = clip(m + alpha d, vmin, vmax), alpha halved up to max_ls times; first trial alpha = 1
  when the memory holds a pair, else the step that moves the fastest cell by step_frac of the
  largest velocity;
* penalty schedule: beta_i = beta0 * growth^i (a small penalty first, growing over the
  iterations, as the section on the role of the penalty advises); when the
  penalty changes the objective changes, so J and g are re-evaluated and the memory cleared;
* the sponge's reference velocity vref is fixed over the iterations (the damping does not
  follow the model).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import Oracle


@dataclass
class Problem:
    """A seeded inversion problem: grid and time axis, per-shot geometry, observed data
    (and the point-source wavelets, used by WRI only)."""
    dx: float
    dt: float
    nt: int
    nb: int
    vref: float
    src_xyz: Sequence[Sequence[float]]
    rec_xyz: Sequence[np.ndarray]
    d: Sequence[np.ndarray]                    # per shot [nt][nr]
    wavelets: Optional[Sequence[np.ndarray]] = None
    eps: Optional[float] = None


@dataclass
class Options:
    mode: str = "esi"            # "esi" or "wri"
    n_outer: int = 3
    n_cg: int = 10               # inner iterations (the paper's numerical tests use 10)
    cg_tol: float = 0.0
    precond: str = "diag"        # ESI inner solve: "none" or "diag" (z = r / (beta B^2))
    beta0: float = 1.0
    growth: float = 1.0
    memory: int = 5
    c1: float = 1e-4
    step_frac: float = 0.02
    max_ls: int = 8
    vmin: float = -math.inf
    vmax: float = math.inf


def esi_objective(orc: Oracle, sh, q: np.ndarray, d: np.ndarray, beta: float,
                  eps: Optional[float] = None) -> float:
    """Eq. "esi": 1/2 ||S q - d||^2 + beta/2 ||B q||^2 with u = A^{-1} q."""
    B = orc.annihilator(sh.src_xyz, eps)
    e = orc.S(sh, q) - np.asarray(d, dtype=np.float64).reshape(orc.nt, sh.nr)
    qq = np.asarray(q, dtype=np.float64).reshape(orc.nt, orc.N)
    return 0.5 * float(np.sum(e * e)) + 0.5 * beta * float(np.sum((B * B)[None, :] * qq * qq))


def evaluate(v: np.ndarray, pb: Problem, beta: float, opt: Options,
             shots: Optional[Sequence[int]] = None) -> Tuple[float, np.ndarray, List[int]]:
    """J and dJ/dv at the inner solution, summed over the given shots (all by default);
    also the inner iteration counts."""
    orc = Oracle(v, pb.dx, pb.dt, pb.nt, pb.nb, vref=pb.vref)
    J, g, its = 0.0, np.zeros(orc.N), []
    for s in (range(len(pb.src_xyz)) if shots is None else shots):
        sh = orc.shot(pb.src_xyz[s], pb.rec_xyz[s])
        d = np.asarray(pb.d[s], dtype=np.float64).reshape(pb.nt, sh.nr)
        if opt.mode == "esi":
            if opt.precond == "diag":
                B = orc.annihilator(sh.src_xyz, pb.eps)
                res = orc.pcg(sh, d, beta, opt.cg_tol, opt.n_cg, minv=1.0 / (beta * B * B),
                              eps=pb.eps)
            else:
                res = orc.cg(sh, d, beta, opt.cg_tol, opt.n_cg, eps=pb.eps)
            q = res["x"]
            J += esi_objective(orc, sh, q, d, beta, pb.eps)
            g += orc.saddle_gradient(sh, q, beta, param="v", eps=pb.eps)
        else:
            f = pb.wavelets[s]
            res = orc.wri_cg(sh, d, f, beta, opt.cg_tol, opt.n_cg)
            q = res["x"]
            J += orc.wri_objective(sh, q, d, f, beta)
            g += orc.wri_gradient(sh, q, f, beta, param="v")
        its.append(int(res["iters"]))
    return J, g, its


def lbfgs_direction(g: np.ndarray, pairs: Sequence[Tuple[np.ndarray, np.ndarray]]) -> np.ndarray:
    """-H g by the two-loop recursion over pairs (oldest first)."""
    q = np.array(g, dtype=np.float64)
    a = []
    for s, y in reversed(pairs):
        rho = 1.0 / float(np.dot(y, s))
        ai = rho * float(np.dot(s, q))
        q -= ai * y
        a.append((rho, ai))
    if pairs:
        s, y = pairs[-1]
        q *= float(np.dot(s, y)) / float(np.dot(y, y))
    for (s, y), (rho, ai) in zip(pairs, reversed(a)):
        b = rho * float(np.dot(y, q))
        q += (ai - b) * s
    return -q


def minimize(fun: Callable[[np.ndarray, int], Tuple[float, np.ndarray]], x0: np.ndarray,
             opt: Options, beta_of: Callable[[int], float] = lambda i: 0.0) -> Dict:
    """The outer loop around an objective fun(x, i) -> (J, g) whose definition may change
    with the iteration index i (the penalty schedule): L-BFGS direction, projected Armijo
    backtracking, pair update.  History per iteration: J at its start and after its step
    (both under that iteration's penalty), the accepted alpha and the trials taken."""
    x = np.array(x0, dtype=np.float64)
    J, g = fun(x, 0)
    pairs: List[Tuple[np.ndarray, np.ndarray]] = []
    hist = {"J_start": [], "J_end": [], "alpha": [], "trials": [], "beta": [],
            "status": "ok"}
    for i in range(opt.n_outer):
        if i > 0 and beta_of(i) != beta_of(i - 1):
            J, g = fun(x, i)
            pairs = []
        hist["beta"].append(beta_of(i))
        hist["J_start"].append(J)
        d = lbfgs_direction(g, pairs)
        if not float(np.dot(g, d)) < 0:
            pairs = []
            d = -g
        if pairs:
            alpha = 1.0
        else:
            dmax = float(np.max(np.abs(d)))
            if dmax == 0:
                hist["status"] = "zero gradient"
                break
            alpha = opt.step_frac * float(np.max(np.abs(x))) / dmax
            if not alpha > 0:
                hist["status"] = "zero step"
                break
        ok = False
        for t in range(opt.max_ls):
            xt = np.clip(x + alpha * d, opt.vmin, opt.vmax)
            Jt, gt = fun(xt, i)
            if Jt <= J + opt.c1 * float(np.dot(g, xt - x)):
                ok = True
                break
            alpha *= 0.5
        hist["trials"].append(t + 1)
        if not ok:
            hist["status"] = "line search failed"
            break
        s, y = xt - x, gt - g
        if float(np.dot(s, y)) > 1e-12 * float(np.linalg.norm(s)) * float(np.linalg.norm(y)):
            pairs.append((s, y))
            pairs = pairs[-opt.memory:]
        x, J, g = xt, Jt, gt
        hist["J_end"].append(J)
        hist["alpha"].append(alpha)
    hist["x_final"] = x
    hist["g_final"] = g
    return hist


def invert(v0: np.ndarray, pb: Problem, opt: Options,
           reduce: Optional[Callable[[float, np.ndarray], Tuple[float, np.ndarray]]] = None,
           shots: Optional[Sequence[int]] = None) -> Dict:
    """Algorithm "nestedloop" on the velocity.  `shots` restricts the evaluation to this
    rank's shots and `reduce` sums J and g over the ranks (identity by default)."""
    shape = np.asarray(v0).shape
    its_all: List[List[int]] = []

    def beta_of(i):
        return opt.beta0 * opt.growth ** i

    def fun(x, i):
        J, g, its = evaluate(x.reshape(shape), pb, beta_of(i), opt, shots)
        its_all.append(its)
        if reduce is not None:
            J, g = reduce(J, g)
        return J, g
    h = minimize(fun, np.asarray(v0, dtype=np.float64).ravel(), opt, beta_of)
    h["v"] = h["x_final"].reshape(shape)
    h["inner_iters"] = its_all
    return h
