"""Pins of the oracle's outer loop (Algorithm "nestedloop") against facts that do not come
from its own code: the dense BFGS inverse-Hessian update, the known minimisers of a quadratic
and of Rosenbrock's function, the Armijo condition, the identity J = 1/2 ||d||^2 -
1/2 <S^T d, q> of Eq. "esi" at the exact inner solution, and central differences of the
reduced objective."""
import numpy as np
import pytest

import oracle
from oracle import outer
from paper_2211_06300_gb300 import synth


def _dense_bfgs_inverse(pairs, n):
    """H_{k+1} = (I - rho s y^T) H_k (I - rho y s^T) + rho s s^T from H_0 = gamma I."""
    s, y = pairs[-1]
    H = (s @ y) / (y @ y) * np.eye(n)
    for s, y in pairs:
        rho = 1.0 / (y @ s)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


def test_two_loop_recursion_equals_the_dense_bfgs_update():
    n = 9
    M = synth.normal(1, (n, n))
    A = M @ M.T + n * np.eye(n)
    pairs = [(synth.normal(10 + k, (n,)), None) for k in range(4)]
    pairs = [(s, A @ s) for s, _ in pairs]
    g = synth.normal(20, (n,))
    H = _dense_bfgs_inverse(pairs, n)
    assert np.allclose(outer.lbfgs_direction(g, pairs), -H @ g, rtol=1e-12, atol=1e-12)
    assert np.allclose(outer.lbfgs_direction(g, []), -g)


def _run(fun, x0, **kw):
    opt = outer.Options(**kw)
    calls = []

    def f(x, i):
        J, g = fun(x)
        calls.append((x.copy(), J, g.copy()))
        return J, g
    return outer.minimize(f, x0, opt), calls


def test_quadratic_reaches_its_minimiser():
    n = 6
    M = synth.normal(2, (n, n))
    A = M @ M.T + np.eye(n)
    b = synth.normal(3, (n,))
    h, _ = _run(lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b), np.ones(n), n_outer=40,
                memory=n, step_frac=1.0)
    x = h["x_final"]
    xs = np.linalg.solve(A, b)
    assert oracle.rel_l2(x, xs) < 1e-8
    assert np.all(np.diff(h["J_end"]) <= 0)


def test_rosenbrock_minimiser_and_armijo_at_every_accepted_step():
    def rosen(x):
        a, b = x
        J = (1 - a) ** 2 + 100 * (b - a * a) ** 2
        g = np.array([-2 * (1 - a) - 400 * a * (b - a * a), 200 * (b - a * a)])
        return J, g
    x0 = np.array([-1.2, 1.0])
    h, calls = _run(rosen, x0, n_outer=200, memory=5, step_frac=0.05, max_ls=30, c1=1e-4)
    assert np.abs(h["x_final"] - 1.0).max() < 1e-6
    # each accepted step meets the Armijo test against the previous accepted point
    xs = [x0] + [None] * 0
    J0, g0 = rosen(x0)
    x_prev, J_prev, g_prev = x0, J0, g0
    for J_end in h["J_end"]:
        # find the accepted evaluation with this J
        x_acc = next(c[0] for c in calls if c[1] == J_end)
        assert J_end <= J_prev + 1e-4 * g_prev @ (x_acc - x_prev) + 1e-15
        x_prev, J_prev, g_prev = x_acc, J_end, rosen(x_acc)[1]


def test_bounds_hold_for_every_trial():
    seen = []

    def fun(x):
        seen.append(x.copy())
        return float(np.sum((x - 5.0) ** 2)), 2 * (x - 5.0)
    h, _ = _run(fun, np.array([1.0, 2.0, 3.0]), n_outer=10, vmin=0.5, vmax=4.0, step_frac=0.5)
    assert all(np.all((x >= 0.5) & (x <= 4.0)) for x in seen)
    assert np.allclose(h["x_final"], 4.0)


def _tiny(nt=10, shape=(10, 11), seed=9):
    dx, dt, nb = 10.0, 1e-3, 3
    v = synth.dipping_layers(shape, dx, seed, nlayers=3, vmin=1500, vmax=2300, nanom=1,
                             sigma=20.0)
    orc = oracle.Oracle(v, dx, dt, nt, nb, vref=2500.0)
    sh = orc.shot((52.0, 0.0, 30.0), [(x, 0.0, 30.0) for x in np.arange(5.0, 105.0, 10.0)])
    return v, orc, sh


def test_esi_objective_identity_at_the_exact_inner_solution():
    _, orc, sh = _tiny()
    beta = 2e-3
    d = synth.normal(31, (orc.nt, sh.nr))
    A = orc.assemble_normal(sh, beta)
    b = orc.ST(sh, d).ravel()
    q = np.linalg.solve(0.5 * (A + A.T), b).reshape(orc.nt, orc.N)
    J = outer.esi_objective(orc, sh, q, d, beta)
    assert J == pytest.approx(0.5 * float(np.sum(d * d)) - 0.5 * float(b @ q.ravel()), rel=1e-10)
    # the inner solution minimises J over q
    assert outer.esi_objective(orc, sh, 1.01 * q, d, beta) > J


def _problem(nt=40, shape=(14, 16), mode="esi"):
    dx, dt, nb = 10.0, 1e-3, 4
    v = synth.dipping_layers(shape, dx, 5, nlayers=3, vmin=1500, vmax=2300, nanom=1, sigma=25.0)
    vt = v + synth.gaussian_blob(shape, dx, 3, amp=60.0, sigma=30.0)
    srcs = [(45.0, 0.0, 40.0), (105.0, 0.0, 40.0)]
    recs = [np.array([(x, 0.0, 40.0) for x in np.arange(5.0, 155.0, 10.0)])] * 2
    f = synth.ricker(nt, dt, 45.0)
    o_true = oracle.Oracle(vt, dx, dt, nt, nb, vref=2500.0)
    d = [o_true.forward(o_true.shot(s, r), wavelet=f)["traces"] for s, r in zip(srcs, recs)]
    pb = outer.Problem(dx, dt, nt, nb, 2500.0, srcs, recs, d, wavelets=[f, f])
    return v, vt, pb


@pytest.mark.parametrize("mode,beta", [("esi", 2e-5), ("wri", 5e-2)])
def test_reduced_gradient_taylor(mode, beta):
    """J(v) at a tight inner solution: its derivative along a smooth direction is the
    saddle-point gradient (variable projection), O(h^2) central differences."""
    v, _, pb = _problem()
    opt = outer.Options(mode=mode, n_cg=4000, cg_tol=1e-13, precond="diag")
    J0, g, _ = outer.evaluate(v, pb, beta, opt)
    dv = synth.gaussian_blob(v.shape, pb.dx, 7, amp=1.0, sigma=30.0)
    errs = []
    for h in (2.0, 1.0):
        Jp = outer.evaluate(v + h * dv, pb, beta, opt)[0]
        Jm = outer.evaluate(v - h * dv, pb, beta, opt)[0]
        fd = (Jp - Jm) / (2 * h)
        errs.append(abs(fd - float(g @ dv.ravel())) / abs(fd))
    assert errs[-1] < 2e-5
    assert errs[0] / errs[1] > 3.0


def test_outer_loop_decreases_the_objective_and_resets_memory_on_a_new_penalty():
    v, _, pb = _problem(nt=30)
    opt = outer.Options(mode="esi", n_outer=4, n_cg=10, beta0=0.1, growth=1.0, vmin=1400,
                        vmax=2600)
    h = outer.invert(v, pb, opt)
    assert h["status"] == "ok"
    assert all(e < s for s, e in zip(h["J_start"], h["J_end"]))
    assert all(h["J_start"][i + 1] == h["J_end"][i] for i in range(len(h["J_end"]) - 1))
    # with a schedule the objective changes at every iteration: J is re-evaluated
    opt2 = outer.Options(mode="esi", n_outer=3, n_cg=10, beta0=0.1, growth=10.0, vmin=1400,
                         vmax=2600)
    h2 = outer.invert(v, pb, opt2)
    assert h2["beta"] == pytest.approx([0.1, 1.0, 10.0])
    assert h2["J_start"][1] != h2["J_end"][0]
    # one iteration: the first trial moves the fastest cell by step_frac of the largest
    # velocity, halved per rejected trial
    h1 = outer.invert(v, pb, outer.Options(mode="esi", n_outer=1, n_cg=10, beta0=0.1,
                                           vmin=1400, vmax=2600))
    step = np.abs(h1["v"] - v).max()
    assert step == pytest.approx(0.02 * v.max() * 0.5 ** (h1["trials"][0] - 1), rel=1e-9)
