"""Pins of the oracle's WRI operators (the CG section: the same CG with B = I and WRI's own
right-hand side, Eq. "normalwri"; Eq. "newq", "wrimisfit", "newadj2", "gradient2") against facts that
do not come from the oracle's WRI code itself: the spectrum of S^T S + beta I, the
data-space closed form of the reduced objective, the large-beta limit, and a Taylor test of
the reduced objective's gradient."""
import numpy as np
import pytest

import oracle
from paper_2211_06300_gb300 import synth


def _tiny(nt=8, shape=(10, 11), seed=9):
    dx, dt, nb = 10.0, 1e-3, 3
    v = synth.dipping_layers(shape, dx, seed, nlayers=3, vmin=1500, vmax=2300, nanom=1,
                             sigma=20.0)
    orc = oracle.Oracle(v, dx, dt, nt, nb)
    src = (52.0, 0.0, 30.0)
    sh = orc.shot(src, [(x, 0.0, 30.0) for x in np.arange(5.0, 105.0, 10.0)])
    f = synth.ricker(nt, dt, 60.0, delay=3 * dt)
    return orc, sh, f


def _assemble(orc, sh, beta):
    n = orc.nt * orc.N
    A = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = orc.wri_matvec(sh, e, beta).ravel()
    return 0.5 * (A + A.T)


def test_wri_spectrum_is_beta_plus_a_rank_limited_psd_part():
    orc, sh, _ = _tiny()
    beta = 3e-3
    A = _assemble(orc, sh, beta)
    ev = np.linalg.eigvalsh(A)
    # S^T S is PSD with rank <= nr * nt (far below the N * nt unknowns): the rest of the
    # spectrum sits exactly at beta
    assert ev[0] == pytest.approx(beta, rel=1e-9)
    above = np.sum(ev > beta * (1 + 1e-6))
    assert 0 < above <= sh.nr * orc.nt
    assert np.sum(np.abs(ev - beta) <= 1e-9 * beta) >= A.shape[0] - sh.nr * orc.nt


def test_wri_cg_reaches_the_cholesky_solution_and_the_closed_form_objective():
    orc, sh, f = _tiny()
    beta = 1e-2
    d = synth.normal(21, (orc.nt, sh.nr))
    res = orc.wri_cg(sh, d, f, beta, tol=1e-13, n_cg=2000)
    A = _assemble(orc, sh, beta)
    L = np.linalg.cholesky(A)
    b = res["b"].ravel()
    x_direct = np.linalg.solve(L.T, np.linalg.solve(L, b))
    assert oracle.rel_l2(res["x"].ravel(), x_direct) < 1e-10
    # reduced objective in data space: J* = 1/2 r0^T (I + S S^T / beta)^{-1} r0, r0 = d - S f
    S = orc.assemble_S(sh)
    r0 = (d - orc.forward(sh, wavelet=f)["traces"]).ravel()
    J_closed = 0.5 * r0 @ np.linalg.solve(np.eye(S.shape[0]) + S @ S.T / beta, r0)
    J = orc.wri_objective(sh, res["x"], d, f, beta)
    assert J == pytest.approx(J_closed, rel=1e-9)
    # a wrong sign of S f in the right-hand side would move the minimiser
    assert orc.wri_objective(sh, res["x"] * 1.01, d, f, beta) > J


def test_wri_large_beta_limit():
    orc, sh, f = _tiny()
    d = synth.normal(22, (orc.nt, sh.nr))
    Sf = orc.forward(sh, wavelet=f)["traces"]
    b = orc.ST(sh, d - Sf)
    # q = (S^T S + beta I)^{-1} b = b / beta - S^T S b / beta^2 + O(beta^-3)
    errs = []
    for beta in (1e8, 1e9):
        x = orc.wri_cg(sh, d, f, beta, tol=1e-14, n_cg=50)["x"]
        errs.append(oracle.rel_l2(x, b / beta))
        second = b / beta - orc.ST(sh, orc.S(sh, b)) / beta ** 2
        assert oracle.rel_l2(x, second) < 1e-3 * errs[-1]
    assert errs[0] / errs[1] == pytest.approx(10.0, rel=1e-3)   # first-order deviation


def test_wri_gradient_taylor():
    """The reduced objective J(m) = min_q J_WRI(m, q): its derivative is the saddle-point
    expression (variable projection), checked by central differences in v."""
    nt, shape, dx, dt, nb = 40, (14, 16), 10.0, 1e-3, 4
    v = synth.dipping_layers(shape, dx, 5, nlayers=3, vmin=1500, vmax=2300, nanom=1, sigma=25.0)
    src = (75.0, 0.0, 40.0)
    recs = [(x, 0.0, 40.0) for x in np.arange(5.0, 155.0, 10.0)]
    f = synth.ricker(nt, dt, 45.0)
    o_true = oracle.Oracle(v + synth.gaussian_blob(shape, dx, 3, amp=60.0, sigma=30.0), dx, dt,
                           nt, nb, vref=2500.0)
    d = o_true.forward(o_true.shot(src, recs), wavelet=f)["traces"]
    beta = 5e-2

    def J_and_q(vv):
        o = oracle.Oracle(vv, dx, dt, nt, nb, vref=2500.0)
        sh = o.shot(src, recs)
        q = o.wri_cg(sh, d, f, beta, tol=1e-14, n_cg=4000)["x"]
        return o.wri_objective(sh, q, d, f, beta), q, o, sh
    J0, q0, o0, sh0 = J_and_q(v)
    g = o0.wri_gradient(sh0, q0, f, beta, param="v").reshape(shape)
    dv = synth.gaussian_blob(shape, dx, 7, amp=1.0, sigma=30.0)
    errs = []
    for h in (4.0, 2.0):
        fd = (J_and_q(v + h * dv)[0] - J_and_q(v - h * dv)[0]) / (2 * h)
        errs.append(abs(fd - float(np.sum(g * dv))) / abs(fd))
    assert errs[-1] < 1e-5
    assert errs[0] / errs[1] > 3.0   # O(h^2)
