"""Pins of the oracle's data-space CG (the section "Switching from the wavefield to data
space": Eq. "wd", "wv", "q" and the Sherman-Morrison-Woodbury identity that derives them)
against the wavefield-space solution by a dense Cholesky solve, the synthetic-data identity
w = S q, and the spectrum of the data-space operator."""
import numpy as np
import pytest

import oracle
from paper_2211_06300_gb300 import synth


def _tiny(nt=8, shape=(10, 11), seed=9):
    dx, dt, nb = 10.0, 1e-3, 3
    v = synth.dipping_layers(shape, dx, seed, nlayers=3, vmin=1500, vmax=2300, nanom=1,
                             sigma=20.0)
    orc = oracle.Oracle(v, dx, dt, nt, nb)
    sh = orc.shot((52.0, 0.0, 30.0), [(x, 0.0, 30.0) for x in np.arange(5.0, 105.0, 10.0)])
    return orc, sh


def test_data_space_solution_equals_the_wavefield_space_solution():
    orc, sh = _tiny()
    beta = 2e-3
    d = synth.normal(31, (orc.nt, sh.nr))
    res = orc.ds_cg(sh, d, beta, tol=1e-14, n_cg=500)
    A = orc.assemble_normal(sh, beta)
    L = np.linalg.cholesky(0.5 * (A + A.T))
    b = orc.ST(sh, d).ravel()
    q_direct = np.linalg.solve(L.T, np.linalg.solve(L, b))
    assert oracle.rel_l2(res["q"].ravel(), q_direct) < 1e-10
    # w is the synthetic data of the extended source: w = S q
    assert oracle.rel_l2(res["w"], orc.S(sh, res["q"])) < 1e-10


def test_data_space_operator_is_identity_plus_psd():
    orc, sh = _tiny()
    beta = 5e-3
    n = orc.nt * sh.nr
    M = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = (e.reshape(orc.nt, sh.nr) + orc.ds_K(sh, e, beta)).ravel()
    assert np.max(np.abs(M - M.T)) <= 1e-12 * np.max(np.abs(M))
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev[0] >= 1.0 - 1e-12 and ev[-1] > 1.0 + 1e-6


def test_synthetic_data_fits_the_observed_data_as_beta_vanishes():
    """d - w = (I + K/beta)^{-1} d = beta (beta I + K_1)^{-1} d (K_1 = K at beta = 1): with K_1
    invertible on the data the misfit falls linearly in beta (the section's remark that
    w -> d as beta -> 0)."""
    orc, sh = _tiny()
    d = orc.forward(sh, wavelet=synth.ricker(orc.nt, orc.dt, 60.0, delay=3 * orc.dt))["traces"]
    d = d + 1e-3 * np.abs(d).max() * synth.normal(33, d.shape)
    mis = [oracle.rel_l2(orc.ds_cg(sh, d, beta, tol=1e-14, n_cg=2000)["w"], d)
           for beta in (1e-7, 1e-8, 1e-9)]
    assert mis[0] < 1e-5
    assert mis[0] / mis[1] == pytest.approx(10.0, rel=0.05)
    assert mis[1] / mis[2] == pytest.approx(10.0, rel=0.01)
