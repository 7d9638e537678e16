"""Pins of the oracle's frequency-domain ESI (the section "Frequency domain inversion by time
domain modelling": Eq. "dtft", "idtft", "normaldtft") against facts that do not come from the
oracle's frequency-domain code itself: numpy's inverse FFT on the DFT grid, the paper's
statement that with as many frequencies as time steps the solve is the time-domain CG, the
Hermitian positive definite structure with a direct solve, and the paper's worked example
(a sum of sines recovered from five frequencies through a Toeplitz operator)."""
import numpy as np

import oracle
from paper_2211_06300_gb300 import synth


def _tiny(nt=8, shape=(10, 11), seed=9):
    dx, dt, nb = 10.0, 1e-3, 3
    v = synth.dipping_layers(shape, dx, seed, nlayers=3, vmin=1500, vmax=2300, nanom=1,
                             sigma=20.0)
    orc = oracle.Oracle(v, dx, dt, nt, nb)
    sh = orc.shot((52.0, 0.0, 30.0), [(x, 0.0, 30.0) for x in np.arange(5.0, 105.0, 10.0)])
    return orc, sh


def test_dtft_matrix_on_the_dft_grid_is_nt_times_the_inverse_fft():
    orc, _ = _tiny(nt=12)
    k = np.array([0, 1, 5, 11])
    F = orc.dtft_matrix(k / (orc.nt * orc.dt))
    x = synth.normal(3, (orc.nt,)) + 1j * synth.normal(4, (orc.nt,))
    assert np.allclose(F @ x, orc.nt * np.fft.ifft(x)[k], rtol=0, atol=1e-12)
    # rows on the grid are orthogonal: F F^H / nt = I
    assert np.allclose(F @ F.conj().T / orc.nt, np.eye(len(k)), atol=1e-12)


def test_full_frequency_grid_reduces_to_the_time_domain_cg():
    """With N_f = N_t grid frequencies the frequency-domain CG is the time-domain CG on
    Eq. "normalewi" seen through F: the same residual history, qbar = F x, q = x."""
    orc, sh = _tiny(nt=8)
    beta = 2e-3
    d = synth.normal(11, (orc.nt, sh.nr))
    freqs = np.arange(orc.nt) / (orc.nt * orc.dt)
    fd = orc.fd_cg(sh, d, beta, freqs, tol=0.0, n_cg=6)
    td = orc.cg(sh, d, beta, tol=0.0, n_cg=6)
    assert np.allclose(fd["rel_res"], td["rel_res"], rtol=1e-9, atol=0)
    assert oracle.rel_l2(fd["q"].real, td["x"]) < 1e-10
    assert np.abs(fd["q"].imag).max() < 1e-10 * np.abs(td["x"]).max()
    F = orc.dtft_matrix(freqs)
    assert oracle.rel_l2(fd["qbar"], F @ td["x"]) < 1e-10


def test_operator_is_hermitian_positive_definite_and_cg_reaches_the_direct_solution():
    orc, sh = _tiny(nt=8, shape=(5, 11))
    beta, freqs = 3e-3, [37.0, 120.5]
    nf, N = len(freqs), orc.N
    n = nf * N
    M = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        M[:, j] = orc.fd_matvec(sh, e, beta, freqs).ravel()
    assert np.abs(M - M.conj().T).max() < 1e-10 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.conj().T)).min() > 0
    # complex linearity (the real and the imaginary part of F^H qbar are modelled apart)
    z = (synth.normal(5, (n,)) + 1j * synth.normal(6, (n,))) * 1e-3
    assert oracle.rel_l2(orc.fd_matvec(sh, 1j * z, beta, freqs).ravel(),
                         1j * orc.fd_matvec(sh, z, beta, freqs).ravel()) < 1e-12
    d = synth.normal(12, (orc.nt, sh.nr))
    res = orc.fd_cg(sh, d, beta, freqs, tol=1e-13, n_cg=3 * n)
    direct = np.linalg.solve(M, res["b"].ravel())
    assert oracle.rel_l2(res["qbar"].ravel(), direct) < 1e-9


def _toeplitz_case(col, both_signs=False):
    """The worked example of the section: x(t) = sum_m sin(2 pi f_m t) on t in [0, 1) with
    N_t = 200 samples and f = 1, 3, 5, 7, 9 Hz; b = A x for a symmetric positive definite
    matrix A standing in for the regularised Hessian; CG on F A F^H xbar = F b over the five
    frequencies; the real signal is 2 Re(F^H xbar / N_t) (its negative frequencies being
    the conjugates of the positive ones)."""
    nt = 200
    orc = oracle.Oracle(np.full((4, 4), 1500.0), 10.0, 1.0 / nt, nt, 1)
    f = [1.0, 3.0, 5.0, 7.0, 9.0]
    t = np.arange(nt) / nt
    x = np.sin(2 * np.pi * np.outer(f, t)).sum(axis=0)
    idx = np.abs(np.subtract.outer(np.arange(nt), np.arange(nt)))
    A = col[idx]
    F = orc.dtft_matrix(f + [-v for v in f] if both_signs else f)

    def M(v):
        q = F.conj().T @ v / nt
        return F @ (A @ q.real) + 1j * (F @ (A @ q.imag))
    b = F @ (A @ x)
    xb = np.zeros(F.shape[0], dtype=np.complex128)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    for _ in range(40):
        Ap = M(p)
        a = rr / np.vdot(p, Ap).real
        xb += a * p
        r -= a * Ap
        rn = np.vdot(r, r).real
        if rn < 1e-28 * np.vdot(b, b).real:
            break
        p = r + rn / rr * p
        rr = rn
    scale = 1.0 if both_signs else 2.0
    rec = scale * (F.conj().T @ xb / nt).real
    naive = scale * (F.conj().T @ b / nt).real   # the band-limited data, A not inverted
    return oracle.rel_l2(rec, x), oracle.rel_l2(naive, x)


def test_worked_example_circulant_operator_is_recovered_exactly():
    # a circulant SPD operator is diagonal in the DFT basis: the five frequencies carry x
    nt = 200
    k = np.arange(nt)
    col = np.exp(-np.minimum(k, nt - k) ** 2 / 8.0)
    col[0] += 0.1
    circ = np.array([[col[(i - j) % nt] for j in range(nt)] for i in range(nt)])
    assert np.linalg.eigvalsh(circ).min() > 0
    orc = oracle.Oracle(np.full((4, 4), 1500.0), 10.0, 1.0 / nt, nt, 1)
    f = [1.0, 3.0, 5.0, 7.0, 9.0]
    t = np.arange(nt) / nt
    x = np.sin(2 * np.pi * np.outer(f, t)).sum(axis=0)
    F = orc.dtft_matrix(f)
    b = F @ (circ @ x)
    Mm = F @ circ @ F.conj().T / nt
    xb = np.linalg.solve(Mm, b)
    assert oracle.rel_l2(2 * (F.conj().T @ xb / nt).real, x) < 1e-12


def test_worked_example_toeplitz_operator():
    """The Kac-Murdock-Szego matrix rho^|i-j| (rho = 0.5, SPD): not shift invariant, so the
    sines' negative-frequency halves leak a little into the five unknowns; the recovered
    signal is within a few per cent, against an O(1) error of the data left uninverted."""
    err, naive = _toeplitz_case(0.5 ** np.arange(200))
    assert err < 5e-2
    assert naive > 1.0
    assert err < naive / 30


def test_worked_example_with_both_signs_is_exact_for_any_spd_operator():
    """CG on F A F^H xbar = F A x returns the A-orthogonal projection of x onto the range of
    F^H; with the frequencies +-f_m the sum of sines lies in that range, so the recovery is
    exact whatever the (here Toeplitz, not shift-invariant) operator."""
    err, _ = _toeplitz_case(0.5 ** np.arange(200), both_signs=True)
    assert err < 1e-12


def test_preconditioned_full_grid_reduces_to_the_time_domain_pcg():
    """The diagonal preconditioner 1 / (beta B^2) acts per cell, so on the full DFT grid the
    preconditioned frequency-domain CG is the preconditioned time-domain CG seen through F."""
    orc, sh = _tiny(nt=8)
    beta = 2e-3
    d = synth.normal(13, (orc.nt, sh.nr))
    B = orc.annihilator(sh.src_xyz)
    minv = 1.0 / (beta * B * B)
    freqs = np.arange(orc.nt) / (orc.nt * orc.dt)
    fd = orc.fd_pcg(sh, d, beta, freqs, 0.0, 6, minv)
    td = orc.pcg(sh, d, beta, 0.0, 6, minv=minv)
    assert np.allclose(fd["rel_res"], td["rel_res"], rtol=1e-9, atol=0)
    assert oracle.rel_l2(fd["q"].real, td["x"]) < 1e-10
    # and it converges to the unpreconditioned solution off the grid as well
    fr = [37.0, 120.5]
    a = orc.fd_pcg(sh, d, beta, fr, 1e-12, 400, minv)
    c = orc.fd_cg(sh, d, beta, fr, 1e-12, 400)
    assert oracle.rel_l2(a["qbar"], c["qbar"]) < 1e-8
