"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: they use closed forms (polynomial
exactness, Fourier symbol, Green's functions, geometric series), invariants
(exact transposes, reciprocity, symmetry/definiteness), brute force at tiny sizes
(dense assembly, Cholesky, least squares) and independent derivatives (Taylor tests).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2211_06300_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_fd8():
    w = {}
    for line in open(os.path.join(GOLDEN, "fd8_coefficients.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, num, den = line.split()
        w[int(k)] = int(num) / int(den)
    return w


# ----------------------------------------------------------------------------- Laplacian
def test_laplacian_stencil_row_matches_fornberg_table():
    w = _golden_fd8()
    n, dx = 21, 2.0
    u = np.zeros((n, n))
    u[10, 10] = 1.0
    out = oracle.laplacian(u, dx) * dx * dx
    # the operator is symmetric: column of the unit impulse = row of the stencil
    assert out[10, 10] == pytest.approx(2 * w[0], abs=1e-14)
    for k in range(1, 5):
        for (a, b) in [(10 + k, 10), (10 - k, 10), (10, 10 + k), (10, 10 - k)]:
            assert out[a, b] == pytest.approx(w[k], abs=1e-14)
    assert np.count_nonzero(np.abs(out) > 1e-15) == 17


@pytest.mark.parametrize("ndim", [2, 3])
def test_laplacian_exact_on_degree_9_polynomials(ndim):
    rng = np.random.default_rng(11)
    n = 24 if ndim == 3 else 40
    dx = 0.05
    coords = [np.arange(n) * dx - 0.5 * n * dx for _ in range(ndim)]
    grids = np.meshgrid(*coords, indexing="ij")
    u = np.zeros([n] * ndim)
    lap = np.zeros_like(u)
    for g in grids:
        a = rng.standard_normal(10)
        u += np.polynomial.polynomial.polyval(g, a)
        d2 = np.polynomial.polynomial.polyder(a, 2)
        lap += np.polynomial.polynomial.polyval(g, d2)
    got = oracle.laplacian(u, dx)
    sl = tuple(slice(4, n - 4) for _ in range(ndim))
    err = np.max(np.abs(got[sl] - lap[sl])) / np.max(np.abs(lap[sl]))
    assert err < 1e-9
    # degree 10 is no longer exact: the truncation error of the order-2p central second
    # difference is -2 (p!)^2 / (2p+2)! h^(2p) u^(2p+2)  (= -h^2 u''''/12 for p = 1)
    u10 = grids[0] ** 10
    got10 = oracle.laplacian(u10, dx)
    exact10 = 90 * grids[0] ** 8
    resid = (got10 - exact10)[sl]
    expected = -2.0 * math.factorial(4) ** 2 / math.factorial(10) * dx ** 8 * math.factorial(10)
    assert np.allclose(resid, expected, rtol=1e-3, atol=0)


def test_laplacian_symmetric_with_zero_extension():
    rng = np.random.default_rng(3)
    u = rng.standard_normal((13, 17))
    v = rng.standard_normal((13, 17))
    a = np.sum(oracle.laplacian(u, 3.0) * v)
    b = np.sum(u * oracle.laplacian(v, 3.0))
    assert abs(a - b) <= 1e-12 * abs(a)


def test_laplacian_nyquist_symbol():
    # (-1)^(i+j) is an eigenvector in the interior; symbol per axis = sum_k w_k 2 cos(k pi)
    w = _golden_fd8()
    per_axis = w[0] + 2 * sum(w[k] * (-1) ** k for k in range(1, 5))
    assert per_axis == pytest.approx(-6.501587301587301, rel=1e-14)
    n, dx = 30, 1.5
    i = np.arange(n)
    u = (-1.0) ** (i[:, None] + i[None, :])
    got = oracle.laplacian(u, dx)[4:-4, 4:-4]
    assert np.allclose(got, 2 * per_axis / dx ** 2 * u[4:-4, 4:-4], rtol=1e-13)


# ----------------------------------------------------------------------------- forward
def _green2d_ricker(r, v, t, f_peak):
    """u(r,t) = (1/2pi) int_{r/v}^t f(t - tau) / sqrt(tau^2 - r^2/v^2) dtau for
    (1/v^2) u_tt - Lap u = delta(x) f(t), via tau = r/v + s^2 (no singularity)."""
    from scipy.integrate import quad
    delay = 1.5 / f_peak

    def f(tt):
        a = (math.pi * f_peak * (tt - delay)) ** 2
        return (1 - 2 * a) * math.exp(-a)
    t0 = r / v
    if t <= t0:
        return 0.0
    smax = math.sqrt(t - t0)
    val, _ = quad(lambda s: 2.0 * f(t - t0 - s * s) / math.sqrt(s * s + 2 * t0), 0.0, smax,
                  limit=400, epsabs=1e-13, epsrel=1e-11)
    return val / (2 * math.pi)


def _homog_trace_2d(dx, dt, nt, offset, v=2000.0, f_peak=15.0):
    L = 1600.0
    n = int(round(L / dx)) + 1
    nb = int(round(200.0 / dx))
    vel = np.full((n, n), v)
    orc = oracle.Oracle(vel, dx, dt, nt, nb)
    c = (n // 2) * dx
    sh = orc.shot((c, 0.0, c), [(c + offset, 0.0, c)])
    tr = orc.forward(sh, wavelet=synth.ricker(nt, dt, f_peak))["traces"][:, 0]
    return tr


@pytest.mark.slow
def test_forward_matches_2d_green_function_and_converges_second_order():
    v, f_peak, offset, T = 2000.0, 15.0, 200.0, 0.45
    errs = []
    for dx, dt in [(10.0, 1e-3), (5.0, 0.5e-3)]:
        nt = int(round(T / dt))
        tr = _homog_trace_2d(dx, dt, nt, offset, v, f_peak)
        t = (np.arange(nt) + 1) * dt          # trace sample n holds u at t_{n+1}
        ref = np.array([_green2d_ricker(offset, v, tt, f_peak) for tt in t])
        errs.append(np.linalg.norm(tr - ref) / np.linalg.norm(ref))
    assert errs[0] < 0.03
    assert 3.0 < errs[0] / errs[1] < 5.0


@pytest.mark.slow
def test_forward_matches_3d_green_function():
    v, f_peak, dx, dt = 2000.0, 15.0, 10.0, 1e-3
    n, nb, nt = 71, 10, 260
    vel = np.full((n, n, n), v)
    orc = oracle.Oracle(vel, dx, dt, nt, nb)
    c = (n // 2) * dx
    offset = 150.0
    sh = orc.shot((c, c, c), [(c + offset, c, c)])
    wav = synth.ricker(nt, dt, f_peak)
    tr = orc.forward(sh, wavelet=wav)["traces"][:, 0]
    t = (np.arange(nt) + 1) * dt
    delay = 1.5 / f_peak
    a = (math.pi * f_peak * (t - offset / v - delay)) ** 2
    ref = (1 - 2 * a) * np.exp(-a) / (4 * math.pi * offset)
    win = t < 0.2      # before waves reflected by the sponge come back
    assert np.linalg.norm(tr[win] - ref[win]) / np.linalg.norm(ref[win]) < 0.03


def test_sponge_absorbs_boundary_reflection():
    # homogeneous grid: with the sponge, the energy that returns from the edge is small
    v, dx, dt, nt, f_peak = 2000.0, 10.0, 1e-3, 700, 15.0
    n = 121
    vel = np.full((n, n), v)
    c = 60 * dx
    wav = synth.ricker(nt, dt, f_peak)

    def trace(nb):
        orc = oracle.Oracle(vel, dx, dt, nt, nb, vref=v)
        sh = orc.shot((c, 0, c), [(c, 0, c)])
        return orc.forward(sh, wavelet=wav)["traces"][:, 0]
    tr_sponge, tr_rigid = trace(20), trace(0)
    late = slice(int(0.45 / dt), nt)        # after the edge reflection arrives (0.6 km two-way at 2 km/s)
    early = slice(0, int(0.15 / dt))
    ratio_sponge = np.max(np.abs(tr_sponge[late])) / np.max(np.abs(tr_sponge[early]))
    ratio_rigid = np.max(np.abs(tr_rigid[late])) / np.max(np.abs(tr_rigid[early]))
    assert ratio_rigid > 0.05
    assert ratio_sponge < 0.1 * ratio_rigid


def _hetero(shape, dx, seed=5):
    v = synth.dipping_layers(shape, dx, seed, nlayers=4, vmin=1500, vmax=2500, nanom=2,
                             sigma=3 * dx)
    return v


def test_reciprocity_is_exact_on_nodes():
    shape, dx, dt, nt, nb = (40, 50), 10.0, 1e-3, 150, 8
    orc = oracle.Oracle(_hetero(shape, dx), dx, dt, nt, nb)
    a = (120.0, 0.0, 100.0)
    b = (330.0, 0.0, 260.0)
    wav = synth.ricker(nt, dt, 20.0)
    ab = orc.forward(orc.shot(a, [b]), wavelet=wav)["traces"][:, 0]
    ba = orc.forward(orc.shot(b, [a]), wavelet=wav)["traces"][:, 0]
    assert np.max(np.abs(ab - ba)) <= 1e-12 * np.max(np.abs(ab))
    assert np.max(np.abs(ab)) > 0


# ----------------------------------------------------------------------------- adjoint
@pytest.mark.parametrize("shape", [(30, 37), (14, 12, 15)])
def test_adjoint_dot_product(shape):
    dx, dt, nt, nb = 10.0, 1e-3, 60, 4
    orc = oracle.Oracle(_hetero(shape, dx), dx, dt, nt, nb)
    src = (0.5 * shape[-1] * dx, 0.5 * shape[1] * dx if len(shape) == 3 else 0.0, 35.0)
    recs = [(x, src[1], 23.0) for x in np.linspace(5.0, (shape[-1] - 2) * dx, 9)]
    sh = orc.shot(src, recs)
    q = synth.normal(7, (nt, orc.N))
    e = synth.normal(8, (nt, sh.nr))
    Sq = orc.forward(sh, q_ext=q)["traces"]
    ad = orc.adjoint(sh, e, want_src=True)
    lhs = np.sum(Sq * e)
    rhs = np.sum(q * ad["out"])
    assert abs(lhs - rhs) / (np.linalg.norm(Sq) * np.linalg.norm(e)) <= 1e-12
    # point-source injection adjoint
    f = synth.normal(9, (nt,))
    Sf = orc.forward(sh, wavelet=f)["traces"]
    lhs = np.sum(Sf * e)
    rhs = np.sum(f * ad["src"])
    assert abs(lhs - rhs) / (np.linalg.norm(Sf) * np.linalg.norm(e)) <= 1e-12


def test_adjoint_equals_dense_transpose():
    shape, dx, dt, nt, nb = (7, 8), 10.0, 1e-3, 6, 2
    orc = oracle.Oracle(_hetero(shape, dx), dx, dt, nt, nb)
    sh = orc.shot((35.0, 0.0, 25.0), [(15.0, 0, 12.0), (52.5, 0, 12.0), (60.0, 0, 50.0)])
    n, m = nt * orc.N, nt * sh.nr
    S = np.zeros((m, n))
    for j in range(n):
        q = np.zeros(n)
        q[j] = 1.0
        S[:, j] = orc.S(sh, q).ravel()
    ST = np.zeros((n, m))
    for i in range(m):
        e = np.zeros(m)
        e[i] = 1.0
        ST[:, i] = orc.ST(sh, e).ravel()
    assert np.max(np.abs(ST - S.T)) <= 1e-14 * np.max(np.abs(S))
    # causality: data sample n depends on q_0..q_n only
    Sb = S.reshape(nt, sh.nr, nt, orc.N)
    for a in range(nt):
        assert np.all(Sb[a, :, a + 1:, :] == 0)


# ----------------------------------------------------------------------------- gradient
@pytest.mark.parametrize("param", ["v", "m"])
def test_gradient_taylor(param):
    shape, dx, dt, nt, nb = (36, 44), 10.0, 1e-3, 160, 8
    v0 = _hetero(shape, dx)
    vref = 2600.0
    src = (215.0, 0.0, 40.0)
    recs = [(x, 0.0, 40.0) for x in np.arange(10.0, 420.0, 20.0)]
    wav = synth.ricker(nt, dt, 20.0)
    v_true = v0 + synth.gaussian_blob(shape, dx, 21, amp=80.0, sigma=50.0)
    o_true = oracle.Oracle(v_true, dx, dt, nt, nb, vref=vref)
    dobs = o_true.forward(o_true.shot(src, recs), wavelet=wav)["traces"]
    o = oracle.Oracle(v0, dx, dt, nt, nb, vref=vref)
    sh = o.shot(src, recs)
    J0, g = o.misfit_gradient(sh, dobs, wavelet=wav, param=param)
    dv = synth.gaussian_blob(shape, dx, 1000, amp=10.0, sigma=60.0)

    def J(vv):
        oo = oracle.Oracle(vv, dx, dt, nt, nb, vref=vref)
        r = oo.forward(oo.shot(src, recs), wavelet=wav)["traces"] - dobs
        return 0.5 * np.sum(r * r)
    if param == "v":
        base, pert = v0, dv
        to_v = lambda x: x
    else:
        base = 1.0 / v0 ** 2
        pert = -2.0 * dv / v0 ** 3          # same physical direction expressed in m
        to_v = lambda m: 1.0 / np.sqrt(m)
    dirderiv = float(np.sum(g * pert.ravel()))
    errs = []
    for h in [0.02, 0.01]:
        fd = (J(to_v(base + h * pert)) - J(to_v(base - h * pert))) / (2 * h)
        errs.append(abs(fd - dirderiv) / abs(dirderiv))
    # central differences: error O(h^2), so halving h divides it by ~4; >= 5 digits agree
    assert errs[1] < 5e-6
    assert 3.0 < errs[0] / errs[1] < 5.0


# ----------------------------------------------------------------------------- normal equation / CG
def _tiny_problem():
    shape, dx, dt, nt, nb = (12, 12), 10.0, 1e-3, 8, 3
    orc = oracle.Oracle(_hetero(shape, dx, seed=9), dx, dt, nt, nb)
    sh = orc.shot((55.0, 0.0, 30.0), [(x, 0.0, 30.0) for x in np.arange(10.0, 115.0, 10.0)])
    return orc, sh


def test_normal_matrix_spd_and_cg_matches_cholesky():
    orc, sh = _tiny_problem()
    beta = 1e-3
    A = orc.assemble_normal(sh, beta)
    assert np.max(np.abs(A - A.T)) <= 1e-12 * np.max(np.abs(A))
    L = np.linalg.cholesky(0.5 * (A + A.T))
    B = orc.annihilator(sh.src_xyz)
    lam_min = np.linalg.eigvalsh(0.5 * (A + A.T))[0]
    assert lam_min >= beta * np.min(B * B) * (1 - 1e-9)
    d = synth.normal(12, (orc.nt, sh.nr))
    b = orc.ST(sh, d).ravel()
    x_direct = np.linalg.solve(L.T, np.linalg.solve(L, b))
    res = orc.cg(sh, d, beta, tol=1e-13, n_cg=3000)
    assert oracle.rel_l2(res["x"].ravel(), x_direct) < 1e-10
    assert np.allclose(res["b"].ravel(), b)


def test_cg_alg1_residual_history_is_true_residual_and_orthogonal():
    orc, sh = _tiny_problem()
    beta = 1e-3
    A = orc.assemble_normal(sh, beta)
    d = synth.normal(13, (orc.nt, sh.nr))
    b = orc.ST(sh, d).ravel()
    xs, rs = [], []
    for k in range(1, 6):
        res = orc.cg(sh, d, beta, tol=0.0, n_cg=k)
        assert res["iters"] == k
        x = res["x"].ravel()
        r_true = b - A @ x
        assert np.linalg.norm(r_true) / np.linalg.norm(b) == pytest.approx(res["rel_res"][-1],
                                                                           rel=1e-8)
        xs.append(x)
        rs.append(r_true)
    rs = [b] + rs
    for i in range(len(rs)):
        for j in range(i):
            assert abs(rs[i] @ rs[j]) <= 1e-8 * np.linalg.norm(rs[i]) * np.linalg.norm(rs[j])
    # the tolerance exit: stops at the first k with ||r_{k+1}|| < tol ||r_0||
    full = orc.cg(sh, d, beta, tol=0.0, n_cg=8)["rel_res"]
    tol = 0.5 * (full[3] + full[2])
    assert full[3] < tol <= full[2]
    early = orc.cg(sh, d, beta, tol=tol, n_cg=8)
    assert early["iters"] == 4


def test_cg_large_beta_limit():
    # beta -> infinity: q -> (beta B^2)^-1 S^T d
    orc, sh = _tiny_problem()
    d = synth.normal(14, (orc.nt, sh.nr))
    beta = 1e8
    B = orc.annihilator(sh.src_xyz)
    x = orc.cg(sh, d, beta, tol=1e-14, n_cg=50)["x"]
    lim = orc.ST(sh, d) / (beta * B * B)[None, :]
    assert oracle.rel_l2(x, lim) < 1e-6


def test_beta_zero_source_wavelet_estimation():
    """beta = 0 with q restricted to the source node: CG on S_f^T S_f f = S_f^T d recovers
    the wavelet that generated d (the special case after Algorithm 1)."""
    shape, dx, dt, nt, nb = (30, 40), 10.0, 1e-3, 60, 6
    orc = oracle.Oracle(_hetero(shape, dx), dx, dt, nt, nb)
    src = (200.0, 0.0, 100.0)
    sh = orc.shot(src, [(x, 0, 100.0) for x in np.arange(100.0, 310.0, 10.0)])
    f_true = synth.ricker(nt, dt, 25.0)
    d = orc.forward(sh, wavelet=f_true)["traces"]

    def S(f):
        return orc.forward(sh, wavelet=f)["traces"]

    def ST(e):
        return orc.adjoint(sh, e, want_out=False, want_src=True)["src"]
    # Algorithm 1 on the nt x nt system
    b = ST(d)
    x = np.zeros(nt)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    r0 = math.sqrt(rr)
    for k in range(4 * nt):
        Ap = ST(S(p))
        alpha = rr / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = r @ r
        if math.sqrt(rr_new) < 1e-13 * r0:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    assert oracle.rel_l2(x, f_true) < 1e-7


def test_saddle_point_gradient_equals_adjoint_state_at_solution():
    shape, dx, dt, nt, nb = (16, 18), 10.0, 1e-3, 24, 4
    orc = oracle.Oracle(_hetero(shape, dx, seed=4), dx, dt, nt, nb)
    src = (85.0, 0.0, 40.0)
    sh = orc.shot(src, [(x, 0, 40.0) for x in np.arange(10.0, 170.0, 10.0)])
    d = orc.forward(sh, wavelet=synth.ricker(nt, dt, 40.0))["traces"]
    beta = 1e-4
    res = orc.cg(sh, d, beta, tol=1e-12, n_cg=4000)
    q = res["x"]
    g_sp = orc.saddle_gradient(sh, q, beta)
    _, g_as = orc.misfit_gradient(sh, d, q_ext=q)
    assert oracle.rel_l2(g_sp, g_as) < 1e-7


# ----------------------------------------------------------------------------- DTFT
def test_dtft_single_sinusoid_closed_form():
    nt, dt, f0 = 300, 2e-3, 7.0
    freqs = [3.0, 7.0, 11.5]
    re = np.zeros((3, 1))
    im = np.zeros((3, 1))
    for n in range(nt):
        t = (n + 1) * dt
        oracle.dtft_accumulate(np.array([math.sin(2 * math.pi * f0 * t)]), t, freqs, re, im)
    w0 = 2 * math.pi * f0 * dt

    def geo(theta):  # sum_{n=1}^{nt} exp(j theta n)
        z = complex(math.cos(theta), math.sin(theta))
        if abs(1 - z) < 1e-15:
            return complex(nt, 0)
        return z * (1 - z ** nt) / (1 - z)
    for m, f in enumerate(freqs):
        w = 2 * math.pi * f * dt
        ref = (geo(w + w0) - geo(w - w0)) / 2j
        assert abs(complex(re[m, 0], im[m, 0]) - ref) <= 1e-11 * max(1.0, abs(ref))


def test_forward_dtft_uses_state_times():
    shape, dx, dt, nt, nb = (20, 24), 10.0, 1e-3, 80, 4
    orc = oracle.Oracle(_hetero(shape, dx), dx, dt, nt, nb)
    sh = orc.shot((115.0, 0, 60.0), [(50.0, 0, 30.0)])
    freqs = [10.0, 25.0]
    out = orc.forward(sh, wavelet=synth.ricker(nt, dt, 25.0), want_u=True, freqs=freqs)
    u = out["u"]
    t = np.arange(nt + 1) * dt
    for m, f in enumerate(freqs):
        ref = np.sum(u[1:] * np.exp(2j * np.pi * f * t[1:])[:, None], axis=0)
        assert oracle.rel_l2(out["dft"][m], ref) < 1e-12


# ----------------------------------------------------------------------------- codecs
def test_bf16_rounding_is_nearest_ties_even():
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-20, 20, 20000)).astype(np.float32)
    codes = oracle._bf16_rne(x)
    y = oracle.bf16_to_f32(codes).astype(np.float64)
    up = oracle.bf16_to_f32((codes + 1).astype(np.uint16)).astype(np.float64)
    dn = oracle.bf16_to_f32((codes - 1).astype(np.uint16)).astype(np.float64)
    xd = x.astype(np.float64)
    e = np.abs(y - xd)
    assert np.all(e <= np.abs(up - xd) + 0.0)
    assert np.all(e <= np.abs(dn - xd) + 0.0)
    # exact ties go to the even code
    ties = (np.arange(1, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32)
    tc = oracle._bf16_rne(ties)
    assert np.all(tc % 2 == 0)


@pytest.mark.parametrize("kind,bound", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_snapshot_codec_roundtrip_bound(kind, bound):
    rng = np.random.default_rng(6)
    u = (rng.standard_normal(50000) * np.exp(rng.uniform(-8, 0, 50000))).astype(np.float32)
    codes, dec = oracle.encode_snapshot(u, kind)
    back = oracle.decode_snapshot(codes, dec, kind).astype(np.float64)
    s = float(np.max(np.abs(u)))
    normal = np.abs(u) * oracle.CODEC_RANGE / s >= 2.0 ** -14
    rel = np.abs(back - u)[normal] / np.abs(u.astype(np.float64))[normal]
    # one rounding to the 16-bit format plus two FP32 roundings of the scale products
    assert np.max(rel) <= bound * (1 + 1e-3) + 3 * 2.0 ** -24
    assert np.max(np.abs(back)) <= s * (1 + bound)


def test_pcg_reaches_the_cholesky_solution_and_reduces_to_cg():
    orc, sh = _tiny_problem()
    beta = 1e-3
    A = orc.assemble_normal(sh, beta)
    d = synth.normal(15, (orc.nt, sh.nr))
    b = orc.ST(sh, d).ravel()
    x_direct = np.linalg.solve(A, b)
    B = orc.annihilator(sh.src_xyz)
    res = orc.pcg(sh, d, beta, tol=1e-13, n_cg=3000, minv=1.0 / (beta * B * B))
    assert oracle.rel_l2(res["x"].ravel(), x_direct) < 1e-9
    # the identity preconditioner gives Algorithm 1's iterates
    a = orc.pcg(sh, d, beta, tol=0.0, n_cg=6, minv=np.ones(orc.N))
    c = orc.cg(sh, d, beta, tol=0.0, n_cg=6)
    assert np.allclose(a["rel_res"], c["rel_res"], rtol=1e-12)
    assert oracle.rel_l2(a["x"], c["x"]) < 1e-12
