"""Pins of the oracle's checkpoint code and of the gradient recomputed from checkpoints,
each with a planted mistake (on the CPU, in a copy of the oracle function) that the pin
must catch.

* ``upsample_even``: multilinear prolongation from the all-even cells.  Pinned by a
  cell-by-cell construction with explicit trilinear weights at random coarse values, by
  exact reproduction of multilinear polynomials, and by hand-computed small cases, including
  an even axis length (the last odd index repeats its left neighbour).
* ``checkpoint_code``: the two-level 16-bit code.  Pinned by exact round trips of fields that
  are multilinear between BF16-representable even cells (the single-level code is not exact
  there), and by the per-element bound: the error is the 16-bit rounding of the residual
  against the interpolation of the decoded coarse part, not of the value.
* ``Oracle.checkpointed_gradient``: the storage section's recomputation from checkpoints.
  Pinned by three identities with the stored-history gradient ``misfit_gradient``: with
  uncompressed checkpoints, with one checkpoint only (the zero initial state), and with a
  lossless code in place of the 16-bit one (the u_n, u_n - u_{n-1} bookkeeping).
"""
import numpy as np
import pytest

import oracle
from paper_2211_06300_gb300 import synth


# ----------------------------------------------------------------------------- prolongation
def _bf16_values(rng, shape):
    """Random BF16-representable values in [-2, -1] U [1, 2], built from their bit patterns."""
    mant = rng.integers(0, 128, size=shape).astype(np.uint32)
    sign = rng.integers(0, 2, size=shape).astype(np.uint32)
    bits = (sign << 31) | (np.uint32(127) << 23) | (mant << 16)
    return bits.view(np.float32).astype(np.float64)


def _trilinear_brute(c, shape):
    """Every cell from the coarse values by explicit weights: along each axis a cell at
    index i lies between even cells 2k and 2k+2 (k = i // 2) at fraction (i % 2) / 2, the
    right one clamped to the last even cell."""
    out = np.zeros(shape)
    for idx in np.ndindex(*shape):
        axes = []
        for i, n in zip(idx, shape):
            k, t = i // 2, (i % 2) / 2.0
            k1 = min(k + 1, (n + 1) // 2 - 1)
            axes.append([(k, 1.0 - t), (k1, t)])
        val = 0.0
        for corner in np.ndindex(*([2] * len(shape))):
            w = 1.0
            cidx = []
            for a, b in enumerate(corner):
                kk, ww = axes[a][b]
                w *= ww
                cidx.append(kk)
            val += w * c[tuple(cidx)]
        out[idx] = val
    return out


def _up_nearest(c, shape):
    """Planted mistake: an odd index copies its left even neighbour."""
    u = np.asarray(c, dtype=np.float64)
    for ax, n in enumerate(shape):
        u = np.repeat(u, 2, axis=ax).take(np.arange(n), axis=ax)
    return u


def _up_axes_reversed(c, shape):
    """Planted mistake: the axes walked in reverse order with the lengths of the forward
    order (a transposed loop)."""
    u = np.asarray(c, dtype=np.float64)
    nd = len(shape)
    for ax in range(nd):
        n = shape[nd - 1 - ax]
        try:
            u = np.moveaxis(u, ax, 0)
            out = np.empty((n,) + u.shape[1:])
            out[0::2] = u[: (n + 1) // 2]
            right = np.concatenate([u[1:], u[-1:]])
            out[1::2] = (0.5 * (u + right))[: n // 2]
            u = np.moveaxis(out, 0, ax)
        except ValueError:
            return np.full(shape, np.nan)
    return u if u.shape == tuple(shape) else np.full(shape, np.nan)


def _up_last_zero(c, shape):
    """Planted mistake: an odd last index averages with zero instead of repeating."""
    u = np.asarray(c, dtype=np.float64)
    for ax, n in enumerate(shape):
        u = np.moveaxis(u, ax, 0)
        out = np.empty((n,) + u.shape[1:])
        out[0::2] = u
        right = np.concatenate([u[1:], np.zeros_like(u[-1:])])
        out[1::2] = (0.5 * (u + right))[: n // 2]
        u = np.moveaxis(out, 0, ax)
    return u


def _prolongation_errors(up):
    """Largest deviation of a prolongation from the pins: brute-force weights on odd and
    even lengths, multilinear polynomials, the hand-computed cases."""
    rng = np.random.default_rng(3)
    errs = []
    for shape in [(7, 5, 9), (6, 5, 4), (9, 11), (8, 3)]:
        c = _bf16_values(rng, tuple((n + 1) // 2 for n in shape))
        errs.append(np.max(np.abs(up(c, shape) - _trilinear_brute(c, shape))))
    # multilinear polynomial: linear in each index, cross terms included (odd lengths)
    for shape in [(7, 5, 9), (9, 11)]:
        idx = [i.astype(np.float64) for i in np.indices(shape)]
        coef = rng.standard_normal(2 ** len(shape))
        f = np.zeros(shape)
        for m in range(2 ** len(shape)):
            term = np.ones(shape)
            for a in range(len(shape)):
                if m >> a & 1:
                    term = term * idx[a]
            f += coef[m] * term
        even = f[tuple(slice(0, None, 2) for _ in shape)]
        errs.append(np.max(np.abs(up(even, shape) - f)) / np.max(np.abs(f)))
    # hand-computed
    errs.append(np.max(np.abs(up(np.array([[[1.0, 5.0, 2.0]]]), (1, 1, 5))
                              - np.array([[[1.0, 3.0, 5.0, 3.5, 2.0]]]))))
    errs.append(np.max(np.abs(up(np.array([[1.0, 5.0]]), (1, 4))
                              - np.array([[1.0, 3.0, 5.0, 5.0]]))))
    errs.append(np.max(np.abs(up(np.array([[1.0, 2.0], [3.0, 4.0]]), (3, 3))
                              - np.array([[1.0, 1.5, 2.0], [2.0, 2.5, 3.0], [3.0, 3.5, 4.0]]))))
    return max(float(e) if np.isfinite(e) else np.inf for e in errs)


def test_prolongation_pins():
    assert _prolongation_errors(oracle.upsample_even) <= 1e-13


@pytest.mark.parametrize("mutant", [_up_nearest, _up_axes_reversed, _up_last_zero])
def test_prolongation_planted_mistakes_fail(mutant):
    assert _prolongation_errors(mutant) > 1e-3


# ----------------------------------------------------------------------------- the code
def _multilinear_between_bf16(shape, seed):
    """A field that is multilinear between BF16-representable values at the even cells
    (odd lengths), built cell by cell; its odd cells need more than BF16's 8 bits."""
    rng = np.random.default_rng(seed)
    c = _bf16_values(rng, tuple((n + 1) // 2 for n in shape))
    c.flat[0] = 2.0   # max |x| = 2: FP16's scale 32768 / max |x| is then a power of two
    return _trilinear_brute(c, shape)


@pytest.mark.parametrize("kind", ["bf16", "f16"])
@pytest.mark.parametrize("shape", [(9, 7, 11), (13, 15)])
def test_code_is_exact_on_fields_multilinear_between_representable_even_cells(kind, shape):
    x = _multilinear_between_bf16(shape, 11)
    if kind == "f16":
        x = x * 2.0 ** 10   # a power of two: the scaled values stay in FP16's normal range
    back = oracle.checkpoint_code(x, shape, kind)
    assert np.array_equal(back, x.ravel())
    if kind == "bf16":
        # a single BF16 rounding of the values is not exact on the same field (FP16's 11
        # bits hold the means of up to eight 8-bit values, so there both codes are exact)
        codes, dec = oracle.encode_snapshot(x.ravel(), kind)
        single = oracle.decode_snapshot(codes, dec, kind).astype(np.float64)
        assert np.max(np.abs(single - x.ravel())) > 0


def _residual_of_decoded_coarse(x, shape, kind):
    """x - U(decoded coarse part), the decoded coarse part rounded to FP32 then 16 bits by
    the same rule as the code's coarse level."""
    even = x[tuple(slice(0, None, 2) for _ in shape)]
    if kind == "bf16":
        dc = oracle.bf16_to_f32(oracle._bf16_rne(even.astype(np.float32))).astype(np.float64)
    else:
        codes, dec = oracle.encode_snapshot(even.ravel(), "f16")
        dc = oracle.decode_snapshot(codes, dec, "f16").astype(np.float64).reshape(even.shape)
    return x - _trilinear_brute(dc, shape)


def _code_bound_violation(code, kind, shape=(9, 8, 13), seed=5):
    """Largest ratio of |decoded - x| to its bound over one smooth-plus-noise field:
    BF16 rounds the FP32 residual r to 8 significant bits (unit roundoff 2^-8); FP16 rounds
    r scaled by 32768 / max|r| to 11 (2^-11, normal range only); both add the FP32 roundings
    of the residual and of the scale products (a few 2^-24 |r|)."""
    rng = np.random.default_rng(seed)
    idx = np.indices(shape).astype(np.float64)
    x = np.sin(0.5 * idx[0] + 0.3) * np.cos(0.4 * idx[-1]) + 0.05 * rng.standard_normal(shape)
    r = _residual_of_decoded_coarse(x, shape, kind).ravel()
    err = np.abs(code(x, shape, kind) - x.ravel())
    if kind == "bf16":
        bound = (2.0 ** -8 + 4 * 2.0 ** -24) * np.abs(r)
        keep = np.abs(r) > 1e-30
    else:
        scale = np.max(np.abs(r.astype(np.float32))) / 32768.0
        keep = np.abs(r) / scale >= 2.0 ** -14
        bound = (2.0 ** -11 + 4 * 2.0 ** -24) * np.abs(r)
    return float(np.max(err[keep] / bound[keep]))


def _code_residual_vs_exact_coarse(x, shape, kind):
    """Planted mistake: the fine part is taken against the exact coarse values while the
    decoder interpolates the decoded ones."""
    x = np.asarray(x, dtype=np.float64).reshape(shape)
    even = x[tuple(slice(0, None, 2) for _ in shape)]
    up_exact = oracle.upsample_even(even, shape)
    up_dec = oracle.upsample_even(oracle._code16(even, kind), shape)
    return (up_dec + oracle._code16(x - up_exact, kind)).ravel()


def _code_single_level(x, shape, kind):
    """Planted mistake: one 16-bit rounding of the values (no coarse level)."""
    codes, dec = oracle.encode_snapshot(np.asarray(x).ravel(), kind)
    return oracle.decode_snapshot(codes, dec, kind).astype(np.float64)


@pytest.mark.parametrize("kind", ["bf16", "f16"])
def test_code_error_is_the_rounding_of_the_interpolation_residual(kind):
    assert _code_bound_violation(oracle.checkpoint_code, kind) <= 1.0


@pytest.mark.parametrize("kind", ["bf16", "f16"])
@pytest.mark.parametrize("mutant", [_code_residual_vs_exact_coarse, _code_single_level])
def test_code_planted_mistakes_fail(kind, mutant):
    assert _code_bound_violation(mutant, kind) > 1.0


def test_code_keeps_zero_and_the_uncompressed_kind():
    shape = (5, 6)
    assert np.array_equal(oracle.checkpoint_code(np.zeros(shape), shape, "bf16"), np.zeros(30))
    assert np.array_equal(oracle.checkpoint_code(np.zeros(shape), shape, "f16"), np.zeros(30))
    x = synth.normal(1, shape)
    assert np.array_equal(oracle.checkpoint_code(x, shape, "f32"), x.ravel())


# ----------------------------------------------------------------------------- the gradient
def _grad_problem():
    shape, dx, dt, nt, nb = (24, 31), 10.0, 1e-3, 70, 5
    v = synth.dipping_layers(shape, dx, 2, nlayers=3, vmin=1500, vmax=2400, nanom=1,
                             sigma=30.0)
    vt = v + synth.gaussian_blob(shape, dx, 4, amp=70.0, sigma=40.0)
    o = oracle.Oracle(v, dx, dt, nt, nb, vref=2600.0)
    ot = oracle.Oracle(vt, dx, dt, nt, nb, vref=2600.0)
    rec = np.stack([np.arange(0.0, 300.0, 15.0), np.zeros(20), np.full(20, 30.0)], axis=1)
    src = np.array([152.5, 0.0, 31.0])
    sh, sht = o.shot(src, rec), ot.shot(src, rec)
    wav = synth.ricker(nt, dt, 25.0)
    d = ot.forward(sht, wavelet=synth.ricker(nt, dt, 21.0, delay=0.06))["traces"]
    return o, sh, d, wav


def _ckpt_grad_state_after(self, sh, dobs, wavelet, every, kind, param="c"):
    """Planted mistake: a segment restarts from (u_n0+1, u_n0), one step late."""
    nt, N = self.nt, self.N
    fw = self.forward(sh, wavelet=wavelet, want_u=True)
    e = fw["traces"] - np.asarray(dobs).reshape(nt, sh.nr)
    U = fw["u"]
    s_hist = np.empty((nt, N))
    for n0 in range(0, nt, every):
        cur = oracle.checkpoint_code(U[min(n0 + 1, nt)], self.shape, kind)
        prev = oracle.checkpoint_code(U[n0], self.shape, kind)
        for n in range(n0, min(nt, n0 + every)):
            q = np.zeros(N)
            np.add.at(q, sh.src_node, sh.src_w * wavelet[n])
            s = oracle.laplacian(cur.reshape(self.shape), self.dx).ravel() + q
            s_hist[n] = s
            nxt = (2.0 * cur - (1.0 - self.kappa) * prev + self.c * s) / (1.0 + self.kappa)
            prev, cur = cur, nxt
    ad = self.adjoint(sh, e, want_out=False, s_hist=s_hist)
    return 0.5 * float(np.sum(e * e)), self.to_param(ad["grad_c"], param)


def _ckpt_grad_difference_sign(self, sh, dobs, wavelet, every, kind, param="c"):
    """Planted mistake: u_n0-1 rebuilt as decoded u_n0 + decoded difference."""
    nt, N = self.nt, self.N
    fw = self.forward(sh, wavelet=wavelet, want_u=True)
    e = fw["traces"] - np.asarray(dobs).reshape(nt, sh.nr)
    U = fw["u"]
    s_hist = np.empty((nt, N))
    for n0 in range(0, nt, every):
        up = U[n0 - 1] if n0 > 0 else np.zeros(N)
        cur = oracle.checkpoint_code(U[n0], self.shape, kind)
        prev = cur + oracle.checkpoint_code(U[n0] - up, self.shape, kind)
        for n in range(n0, min(nt, n0 + every)):
            q = np.zeros(N)
            np.add.at(q, sh.src_node, sh.src_w * wavelet[n])
            s = oracle.laplacian(cur.reshape(self.shape), self.dx).ravel() + q
            s_hist[n] = s
            nxt = (2.0 * cur - (1.0 - self.kappa) * prev + self.c * s) / (1.0 + self.kappa)
            prev, cur = cur, nxt
    ad = self.adjoint(sh, e, want_out=False, s_hist=s_hist)
    return 0.5 * float(np.sum(e * e)), self.to_param(ad["grad_c"], param)


def _lossless(x, shape, kind):
    return np.asarray(x, dtype=np.float64).ravel().copy()


def _identity_errors(fn, monkeypatch):
    """Deviations from misfit_gradient: uncompressed checkpoints every 9 steps, BF16 with a
    single checkpoint (every >= nt), and BF16 bookkeeping with a lossless code."""
    o, sh, d, wav = _grad_problem()
    J, g = o.misfit_gradient(sh, d, wavelet=wav, param="v")
    out = []
    Jk, gk = fn(o, sh, d, wav, 9, "f32", param="v")
    out.append(max(oracle.rel_l2(gk, g), abs(Jk - J) / J))
    out.append(oracle.rel_l2(fn(o, sh, d, wav, o.nt, "bf16", param="v")[1], g))
    with monkeypatch.context() as m:
        m.setattr(oracle, "checkpoint_code", _lossless)
        out.append(oracle.rel_l2(fn(o, sh, d, wav, 9, "bf16", param="v")[1], g))
    return out


def test_checkpointed_gradient_identities(monkeypatch):
    f32, single, lossless = _identity_errors(oracle.Oracle.checkpointed_gradient, monkeypatch)
    assert f32 <= 1e-14
    assert single <= 1e-14
    assert lossless <= 1e-12


def test_checkpointed_gradient_with_bf16_code_moves_the_gradient_a_little():
    o, sh, d, wav = _grad_problem()
    _, g = o.misfit_gradient(sh, d, wavelet=wav, param="v")
    err = oracle.rel_l2(o.checkpointed_gradient(sh, d, wav, 9, "bf16", param="v")[1], g)
    assert 1e-7 < err < 1e-2


@pytest.mark.parametrize("mutant", [_ckpt_grad_state_after, _ckpt_grad_difference_sign])
def test_checkpointed_gradient_planted_mistakes_fail(mutant, monkeypatch):
    errs = _identity_errors(mutant, monkeypatch)
    assert max(errs) > 1e-3
