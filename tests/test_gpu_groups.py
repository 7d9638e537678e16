"""Concurrent shot groups (esi_set_shot_groups): the context's shots split into child
contexts on streams and host threads of their own.  Shots are independent systems (one
extended source and one normal equation each), so every per-shot output must equal the
ungrouped context's and the oracle's; the gradient, a sum over shots, is the groups' partial
sums added in group order."""
import numpy as np
import pytest

import oracle
from paper_2211_06300_gb300 import synth
from test_gpu_parity import _ctx, _dev, _multishot_3d, _orc, _ragged_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case():
    v, geom, p = _ragged_case(nt=80)
    # every shot with data above FP32 resolution: shot 1's single receiver near its source
    geom.rec_xyz[geom.rec_offset[1]] = (geom.src_xyz[1, 0] + 55.0, 0.0, 30.0)
    return v, geom, p


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("groups", [2, 3])
@pytest.mark.parametrize("precond", ["none", "diag"])
def test_grouped_cg_equals_the_single_context_and_the_oracle(prec, groups, precond):
    v, geom, p = _case()
    nt = p["nt"]
    o, shots = _orc(v, geom, p)
    wav = synth.ricker(nt, p["dt"], 25.0)
    d = np.concatenate([o.forward(sh, wavelet=wav)["traces"].ravel() for sh in shots])
    lam, tol, nmax = 2e-4, 0.05, 8
    ctx1 = _ctx(v, geom, p, prec)
    q1, r1 = ctx1.cg_solve(_dev(d, prec), lam=lam, tol=tol, max_iter=nmax, precond=precond, hist=nmax)
    ctxg = _ctx(v, geom, p, prec)
    ctxg.set_shot_groups(groups)
    qg, rg = ctxg.cg_solve(_dev(d, prec), lam=lam, tol=tol, max_iter=nmax, precond=precond, hist=nmax)
    # per shot, the same launches with the same per-shot reductions: the same numbers
    assert list(rg["iters"]) == list(r1["iters"])
    for s in range(geom.ns):
        assert np.allclose(rg["rel_res"][s], r1["rel_res"][s], rtol=1e-12, atol=0), s
    assert torch.allclose(qg, q1, rtol=1e-12, atol=0)
    tolp = {"f64": 1e-12, "f32": 1e-4}[prec]
    for s, sh in enumerate(shots):
        o0, o1 = geom.rec_offset[s], geom.rec_offset[s + 1]
        ds = d[nt * o0:nt * o1].reshape(nt, -1)
        if precond == "diag":
            B = o.annihilator(sh.src_xyz)
            ref = o.pcg(sh, ds, lam, tol, nmax, minv=1.0 / (lam * B * B))
        else:
            ref = o.cg(sh, ds, lam, tol, nmax)
        assert rg["iters"][s] == ref["iters"], s
        assert np.allclose(rg["rel_res"][s], ref["rel_res"], rtol=tolp, atol=0), s
        assert oracle.rel_l2(qg[s].reshape(nt, -1).double().cpu().numpy(), ref["x"]) <= \
            (tolp if prec == "f64" else 1e-3), s
    assert ctxg.launches > 0


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_grouped_gradients_are_the_sum_of_the_groups(prec):
    """Saddle-point gradient (and its objective) and the adjoint-state gradient with
    checkpoints, three shots in two groups, against the single context."""
    v, geom, p = _case()
    nt = p["nt"]
    o, shots = _orc(v, geom, p)
    q = synth.normal(8, (geom.ns, nt) + v.shape) * 1e-2
    wav = np.stack([synth.ricker(nt, p["dt"], 25.0)] * geom.ns)
    d = np.concatenate([o.forward(sh, wavelet=wav[s])["traces"].ravel() for s, sh in enumerate(shots)])
    ctx1, ctxg = _ctx(v, geom, p, prec), _ctx(v, geom, p, prec)
    ctxg.set_shot_groups(2)
    tol = {"f64": 1e-12, "f32": 1e-5}[prec]
    g1, J1 = ctx1.gradient(ext=_dev(q, prec), dobs=_dev(d, prec), mode="saddle", beta=0.3, param="v")
    gg, Jg = ctxg.gradient(ext=_dev(q, prec), dobs=_dev(d, prec), mode="saddle", beta=0.3, param="v")
    assert oracle.rel_l2(gg.double().cpu().numpy(), g1.double().cpu().numpy()) <= tol
    assert Jg == pytest.approx(J1, rel=tol)
    wav2 = np.stack([synth.ricker(nt, p["dt"], 21.0, delay=0.05)] * geom.ns)
    g1, J1 = ctx1.gradient(wavelet=_dev(wav2, prec), dobs=_dev(d, prec), param="m", ckpt_every=9)
    gg, Jg = ctxg.gradient(wavelet=_dev(wav2, prec), dobs=_dev(d, prec), param="m", ckpt_every=9)
    assert oracle.rel_l2(gg.double().cpu().numpy(), g1.double().cpu().numpy()) <= tol
    assert Jg == pytest.approx(J1, rel=tol)
    if prec == "f64":   # and the oracle's sum over shots
        g_ref = sum(o.misfit_gradient(sh, d[nt * geom.rec_offset[s]:nt * geom.rec_offset[s + 1]],
                                      wavelet=wav2[s], param="m")[1] for s, sh in enumerate(shots))
        assert oracle.rel_l2(gg.cpu().numpy().ravel(), g_ref) <= 1e-12


@pytest.mark.parametrize("half", [True, False])
def test_grouped_dtft_extract_equals_the_single_context(half):
    v, geom, p = _case()
    nt = p["nt"]
    wav = _dev(np.stack([synth.ricker(nt, p["dt"], 25.0)] * geom.ns), "f32")
    ctx1, ctxg = _ctx(v, geom, p, "f32"), _ctx(v, geom, p, "f32")
    ctxg.set_shot_groups(3)
    freqs = [10.0, 17.5, 31.0]
    t1, tg = ctx1.empty_traces(), ctxg.empty_traces()
    U1, s1 = ctx1.dft_extract(freqs, wavelet=wav, half=half, traces=t1)
    Ug, sg = ctxg.dft_extract(freqs, wavelet=wav, half=half, traces=tg)
    assert torch.equal(t1, tg)
    assert torch.equal(U1, Ug)
    if half:
        assert np.array_equal(np.asarray(s1), np.asarray(sg))


def test_grouped_3d_cg_per_shot_stopping_fp64():
    """Three 3D shots in three groups (one each), stopping after 6, 4 and 8 iterations."""
    v, geom, p = _multishot_3d()
    nt = p["nt"]
    o, shots = _orc(v, geom, p)
    wav = synth.ricker(nt, p["dt"], 30.0)
    d = np.concatenate([o.forward(sh, wavelet=wav)["traces"].ravel() for sh in shots])
    lam, tol, nmax = 1e-2, 0.04, 10
    ctx = _ctx(v, geom, p, "f64")
    ctx.set_shot_groups(3)
    q, rep = ctx.cg_solve(_dev(d, "f64"), lam=lam, tol=tol, max_iter=nmax)
    for s, sh in enumerate(shots):
        o0, o1 = geom.rec_offset[s], geom.rec_offset[s + 1]
        ref = o.cg(sh, d[nt * o0:nt * o1].reshape(nt, -1), lam, tol, nmax)
        assert rep["iters"][s] == ref["iters"], s
        assert np.allclose(rep["rel_res"][s], ref["rel_res"], rtol=1e-12, atol=0), s
        assert oracle.rel_l2(q[s].reshape(nt, -1).cpu().numpy(), ref["x"]) <= 1e-12, s


def test_groups_follow_the_velocity_and_report_their_work():
    esi = pytest.importorskip("paper_2211_06300_gb300.esi")
    v, geom, p = _case()
    nt = p["nt"]
    v2 = v * 1.03
    # the sponge keeps the reference velocity of the context's creation (v.max())
    o2, shots2 = _orc(v2, geom, p, vref=float(v.max()))
    wav = synth.ricker(nt, p["dt"], 25.0)
    d = np.concatenate([o2.forward(sh, wavelet=wav)["traces"].ravel() for sh in shots2])
    ctx = _ctx(v, geom, p, "f64")
    ctx.set_shot_groups(2)
    ctx.set_velocity(_dev(v2, "f64"))
    ctx.set_profiling(True)
    q, rep = ctx.cg_solve(_dev(d, "f64"), lam=2e-4, tol=0.0, max_iter=3)
    prof = ctx.profile()
    ctx.set_profiling(False)
    for s, sh in enumerate(shots2):
        o0, o1 = geom.rec_offset[s], geom.rec_offset[s + 1]
        ref = o2.cg(sh, d[nt * o0:nt * o1].reshape(nt, -1), 2e-4, 0.0, 3)
        assert oracle.rel_l2(q[s].reshape(nt, -1).cpu().numpy(), ref["x"]) <= 1e-12, s
    # the groups' launches are counted and profiled: 3 products of two propagations of
    # nt steps for every shot, plus b = S^T d
    steps = sum(k["launches"] for k in prof if k["name"].startswith("fd2_step"))
    assert steps >= (2 * 3 + 1) * nt
    with pytest.raises(esi.EsiError):
        ctx.set_shot_groups(0)
    with pytest.raises(esi.EsiError):
        ctx.set_shot_groups(geom.ns + 1)
    ctx.set_shot_groups(1)   # removes the groups: the context solves alone again
    q1, _ = ctx.cg_solve(_dev(d, "f64"), lam=2e-4, tol=0.0, max_iter=3)
    assert torch.allclose(q1, q, rtol=1e-12, atol=0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_grouped_modelling_and_normal_operator_equal_the_single_context(prec):
    """Forward modelling (point and extended sources), the adjoint with its source-point
    output, and the normal operator, three shots in two groups: per shot, the same numbers."""
    v, geom, p = _case()
    nt = p["nt"]
    wav = _dev(np.stack([synth.ricker(nt, p["dt"], f) for f in (25.0, 21.0, 30.0)]), prec)
    q = _dev(synth.normal(9, (geom.ns, nt) + v.shape) * 1e-3, prec)
    ctx1, ctxg = _ctx(v, geom, p, prec), _ctx(v, geom, p, prec)
    ctxg.set_shot_groups(2)
    d1, dg = ctx1.forward(wavelet=wav, ext=q), ctxg.forward(wavelet=wav, ext=q)
    assert torch.equal(d1, dg)
    f1, w1 = ctx1.adjoint(d1, want_wavelet=True)
    fg, wg = ctxg.adjoint(d1, want_wavelet=True)
    assert torch.equal(f1, fg) and torch.equal(w1, wg)
    a1, ag = ctx1.normal_apply(q, 3e-4), ctxg.normal_apply(q, 3e-4)
    assert torch.equal(a1, ag)


def test_grouped_wri_data_space_and_frequency_domain_solves_fp64():
    """The WRI, data-space and frequency-domain solves with three shots in three groups:
    iterates and residual histories of the single context."""
    v, geom, p = _case()
    nt = p["nt"]
    o, shots = _orc(v, geom, p, vref=float(v.max()))
    wav = np.stack([synth.ricker(nt, p["dt"], 25.0)] * geom.ns)
    d = np.concatenate([o.forward(sh, wavelet=wav[s])["traces"].ravel() for s, sh in enumerate(shots)])
    dn = d + synth.normal(44, d.shape) * np.abs(d).max()
    ctx1 = _ctx(v, geom, p, "f64", vref=float(v.max()))
    ctxg = _ctx(v, geom, p, "f64", vref=float(v.max()))
    ctxg.set_shot_groups(3)
    runs = [dict(d=dn, lam=0.05, kw=dict(wri_wavelet=_dev(wav, "f64"))),
            dict(d=d, lam=2e-4, kw=dict(data_space=True)),
            dict(d=d, lam=2e-4, kw=dict(freqs=[8.0, 15.5, 23.0], precond="diag"))]
    for run in runs:
        x1, r1 = ctx1.cg_solve(_dev(run["d"], "f64"), lam=run["lam"], tol=0.0, max_iter=4, **run["kw"])
        xg, rg = ctxg.cg_solve(_dev(run["d"], "f64"), lam=run["lam"], tol=0.0, max_iter=4, **run["kw"])
        assert list(rg["iters"]) == list(r1["iters"]), run["kw"]
        for s in range(geom.ns):
            assert np.allclose(rg["rel_res"][s], r1["rel_res"][s], rtol=1e-12, atol=0), (run["kw"], s)
        assert torch.allclose(xg, x1, rtol=1e-12, atol=1e-300), run["kw"]


@pytest.mark.parametrize("mode", ["esi", "wri"])
def test_grouped_outer_loop_follows_the_single_context_fp64(mode):
    """esi_invert with two shot groups: its inner solves and gradients run on the groups (the
    gradient's partial sums are added in group order, a rounding-order difference), and the
    loop takes the same steps as on the single context."""
    from test_gpu_outer import _ctx as _octx, _dcat, _dev as _odev, _problem
    v, geom, pb, f = _problem()
    kw = dict(mode=mode, n_outer=3, n_cg=10, precond="diag", beta0=0.1, growth=1.0,
              vmin=1400.0, vmax=2600.0)
    outs = []
    for groups in (1, 2):
        ctx = _octx(v, geom, pb, torch.float64)
        if groups > 1:
            ctx.set_shot_groups(groups)
        vel = _odev(v, torch.float64)
        wav = _odev(np.stack([f] * geom.ns), torch.float64) if mode == "wri" else None
        g, rep = ctx.invert(_dcat(pb, torch.float64), vel, wavelet=wav, **kw)
        outs.append((vel.cpu().numpy(), g.cpu().numpy(), rep))
    (v1, g1, r1), (v2, g2, r2) = outs
    assert r2["stop"] == r1["stop"] and r2["trials"] == r1["trials"]
    assert np.allclose(r2["J_start"], r1["J_start"], rtol=1e-10, atol=0)
    assert np.allclose(r2["J_end"], r1["J_end"], rtol=1e-10, atol=0)
    assert oracle.rel_l2(v2 - v, v1 - v) < 1e-8
    assert oracle.rel_l2(g2.ravel(), g1.ravel()) < 1e-8
