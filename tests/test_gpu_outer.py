"""Parity of the CUDA outer loop (esi_invert, Algorithm "nestedloop") and of the objective the
saddle-point gradient returns (Eq. "esi", "wrimisfit") with the FP64 oracle."""
import numpy as np
import pytest

import oracle
from oracle import outer
from paper_2211_06300_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _esi():
    from paper_2211_06300_gb300 import esi
    return esi


def _dev(a, dt):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _problem(nt=40, shape=(14, 36), ns=3):
    """Three shots (a full receiver line, a sparse off-node one, a single receiver at the last
    column) over a 14 x 36 model: a partial tile in both directions, padded x pitch."""
    dx, dt, nb = 10.0, 1e-3, 4
    v = synth.dipping_layers(shape, dx, 5, nlayers=3, vmin=1500, vmax=2300, nanom=1, sigma=25.0)
    vt = v + synth.gaussian_blob(shape, dx, 3, amp=60.0, sigma=30.0)
    xs = [55.0, 175.5, 300.0][:ns]
    rx = [np.arange(5.0, 355.0, 10.0), np.arange(0.0, 350.0, 23.0), np.array([347.5])][:ns]
    geom = synth.surface_line(ns, xs, 40.0, rx, 40.0)
    f = synth.ricker(nt, dt, 45.0)
    o_true = oracle.Oracle(vt, dx, dt, nt, nb, vref=2500.0)
    d = [o_true.forward(o_true.shot(geom.src_xyz[s], geom.receivers(s)), wavelet=f)["traces"]
         for s in range(ns)]
    pb = outer.Problem(dx, dt, nt, nb, 2500.0, [geom.src_xyz[s] for s in range(ns)],
                       [geom.receivers(s) for s in range(ns)], d, wavelets=[f] * ns)
    return v, geom, pb, f


def _ctx(v, geom, pb, dt):
    return _esi().Context(_dev(v, dt), pb.dx, pb.dt, pb.nt, pb.nb, geom, vref=pb.vref)


def _dcat(pb, dt):
    return _dev(np.concatenate([x.ravel() for x in pb.d]), dt)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("mode", ["esi", "wri"])
def test_objective_from_the_saddle_gradient_matches_oracle(prec, mode):
    v, geom, pb, f = _problem()
    dt = torch.float64 if prec == "f64" else torch.float32
    ctx = _ctx(v, geom, pb, dt)
    nt = pb.nt
    beta = 0.1 if mode == "esi" else 5e-2
    q = synth.normal(17, (geom.ns, nt) + v.shape) * 1e-3
    kw = dict(wavelet=_dev(np.stack([f] * geom.ns), dt)) if mode == "wri" else {}
    g, J = ctx.gradient(ext=_dev(q, dt), dobs=_dcat(pb, dt),
                        mode="saddle" if mode == "esi" else "wri", beta=beta, param="v", **kw)
    o = oracle.Oracle(v, pb.dx, pb.dt, nt, pb.nb, vref=pb.vref)
    J_ref, g_ref = 0.0, 0.0
    for s in range(geom.ns):
        sh = o.shot(geom.src_xyz[s], geom.receivers(s))
        qs = q[s].reshape(nt, -1)
        if mode == "esi":
            J_ref += outer.esi_objective(o, sh, qs, pb.d[s], beta)
            g_ref = g_ref + o.saddle_gradient(sh, qs, beta, param="v")
        else:
            J_ref += o.wri_objective(sh, qs, pb.d[s], f, beta)
            g_ref = g_ref + o.wri_gradient(sh, qs, f, beta, param="v")
    assert J == pytest.approx(J_ref, rel=1e-12 if prec == "f64" else 1e-5)
    assert oracle.rel_l2(g.double().cpu().numpy().ravel(), g_ref) <= \
        (1e-12 if prec == "f64" else 1e-4)


@pytest.mark.parametrize("mode,precond,beta0,growth", [("esi", "diag", 0.1, 1.0),
                                                       ("esi", "diag", 0.1, 3.0),
                                                       ("esi", "none", 0.1, 1.0),
                                                       ("wri", "none", 5e-2, 1.0)])
def test_outer_loop_fp64_matches_oracle(mode, precond, beta0, growth):
    v, geom, pb, f = _problem()
    opt = outer.Options(mode=mode, n_outer=3, n_cg=10, precond=precond, beta0=beta0,
                        growth=growth, vmin=1400.0, vmax=2600.0)
    ref = outer.invert(v, pb, opt)
    ctx = _ctx(v, geom, pb, torch.float64)
    vel = _dev(v, torch.float64)
    wav = _dev(np.stack([f] * geom.ns), torch.float64) if mode == "wri" else None
    g, rep = ctx.invert(_dcat(pb, torch.float64), vel, mode=mode, n_outer=3, n_cg=10,
                        precond=precond, beta0=beta0, growth=growth, vmin=1400.0, vmax=2600.0,
                        wavelet=wav)
    assert rep["stop"] == ref["status"] == "ok"
    assert rep["trials"] == ref["trials"]
    assert np.allclose(rep["beta"], ref["beta"], rtol=1e-15)
    assert np.allclose(rep["J_start"], ref["J_start"], rtol=1e-9, atol=0)
    assert np.allclose(rep["J_end"], ref["J_end"], rtol=1e-9, atol=0)
    assert np.allclose(rep["alpha"], ref["alpha"], rtol=1e-8, atol=0)
    # the model update (the CG iterates carry rounding-order differences amplified by the
    # conditioning of the inner systems, as in the CG parity tests)
    assert oracle.rel_l2(vel.cpu().numpy() - v, ref["v"] - v) < 1e-6
    assert oracle.rel_l2(g.cpu().numpy().ravel(), ref["g_final"]) < 1e-6


def test_outer_loop_fp32_follows_the_oracle():
    """FP32 with the inner solves taken to 1e-4: a truncated (10-iteration) inner CG amplifies
    FP32 rounding of its iterates into per-cent differences of J, so the comparison with the
    FP64 oracle uses converged inner solutions."""
    v, geom, pb, f = _problem()
    opt = outer.Options(mode="esi", n_outer=3, n_cg=400, cg_tol=1e-4, precond="diag",
                        beta0=0.1, vmin=1400.0, vmax=2600.0)
    ref = outer.invert(v, pb, opt)
    ctx = _ctx(v, geom, pb, torch.float32)
    vel = _dev(v, torch.float32)
    _, rep = ctx.invert(_dcat(pb, torch.float32), vel, n_outer=3, n_cg=400, cg_tol=1e-4,
                        precond="diag", beta0=0.1, vmin=1400.0, vmax=2600.0)
    assert rep["stop"] == "ok" and rep["trials"] == ref["trials"]
    assert np.allclose(rep["J_end"], ref["J_end"], rtol=2e-3, atol=0)
    assert oracle.rel_l2(vel.double().cpu().numpy() - v, ref["v"] - v) < 5e-2


def test_reduce_callback_sees_every_evaluation_and_scaling_leaves_the_path():
    """A reduce that doubles J and g (two identical ranks) leaves the iterates unchanged: the
    first step, L-BFGS and the Armijo test are invariant to scaling the objective by 2."""
    v, geom, pb, f = _problem()
    runs = []
    for scale in (None, 2.0):
        ctx = _ctx(v, geom, pb, torch.float64)
        vel = _dev(v, torch.float64)
        calls = []

        def red(J, g, scale=scale):
            calls.append(J)
            g.mul_(scale)
            return scale * J
        _, rep = ctx.invert(_dcat(pb, torch.float64), vel, n_outer=3, n_cg=10, beta0=0.1,
                            vmin=1400.0, vmax=2600.0, reduce=None if scale is None else red)
        runs.append((vel.cpu().numpy(), rep, len(calls)))
    (v1, r1, _), (v2, r2, nc) = runs
    assert nc == r2["evaluations"] > 3
    assert r1["trials"] == r2["trials"]
    assert np.allclose(np.asarray(r2["J_end"]), 2 * np.asarray(r1["J_end"]), rtol=1e-12)
    assert oracle.rel_l2(v2, v1) < 1e-12


def test_outer_loop_rejects_bad_options():
    v, geom, pb, f = _problem()
    esi = _esi()
    ctx = _ctx(v, geom, pb, torch.float64)
    vel = _dev(v, torch.float64)
    d = _dcat(pb, torch.float64)
    with pytest.raises(esi.EsiError):
        ctx.invert(d, vel, vmin=2000.0, vmax=1500.0)
    with pytest.raises(esi.EsiError):
        ctx.invert(d, vel, mode="wri")          # no point sources
    with pytest.raises(esi.EsiError):
        ctx.invert(d, vel, memory=0)
    assert np.array_equal(vel.cpu().numpy(), v)  # nothing ran


def test_outer_loop_on_zero_data_stops_at_a_zero_gradient():
    """Zero data: the inner solution is q = 0, so J = 0 and g = 0 and the loop stops before
    its first step, leaving the model as it was."""
    v, geom, pb, f = _problem()
    ctx = _ctx(v, geom, pb, torch.float64)
    vel = _dev(v, torch.float64)
    d0 = torch.zeros(sum(x.size for x in pb.d), dtype=torch.float64, device="cuda")
    g, rep = ctx.invert(d0, vel, n_outer=2, n_cg=5, beta0=0.1, vmin=1400.0, vmax=2600.0)
    assert rep["stop"] == "zero gradient" and rep["iters_done"] == 0
    assert rep["evaluations"] == 1
    assert torch.count_nonzero(g).item() == 0
    assert np.array_equal(vel.cpu().numpy(), v)


def test_failed_line_search_leaves_the_model_and_reports_it():
    """A strict Armijo constant and two trials of a large first step: the line search fails
    on both sides, the loop stops with the model unchanged and reports the trials."""
    v, geom, pb, f = _problem()
    kw = dict(n_outer=2, n_cg=10, beta0=0.1, vmin=1000.0, vmax=2900.0, step_frac=0.5,
              max_ls=2, c1=0.9)
    ref = outer.invert(v, pb, outer.Options(mode="esi", **kw))
    ctx = _ctx(v, geom, pb, torch.float64)
    vel = _dev(v, torch.float64)
    _, rep = ctx.invert(_dcat(pb, torch.float64), vel, **kw)
    assert ref["status"] == rep["stop"] == "line search failed"
    assert rep["trials"] == ref["trials"] == [2] and rep["iters_done"] == 0
    assert rep["evaluations"] == 3
    assert np.allclose(rep["J_start"], ref["J_start"], rtol=1e-9, atol=0)
    assert np.array_equal(vel.cpu().numpy(), v)
