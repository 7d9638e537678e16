"""Parity of the misfit-landscape scan (section "Misfit landscape in transmission case") with
the FP64 oracle: the FWI, WRI and ESI objectives at three velocity errors, fixed penalties."""
import numpy as np
import pytest

import oracle
from oracle import outer
from paper_2211_06300_gb300 import landscape, synth

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_scan_matches_oracle_fp64():
    shape, dx, dt, nt, nb, fp = (36, 40), 10.0, 1e-3, 160, 6, 30.0
    v = landscape.layered_model(shape, dx, seed=5, nlayers=3)
    eps = [-0.3, 0.0, 0.2]
    betas = {"wri": {100.0: 2e-2, 0.01: 2e-6}, "esi": {100.0: 1e-3, 0.01: 1e-7}}
    r = landscape.scan(v, dx, dt, nt, nb, fp, eps, n_cg=10, dtype="f64", betas=betas,
                       cg_tol=0.0)
    assert r["breakdowns"] == []
    geom = landscape.acquisition(shape, dx, nb)
    vref = float(v.max()) * 1.3
    f = synth.ricker(nt, dt, fp)
    o_t = oracle.Oracle(v, dx, dt, nt, nb, vref=vref)
    d = o_t.forward(o_t.shot(geom.src_xyz[0], geom.receivers(0)), wavelet=f)["traces"]
    for k, e in enumerate(eps):
        o = oracle.Oracle(v * (1 + e), dx, dt, nt, nb, vref=vref)
        sh = o.shot(geom.src_xyz[0], geom.receivers(0))
        J_fwi = o.misfit_gradient(sh, d, wavelet=f, param="v")[0]
        assert r["fwi"][k] == pytest.approx(J_fwi, rel=1e-9, abs=1e-20)
        B = o.annihilator(sh.src_xyz)
        for b in (100.0, 0.01):
            bw, be = betas["wri"][b], betas["esi"][b]
            q = o.wri_cg(sh, d, f, bw, 0.0, 10)["x"]
            assert r["wri"][b][k] == pytest.approx(o.wri_objective(sh, q, d, f, bw), rel=1e-9,
                                                   abs=1e-20)
            q = o.pcg(sh, d, be, 0.0, 10, minv=1.0 / (be * B * B))["x"]
            assert r["esi"][b][k] == pytest.approx(outer.esi_objective(o, sh, q, d, be), rel=1e-9)
