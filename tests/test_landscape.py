"""Host logic of the misfit-landscape experiment: the 1D layered model, the acquisition frame
(source on a receiver at the top-left corner, three receiver lines) and the basin summary."""
import numpy as np

from paper_2211_06300_gb300 import landscape


def test_layered_model_is_one_dimensional_and_increasing():
    v = landscape.layered_model((61, 47), 10.0, seed=3, nlayers=4)
    assert np.all(v == v[:, :1])
    col = v[:, 0]
    assert np.all(np.diff(col) >= 0) and col[0] == 1500.0 and col[-1] == 3000.0
    assert len(np.unique(col)) == 4


def test_acquisition_frame():
    shape, dx, nb = (50, 60), 10.0, 6
    g = landscape.acquisition(shape, dx, nb, step=2)
    src = g.src_xyz[0]
    rec = g.receivers(0)
    assert any(np.allclose(r, src) for r in rec)                 # source on a receiver
    xs = sorted(set(rec[:, 0]))
    assert xs[0] == src[0] and xs[-1] == (shape[1] - nb - 3) * dx
    assert np.all(rec[:, 2] >= src[2]) and rec[:, 2].max() <= (shape[0] - nb - 3) * dx
    on_top = rec[:, 2] == src[2]
    on_sides = (rec[:, 0] == xs[0]) | (rec[:, 0] == xs[-1])
    assert np.all(on_top | on_sides)


def test_basin_summary():
    eps = np.linspace(-0.5, 0.5, 11)
    conv = landscape.basin(eps, (eps - 0.1) ** 2)
    assert conv["local_minima_eps"] == [eps[6]] and conv["basin_eps"] == [-0.5, 0.5]
    wavy = (eps ** 2) - 0.2 * np.cos(12 * eps) * (np.abs(eps) > 0.25)
    w = landscape.basin(eps, wavy)
    assert len(w["local_minima_eps"]) > 1
    assert w["basin_eps"][0] > -0.5 or w["basin_eps"][1] < 0.5
