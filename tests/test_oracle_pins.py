"""Pins of the oracle's geometry and boundary functions against values fixed by the
mathematics, each with a planted mistake (on the CPU, in a copy of the oracle function)
that the pin must catch.

* ``point_weights``: the sampling operator R of Eq. "fwi" and the point-source injection
  at positions off the grid nodes (bilinear in 2D, trilinear in 3D).  Pinned by exact
  reproduction of every function that is linear in each axis, partition of unity,
  hand-computed weights at an asymmetric point, and the analytic 2D Green's function with
  source and receiver both off the nodes.
* ``Oracle.annihilator``: B = ||x - x_s|| + eps of the ESI section (the small positive
  number of the Numerical tests section is eps = dx).  Pinned by hand-computed distances
  on Pythagorean triples with a source whose x and z differ, and by the beta B^2 term of
  the normal operator (Eq. "normalewi") at those cells.
* ``sponge_kappa``: the absorbing boundary of the Numerical tests section, read as a
  damping term eta u_t with eta = eta_max sum_axes (d/nb)^2.  Pinned by its values at
  interior, face, ramp and corner cells, and by the closed-form decay of the damped
  recurrence at a sponge cell.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2211_06300_gb300 import synth
from test_oracle import _green2d_ricker


# ----------------------------------------------------------------------------- helpers
def _node_xyz(flat, shape, dx):
    """Position (x, y, z) in metres of a flat node index on a (nz, nx) or (nz, ny, nx)
    grid, node (iz, iy, ix) sitting at (ix dx, iy dx, iz dx)."""
    if len(shape) == 2:
        iz, ix = divmod(int(flat), shape[1])
        return ix * dx, 0.0, iz * dx
    nz, ny, nx = shape
    iz, rem = divmod(int(flat), ny * nx)
    iy, ix = divmod(rem, nx)
    return ix * dx, iy * dx, iz * dx


def _multilinear_error(pw, shape, dx, seed):
    """Largest error of sum_i w_i f(node_i) against f(p) over random points p, for random
    functions f linear in each axis (f = sum of coefficients x products of distinct axes).
    Bilinear / trilinear interpolation reproduces every such function exactly."""
    rng = np.random.default_rng(seed)
    nd = len(shape)
    ext = [shape[-1] - 1, 0 if nd == 2 else shape[1] - 1, shape[0] - 1]   # x, y, z cells
    worst = 0.0
    for _ in range(40):
        a = rng.standard_normal(8)

        def f(x, y, z):
            return (a[0] + a[1] * x + a[2] * y + a[3] * z + a[4] * x * y + a[5] * x * z
                    + a[6] * y * z + a[7] * x * y * z) if nd == 3 else \
                   (a[0] + a[1] * x + a[3] * z + a[5] * x * z)
        p = [rng.uniform(0, e) * dx if e > 0 else 0.0 for e in ext]
        try:
            nodes, w = pw(p, shape, dx)
        except ValueError:              # a mistaken axis order can leave the grid
            return math.inf
        got = sum(wi * f(*_node_xyz(n, shape, dx)) for n, wi in zip(nodes, w))
        worst = max(worst, abs(got - f(*p)) / (1.0 + abs(f(*p))))
    return worst


# planted mistakes (the oracle function with one error each)
_POINT_WEIGHTS = oracle.point_weights


def _pw_weights_swapped(pos, shape, dx):
    """(1 - w, w) exchanged on every axis: the point mirrored inside its cell."""
    f = [p / dx - math.floor(p / dx) for p in pos]
    mirrored = [(math.floor(p / dx) + 1 - fr) * dx if fr else p for p, fr in zip(pos, f)]
    return _POINT_WEIGHTS(mirrored, shape, dx)


def _pw_axes_exchanged(pos, shape, dx):
    """x and z exchanged (node order (x, z) instead of (z, x))."""
    x, y, z = pos
    return _POINT_WEIGHTS((z, y, x), shape, dx)


# ----------------------------------------------------------------------------- point_weights
@pytest.mark.parametrize("shape", [(13, 21), (7, 9, 11)])
def test_point_weights_reproduce_multilinear_functions(shape):
    assert _multilinear_error(oracle.point_weights, shape, 2.5, seed=1) < 1e-12
    # each planted mistake breaks exact reproduction
    assert _multilinear_error(_pw_weights_swapped, shape, 2.5, seed=1) > 1e-3
    assert _multilinear_error(_pw_axes_exchanged, shape, 2.5, seed=1) > 1e-3


@pytest.mark.parametrize("shape", [(13, 21), (7, 9, 11)])
def test_point_weights_partition_of_unity_and_node_count(shape):
    rng = np.random.default_rng(2)
    nd = len(shape)
    for _ in range(50):
        p = [rng.uniform(0, shape[-1] - 1), rng.uniform(0, shape[1] - 1) if nd == 3 else 0.0,
             rng.uniform(0, shape[0] - 1)]
        nodes, w = oracle.point_weights(p, shape, 1.0)
        assert len(nodes) == 2 ** nd
        assert abs(w.sum() - 1.0) < 1e-14
        assert np.all(w > 0)
    # on a node: one node, weight 1; on a cell face: two nodes
    nodes, w = oracle.point_weights((3.0, 0.0, 4.0), (13, 21), 1.0)
    assert list(nodes) == [4 * 21 + 3] and list(w) == [1.0]
    nodes, w = oracle.point_weights((3.5, 0.0, 4.0), (13, 21), 1.0)
    assert sorted(nodes.tolist()) == [4 * 21 + 3, 4 * 21 + 4]
    assert np.allclose(w, [0.5, 0.5], rtol=0, atol=0)
    with pytest.raises(ValueError):
        oracle.point_weights((20.5, 0.0, 1.0), (13, 21), 1.0)     # x beyond the last node


def test_point_weights_hand_computed_asymmetric_point():
    # dx = 5 m, point x = 11 m (2.2 cells), z = 8 m (1.6 cells) on a 10 x 12 (nz x nx) grid:
    # x weights 0.8 at ix = 2 and 0.2 at ix = 3; z weights 0.4 at iz = 1 and 0.6 at iz = 2
    nodes, w = oracle.point_weights((11.0, 0.0, 8.0), (10, 12), 5.0)
    got = dict(zip(nodes.tolist(), w.tolist()))
    expected = {1 * 12 + 2: 0.32, 1 * 12 + 3: 0.08, 2 * 12 + 2: 0.48, 2 * 12 + 3: 0.12}
    assert set(got) == set(expected)
    for k, v in expected.items():
        assert got[k] == pytest.approx(v, abs=1e-15)
    # 3D: x = 2.25, y = 1.5, z = 0.75 cells of dx = 2 m on a 4 x 5 x 6 grid
    nodes, w = oracle.point_weights((4.5, 3.0, 1.5), (4, 5, 6), 2.0)
    got = dict(zip(nodes.tolist(), w.tolist()))
    wx = {2: 0.75, 3: 0.25}
    wy = {1: 0.5, 2: 0.5}
    wz = {0: 0.25, 1: 0.75}
    expected = {(iz * 5 + iy) * 6 + ix: wz[iz] * wy[iy] * wx[ix]
                for iz in wz for iy in wy for ix in wx}
    assert set(got) == set(expected)
    for k, v in expected.items():
        assert got[k] == pytest.approx(v, abs=1e-15)


def _offnode_green_error(dx, dt, f_peak=10.0, T=0.45, v=2000.0):
    """Relative L2 error of the oracle trace against the analytic 2D Green's function
    convolved with a Ricker wavelet, source and receiver both off the grid nodes in both
    axes (x and z at different fractions of a cell)."""
    n = int(round(1600.0 / dx)) + 1
    nb = int(round(200.0 / dx))
    nt = int(round(T / dt))
    orc = oracle.Oracle(np.full((n, n), v), dx, dt, nt, nb)
    s = (803.7, 0.0, 806.1)
    r = (1007.9, 0.0, 795.6)
    offset = math.hypot(r[0] - s[0], r[2] - s[2])
    tr = orc.forward(orc.shot(s, [r]), wavelet=synth.ricker(nt, dt, f_peak))["traces"][:, 0]
    t = (np.arange(nt) + 1) * dt
    ref = np.array([_green2d_ricker(offset, v, tt, f_peak) for tt in t])
    return np.linalg.norm(tr - ref) / np.linalg.norm(ref)


@pytest.mark.slow
def test_offnode_source_and_receiver_match_2d_green_function(monkeypatch):
    # bilinear injection and sampling are second-order accurate: the error falls about
    # 4x when dx and dt halve (measured 2.4 % -> 0.66 %)
    e10 = _offnode_green_error(10.0, 1e-3)
    e5 = _offnode_green_error(5.0, 0.5e-3)
    assert e10 < 0.035
    assert 3.0 < e10 / e5 < 5.0
    # the weights mirrored inside the cell move both points by a fraction of a cell: the
    # trace arrives at the wrong time (measured 27 %)
    monkeypatch.setattr(oracle, "point_weights", _pw_weights_swapped)
    assert _offnode_green_error(10.0, 1e-3) > 0.15


# ----------------------------------------------------------------------------- annihilator
def _annihilator_cases():
    """(shape, dx, source (x, y, z), {flat cell: B}) with B worked out by hand on
    Pythagorean triples, the source's x and z different so that exchanging axes changes
    the distances."""
    # 2D, dx = 10 m, source at x = 30 m, z = 20 m = node (iz 2, ix 3) of a 9 x 11 grid
    nx = 11
    c2 = {2 * nx + 3: 10.0,          # the source node: distance 0, B = eps = dx
          2 * nx + 6: 40.0,          # (x 60, z 20): 30 m along x
          6 * nx + 3: 50.0,          # (x 30, z 60): 40 m along z
          6 * nx + 6: 60.0,          # (x 60, z 60): 30-40-50 triangle
          8 * nx + 10: 10.0 + math.sqrt(70.0 ** 2 + 60.0 ** 2),
          0: 10.0 + math.sqrt(30.0 ** 2 + 20.0 ** 2)}
    # 3D, dx = 5 m, source at (x 10, y 15, z 20) = node (iz 4, iy 3, ix 2) of 7 x 8 x 9
    ny, nx3 = 8, 9
    c3 = {(4 * ny + 3) * nx3 + 2: 5.0,
          (4 * ny + 3) * nx3 + 5: 20.0,          # 15 m along x
          (4 * ny + 7) * nx3 + 2: 25.0,          # 20 m along y
          (0 * ny + 3) * nx3 + 2: 25.0,          # 20 m along z
          (4 * ny + 7) * nx3 + 5: 30.0,          # 15-20-25 triangle in the x-y plane
          (0 * ny + 3) * nx3 + 8: 5.0 + math.sqrt(30.0 ** 2 + 20.0 ** 2)}   # x 40, z 0
    return [((9, 11), 10.0, (30.0, 0.0, 20.0), c2), ((7, 8, 9), 5.0, (10.0, 15.0, 20.0), c3)]


def _annihilator_error(fn):
    worst = 0.0
    for shape, dx, src, cells in _annihilator_cases():
        B = fn(shape, dx, src)
        for k, v in cells.items():
            worst = max(worst, abs(B[k] - v) / v)
    return worst


def _oracle_B(shape, dx, src, eps=None):
    orc = oracle.Oracle(np.full(shape, 2000.0), dx, 1e-4, 4, 0)
    return orc.annihilator(src, eps)


def test_annihilator_hand_computed_distances():
    assert _annihilator_error(_oracle_B) < 1e-14
    # the source node carries B = eps, and an explicit eps replaces dx
    B = _oracle_B((9, 11), 10.0, (30.0, 0.0, 20.0), eps=0.5)
    assert B[2 * 11 + 3] == 0.5 and B[2 * 11 + 6] == pytest.approx(30.5, abs=1e-13)
    # B is smallest at the source node, also for a source between nodes
    B = _oracle_B((9, 11), 10.0, (33.0, 0.0, 18.0))
    assert int(np.argmin(B)) == 2 * 11 + 3
    assert B.min() == pytest.approx(10.0 + math.hypot(3.0, 2.0), abs=1e-13)


def test_annihilator_planted_mistakes_fail():
    def squared(shape, dx, src):
        return (_oracle_B(shape, dx, src, eps=0.0)) ** 2 + dx

    def no_eps(shape, dx, src):
        return _oracle_B(shape, dx, src, eps=0.0)

    def axes_exchanged(shape, dx, src):
        return _oracle_B(shape, dx, (src[2], src[1], src[0]))
    for bad in (squared, no_eps, axes_exchanged):
        assert _annihilator_error(bad) > 0.05


def test_normal_operator_adds_beta_b_squared():
    # A(beta1) p - A(beta2) p = (beta1 - beta2) B^2 p: a unit impulse at a cell whose B is
    # known by hand picks out B^2 there
    shape, dx, dt, nt, nb = (9, 11), 10.0, 1e-3, 6, 2
    orc = oracle.Oracle(np.full(shape, 1500.0), dx, dt, nt, nb)
    sh = orc.shot((30.0, 0.0, 20.0), [(50.0, 0.0, 40.0)])
    for cell, B in [(2 * 11 + 6, 40.0), (6 * 11 + 6, 60.0), (2 * 11 + 3, 10.0)]:
        p = np.zeros((nt, orc.N))
        p[3, cell] = 1.0
        diff = orc.normal_matvec(sh, p, 7.0) - orc.normal_matvec(sh, p, 2.0)
        assert diff[3, cell] == pytest.approx(5.0 * B * B, rel=1e-12)
        diff[3, cell] = 0.0
        assert np.max(np.abs(diff)) <= 1e-12 * B * B


# ----------------------------------------------------------------------------- sponge
def _kappa_face(v, R, nb, dx, dt):
    # eta_max = 3 v ln(1/R) / (2 nb dx): for v = 2000 m/s, R = 1e-3, nb = 10, dx = 10 m
    # this is 6000 * 6.907755278982137 / 200 = 207.23265836946411 s^-1, kappa = eta dt / 2
    return 207.23265836946411 * dt / 2.0


def _sponge_error(fn):
    """Largest relative error of the profile at hand-picked cells of a 40 x 50 grid
    (nb = 10): interior 0, outermost face cell kappa_face, the quadratic ramp, and the
    corner sum of the two axes; plus the 3D corner (three axes)."""
    nb, dx, dt, v = 10, 10.0, 1e-3, 2000.0
    kf = _kappa_face(v, 1e-3, nb, dx, dt)
    k = fn((40, 50), nb, dx, dt, v).reshape(40, 50)
    cases = [((20, 25), 0.0), ((nb, nb), 0.0), ((40 - 1 - nb, 50 - 1 - nb), 0.0),
             ((20, 0), kf), ((20, 49), kf), ((0, 25), kf), ((39, 25), kf),
             ((20, 5), kf * 0.25), ((20, 44), kf * 0.25), ((20, nb - 1), kf * 0.01),
             ((3, 25), kf * 0.49), ((0, 0), 2 * kf), ((39, 49), 2 * kf),
             ((5, 2), kf * (0.25 + 0.64))]
    worst = 0.0
    for (iz, ix), ref in cases:
        worst = max(worst, abs(k[iz, ix] - ref) / kf)
    k3 = fn((24, 25, 26), nb, dx, dt, v).reshape(24, 25, 26)
    worst = max(worst, abs(k3[0, 0, 0] - 3 * kf) / kf, abs(k3[12, 12, 13]) / kf,
                abs(k3[12, 0, 13] - kf) / kf)
    return worst


def test_sponge_profile_values():
    assert _sponge_error(oracle.sponge_kappa) < 1e-13

    def linear_ramp(shape, nb, dx, dt, v):       # (d/nb) instead of (d/nb)^2
        return _ramp_power(shape, nb, dx, dt, v, 1.0)

    def full_eta(shape, nb, dx, dt, v):          # kappa = eta dt instead of eta dt / 2
        return 2.0 * oracle.sponge_kappa(shape, nb, dx, dt, v)

    def max_not_sum(shape, nb, dx, dt, v):       # corners take the larger axis, not the sum
        return _ramp_power(shape, nb, dx, dt, v, 2.0, combine=np.maximum)
    for bad in (linear_ramp, full_eta, max_not_sum):
        assert _sponge_error(bad) > 0.05


def _ramp_power(shape, nb, dx, dt, v, power, combine=np.add):
    eta_max = 3.0 * v * math.log(1e3) / (2.0 * nb * dx)
    out = np.zeros(shape)
    for axis, n in enumerate(shape):
        i = np.arange(n)
        d = np.maximum(np.maximum(nb - i, i - (n - 1 - nb)), 0) / nb
        sh = [1] * len(shape)
        sh[axis] = n
        out = combine(out, (d ** power).reshape(sh))
    return eta_max * out * dt / 2.0


def test_damped_recurrence_at_a_sponge_cell_has_closed_form():
    # With c ~ 0 (a tiny velocity, the sponge set by vref) the scheme at one cell reduces to
    # (1 + k) u_{n+1} = 2 u_n - (1 - k) u_{n-1} + c q_n, whose roots are 1 and
    # rho = (1 - k)/(1 + k).  An impulse q_0 = 1/dx^2 on the node gives
    # u_n = u_1 (1 - rho^n) / (1 - rho), u_1 = c / (dx^2 (1 + k)): the cell relaxes to
    # c / (2 k dx^2) instead of growing linearly as it does where k = 0.
    shape, dx, dt, nt, nb = (30, 30), 10.0, 1e-3, 60, 10
    v = np.full(shape, 1e-4)
    orc = oracle.Oracle(v, dx, dt, nt, nb, vref=2000.0)
    wav = np.zeros(nt)
    wav[0] = 1.0
    c = 1e-8 * dt * dt
    for (iz, ix) in [(2, 15), (15, 15)]:       # a sponge cell (d = 8 along z) and the interior
        pos = (ix * dx, 0.0, iz * dx)
        tr = orc.forward(orc.shot(pos, [pos]), wavelet=wav)["traces"][:, 0]
        k = _kappa_face(2000.0, 1e-3, nb, dx, dt) * ((nb - iz) / nb) ** 2 if iz < nb else 0.0
        n = np.arange(1, nt + 1)
        u1 = c / (dx * dx * (1 + k))
        if k > 0:
            rho = (1 - k) / (1 + k)
            ref = u1 * (1 - rho ** n) / (1 - rho)
        else:
            ref = u1 * n
        assert np.max(np.abs(tr - ref)) <= 1e-9 * np.max(np.abs(ref))
