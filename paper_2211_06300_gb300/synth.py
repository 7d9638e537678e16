"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the CPU oracle.

This module only *generates inputs*: velocity models, acquisition geometries, source
wavelets and random test vectors.  It contains none of the method's arithmetic (no
stencil, no interpolation weights, no sponge profile, no operator) so that the oracle
and the GPU path stay independent while being fed identical data.

Workload recipes (the paper prints no numeric geometry for its experiments, so these
are synthetic stand-ins of the same shape class, cf. the two-layer reflection test and
the Marmousi-II surface acquisition of the Numerical tests section):

* ``two_layer``      : 1500 / 2500 m/s, interface depth given in metres.
* ``dipping_layers`` : ``nlayers`` layers with velocities linspace(vmin, vmax) in depth,
                       interfaces at evenly spaced mean depths with a random dip in
                       [-10, 10] degrees (clipped so they never cross), plus ``nanom``
                       Gaussian anomalies of amplitude +-``anom_amp`` and width ``sigma``.
* ``smooth``         : Gaussian smoothing of a model (starting models).
* ``ricker``         : unit-peak Ricker wavelet, delay 1.5 / f_peak.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np


def ricker(nt: int, dt: float, f_peak: float, delay: Optional[float] = None) -> np.ndarray:
    """Unit-peak Ricker wavelet sampled at t_n = n*dt, n = 0..nt-1 (float64)."""
    if delay is None:
        delay = 1.5 / f_peak
    t = np.arange(nt, dtype=np.float64) * dt - delay
    a = (math.pi * f_peak * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def two_layer(shape: Sequence[int], dx: float, v_top: float, v_bottom: float,
              z_interface: float) -> np.ndarray:
    """Two-layer model; ``shape`` is (nz, nx) or (nz, ny, nx); z is axis 0."""
    v = np.full(tuple(shape), v_top, dtype=np.float64)
    nz = shape[0]
    z = np.arange(nz) * dx
    v[z >= z_interface, ...] = v_bottom
    return v


def dipping_layers(shape: Sequence[int], dx: float, seed: int, nlayers: int = 8,
                   vmin: float = 1500.0, vmax: float = 4500.0, nanom: int = 5,
                   anom_amp: float = 300.0, sigma: float = 100.0,
                   max_dip_deg: float = 10.0, z_top: float = 0.0) -> np.ndarray:
    """Seeded layered model with dipping interfaces and Gaussian anomalies.

    Works for 2D (nz, nx) and 3D (nz, ny, nx) shapes; in 3D each interface is a plane
    with a random dip along x and along y.
    """
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    ndim = len(shape)
    nz = shape[0]
    zc = np.arange(nz, dtype=np.float64) * dx
    vel = np.linspace(vmin, vmax, nlayers)
    depth = nz * dx
    mean_depths = z_top + (depth - z_top) * (np.arange(1, nlayers) / nlayers)
    if ndim == 2:
        xs = np.arange(shape[1]) * dx
        coords = [xs - xs.mean()]
    else:
        ys = np.arange(shape[1]) * dx
        xs = np.arange(shape[2]) * dx
        coords = [ys - ys.mean(), xs - xs.mean()]
    dips = rng.uniform(-max_dip_deg, max_dip_deg, size=(nlayers - 1, ndim - 1))
    # interface depth surfaces, shape = lateral shape
    lat_shape = shape[1:]
    surf = np.empty((nlayers - 1,) + lat_shape)
    for k in range(nlayers - 1):
        s = np.full(lat_shape, mean_depths[k])
        if ndim == 2:
            s = s + np.tan(np.radians(dips[k, 0])) * coords[0]
        else:
            s = s + np.tan(np.radians(dips[k, 0])) * coords[0][:, None] \
                  + np.tan(np.radians(dips[k, 1])) * coords[1][None, :]
        surf[k] = s
    # non-crossing: each interface at least one cell below the previous one
    for k in range(1, nlayers - 1):
        surf[k] = np.maximum(surf[k], surf[k - 1] + dx)
    zgrid = zc.reshape((nz,) + (1,) * (ndim - 1))
    layer = np.zeros(shape, dtype=np.int64)
    for k in range(nlayers - 1):
        layer += (zgrid >= surf[k][None, ...]).astype(np.int64)
    v = vel[layer]
    # Gaussian anomalies
    grids = np.meshgrid(*[np.arange(n) * dx for n in shape], indexing="ij")
    for _ in range(nanom):
        centre = [rng.uniform(0.15, 0.85) * n * dx for n in shape]
        amp = anom_amp * (1.0 if rng.uniform() < 0.5 else -1.0)
        r2 = sum((g - c) ** 2 for g, c in zip(grids, centre))
        v = v + amp * np.exp(-0.5 * r2 / sigma ** 2)
    return v


def smooth(v: np.ndarray, sigma_m: float, dx: float) -> np.ndarray:
    """Gaussian smoothing (reflecting edges), used for starting models."""
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(v, sigma=sigma_m / dx, mode="nearest")


def gaussian_blob(shape: Sequence[int], dx: float, seed: int, amp: float = 10.0,
                  sigma: float = 100.0, margin: float = 0.2) -> np.ndarray:
    """A seeded smooth model perturbation (used for directional-derivative tests)."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.arange(n) * dx for n in shape], indexing="ij")
    centre = [rng.uniform(margin, 1.0 - margin) * n * dx for n in shape]
    r2 = sum((g - c) ** 2 for g, c in zip(grids, centre))
    sign = 1.0 if rng.uniform() < 0.5 else -1.0
    return sign * amp * np.exp(-0.5 * r2 / sigma ** 2)


def normal(seed: int, shape: Sequence[int]) -> np.ndarray:
    """i.i.d. N(0,1) float64 test vector."""
    return np.random.default_rng(seed).standard_normal(tuple(shape))


@dataclasses.dataclass
class Geometry:
    """Acquisition geometry in metres; positions are (x, y, z) triples (y = 0 in 2D).

    Receivers are CSR-packed: shot s owns rec_xyz[rec_offset[s]:rec_offset[s+1]].
    """
    src_xyz: np.ndarray          # (ns, 3)
    rec_offset: np.ndarray       # (ns + 1,) int64
    rec_xyz: np.ndarray          # (total, 3)

    @property
    def ns(self) -> int:
        return int(self.src_xyz.shape[0])

    def nrec(self, s: int) -> int:
        return int(self.rec_offset[s + 1] - self.rec_offset[s])

    def receivers(self, s: int) -> np.ndarray:
        return self.rec_xyz[self.rec_offset[s]:self.rec_offset[s + 1]]

    def select(self, shots: Sequence[int]) -> "Geometry":
        src = self.src_xyz[list(shots)]
        recs = [self.receivers(s) for s in shots]
        off = np.zeros(len(recs) + 1, dtype=np.int64)
        off[1:] = np.cumsum([len(r) for r in recs])
        return Geometry(src, off, np.concatenate(recs, axis=0) if recs else np.zeros((0, 3)))


def surface_line(ns: int, src_x: Sequence[float], src_z: float,
                 rec_x_per_shot: Sequence[np.ndarray], rec_z: float) -> Geometry:
    src = np.zeros((ns, 3))
    src[:, 0] = np.asarray(src_x, dtype=np.float64)
    src[:, 2] = src_z
    off = np.zeros(ns + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) for r in rec_x_per_shot])
    rec = np.zeros((int(off[-1]), 3))
    for s in range(ns):
        rx = np.asarray(rec_x_per_shot[s], dtype=np.float64)
        rec[off[s]:off[s + 1], 0] = rx
        rec[off[s]:off[s + 1], 2] = rec_z
    return Geometry(src, off, rec)


def surface_grid_3d(src_xyz: Tuple[float, float, float], rec_x: np.ndarray, rec_y: np.ndarray,
                    rec_z: float) -> Geometry:
    gx, gy = np.meshgrid(rec_x, rec_y, indexing="xy")
    rec = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, rec_z)], axis=1)
    off = np.array([0, rec.shape[0]], dtype=np.int64)
    return Geometry(np.asarray([src_xyz], dtype=np.float64), off, rec)


# --------------------------------------------------------------------------------------
# Workload recipes.  Sizes follow the five workloads the method is benchmarked on.
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    shape: Tuple[int, ...]       # (nz, nx) or (nz, ny, nx), sponge included
    dx: float
    dt: float
    nt: int
    nb: int
    f_peak: float
    v_true: np.ndarray
    v_start: np.ndarray
    geom: Geometry
    dtype: str                   # "f32" or "f64"
    beta: Optional[float] = None

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def ncell(self) -> int:
        return int(np.prod(self.shape))

    def wavelets(self) -> np.ndarray:
        w = ricker(self.nt, self.dt, self.f_peak)
        return np.tile(w, (self.geom.ns, 1))


def workload_small_2d(nt: int = 500) -> Workload:
    """101 x 101 (20-cell sponge), dx 10 m, dt 1 ms, nt 500, FP64; two layers 1500/2500 m/s
    with the interface at 500 m; one 15 Hz Ricker at (505 m, 20 m); 101 receivers at 20 m."""
    shape = (101, 101)
    dx = 10.0
    v = two_layer(shape, dx, 1500.0, 2500.0, 500.0)
    geom = surface_line(1, [505.0], 20.0, [np.arange(101) * dx], 20.0)
    return Workload("2d-101x101-two-layer-fp64", shape, dx, 1e-3, nt, 20, 15.0, v,
                    np.full(shape, 1500.0), geom, "f64", beta=1.0)


def workload_esi_2d(nt: int = 3000, ns: int = 16, seed: int = 2) -> Workload:
    """801 x 241 (z = 241 rows, x = 801 columns), dx 12.5 m, dt 1 ms, nt 3000, FP32;
    8 dipping layers 1500-4500 m/s + 5 Gaussian anomalies; ``ns`` 8 Hz Ricker shots
    evenly spaced over the interior columns, 801 receivers on every column, source and
    receivers on row nb + 2."""
    shape = (241, 801)
    dx, nb = 12.5, 20
    v = dipping_layers(shape, dx, seed, z_top=(nb + 4) * dx)
    v0 = smooth(v, 250.0, dx)
    zr = (nb + 2) * dx
    interior = np.linspace(nb + 2, shape[1] - 1 - nb - 2, ns)
    src_x = np.round(interior) * dx
    rec = [np.arange(shape[1]) * dx for _ in range(ns)]
    geom = surface_line(ns, src_x, zr, rec, zr)
    return Workload(f"2d-801x241-nt{nt}-{ns}shots-dipping-fp32", shape, dx, 1e-3, nt, nb, 8.0,
                    v, v0, geom, "f32")


def workload_batched_2d(nt: int = 3000, ns: int = 64, seed: int = 3) -> Workload:
    """1201 x 301 grid, 64 shots with uneven apertures of 201..801 receivers (centred on
    the source, clipped to the grid), dx 12.5 m, dt 1 ms, nt 3000, FP32."""
    shape = (301, 1201)
    dx, nb = 12.5, 20
    rng = np.random.default_rng(seed + 1000)
    v = dipping_layers(shape, dx, seed, z_top=(nb + 4) * dx)
    v0 = smooth(v, 250.0, dx)
    zr = (nb + 2) * dx
    cols = np.round(np.linspace(nb + 2, shape[1] - 1 - nb - 2, ns)).astype(int)
    rec = []
    for c in cols:
        ap = int(rng.integers(201, 802))
        lo = max(0, c - ap // 2)
        hi = min(shape[1], lo + ap)
        lo = max(0, hi - ap)
        rec.append(np.arange(lo, hi) * dx)
    geom = surface_line(ns, cols * dx, zr, rec, zr)
    return Workload(f"2d-1201x301-nt{nt}-{ns}shots-uneven-fp32", shape, dx, 1e-3, nt, nb, 8.0,
                    v, v0, geom, "f32")


def workload_3d(n: int = 400, nt: int = 2000, seed: int = 4) -> Workload:
    """n^3 grid (default 400^3), dx 10 m, dt 0.8 ms, nt 2000, FP32; layered + anomaly
    model (1500-4500 m/s); one 10 Hz shot at the centre column on row nb + 2; a
    160 x 160 receiver grid every 2nd node, centred, on the same row."""
    shape = (n, n, n)
    dx, nb = 10.0, 20
    v = dipping_layers(shape, dx, seed, z_top=(nb + 4) * dx)
    zr = (nb + 2) * dx
    c = (n // 2) * dx
    nrec = min(160, (n - 2 * nb) // 2)
    r = (np.arange(nrec) - (nrec - 1) / 2.0) * 2 * dx + c
    r = np.round(r / dx) * dx
    geom = surface_grid_3d((c, c, zr), r, r, zr)
    return Workload(f"3d-{n}^3-nt{nt}-fp32", shape, dx, 0.8e-3, nt, nb, 10.0, v,
                    smooth(v, 250.0, dx) if n <= 160 else v, geom, "f32")
