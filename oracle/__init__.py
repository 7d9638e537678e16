"""FP64 CPU oracle for the time-domain ESI hot path (Yang & Zhou, arXiv 2211.06300).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
It shares no code with the CUDA library and never imports it.

The heavy loops (stencil, time stepping, transpose solve, DTFT sums) are plain C in
``esi_oracle.c``; this module adds what is naturally written with numpy:

* the sponge profile (absorbing boundary, Numerical tests section) and ``c = v^2 dt^2``;
* bilinear (2D) / trilinear (3D) point sampling and injection weights;
* the annihilator ``B = ||x - x_s|| + eps`` (ESI section, "B = ||x - x_s||"; the small
  positive number of the Numerical tests section is ``eps = dx``);
* the ESI normal operator ``S^T S + beta B^T B`` (Eq. "normalewi", matrix-vector product
  bullet of the CG section) and Algorithm 1 (CG) written step by step;
* the zero-lag cross-correlation gradient (Eq. "gradient", "gradewi") in both the
  adjoint-state form and the saddle-point form of Algorithm 2 (lambda = beta B^H B q);
* the frequency-domain ESI system F (S^T S + beta B^T B) F^H qbar = F S^T d (Eq. "dtft",
  "idtft", "normaldtft") and its CG with the real part of the Hermitian inner product;
* dense assembly of the normal matrix at tiny sizes and its Cholesky solution;
* FP16 / BF16 snapshot codecs with a per-snapshot scale, the two-level checkpoint code
  (all-even cells plus the interpolation residual) and the gradient recomputed from
  checkpoints in that code.

Where the paper leaves a point open, this module takes one reading and states it
where it is used: state u_{n+1} is produced by step n from q_n; sample n of a trace is
R u_{n+1}; the DTFT sums the states at their own times (n+1) dt; points off the grid
use bilinear/trilinear weights, point sources carry 1/dx^d; the sponge is a linear
damping term on all sides; inner products are plain Euclidean sums.  Every function
below is pinned by a ``-m "not gpu"`` test.  The learned CG preconditioner has no
oracle (parity unpinned): the true CG residual is its only judge.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "esi_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile esi_oracle.c into liboracle.so with gcc (plain -O2, optional OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared"]
        if openmp:
            cmd.append("-fopenmp")
        cmd += [_SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.orc_laplacian.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_long, ctypes.c_long,
                                    ctypes.c_double, _D, _D]
        L.orc_dtft_accumulate.argtypes = [ctypes.c_long, _D, ctypes.c_double, ctypes.c_int, _D,
                                          _D, _D]
        L.orc_forward.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_long, ctypes.c_long,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int, _D, _D, _D,
                                  ctypes.c_long, _L, _D, _D, ctypes.c_long, _L, _L, _D, _D, _D,
                                  _D, ctypes.c_int, _D, _D, _D]
        L.orc_adjoint.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_long, ctypes.c_long,
                                  ctypes.c_double, ctypes.c_int, _D, _D, ctypes.c_long, _L, _L,
                                  _D, _D, _D, ctypes.c_long, _L, _D, _D, _D, _D]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _lp(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(_L)


def _dims(shape: Sequence[int]) -> Tuple[int, int, int, int]:
    if len(shape) == 2:
        return 2, int(shape[0]), 1, int(shape[1])
    if len(shape) == 3:
        return 3, int(shape[0]), int(shape[1]), int(shape[2])
    raise ValueError("grid must be 2D (nz, nx) or 3D (nz, ny, nx)")


def laplacian(u: np.ndarray, dx: float) -> np.ndarray:
    """8th-order Laplacian with zero values outside the grid."""
    nd, nz, ny, nx = _dims(u.shape)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    lib().orc_laplacian(nd, nz, ny, nx, dx, _dp(u), _dp(out))
    return out


def dtft_accumulate(u: np.ndarray, t: float, freqs: Sequence[float], re: np.ndarray,
                    im: np.ndarray) -> None:
    """re/im[m] += u * exp(+j 2 pi f_m t)  (Eq. "dtft"), in place."""
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64).ravel()
    lib().orc_dtft_accumulate(u.size, _dp(u), t, f.size, _dp(f), _dp(re), _dp(im))


def sponge_kappa(shape: Sequence[int], nb: int, dx: float, dt: float, vref: float,
                 R: float = 1e-3) -> np.ndarray:
    """kappa = eta * dt / 2 with eta = eta_max * sum_axes (d/nb)^2, d the number of cells
    into the sponge along that axis (d = nb at the outermost cell), and
    eta_max = 3 vref ln(1/R) / (2 nb dx)."""
    kappa = np.zeros(tuple(shape))
    if nb <= 0:
        return kappa
    eta_max = 3.0 * vref * math.log(1.0 / R) / (2.0 * nb * dx)
    for axis, n in enumerate(shape):
        i = np.arange(n)
        d = np.maximum(np.maximum(nb - i, i - (n - 1 - nb)), 0).astype(np.float64)
        prof = (d / nb) ** 2
        sh = [1] * len(shape)
        sh[axis] = n
        kappa = kappa + prof.reshape(sh)
    return eta_max * kappa * dt / 2.0


def point_weights(pos_xyz: Sequence[float], shape: Sequence[int], dx: float
                  ) -> Tuple[np.ndarray, np.ndarray]:
    """Bilinear (2D) / trilinear (3D) weights of the point (x, y, z) metres on the grid
    whose node (iz, iy, ix) sits at (ix dx, iy dx, iz dx).  Zero weights are dropped.
    Returns (flat node indices, weights)."""
    nd, nz, ny, nx = _dims(shape)
    x, y, z = (float(p) for p in pos_xyz)
    axes = [(z, nz), (x, nx)] if nd == 2 else [(z, nz), (y, ny), (x, nx)]
    per_axis = []
    for p, n in axes:
        f = p / dx
        i0 = math.floor(f)
        w1 = f - i0
        pts = [(i0, 1.0 - w1), (i0 + 1, w1)]
        pts = [(i, w) for i, w in pts if w != 0.0]
        for i, _ in pts:
            if i < 0 or i >= n:
                raise ValueError(f"point {pos_xyz} outside the grid")
        per_axis.append(pts)
    nodes, weights = [], []
    if nd == 2:
        for iz, wz in per_axis[0]:
            for ix, wx in per_axis[1]:
                nodes.append(iz * nx + ix)
                weights.append(wz * wx)
    else:
        for iz, wz in per_axis[0]:
            for iy, wy in per_axis[1]:
                for ix, wx in per_axis[2]:
                    nodes.append((iz * ny + iy) * nx + ix)
                    weights.append(wz * wy * wx)
    return np.asarray(nodes, dtype=np.int64), np.asarray(weights, dtype=np.float64)


class Shot:
    """One shot's sampling operator R (CSR) and point-source injection list."""

    def __init__(self, shape, dx, src_xyz, rec_xyz):
        nd = len(shape)
        self.src_xyz = np.asarray(src_xyz, dtype=np.float64)
        n, w = point_weights(self.src_xyz, shape, dx)
        self.src_node = n
        self.src_w = w / dx ** nd              # discrete delta: weight / dx^d
        ptr = [0]
        nodes, ws = [], []
        for r in np.asarray(rec_xyz, dtype=np.float64).reshape(-1, 3):
            n, w = point_weights(r, shape, dx)
            nodes.append(n)
            ws.append(w)
            ptr.append(ptr[-1] + len(n))
        self.r_ptr = np.asarray(ptr, dtype=np.int64)
        self.r_node = np.concatenate(nodes) if nodes else np.zeros(0, np.int64)
        self.r_w = np.concatenate(ws) if ws else np.zeros(0)
        self.nr = len(ptr) - 1


class Oracle:
    """The discrete ESI operators on one velocity model (FP64)."""

    def __init__(self, v: np.ndarray, dx: float, dt: float, nt: int, nb: int,
                 R: float = 1e-3, vref: Optional[float] = None):
        self.v = np.ascontiguousarray(v, dtype=np.float64)
        self.shape = tuple(v.shape)
        self.ndim, self.nz, self.ny, self.nx = _dims(self.shape)
        self.N = int(np.prod(self.shape))
        self.dx, self.dt, self.nt, self.nb = float(dx), float(dt), int(nt), int(nb)
        self.vref = float(self.v.max() if vref is None else vref)
        self.c = (self.v ** 2 * dt * dt).ravel().copy()
        self.kappa = sponge_kappa(self.shape, nb, dx, dt, self.vref, R).ravel().copy()

    # ---------------------------------------------------------------- geometry
    def shot(self, src_xyz, rec_xyz) -> Shot:
        return Shot(self.shape, self.dx, src_xyz, rec_xyz)

    def annihilator(self, src_xyz, eps: Optional[float] = None) -> np.ndarray:
        """B(x) = ||x - x_s|| + eps (metres), eps = dx by default."""
        eps = self.dx if eps is None else eps
        grids = np.meshgrid(*[np.arange(n) * self.dx for n in self.shape], indexing="ij")
        if self.ndim == 2:
            pos = (src_xyz[2], src_xyz[0])
        else:
            pos = (src_xyz[2], src_xyz[1], src_xyz[0])
        r2 = sum((g - p) ** 2 for g, p in zip(grids, pos))
        return (np.sqrt(r2) + eps).ravel()

    # ---------------------------------------------------------------- modelling
    def forward(self, sh: Shot, wavelet: Optional[np.ndarray] = None,
                q_ext: Optional[np.ndarray] = None, want_s: bool = False,
                want_u: bool = False, freqs: Optional[Sequence[float]] = None) -> Dict:
        nt, N = self.nt, self.N
        traces = np.zeros((nt, sh.nr))
        s_hist = np.zeros((nt, N)) if want_s else None
        u_hist = np.zeros((nt + 1, N)) if want_u else None
        f = np.ascontiguousarray(freqs if freqs is not None else [], dtype=np.float64)
        nf = f.size
        dre = np.zeros((nf, N)) if nf else None
        dim = np.zeros((nf, N)) if nf else None
        if wavelet is not None:
            wav = np.ascontiguousarray(wavelet, dtype=np.float64)
            ns_ = sh.src_node.size
        else:
            wav, ns_ = None, 0
        q = None if q_ext is None else np.ascontiguousarray(q_ext, dtype=np.float64).reshape(nt, N)
        lib().orc_forward(self.ndim, self.nz, self.ny, self.nx, self.dx, self.dt, nt,
                          _dp(self.c), _dp(self.kappa), _dp(q), ns_, _lp(sh.src_node),
                          _dp(sh.src_w), _dp(wav), sh.nr, _lp(sh.r_ptr), _lp(sh.r_node),
                          _dp(sh.r_w), _dp(traces), _dp(s_hist), _dp(u_hist), nf,
                          _dp(f) if nf else None, _dp(dre), _dp(dim))
        out = {"traces": traces}
        if want_s:
            out["s"] = s_hist
        if want_u:
            out["u"] = u_hist
        if nf:
            out["dft"] = dre + 1j * dim
        return out

    def adjoint(self, sh: Shot, e: np.ndarray, want_out: bool = True, want_src: bool = False,
                s_hist: Optional[np.ndarray] = None) -> Dict:
        nt, N = self.nt, self.N
        e = np.ascontiguousarray(e, dtype=np.float64).reshape(nt, sh.nr)
        out = np.zeros((nt, N)) if want_out else None
        src_adj = np.zeros(nt) if want_src else None
        grad = np.zeros(N) if s_hist is not None else None
        lib().orc_adjoint(self.ndim, self.nz, self.ny, self.nx, self.dx, nt, _dp(self.c),
                          _dp(self.kappa), sh.nr, _lp(sh.r_ptr), _lp(sh.r_node), _dp(sh.r_w),
                          _dp(e), _dp(out), sh.src_node.size, _lp(sh.src_node),
                          _dp(sh.src_w), _dp(src_adj),
                          _dp(s_hist) if s_hist is not None else None, _dp(grad))
        res = {}
        if want_out:
            res["out"] = out
        if want_src:
            res["src"] = src_adj
        if grad is not None:
            res["grad_c"] = grad
        return res

    # ---------------------------------------------------------------- gradients
    def to_param(self, g_c: np.ndarray, param: str) -> np.ndarray:
        """Chain rule from c = v^2 dt^2 to v (g_v = 2 v dt^2 g_c) or to m = 1/v^2
        (g_m = -dt^2 v^4 g_c)."""
        v = self.v.ravel()
        if param == "c":
            return g_c
        if param == "v":
            return 2.0 * v * self.dt ** 2 * g_c
        if param == "m":
            return -(self.dt ** 2) * v ** 4 * g_c
        raise ValueError(param)

    def misfit_gradient(self, sh: Shot, dobs: np.ndarray, wavelet=None, q_ext=None,
                        param: str = "c") -> Tuple[float, np.ndarray]:
        """Adjoint-state gradient of J = 1/2 ||R u - d||^2 (Eq. "FWI_lambda", "gradient"):
        residual e = R u - d drives the adjoint; g_c = sum_n mu_{n+1} s_n."""
        fw = self.forward(sh, wavelet=wavelet, q_ext=q_ext, want_s=True)
        e = fw["traces"] - np.asarray(dobs, dtype=np.float64).reshape(self.nt, sh.nr)
        ad = self.adjoint(sh, e, want_out=False, s_hist=fw["s"])
        return 0.5 * float(np.sum(e * e)), self.to_param(ad["grad_c"], param)

    def saddle_gradient(self, sh: Shot, q: np.ndarray, beta: float, param: str = "c",
                        eps: Optional[float] = None) -> np.ndarray:
        """Algorithm 2's gradient: u = A^{-1} q, adjoint field taken from the extended
        source (lambda = beta B^H B q), correlated with the forward field.  With the
        discrete adjoint convention (S^T e)_n = c mu_{n+1}, the adjoint field of the
        residual at the normal-equation solution is mu_{n+1} = -beta B^2 q_n / c."""
        B = self.annihilator(sh.src_xyz, eps)
        fw = self.forward(sh, q_ext=q, want_s=True)
        qq = np.asarray(q, dtype=np.float64).reshape(self.nt, self.N)
        mu = -beta * (B * B)[None, :] * qq / self.c[None, :]
        return self.to_param(np.sum(mu * fw["s"], axis=0), param)

    # ---------------------------------------------------------------- ESI normal equation
    def S(self, sh: Shot, q: np.ndarray) -> np.ndarray:
        return self.forward(sh, q_ext=q)["traces"]

    def ST(self, sh: Shot, e: np.ndarray) -> np.ndarray:
        return self.adjoint(sh, e)["out"]

    def normal_matvec(self, sh: Shot, p: np.ndarray, beta: float,
                      eps: Optional[float] = None) -> np.ndarray:
        """A p = S^T S p + beta B^T B p (the CG section's matrix-vector product: forward
        modelling with p as the source, sampling, adjoint modelling, plus beta B^2 p)."""
        B = self.annihilator(sh.src_xyz, eps)
        p = np.asarray(p, dtype=np.float64).reshape(self.nt, self.N)
        return self.ST(sh, self.S(sh, p)) + beta * (B * B)[None, :] * p

    def cg(self, sh: Shot, d: np.ndarray, beta: float, tol: float, n_cg: int,
           eps: Optional[float] = None) -> Dict:
        """Algorithm 1 applied to (S^T S + beta B^T B) q = S^T d, verbatim: x0 = 0,
        r0 = b, p0 = r0; exit when ||r_{k+1}|| < tol ||r_0|| or k = N_CG - 1."""
        b = self.ST(sh, d)
        x = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        rr = float(np.sum(r * r))
        r0 = math.sqrt(rr)
        hist, alphas, betas = [], [], []
        k = -1   # b = 0: x_0 = 0 is exact and no iteration runs
        for k in range(n_cg if r0 > 0 else 0):
            Ap = self.normal_matvec(sh, p, beta, eps)
            alpha = rr / float(np.sum(p * Ap))
            x = x + alpha * p
            r = r - alpha * Ap
            rr_new = float(np.sum(r * r))
            hist.append(math.sqrt(rr_new) / r0 if r0 > 0 else 0.0)
            alphas.append(alpha)
            if math.sqrt(rr_new) < tol * r0 or k == n_cg - 1:
                break
            bk = rr_new / rr
            betas.append(bk)
            p = r + bk * p
            rr = rr_new
        return {"x": x, "rel_res": np.asarray(hist), "alpha": np.asarray(alphas),
                "beta": np.asarray(betas), "iters": k + 1, "b": b}

    def pcg(self, sh: Shot, d: np.ndarray, beta: float, tol: float, n_cg: int,
            minv: np.ndarray, eps: Optional[float] = None) -> Dict:
        """Algorithm 1 with a fixed SPD preconditioner M^{-1} = diag(minv) (per cell, the same
        at every time step): z = M^{-1} r, alpha = <r,z>/<p,Ap>, beta_k = <r',z'>/<r,z>,
        p = z + beta_k p; stopping test on ||r|| as in Algorithm 1."""
        b = self.ST(sh, d)
        x = np.zeros_like(b)
        r = b.copy()
        z = r * minv[None, :]
        p = z.copy()
        rz = float(np.sum(r * z))
        r0 = math.sqrt(float(np.sum(r * r)))
        hist = []
        k = -1   # b = 0: x_0 = 0 is exact and no iteration runs
        for k in range(n_cg if r0 > 0 else 0):
            Ap = self.normal_matvec(sh, p, beta, eps)
            alpha = rz / float(np.sum(p * Ap))
            x = x + alpha * p
            r = r - alpha * Ap
            rn = math.sqrt(float(np.sum(r * r)))
            hist.append(rn / r0)
            if rn < tol * r0 or k == n_cg - 1:
                break
            z = r * minv[None, :]
            rz_new = float(np.sum(r * z))
            p = z + (rz_new / rz) * p
            rz = rz_new
        return {"x": x, "rel_res": np.asarray(hist), "iters": k + 1}

    # ---------------------------------------------------------------- WRI (B = I)
    # The CG section notes that the same CG serves WRI once B is the identity and the
    # right-hand side is WRI's own: Eq. "normalwri", (S^H S + beta I) q = S^H (d - S f), with
    # u = A^{-1}(f + q) (Eq. "newq") and the gradient beta <A u - f, dA/dm u> = <lambda,
    # dA/dm u>, lambda = beta q (Eq. "newadj2", "gradient2").
    def wri_rhs(self, sh: Shot, d: np.ndarray, wavelet: np.ndarray) -> np.ndarray:
        """b = S^T (d - S f): the data residual of the point sources, back-propagated."""
        Sf = self.forward(sh, wavelet=wavelet)["traces"]
        return self.ST(sh, np.asarray(d, dtype=np.float64).reshape(self.nt, sh.nr) - Sf)

    def wri_matvec(self, sh: Shot, p: np.ndarray, beta: float) -> np.ndarray:
        """(S^T S + beta I) p."""
        p = np.asarray(p, dtype=np.float64).reshape(self.nt, self.N)
        return self.ST(sh, self.S(sh, p)) + beta * p

    def wri_cg(self, sh: Shot, d: np.ndarray, wavelet: np.ndarray, beta: float, tol: float,
               n_cg: int) -> Dict:
        """Algorithm 1 on the WRI system, verbatim as in cg()."""
        b = self.wri_rhs(sh, d, wavelet)
        x = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        rr = float(np.sum(r * r))
        r0 = math.sqrt(rr)
        hist = []
        k = -1   # b = 0: x_0 = 0 is exact and no iteration runs
        for k in range(n_cg if r0 > 0 else 0):
            Ap = self.wri_matvec(sh, p, beta)
            alpha = rr / float(np.sum(p * Ap))
            x = x + alpha * p
            r = r - alpha * Ap
            rr_new = float(np.sum(r * r))
            hist.append(math.sqrt(rr_new) / r0 if r0 > 0 else 0.0)
            if math.sqrt(rr_new) < tol * r0 or k == n_cg - 1:
                break
            p = r + (rr_new / rr) * p
            rr = rr_new
        return {"x": x, "rel_res": np.asarray(hist), "iters": k + 1, "b": b}

    def wri_objective(self, sh: Shot, q: np.ndarray, d: np.ndarray, wavelet: np.ndarray,
                      beta: float) -> float:
        """J_WRI = 1/2 ||R u - d||^2 + beta/2 ||q||^2 with u = A^{-1}(f + q) (Eq. "wrimisfit")."""
        tr = self.forward(sh, wavelet=wavelet, q_ext=q)["traces"]
        e = tr - np.asarray(d, dtype=np.float64).reshape(self.nt, sh.nr)
        return 0.5 * float(np.sum(e * e)) + 0.5 * beta * float(np.sum(np.asarray(q) ** 2))

    def wri_gradient(self, sh: Shot, q: np.ndarray, wavelet: np.ndarray, beta: float,
                     param: str = "c") -> np.ndarray:
        """The WRI saddle-point gradient: u = A^{-1}(f + q), lambda = beta q.  With the discrete
        adjoint convention (S^T e)_n = c mu_{n+1}, the adjoint field of the residual at the
        solution is mu_{n+1} = -beta q_n / c; g_c = sum_n mu_{n+1} (Lap u_n + f_n + q_n)."""
        fw = self.forward(sh, wavelet=wavelet, q_ext=q, want_s=True)
        qq = np.asarray(q, dtype=np.float64).reshape(self.nt, self.N)
        mu = -beta * qq / self.c[None, :]
        return self.to_param(np.sum(mu * fw["s"], axis=0), param)

    # ---------------------------------------------------------------- data-space CG
    # The section "Switching from the wavefield to data space": with w := R u the synthetic
    # data, Eq. "wd" reads (I + S (beta B^H B)^{-1} S^H) w = S (beta B^H B)^{-1} S^H d, an
    # SPD system in data space (nr x nt unknowns per shot) solved by CG; then Eq. "q" gives
    # q = (beta B^H B)^{-1} S^H (d - w).
    def ds_K(self, sh: Shot, e: np.ndarray, beta: float, eps: Optional[float] = None) -> np.ndarray:
        """K e = S (beta B^2)^{-1} S^T e: adjoint modelling of e, scaling, forward modelling."""
        B = self.annihilator(sh.src_xyz, eps)
        lam = self.ST(sh, np.asarray(e, dtype=np.float64).reshape(self.nt, sh.nr))
        return self.S(sh, lam / (beta * B * B)[None, :])

    def ds_cg(self, sh: Shot, d: np.ndarray, beta: float, tol: float, n_cg: int,
              eps: Optional[float] = None) -> Dict:
        """Algorithm 1 on (I + K) w = K d, then q = (beta B^2)^{-1} S^T (d - w)."""
        d = np.asarray(d, dtype=np.float64).reshape(self.nt, sh.nr)
        b = self.ds_K(sh, d, beta, eps)
        x = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        rr = float(np.sum(r * r))
        r0 = math.sqrt(rr)
        hist = []
        k = -1   # b = 0: x_0 = 0 is exact and no iteration runs
        for k in range(n_cg if r0 > 0 else 0):
            Ap = p + self.ds_K(sh, p, beta, eps)
            alpha = rr / float(np.sum(p * Ap))
            x = x + alpha * p
            r = r - alpha * Ap
            rr_new = float(np.sum(r * r))
            hist.append(math.sqrt(rr_new) / r0 if r0 > 0 else 0.0)
            if math.sqrt(rr_new) < tol * r0 or k == n_cg - 1:
                break
            p = r + (rr_new / rr) * p
            rr = rr_new
        B = self.annihilator(sh.src_xyz, eps)
        q = self.ST(sh, d - x) / (beta * B * B)[None, :]
        return {"w": x, "q": q, "rel_res": np.asarray(hist), "iters": k + 1, "b": b}

    # ---------------------------------------------------------- frequency-domain ESI
    def dtft_matrix(self, freqs: Sequence[float]) -> np.ndarray:
        """F of Eq. "dtft" over the source's time index: F[m, n] = exp(+j 2 pi f_m n dt),
        shape [nf, nt].  The inverse of Eq. "idtft" is F^H / nt."""
        f = np.asarray(freqs, dtype=np.float64)
        n = np.arange(self.nt, dtype=np.float64)
        return np.exp(2j * np.pi * np.outer(f, n) * self.dt)

    def fd_matvec(self, sh: Shot, qbar: np.ndarray, beta: float, freqs: Sequence[float],
                  eps: Optional[float] = None) -> np.ndarray:
        """M qbar = F (S^T S + beta B^T B) F^H qbar / nt (left side of Eq. "normaldtft"): the
        inverse DTFT to a complex time series, the real normal operator on its real and its
        imaginary part, the DTFT back to the frequencies."""
        F = self.dtft_matrix(freqs)
        qb = np.asarray(qbar, dtype=np.complex128).reshape(len(freqs), self.N)
        q = F.conj().T @ qb / self.nt
        Aq = self.normal_matvec(sh, q.real, beta, eps) + 1j * self.normal_matvec(sh, q.imag, beta, eps)
        return F @ Aq

    def fd_cg(self, sh: Shot, d: np.ndarray, beta: float, freqs: Sequence[float], tol: float,
              n_cg: int, eps: Optional[float] = None) -> Dict:
        """Algorithm 1 on Eq. "normaldtft", right-hand side F S^T d (the observed data taken
        as the time series d = F^H dbar / nt), inner products Re <x, y> (M is Hermitian
        positive definite).  Also returns q = F^H qbar / nt."""
        F = self.dtft_matrix(freqs)
        b = F @ self.ST(sh, np.asarray(d, dtype=np.float64).reshape(self.nt, sh.nr))
        x = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        rr = float(np.vdot(r, r).real)
        r0 = math.sqrt(rr)
        hist = []
        k = -1   # b = 0: x_0 = 0 is exact and no iteration runs
        for k in range(n_cg if r0 > 0 else 0):
            Ap = self.fd_matvec(sh, p, beta, freqs, eps)
            alpha = rr / float(np.vdot(p, Ap).real)
            x = x + alpha * p
            r = r - alpha * Ap
            rr_new = float(np.vdot(r, r).real)
            hist.append(math.sqrt(rr_new) / r0 if r0 > 0 else 0.0)
            if math.sqrt(rr_new) < tol * r0 or k == n_cg - 1:
                break
            p = r + (rr_new / rr) * p
            rr = rr_new
        return {"qbar": x, "q": F.conj().T @ x / self.nt, "rel_res": np.asarray(hist),
                "iters": k + 1, "b": b}

    def fd_pcg(self, sh: Shot, d: np.ndarray, beta: float, freqs: Sequence[float], tol: float,
               n_cg: int, minv: np.ndarray, eps: Optional[float] = None) -> Dict:
        """fd_cg with a fixed preconditioner z = minv r per cell, the same at every frequency
        (minv = 1 / (beta B^2): on the DFT grid F F^H / nt = I, so this is the inverse of the
        penalty term of Eq. "normaldtft"); beta_k = Re<r', z'> / Re<r, z>, stopping on ||r||."""
        F = self.dtft_matrix(freqs)
        b = F @ self.ST(sh, np.asarray(d, dtype=np.float64).reshape(self.nt, sh.nr))
        x = np.zeros_like(b)
        r = b.copy()
        z = r * minv[None, :]
        p = z.copy()
        rz = float(np.vdot(r, z).real)
        r0 = math.sqrt(float(np.vdot(r, r).real))
        hist = []
        k = -1   # b = 0: x_0 = 0 is exact and no iteration runs
        for k in range(n_cg if r0 > 0 else 0):
            Ap = self.fd_matvec(sh, p, beta, freqs, eps)
            alpha = rz / float(np.vdot(p, Ap).real)
            x = x + alpha * p
            r = r - alpha * Ap
            rn = math.sqrt(float(np.vdot(r, r).real))
            hist.append(rn / r0)
            if rn < tol * r0 or k == n_cg - 1:
                break
            z = r * minv[None, :]
            rz_new = float(np.vdot(r, z).real)
            p = z + (rz_new / rz) * p
            rz = rz_new
        return {"qbar": x, "q": F.conj().T @ x / self.nt, "rel_res": np.asarray(hist),
                "iters": k + 1, "b": b}

    def assemble_S(self, sh: Shot) -> np.ndarray:
        """Dense data operator S (columns S e_j over space-time; tiny sizes only)."""
        n = self.nt * self.N
        M = np.empty((self.nt * sh.nr, n))
        for j in range(n):
            ej = np.zeros(n)
            ej[j] = 1.0
            M[:, j] = self.S(sh, ej.reshape(self.nt, self.N)).ravel()
        return M

    def assemble_normal(self, sh: Shot, beta: float, eps: Optional[float] = None) -> np.ndarray:
        """Dense normal matrix, column j = A e_j (tiny sizes only)."""
        n = self.nt * self.N
        A = np.empty((n, n))
        for j in range(n):
            ej = np.zeros(n)
            ej[j] = 1.0
            A[:, j] = self.normal_matvec(sh, ej, beta, eps).ravel()
        return A


# -------------------------------------------------------------------- snapshot codecs
CODEC_RANGE = 32768.0   # max |u| of a snapshot maps to this code magnitude


def _bf16_rne(x32: np.ndarray) -> np.ndarray:
    """Round float32 to the nearest bfloat16 (ties to even); returns the uint16 codes."""
    b = x32.astype(np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = (b + 0x7FFF + lsb) >> 16
    nan = np.isnan(x32)
    out = r.astype(np.uint16)
    out[nan] = 0x7FC0
    return out


def bf16_to_f32(codes: np.ndarray) -> np.ndarray:
    return (codes.astype(np.uint32) << 16).view(np.float32)


def encode_snapshot(u32: np.ndarray, kind: str) -> Tuple[np.ndarray, np.float32]:
    """Per-snapshot scaled codec, decisions taken in FP32: s = max|u|,
    code = round16(fl32(u * fl32(CODEC_RANGE / s))).  Returns (codes, decode scale
    fl32(s / CODEC_RANGE))."""
    u32 = np.asarray(u32, dtype=np.float32)
    s = np.float32(np.max(np.abs(u32))) if u32.size else np.float32(0)
    if s == 0:
        inv = np.float32(0)
    else:
        inv = np.float32(np.float32(CODEC_RANGE) / s)
    y = (u32 * inv).astype(np.float32)
    if kind == "f16":
        codes = y.astype(np.float16).view(np.uint16)
    elif kind == "bf16":
        codes = _bf16_rne(y)
    else:
        raise ValueError(kind)
    dec = np.float32(s / np.float32(CODEC_RANGE))
    return codes, dec


def decode_snapshot(codes: np.ndarray, dec: np.float32, kind: str) -> np.ndarray:
    if kind == "f16":
        h = codes.view(np.float16).astype(np.float32)
    else:
        h = bf16_to_f32(codes)
    return (h * np.float32(dec)).astype(np.float32)


def _code16(x: np.ndarray, kind: str) -> np.ndarray:
    """x taken to FP32, then to a 16-bit format and back (FP64 result): BF16 unscaled,
    FP16 through the per-part scale of encode_snapshot."""
    if kind == "bf16":
        return bf16_to_f32(_bf16_rne(np.asarray(x, dtype=np.float32))).astype(np.float64)
    if kind == "f16":
        codes, dec = encode_snapshot(x, "f16")
        return decode_snapshot(codes, dec, "f16").astype(np.float64)
    raise ValueError(kind)


def upsample_even(c: np.ndarray, shape: Sequence[int]) -> np.ndarray:
    """Multilinear prolongation from the cells whose indices are all even to the whole grid:
    along each axis an even index 2k takes c[k], an odd index the mean of its even
    neighbours, and an odd last index (even axis length) repeats its left neighbour."""
    u = np.asarray(c, dtype=np.float64)
    for ax, n in enumerate(shape):
        u = np.moveaxis(u, ax, 0)
        out = np.empty((n,) + u.shape[1:])
        out[0::2] = u
        right = np.concatenate([u[1:], u[-1:]])
        out[1::2] = (0.5 * (u + right))[: n // 2]
        u = np.moveaxis(out, 0, ax)
    return u


def checkpoint_code(x: np.ndarray, shape: Sequence[int], kind: str) -> np.ndarray:
    """Round trip of one snapshot through the two-level 16-bit checkpoint code.

    The paper replaces the stored wavefield history by recomputation from checkpoints
    (storage section, time-reversal discussion); it fixes no checkpoint format, so this is
    the library's: the coarse part is x at the all-even cells, coded to 16 bits; the fine
    part is x - U(decoded coarse) at every cell, coded to 16 bits; the decoded snapshot is
    U(decoded coarse) + decoded fine, U the prolongation of upsample_even.  Rounding then
    errs by the 16-bit precision of the interpolation residual, not of x.  kind "f32" keeps
    the snapshot as it is (an uncompressed copy in the working precision)."""
    x = np.asarray(x, dtype=np.float64).reshape(tuple(shape))
    if kind == "f32":
        return x.ravel().copy()
    coarse = _code16(x[tuple(slice(0, None, 2) for _ in shape)], kind)
    up = upsample_even(coarse, shape)
    return (up + _code16(x - up, kind)).ravel()


def _oracle_checkpointed_gradient(self: "Oracle", sh: Shot, dobs: np.ndarray, wavelet,
                                  every: int, kind: str, param: str = "c"
                                  ) -> Tuple[float, np.ndarray]:
    """misfit_gradient with the forward history recomputed from checkpoints (storage
    section: recompute instead of storing every step).  Every `every` steps n0 the pair
    (u_n0, u_n0-1) is kept: u_n0 and the difference u_n0 - u_n0-1 each through
    checkpoint_code (kind "f32": both states as they are); each segment restarts step n0
    from the decoded pair, u_n0-1 = decoded u_n0 - decoded difference, and its steps'
    s_n = Lap u_n + q_n (the same update as ``forward``) enter the correlation.  The
    residual and J come from the uncompressed forward run."""
    nt, N = self.nt, self.N
    fw = self.forward(sh, wavelet=wavelet, want_u=True)
    e = fw["traces"] - np.asarray(dobs, dtype=np.float64).reshape(nt, sh.nr)
    U = fw["u"]                      # U[n] = u_n, U[0] = u_0 = 0; u_{-1} = 0
    wav = np.asarray(wavelet, dtype=np.float64)
    s_hist = np.empty((nt, N))
    for n0 in range(0, nt, int(every)):
        u_prev_true = U[n0 - 1] if n0 > 0 else np.zeros(N)
        cur = checkpoint_code(U[n0], self.shape, kind)
        if kind == "f32":
            prev = checkpoint_code(u_prev_true, self.shape, kind)
        else:
            prev = cur - checkpoint_code(U[n0] - u_prev_true, self.shape, kind)
        for n in range(n0, min(nt, n0 + int(every))):
            q = np.zeros(N)
            np.add.at(q, sh.src_node, sh.src_w * wav[n])
            s = laplacian(cur.reshape(self.shape), self.dx).ravel() + q
            s_hist[n] = s
            nxt = (2.0 * cur - (1.0 - self.kappa) * prev + self.c * s) / (1.0 + self.kappa)
            prev, cur = cur, nxt
    ad = self.adjoint(sh, e, want_out=False, s_hist=s_hist)
    return 0.5 * float(np.sum(e * e)), self.to_param(ad["grad_c"], param)


Oracle.checkpointed_gradient = _oracle_checkpointed_gradient


def rel_l2(a, b) -> float:
    """||a - b|| / ||b|| (real or complex)."""
    a = np.asarray(a)
    b = np.asarray(b)
    a = a.astype(np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = b.astype(a.dtype)
    den = float(np.linalg.norm(b.ravel()))
    return float(np.linalg.norm((a - b).ravel())) / (den if den > 0 else 1.0)
