"""Thin ctypes binding of libesi (the C ABI in include/esi.h).

Argument marshalling only: PyTorch provides device memory and the stream; every
arithmetic step runs in the library's CUDA kernels.  There is no CPU fallback: loading
fails loudly when the library is missing or no CUDA device is available.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libesi.so")

ESI_OK, ESI_ERR_ARG, ESI_ERR_CFL, ESI_ERR_OOM, ESI_ERR_CUDA = 0, 1, 2, 3, 4
ESI_ERR_BREAKDOWN, ESI_ERR_TIMEOUT, ESI_ERR_NOT_CONVERGED, ESI_ERR_UNSUPPORTED = 5, 6, 7, 8
ESI_F32, ESI_F64 = 0, 1
GRAD_ADJOINT_STATE, GRAD_SADDLE_POINT, GRAD_WRI_SADDLE = 0, 1, 2
GRAD_MODES = {"adjoint": GRAD_ADJOINT_STATE, "saddle": GRAD_SADDLE_POINT, "wri": GRAD_WRI_SADDLE}
PARAMS = {"c": 0, "v": 1, "m": 2}
CKPT = {"f32": 0, "f16": 1, "bf16": 2}
DFT_C64, DFT_C32_HALF = 0, 1
PC = {"none": 0, "diag": 1, "learned": 2}

# every symbol the header declares (checked by the CPU test-suite)
EXPORTS = ["esi_create", "esi_destroy", "esi_set_stream", "esi_set_velocity", "esi_forward",
           "esi_adjoint", "esi_gradient", "esi_dft_extract", "esi_cg_solve", "esi_pc_load",
           "esi_status_string", "esi_last_error", "esi_launch_count", "esi_set_profiling",
           "esi_get_profile", "esi_forward_noalloc", "esi_normal_apply", "esi_pc_param_count",
           "esi_pc_fallbacks", "esi_pc_pack", "esi_pc_create", "esi_pc_destroy",
           "esi_pc_last_error", "esi_pc_set_params", "esi_pc_get_params", "esi_pc_apply",
           "esi_pc_grad", "esi_pc_vjp", "esi_pc_train_step", "esi_wri_solve", "esi_dscg_solve",
           "esi_fdcg_solve", "esi_invert", "esi_set_shot_groups"]


class EsiGrid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nz", ctypes.c_int), ("ny", ctypes.c_int),
                ("nx", ctypes.c_int), ("dx", ctypes.c_double), ("nb", ctypes.c_int),
                ("sponge_R", ctypes.c_double), ("sponge_vref", ctypes.c_double),
                ("dtype", ctypes.c_int)]


class EsiGeometry(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int), ("src_xyz", ctypes.POINTER(ctypes.c_double)),
                ("rec_offset", ctypes.POINTER(ctypes.c_longlong)),
                ("rec_xyz", ctypes.POINTER(ctypes.c_double))]


class EsiGradOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("param", ctypes.c_int), ("ckpt_every", ctypes.c_int),
                ("ckpt_kind", ctypes.c_int), ("beta", ctypes.c_double), ("eps", ctypes.c_double)]


class EsiCgReport(ctypes.Structure):
    _fields_ = [("iters_max", ctypes.c_int), ("converged", ctypes.c_int),
                ("max_hist", ctypes.c_int), ("iters", ctypes.POINTER(ctypes.c_int)),
                ("rel_res", ctypes.POINTER(ctypes.c_double)), ("ms_matvec", ctypes.c_double),
                ("ms_vector", ctypes.c_double), ("ms_precond", ctypes.c_double),
                ("ms_total", ctypes.c_double)]


REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                             ctypes.c_void_p, ctypes.c_longlong)


class EsiInvertOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("n_outer", ctypes.c_int), ("n_cg", ctypes.c_int),
                ("cg_tol", ctypes.c_double), ("precond", ctypes.c_int),
                ("beta0", ctypes.c_double), ("growth", ctypes.c_double),
                ("memory", ctypes.c_int), ("c1", ctypes.c_double),
                ("step_frac", ctypes.c_double), ("max_ls", ctypes.c_int),
                ("vmin", ctypes.c_double), ("vmax", ctypes.c_double), ("eps", ctypes.c_double),
                ("reduce", REDUCE_FN), ("reduce_user", ctypes.c_void_p)]


class EsiInvertReport(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("J_start", ctypes.POINTER(ctypes.c_double)),
                ("J_end", ctypes.POINTER(ctypes.c_double)),
                ("alpha", ctypes.POINTER(ctypes.c_double)),
                ("beta", ctypes.POINTER(ctypes.c_double)),
                ("trials", ctypes.POINTER(ctypes.c_int)), ("iters_done", ctypes.c_int),
                ("evaluations", ctypes.c_int), ("cg_iters_total", ctypes.c_int),
                ("stop_reason", ctypes.c_int), ("ms_total", ctypes.c_double)]


STOP_REASONS = {0: "ok", 1: "line search failed", 2: "zero gradient"}


class EsiKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_longlong),
                ("cells", ctypes.c_longlong), ("bytes_per_cell", ctypes.c_double),
                ("ms", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return LIB_PATH


def load_library(require_gpu: bool = True) -> ctypes.CDLL:
    """Load libesi.so (built by paper_2211_06300_gb300.build).  Raises when missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libesi.so not built ({LIB_PATH}); run paper_2211_06300_gb300.build")
    if require_gpu:
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libesi needs a CUDA device; none is available")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.esi_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(EsiGrid),
                             ctypes.POINTER(EsiGeometry), vp, d, i, vp]
    L.esi_destroy.argtypes = [vp]
    L.esi_destroy.restype = None
    L.esi_set_stream.argtypes = [vp, vp]
    L.esi_set_velocity.argtypes = [vp, vp]
    L.esi_set_shot_groups.argtypes = [vp, i, vp]
    L.esi_forward.argtypes = [vp, vp, vp, vp]
    L.esi_forward_noalloc.argtypes = [vp, vp, vp, vp]
    L.esi_adjoint.argtypes = [vp, vp, vp, vp]
    L.esi_gradient.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(EsiGradOpts), vp,
                               ctypes.POINTER(d)]
    L.esi_dft_extract.argtypes = [vp, vp, vp, ctypes.POINTER(d), i, vp, i,
                                  ctypes.POINTER(ctypes.c_float), vp]
    L.esi_cg_solve.argtypes = [vp, d, d, i, vp, vp, i, d, ctypes.POINTER(EsiCgReport)]
    L.esi_wri_solve.argtypes = [vp, d, d, i, vp, vp, vp, ctypes.POINTER(EsiCgReport)]
    L.esi_dscg_solve.argtypes = [vp, d, d, i, vp, vp, vp, d, ctypes.POINTER(EsiCgReport)]
    L.esi_fdcg_solve.argtypes = [vp, d, d, i, vp, ctypes.POINTER(d), i, i, vp, d,
                                 ctypes.POINTER(EsiCgReport)]
    L.esi_pc_load.argtypes = [vp, vp, ctypes.c_size_t]
    L.esi_invert.argtypes = [vp, ctypes.POINTER(EsiInvertOpts), vp, vp, vp, vp,
                             ctypes.POINTER(EsiInvertReport)]
    L.esi_normal_apply.argtypes = [vp, d, d, vp, vp]
    L.esi_pc_param_count.argtypes = []
    L.esi_pc_param_count.restype = ctypes.c_size_t
    L.esi_pc_fallbacks.argtypes = [vp]
    L.esi_pc_fallbacks.restype = ctypes.c_longlong
    L.esi_pc_pack.argtypes = [vp, vp, d, d, i, i, vp]
    L.esi_pc_create.argtypes = [ctypes.POINTER(vp), i, i, i, vp]
    L.esi_pc_destroy.argtypes = [vp]
    L.esi_pc_destroy.restype = None
    L.esi_pc_last_error.argtypes = [vp]
    L.esi_pc_last_error.restype = ctypes.c_char_p
    L.esi_pc_set_params.argtypes = [vp, vp]
    L.esi_pc_get_params.argtypes = [vp, vp]
    L.esi_pc_apply.argtypes = [vp, vp, i, vp]
    L.esi_pc_grad.argtypes = [vp, vp, vp, i, vp, ctypes.POINTER(d)]
    L.esi_pc_vjp.argtypes = [vp, vp, vp, i, vp]
    L.esi_pc_train_step.argtypes = [vp, vp, vp, i, d, ctypes.POINTER(d)]
    L.esi_status_string.argtypes = [i]
    L.esi_status_string.restype = ctypes.c_char_p
    L.esi_last_error.argtypes = [vp]
    L.esi_last_error.restype = ctypes.c_char_p
    L.esi_launch_count.argtypes = [vp]
    L.esi_launch_count.restype = ctypes.c_longlong
    L.esi_set_profiling.argtypes = [vp, i]
    L.esi_set_profiling.restype = i
    L.esi_get_profile.argtypes = [vp, ctypes.POINTER(EsiKernelStat), i]
    L.esi_get_profile.restype = i
    for name in ("esi_create", "esi_set_stream", "esi_set_velocity", "esi_forward",
                 "esi_forward_noalloc", "esi_normal_apply", "esi_pc_pack", "esi_pc_create",
                 "esi_pc_set_params", "esi_pc_get_params", "esi_pc_apply", "esi_pc_grad",
                 "esi_pc_vjp", "esi_pc_train_step",
                 "esi_adjoint", "esi_gradient", "esi_dft_extract", "esi_cg_solve",
                 "esi_pc_load", "esi_wri_solve", "esi_dscg_solve", "esi_fdcg_solve", "esi_invert",
                 "esi_set_shot_groups"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class EsiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libesi takes CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("libesi takes contiguous tensors")
    return t.data_ptr()


class Context:
    """An ESI operator on one velocity model and acquisition (``esi_create``).

    ``v``: CUDA tensor (nz, nx) or (nz, ny, nx), float32 or float64 (the precision of
    every field of this context).  ``geom``: a ``synth.Geometry`` (positions in metres).
    """

    def __init__(self, v, dx: float, dt: float, nt: int, nb: int, geom, sponge_R: float = 1e-3,
                 vref: float = 0.0, stream=None):
        import torch
        self.L = load_library()
        self.torch = torch
        if v.dim() not in (2, 3):
            raise ValueError("velocity must be 2D or 3D")
        self.dtype = v.dtype
        if v.dtype not in (torch.float32, torch.float64):
            raise ValueError("velocity must be float32 or float64")
        self.device = v.device
        self.shape = tuple(v.shape)
        self.ndim = v.dim()
        self.N = int(np.prod(self.shape))
        self.nt, self.dx, self.dt, self.nb = int(nt), float(dx), float(dt), int(nb)
        self.geom = geom
        self.ns = geom.ns
        self.total_rec = int(geom.rec_offset[-1])
        g = EsiGrid()
        g.ndim = self.ndim
        if self.ndim == 2:
            g.nz, g.ny, g.nx = self.shape[0], 1, self.shape[1]
        else:
            g.nz, g.ny, g.nx = self.shape
        g.dx, g.nb, g.sponge_R, g.sponge_vref = self.dx, self.nb, sponge_R, vref
        g.dtype = ESI_F64 if v.dtype == torch.float64 else ESI_F32
        self._src = np.ascontiguousarray(geom.src_xyz, dtype=np.float64)
        self._off = np.ascontiguousarray(geom.rec_offset, dtype=np.int64)
        self._rec = np.ascontiguousarray(geom.rec_xyz, dtype=np.float64).reshape(-1, 3)
        if self._rec.size == 0:
            self._rec = np.zeros((1, 3))
        gm = EsiGeometry()
        gm.ns = self.ns
        gm.src_xyz = self._src.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        gm.rec_offset = self._off.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
        gm.rec_xyz = self._rec.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self._v = v.contiguous()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.L.esi_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(gm),
                                   _ptr(self._v), self.dt, self.nt,
                                   ctypes.c_void_p(stream.cuda_stream))
        if st != ESI_OK:
            raise EsiError(st, self.L.esi_last_error(None).decode() or
                           self.L.esi_status_string(st).decode())
        self.h = h

    # ---------------------------------------------------------------- helpers
    def _check(self, st: int, allow=(ESI_OK,)):
        if st not in allow:
            raise EsiError(st, self.L.esi_last_error(self.h).decode() or
                           self.L.esi_status_string(st).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.L.esi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty_traces(self):
        return self.torch.empty(self.nt * self.total_rec, dtype=self.dtype, device=self.device)

    def empty_field(self, ns: Optional[int] = None):
        ns = self.ns if ns is None else ns
        return self.torch.empty((ns, self.nt) + self.shape, dtype=self.dtype, device=self.device)

    def traces_of(self, traces, s: int):
        """View of shot s in a CSR seismogram buffer as (nt, nrec)."""
        o0, o1 = int(self.geom.rec_offset[s]), int(self.geom.rec_offset[s + 1])
        return traces[self.nt * o0:self.nt * o1].view(self.nt, o1 - o0)

    @property
    def launches(self) -> int:
        return int(self.L.esi_launch_count(self.h))

    def set_profiling(self, on: bool = True):
        self._check(self.L.esi_set_profiling(self.h, 1 if on else 0))

    def profile(self):
        """Per kernel variant: launches, cells, algorithmic bytes per cell, device ms."""
        n = self.L.esi_get_profile(self.h, None, 0)
        arr = (EsiKernelStat * max(n, 1))()
        n = self.L.esi_get_profile(self.h, arr, n)
        return [{"name": arr[i].name.decode(), "launches": int(arr[i].launches),
                 "cells": int(arr[i].cells), "bytes_per_cell": float(arr[i].bytes_per_cell),
                 "ms": float(arr[i].ms)} for i in range(n)]

    # ---------------------------------------------------------------- operators
    def set_velocity(self, v):
        self._v = v.contiguous()
        self._check(self.L.esi_set_velocity(self.h, _ptr(self._v)))

    def set_shot_groups(self, groups: int):
        """esi_set_shot_groups: run the shots as `groups` concurrent groups (1 removes them)."""
        with self.torch.cuda.device(self.device):
            self._check(self.L.esi_set_shot_groups(self.h, int(groups), _ptr(self._v)))

    def forward(self, wavelet=None, ext=None, out=None):
        out = self.empty_traces() if out is None else out
        self._check(self.L.esi_forward(self.h, _ptr(wavelet), _ptr(ext), _ptr(out)))
        return out

    def normal_apply(self, p, lam: float, eps: float = 0.0, out=None):
        """A p = S^T S p + lam B^2 p (esi_normal_apply)."""
        out = self.empty_field() if out is None else out
        self._check(self.L.esi_normal_apply(self.h, float(lam), float(eps), _ptr(p), _ptr(out)))
        return out

    def pc_images_shape(self):
        ng = (self.nt + 15) // 16
        return (self.ns * ng, (self.shape[0] + 1) // 2, (self.shape[-1] + 1) // 2, 16)

    def pc_pack(self, field, lam: float = 0.0, scale: bool = False, eps: float = 0.0, out=None,
                pitched: bool = False):
        """Pack a [ns][nt][...] field into the network's BF16 images (esi_pc_pack); pitched:
        the field's rows are px = 32 ceil(nx / 32) wide, pad columns zero."""
        out = self.torch.empty(self.pc_images_shape(), dtype=self.torch.bfloat16,
                               device=self.device) if out is None else out
        self._check(self.L.esi_pc_pack(self.h, _ptr(field), float(lam), float(eps),
                                       1 if scale else 0, 1 if pitched else 0, _ptr(out)))
        return out

    def pc_load(self, params):
        """Load trained preconditioner parameters (FP32 CUDA tensor, esi_pc_param_count())."""
        params = params.contiguous()
        self._check(self.L.esi_pc_load(self.h, _ptr(params), params.numel() * 4))

    @property
    def pc_fallbacks(self) -> int:
        return int(self.L.esi_pc_fallbacks(self.h))

    def forward_noalloc(self, out, wavelet=None, ext=None):
        """esi_forward_noalloc: forward modelling whose wave states live in the library's
        fixed device array (no device allocation); ``out`` must be preallocated."""
        self._check(self.L.esi_forward_noalloc(self.h, _ptr(wavelet), _ptr(ext), _ptr(out)))
        return out

    def adjoint(self, traces, want_field: bool = True, want_wavelet: bool = False, out=None):
        f = (self.empty_field() if out is None else out) if want_field else None
        w = self.torch.empty((self.ns, self.nt), dtype=self.dtype, device=self.device) \
            if want_wavelet else None
        self._check(self.L.esi_adjoint(self.h, _ptr(traces), _ptr(f), _ptr(w)))
        return f, w

    def gradient(self, wavelet=None, ext=None, dobs=None, adj_src=None, mode: str = "adjoint",
                 param: str = "v", ckpt_every: int = 20, ckpt: str = "f32", beta: float = 0.0,
                 eps: float = 0.0, out=None):
        o = EsiGradOpts()
        o.mode = GRAD_MODES[mode]
        o.param = PARAMS[param]
        o.ckpt_every = int(ckpt_every)
        o.ckpt_kind = CKPT[ckpt]
        o.beta = float(beta)
        o.eps = float(eps)
        g = self.torch.empty(self.shape, dtype=self.dtype, device=self.device) if out is None else out
        mis = ctypes.c_double(0.0)
        self._check(self.L.esi_gradient(self.h, _ptr(wavelet), _ptr(ext), _ptr(dobs), _ptr(adj_src),
                                        ctypes.byref(o), _ptr(g), ctypes.byref(mis)))
        return g, float(mis.value)

    def dft_extract(self, freqs: Sequence[float], wavelet=None, ext=None, half: bool = False,
                    traces=None):
        f = np.ascontiguousarray(freqs, dtype=np.float64)
        nf = f.size
        if half:
            out = self.torch.empty((self.ns, nf) + self.shape + (2,), dtype=self.torch.float16,
                                   device=self.device)
            scales = np.zeros(self.ns * nf, dtype=np.float32)
            sp = scales.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
            kind = DFT_C32_HALF
        else:
            out = self.torch.empty((self.ns, nf) + self.shape + (2,), dtype=self.dtype,
                                   device=self.device)
            scales, sp, kind = None, None, DFT_C64
        self._check(self.L.esi_dft_extract(self.h, _ptr(wavelet), _ptr(ext),
                                           f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nf,
                                           _ptr(out), kind, sp, _ptr(traces)))
        return out, (scales.reshape(self.ns, nf) if scales is not None else None)

    def cg_solve(self, dobs, lam: float, tol: float, max_iter: int, precond: str = "none",
                 eps: float = 0.0, out=None, hist: int = 0, wri_wavelet=None,
                 data_space: bool = False, w_out=None, freqs=None):
        """ESI normal equation by Algorithm 1; with wri_wavelet (the point sources f) the WRI
        system (S^T S + lam I) q = S^T (d - S f) instead (esi_wri_solve); with data_space the
        ESI system through the data-space form (esi_dscg_solve; w_out receives w); with freqs
        (Hz) the frequency-domain system F A F^H qbar / nt = F S^T d (esi_fdcg_solve), whose
        solution qbar is returned as [ns][nf][*shape][2] (re, im)."""
        if freqs is not None:
            f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64).ravel())
            q = (self.torch.empty((self.ns, f.size) + self.shape + (2,), dtype=self.dtype,
                                  device=self.device) if out is None else out)
        else:
            q = self.empty_field() if out is None else out
        rep = EsiCgReport()
        hist = max(int(hist), int(max_iter))
        rel = np.zeros((self.ns, hist), dtype=np.float64)
        its = np.zeros(self.ns, dtype=np.int32)
        rep.max_hist = hist
        rep.iters = its.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        rep.rel_res = rel.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if freqs is not None:
            call = self.L.esi_fdcg_solve(self.h, float(lam), float(tol), int(max_iter),
                                         _ptr(dobs),
                                         f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         int(f.size), PC[precond], _ptr(q), float(eps),
                                         ctypes.byref(rep))
        elif data_space:
            call = self.L.esi_dscg_solve(self.h, float(lam), float(tol), int(max_iter),
                                         _ptr(dobs), _ptr(q), _ptr(w_out), float(eps),
                                         ctypes.byref(rep))
        elif wri_wavelet is not None:
            call = self.L.esi_wri_solve(self.h, float(lam), float(tol), int(max_iter),
                                        _ptr(wri_wavelet), _ptr(dobs), _ptr(q), ctypes.byref(rep))
        else:
            call = self.L.esi_cg_solve(self.h, float(lam), float(tol), int(max_iter),
                                       _ptr(dobs), _ptr(q), PC[precond], float(eps),
                                       ctypes.byref(rep))
        st = self._check(call, allow=(ESI_OK, ESI_ERR_NOT_CONVERGED))
        report = {"iters": its.copy(), "rel_res": [rel[s, :its[s]].copy() for s in range(self.ns)],
                  "converged": bool(rep.converged), "iters_max": int(rep.iters_max),
                  "ms_matvec": rep.ms_matvec, "ms_vector": rep.ms_vector,
                  "ms_precond": rep.ms_precond,
                  "ms_total": rep.ms_total, "status": st}
        return q, report

    def wri_solve(self, wavelet, dobs, lam: float, tol: float, max_iter: int, out=None,
                  hist: int = 0):
        """esi_wri_solve: (S^T S + lam I) q = S^T (d - S f) by Algorithm 1."""
        return self.cg_solve(dobs, lam, tol, max_iter, out=out, hist=hist, wri_wavelet=wavelet)

    def dscg_solve(self, dobs, lam: float, tol: float, max_iter: int, eps: float = 0.0,
                   out=None, w_out=None, hist: int = 0):
        """esi_dscg_solve: the ESI normal equation in data space; w_out receives w."""
        return self.cg_solve(dobs, lam, tol, max_iter, eps=eps, out=out, hist=hist,
                             data_space=True, w_out=w_out)

    def fdcg_solve(self, dobs, freqs, lam: float, tol: float, max_iter: int,
                   precond: str = "none", eps: float = 0.0, out=None, hist: int = 0):
        """esi_fdcg_solve: the frequency-domain ESI system at `freqs` (Hz); returns qbar
        [ns][nf][*shape][2] (re, im) and the report."""
        return self.cg_solve(dobs, lam, tol, max_iter, precond=precond, eps=eps, out=out,
                             hist=hist, freqs=freqs)

    def invert(self, dobs, velocity, mode: str = "esi", n_outer: int = 3, n_cg: int = 10,
               cg_tol: float = 0.0, precond: str = "diag", beta0: float = 1.0,
               growth: float = 1.0, memory: int = 5, c1: float = 1e-4, step_frac: float = 0.02,
               max_ls: int = 8, vmin: float = 1.0, vmax: float = 1e9, eps: float = 0.0,
               wavelet=None, grad=None, reduce=None):
        """Algorithm "nestedloop" (esi_invert): velocity (tensor, updated in place) from the
        observed data by n_outer L-BFGS steps on the ESI (mode "esi") or WRI ("wri") reduced
        objective.  `reduce(J, grad) -> J_total`, for shots sharded over ranks, sums J and the
        gradient tensor in place over the ranks.  Returns (gradient, report dict)."""
        g = self.torch.empty(self.shape, dtype=self.dtype, device=self.device) if grad is None else grad
        o = EsiInvertOpts()
        o.mode = GRAD_MODES["saddle" if mode == "esi" else mode]
        o.n_outer, o.n_cg, o.cg_tol = int(n_outer), int(n_cg), float(cg_tol)
        o.precond = PC[precond]
        o.beta0, o.growth, o.memory = float(beta0), float(growth), int(memory)
        o.c1, o.step_frac, o.max_ls = float(c1), float(step_frac), int(max_ls)
        o.vmin, o.vmax, o.eps = float(vmin), float(vmax), float(eps)
        cb = None
        if reduce is not None:
            def _cb(user, jp, gp, n):
                try:
                    jp[0] = float(reduce(float(jp[0]), g))
                    self.torch.cuda.current_stream().synchronize()
                    return 0
                except Exception:   # reported to the caller as ESI_ERR_ARG
                    return 1
            cb = REDUCE_FN(_cb)
            o.reduce = cb
        k = max(int(n_outer), 1)
        arr = {n: np.zeros(k) for n in ("J_start", "J_end", "alpha", "beta")}
        trials = np.zeros(k, dtype=np.int32)
        rep = EsiInvertReport()
        rep.max_iters = k
        for n, a in arr.items():
            setattr(rep, n, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        rep.trials = trials.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        self._check(self.L.esi_invert(self.h, ctypes.byref(o), _ptr(wavelet), _ptr(dobs),
                                      _ptr(velocity), _ptr(g), ctypes.byref(rep)))
        n = rep.iters_done
        tried = n + (1 if rep.stop_reason == 1 else 0)   # a failed line search was tried
        out = {"iters_done": n, "evaluations": rep.evaluations,
               "cg_iters_total": rep.cg_iters_total,
               "stop": STOP_REASONS.get(rep.stop_reason, str(rep.stop_reason)),
               "ms_total": rep.ms_total, "trials": trials[:tried].tolist(),
               "J_start": arr["J_start"][:tried].tolist(), "beta": arr["beta"][:tried].tolist(),
               "J_end": arr["J_end"][:n].tolist(), "alpha": arr["alpha"][:n].tolist()}
        del cb
        return g, out



class PCNet:
    """A stand-alone preconditioner network (esi_pc_*) for h x w images, batches <= max_batch."""

    def __init__(self, h: int, w: int, max_batch: int, stream=None):
        import torch
        self.torch = torch
        self.L = load_library()
        self.h_img, self.w_img = int(h), int(w)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h_ = ctypes.c_void_p()
        st = self.L.esi_pc_create(ctypes.byref(h_), self.h_img, self.w_img, int(max_batch),
                                  ctypes.c_void_p(stream.cuda_stream))
        if st != ESI_OK:
            raise EsiError(st, self.L.esi_pc_last_error(None).decode())
        self.h = h_

    @staticmethod
    def param_count() -> int:
        return int(load_library(require_gpu=False).esi_pc_param_count())

    def _check(self, st):
        if st != ESI_OK:
            raise EsiError(st, self.L.esi_pc_last_error(self.h).decode())

    def set_params(self, params):
        params = params.contiguous()
        self._check(self.L.esi_pc_set_params(self.h, _ptr(params)))

    def get_params(self):
        out = self.torch.empty(self.param_count(), dtype=self.torch.float32, device="cuda")
        self._check(self.L.esi_pc_get_params(self.h, _ptr(out)))
        return out

    def apply(self, x):
        y = self.torch.empty(x.shape, dtype=self.torch.float32, device=x.device)
        self._check(self.L.esi_pc_apply(self.h, _ptr(x), int(x.shape[0]), _ptr(y)))
        return y

    def grad(self, x, e):
        g = self.torch.empty(self.param_count(), dtype=self.torch.float32, device=x.device)
        loss = ctypes.c_double(0.0)
        self._check(self.L.esi_pc_grad(self.h, _ptr(x), _ptr(e), int(x.shape[0]), _ptr(g),
                                       ctypes.byref(loss)))
        return g, float(loss.value)

    def vjp(self, x, gy, out=None):
        """Parameter gradient of <gy, y(x)> (esi_pc_vjp)."""
        g = self.torch.empty(self.param_count(), dtype=self.torch.float32, device=x.device) \
            if out is None else out
        self._check(self.L.esi_pc_vjp(self.h, _ptr(x), _ptr(gy), int(x.shape[0]), _ptr(g)))
        return g

    def train_step(self, x, e, lr: float) -> float:
        loss = ctypes.c_double(0.0)
        self._check(self.L.esi_pc_train_step(self.h, _ptr(x), _ptr(e), int(x.shape[0]),
                                             float(lr), ctypes.byref(loss)))
        return float(loss.value)

    def close(self):
        if getattr(self, "h", None):
            self.L.esi_pc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
