"""GB300-native anisotropic 3PCF (Galactos, arXiv 1709.00086) -- Python binding.

Thin ctypes layer over ``libg3pcf.so`` (see ``include/g3pcf.h``): argument
marshalling only; every step of the computation runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream.  If the
library has not been built, the binding raises instead of computing anything
another way.

    plan = Plan(nbins=10, rmin=0, rmax=200, lmax=10, box=1000, los_mode=0)
    zeta, counts = plan.compute(pos_cuda, w_cuda)      # zeta: (zeta_size,) complex128
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libg3pcf.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "g3pcf.h")

LOS_Z_PERIODIC, LOS_Z_OPEN, LOS_RADIAL_OPEN = 0, 1, 2
OPT_CHUNK_ROWS, OPT_CELLS_PER_RMAX, OPT_KFLUSH, OPT_PAIR_KERNELS, OPT_LIST_BYTES = 1, 2, 3, 4, 5
OPT_BASIS = 7
OPT_X_REFINE = 8
OPT_GRAD_PRECISION = 9
OPT_TEST_FAIL_ALLOC, OPT_TEST_TC_TIMEOUT = 10, 11
OPT_TC_OPERANDS = 12
F_POS_F64, F_CONTRACT_FP32, F_NO_SYNC, F_KEEP_ALM, F_GRAPH = 1, 2, 4, 8, 16
ERRORS = {0: "OK", -1: "ERR_ARG", -2: "ERR_RANGE", -3: "ERR_RMAX", -4: "ERR_ALLOC",
          -5: "ERR_CUDA", -6: "ERR_TIMEOUT", -7: "ERR_STATE", -8: "ERR_UNSUPPORTED"}

_lib = None


class G3PCFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code
        self.name = ERRORS.get(code, "?")


def lib():
    """Load libg3pcf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libg3pcf.so is not built; run `python -m paper_1709_00086_gb300.build` "
                               "(or __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.g3pcf_zeta_size.restype = I64
        L.g3pcf_zeta_size.argtypes = [I, I]
        L.g3pcf_last_error.restype = ctypes.c_char_p
        L.g3pcf_last_error.argtypes = []
        L.g3pcf_plan.argtypes = [ctypes.POINTER(P), I, D, D, I, D, I]
        L.g3pcf_set_stream.argtypes = [P, P]
        L.g3pcf_compute.argtypes = [P, P, P, I64, P]
        L.g3pcf_compute_ex.argtypes = [P, P, P, I64, I64, P, P, I]
        L.g3pcf_compute_batch.argtypes = [P, P, P, P, I, P, P, I]
        L.g3pcf_backward.argtypes = [P, P, P, P]
        L.g3pcf_alm.argtypes = [P, P, I64, P]
        L.g3pcf_status.argtypes = [P]
        L.g3pcf_stats.argtypes = [P, P, I]
        L.g3pcf_destroy.argtypes = [P]
        L.g3pcf_autotune.argtypes = [P, P, P, I64, I, P]
        L.g3pcf_autotune.restype = I
        L.g3pcf_autotune_cached.argtypes = [P, P, P, I64, I, ctypes.c_char_p, P]
        L.g3pcf_autotune_cached.restype = I
        L.g3pcf_isotropic.argtypes = [I, I, I, P, P, P]
        L.g3pcf_isotropic.restype = I
        L.g3pcf_zeta_combine.argtypes = [I, I, I, P, P, P, P]
        L.g3pcf_zeta_combine.restype = I
        L.g3pcf_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), P]
        L.g3pcf_fp32_peak.restype = I
        L.g3pcf_set_option.argtypes = [P, I, I64]
        L.g3pcf_set_option.restype = I
        L.g3pcf_zeta_from_alm_noalloc.argtypes = [I, I, P, I64, P, I64, P, P]
        L.g3pcf_zeta_from_alm_noalloc.restype = I
        for f in ("g3pcf_plan", "g3pcf_set_stream", "g3pcf_compute", "g3pcf_compute_ex",
                  "g3pcf_compute_batch", "g3pcf_backward", "g3pcf_alm", "g3pcf_status",
                  "g3pcf_stats", "g3pcf_destroy"):
            getattr(L, f).restype = I
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise G3PCFError(rc, lib().g3pcf_last_error().decode())


def fp32_peak_tflops(stream=None) -> float:
    """Measured FP32 FMA throughput of the current device (TFLOP/s)."""
    v = ctypes.c_double(0.0)
    _check(lib().g3pcf_fp32_peak(ctypes.byref(v), stream))
    return v.value


def isotropic(z, nbins: int, lmax: int):
    """Isotropic Legendre 3PCF zeta_l(b1, b2) from zeta (g3pcf_isotropic).

    z: CUDA complex128 tensor (zsize,) or (ncat, zsize) as returned by Plan.compute /
    compute_batch (or its float64 (..., 2) real view).  Returns (lmax+1, nbins, nbins) or
    (ncat, lmax+1, nbins, nbins) float64."""
    import torch
    zz = (torch.view_as_real(z) if z.is_complex() else z).contiguous()
    single = zz.dim() == 2
    ncat = 1 if single else zz.shape[0]
    out = torch.empty((ncat, lmax + 1, nbins, nbins), dtype=torch.float64, device=zz.device)
    stream = torch.cuda.current_stream(zz.device).cuda_stream
    _check(lib().g3pcf_isotropic(nbins, lmax, ncat, _ptr(zz), _ptr(out), stream))
    return out[0] if single else out


def zeta_combine(zb, coef, nbins: int, lmax: int):
    """sum_c coef[c] zeta_c of a batch of zeta blocks (g3pcf_zeta_combine): zb is
    (ncat, zsize) complex or (ncat, zsize, 2) float64 on a CUDA device; returns a
    complex (zsize,) tensor on that device."""
    import torch
    zr = torch.view_as_real(zb) if zb.is_complex() else zb
    zr = zr.contiguous()
    c = np.ascontiguousarray(coef, dtype=np.float64)
    ncat = zr.shape[0]
    if c.size != ncat:
        raise ValueError("one coefficient per catalog")
    out = torch.empty((zr.shape[1], 2), dtype=torch.float64, device=zr.device)
    _check(lib().g3pcf_zeta_combine(int(nbins), int(lmax), int(ncat), _ptr(zr),
                                    c.ctypes.data_as(ctypes.c_void_p), _ptr(out),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return torch.view_as_complex(out)


def zeta_size(nbins: int, lmax: int) -> int:
    return int(lib().g3pcf_zeta_size(nbins, lmax))


def nlm(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A g3pcf plan: binning, harmonic order, box and line-of-sight mode."""

    def __init__(self, nbins: int, rmin: float, rmax: float, lmax: int, box: float,
                 los_mode: int = LOS_Z_PERIODIC):
        self.nbins, self.rmin, self.rmax, self.lmax = int(nbins), float(rmin), float(rmax), int(lmax)
        self.box, self.los_mode = float(box), int(los_mode)
        h = ctypes.c_void_p()
        _check(lib().g3pcf_plan(ctypes.byref(h), self.nbins, self.rmin, self.rmax, self.lmax,
                                self.box, self.los_mode))
        self._h = h
        self.zsize = zeta_size(self.nbins, self.lmax)
        self._last_n = 0
        self._token = 0  # increments with every forward on this plan

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().g3pcf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        import torch
        _check(lib().g3pcf_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

    def compute(self, pos, w, n_primary=None, fp32_contraction=False, keep_alm=False,
                with_counts=True, sync=True, out=None, graph=False, counts_out=None):
        """zeta (complex128 tensor, zsize) and counts (int64 tensor, nbins) on pos's device."""
        import torch
        if not (pos.is_cuda and w.is_cuda):
            raise ValueError("pos and w must be CUDA tensors")
        pos = pos.contiguous()
        w = w.contiguous()
        if w.dtype != torch.float32:
            raise ValueError("w must be float32")
        if pos.dim() != 2 or pos.shape[1] != 3:
            raise ValueError("pos must be (n, 3)")
        n = pos.shape[0]
        flags = 0
        if pos.dtype == torch.float64:
            flags |= F_POS_F64
        elif pos.dtype != torch.float32:
            raise ValueError("pos must be float32 or float64")
        if fp32_contraction:
            flags |= F_CONTRACT_FP32
        if keep_alm:
            flags |= F_KEEP_ALM
        if not sync:
            flags |= F_NO_SYNC
        if graph:
            flags |= F_GRAPH
        zeta = out if out is not None else torch.empty((self.zsize, 2), dtype=torch.float64,
                                                       device=pos.device)
        counts = None
        if with_counts:
            counts = counts_out if counts_out is not None else torch.empty(
                self.nbins, dtype=torch.int64, device=pos.device)
        npri = -1 if n_primary is None else int(n_primary)
        self._stream()
        _check(lib().g3pcf_compute_ex(self._h, _ptr(pos), _ptr(w), n, npri, _ptr(zeta), _ptr(counts),
                                      flags))
        self._last_n = n
        self._token += 1
        return torch.view_as_complex(zeta), counts

    def compute_batch(self, pos, w, offsets, fp32_contraction=False, sync=True, graph=False,
                      out=None, counts_out=None, keep_alm=False):
        """Batched zeta over catalogs [offsets[c], offsets[c+1]): (ncat, zsize) complex.

        graph=True replays a captured CUDA graph for repeated calls with the same
        buffers (pass the same out/counts_out tensors)."""
        import torch
        pos = pos.contiguous()
        w = w.contiguous()
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        ncat = offs.size - 1
        zeta = out if out is not None else torch.empty((ncat, self.zsize, 2), dtype=torch.float64,
                                                       device=pos.device)
        counts = counts_out if counts_out is not None else torch.empty(
            (ncat, self.nbins), dtype=torch.int64, device=pos.device)
        flags = ((F_CONTRACT_FP32 if fp32_contraction else 0) | (0 if sync else F_NO_SYNC) |
                 (F_GRAPH if graph else 0) | (F_KEEP_ALM if keep_alm else 0))
        self._stream()
        self._token += 1
        self._last_n = int(pos.shape[0])
        _check(lib().g3pcf_compute_batch(self._h, _ptr(pos), _ptr(w),
                                         offs.ctypes.data_as(ctypes.c_void_p), ncat, _ptr(zeta),
                                         _ptr(counts), flags))
        return torch.view_as_complex(zeta), counts

    def alm(self, primaries) -> np.ndarray:
        """a_lm(i, b) of the last forward: (np, nbins, nlm) complex128 (host)."""
        prim = np.ascontiguousarray(primaries, dtype=np.int64)
        out = np.zeros((prim.size, self.nbins, nlm(self.lmax)), dtype=np.complex128)
        _check(lib().g3pcf_alm(self._h, prim.ctypes.data_as(ctypes.c_void_p), prim.size,
                               out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def backward(self, dzeta):
        """(dpos (n,3) float64, dw (n,) float64) for the last forward (compute or
        compute_batch; for a batch dzeta is (ncat, zsize) like its zeta)."""
        import torch
        dz = torch.view_as_real(dzeta) if dzeta.is_complex() else dzeta
        dz = dz.contiguous().to(torch.float64)
        n = self._last_n
        dpos = torch.empty((n, 3), dtype=torch.float64, device=dz.device)
        dw = torch.empty(n, dtype=torch.float64, device=dz.device)
        self._stream()
        _check(lib().g3pcf_backward(self._h, _ptr(dz), _ptr(dpos), _ptr(dw)))
        return dpos, dw

    def autotune(self, pos, w) -> dict:
        """Pick cells-per-rmax and flush size for this data (see g3pcf_autotune)."""
        import torch
        pos = pos.contiguous()
        w = w.contiguous()
        flags = F_POS_F64 if pos.dtype == torch.float64 else 0
        out = np.zeros(3, dtype=np.int64)
        self._stream()
        _check(lib().g3pcf_autotune(self._h, _ptr(pos), _ptr(w), pos.shape[0], flags,
                                    out.ctypes.data_as(ctypes.c_void_p)))
        return {"cells_per_rmax": int(out[0]), "kflush": int(out[1]), "pair_us": int(out[2])}

    def autotune_cached(self, pos, w, cache_path=None) -> dict:
        """Tune cell resolution and x refinement (pair lists) or flush size (fused
        kernel), then the contraction's operand source, on a sample of this data,
        through the on-disk cache cache_path (see g3pcf_autotune_cached)."""
        import torch
        pos = pos.contiguous()
        w = w.contiguous()
        flags = F_POS_F64 if pos.dtype == torch.float64 else 0
        out = np.zeros(6, dtype=np.int64)
        self._stream()
        _check(lib().g3pcf_autotune_cached(self._h, _ptr(pos), _ptr(w), pos.shape[0], flags,
                                           None if cache_path is None else str(cache_path).encode(),
                                           out.ctypes.data_as(ctypes.c_void_p)))
        return {"cells_per_rmax": int(out[0]), "x_refine": int(out[1]), "kflush": int(out[2]),
                "pair_us": int(out[3]), "from_cache": bool(out[4]), "tc_operands": int(out[5])}

    def set_option(self, option: int, value: int):
        """Tuning knob (OPT_CHUNK_ROWS, OPT_CELLS_PER_RMAX, OPT_KFLUSH, OPT_PAIR_KERNELS,
        OPT_LIST_BYTES, OPT_BASIS, OPT_X_REFINE, OPT_GRAD_PRECISION, OPT_TC_OPERANDS; 0 = automatic)."""
        _check(lib().g3pcf_set_option(self._h, int(option), int(value)))

    def status(self):
        _check(lib().g3pcf_status(self._h))

    def stats(self) -> dict:
        v = np.zeros(15)
        _check(lib().g3pcf_stats(self._h, v.ctypes.data_as(ctypes.c_void_p), 15))
        keys = ["index_ms", "pair_ms", "contract_ms", "reduce_ms", "total_ms", "pairs", "primaries",
                "cells_per_rmax", "launches", "candidates", "list_passes", "scan_ms", "accum_ms",
                "accum_launches", "tc_operands_from_pairs"]
        return dict(zip(keys, v.tolist()))


class _Zeta:
    """torch.autograd.Function computing zeta (real view (zsize, 2)) of (pos, w)."""

    @staticmethod
    def _fn():
        import torch

        class ZetaFunction(torch.autograd.Function):
            @staticmethod
            def forward(ctx, pos, w, plan, n_primary, fp32_contraction):
                z, _ = plan.compute(pos.detach(), w.detach(), n_primary=n_primary,
                                    fp32_contraction=fp32_contraction, keep_alm=True)
                ctx.plan = plan
                ctx.token = plan._token
                ctx.args = (n_primary, fp32_contraction)
                ctx.save_for_backward(pos, w)
                return torch.view_as_real(z).clone()

            @staticmethod
            def backward(ctx, gz):
                pos, w = ctx.saved_tensors
                plan = ctx.plan
                if plan._token != ctx.token:  # the plan ran another forward since: redo ours
                    plan.compute(pos.detach(), w.detach(), n_primary=ctx.args[0],
                                 fp32_contraction=ctx.args[1], keep_alm=True)
                dpos, dw = plan.backward(gz)
                return dpos.to(pos.dtype), dw.to(w.dtype), None, None, None

        return ZetaFunction


_ZETA_FN = None


def zeta(pos, w, plan: "Plan", n_primary=None, fp32_contraction=False):
    """Differentiable zeta (real view, shape (zsize, 2), float64) of pos (n,3) and w (n,).

    Gradients with respect to pos and w come from the library's adjoint
    (g3pcf_backward; z line-of-sight modes), with the pair set and bins held
    at the forward positions.
    """
    global _ZETA_FN
    if _ZETA_FN is None:
        _ZETA_FN = _Zeta._fn()
    return _ZETA_FN.apply(pos, w, plan, n_primary, fp32_contraction)


def zeta_blocks(z, nbins: int, lmax: int):
    """Split a flat complex zeta (numpy or torch) into per-m K_m x K_m blocks."""
    z = z.detach().cpu().numpy() if hasattr(z, "detach") else np.asarray(z)
    out, off = [], 0
    for m in range(lmax + 1):
        K = nbins * (lmax + 1 - m)
        out.append(z[off:off + K * K].reshape(K, K))
        off += K * K
    return out
