"""FP64 CPU oracle for the anisotropic 3PCF (Galactos, arXiv 1709.00086, Sec. 3.1).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow definition the CUDA
path is checked against; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with ``paper_1709_00086_gb300`` and never imports it.

Functions follow the paper's notation: ``nbins`` radial shells between ``rmin``
and ``rmax`` (Sec. 3.1: "the secondaries are binned into spherical shells"),
spherical harmonics up to ``lmax`` (Sec. 3.3.2: l = 10), multipoles
``a_lm(i, b) = sum_j w_j Y_lm(rhat_ij)`` (Sec. 3.1, the discrete form of the
shell integral) and ``zeta^m_{ll'}(b1,b2) = sum_i w_i a_lm(i,b1) a*_l'm(i,b2)``
(Sec. 3.1, product of coefficients about one primary summed over primaries).

LOS modes: 0 = z axis, periodic box (minimum image); 1 = z axis, open box;
2 = radial from the box centre, open box (Sec. 3.1 and Fig. 2: rotate so the
primary's line of sight is the z axis).

Parity pins for every function live in ``tests/test_oracle_*.py``.  Nothing
here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

LOS_Z_PERIODIC, LOS_Z_OPEN, LOS_RADIAL_OPEN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64, I, D = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_zeta_size.restype = I64
        lib.orc_zeta_size.argtypes = [I, I]
        lib.orc_edges.argtypes = [I, D, D, P]
        lib.orc_ylm.argtypes = [I, P, I64, P]
        lib.orc_ylm_grad.argtypes = [I, P, I64, P]
        lib.orc_alm.argtypes = [P, P, I64, P, I64, D, I, I, D, D, I, P, P, I]
        lib.orc_zeta.argtypes = [P, P, P, I64, I64, D, I, I, D, D, I, P, P, I]
        lib.orc_zeta_from_alm.argtypes = [P, P, I64, I, I, P]
        lib.orc_zeta_triplets.argtypes = [P, P, I64, D, I, I, D, D, I, P]
        lib.orc_iso_legendre.argtypes = [P, P, I64, D, I, I, D, D, I, P]
        lib.orc_grad.argtypes = [P, P, I64, D, I, I, D, D, I, P, P, P, I]
        lib.orc_grad_sel.argtypes = [P, P, I64, D, I, I, D, D, I, P, P, I64, P, P, I]
        lib.orc_mono_count.restype = I64
        lib.orc_mono_count.argtypes = [I]
        lib.orc_alm_monomial.argtypes = [P, P, I64, P, I64, D, I, I, D, D, I, P, I]
        for f in ("orc_edges", "orc_ylm", "orc_ylm_grad", "orc_alm", "orc_zeta",
                  "orc_zeta_from_alm", "orc_zeta_triplets", "orc_iso_legendre", "orc_grad", "orc_grad_sel",
                  "orc_alm_monomial"):
            getattr(lib, f).restype = I
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def nlm(lmax: int) -> int:
    """Number of (l, m >= 0) pairs up to lmax."""
    return (lmax + 1) * (lmax + 2) // 2


def lm_index(l: int, m: int) -> int:
    return l * (l + 1) // 2 + m


def zeta_block_sizes(nbins: int, lmax: int):
    """K_m = nbins * (lmax + 1 - m), m = 0..lmax."""
    return [nbins * (lmax + 1 - m) for m in range(lmax + 1)]


def zeta_blocks(flat, nbins: int, lmax: int):
    """Split a flat complex zeta vector into per-m K_m x K_m complex blocks."""
    flat = np.asarray(flat)
    if flat.dtype != np.complex128:
        flat = flat.view(np.complex128)
    out, off = [], 0
    for K in zeta_block_sizes(nbins, lmax):
        out.append(flat[off:off + K * K].reshape(K, K))
        off += K * K
    return out


def edges2(nbins: int, rmin: float, rmax: float) -> np.ndarray:
    """Squared bin edges e_k^2 (e_0 = rmin, e_B = rmax, linear in between)."""
    out = np.zeros(nbins + 1)
    if _load().orc_edges(nbins, rmin, rmax, _ptr(out)) != 0:
        raise ValueError("bad binning")
    return out


def ylm(lmax: int, d) -> np.ndarray:
    """Y_lm(d/|d|) for m >= 0: array (n, nlm) complex (std::sph_legendre based)."""
    d = _f64(np.atleast_2d(d))
    out = np.zeros((d.shape[0], nlm(lmax)), dtype=np.complex128)
    _load().orc_ylm(lmax, _ptr(d), d.shape[0], _ptr(out))
    return out


def ylm_grad(lmax: int, d) -> np.ndarray:
    """grad_d Y_lm(d/|d|): array (n, nlm, 3) complex (solid-harmonic ladder)."""
    d = _f64(np.atleast_2d(d))
    out = np.zeros((d.shape[0], nlm(lmax), 3), dtype=np.complex128)
    _load().orc_ylm_grad(lmax, _ptr(d), d.shape[0], _ptr(out))
    return out


def alm(pos, w, primaries, box, nbins, rmin, rmax, lmax, los_mode=0, nthreads=0,
        return_counts=False):
    """Per-primary multipoles a_lm(i, b): array (np, nbins, nlm) complex."""
    pos, w = _f64(pos), _f64(w)
    prim = np.ascontiguousarray(primaries, dtype=np.int64)
    out = np.zeros((prim.size, nbins, nlm(lmax)), dtype=np.complex128)
    counts = np.zeros(nbins, dtype=np.int64)
    rc = _load().orc_alm(_ptr(pos), _ptr(w), pos.shape[0], _ptr(prim), prim.size, box, los_mode,
                         nbins, rmin, rmax, lmax, _ptr(out), _ptr(counts), nthreads)
    if rc != 0:
        raise ValueError("orc_alm failed (%d)" % rc)
    return (out, counts) if return_counts else out


def mono_count(lmax):
    """Number of monomial power sums x^a y^b z^c with a + b + c <= lmax (Sec. 3.3.2)."""
    return int(_load().orc_mono_count(lmax))


def alm_monomial(pos, w, primaries, box, nbins, rmin, rmax, lmax, los_mode=0, nthreads=0):
    """Per-primary multipoles through the paper's monomial power sums (Sec. 3.3.2):
    per bin M_abc = sum_j w_j xhat^a yhat^b zhat^c, a + b + c <= lmax, converted
    with the expansion of Y_lm in those monomials.  Same layout as ``alm``."""
    pos, w = _f64(pos), _f64(w)
    prim = np.ascontiguousarray(primaries, dtype=np.int64)
    out = np.zeros((prim.size, nbins, nlm(lmax)), dtype=np.complex128)
    rc = _load().orc_alm_monomial(_ptr(pos), _ptr(w), pos.shape[0], _ptr(prim), prim.size, box,
                                  los_mode, nbins, rmin, rmax, lmax, _ptr(out), nthreads)
    if rc != 0:
        raise ValueError("orc_alm_monomial failed (%d)" % rc)
    return out


def zeta(pos, w, box, nbins, rmin, rmax, lmax, los_mode=0, n_primary=None, nthreads=0,
         pos_bins=None):
    """zeta (flat complex, per-m blocks) and counts (int64 per bin)."""
    pos, w = _f64(pos), _f64(w)
    pb = _f64(pos_bins) if pos_bins is not None else None
    n = pos.shape[0]
    npri = n if n_primary is None else int(n_primary)
    out = np.zeros(_load().orc_zeta_size(nbins, lmax), dtype=np.complex128)
    counts = np.zeros(nbins, dtype=np.int64)
    rc = _load().orc_zeta(_ptr(pos), _ptr(pb), _ptr(w), n, npri, box, los_mode, nbins, rmin,
                          rmax, lmax, _ptr(out), _ptr(counts), nthreads)
    if rc != 0:
        raise ValueError("orc_zeta failed (%d)" % rc)
    return out, counts


def zeta_from_alm(a, wprim, nbins, lmax):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    wprim = _f64(wprim)
    out = np.zeros(_load().orc_zeta_size(nbins, lmax), dtype=np.complex128)
    _load().orc_zeta_from_alm(_ptr(a), _ptr(wprim), wprim.size, nbins, lmax, _ptr(out))
    return out


def zeta_triplets(pos, w, box, nbins, rmin, rmax, lmax, los_mode=0):
    """O(N^3) brute-force triplet sum (tiny N)."""
    pos, w = _f64(pos), _f64(w)
    out = np.zeros(_load().orc_zeta_size(nbins, lmax), dtype=np.complex128)
    _load().orc_zeta_triplets(_ptr(pos), _ptr(w), pos.shape[0], box, los_mode, nbins, rmin,
                              rmax, lmax, _ptr(out))
    return out


def iso_legendre(pos, w, box, nbins, rmin, rmax, lmax, los_mode=0):
    """Isotropic Legendre 3PCF by brute force: (lmax+1, nbins, nbins)."""
    pos, w = _f64(pos), _f64(w)
    out = np.zeros((lmax + 1, nbins, nbins))
    _load().orc_iso_legendre(_ptr(pos), _ptr(w), pos.shape[0], box, los_mode, nbins, rmin,
                             rmax, lmax, _ptr(out))
    return out


def grad(pos, w, G, box, nbins, rmin, rmax, lmax, los_mode=0, nthreads=0):
    """Reference (dpos, dw) of L = sum |zeta - zeta_t|^2 given G = zeta - zeta_t."""
    pos, w = _f64(pos), _f64(w)
    G = np.ascontiguousarray(G, dtype=np.complex128)
    n = pos.shape[0]
    dpos = np.zeros((n, 3))
    dw = np.zeros(n)
    rc = _load().orc_grad(_ptr(pos), _ptr(w), n, box, los_mode, nbins, rmin, rmax, lmax,
                          _ptr(G), _ptr(dpos), _ptr(dw), nthreads)
    if rc != 0:
        raise ValueError("orc_grad failed (%d)" % rc)
    return dpos, dw


def grad_sel(pos, w, G, box, nbins, rmin, rmax, lmax, sel, los_mode=0, nthreads=0):
    """Reference (dpos, dw) of ``grad`` for the chosen galaxies ``sel`` only:
    arrays (len(sel), 3) and (len(sel),), in the order of ``sel``.  Evaluates the
    multipoles of the chosen galaxies and of the primaries within rmax of them."""
    pos, w = _f64(pos), _f64(w)
    G = np.ascontiguousarray(G, dtype=np.complex128)
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    dpos = np.zeros((sel.size, 3))
    dw = np.zeros(sel.size)
    rc = _load().orc_grad_sel(_ptr(pos), _ptr(w), pos.shape[0], box, los_mode, nbins, rmin, rmax, lmax,
                              _ptr(G), _ptr(sel), sel.size, _ptr(dpos), _ptr(dw), nthreads)
    if rc != 0:
        raise ValueError("orc_grad_sel failed (%d)" % rc)
    return dpos, dw


def loss(zeta_flat, zeta_target):
    """L = sum over all stored entries |zeta - zeta_t|^2."""
    d = np.asarray(zeta_flat) - np.asarray(zeta_target)
    return float(np.sum(d.real ** 2 + d.imag ** 2))
