"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np

import oracle


def maxrel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def to_dev(cat, torch):
    pos = torch.from_numpy(np.ascontiguousarray(cat.pos)).cuda()
    w = torch.from_numpy(np.ascontiguousarray(cat.w)).cuda()
    return pos, w


def oracle_zeta(cat, n_primary=None, nthreads=0):
    return oracle.zeta(cat.pos.astype(np.float64), cat.w.astype(np.float64), cat.box, cat.nbins,
                       cat.rmin, cat.rmax, cat.lmax, los_mode=cat.los_mode, n_primary=n_primary,
                       nthreads=nthreads)


def oracle_alm(cat, prims):
    return oracle.alm(cat.pos.astype(np.float64), cat.w.astype(np.float64), prims, cat.box,
                      cat.nbins, cat.rmin, cat.rmax, cat.lmax, los_mode=cat.los_mode)
