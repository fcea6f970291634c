"""Seeded synthetic galaxy catalogs (inputs only; no 3PCF arithmetic here).

The paper measures on the Outer Rim halo catalog (Sec. 4.2), which is not
available; these generators stand in for it with the box sizes, search radius
and clustering recipe of the workloads this library is measured on:

* ``uniform``   -- points uniform in a cube of side L (NumPy PCG64).
* ``clustered`` -- a fraction ``f_uniform`` uniform, the rest assigned
  uniformly at random to ``n_centres`` uniform centres and displaced by an
  isotropic Gaussian of width ``sigma`` (Mpc/h); periodic boxes wrap the
  displaced points, open boxes redraw the ones that leave the box.

Positions are drawn in FP64, wrapped into [0, L), and cast to the requested
dtype; an FP32 value that rounds up to L is mapped to 0.  Weights are 1 or
U(0.5, 1.5) in FP32.  Both the oracle tests and the CUDA tests draw from here;
this module holds none of the method's arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Catalog:
    pos: np.ndarray          # (n, 3) float64 or float32, in [0, box)
    w: np.ndarray            # (n,) float32
    box: float
    nbins: int
    rmin: float
    rmax: float
    lmax: int
    los_mode: int            # 0 periodic z, 1 open z, 2 open radial
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def params(self) -> dict:
        return dict(nbins=self.nbins, rmin=self.rmin, rmax=self.rmax, lmax=self.lmax,
                    box=self.box, los_mode=self.los_mode)


def _wrap_cast(x: np.ndarray, box: float, dtype) -> np.ndarray:
    x = np.mod(x, box)
    x = x.astype(dtype)
    x[x >= dtype(box)] = 0
    x[x < 0] = 0
    return np.ascontiguousarray(x)


def uniform_positions(rng: np.random.Generator, n: int, box: float, dtype=np.float64):
    return _wrap_cast(rng.uniform(0.0, box, size=(n, 3)), box, dtype)


def clustered_positions(rng: np.random.Generator, n: int, box: float, n_centres: int = 10000,
                        sigma: float = 5.0, f_uniform: float = 0.6, periodic: bool = True,
                        dtype=np.float32):
    n_uni = int(round(f_uniform * n))
    n_blob = n - n_uni
    uni = rng.uniform(0.0, box, size=(n_uni, 3))
    centres = rng.uniform(0.0, box, size=(n_centres, 3))
    owner = rng.integers(0, n_centres, size=n_blob)
    blob = centres[owner] + rng.normal(0.0, sigma, size=(n_blob, 3))
    if not periodic:
        bad = np.any((blob < 0) | (blob >= box), axis=1)
        while np.any(bad):
            k = int(bad.sum())
            blob[bad] = centres[owner[bad]] + rng.normal(0.0, sigma, size=(k, 3))
            bad = np.any((blob < 0) | (blob >= box), axis=1)
    pos = np.concatenate([uni, blob], axis=0)
    pos = pos[rng.permutation(n)]
    return _wrap_cast(pos, box, dtype)


def weights(rng: np.random.Generator, n: int, kind: str = "uniform_0.5_1.5"):
    if kind == "ones":
        return np.ones(n, dtype=np.float32)
    return rng.uniform(0.5, 1.5, size=n).astype(np.float32)


# --- the five measured workloads -------------------------------------------

def plain_uniform(n: int = 20000, seed: int = 1) -> Catalog:
    """N uniform points, periodic cube L=1000, FP64 positions, w = 1, Rmax=200,
    10 bins on [0, 200], lmax=10, LOS = z."""
    rng = np.random.default_rng(seed)
    pos = uniform_positions(rng, n, 1000.0, np.float64)
    return Catalog(pos, weights(rng, n, "ones"), 1000.0, 10, 0.0, 200.0, 10, 0,
                   name="uniform-20k-L1000")


def clustered_2m(n: int = 2_000_000, seed: int = 2, box: float = 1500.0) -> Catalog:
    """60% uniform + 40% in sigma=5 blobs about 10,000 centres, periodic L=1500,
    FP32 positions, w ~ U(0.5,1.5), Rmax=200, 10 bins, lmax=10, LOS = z."""
    rng = np.random.default_rng(seed)
    pos = clustered_positions(rng, n, box, periodic=True, dtype=np.float32)
    return Catalog(pos, weights(rng, n), box, 10, 0.0, 200.0, 10, 0,
                   name="clustered-%d-L%g" % (n, box))


def batch_sizes(ncat: int = 64, seed: int = 3, lo: float = 3.0, hi: float = 6.0):
    rng = np.random.default_rng(seed)
    return [int(round(10.0 ** u)) for u in rng.uniform(lo, hi, size=ncat)]


def batched(ncat: int = 64, seed: int = 3, sizes=None, box: float = 600.0):
    """ncat independent uniform catalogs in periodic cubes of side 600, sizes
    log-uniform in [1e3, 1e6], w ~ U(0.5,1.5), Rmax=150, 12 bins, lmax=8, LOS=z.
    Catalog c is drawn from seed (seed, c)."""
    if sizes is None:
        sizes = batch_sizes(ncat, seed)
    cats = []
    for c, n in enumerate(sizes):
        rng = np.random.default_rng([seed, c])
        pos = uniform_positions(rng, n, box, np.float32)
        cats.append(Catalog(pos, weights(rng, n), box, 12, 0.0, 150.0, 8, 0,
                            name="batch-%d" % c))
    return cats


def differentiation(n: int = 500_000, seed: int = 4, box: float = 800.0) -> Catalog:
    """Clustered as the 2M catalog (10,000 centres), periodic L=800, FP32,
    Rmax=120, 8 bins, lmax=6, LOS = z.  The target zeta uses seed 5."""
    rng = np.random.default_rng(seed)
    pos = clustered_positions(rng, n, box, periodic=True, dtype=np.float32)
    return Catalog(pos, weights(rng, n), box, 8, 0.0, 120.0, 6, 0,
                   name="diff-%d-L%g" % (n, box))


def large_radial(n: int = 50_000_000, seed: int = 7, box: float = 3000.0) -> Catalog:
    """Clustered (10,000 centres), open cube L=3000 observed from its centre,
    per-primary radial LOS, FP32, w ~ U(0.5,1.5), Rmax=200, 10 bins, lmax=10."""
    rng = np.random.default_rng(seed)
    pos = clustered_positions(rng, n, box, periodic=False, dtype=np.float32)
    return Catalog(pos, weights(rng, n), box, 10, 0.0, 200.0, 10, 2,
                   name="radial-%d-L%g" % (n, box))


def data_minus_randoms(data: Catalog, nrand_factor: int = 2, seed: int = 0) -> Catalog:
    """A D - R catalog (the random-catalog correction of Sec. 6): the data points
    with their weights followed by nrand_factor x n uniform randoms in the same
    box with the equal negative weight -sum(w_D) / n_R, so the total weight is ~0.
    The randoms take the data's position dtype; the parameters are the data's."""
    rng = np.random.default_rng(seed)
    n_r = nrand_factor * data.n
    rpos = uniform_positions(rng, n_r, data.box, data.pos.dtype.type)
    alpha = float(np.sum(data.w, dtype=np.float64)) / max(n_r, 1)
    rw = np.full(n_r, -alpha, dtype=np.float32)
    return Catalog(np.concatenate([data.pos, rpos]), np.concatenate([data.w, rw]), data.box,
                   data.nbins, data.rmin, data.rmax, data.lmax, data.los_mode,
                   name="%s-minus-%dR" % (data.name, nrand_factor))


def random_catalogs(data: Catalog, n_randoms: int, nrand_factor: int = 2, seed: int = 0):
    """n_randoms random catalogs for the random-catalog correction of Sec. 6.  R_k
    holds nrand_factor x n uniform points in the data's box (drawn from seed (seed, k))
    with the equal positive weight alpha = sum(w_D) / n_R, so that its total weight
    is the data's; D - R_k is the data followed by R_k at weight -alpha.  Returns
    ([D - R_0, ...], [R_0, ...]) with the data's parameters."""
    n_r = nrand_factor * data.n
    alpha = float(np.sum(data.w, dtype=np.float64)) / max(n_r, 1)
    dr, rr = [], []
    for k in range(n_randoms):
        rng = np.random.default_rng([seed, k])
        rpos = uniform_positions(rng, n_r, data.box, data.pos.dtype.type)
        rr.append(Catalog(rpos, np.full(n_r, alpha, dtype=np.float32), data.box, data.nbins, data.rmin,
                          data.rmax, data.lmax, data.los_mode, name="R%d" % k))
        dr.append(Catalog(np.concatenate([data.pos, rpos]),
                          np.concatenate([data.w, np.full(n_r, -alpha, dtype=np.float32)]), data.box,
                          data.nbins, data.rmin, data.rmax, data.lmax, data.los_mode,
                          name="%s-minus-R%d" % (data.name, k)))
    return dr, rr


def small_case(kind: str, n: int, seed: int, box: float, nbins: int, rmin: float, rmax: float,
               lmax: int, los_mode: int = 0, dtype=np.float32, weight_kind="uniform_0.5_1.5"):
    """A small catalog with an explicit recipe, for parity tests."""
    rng = np.random.default_rng(seed)
    periodic = los_mode == 0
    if kind == "uniform":
        pos = uniform_positions(rng, n, box, dtype)
    else:
        pos = clustered_positions(rng, n, box, n_centres=max(1, n // 40), periodic=periodic,
                                  dtype=dtype)
    return Catalog(pos, weights(rng, n, weight_kind), box, nbins, rmin, rmax, lmax, los_mode,
                   name="%s-%d" % (kind, n))
