"""Pin for the oracle's reference gradient of L = sum |zeta - zeta_t|^2.

The adjoint is not in the paper; its definition is the derivative of the
paper's zeta (Sec. 3.1) with the pair set and radial bins held fixed.  The
oracle's analytic gradient is pinned to FP64 central finite differences of the
oracle's own loss with frozen pair geometry (``pos_bins``).
"""
import numpy as np
import pytest

import oracle
from paper_1709_00086_gb300 import catalogs


def _setup(seed=5):
    box, nb, lmax = 20.0, 3, 4
    rng = np.random.default_rng(seed)
    n = 45
    pos = rng.uniform(0, box, size=(n, 3))
    w = rng.uniform(0.5, 1.5, size=n)
    kw = dict(box=box, nbins=nb, rmin=0.5, rmax=7.0, lmax=lmax, los_mode=0)
    rng_t = np.random.default_rng(seed + 100)
    pos_t = rng_t.uniform(0, box, size=(n, 3))
    w_t = rng_t.uniform(0.5, 1.5, size=n)
    zt, _ = oracle.zeta(pos_t, w_t, **kw)
    return pos, w, zt, kw


def test_gradient_matches_central_differences():
    pos, w, zt, kw = _setup()
    z, _ = oracle.zeta(pos, w, **kw)
    dpos, dw = oracle.grad(pos, w, z - zt, **kw)

    def L(p, ww):
        zz, _ = oracle.zeta(p, ww, pos_bins=pos, **kw)
        return oracle.loss(zz, zt)

    rng = np.random.default_rng(9)
    h = 1e-5
    for k in rng.choice(pos.shape[0], size=6, replace=False):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[k, a] += h
            pm[k, a] -= h
            fd = (L(pp, w) - L(pm, w)) / (2 * h)
            assert abs(fd - dpos[k, a]) < 1e-6 * max(1.0, np.abs(dpos).max()), (k, a, fd, dpos[k, a])
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (L(pos, wp) - L(pos, wm)) / (2 * h)
        assert abs(fd - dw[k]) < 1e-6 * max(1.0, np.abs(dw).max()), (k, fd, dw[k])


def test_gradient_sums_translation_invariance():
    # L is invariant under a rigid translation of all points (periodic box), so
    # the position gradient sums to zero over galaxies.
    pos, w, zt, kw = _setup(seed=8)
    z, _ = oracle.zeta(pos, w, **kw)
    dpos, _ = oracle.grad(pos, w, z - zt, **kw)
    assert np.abs(dpos.sum(axis=0)).max() < 1e-9 * np.abs(dpos).max()


def test_radial_mode_rejected():
    pos, w, zt, kw = _setup()
    kw = dict(kw, los_mode=2)
    with pytest.raises(ValueError):
        oracle.grad(pos, w, zt, **kw)


@pytest.mark.parametrize("los_mode", [0, 1])
def test_grad_sel_matches_full_gradient(los_mode):
    # the chosen-galaxy gradient (used on catalogs too large for orc_grad) equals
    # the full reference gradient at those galaxies: same terms, fewer primaries
    cat = catalogs.small_case("clustered", 500, seed=70 + los_mode, box=220.0, nbins=6, rmin=5.0,
                              rmax=50.0, lmax=5, los_mode=los_mode)
    pos, w = cat.pos.astype(np.float64), cat.w.astype(np.float64)
    K = sum(k * k for k in oracle.zeta_block_sizes(cat.nbins, cat.lmax))
    rng = np.random.default_rng(71)
    G = rng.normal(size=K) + 1j * rng.normal(size=K)
    dpos, dw = oracle.grad(pos, w, G, cat.box, cat.nbins, cat.rmin, cat.rmax, cat.lmax, los_mode=los_mode)
    sel = rng.choice(cat.n, 40, replace=False)
    spos, sw = oracle.grad_sel(pos, w, G, cat.box, cat.nbins, cat.rmin, cat.rmax, cat.lmax, sel,
                               los_mode=los_mode)
    assert np.abs(spos - dpos[sel]).max() <= 1e-12 * np.abs(dpos).max()
    assert np.abs(sw - dw[sel]).max() <= 1e-12 * np.abs(dw).max()
    # a chosen galaxy with no neighbours gets only its (zero) primary terms
    far = np.concatenate([pos, [[0.5 * cat.box, 0.5 * cat.box, 0.5 * cat.box]]])
    far_w = np.concatenate([w, [1.0]])
    keep = np.linalg.norm(far[:-1] - far[-1], axis=1) > cat.rmax + 1.0
    far = np.concatenate([far[:-1][keep], far[-1:]])
    far_w = np.concatenate([far_w[:-1][keep], far_w[-1:]])
    spos, sw = oracle.grad_sel(far, far_w, G, cat.box, cat.nbins, cat.rmin, cat.rmax, cat.lmax,
                               [far.shape[0] - 1], los_mode=los_mode)
    assert np.all(spos == 0.0) and np.all(sw == 0.0)
