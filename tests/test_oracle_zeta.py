"""Pins for the oracle's zeta, counts and multipoles (Sec. 3.1 of the paper).

Each pin is something the oracle's own code does not re-derive: an O(N^3)
triplet sum, the addition theorem against the isotropic Legendre 3PCF
(Sec. 2.2), a pure-counting identity checked with an independent numpy pair
search, Unsold's theorem for one pair, Hermitian symmetry, and invariance under
rotations about the line of sight (Sec. 3.1: axisymmetry about the LOS gives
equal m), translations and point reflection.
"""
import numpy as np
import pytest

import oracle

FOURPI = 4.0 * np.pi


def _cat(n, box, seed, dtype=np.float64, lattice=None):
    rng = np.random.default_rng(seed)
    if lattice:
        pos = rng.integers(0, int(box * lattice), size=(n, 3)) / lattice
    else:
        pos = rng.uniform(0, box, size=(n, 3))
    pos = pos.astype(dtype).astype(np.float64)
    w = rng.uniform(0.5, 1.5, size=n).astype(np.float32).astype(np.float64)
    return pos, w


def _maxrel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("los_mode,box", [(0, 10.0), (1, 10.0), (2, 10.0)])
def test_factorised_equals_triplet_brute_force(los_mode, box):
    pos, w = _cat(28, box, seed=10 + los_mode)
    kw = dict(box=box, nbins=3, rmin=0.5, rmax=4.5, lmax=4, los_mode=los_mode)
    z, counts = oracle.zeta(pos, w, **kw)
    zt = oracle.zeta_triplets(pos, w, **kw)
    assert counts.sum() > 50
    assert _maxrel(z, zt) < 1e-12


def test_addition_theorem_recovers_isotropic_legendre():
    # sum_m zeta^m_ll with the m<0 blocks folded in: zeta^0_ll + 2 Re sum_{m>0}
    # zeta^m_ll = (2l+1)/(4pi) sum w_i w_j w_k P_l(rhat_ij . rhat_ik)
    box, nb, lmax = 10.0, 3, 6
    pos, w = _cat(30, box, seed=21)
    kw = dict(box=box, nbins=nb, rmin=0.0, rmax=4.9, lmax=lmax, los_mode=0)
    z, _ = oracle.zeta(pos, w, **kw)
    blocks = oracle.zeta_blocks(z, nb, lmax)
    iso = oracle.iso_legendre(pos, w, **kw)
    for l in range(lmax + 1):
        acc = np.zeros((nb, nb))
        for m in range(l + 1):
            r0 = (l - m) * nb
            blk = blocks[m][r0:r0 + nb, r0:r0 + nb]
            acc += (1.0 if m == 0 else 2.0) * blk.real
        assert _maxrel(acc, iso[l]) < 1e-11, l


def _numpy_pairs(pos, box, periodic, e2):
    """Independent pair search: all ordered (i, j) and their bins."""
    d = pos[None, :, :] - pos[:, None, :]
    if periodic:
        d = d - box * np.round(d / box)
    r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    b = np.searchsorted(e2, r2, side="right") - 1
    ok = (r2 > 0) & (r2 >= e2[0]) & (r2 < e2[-1])
    return np.where(ok, b, -1)


@pytest.mark.parametrize("los_mode", [0, 1])
def test_monopole_counts_identity(los_mode):
    # 4 pi zeta^0_00(b1,b2) = sum_i w_i W_i(b1) W_i(b2),  W_i(b) = sum_{j in b} w_j
    box, nb, lmax = 50.0, 5, 2
    pos, w = _cat(300, box, seed=31 + los_mode)
    kw = dict(box=box, nbins=nb, rmin=1.0, rmax=20.0, lmax=lmax, los_mode=los_mode)
    z, counts = oracle.zeta(pos, w, **kw)
    bins = _numpy_pairs(pos, box, los_mode == 0, oracle.edges2(nb, 1.0, 20.0))
    W = np.zeros((pos.shape[0], nb))
    for b in range(nb):
        W[:, b] = ((bins == b) * w[None, :]).sum(axis=1)
    want = np.einsum("i,ia,ib->ab", w, W, W)
    blk = oracle.zeta_blocks(z, nb, lmax)[0][:nb, :nb]
    assert _maxrel(FOURPI * blk.real, want) < 1e-12
    assert np.abs(blk.imag).max() < 1e-12 * np.abs(want).max()
    np.testing.assert_array_equal(counts, [(bins == b).sum() for b in range(nb)])


def test_unsold_single_pair():
    # One primary and one secondary: zeta^0_ll(b,b) + 2 sum_{m>0} zeta^m_ll(b,b)
    # = w_i w_j^2 (2l+1)/4pi (Unsold), all other shells empty.
    lmax, nb = 10, 4
    pos = np.array([[5.0, 5.0, 5.0], [6.3, 4.1, 7.7]])
    w = np.array([0.7, 1.3])
    z, counts = oracle.zeta(pos, w, box=20.0, nbins=nb, rmin=0.0, rmax=4.0, lmax=lmax,
                            los_mode=0, n_primary=1)
    r = np.linalg.norm(pos[1] - pos[0])
    b = int(r // 1.0)
    assert counts.tolist() == [1 if k == b else 0 for k in range(nb)]
    blocks = oracle.zeta_blocks(z, nb, lmax)
    for l in range(lmax + 1):
        s = sum((1.0 if m == 0 else 2.0) * blocks[m][(l - m) * nb + b, (l - m) * nb + b].real
                for m in range(l + 1))
        assert abs(s - 0.7 * 1.3 ** 2 * (2 * l + 1) / FOURPI) < 1e-13


@pytest.mark.parametrize("los_mode", [0, 2])
def test_hermitian(los_mode):
    box, nb, lmax = 40.0, 4, 6
    pos, w = _cat(200, box, seed=41)
    z, _ = oracle.zeta(pos, w, box=box, nbins=nb, rmin=0.0, rmax=12.0, lmax=lmax, los_mode=los_mode)
    for blk in oracle.zeta_blocks(z, nb, lmax):
        assert np.abs(blk - blk.conj().T).max() < 1e-12 * np.abs(blk).max()


def _zeta(pos, w, **kw):
    return oracle.zeta(pos, w, **kw)


def test_periodic_quarter_turn_translation_and_reflection():
    # Lattice positions (multiples of 1/8) make every separation exact, so the
    # pair set is identical after each transform.
    box, nb, lmax = 32.0, 4, 6
    pos, w = _cat(250, box, seed=51, lattice=8)
    kw = dict(box=box, nbins=nb, rmin=0.0, rmax=10.0, lmax=lmax, los_mode=0)
    z, c = _zeta(pos, w, **kw)
    # quarter turn about z: (x, y) -> (y, -x) mod L; a_lm -> e^{-im pi/2} a_lm
    rot = np.stack([pos[:, 1], np.mod(-pos[:, 0], box), pos[:, 2]], axis=1)
    zr, cr = _zeta(rot, w, **kw)
    np.testing.assert_array_equal(c, cr)
    assert _maxrel(zr, z) < 1e-12
    # translation by an exactly representable shift
    tr = np.mod(pos + np.array([3.125, -7.5, 11.0]), box)
    zt, ct = _zeta(tr, w, **kw)
    np.testing.assert_array_equal(c, ct)
    assert _maxrel(zt, z) < 1e-12
    # point reflection: Y_lm(-r) = (-1)^l Y_lm(r) -> zeta^m_{ll'} * (-1)^(l+l')
    ref = np.mod(-pos, box)
    zf, cf = _zeta(ref, w, **kw)
    np.testing.assert_array_equal(c, cf)
    sign = []
    for m in range(lmax + 1):
        ls = np.repeat(np.arange(m, lmax + 1), nb)
        sign.append(np.outer((-1.0) ** ls, (-1.0) ** ls).ravel())
    sign = np.concatenate(sign)
    assert _maxrel(zf, sign * z) < 1e-12


def _rotz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])


def test_open_box_rotation_about_z_axis():
    # Any angle about the LOS (z) leaves zeta invariant (equal-m products).
    box, nb, lmax = 100.0, 4, 8
    rng = np.random.default_rng(61)
    n = 220
    rad = 40 * np.sqrt(rng.uniform(0, 1, n))
    ang = rng.uniform(0, 2 * np.pi, n)
    pos = np.stack([50 + rad * np.cos(ang), 50 + rad * np.sin(ang), rng.uniform(5, 95, n)], axis=1)
    w = rng.uniform(0.5, 1.5, n)
    kw = dict(box=box, nbins=nb, rmin=0.0, rmax=30.0, lmax=lmax, los_mode=1)
    z, c = _zeta(pos, w, **kw)
    R = _rotz(0.7)
    rot = (pos - 50.0) @ R.T + 50.0
    zr, cr = _zeta(rot, w, **kw)
    np.testing.assert_array_equal(c, cr)
    assert _maxrel(zr, z) < 1e-11


def test_radial_rotation_about_observer():
    # Radial LOS: a rigid rotation about the observer (box centre) rotates every
    # primary's LOS with it, so zeta is invariant.
    box, nb, lmax = 100.0, 4, 8
    rng = np.random.default_rng(71)
    n = 220
    v = rng.normal(size=(n, 3))
    v *= (45 * rng.uniform(0, 1, (n, 1)) ** (1 / 3)) / np.linalg.norm(v, axis=1, keepdims=True)
    pos = 50.0 + v
    w = rng.uniform(0.5, 1.5, n)
    kw = dict(box=box, nbins=nb, rmin=0.0, rmax=25.0, lmax=lmax, los_mode=2)
    z, c = _zeta(pos, w, **kw)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, cc, d = q
    R = np.array([[a * a + b * b - cc * cc - d * d, 2 * (b * cc - a * d), 2 * (b * d + a * cc)],
                  [2 * (b * cc + a * d), a * a - b * b + cc * cc - d * d, 2 * (cc * d - a * b)],
                  [2 * (b * d - a * cc), 2 * (cc * d + a * b), a * a - b * b - cc * cc + d * d]])
    rot = v @ R.T + 50.0
    zr, cr = _zeta(rot, w, **kw)
    np.testing.assert_array_equal(c, cr)
    assert _maxrel(zr, z) < 1e-11


def test_radial_frame_equals_explicit_rotation():
    # One primary, radial LOS: equal to the z-LOS result on separations that an
    # independent rotation (mapping the LOS to +z) has been applied to.
    box, nb, lmax = 100.0, 3, 6
    rng = np.random.default_rng(81)
    xi = np.array([71.0, 38.0, 22.0])
    sec = xi + rng.normal(size=(120, 3)) * 8.0
    pos = np.vstack([xi, sec])
    w = rng.uniform(0.5, 1.5, pos.shape[0])
    kw = dict(box=box, nbins=nb, rmin=0.0, rmax=20.0, lmax=lmax)
    z_rad, c_rad = oracle.zeta(pos, w, los_mode=2, n_primary=1, **kw)
    nhat = (xi - 50.0) / np.linalg.norm(xi - 50.0)
    # rotation taking nhat to z built from an orthonormal basis (e1, e2, nhat)
    e1 = np.cross(nhat, [1.0, 0.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(nhat, e1)
    R = np.stack([e1, e2, nhat])
    assert np.allclose(R @ nhat, [0, 0, 1])
    rsec = 50.0 + (sec - xi) @ R.T
    pos2 = np.vstack([[50.0, 50.0, 50.0], rsec])
    z_z, c_z = oracle.zeta(pos2, w, los_mode=1, n_primary=1, **kw)
    np.testing.assert_array_equal(c_rad, c_z)
    assert _maxrel(z_rad, z_z) < 1e-11


def test_half_open_bins_on_exact_lattice():
    # Integer lattice, edges at integers: r^2 and e^2 are exact, so the
    # half-open rule e_b^2 <= r^2 < e_{b+1}^2 can be checked in integers.
    box, nb = 16.0, 4
    g = np.arange(0, 16, 2.0)
    pos = np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).T.copy()
    w = np.ones(pos.shape[0])
    z, counts = oracle.zeta(pos, w, box=box, nbins=nb, rmin=2.0, rmax=6.0, lmax=0, los_mode=0)
    ip = pos.astype(np.int64)
    d = ip[None] - ip[:, None]
    d = d - 16 * np.round(d / 16).astype(np.int64)
    r2 = (d ** 2).sum(-1)
    want = [int(((r2 >= (2 + b) ** 2) & (r2 < (3 + b) ** 2)).sum()) for b in range(nb)]
    np.testing.assert_array_equal(counts, want)
    # r = 2 exactly belongs to bin 0; r = 6 exactly is excluded
    assert (r2 == 4).sum() > 0 and (r2 == 36).sum() > 0
    assert counts[0] == ((r2 >= 4) & (r2 < 9)).sum() >= (r2 == 4).sum()
    assert counts.sum() == ((r2 >= 4) & (r2 < 36)).sum()


def test_alm_and_zeta_agree():
    box, nb, lmax = 30.0, 3, 5
    pos, w = _cat(150, box, seed=91)
    kw = dict(box=box, nbins=nb, rmin=0.0, rmax=9.0, lmax=lmax, los_mode=0)
    z, counts = oracle.zeta(pos, w, **kw)
    a, c2 = oracle.alm(pos, w, np.arange(150), return_counts=True, **kw)
    np.testing.assert_array_equal(counts, c2)
    assert _maxrel(oracle.zeta_from_alm(a, w, nb, lmax), z) < 1e-13


def test_n_primary_subset_and_self_pair_exclusion():
    box, nb, lmax = 30.0, 3, 4
    pos, w = _cat(120, box, seed=101)
    pos[7] = pos[3]          # a coincident pair (r = 0) must be skipped
    kw = dict(box=box, nbins=nb, rmin=0.0, rmax=9.0, lmax=lmax, los_mode=0)
    z_sub, c_sub = oracle.zeta(pos, w, n_primary=40, **kw)
    a = oracle.alm(pos, w, np.arange(40), **kw)
    assert _maxrel(oracle.zeta_from_alm(a, w[:40], nb, lmax), z_sub) < 1e-13
    bins = _numpy_pairs(pos, box, True, oracle.edges2(nb, 0.0, 9.0))
    np.testing.assert_array_equal(c_sub, [(bins[:40] == b).sum() for b in range(nb)])
