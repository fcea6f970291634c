"""Pins for the oracle's spherical harmonics and their gradient.

Y_lm enters the method through the multipole sum a_lm = sum_j Y_lm(rhat_j)
(Sec. 3.1); the paper does not fix a normalisation, so the oracle uses the
orthonormal, Condon-Shortley-phased harmonics.  These tests pin that choice to
closed forms, to SciPy, to a quadrature of the orthonormality relation and to
Unsold's theorem, and pin the ladder-operator gradient to finite differences.
"""
import numpy as np
import pytest

import oracle

FOURPI = 4.0 * np.pi


def _dirs(n, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, 3)) * rng.uniform(0.5, 50.0, size=(n, 1))


def test_closed_forms():
    d = _dirs(64)
    Y = oracle.ylm(2, d)
    r = np.linalg.norm(d, axis=1)
    ct = d[:, 2] / r
    st = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2) / r
    eiphi = (d[:, 0] + 1j * d[:, 1]) / np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
    np.testing.assert_allclose(Y[:, oracle.lm_index(0, 0)], 1 / np.sqrt(FOURPI), atol=1e-15)
    np.testing.assert_allclose(Y[:, oracle.lm_index(1, 0)], np.sqrt(3 / FOURPI) * ct, atol=1e-14)
    np.testing.assert_allclose(Y[:, oracle.lm_index(1, 1)], -np.sqrt(3 / (8 * np.pi)) * st * eiphi,
                               atol=1e-14)
    np.testing.assert_allclose(Y[:, oracle.lm_index(2, 2)],
                               0.25 * np.sqrt(15 / (2 * np.pi)) * st ** 2 * eiphi ** 2, atol=1e-14)
    np.testing.assert_allclose(Y[:, oracle.lm_index(2, 0)],
                               0.25 * np.sqrt(5 / np.pi) * (3 * ct ** 2 - 1), atol=1e-14)


def test_on_axis():
    # Y_lm(z) = delta_m0 sqrt((2l+1)/4pi); Y_lm(-z) = (-1)^l delta_m0 sqrt(...)
    lmax = 10
    for sgn in (1.0, -1.0):
        Y = oracle.ylm(lmax, [[0.0, 0.0, 3.0 * sgn]])[0]
        for l in range(lmax + 1):
            for m in range(l + 1):
                want = np.sqrt((2 * l + 1) / FOURPI) * (sgn ** l) if m == 0 else 0.0
                assert abs(Y[oracle.lm_index(l, m)] - want) < 1e-13


def test_against_scipy():
    special = pytest.importorskip("scipy.special")
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    lmax = 10
    d = _dirs(200, seed=3)
    Y = oracle.ylm(lmax, d)
    r = np.linalg.norm(d, axis=1)
    th = np.arccos(d[:, 2] / r)
    ph = np.arctan2(d[:, 1], d[:, 0])
    for l in range(lmax + 1):
        for m in range(l + 1):
            np.testing.assert_allclose(Y[:, oracle.lm_index(l, m)], special.sph_harm_y(l, m, th, ph),
                                       atol=1e-13)


def test_orthonormality_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi integrates band-limited
    # products exactly: int Y_lm conj(Y_l'm') dOmega = delta delta.
    lmax = 10
    nq = 2 * lmax + 2
    x, wq = np.polynomial.legendre.leggauss(nq)
    nphi = 2 * lmax + 3
    phi = 2 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1 - x ** 2)
    dirs = np.stack([np.outer(st, np.cos(phi)).ravel(), np.outer(st, np.sin(phi)).ravel(),
                     np.repeat(x, nphi)], axis=1)
    weights = np.repeat(wq, nphi) * (2 * np.pi / nphi)
    Y = oracle.ylm(lmax, dirs)
    gram = (Y.conj().T * weights) @ Y
    np.testing.assert_allclose(gram, np.eye(Y.shape[1]), atol=1e-12)


def test_unsold():
    lmax = 10
    Y = oracle.ylm(lmax, _dirs(50, seed=5))
    for l in range(lmax + 1):
        s = np.abs(Y[:, oracle.lm_index(l, 0)]) ** 2
        for m in range(1, l + 1):
            s = s + 2 * np.abs(Y[:, oracle.lm_index(l, m)]) ** 2
        np.testing.assert_allclose(s, (2 * l + 1) / FOURPI, rtol=1e-13)


def test_gradient_matches_finite_differences():
    lmax = 10
    d = _dirs(40, seed=7)
    G = oracle.ylm_grad(lmax, d)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1.0
        scale = np.linalg.norm(d, axis=1, keepdims=True)
        fd = (oracle.ylm(lmax, d + h * scale * e) - oracle.ylm(lmax, d - h * scale * e)) / (2 * h * scale)
        # gradient of a degree-0 homogeneous function scales as 1/r
        np.testing.assert_allclose(G[:, :, a] * scale, fd * scale, atol=2e-7)


def test_gradient_is_tangential():
    # Y_lm(d/|d|) is invariant under radial scaling: d . grad Y = 0.
    lmax = 10
    d = _dirs(30, seed=11)
    G = oracle.ylm_grad(lmax, d)
    radial = np.einsum("na,nka->nk", d.astype(complex), G)
    assert np.abs(radial).max() < 1e-12
