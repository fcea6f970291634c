"""The oracle's monomial route to a_lm (the paper's power sums, Sec. 3.3.2)
against the count the paper prints and against the library-based definition
(std::sph_legendre) of the multipoles.  CPU only."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "monomial_count.txt")


def _golden_counts():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                lmax, count = line.split()
                rows.append((int(lmax), int(count)))
    return rows


def test_monomial_count_printed_in_the_paper():
    rows = _golden_counts()
    assert rows == [(10, 286)]
    for lmax, count in rows:
        assert oracle.mono_count(lmax) == count


def test_monomial_count_closed_form():
    # brute-force enumeration of a + b + c <= l against (l+1)(l+2)(l+3)/6
    for lmax in range(0, 13):
        brute = sum(1 for a in range(lmax + 1) for b in range(lmax + 1) for c in range(lmax + 1)
                    if a + b + c <= lmax)
        assert oracle.mono_count(lmax) == brute == (lmax + 1) * (lmax + 2) * (lmax + 3) // 6


@pytest.mark.parametrize("los_mode", [0, 1, 2])
@pytest.mark.parametrize("lmax", [0, 3, 10])
def test_monomial_route_equals_spherical_harmonics(los_mode, lmax):
    # same pairs, bins and frame; the sums of w x^a y^b z^c converted to a_lm
    # agree with sum w Y_lm computed from std::sph_legendre
    rng = np.random.default_rng(81 + 3 * lmax + los_mode)
    pos = rng.uniform(0.0, 100.0, (500, 3))
    w = rng.uniform(0.5, 1.5, 500)
    prims = np.array([0, 7, 123, 499])
    a = oracle.alm(pos, w, prims, 100.0, 5, 3.0, 45.0, lmax, los_mode=los_mode)
    b = oracle.alm_monomial(pos, w, prims, 100.0, 5, 3.0, 45.0, lmax, los_mode=los_mode)
    assert np.abs(a).max() > 0
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_monomial_route_single_pair_is_ylm():
    # one secondary of weight 1 in bin 0: the converted sums are Y_lm(rhat)
    d = np.array([[0.3, -0.7, 0.4]])
    pos = np.vstack([np.zeros(3) + 50.0, 50.0 + d[0] * 10.0 / np.linalg.norm(d[0])])
    w = np.ones(2)
    b = oracle.alm_monomial(pos, w, [0], 100.0, 1, 5.0, 20.0, 10, los_mode=1)
    y = oracle.ylm(10, d)
    np.testing.assert_allclose(b[0, 0], y[0], rtol=0, atol=1e-13)
