"""Isotropic Legendre 3PCF (g3pcf_isotropic, Sec. 2.2 via the addition
theorem) against the oracle's brute-force triplet sum
(2l+1)/(4 pi) sum_i w_i sum_{j in b1, k in b2} w_j w_k P_l(rhat_ij . rhat_ik),
and D - R style catalogs (data plus randoms with negative weights, Sec. 6)
through the forward path.  Tolerance 1e-5 of the largest entry (FP32 path)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1709_00086_gb300 as g3  # noqa: E402
from paper_1709_00086_gb300 import catalogs  # noqa: E402

from gpu_util import maxrel, oracle_zeta, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.mark.parametrize("los_mode", [0, 1, 2])
def test_isotropic_matches_triplet_sum(los_mode):
    cat = catalogs.small_case("clustered", 160, seed=70 + los_mode, box=60.0, nbins=4, rmin=2.0,
                              rmax=25.0, lmax=6, los_mode=los_mode, dtype=np.float64)
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    z, _ = plan.compute(pos, w, fp32_contraction=True)
    iso = g3.isotropic(z, cat.nbins, cat.lmax).cpu().numpy()
    ref = oracle.iso_legendre(cat.pos.astype(np.float64), cat.w.astype(np.float64), cat.box,
                              cat.nbins, cat.rmin, cat.rmax, cat.lmax, los_mode=los_mode)
    assert iso.shape == (cat.lmax + 1, cat.nbins, cat.nbins)
    assert maxrel(iso, ref) < TOL


def test_isotropic_batch_layout_and_lmax10():
    cats = catalogs.batched(ncat=3, seed=73, sizes=[700, 0, 1200], box=400.0)
    plan = g3.Plan(**cats[0].params())
    pos = torch.from_numpy(np.concatenate([c.pos for c in cats])).cuda()
    w = torch.from_numpy(np.concatenate([c.w for c in cats])).cuda()
    offs = np.cumsum([0] + [c.n for c in cats])
    zb, _ = plan.compute_batch(pos, w, offs, fp32_contraction=True)
    iso = g3.isotropic(zb, plan.nbins, plan.lmax).cpu().numpy()
    assert iso.shape == (3, plan.lmax + 1, plan.nbins, plan.nbins)
    for k, cat in enumerate(cats):
        zo, _ = oracle_zeta(cat)
        blocks = oracle.zeta_blocks(zo, cat.nbins, cat.lmax)
        ref = np.zeros((cat.lmax + 1, cat.nbins, cat.nbins))
        for l in range(cat.lmax + 1):
            for m in range(l + 1):
                r0 = (l - m) * cat.nbins
                ref[l] += (1.0 if m == 0 else 2.0) * blocks[m][r0:r0 + cat.nbins, r0:r0 + cat.nbins].real
        if np.abs(ref).max() == 0:
            assert np.abs(iso[k]).max() == 0
        else:
            assert maxrel(iso[k], ref) < TOL, k


@pytest.mark.parametrize("tc", [False, True])
def test_data_minus_randoms_catalog(tc):
    cat = catalogs.data_minus_randoms(catalogs.small_case("clustered", 3000, seed=75, box=400.0,
                                                          nbins=8, rmin=5.0, rmax=90.0, lmax=8,
                                                          los_mode=1),
                                      nrand_factor=2, seed=76)
    assert (cat.w < 0).any() and abs(float(cat.w.sum())) < 1e-2 * float(np.abs(cat.w).sum())
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    z, c = plan.compute(pos, w, n_primary=1500, fp32_contraction=not tc)
    zo, co = oracle_zeta(cat, n_primary=1500)
    np.testing.assert_array_equal(c.cpu().numpy(), co)
    assert maxrel(z.cpu().numpy(), zo) < (1e-4 if tc else TOL)
