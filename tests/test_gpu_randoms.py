"""Many random catalogs in one batched forward (the random-catalog correction
of the paper's Sec. 6): a batch of D - R_k catalogs (the data with the k-th
random catalog at negative weight) and of the randoms R_k, combined on the
device by g3pcf_zeta_combine into the mean zeta of the D - R field and of the
randoms, against the oracle's zeta of every catalog averaged on the host.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1709_00086_gb300 as g3  # noqa: E402
from paper_1709_00086_gb300 import catalogs  # noqa: E402

from gpu_util import maxrel, oracle_zeta  # noqa: E402

pytestmark = pytest.mark.gpu
N_R = 4


@pytest.mark.parametrize("fp32,tol", [(True, 1e-5), (False, 1e-4)])
def test_many_random_catalogs_combined_on_device(fp32, tol):
    data = catalogs.small_case("clustered", 1200, seed=81, box=300.0, nbins=6, rmin=0.0, rmax=60.0,
                               lmax=5)
    dr, rr = catalogs.random_catalogs(data, N_R, nrand_factor=2, seed=82)
    cats = dr + rr
    plan = g3.Plan(**data.params())
    pos = torch.from_numpy(np.concatenate([c.pos for c in cats])).cuda()
    w = torch.from_numpy(np.concatenate([c.w for c in cats])).cuda()
    offs = np.cumsum([0] + [c.n for c in cats])
    zb, cb = plan.compute_batch(pos, w, offs, fp32_contraction=fp32)
    z_n = g3.zeta_combine(zb[:N_R], [1.0 / N_R] * N_R, data.nbins, data.lmax).cpu().numpy()
    z_r = g3.zeta_combine(zb[N_R:], [1.0 / N_R] * N_R, data.nbins, data.lmax).cpu().numpy()
    ref = [oracle_zeta(c) for c in cats]
    for k, (zo, co) in enumerate(ref):
        np.testing.assert_array_equal(cb[k].cpu().numpy(), co)
    zn_ref = np.mean([zo for zo, _ in ref[:N_R]], axis=0)
    zr_ref = np.mean([zo for zo, _ in ref[N_R:]], axis=0)
    assert maxrel(z_n, zn_ref) < tol
    assert maxrel(z_r, zr_ref) < tol
    # the combination itself is a fixed-order FP64 sum of the blocks
    zbn = zb.cpu().numpy()
    assert np.abs(z_n - zbn[:N_R].sum(0) / N_R).max() <= 1e-14 * np.abs(zbn[:N_R]).max()


def test_zeta_combine_weights_and_reruns():
    # arbitrary coefficients, one catalog, and bit-identical reruns
    rng = np.random.default_rng(3)
    nb, L = 4, 3
    zs = g3.zeta_size(nb, L)
    zb = torch.from_numpy(rng.normal(size=(5, zs, 2))).cuda()
    coef = rng.normal(size=5)
    out = g3.zeta_combine(zb, coef, nb, L).cpu().numpy()
    ref = np.tensordot(coef, zb.cpu().numpy()[..., 0] + 1j * zb.cpu().numpy()[..., 1], axes=1)
    assert np.abs(out - ref).max() <= 1e-14 * np.abs(ref).max()
    again = g3.zeta_combine(zb, coef, nb, L).cpu().numpy()
    assert np.array_equal(out, again)
    one = g3.zeta_combine(zb[2:3], [2.0], nb, L).cpu().numpy()
    assert np.array_equal(one, 2.0 * (zb.cpu().numpy()[2, :, 0] + 1j * zb.cpu().numpy()[2, :, 1]))
