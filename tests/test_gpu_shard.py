"""Spatial sharding (the paper's Sec. 3.2) with the CUDA forward as the local
step: the k-d regions of a catalog, each forwarded with its primaries first
and its rmax halo after them (n_primary), one after another on this GPU, sum
to the zeta and pair counts of the whole catalog (oracle and the single
forward).  The multi-process exchange itself is covered on CPU ranks in
test_shard_gloo.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1709_00086_gb300 as g3  # noqa: E402
from paper_1709_00086_gb300 import catalogs, shard  # noqa: E402

from gpu_util import maxrel, oracle_zeta, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("los_mode,nparts", [(0, 2), (0, 4), (1, 3)])
def test_regions_sum_to_the_whole_catalog(los_mode, nparts):
    cat = catalogs.small_case("clustered", 6000, seed=95 + nparts, box=400.0, nbins=8, rmin=0.0,
                              rmax=80.0, lmax=6, los_mode=los_mode)
    plan = g3.Plan(**cat.params())

    def compute(p, w, npri):
        z, c = plan.compute(torch.from_numpy(p).cuda(), torch.from_numpy(w).cuda(), n_primary=npri,
                            fp32_contraction=True)
        return z.cpu().numpy(), c.cpu().numpy()

    z, c, npri = shard.sharded_zeta_local(cat.pos, cat.w, nparts, compute, cat.box, cat.rmax, los_mode == 0)
    assert sum(npri) == cat.n
    zo, co = oracle_zeta(cat)
    np.testing.assert_array_equal(c, co)
    assert maxrel(z, zo) < 1e-5
    zw, cw = plan.compute(*to_dev(cat, torch), fp32_contraction=True)
    np.testing.assert_array_equal(cw.cpu().numpy(), c)
