"""Both forward pair stages (fused bucket kernel; count / scan / accumulate
over pair lists) against the FP64 oracle, and the list path split into many
passes by a small list budget.  Counts bit-exact, zeta within 1e-5 of
max|zeta| (FP32 contraction), multipoles within 1e-5 of their largest entry.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1709_00086_gb300 as g3  # noqa: E402
from paper_1709_00086_gb300 import catalogs  # noqa: E402

from gpu_util import maxrel, oracle_alm, oracle_zeta, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = {
    # periodic, FP64 input, every point a primary
    "uniform_f64": lambda: catalogs.plain_uniform(n=2500, seed=41),
    # clustered, FP32 input, open box, LOS z
    "clustered_open": lambda: catalogs.small_case("clustered", 5000, seed=42, box=400.0, nbins=8,
                                                  rmin=5.0, rmax=90.0, lmax=8, los_mode=1),
    # radial LOS (rotation per primary)
    "clustered_radial": lambda: catalogs.small_case("clustered", 5000, seed=43, box=400.0, nbins=6,
                                                    rmin=0.0, rmax=80.0, lmax=10, los_mode=2),
    # many bins, low order
    "bins32": lambda: catalogs.small_case("uniform", 4000, seed=44, box=300.0, nbins=32,
                                          rmin=2.0, rmax=70.0, lmax=3, los_mode=0),
}


def _forward(cat, kernels, list_bytes=0, n_primary=None, keep_alm=False):
    plan = g3.Plan(**cat.params())
    plan.set_option(g3.OPT_PAIR_KERNELS, kernels)
    plan.set_option(g3.OPT_LIST_BYTES, list_bytes)
    pos, w = to_dev(cat, torch)
    z, c = plan.compute(pos, w, n_primary=n_primary, fp32_contraction=True, keep_alm=keep_alm)
    return plan, z.cpu().numpy(), c.cpu().numpy()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("kernels", [1, 2])
def test_pair_stage_matches_oracle(name, kernels):
    cat = CASES[name]()
    npri = min(cat.pos.shape[0], 600)
    plan, z, c = _forward(cat, kernels, n_primary=npri, keep_alm=True)
    zo, co = oracle_zeta(cat, n_primary=npri)
    np.testing.assert_array_equal(c, co)
    assert maxrel(z, zo) < TOL
    prims = np.array([0, 1, npri // 2, npri - 1])
    a = plan.alm(prims)
    ao = oracle_alm(cat, prims)
    for k in range(prims.size):
        assert maxrel(a[k], ao[k]) < TOL, k


def test_list_passes_bit_identical_to_one_pass():
    # 1 MiB of lists holds ~8,000 chunks: the 20,000-point clustered catalog
    # needs many passes; per-primary lists do not depend on the pass split
    cat = catalogs.clustered_2m(n=20000, seed=45, box=500.0)
    _, z1, c1 = _forward(cat, 2)
    _, zp, cp = _forward(cat, 2, list_bytes=1 << 20)
    np.testing.assert_array_equal(c1, cp)
    np.testing.assert_array_equal(z1, zp)


def test_list_and_fused_agree_on_counts_and_zeta():
    cat = catalogs.clustered_2m(n=20000, seed=46, box=500.0)
    _, zl, cl = _forward(cat, 2)
    _, zf, cf = _forward(cat, 1)
    np.testing.assert_array_equal(cl, cf)
    assert maxrel(zl, zf) < TOL


def test_list_path_batch_matches_single_calls():
    cats = catalogs.batched(ncat=3, seed=47, sizes=[3000, 1200, 2200], box=400.0)
    plan = g3.Plan(**cats[0].params())
    plan.set_option(g3.OPT_PAIR_KERNELS, 2)
    plan.set_option(g3.OPT_LIST_BYTES, 1 << 20)
    pos = torch.from_numpy(np.concatenate([c.pos for c in cats])).cuda()
    w = torch.from_numpy(np.concatenate([c.w for c in cats])).cuda()
    offs = np.cumsum([0] + [c.n for c in cats])
    zb, cb = plan.compute_batch(pos, w, offs, fp32_contraction=True)
    for k, cat in enumerate(cats):
        zo, co = oracle_zeta(cat)
        np.testing.assert_array_equal(cb[k].cpu().numpy(), co)
        assert maxrel(zb[k].cpu().numpy(), zo) < TOL, k


@pytest.mark.parametrize("name", ["uniform_f64", "clustered_radial", "bins32"])
def test_monomial_basis_matches_oracle(name):
    # the paper's monomial power sums (Sec. 3.3.2), FP64 accumulation and conversion
    cat = CASES[name]()
    npri = min(cat.pos.shape[0], 400)
    plan = g3.Plan(**cat.params())
    plan.set_option(g3.OPT_BASIS, 1)
    pos, w = to_dev(cat, torch)
    z, c = plan.compute(pos, w, n_primary=npri, fp32_contraction=True, keep_alm=True)
    zo, co = oracle_zeta(cat, n_primary=npri)
    np.testing.assert_array_equal(c.cpu().numpy(), co)
    assert maxrel(z.cpu().numpy(), zo) < TOL
    prims = np.array([0, npri // 3, npri - 1])
    a = plan.alm(prims)
    ao = oracle_alm(cat, prims)
    for k in range(prims.size):
        assert maxrel(a[k], ao[k]) < TOL, k


@pytest.mark.parametrize("name", ["uniform_f64", "clustered_open", "clustered_radial"])
@pytest.mark.parametrize("xref", [1, 3, 16])
def test_x_refinement_matches_oracle(name, xref):
    # cells 1, 3 or 16 times narrower along x than along y and z: the slot
    # ranges change, the pair decisions must not
    cat = CASES[name]()
    npri = min(cat.pos.shape[0], 500)
    plan = g3.Plan(**cat.params())
    plan.set_option(g3.OPT_X_REFINE, xref)
    pos, w = to_dev(cat, torch)
    z, c = plan.compute(pos, w, n_primary=npri, fp32_contraction=True)
    zo, co = oracle_zeta(cat, n_primary=npri)
    np.testing.assert_array_equal(c.cpu().numpy(), co)
    assert maxrel(z.cpu().numpy(), zo) < TOL


def test_cell_keys_at_their_limit():
    # 16 catalogs on a 256^3 grid (s = 8, rmax = box / 32): with the default x
    # refinement of 8 the cell keys would reach 2^31, so the grid takes a
    # coarser x step (16 * 256^3 * 4 cells, a 4.3 GB cell-start table)
    box, rmax = 1000.0, 31.25
    cats = []
    for c in range(16):
        rng = np.random.default_rng([49, c])
        pos = catalogs.uniform_positions(rng, 4000, box, np.float32)
        cats.append(catalogs.Catalog(pos, catalogs.weights(rng, 4000), box, 4, 2.0, rmax, 2, 0))
    plan = g3.Plan(**cats[0].params())
    plan.set_option(g3.OPT_CELLS_PER_RMAX, 8)
    pos = torch.from_numpy(np.concatenate([c.pos for c in cats])).cuda()
    w = torch.from_numpy(np.concatenate([c.w for c in cats])).cuda()
    offs = np.cumsum([0] + [c.n for c in cats])
    zb, cb = plan.compute_batch(pos, w, offs, fp32_contraction=True)
    assert plan.stats()["cells_per_rmax"] == 8.0
    for k in (0, 7, 15):
        zo, co = oracle_zeta(cats[k])
        np.testing.assert_array_equal(cb[k].cpu().numpy(), co)
        assert maxrel(zb[k].cpu().numpy(), zo) < TOL, k
