"""Parity of the CUDA forward path against the FP64 oracle.

Counts per bin must be bit-exact; zeta within 1e-5 of max|zeta| for the
FP32 path (pair stage FP32 + FP32 contraction) and 1e-4 for the split-BF16
tensor-core contraction; per-primary multipoles within 1e-5 of their largest
entry.  Sizes are chosen so the oracle finishes in seconds while the GPU path
still runs many warps, several candidate pieces per primary and ragged
bucket flushes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1709_00086_gb300 as g3  # noqa: E402
from paper_1709_00086_gb300 import catalogs  # noqa: E402

from gpu_util import maxrel, oracle_alm, oracle_zeta, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_TC = 1e-4


def _run(cat, n_primary=None, fp32=True, keep_alm=False):
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    z, c = plan.compute(pos, w, n_primary=n_primary, fp32_contraction=fp32, keep_alm=keep_alm)
    return plan, z.cpu().numpy(), c.cpu().numpy()


def test_uniform_fp64_positions_counts_and_zeta():
    # the plain-method recipe (uniform, periodic L=1000, FP64 positions, w=1,
    # Rmax=200, 10 bins, lmax=10) at N=3000
    cat = catalogs.plain_uniform(n=3000, seed=11)
    plan, z, c = _run(cat, keep_alm=True)
    zo, co = oracle_zeta(cat)
    np.testing.assert_array_equal(c, co)
    assert maxrel(z, zo) < TOL_FP32
    prims = np.array([0, 1, 17, 1234, 2999])
    a = plan.alm(prims)
    ao = oracle_alm(cat, prims)
    for k in range(prims.size):
        assert maxrel(a[k], ao[k]) < TOL_FP32, k


@pytest.mark.parametrize("tc", [False, True])
def test_clustered_fp32_subset_of_primaries(tc):
    # clustered recipe (60% uniform + sigma=5 blobs), FP32 positions, weights
    # U(0.5,1.5); 300 primaries against all 30,000 secondaries
    cat = catalogs.clustered_2m(n=30000, seed=12, box=600.0)
    npri = 300
    plan, z, c = _run(cat, n_primary=npri, fp32=not tc)
    zo, co = oracle_zeta(cat, n_primary=npri)
    np.testing.assert_array_equal(c, co)
    assert maxrel(z, zo) < (TOL_TC if tc else TOL_FP32)


def test_exact_edges_on_integer_lattice():
    # points on an integer lattice in FP32: many separations fall exactly on
    # bin edges (r = 2, 3, ... exactly); the half-open rule must match
    g = np.arange(0, 24, 1.0)
    pos = np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).T.astype(np.float32)
    rng = np.random.default_rng(3)
    w = rng.uniform(0.5, 1.5, pos.shape[0]).astype(np.float32)
    cat = catalogs.Catalog(pos, w, 24.0, 5, 1.0, 6.0, 4, 0)
    plan, z, c = _run(cat, n_primary=400)
    zo, co = oracle_zeta(cat, n_primary=400)
    np.testing.assert_array_equal(c, co)
    assert maxrel(z, zo) < TOL_FP32


@pytest.mark.parametrize("los_mode", [1, 2])
def test_open_box_z_and_radial(los_mode):
    cat = catalogs.small_case("clustered", 6000, seed=20 + los_mode, box=400.0, nbins=8,
                              rmin=5.0, rmax=90.0, lmax=8, los_mode=los_mode)
    plan, z, c = _run(cat, n_primary=600, keep_alm=True)
    zo, co = oracle_zeta(cat, n_primary=600)
    np.testing.assert_array_equal(c, co)
    assert maxrel(z, zo) < TOL_FP32
    if los_mode == 1:
        prims = np.array([3, 77, 599])
        a = plan.alm(prims)
        ao = oracle_alm(cat, prims)
        for k in range(prims.size):
            assert maxrel(a[k], ao[k]) < TOL_FP32


@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 33])
def test_tiny_catalogs(n):
    rng = np.random.default_rng(n)
    pos = rng.uniform(0, 10.0, size=(n, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, n).astype(np.float32)
    cat = catalogs.Catalog(pos, w, 10.0, 3, 0.0, 4.5, 3, 0)
    plan, z, c = _run(cat)
    zo, co = oracle_zeta(cat)
    np.testing.assert_array_equal(c, co)
    if np.abs(zo).max() == 0:
        assert np.abs(z).max() == 0
    else:
        assert maxrel(z, zo) < TOL_FP32


@pytest.mark.parametrize("nbins,lmax", [(1, 0), (1, 10), (32, 2), (7, 5), (32, 10)])
def test_degenerate_shapes(nbins, lmax):
    cat = catalogs.small_case("uniform", 1500, seed=nbins * 13 + lmax, box=100.0, nbins=nbins,
                              rmin=0.0, rmax=25.0, lmax=lmax)
    plan, z, c = _run(cat, n_primary=300)
    zo, co = oracle_zeta(cat, n_primary=300)
    np.testing.assert_array_equal(c, co)
    assert maxrel(z, zo) < TOL_FP32


def test_n_primary_zero_and_coincident_points():
    cat = catalogs.small_case("uniform", 500, seed=5, box=50.0, nbins=4, rmin=0.0, rmax=12.0, lmax=4)
    cat.pos[10] = cat.pos[3]
    cat.pos[11] = cat.pos[3]
    plan, z, c = _run(cat, n_primary=0)
    assert np.abs(z).max() == 0 and c.sum() == 0
    plan, z, c = _run(cat, n_primary=50)
    zo, co = oracle_zeta(cat, n_primary=50)
    np.testing.assert_array_equal(c, co)
    assert maxrel(z, zo) < TOL_FP32


def test_range_error_reported():
    cat = catalogs.small_case("uniform", 200, seed=7, box=50.0, nbins=4, rmin=0.0, rmax=12.0, lmax=2)
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    pos[5, 1] = 50.0  # == box: outside [0, box)
    with pytest.raises(g3.G3PCFError) as ei:
        plan.compute(pos, w)
    assert ei.value.name == "ERR_RANGE"
    pos[5, 1] = float("nan")
    with pytest.raises(g3.G3PCFError) as ei:
        plan.compute(pos, w)
    assert ei.value.name == "ERR_RANGE"
    # the plan stays usable
    pos[5, 1] = 1.0
    plan.compute(pos, w)


def test_deterministic_reruns():
    cat = catalogs.clustered_2m(n=20000, seed=8, box=500.0)
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    z1, c1 = plan.compute(pos, w, n_primary=2000)
    z2, c2 = plan.compute(pos, w, n_primary=2000)
    assert torch.equal(z1, z2) and torch.equal(c1, c2)


def test_batch_matches_single_catalog_calls():
    cats = catalogs.batched(ncat=5, seed=3, sizes=[1500, 400, 1200, 0, 900], box=400.0)
    plan = g3.Plan(**cats[0].params())
    pos = torch.from_numpy(np.concatenate([c.pos for c in cats])).cuda()
    w = torch.from_numpy(np.concatenate([c.w for c in cats])).cuda()
    offs = np.cumsum([0] + [c.n for c in cats])
    zb, cb = plan.compute_batch(pos, w, offs, fp32_contraction=True)
    for k, cat in enumerate(cats):
        zo, co = oracle_zeta(cat)
        np.testing.assert_array_equal(cb[k].cpu().numpy(), co)
        if np.abs(zo).max() == 0:
            assert torch.abs(zb[k]).max().item() == 0
        else:
            assert maxrel(zb[k].cpu().numpy(), zo) < TOL_FP32


def test_tc_contraction_multi_segment_matches_fp32():
    # 60,000 primaries: the tensor-core contraction runs 8 segments x all
    # tiles; it must agree with the plain-FP32 contraction of the same
    # multipoles to the split-BF16 tolerance.
    cat = catalogs.clustered_2m(n=60000, seed=14, box=700.0)
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    z32, c32 = plan.compute(pos, w, fp32_contraction=True)
    ztc, ctc = plan.compute(pos, w, fp32_contraction=False)
    assert torch.equal(c32, ctc)
    assert maxrel(ztc.cpu().numpy(), z32.cpu().numpy()) < TOL_TC


def test_batch_tensor_core_path():
    cats = catalogs.batched(ncat=4, seed=5, sizes=[700, 1300, 90, 1000], box=400.0)
    plan = g3.Plan(**cats[0].params())
    pos = torch.from_numpy(np.concatenate([c.pos for c in cats])).cuda()
    w = torch.from_numpy(np.concatenate([c.w for c in cats])).cuda()
    offs = np.cumsum([0] + [c.n for c in cats])
    zb, cb = plan.compute_batch(pos, w, offs, fp32_contraction=False)
    for k, cat in enumerate(cats):
        zo, co = oracle_zeta(cat)
        np.testing.assert_array_equal(cb[k].cpu().numpy(), co)
        assert maxrel(zb[k].cpu().numpy(), zo) < TOL_TC


def test_tc_operand_paths_bit_identical():
    # The bf16 operands written by the pair stage and those formed inside the
    # contraction kernel are the same numbers (the same FP32 row times the same
    # sqrt(w), split the same way), summed in the same order: zeta must agree
    # bit for bit, on one catalog over many segments and on a ragged batch.
    cat = catalogs.clustered_2m(n=60000, seed=21, box=700.0)
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    zc, cc = plan.compute(pos, w)
    assert plan.stats()["tc_operands_from_pairs"] == 0.0
    plan.set_option(g3.OPT_TC_OPERANDS, 1)
    zd, cd = plan.compute(pos, w)
    assert plan.stats()["tc_operands_from_pairs"] == 1.0
    assert torch.equal(cd, cc)
    assert torch.equal(zd, zc)
    plan.close()

    cats = catalogs.batched(ncat=5, seed=6, sizes=[700, 1300, 0, 90, 1000], box=400.0)
    plan = g3.Plan(**cats[0].params())
    pos = torch.from_numpy(np.concatenate([c.pos for c in cats])).cuda()
    w = torch.from_numpy(np.concatenate([c.w for c in cats])).cuda()
    offs = np.cumsum([0] + [c.n for c in cats])
    zc, _ = plan.compute_batch(pos, w, offs)
    plan.set_option(g3.OPT_TC_OPERANDS, 1)
    zd, _ = plan.compute_batch(pos, w, offs)
    assert plan.stats()["tc_operands_from_pairs"] == 1.0
    assert torch.equal(zd, zc)
    for k, c in enumerate(cats):
        zo, _ = oracle_zeta(c)
        if np.abs(zo).max() > 0:
            assert maxrel(zd[k].cpu().numpy(), zo) < TOL_TC
    plan.close()

    # FP64 positions and a subset of primaries (a ragged 1,111 of 4,000 points)
    cat = catalogs.small_case("uniform", 4000, seed=31, box=300.0, nbins=7, rmin=2.0, rmax=70.0, lmax=7,
                              dtype=np.float64)
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    zc, cc = plan.compute(pos, w, n_primary=1111)
    plan.set_option(g3.OPT_TC_OPERANDS, 1)
    zd, cd = plan.compute(pos, w, n_primary=1111)
    assert plan.stats()["tc_operands_from_pairs"] == 1.0
    assert torch.equal(cd, cc) and torch.equal(zd, zc)
    zo, co = oracle_zeta(cat, n_primary=1111)
    np.testing.assert_array_equal(cd.cpu().numpy(), co)
    assert maxrel(zd.cpu().numpy(), zo) < TOL_TC
    plan.close()


def test_tc_operands_fall_back_with_negative_weights():
    # data plus randoms at negative weight: the sqrt(w) operands cannot be formed,
    # so the contraction forms its own from the FP32 rows; zeta matches the oracle
    cat = catalogs.data_minus_randoms(catalogs.small_case("clustered", 1500, seed=9, box=400.0, nbins=6, rmin=5.0,
                                                          rmax=80.0, lmax=6),
                                      nrand_factor=2, seed=10)
    plan = g3.Plan(**cat.params())
    plan.set_option(g3.OPT_TC_OPERANDS, 1)
    pos, w = to_dev(cat, torch)
    z, c = plan.compute(pos, w)
    assert plan.stats()["tc_operands_from_pairs"] == 0.0
    zo, co = oracle_zeta(cat)
    np.testing.assert_array_equal(c.cpu().numpy(), co)
    assert maxrel(z.cpu().numpy(), zo) < TOL_TC
    plan.close()


@pytest.mark.parametrize("tc", [False, True])
def test_chunked_passes_match_single_pass(tc):
    # primaries processed in 5 chunks (multipoles of earlier chunks are
    # contracted and dropped) give the zeta of a single pass
    cat = catalogs.clustered_2m(n=30000, seed=15, box=600.0)
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    z1, c1 = plan.compute(pos, w, fp32_contraction=not tc)
    plan.set_option(g3.OPT_CHUNK_ROWS, 6400)
    z2, c2 = plan.compute(pos, w, fp32_contraction=not tc)
    assert torch.equal(c1, c2)
    # the FP32 form adds the same FP32 partial sums in both cases (1e-6); the
    # tensor-core form's FP32 accumulation runs in tensor memory follow the
    # segments, which differ between the two, so its sums round differently at
    # the 1e-6 level (both stay within 1e-4 of the FP64 oracle; a chunking
    # mistake would show at order one)
    assert maxrel(z2.cpu().numpy(), z1.cpu().numpy()) < (1e-5 if tc else 1e-6)
    with pytest.raises(g3.G3PCFError) as ei:
        plan.alm([0])
    assert ei.value.name == "ERR_STATE"
    # stage times of a chunked call are summed over its chunks: they add up to
    # the total, and the pair stage holds every list scan and accumulate
    st = plan.stats()
    parts = st["index_ms"] + st["pair_ms"] + st["contract_ms"] + st["reduce_ms"]
    assert abs(parts - st["total_ms"]) <= 0.02 * st["total_ms"] + 0.05
    assert st["pair_ms"] >= st["scan_ms"] + st["accum_ms"]
