"""CUDA-graph replay of the batched forward and the autotuner.

A captured graph runs the pair lists with passes planned on the device, so it
must reproduce a plain call bit for bit (the same per-primary lists and kernels;
every reduction has a fixed order), and the fused pair kernel within tolerance;
a replay after the input buffers were overwritten in place must compute the new
data, and data whose lists outgrow the captured pool fall back to an uncaptured
call.  The autotuner must return settings inside their ranges and leave
the plan producing the oracle's counts and zeta.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1709_00086_gb300 as g3  # noqa: E402
from paper_1709_00086_gb300 import catalogs  # noqa: E402

from gpu_util import maxrel, oracle_zeta, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


def _batch(seed):
    cats = catalogs.batched(ncat=5, seed=seed, sizes=[900, 3000, 50, 1800, 400], box=400.0)
    pos = np.concatenate([c.pos for c in cats])
    w = np.concatenate([c.w for c in cats])
    offs = np.cumsum([0] + [c.n for c in cats])
    return cats, pos, w, offs


@pytest.mark.parametrize("tc", [False, True])
def test_graph_replay_matches_plain_and_follows_new_data(tc):
    cats, pos, w, offs = _batch(9)
    plan = g3.Plan(**cats[0].params())
    dpos = torch.from_numpy(pos).cuda()
    dw = torch.from_numpy(w).cuda()
    plan.set_option(g3.OPT_PAIR_KERNELS, 1)
    zf, cf = plan.compute_batch(dpos, dw, offs, fp32_contraction=not tc)  # fused kernel
    plan.set_option(g3.OPT_PAIR_KERNELS, 0)
    z0, c0 = plan.compute_batch(dpos, dw, offs, fp32_contraction=not tc)  # pair lists
    assert torch.equal(cf, c0)
    assert maxrel(zf.cpu().numpy(), z0.cpu().numpy()) < (1e-4 if tc else 1e-5)
    zbuf = torch.empty((len(cats), plan.zsize, 2), dtype=torch.float64, device="cuda")
    cbuf = torch.empty((len(cats), plan.nbins), dtype=torch.int64, device="cuda")
    for _ in range(3):  # capture, then two replays
        z1, c1 = plan.compute_batch(dpos, dw, offs, fp32_contraction=not tc, graph=True,
                                    out=zbuf, counts_out=cbuf)
        assert torch.equal(z1, z0) and torch.equal(c1, c0)
    # new data in the same buffers: the replay computes it
    cats2, pos2, w2, _ = _batch(10)
    dpos.copy_(torch.from_numpy(pos2))
    dw.copy_(torch.from_numpy(w2))
    z2, c2 = plan.compute_batch(dpos, dw, offs, fp32_contraction=not tc, graph=True,
                                out=zbuf, counts_out=cbuf)
    for k, cat in enumerate(cats2):
        zo, co = oracle_zeta(cat)
        np.testing.assert_array_equal(c2[k].cpu().numpy(), co)
        if np.abs(zo).max() > 0:
            assert maxrel(z2[k].cpu().numpy(), zo) < (1e-4 if tc else 1e-5)


def test_graph_single_catalog_and_plain_call_drops_graph():
    cat = catalogs.small_case("clustered", 5000, seed=3, box=300.0, nbins=6, rmin=0.0, rmax=60.0,
                              lmax=6)
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    zb = torch.empty((plan.zsize, 2), dtype=torch.float64, device="cuda")
    cb = torch.empty(plan.nbins, dtype=torch.int64, device="cuda")
    za, ca = plan.compute(pos, w, n_primary=700, graph=True, out=zb, counts_out=cb)
    za = za.clone()
    zp, cp = plan.compute(pos, w, n_primary=300)  # a plain call in between
    zc, cc = plan.compute(pos, w, n_primary=700, graph=True, out=zb, counts_out=cb)
    assert torch.equal(za, zc)
    zo, co = oracle_zeta(cat, n_primary=700)
    np.testing.assert_array_equal(cc.cpu().numpy(), co)
    assert maxrel(zc.cpu().numpy(), zo) < 1e-4


def test_autotune_choices_and_result():
    cat = catalogs.clustered_2m(n=60000, seed=21, box=700.0)
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    best = plan.autotune(pos, w)
    assert 1 <= best["cells_per_rmax"] <= 8 and 2 <= best["kflush"] <= 16 and best["pair_us"] > 0
    z, c = plan.compute(pos, w, n_primary=300)
    zo, co = oracle_zeta(cat, n_primary=300)
    np.testing.assert_array_equal(c.cpu().numpy(), co)
    assert maxrel(z.cpu().numpy(), zo) < 1e-4


def test_autotune_cache_round_trip_and_tuned_parity(tmp_path):
    # the first tune times the sweep and appends its winner to the cache; a new
    # plan with the same shape and density reads it back without timing; a
    # tuned forward (and a batch over the tuned grid) still matches the oracle
    cat = catalogs.clustered_2m(n=60000, seed=23, box=700.0)
    cache = tmp_path / "tune.txt"
    pos, w = to_dev(cat, torch)
    p1 = g3.Plan(**cat.params())
    t1 = p1.autotune_cached(pos, w, cache)
    assert not t1["from_cache"] and t1["pair_us"] > 0
    assert 1 <= t1["cells_per_rmax"] <= 8 and t1["x_refine"] in (4, 8, 16) and t1["tc_operands"] in (0, 1)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1 and "nbins=10 lmax=10" in lines[0]
    p2 = g3.Plan(**cat.params())
    t2 = p2.autotune_cached(pos, w, cache)
    assert t2["from_cache"] and (t2["cells_per_rmax"], t2["x_refine"], t2["tc_operands"]) == (
        t1["cells_per_rmax"], t1["x_refine"], t1["tc_operands"])
    assert len(cache.read_text().strip().splitlines()) == 1
    z, c = p2.compute(pos, w, n_primary=300, fp32_contraction=True)
    zo, co = oracle_zeta(cat, n_primary=300)
    np.testing.assert_array_equal(c.cpu().numpy(), co)
    assert maxrel(z.cpu().numpy(), zo) < 1e-5
    # the tuned tensor-core forward, with the operand source the tuner kept
    ztc, ctc = p2.compute(pos, w, n_primary=300)
    assert p2.stats()["tc_operands_from_pairs"] == float(t1["tc_operands"])
    np.testing.assert_array_equal(ctc.cpu().numpy(), co)
    assert maxrel(ztc.cpu().numpy(), zo) < 1e-4
    # every x refinement and resolution the tuner may pick gives the same counts
    for s, x in ((max(1, t1["cells_per_rmax"] - 1), 4), (t1["cells_per_rmax"] + 1, 16)):
        p3 = g3.Plan(**cat.params())
        p3.set_option(g3.OPT_CELLS_PER_RMAX, min(s, 8))
        p3.set_option(g3.OPT_X_REFINE, x)
        _, c3 = p3.compute(pos, w, n_primary=300, fp32_contraction=True)
        np.testing.assert_array_equal(c3.cpu().numpy(), co)


def test_graph_replay_with_denser_data_falls_back():
    # capture on a catalog of scattered points, then overwrite the buffers with
    # a tightly clustered catalog of the same size: its lists outgrow the pool
    # planned at capture; the call must still return the right zeta
    n = 4000
    sparse = catalogs.small_case("uniform", n, seed=81, box=400.0, nbins=6, rmin=0.0, rmax=60.0, lmax=4)
    dense = catalogs.small_case("clustered", n, seed=82, box=400.0, nbins=6, rmin=0.0, rmax=60.0, lmax=4)
    dense.pos[:] = (dense.pos * 0.25).astype(dense.pos.dtype)  # everything in one corner
    plan = g3.Plan(**sparse.params())
    dpos, dw = to_dev(sparse, torch)
    zb = torch.empty((plan.zsize, 2), dtype=torch.float64, device="cuda")
    cb = torch.empty(plan.nbins, dtype=torch.int64, device="cuda")
    plan.compute(dpos, dw, graph=True, out=zb, counts_out=cb, fp32_contraction=True)
    dpos.copy_(torch.from_numpy(dense.pos))
    dw.copy_(torch.from_numpy(dense.w))
    z, c = plan.compute(dpos, dw, graph=True, out=zb, counts_out=cb, fp32_contraction=True)
    zo, co = oracle_zeta(dense)
    np.testing.assert_array_equal(c.cpu().numpy(), co)
    assert maxrel(z.cpu().numpy(), zo) < 1e-5
    # and the next graph call captures again and agrees
    z2, c2 = plan.compute(dpos, dw, graph=True, out=zb, counts_out=cb, fp32_contraction=True)
    assert torch.equal(c2, c) and maxrel(z2.cpu().numpy(), zo) < 1e-5
