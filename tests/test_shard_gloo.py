"""Spatial sharding (the paper's Sec. 3.2): k-d regions, rmax halos and the
final sum of zeta over ranks.  The host logic runs here on CPU: the partition
and halo are checked by brute force, and two gloo ranks -- each holding half
of a catalog, with the oracle as the local forward -- must reproduce the
oracle's zeta and pair counts of the whole catalog."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_1709_00086_gb300 import catalogs, shard  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case(los_mode):
    return catalogs.small_case("clustered", 700, seed=90 + los_mode, box=200.0, nbins=5, rmin=0.0,
                               rmax=45.0, lmax=4, los_mode=los_mode)


@pytest.mark.parametrize("nparts", [2, 3, 5])
@pytest.mark.parametrize("los_mode", [0, 1])
def test_kd_regions_own_every_point_once_and_halos_hold_every_secondary(nparts, los_mode):
    cat = _case(los_mode)
    pos = cat.pos.astype(np.float64)
    lo, hi, owner = shard.kd_regions(pos, nparts, cat.box)
    # regions tile the box and every point is owned by the region that contains it
    assert np.isclose(np.prod(hi - lo, axis=1).sum(), cat.box ** 3)
    np.testing.assert_array_equal(shard.kd_owner(pos, lo, hi), owner)
    counts = np.bincount(owner, minlength=nparts)
    assert counts.sum() == cat.n and counts.max() - counts.min() <= nparts  # balanced
    e2 = oracle.edges2(cat.nbins, cat.rmin, cat.rmax)
    for r in range(nparts):
        lpos, lw, npri, idx = shard.local_catalog(pos, cat.w, owner, r, lo, hi, cat.rmax, cat.box,
                                                  los_mode == 0)
        assert npri == counts[r] and np.all(owner[idx[:npri]] == r)
        have = set(idx.tolist())
        for i in idx[:npri]:  # brute force: every accepted secondary of a primary is present
            d = pos - pos[i]
            if los_mode == 0:
                d -= cat.box * np.round(d / cat.box)
            r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
            js = np.nonzero((r2 > 0) & (r2 >= e2[0]) & (r2 < e2[-1]))[0]
            assert have.issuperset(js.tolist())


def _rank(rank, ws, port, los_mode, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    cat = _case(los_mode)
    mine = np.arange(rank, cat.n, ws)  # an arbitrary initial split of the points

    def compute(p, w, npri):
        return oracle.zeta(p.astype(np.float64), w.astype(np.float64), cat.box, cat.nbins, cat.rmin,
                           cat.rmax, cat.lmax, los_mode=los_mode, n_primary=npri, nthreads=1)

    z, c = shard.sharded_zeta(cat.pos[mine], cat.w[mine], compute, cat.box, cat.rmax, los_mode == 0)
    out[rank] = (z, c)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("los_mode", [0, 1])
def test_two_ranks_reproduce_the_whole_catalog(los_mode):
    ws = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, _free_port(), los_mode, out), nprocs=ws, join=True)
        res = dict(out)
    cat = _case(los_mode)
    zo, co = oracle.zeta(cat.pos.astype(np.float64), cat.w.astype(np.float64), cat.box, cat.nbins,
                         cat.rmin, cat.rmax, cat.lmax, los_mode=los_mode)
    for r in range(ws):
        z, c = res[r]
        np.testing.assert_array_equal(c, co)
        assert np.abs(z - zo).max() <= 1e-12 * np.abs(zo).max()
