"""Spatial sharding of one catalog over several processes (the paper's Sec. 3.2).

The paper distributes the galaxies over nodes with a k-d tree: the volume is
split recursively at the median of the widest dimension until there is one
region per node, each node receives the galaxies of its region (its
primaries) plus every galaxy within rmax of the region (its halo, the
secondaries it needs but does not own), computes the multipoles and zeta of
its own primaries, and the per-node zeta are summed at the end.  This module
holds that host-side logic:

* ``kd_regions``   -- the balanced k-d split of the points into axis-aligned
                      regions, one per rank (counts proportional to the ranks
                      on each side of a split, so any number of ranks works);
* ``halo_mask``    -- the points within rmax of a region (periodic images in a
                      periodic box);
* ``local_catalog``-- one rank's primaries followed by its halo;
* ``sharded_zeta`` -- the whole exchange over ``torch.distributed``: regions
                      from the gathered coordinates, the points each rank needs
                      sent to it (every rank contributes the points it holds),
                      the local forward with n_primary, and one FP64 sum
                      all-reduce of zeta plus an int64 one of the pair counts.

The local forward is a callable ``compute(pos, w, n_primary) -> (zeta, counts)``
(the library's ``Plan.compute`` on a GPU).  The halo is copied into each rank's
own memory before the forward: no kernel reads another device's memory.
"""
from __future__ import annotations

import numpy as np


def kd_regions(pos: np.ndarray, nparts: int, box: float):
    """Balanced k-d split of the points into nparts axis-aligned regions.

    Returns (lo, hi, owner): lo/hi (nparts, 3) region bounds, half-open
    [lo, hi) per axis and covering [0, box)^3 together, and owner (n,) the
    region of every point.  A region of k ranks is split across its widest
    axis at the coordinate that leaves round(n k_left / k) of its points on the
    left (k_left = k // 2); ties at the split coordinate all go right, so the
    owner is a pure function of the coordinate."""
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    lo = np.zeros((nparts, 3))
    hi = np.full((nparts, 3), float(box))
    owner = np.zeros(n, dtype=np.int64)

    def split(idx, r0, k, rlo, rhi):
        if k == 1:
            lo[r0], hi[r0] = rlo, rhi
            owner[idx] = r0
            return
        axis = int(np.argmax(rhi - rlo))
        kl = k // 2
        if idx.size == 0:
            cut = 0.5 * (rlo[axis] + rhi[axis])
        else:
            x = np.sort(pos[idx, axis])
            nl = int(round(idx.size * kl / k))
            cut = x[nl] if nl < idx.size else rhi[axis]
            cut = min(max(cut, rlo[axis]), rhi[axis])
        left = idx[pos[idx, axis] < cut]
        right = idx[pos[idx, axis] >= cut]
        llo, lhi = rlo.copy(), rhi.copy()
        lhi[axis] = cut
        rlo2, rhi2 = rlo.copy(), rhi.copy()
        rlo2[axis] = cut
        split(left, r0, kl, llo, lhi)
        split(right, r0 + kl, k - kl, rlo2, rhi2)

    split(np.arange(n), 0, int(nparts), np.zeros(3), np.full(3, float(box)))
    return lo, hi, owner


def _axis_gap(x, a, b, box, periodic):
    """Distance along one axis from coordinates x to the interval [a, b)."""
    d = np.maximum(np.maximum(a - x, x - b), 0.0)
    if periodic:  # the nearer periodic image of the interval
        d = np.minimum(d, np.maximum(np.maximum(a - (x - box), (x - box) - b), 0.0))
        d = np.minimum(d, np.maximum(np.maximum(a - (x + box), (x + box) - b), 0.0))
    return d


def halo_mask(pos: np.ndarray, lo, hi, rmax: float, box: float, periodic: bool) -> np.ndarray:
    """Points within rmax of the region [lo, hi) (minimum image in a periodic
    box); a conservative margin of 1e-9 rmax keeps points exactly at rmax."""
    pos = np.asarray(pos, dtype=np.float64)
    g2 = np.zeros(pos.shape[0])
    for a in range(3):
        g = _axis_gap(pos[:, a], lo[a], hi[a], box, periodic)
        g2 += g * g
    r = rmax * (1.0 + 1e-9)
    return g2 <= r * r


def local_catalog(pos, w, owner, rank: int, lo, hi, rmax: float, box: float, periodic: bool):
    """Rank's primaries (its region's points, in input order) followed by its
    halo: returns (pos, w, n_primary, index) with index the input positions."""
    own = np.nonzero(owner == rank)[0]
    halo = np.nonzero(halo_mask(pos, lo[rank], hi[rank], rmax, box, periodic) & (owner != rank))[0]
    idx = np.concatenate([own, halo])
    return (np.ascontiguousarray(np.asarray(pos)[idx]), np.ascontiguousarray(np.asarray(w)[idx]),
            int(own.size), idx)


def sharded_zeta(pos_local, w_local, compute, box: float, rmax: float, periodic: bool, group=None,
                 device="cpu"):
    """zeta and pair counts of the union of every rank's points, sharded by k-d region.

    pos_local / w_local: this rank's share of the catalog (numpy, any split of
    the points over the ranks).  compute(pos, w, n_primary) returns (zeta,
    counts) of the local catalog (complex zeta, int64 counts; numpy or torch).
    Steps: the coordinates are gathered to fix the regions (identical on every
    rank), every rank sends each other rank the points of its share that the
    other needs (its primaries and halo), the local forward runs with those
    primaries first, and zeta (FP64) and the counts (int64) are summed over the
    ranks.  Returns (zeta, counts) as numpy arrays, the same on every rank."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    pos_local = np.ascontiguousarray(pos_local, dtype=np.asarray(pos_local).dtype)
    w_local = np.ascontiguousarray(w_local, dtype=np.float32)
    shares = [None] * ws
    dist.all_gather_object(shares, pos_local.astype(np.float64), group=group)
    allpos = np.concatenate(shares) if ws > 0 else pos_local
    lo, hi, _ = kd_regions(allpos, ws, box)
    # what this rank sends to every rank r: its points owned by r, then its points in r's halo
    mine_owner = kd_owner(pos_local, lo, hi)
    out = []
    for r in range(ws):
        o = mine_owner == r
        h = halo_mask(pos_local, lo[r], hi[r], rmax, box, periodic) & ~o
        out.append((pos_local[o], w_local[o], pos_local[h], w_local[h]))
    recv = [None] * ws
    dist.all_gather_object(recv, out, group=group)
    parts = [recv[src][rank] for src in range(ws)]
    ppos = np.concatenate([p[0] for p in parts] + [p[2] for p in parts])
    pw = np.concatenate([p[1] for p in parts] + [p[3] for p in parts])
    npri = int(sum(p[0].shape[0] for p in parts))
    z, c = compute(np.ascontiguousarray(ppos), np.ascontiguousarray(pw), npri)
    z = torch.as_tensor(np.asarray(z.cpu() if hasattr(z, "cpu") else z))
    zr = torch.view_as_real(z.to(torch.complex128)).contiguous().to(device)
    cc = torch.as_tensor(np.asarray(c.cpu() if hasattr(c, "cpu") else c), dtype=torch.int64).to(device)
    dist.all_reduce(zr, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(cc, op=dist.ReduceOp.SUM, group=group)
    return torch.view_as_complex(zr.cpu()).numpy(), cc.cpu().numpy()


def kd_owner(pos, lo, hi) -> np.ndarray:
    """Region of every point for regions from kd_regions (half-open bounds)."""
    pos = np.asarray(pos, dtype=np.float64)
    inside = np.all((pos[:, None, :] >= lo[None]) & (pos[:, None, :] < hi[None]), axis=2)
    owner = np.argmax(inside, axis=1)
    if not np.all(inside.any(axis=1)):
        raise ValueError("a point lies outside every region (positions must be in [0, box))")
    return owner


def sharded_zeta_local(pos, w, nparts: int, compute, box: float, rmax: float, periodic: bool):
    """The same decomposition run in one process: every region's local forward in
    turn (no collective; the regions' results are summed on the host in rank
    order).  Returns (zeta, counts, npri) with npri the primaries per region."""
    pos = np.asarray(pos)
    lo, hi, owner = kd_regions(pos, nparts, box)
    zsum, csum, npri = None, None, []
    for r in range(nparts):
        lpos, lw, n_p, _ = local_catalog(pos, w, owner, r, lo, hi, rmax, box, periodic)
        z, c = compute(lpos, lw, n_p)
        z = np.asarray(z.cpu() if hasattr(z, "cpu") else z)
        c = np.asarray(c.cpu() if hasattr(c, "cpu") else c, dtype=np.int64)
        zsum = z.astype(np.complex128) if zsum is None else zsum + z
        csum = c.copy() if csum is None else csum + c
        npri.append(n_p)
    return zsum, csum, npri
