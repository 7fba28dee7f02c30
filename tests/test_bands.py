"""Latitude-band split bookkeeping (the paper's process blocks, Section 3) on
the CPU: the partition covers every row once in whole tiles; with gloo at
world sizes 2 and 3 the halo exchange delivers exactly the neighbours' rows,
so the operator on a halo-padded band reproduces the global operator's rows
and the row-local line preconditioner needs no exchange; and the gathered
per-tile partial sums are the single-process array, in tile order, on every
rank."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2103_07210_gb300 import bands  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("nlat,world,tile_h", [(32, 2, 4), (33, 2, 4), (7, 3, 1), (512, 4, 4), (37, 5, 3), (5, 5, 1)])
def test_partition_covers_each_row_once_in_whole_tiles(nlat, world, tile_h):
    bs = bands.partition(nlat, world, tile_h)
    nt = bands.n_tiles(nlat, tile_h)
    assert len(bs) == world and bs[0].r0 == 0 and bs[-1].r1 == nlat and bs[-1].t1 == nt
    for a, b in zip(bs, bs[1:]):
        assert a.t1 == b.t0 and a.r1 == b.r0 and a.above == b.rank and b.below == a.rank
    assert bs[0].below is None and bs[-1].above is None
    counts = [b.tiles for b in bs]
    assert min(counts) >= 1 and max(counts) - min(counts) <= 1
    for b in bs:
        assert b.r0 == b.t0 * tile_h and b.r1 == min(b.t1 * tile_h, nlat)


def test_partition_refuses_more_ranks_than_tiles():
    with pytest.raises(ValueError):
        bands.partition(8, 3, 4)
    with pytest.raises(ValueError):
        bands.partition(0, 1)


def _rank_main(rank, ws, port, nlon, nlat, tile_h, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2103_07210_gb300 import bands as B, inputs
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        e = inputs.uniform_pm1(5, (nlat, nlon))  # every rank draws the same global vector
        bs = B.partition(nlat, ws, tile_h)
        me = bs[rank]
        buf = B.padded(me, nlon)
        buf[1:me.rows + 1] = torch.from_numpy(e[me.r0:me.r1])
        B.exchange_halos(buf, me)
        # per-tile partials of a stand-in quantity (each tile's own sum of squares), S = 3 columns
        loc = torch.zeros(me.tiles, 3, dtype=torch.float64)
        for t in range(me.t0, me.t1):
            rows = e[t * tile_h:min((t + 1) * tile_h, nlat)]
            loc[t - me.t0] = torch.tensor([float((rows * rows).sum()), float(t), float(rank)], dtype=torch.float64)
        allp = B.gather_partials(loc, bs, rank)
        q.put((rank, buf.numpy().copy(), allp.numpy().copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,nlon,nlat,tile_h", [(2, 24, 13, 2), (3, 16, 20, 3), (2, 8, 2, 1)])
def test_band_split_with_gloo(ws, nlon, nlat, tile_h):
    import oracle
    from paper_2103_07210_gb300 import inputs
    ctx = torch.multiprocessing.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, nlon, nlat, tile_h, qu)) for r in range(ws)]
    for p in procs:
        p.start()
    got = dict((r, (b, a)) for r, b, a in (qu.get(timeout=180) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    e = inputs.uniform_pm1(5, (nlat, nlon))
    p = inputs.hill_problem(nlon, nlat)
    Le = oracle.apply_L(p.D, p.mu, e)
    Pe = oracle.solve_P(p.D, p.mu, e)
    bs = bands.partition(nlat, ws, tile_h)
    ref = np.array([[float((e[t * tile_h:min((t + 1) * tile_h, nlat)] ** 2).sum()), t,
                     next(b.rank for b in bs if b.t0 <= t < b.t1)] for t in range(bands.n_tiles(nlat, tile_h))])
    for b in bs:
        buf, allp = got[b.rank]
        # own rows untouched, halos are exactly the neighbours' boundary rows (zero at a pole)
        assert np.array_equal(buf[1:b.rows + 1], e[b.r0:b.r1])
        assert np.array_equal(buf[0], e[b.r0 - 1] if b.below is not None else np.zeros(nlon))
        assert np.array_equal(buf[-1], e[b.r1] if b.above is not None else np.zeros(nlon))
        # the padded band is all the operator needs: embedded alone, it gives the global rows bitwise
        emb = np.zeros_like(e)
        lo, hi = max(b.r0 - 1, 0), min(b.r1 + 1, nlat)
        emb[lo:hi] = buf[lo - b.r0 + 1:hi - b.r0 + 1]
        assert np.array_equal(oracle.apply_L(p.D, p.mu, emb)[b.r0:b.r1], Le[b.r0:b.r1])
        # the line preconditioner is row-local: own rows alone give the global rows
        own = np.zeros_like(e)
        own[b.r0:b.r1] = e[b.r0:b.r1]
        assert np.array_equal(oracle.solve_P(p.D, p.mu, own)[b.r0:b.r1], Pe[b.r0:b.r1])
        # every rank gathered the single-process per-tile array, in tile order
        assert np.array_equal(allp, ref)
