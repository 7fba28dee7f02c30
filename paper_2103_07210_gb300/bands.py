"""Latitude-band split of one solve over ranks: partition, halo exchange and
the gather of per-tile partial sums.

The paper runs FT-GCR(k) over MPI processes, each holding a contiguous block
of the grid, with global reductions for the inner products (Section 3,
Section 4).  On the lat-lon grid the natural block is a band of whole latitude
rows:

- the line preconditioner couples only points of one row (Section 2, the
  bespoke left preconditioner), so every rank solves its own rows with no
  exchange;
- the 5-point operator reaches one row up and one row down, so L(e) on a band
  needs one halo row of e on each side that has a neighbour (the pole faces
  carry no flux and need none);
- the fault test, the exit test, beta and the alpha_l need the global inner
  products; every rank must reach the same decisions, so the per-tile partial
  sums are gathered in tile order rather than all-reduced, and every rank
  then reduces the same array in the same fixed order.

Bands are made of whole row tiles (the tiling a single-GPU solve of the same
grid uses), so the gathered array is exactly the one the single-GPU kernel
reduces, and a band-split solve reaches the single-GPU decisions.

This module holds the bookkeeping only (which rows and tiles a rank owns,
which rows it sends and receives, where gathered partials go), on whatever
device the tensors live (NCCL on GPUs, gloo on CPU).  It does no arithmetic of
the method.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch
import torch.distributed as dist


@dataclass(frozen=True)
class Band:
    """Rank `rank`'s share: row tiles [t0, t1) of height `tile_h`, i.e. rows
    [r0, r1) of the nlat rows; `below` / `above` are the ranks holding rows
    r0 - 1 and r1 (None at a pole)."""
    rank: int
    t0: int
    t1: int
    r0: int
    r1: int
    below: int | None
    above: int | None

    @property
    def rows(self) -> int:
        return self.r1 - self.r0

    @property
    def tiles(self) -> int:
        return self.t1 - self.t0


def n_tiles(nlat: int, tile_h: int) -> int:
    return -(-nlat // tile_h)


def partition(nlat: int, world: int, tile_h: int = 1) -> list[Band]:
    """Split the ceil(nlat / tile_h) row tiles into `world` contiguous bands
    whose tile counts differ by at most one (the first nt % world ranks take
    the extra tile).  The last tile may be short (nlat not a multiple of
    tile_h).  Raises ValueError when a rank would get no tile."""
    if nlat < 1 or world < 1 or tile_h < 1:
        raise ValueError("nlat, world and tile_h must be positive")
    nt = n_tiles(nlat, tile_h)
    if world > nt:
        raise ValueError(f"{world} ranks for {nt} row tiles: a rank would hold no rows")
    base, extra = divmod(nt, world)
    bands = []
    t0 = 0
    for q in range(world):
        t1 = t0 + base + (1 if q < extra else 0)
        bands.append(Band(q, t0, t1, t0 * tile_h, min(t1 * tile_h, nlat), q - 1 if q > 0 else None,
                          q + 1 if q + 1 < world else None))
        t0 = t1
    return bands


def padded(band: Band, nlon: int, dtype=torch.float64, device="cpu") -> torch.Tensor:
    """A rank's working array for a vector that needs halos: rows + 2 rows of
    nlon; row 0 holds global row r0 - 1, rows 1..rows the band's own rows, the
    last row global row r1.  Halo rows at a pole stay zero."""
    return torch.zeros(band.rows + 2, nlon, dtype=dtype, device=device)


def exchange_halos(buf: torch.Tensor, band: Band, group=None) -> None:
    """Fill buf's halo rows from the neighbouring ranks: send the first own
    row down and the last own row up, receive row r0 - 1 into row 0 and row r1
    into the last row.  Non-blocking sends and receives, then wait for all."""
    h = band.rows
    if buf.shape[0] != h + 2 or not buf.is_contiguous():
        raise ValueError("buf must be the contiguous (rows + 2) x nlon array of this band")
    reqs = []
    if band.below is not None:
        reqs.append(dist.isend(buf[1].contiguous(), band.below, group=group))
        reqs.append(dist.irecv(buf[0], band.below, group=group))
    if band.above is not None:
        reqs.append(dist.isend(buf[h].contiguous(), band.above, group=group))
        reqs.append(dist.irecv(buf[h + 1], band.above, group=group))
    for r in reqs:
        r.wait()


def gather_partials(local: torch.Tensor, bands: list[Band], rank: int, group=None) -> torch.Tensor:
    """All-gather every rank's per-tile partial sums, [its tiles, S], into the
    global [tiles, S] array in tile order (ranks padded to the largest band for
    the collective).  Every rank gets the same array."""
    me = bands[rank]
    if local.shape[0] != me.tiles:
        raise ValueError("local partials must have one row per tile of this band")
    mx = max(b.tiles for b in bands)
    S = local.shape[1]
    pad = torch.zeros(mx, S, dtype=local.dtype, device=local.device)
    pad[: me.tiles] = local
    got = [torch.empty_like(pad) for _ in bands]
    dist.all_gather(got, pad, group=group)
    return torch.cat([g[: b.tiles] for g, b in zip(got, bands)], dim=0)
