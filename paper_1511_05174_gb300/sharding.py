"""Row-band sharding of one image over ranks, with the overlap-add halo exchange.

Every patch is an independent problem (Sec. II-B), so the patch grid of one
image splits over ranks without any exchange in the solve.  Only the
overlap-add of Sec. IV couples neighbouring patches: a pixel is the mean of
the synthesized patches that cover it, and near a band boundary those patches
belong to two ranks.  Here the grid's patch rows are cut into contiguous bands
(one per rank); each rank reconstructs the sub-image its band covers (the
library's own csp_reconstruct on those measurement rows: its patch grid is
exactly the band's patches), turns its band image back into per-pixel sums,
and adds the sums of the rows it shares with its neighbours -- the P - stride
halo rows of each boundary -- before dividing by the total coverage.  The halo
travels by torch.distributed point-to-point messages (gloo for host tensors,
NCCL for device tensors); nothing else crosses ranks.

Bands start on an even image row when the stride is even, so the Bayer phase of
a patch is the same in the band as in the whole image.
"""

from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def patch_origins(extent: int, P: int, stride: int) -> np.ndarray:
    """Patch origins along one axis: 0, s, 2s, ... <= extent - P, plus extent - P
    when the stride misses it (the library's grid)."""
    if extent < P:
        return np.zeros(0, np.int64)
    o = list(range(0, extent - P + 1, stride))
    if o[-1] != extent - P:
        o.append(extent - P)
    return np.asarray(o, np.int64)


def band_split(n_rows: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous ranges [iy0, iy1) of patch rows, one per rank, sizes differing
    by at most one (empty ranges when world > n_rows)."""
    q, r = divmod(n_rows, world)
    out, a = [], 0
    for k in range(world):
        b = a + q + (1 if k < r else 0)
        out.append((a, b))
        a = b
    return out


def band_image_rows(origins: np.ndarray, P: int, band: Tuple[int, int]) -> Tuple[int, int]:
    """Image rows [r0, r1) covered by the patch rows of `band`."""
    iy0, iy1 = band
    if iy1 <= iy0:
        return (0, 0)
    return int(origins[iy0]), int(origins[iy1 - 1]) + P


def row_coverage(origins: np.ndarray, P: int, band: Tuple[int, int], r0: int, r1: int) -> np.ndarray:
    """Number of the band's patch rows covering each image row of [r0, r1)."""
    cnt = np.zeros(r1 - r0, np.int64)
    for iy in range(*band):
        cnt[origins[iy] - r0:origins[iy] + P - r0] += 1
    return cnt


class BandPlan:
    """The band of one rank: its patch rows, the image rows it reconstructs, the
    halo rows it shares with the previous and the next rank, and the rows whose
    final values it owns (each shared row is owned by the lower rank)."""

    def __init__(self, H: int, P: int, stride: int, world: int, rank: int):
        self.origins = patch_origins(H, P, stride)
        self.bands = band_split(len(self.origins), world)
        self.rank, self.world, self.P, self.H = rank, world, P, H
        self.band = self.bands[rank]
        self.rows = band_image_rows(self.origins, P, self.band)
        self.row_count = row_coverage(self.origins, P, self.band, *self.rows) if self.rows[1] > self.rows[0] else \
            np.zeros(0, np.int64)
        prev = band_image_rows(self.origins, P, self.bands[rank - 1]) if rank > 0 else (0, 0)
        nxt = band_image_rows(self.origins, P, self.bands[rank + 1]) if rank + 1 < world else (0, 0)
        r0, r1 = self.rows
        # rows shared with the neighbours (absolute image rows)
        self.halo_prev = (r0, min(r1, prev[1])) if rank > 0 and prev[1] > r0 else (r0, r0)
        self.halo_next = (max(r0, nxt[0]), r1) if rank + 1 < world and nxt[1] > nxt[0] and nxt[0] < r1 else (r1, r1)
        # rows this rank writes to the final image: its rows minus those the previous rank owns
        self.own = (self.halo_prev[1], r1) if rank > 0 else (r0, r1)

    @property
    def n_patch_rows(self) -> int:
        return self.band[1] - self.band[0]


def band_sums(band_image: np.ndarray, plan: BandPlan, col_count: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Per-pixel sums over the band's patches and their coverage counts, from
    the band's overlap-add image (mean over the band's covering patches):
    sum = mean x count, count = row count x column count."""
    cnt = plan.row_count[:, None] * col_count[None, :]
    return band_image * cnt[None], np.broadcast_to(cnt[None], band_image.shape).astype(band_image.dtype)


def exchange_halos(sums, counts, plan: BandPlan, dist_mod=None):
    """Adds the neighbours' sums and counts on the shared halo rows (in place):
    each boundary's rows go both ways, so both ranks end with the whole image's
    totals there.  `sums` / `counts`: tensors [planes, rows, W] over the band's
    image rows.  The exchange order (send down, then up; the two ends of each
    boundary in opposite order) keeps blocking point-to-point messages from
    waiting on each other."""
    import torch.distributed as dist
    dist = dist_mod or dist
    r0 = plan.rows[0]
    lo = slice(plan.halo_prev[0] - r0, plan.halo_prev[1] - r0)
    hi = slice(plan.halo_next[0] - r0, plan.halo_next[1] - r0)
    has_prev = plan.halo_prev[1] > plan.halo_prev[0]
    has_next = plan.halo_next[1] > plan.halo_next[0]
    for t in (sums, counts):
        send_hi = t[:, hi, :].contiguous() if has_next else None
        send_lo = t[:, lo, :].contiguous() if has_prev else None
        recv_hi = send_hi.clone() if has_next else None
        recv_lo = send_lo.clone() if has_prev else None
        # step 1: rank r sends its next-boundary rows to r + 1, which receives them as its previous-boundary rows
        if plan.rank % 2 == 0:
            if has_next:
                dist.send(send_hi, plan.rank + 1)
                dist.recv(recv_hi, plan.rank + 1)
            if has_prev:
                dist.recv(recv_lo, plan.rank - 1)
                dist.send(send_lo, plan.rank - 1)
        else:
            if has_prev:
                dist.recv(recv_lo, plan.rank - 1)
                dist.send(send_lo, plan.rank - 1)
            if has_next:
                dist.send(send_hi, plan.rank + 1)
                dist.recv(recv_hi, plan.rank + 1)
        if has_next:
            t[:, hi, :] += recv_hi
        if has_prev:
            t[:, lo, :] += recv_lo
    return sums, counts


def finish_rows(sums, counts, plan: BandPlan):
    """Final pixel values of the rows this rank owns: total sum / total count
    (0 where nothing covers a pixel), as [planes, own rows, W]."""
    r0 = plan.rows[0]
    sl = slice(plan.own[0] - r0, plan.own[1] - r0)
    s, c = sums[:, sl, :], counts[:, sl, :]
    out = s / c.clamp_min(1)
    return out.masked_fill(c == 0, 0)
