"""Row-band sharding of one image with the overlap-add halo exchange, on CPU
gloo ranks (127.0.0.1).

Each rank reconstructs only the sub-image its band of patch rows covers (here
with the FP64 oracle standing in for the per-rank GPU solve: what is tested is
the band split and the halo sum), then the ranks add their sums on the shared
halo rows; the assembled image must equal the single-image overlap-add of the
oracle's codes (Sec. IV: every pixel is the mean of the patches that cover it)."""

import copy
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1511_05174_gb300 import sharding  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _band_workload(w, plan):
    """The sub-problem of one band: the measurement rows it covers, its patches."""
    g = w.geometry
    r0, r1 = plan.rows
    nx = len(sharding.patch_origins(g.W, g.P, g.stride))
    sub = copy.copy(w)
    sub.geometry = copy.copy(g)
    sub.geometry.H = r1 - r0
    sub.meas = w.meas[r0:r1] if w.meas.ndim == 2 else w.meas[:, r0:r1]
    sub.truth = w.truth[:, r0:r1]
    iy0, iy1 = plan.band
    sub.K_levels = [k[iy0 * nx:iy1 * nx] for k in w.K_levels]
    return sub


def _make(name, H, W, stride):
    import synthetic
    w = synthetic.make_workload(name, H=H, W=W, links="model")
    w.geometry.stride = stride
    B = w.n_patches
    w.K_levels = [np.full(B, int(k[0]), np.int32) for k in w.K_levels]
    return w


def _worker(rank, world, port, spec, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1511_05174_gb300 import sharding as sh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _make(*spec)
        g = w.geometry
        plan = sh.BandPlan(g.H, g.P, g.stride, world, rank)
        ox = sh.patch_origins(g.W, g.P, g.stride)
        col_count = np.zeros(g.W, np.int64)
        for x in ox:
            col_count[x:x + g.P] += 1
        sub = _band_workload(w, plan)
        assert sub.n_patches == plan.n_patch_rows * len(ox)
        o, a, k, _ = oracle.cross_scale_omp(sub, nthreads=1)
        band_img = oracle.aggregate(sub, o, a, k)
        s, c = sh.band_sums(band_img, plan, col_count)
        s, c = torch.from_numpy(np.ascontiguousarray(s)), torch.from_numpy(np.ascontiguousarray(c))
        sh.exchange_halos(s, c, plan)
        rows = sh.finish_rows(s, c, plan)
        q.put((rank, plan.own, rows.numpy(), plan.halo_prev, plan.halo_next))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("spec,world", [
    (("bayer", 64, 48, 2), 2),     # Bayer RGGB, stride 2: 6-row halos
    (("denoise", 64, 40, 3), 3),   # ragged: the last origin is clamped to H - P
])
def test_band_sharded_overlap_add_equals_single_image(spec, world):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, spec, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = _make(*spec)
    g = w.geometry
    o, a, k, _ = oracle.cross_scale_omp(w, nthreads=1)
    ref = oracle.aggregate(w, o, a, k)
    img = np.full_like(ref, np.nan)
    P, s = g.P, g.stride
    for rank, own, rows, hp, hn in out:
        img[:, own[0]:own[1]] = rows
        if rank > 0:
            assert hp[1] - hp[0] == P - s  # the halo of an interior boundary: P - stride rows
    assert np.isfinite(img).all()       # the owned rows tile the image
    np.testing.assert_allclose(img, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_band_plan_covers_every_patch_row_once():
    for H, P, st, world in [(512, 8, 2, 8), (64, 8, 3, 3), (40, 8, 8, 4), (16, 8, 4, 5)]:
        plans = [sharding.BandPlan(H, P, st, world, r) for r in range(world)]
        origins = sharding.patch_origins(H, P, st)
        rows = [i for p in plans for i in range(*p.band)]
        assert rows == list(range(len(origins)))
        owned = [y for p in plans if p.n_patch_rows for y in range(*p.own)]
        assert owned == list(range(H))
