"""Serving engine (continuous batching): a job's image through the server equals
the same image reconstructed alone through a Context, whatever batch it
shares; admission by the memory budget, timeouts and job bookkeeping."""

import numpy as np
import pytest

import synthetic
from paper_1511_05174_gb300 import _binding as b
from paper_1511_05174_gb300.server import Server

from _gpu_util import run_gpu

pytestmark = pytest.mark.gpu


def _w(name, H, W, seed=0, **kw):
    # every image of a model shares its dictionaries and links (dict_seed 0)
    return synthetic.make_workload(name, seed=seed, H=H, W=W, dict_seed=0, **kw)


def _alone(w, mode, prec):
    r = run_gpu(w, mode, prec)
    r["ctx"].close()
    return r["img"].astype(np.float32)


def _codes(w):
    return w.sensing.codes if w.sensing.kind == "coded_exposure" else None


@pytest.mark.parametrize("name,kw,prec", [
    ("denoise", dict(), "fp32"),
    ("bayer", dict(), "bf16"),
    ("video", dict(T0=1024), "fp32"),
])
def test_mixed_batch_equals_alone(name, kw, prec):
    # jobs of one model with different extents and contents, submitted in a burst
    sizes = [(64, 64), (48, 56), (64, 80), (40, 40), (56, 64), (64, 64)]
    ws = [_w(name, H, W, seed=10 + i, **kw) for i, (H, W) in enumerate(sizes)]
    with Server(0, n_streams=2) as srv:
        mid = srv.add_workload_model(ws[0], "cross_scale", prec)
        ids = [srv.submit(mid, w.meas, w.geometry.H, w.geometry.W, codes=_codes(w)) for w in ws]
        imgs = [srv.result(j, timeout_s=60) for j in ids]
        infos = [srv.info(j) for j in ids]
    for w, img, info in zip(ws, imgs, infos):
        ref = _alone(w, "cross_scale", prec)
        assert np.array_equal(img, ref), (w.geometry.H, w.geometry.W, info)
        assert info["status"] == b.CSP_OK
        assert info["patches"] == w.n_patches
        assert info["batch_patches"] >= info["patches"] and info["batch_jobs"] >= 1
        assert info["t_submit"] <= info["t_admit"] <= info["t_done"]
        # stage times: the per-patch operator builds are part of the solve, and
        # only coded-exposure jobs have them
        assert 0.0 <= info["build_ms"] <= info["solve_ms"] + 1e-3
        assert (info["build_ms"] > 0.0) == (name == "video")


def test_video_job_in_slices_equals_alone():
    # 3,969 patches with ~350 KB of per-patch operators each: the server builds
    # them for one 512 MiB slice (~1,500 patches) at a time
    w = _w("video", 256, 256, seed=3, T0=1024)
    with Server(0, mem_budget_bytes=1 << 30) as srv:
        mid = srv.add_workload_model(w, "cross_scale", "fp32")
        j = srv.submit(mid, w.meas, 256, 256, codes=w.sensing.codes)
        img = srv.result(j, 120).copy()
        info = srv.info(j)
    assert np.array_equal(img, _alone(w, "cross_scale", "fp32"))
    assert 0.0 < info["build_ms"] <= info["solve_ms"] + 1e-3  # every slice's build counted


def test_two_models_interleaved():
    wd = [_w("denoise", 64, 64, seed=s) for s in (1, 2, 3)]
    wb = [_w("bayer", 64, 64, seed=s) for s in (4, 5, 6)]
    with Server(0, n_streams=3) as srv:
        md = srv.add_workload_model(wd[0], "plain", "fp32")
        mb = srv.add_workload_model(wb[0], "cross_scale", "fp32")
        jobs = []
        for x, y in zip(wd, wb):
            jobs.append((x, "plain", srv.submit(md, x.meas, 64, 64)))
            jobs.append((y, "cross_scale", srv.submit(mb, y.meas, 64, 64)))
        out = [(w, mode, srv.result(j, 60).copy()) for w, mode, j in jobs]
    for w, mode, img in out:
        assert np.array_equal(img, _alone(w, mode, "fp32"))


def test_burst_is_coalesced():
    small = [_w("bayer", 64, 64, seed=20 + i) for i in range(8)]
    with Server(0, n_streams=1) as srv:
        mid = srv.add_workload_model(small[0], "cross_scale", "bf16")
        srv.pause(True)
        ids = [srv.submit(mid, w.meas, 64, 64) for w in small]
        assert not any(srv.poll(j) for j in ids)
        srv.pause(False)
        for j in ids:
            assert srv.wait(j, 60) == b.CSP_OK
        infos = [srv.info(j) for j in ids]
        imgs = [srv.result(j).copy() for j in ids]
    # queued together, admitted together: one batch, one solve
    assert all(i["batch_jobs"] == 8 for i in infos)
    assert all(i["batch_patches"] == sum(w.n_patches for w in small) for i in infos)
    for w, img in zip(small, imgs):
        assert np.array_equal(img, _alone(w, "cross_scale", "bf16"))


def test_max_batch_splits_burst():
    small = [_w("denoise", 64, 64, seed=40 + i) for i in range(4)]
    B1 = small[0].n_patches
    with Server(0, n_streams=1, max_batch_patches=2 * B1) as srv:
        mid = srv.add_workload_model(small[0], "cross_scale", "fp32")
        srv.pause(True)
        ids = [srv.submit(mid, w.meas, 64, 64) for w in small]
        srv.pause(False)
        infos = [srv.info(j) for j in ids if srv.wait(j, 60) == b.CSP_OK]
    assert len(infos) == 4
    assert all(i["batch_jobs"] == 2 and i["batch_patches"] == 2 * B1 for i in infos)


def test_budget_rejects_oversized_job():
    w = _w("bayer", 512, 512)
    with Server(0, mem_budget_bytes=1 << 20) as srv:
        mid = srv.add_workload_model(w, "cross_scale", "fp32")
        with pytest.raises(b.CspError) as e:
            srv.submit(mid, w.meas, 512, 512)
        assert e.value.status == b.CSP_ERR_OOM
        small = _w("bayer", 16, 16)
        j = srv.submit(mid, small.meas, 16, 16)
        assert srv.wait(j, 60) == b.CSP_OK


def test_budget_serialises_jobs():
    # a budget that holds one 256x256 Bayer job (about 45 MB) at a time
    ws = [_w("bayer", 256, 256, seed=30 + i) for i in range(3)]
    with Server(0, mem_budget_bytes=64 << 20, n_streams=4) as srv:
        mid = srv.add_workload_model(ws[0], "cross_scale", "fp32")
        srv.pause(True)
        ids = [srv.submit(mid, w.meas, 256, 256) for w in ws]
        srv.pause(False)
        imgs = [srv.result(j, 60).copy() for j in ids]
        infos = [srv.info(j) for j in ids]
    assert all(i["status"] == b.CSP_OK and i["batch_jobs"] == 1 for i in infos)
    for k in range(1, 3):  # admitted only after the previous job released its memory
        assert infos[k]["t_admit"] >= infos[k - 1]["t_done"]
    for w, img in zip(ws, imgs):
        assert np.array_equal(img, _alone(w, "cross_scale", "fp32"))


def test_wait_timeout_poll_and_release():
    w = _w("denoise", 64, 64)
    with Server(0) as srv:
        mid = srv.add_workload_model(w, "cross_scale", "fp32")
        srv.pause(True)
        j = srv.submit(mid, w.meas, 64, 64)
        assert not srv.poll(j)
        assert srv.wait(j, 0.01) == b.CSP_ERR_TIMEOUT
        assert srv.info(j)["status"] == b.CSP_ERR_NOT_READY
        with pytest.raises(b.CspError) as e:
            srv.release(j)
        assert e.value.status == b.CSP_ERR_NOT_READY
        srv.pause(False)
        assert srv.wait(j, 60) == b.CSP_OK and srv.poll(j)
        srv.release(j)
        with pytest.raises(b.CspError):
            srv.info(j)
        with pytest.raises(b.CspError):
            srv.poll(123456789)


def test_destroy_runs_queued_jobs():
    w = _w("denoise", 64, 64)
    ref = _alone(w, "cross_scale", "fp32")
    srv = Server(0)
    mid = srv.add_workload_model(w, "cross_scale", "fp32")
    srv.pause(True)
    out = np.zeros((1, 64, 64), np.float32)
    srv.submit(mid, w.meas, 64, 64, out=out)
    srv.close()  # resumes, runs the queued job, then frees everything
    assert np.array_equal(out, ref)


def test_invalid_model_and_job():
    w = _w("denoise", 64, 64)
    with Server(0) as srv:
        lf = _w("lightfield", 48, 48, T0=2048)
        with pytest.raises(b.CspError) as e:
            srv.add_workload_model(lf, "cross_scale", "fp32")
        assert e.value.status == b.CSP_ERR_UNSUPPORTED
        mid = srv.add_workload_model(w, "cross_scale", "fp32")
        with pytest.raises(b.CspError):
            srv._models[mid + 5] = srv._models[mid]  # the binding knows it, the server does not
            srv.submit(mid + 5, w.meas, 64, 64)
        with pytest.raises(b.CspError):
            srv.submit(mid, w.meas[:, :4, :4], 4, 4)  # smaller than a patch
