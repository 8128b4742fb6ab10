"""Serving engine over the C ABI: continuous batching of reconstruction jobs.

Marshalling only.  The scheduler (admission by device-memory budget,
coalescing of same-model jobs into one batched solve, streams, copies) runs
in libcsp.so; this class keeps the host arrays of queued jobs alive until
they are done.
"""

from __future__ import annotations

from typing import Dict, Optional, Sequence

import numpy as np

from . import _binding as b


class Server:
    """One serving engine on one CUDA device (see the serving section of csp.h)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, max_batch_patches: int = 0,
                 n_streams: int = 0):
        self._srv = b.csp_server_create(device, mem_budget_bytes, max_batch_patches, n_streams)
        self._models: Dict[int, dict] = {}
        self._jobs: Dict[int, tuple] = {}

    def close(self) -> None:
        if getattr(self, "_srv", None):
            b.csp_server_destroy(self._srv)
            self._srv = None
            self._jobs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_model(self, plane_grid: Sequence[int], P: int, stride: int, level_factors: Sequence[Sequence[int]],
                  sense_kind: str, dicts: Sequence[np.ndarray], parents: Sequence[np.ndarray] = (),
                  mode: str = "cross_scale", precision: str = "fp32", K: Sequence[int] = (),
                  Kmax: Optional[int] = None) -> int:
        """Register a model (dictionaries, links, patch geometry, sensing kind,
        solve parameters).  Returns its id."""
        d = b.csp_model_desc()
        g = d.geom
        g.H = g.W = P
        g.plane_rows, g.plane_cols = int(plane_grid[0]), int(plane_grid[1])
        g.P, g.stride = int(P), int(stride)
        g.n_levels = len(level_factors)
        for l, f in enumerate(level_factors):
            for c in range(4):
                g.factors[l][c] = int(f[c])
        d.sense_kind = b.SENSE[sense_kind]
        keep = []
        for l, D in enumerate(dicts):
            a = np.ascontiguousarray(D, dtype=np.float32)
            keep.append(a)
            d.D[l] = a.ctypes.data
            d.T[l] = a.shape[0]
        for l, p in enumerate(parents):
            a = np.ascontiguousarray(p, dtype=np.int32)
            keep.append(a)
            d.parent[l] = a.ctypes.data
        p = d.params
        p.mode = b.MODE[mode]
        p.precision = b.PREC[precision]
        for l, k in enumerate(K):
            p.K[l] = int(k)
        p.Kmax = int(Kmax if Kmax is not None else max(K))
        mid = b.csp_server_add_model(self._srv, d)
        self._models[mid] = {"planes": int(plane_grid[0]) * int(plane_grid[1]), "sense_kind": sense_kind}
        del keep
        return mid

    def add_workload_model(self, w, mode: str = "cross_scale", precision: str = "fp32",
                           K: Optional[Sequence[int]] = None, Kmax: Optional[int] = None) -> int:
        """Register the model of a workload object (geometry, sensing kind,
        dictionaries, links); K defaults to the workload's uniform budgets."""
        g = w.geometry
        if K is None:
            K = [int(np.max(k)) for k in w.K_levels]
        return self.add_model(g.plane_grid, g.P, g.stride, g.level_factors, w.sensing.kind, w.dicts, w.parents,
                              mode, precision, K, Kmax)

    def submit(self, model_id: int, meas: np.ndarray, H: int, W: int, codes: Optional[np.ndarray] = None,
               out: Optional[np.ndarray] = None) -> int:
        """Queue a job; returns its id.  `out` ([planes, H, W] float32) receives
        the image once the job is done."""
        planes = self._models[model_id]["planes"]
        meas = np.ascontiguousarray(meas, dtype=np.float32)
        if out is None:
            out = np.empty((planes, H, W), dtype=np.float32)
        assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == planes * H * W
        c = None if codes is None else np.ascontiguousarray(codes, dtype=np.uint8)
        jd = b.csp_job_desc(model_id, int(H), int(W), meas.ctypes.data, None if c is None else c.ctypes.data,
                            out.ctypes.data)
        jid = b.csp_submit(self._srv, jd)
        self._jobs[jid] = (meas, out)
        return jid

    def pause(self, paused: bool = True) -> None:
        """Stop (or resume) admitting jobs; batches in flight complete."""
        b.csp_server_pause(self._srv, paused)

    def poll(self, job_id: int) -> bool:
        return b.csp_poll(self._srv, job_id)

    def wait(self, job_id: int, timeout_s: Optional[float] = None) -> int:
        """Status code (CSP_OK, CSP_ERR_TIMEOUT, ...)."""
        return b.csp_wait(self._srv, job_id, -1 if timeout_s is None else int(timeout_s * 1e6))

    def result(self, job_id: int, timeout_s: Optional[float] = None) -> np.ndarray:
        """Waits for the job and returns its image; raises CspError on failure."""
        st = self.wait(job_id, timeout_s)
        if st != b.CSP_OK:
            raise b.CspError(st, b.csp_server_last_error(self._srv))
        return self._jobs[job_id][1]

    def info(self, job_id: int) -> dict:
        i = b.csp_job_info_get(self._srv, job_id)
        return {"patches": i.patches, "t_submit": i.t_submit, "t_admit": i.t_admit, "t_done": i.t_done,
                "batch_jobs": i.batch_jobs, "batch_patches": i.batch_patches, "status": i.status,
                "enqueue_ms": i.enqueue_ms, "copy_in_ms": i.copy_in_ms, "solve_ms": i.solve_ms,
                "aggregate_ms": i.aggregate_ms, "copy_out_ms": i.copy_out_ms, "t_gpu_done": i.t_gpu_done,
                "host_out_ms": i.host_out_ms, "build_ms": i.build_ms}

    def release(self, job_id: int) -> None:
        b.csp_job_release(self._srv, job_id)
        self._jobs.pop(job_id, None)
