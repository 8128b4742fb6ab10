"""Context object over the C ABI, taking torch tensors for device buffers.

Marshalling only: pointers, sizes and the current CUDA stream are handed to
libcsp.so, which does all the work.  Device tensors come from PyTorch, which
here is the allocator and the stream provider.
"""

from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _binding as b


def _stream_ptr(stream: Optional[torch.cuda.Stream], device) -> int:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return int(s.cuda_stream)


class Context:
    """One library context on one CUDA device (see include/csp.h)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.device = torch.device("cuda", device)
        self._ctx = b.csp_create(device, mem_budget_bytes)
        self.geometry = None
        self.M = None
        self.B = None
        self.n_levels = 0
        self._planes = 0

    def close(self) -> None:
        if getattr(self, "_ctx", None):
            b.csp_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- set-up -------------------------------------------------------------
    def set_geometry(self, H: int, W: int, plane_grid: Sequence[int], P: int, stride: int,
                     level_factors: Sequence[Sequence[int]]) -> None:
        g = b.csp_geometry()
        g.H, g.W = H, W
        g.plane_rows, g.plane_cols = int(plane_grid[0]), int(plane_grid[1])
        g.P, g.stride = P, stride
        g.n_levels = len(level_factors)
        for l, f in enumerate(level_factors):
            for c in range(4):
                g.factors[l][c] = int(f[c])
        b.csp_set_geometry(self._ctx, g)
        self.geometry = (H, W, tuple(plane_grid), P, stride, [tuple(f) for f in level_factors])
        self.n_levels = len(level_factors)
        self._planes = int(plane_grid[0]) * int(plane_grid[1])

    def set_sensing(self, kind: str, codes: Optional[np.ndarray] = None, shots: int = 0) -> None:
        """codes: uint8 codes (coded exposure / aperture) or, for "dense", Phi
        float32 [M, N] (shots = M is then taken from its shape)."""
        s = b.csp_sensing()
        s.kind = b.SENSE[kind]
        self._codes = None
        if kind == "dense":
            self._codes = np.ascontiguousarray(codes, dtype=np.float32)
            s.phi = self._codes.ctypes.data
            shots = self._codes.shape[0]
        elif codes is not None:
            self._codes = np.ascontiguousarray(codes, dtype=np.uint8)
            s.codes = self._codes.ctypes.data
        s.shots = int(shots)
        b.csp_set_sensing(self._ctx, s)
        self.B, self.M = b.csp_problem_size(self._ctx)
        self.sense_kind = kind
        self.shots = shots

    def load_dictionary(self, level: int, D) -> None:
        """D: [T, N] float32 (numpy or torch, host or device), atom-major."""
        if isinstance(D, torch.Tensor):
            Dt = D.detach().to(torch.float32).contiguous()
            on_dev = int(Dt.is_cuda)
            ptr = Dt.data_ptr()
            T, N = Dt.shape
            keep = Dt
        else:
            keep = np.ascontiguousarray(D, dtype=np.float32)
            T, N = keep.shape
            on_dev, ptr = 0, keep.ctypes.data
        b.csp_load_dictionary(self._ctx, level, ptr, int(N), int(T), on_dev)
        del keep

    def load_links(self, level: int, parent: Optional[np.ndarray] = None, T_l: int = 0, Q: int = 0) -> None:
        if parent is not None:
            p = np.ascontiguousarray(parent, dtype=np.int32)
            b.csp_load_scale_links(self._ctx, level, p.ctypes.data, int(p.shape[0]), 0)
        else:
            b.csp_load_scale_links(self._ctx, level, None, int(T_l), int(Q))

    def load_workload(self, w) -> None:
        """Geometry, sensing, dictionaries and links of a workload object with
        fields geometry, sensing, dicts, parents."""
        g = w.geometry
        self.set_geometry(g.H, g.W, g.plane_grid, g.P, g.stride, g.level_factors)
        s = w.sensing
        shots = int(s.codes.shape[0]) if s.kind == "coded_aperture" else 0
        self.set_sensing(s.kind, s.codes, shots)
        for l, D in enumerate(w.dicts):
            self.load_dictionary(l, D)
        for l, p in enumerate(w.parents):
            self.load_links(l, p)

    # ---- compute ------------------------------------------------------------
    def extract(self, meas: torch.Tensor, Y: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        meas = meas.contiguous()
        assert meas.dtype == torch.float32 and meas.is_cuda
        if Y is None:
            Y = torch.empty((self.B, self.M), dtype=torch.float32, device=self.device)
        b.csp_extract_patches(self._ctx, meas.data_ptr(), Y.data_ptr(), _stream_ptr(stream, self.device))
        return Y

    @staticmethod
    def params(mode: str = "cross_scale", precision: str = "fp32", K: Sequence[int] = (),
               K_patch: Optional[Sequence[Optional[torch.Tensor]]] = None, Kmax: Optional[int] = None):
        p = b.csp_solve_params()
        p.mode = b.MODE[mode]
        p.precision = b.PREC[precision]
        for l, k in enumerate(K):
            p.K[l] = int(k)
        if K_patch is not None:
            for l, t in enumerate(K_patch):
                p.K_patch[l] = None if t is None else t.data_ptr()
        p.Kmax = int(Kmax if Kmax is not None else (max(K) if K else 0))
        return p

    def solve(self, Y: torch.Tensor, mode: str = "cross_scale", precision: str = "fp32",
              K: Sequence[int] = (), K_patch=None, Kmax: Optional[int] = None, out=None, stream=None):
        """Returns (support int32 [B, Kmax], coef float32 [B, Kmax], k_eff int8 [B])."""
        Y = Y.contiguous()
        assert Y.dtype == torch.float32 and Y.is_cuda
        Bn = Y.shape[0]
        p = self.params(mode, precision, K, K_patch, Kmax)
        if out is None:
            sup = torch.empty((Bn, p.Kmax), dtype=torch.int32, device=self.device)
            coef = torch.empty((Bn, p.Kmax), dtype=torch.float32, device=self.device)
            keff = torch.empty((Bn,), dtype=torch.int8, device=self.device)
        else:
            sup, coef, keff = out
        b.csp_solve(self._ctx, p, Y.data_ptr(), Bn, sup.data_ptr(), coef.data_ptr(), keff.data_ptr(),
                    _stream_ptr(stream, self.device))
        return sup, coef, keff

    def autotune(self, Y: torch.Tensor, mode: str = "cross_scale", precision: str = "fp32", K: Sequence[int] = (),
                 K_patch=None, Kmax: Optional[int] = None, stream=None):
        """Times each kernel variant on this batch and keeps the fastest.
        Returns {"restricted_variant": v, "ms": [...]}."""
        Y = Y.contiguous()
        Bn = Y.shape[0]
        p = self.params(mode, precision, K, K_patch, Kmax)
        sup = torch.empty((Bn, p.Kmax), dtype=torch.int32, device=self.device)
        coef = torch.empty((Bn, p.Kmax), dtype=torch.float32, device=self.device)
        keff = torch.empty((Bn,), dtype=torch.int8, device=self.device)
        r = b.csp_autotune(self._ctx, p, Y.data_ptr(), Bn, sup.data_ptr(), coef.data_ptr(), keff.data_ptr(),
                           _stream_ptr(stream, self.device))
        return {"restricted_variant": r.restricted_variant, "ms": list(r.ms), "top_level_form": r.top_level_form,
                "ms_top": list(r.ms_top)}

    def set_graph_mode(self, on: bool = True) -> None:
        """Replay identical solves from a CUDA graph (see csp_set_graph_mode)."""
        b.csp_set_graph_mode(self._ctx, on)

    def set_pipeline(self, on: bool = True) -> None:
        """Pipelined cross-scale solve on two streams (see csp_set_pipeline)."""
        b.csp_set_pipeline(self._ctx, on)

    def set_work_order(self, order: int) -> None:
        """0 static grids in patch order; 1 patches sorted by budget (largest
        first) and the restricted levels on a work queue (csp_set_work_order)."""
        b.csp_set_work_order(self._ctx, order)

    def set_wait_test(self, on: bool) -> None:
        """Failure-detection test hook (see csp_set_wait_test)."""
        b.csp_set_wait_test(self._ctx, on)

    def set_top_level_form(self, form: int) -> None:
        """0 automatic, 1 per-iteration kernels, 2 fused full-dictionary kernel,
        3 Gram form (correlation GEMM once, Gram-Schmidt iteration over every atom)."""
        b.csp_set_top_level_form(self._ctx, form)

    def set_aggregate_path(self, path: int) -> None:
        """0 automatic, 1 two-pass, 2 fused shared-memory tiles (same image)."""
        b.csp_set_aggregate_path(self._ctx, path)

    def set_kernel_variant(self, restricted_variant: int) -> None:
        b.csp_set_kernel_variant(self._ctx, restricted_variant)

    def stats(self):
        st = b.csp_solve_stats_get(self._ctx)
        return {"patches": st.patches, "fp64_fallbacks": st.fp64_fallbacks, "early_stops": st.early_stops,
                "overflow": st.overflow, "restricted_scores": st.restricted_scores,
                "synthesized": bool(st.synthesized)}

    def profile(self, on: bool = True) -> None:
        b.csp_profile_enable(self._ctx, on)

    def profile_read(self, reset: bool = False):
        return b.csp_profile_read(self._ctx, reset)

    def aggregate(self, sup: torch.Tensor, coef: torch.Tensor, keff: torch.Tensor,
                  img: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        H, W = self.geometry[0], self.geometry[1]
        if img is None:
            img = torch.empty((self._planes, H, W), dtype=torch.float32, device=self.device)
        b.csp_aggregate(self._ctx, sup.data_ptr(), coef.data_ptr(), keff.data_ptr(), sup.shape[0], sup.shape[1],
                        img.data_ptr(), _stream_ptr(stream, self.device))
        return img

    def reconstruct(self, meas: torch.Tensor, img: Optional[torch.Tensor] = None, mode: str = "cross_scale",
                    precision: str = "fp32", K: Sequence[int] = (), Kmax: Optional[int] = None,
                    stream=None) -> torch.Tensor:
        """Extraction, solve and aggregation on device tensors in one call
        (csp_reconstruct); returns the image [planes, H, W]."""
        meas = meas.contiguous()
        assert meas.dtype == torch.float32 and meas.is_cuda
        H, W = self.geometry[0], self.geometry[1]
        if img is None:
            img = torch.empty((self._planes, H, W), dtype=torch.float32, device=self.device)
        p = self.params(mode, precision, K, None, Kmax)
        b.csp_reconstruct(self._ctx, p, meas.data_ptr(), img.data_ptr(), _stream_ptr(stream, self.device))
        return img

    # ---- dictionary learning (modified K-SVD) -------------------------------
    def downsample(self, level: int, X: torch.Tensor, out: Optional[torch.Tensor] = None,
                   stream=None) -> torch.Tensor:
        """W_level applied to level-0 vectors X [N, N0] (csp_downsample)."""
        X = X.contiguous()
        assert X.dtype == torch.float32 and X.is_cuda
        fy, fx, sy, sx = self.geometry[5][level]
        n_low = X.shape[1] // (fy * fx * sy * sx)
        if out is None:
            out = torch.empty((X.shape[0], n_low), dtype=torch.float32, device=self.device)
        b.csp_downsample(self._ctx, level, X.data_ptr(), X.shape[0], out.data_ptr(), _stream_ptr(stream, self.device))
        return out

    def ksvd_update(self, D: torch.Tensor, X: torch.Tensor, sup: torch.Tensor, coef: torch.Tensor,
                    keff: torch.Tensor, replace_unused: bool = False, repl_parent: Optional[torch.Tensor] = None,
                    repl_support: Optional[torch.Tensor] = None, err_out: Optional[torch.Tensor] = None,
                    stream=None, approximate: bool = False) -> None:
        """One K-SVD dictionary-update sweep in place on D [T, M] and coef
        [N, Kmax] (csp_ksvd_update); err_out (float32 [1]) receives
        ||X - D S||_F^2 after the sweep; approximate: one alternating step per
        atom instead of the singular vector."""
        for t in (D, X, sup, coef, keff):
            assert t.is_cuda and t.is_contiguous()
        T, M = D.shape
        Kc = int(repl_support.shape[1]) if repl_support is not None else 0
        b.csp_ksvd_update(self._ctx, D.data_ptr(), int(M), int(T), X.data_ptr(), int(X.shape[0]), sup.data_ptr(),
                          coef.data_ptr(), keff.data_ptr(), int(sup.shape[1]), int(bool(replace_unused)),
                          int(bool(approximate)),
                          repl_parent.data_ptr() if repl_parent is not None else None,
                          repl_support.data_ptr() if repl_support is not None else None, Kc,
                          err_out.data_ptr() if err_out is not None else None, _stream_ptr(stream, self.device))

    def ksvd_stats(self):
        """(power-method steps, replaced atoms, cluster ranks) of the last ksvd_update."""
        return b.csp_ksvd_stats_get(self._ctx)

    def ksvd_init_atoms(self, D: torch.Tensor, X: torch.Tensor, u: torch.Tensor,
                        parent: Optional[torch.Tensor] = None, sup_low: Optional[torch.Tensor] = None,
                        keff_low: Optional[torch.Tensor] = None, T_low: int = 0, stream=None) -> None:
        """Initialisation picks (csp_ksvd_init_atoms); u: float64 [T] on the device."""
        assert u.dtype == torch.float64 and u.is_cuda
        T, M = D.shape
        Kc = int(sup_low.shape[1]) if sup_low is not None else 0
        b.csp_ksvd_init_atoms(self._ctx, D.data_ptr(), int(M), int(T), X.data_ptr(), int(X.shape[0]),
                              parent.data_ptr() if parent is not None else None,
                              sup_low.data_ptr() if sup_low is not None else None,
                              keff_low.data_ptr() if keff_low is not None else None, Kc, int(T_low),
                              u.data_ptr(), _stream_ptr(stream, self.device))

    def reconstruct_host(self, meas: np.ndarray, img: np.ndarray, mode: str = "cross_scale",
                         precision: str = "fp32", K: Sequence[int] = (), Kmax: Optional[int] = None,
                         stream=None) -> np.ndarray:
        """End to end from host memory (pinned numpy views recommended)."""
        p = self.params(mode, precision, K, None, Kmax)
        b.csp_reconstruct_host(self._ctx, p, meas.ctypes.data if isinstance(meas, np.ndarray) else meas.data_ptr(),
                               img.ctypes.data if isinstance(img, np.ndarray) else img.data_ptr(),
                               _stream_ptr(stream, self.device))
        return img
