"""Modified K-SVD (Sec. III, "Learning cross-scale sparse models") on the GPU.

Orchestration only: every step runs in libcsp.so.

* Step 1: K-SVD on the downsampled training signals W x_i (csp_downsample):
  plain OMP against D_low (csp_solve) and a dictionary-update sweep
  (csp_ksvd_update), from heuristic 1 of Sec. III, "Initialization of
  dictionary" (csp_ksvd_init_atoms); the last coding gives the coarse
  supports Omega_low.
* Step 2: K-SVD on the x_i with the coding restricted to f(Omega_low) --
  Algorithm 2 (csp_solve, cross-scale mode) over the pair (D_high, D_low) --
  from heuristic 2; unused atoms are replaced by heuristics 3 and 4.
"""

from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
import torch

from .context import Context


class ModifiedKSVD:
    """Learns (D_high, D_low) for patches of `P` x `P` pixels on a plane grid,
    with the scale factors `level_factors` ([(1, 1, 1, 1), (fy, fx, sy, sx)])
    and the scale links parent[j] (coarse atom of fine atom j)."""

    def __init__(self, P: int, plane_grid: Sequence[int], level_factors, parent: np.ndarray, K_high: int,
                 K_low: int, device: int = 0, precision: str = "fp32", replace_unused: bool = True,
                 approximate: bool = False):
        if len(level_factors) != 2:
            raise ValueError("two scales")
        fy, fx, sy, sx = level_factors[1]
        if sy != sx or P % sy:
            raise ValueError("the coarse patch must be square")
        self.parent = np.ascontiguousarray(parent, np.int32)
        self.T_high = int(self.parent.shape[0])
        self.K_high, self.K_low = int(K_high), int(K_low)
        self.precision = precision
        self.replace = bool(replace_unused)
        self.approximate = bool(approximate)   # one alternating step per atom instead of the SVD
        Ly, Lx = int(plane_grid[0]), int(plane_grid[1])
        self.fine = Context(device)          # both scales; Step 2 coding and W
        self.fine.set_geometry(P, P, (Ly, Lx), P, P, level_factors)
        self.fine.set_sensing("identity")
        self.coarse = Context(device)        # the coarse scale alone; Step 1 coding
        Pl = P // sy
        self.coarse.set_geometry(Pl, Pl, (Ly // fy, Lx // fx), Pl, Pl, [(1, 1, 1, 1)])
        self.coarse.set_sensing("identity")
        self.dev = self.fine.device
        self.parent_dev = torch.from_numpy(self.parent).to(self.dev)

    def fit(self, X: torch.Tensor, u_low: np.ndarray, u_high: np.ndarray, iters_low: int, iters_high: int):
        """X: float32 [n, N0] on the device.  u_low [T_low], u_high [T_high]:
        uniform numbers of the initialisation picks.  Returns (D_low, D_high,
        sup_low, keff_low, err_low, err_high), the errors ||X - D S||_F^2 after
        every sweep."""
        X = X.contiguous()
        dev = self.dev
        T_low = len(u_low)
        X_low = self.fine.downsample(1, X)
        D_low = torch.zeros((T_low, X_low.shape[1]), dtype=torch.float32, device=dev)
        self.coarse.ksvd_init_atoms(D_low, X_low, torch.as_tensor(np.asarray(u_low, np.float64), device=dev))
        err = torch.zeros(1, dtype=torch.float32, device=dev)
        err_low, err_high = [], []
        for _ in range(iters_low):
            self.coarse.load_dictionary(0, D_low)
            sup, coef, keff = self.coarse.solve(X_low, mode="plain", precision=self.precision, K=(self.K_low,))
            self.coarse.ksvd_update(D_low, X_low, sup, coef, keff, self.replace, err_out=err,
                                    approximate=self.approximate)
            err_low.append(float(err.item()))
        self.coarse.load_dictionary(0, D_low)
        sup_low, _, keff_low = self.coarse.solve(X_low, mode="plain", precision=self.precision, K=(self.K_low,))
        D_high = torch.zeros((self.T_high, X.shape[1]), dtype=torch.float32, device=dev)
        self.fine.ksvd_init_atoms(D_high, X, torch.as_tensor(np.asarray(u_high, np.float64), device=dev),
                                  self.parent_dev, sup_low, keff_low, T_low)
        for _ in range(iters_high):
            sup, coef, keff = self.code_high(D_high, D_low, X)
            self.fine.ksvd_update(D_high, X, sup, coef, keff, self.replace, self.parent_dev, sup_low, err_out=err,
                                  approximate=self.approximate)
            err_high.append(float(err.item()))
        return D_low, D_high, sup_low, keff_low, err_low, err_high

    def code_high(self, D_high: torch.Tensor, D_low: torch.Tensor, X: torch.Tensor):
        """Step 2 coding: Algorithm 2 over (D_high, D_low) and the links."""
        self.fine.load_dictionary(0, D_high)
        self.fine.load_dictionary(1, D_low)
        self.fine.load_links(0, self.parent)
        return self.fine.solve(X, mode="cross_scale", precision=self.precision, K=(self.K_high, self.K_low))

    def close(self) -> None:
        self.fine.close()
        self.coarse.close()
