"""FP64 CPU oracle for plain and cross-scale (zero-tree) OMP on patch workloads.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the CPU
baseline leg of the benchmark, never by the product path.  It shares no code
with the CUDA library; its only shared dependency is the seeded input
generator in ``synthetic``.

Paper passages followed (arXiv 1511.05174):

* Sec. II-A notation: support Omega, restriction D_|Omega.
* Sec. II-B, Algorithm 1 (OMP): proxy, support merge, projection, residue --
  implemented in ``omp_oracle.c`` with least squares solved from scratch by
  Householder QR every iteration.
* Sec. III-A signal model and operators W (uniform downsampler) and U
  (nearest-neighbour upsampler, W U = I).
* Sec. III-B cross-scale map f: children of each coarse atom (the block rule
  i -> (i-1)Q + {1..Q} is the special case parent(j) = floor(j / Q)).
* Sec. III-C measurement model y = Phi x + e, coarse problem (P_low) with the
  operator Phi U D_low, fine problem (P_high) restricted to f(Omega_low).
* Algorithm 2 (zero-tree OMP): for Phi = I the coarse step runs on W x
  against D_low (``coarse_form="wx"``); (P_low) is the general form
  (``coarse_form="p_low"``).  Both give the same supports (the W-form residual
  is W applied to the (P_low) residual and the upsampled atoms have norms
  scaled by a common factor).
* Sec. IV: SNR = 20 log10(||x|| / ||x - x_hat||); overlapping patches (the
  aggregation rule is not stated -- uniform averaging over covering patches).
"""

from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

EPS_R = 1e-28   # stop when ||r||^2 <= EPS_R ||y||^2
EPS_D = 1e-10   # drop an atom whose QR pivot |R_kk| <= EPS_D ||a_k||

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_omp_batch.restype = ctypes.c_int
        lib.oracle_omp_batch.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p]
        lib.oracle_num_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def num_threads() -> int:
    return int(_lib().oracle_num_threads())


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# --------------------------------------------------------------------------
# OMP over independent problems (Algorithm 1)
# --------------------------------------------------------------------------

def omp_batch(mats: Sequence[np.ndarray], Y: np.ndarray, K, normalize: bool = True,
              eps_r: float = EPS_R, eps_d: float = EPS_D, nthreads: int = 0,
              return_flops: bool = False):
    """OMP for each problem b: y = Y[b] against the atom-major matrix mats[b]
    ([T_b, M]; entries may be the same array object).  K: int or [B] ints.
    Returns omega [B, Kmax] (column indices, -1 padded), alpha [B, Kmax],
    k_eff [B], rsq [B] (final ||r||^2) and, optionally, proxy flops [B]."""
    B = len(mats)
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(B, -1)
    M = Y.shape[1] if B else 0
    Karr = np.broadcast_to(np.asarray(K, dtype=np.int32), (B,)).copy()
    Kmax = int(Karr.max()) if B else 0
    Kmax = max(Kmax, 1)
    keep = []
    ptrs = np.zeros(B, dtype=np.uintp)
    cols = np.zeros(B, dtype=np.int32)
    cache = {}
    for b, A in enumerate(mats):
        key = id(A)
        if key not in cache:
            Ad = np.ascontiguousarray(A, dtype=np.float64)
            if Ad.ndim != 2 or (Ad.shape[0] and Ad.shape[1] != M):
                raise ValueError("each matrix must be [T, M]")
            keep.append(Ad)
            cache[key] = (_ptr(Ad) if Ad.size else 0, Ad.shape[0])
        ptrs[b], cols[b] = cache[key]
    omega = np.full((B, Kmax), -1, np.int32)
    alpha = np.zeros((B, Kmax))
    k_eff = np.zeros(B, np.int32)
    rsq = np.zeros(B)
    flops = np.zeros(B, np.int64)
    if B:
        _lib().oracle_omp_batch(B, M, _ptr(ptrs), _ptr(cols), _ptr(Y), _ptr(Karr), Kmax, eps_r, eps_d,
                                int(bool(normalize)), int(nthreads), _ptr(omega), _ptr(alpha),
                                _ptr(k_eff), _ptr(rsq), _ptr(flops))
    if return_flops:
        return omega, alpha, k_eff, rsq, flops
    return omega, alpha, k_eff, rsq


# --------------------------------------------------------------------------
# Geometry, W, U and Phi
# --------------------------------------------------------------------------

def patch_origins(extent: int, P: int, stride: int) -> np.ndarray:
    """Origins 0, s, 2s, ... <= extent - P, plus extent - P if the stride misses it."""
    if extent < P:
        return np.zeros(0, np.int64)
    o = list(range(0, extent - P + 1, stride))
    if o[-1] != extent - P:
        o.append(extent - P)
    return np.asarray(o, np.int64)


def patch_grid(g) -> Tuple[np.ndarray, np.ndarray]:
    """Patch origins in raster order: patch b = iy * nx + ix."""
    oy = patch_origins(g.H, g.P, g.stride)
    ox = patch_origins(g.W, g.P, g.stride)
    yy, xx = np.meshgrid(oy, ox, indexing="ij")
    return yy.ravel(), xx.ravel()


def level_shape(g, l: int) -> Tuple[int, int, int, int]:
    fy, fx, sy, sx = g.level_factors[l]
    Ly, Lx = g.plane_grid
    return Ly // fy, Lx // fx, g.P // sy, g.P // sx


def W_down(V: np.ndarray, g, l: int) -> np.ndarray:
    """Uniform (box) downsampler from level 0 to level l, applied to rows of V."""
    Ly, Lx = g.plane_grid
    fy, fx, sy, sx = g.level_factors[l]
    n = V.shape[0]
    X = V.reshape(n, Ly // fy, fy, Lx // fx, fx, g.P // sy, sy, g.P // sx, sx)
    return X.mean(axis=(2, 4, 6, 8)).reshape(n, -1)


def U_up(V: np.ndarray, g, l: int) -> np.ndarray:
    """Nearest-neighbour upsampler from level l to level 0 (W U = I)."""
    Lyl, Lxl, Pyl, Pxl = level_shape(g, l)
    fy, fx, sy, sx = g.level_factors[l]
    n = V.shape[0]
    X = V.reshape(n, Lyl, 1, Lxl, 1, Pyl, 1, Pxl, 1)
    X = np.broadcast_to(X, (n, Lyl, fy, Lxl, fx, Pyl, sy, Pxl, sx))
    return X.reshape(n, -1).copy()


def bayer_channel(y: np.ndarray, x: np.ndarray) -> np.ndarray:
    """RGGB: (even, even) red = 0, (odd, odd) blue = 2, else green = 1."""
    return np.where((y % 2 == 0) & (x % 2 == 0), 0, np.where((y % 2 == 1) & (x % 2 == 1), 2, 1))


def meas_dim(g, sensing) -> int:
    if sensing.kind == "identity":
        return g.planes * g.P * g.P
    if sensing.kind in ("bayer_rggb", "coded_exposure"):
        return g.P * g.P
    if sensing.kind == "coded_aperture":
        return sensing.codes.shape[0] * g.P * g.P
    if sensing.kind == "dense":
        return sensing.codes.shape[0]
    raise ValueError(sensing.kind)


def phi_apply(sensing, g, oy: int, ox: int, V: np.ndarray) -> np.ndarray:
    """Phi_p applied to rows of V ([n, N] level-0 patch vectors) for the patch
    at origin (oy, ox): y = Phi x (Sec. III-C)."""
    n = V.shape[0]
    P = g.P
    X = V.reshape(n, g.planes, P, P)
    if sensing.kind == "identity":
        return V.copy()
    if sensing.kind == "bayer_rggb":
        yy, xx = np.meshgrid(oy + np.arange(P), ox + np.arange(P), indexing="ij")
        ch = bayer_channel(yy, xx)
        out = np.take_along_axis(X, np.broadcast_to(ch[None, None], (n, 1, P, P)), axis=1)[:, 0]
        return out.reshape(n, P * P)
    if sensing.kind == "coded_exposure":
        c = sensing.codes[:, oy:oy + P, ox:ox + P].astype(np.float64)   # [F, P, P]
        return (X * c[None]).sum(axis=1).reshape(n, P * P)
    if sensing.kind == "coded_aperture":
        c = sensing.codes.astype(np.float64)                             # [S, V]
        return np.einsum("sv,nvyx->nsyx", c, X).reshape(n, -1)
    if sensing.kind == "dense":                                          # one Phi [M, N] for every patch
        return V @ sensing.codes.astype(np.float64).T
    raise ValueError(sensing.kind)


def sensing_matrix(sensing, g, oy: int, ox: int) -> np.ndarray:
    """Dense Phi_p ([M, N]) for the patch at (oy, ox)."""
    N = g.planes * g.P * g.P
    return phi_apply(sensing, g, oy, ox, np.eye(N)).T.copy()


def phi_key(sensing, oy: int, ox: int, b: int):
    """Patches with the same key share Phi_p."""
    if sensing.kind in ("identity", "coded_aperture", "dense"):
        return 0
    if sensing.kind == "bayer_rggb":
        return (int(oy) % 2, int(ox) % 2)
    return ("patch", b)


# --------------------------------------------------------------------------
# Patch extraction and the per-level problems
# --------------------------------------------------------------------------

def extract_patches(w) -> np.ndarray:
    """Y [B, M] float64: the patch vectors of the measurement image."""
    g, s = w.geometry, w.sensing
    oy, ox = patch_grid(g)
    P = g.P
    m = w.meas.astype(np.float64)
    B = len(oy)
    if s.kind == "dense":  # the measurements are per patch already
        return m.reshape(B, -1).copy()
    out = np.zeros((B, meas_dim(g, s)))
    for b in range(B):
        if s.kind == "identity":
            out[b] = m[:, oy[b]:oy[b] + P, ox[b]:ox[b] + P].ravel()
        elif s.kind in ("bayer_rggb", "coded_exposure"):
            out[b] = m[oy[b]:oy[b] + P, ox[b]:ox[b] + P].ravel()
        else:
            out[b] = m[:, oy[b]:oy[b] + P, ox[b]:ox[b] + P].ravel()
    return out


def children_lists(parent: np.ndarray, n_parent: int) -> List[np.ndarray]:
    """f: the atoms of the finer level linked to each coarse atom, ascending."""
    return [np.flatnonzero(parent == p) for p in range(n_parent)]


def plain_omp(w, Y: Optional[np.ndarray] = None, patches: Optional[np.ndarray] = None,
              nthreads: int = 0, K: Optional[np.ndarray] = None):
    """Algorithm 1 on every patch against the fine effective dictionary."""
    if Y is None:
        Y = extract_patches(w)
    sel = np.arange(Y.shape[0]) if patches is None else np.asarray(patches)
    Kp = w.K_levels[0][sel] if K is None else np.broadcast_to(K, sel.shape)
    # chunks of patches bound the memory of per-patch effective dictionaries;
    # every problem is solved on its own, so chunking changes no result
    chunk = 512 if w.sensing.kind in ("coded_exposure",) else max(len(sel), 1)
    outs = []
    for c0 in range(0, len(sel), chunk):
        Yl, mats = _level_subset(w, 0, Y, sel[c0:c0 + chunk], "p_low")
        outs.append(omp_batch(mats, Yl, Kp[c0:c0 + chunk], nthreads=nthreads))
    if len(outs) == 1:
        return outs[0]
    if not outs:
        return omp_batch([], np.zeros((0, Y.shape[1])), Kp)
    Kmax = max(o[0].shape[1] for o in outs)
    return (np.concatenate([np.pad(o[0], ((0, 0), (0, Kmax - o[0].shape[1])), constant_values=-1) for o in outs]),
            np.concatenate([np.pad(o[1], ((0, 0), (0, Kmax - o[1].shape[1]))) for o in outs]),
            np.concatenate([o[2] for o in outs]), np.concatenate([o[3] for o in outs]))


def _level_subset(w, l, Y, sel, form):
    """level_problem for a subset of patches (keeps per-patch memory bounded)."""
    g, s = w.geometry, w.sensing
    D = w.dicts[l].astype(np.float64)
    oy, ox = patch_grid(g)
    Ysub = Y[sel]
    if s.kind == "identity" and form == "wx":
        return (W_down(Ysub, g, l) if l else Ysub.copy()), [D] * len(sel)
    UD = U_up(D, g, l) if l else D
    cache = {}
    mats = []
    for b in sel:
        k = phi_key(s, oy[b], ox[b], int(b))
        if k not in cache:
            cache[k] = phi_apply(s, g, int(oy[b]), int(ox[b]), UD)
        mats.append(cache[k])
    return Ysub, mats


def cross_scale_omp(w, Y: Optional[np.ndarray] = None, patches: Optional[np.ndarray] = None,
                    coarse_form: str = "wx", nthreads: int = 0, return_levels: bool = False,
                    chunk: int = 256):
    """Algorithm 2 generalised to L levels (the zero tree of Fig. 3).

    Coarsest level: OMP over all atoms with K_{L-1}.  Each finer level l:
    candidates C_l = f(Omega_{l+1}) (children of the atoms chosen one level up,
    ascending), then OMP restricted to C_l with K_l (stops when C_l runs out).
    Returns level-0 (omega, alpha, k_eff, rsq) with omega in fine atom indices."""
    if Y is None:
        Y = extract_patches(w)
    sel = np.arange(Y.shape[0]) if patches is None else np.asarray(patches)
    L = w.n_levels
    children = [children_lists(w.parents[l], w.dicts[l + 1].shape[0]) for l in range(L - 1)]
    levels = []
    prev_omega = None
    prev_keff = None
    for l in range(L - 1, -1, -1):
        form = coarse_form
        Kl = w.K_levels[l][sel]
        outs = []
        for c0 in range(0, len(sel), chunk):
            csel = sel[c0:c0 + chunk]
            Yl, mats = _level_subset(w, l, Y, csel, form)
            if l == L - 1:
                outs.append(omp_batch(mats, Yl, Kl[c0:c0 + chunk], nthreads=nthreads))
                continue
            sub_mats, cand_lists = [], []
            for j, b in enumerate(csel):
                jj = c0 + j
                om = prev_omega[jj, :prev_keff[jj]]
                C = np.sort(np.concatenate([children[l][p] for p in om])) if len(om) else np.zeros(0, np.int64)
                cand_lists.append(C)
                sub_mats.append(mats[j][C])
            o, a, k, r = omp_batch(sub_mats, Yl, Kl[c0:c0 + chunk], nthreads=nthreads)
            for j, C in enumerate(cand_lists):   # column position -> atom index
                valid = o[j] >= 0
                o[j, valid] = C[o[j, valid]]
            outs.append((o, a, k, r))
        Kmax = max(int(Kl.max()) if len(Kl) else 1, 1)
        omega = np.concatenate([np.pad(o[0], ((0, 0), (0, Kmax - o[0].shape[1])), constant_values=-1) for o in outs]) if outs else np.zeros((0, Kmax), np.int32)
        alpha = np.concatenate([np.pad(o[1], ((0, 0), (0, Kmax - o[1].shape[1]))) for o in outs]) if outs else np.zeros((0, Kmax))
        keff = np.concatenate([o[2] for o in outs]) if outs else np.zeros(0, np.int32)
        rsq = np.concatenate([o[3] for o in outs]) if outs else np.zeros(0)
        levels.append((omega, alpha, keff, rsq))
        prev_omega, prev_keff = omega, keff
    if return_levels:
        return levels[::-1]  # index by level
    return levels[-1]


# --------------------------------------------------------------------------
# Synthesis, aggregation and quality metrics
# --------------------------------------------------------------------------

def synthesize(D0: np.ndarray, omega: np.ndarray, alpha: np.ndarray, k_eff: np.ndarray) -> np.ndarray:
    """x_hat_p = D_|Omega alpha for every patch ([B, N])."""
    D = D0.astype(np.float64)
    B = omega.shape[0]
    out = np.zeros((B, D.shape[1]))
    for b in range(B):
        k = int(k_eff[b])
        if k:
            out[b] = D[omega[b, :k]].T @ alpha[b, :k]
    return out


def aggregate(w, omega: np.ndarray, alpha: np.ndarray, k_eff: np.ndarray) -> np.ndarray:
    """Overlap-add of the synthesized patches, divided by the coverage count."""
    g = w.geometry
    X = synthesize(w.dicts[0], omega, alpha, k_eff)
    oy, ox = patch_grid(g)
    P = g.P
    acc = np.zeros((g.planes, g.H, g.W))
    cnt = np.zeros((g.H, g.W))
    for b in range(len(oy)):
        acc[:, oy[b]:oy[b] + P, ox[b]:ox[b] + P] += X[b].reshape(g.planes, P, P)
        cnt[oy[b]:oy[b] + P, ox[b]:ox[b] + P] += 1
    return np.where(cnt > 0, acc / np.maximum(cnt, 1), 0.0)


def psnr(gt: np.ndarray, est: np.ndarray) -> float:
    """10 log10(peak^2 / MSE), peak = max(gt) - min(gt)."""
    mse = float(np.mean((gt - est) ** 2))
    peak = float(gt.max() - gt.min())
    return float("inf") if mse == 0 else 10.0 * np.log10(peak * peak / mse)


def snr(gt: np.ndarray, est: np.ndarray) -> float:
    """Sec. IV: 20 log10(||x|| / ||x - x_hat||)."""
    e = float(np.linalg.norm(gt - est))
    return float("inf") if e == 0 else 20.0 * np.log10(float(np.linalg.norm(gt)) / e)
