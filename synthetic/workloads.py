"""Seeded synthetic workloads with the shapes of the paper's experiments.

The paper's datasets (Kodak, peppers, videos, light fields) and its trained
dictionaries are not available, so every workload here is synthetic: unit-norm
Gaussian atoms stand in for trained atoms and K-sparse N(0, 1) codes for the
sparse representations (signal model of Sec. III-A).

Workloads (sizes follow the configurations this library is measured on):

* ``denoise``    -- Phi = I, 64x64 grey image, 8x8 patches, stride 8, D 64x256.
* ``bayer``      -- RGGB mosaic of a 512x512 RGB image, 8x8x3 patches, stride 2,
                    D 192x1024, 64 measurements per patch.
* ``video``      -- per-pixel coded exposure of 8 frames (256x256), 8x8x8
                    patches, stride 4, D 512x4096, three scales.
* ``lightfield`` -- 4 coded-aperture shots of 4x4 views (256x256), 4x4x8x8
                    patches, stride 4, D 1024x8192, three scales, K in [8, 20]
                    drawn per patch.

Three readings of the scale links exist:

* ``links="paper"`` (default): each coarser level has T/Q atoms (Q = 4), made by
  box-downsampling a seeded subset of the finer atoms and renormalising; every
  finer atom is linked to the coarse atom its own downsampled, renormalised
  version correlates with most (ties to the lowest index).  Child counts are
  uneven with mean Q.
* ``links="literal"``: every level keeps all T atoms (downsampled and
  renormalised) and each atom is linked to its own downsampled copy, i.e. the
  identity map; the coarse sparsity equals the fine one.
* ``links="model"``: dictionaries built so that the signal model of
  Sec. III-A holds exactly -- coarse atoms are unit Gaussian, fine atom i is a
  child of coarse atom i // Q (block rule of Sec. III-B) whose box-downsampled,
  renormalised copy is its parent (parent structure plus a detail in the null
  space of W), and the truth codes are sign-coherent within each subtree so a
  tile's coarse code W x never cancels.  The solver's coarser budgets are
  ceil(1.5 K_l) of the truth's (capped by the finer budget): a patch that
  straddles tiles mixes several tiles' coarse codes.

Vector layout of a patch at any level: index ``((ly * Lx + lx) * Py + py) * Px + px``
for plane-grid position (ly, lx) (colour channel, frame or view) and pixel
(py, px).  Dictionaries are atom-major float32 arrays of shape [T, N].
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

WORKLOAD_NAMES = ("denoise", "bayer", "video", "lightfield", "inpaint", "cs_dense")

# Stream indices of the seed sequence; one independent stream per ingredient.
_S_DICT, _S_SUBSET, _S_SUPPORT, _S_VALUES, _S_NOISE, _S_CODES, _S_KPATCH, _N_STREAMS = range(8)


@dataclasses.dataclass
class Geometry:
    """Signal and patch geometry.

    The signal is a stack of ``Ly*Lx`` planes of ``H x W`` pixels (colour
    channels, frames or views arranged on a plane grid).  Patches cover all
    planes and ``P x P`` pixels; patch origins step by ``stride`` along each
    axis.  ``level_factors[l] = (fy, fx, sy, sx)`` are the downsampling
    factors of level ``l`` relative to the finest level (plane-grid rows,
    plane-grid columns, pixel rows, pixel columns); level 0 is (1, 1, 1, 1).
    """

    kind: str
    H: int
    W: int
    plane_grid: Tuple[int, int]
    P: int
    stride: int
    level_factors: List[Tuple[int, int, int, int]]

    @property
    def planes(self) -> int:
        return self.plane_grid[0] * self.plane_grid[1]

    @property
    def n_levels(self) -> int:
        return len(self.level_factors)

    def level_shape(self, level: int) -> Tuple[int, int, int, int]:
        """(Ly, Lx, Py, Px) of a patch vector at ``level``."""
        fy, fx, sy, sx = self.level_factors[level]
        Ly, Lx = self.plane_grid
        return Ly // fy, Lx // fx, self.P // sy, self.P // sx

    def level_dim(self, level: int) -> int:
        return int(np.prod(self.level_shape(level)))


@dataclasses.dataclass
class Sensing:
    """Camera model.  ``codes`` is uint8: coded exposure [F, H, W]; coded
    aperture [S, V] (shot x view); None for identity and Bayer."""

    kind: str  # "identity" | "bayer_rggb" | "coded_exposure" | "coded_aperture" | "dense"
    codes: Optional[np.ndarray] = None


@dataclasses.dataclass
class Workload:
    name: str
    geometry: Geometry
    sensing: Sensing
    dicts: List[np.ndarray]          # per level, float32 [T_l, N_l], level 0 finest
    parents: List[np.ndarray]        # per level l < L-1, int32 [T_l] into level l+1
    K_levels: List[np.ndarray]       # per level, int32 [B] sparsity of the solve
    truth: np.ndarray                # float64 [planes, H, W]
    meas: np.ndarray                 # float32 measurement image
    sigma: float
    seed: int
    links: str
    tile_codes: Optional[list] = None  # per P x P tile of the truth, raster order: (support, values)

    @property
    def n_patches(self) -> int:
        g = self.geometry
        return patch_count_1d(g.H, g.P, g.stride) * patch_count_1d(g.W, g.P, g.stride)

    @property
    def n_levels(self) -> int:
        return len(self.dicts)


def patch_count_1d(extent: int, P: int, stride: int) -> int:
    """Number of patch origins along one axis: 0, s, 2s, ... <= extent-P, plus
    extent-P when the stride misses it."""
    if extent < P:
        return 0
    n = (extent - P) // stride + 1
    if (extent - P) % stride:
        n += 1
    return n


def _unit_gaussian(rng: np.random.Generator, T: int, N: int) -> np.ndarray:
    D = rng.standard_normal((T, N))
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    return D


def _box_down(V: np.ndarray, shape: Tuple[int, int, int, int], f: Tuple[int, int, int, int]) -> np.ndarray:
    """Box-average rows of V (each a patch vector of ``shape``) by factors f.
    Used only to build coarse dictionaries (a stand-in for training)."""
    Ly, Lx, Py, Px = shape
    fy, fx, sy, sx = f
    T = V.shape[0]
    X = V.reshape(T, Ly // fy, fy, Lx // fx, fx, Py // sy, sy, Px // sx, sx)
    return X.mean(axis=(2, 4, 6, 8)).reshape(T, -1)


def _colnorm(V: np.ndarray) -> np.ndarray:
    n = np.linalg.norm(V, axis=1, keepdims=True)
    if np.any(n <= 1e-12):
        raise ValueError("degenerate downsampled atom")
    return V / n


def _rel_factor(g: Geometry, l: int) -> Tuple[int, int, int, int]:
    a, b = g.level_factors[l], g.level_factors[l + 1]
    r = tuple(bb // aa for aa, bb in zip(a, b))
    assert all(aa * rr == bb for aa, rr, bb in zip(a, r, b)), "level factors must nest"
    return r  # type: ignore[return-value]


def _up_rel(V: np.ndarray, shape_fine: Tuple[int, int, int, int], f: Tuple[int, int, int, int]) -> np.ndarray:
    """Nearest-neighbour upsampling of rows of V (patch vectors of the coarser
    level) to the finer level of ``shape_fine`` by factors f (U of Sec. III-A)."""
    Ly, Lx, Py, Px = shape_fine
    fy, fx, sy, sx = f
    T = V.shape[0]
    X = V.reshape(T, Ly // fy, 1, Lx // fx, 1, Py // sy, 1, Px // sx, 1)
    X = np.broadcast_to(X, (T, Ly // fy, fy, Lx // fx, fx, Py // sy, sy, Px // sx, sx))
    return X.reshape(T, -1).copy()


def _build_model_dictionaries(g: Geometry, T0: int, Q: int, rho: float, rng_dict):
    """Dictionaries that satisfy the signal model of Sec. III-A exactly.

    The coarsest level holds T0 / Q^(L-1) unit-norm Gaussian atoms.  Going one
    level finer, atom i is a child of coarse atom floor(i / Q) (the block rule
    of Sec. III-B) and equals sqrt(rho) * U c_p / ||U c_p|| + sqrt(1 - rho) * n_i,
    n_i a unit Gaussian direction in the null space of the level's box
    downsampler W (I - U W projects onto it, since U W replaces each block by its
    mean).  The two parts are orthogonal, so every atom has unit norm, and
    W d_i is proportional to c_p: the downsampled, renormalised child IS its
    parent.  A K-sparse fine code whose support lies in the children of K_low
    coarse atoms therefore gives a coarse signal W x that is K_low-sparse over
    the coarse dictionary (property 2), with the fine support inside f of the
    coarse one (property 3).  rho is the share of an atom's energy carried by
    its parent's (block-constant) structure."""
    if not 0.0 < rho < 1.0:
        raise ValueError("rho must lie in (0, 1)")
    L = g.n_levels
    T_top = T0 // Q ** (L - 1)
    if T_top * Q ** (L - 1) != T0:
        raise ValueError("T must be divisible by Q^(levels - 1)")
    dicts = [None] * L
    parents: List[np.ndarray] = [None] * (L - 1)
    dicts[L - 1] = _unit_gaussian(rng_dict, T_top, g.level_dim(L - 1))
    for l in range(L - 2, -1, -1):
        f = _rel_factor(g, l)
        shape = g.level_shape(l)
        Tl = dicts[l + 1].shape[0] * Q
        parent = (np.arange(Tl) // Q).astype(np.int32)
        up = _up_rel(dicts[l + 1], shape, f)[parent]
        up /= np.linalg.norm(up, axis=1, keepdims=True)
        G = rng_dict.standard_normal((Tl, g.level_dim(l)))
        n = G - _up_rel(_box_down(G, shape, f), shape, f)
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        dicts[l] = np.sqrt(rho) * up + np.sqrt(1.0 - rho) * n
        parents[l] = parent
    return [d.astype(np.float32) for d in dicts], parents


def _build_dictionaries(g: Geometry, T0: int, Q: int, links: str, rng_dict, rng_subset, rho: float = 0.5):
    if links == "model":
        return _build_model_dictionaries(g, T0, Q, rho, rng_dict)
    L = g.n_levels
    dicts = [_unit_gaussian(rng_dict, T0, g.level_dim(0))]
    parents: List[np.ndarray] = []
    for l in range(L - 1):
        f = _rel_factor(g, l)
        down = _colnorm(_box_down(dicts[l], g.level_shape(l), f))
        if links == "literal":
            dicts.append(down.copy())
            parents.append(np.arange(dicts[l].shape[0], dtype=np.int32))
        elif links == "paper":
            Tl = dicts[l].shape[0]
            if Tl % Q:
                raise ValueError("T must be divisible by Q")
            subset = np.sort(rng_subset.choice(Tl, Tl // Q, replace=False))
            coarse = down[subset]
            corr = np.abs(down @ coarse.T)           # [T_l, T_{l+1}]
            parents.append(np.argmax(corr, axis=1).astype(np.int32))  # first max = lowest index
            dicts.append(coarse)
        else:
            raise ValueError(f"unknown links reading {links!r}")
    # Round once to float32: both the GPU path and the oracle read these values.
    dicts = [d.astype(np.float32) for d in dicts]
    return dicts, parents


def _children(parent: np.ndarray, n_parent: int) -> List[np.ndarray]:
    order = np.argsort(parent, kind="stable")
    counts = np.bincount(parent, minlength=n_parent)
    offs = np.concatenate([[0], np.cumsum(counts)])
    return [np.sort(order[offs[p]:offs[p + 1]]) for p in range(n_parent)]


def _truth_support(rng, children: List[List[np.ndarray]], T_top: int, K_lv: Sequence[int]) -> np.ndarray:
    """Descend the scale tree: K_lv[-1] random coarsest atoms, then at each finer
    level keep K_lv[l] of the children of the atoms kept above."""
    L = len(K_lv)
    S = np.sort(rng.choice(T_top, min(K_lv[L - 1], T_top), replace=False))
    for l in range(L - 2, -1, -1):
        cands = np.concatenate([children[l][p] for p in S]) if len(S) else np.zeros(0, np.int64)
        k = min(int(K_lv[l]), len(cands))
        S = np.sort(rng.choice(cands, k, replace=False)) if k else cands[:0]
    return S


def _coarsest_ancestor(parents: List[np.ndarray]) -> np.ndarray:
    """For every fine atom, its ancestor at the coarsest level."""
    a = np.arange(len(parents[0]) if parents else 0)
    for p in parents:
        a = p[a]
    return a


def _truth_image(g: Geometry, D0: np.ndarray, children, T_top, K_tile_levels, rng_sup, rng_val,
                 ancestor: Optional[np.ndarray] = None):
    """Ground truth: non-overlapping P x P tiles, each D0 s with a zero-tree
    support.  Values are N(0, 1); with ``ancestor`` (the coarsest ancestor of
    each fine atom) the values are sign-coherent: every atom of a subtree takes
    its root's random sign and an |N(0, 1)| magnitude, so the coarse code that
    W x aggregates from the children never cancels and every ancestor of the
    fine support stays in the coarse support (property 3 of Sec. III-A)."""
    Ly, Lx = g.plane_grid
    P = g.P
    if g.H % P or g.W % P:
        raise ValueError("image extent must be a multiple of the patch side")
    ty, tx = g.H // P, g.W // P
    img = np.zeros((Ly * Lx, g.H, g.W))
    codes = []
    t = 0
    for by in range(ty):
        for bx in range(tx):
            S = _truth_support(rng_sup, children, T_top, [k[t] for k in K_tile_levels])
            s = rng_val.standard_normal(len(S))
            if ancestor is not None and len(S):
                roots, inv = np.unique(ancestor[S], return_inverse=True)
                sign = np.where(rng_val.random(len(roots)) < 0.5, -1.0, 1.0)
                s = np.abs(s) * sign[inv]
            x = (D0[S].astype(np.float64).T @ s) if len(S) else np.zeros(D0.shape[1])
            img[:, by * P:(by + 1) * P, bx * P:(bx + 1) * P] = x.reshape(Ly * Lx, P, P)
            codes.append((S, s))
            t += 1
    return img, codes


def _simulate_camera(sensing: Sensing, truth: np.ndarray, sigma: float, rng_noise) -> np.ndarray:
    """Forward camera model y = Phi x + e (Sec. III-C), per measurement pixel."""
    planes, H, W = truth.shape
    if sensing.kind == "identity":
        m = truth.copy()
    elif sensing.kind == "bayer_rggb":
        if planes != 3:
            raise ValueError("Bayer sensing needs 3 colour planes")
        yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        ch = np.where((yy % 2 == 0) & (xx % 2 == 0), 0, np.where((yy % 2 == 1) & (xx % 2 == 1), 2, 1))
        m = np.take_along_axis(truth, ch[None], axis=0)[0]
    elif sensing.kind == "coded_exposure":
        m = (sensing.codes.astype(np.float64) * truth).sum(axis=0)
    elif sensing.kind == "coded_aperture":
        m = np.einsum("sv,vhw->shw", sensing.codes.astype(np.float64), truth)
    else:
        raise ValueError(sensing.kind)
    m = m + sigma * rng_noise.standard_normal(m.shape)
    return m.astype(np.float32)


def _presets(name: str, links: str):
    """(geometry kwargs, T0, K per level (fine->coarse, may be callables of K0), sigma, sensing kind)."""
    if name == "denoise":
        geo = dict(kind="image", H=64, W=64, plane_grid=(1, 1), P=8, stride=8,
                   level_factors=[(1, 1, 1, 1), (1, 1, 2, 2)])
        return geo, 256, [4, 2] if links != "literal" else [4, 4], 0.01, "identity"
    if name == "bayer":
        geo = dict(kind="image", H=512, W=512, plane_grid=(1, 3), P=8, stride=2,
                   level_factors=[(1, 1, 1, 1), (1, 1, 2, 2)])
        return geo, 1024, [8, 4] if links != "literal" else [8, 8], 0.005, "bayer_rggb"
    if name == "video":
        geo = dict(kind="video", H=256, W=256, plane_grid=(1, 8), P=8, stride=4,
                   level_factors=[(1, 1, 1, 1), (1, 1, 2, 2), (1, 2, 2, 2)])
        return geo, 4096, [16, 8, 4] if links != "literal" else [16, 16, 16], 0.005, "coded_exposure"
    if name == "lightfield":
        geo = dict(kind="lightfield", H=256, W=256, plane_grid=(4, 4), P=8, stride=4,
                   level_factors=[(1, 1, 1, 1), (2, 2, 1, 1), (2, 2, 2, 2)])
        return geo, 8192, None, 0.005, "coded_aperture"
    if name == "inpaint":
        # grayscale image with a random half of the pixels kept (N/M = 2): the
        # per-pixel retention mask is a one-frame coded exposure y = c * x
        geo = dict(kind="image", H=512, W=512, plane_grid=(1, 1), P=8, stride=4,
                   level_factors=[(1, 1, 1, 1), (1, 1, 2, 2)])
        return geo, 1024, [8, 4] if links != "literal" else [8, 8], 0.005, "coded_exposure"
    if name == "cs_dense":
        # compressive sensing of each patch with one dense Gaussian Phi (32 x 64)
        geo = dict(kind="image", H=128, W=128, plane_grid=(1, 1), P=8, stride=4,
                   level_factors=[(1, 1, 1, 1), (1, 1, 2, 2)])
        return geo, 512, [6, 3] if links != "literal" else [6, 6], 0.005, "dense"
    raise ValueError(f"unknown workload {name!r}; expected one of {WORKLOAD_NAMES}")


DENSE_M = 32  # measurements per patch of the dense-Phi workload
MODEL_RHO = 0.5  # links="model": share of a fine atom's energy in its parent's structure


def _patch_origins(extent: int, P: int, stride: int) -> np.ndarray:
    """Origins 0, s, 2s, ... <= extent - P, plus extent - P if the stride misses it."""
    o = list(range(0, extent - P + 1, stride))
    if o[-1] != extent - P:
        o.append(extent - P)
    return np.asarray(o, np.int64)


def _simulate_patches(phi: np.ndarray, truth: np.ndarray, g: Geometry, sigma: float, rng_noise) -> np.ndarray:
    """Per-patch measurements y_p = Phi x_p + e (Sec. III-C) of every patch of
    the grid, raster order: [B, M]."""
    P = g.P
    oy, ox = _patch_origins(g.H, P, g.stride), _patch_origins(g.W, P, g.stride)
    X = np.stack([truth[:, y:y + P, x:x + P].ravel() for y in oy for x in ox])
    m = X @ phi.astype(np.float64).T
    m = m + sigma * rng_noise.standard_normal(m.shape)
    return m.astype(np.float32)


def make_workload(name: str, seed: int = 0, links: str = "paper", H: Optional[int] = None,
                  W: Optional[int] = None, T0: Optional[int] = None, sigma: Optional[float] = None,
                  Q: int = 4, K_range: Tuple[int, int] = (8, 20), shots: int = 4,
                  dict_seed: Optional[int] = None, rho: float = MODEL_RHO) -> Workload:
    """Build one seeded workload.  ``H``/``W``/``T0``/``sigma`` override the
    full-size preset (tests use small images); everything else keeps the
    preset's structure.  ``dict_seed`` (default: ``seed``) seeds the
    dictionaries and scale links alone, so that several images (jobs) can
    share one model."""
    geo_kw, T0_def, K_lv, sigma_def, skind = _presets(name, links)
    if H is not None:
        geo_kw["H"] = H
    if W is not None:
        geo_kw["W"] = W
    g = Geometry(**geo_kw)
    T0 = T0 or T0_def
    sigma = sigma_def if sigma is None else sigma
    ss = np.random.SeedSequence(seed).spawn(_N_STREAMS)
    rng = [np.random.default_rng(s) for s in ss]
    if dict_seed is not None and dict_seed != seed:
        dss = np.random.SeedSequence(dict_seed).spawn(_N_STREAMS)
        rng[_S_DICT], rng[_S_SUBSET] = np.random.default_rng(dss[_S_DICT]), np.random.default_rng(dss[_S_SUBSET])

    dicts, parents = _build_dictionaries(g, T0, Q, links, rng[_S_DICT], rng[_S_SUBSET], rho)
    L = g.n_levels
    children = [_children(parents[l], dicts[l + 1].shape[0]) for l in range(L - 1)]

    B = patch_count_1d(g.H, g.P, g.stride) * patch_count_1d(g.W, g.P, g.stride)
    n_tiles = (g.H // g.P) * (g.W // g.P)
    if K_lv is None:  # per-patch K in K_range, coarser levels ceil(K / 2^l) (literal: K)
        k_lo, k_hi = K_range
        Kp = rng[_S_KPATCH].integers(k_lo, k_hi + 1, size=B)
        Kt = rng[_S_KPATCH].integers(k_lo, k_hi + 1, size=n_tiles)
        div = (lambda K, l: -(-K // (2 ** l))) if links != "literal" else (lambda K, l: K)
        K_levels = [np.asarray(div(Kp, l), np.int32) for l in range(L)]
        K_tile = [np.asarray(div(Kt, l), np.int32) for l in range(L)]
    else:
        K_levels = [np.full(B, k, np.int32) for k in K_lv]
        K_tile = [np.full(n_tiles, k, np.int32) for k in K_lv]
    if links == "model":  # the solver's coarser budgets exceed the truth's (off-grid patches mix tiles)
        K_levels = [K_levels[0]] + [np.minimum(K_levels[l - 1], -(-3 * K_levels[l] // 2)).astype(np.int32)
                                    for l in range(1, L)]

    if skind == "coded_exposure":
        codes = (rng[_S_CODES].random((g.planes, g.H, g.W)) < 0.5).astype(np.uint8)
    elif skind == "coded_aperture":
        codes = (rng[_S_CODES].random((shots, g.planes)) < 0.5).astype(np.uint8)
    elif skind == "dense":
        N = g.planes * g.P * g.P
        codes = (rng[_S_CODES].standard_normal((DENSE_M, N)) / np.sqrt(DENSE_M)).astype(np.float32)
    else:
        codes = None
    sensing = Sensing(skind, codes)

    truth, tile_codes = _truth_image(g, dicts[0], children, dicts[-1].shape[0], K_tile, rng[_S_SUPPORT],
                                     rng[_S_VALUES], _coarsest_ancestor(parents) if links == "model" else None)
    if skind == "dense":  # per-patch measurements [B, M]
        meas = _simulate_patches(codes, truth, g, sigma, rng[_S_NOISE])
    else:
        meas = _simulate_camera(sensing, truth, sigma, rng[_S_NOISE])
    return Workload(name, g, sensing, dicts, parents, K_levels, truth, meas, sigma, seed, links, tile_codes)


def make_independent_problems(B: int, M: int, T: int, K: int, seed: int = 0, sigma: float = 0.0,
                              unit_norm: bool = False, K_true: Optional[int] = None):
    """Independent problems y_p = A s_p + e_p with one shared A (M x T, stored
    atom-major [T, M] float32).  Column norms are drawn in [0.5, 2] unless
    ``unit_norm``.  Returns (A, Y [B, M] float32, true supports [B, K_true])."""
    ss = np.random.SeedSequence(seed).spawn(4)
    r = [np.random.default_rng(s) for s in ss]
    A = _unit_gaussian(r[0], T, M)
    if not unit_norm:
        A *= r[0].uniform(0.5, 2.0, size=(T, 1))
    A = A.astype(np.float32)
    Kt = K if K_true is None else K_true
    sup = np.stack([np.sort(r[1].choice(T, Kt, replace=False)) for _ in range(B)]) if B else np.zeros((0, Kt), np.int64)
    vals = r[2].standard_normal((B, Kt))
    Y = np.einsum("bk,bkm->bm", vals, A.astype(np.float64)[sup]) if B else np.zeros((0, M))
    Y = Y + sigma * r[3].standard_normal(Y.shape)
    return A, Y.astype(np.float32), sup.astype(np.int32)


@dataclasses.dataclass
class TrainingSet:
    """Training signals for learning a cross-scale dictionary pair.

    ``X`` [n, N0] float32 holds level-0 patch vectors x = D0_S s + e with
    zero-tree supports S drawn through the scale links of ``parents`` (the
    signal model of Sec. III-A) and s ~ N(0, 1).  ``dicts``/``parents`` are the
    generating model (the learner never sees them).  ``u_low`` [T_low] and
    ``u_high`` [T_high] are uniform numbers in [0, 1) for the random picks of
    the initialisation heuristics."""

    geometry: Geometry
    X: np.ndarray
    dicts: List[np.ndarray]
    parents: List[np.ndarray]
    K_high: int
    K_low: int
    u_low: np.ndarray
    u_high: np.ndarray
    sigma: float
    seed: int


def make_training_set(name: str = "denoise", n: int = 4096, seed: int = 0, T0: Optional[int] = None,
                      sigma: Optional[float] = None, Q: int = 4) -> TrainingSet:
    """Seeded two-scale training set with the patch shape, atom counts and
    sparsities of workload ``name`` (``denoise``: 8x8 grey, T 256/64, K 4/2;
    ``bayer``: 8x8 RGB, T 1024/256, K 8/4)."""
    geo_kw, T0_def, K_lv, sigma_def, _ = _presets(name, "paper")
    g = Geometry(**geo_kw)
    if g.n_levels != 2 or K_lv is None:
        raise ValueError("training sets are defined for the two-scale presets")
    T0 = T0 or T0_def
    sigma = sigma_def if sigma is None else sigma
    ss = np.random.SeedSequence([seed, 0x6b737664]).spawn(_N_STREAMS)
    rng = [np.random.default_rng(s) for s in ss]
    dicts, parents = _build_dictionaries(g, T0, Q, "paper", rng[_S_DICT], rng[_S_SUBSET])
    children = [_children(parents[0], dicts[1].shape[0])]
    D0 = dicts[0].astype(np.float64)
    X = np.zeros((n, D0.shape[1]))
    for i in range(n):
        S = _truth_support(rng[_S_SUPPORT], children, dicts[1].shape[0], K_lv)
        X[i] = D0[S].T @ rng[_S_VALUES].standard_normal(len(S))
    X += sigma * rng[_S_NOISE].standard_normal(X.shape)
    u_low = rng[_S_CODES].random(dicts[1].shape[0])
    u_high = rng[_S_CODES].random(T0)
    return TrainingSet(g, X.astype(np.float32), dicts, parents, int(K_lv[0]), int(K_lv[1]),
                       u_low, u_high, sigma, seed)
