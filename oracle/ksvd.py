"""FP64 CPU oracle of the dictionary-update step of K-SVD and of the modified
K-SVD that learns a cross-scale dictionary pair.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the CPU
baseline leg of the benchmark, never by the product path.  It shares no code
with the CUDA library.

Passages followed (arXiv 1511.05174):

* Sec. II, "Dictionary learning": K-SVD learns D with X ~ D S, S K-sparse, alternating
  sparse coding and a dictionary update.  The update step is the one of the
  cited K-SVD paper: atoms are visited one after another; atom k is replaced
  by the leading left singular vector of the error matrix E_k of the signals
  that use it (their residuals with atom k's contribution added back), and
  those signals' coefficients on atom k by E_k^T d_k, so each visit is the
  best rank-one fit of E_k restricted to the existing support.
* Sec. III, "Learning cross-scale sparse models": Step 1 runs K-SVD on the
  downsampled training set W X and keeps the coarse supports; Step 2 runs
  K-SVD on X with the sparse-coding step restricted to the children
  f(Omega_low) of each signal's coarse support (zero-tree OMP).
* Sec. III, "Initialization of dictionary", heuristics 1-4: the coarse
  dictionary starts from randomly picked (downsampled) training signals; the
  children of coarse atom k start from randomly picked signals of X|Omega_k
  (the signals whose coarse support holds k); an unused atom is replaced by
  the least-represented training signal, for a fine atom the least-represented
  signal of X|Omega_k of its parent k.

Readings taken where the passages are silent:

* Sign of the singular vector: the one with <d_new, d_old> >= 0 (an SVD fixes
  it only up to sign; this keeps an atom's sign across sweeps).
* E_k = 0 (every user of atom k is represented exactly without it): the atom
  is left as it is and its coefficients become E_k^T d_k = 0.
* "Least represented": the largest residual norm ||x_i - D s_i||^2 at the time
  the unused atom is visited, ties to the lowest index; the new atom is the
  signal itself normalised, and that signal is not picked again in the sweep.
  Signals with a zero norm are never picked.
* Random picks (initialisation) are passed in as uniform numbers u in [0, 1):
  the pick from an ordered list of n items is item floor(u n).

Approximate update (an option; Rubinstein, Zibulevsky and Elad, "Efficient
implementation of the K-SVD algorithm using Batch Orthogonal Matching
Pursuit", 2008): instead of the leading singular vector, one alternating step
from the current coefficients -- d_k = E_k^T alpha_k / ||E_k^T alpha_k||, then
alpha_k = E_k d_k -- each half minimises ||E_k - alpha d^T||_F over its own
variable, so the error never grows.  E_k^T alpha_k = 0 keeps the atom.
"""

from __future__ import annotations

from typing import List, Optional

import numpy as np

from .reference import omp_batch


def residuals(D: np.ndarray, X: np.ndarray, omega: np.ndarray, alpha: np.ndarray,
              k_eff: np.ndarray) -> np.ndarray:
    """R [N, M] with r_i = x_i - sum_j alpha_ij d_{omega_ij} (j < k_eff_i)."""
    D = np.asarray(D, np.float64)
    R = np.array(X, np.float64, copy=True)
    valid = np.arange(omega.shape[1])[None, :] < np.asarray(k_eff).reshape(-1, 1)
    for i0 in range(0, R.shape[0], 4096):      # blocks of signals bound the [n, K, M] temporary
        v = valid[i0:i0 + 4096]
        a = np.where(v, np.asarray(alpha[i0:i0 + 4096], np.float64), 0.0)
        idx = np.where(v, omega[i0:i0 + 4096], 0)
        R[i0:i0 + 4096] -= np.einsum("nk,nkm->nm", a, D[idx])
    return R


def atom_users(omega: np.ndarray, k_eff: np.ndarray, T: int):
    """For every atom k, the (signal i, slot j) pairs with omega[i, j] = k, i ascending."""
    valid = np.arange(omega.shape[1])[None, :] < np.asarray(k_eff).reshape(-1, 1)
    I, J = np.nonzero(valid)                       # row-major: i ascending
    atoms = np.asarray(omega)[I, J]
    order = np.argsort(atoms, kind="stable")
    cuts = np.searchsorted(atoms[order], np.arange(T + 1))
    return [list(zip(I[order[cuts[k]:cuts[k + 1]]].tolist(), J[order[cuts[k]:cuts[k + 1]]].tolist()))
            for k in range(T)]


def _eligible(k: int, taken, X_norm2, repl_parent, repl_support) -> np.ndarray:
    """Signals that may replace unused atom k: not yet taken, nonzero, and (with
    coarse parents) holding atom k's parent in their coarse support."""
    ok = ~taken & (X_norm2 > 0.0)
    if repl_parent is not None:
        ok &= np.any(np.asarray(repl_support) == int(repl_parent[k]), axis=1)
    return ok


def ksvd_update(D: np.ndarray, X: np.ndarray, omega: np.ndarray, alpha: np.ndarray,
                k_eff: np.ndarray, replace_unused: bool = False,
                repl_parent: Optional[np.ndarray] = None,
                repl_support: Optional[np.ndarray] = None, approximate: bool = False):
    """One dictionary-update sweep of K-SVD over atoms k = 0 .. T-1 in order.

    D: [T, M] atoms (rows); X: [N, M] training signals; omega/alpha [N, Kmax]
    supports (atom ids, -1 padded) and coefficients; k_eff [N].
    replace_unused: heuristics 3/4 for atoms without users; with repl_parent
    ([T], coarse parent of each atom) and repl_support ([N, Kc] coarse
    supports, -1 padded) only signals whose coarse support holds the atom's
    parent may replace it (heuristic 4), else any signal (heuristic 3).
    approximate: the one-step update from the current coefficients (module
    docstring) instead of the singular vector.
    Returns (D_new [T, M], alpha_new [N, Kmax], replaced: list of (k, i))."""
    D = np.array(D, np.float64, copy=True)
    A = np.array(alpha, np.float64, copy=True)
    X = np.asarray(X, np.float64)
    T = D.shape[0]
    R = residuals(D, X, omega, A, k_eff)
    users = atom_users(omega, k_eff, T)
    X_norm2 = np.einsum("ij,ij->i", X, X)
    taken = np.zeros(X.shape[0], bool)
    replaced = []
    for k in range(T):
        us = users[k]
        if not us:
            if not replace_unused:
                continue
            err = np.einsum("ij,ij->i", R, R)
            ok = _eligible(k, taken, X_norm2, repl_parent, repl_support)
            best_i = int(np.argmax(np.where(ok, err, -1.0))) if ok.any() else -1  # first maximum
            if best_i >= 0:
                D[k] = X[best_i] / np.sqrt(X_norm2[best_i])
                taken[best_i] = True
                replaced.append((k, best_i))
            continue
        I = np.array([u[0] for u in us])
        J = np.array([u[1] for u in us])
        E = R[I] + A[I, J][:, None] * D[k][None, :]        # rows e_i, [n, M]
        if approximate:
            g = E.T @ A[I, J]                              # E_k^T alpha_k
            ng = np.linalg.norm(g)
            u = g / ng if ng > 0.0 else D[k].copy()
            a = E @ u
            D[k] = u
            A[I, J] = a
            R[I] = E - a[:, None] * u[None, :]
            continue
        U, s, _ = np.linalg.svd(E.T, full_matrices=False)  # E^T = M x n
        if s[0] == 0.0:
            A[I, J] = E @ D[k]
            R[I] = E - A[I, J][:, None] * D[k][None, :]
            continue
        u = U[:, 0]
        if u @ D[k] < 0.0:
            u = -u
        a = E @ u
        D[k] = u
        A[I, J] = a
        R[I] = E - a[:, None] * u[None, :]
    return D, A, replaced


def pick(u: float, n: int) -> int:
    """Item floor(u n) of an ordered list of n items (u in [0, 1))."""
    return min(int(np.floor(u * n)), n - 1)


def init_coarse(X_low: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Heuristic 1: atom t = normalised training signal pick(u_t, n) of W X."""
    X_low = np.asarray(X_low, np.float64)
    D = np.zeros((len(u), X_low.shape[1]))
    for t, ut in enumerate(u):
        x = X_low[pick(float(ut), X_low.shape[0])]
        D[t] = x / np.linalg.norm(x)
    return D


def coarse_users(omega_low: np.ndarray, keff_low: np.ndarray, T_low: int) -> List[np.ndarray]:
    """Omega_k of the initialisation heuristics: the signals whose coarse
    support holds atom k, ascending."""
    return [np.array(sorted(i for i, _ in us), np.int64)
            for us in atom_users(omega_low, keff_low, T_low)]


def init_children(X: np.ndarray, parent: np.ndarray, omega_low: np.ndarray, keff_low: np.ndarray,
                  T_low: int, u: np.ndarray) -> np.ndarray:
    """Heuristic 2: fine atom j (a child of coarse atom parent[j]) = the
    normalised signal pick(u_j, |Omega_k|) of X|Omega_k, k = parent[j]; from
    all of X when no signal uses k."""
    X = np.asarray(X, np.float64)
    om = coarse_users(omega_low, keff_low, T_low)
    D = np.zeros((len(parent), X.shape[1]))
    for j, k in enumerate(parent):
        pool = om[int(k)]
        i = int(pool[pick(float(u[j]), len(pool))]) if len(pool) else pick(float(u[j]), X.shape[0])
        D[j] = X[i] / np.linalg.norm(X[i])
    return D


def restricted_coding(D_high: np.ndarray, X: np.ndarray, parent: np.ndarray, T_low: int,
                      omega_low: np.ndarray, keff_low: np.ndarray, K_high: int, nthreads: int = 0):
    """Step 2 sparse coding: OMP of each x_i over the children f(Omega_low,i)
    of its coarse support (the finer step of Algorithm 2)."""
    children = [np.flatnonzero(parent == p) for p in range(T_low)]
    D_high = np.asarray(D_high, np.float64)
    mats, cands = [], []
    for i in range(X.shape[0]):
        om = omega_low[i, :int(keff_low[i])]
        C = np.sort(np.concatenate([children[p] for p in om])) if len(om) else np.zeros(0, np.int64)
        cands.append(C)
        mats.append(D_high[C])
    o, a, k, r = omp_batch(mats, np.asarray(X, np.float64), K_high, nthreads=nthreads)
    for i, C in enumerate(cands):
        v = o[i] >= 0
        o[i, v] = C[o[i, v]]
    return o, a, k, r


def modified_ksvd(X: np.ndarray, X_low: np.ndarray, parent: np.ndarray, K_low: int, K_high: int,
                  u_low: np.ndarray, u_high: np.ndarray, iters_low: int, iters_high: int,
                  replace_unused: bool = True, nthreads: int = 0, approximate: bool = False):
    """Sec. III, learning cross-scale models: Step 1 (K-SVD on W X from heuristic 1), Step 2 (K-SVD on X
    from heuristic 2 with the coding restricted to f(Omega_low)).

    Each iteration codes every signal, then sweeps the atoms.  Returns
    (D_low, D_high, omega_low, keff_low, err_low, err_high): err_* are the
    squared Frobenius errors ||X - D S||_F^2 after each dictionary update."""
    n = X.shape[0]
    T_low = len(u_low)
    D_low = init_coarse(X_low, u_low)
    err_low = []
    for _ in range(iters_low):
        o, a, k, _ = omp_batch([D_low] * n, X_low, K_low, nthreads=nthreads)
        D_low, a, _ = ksvd_update(D_low, X_low, o, a, k, replace_unused, approximate=approximate)
        err_low.append(float(np.sum(residuals(D_low, X_low, o, a, k) ** 2)))
    om_low, _, ke_low, _ = omp_batch([D_low] * n, X_low, K_low, nthreads=nthreads)
    D_high = init_children(X, parent, om_low, ke_low, T_low, u_high)
    err_high = []
    for _ in range(iters_high):
        o, a, k, _ = restricted_coding(D_high, X, parent, T_low, om_low, ke_low, K_high, nthreads)
        D_high, a, _ = ksvd_update(D_high, X, o, a, k, replace_unused, parent, om_low, approximate)
        err_high.append(float(np.sum(residuals(D_high, X, o, a, k) ** 2)))
    return D_low, D_high, om_low, ke_low, err_low, err_high
