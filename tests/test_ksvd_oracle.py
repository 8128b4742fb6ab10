"""Pins of the K-SVD oracle (oracle/ksvd.py) against facts that do not come
from it: exhaustive search over unit vectors in the plane, closed forms of
rank-one data, Eckart-Young, and invariants of the update.  All CPU.

Passages: Sec. II, "Dictionary learning" (K-SVD: alternate sparse coding and
an atom-by-atom rank-one dictionary update); Sec. III, "Learning cross-scale
sparse models" (Steps 1 and 2) and "Initialization of dictionary"
(heuristics 1-4).
"""

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

import oracle
from oracle import ksvd
import synthetic


def _random_problem(rng, N, M, T, K):
    D = rng.standard_normal((T, M))
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    X = rng.standard_normal((N, M))
    om = np.stack([np.sort(rng.choice(T, K, replace=False)) for _ in range(N)]).astype(np.int32)
    al = rng.standard_normal((N, K))
    ke = np.full(N, K, np.int32)
    return D, X, om, al, ke


def _objective(D, X, om, al, ke):
    err = 0.0
    for i in range(X.shape[0]):
        r = X[i] - sum(al[i, j] * D[om[i, j]] for j in range(int(ke[i])))
        err += float(r @ r)
    return err


def test_plane_sweep_matches_exhaustive_search():
    """M = 2: each visit maximises ||E_k^T d|| over unit d = (cos t, sin t);
    a sequential sweep written from that definition with a bounded scalar
    search (no SVD) gives the oracle's atoms and coefficients."""
    rng = np.random.default_rng(3)
    N, M, T, K = 9, 2, 3, 2
    D, X, om, al, ke = _random_problem(rng, N, M, T, K)
    Dn, An, _ = ksvd.ksvd_update(D, X, om, al, ke)

    Dr, Ar = D.copy(), al.copy()
    for k in range(T):
        rows = [(i, j) for i in range(N) for j in range(K) if om[i, j] == k]
        E = np.stack([X[i] - sum(Ar[i, jj] * Dr[om[i, jj]] for jj in range(K) if jj != j)
                      for i, j in rows])

        def neg(t):
            d = np.array([np.cos(t), np.sin(t)])
            return -float(np.sum((E @ d) ** 2))
        grid = np.linspace(0.0, np.pi, 4001)
        t0 = grid[np.argmin([neg(t) for t in grid])]
        t = scipy.optimize.minimize_scalar(neg, bounds=(t0 - 1e-3, t0 + 1e-3), method="bounded",
                                           options={"xatol": 1e-12}).x
        d = np.array([np.cos(t), np.sin(t)])
        if d @ Dr[k] < 0:
            d = -d
        Dr[k] = d
        for (i, j), a in zip(rows, E @ d):
            Ar[i, j] = a
    np.testing.assert_allclose(Dn, Dr, atol=1e-7)
    np.testing.assert_allclose(An, Ar, atol=1e-6)


def test_rank_one_users_recover_the_atom():
    """K = 1 and x_i = c_i g_{k_i}: E_k is rank one, so the sweep returns
    d_k = +-g_k (sign of the starting atom) and alpha_i = +-c_i exactly."""
    rng = np.random.default_rng(5)
    N, M, T = 40, 7, 5
    G = rng.standard_normal((T, M))
    G /= np.linalg.norm(G, axis=1, keepdims=True)
    k_of = np.arange(N) % T
    c = rng.uniform(0.5, 2.0, N) * rng.choice([-1, 1], N)
    X = c[:, None] * G[k_of]
    D0 = G + 0.3 * rng.standard_normal((T, M))
    D0 /= np.linalg.norm(D0, axis=1, keepdims=True)
    D0[1] = -D0[1]                       # start one atom on the opposite sign
    om = k_of[:, None].astype(np.int32)
    al = rng.standard_normal((N, 1))
    Dn, An, _ = ksvd.ksvd_update(D0, X, om, al, np.ones(N, np.int32))
    s = np.sign(np.sum(D0 * G, axis=1))
    np.testing.assert_allclose(Dn, s[:, None] * G, atol=1e-12)
    np.testing.assert_allclose(An[:, 0], s[k_of] * c, atol=1e-12)
    assert np.allclose(ksvd.residuals(Dn, X, om, An, np.ones(N)), 0.0, atol=1e-12)


def test_visit_reaches_eckart_young_and_the_objective_never_grows():
    """A single atom used by every signal: after its visit the error is
    ||X||_F^2 - lambda_max(X^T X) (eigvalsh, not an SVD).  Over a sweep of
    many atoms the total error never grows, atoms stay unit norm, and padded
    slots stay zero."""
    rng = np.random.default_rng(11)
    N, M = 50, 6
    X = rng.standard_normal((N, M))
    d0 = rng.standard_normal((1, M))
    d0 /= np.linalg.norm(d0)
    D1, A1, _ = ksvd.ksvd_update(d0, X, np.zeros((N, 1), np.int32), rng.standard_normal((N, 1)),
                                 np.ones(N, np.int32))
    e1 = float(np.sum((X - A1[:, :1] * D1[0]) ** 2))
    lam = scipy.linalg.eigvalsh(X.T @ X)[-1]
    assert e1 == pytest.approx(float(np.sum(X * X)) - lam, rel=1e-10)

    N, M, T, K = 120, 6, 10, 3
    D, X, om, al, ke = _random_problem(rng, N, M, T, K)
    ke[::7] = 2
    om[::7, 2] = -1
    al[::7, 2] = 0.0
    before = _objective(D, X, om, al, ke)
    Dn, An, _ = ksvd.ksvd_update(D, X, om, al, ke)
    after = _objective(Dn, X, om, An, ke)
    assert after <= before * (1 + 1e-12)
    np.testing.assert_allclose(np.linalg.norm(Dn, axis=1), 1.0, atol=1e-12)
    assert np.all(An[::7, 2] == 0.0)


def test_unused_atom_replacement_heuristics():
    """Heuristic 3: an unused atom becomes the normalised signal with the
    largest residual (computed here from the definition), which is not picked
    twice.  Heuristic 4: only signals whose coarse support holds the atom's
    parent qualify."""
    rng = np.random.default_rng(2)
    N, M, T, K = 30, 5, 6, 2
    D, X, om, al, ke = _random_problem(rng, N, M, T, K)
    om[om == 4] = 5                       # atoms 3 and 4 unused
    om[om == 3] = 0
    for i in range(N):                    # keep supports distinct
        if om[i, 0] == om[i, 1]:
            om[i, 1] = 1 if om[i, 0] != 1 else 2
    Dn, An, rep = ksvd.ksvd_update(D, X, om, al, ke, replace_unused=True)
    assert [k for k, _ in rep] == [3, 4]
    i3, i4 = rep[0][1], rep[1][1]
    assert i3 != i4
    np.testing.assert_allclose(Dn[3], X[i3] / np.linalg.norm(X[i3]), atol=1e-12)
    np.testing.assert_allclose(Dn[4], X[i4] / np.linalg.norm(X[i4]), atol=1e-12)
    # atom 5 (visited after) changes residuals; at the visit of atoms 3 and 4 only
    # atoms 0..2 had been updated: rebuild that state from the final atoms 0..2
    D_mid = D.copy()
    D_mid[:3] = Dn[:3]
    A_mid = al.copy()
    A_mid[om <= 2] = An[om <= 2]
    e_mid = np.array([np.sum((X[i] - sum(A_mid[i, j] * D_mid[om[i, j]] for j in range(K))) ** 2)
                      for i in range(N)])
    assert i3 == int(np.argmax(e_mid))
    e2 = e_mid.copy()
    e2[i3] = -1
    assert i4 == int(np.argmax(e2))
    # heuristic 4: parent of atom 3 is coarse atom 1; only signals 0..9 hold it
    parent = np.array([0, 0, 1, 1, 2, 2], np.int32)
    sup_low = np.full((N, 1), 0, np.int32)
    sup_low[:10, 0] = 1
    sup_low[10:20, 0] = 2
    _, _, rep4 = ksvd.ksvd_update(D, X, om, al, ke, True, parent, sup_low)
    k3 = dict(rep4)[3]
    assert k3 < 10 and k3 == int(np.argmax(np.where(np.arange(N) < 10, e_mid, -1)))
    assert 10 <= dict(rep4)[4] < 20


def test_initialisation_picks():
    """Heuristics 1 and 2 with the floor(u n) pick rule on hand-checked lists."""
    X_low = np.arange(1, 13, dtype=float).reshape(6, 2)
    D = ksvd.init_coarse(X_low, np.array([0.0, 0.5, 0.999]))
    for t, i in enumerate([0, 3, 5]):
        np.testing.assert_allclose(D[t], X_low[i] / np.linalg.norm(X_low[i]))
    X = np.arange(1, 19, dtype=float).reshape(6, 3)
    om_low = np.array([[0, 1], [1, -1], [0, -1], [1, 0], [2, -1], [1, -1]], np.int32)
    ke_low = np.array([2, 1, 1, 2, 1, 1])
    parent = np.array([0, 0, 1, 1, 3])
    u = np.array([0.0, 0.99, 0.26, 0.5, 0.75])
    D = ksvd.init_children(X, parent, om_low, ke_low, 4, u)
    # Omega_0 = {0, 2, 3}, Omega_1 = {0, 1, 3, 5}, Omega_3 = {} (pick from all 6)
    for j, i in enumerate([0, 3, 1, 3, 4]):
        np.testing.assert_allclose(D[j], X[i] / np.linalg.norm(X[i]))


def test_modified_ksvd_reduces_error_and_keeps_zero_tree_supports():
    """Steps 1 and 2 on a planted two-scale training set: each step's error
    falls with every iteration, and every Step-2 support lies in the
    children of the signal's coarse support."""
    ts = synthetic.make_training_set("denoise", 600, seed=4, T0=64)
    g = ts.geometry
    X = ts.X.astype(np.float64)
    X_low = oracle.W_down(X, g, 1)
    parent = ts.parents[0]
    D_low, D_high, om_low, ke_low, el, eh = ksvd.modified_ksvd(
        X, X_low, parent, ts.K_low, ts.K_high, ts.u_low, ts.u_high, 3, 3)
    assert np.all(np.diff(el) < 0) and np.all(np.diff(eh) < 0)
    assert eh[-1] < 0.35 * float(np.sum(X * X))
    o, _, k, _ = ksvd.restricted_coding(D_high, X, parent, D_low.shape[0], om_low, ke_low, ts.K_high)
    for i in range(len(X)):
        allowed = set(np.flatnonzero(np.isin(parent, om_low[i, :ke_low[i]])))
        assert set(o[i, :k[i]]) <= allowed


def test_approximate_update_is_exact_on_rank_one_and_never_grows_the_error():
    """Approximate update (one alternating step from the current coefficients):
    on rank-one users it gives the singular vector like the exact update; on
    general data each visit minimises the error over d for fixed alpha and
    over alpha for fixed d, so the objective never grows, and it stays at or
    above the exact update's (Eckart-Young bound per visit)."""
    rng = np.random.default_rng(8)
    N, M, T = 40, 7, 5
    G = rng.standard_normal((T, M))
    G /= np.linalg.norm(G, axis=1, keepdims=True)
    k_of = np.arange(N) % T
    c = rng.uniform(0.5, 2.0, N) * rng.choice([-1, 1], N)
    X = c[:, None] * G[k_of]
    D0 = G + 0.3 * rng.standard_normal((T, M))
    D0 /= np.linalg.norm(D0, axis=1, keepdims=True)
    om = k_of[:, None].astype(np.int32)
    al = c[:, None] * np.sum(D0[k_of] * G[k_of], axis=1, keepdims=True)   # alpha = <x, d0>
    Da, Aa, _ = ksvd.ksvd_update(D0, X, om, al, np.ones(N, np.int32), approximate=True)
    De, Ae, _ = ksvd.ksvd_update(D0, X, om, al, np.ones(N, np.int32))
    np.testing.assert_allclose(Da, De, atol=1e-12)
    np.testing.assert_allclose(Aa, Ae, atol=1e-12)

    N, M, T, K = 150, 6, 12, 3
    D, X, om, al, ke = _random_problem(rng, N, M, T, K)
    before = _objective(D, X, om, al, ke)
    Da, Aa, _ = ksvd.ksvd_update(D, X, om, al, ke, approximate=True)
    after = _objective(Da, X, om, Aa, ke)
    assert after <= before * (1 + 1e-12)
    np.testing.assert_allclose(np.linalg.norm(Da, axis=1), 1.0, atol=1e-12)
    # one visit alone: approximate error >= exact error (exact is optimal)
    users = np.array([i for i in range(N) if 0 in om[i, :ke[i]]])
    sl = np.array([list(om[i]).index(0) for i in users])
    E = np.stack([X[i] - sum(al[i, j] * D[om[i, j]] for j in range(ke[i]) if om[i, j] != 0) for i in users])
    lam = scipy.linalg.eigvalsh(E.T @ E)[-1]
    D1, A1, _ = ksvd.ksvd_update(D[:1], E, np.zeros((len(users), 1), np.int32), al[users, sl][:, None],
                                 np.ones(len(users), np.int32), approximate=True)
    e1 = float(np.sum((E - A1[:, :1] * D1[0]) ** 2))
    assert e1 >= float(np.sum(E * E)) - lam - 1e-9


def test_step2_coding_is_the_fine_step_of_algorithm_2():
    """Step 2's coarse supports are those of Step 1's final coding (plain OMP
    on W x against the learned D_low): Step 2's coding (OMP over the children
    of those supports) then equals the finer level of Algorithm 2 run on the
    same pair of dictionaries, which recomputes the coarse supports from W x."""
    ts = synthetic.make_training_set("denoise", 300, seed=9, T0=64)
    g = ts.geometry
    X = ts.X.astype(np.float64)
    X_low = oracle.W_down(X, g, 1)
    D_high, D_low = ts.dicts[0].astype(np.float64), ts.dicts[1].astype(np.float64)
    parent = ts.parents[0]
    om_low, _, ke_low, _ = oracle.omp_batch([D_low] * len(X), X_low, ts.K_low)
    o, a, k, _ = ksvd.restricted_coding(D_high, X, parent, D_low.shape[0], om_low, ke_low, ts.K_high)

    class W:  # the two-level identity problem of these signals, one "patch" per signal
        pass
    w = W()
    w.geometry = g
    w.sensing = synthetic.Sensing("identity")
    w.dicts = [D_high, D_low]
    w.parents = [parent]
    w.n_levels = 2
    w.K_levels = [np.full(len(X), ts.K_high, np.int32), np.full(len(X), ts.K_low, np.int32)]
    o2, a2, k2, _ = oracle.cross_scale_omp(w, Y=X)
    np.testing.assert_array_equal(k, k2)
    for i in range(len(X)):
        assert list(o[i, :k[i]]) == list(o2[i, :k2[i]])
        np.testing.assert_allclose(a[i, :k[i]], a2[i, :k2[i]], rtol=1e-12, atol=1e-12)


def test_zero_error_matrix_keeps_the_atom():
    """E_k = 0: every user of atom k is represented exactly without it (here
    x_i = d_1 with coefficient 0 on d_0).  The update keeps d_0 unchanged (no
    singular vector exists; any unit vector would fit), sets its coefficients
    to E_k^T d_k = 0 and leaves the residuals at zero; atom 1's visit then sees
    the rank-one matrix of its users and keeps d_1 (the signals are d_1)."""
    rng = np.random.default_rng(31)
    D = rng.standard_normal((2, 12))
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    X = np.stack([D[1] * c for c in (1.0, -2.0, 0.5)])
    om = np.tile(np.array([[0, 1]], np.int32), (3, 1))
    al = np.stack([[0.0, 1.0], [0.0, -2.0], [0.0, 0.5]])
    ke = np.full(3, 2, np.int32)
    for approx in (False, True):
        Dn, An, rep = ksvd.ksvd_update(D, X, om, al, ke, approximate=approx)
        assert rep == []
        np.testing.assert_array_equal(Dn[0], D[0])
        np.testing.assert_array_equal(An[:, 0], 0.0)
        np.testing.assert_allclose(Dn[1], D[1], atol=1e-12)
        np.testing.assert_allclose(An[:, 1], [1.0, -2.0, 0.5], atol=1e-12)
        np.testing.assert_allclose(ksvd.residuals(Dn, X, om, An, ke), 0.0, atol=1e-12)
