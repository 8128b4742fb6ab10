"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test names the paper passage (arXiv 1511.05174) or the mathematical fact
it rests on.  All run on the CPU.
"""

import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _omp(A_tm, y, K, **kw):
    o, a, k, r = oracle.omp_batch([A_tm], y[None], K, **kw)
    return o[0, :k[0]], a[0, :k[0]], int(k[0]), float(r[0])


def _two_ortho_bases():
    """[I | H/4], 16 x 32, coherence 1/4 (Hadamard entries +-1/4 after scaling)."""
    H = scipy.linalg.hadamard(16) / 4.0
    return np.hstack([np.eye(16), H])  # M x T


# ---------------------------------------------------------------- projection

def test_k1_closed_form():
    """Algorithm 1 with K = 1: alpha = <a, y> / ||a||^2 for the chosen atom."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((20, 12)) * rng.uniform(0.5, 2, size=12)  # M x T
    for _ in range(20):
        y = rng.standard_normal(20)
        om, al, k, _ = _omp(A.T, y, 1)
        a = A[:, om[0]]
        assert k == 1
        assert al[0] == pytest.approx(a @ y / (a @ a), rel=1e-12)


def test_projection_matches_lapack_lstsq():
    """Projection step = least squares; LAPACK's gelsd (numpy lstsq) agrees."""
    rng = np.random.default_rng(2)
    for M, T, K in [(16, 32, 4), (30, 50, 8), (64, 256, 12)]:
        A = rng.standard_normal((M, T))
        y = rng.standard_normal(M)
        om, al, k, rsq = _omp(A.T, y, K)
        ref, *_ = np.linalg.lstsq(A[:, om], y, rcond=None)
        np.testing.assert_allclose(al, ref, rtol=1e-9, atol=1e-12)
        assert rsq == pytest.approx(float(np.sum((y - A[:, om] @ ref) ** 2)), rel=1e-8)


def test_residual_orthogonal_to_selected_atoms():
    """LS optimality: A_Omega^T r = 0 (normal equations)."""
    rng = np.random.default_rng(3)
    M, T, K = 64, 256, 10
    A = rng.standard_normal((M, T))
    for _ in range(10):
        y = rng.standard_normal(M)
        om, al, k, _ = _omp(A.T, y, K)
        r = y - A[:, om] @ al
        assert np.max(np.abs(A[:, om].T @ r)) <= 1e-10 * np.linalg.norm(A, 2) * np.linalg.norm(y)


def test_residual_monotone():
    """||r_n|| <= ||r_{n-1}||: each support contains the previous one."""
    rng = np.random.default_rng(4)
    M, T = 32, 96
    A = rng.standard_normal((M, T))
    y = rng.standard_normal(M)
    prev = float(y @ y)
    for K in range(1, 16):
        _, _, _, rsq = _omp(A.T, y, K)
        assert rsq <= prev * (1 + 1e-12)
        prev = rsq


# ---------------------------------------------------------------- proxy / greedy sequence

def _brute_force_greedy(A, y, K):
    """Independent greedy re-implementation: fresh lstsq each step, angle proxy,
    lowest index on ties."""
    norms = np.linalg.norm(A, axis=0)
    S = []
    r = y.copy()
    for _ in range(K):
        sc = np.abs(A.T @ r) / norms
        sc[S] = -1
        k = int(np.flatnonzero(sc == sc.max())[0])
        S.append(k)
        c, *_ = np.linalg.lstsq(A[:, S], y, rcond=None)
        r = y - A[:, S] @ c
    return S


def test_greedy_sequence_brute_force():
    rng = np.random.default_rng(5)
    for trial in range(50):
        A = rng.standard_normal((16, 32)) * rng.uniform(0.5, 2, size=32)
        y = rng.standard_normal(16)
        K = 1 + trial % 4
        om, _, _, _ = _omp(A.T, y, K)
        assert list(om) == _brute_force_greedy(A, y, K)


def test_tie_break_lowest_index():
    """Equal scores: the lowest atom index wins (duplicate atoms at 3 and 7)."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((8, 10))
    A[:, 7] = A[:, 3]
    y = A[:, 3] * 2.0
    om, al, k, _ = _omp(A.T, y, 1)
    assert om[0] == 3 and al[0] == pytest.approx(2.0)


def test_unnormalised_proxy_flag():
    """normalize=0 is Algorithm 1's |<d_i, r>| literally: with unequal norms the
    larger atom can win although the smaller is closer in angle."""
    A = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    A[:, 1] = np.array([0.6, 0.8, 0.0]) * 10.0
    y = np.array([1.0, 0.1, 0.0])
    om_n, _, _, _ = _omp(A.T, y, 1, normalize=True)
    om_u, _, _, _ = _omp(A.T, y, 1, normalize=False)
    assert om_n[0] == 0 and om_u[0] == 1


# ---------------------------------------------------------------- support optimality

def _exhaustive_best(A, y, K):
    best, best_S = math.inf, None
    for S in itertools.combinations(range(A.shape[1]), K):
        c, *_ = np.linalg.lstsq(A[:, list(S)], y, rcond=None)
        e = float(np.sum((y - A[:, list(S)] @ c) ** 2))
        if e < best - 1e-12:
            best, best_S = e, set(S)
    return best, best_S


@pytest.mark.parametrize("K", [1, 2])
def test_exhaustive_search_two_orthobases(K):
    """Problem (P0), Sec. II-B, on [I | H/4]: coherence 1/4 < 1/(2K-1), so OMP
    recovers every K-sparse signal exactly (Tropp 2004, exact recovery
    condition); the exhaustive minimiser over all C(32, K) supports, the true
    support and OMP's support coincide."""
    A = _two_ortho_bases()
    rng = np.random.default_rng(7 + K)
    for _ in range(25):
        S = sorted(rng.choice(32, K, replace=False))
        y = A[:, S] @ (rng.standard_normal(K) + np.sign(rng.standard_normal(K)))
        best, best_S = _exhaustive_best(A, y, K)
        om, al, k, rsq = _omp(A.T, y, K)
        assert best_S == set(S) == set(om)
        assert rsq <= 1e-20 * float(y @ y) + 1e-30


@pytest.mark.parametrize("K", [1, 2])
def test_exhaustive_search_gaussian_bound(K):
    """Random 16 x 32 Gaussian: OMP's error is never below the exhaustive
    optimum, and with K = 1 the two coincide (one greedy step is exhaustive)."""
    rng = np.random.default_rng(17 + K)
    A = rng.standard_normal((16, 32))
    for _ in range(25):
        y = rng.standard_normal(16)
        best, best_S = _exhaustive_best(A, y, K)
        om, al, k, rsq = _omp(A.T, y, K)
        assert rsq >= best - 1e-10
        if K == 1:
            # the best single atom maximises |<a, y>| / ||a|| (residual ||y||^2 - <a,y>^2/||a||^2)
            assert set(om) == best_S


def test_exact_recovery_noiseless_denoise_sizes():
    """Noiseless K-sparse signals with the denoise sizes (D 64 x 256, K = 4):
    the residual vanishes (down to the float32 rounding of the stored y) and the
    support is recovered on almost every patch."""
    A, Y, sup = synthetic.make_independent_problems(64, 64, 256, 4, seed=11, unit_norm=True)
    o, a, k, rsq = oracle.omp_batch([A] * 64, Y, 4)
    yy = np.sum(Y.astype(np.float64) ** 2, axis=1)
    hits = sum(set(o[b, :k[b]]) == set(sup[b]) for b in range(64))
    assert hits >= 62
    good = np.array([set(o[b, :k[b]]) == set(sup[b]) for b in range(64)])
    assert np.all(rsq[good] <= 1e-12 * yy[good])


# ---------------------------------------------------------------- degenerate cases

def test_zero_measurement_gives_empty_support():
    A = np.random.default_rng(8).standard_normal((10, 20))
    om, al, k, rsq = _omp(A.T, np.zeros(10), 5)
    assert k == 0 and rsq == 0.0


def test_dependent_atom_stops_early_without_nan():
    """Atom 5 = atom 1 + atom 2: once 1 and 2 are chosen, 5 adds nothing; a
    candidate set {1, 2, 5} exhausts after two atoms with no NaN."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((12, 3))
    A[:, 2] = A[:, 0] + A[:, 1]
    y = A[:, 0] + 0.5 * A[:, 1] + 1e-3 * rng.standard_normal(12)
    om, al, k, rsq = _omp(A.T, y, 3)
    assert k == 2 and np.all(np.isfinite(al))


def test_zero_column_is_never_chosen():
    A = np.random.default_rng(10).standard_normal((8, 6))
    A[:, 0] = 0.0
    om, al, k, _ = _omp(A.T, np.ones(8), 6)
    assert 0 not in om and k == 5


# ---------------------------------------------------------------- operators and geometry

def test_patch_origins_ragged_tail():
    assert list(oracle.patch_origins(10, 4, 4)) == [0, 4, 6]
    assert list(oracle.patch_origins(12, 4, 4)) == [0, 4, 8]
    assert list(oracle.patch_origins(512, 8, 2))[-1] == 504 and len(oracle.patch_origins(512, 8, 2)) == 253
    assert len(oracle.patch_origins(3, 4, 1)) == 0
    assert synthetic.patch_count_1d(10, 4, 4) == 3


@pytest.mark.parametrize("name", ["denoise", "bayer", "video", "lightfield", "inpaint", "cs_dense"])
def test_WU_identity_and_nearest_neighbour(name):
    """W U = I on R^{N_low} (Sec. III-C), U replicates each coarse entry."""
    w = synthetic.make_workload(name, H=16, W=16, T0=64)
    g = w.geometry
    rng = np.random.default_rng(0)
    for l in range(1, g.n_levels):
        Nl = g.level_dim(l)
        V = rng.standard_normal((3, Nl))
        np.testing.assert_allclose(oracle.W_down(oracle.U_up(V, g, l), g, l), V, atol=1e-14)
        e = np.zeros((1, Nl)); e[0, 0] = 1.0
        u = oracle.U_up(e, g, l)
        assert np.count_nonzero(u) == g.level_dim(0) // Nl and set(np.unique(u)) == {0.0, 1.0}


@pytest.mark.parametrize("name", ["denoise", "bayer", "video", "lightfield", "inpaint", "cs_dense"])
def test_extraction_matches_camera_model(name):
    """Noiseless: the extracted patch equals Phi_p applied to the ground-truth
    patch (y = Phi x, Sec. III-C).  The camera simulation lives in the input
    generator, written independently of the oracle's Phi."""
    w = synthetic.make_workload(name, H=24, W=24, T0=64, sigma=0.0)
    g = w.geometry
    Y = oracle.extract_patches(w)
    oy, ox = oracle.patch_grid(g)
    for b in range(0, len(oy), 7):
        x = w.truth[:, oy[b]:oy[b] + g.P, ox[b]:ox[b] + g.P].reshape(1, -1)
        np.testing.assert_allclose(oracle.phi_apply(w.sensing, g, int(oy[b]), int(ox[b]), x)[0], Y[b],
                                   rtol=1e-6, atol=1e-6)


def test_inpainting_operator_keeps_the_retained_pixels():
    """Random pixel retention (the paper's inpainting task, Sec. IV): the
    operator of a patch is the diagonal 0/1 mask of its retained pixels, so
    every effective atom is the atom with the removed pixels set to zero and
    OMP's angle score uses the norm over the retained pixels only."""
    w = synthetic.make_workload("inpaint", H=16, W=16, T0=64)
    g = w.geometry
    oy, ox = oracle.patch_grid(g)
    for b in range(0, len(oy), 5):
        Phi = oracle.sensing_matrix(w.sensing, g, int(oy[b]), int(ox[b]))
        mask = w.sensing.codes[0, oy[b]:oy[b] + g.P, ox[b]:ox[b] + g.P].reshape(-1).astype(float)
        np.testing.assert_array_equal(Phi, np.diag(mask))
    assert 0.4 < w.sensing.codes.mean() < 0.6  # N/M = 2


def test_bayer_matrix_rows_are_rggb_selectors():
    w = synthetic.make_workload("bayer", H=16, W=16, T0=64)
    g = w.geometry
    for oy, ox in [(0, 0), (0, 1), (1, 0), (1, 1)]:
        Phi = oracle.sensing_matrix(w.sensing, g, oy, ox)
        assert Phi.shape == (64, 192)
        assert np.all(Phi.sum(axis=1) == 1)
        py, px = 0, 0
        ch = int(np.flatnonzero(Phi[0])[0]) // 64
        assert ch == {(0, 0): 0, (0, 1): 1, (1, 0): 1, (1, 1): 2}[(oy, ox)]


def test_aggregation_reproduces_image_with_pixel_dictionary():
    """D = I (one atom per pixel), alpha = the true patch: overlap-add with
    averaging returns the image exactly, at any stride."""
    w = synthetic.make_workload("bayer", H=24, W=24, T0=64, sigma=0.0)
    g = w.geometry
    N = g.planes * g.P * g.P
    w.dicts = [np.eye(N, dtype=np.float32)] + w.dicts[1:]
    oy, ox = oracle.patch_grid(g)
    B = len(oy)
    om = np.tile(np.arange(N, dtype=np.int32), (B, 1))
    al = np.stack([w.truth[:, oy[b]:oy[b] + g.P, ox[b]:ox[b] + g.P].ravel() for b in range(B)])
    img = oracle.aggregate(w, om, al, np.full(B, N))
    np.testing.assert_allclose(img, w.truth, atol=1e-12)


def test_snr_psnr_closed_forms():
    gt = np.zeros((1, 4, 4)); gt[0, 0, 0] = 2.0   # ||x|| = 2, peak 2
    est = gt.copy(); est[0, 1, 1] = 0.2           # error norm 0.2, MSE 0.04/16
    assert oracle.snr(gt, est) == pytest.approx(20.0)
    assert oracle.psnr(gt, est) == pytest.approx(10 * math.log10(4.0 / (0.04 / 16)))


# ---------------------------------------------------------------- cross-scale (Algorithm 2)

def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([c.strip() for c in line.split("|")])
    return rows


def _block_parents(T_high, Q):
    return (np.arange(T_high) // Q).astype(np.int32)


def test_block_map_golden():
    """Sec. III-B block rule, 1-based in the paper; parent(j) = floor(j / Q) 0-based."""
    for Q, om, f in _read_golden("block_map.txt"):
        Q = int(Q)
        om = [int(v) - 1 for v in om.split(",")]
        f = [int(v) - 1 for v in f.split(",")]
        T_low = max(om) + 2
        ch = oracle.children_lists(_block_parents(T_low * Q, Q), T_low)
        got = sorted(np.concatenate([ch[p] for p in om]).tolist())
        assert got == f
        assert len(got) == Q * len(om)


def _tiny_denoise(links_parent, T_high, T_low, K_high, K_low, sigma=0.01, seed=0):
    w = synthetic.make_workload("denoise", seed=seed, T0=T_high, sigma=sigma)
    g = w.geometry
    rng = np.random.default_rng(seed + 100)
    D_low = rng.standard_normal((T_low, g.level_dim(1)))
    D_low /= np.linalg.norm(D_low, axis=1, keepdims=True)
    w.dicts = [w.dicts[0], D_low.astype(np.float32)]
    w.parents = [links_parent.astype(np.int32)]
    B = w.n_patches
    w.K_levels = [np.full(B, K_high, np.int32), np.full(B, K_low, np.int32)]
    return w


def test_speedup_model_proxy_flops_golden():
    """Proxy work of plain vs zero-tree OMP (Sec. III-C, theoretical speedup):
    with the (P_low) operator (same dimension N) and K_low = K_high the
    counted proxy flops give exactly T_high / (T_low + K_low Q)."""
    for params, ratio in _read_golden("speedup_model.txt"):
        Th, Tl, K, Q = (int(v) for v in params.split())
        ratio = float(ratio)
        w = _tiny_denoise(_block_parents(Th, Q), Th, Tl, K, K)
        Y = oracle.extract_patches(w)
        N = Y.shape[1]
        D0 = w.dicts[0].astype(np.float64)
        _, _, k0, _, f_plain = oracle.omp_batch([D0] * len(Y), Y, K, return_flops=True)
        UD = oracle.U_up(w.dicts[1].astype(np.float64), w.geometry, 1)
        oc, _, kc, _, f_c = oracle.omp_batch([UD] * len(Y), Y, K, return_flops=True)
        ch = oracle.children_lists(w.parents[0], Tl)
        f_f = 0
        for b in range(len(Y)):
            C = np.sort(np.concatenate([ch[p] for p in oc[b, :kc[b]]]))
            assert len(C) == Q * K                       # |f(Omega)| = Q K_low
            *_, fl = oracle.omp_batch([D0[C]], Y[b:b + 1], K, return_flops=True)
            f_f += int(fl[0])
        assert np.all(k0 == K) and np.all(kc == K)
        assert int(f_plain.sum()) == 2 * N * Th * K * len(Y)
        assert int(f_c.sum()) + f_f == 2 * N * (Tl * K + Q * K * K) * len(Y)
        assert f_plain.sum() / (f_c.sum() + f_f) == pytest.approx(ratio, rel=1e-9)


def test_cross_scale_with_all_atoms_equals_plain():
    """One coarse atom whose children are all fine atoms and K_low = 1: the
    candidate set f(Omega_low) is the whole dictionary, so Algorithm 2's fine
    step is Algorithm 1 -- identical output."""
    w = _tiny_denoise(np.zeros(256, np.int32), 256, 1, 4, 1)
    o_p, a_p, k_p, _ = oracle.plain_omp(w)
    o_c, a_c, k_c, _ = oracle.cross_scale_omp(w)
    np.testing.assert_array_equal(o_p, o_c)
    np.testing.assert_array_equal(a_p, a_c)
    np.testing.assert_array_equal(k_p, k_c)


@pytest.mark.parametrize("links", ["paper", "literal"])
def test_coarse_form_equivalence_identity(links):
    """Phi = I: Algorithm 2's coarse step on W x against D_low and (P_low) on x
    against U D_low choose the same atoms with the same coefficients."""
    w = synthetic.make_workload("denoise", links=links)
    lv_w = oracle.cross_scale_omp(w, coarse_form="wx", return_levels=True)
    lv_p = oracle.cross_scale_omp(w, coarse_form="p_low", return_levels=True)
    for (o1, a1, k1, _), (o2, a2, k2, _) in zip(lv_w, lv_p):
        np.testing.assert_array_equal(o1, o2)
        np.testing.assert_array_equal(k1, k2)
        np.testing.assert_allclose(a1, a2, rtol=1e-9, atol=1e-12)


def test_literal_links_fine_step_is_ls_on_coarse_support():
    """Identity links and K_low = K_high: f(Omega_low) = Omega_low, so the fine
    step chooses all of it and returns the least-squares fit on it."""
    w = synthetic.make_workload("denoise", links="literal")
    lv = oracle.cross_scale_omp(w, return_levels=True)
    o0, a0, k0, _ = lv[0]
    o1, a1, k1, _ = lv[1]
    Y = oracle.extract_patches(w)
    D0 = w.dicts[0].astype(np.float64)
    for b in range(len(Y)):
        assert set(o0[b, :k0[b]]) == set(o1[b, :k1[b]])
        ref, *_ = np.linalg.lstsq(D0[o0[b, :k0[b]]].T, Y[b], rcond=None)
        np.testing.assert_allclose(a0[b, :k0[b]], ref, rtol=1e-8, atol=1e-10)


def test_fine_support_lies_in_predicted_set():
    """Cross-scale prediction property (Sec. III-A): Omega_high is a subset of
    f(Omega_low), for every level of a three-scale tree."""
    w = synthetic.make_workload("video", H=16, W=16, T0=256)
    lv = oracle.cross_scale_omp(w, return_levels=True)
    for l in range(w.n_levels - 1):
        ch = oracle.children_lists(w.parents[l], w.dicts[l + 1].shape[0])
        o_f, _, k_f, _ = lv[l]
        o_c, _, k_c, _ = lv[l + 1]
        for b in range(o_f.shape[0]):
            allowed = set(np.concatenate([ch[p] for p in o_c[b, :k_c[b]]]).tolist()) if k_c[b] else set()
            assert set(o_f[b, :k_f[b]].tolist()) <= allowed
            assert k_f[b] == min(int(w.K_levels[l][b]), len(allowed))


# ---------------------------------------------------------------- per-patch operators

@pytest.mark.parametrize("name,H", [("bayer", 24), ("inpaint", 24), ("video", 16)])
def test_per_patch_operator_selection_equals_direct_construction(name, H):
    """Sec. III-C, y_p = Phi_p x_p: the oracle hands every patch the effective
    dictionary of its own operator (Bayer: one per mosaic phase (oy % 2, ox % 2),
    shared by the patches of that phase; per-pixel codes: one per patch).  At
    stride 1 every phase occurs; the oracle's plain and cross-scale OMP must equal
    OMP against Phi_p U_l D^(l) written out densely for each patch on its own,
    from its origin, with no sharing between patches."""
    kw = dict(T0=256) if name == "video" else {}
    w = synthetic.make_workload(name, H=H, W=H, **kw)
    w.geometry.stride = 1
    B = w.n_patches
    w.K_levels = [np.full(B, int(k[0]), np.int32) for k in w.K_levels]
    g, s = w.geometry, w.sensing
    Y = oracle.extract_patches(w)
    oy, ox = oracle.patch_grid(g)
    assert {(int(a) % 2, int(b) % 2) for a, b in zip(oy, ox)} == {(0, 0), (0, 1), (1, 0), (1, 1)}

    def level_mats(l):
        D = w.dicts[l].astype(np.float64)
        UD = oracle.U_up(D, g, l) if l else D
        return [UD @ oracle.sensing_matrix(s, g, int(oy[b]), int(ox[b])).T for b in range(B)]

    o, a, k, _ = oracle.plain_omp(w, Y=Y)
    o2, a2, k2, _ = oracle.omp_batch(level_mats(0), Y, w.K_levels[0])
    np.testing.assert_array_equal(k, k2)
    np.testing.assert_array_equal(o, o2)
    np.testing.assert_allclose(a, a2, rtol=1e-9, atol=1e-12)

    # Algorithm 2 level by level with the directly built operators (P_low form)
    L = w.n_levels
    om, ke = None, None
    for l in range(L - 1, -1, -1):
        mats = level_mats(l)
        if l == L - 1:
            om, al, ke, _ = oracle.omp_batch(mats, Y, w.K_levels[l])
            continue
        ch = oracle.children_lists(w.parents[l], w.dicts[l + 1].shape[0])
        C = [np.sort(np.concatenate([ch[p] for p in om[b, :ke[b]]])) for b in range(B)]
        om, al, ke, _ = oracle.omp_batch([mats[b][C[b]] for b in range(B)], Y, w.K_levels[l])
        om = np.array([[C[b][j] if j >= 0 else -1 for j in om[b]] for b in range(B)], np.int32)
    o, a, k, _ = oracle.cross_scale_omp(w, Y=Y, coarse_form="p_low")
    np.testing.assert_array_equal(k, ke)
    np.testing.assert_array_equal(o[:, :om.shape[1]], om)
    np.testing.assert_allclose(a[:, :al.shape[1]], al, rtol=1e-9, atol=1e-12)
