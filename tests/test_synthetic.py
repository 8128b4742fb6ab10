"""The seeded input generator: reproducible, and one model can serve many
images (dictionaries and links seeded apart from the image content)."""

import itertools

import numpy as np
import pytest

import synthetic


def test_same_seed_same_workload():
    a = synthetic.make_workload("denoise", seed=3)
    b = synthetic.make_workload("denoise", seed=3)
    assert all(np.array_equal(x, y) for x, y in zip(a.dicts, b.dicts))
    assert np.array_equal(a.meas, b.meas)


def test_dict_seed_shares_the_model_only():
    base = synthetic.make_workload("bayer", seed=0, H=32, W=32)
    same = synthetic.make_workload("bayer", seed=0, H=32, W=32, dict_seed=0)
    other = synthetic.make_workload("bayer", seed=5, H=48, W=40, dict_seed=0)
    # dict_seed equal to seed changes nothing
    assert np.array_equal(base.meas, same.meas)
    # another image of the same model: same dictionaries and links, other content
    assert all(np.array_equal(x, y) for x, y in zip(base.dicts, other.dicts))
    assert all(np.array_equal(x, y) for x, y in zip(base.parents, other.parents))
    assert other.meas.shape == (48, 40)
    assert not np.array_equal(base.meas, other.meas[:32, :32])
    # and without dict_seed a different seed is a different model
    plain = synthetic.make_workload("bayer", seed=5, H=32, W=32)
    assert not np.array_equal(base.dicts[0], plain.dicts[0])


def test_video_codes_follow_the_image_seed():
    a = synthetic.make_workload("video", seed=1, H=24, W=24, T0=256, dict_seed=0)
    b = synthetic.make_workload("video", seed=2, H=24, W=24, T0=256, dict_seed=0)
    assert np.array_equal(a.dicts[0], b.dicts[0])
    assert not np.array_equal(a.sensing.codes, b.sensing.codes)


def _box(V, shape, f):
    Ly, Lx, Py, Px = shape
    fy, fx, sy, sx = f
    return V.reshape(len(V), Ly // fy, fy, Lx // fx, fx, Py // sy, sy, Px // sx, sx).mean(axis=(2, 4, 6, 8)).reshape(len(V), -1)


@pytest.mark.parametrize("name,kw", [("bayer", dict(H=32, W=32)), ("video", dict(H=16, W=16, T0=256)),
                                     ("lightfield", dict(H=16, W=16, T0=512))])
def test_model_links_downsampled_child_is_its_parent(name, kw):
    """links="model": the block rule of Sec. III-B (parent = i // Q), unit-norm
    atoms, and the box-downsampled, renormalised child equals its parent (so the
    coarse dictionary is the set of downsampled fine atoms, property 2 of
    Sec. III-A holds exactly)."""
    w = synthetic.make_workload(name, links="model", **kw)
    g = w.geometry
    for l in range(w.n_levels - 1):
        T = w.dicts[l].shape[0]
        np.testing.assert_array_equal(w.parents[l], np.arange(T) // 4)
        np.testing.assert_allclose(np.linalg.norm(w.dicts[l].astype(np.float64), axis=1), 1.0, atol=1e-6)
        f = tuple(b // a for a, b in zip(g.level_factors[l], g.level_factors[l + 1]))
        down = _box(w.dicts[l].astype(np.float64), g.level_shape(l), f)
        down /= np.linalg.norm(down, axis=1, keepdims=True)
        np.testing.assert_allclose(down, w.dicts[l + 1][w.parents[l]].astype(np.float64), atol=2e-6)


def test_model_links_coarse_code_of_a_tile_is_its_ancestors():
    """links="model", noiseless tiles: W x of every P x P tile equals
    sum_i s_i W d_i = sum_p a_p c_p over the parents p of its fine support,
    with |a_p| = sum over p's chosen children of |s_i| ||W d_i|| (the
    sign-coherent codes never cancel), so the coarse support is exactly the
    parent set of the fine support (properties 2 and 3 of Sec. III-A)."""
    w = synthetic.make_workload("bayer", H=64, W=64, links="model", sigma=0.0)
    g = w.geometry
    P = g.P
    D0 = w.dicts[0].astype(np.float64)
    Dl = w.dicts[1].astype(np.float64)
    t = 0
    for by in range(0, g.H, P):
        for bx in range(0, g.W, P):
            S, s = w.tile_codes[t]
            t += 1
            x = w.truth[:, by:by + P, bx:bx + P].reshape(1, -1)
            np.testing.assert_allclose(x[0], D0[S].T @ s, atol=1e-12)
            xl = _box(x, g.level_shape(0), g.level_factors[1])[0]
            par = np.unique(w.parents[0][S])
            assert 1 <= len(par) <= 4
            a, *_ = np.linalg.lstsq(Dl[par].T, xl, rcond=None)
            assert np.linalg.norm(xl - Dl[par].T @ a) <= 1e-5 * np.linalg.norm(xl)
            wn = np.linalg.norm(_box(D0[S], g.level_shape(0), g.level_factors[1]), axis=1)
            for j, p in enumerate(par):
                mine = w.parents[0][S] == p
                assert abs(a[j]) == pytest.approx(np.sum(np.abs(s[mine]) * wn[mine]), rel=1e-4)
                assert len(set(np.sign(s[mine]))) == 1
