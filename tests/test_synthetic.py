"""The seeded input generator: reproducible, and one model can serve many
images (dictionaries and links seeded apart from the image content)."""

import numpy as np

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
