"""The seeded input recipe: determinism, shapes and ranges."""
import numpy as np

from paper_2001_09632_gb300 import synth


def test_image_deterministic_and_in_range():
    a = synth.gen_image(256, 256, 12)
    b = synth.gen_image(256, 256, 12)
    c = synth.gen_image(256, 256, 13)
    assert a.dtype == np.uint8 and a.shape == (256, 256)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.std() > 10                       # shapes + texture, not flat


def test_video_drift_static_texture():
    v = synth.gen_video(3, 64, 96, seed=5)
    assert v.shape == (3, 64, 96) and v.dtype == np.uint8
    assert not np.array_equal(v[0], v[1])
    v2 = synth.gen_video(2, 64, 96, seed=5, first_frame=1)
    assert np.array_equal(v[1:], v2)


def test_uneven_batch_mix():
    batch = synth.gen_uneven_batch(10, 0, sizes=((32, 32), (64, 64), (48, 80)))
    shapes = [img.shape for img, _ in batch]
    assert shapes.count((32, 32)) == 4 and shapes.count((64, 64)) == 4 and shapes.count((48, 80)) == 2
    assert [B for _, B in batch][:4] == [8, 16, 32, 8]
