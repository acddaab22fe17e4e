"""The seeded input generators keep the properties their recipes state: the
same seed gives the same frames, the known-motion set-up's moved frames are
the original displaced by the stated vectors (before noise), the contrast
map leaves at least 30 % of the frame flat, and the 10 fps load scenes are every
third frame of the 30 fps ones."""
import numpy as np

import synth


def test_generators_are_deterministic():
    a, ga = synth.global_motion_sequence(3, 176, 144, n_moved=4)
    b, gb = synth.global_motion_sequence(3, 176, 144, n_moved=4)
    assert np.array_equal(a, b) and np.array_equal(ga, gb)
    assert np.array_equal(synth.load_sequence("smooth-fast", 30, 9), synth.load_sequence("smooth-fast", 30, 9))
    assert np.array_equal(synth.config_sequence("qcif", 5, 3), synth.config_sequence("qcif", 5, 3))


def test_global_motion_frames_are_the_original_displaced():
    frames, g = synth.global_motion_sequence(11, 176, 144, n_moved=9, noise_sigma=0.0)
    assert frames.shape == (10, 144, 176) and g.shape == (9, 2)
    assert len({(int(x), int(y)) for x, y in g}) == 9            # distinct vectors
    assert np.all(np.abs(g) <= 8)
    H, W = frames.shape[1:]
    for k, (gx, gy) in enumerate(g):
        ys = np.clip(np.arange(H) + int(gy), 0, H - 1)
        xs = np.clip(np.arange(W) + int(gx), 0, W - 1)
        # frame_k(x, y) = frame_0(clamp(x + gx), clamp(y + gy)): g is the
        # motion vector a block matcher should find
        assert np.array_equal(frames[k + 1], frames[0][np.ix_(ys, xs)]), k


def test_contrast_texture_is_at_least_30_percent_flat():
    """Zero contrast on 30 % of the frame (rank below 0.3), plus the margin
    where the squared contrast rounds the texture to 128; textured elsewhere."""
    for seed in (2, 7):
        t = synth.contrast_texture(np.random.default_rng(seed), 352, 288)
        flat = np.mean(t == 128)
        assert 0.30 <= flat < 0.6, flat
        assert np.mean(np.abs(t.astype(int) - 128) > 10) > 0.12


def test_load_scenes_at_10_fps_are_every_third_frame():
    for name in synth.LOAD_RECIPES:
        f30 = synth.load_sequence(name, 30, 500, n_frames=28)
        f10 = synth.load_sequence(name, 10, 500)
        assert f10.shape == (10, 144, 176)
        assert np.array_equal(f10, f30[::3]), name
