"""The seeded input generator: Philox4x32-10 known answers and the
self-written log/sin/cos used by Box-Muller."""
import numpy as np

from lrsgen import philox4x32_10, ln_pos, sincos_turns, normals, GaussianInstance


def _run(c, k):
    out = philox4x32_10([np.uint64(x) for x in c], [np.uint64(x) for x in k])
    return [int(o) for o in out]


def test_philox4x32_10_known_answers():
    # Known-answer vectors published with the Random123 library (Salmon et al., SC'11).
    assert _run([0, 0, 0, 0], [0, 0]) == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]
    assert _run([0xffffffff] * 4, [0xffffffff] * 2) == \
        [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]
    assert _run([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0]) == \
        [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]


def test_series_log_sin_cos_accuracy():
    u = np.random.default_rng(0).random(20000) + 1e-300
    assert np.max(np.abs(ln_pos(u) - np.log(u)) / np.abs(np.log(u))) < 1e-14
    v = np.random.default_rng(1).random(20000)
    s, c = sincos_turns(v)
    assert np.max(np.abs(s - np.sin(2 * np.pi * v))) < 1e-14
    assert np.max(np.abs(c - np.cos(2 * np.pi * v))) < 1e-14


def test_normals_moments_and_offsets():
    z = normals(7, 1, 2, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    np.testing.assert_array_equal(normals(7, 1, 2, 9, 3), z[3:12])


def test_instance_shapes_and_supports():
    g = GaussianInstance(n=50, q=20, r=3, m=15, rho=4, seed=5)
    assert g.A.shape == (20, 15, 50) and g.A.dtype == np.float32
    assert g.Y.shape == (20, 15) and g.Y.dtype == np.float32
    assert np.all(np.diff(g.S_idx, axis=1) > 0)
    np.testing.assert_allclose(g.Ustar.T @ g.Ustar, np.eye(3), atol=1e-13)
    mags = np.abs(g.S_val) / g.rms_L
    assert mags.min() >= 1 and mags.max() <= 10
