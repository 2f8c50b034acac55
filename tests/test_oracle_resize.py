"""Pins for the crop-and-resize oracle (Sec. 3.1 front end): identity,
constants, 2x down- and up-sampling against their closed forms, the integer
coordinate rule against a floating-point restatement, and crops."""
import numpy as np

import oracle


def test_identity_and_constant():
    rng = np.random.default_rng(0)
    img = rng.integers(0, 256, (37, 53), dtype=np.uint8)
    assert np.array_equal(oracle.resize(img, (37, 53)), img)
    for shape in ((260, 260), (5, 300), (1, 1)):
        assert (oracle.resize(np.full((40, 70), 201, np.uint8), shape) == 201).all()


def test_half_size_is_rounded_block_mean():
    rng = np.random.default_rng(1)
    img = rng.integers(0, 256, (40, 62), dtype=np.uint8).astype(np.int64)
    blocks = img[0::2, 0::2] + img[1::2, 0::2] + img[0::2, 1::2] + img[1::2, 1::2]
    assert np.array_equal(oracle.resize(img.astype(np.uint8), (20, 31)), ((blocks + 2) // 4).astype(np.uint8))


def test_double_width_closed_form():
    rng = np.random.default_rng(2)
    img = rng.integers(0, 256, (9, 23), dtype=np.uint8)
    out = oracle.resize(img, (9, 46)).astype(np.int64)
    p = img.astype(np.int64)
    left = np.concatenate([p[:, :1], p[:, :-1]], axis=1)   # p[m-1], clamped
    right = np.concatenate([p[:, 1:], p[:, -1:]], axis=1)  # p[m+1], clamped
    # even outputs sample m - 1/4, odd ones m + 1/4 (weights 3/4, 1/4), rounded half up
    even = (left + 3 * p + 2) // 4
    odd = (3 * p + right + 2) // 4
    even[:, 0] = p[:, 0]  # m - 1/4 < 0 clamps to the first pixel
    odd[:, -1] = p[:, -1]  # m + 1/4 > last clamps to the last pixel
    assert np.array_equal(out[:, 0::2], even)
    assert np.array_equal(out[:, 1::2], odd)


def test_coordinate_rule_matches_float():
    for n_src in (1, 2, 7, 130, 490, 640):
        for n_dst in (1, 3, 260, 261, 999):
            for i in range(n_dst):
                y = (i + 0.5) * n_src / n_dst - 0.5
                i0, w1 = oracle.resize_coord(i, n_src, n_dst)
                if y <= 0:
                    assert (i0, w1) == (0, 0)
                    continue
                f0 = int(np.floor(y))
                w = (y - f0) * 2048
                if abs(w - np.floor(w) - 0.5) < 1e-6:  # halves: decided by the exact rule
                    continue
                w = int(np.floor(w + 0.5))
                if w == 2048:
                    f0, w = f0 + 1, 0
                if f0 >= n_src - 1:
                    f0, w = n_src - 1, 0
                assert (i0, w1) == (f0, w), (n_src, n_dst, i)


def test_crop_equals_resize_of_the_cut():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (120, 160), dtype=np.uint8)
    for crop in ((10, 20, 90, 100), (0, 0, 120, 160), (119, 159, 1, 1), (5, 7, 33, 140)):
        cy, cx, ch, cw = crop
        assert np.array_equal(oracle.resize(img, (61, 47), crop=crop),
                              oracle.resize(np.ascontiguousarray(img[cy:cy + ch, cx:cx + cw]), (61, 47)))
