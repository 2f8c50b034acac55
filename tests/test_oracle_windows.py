"""Pins for the sliding-window oracle (Sec. 3.2, Table 3): the printed
window counts, a brute-force enumeration of window starts, numpy counts over
window slices, agreement with the region-grid histograms where the two grids
coincide, and mass invariants."""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(__file__)


def test_table3_window_counts():
    with open(os.path.join(HERE, "golden", "table3_windows.json")) as f:
        g = json.load(f)
    for row in g["rows"]:
        w = row["window"]
        assert oracle.window_count(g["side"], w, w) ** 2 == row["count"], row


def _starts_brute(n, w, s):
    # windows are added until one reaches the end of the axis
    starts = [0]
    while starts[-1] + w < n:
        starts.append(starts[-1] + s)
    return starts


def test_window_count_matches_enumeration():
    for n in range(1, 90):
        for w in range(1, 40, 3):
            for s in range(1, 45, 4):
                assert oracle.window_count(n, w, s) == len(_starts_brute(n, w, s)), (n, w, s)
    with pytest.raises(ValueError):
        oracle.window_count(10, 0, 1)


def _brute_windows(cm, H, W, wh, ww, sh, sw, k):
    """Counts of codes inside each window's interior rectangle, by numpy."""
    nb = len(oracle.compact_codes(k)) if k else 256
    lut = np.array([oracle.bin_of_code(c, k) if k else c for c in range(256)])
    rs, cs = _starts_brute(H, wh, sh), _starts_brute(W, ww, sw)
    out = np.zeros((len(rs), len(cs), nb), dtype=np.uint32)
    for a, x0 in enumerate(rs):
        xl, xh = max(x0, 1), min(x0 + wh, H, H - 1)
        for b, y0 in enumerate(cs):
            yl, yh = max(y0, 1), min(y0 + ww, W, W - 1)
            if xh <= xl or yh <= yl:
                continue
            bins = lut[cm[xl - 1:xh - 1, yl - 1:yh - 1].ravel()]
            bins = bins[bins >= 0]
            out[a, b] = np.bincount(bins, minlength=nb)
    return out


def test_window_hist_brute_force():
    rng = np.random.default_rng(7)
    for trial in range(40):
        H, W = int(rng.integers(3, 60)), int(rng.integers(3, 60))
        wh, ww = int(rng.integers(1, 30)), int(rng.integers(1, 30))
        sh, sw = int(rng.integers(1, 35)), int(rng.integers(1, 35))  # gaps, overlaps and w > n
        k = int(rng.integers(0, 8))
        img = rng.integers(0, 256, (H, W), dtype=np.uint8)
        if trial % 3 == 0:
            img = (img > 128).astype(np.uint8) * 255  # ties
        cm = oracle.codes(img, k=max(k, 1))
        got = oracle.window_hist(cm, H, W, wh, ww, sh, sw, k)
        assert np.array_equal(got, _brute_windows(cm, H, W, wh, ww, sh, sw, k)), (H, W, wh, ww, sh, sw, k)


def test_windows_equal_regions_where_grids_coincide():
    img = np.random.default_rng(3).integers(0, 256, (280, 210), dtype=np.uint8)
    for k in (1, 3, 5):
        cm = oracle.codes(img, k=k)
        # 70-pixel windows at stride 70 = the floor-bound 4 x 3 region grid
        w = oracle.window_hist(cm, 280, 210, 70, 70, 70, 70, k)
        r = oracle.region_hist(cm, 280, 210, 4, 3, k)
        assert np.array_equal(w, r)
        # a window at least as large as the image is the whole-image histogram
        whole = oracle.window_hist(cm, 280, 210, 300, 500, 7, 9, k)
        assert whole.shape[:2] == (1, 1)
        assert np.array_equal(whole[0, 0], oracle.region_hist(cm, 280, 210, 1, 1, k)[0, 0])


def test_window_mass():
    rng = np.random.default_rng(11)
    H, W = 77, 64
    img = rng.integers(0, 256, (H, W), dtype=np.uint8)
    cm = oracle.codes(img, k=3)
    # non-overlapping windows count every interior pixel once
    h = oracle.window_hist(cm, H, W, 10, 10, 10, 10, 3)
    assert int(h.sum()) == (H - 2) * (W - 2)
    # overlapping windows: each window holds exactly its interior pixels
    wh, ww, sh, sw = 20, 16, 10, 8
    h = oracle.window_hist(cm, H, W, wh, ww, sh, sw, 0)
    for a, x0 in enumerate(_starts_brute(H, wh, sh)):
        rows = max(0, min(x0 + wh, H - 1) - max(x0, 1))
        for b, y0 in enumerate(_starts_brute(W, ww, sw)):
            cols = max(0, min(y0 + ww, W - 1) - max(y0, 1))
            assert int(h[a, b].sum()) == rows * cols
