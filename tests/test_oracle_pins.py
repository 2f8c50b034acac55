"""Pins for the CPU oracle: worked examples, closed forms, invariants and
independent formulations, chosen so that a dropped term, a wrong sign or
index, a transposed or flipped mask, or a wrong tie rule fails at least one.
All CPU-only."""
import itertools
import json
import os
from math import comb

import numpy as np
import pytest
from scipy import ndimage

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")
RING = [(0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1), (1, 0), (1, 1)]  # E, NE, ..., SE


def _examples():
    with open(GOLDEN) as f:
        return json.load(f)["examples"]


@pytest.mark.parametrize("ex", _examples(), ids=lambda e: e["name"])
def test_worked_example(orc, ex):
    img = np.array(ex["image"], dtype=np.uint8)
    assert list(orc.responses(img, 1, 1)) == ex["m"]
    assert list(orc.aldp_responses(img, 1, 1)) == ex["m"]
    assert list(orc.ringsum_responses(img, 1, 1)) == ex["m"]
    for k, code in ex["ldp"].items():
        assert orc.code_from_responses(ex["m"], int(k)) == code
        assert orc.codes(img, int(k))[0, 0] == code
    assert orc.lbp_code(img, 1, 1) == ex["lbp"]
    assert orc.codes(img, mode=orc.MODE_LBP)[0, 0] == ex["lbp"]


def test_mask_structure(orc):
    """Each M_i: centre 0, 5 on ring positions i-1, i, i+1, -3 on the other
    five (Sec. 2.2.1); consecutive masks are one ring step apart."""
    for i in range(8):
        M = orc.kirsch_mask(i)
        assert M[1, 1] == 0
        assert M.sum() == 0
        for j, (dx, dy) in enumerate(RING):
            want = 5 if (j - i) % 8 in (7, 0, 1) else -3
            assert M[1 + dx, 1 + dy] == want, (i, j)
    # M_0 lights the right column (East), M_2 the top row (North)
    assert (orc.kirsch_mask(0)[:, 2] == 5).all()
    assert (orc.kirsch_mask(2)[0, :] == 5).all()


def _rand_img(rng, H, W, kind):
    if kind == "u8":
        return rng.integers(0, 256, (H, W), dtype=np.uint8)
    if kind == "bin255":
        return (rng.integers(0, 2, (H, W)) * 255).astype(np.uint8)
    if kind == "bin1":
        return rng.integers(0, 2, (H, W)).astype(np.uint8)
    if kind == "few":
        return rng.choice(np.array([0, 3, 8, 200], dtype=np.uint8), (H, W))
    raise ValueError(kind)


def test_eq1_is_a_correlation_library(orc):
    """Eq. 1 reduces to scipy.ndimage.correlate with each mask."""
    rng = np.random.default_rng(1)
    img = rng.integers(0, 256, (13, 17), dtype=np.uint8)
    for i in range(8):
        ref = ndimage.correlate(img.astype(np.int64), orc.kirsch_mask(i).astype(np.int64), mode="constant")
        for x in range(1, 12):
            for y in range(1, 16):
                assert orc.responses(img, x, y)[i] == ref[x, y]


def test_brute_force_three_routes(orc):
    """Literal masks + stable sort == paper's ALDP (Eqs. 7-29) + rank count ==
    ring sums, on many tiny images including heavy ties."""
    rng = np.random.default_rng(2)
    kinds = ["u8", "bin255", "bin1", "few"]
    n = 0
    for trial in range(160):
        H = int(rng.integers(3, 18))
        W = int(rng.integers(3, 14))
        img = _rand_img(rng, H, W, kinds[trial % 4])
        for x in range(1, H - 1):
            for y in range(1, W - 1):
                m = orc.responses(img, x, y)
                assert (m == orc.aldp_responses(img, x, y)).all()
                assert (m == orc.ringsum_responses(img, x, y)).all()
                for k in range(1, 8):
                    assert orc.code_from_responses(m, k) == orc.rank_code_from_responses(m, k)
                n += 1
        k = int(rng.integers(1, 8))
        assert (orc.codes(img, k) == orc.aldp_codes(img, k)).all()
    assert n > 5000


def test_definitional_topk(orc):
    """Pin 10: for each pixel, every set bit beats every unset bit."""
    rng = np.random.default_rng(3)
    for trial in range(60):
        img = _rand_img(rng, 9, 11, ["u8", "bin255", "few"][trial % 3])
        for k in range(1, 8):
            cm = orc.codes(img, k)
            for x in range(1, 8):
                for y in range(1, 10):
                    a = np.abs(orc.responses(img, x, y).astype(np.int64))
                    c = int(cm[x - 1, y - 1])
                    assert bin(c).count("1") == k
                    on = [i for i in range(8) if c >> i & 1]
                    off = [i for i in range(8) if not c >> i & 1]
                    for i in on:
                        for j in off:
                            assert a[i] > a[j] or (a[i] == a[j] and i < j)


def test_constant_and_zero_sum(orc):
    for v in (0, 1, 77, 255):
        img = np.full((6, 7), v, dtype=np.uint8)
        for k in range(1, 8):
            assert (orc.codes(img, k) == (1 << k) - 1).all()
        assert (orc.codes(img, mode=orc.MODE_LBP) == 255).all()
        h, _ = orc.extract(img, k=3, R=1, C=1, compact=False)
        assert h[0, 0, 7] == 4 * 5 and h.sum() == 20
        hc, _ = orc.extract(img, k=3, R=1, C=1, compact=True)
        assert hc[0, 0, 0] == 20


def _tie_free(orc, img, x, y, k):
    a = sorted(np.abs(orc.responses(img, x, y).astype(np.int64)), reverse=True)
    return a[k - 1] != a[k]


def _rotl8(c, s):
    return ((c << s) | (c >> (8 - s))) & 0xFF


def test_rotation_rotates_codes(orc):
    """rot90 counter-clockwise maps E to N: tie-free codes rotate left by 2."""
    rng = np.random.default_rng(4)
    checked = 0
    for trial in range(6):
        img = rng.integers(0, 256, (12, 15), dtype=np.uint8)
        rot = np.ascontiguousarray(np.rot90(img))  # rot[i, j] = img[j, W-1-i]
        H, W = img.shape
        for k in (1, 2, 3, 4, 6):
            a, b = orc.codes(img, k), orc.codes(rot, k)
            for x in range(1, H - 1):
                for y in range(1, W - 1):
                    if _tie_free(orc, img, x, y, k):
                        assert b[W - 1 - y - 1, x - 1] == _rotl8(int(a[x - 1, y - 1]), 2)
                        checked += 1
    assert checked > 2000


def test_mirror_reflects_codes(orc):
    """Flipping columns maps direction i to (4 - i) mod 8 (tie-free pixels)."""
    rng = np.random.default_rng(5)
    for trial in range(4):
        img = rng.integers(0, 256, (10, 13), dtype=np.uint8)
        mir = np.ascontiguousarray(img[:, ::-1])
        H, W = img.shape
        for k in (1, 3, 5):
            a, b = orc.codes(img, k), orc.codes(mir, k)
            for x in range(1, H - 1):
                for y in range(1, W - 1):
                    if _tie_free(orc, img, x, y, k):
                        c = int(a[x - 1, y - 1])
                        want = sum(1 << ((4 - i) % 8) for i in range(8) if c >> i & 1)
                        assert b[x - 1, W - 1 - y - 1] == want


def test_inversion_and_offset(orc):
    """255 - I negates every m (|m| unchanged: identical codes, ties included);
    I + c leaves m and LBP unchanged."""
    rng = np.random.default_rng(6)
    for kind in ("u8", "bin255", "few"):
        img = _rand_img(rng, 11, 12, kind)
        for k in range(1, 8):
            assert (orc.codes(255 - img, k) == orc.codes(img, k)).all()
        low = (img // 2).astype(np.uint8)
        for k in (1, 3, 7):
            assert (orc.codes(low + 100, k) == orc.codes(low, k)).all()
        assert (orc.codes(low + 100, mode=orc.MODE_LBP) == orc.codes(low, mode=orc.MODE_LBP)).all()


def test_compact_bins_colex_closed_form(orc):
    """Eq. 6 ordering (ascending code value) equals the colex rank
    sum_j C(b_j, j) over set bits b_1 < ... < b_k."""
    for k in range(0, 9):
        lst = orc.compact_codes(k)
        assert len(lst) == comb(8, k)
        for b, code in enumerate(lst):
            bits = [i for i in range(8) if code >> i & 1]
            assert sum(comb(bj, j + 1) for j, bj in enumerate(bits)) == b
            assert orc.bin_of_code(code, k) == b
    assert orc.bin_of_code(7, 3) == 0 and orc.bin_of_code(224, 3) == 55
    assert orc.bin_of_code(255, 3) == -1


def test_region_band_closed_form(orc):
    """Row band of pixel x = floor((R*x + R - 1) / H) matches the bounds loop."""
    for H in list(range(1, 60)) + [490, 640, 1024, 2048]:
        for R in range(1, 17):
            owner = np.full(H, -1)
            for b in range(R):
                lo, hi = orc.band(H, R, b)
                assert lo == b * H // R and hi == (b + 1) * H // R
                owner[lo:hi] = b
            xs = np.arange(H)
            assert (owner == (R * xs + R - 1) // H).all()


def test_region_hist_brute_force(orc):
    """Region histograms equal a direct count over each region's interior
    pixels; masses and raw/compact agreement (Eq. 4-5)."""
    rng = np.random.default_rng(7)
    for (H, W, R, C, k) in [(17, 23, 3, 4, 3), (9, 9, 1, 1, 2), (30, 12, 7, 6, 3), (5, 40, 2, 16, 4),
                            (12, 12, 12, 12, 1), (3, 3, 2, 2, 5)]:
        img = rng.integers(0, 256, (H, W), dtype=np.uint8)
        raw, cm = orc.extract(img, k=k, R=R, C=C, compact=False)
        cpt, cm2 = orc.extract(img, k=k, R=R, C=C, compact=True)
        assert (cm == cm2).all()
        assert raw.sum() == (H - 2) * (W - 2) == cpt.sum()
        lst = orc.compact_codes(k)
        for ri in range(R):
            for rj in range(C):
                x0, x1 = max(ri * H // R, 1), min((ri + 1) * H // R, H - 1)
                y0, y1 = max(rj * W // C, 1), min((rj + 1) * W // C, W - 1)
                sub = cm[x0 - 1:max(x1 - 1, x0 - 1), y0 - 1:max(y1 - 1, y0 - 1)]
                want = np.bincount(sub.ravel(), minlength=256)
                assert (raw[ri, rj] == want).all()
                assert (cpt[ri, rj] == want[lst]).all()
        whole, _ = orc.extract(img, k=k, R=1, C=1, compact=False)
        assert (raw.sum(axis=(0, 1)) == whole[0, 0]).all()


def test_lbp_brute_force(orc):
    """LBP: bit j = [p_j >= centre], recomputed from numpy shifts."""
    rng = np.random.default_rng(8)
    img = rng.integers(0, 4, (14, 19), dtype=np.uint8) * 60
    cm = orc.codes(img, mode=orc.MODE_LBP)
    c = img[1:-1, 1:-1].astype(int)
    want = np.zeros_like(c)
    for j, (dx, dy) in enumerate(RING):
        nb = img[1 + dx:img.shape[0] - 1 + dx, 1 + dy:img.shape[1] - 1 + dy].astype(int)
        want |= (nb >= c).astype(int) << j
    assert (cm == want).all()


def test_popcount_on_synthetic(orc):
    import synth

    img = synth.image(0, 64, 80, 3.0)
    for k in range(1, 8):
        cm = orc.codes(img, k)
        assert (np.unpackbits(cm[..., None], axis=-1).sum(-1) == k).all()


def test_batch_driver_matches_single(orc):
    import synth

    Hs, Ws = [20, 33, 7], [25, 9, 40]
    pitches = [32, 16, 48]
    offs = np.array([0, 20 * 32, 20 * 32 + 33 * 16], dtype=np.int64)
    buf = np.zeros(int(offs[-1] + 7 * 48), dtype=np.uint8)
    synth.batch_into(buf, [5, 6, 7], Hs, Ws, pitches, offs)
    hists, maps = orc.extract_batch(buf, offs, Hs, Ws, pitches, k=3, R=2, C=3, want_codes=True, threads=3)
    for i in range(3):
        img = buf[offs[i]:offs[i] + Hs[i] * pitches[i]].reshape(Hs[i], pitches[i])
        h, cm = orc.extract(img, k=3, R=2, C=3, W=Ws[i])
        assert (h == hists[i]).all() and (cm == maps[i]).all()


def test_rejects_bad_arguments(orc):
    img = np.zeros((2, 5), dtype=np.uint8)
    with pytest.raises(ValueError):
        orc.extract(img)
    with pytest.raises(ValueError):
        orc.codes(np.zeros((4, 4), np.uint8), k=0)
    with pytest.raises(ValueError):
        orc.codes(np.zeros((4, 4), np.uint8), k=8)


def test_timed_cpu_routes_equal_the_oracle(orc):
    """The driver bench.py times (three response routes, the same code step
    and histograms) gives the oracle's histograms on every route, in both
    builds, raw and compact, on several threads; the responses alone agree."""
    import synth

    imgs = synth.batch(list(range(5)), 37, 53, 3.0)
    flat = np.ascontiguousarray(imgs.reshape(-1))
    offs = np.arange(5, dtype=np.int64) * (37 * 53)
    for R, C, compact, k in ((7, 6, True, 3), (1, 1, False, 2)):
        ref, _ = orc.extract_batch(flat, offs, [37] * 5, [53] * 5, [53] * 5, k=k, R=R, C=C, compact=compact)
        for route in (orc.ROUTE_MASKS, orc.ROUTE_ALDP, orc.ROUTE_RINGSUM):
            for timed in (False, True):
                got = orc.route_extract_batch(route, flat, offs, 37, 53, 53, k=k, R=R, C=C, compact=compact,
                                              threads=3, timed=timed)
                assert np.array_equal(got, ref), (route, timed)
    sums = {orc.route_response_sum(r, flat, offs, 37, 53, 53, timed=t) for r in range(3) for t in (False, True)}
    m = sum(np.abs(orc.responses(imgs[i], x, y)).sum() for i in range(5) for x in range(1, 36) for y in range(1, 52))
    assert sums == {int(m)}
