"""Pins for the Eq. 2-3 code variants of the oracle: hand-derived codes of
worked examples A and B under every reading, and invariants that tie each
variant to an independent formulation."""
import json
import os

import numpy as np

import oracle

HERE = os.path.dirname(__file__)
VARIANTS = {"abs_exact": 0, "raw_exact": 1, "abs_thresh": 2, "raw_thresh": 3}
MODES = {0: oracle.MODE_LDP, 1: oracle.MODE_LDP_RAW, 2: oracle.MODE_LDP_THRESH, 3: oracle.MODE_LDP_RAW_THRESH}


def _golden():
    with open(os.path.join(HERE, "golden", "eq2_readings.json")) as f:
        return json.load(f)["examples"]


def _examples():
    with open(os.path.join(HERE, "golden", "worked_examples.json")) as f:
        return {e["name"]: e for e in json.load(f)["examples"]}


def test_hand_derived_readings():
    images = _examples()
    for ex in _golden():
        img = np.array(images[ex["name"]]["image"], dtype=np.uint8)
        assert images[ex["name"]]["m"] == ex["m"]
        for name, var in VARIANTS.items():
            for k in range(1, 8):
                want = ex[name][k - 1]
                assert oracle.code_variant(ex["m"], k, var) == want, (ex["name"], name, k)
                assert int(oracle.codes(img, k=k, mode=MODES[var])[0, 0]) == want, (ex["name"], name, k)
    # variant 0 is the default code
    for ex in _golden():
        for k in range(1, 8):
            assert oracle.code_variant(ex["m"], k, 0) == oracle.code_from_responses(ex["m"], k)


def _bits(c):
    return [i for i in range(8) if c >> i & 1]


def test_variant_invariants():
    rng = np.random.default_rng(5)
    for trial in range(3000):
        if trial % 3 == 0:
            m = rng.integers(-3, 4, 8) * 255  # many ties
        else:
            m = rng.integers(-3825, 3826, 8)
        k = int(rng.integers(1, 8))
        for raw in (0, 1):
            v = m if raw else np.abs(m)
            exact = oracle.code_variant(m, k, raw)
            thresh = oracle.code_variant(m, k, 2 + raw)
            assert bin(exact).count("1") == k
            # exact: every set bit beats every clear one (value, then lower index)
            for i in _bits(exact):
                for j in set(range(8)) - set(_bits(exact)):
                    assert v[i] > v[j] or (v[i] == v[j] and i < j)
            # threshold: exactly the values at or above the k-th largest (numpy order)
            t = np.sort(v)[::-1][k - 1]
            assert thresh == sum(1 << i for i in range(8) if v[i] >= t)
            assert thresh & exact == exact
            if len(set(v.tolist())) == 8:
                assert thresh == exact


def test_inversion_and_complement():
    """I -> 255 - I flips every m_i: the |m| readings are unchanged, and for
    tie-free responses the raw ranking of -m picks the complement of the
    8-k largest m."""
    rng = np.random.default_rng(9)
    for _ in range(50):
        img = rng.integers(0, 256, (12, 15), dtype=np.uint8)
        inv = 255 - img
        for k in range(1, 8):
            for mode in (oracle.MODE_LDP, oracle.MODE_LDP_THRESH):
                assert np.array_equal(oracle.codes(img, k=k, mode=mode), oracle.codes(inv, k=k, mode=mode))
        for x in range(1, 11):
            for y in range(1, 14):
                m = oracle.responses(img, x, y)
                if len(set(m.tolist())) < 8:
                    continue
                for k in range(1, 8):
                    assert oracle.code_variant(-m, k, 1) == (~oracle.code_variant(m, 8 - k, 1)) & 0xFF
