"""Pins for the descriptor-distance oracle: a hand-worked example, the
identity |a - b| + 2 min(a, b) = a + b tying L1 to intersection, bounds
that sandwich chi-square, symmetry and zero self-distance, and a numpy
restatement on random data."""
import numpy as np

import oracle


def test_hand_example():
    q = np.array([[1, 0, 3]])
    g = np.array([[0, 2, 1]])
    assert oracle.hist_distance(q, g, oracle.DIST_L1)[0, 0] == 5          # 1 + 2 + 2
    assert oracle.hist_distance(q, g, oracle.DIST_INTERSECT)[0, 0] == 1   # 0 + 0 + 1
    assert oracle.hist_distance(q, g, oracle.DIST_CHI2)[0, 0] == 4.0      # 1/1 + 4/2 + 4/4
    assert oracle.hist_distance(np.zeros((1, 4)), np.zeros((1, 4)), oracle.DIST_CHI2)[0, 0] == 0.0


def test_identities_and_bounds():
    rng = np.random.default_rng(0)
    q = rng.integers(0, 5000, (7, 300)).astype(np.uint32)
    g = rng.integers(0, 5000, (9, 300)).astype(np.uint32)
    q[:, ::7] = 0
    g[:, ::5] = 0
    l1 = oracle.hist_distance(q, g, oracle.DIST_L1).astype(np.int64)
    it = oracle.hist_distance(q, g, oracle.DIST_INTERSECT).astype(np.int64)
    chi = oracle.hist_distance(q, g, oracle.DIST_CHI2)
    tot = q.sum(1, dtype=np.int64)[:, None] + g.sum(1, dtype=np.int64)[None, :]
    assert np.array_equal(l1 + 2 * it, tot)
    # (a-b)^2/(a+b) <= |a-b| termwise; Cauchy-Schwarz: (sum |a-b|)^2 <= chi2 * sum (a+b)
    assert (chi <= l1 + 1e-9).all()
    assert (l1.astype(np.float64) ** 2 <= chi * tot * (1 + 1e-12)).all()
    # symmetry, self-distance
    assert np.array_equal(oracle.hist_distance(g, q, oracle.DIST_L1).T, l1.astype(np.uint64))
    assert np.allclose(oracle.hist_distance(g, q, oracle.DIST_CHI2).T, chi, rtol=0, atol=0)
    assert (np.diag(oracle.hist_distance(q, q, oracle.DIST_L1)) == 0).all()
    assert (np.diag(oracle.hist_distance(q, q, oracle.DIST_CHI2)) == 0).all()
    assert np.array_equal(np.diag(oracle.hist_distance(q, q, oracle.DIST_INTERSECT)), q.sum(1, dtype=np.uint64))


def test_numpy_restatement():
    rng = np.random.default_rng(1)
    q = rng.integers(0, 300, (5, 57)).astype(np.uint32)
    g = rng.integers(0, 300, (6, 57)).astype(np.uint32)
    q[q < 50] = 0
    qf, gf = q[:, None, :].astype(np.float64), g[None, :, :].astype(np.float64)
    s = qf + gf
    with np.errstate(divide="ignore", invalid="ignore"):
        chi = np.where(s > 0, (qf - gf) ** 2 / np.where(s > 0, s, 1), 0).sum(-1)
    assert np.allclose(oracle.hist_distance(q, g, oracle.DIST_CHI2), chi, rtol=1e-12, atol=0)
    assert np.array_equal(oracle.hist_distance(q, g, oracle.DIST_L1), np.abs(qf - gf).sum(-1).astype(np.uint64))
    assert np.array_equal(oracle.hist_distance(q, g, oracle.DIST_INTERSECT),
                          np.minimum(qf, gf).sum(-1).astype(np.uint64))
