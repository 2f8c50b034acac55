"""GPU parity of the descriptor distances: L1 and intersection bit-exact,
chi-square within (D + 5) * 2^-24 relative (fp32 terms, hardware reciprocal
within 2^-23, D non-negative terms summed), against the fp64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import oracle
    import paper_1810_11518_gb300 as ldp
    import synth

    return torch, ldp, oracle, synth


def _check(env, q, g):
    torch, ldp, oracle, synth = env
    dq = torch.from_numpy(q.astype(np.int32)).cuda()
    dg = torch.from_numpy(g.astype(np.int32)).cuda()
    D = q.shape[1]
    for metric in (ldp.DIST_L1, ldp.DIST_INTERSECT):
        got = ldp.hist_distance(dq, dg, metric)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy().astype(np.uint64), oracle.hist_distance(q, g, metric)), metric
    got = ldp.hist_distance(dq, dg, ldp.DIST_CHI2).cpu().numpy().astype(np.float64)
    ref = oracle.hist_distance(q, g, oracle.DIST_CHI2)
    bound = (D + 5) * 2.0 ** -24
    assert (np.abs(got - ref) <= bound * ref).all(), float(np.max(np.abs(got - ref) / np.maximum(ref, 1e-300)))


@pytest.mark.parametrize("nq,ng,D", [(1, 1, 1), (3, 70, 33), (64, 64, 32), (65, 129, 2352), (130, 7, 100)])
def test_random_descriptors(env, nq, ng, D):
    rng = np.random.default_rng(nq * 1000 + ng + D)
    q = rng.integers(0, 3000, (nq, D)).astype(np.uint32)
    g = rng.integers(0, 3000, (ng, D)).astype(np.uint32)
    q[rng.random(q.shape) < 0.3] = 0   # empty bins, some shared with g
    g[rng.random(g.shape) < 0.3] = 0
    _check(env, q, g)


def test_large_counts_and_identical_rows(env):
    rng = np.random.default_rng(3)
    q = rng.integers(0, 1 << 23, (20, 300)).astype(np.uint32)
    g = np.concatenate([q[:5], rng.integers(0, 1 << 23, (30, 300)).astype(np.uint32)])
    _check(env, q, g)
    torch, ldp, oracle, synth = env
    d = ldp.hist_distance(torch.from_numpy(q.astype(np.int32)).cuda(), torch.from_numpy(g.astype(np.int32)).cuda(),
                          ldp.DIST_CHI2).cpu().numpy()
    assert (d[np.arange(5), np.arange(5)] == 0).all()


def test_ldp_descriptors(env):
    """Region histograms of real LDP code maps as the descriptors."""
    torch, ldp, oracle, synth = env
    descs = []
    for s in range(40):
        img = synth.image(2000 + s, 98, 130, 3.0)
        h, _ = ldp.region_hist(torch.from_numpy(img).cuda(), k=3, regions=(7, 6), with_codes=False)
        descs.append(h.reshape(-1))
    allq = torch.stack(descs)
    torch.cuda.synchronize()
    q = allq.cpu().numpy().astype(np.uint32)
    _check(env, q[:13], q)
    # strided rows: every other descriptor, leading dimension 2 D
    got = ldp.hist_distance(allq[::2], allq[1::2], ldp.DIST_L1).cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, oracle.hist_distance(q[::2], q[1::2], oracle.DIST_L1))
