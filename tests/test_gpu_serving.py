"""The continuous-batching request runtime: every request's results equal
the same image processed alone and the CPU oracle (tolerance 0, integer
work), whatever else is in flight; admission by device memory; Poisson load."""
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
    from paper_1810_11518_gb300 import serving

    return torch, ldp, oracle, synth, serving


def _pool(env, n, seed0):
    torch, ldp, oracle, synth, serving = env
    sizes = [synth.sizes(seed0 + i, 3, 700) for i in range(n)]
    imgs = []
    for i, (H, W) in enumerate(sizes):
        t = torch.empty((H, W), dtype=torch.uint8, pin_memory=True)
        a = t.numpy()
        a[...] = synth.image(seed0 + i, H, W, 3.0)
        imgs.append((t, a))
    return imgs


def _outputs(env, imgs, hist_len):
    torch = env[0]
    outs = []
    for t, a in imgs:
        H, W = a.shape
        c = torch.full((H - 2, W - 2), 0xEE, dtype=torch.uint8, pin_memory=True).numpy()
        h = torch.full((hist_len,), -1, dtype=torch.int32, pin_memory=True).numpy()
        outs.append((c, h))
    return outs


def _wait(srv, n):
    import time

    got = {}
    t0 = time.time()
    while len(got) < n:
        for c in srv.poll():
            got[c[0]] = c
        assert time.time() - t0 < 60, "requests did not complete"
        time.sleep(0.001)
    return got


def test_mix_equals_alone_and_oracle(env):
    torch, ldp, oracle, synth, serving = env
    imgs = _pool(env, 120, 7000)
    with serving.Server(k=3, regions=(7, 6), max_batch=32, streams=3, arena_bytes=64 << 20) as srv:
        # all at once: batches form and overlap on the device
        mix = _outputs(env, imgs, srv.hist_len)
        for i, ((t, a), (c, h)) in enumerate(zip(imgs, mix)):
            srv.submit(a, tag=i, codes=c, hist=h)
        got = _wait(srv, len(imgs))
        st = srv.stats()
        assert st["batches"] < len(imgs) and st["arena_used"] == 0
        # each request alone
        alone = _outputs(env, imgs, srv.hist_len)
        for i, ((t, a), (c, h)) in enumerate(zip(imgs, alone)):
            srv.submit(a, tag=1000 + i, codes=c, hist=h)
            _wait(srv, 1)
    for i, (t, a) in enumerate(imgs):
        h_ref, c_ref = oracle.extract(a, k=3, R=7, C=6, compact=True)
        assert np.array_equal(mix[i][0], alone[i][0]) and np.array_equal(mix[i][1], alone[i][1]), i
        assert np.array_equal(mix[i][0], c_ref), i
        assert np.array_equal(mix[i][1].astype(np.uint32), h_ref.reshape(-1)), i
        g = got[i]
        assert g[1] <= g[2] <= g[3]


def test_admission_by_device_memory(env):
    """A 2 MiB arena holds only a few requests at a time; all still complete,
    in order of admission, and the arena drains."""
    torch, ldp, oracle, synth, serving = env
    imgs = _pool(env, 40, 8000)
    with serving.Server(k=3, regions=(2, 2), max_batch=64, streams=2, arena_bytes=2 << 20) as srv:
        outs = _outputs(env, imgs, srv.hist_len)
        for i, ((t, a), (c, h)) in enumerate(zip(imgs, outs)):
            srv.submit(a, tag=i, codes=c, hist=h)
        got = _wait(srv, len(imgs))
        assert srv.stats()["arena_used"] == 0
        assert srv.stats()["batches"] > 2
    for i, (t, a) in enumerate(imgs):
        h_ref, c_ref = oracle.extract(a, k=3, R=2, C=2, compact=True)
        assert np.array_equal(outs[i][0], c_ref) and np.array_equal(outs[i][1].astype(np.uint32), h_ref.reshape(-1))


def test_rejects_oversized_and_bad_requests(env):
    torch, ldp, oracle, synth, serving = env
    with serving.Server(arena_bytes=1 << 20) as srv:
        big = np.zeros((1100, 1100), dtype=np.uint8)
        with pytest.raises(ldp.LdpError):
            srv.submit(big, tag=1)
        with pytest.raises(ldp.LdpError):
            srv.submit(np.zeros((2, 9), dtype=np.uint8), tag=2)


def test_poisson_load_short(env):
    torch, ldp, oracle, synth, serving = env
    pool = serving.RequestPool(64, "uneven", seed0=9000)
    with serving.Server(streams=3, max_batch=128, arena_bytes=256 << 20) as srv:
        res = serving.run_load(srv, pool, rate=4000, seconds=0.5, warmup=0.1, seed=1)
    assert res["requests"] > 1000
    assert 0 < res["p50_ms"] <= res["p99_ms"] < 100
    assert res["sustained_mpix_s"] > 0
