"""GPU parity of the batched path: one persistent (CUDA-graph) launch over
images of uneven sizes, against the CPU oracle, bit for bit."""
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


def _make(env, seeds, lo=3, hi=300, hist_len=7 * 6 * 56, sizes=None):
    torch, ldp, oracle, synth = env
    if sizes is None:
        sizes = [synth.sizes(s, lo, hi) for s in seeds]
    Hs = [h for h, _ in sizes]
    Ws = [w for _, w in sizes]
    lay = ldp.BatchLayout.build(Hs, Ws, hist_len=hist_len)
    host = np.zeros(lay.img_bytes, dtype=np.uint8)
    synth.batch_into(host, seeds, Hs, Ws, lay.pitches, lay.img_off)
    d_img = torch.from_numpy(host).cuda()
    d_codes = torch.zeros(lay.code_bytes, dtype=torch.uint8, device="cuda")
    d_hist = torch.zeros(lay.n * lay.hist_len, dtype=torch.int32, device="cuda")
    return lay, host, d_img, d_codes, d_hist


def _check(env, lay, host, d_codes, d_hist, k=3, R=7, C=6, compact=True, mode=0, idx=None):
    torch, ldp, oracle, synth = env
    torch.cuda.synchronize()
    cc = d_codes.cpu().numpy()
    hc = d_hist.cpu().numpy().astype(np.uint32)
    for i in (range(lay.n) if idx is None else idx):
        h_ref, c_ref = oracle.extract(lay.image(host, i), k=k, R=R, C=C, compact=compact, mode=mode,
                                      W=int(lay.Ws[i]))
        assert np.array_equal(lay.codes(cc, i), c_ref), i
        assert np.array_equal(hc[i * lay.hist_len:(i + 1) * lay.hist_len].reshape(h_ref.shape), h_ref), i


@pytest.mark.parametrize("graph", [True, False])
def test_uneven_batch(env, graph):
    torch, ldp, oracle, synth = env
    seeds = list(range(500, 540))
    lay, host, d_img, d_codes, d_hist = _make(env, seeds)
    d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
    d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
    with ldp.BatchPlan(64, lay.pixels, k=3, regions=(7, 6), graph=graph) as plan:
        plan.run(d_desc, d_count, d_hist)
        _check(env, lay, host, d_codes, d_hist)
        assert ldp.device_status() == 0


def test_count_read_on_device_and_replay(env):
    """One captured graph serves different image counts: the count lives in
    device memory; histograms of images past the count are left alone."""
    torch, ldp, oracle, synth = env
    seeds = list(range(600, 620))
    lay, host, d_img, d_codes, d_hist = _make(env, seeds, lo=20, hi=200)
    d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
    d_count = torch.tensor([5], dtype=torch.int32, device="cuda")
    with ldp.BatchPlan(32, lay.pixels, k=3, regions=(7, 6)) as plan:
        d_hist.fill_(-1)
        plan.run(d_desc, d_count, d_hist)
        torch.cuda.synchronize()
        _check(env, lay, host, d_codes, d_hist, idx=range(5))
        assert (d_hist[5 * lay.hist_len:] == -1).all()
        d_count.fill_(lay.n)
        plan.run(d_desc, d_count, d_hist)
        _check(env, lay, host, d_codes, d_hist)


def test_all_k_and_variants(env):
    torch, ldp, oracle, synth = env
    seeds = list(range(700, 712))
    for k in range(1, 8):
        nb = ldp.hist_bins(k)
        lay, host, d_img, d_codes, d_hist = _make(env, seeds, lo=3, hi=260, hist_len=4 * 3 * nb)
        d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
        d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
        with ldp.BatchPlan(16, lay.pixels, k=k, regions=(4, 3)) as plan:
            for v in range(ldp.num_variants()):
                plan.set_config(v, 0 if v % 2 == 0 else 1)
                d_codes.zero_()
                plan.run(d_desc, d_count, d_hist)
                _check(env, lay, host, d_codes, d_hist, k=k, R=4, C=3)


def test_lbp_batch_every_variant(env):
    """LBP through every tile variant on a batch with images of 3 to 6 rows
    (input rows read ahead are clamped to the image's last row) beside larger
    ones, 7x6 regions (the region-row slot variants flush per region row)."""
    torch, ldp, oracle, synth = env
    sizes = [(3, 40), (4, 133), (5, 7), (6, 300), (3, 3), (97, 5), (130, 260), (257, 129), (64, 1000)]
    seeds = list(range(900, 900 + len(sizes)))
    lay, host, d_img, d_codes, d_hist = _make(env, seeds, hist_len=7 * 6 * 256, sizes=sizes)
    d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
    d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
    for v in range(ldp.num_variants()):
        with ldp.BatchPlan(lay.n, lay.pixels, regions=(7, 6), lbp=True) as plan:
            plan.set_config(v, 0)
            d_codes.zero_()
            plan.run(d_desc, d_count, d_hist)
            _check(env, lay, host, d_codes, d_hist, R=7, C=6, compact=False, mode=oracle.MODE_LBP)
        assert ldp.device_status() == 0, ldp.variant_name(v)


def test_lbp_batch_and_raw_bins(env):
    torch, ldp, oracle, synth = env
    seeds = list(range(800, 816))
    lay, host, d_img, d_codes, d_hist = _make(env, seeds, lo=3, hi=200, hist_len=2 * 2 * 256)
    d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
    d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
    with ldp.BatchPlan(16, lay.pixels, regions=(2, 2), lbp=True) as plan:
        plan.run(d_desc, d_count, d_hist)
        _check(env, lay, host, d_codes, d_hist, R=2, C=2, compact=False, mode=oracle.MODE_LBP)
    with ldp.BatchPlan(16, lay.pixels, k=2, regions=(2, 2), compact=False) as plan:
        plan.run(d_desc, d_count, d_hist)
        _check(env, lay, host, d_codes, d_hist, k=2, R=2, C=2, compact=False)


def test_codes_optional_and_hist_only(env):
    torch, ldp, oracle, synth = env
    seeds = list(range(900, 908))
    lay, host, d_img, d_codes, d_hist = _make(env, seeds, lo=10, hi=150)
    descs = lay.descs(d_img.data_ptr(), d_codes.data_ptr())
    descs["codes"][::2] = 0  # even images: histogram only
    d_desc = torch.from_numpy(descs.view(np.uint8)).cuda()
    d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
    with ldp.BatchPlan(8, lay.pixels, k=3, regions=(7, 6)) as plan:
        plan.run(d_desc, d_count, d_hist)
        torch.cuda.synchronize()
    cc = d_codes.cpu().numpy()
    hc = d_hist.cpu().numpy().astype(np.uint32)
    for i in range(lay.n):
        h_ref, c_ref = oracle.extract(lay.image(host, i), k=3, R=7, C=6, W=int(lay.Ws[i]))
        assert np.array_equal(hc[i * lay.hist_len:(i + 1) * lay.hist_len].reshape(h_ref.shape), h_ref)
        if i % 2:
            assert np.array_equal(lay.codes(cc, i), c_ref)
        else:
            assert (lay.codes(cc, i) == 0).all()


def test_invalid_descriptor_skipped_and_flagged(env):
    torch, ldp, oracle, synth = env
    seeds = list(range(950, 954))
    lay, host, d_img, d_codes, d_hist = _make(env, seeds, lo=10, hi=90)
    descs = lay.descs(d_img.data_ptr(), d_codes.data_ptr())
    descs["H"][1] = 2  # invalid: below 3 rows
    d_desc = torch.from_numpy(descs.view(np.uint8)).cuda()
    d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
    ldp.device_status()  # clear
    with ldp.BatchPlan(8, lay.pixels, k=3, regions=(7, 6)) as plan:
        plan.run(d_desc, d_count, d_hist)
        _check(env, lay, host, d_codes, d_hist, idx=[0, 2, 3])
        assert (d_hist[lay.hist_len:2 * lay.hist_len] == 0).all()
    assert ldp.device_status() & 1
    assert ldp.device_status() == 0


def test_plan_errors(env):
    torch, ldp, oracle, synth = env
    with ldp.BatchPlan(4, 10000, k=3, regions=(1, 1)) as plan:
        d = torch.zeros(40, dtype=torch.uint8, device="cuda")
        n = torch.zeros(1, dtype=torch.int32, device="cuda")
        with pytest.raises(ldp.LdpError):
            ldp._abi.call("lbp_batch_run", plan._h, ctypes_ptr(d), ctypes_ptr(n), None, None)
        plan.run(d, n, None)  # zero images: a valid no-op
        torch.cuda.synchronize()


def ctypes_ptr(t):
    import ctypes

    return ctypes.c_void_p(t.data_ptr())
