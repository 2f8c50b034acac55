"""GPU parity of the sliding-window histograms (Sec. 3.2): cell histograms of
gcd(size, stride) cells summed into windows, against the CPU oracle bit for
bit, single images and batches.  The cases cover the three routes: stride =
size (cells are the windows), the fused pass (column stride dividing the
width: cell rows in shared memory), and cells through device scratch."""
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


def _h(t):
    return t.cpu().numpy().astype(np.uint32)


@pytest.mark.parametrize("H,W,window,stride", [
    (280, 280, (10, 10), None), (280, 280, (25, 25), None), (280, 280, (100, 100), None),  # Table 3
    (260, 260, (20, 20), None), (260, 260, (50, 50), None),
    (77, 150, (20, 16), (10, 8)),     # overlapping
    (77, 150, (9, 12), (15, 20)),     # gaps between windows
    (64, 90, (100, 200), (7, 9)),     # one window larger than the image
    (3, 3, (1, 1), (1, 1)),           # one interior pixel, 1-pixel windows
    (33, 517, (6, 35), (4, 21)),      # ragged cells, gcd 2 x 7
    (61, 203, (8, 16), (24, 8)),      # fused: gaps between window rows, columns overlap
    (40, 300, (30, 6), (10, 2)),      # fused: three cell rows and three cells per window
    (700, 900, (20, 20), (10, 10)),   # fused: bands of window rows per CTA
    (57, 1030, (4, 9), (2, 3)),       # fused: 344 cells per ring row
    (50, 60, (80, 80), (40, 40)),     # fused: one window, larger than the image
    (30, 30, (64, 64), (16, 16)),     # fused: a window wider than the image's cells (zero cells past it)
    (45, 18, (10, 10), (5, 5)),       # fused: rows of 16 codes (the narrowest read in whole words)
    (40, 14, (6, 4), (3, 2)),         # fused: rows of 12 codes (aligned, read byte by byte)
    (31, 642, (20, 20), (10, 10)),    # fused: 640 codes a row, cells of ten columns in whole words
])
def test_single_image_windows(env, H, W, window, stride):
    torch, ldp, oracle, synth = env
    img = synth.image(H * 7 + W, H, W, 3.0)
    d = torch.from_numpy(img).cuda()
    for k, compact in ((3, True), (1, True), (4, True), (6, False)):
        h, c = ldp.window_hist(d, k=k, window=window, stride=stride, compact=compact)
        torch.cuda.synchronize()
        h_ref, c_ref = oracle.extract_windows(img, k=k, window=window, stride=stride, compact=compact)
        assert np.array_equal(c.cpu().numpy(), c_ref), (k, window, stride)
        assert np.array_equal(_h(h), h_ref), (k, window, stride)
    # histogram only: the code map lives in the scratch
    h2, c2 = ldp.window_hist(d, k=3, window=window, stride=stride, with_codes=False)
    torch.cuda.synchronize()
    assert c2 is None
    assert np.array_equal(_h(h2), oracle.extract_windows(img, k=3, window=window, stride=stride)[0])


def test_lbp_windows(env):
    torch, ldp, oracle, synth = env
    img = synth.image(5, 130, 171, 3.0)
    d = torch.from_numpy(img).cuda()
    for window, stride in (((20, 20), None), ((30, 24), (15, 12))):
        h, c = ldp.lbp_window_hist(d, window=window, stride=stride)
        torch.cuda.synchronize()
        h_ref, c_ref = oracle.extract_windows(img, window=window, stride=stride, compact=False,
                                              mode=oracle.MODE_LBP)
        assert np.array_equal(c.cpu().numpy(), c_ref)
        assert np.array_equal(_h(h), h_ref)


def test_ties_and_flat_images(env):
    torch, ldp, oracle, synth = env
    rng = np.random.default_rng(3)
    for img in ((rng.integers(0, 2, (61, 83)) * 255).astype(np.uint8), np.full((40, 50), 7, np.uint8)):
        d = torch.from_numpy(img).cuda()
        for k in (2, 3, 5):
            h, _ = ldp.window_hist(d, k=k, window=(12, 10), stride=(4, 5))
            torch.cuda.synchronize()
            assert np.array_equal(_h(h), oracle.extract_windows(img, k=k, window=(12, 10), stride=(4, 5))[0])


@pytest.mark.parametrize("window,stride,gap", [((20, 20), None, 0), ((24, 16), (12, 8), 0),
                                               ((24, 16), (12, 8), 1), ((20, 20), (15, 15), 0)])
def test_batch_windows_from_plan_codes(env, window, stride, gap):
    """Code maps of an uneven batch from one persistent launch (codes only),
    then the windows of every image in one call (gap = 1: histogram offsets
    that are not multiples of four words)."""
    torch, ldp, oracle, synth = env
    seeds = np.arange(900, 941)
    sizes = [synth.sizes(int(s), 3, 260) for s in seeds]
    Hs, Ws = [h for h, _ in sizes], [w for _, w in sizes]
    k = 3
    sh, sw = window if stride is None else stride
    nwin = [ldp.window_count(h, window[0], sh) * ldp.window_count(w, window[1], sw) for h, w in sizes]
    lay = ldp.BatchLayout.build(Hs, Ws, hist_len=0)
    host = np.zeros(lay.img_bytes, dtype=np.uint8)
    synth.batch_into(host, seeds, Hs, Ws, lay.pitches, lay.img_off)
    d_img = torch.from_numpy(host).cuda()
    d_codes = torch.zeros(lay.code_bytes, dtype=torch.uint8, device="cuda")
    descs = lay.descs(d_img.data_ptr(), d_codes.data_ptr())
    offs = np.concatenate([[0], np.cumsum(np.array(nwin) * 56 + gap)[:-1]]).astype(np.uint64) + gap
    descs["hist_offset"] = offs
    d_desc = torch.from_numpy(descs.view(np.uint8)).cuda()
    d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
    with ldp.BatchPlan(lay.n, lay.pixels, k=k, regions=(1, 1)) as plan:
        plan.run(d_desc, d_count, None)
    d_hist = torch.full((int(sum(nwin)) * 56 + gap * (lay.n + 1),), -1, dtype=torch.int32, device="cuda")
    ldp.batch_window_hist(d_desc, lay.n, (max(Hs), max(Ws)), k, window, stride, hist=d_hist)
    torch.cuda.synchronize()
    hist = _h(d_hist)
    for i in range(lay.n):
        img = np.ascontiguousarray(lay.image(host, i))
        ref, _ = oracle.extract_windows(img, k=k, window=window, stride=stride)
        o = int(offs[i])
        assert np.array_equal(hist[o:o + ref.size].reshape(ref.shape), ref), (i, Hs[i], Ws[i])
    if gap:  # the words between the images' histograms are untouched
        for i in range(lay.n):
            assert int(d_hist[int(offs[i]) - 1]) == -1


@pytest.mark.parametrize("window,stride", [((20, 20), (10, 10)), ((20, 20), (15, 15)), ((10, 10), None)])
def test_batch_windows_reject_images_past_the_bounds(env, window, stride):
    """An image larger than max_H x max_W is skipped on every route (fused,
    cells through scratch, stride = size): its histogram words are left as
    they were and the device status word reports a bad descriptor; the
    other images are exact."""
    torch, ldp, oracle, synth = env
    Hs, Ws = [60, 90, 60], [80, 70, 130]  # image 2 is wider than max_W = 100
    lay = ldp.BatchLayout.build(Hs, Ws, hist_len=0)
    host = np.zeros(lay.img_bytes, dtype=np.uint8)
    synth.batch_into(host, np.arange(3) + 50, Hs, Ws, lay.pitches, lay.img_off)
    d_img = torch.from_numpy(host).cuda()
    d_codes = torch.zeros(lay.code_bytes, dtype=torch.uint8, device="cuda")
    descs = lay.descs(d_img.data_ptr(), d_codes.data_ptr())
    sh, sw = window if stride is None else stride
    nwin = [ldp.window_count(h, window[0], sh) * ldp.window_count(w, window[1], sw) for h, w in zip(Hs, Ws)]
    offs = np.concatenate([[0], np.cumsum(np.array(nwin) * 56)[:-1]]).astype(np.uint64)
    descs["hist_offset"] = offs
    d_desc = torch.from_numpy(descs.view(np.uint8)).cuda()
    d_count = torch.tensor([3], dtype=torch.int32, device="cuda")
    with ldp.BatchPlan(3, lay.pixels, k=3, regions=(1, 1)) as plan:
        plan.run(d_desc, d_count, None)
    ldp.device_status()  # clear
    d_hist = torch.full((int(sum(nwin)) * 56,), -1, dtype=torch.int32, device="cuda")
    ldp.batch_window_hist(d_desc, 3, (100, 100), 3, window, stride, hist=d_hist)
    torch.cuda.synchronize()
    assert ldp.device_status() & 1
    hist = _h(d_hist)
    for i in range(2):
        ref, _ = oracle.extract_windows(np.ascontiguousarray(lay.image(host, i)), k=3, window=window, stride=stride)
        assert np.array_equal(hist[int(offs[i]):int(offs[i]) + ref.size].reshape(ref.shape), ref), i
    assert (d_hist[int(offs[2]):].cpu().numpy() == -1).all()
    assert ldp.device_status() == 0
