"""Guard bands: every output buffer sits inside a larger one filled with a
sentinel, and nothing outside the output changes -- region histograms (shared
and global-atomic paths), sliding windows, batch histograms with gaps
between images, codes with pitch padding, resized images and distance
matrices."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SENT = -1515870811  # 0xA5A5A5A5 as int32
GUARD = 4096


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


def _guarded(torch, n, dtype=None):
    torch_dtype = dtype or torch.int32
    buf = torch.full((n + 2 * GUARD,), SENT if torch_dtype == torch.int32 else 0xA5, dtype=torch_dtype,
                     device="cuda")
    return buf, buf[GUARD:GUARD + n]


def _guards_intact(buf, n, sent):
    b = buf.cpu().numpy()
    return (b[:GUARD] == sent).all() and (b[GUARD + n:] == sent).all()


def test_region_and_window_histograms(env):
    torch, ldp, oracle, synth = env
    img = synth.image(21, 150, 261, 3.0)
    d = torch.from_numpy(img).cuda()
    for regions in ((7, 6), (60, 90)):  # shared-memory and global-atomic paths
        n = regions[0] * regions[1] * 56
        buf, view = _guarded(torch, n)
        ldp.region_hist(d, k=3, regions=regions, hist=view, with_codes=False)
        torch.cuda.synchronize()
        assert _guards_intact(buf, n, SENT), regions
        assert np.array_equal(view.cpu().numpy().astype(np.uint32).reshape(regions + (56,)),
                              oracle.extract(img, k=3, R=regions[0], C=regions[1], want_codes=False)[0])
    for window, stride in (((20, 20), None), ((30, 24), (10, 8))):
        sh, sw = window if stride is None else stride
        n = ldp.window_count(150, window[0], sh) * ldp.window_count(261, window[1], sw) * 56
        buf, view = _guarded(torch, n)
        ldp.window_hist(d, k=3, window=window, stride=stride, hist=view, with_codes=False)
        torch.cuda.synchronize()
        assert _guards_intact(buf, n, SENT), window


def test_batch_histograms_with_gaps(env):
    torch, ldp, oracle, synth = env
    sizes = [synth.sizes(s, 3, 200) for s in range(300, 320)]
    Hs, Ws = [h for h, _ in sizes], [w for _, w in sizes]
    hist_len = 5 * 4 * 56
    stride = hist_len + 37  # a gap after every image's histogram
    lay = ldp.BatchLayout.build(Hs, Ws, hist_len=hist_len)
    host = np.zeros(lay.img_bytes, dtype=np.uint8)
    synth.batch_into(host, np.arange(300, 320), Hs, Ws, lay.pitches, lay.img_off)
    d_img = torch.from_numpy(host).cuda()
    d_codes = torch.full((lay.code_bytes,), 0xA5, dtype=torch.uint8, device="cuda")
    descs = lay.descs(d_img.data_ptr(), d_codes.data_ptr())
    descs["hist_offset"] = np.arange(lay.n, dtype=np.uint64) * np.uint64(stride)
    d_desc = torch.from_numpy(descs.view(np.uint8)).cuda()
    d_hist = torch.full((lay.n * stride,), SENT, dtype=torch.int32, device="cuda")
    with ldp.BatchPlan(lay.n, lay.pixels, k=3, regions=(5, 4)) as plan:
        plan.run(d_desc, torch.tensor([lay.n], dtype=torch.int32, device="cuda"), d_hist)
    torch.cuda.synchronize()
    h = d_hist.cpu().numpy()
    codes = d_codes.cpu().numpy()
    for i in range(lay.n):
        assert (h[i * stride + hist_len:(i + 1) * stride] == SENT).all(), i
        H, W = Hs[i], Ws[i]
        cp, co = int(lay.code_pitches[i]), int(lay.code_off[i])
        block = codes[co:co + (H - 2) * cp].reshape(H - 2, cp)
        assert (block[:, W - 2:] == 0xA5).all(), i  # pitch padding untouched
        h_ref, c_ref = oracle.extract(np.ascontiguousarray(lay.image(host, i)), k=3, R=5, C=4)
        assert np.array_equal(block[:, :W - 2], c_ref), i


def test_resize_and_distances(env):
    torch, ldp, oracle, synth = env
    frame = torch.from_numpy(synth.image(5, 200, 300, 3.0)).cuda()
    OH, OW = 61, 47
    buf = torch.full((OH + 4, OW + 16), 0xA5, dtype=torch.uint8, device="cuda")
    view = buf[2:2 + OH, 8:8 + OW]
    ldp.resize(frame, (OH, OW), crop=(10, 20, 150, 200), out=view)
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    mask = np.ones_like(b, dtype=bool)
    mask[2:2 + OH, 8:8 + OW] = False
    assert (b[mask] == 0xA5).all()
    q = torch.randint(0, 1000, (7, 100), dtype=torch.int32, device="cuda")
    g = torch.randint(0, 1000, (9, 100), dtype=torch.int32, device="cuda")
    out = torch.full((7 + 2, 9 + 5), -7, dtype=torch.int64, device="cuda")
    ldp.hist_distance(q, g, ldp.DIST_L1, out=out[1:8, 2:11])
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    inner = np.zeros_like(o, dtype=bool)
    inner[1:8, 2:11] = True
    assert (o[~inner] == -7).all()
    assert np.array_equal(o[1:8, 2:11].astype(np.uint64),
                          oracle.hist_distance(q.cpu().numpy(), g.cpu().numpy(), oracle.DIST_L1))
