"""The host-to-host pipeline (copies and compute overlapped over chunks):
results in the host buffers equal the oracle bit for bit, for chunk limits
that cut the batch in many places, one to four buffers, LBP, raw bins and
without codes."""
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


def _batch(env, n, seed0, lo=3, hi=260):
    torch, ldp, oracle, synth = env
    seeds = np.arange(seed0, seed0 + n)
    sizes = [synth.sizes(int(s), lo, hi) for s in seeds]
    Hs, Ws = [h for h, _ in sizes], [w for _, w in sizes]
    lay = ldp.BatchLayout.build(Hs, Ws, hist_len=0)
    h_img = torch.zeros(lay.img_bytes, dtype=torch.uint8, pin_memory=True)
    synth.batch_into(h_img.numpy(), seeds, Hs, Ws, lay.pitches, lay.img_off)
    return lay, h_img


@pytest.mark.parametrize("chunk_images,chunk_px,nbuf", [(5, 1 << 24, 3), (64, 200_000, 2), (1000, 1 << 26, 1),
                                                        (7, 70_000, 4)])
def test_pipeline_matches_oracle(env, chunk_images, chunk_px, nbuf):
    torch, ldp, oracle, synth = env
    lay, h_img = _batch(env, 45, 3100)
    with ldp.Pipeline(chunk_images, chunk_px, k=3, regions=(5, 4), nbuf=nbuf) as pipe:
        h_hist = torch.full((lay.n * pipe.hist_len,), -1, dtype=torch.int32, pin_memory=True)
        h_codes = torch.zeros(lay.code_bytes, dtype=torch.uint8, pin_memory=True)
        for _ in range(2):  # a second run reuses the grown buffers
            pipe.run(h_img, lay, h_hist, h_codes)
            torch.cuda.current_stream().synchronize()
        hist, codes, img = h_hist.numpy().astype(np.uint32), h_codes.numpy(), h_img.numpy()
        for i in range(lay.n):
            im = np.ascontiguousarray(lay.image(img, i))
            h_ref, c_ref = oracle.extract(im, k=3, R=5, C=4)
            assert np.array_equal(hist[i * pipe.hist_len:(i + 1) * pipe.hist_len].reshape(h_ref.shape), h_ref), i
            H, W = im.shape
            co, cp = int(lay.code_off[i]), int(lay.code_pitches[i])
            assert np.array_equal(codes[co:co + (H - 2) * cp].reshape(H - 2, cp)[:, :W - 2], c_ref), i


def test_pipeline_lbp_raw_and_no_codes(env):
    torch, ldp, oracle, synth = env
    lay, h_img = _batch(env, 30, 3300)
    img = h_img.numpy()
    with ldp.Pipeline(8, 1 << 22, regions=(2, 3), lbp=True) as pipe:
        h_hist = torch.zeros(lay.n * pipe.hist_len, dtype=torch.int32, pin_memory=True)
        pipe.run(h_img, lay, h_hist)
        torch.cuda.current_stream().synchronize()
        hist = h_hist.numpy().astype(np.uint32)
        for i in range(lay.n):
            h_ref, _ = oracle.extract(np.ascontiguousarray(lay.image(img, i)), R=2, C=3, mode=oracle.MODE_LBP,
                                      compact=False)
            assert np.array_equal(hist[i * 1536:(i + 1) * 1536].reshape(h_ref.shape), h_ref), i
    with ldp.Pipeline(11, 1 << 22, k=5, regions=(3, 3), compact=False) as pipe:
        h_hist = torch.zeros(lay.n * pipe.hist_len, dtype=torch.int32, pin_memory=True)
        pipe.run(h_img, lay, h_hist)
        torch.cuda.current_stream().synchronize()
        hist = h_hist.numpy().astype(np.uint32)
        for i in range(lay.n):
            h_ref, _ = oracle.extract(np.ascontiguousarray(lay.image(img, i)), k=5, R=3, C=3, compact=False)
            assert np.array_equal(hist[i * pipe.hist_len:(i + 1) * pipe.hist_len].reshape(h_ref.shape), h_ref), i


def test_pipeline_orders_after_the_callers_stream(env):
    """Images written on the caller's stream right before the run are the ones extracted."""
    torch, ldp, oracle, synth = env
    lay, h_img = _batch(env, 12, 3500, lo=40, hi=120)
    ref = h_img.clone()
    h_img.zero_()
    s = torch.cuda.Stream()
    d_tmp = ref.cuda()
    with torch.cuda.stream(s):
        torch.cuda._sleep(20_000_000)  # keep the stream busy, then fill the host images from the device
        h_img.copy_(d_tmp, non_blocking=True)
    with ldp.Pipeline(4, 1 << 20, k=3, regions=(1, 1)) as pipe:
        h_hist = torch.zeros(lay.n * pipe.hist_len, dtype=torch.int32, pin_memory=True)
        pipe.run(h_img, lay, h_hist, stream=s)
        s.synchronize()
        hist = h_hist.numpy().astype(np.uint32)
        for i in range(lay.n):
            h_ref, _ = oracle.extract(np.ascontiguousarray(lay.image(ref.numpy(), i)), k=3)
            assert np.array_equal(hist[i * 56:(i + 1) * 56], h_ref.reshape(-1)), i
