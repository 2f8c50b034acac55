"""GPU parity of the crop-and-resize front end (Sec. 3.1) against the
oracle, bit for bit, and the front end chained into batched extraction."""
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


@pytest.mark.parametrize("shape,crop,out_hw", [
    ((490, 640), None, (260, 260)),             # whole frame -> face size
    ((490, 640), (100, 180, 300, 280), (260, 260)),
    ((37, 53), None, (37, 53)),                 # identity
    ((40, 62), None, (20, 31)),                 # exact 2x
    ((9, 23), None, (9, 46)),                   # 2x upsampling
    ((120, 160), (119, 159, 1, 1), (7, 5)),     # one source pixel
    ((50, 700), (3, 10, 44, 600), (333, 17)),   # extreme aspect change
    ((1, 1), None, (4, 300)),
    ((6, 9), None, (3, 4101)),                  # wider than the column table
    ((300, 200), (0, 0, 300, 199), (130, 4096)),  # widest output with the table
    ((20, 32), None, (41, 97)),                 # aligned rows, upsampling (source words)
    ((90, 400), None, (30, 130)),               # aligned rows, about 3x down (source words)
    ((60, 512), (0, 1, 60, 509), (15, 126)),    # about 4x down: groups past 16 bytes gather bytes
])
def test_resize_parity(env, shape, crop, out_hw):
    torch, ldp, oracle, synth = env
    img = synth.image(shape[0] * 3 + shape[1], shape[0], shape[1], 3.0) if min(shape) >= 3 else \
        np.random.default_rng(0).integers(0, 256, shape, dtype=np.uint8)
    d = torch.from_numpy(img).cuda()
    got = ldp.resize(d, out_hw, crop=crop)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), oracle.resize(img, out_hw, crop=crop))
    # padded source and destination rows
    big = torch.zeros((shape[0], shape[1] + 13), dtype=torch.uint8, device="cuda")
    big[:, :shape[1]] = d
    dst = torch.zeros((out_hw[0], out_hw[1] + 7), dtype=torch.uint8, device="cuda")
    ldp.resize(big[:, :shape[1]], out_hw, crop=crop, out=dst[:, :out_hw[1]])
    torch.cuda.synchronize()
    assert np.array_equal(dst[:, :out_hw[1]].cpu().numpy(), oracle.resize(img, out_hw, crop=crop))
    assert (dst[:, out_hw[1]:].cpu().numpy() == 0).all()


def test_batch_resize_then_extract(env):
    """Crops of uneven frames -> 260 x 260 in one launch -> one persistent LDP
    launch over the crops, against oracle resize + oracle extraction."""
    torch, ldp, oracle, synth = env
    rng = np.random.default_rng(4)
    n = 24
    frames = [synth.image(700 + i, int(rng.integers(200, 500)), int(rng.integers(200, 640)), 3.0)
              for i in range(n)]
    crops = []
    for f in frames:
        H, W = f.shape
        ch, cw = int(rng.integers(60, H + 1)), int(rng.integers(60, W + 1))
        crops.append((int(rng.integers(0, H - ch + 1)), int(rng.integers(0, W - cw + 1)), ch, cw))
    d_frames = [torch.from_numpy(f).cuda() for f in frames]
    OH = OW = 260
    lay = ldp.BatchLayout.build([OH] * n, [OW] * n, hist_len=7 * 6 * 56)
    d_img = torch.zeros(lay.img_bytes, dtype=torch.uint8, device="cuda")
    cd = np.zeros(n, dtype=ldp.CROP_DTYPE)
    for i, (f, c) in enumerate(zip(d_frames, crops)):
        cd[i] = (f.data_ptr(), d_img.data_ptr() + int(lay.img_off[i]), f.shape[0], f.shape[1], f.stride(0),
                 c[0], c[1], c[2], c[3], int(lay.pitches[i]))
    ldp.batch_resize(torch.from_numpy(cd.view(np.uint8)).cuda(), n, (OH, OW))
    d_codes = torch.zeros(lay.code_bytes, dtype=torch.uint8, device="cuda")
    d_hist = torch.zeros(n * lay.hist_len, dtype=torch.int32, device="cuda")
    d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
    with ldp.BatchPlan(n, lay.pixels, k=3, regions=(7, 6)) as plan:
        plan.run(d_desc, torch.tensor([n], dtype=torch.int32, device="cuda"), d_hist)
    torch.cuda.synchronize()
    assert ldp.device_status() == 0
    host = d_img.cpu().numpy()
    hist = d_hist.cpu().numpy().astype(np.uint32)
    for i in range(n):
        ref_img = oracle.resize(frames[i], (OH, OW), crop=crops[i])
        assert np.array_equal(lay.image(host, i), ref_img), i
        h_ref, _ = oracle.extract(ref_img, k=3, R=7, C=6)
        assert np.array_equal(hist[i * lay.hist_len:(i + 1) * lay.hist_len].reshape(h_ref.shape), h_ref), i


def test_batch_resize_rejects_bad_crop(env):
    torch, ldp, oracle, synth = env
    f = torch.from_numpy(synth.image(1, 100, 100, 3.0)).cuda()
    dst = torch.zeros((2, 32, 32), dtype=torch.uint8, device="cuda")
    cd = np.zeros(2, dtype=ldp.CROP_DTYPE)
    cd[0] = (f.data_ptr(), dst[0].data_ptr(), 100, 100, 100, 0, 0, 100, 100, 32)
    cd[1] = (f.data_ptr(), dst[1].data_ptr(), 100, 100, 100, 50, 0, 60, 100, 32)  # past the bottom
    ldp.device_status()  # clear
    ldp.batch_resize(torch.from_numpy(cd.view(np.uint8)).cuda(), 2, (32, 32))
    torch.cuda.synchronize()
    assert ldp.device_status() & 8
    assert np.array_equal(dst[0].cpu().numpy(), oracle.resize(f.cpu().numpy(), (32, 32)))
    assert (dst[1].cpu().numpy() == 0).all()
