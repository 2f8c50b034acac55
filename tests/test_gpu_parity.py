"""GPU parity: every result of the CUDA path against the CPU oracle, bit for
bit (integer work: tolerance 0), through the C-ABI."""
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


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _hist_np(h):
    return h.cpu().numpy().astype(np.uint32)


def test_640x490_plain_whole_image(env):
    """640x490 image from seed 0 (sigma 3), k = 3, 638x488 codes and one
    256-bin whole-image histogram."""
    torch, ldp, oracle, synth = env
    img = synth.image(0, 490, 640, 3.0)
    h, c = ldp.region_hist(_dev(torch, img), k=3, regions=(1, 1), compact=False)
    torch.cuda.synchronize()
    h_ref, c_ref = oracle.extract(img, k=3, R=1, C=1, compact=False)
    assert c.shape == (488, 638)
    assert np.array_equal(c.cpu().numpy(), c_ref)
    assert np.array_equal(_hist_np(h), h_ref)
    assert int(h.sum()) == 488 * 638


@pytest.mark.parametrize("k", range(1, 8))
def test_all_k_regions(env, k):
    torch, ldp, oracle, synth = env
    img = synth.image(100 + k, 203, 333, 3.0)  # several tiles and a ragged tail both ways
    d = _dev(torch, img)
    for regions, compact in (((7, 6), True), ((3, 5), False), ((1, 1), True)):
        h, c = ldp.region_hist(d, k=k, regions=regions, compact=compact)
        torch.cuda.synchronize()
        h_ref, c_ref = oracle.extract(img, k=k, R=regions[0], C=regions[1], compact=compact)
        assert np.array_equal(c.cpu().numpy(), c_ref), (k, regions)
        assert np.array_equal(_hist_np(h), h_ref), (k, regions)
    c2 = ldp.codes(d, k=k)
    torch.cuda.synchronize()
    assert np.array_equal(c2.cpu().numpy(), c_ref)


def test_lbp(env):
    torch, ldp, oracle, synth = env
    img = synth.image(7, 150, 261, 3.0)
    d = _dev(torch, img)
    c = ldp.lbp_codes(d)
    h, c2 = ldp.lbp_region_hist(d, regions=(4, 3))
    torch.cuda.synchronize()
    h_ref, c_ref = oracle.extract(img, R=4, C=3, mode=oracle.MODE_LBP, compact=False)
    assert np.array_equal(c.cpu().numpy(), c_ref)
    assert np.array_equal(c2.cpu().numpy(), c_ref)
    assert np.array_equal(_hist_np(h), h_ref)


def test_worked_examples_on_gpu(env):
    import json
    import os

    torch, ldp, oracle, synth = env
    with open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")) as f:
        exs = json.load(f)["examples"]
    for ex in exs:
        img = np.array(ex["image"], dtype=np.uint8)
        d = _dev(torch, img)
        for k, code in ex["ldp"].items():
            c = ldp.codes(d, k=int(k))
            torch.cuda.synchronize()
            assert int(c[0, 0]) == code, (ex["name"], k)
        assert int(ldp.lbp_codes(d)[0, 0]) == ex["lbp"]


@pytest.mark.parametrize("H,W", [(3, 3), (3, 50), (50, 3), (4, 4), (5, 7), (17, 131), (130, 5),
                                 (65, 129), (66, 130), (129, 258), (300, 17)])
def test_edge_sizes(env, H, W):
    torch, ldp, oracle, synth = env
    rng = np.random.default_rng(H * 1000 + W)
    for kind in range(3):
        if kind == 0:
            img = rng.integers(0, 256, (H, W), dtype=np.uint8)
        elif kind == 1:
            img = (rng.integers(0, 2, (H, W)) * 255).astype(np.uint8)  # heavy ties
        else:
            img = np.full((H, W), 9, dtype=np.uint8)
        d = _dev(torch, img)
        for k in (1, 3, 6):
            h, c = ldp.region_hist(d, k=k, regions=(2, 3), compact=True)
            torch.cuda.synchronize()
            h_ref, c_ref = oracle.extract(img, k=k, R=2, C=3, compact=True)
            assert np.array_equal(c.cpu().numpy(), c_ref)
            assert np.array_equal(_hist_np(h), h_ref)


def test_pitch_and_unaligned_pointers(env):
    """Any pitch and any alignment, for every tile variant (staged variants
    copy rows they cannot bulk-copy with plain loads)."""
    torch, ldp, oracle, synth = env
    img = synth.image(11, 77, 150, 3.0)
    h_ref, c_ref = oracle.extract(img, k=3, R=3, C=4, compact=True)
    try:
        for v in range(ldp.num_variants()):
            ldp.set_plain_variant(v)
            for pitch, off in ((150, 0), (160, 0), (151, 0), (163, 5), (150, 1), (256, 3)):
                big = torch.zeros(77 * pitch + off + 64, dtype=torch.uint8, device="cuda")
                view = big[off:off + 77 * pitch].view(77, pitch)[:, :150]
                view.copy_(_dev(torch, img))
                for cpitch, coff in ((148, 0), (149, 1), (160, 7)):
                    cbuf = torch.zeros((75 * cpitch + coff,), dtype=torch.uint8, device="cuda")
                    cview = cbuf[coff:coff + 75 * cpitch].view(75, cpitch)[:, :148]
                    h, c = ldp.region_hist(view, k=3, regions=(3, 4), codes_out=cview)
                    torch.cuda.synchronize()
                    assert np.array_equal(c.cpu().numpy(), c_ref), (v, pitch, off, cpitch, coff)
                    assert np.array_equal(_hist_np(h), h_ref)
                    # bytes outside the code rectangle are untouched
                    full = cbuf.cpu().numpy()
                    inside = np.zeros_like(full, dtype=bool)
                    for r in range(75):
                        inside[coff + r * cpitch: coff + r * cpitch + 148] = True
                    assert (full[~inside] == 0).all()
            # an image whose buffer ends exactly at its last byte (no pitch padding on the last row)
            H, W, P = 70, 133, 144
            tight = torch.zeros((H - 1) * P + W, dtype=torch.uint8, device="cuda")
            img2 = synth.image(12, H, W, 3.0)
            rows = np.zeros((H, P), dtype=np.uint8)
            rows[:, :W] = img2
            tight.copy_(_dev(torch, rows.reshape(-1)[:(H - 1) * P + W]))
            view2 = torch.as_strided(tight, (H, W), (P, 1))
            h, c = ldp.region_hist(view2, k=3, regions=(2, 2))
            torch.cuda.synchronize()
            h_ref2, c_ref2 = oracle.extract(img2, k=3, R=2, C=2)
            assert np.array_equal(c.cpu().numpy(), c_ref2) and np.array_equal(_hist_np(h), h_ref2), v
    finally:
        ldp.set_plain_variant(-1)


def test_many_small_regions_global_path(env):
    """A region grid finer than a tile (more than 16 regions per tile)
    takes the direct global-atomic path."""
    torch, ldp, oracle, synth = env
    img = synth.image(12, 140, 270, 3.0)
    d = _dev(torch, img)
    for R, C in ((140, 270), (35, 90), (200, 300), (17, 40)):
        h, c = ldp.region_hist(d, k=3, regions=(R, C), compact=True)
        torch.cuda.synchronize()
        h_ref, _ = oracle.extract(img, k=3, R=R, C=C, compact=True)
        assert np.array_equal(_hist_np(h), h_ref), (R, C)


def test_histogram_is_overwritten(env):
    torch, ldp, oracle, synth = env
    img = synth.image(13, 64, 64, 3.0)
    d = _dev(torch, img)
    hist = torch.full((2, 2, 56), 12345, dtype=torch.int32, device="cuda")
    ldp.region_hist(d, k=3, regions=(2, 2), hist=hist, with_codes=False)
    ldp.region_hist(d, k=3, regions=(2, 2), hist=hist, with_codes=False)
    torch.cuda.synchronize()
    h_ref, _ = oracle.extract(img, k=3, R=2, C=2, compact=True, want_codes=False)
    assert np.array_equal(_hist_np(hist), h_ref)


def test_streams(env):
    torch, ldp, oracle, synth = env
    imgs = [synth.image(20 + i, 90, 120, 3.0) for i in range(4)]
    streams = [torch.cuda.Stream() for _ in range(4)]
    outs = []
    for img, s in zip(imgs, streams):
        with torch.cuda.stream(s):
            d = _dev(torch, img)
            outs.append(ldp.region_hist(d, k=3, regions=(2, 2), stream=s))
    torch.cuda.synchronize()
    for img, (h, c) in zip(imgs, outs):
        h_ref, c_ref = oracle.extract(img, k=3, R=2, C=2)
        assert np.array_equal(c.cpu().numpy(), c_ref) and np.array_equal(_hist_np(h), h_ref)


def test_all_variants(env):
    torch, ldp, oracle, synth = env
    img = synth.image(30, 261, 400, 3.0)
    d = _dev(torch, img)
    h_ref, c_ref = oracle.extract(img, k=3, R=7, C=6)
    try:
        for v in range(ldp.num_variants()):
            ldp.set_plain_variant(v)
            h, c = ldp.region_hist(d, k=3, regions=(7, 6))
            torch.cuda.synchronize()
            assert np.array_equal(c.cpu().numpy(), c_ref), ldp.variant_name(v)
            assert np.array_equal(_hist_np(h), h_ref), ldp.variant_name(v)
    finally:
        ldp.set_plain_variant(-1)
