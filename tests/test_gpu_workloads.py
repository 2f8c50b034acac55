"""GPU parity at the workload sizes: the batched persistent path, in the
launch configuration bench.py uses (autotuned tile variant), against the CPU
oracle bit for bit.

- 4096 images of 640x490 (seeds 0..4095): every image's k=3 codes and 7x6x56
  histograms, and every image's LBP codes and 256-bin histogram.
- 2048 images, H and W uniform on [64, 1024]: every image.
- 64 images of 8192x8192 (sigma 6), k = 1..4, 16x16 region histograms: 8 full
  images per k against the oracle, and on all 64 images the invariants that
  hold at any size (histogram mass, popcount of every code, region sums).
"""
import os

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


def _configured_plan(env, lay, k, regions, lbp=False):
    torch, ldp, oracle, synth = env
    from paper_1810_11518_gb300 import autotune

    plan = ldp.BatchPlan(lay.n, lay.pixels, k=k, regions=regions, lbp=lbp)
    props = torch.cuda.get_device_properties(0)
    ent = autotune.lookup(torch.cuda.get_device_name(0), props.multi_processor_count, "batch", 0 if lbp else k,
                          "lbp+hist+codes" if lbp else "hist+codes", lay.pixels / lay.n)
    if ent:
        plan.set_config(ent["variant"], ent["ctas_per_sm"])
    return plan


def _device_batch(env, lay, host, hist_len):
    torch = env[0]
    d_img = torch.from_numpy(host).cuda()
    d_codes = torch.zeros(lay.code_bytes, dtype=torch.uint8, device="cuda")
    d_hist = torch.zeros(lay.n * hist_len, dtype=torch.int32, device="cuda")
    descs = lay.descs(d_img.data_ptr(), d_codes.data_ptr())
    descs["hist_offset"] = np.arange(lay.n, dtype=np.uint64) * np.uint64(hist_len)
    d_desc = torch.from_numpy(descs.view(np.uint8)).cuda()
    d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
    return d_img, d_codes, d_hist, d_desc, d_count


def _compare_all(env, lay, host, d_codes, d_hist, hist_len, k, R, C, compact, mode, idx=None):
    torch, ldp, oracle, synth = env
    idx = np.arange(lay.n) if idx is None else np.asarray(idx)
    # the oracle reads the images where they are (offsets and pitches), all host threads
    h_ref, c_ref = oracle.extract_batch(host, lay.img_off[idx], lay.Hs[idx], lay.Ws[idx], lay.pitches[idx],
                                        k=k, R=R, C=C, compact=compact, mode=mode, want_codes=True)
    hc = d_hist.cpu().numpy().astype(np.uint32).reshape(lay.n, hist_len)
    cc = d_codes.cpu().numpy()
    for j, i in enumerate(idx):
        assert np.array_equal(hc[i], h_ref[j].reshape(-1)), f"histogram of image {i}"
        assert np.array_equal(lay.codes(cc, i), c_ref[j]), f"codes of image {i}"


def test_4096_images_640x490_ldp_and_lbp(env):
    torch, ldp, oracle, synth = env
    n, H, W = 4096, 490, 640
    lay = ldp.BatchLayout.build([H] * n, [W] * n, hist_len=7 * 6 * 56)
    host = np.zeros(lay.img_bytes, dtype=np.uint8)
    synth.batch_into(host, np.arange(n), lay.Hs, lay.Ws, lay.pitches, lay.img_off, sigma=3.0)
    d_img, d_codes, d_hist, d_desc, d_count = _device_batch(env, lay, host, 7 * 6 * 56)
    with _configured_plan(env, lay, 3, (7, 6)) as plan:
        plan.run(d_desc, d_count, d_hist)
        torch.cuda.synchronize()
    _compare_all(env, lay, host, d_codes, d_hist, 7 * 6 * 56, 3, 7, 6, True, oracle.MODE_LDP)
    # LBP on the same images: codes + one 256-bin whole-image histogram
    d_img, d_codes, d_hist, d_desc, d_count = _device_batch(env, lay, host, 256)
    with _configured_plan(env, lay, 3, (1, 1), lbp=True) as plan:
        plan.run(d_desc, d_count, d_hist)
        torch.cuda.synchronize()
    _compare_all(env, lay, host, d_codes, d_hist, 256, 3, 1, 1, False, oracle.MODE_LBP)


def test_2048_uneven_images(env):
    torch, ldp, oracle, synth = env
    n = 2048
    sizes = [synth.sizes(s, 64, 1024) for s in range(n)]
    Hs, Ws = [h for h, _ in sizes], [w for _, w in sizes]
    lay = ldp.BatchLayout.build(Hs, Ws, hist_len=7 * 6 * 56)
    host = np.zeros(lay.img_bytes, dtype=np.uint8)
    synth.batch_into(host, np.arange(n), lay.Hs, lay.Ws, lay.pitches, lay.img_off, sigma=3.0)
    d_img, d_codes, d_hist, d_desc, d_count = _device_batch(env, lay, host, 7 * 6 * 56)
    with _configured_plan(env, lay, 3, (7, 6)) as plan:
        plan.run(d_desc, d_count, d_hist)
        torch.cuda.synchronize()
        assert ldp.device_status() == 0
    _compare_all(env, lay, host, d_codes, d_hist, 7 * 6 * 56, 3, 7, 6, True, oracle.MODE_LDP)


@pytest.fixture(scope="module")
def large_batch(env):
    torch, ldp, oracle, synth = env
    n, S = 64, 8192
    lay = ldp.BatchLayout.build([S] * n, [S] * n, hist_len=16 * 16 * 70)
    host = np.zeros(lay.img_bytes, dtype=np.uint8)
    synth.batch_into(host, np.arange(n), lay.Hs, lay.Ws, lay.pitches, lay.img_off, sigma=6.0)
    return lay, host


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_64_images_8192_squared(env, large_batch, k):
    torch, ldp, oracle, synth = env
    lay, host = large_batch
    nb = ldp.hist_bins(k)
    hist_len = 16 * 16 * nb
    d_img, d_codes, d_hist, d_desc, d_count = _device_batch(env, lay, host, hist_len)
    with _configured_plan(env, lay, k, (16, 16)) as plan:
        plan.run(d_desc, d_count, d_hist)
        torch.cuda.synchronize()
    # invariants on every image, computed on the device
    S = 8192
    hv = d_hist.view(lay.n, 16, 16, nb).to(torch.int64)
    assert (hv.sum(dim=(1, 2, 3)) == (S - 2) ** 2).all()
    # region band b holds rows [512 b, 512 (b+1)); the border row / column is not counted
    band = torch.full((16,), 512, dtype=torch.int64, device="cuda")
    band[0] -= 1
    band[-1] -= 1
    assert (hv.sum(dim=3) == band[:, None] * band[None, :]).all()
    # every code has popcount k, and the code map's value counts equal the
    # histograms summed over regions (compact bin b <-> b-th code of popcount k)
    codes_k = torch.tensor(oracle.compact_codes(k), dtype=torch.int64, device="cuda")
    cp = int(lay.code_pitches[0])
    for i in range(lay.n):
        cm = d_codes[int(lay.code_off[i]):int(lay.code_off[i]) + (S - 2) * cp].view(S - 2, cp)[:, :S - 2]
        counts = torch.bincount(cm.reshape(-1).to(torch.int64), minlength=256)
        assert int(counts.sum()) == (S - 2) ** 2
        assert int(counts[codes_k].sum()) == (S - 2) ** 2, f"image {i}: a code without popcount {k}"
        assert torch.equal(counts[codes_k], hv[i].sum(dim=(0, 1))), f"image {i}: codes and histograms disagree"
    # full oracle comparison on 8 of the 64 images
    _compare_all(env, lay, host, d_codes, d_hist, hist_len, k, 16, 16, True, oracle.MODE_LDP,
                 idx=[0, 9, 18, 27, 36, 45, 54, 63])
