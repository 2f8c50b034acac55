"""The checked build (-DLDP_CHECKED: every shared- and global-memory index of
the tile loop, the window kernels and the resize gathers tested against its
buffer, violations recorded in the device status word instead of trapping)
runs the parity cases with no violation.
It stands in for a memory checker, which this environment does not offer.
The cases run in a child process that loads the checked library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch, sys
sys.path.insert(0, ROOT)
import oracle, synth
import paper_1810_11518_gb300 as ldp
assert ldp.load()._name.endswith("libldp_checked.so")
ldp.device_status()
rng = np.random.default_rng(0)
cases = [synth.image(1, 203, 333, 3.0), synth.image(2, 3, 3, 3.0), synth.image(3, 70, 131, 3.0),
         (rng.integers(0, 2, (66, 130)) * 255).astype(np.uint8)]
for img in cases:
    d = torch.from_numpy(img).cuda()
    for k in (1, 3, 6):
        for regions, compact in (((7, 6), True), ((2, 3), False), ((40, 60), True)):
            h, c = ldp.region_hist(d, k=k, regions=regions, compact=compact)
            h_ref, c_ref = oracle.extract(img, k=k, R=regions[0], C=regions[1], compact=compact)
            assert np.array_equal(c.cpu().numpy(), c_ref) and np.array_equal(h.cpu().numpy().astype(np.uint32), h_ref)
    for cm, om in ((ldp.CODE_RAW, oracle.MODE_LDP_RAW), (ldp.CODE_ABS_THRESH, oracle.MODE_LDP_THRESH)):
        h, c = ldp.region_hist(d, k=3, regions=(3, 3), compact=False, code_mode=cm)
        assert np.array_equal(h.cpu().numpy().astype(np.uint32), oracle.extract(img, k=3, R=3, C=3, compact=False, mode=om)[0])
    h, c = ldp.lbp_region_hist(d, regions=(2, 2))
    assert np.array_equal(h.cpu().numpy().astype(np.uint32), oracle.extract(img, R=2, C=2, mode=oracle.MODE_LBP, compact=False)[0])
# a batch of uneven images through every tile variant
sizes = [synth.sizes(s, 3, 300) for s in range(40)]
Hs, Ws = [h for h, _ in sizes], [w for _, w in sizes]
lay = ldp.BatchLayout.build(Hs, Ws, hist_len=7 * 6 * 56)
host = np.zeros(lay.img_bytes, dtype=np.uint8)
synth.batch_into(host, np.arange(40), Hs, Ws, lay.pitches, lay.img_off)
d_img = torch.from_numpy(host).cuda()
d_codes = torch.zeros(lay.code_bytes, dtype=torch.uint8, device="cuda")
d_hist = torch.zeros(lay.n * lay.hist_len, dtype=torch.int32, device="cuda")
d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
for v in range(ldp.num_variants()):
    with ldp.BatchPlan(lay.n, lay.pixels, k=3, regions=(7, 6)) as plan:
        plan.set_config(v, 0)
        plan.run(d_desc, d_count, d_hist)
    hist = d_hist.cpu().numpy().astype(np.uint32)
    for i in range(lay.n):
        h_ref, _ = oracle.extract(np.ascontiguousarray(lay.image(host, i)), k=3, R=7, C=6)
        assert np.array_equal(hist[i * lay.hist_len:(i + 1) * lay.hist_len].reshape(h_ref.shape), h_ref), (v, i)
# sliding windows on every route (fused ring, stride = size, cells through scratch), single and batched
img = synth.image(5, 77, 150, 3.0)
d = torch.from_numpy(img).cuda()
for window, stride in (((20, 16), (10, 8)), ((12, 10), (4, 5)), ((20, 20), None), ((9, 12), (15, 20)),
                       ((64, 64), (16, 16))):
    for k, compact in ((3, True), (4, True), (6, False)):
        h, _ = ldp.window_hist(d, k=k, window=window, stride=stride, compact=compact, with_codes=False)
        h_ref, _ = oracle.extract_windows(img, k=k, window=window, stride=stride, compact=compact)
        assert np.array_equal(h.cpu().numpy().astype(np.uint32), h_ref), (window, stride, k)
    descs = lay.descs(d_img.data_ptr(), d_codes.data_ptr())
    sh, sw = window if stride is None else stride
    nwin = [ldp.window_count(h_, window[0], sh) * ldp.window_count(w_, window[1], sw) for h_, w_ in zip(Hs, Ws)]
    offs = np.concatenate([[0], np.cumsum(np.array(nwin) * 56)[:-1]]).astype(np.uint64)
    descs["hist_offset"] = offs
    wd = torch.from_numpy(descs.view(np.uint8)).cuda()
    wh = torch.zeros(int(sum(nwin)) * 56, dtype=torch.int32, device="cuda")
    ldp.batch_window_hist(wd, lay.n, (max(Hs), max(Ws)), 3, window, stride, hist=wh)
    wh = wh.cpu().numpy().astype(np.uint32)
    for i in range(0, lay.n, 7):
        ref, _ = oracle.extract_windows(np.ascontiguousarray(lay.image(host, i)), k=3, window=window, stride=stride)
        assert np.array_equal(wh[int(offs[i]):int(offs[i]) + ref.size].reshape(ref.shape), ref), (window, i)
# crop-and-resize, both column paths
for shape, crop, out_hw in (((490, 640), (100, 180, 300, 280), (260, 260)), ((9, 23), None, (9, 46)),
                            ((6, 9), None, (3, 4101))):
    src = synth.image(shape[0] + shape[1], shape[0], shape[1], 3.0)
    got = ldp.resize(torch.from_numpy(src).cuda(), out_hw, crop=crop)
    assert np.array_equal(got.cpu().numpy(), oracle.resize(src, out_hw, crop=crop)), shape
torch.cuda.synchronize()
print("status", ldp.device_status())
"""


def test_checked_build_runs_clean():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    from paper_1810_11518_gb300 import build as libbuild

    __graft_entry__.build()
    lib = libbuild.build(checked=True)
    env = dict(os.environ, LDP_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "status 0" in r.stdout, r.stdout[-2000:]
