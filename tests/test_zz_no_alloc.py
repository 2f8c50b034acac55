"""The allocation-free batch entry point (ldp_batch_run_noalloc), called
through the C-ABI and checked against the regular plan-based batch run and
the CPU oracle (Eqs. 1-6, bit for bit) on the same inputs, on two calls in a
row.

It exists for callers that cannot allocate device memory while they run:
memory budgeted once at start-up, or owned by another allocator's pool, or
loops that must not risk an allocation failure or the device-wide
synchronisation that cudaFree can cause.  Its work list lives in one static
device array shared by all calls, so the second call below also checks
that stale contents left by the first call do not leak into its results.

This file is named to be collected last."""
import ctypes

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
    import paper_1810_11518_gb300 as ldp
    import synth
    from paper_1810_11518_gb300 import _abi

    return torch, ldp, synth, _abi


def _batch(env, seeds, lo, hi, k):
    torch, ldp, synth, _abi = env
    sizes = [synth.sizes(s, lo, hi) for s in seeds]
    Hs, Ws = [h for h, _ in sizes], [w for _, w in sizes]
    lay = ldp.BatchLayout.build(Hs, Ws, hist_len=7 * 6 * ldp.hist_bins(k))
    host = np.zeros(lay.img_bytes, dtype=np.uint8)
    synth.batch_into(host, seeds, Hs, Ws, lay.pitches, lay.img_off)
    d_img = torch.from_numpy(host).cuda()
    return lay, host, d_img, max(max(Hs), max(Ws))


def _run_both(env, lay, d_img, max_side, k):
    """(codes, hist) from the plan-based run and from the no-alloc run."""
    torch, ldp, synth, _abi = env
    lib = _abi.load()
    out = []
    for noalloc in (False, True):
        d_codes = torch.full((lay.code_bytes,), 0xEE, dtype=torch.uint8, device="cuda")
        d_hist = torch.full((lay.n * lay.hist_len,), -7, dtype=torch.int32, device="cuda")
        d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
        if noalloc:
            rc = lib.ldp_batch_run_noalloc(ctypes.c_void_p(d_desc.data_ptr()), lay.n, lay.pixels, max_side, k,
                                           _abi.RegionSpec(7, 6, 1), ctypes.c_void_p(d_hist.data_ptr()), None)
            assert rc == 0, lib.ldp_last_error()
        else:
            d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
            with ldp.BatchPlan(lay.n, lay.pixels, k=k, regions=(7, 6)) as plan:
                plan.run(d_desc, d_count, d_hist)
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        out.append((d_codes.cpu().numpy(), d_hist.cpu().numpy()))
    return out


def test_noalloc_matches_plan_run_twice(env):
    import oracle

    torch, ldp, synth, _abi = env
    # first call: 24 uneven images; second call: a different, smaller batch
    # with another k, so the shared array holds the first call's leftovers
    for seeds, lo, hi, k in ((list(range(3000, 3024)), 3, 400, 3), (list(range(3100, 3107)), 30, 260, 2)):
        lay, host, d_img, max_side = _batch(env, seeds, lo, hi, k)
        (c_ref, h_ref), (c_na, h_na) = _run_both(env, lay, d_img, max_side, k)
        for i in range(lay.n):  # compare inside each code rectangle, tolerance 0
            assert np.array_equal(lay.codes(c_na, i), lay.codes(c_ref, i)), i
            # and against the oracle, image by image
            ho, co = oracle.extract(lay.image(host, i), k=k, R=7, C=6, compact=True, W=int(lay.Ws[i]))
            assert np.array_equal(lay.codes(c_na, i), co), i
            assert np.array_equal(h_na[i * lay.hist_len:(i + 1) * lay.hist_len].astype(np.uint32),
                                  ho.reshape(-1)), i
        assert np.array_equal(h_na, h_ref)
        assert (h_ref.reshape(lay.n, -1).sum(axis=1) == (lay.Hs - 2) * (lay.Ws - 2)).all()
    assert ldp.device_status() == 0


def test_noalloc_rejects_oversized_batch(env):
    torch, ldp, synth, _abi = env
    lib = _abi.load()
    d = torch.zeros(40, dtype=torch.uint8, device="cuda")
    rc = lib.ldp_batch_run_noalloc(ctypes.c_void_p(d.data_ptr()), 1, 1 << 36, 1 << 16, 3, _abi.RegionSpec(7, 6, 1),
                                   None, None)
    assert rc == _abi.LDP_EINVAL
    assert b"static work list" in lib.ldp_last_error()
