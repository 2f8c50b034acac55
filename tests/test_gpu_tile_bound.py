"""Batch plans on tall and narrow images: every tile variant, including the
8- and 16-row ones, covers every interior pixel (codes and region histograms
bit for bit against the oracle, Eqs. 1-6) and leaves the device status word
clear; the autotuner never keeps a variant whose run was cut short."""
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


def _batch(env, sizes, seed0):
    torch, ldp, oracle, synth = env
    Hs, Ws = [h for h, _ in sizes], [w for _, w in sizes]
    lay = ldp.BatchLayout.build(Hs, Ws, hist_len=7 * 6 * 56)
    host = np.zeros(lay.img_bytes, dtype=np.uint8)
    synth.batch_into(host, list(range(seed0, seed0 + len(sizes))), Hs, Ws, lay.pitches, lay.img_off)
    d_img = torch.from_numpy(host).cuda()
    d_codes = torch.full((lay.code_bytes,), 0xEE, dtype=torch.uint8, device="cuda")
    d_hist = torch.full((lay.n * lay.hist_len,), -1, dtype=torch.int32, device="cuda")
    d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
    d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
    return lay, host, d_codes, d_hist, d_desc, d_count


def _check(env, lay, host, d_codes, d_hist):
    torch, ldp, oracle, synth = env
    torch.cuda.synchronize()
    cc, hc = d_codes.cpu().numpy(), d_hist.cpu().numpy().astype(np.uint32)
    for i in range(lay.n):
        h_ref, c_ref = oracle.extract(lay.image(host, i), k=3, R=7, C=6, compact=True, W=int(lay.Ws[i]))
        assert np.array_equal(lay.codes(cc, i), c_ref), i
        assert np.array_equal(hc[i * lay.hist_len:(i + 1) * lay.hist_len].reshape(h_ref.shape), h_ref), i


# one column or row of output pixels per image, tall and wide, next to ordinary ones
SIZES = [(20000, 3), (9000, 5), (3, 20000), (3, 3), (1000, 7), (4, 1500), (64, 64), (131, 259)]


def test_tall_narrow_batch_every_variant(env):
    torch, ldp, oracle, synth = env
    lay, host, d_codes, d_hist, d_desc, d_count = _batch(env, SIZES, 41000)
    ldp.device_status()
    for v in range(ldp.num_variants()):
        d_codes.fill_(0xEE)
        d_hist.fill_(-1)
        with ldp.BatchPlan(lay.n, lay.pixels, k=3, regions=(7, 6)) as plan:
            plan.set_config(v, 0)
            plan.run(d_desc, d_count, d_hist)
            _check(env, lay, host, d_codes, d_hist)
        assert ldp.device_status() == 0, ldp.variant_name(v)


def test_set_config_grows_the_work_list_of_a_used_plan(env):
    """One plan, run with 64-row tiles first (graph captured), then switched
    to 8-row tiles: the larger work list replaces the old one."""
    torch, ldp, oracle, synth = env
    lay, host, d_codes, d_hist, d_desc, d_count = _batch(env, SIZES[:3], 42000)
    names = [ldp.variant_name(v) for v in range(ldp.num_variants())]
    v8 = next(v for v, n in enumerate(names) if n.startswith("r8w"))
    with ldp.BatchPlan(lay.n, lay.pixels, k=3, regions=(7, 6)) as plan:
        plan.run(d_desc, d_count, d_hist)
        _check(env, lay, host, d_codes, d_hist)
        plan.set_config(v8, 0)
        d_codes.fill_(0xEE)
        plan.run(d_desc, d_count, d_hist)
        _check(env, lay, host, d_codes, d_hist)
    assert ldp.device_status() == 0


def test_autotune_drops_truncated_variants(env):
    """A plan created with max_pixels below the batch's real pixel count (the
    caller broke its own bound): variants of 64 rows and more still fit the
    work list, the 4-, 8- and 16-row ones do not and are clamped on the device.
    Those would time fastest (less work); the tuner must flag and skip them."""
    torch, ldp, oracle, synth = env
    from paper_1810_11518_gb300 import autotune

    lay, host, d_codes, d_hist, d_desc, d_count = _batch(env, [(20000, 3)] * 4, 43000)
    assert lay.pixels == 240000
    with ldp.BatchPlan(lay.n, 180000, k=3, regions=(7, 6)) as plan:
        res = autotune.tune_plan(plan, d_desc, d_count, d_hist, ctas_options=(0,), reps=2, warmup=1)
        flagged = {r["name"] for r in res["all"] if r["status"]}
        short = {ldp.variant_name(v) for v in range(ldp.num_variants())
                 if ldp.variant_name(v).startswith(("r4w", "r8w", "r16w"))}
        assert short and flagged == short
        assert all(r["status"] & 2 for r in res["all"] if r["status"])
        assert res["name"] not in flagged
        d_codes.fill_(0xEE)
        plan.run(d_desc, d_count, d_hist)  # the chosen configuration is complete
        _check(env, lay, host, d_codes, d_hist)
    assert ldp.device_status() == 0
