"""Error paths, exercised without faulting the GPU: failures are injected on
the host (ldp_test_inject_fault) the way a real out-of-memory or launch
failure would surface, and the device-side bounded wait of the staged tile
variants is made to run out (checked build, a stage that is never filled, so
no copy is in flight for it).  Each test checks the error code, the message
and that the library stays usable afterwards."""
import os
import subprocess
import sys
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    from paper_1810_11518_gb300 import _abi, serving

    yield torch, ldp, oracle, synth, _abi, serving
    ldp.inject_fault(ldp.FAULT_DEVICE_ALLOC, 0)
    ldp.inject_fault(ldp.FAULT_SERVER_LAUNCH, 0)


def test_plan_allocation_failure(env):
    torch, ldp, oracle, synth, _abi, serving = env
    ldp.inject_fault(ldp.FAULT_DEVICE_ALLOC, 1)
    with pytest.raises(ldp.LdpError) as ei:
        ldp.BatchPlan(16, 1 << 20, k=3)
    assert ei.value.status == _abi.LDP_ENOMEM and "work list" in str(ei.value)
    # the fault is used up: the next plan is created and runs; growing its
    # work list for 8-row tiles fails once and leaves the plan as it was
    img = synth.image(7, 300, 200, 3.0)
    lay = ldp.BatchLayout.build([300], [200], hist_len=7 * 6 * 56)
    host = np.zeros(lay.img_bytes, dtype=np.uint8)
    synth.batch_into(host, [7], [300], [200], lay.pitches, lay.img_off)
    d_img = torch.from_numpy(host).cuda()
    d_codes = torch.zeros(lay.code_bytes, dtype=torch.uint8, device="cuda")
    d_hist = torch.zeros(lay.hist_len, dtype=torch.int32, device="cuda")
    d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
    d_count = torch.tensor([1], dtype=torch.int32, device="cuda")
    v8 = next(v for v in range(ldp.num_variants()) if ldp.variant_name(v).startswith("r8w"))
    with ldp.BatchPlan(16, lay.pixels, k=3) as plan:
        ldp.inject_fault(ldp.FAULT_DEVICE_ALLOC, 1)
        with pytest.raises(ldp.LdpError) as ei:
            plan.set_config(v8, 0)
        assert ei.value.status == _abi.LDP_ENOMEM
        plan.run(d_desc, d_count, d_hist)
        torch.cuda.synchronize()
    h_ref, c_ref = oracle.extract(img, k=3, R=7, C=6)
    assert np.array_equal(lay.codes(d_codes.cpu().numpy(), 0), c_ref)
    assert np.array_equal(d_hist.cpu().numpy().astype(np.uint32).reshape(h_ref.shape), h_ref)
    assert ldp.device_status() == 0


@pytest.mark.parametrize("after", [0, 1, 4, 6])
def test_server_allocation_failure(env, after):
    """The arena (the first device allocation), a per-stream buffer or a
    stream's batch plan fails: the create call returns ENOMEM, frees what it
    had, and a server created afterwards works."""
    torch, ldp, oracle, synth, _abi, serving = env
    ldp.inject_fault(ldp.FAULT_DEVICE_ALLOC, 1, after=after)
    with pytest.raises(ldp.LdpError) as ei:
        serving.Server(streams=2, arena_bytes=8 << 20)
    assert ei.value.status == _abi.LDP_ENOMEM
    ldp.inject_fault(ldp.FAULT_DEVICE_ALLOC, 0)
    img = synth.image(11, 120, 90, 3.0)
    h = np.zeros(7 * 6 * 56, dtype=np.uint32)
    with serving.Server(streams=2, arena_bytes=8 << 20) as srv:
        srv.submit(img, tag=5, hist=h)
        t0 = time.time()
        got = []
        while not got:
            got = srv.poll()
            assert time.time() - t0 < 30
    assert np.array_equal(h, oracle.extract(img, k=3, R=7, C=6)[0].reshape(-1))


def test_server_launch_failure_surfaces_as_ecuda(env):
    """A serving batch whose launch fails: later submit / poll calls return
    LDP_ECUDA with the CUDA error in the message; destroy still returns (it
    neither hangs on the failed batch nor leaks its arena ranges)."""
    torch, ldp, oracle, synth, _abi, serving = env
    imgs = [synth.image(20 + i, 64 + i, 80, 3.0) for i in range(6)]
    srv = serving.Server(streams=2, max_batch=4, arena_bytes=8 << 20)
    try:
        ldp.inject_fault(ldp.FAULT_SERVER_LAUNCH, 1)
        srv.submit(imgs[0], tag=0)
        t0 = time.time()
        with pytest.raises(ldp.LdpError) as ei:
            while True:
                srv.poll()
                assert time.time() - t0 < 30, "the launch failure never surfaced"
                time.sleep(0.001)
        assert ei.value.status == _abi.LDP_ECUDA and "injected" in str(ei.value)
        with pytest.raises(ldp.LdpError) as ei:
            srv.submit(imgs[1], tag=1)
        assert ei.value.status == _abi.LDP_ECUDA
        assert srv.stats()["arena_used"] == 0  # the failed batch gave its ranges back
    finally:
        t0 = time.time()
        srv.close()
        assert time.time() - t0 < 30
    # a new server is unaffected
    with serving.Server(streams=2, arena_bytes=8 << 20) as srv2:
        h = np.zeros(7 * 6 * 56, dtype=np.uint32)
        srv2.submit(imgs[2], tag=2, hist=h)
        t0 = time.time()
        while not srv2.poll():
            assert time.time() - t0 < 30
    assert np.array_equal(h, oracle.extract(imgs[2], k=3, R=7, C=6)[0].reshape(-1))


def test_fault_hook_arguments(env):
    torch, ldp, oracle, synth, _abi, serving = env
    for kind, count, after in ((7, 1, 0), (ldp.FAULT_DEVICE_ALLOC, -1, 0), (ldp.FAULT_SERVER_LAUNCH, 1, -2)):
        with pytest.raises(ldp.LdpError) as ei:
            ldp.inject_fault(kind, count, after=after)
        assert ei.value.status == _abi.LDP_EINVAL
    with pytest.raises(ldp.LdpError) as ei:  # the release build has no stage-wait hook
        ldp.inject_fault(ldp.FAULT_STAGE_WAIT, 1)
    assert ei.value.status == _abi.LDP_ENOTIMPL


# Checked build, in a child process: the staged variants' bounded mbarrier
# wait runs out on a stage that is never filled (no copy in flight), the call
# returns LDP_ETIMEOUT, the status word holds bit 2, and with the hook off the
# same launch is bit-exact again.  A batch whose descriptors exceed the plan's
# max_pixels is reported as LDP_EINVAL.
CHILD = r"""
import numpy as np, torch, sys
sys.path.insert(0, ROOT)
import oracle, synth
import paper_1810_11518_gb300 as ldp
from paper_1810_11518_gb300 import _abi
assert ldp.load()._name.endswith("libldp_checked.so")
ldp.device_status()
staged = [v for v in range(ldp.num_variants()) if ldp.variant_name(v).rstrip("s").endswith("t1")]
assert staged
img = synth.image(31, 40, 200, 3.0)
d = torch.from_numpy(img).cuda()
h_ref, c_ref = oracle.extract(img, k=3, R=7, C=6)
for v in staged:
    ldp.set_plain_variant(v)
    ldp.inject_fault(ldp.FAULT_STAGE_WAIT, 1)
    try:
        ldp.region_hist(d, k=3, regions=(7, 6))
        raise AssertionError("no timeout reported")
    except ldp.LdpError as e:
        assert e.status == _abi.LDP_ETIMEOUT, e
    st = ldp.device_status()
    assert st & 4 and not st & 16, st
    ldp.inject_fault(ldp.FAULT_STAGE_WAIT, 0)
    h, c = ldp.region_hist(d, k=3, regions=(7, 6))
    assert np.array_equal(c.cpu().numpy(), c_ref)
    assert np.array_equal(h.cpu().numpy().astype(np.uint32), h_ref)
    assert ldp.device_status() == 0
ldp.set_plain_variant(-1)
# descriptors beyond the plan's max_pixels
lay = ldp.BatchLayout.build([20000] * 4, [3] * 4, hist_len=7 * 6 * 56)
host = np.zeros(lay.img_bytes, dtype=np.uint8)
synth.batch_into(host, [1, 2, 3, 4], lay.Hs, lay.Ws, lay.pitches, lay.img_off)
d_img = torch.from_numpy(host).cuda()
d_codes = torch.zeros(lay.code_bytes, dtype=torch.uint8, device="cuda")
d_hist = torch.zeros(lay.n * lay.hist_len, dtype=torch.int32, device="cuda")
d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
v8 = next(v for v in range(ldp.num_variants()) if ldp.variant_name(v).startswith("r8w"))
with ldp.BatchPlan(lay.n, 180000, k=3) as plan:
    plan.set_config(v8, 0)
    try:
        plan.run(d_desc, d_count, d_hist)
        raise AssertionError("truncated batch not reported")
    except ldp.LdpError as e:
        assert e.status == _abi.LDP_EINVAL and "max_pixels" in str(e), e
assert ldp.device_status() & 2
print("failures ok")
"""


def test_checked_build_wait_timeout_and_truncation():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    from paper_1810_11518_gb300 import build as libbuild

    __graft_entry__.build()
    lib = libbuild.build(checked=True)
    env = dict(os.environ, LDP_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "failures ok" in r.stdout
