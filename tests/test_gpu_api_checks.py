"""The Python face checks every caller buffer before its address reaches a
kernel: host tensors where device memory is expected (and the reverse),
wrong dtypes and short buffers raise instead of launching."""
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

    return torch, ldp


def test_device_buffers_are_checked(env):
    torch, ldp = env
    d = torch.randint(0, 256, (40, 50), dtype=torch.uint8, device="cuda")
    with pytest.raises(TypeError):
        ldp.region_hist(d, k=3, regions=(2, 2), hist=torch.zeros((2, 2, 56), dtype=torch.int32))
    with pytest.raises(TypeError):
        ldp.region_hist(d, k=3, regions=(2, 2), hist=torch.zeros((2, 2, 56), dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        ldp.region_hist(d, k=3, regions=(2, 2), hist=torch.zeros((2, 2, 55), dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        ldp.lbp_region_hist(d, regions=(2, 2), hist=torch.zeros((2, 2, 255), dtype=torch.int32, device="cuda"))
    with pytest.raises(TypeError):
        ldp.window_hist(d, k=3, window=(10, 10), hist=torch.zeros(4 * 5 * 56, dtype=torch.int32))
    with pytest.raises(ValueError):
        ldp.resize(d, (20, 20), out=torch.zeros((20, 20), dtype=torch.uint8))
    q = torch.zeros((3, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        ldp.hist_distance(q, q, ldp.DIST_L1, out=torch.zeros((3, 3), dtype=torch.int64))
    with pytest.raises(TypeError):
        ldp.batch_resize(torch.zeros(48, dtype=torch.uint8), 1)
    with pytest.raises(ValueError):
        ldp.batch_resize(torch.zeros(40, dtype=torch.uint8, device="cuda"), 1)
    descs = torch.zeros(40, dtype=torch.uint8, device="cuda")
    with pytest.raises(TypeError):
        ldp.batch_window_hist(descs, 1, (40, 50), 3, (10, 10), hist=None)
    with pytest.raises(ValueError):
        ldp.batch_window_hist(descs, 2, (40, 50), 3, (10, 10), hist=torch.zeros(8, dtype=torch.int32, device="cuda"))
    count = torch.ones(1, dtype=torch.int32, device="cuda")
    with ldp.BatchPlan(1, 40 * 50, k=3, regions=(1, 1)) as plan:
        with pytest.raises(TypeError):
            plan.run(torch.zeros(40, dtype=torch.uint8), count, None)
        with pytest.raises(TypeError):
            plan.run(descs, torch.ones(1, dtype=torch.int64, device="cuda"), None)
        with pytest.raises(TypeError):
            plan.run(descs, count, torch.zeros(56, dtype=torch.int32))
    assert ldp.device_status() == 0


def test_host_buffers_are_checked(env):
    torch, ldp = env
    lay = ldp.BatchLayout.build([30, 40], [50, 60], hist_len=56)
    with ldp.Pipeline(2, 40 * 60, k=3, regions=(1, 1)) as pipe:
        h_img = torch.zeros(lay.img_bytes, dtype=torch.uint8, pin_memory=True)
        h_hist = torch.zeros(2 * pipe.hist_len, dtype=torch.int32, pin_memory=True)
        with pytest.raises(TypeError):
            pipe.run(h_img.cuda(), lay, h_hist)
        with pytest.raises(ValueError):
            pipe.run(h_img[:-1], lay, h_hist)
        with pytest.raises(ValueError):
            pipe.run(h_img, lay, h_hist[:-1])
        with pytest.raises(ValueError):
            pipe.run(h_img, lay, h_hist, torch.zeros(lay.code_bytes - 1, dtype=torch.uint8))
        pipe.run(h_img, lay, h_hist)  # the checked call itself goes through
        torch.cuda.synchronize()
    assert (h_hist.numpy().reshape(2, -1).sum(axis=1) == np.array([28 * 48, 38 * 58])).all()
