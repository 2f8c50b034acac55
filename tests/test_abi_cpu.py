"""The C-ABI library on a machine without a GPU: it builds, loads, exports
every function include/ldp.h declares, and rejects bad arguments on the host
before any CUDA call.  No compute call is made here."""
import ctypes
import os
import re
from math import comb

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_11518_gb300 import _abi
    from paper_1810_11518_gb300 import build as libbuild

    libbuild.build()
    return _abi.load()


def _declared():
    with open(os.path.join(ROOT, "include", "ldp.h")) as f:
        src = f.read()
    return re.findall(r"LDP_API\s+(?:int|uint64_t|const char \*)\s*(\w+)\(", src)


def test_exports_every_declared_symbol(lib):
    from paper_1810_11518_gb300 import _abi

    names = _declared()
    assert len(names) >= 17
    assert sorted(names) == sorted(_abi.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_variants_listed(lib):
    from paper_1810_11518_gb300 import build as libbuild

    nv = lib.ldp_num_variants()
    assert nv == len(libbuild.variants()) and nv >= 1
    for v in range(nv):
        name = lib.ldp_variant_name(v).decode()
        assert re.fullmatch(r"r\d+w\d+b\d+t[01][sf]?", name)
    assert lib.ldp_variant_name(nv) == b""
    assert lib.ldp_set_plain_variant(nv) == 1
    assert lib.ldp_set_plain_variant(-2) == 1
    assert lib.ldp_set_plain_variant(-1) == 0  # by image size (the default)


def test_host_helpers(lib):
    import oracle

    for k in range(0, 9):
        assert lib.ldp_hist_bins(k) == comb(8, k)
    assert lib.ldp_hist_bins(9) == -1
    for k in range(1, 8):
        for code in range(256):
            assert lib.ldp_bin_of_code(code, k) == oracle.bin_of_code(code, k)
    assert lib.ldp_version() >= 100


def test_argument_errors_without_gpu(lib):
    from paper_1810_11518_gb300 import _abi

    fake = ctypes.c_void_p(0x1000)
    rs = _abi.RegionSpec(7, 6, 1)
    EINVAL = _abi.LDP_EINVAL
    assert lib.ldp_codes(None, 10, 10, 10, 3, fake, 8, None) == EINVAL
    assert lib.ldp_codes(fake, 2, 10, 10, 3, fake, 8, None) == EINVAL
    assert lib.ldp_codes(fake, 10, 2, 10, 3, fake, 8, None) == EINVAL
    assert lib.ldp_codes(fake, 10, 10, 9, 3, fake, 8, None) == EINVAL
    assert lib.ldp_codes(fake, 10, 10, 10, 3, fake, 7, None) == EINVAL
    assert lib.ldp_codes(fake, 10, 10, 10, 0, fake, 8, None) == EINVAL
    assert lib.ldp_codes(fake, 10, 10, 10, 8, fake, 8, None) == EINVAL
    assert lib.ldp_codes(fake, 10, 10, 10, 3, None, 8, None) == EINVAL
    assert lib.ldp_codes(fake, (1 << 20) + 1, 10, 10, 3, fake, 8, None) == EINVAL
    assert b"pitch" in lib.ldp_last_error() or lib.ldp_last_error()
    assert lib.ldp_region_hist(fake, 10, 10, 10, 3, _abi.RegionSpec(0, 6, 1), fake, None, 0, None) == EINVAL
    assert lib.ldp_region_hist(fake, 10, 10, 10, 3, _abi.RegionSpec(7, 6, 2), fake, None, 0, None) == EINVAL
    assert lib.ldp_region_hist(fake, 10, 10, 10, 3, rs, None, None, 0, None) == EINVAL
    assert lib.lbp_codes(fake, 10, 10, 10, None, 8, None) == EINVAL
    assert lib.lbp_region_hist(fake, 10, 10, 10, 0, 1, fake, None, 0, None) == EINVAL
    h = ctypes.c_void_p()
    assert lib.ldp_batch_plan_create(None, 4, 1000, 3, rs, 0) == EINVAL
    assert lib.ldp_batch_plan_create(ctypes.byref(h), 0, 1000, 3, rs, 0) == EINVAL
    assert lib.ldp_batch_plan_create(ctypes.byref(h), 4, 1000, 9, rs, 0) == EINVAL
    assert lib.ldp_batch_run(None, fake, fake, fake, None) == EINVAL
    assert lib.ldp_batch_plan_destroy(None) == 0
    out = ctypes.c_int()
    assert lib.ldp_device_status(None, None) == EINVAL


def test_layout_alignment():
    import paper_1810_11518_gb300 as ldp

    lay = ldp.BatchLayout.build([3, 100, 490], [3, 77, 640], hist_len=2352)
    assert (lay.pitches % 16 == 0).all() and (lay.img_off % 16 == 0).all()
    assert (lay.code_pitches % 16 == 0).all() and (lay.code_off % 16 == 0).all()
    assert (lay.pitches >= lay.Ws).all() and (lay.code_pitches >= lay.Ws - 2).all()
    d = lay.descs(1 << 20, 1 << 30)
    assert d["hist_offset"].tolist() == [0, 2352, 4704]
    assert d.itemsize == 40


def test_window_host_logic_without_gpu(lib):
    import oracle
    from paper_1810_11518_gb300 import _abi

    EINVAL = _abi.LDP_EINVAL
    for n in range(0, 70, 3):
        for w in range(1, 30, 4):
            for s in range(1, 33, 5):
                assert lib.ldp_window_count(n, w, s) == oracle.window_count(n, w, s)
    assert lib.ldp_window_count(10, 0, 1) == -1 and lib.ldp_window_count(10, 3, 0) == -1
    ws = _abi.WindowSpec(20, 20, 10, 10, 1)
    code_map = ((488 * 638 + 255) // 256) * 256
    # overlapping windows whose column stride divides the width: one fused
    # pass with the cells in shared memory, scratch for the code map only
    assert lib.ldp_window_scratch_bytes(490, 640, 3, ws, 0) == code_map
    assert lib.ldp_window_scratch_bytes(490, 640, 3, ws, 1) == 0
    assert lib.ldp_batch_window_scratch_bytes(8, 490, 640, 0, _abi.WindowSpec(20, 20, 10, 10, 0)) == 0
    # a column stride that does not divide the width: cells of gcd(20, 15) = 5
    # pixels go through device scratch
    ws15 = _abi.WindowSpec(20, 20, 15, 15, 1)
    cells = 98 * 128 * 56 * 4
    assert lib.ldp_window_scratch_bytes(490, 640, 3, ws15, 0) == code_map + cells
    assert lib.ldp_window_scratch_bytes(490, 640, 3, ws15, 1) == cells
    assert lib.ldp_batch_window_scratch_bytes(8, 490, 640, 0, _abi.WindowSpec(20, 20, 15, 15, 0)) == \
        8 * 98 * 128 * 256 * 4
    # rows of cells too wide for shared memory (1-pixel cells, 256 bins): scratch again
    ws1 = _abi.WindowSpec(4, 4, 1, 1, 0)
    assert lib.ldp_window_scratch_bytes(490, 640, 0, ws1, 1) == 490 * 640 * 256 * 4
    # stride = size: the cells are the windows, no cell scratch
    assert lib.ldp_window_scratch_bytes(490, 640, 3, _abi.WindowSpec(20, 20, 20, 20, 1), 1) == 0
    assert lib.ldp_window_scratch_bytes(490, 640, 0, _abi.WindowSpec(20, 20, 20, 20, 1), 1) == 0  # bad spec
    fake = ctypes.c_void_p(0x1000)
    assert lib.ldp_window_hist(fake, 10, 10, 10, 3, _abi.WindowSpec(0, 4, 4, 4, 1), fake, None, 0, None, 0,
                               None) == EINVAL
    assert lib.ldp_window_hist(fake, 10, 10, 10, 3, _abi.WindowSpec(4, 4, 4, 4, 2), fake, None, 0, None, 0,
                               None) == EINVAL
    # the code map needs scratch when no code buffer is given
    assert lib.ldp_window_hist(fake, 10, 10, 10, 3, _abi.WindowSpec(4, 4, 4, 4, 1), fake, None, 0, None, 0,
                               None) == EINVAL
    assert lib.lbp_window_hist(fake, 10, 10, 10, _abi.WindowSpec(4, 4, 4, 4, 1), fake, fake, 8, None, 0,
                               None) == EINVAL
    assert lib.ldp_batch_window_hist(None, 1, 10, 10, 3, ws, fake, None, 0, None) == EINVAL
    assert lib.ldp_batch_window_hist(fake, 1, 10, 10, 3, ws15, fake, None, 0, None) == EINVAL  # no scratch


def test_code_mode_arguments_without_gpu(lib):
    from paper_1810_11518_gb300 import _abi

    EINVAL = _abi.LDP_EINVAL
    fake = ctypes.c_void_p(0x1000)
    assert lib.ldp_codes_ex(fake, 10, 10, 10, 3, 4, fake, 8, None) == EINVAL   # no such mode
    assert lib.ldp_codes_ex(fake, 10, 10, 10, 3, -1, fake, 8, None) == EINVAL
    assert lib.ldp_codes_ex(fake, 10, 10, 10, 0, 1, fake, 8, None) == EINVAL   # k
    # threshold modes count raw bins only
    for m in (_abi.LDP_CODE_ABS_THRESH, _abi.LDP_CODE_RAW_THRESH):
        assert lib.ldp_region_hist_ex(fake, 10, 10, 10, 3, m, _abi.RegionSpec(2, 2, 1), fake, None, 0,
                                      None) == EINVAL
        h = ctypes.c_void_p()
        assert lib.ldp_batch_plan_create(ctypes.byref(h), 4, 1000, 3, _abi.RegionSpec(2, 2, 1),
                                         _abi.plan_code_mode(m)) == EINVAL
    h = ctypes.c_void_p()
    assert lib.ldp_batch_plan_create(ctypes.byref(h), 4, 1000, 3, _abi.RegionSpec(2, 2, 0),
                                     _abi.LDP_PLAN_LBP | _abi.plan_code_mode(1)) == EINVAL


def test_resize_arguments_without_gpu(lib):
    import paper_1810_11518_gb300 as ldp
    from paper_1810_11518_gb300 import _abi

    EINVAL = _abi.LDP_EINVAL
    fake = ctypes.c_void_p(0x1000)
    assert ldp.CROP_DTYPE.itemsize == 48
    ok = (fake, 100, 120, 128, 10, 20, 50, 60, fake, 26, 26, 26, None)
    bad = [
        (None,) + ok[1:],
        ok[:4] + (-1,) + ok[5:],             # crop above the image
        ok[:4] + (60, 20, 50, 60) + ok[8:],  # crop past the bottom
        ok[:6] + (0,) + ok[7:],              # empty crop
        ok[:3] + (119,) + ok[4:],            # pitch < W
        ok[:9] + (0,) + ok[10:],             # OH
        ok[:11] + (25, None),                # dst_pitch < OW
    ]
    for args in bad:
        assert lib.ldp_resize(*args) == EINVAL, args
    assert lib.ldp_batch_resize(None, 1, 26, 26, None) == EINVAL
    assert lib.ldp_batch_resize(fake, 0, 26, 26, None) == EINVAL
    assert lib.ldp_batch_resize(fake, 1, 0, 26, None) == EINVAL


def test_distance_arguments_without_gpu(lib):
    from paper_1810_11518_gb300 import _abi

    EINVAL = _abi.LDP_EINVAL
    f = ctypes.c_void_p(0x1000)
    ok = [f, 4, 10, f, 5, 10, 10, _abi.LDP_DIST_CHI2, f, 5, None]
    for pos, val in ((0, None), (1, 0), (2, 9), (5, 9), (6, 0), (7, 3), (7, -1), (8, None), (9, 4)):
        args = list(ok)
        args[pos] = val
        assert lib.ldp_hist_distance(*args) == EINVAL, (pos, val)


def test_pipeline_arguments_without_gpu(lib):
    from paper_1810_11518_gb300 import _abi

    EINVAL = _abi.LDP_EINVAL
    h = ctypes.c_void_p()
    rs = _abi.RegionSpec(7, 6, 1)
    assert lib.ldp_pipeline_create(None, 16, 1 << 20, 3, rs, 3, 0) == EINVAL
    assert lib.ldp_pipeline_create(ctypes.byref(h), 0, 1 << 20, 3, rs, 3, 0) == EINVAL
    assert lib.ldp_pipeline_create(ctypes.byref(h), 16, 4, 3, rs, 3, 0) == EINVAL
    assert lib.ldp_pipeline_create(ctypes.byref(h), 16, 1 << 20, 3, rs, 0, 0) == EINVAL
    assert lib.ldp_pipeline_create(ctypes.byref(h), 16, 1 << 20, 3, rs, 9, 0) == EINVAL
    assert lib.ldp_pipeline_create(ctypes.byref(h), 16, 1 << 20, 3, rs, 3, _abi.LDP_PLAN_NO_GRAPH) == EINVAL
    f = ctypes.c_void_p(0x1000)
    assert lib.ldp_pipeline_run(None, 1, f, f, f, f, f, None, None, None, f, None) == EINVAL
    assert lib.ldp_pipeline_destroy(None) == 0


def test_autotune_cache_names_compiled_variants():
    """Every tuned entry shipped with the package names a variant of the
    compiled list, by index and by name, so a change of the variant list
    cannot silently re-point the cache."""
    import json
    import os

    from paper_1810_11518_gb300 import autotune
    from paper_1810_11518_gb300 import build as libbuild

    names = [f"r{rpw}w{nw}b{mb}t{st}" + {0: "", 1: "s", 2: "f"}[sp] for _, rpw, nw, mb, st, sp in libbuild.variants()]
    with open(autotune.DEFAULT_CACHE) as f:
        cache = json.load(f)
    assert cache
    for key, ent in cache.items():
        assert 0 <= ent["variant"] < len(names), key
        assert ent["name"] == names[ent["variant"]], key
        assert ent["ctas_per_sm"] >= 0
    assert os.path.basename(autotune.DEFAULT_CACHE) == "autotune_cache.json"


def test_fault_hook_without_gpu(lib):
    """The test-only fault hook checks its arguments on the host; the
    stage-wait fault exists only in the checked build."""
    from paper_1810_11518_gb300 import _abi

    assert lib.ldp_test_inject_fault(9, 0, 1, None) == _abi.LDP_EINVAL
    assert lib.ldp_test_inject_fault(_abi.LDP_FAULT_DEVICE_ALLOC, -1, 1, None) == _abi.LDP_EINVAL
    assert lib.ldp_test_inject_fault(_abi.LDP_FAULT_SERVER_LAUNCH, 0, -1, None) == _abi.LDP_EINVAL
    assert lib.ldp_test_inject_fault(_abi.LDP_FAULT_STAGE_WAIT, 0, 1, None) == _abi.LDP_ENOTIMPL
    assert lib.ldp_test_inject_fault(_abi.LDP_FAULT_STAGE_WAIT, 1, 1, None) == _abi.LDP_EINVAL
    for kind in (_abi.LDP_FAULT_DEVICE_ALLOC, _abi.LDP_FAULT_SERVER_LAUNCH):
        assert lib.ldp_test_inject_fault(kind, 2, 1, None) == 0
        assert lib.ldp_test_inject_fault(kind, 0, 0, None) == 0  # cleared again
