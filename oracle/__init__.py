"""CPU ORACLE for LDP / LBP extraction -- test infrastructure only.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It compiles and wraps the plain C
oracle in this directory (``oracle_ldp.c``: literal Kirsch masks, Eq. 1-6 of
Ayami & Shabat, arXiv:1810.11518; ``aldp.c``: the paper's Eqs. 7-29 scheme and
the ring-sum identity).  It shares no code with the CUDA library.

Every function here is pinned by ``tests/test_oracle_*.py`` against worked
examples, closed forms, invariants and independent formulations; none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("oracle_ldp.c", "aldp.c", "cpu_routes.c")]
_HDR = os.path.join(_HERE, "oracle_ldp.h")
_LIB = os.path.join(_HERE, "_oracle.so")
# the same sources built -O3 with link-time inlining across them, for the
# timed CPU baselines only (the sources are unchanged; no -march, so the
# build is the same on every host)
_LIB_TIMED = os.path.join(_HERE, "_oracle_o3.so")
_lock = threading.Lock()
_lib = None
_lib_timed = None

ROUTE_MASKS, ROUTE_ALDP, ROUTE_RINGSUM = 0, 1, 2
ROUTE_NAMES = {ROUTE_MASKS: "literal masks (Eq. 1)", ROUTE_ALDP: "paper's column sums (Eqs. 7-29)",
               ROUTE_RINGSUM: "ring sums (m_i = 8 S3_i - 3 S8)"}

MODE_LDP = 0
MODE_LBP = 1
MODE_LDP_RAW = 2         # rank by the signed response m_i, exactly k bits
MODE_LDP_THRESH = 3      # rank by |m_i|, every bit tied with the k-th set
MODE_LDP_RAW_THRESH = 4  # rank by m_i, every bit tied with the k-th set


def build(force: bool = False, timed: bool = False) -> str:
    """Compile the oracle into oracle/_oracle.so (plain C, -O2, no -march);
    timed=True: the same sources into oracle/_oracle_o3.so with -O3 -flto,
    the build the CPU baselines are timed on."""
    lib, flags = (_LIB_TIMED, ["-O3", "-flto"]) if timed else (_LIB, ["-O2"])
    newest = max(os.path.getmtime(p) for p in _SRCS + [_HDR])
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc"] + flags + ["-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp] + _SRCS)
        os.replace(tmp, lib)
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i32, i64p = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
            lib.oracle_kirsch_mask.argtypes = [i32, vp]
            lib.oracle_kirsch_mask.restype = None
            for fn in (lib.oracle_responses, lib.aldp_responses, lib.ringsum_responses):
                fn.argtypes = [vp, i32, i32, i32, i32, i32, vp]
                fn.restype = None
            lib.oracle_code_from_responses.argtypes = [vp, i32]
            lib.rank_code_from_responses.argtypes = [vp, i32]
            lib.oracle_code_variant.argtypes = [vp, i32, i32]
            lib.oracle_lbp_code.argtypes = [vp, i32, i32, i32, i32, i32]
            lib.oracle_codes_rect.argtypes = [vp, i32, i32, i32, i32, i32, i32, i32, i32, i32, vp, i32]
            lib.oracle_compact_codes.argtypes = [i32, vp]
            lib.oracle_bin_of_code.argtypes = [i32, i32]
            lib.oracle_band.argtypes = [i32, i32, i32, vp, vp]
            lib.oracle_band.restype = None
            lib.oracle_region_hist.argtypes = [vp, i32, i32, i32, i32, i32, i32, vp]
            lib.oracle_extract.argtypes = [vp, i32, i32, i32, i32, i32, i32, i32, i32, vp, vp, i32]
            lib.oracle_extract_batch.argtypes = [i32, vp, i64p, vp, vp, vp, i32, i32, i32, i32, i32,
                                                 vp, i64p, vp, i64p, vp, i32]
            lib.aldp_codes.argtypes = [vp, i32, i32, i32, i32, vp, i32]
            lib.oracle_window_count.argtypes = [i32, i32, i32]
            lib.oracle_resize_bilinear.argtypes = [vp, i32, i32, i32, i32, i32, i32, i32, vp, i32, i32, i32]
            lib.oracle_resize_coord.argtypes = [i32, i32, i32, vp, vp]
            lib.oracle_resize_coord.restype = None
            lib.oracle_hist_distance.argtypes = [vp, i32, i32, vp, i32, i32, i32, i32, vp, i32]
            lib.oracle_window_hist.argtypes = [vp, i32, i32, i32, i32, i32, i32, i32, i32, vp]
            lib.route_extract_batch.argtypes = [i32, i32, vp, vp, i32, i32, i32, i32, i32, i32, i32, vp, i32]
            lib.route_response_sum.argtypes = [i32, i32, vp, vp, i32, i32, i32]
            lib.route_response_sum.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _load_timed():
    global _lib_timed
    with _lock:
        if _lib_timed is None:
            lib = ctypes.CDLL(build(timed=True))
            lib.route_extract_batch.argtypes = [ctypes.c_int] * 2 + [ctypes.c_void_p] * 2 + [ctypes.c_int] * 7 + \
                                               [ctypes.c_void_p, ctypes.c_int]
            lib.route_response_sum.argtypes = [ctypes.c_int] * 2 + [ctypes.c_void_p] * 2 + [ctypes.c_int] * 3
            lib.route_response_sum.restype = ctypes.c_int64
            _lib_timed = lib
    return _lib_timed


def _u8(img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    if img.ndim != 2:
        raise ValueError("image must be 2-D")
    return img


def kirsch_mask(i: int) -> np.ndarray:
    out = np.zeros(9, dtype=np.int32)
    _load().oracle_kirsch_mask(i, out.ctypes.data)
    return out.reshape(3, 3)


def _resp(fn, img, x, y):
    img = _u8(img)
    m = np.zeros(8, dtype=np.int32)
    fn(img.ctypes.data, img.shape[0], img.shape[1], img.shape[1], x, y, m.ctypes.data)
    return m


def responses(img, x, y):
    """Eq. 1 at (row x, column y)."""
    return _resp(_load().oracle_responses, img, x, y)


def aldp_responses(img, x, y):
    """Eqs. 7-29 at (row x, column y)."""
    return _resp(_load().aldp_responses, img, x, y)


def ringsum_responses(img, x, y):
    return _resp(_load().ringsum_responses, img, x, y)


def code_from_responses(m, k: int = 3) -> int:
    m = np.ascontiguousarray(m, dtype=np.int32)
    return int(_load().oracle_code_from_responses(m.ctypes.data, k))


def code_variant(m, k: int = 3, variant: int = 0) -> int:
    """Eq. 2-3 readings: 0 |m| exact-k, 1 raw m exact-k, 2 |m| threshold, 3 raw m threshold."""
    m = np.ascontiguousarray(m, dtype=np.int32)
    return int(_load().oracle_code_variant(m.ctypes.data, k, variant))


def rank_code_from_responses(m, k: int = 3) -> int:
    m = np.ascontiguousarray(m, dtype=np.int32)
    return int(_load().rank_code_from_responses(m.ctypes.data, k))


def lbp_code(img, x, y) -> int:
    img = _u8(img)
    return int(_load().oracle_lbp_code(img.ctypes.data, img.shape[0], img.shape[1], img.shape[1], x, y))


def codes(img, k: int = 3, mode: int = MODE_LDP, W: int | None = None) -> np.ndarray:
    """Interior code map, shape (H-2, W-2). img may carry pitch padding: pass W."""
    img = _u8(img)
    H, P = img.shape
    W = P if W is None else W
    out = np.zeros((H - 2, W - 2), dtype=np.uint8)
    rc = _load().oracle_codes_rect(img.ctypes.data, H, W, P, mode, k, 1, H - 1, 1, W - 1,
                                   out.ctypes.data, W - 2)
    if rc:
        raise ValueError("oracle_codes_rect rejected the arguments")
    return out


def codes_rect(img, x0, x1, y0, y1, k: int = 3, mode: int = MODE_LDP, W: int | None = None) -> np.ndarray:
    """Codes of interior pixels rows [x0,x1), cols [y0,y1) (image coordinates)."""
    img = _u8(img)
    H, P = img.shape
    W = P if W is None else W
    out = np.zeros((x1 - x0, y1 - y0), dtype=np.uint8)
    rc = _load().oracle_codes_rect(img.ctypes.data, H, W, P, mode, k, x0, x1, y0, y1,
                                   out.ctypes.data, max(1, y1 - y0))
    if rc:
        raise ValueError("oracle_codes_rect rejected the arguments")
    return out


def aldp_codes(img, k: int = 3, W: int | None = None) -> np.ndarray:
    img = _u8(img)
    H, P = img.shape
    W = P if W is None else W
    out = np.zeros((H - 2, W - 2), dtype=np.uint8)
    if _load().aldp_codes(img.ctypes.data, H, W, P, k, out.ctypes.data, W - 2):
        raise ValueError("aldp_codes rejected the arguments")
    return out


def compact_codes(k: int) -> list[int]:
    n = _load().oracle_compact_codes(k, None)
    buf = np.zeros(max(n, 1), dtype=np.int32)
    _load().oracle_compact_codes(k, buf.ctypes.data)
    return [int(v) for v in buf[:n]]


def bin_of_code(code: int, k: int) -> int:
    return int(_load().oracle_bin_of_code(code, k))


def band(n: int, nb: int, b: int) -> tuple[int, int]:
    lo, hi = ctypes.c_int(), ctypes.c_int()
    _load().oracle_band(n, nb, b, ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def nbins(mode: int, k: int, compact: bool) -> int:
    return len(compact_codes(k)) if (mode in (MODE_LDP, MODE_LDP_RAW) and compact) else 256


def region_hist(code_map, H, W, R, C, nbins_k) -> np.ndarray:
    """Histograms from a full interior code map of shape (H-2, W-2)."""
    code_map = np.ascontiguousarray(code_map, dtype=np.uint8)
    nb = len(compact_codes(nbins_k)) if nbins_k else 256
    out = np.zeros((R, C, nb), dtype=np.uint32)
    rc = _load().oracle_region_hist(code_map.ctypes.data, H, W, code_map.shape[1], R, C, nbins_k,
                                    out.ctypes.data)
    if rc:
        raise ValueError("oracle_region_hist rejected the arguments")
    return out


def window_count(n: int, w: int, s: int) -> int:
    """Windows of size w at stride s along an axis of n pixels (Sec. 3.2)."""
    c = _load().oracle_window_count(n, w, s)
    if c < 0:
        raise ValueError("window size and stride must be positive")
    return c


def window_hist(code_map, H, W, wh, ww, sh, sw, nbins_k) -> np.ndarray:
    """Sliding-window histograms from a full interior code map of shape (H-2, W-2):
    shape (window rows, window columns, nbins)."""
    code_map = np.ascontiguousarray(code_map, dtype=np.uint8)
    nb = len(compact_codes(nbins_k)) if nbins_k else 256
    out = np.zeros((window_count(H, wh, sh), window_count(W, ww, sw), nb), dtype=np.uint32)
    rc = _load().oracle_window_hist(code_map.ctypes.data, H, W, code_map.shape[1], wh, ww, sh, sw, nbins_k,
                                    out.ctypes.data)
    if rc:
        raise ValueError("oracle_window_hist rejected the arguments")
    return out


def extract_windows(img, k: int = 3, window=(20, 20), stride=None, compact: bool = True,
                    mode: int = MODE_LDP):
    """(window histograms, codes) for one image; stride defaults to the window size."""
    img = _u8(img)
    H, W = img.shape
    stride = tuple(window) if stride is None else tuple(stride)
    cm = codes(img, k=k, mode=mode)
    nbk = k if (mode in (MODE_LDP, MODE_LDP_RAW) and compact) else 0
    return window_hist(cm, H, W, window[0], window[1], stride[0], stride[1], nbk), cm


DIST_L1, DIST_INTERSECT, DIST_CHI2 = 0, 1, 2


def hist_distance(q, g, metric: int = DIST_CHI2) -> np.ndarray:
    """(nq, ng) distances between descriptor rows: uint64 for L1 / intersection, float64 for chi-square."""
    q = np.ascontiguousarray(q, dtype=np.uint32).reshape(len(q), -1)
    g = np.ascontiguousarray(g, dtype=np.uint32).reshape(len(g), -1)
    if q.shape[1] != g.shape[1]:
        raise ValueError("descriptor lengths differ")
    out = np.zeros((q.shape[0], g.shape[0]), dtype=np.float64 if metric == DIST_CHI2 else np.uint64)
    rc = _load().oracle_hist_distance(q.ctypes.data, q.shape[0], q.shape[1], g.ctypes.data, g.shape[0],
                                      g.shape[1], q.shape[1], metric, out.ctypes.data, g.shape[0])
    if rc:
        raise ValueError("oracle_hist_distance rejected the arguments")
    return out


def resize_coord(i: int, n_src: int, n_dst: int) -> tuple[int, int]:
    a, b = ctypes.c_int(), ctypes.c_int()
    _load().oracle_resize_coord(i, n_src, n_dst, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def resize(img, out_hw=(260, 260), crop=None) -> np.ndarray:
    """Bilinear crop-and-resize (Sec. 3.1 front end); crop = (y, x, h, w), default the whole image."""
    img = _u8(img)
    H, W = img.shape
    cy, cx, ch, cw = (0, 0, H, W) if crop is None else crop
    OH, OW = out_hw
    out = np.zeros((OH, OW), dtype=np.uint8)
    rc = _load().oracle_resize_bilinear(img.ctypes.data, H, W, W, cy, cx, ch, cw, out.ctypes.data, OH, OW, OW)
    if rc:
        raise ValueError("oracle_resize_bilinear rejected the arguments")
    return out


def extract(img, k: int = 3, R: int = 1, C: int = 1, compact: bool = True, mode: int = MODE_LDP,
            W: int | None = None, want_codes: bool = True):
    """(hist of shape (R, C, nbins), codes (H-2, W-2) or None) for one image."""
    img = _u8(img)
    H, P = img.shape
    W = P if W is None else W
    nb = nbins(mode, k, compact)
    hist = np.zeros((R, C, nb), dtype=np.uint32)
    cm = np.zeros((H - 2, W - 2), dtype=np.uint8) if want_codes else None
    rc = _load().oracle_extract(img.ctypes.data, H, W, P, mode, k, R, C, int(compact), hist.ctypes.data,
                                cm.ctypes.data if want_codes else None, W - 2)
    if rc:
        raise ValueError("oracle_extract rejected the arguments")
    return hist, cm


def extract_batch(buf: np.ndarray, img_off, Hs, Ws, pitches, k: int = 3, R: int = 7, C: int = 6,
                  compact: bool = True, mode: int = MODE_LDP, threads: int | None = None,
                  want_codes: bool = False):
    """Many images from one flat uint8 buffer.  Returns (hists (n, R, C, nb), list of code maps or None)."""
    n = len(img_off)
    img_off = np.ascontiguousarray(img_off, dtype=np.int64)
    Hs = np.ascontiguousarray(Hs, dtype=np.int32)
    Ws = np.ascontiguousarray(Ws, dtype=np.int32)
    pitches = np.ascontiguousarray(pitches, dtype=np.int32)
    nb = nbins(mode, k, compact)
    hist = np.zeros((n, R, C, nb), dtype=np.uint32)
    hist_off = np.arange(n, dtype=np.int64) * (R * C * nb)
    code_buf = code_off = cps = None
    if want_codes:
        sizes = (Hs.astype(np.int64) - 2) * (Ws.astype(np.int64) - 2)
        code_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        code_buf = np.zeros(int(sizes.sum()), dtype=np.uint8)
        cps = np.ascontiguousarray(Ws - 2, dtype=np.int32)
    rc = _load().oracle_extract_batch(
        n, buf.ctypes.data, img_off.ctypes.data, Hs.ctypes.data, Ws.ctypes.data, pitches.ctypes.data,
        mode, k, R, C, int(compact), hist.ctypes.data, hist_off.ctypes.data,
        code_buf.ctypes.data if want_codes else None, code_off.ctypes.data if want_codes else None,
        cps.ctypes.data if want_codes else None, threads or max(1, os.cpu_count() or 1))
    if rc:
        raise ValueError("oracle_extract_batch failed")
    maps = None
    if want_codes:
        maps = [code_buf[code_off[i]:code_off[i] + (Hs[i] - 2) * (Ws[i] - 2)].reshape(Hs[i] - 2, Ws[i] - 2)
                for i in range(n)]
    return hist, maps


def route_extract_batch(route: int, buf: np.ndarray, img_off, H: int, W: int, pitch: int, k: int = 3, R: int = 7,
                        C: int = 6, compact: bool = True, threads: int = 1, timed: bool = False) -> np.ndarray:
    """Region histograms (n, R, C, bins) of n H x W images of one flat buffer
    along one response route (ROUTE_MASKS / ROUTE_ALDP / ROUTE_RINGSUM), all
    ending in the oracle's code step and histograms.  timed=True runs the -O3
    build the CPU baselines are timed on."""
    n = len(img_off)
    img_off = np.ascontiguousarray(img_off, dtype=np.int64)
    hist = np.zeros((n, R, C, nbins(MODE_LDP, k, compact)), dtype=np.uint32)
    lib = _load_timed() if timed else _load()
    rc = lib.route_extract_batch(int(route), n, buf.ctypes.data, img_off.ctypes.data, H, W, pitch, k, R, C,
                                 int(compact), hist.ctypes.data, int(threads))
    if rc:
        raise ValueError("route_extract_batch rejected the arguments")
    return hist


def route_response_sum(route: int, buf: np.ndarray, img_off, H: int, W: int, pitch: int,
                       timed: bool = False) -> int:
    """Sum of |m_i| over every interior pixel and direction of n images, with
    the responses of one route only (no code step), single-threaded."""
    img_off = np.ascontiguousarray(img_off, dtype=np.int64)
    lib = _load_timed() if timed else _load()
    return int(lib.route_response_sum(int(route), len(img_off), buf.ctypes.data, img_off.ctypes.data, H, W, pitch))
