"""LDP / LBP feature extraction on GB300 (sm_103a).

Python face of libldp (include/ldp.h).  PyTorch provides device memory and
streams; every pixel is processed by the library's CUDA kernels.  Images are
``torch.uint8`` CUDA tensors of shape (H, W) whose rows may be padded
(``stride(0)`` is the pitch, ``stride(1)`` must be 1).

Method: Ayami & Shabat, arXiv:1810.11518 -- Kirsch responses (Eq. 1), the
LDP code of the k largest |m_i| (Eq. 2-3, ties to the lower index), region
histograms (Eq. 4-6, Sec. 3.2) and LBP (Sec. 2.1).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from math import comb

import numpy as np

from . import _abi
from ._abi import LdpError, RegionSpec, WindowSpec

__all__ = ["codes", "region_hist", "lbp_codes", "lbp_region_hist", "hist_bins", "bin_of_code",
           "BatchPlan", "BatchLayout", "DESC_DTYPE", "LdpError", "device_status", "num_variants",
           "variant_name", "set_plain_variant", "load", "batch_run_noalloc", "window_count", "window_hist",
           "lbp_window_hist", "batch_window_hist", "resize", "batch_resize", "CROP_DTYPE", "hist_distance", "Pipeline", "DIST_L1",
           "DIST_INTERSECT", "DIST_CHI2", "CODE_ABS", "CODE_RAW", "CODE_ABS_THRESH", "CODE_RAW_THRESH"]

DESC_DTYPE = np.dtype([("img", "<u8"), ("H", "<i4"), ("W", "<i4"), ("pitch", "<i4"),
                       ("code_pitch", "<i4"), ("codes", "<u8"), ("hist_offset", "<u8")])
assert DESC_DTYPE.itemsize == 40

# ldp_crop_desc: one crop of a batch resize (include/ldp.h)
CROP_DTYPE = np.dtype([("src", "<u8"), ("dst", "<u8"), ("H", "<i4"), ("W", "<i4"), ("pitch", "<i4"),
                       ("cy", "<i4"), ("cx", "<i4"), ("ch", "<i4"), ("cw", "<i4"), ("dst_pitch", "<i4")])
assert CROP_DTYPE.itemsize == 48


def load():
    """Loads libldp.so; raises if it is missing."""
    return _abi.load()


def _torch():
    import torch

    return torch


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _img(img):
    torch = _torch()
    if not isinstance(img, torch.Tensor) or img.dtype != torch.uint8 or not img.is_cuda:
        raise TypeError("image must be a torch.uint8 CUDA tensor")
    if img.dim() != 2 or img.stride(1) != 1:
        raise ValueError("image must be 2-D with unit column stride")
    H, W = img.shape
    return ctypes.c_void_p(img.data_ptr()), int(H), int(W), int(img.stride(0))


def _cuda(t, name, dtype=None, min_numel=None, contiguous=False):
    """A caller's device buffer, checked before its address reaches a kernel."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be a {dtype} tensor")
    if contiguous and not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name} holds {t.numel()} elements, at least {min_numel} are needed")
    return t


def _host(t, name, dtype, min_numel):
    """A caller's host buffer (pinned for overlapped copies), checked likewise."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} host tensor")
    if t.numel() < min_numel:
        raise ValueError(f"{name} holds {t.numel()} elements, at least {min_numel} are needed")
    return t


def _alloc_codes(img, H, W, out):
    torch = _torch()
    if out is not None:
        if out.dtype != torch.uint8 or not out.is_cuda or out.dim() != 2 or out.stride(1) != 1:
            raise ValueError("out must be a 2-D uint8 CUDA tensor")
        if tuple(out.shape) != (H - 2, W - 2):
            raise ValueError(f"out must have shape {(H - 2, W - 2)}")
        return out, int(out.stride(0))
    pc = (W - 2 + 15) // 16 * 16
    buf = torch.empty((H - 2, pc), dtype=torch.uint8, device=img.device)
    return buf[:, :W - 2], pc


def hist_bins(k: int) -> int:
    return int(_abi.load().ldp_hist_bins(k))


def bin_of_code(code: int, k: int) -> int:
    return int(_abi.load().ldp_bin_of_code(code, k))


CODE_ABS, CODE_RAW, CODE_ABS_THRESH, CODE_RAW_THRESH = (_abi.LDP_CODE_ABS, _abi.LDP_CODE_RAW,
                                                       _abi.LDP_CODE_ABS_THRESH, _abi.LDP_CODE_RAW_THRESH)


def codes(img, k: int = 3, out=None, stream=None, code_mode: int = CODE_ABS):
    """LDP codes (Eq. 1-3) of the interior: uint8 tensor (H-2, W-2).

    code_mode picks the reading of Eq. 2-3 (CODE_ABS: the k largest |m_i|,
    the default; CODE_RAW: the k largest m_i; *_THRESH: every response tied
    with the k-th is set as well)."""
    p, H, W, P = _img(img)
    out, pc = _alloc_codes(img, H, W, out)
    if code_mode == CODE_ABS:
        _abi.call("ldp_codes", p, H, W, P, k, ctypes.c_void_p(out.data_ptr()), pc, _stream(stream))
    else:
        _abi.call("ldp_codes_ex", p, H, W, P, k, int(code_mode), ctypes.c_void_p(out.data_ptr()), pc,
                  _stream(stream))
    return out


def region_hist(img, k: int = 3, regions=(1, 1), compact: bool = True, with_codes: bool = True,
                hist=None, codes_out=None, stream=None, code_mode: int = CODE_ABS):
    """Fused LDP codes + R x C region histograms (Eq. 1-6); code_mode as in codes()
    (the threshold modes need compact=False).

    Returns (hist int32 tensor (R, C, nbins) holding uint32 counts, codes or None)."""
    torch = _torch()
    p, H, W, P = _img(img)
    R, C = regions
    nb = comb(8, k) if compact else 256
    if hist is None:
        hist = torch.empty((R, C, nb), dtype=torch.int32, device=img.device)
    else:
        _cuda(hist, "hist", torch.int32, R * C * nb, contiguous=True)
    cptr, pc, out = None, 0, None
    if with_codes:
        out, pc = _alloc_codes(img, H, W, codes_out)
        cptr = ctypes.c_void_p(out.data_ptr())
    if code_mode == CODE_ABS:
        _abi.call("ldp_region_hist", p, H, W, P, k, RegionSpec(R, C, int(compact)),
                  ctypes.c_void_p(hist.data_ptr()), cptr, pc, _stream(stream))
    else:
        _abi.call("ldp_region_hist_ex", p, H, W, P, k, int(code_mode), RegionSpec(R, C, int(compact)),
                  ctypes.c_void_p(hist.data_ptr()), cptr, pc, _stream(stream))
    return hist, out


def lbp_codes(img, out=None, stream=None):
    """LBP codes (Sec. 2.1) of the interior: uint8 tensor (H-2, W-2)."""
    p, H, W, P = _img(img)
    out, pc = _alloc_codes(img, H, W, out)
    _abi.call("lbp_codes", p, H, W, P, ctypes.c_void_p(out.data_ptr()), pc, _stream(stream))
    return out


def lbp_region_hist(img, regions=(1, 1), with_codes: bool = True, hist=None, codes_out=None, stream=None):
    """Fused LBP codes + R x C region histograms of 256 bins."""
    torch = _torch()
    p, H, W, P = _img(img)
    R, C = regions
    if hist is None:
        hist = torch.empty((R, C, 256), dtype=torch.int32, device=img.device)
    else:
        _cuda(hist, "hist", torch.int32, R * C * 256, contiguous=True)
    cptr, pc, out = None, 0, None
    if with_codes:
        out, pc = _alloc_codes(img, H, W, codes_out)
        cptr = ctypes.c_void_p(out.data_ptr())
    _abi.call("lbp_region_hist", p, H, W, P, R, C, ctypes.c_void_p(hist.data_ptr()), cptr, pc, _stream(stream))
    return hist, out


def window_count(n: int, w: int, s: int) -> int:
    """Sliding windows of size w at stride s along an axis of n pixels (Sec. 3.2)."""
    c = int(_abi.load().ldp_window_count(n, w, s))
    if c < 0:
        raise ValueError("window size and stride must be positive")
    return c


def _window_run(fn, img, k, window, stride, compact, with_codes, hist, codes_out, stream):
    torch = _torch()
    p, H, W, P = _img(img)
    wh, ww = window
    sh, sw = (wh, ww) if stride is None else stride
    ws = WindowSpec(wh, ww, sh, sw, int(compact))
    nb = comb(8, k) if compact else 256
    shape = (window_count(H, wh, sh), window_count(W, ww, sw), nb)
    if hist is None:
        hist = torch.empty(shape, dtype=torch.int32, device=img.device)
    else:
        _cuda(hist, "hist", torch.int32, shape[0] * shape[1] * nb, contiguous=True)
    cptr, pc, out = None, 0, None
    if with_codes:
        out, pc = _alloc_codes(img, H, W, codes_out)
        cptr = ctypes.c_void_p(out.data_ptr())
    need = int(_abi.load().ldp_window_scratch_bytes(H, W, k if fn == "ldp_window_hist" else 0, ws,
                                                    int(with_codes)))
    scratch = torch.empty(max(need, 1), dtype=torch.uint8, device=img.device) if need else None
    sptr = ctypes.c_void_p(scratch.data_ptr()) if scratch is not None else None
    args = [p, H, W, P] + ([k] if fn == "ldp_window_hist" else []) + [
        ws, ctypes.c_void_p(hist.data_ptr()), cptr, pc, sptr, need, _stream(stream)]
    _abi.call(fn, *args)
    if scratch is not None:  # keep the scratch alive until the kernels have read it
        scratch.record_stream(torch.cuda.current_stream() if stream is None else stream)
    return hist, out


def window_hist(img, k: int = 3, window=(20, 20), stride=None, compact: bool = True, with_codes: bool = True,
                hist=None, codes_out=None, stream=None):
    """LDP codes + sliding-window histograms (Sec. 3.2): windows of window = (wh, ww)
    pixels whose origins step by stride (default: the window size).

    Returns (hist int32 tensor (window rows, window cols, nbins) of uint32 counts, codes or None)."""
    return _window_run("ldp_window_hist", img, k, window, stride, compact, with_codes, hist, codes_out, stream)


def lbp_window_hist(img, window=(20, 20), stride=None, with_codes: bool = True, hist=None, codes_out=None,
                    stream=None):
    """LBP codes + 256-bin sliding-window histograms."""
    return _window_run("lbp_window_hist", img, 0, window, stride, False, with_codes, hist, codes_out, stream)


def batch_window_hist(d_descs, count: int, max_hw, k: int, window, stride=None, compact: bool = True,
                      hist=None, stream=None):
    """Window histograms of `count` code maps already in device memory (descriptors
    `d_descs`, a CUDA tensor of DESC_DTYPE records; windows of image i at
    hist + hist_offset, hist a CUDA int32 tensor covering every offset).
    k = 0: raw 256 bins (LBP maps)."""
    torch = _torch()
    _cuda(d_descs, "d_descs", min_numel=count * DESC_DTYPE.itemsize // d_descs.element_size())
    _cuda(hist, "hist", torch.int32)
    wh, ww = window
    sh, sw = (wh, ww) if stride is None else stride
    ws = WindowSpec(wh, ww, sh, sw, int(compact))
    need = int(_abi.load().ldp_batch_window_scratch_bytes(count, max_hw[0], max_hw[1], k, ws))
    scratch = torch.empty(need, dtype=torch.uint8, device=hist.device) if need else None
    _abi.call("ldp_batch_window_hist", ctypes.c_void_p(d_descs.data_ptr()), count, max_hw[0], max_hw[1], k, ws,
              ctypes.c_void_p(hist.data_ptr()), ctypes.c_void_p(scratch.data_ptr()) if scratch is not None else None,
              need, _stream(stream))
    if scratch is not None:
        scratch.record_stream(torch.cuda.current_stream() if stream is None else stream)
    return hist


def resize(img, out_hw=(260, 260), crop=None, out=None, stream=None):
    """Bilinear crop-and-resize (Sec. 3.1 front end: faces resized to 260 x 260).
    crop = (y, x, h, w) of the source (default: all of it).  Returns uint8 (OH, OW)."""
    torch = _torch()
    p, H, W, P = _img(img)
    cy, cx, ch, cw = (0, 0, H, W) if crop is None else crop
    OH, OW = out_hw
    if out is None:
        out = torch.empty((OH, OW), dtype=torch.uint8, device=img.device)
    elif (not out.is_cuda or out.dtype != torch.uint8 or out.dim() != 2 or tuple(out.shape) != (OH, OW)
          or out.stride(1) != 1):
        raise ValueError(f"out must be a uint8 CUDA tensor of shape {(OH, OW)} with unit column stride")
    _abi.call("ldp_resize", p, H, W, P, cy, cx, ch, cw, ctypes.c_void_p(out.data_ptr()), OH, OW,
              int(out.stride(0)), _stream(stream))
    return out


def batch_resize(d_descs, count: int, out_hw=(260, 260), stream=None) -> None:
    """Every crop of `d_descs` (a CUDA tensor of CROP_DTYPE records) resized to out_hw in one launch;
    rejected descriptors are skipped and reported by device_status() (bit 3)."""
    _cuda(d_descs, "d_descs", min_numel=count * CROP_DTYPE.itemsize // d_descs.element_size())
    _abi.call("ldp_batch_resize", ctypes.c_void_p(d_descs.data_ptr()), int(count), int(out_hw[0]),
              int(out_hw[1]), _stream(stream))


DIST_L1, DIST_INTERSECT, DIST_CHI2 = _abi.LDP_DIST_L1, _abi.LDP_DIST_INTERSECT, _abi.LDP_DIST_CHI2


def hist_distance(q, g, metric: int = DIST_CHI2, out=None, stream=None):
    """Distances between descriptor rows (e.g. flattened region / window
    histograms): q (nq, D) and g (ng, D) CUDA int32 tensors holding uint32
    counts, unit column stride.  Returns (nq, ng): int64 for L1 /
    intersection, float32 for chi-square."""
    torch = _torch()
    for t in (q, g):
        if not t.is_cuda or t.dim() != 2 or t.stride(1) != 1 or t.dtype not in (torch.int32,):
            raise ValueError("descriptors must be 2-D int32 CUDA tensors with unit column stride")
    if q.shape[1] != g.shape[1]:
        raise ValueError("descriptor lengths differ")
    nq, D = q.shape
    ng = g.shape[0]
    dt = torch.float32 if metric == DIST_CHI2 else torch.int64
    if out is None:
        out = torch.empty((nq, ng), dtype=dt, device=q.device)
    elif not out.is_cuda or out.dtype != dt or tuple(out.shape) != (nq, ng) or out.stride(1) != 1:
        raise ValueError(f"out must be a {dt} CUDA tensor of shape {(nq, ng)} with unit column stride")
    _abi.call("ldp_hist_distance", ctypes.c_void_p(q.data_ptr()), nq, int(q.stride(0)),
              ctypes.c_void_p(g.data_ptr()), ng, int(g.stride(0)), D, int(metric),
              ctypes.c_void_p(out.data_ptr()), int(out.stride(0)), _stream(stream))
    return out


class Pipeline:
    """Extraction of images in (pinned) host memory with copies and compute
    overlapped: chunks of consecutive images rotate over nbuf device buffers,
    each with its own stream and batch plan (ldp_pipeline_* in include/ldp.h)."""

    def __init__(self, chunk_images: int, chunk_pixels: int, k: int = 3, regions=(7, 6), compact: bool = True,
                 lbp: bool = False, nbuf: int = 3, code_mode: int = CODE_ABS):
        self.k = k
        self.regions = tuple(regions)
        exact = not lbp and code_mode in (CODE_ABS, CODE_RAW)
        self.nbins = comb(8, k) if (compact and exact) else 256
        flags = (_abi.LDP_PLAN_LBP if lbp else 0) | _abi.plan_code_mode(code_mode)
        h = ctypes.c_void_p()
        _abi.call("ldp_pipeline_create", ctypes.byref(h), int(chunk_images), int(chunk_pixels), int(k),
                  RegionSpec(self.regions[0], self.regions[1], int(compact and not lbp)), int(nbuf), flags)
        self._h = h

    @property
    def hist_len(self) -> int:
        return self.regions[0] * self.regions[1] * self.nbins

    def set_config(self, variant: int, ctas_per_sm: int = 0) -> None:
        _abi.call("ldp_pipeline_set_config", self._h, int(variant), int(ctas_per_sm))

    def run(self, h_img, layout: "BatchLayout", h_hist, h_codes=None, stream=None) -> None:
        """Queues the extraction of every image of `layout` held in the host
        buffer h_img (uint8) into h_hist (int32, n x hist_len) and, when given,
        h_codes (uint8, layout.code_bytes).  Results are in place once
        `stream` (default: the current stream) has been synchronised."""
        arrs = [np.ascontiguousarray(layout.img_off, dtype=np.int64),
                np.ascontiguousarray(layout.Hs, dtype=np.int32), np.ascontiguousarray(layout.Ws, dtype=np.int32),
                np.ascontiguousarray(layout.pitches, dtype=np.int32),
                np.ascontiguousarray(layout.code_off, dtype=np.int64),
                np.ascontiguousarray(layout.code_pitches, dtype=np.int32)]
        torch = _torch()
        _host(h_img, "h_img", torch.uint8, layout.img_bytes)
        _host(h_hist, "h_hist", torch.int32, layout.n * self.hist_len)
        if h_codes is not None:
            _host(h_codes, "h_codes", torch.uint8, layout.code_bytes)
        cptr = ctypes.c_void_p(h_codes.data_ptr()) if h_codes is not None else None
        _abi.call("ldp_pipeline_run", self._h, layout.n, ctypes.c_void_p(h_img.data_ptr()),
                  *[ctypes.c_void_p(a.ctypes.data) for a in arrs[:4]], cptr,
                  *[ctypes.c_void_p(a.ctypes.data) for a in arrs[4:]], ctypes.c_void_p(h_hist.data_ptr()),
                  _stream(stream))

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _abi.call("ldp_pipeline_destroy", self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def num_variants() -> int:
    return int(_abi.load().ldp_num_variants())


def variant_name(v: int) -> str:
    return _abi.load().ldp_variant_name(v).decode()


def set_plain_variant(v: int) -> None:
    _abi.call("ldp_set_plain_variant", v)


def device_status(stream=None) -> int:
    out = ctypes.c_int(0)
    _abi.call("ldp_device_status", _stream(stream), ctypes.byref(out))
    return out.value


FAULT_DEVICE_ALLOC = _abi.LDP_FAULT_DEVICE_ALLOC
FAULT_SERVER_LAUNCH = _abi.LDP_FAULT_SERVER_LAUNCH
FAULT_STAGE_WAIT = _abi.LDP_FAULT_STAGE_WAIT


def inject_fault(kind: int, count: int, after: int = 0, stream=None) -> None:
    """Test hook: after `after` more library operations of `kind` succeed,
    makes the next `count` fail on the host the way a real failure would
    (device allocations, serving batch launches) or, in the checked build,
    makes the staged tile variants give up on input-stage group `count`
    (ldp_test_inject_fault in ldp.h)."""
    _abi.call("ldp_test_inject_fault", int(kind), int(after), int(count), _stream(stream))


def batch_run_noalloc(d_descs, count: int, max_pixels: int, max_side: int, d_hist, k: int = 3,
                      regions=(7, 6), compact: bool = True, stream=None) -> None:
    """Batched LDP run that allocates no device memory (static work list of
    2^21 ints shared by all calls; see ldp_batch_run_noalloc in ldp.h).
    For callers that budget device memory once and cannot allocate per batch.
    Calls must not overlap on the GPU."""
    _cuda(d_descs, "d_descs", min_numel=count * DESC_DTYPE.itemsize // d_descs.element_size())
    if d_hist is not None:
        _cuda(d_hist, "d_hist", _torch().int32)
    hist_ptr = ctypes.c_void_p(d_hist.data_ptr()) if d_hist is not None else None
    _abi.call("ldp_batch_run_noalloc", ctypes.c_void_p(d_descs.data_ptr()), int(count), int(max_pixels),
              int(max_side), int(k), RegionSpec(regions[0], regions[1], int(compact)), hist_ptr, _stream(stream))


@dataclass
class BatchLayout:
    """Host-side layout of n images packed in one flat uint8 buffer, their
    code maps in another, and their histograms in one int32 buffer.  Pitches
    are rounded up to 16 bytes so every row starts 16-byte aligned."""

    Hs: np.ndarray
    Ws: np.ndarray
    pitches: np.ndarray
    img_off: np.ndarray
    code_pitches: np.ndarray
    code_off: np.ndarray
    hist_len: int
    img_bytes: int
    code_bytes: int

    @staticmethod
    def build(Hs, Ws, hist_len: int, align: int = 16) -> "BatchLayout":
        Hs = np.asarray(Hs, dtype=np.int64)
        Ws = np.asarray(Ws, dtype=np.int64)
        pitches = (Ws + align - 1) // align * align
        sizes = Hs * pitches
        img_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        cps = np.maximum((Ws - 2 + align - 1) // align * align, align)
        csz = np.maximum(Hs - 2, 0) * cps
        code_off = np.concatenate([[0], np.cumsum(csz)[:-1]]).astype(np.int64)
        return BatchLayout(Hs, Ws, pitches, img_off, cps, code_off, int(hist_len),
                           int(sizes.sum()), int(max(csz.sum(), 16)))

    @property
    def n(self) -> int:
        return len(self.Hs)

    @property
    def pixels(self) -> int:
        return int((self.Hs * self.Ws).sum())

    def descs(self, img_base: int, code_base: int | None) -> np.ndarray:
        d = np.zeros(self.n, dtype=DESC_DTYPE)
        d["img"] = img_base + self.img_off
        d["H"] = self.Hs
        d["W"] = self.Ws
        d["pitch"] = self.pitches
        d["code_pitch"] = self.code_pitches
        d["codes"] = (code_base + self.code_off) if code_base else 0
        d["hist_offset"] = np.arange(self.n, dtype=np.uint64) * np.uint64(self.hist_len)
        return d

    def image(self, buf, i: int):
        """View of image i inside a flat buffer (numpy or torch), shape (H, W)."""
        o, H, W, P = int(self.img_off[i]), int(self.Hs[i]), int(self.Ws[i]), int(self.pitches[i])
        return buf[o:o + H * P].reshape(H, P)[:, :W]

    def codes(self, buf, i: int):
        o, H, W, P = int(self.code_off[i]), int(self.Hs[i]), int(self.Ws[i]), int(self.code_pitches[i])
        return buf[o:o + (H - 2) * P].reshape(H - 2, P)[:, :W - 2]


class BatchPlan:
    """A plan for one persistent launch over up to max_images images of any
    sizes (the library's work list and CUDA graph live inside)."""

    def __init__(self, max_images: int, max_pixels: int, k: int = 3, regions=(7, 6), compact: bool = True,
                 lbp: bool = False, graph: bool = True, code_mode: int = CODE_ABS, tuned: bool = True):
        """tuned: take the tile variant the shipped autotune cache holds for
        this device and workload class (k or LBP, pixels per image =
        max_pixels / max_images), when it holds one; `config` records it.
        set_config overrides it."""
        self.lbp = lbp
        self.config = None
        self.k = k
        self.regions = tuple(regions)
        self.compact = bool(compact) and not lbp
        self.nbins = comb(8, k) if self.compact else 256
        flags = ((_abi.LDP_PLAN_LBP if lbp else 0) | (0 if graph else _abi.LDP_PLAN_NO_GRAPH) |
                 _abi.plan_code_mode(code_mode))
        h = ctypes.c_void_p()
        _abi.call("ldp_batch_plan_create", ctypes.byref(h), int(max_images), int(max_pixels), int(k),
                  RegionSpec(self.regions[0], self.regions[1], int(self.compact)), flags)
        self._h = h
        if tuned and code_mode == CODE_ABS:
            self._apply_cache(max_images, max_pixels)

    def _apply_cache(self, max_images: int, max_pixels: int) -> None:
        from . import autotune

        torch = _torch()
        if not torch.cuda.is_available():
            return
        dev = torch.cuda.current_device()
        props = torch.cuda.get_device_properties(dev)
        ent = autotune.lookup(torch.cuda.get_device_name(dev), props.multi_processor_count, "batch",
                              0 if self.lbp else self.k, ("lbp+" if self.lbp else "") + "hist+codes",
                              max_pixels / max(1, max_images))
        if ent:
            self.set_config(ent["variant"], ent["ctas_per_sm"])
            self.config = {"variant": ent["variant"], "ctas_per_sm": ent["ctas_per_sm"], "from": "autotune cache"}

    @property
    def hist_len(self) -> int:
        return self.regions[0] * self.regions[1] * self.nbins

    def set_config(self, variant: int, ctas_per_sm: int = 0) -> None:
        _abi.call("ldp_batch_plan_set_config", self._h, int(variant), int(ctas_per_sm))
        self.config = {"variant": int(variant), "ctas_per_sm": int(ctas_per_sm), "from": "set_config"}

    def run(self, d_descs, d_count, d_hist, stream=None) -> None:
        """d_descs: device buffer of DESC_DTYPE records; d_count: device int32
        holding the image count; d_hist: device int32 buffer (or None)."""
        fn = "lbp_batch_run" if self.lbp else "ldp_batch_run"
        _cuda(d_descs, "d_descs")
        _cuda(d_count, "d_count", _torch().int32, 1)
        if d_hist is not None:
            _cuda(d_hist, "d_hist", _torch().int32)
        hist_ptr = ctypes.c_void_p(d_hist.data_ptr()) if d_hist is not None else None
        _abi.call(fn, self._h, ctypes.c_void_p(d_descs.data_ptr()), ctypes.c_void_p(d_count.data_ptr()),
                  hist_ptr, _stream(stream))

    def enable_timing(self, capacity: int) -> None:
        """Record CUDA events around the persistent kernel of the next `capacity` runs."""
        _abi.call("ldp_batch_plan_enable_timing", self._h, int(capacity))

    def kernel_times(self, capacity: int = 1 << 16) -> list[float]:
        """Milliseconds of the persistent kernel of each recorded run (waits for them)."""
        buf = (ctypes.c_float * capacity)()
        n = ctypes.c_int(0)
        _abi.call("ldp_batch_plan_kernel_times", self._h, buf, capacity, ctypes.byref(n))
        return [float(buf[i]) for i in range(n.value)]

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _abi.load().ldp_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
