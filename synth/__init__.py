"""Seeded synthetic uint8 images (stand-in for the paper's CK+ crops, Sec. 3.1).

This package only makes input bytes.  It holds none of the LDP/LBP arithmetic,
so the CPU oracle and the CUDA library can both be fed from it without sharing
any of the method's code.  The C source documents the exact recipe.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into synth/_synth.so (host code, x86 or Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_draw.restype = ctypes.c_uint64
            lib.synth_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_sizes.restype = None
            lib.synth_sizes.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            lib.synth_image.restype = ctypes.c_int
            lib.synth_image.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
            lib.synth_batch.restype = ctypes.c_int
            lib.synth_batch.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_int]
            _lib = lib
    return _lib


def default_threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def draw(seed: int, n: int) -> int:
    """Output number n of image seed's SplitMix64 stream."""
    return int(_load().synth_draw(seed, n))


def sizes(seed: int, lo: int = 64, hi: int = 1024) -> tuple[int, int]:
    """(H, W), each uniform on the integers [lo, hi], from the first two draws."""
    h, w = ctypes.c_int(), ctypes.c_int()
    _load().synth_sizes(seed, lo, hi, ctypes.byref(h), ctypes.byref(w))
    return h.value, w.value


def image(seed: int, H: int, W: int, sigma: float = 3.0, pitch: int | None = None,
          threads: int | None = None) -> np.ndarray:
    """One H x W uint8 image (array shape (H, pitch); columns >= W are zero)."""
    pitch = W if pitch is None else pitch
    out = np.zeros((H, pitch), dtype=np.uint8)
    rc = _load().synth_image(seed, H, W, float(sigma), out.ctypes.data, pitch,
                             threads or default_threads())
    if rc:
        raise RuntimeError(f"synth_image failed ({rc})")
    return out


def batch_into(buf: np.ndarray, seeds, Hs, Ws, pitches, offsets, sigma: float = 3.0,
               threads: int | None = None) -> None:
    """Images i = 0..n-1 written into the flat uint8 buffer at offsets[i] with pitch pitches[i]."""
    n = len(seeds)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    Hs = np.ascontiguousarray(Hs, dtype=np.int32)
    Ws = np.ascontiguousarray(Ws, dtype=np.int32)
    pitches = np.ascontiguousarray(pitches, dtype=np.int32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    assert buf.dtype == np.uint8 and buf.flags.c_contiguous
    end = offsets + (Hs.astype(np.int64) - 1) * pitches + Ws
    if n and (offsets.min() < 0 or end.max() > buf.size or (pitches < Ws).any()):
        raise ValueError("image layout exceeds the buffer")
    rc = _load().synth_batch(n, seeds.ctypes.data, Hs.ctypes.data, Ws.ctypes.data, pitches.ctypes.data,
                             offsets.ctypes.data, float(sigma), buf.ctypes.data,
                             threads or default_threads())
    if rc:
        raise RuntimeError(f"synth_batch failed ({rc})")


def batch(seeds, H: int, W: int, sigma: float = 3.0, pitch: int | None = None,
          threads: int | None = None) -> np.ndarray:
    """Equal-size images stacked as an array of shape (n, H, pitch)."""
    n = len(seeds)
    pitch = W if pitch is None else pitch
    out = np.zeros((n, H, pitch), dtype=np.uint8)
    offs = np.arange(n, dtype=np.int64) * (H * pitch)
    batch_into(out.reshape(-1), seeds, [H] * n, [W] * n, [pitch] * n, offs, sigma, threads)
    return out
