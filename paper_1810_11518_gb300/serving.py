"""Continuous-batching serving of single-image LDP requests.

`Server` wraps the native request runtime of libldp (ldp_server_* in
include/ldp.h): requests are admitted into a resident device arena as
memory frees up, batched as they arrive, and run on several streams so
batches overlap on the device.  `run_load` drives it with Poisson arrivals
from a seeded generator and reports p50/p99 latency and sustained Mpixel/s.

    python -m paper_1810_11518_gb300.serving --rates 5000 20000 50000 --seconds 10 --warmup 2
"""
from __future__ import annotations

import ctypes
import json
import time
from math import comb

import numpy as np

from . import _abi


class Server:
    def __init__(self, k: int = 3, regions=(7, 6), compact: bool = True, max_batch: int = 256,
                 streams: int = 3, arena_bytes: int = 1 << 30, variant: int = -1, ctas_per_sm: int = 0):
        self.k, self.regions, self.compact = k, tuple(regions), bool(compact)
        self.hist_len = regions[0] * regions[1] * (comb(8, k) if compact else 256)
        cfg = _abi.ServerConfig(max_batch, streams, arena_bytes, k,
                                _abi.RegionSpec(regions[0], regions[1], int(compact)), variant, ctas_per_sm)
        h = ctypes.c_void_p()
        _abi.call("ldp_server_create", ctypes.byref(h), ctypes.byref(cfg))
        self._h = h
        self._buf = (_abi.Completion * 4096)()

    def submit(self, img: np.ndarray, tag: int, codes: np.ndarray | None = None,
               hist: np.ndarray | None = None) -> None:
        """img: (H, W) uint8 view (row stride = pitch), ideally in pinned memory;
        codes: (H-2, W-2) uint8 view or None; hist: hist_len uint32/int32 or None.
        All must stay alive and untouched until the request completes."""
        H, W = img.shape
        _abi.call("ldp_server_submit", self._h, ctypes.c_void_p(img.ctypes.data), H, W, img.strides[0],
                  ctypes.c_void_p(codes.ctypes.data) if codes is not None else None,
                  codes.strides[0] if codes is not None else 0,
                  ctypes.c_void_p(hist.ctypes.data) if hist is not None else None, tag)

    def poll(self) -> list[tuple[int, int, int, int]]:
        """Completed requests: (tag, t_submit_ns, t_start_ns, t_done_ns)."""
        out = []
        n = ctypes.c_int(0)
        while True:
            _abi.call("ldp_server_poll", self._h, self._buf, len(self._buf), ctypes.byref(n))
            out.extend((c.tag, c.t_submit_ns, c.t_start_ns, c.t_done_ns) for c in self._buf[:n.value])
            if n.value < len(self._buf):
                return out

    def stats(self) -> dict:
        st = _abi.ServerStats()
        _abi.call("ldp_server_stats", self._h, ctypes.byref(st))
        return {f: int(getattr(st, f)) for f, _ in _abi.ServerStats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _abi.load().ldp_server_destroy(self._h)
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


class RequestPool:
    """Synthetic request images in pinned host memory, drawn from a size
    distribution: 'uneven' (H, W uniform on [64, 1024]) or 'faces' (640x490).
    Rows are padded to 16-byte pitches so each upload is one linear copy."""

    def __init__(self, n: int = 512, dist: str = "uneven", seed0: int = 100_000):
        import torch

        import synth

        if dist == "faces":
            sizes = [(490, 640)] * n
        else:
            sizes = [synth.sizes(seed0 + i, 64, 1024) for i in range(n)]
        self.Hs = np.array([h for h, _ in sizes], dtype=np.int64)
        self.Ws = np.array([w for _, w in sizes], dtype=np.int64)
        self.pitches = (self.Ws + 15) // 16 * 16
        self.off = np.concatenate([[0], np.cumsum(self.Hs * self.pitches)[:-1]]).astype(np.int64)
        total = int((self.Hs * self.pitches).sum())
        self._pinned = torch.zeros(total, dtype=torch.uint8, pin_memory=True)
        self.buf = self._pinned.numpy()
        synth.batch_into(self.buf, np.arange(n) + seed0, self.Hs, self.Ws, self.pitches, self.off)
        self.n = n

    def image(self, i: int) -> np.ndarray:
        o, H, W, P = int(self.off[i]), int(self.Hs[i]), int(self.Ws[i]), int(self.pitches[i])
        return self.buf[o:o + H * P].reshape(H, P)[:, :W]


def run_load(server: Server, pool: RequestPool, rate: float, seconds: float, warmup: float = 0.0,
             seed: int = 0, ring: int = 16384) -> dict:
    """Poisson arrivals at `rate` req/s for warmup + seconds.  Returns, over the
    requests arriving after the warm-up: latency percentiles from the
    scheduled arrival to results in host memory (p50/p99, so client lag is
    included), the same from the actual submit, sustained Mpixel/s (their
    pixels over first arrival .. last completion), and the client's lag."""
    import gc

    import torch

    rng = np.random.default_rng(seed)
    hist_ring = torch.empty((ring, server.hist_len), dtype=torch.int32, pin_memory=True).numpy()
    # raw pointers keep the per-request host cost to one C call
    lib = _abi.load()
    submit = lib.ldp_server_submit
    h = server._h
    img_ptr = [int(pool.buf.ctypes.data + int(pool.off[j])) for j in range(pool.n)]
    hist_base, hist_stride = int(hist_ring.ctypes.data), hist_ring.strides[0]
    total_s = warmup + seconds
    n_req = int(rate * total_s * 1.2) + 16
    gaps = rng.exponential(1.0 / rate, size=n_req)
    arrivals = np.cumsum(gaps)
    pick = rng.integers(0, pool.n, size=n_req)
    done: dict[int, tuple] = {}
    submitted_px = []
    gc_was = gc.isenabled()
    gc.disable()  # no collector pauses inside the arrival schedule
    t0_ns = time.monotonic_ns()  # the runtime stamps with the same monotonic clock
    lag_max = 0.0
    i = 0
    while True:
        now = (time.monotonic_ns() - t0_ns) * 1e-9
        if i < n_req and arrivals[i] <= total_s:
            if arrivals[i] > now:
                # poll while waiting for the next arrival
                for c in server.poll():
                    done[c[0]] = c
                continue
            if i - len(done) >= ring:  # result ring full: wait for completions
                for c in server.poll():
                    done[c[0]] = c
                continue
            lag_max = max(lag_max, now - arrivals[i])
            j = int(pick[i])
            Hj, Wj = int(pool.Hs[j]), int(pool.Ws[j])
            rc = submit(h, img_ptr[j], Hj, Wj, int(pool.pitches[j]), None, 0, hist_base + (i % ring) * hist_stride, i)
            if rc:
                _abi.check(rc, "ldp_server_submit")
            submitted_px.append(Hj * Wj)
            i += 1
        else:
            break
    n_sub = i
    while len(done) < n_sub:
        for c in server.poll():
            done[c[0]] = c
        time.sleep(0.0002)
    if gc_was:
        gc.enable()
    # measured window: requests arriving after warm-up
    lat, lat_sub, px, last_done, first_arr = [], [], 0, 0, None
    for tag in range(n_sub):
        if arrivals[tag] < warmup:
            continue
        c = done[tag]
        arr_ns = t0_ns + int(arrivals[tag] * 1e9)
        first_arr = arr_ns if first_arr is None else first_arr
        lat.append((c[3] - arr_ns) / 1e6)
        lat_sub.append((c[3] - c[1]) / 1e6)
        px += submitted_px[tag]
        last_done = max(last_done, c[3])
    lat = np.array(lat) if lat else np.array([0.0])
    lat_sub = np.array(lat_sub) if lat_sub else np.array([0.0])
    window = max((last_done - (first_arr or last_done)) * 1e-9, 1e-9)
    st = server.stats()
    return {"rate_req_s": rate, "requests": len(lat), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "p50_from_submit_ms": float(np.percentile(lat_sub, 50)),
            "p99_from_submit_ms": float(np.percentile(lat_sub, 99)),
            "sustained_mpix_s": px / window / 1e6, "achieved_req_s": len(lat) / window,
            "client_lag_max_ms": lag_max * 1e3, "batches": st["batches"],
            "mean_batch": st["completed"] / max(st["batches"], 1)}


def main():
    import argparse
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", type=float, nargs="+", default=[5000, 20000, 50000])
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--warmup", type=float, default=2.0)
    ap.add_argument("--dist", default="uneven", choices=["uneven", "faces"])
    ap.add_argument("--streams", type=int, default=3)
    ap.add_argument("--max-batch", type=int, default=256)
    a = ap.parse_args()
    pool = RequestPool(512, a.dist)
    for r in a.rates:
        with Server(streams=a.streams, max_batch=a.max_batch) as srv:
            res = run_load(srv, pool, r, a.seconds, a.warmup, seed=int(r))
        res["dist"] = a.dist
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
