"""Autotuner for the persistent batch kernel.

Searches the compiled tile variants (tile rows x warps per CTA x register cap)
and the number of resident CTAs per SM on the caller's own batch, timing only
the persistent kernel with the CUDA events a plan records inside its graph.
Results are cached as JSON keyed by device name, SM count, descriptor (LDP k
or LBP), histogram / codes mode and image-size class.

The cache file is `autotune_cache.json` next to this module (tuned entries
for the GB300 ship with the package); `LDP_AUTOTUNE_CACHE` points elsewhere.

    python -m paper_1810_11518_gb300.autotune --out cache.json   # tune the standard workloads
"""
from __future__ import annotations

import json
import os
import statistics

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "autotune_cache.json")


def cache_path() -> str:
    return os.environ.get("LDP_AUTOTUNE_CACHE", DEFAULT_CACHE)


def size_class(pixels_per_image: float) -> str:
    """Images of similar size share a tuned configuration."""
    if pixels_per_image < 200_000:
        return "small"
    if pixels_per_image < 2_000_000:
        return "medium"
    return "large"


def make_key(device: str, sms: int, path: str, k: int, mode: str, pixels_per_image: float,
             mixed: bool = False) -> str:
    """Cache key; batches of images of different sizes (mixed) are tuned
    apart from batches of one size in the same size class."""
    return f"{device}|{sms}|{path}|k{k}|{mode}|{size_class(pixels_per_image)}" + ("|mixed" if mixed else "")


def load_cache(path: str | None = None) -> dict:
    try:
        with open(path or cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(device: str, sms: int, path: str, k: int, mode: str, pixels_per_image: float,
           cache: dict | None = None, mixed: bool = False) -> dict | None:
    """The cached {"variant", "ctas_per_sm", ...} for this workload, or None."""
    c = load_cache() if cache is None else cache
    return c.get(make_key(device, sms, path, k, mode, pixels_per_image, mixed))


def tune_plan(plan, d_desc, d_count, d_hist, ctas_options=(0, 4), reps: int = 8, warmup: int = 2) -> dict:
    """Times every (variant, ctas_per_sm) on this batch; leaves the best set
    on the plan and returns it with all measurements (kernel ms, median).

    A candidate whose runs set a bit of the device status word (work cut
    short: more tiles than the work list holds, an image rejected, a wait
    that gave up) did not do the whole batch: it is recorded with its status
    and never chosen.  RuntimeError when every candidate does so."""
    import paper_1810_11518_gb300 as ldp

    results = []
    ldp.device_status()  # start from a clear status word
    for v in range(ldp.num_variants()):
        for cps in ctas_options:
            plan.set_config(v, cps)
            for _ in range(warmup):
                plan.run(d_desc, d_count, d_hist)
            status = ldp.device_status()
            if status:
                results.append({"variant": v, "name": ldp.variant_name(v), "ctas_per_sm": cps,
                                "kernel_ms": None, "status": status})
                continue
            plan.enable_timing(reps)
            for _ in range(reps):
                plan.run(d_desc, d_count, d_hist)
            ms = statistics.median(plan.kernel_times(reps))
            status = ldp.device_status()
            results.append({"variant": v, "name": ldp.variant_name(v), "ctas_per_sm": cps,
                            "kernel_ms": None if status else ms, "status": status})
    timed = [r for r in results if r["status"] == 0]
    if not timed:
        raise RuntimeError("autotune: every variant set the device status word "
                           f"({sorted({r['status'] for r in results})}); the batch exceeds the plan or is invalid")
    best = min(timed, key=lambda r: r["kernel_ms"])
    plan.set_config(best["variant"], best["ctas_per_sm"])
    return {"variant": best["variant"], "name": best["name"], "ctas_per_sm": best["ctas_per_sm"],
            "kernel_ms": best["kernel_ms"], "all": results}


def store(key: str, entry: dict, path: str | None = None) -> None:
    path = path or cache_path()
    c = load_cache(path)
    c[key] = {k: v for k, v in entry.items() if k != "all"}
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _tune_workload(name, Hs, Ws, seeds, k, lbp, sigma, out, hist=True):
    import numpy as np
    import torch

    import paper_1810_11518_gb300 as ldp
    import synth

    nb = 256 if lbp else ldp.hist_bins(k)
    R, C = (16, 16) if name == "large" else (7, 6)
    lay = ldp.BatchLayout.build(Hs, Ws, hist_len=R * C * nb)
    host = np.zeros(lay.img_bytes, dtype=np.uint8)
    synth.batch_into(host, seeds, lay.Hs, lay.Ws, lay.pitches, lay.img_off, sigma=sigma)
    d_img = torch.from_numpy(host).cuda()
    d_codes = torch.empty(lay.code_bytes, dtype=torch.uint8, device="cuda")
    d_hist = torch.empty(lay.n * lay.hist_len, dtype=torch.int32, device="cuda")
    d_desc = torch.from_numpy(lay.descs(d_img.data_ptr(), d_codes.data_ptr()).view(np.uint8)).cuda()
    d_count = torch.tensor([lay.n], dtype=torch.int32, device="cuda")
    dev = torch.cuda.get_device_properties(0)
    with ldp.BatchPlan(lay.n, lay.pixels, k=k, regions=(R, C), lbp=lbp) as plan:
        res = tune_plan(plan, d_desc, d_count, d_hist if hist else None)
    mode = ("lbp+" if lbp else "") + ("hist+codes" if hist else "codes")
    key = make_key(torch.cuda.get_device_name(0), dev.multi_processor_count, "batch", k if not lbp else 0, mode,
                   lay.pixels / lay.n, mixed=len(set(zip(Hs, Ws))) > 1)
    store(key, res, out)
    print(key, res["name"], res["ctas_per_sm"], f"{res['kernel_ms']:.4f} ms", flush=True)


def main():
    import argparse
    import sys

    sys.path.insert(0, os.path.dirname(HERE))
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=cache_path())
    ap.add_argument("--images", type=int, default=1024)
    a = ap.parse_args()
    import synth

    n = a.images
    seeds = list(range(n))
    # uneven 64..1024 (a "mixed" entry of the faces' size class), 640x490
    # faces (LDP k = 1..4 and LBP), 260x260 face crops (codes only, the front
    # end's extraction), 8192^2 stress
    sizes = [synth.sizes(s) for s in range(n)]
    _tune_workload("uneven", [h for h, _ in sizes], [w for _, w in sizes], seeds, 3, False, 3.0, a.out)
    for k in (3, 1, 2, 4):
        _tune_workload("medium", [490] * n, [640] * n, seeds, k, False, 3.0, a.out)
    _tune_workload("medium", [490] * n, [640] * n, seeds, 3, True, 3.0, a.out)
    _tune_workload("crops", [260] * n, [260] * n, seeds, 3, False, 3.0, a.out, hist=False)
    for k in (1, 2, 3, 4):
        _tune_workload("large", [8192] * 4, [8192] * 4, list(range(4)), k, False, 6.0, a.out)


if __name__ == "__main__":
    main()
