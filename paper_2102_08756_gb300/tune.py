"""Autotuner of the history-convolution launch (Section 2.3, the per-mode
truncated time convolution): picks the kernel variant (register prefetch, or
one of the TMA pipeline shapes), the orbit records per CTA (64, 128 or 256:
the modes-per-CTA tile) and the lags per CTA (the history-chunk tile) for a
live handle by timing the convolution stage with the library's own per-stage
CUDA events.

Each trial runs real steps of the handle, so its history advances; tune a
handle whose history is already representative (for the full-history cost,
after n_cut steps).  Results can be cached in a JSON file keyed by grid,
history length, precision, compensation and GPU name.
"""
from __future__ import annotations

import json
import os

import torch

VARIANTS = (1, 2, 3, 0)
TILES = (64, 128, 256)


def _key(h, gpu_name):
    return f"{h.n1}x{h.n3}:{h.n_cut}:{h.precision}:{int(bool(h.kahan))}:{gpu_name}"


def autotune(h, u, v, steps=6, chunkings=None, tiles=TILES, cache=None, verbose=False):
    """Time every (variant, orbit tile, lags_per_cta) candidate on handle ``h``
    with the input fields (u, v) and keep the fastest (the register-prefetch
    variant 0 has the fixed 128-record tile; a tile the handle's record count
    is not a multiple of is skipped).  Returns (best, table)."""
    gpu = torch.cuda.get_device_name(h.device)
    if cache and os.path.exists(cache):
        db = json.load(open(cache))
        hit = db.get(_key(h, gpu))
        if hit:
            h.set_conv_tile(hit.get("tile", 128))
            h.set_conv_config(hit["variant"], hit["lags_per_cta"])
            return hit, None
    if chunkings is None:
        chunkings = sorted({0} | {c for c in (256, 512, 1024, 2048) if c < h.n_cut})
    tau = torch.empty_like(u)
    table = []
    for var in VARIANTS:
        for tile in (tiles if var >= 1 else (128,)):
            try:
                h.set_conv_tile(tile)
            except RuntimeError:
                continue
            for lpc in chunkings:
                try:
                    h.set_conv_config(var, lpc)
                except RuntimeError:
                    continue
                h.step(u, v, tau)                     # warm-up of this launch shape
                h.set_profiling(True)
                for _ in range(steps):
                    h.step(u, v, tau)
                times, n = h.stage_times()
                h.set_profiling(False)
                h.check()
                row = {"variant": var, "tile": tile, "lags_per_cta": lpc,
                       "conv_ms": times["convolution"] / n}
                table.append(row)
                if verbose:
                    print(row, flush=True)
    best = min(table, key=lambda r: r["conv_ms"])
    h.set_conv_tile(best["tile"])
    h.set_conv_config(best["variant"], best["lags_per_cta"])
    if cache:
        db = json.load(open(cache)) if os.path.exists(cache) else {}
        db[_key(h, gpu)] = best
        with open(cache, "w") as f:
            json.dump(db, f, indent=1)
    return best, table


def autotune_hybrid_batch(b, stream, shapes=(1, 2, 3, 4, 5, 6), lags=(256, 512, 1024, 2048),
                          tiles=TILES, steps=4):
    """Time whole captured ensemble steps of a hybrid batch for every (launch
    shape: 1-3 persistent, 4-6 one CTA per item; orbit records per CTA; lags per
    work item) of the batched convolution and keep the fastest (the batch is
    left captured with it).  Each trial advances the ensemble by ``steps + 1``
    steps."""
    from . import sbim as B
    table = []
    for tile in tiles:
        for shape in shapes:
            for lpi in lags:
                try:
                    B.sbim_hybrid_batch_set_conv_config(b, shape, lpi)
                    B.sbim_hybrid_batch_set_conv_tile(b, tile)
                    B.sbim_hybrid_batch_capture(b)
                except RuntimeError:
                    continue
                B.sbim_hybrid_batch_replay(b)              # warm-up of this launch
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    B.sbim_hybrid_batch_replay(b)
                e1.record(stream)
                stream.synchronize()
                table.append({"shape": shape, "tile": tile, "lags_per_item": lpi,
                              "step_ms": e0.elapsed_time(e1) / steps})
    best = min(table, key=lambda r: r["step_ms"])
    B.sbim_hybrid_batch_set_conv_config(b, best["shape"], best["lags_per_item"])
    B.sbim_hybrid_batch_set_conv_tile(b, best["tile"])
    B.sbim_hybrid_batch_capture(b)
    return {"best": best, "trials": table}
