"""Autotuner of the batched kernel: cells per tile (thread block) for each group type.

For every (lattice, storage, equation) of the serving mix it builds a small synthetic batch of
mid-sized solves, times a few batched steps with each candidate tile size (64, 128, 256 cells),
and keeps the fastest. Results are cached per GPU name in ``_tune/tiles.json`` (git-ignored) and
handed to ``lbm.Batch.set_tile`` by the serving engine.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import inputs as I
from . import workloads as W

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune", "tiles.json")
CANDIDATES = (64, 128, 256)
GROUPS = [(name, eq) for name in I.SERVING_2D for eq in ("nse", "ncde")] + [(name, "nse") for name in I.SERVING_3D]


def _solves(lbm, lat, spec, eq, store):
    grids = [(96, 96, 96), (64, 64, 64)] if spec.d == 3 else [(512, 384), (256, 256)]
    out = []
    for k, n in enumerate(grids):
        m = lbm.Model(lat, eq, n, store=store)
        s = W.rates_nse(spec.d, 0.05, spec.cs2[0]) if eq == "nse" else W.rates_ncde(spec.d, 0.1, spec.cs2[0])
        m.set_relaxation(s, 1.0)
        if eq == "nse":
            rho, u = I.rest_state(n, spec.d)
            m.init_fields(rho, u)
        else:
            m.set_ncde((0.02, 0.01, 0.0)[:spec.d], 1.0)
            m.init_fields(I.gaussian_hill(n, spec.c, n[0] / 8, 1.0))
        out.append(m)
    return out


def autotune(stores=("f32", "f16_dev"), steps=24, use_cache=True):
    """Return {(kind, store, eq): cells_per_tile}; times each candidate on the current GPU."""
    import torch
    from . import lbm
    gpu = torch.cuda.get_device_name()
    if use_cache and os.path.exists(CACHE):
        cached = json.load(open(CACHE))
        if cached.get("gpu") == gpu:
            return {tuple(k.split("|")): v for k, v in cached["tiles"].items()}
    tiles, timings = {}, {}
    for name, eq in GROUPS:
        spec = W.LATTICES[name]
        lat = lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w)
        for store in stores:
            models = _solves(lbm, lat, spec, eq, store)
            b = lbm.Batch(8)
            for m in models:
                b.add(m)
            best = None
            for cells in CANDIDATES:
                b.set_tile(spec.kind, store, eq, cells)
                b.step(8)          # rebuild and warm up
                b.synchronize()
                stream = torch.cuda.ExternalStream(b.stream)
                t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0.record(stream)
                b.step(steps)
                t1.record(stream)
                t1.synchronize()
                ms = t0.elapsed_time(t1) / steps
                timings[f"{spec.kind}|{store}|{eq}|{cells}"] = ms
                if best is None or ms < best[1]:
                    best = (cells, ms)
            tiles[(spec.kind, store, eq)] = best[0]
            b.close()
            for m in models:
                m.close()
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    json.dump({"gpu": gpu, "tiles": {"|".join(k): v for k, v in tiles.items()}, "ms_per_step": timings},
              open(CACHE, "w"), indent=1)
    return tiles


if __name__ == "__main__":
    print(json.dumps({"|".join(k): v for k, v in autotune(use_cache=False).items()}, indent=1))
