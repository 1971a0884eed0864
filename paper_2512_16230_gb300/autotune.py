"""Autotuner of the batched engine's launch shapes.

For every group of the serving mix (lattice, storage, equation) it builds a batch from solves
whose grids are those of the seeded serving request stream itself (the first requests of the
group's flow classes, grids capped in size so that the work-list kernel, not the single-solve
path, runs them), times batched steps for every candidate (cells per tile) x (resident blocks per
SM, 0 = the occupancy limit), and keeps the fastest. Then it times the solo threshold -- members of
at least that many cells run on the single-solve kernels -- on a batch of the stream's 3D solves at
their full sizes and on the largest of them alone, and keeps the smallest sum of the two. Results
and every timing are cached per GPU name in ``_tune/tuning.json`` (git-ignored) and applied to a
batch by ``apply``.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import inputs as I
from . import workloads as W

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune", "tuning.json")
TILES = (64, 128, 256)
PER_SM = (0, 2, 4)
SOLO = (1 << 18, 1 << 19, 1 << 20, 1 << 21, 0)   # objective: a mixed batch plus its largest solve alone
FLOWS = {"nse": ("tgv2d", "kolmogorov"), "ncde": ("ncde",)}
GROUPS = [(lat, eq) for lat in I.SERVING_2D for eq in ("nse", "ncde")] + [(lat, "nse") for lat in I.SERVING_3D]
MAX_GROUP_CELLS = {2: 1 << 18, 3: 1 << 19}     # grids of the group batches: below the solo threshold


def _stream(n=4000):
    return I.serving_requests(n, seed=0, rate_per_s=20.0)


def _class_requests(lattice, eq, count, max_cells=None):
    out = []
    for req in _stream():
        if req["lattice"] == lattice and req["flow"] in FLOWS[eq]:
            if max_cells is None or int(np.prod(req["grid"])) <= max_cells:
                out.append(req)
        if len(out) == count:
            break
    return out


def _model(lbm, lat_cache, req, store):
    wl = W.serving_workload(req, store)
    if req["lattice"] not in lat_cache:
        spec = W.LATTICES[req["lattice"]]
        lat_cache[req["lattice"]] = lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w)
    m = lbm.Model(lat_cache[req["lattice"]], wl.eq, wl.n, store=store)
    m.set_relaxation(wl.s, wl.s_high)
    if wl.force is not None:
        m.set_force(*wl.force)
    if wl.u_const is not None:
        m.set_ncde(wl.u_const, wl.nonlin)
    rho, u = wl.fields()
    m.init_fields(rho, None if u is None else np.ascontiguousarray(u))
    return m


def _time_steps(torch, batch, steps):
    batch.step(8)          # rebuild, warm-up, graph capture
    batch.synchronize()
    stream = torch.cuda.ExternalStream(batch.stream)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    batch.step(steps)
    t1.record(stream)
    t1.synchronize()
    return t0.elapsed_time(t1) / steps


def autotune(stores=("f32", "f16_dev"), steps=16, solves=6, use_cache=True):
    """Return {"tiles": {(kind, store, eq): cells}, "per_sm": {(kind, store, eq): blocks},
    "solo_cells": cells, "ms_per_step": {...}} for the current GPU."""
    import torch
    from . import lbm
    gpu = torch.cuda.get_device_name()
    if use_cache and os.path.exists(CACHE):
        cached = json.load(open(CACHE))
        if cached.get("gpu") == gpu:
            return _decode(cached)
    tiles, per_sm, timings = {}, {}, {}
    lat_cache = {}
    for lattice, eq in GROUPS:
        spec = W.LATTICES[lattice]
        reqs = _class_requests(lattice, eq, solves, MAX_GROUP_CELLS[spec.d])
        for store in stores:
            models = [_model(lbm, lat_cache, r, store) for r in reqs]
            b = lbm.Batch(len(models) + 1)
            b.set_solo_threshold(0)
            for m in models:
                b.add(m)
            best = None
            for cells in TILES:
                for blocks in PER_SM:
                    b.set_tile(spec.kind, store, eq, cells)
                    b.set_blocks_per_sm(spec.kind, store, eq, blocks)
                    ms = _time_steps(torch, b, steps)
                    timings[f"{spec.kind}|{store}|{eq}|tile={cells}|per_sm={blocks}"] = ms
                    if best is None or ms < best[2]:
                        best = (cells, blocks, ms)
            key = (spec.kind, store, eq)
            tiles[key], per_sm[key] = best[0], best[1]
            timings[f"{spec.kind}|{store}|{eq}|grids"] = [list(r["grid"]) for r in reqs]
            b.close()
            for m in models:
                m.close()
            torch.cuda.empty_cache()
    # solo threshold: the stream's 3D solves at their full sizes (FP32, as served)
    reqs = [r for r in _stream() if r["flow"] == "kolmogorov"][:8]
    models = [_model(lbm, lat_cache, r, "f32") for r in reqs]
    b = lbm.Batch(len(models) + 1)
    for key, cells in tiles.items():
        b.set_tile(*key, cells)
        b.set_blocks_per_sm(*key, per_sm[key])
    for m in models:
        b.add(m)
    # the largest of them alone as well: the case where the single-solve kernels decide a latency
    big = max(models, key=lambda m: m.ncells)
    lone = lbm.Batch(2)
    for key, cells in tiles.items():
        lone.set_tile(*key, cells)
        lone.set_blocks_per_sm(*key, per_sm[key])
    best = None
    for solo in SOLO:
        b.set_solo_threshold(solo)
        ms = _time_steps(torch, b, steps)
        timings[f"solo_cells={solo}"] = ms
        b.remove(big)
        lone.add(big)
        lone.set_solo_threshold(solo)
        ms1 = _time_steps(torch, lone, steps)
        lone.remove(big)
        b.add(big)
        timings[f"solo_cells={solo}|largest_alone"] = ms1
        if best is None or ms + ms1 < best[1]:
            best = (solo, ms + ms1)
    timings["solo_grids"] = [list(r["grid"]) for r in reqs]
    lone.close()
    b.close()
    for m in models:
        m.close()
    torch.cuda.empty_cache()
    out = {"gpu": gpu, "tiles": {"|".join(k): v for k, v in tiles.items()},
           "per_sm": {"|".join(k): v for k, v in per_sm.items()}, "solo_cells": best[0], "ms_per_step": timings}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    json.dump(out, open(CACHE, "w"), indent=1)
    return _decode(out)


def _decode(d):
    return {"tiles": {tuple(k.split("|")): v for k, v in d["tiles"].items()},
            "per_sm": {tuple(k.split("|")): v for k, v in d.get("per_sm", {}).items()},
            "solo_cells": d.get("solo_cells", 1 << 19), "ms_per_step": d.get("ms_per_step", {})}


def apply(batch, tuning):
    """Set a batch's tile sizes, resident blocks per SM and solo threshold from a tuning."""
    if not tuning:
        return
    for key, cells in tuning.get("tiles", {}).items():
        batch.set_tile(*key, cells)
    for key, blocks in tuning.get("per_sm", {}).items():
        batch.set_blocks_per_sm(*key, blocks)
    if "solo_cells" in tuning:
        batch.set_solo_threshold(tuning["solo_cells"])


def summary(tuning):
    """The chosen shapes, as printed by the benchmark."""
    return {"tiles": {"|".join(k): v for k, v in tuning["tiles"].items()},
            "per_sm": {"|".join(k): v for k, v in tuning["per_sm"].items()},
            "solo_cells": tuning["solo_cells"]}


if __name__ == "__main__":
    t = autotune(use_cache=False)
    print(json.dumps(dict(summary(t), ms_per_step=t["ms_per_step"]), indent=1))
