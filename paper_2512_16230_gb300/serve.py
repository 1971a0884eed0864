"""Serving many lattice-Boltzmann solves on one GPU.

Two request loops over the same seeded request stream (``inputs.serving_requests``):

* ``serve_batched`` -- continuous batching. Requests are admitted, in arrival order, as soon as
  they have arrived and their device workspace fits the HBM budget and a slot is free; every
  admitted solve stays resident and joins one ``lbm.Batch``, which advances all resident solves
  together (one persistent launch per group of solves per step, steps replayed from a CUDA graph).
  The loop enqueues the batch in ticks of at most ``tick`` steps, never past the earliest
  completion, and keeps one tick queued ahead of the one running, so that the host work between
  ticks overlaps the device: the initial fields of arrived requests are generated on worker
  threads, a new solve is initialised on its own stream while the batch runs, and a finished
  solve leaves the batch without a host wait -- its fields are computed on the device and copied
  into pinned host memory behind an event, and its memory is released once that event is done.
* ``serve_sequential`` -- the plain path: one solve at a time in arrival order, FP32, each step one
  launch of the single-solve kernel, fields read back synchronously.

Both record arrival, admission and completion times per request (a batched completion is the
device time of its read-back event, on the host clock); ``summarize`` turns them into solves/s,
latency percentiles and cell updates per second. The host logic (admission, ticks, retirement,
accounting) is independent of the GPU: ``FakeEngine`` drives it on the CPU in tests.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import time
from dataclasses import dataclass

import numpy as np

from . import inputs as I
from . import workloads as W

# The flow classes of the serving mix, and for each the longest run that FP16-deviation storage
# serves within the 1e-3 relative L2 bound on u (or phi) against the FP64 oracle, on the smallest
# and on the largest served grids (0: never). The rounding error of 16-bit storage grows with the
# run (a random walk of the rounded momentum in the vortices) and with the grid (on fine grids the
# per-step change of a population -- the forcing of the Kolmogorov flow, the diffusion of the hill
# -- falls below a unit of the stored deviation and is rounded away), so only short vortex runs
# qualify; every other request is served in FP32. The serving-precision tests check each threshold.
SERVING_CLASSES = ([(flow, lat) for flow in ("tgv2d", "ncde") for lat in I.SERVING_2D]
                   + [("kolmogorov", lat) for lat in I.SERVING_3D])
F16_MAX_STEPS = {
    ("tgv2d", "rD2Q17"): 200, ("tgv2d", "rD2Q21"): 200, ("tgv2d", "rD2Q25"): 200,
    ("ncde", "rD2Q17"): 0, ("ncde", "rD2Q21"): 0, ("ncde", "rD2Q25"): 0,
    ("kolmogorov", "rD3Q33"): 0, ("kolmogorov", "rD3Q45"): 0, ("kolmogorov", "rD3Q53-cubic"): 0,
}


def served_in_f16(flow, lattice, steps):
    return steps <= F16_MAX_STEPS.get((flow, lattice), 0)


def store_for(req, policy):
    """Storage of a request under a serving policy: "as_requested" (FP32 requests in FP32, 16-bit
    ones as FP16 deviations), "f16_dev" (every request as FP16 deviations: the reduced-precision
    path) -- in both, FP16 only where the class and run length keep the error within the bound
    (F16_MAX_STEPS), FP32 otherwise -- or a storage name applied to every request."""
    if policy in ("as_requested", "f16_dev"):
        if policy == "as_requested" and req["store"] == "f32":
            return "f32"
        return "f16_dev" if served_in_f16(req["flow"], req["lattice"], req["steps"]) else "f32"
    return policy


@dataclass
class Record:
    rid: int
    arrival: float
    admitted: float = float("nan")
    finished: float = float("nan")
    steps: int = 0
    cells: int = 0
    lattice: str = ""
    store: str = ""
    q: int = 0


class GpuEngine:
    """Creates, batches and retires models through the CUDA library.

    Protocol of the batched loop: ``prepare`` (host fields of an arrived request, on a worker
    thread), ``create`` + ``add`` (initialise on the model's own stream, join the batch), ``step``
    (enqueue a tick, return its event), ``wait`` (a tick's event), ``finish`` (leave the batch and
    start the read-back, return a handle), ``done`` / ``finish_time`` / ``release`` (poll the
    read-back, its completion time on the host clock, free the model)."""

    def __init__(self, max_solves=4096, tuning=None, keep_results=False, workers=4):
        import torch
        from . import autotune
        from . import lbm
        self.torch = torch
        self.lbm = lbm
        self.batch = lbm.Batch(max_solves)
        self.stream = torch.cuda.ExternalStream(self.batch.stream)
        self._lattices = {}
        self.keep_results = keep_results
        self.results = {}
        self.pool = cf.ThreadPoolExecutor(max_workers=workers)
        self.ref = None
        autotune.apply(self.batch, tuning)

    def lattice(self, name):
        if name not in self._lattices:
            spec = W.LATTICES[name]
            self._lattices[name] = self.lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w)
        return self._lattices[name]

    def nbytes(self, req, store):
        wl = W.serving_workload(req, store)
        return self.lbm.workspace_bytes(self.lattice(req["lattice"]), wl.eq, wl.n, store)

    def start_clock(self, t0):
        """A device timestamp paired with the host clock value t0 (completion times of read-backs
        are measured from it)."""
        ev = self.torch.cuda.Event(enable_timing=True)
        ev.record(self.torch.cuda.current_stream())
        ev.synchronize()
        self.ref = (ev, t0)

    @staticmethod
    def _fields(req, store):
        rho, u = W.serving_workload(req, store).fields()
        return rho, None if u is None else np.ascontiguousarray(u)

    def prepare(self, req, store):
        return self.pool.submit(self._fields, req, store)

    def create(self, req, store, prepared=None, stream=None):
        wl = W.serving_workload(req, store)
        lat = self.lattice(req["lattice"])
        m = self.lbm.Model(lat, wl.eq, wl.n, store=store, stream=stream)
        m.rid = req["rid"]
        m.set_relaxation(wl.s, wl.s_high)
        if wl.force is not None:
            m.set_force(*wl.force)
        if wl.u_const is not None:
            m.set_ncde(wl.u_const, wl.nonlin)
        rho, u = prepared.result() if prepared is not None else self._fields(req, store)
        m.init_fields(rho, u)
        return m, m.workspace_bytes, lat.Q

    def add(self, m):
        self.batch.add(m)

    def step(self, k):
        self.batch.step(k)
        ev = self.torch.cuda.Event()
        ev.record(self.stream)
        return ev

    def wait(self, token):
        token.synchronize()

    def finish(self, m):
        torch = self.torch
        self.batch.remove(m)          # the model's stream now waits for the batch's queued steps
        shape = tuple(reversed(m.n))
        rho_d = torch.empty(shape, dtype=torch.float64, device="cuda")
        u_d = torch.empty((m.d,) + shape, dtype=torch.float64, device="cuda") if m.eq == "nse" else None
        m.read_fields(rho_d, u_d)     # on the model's stream (the current one)
        rho_h = torch.empty(shape, dtype=torch.float64, pin_memory=True)
        rho_h.copy_(rho_d, non_blocking=True)
        u_h = None
        if u_d is not None:
            u_h = torch.empty(u_d.shape, dtype=torch.float64, pin_memory=True)
            u_h.copy_(u_d, non_blocking=True)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(torch.cuda.current_stream())
        return (m, ev, rho_h, u_h, rho_d, u_d)

    def done(self, h):
        return h[1].query()

    def finish_time(self, h):
        ev0, t0 = self.ref
        return t0 + ev0.elapsed_time(h[1]) / 1e3

    def release(self, h):
        m, ev, rho_h, u_h = h[0], h[1], h[2], h[3]
        ev.synchronize()
        if self.keep_results:
            self.results[m.rid] = (rho_h.numpy().copy(), None if u_h is None else u_h.numpy().copy())
        m.close()

    def run_alone(self, m, steps):
        m.step(steps)
        out = m.read_fields()
        if self.keep_results:
            self.results[m.rid] = out
        m.close()

    def close(self):
        self.pool.shutdown(wait=True)
        self.batch.close()


class FakeEngine:
    """CPU stand-in with the same interface: a tick of the batch costs time proportional to the
    resident cells (tests of the host logic)."""

    def __init__(self, seconds_per_cell_step=1e-12, bytes_per_cell=400, clock=time.perf_counter):
        self.spc = seconds_per_cell_step
        self.bpc = bytes_per_cell
        self.clock = clock
        self.resident = {}
        self.serial = 0
        self.steps_taken = collections.Counter()

    def nbytes(self, req, store):
        return int(np.prod(req["grid"])) * self.bpc

    def start_clock(self, t0):
        pass

    def prepare(self, req, store):
        return None

    def create(self, req, store, prepared=None, stream=None):
        self.serial += 1
        m = self.serial
        cells = int(np.prod(req["grid"]))
        self.resident[m] = cells
        return m, cells * self.bpc, 53

    def add(self, m):
        pass

    def step(self, k):
        for key in self.resident:
            self.steps_taken[key] += k
        time.sleep(self.spc * k * sum(self.resident.values()))
        return None

    def wait(self, token):
        pass

    def finish(self, m):
        return (m, self.clock())

    def done(self, h):
        return True

    def finish_time(self, h):
        return h[1]

    def release(self, h):
        self.resident.pop(h[0])

    def run_alone(self, m, steps):
        self.steps_taken[m] += steps
        time.sleep(self.spc * steps * self.resident.pop(m))

    def close(self):
        pass


@dataclass
class Running:
    req: dict
    model: object
    nbytes: int
    record: Record
    done: int = 0
    handle: object = None


def step_bytes(req, store):
    """Algorithmic bytes one time step of a request moves: every population read and written once."""
    q = int(req["lattice"].split("Q")[1].split("-")[0])
    return int(np.prod(req["grid"])) * 2 * q * (4 if store == "f32" else 2)


def serve_batched(requests, engine, budget_bytes=150e9, max_resident=512, tick=64, clock=time.perf_counter,
                  store_policy="as_requested", ahead=1, prepare_depth=16, max_step_bytes=None,
                  large_step_bytes=None):
    """Continuous batching over ``requests`` (sorted by arrival); ``store_policy`` as in
    ``store_for``; ``ahead`` ticks stay queued beyond the one the device runs; the host fields of
    up to ``prepare_depth`` arrived requests are generated ahead of their admission.
    Admission is in arrival order. ``max_step_bytes`` bounds the work of the resident solves per
    batch step (a new arrival waits while it would exceed the bound, unless nothing runs).
    ``large_step_bytes``: a request moving at least that much per step is large; large requests run
    one at a time, in arrival order, and the small ones behind a waiting large one are admitted
    past it (they never delay its admission, which only waits for the running large one), so that
    a large solve shares the device with small ones only and a small one never queues behind a
    large one. Returns the records and the elapsed wall time."""
    pending = collections.deque(sorted(requests, key=lambda r: r["arrival"]))
    prepared = {}
    running, retiring, records = [], [], []
    queued = collections.deque()
    used = 0
    work = 0          # step bytes of the running solves
    peak_used = [0]
    t0 = clock()
    engine.start_clock(t0)
    while pending or running or retiring:
        now = clock() - t0
        # host fields of arrived requests, on worker threads
        for req in list(pending)[:prepare_depth]:
            if req["arrival"] > now:
                break
            if req["rid"] not in prepared:
                prepared[req["rid"]] = engine.prepare(req, store_for(req, store_policy))
        # admission in arrival order while memory and slots allow
        large_running = large_step_bytes is not None and any(
            step_bytes(r.req, r.record.store) >= large_step_bytes for r in running)
        skipped = collections.deque()
        while pending and pending[0]["arrival"] <= now and len(running) < max_resident:
            req = pending[0]
            store = store_for(req, store_policy)
            sb = step_bytes(req, store)
            if large_step_bytes is not None and sb >= large_step_bytes and large_running:
                skipped.append(pending.popleft())   # waits for the running large one; small ones pass
                continue
            if used + engine.nbytes(req, store) > budget_bytes and (running or retiring):
                break          # does not fit yet: admit after a retirement frees memory
            if max_step_bytes is not None and running and work + sb > max_step_bytes:
                break          # the device is busy enough: admit when a running solve finishes
            pending.popleft()
            work += sb
            if large_step_bytes is not None and sb >= large_step_bytes:
                large_running = True
            m, nbytes, q = engine.create(req, store, prepared.pop(req["rid"], None))
            engine.add(m)
            used += nbytes
            rec = Record(req["rid"], req["arrival"], admitted=clock() - t0, steps=req["steps"],
                         cells=int(np.prod(req["grid"])), lattice=req["lattice"], store=store, q=q)
            running.append(Running(req, m, nbytes, rec))
            peak_used[0] = max(peak_used[0], used)
        pending.extendleft(reversed(skipped))        # the waiting large ones keep their places
        # read-backs that have completed: the result is on the host, the memory is free
        still = []
        for r in retiring:
            if engine.done(r.handle):
                r.record.finished = engine.finish_time(r.handle) - t0
                engine.release(r.handle)
                used -= r.nbytes
                records.append(r.record)
            else:
                still.append(r)
        retiring = still
        if running:
            k = min(tick, min(r.req["steps"] - r.done for r in running))
            queued.append(engine.step(k))
            for r in running:
                r.done += k
            still = []
            for r in running:
                if r.done >= r.req["steps"]:
                    r.handle = engine.finish(r.model)
                    retiring.append(r)
                    work -= step_bytes(r.req, r.record.store)
                else:
                    still.append(r)
            running = still
            while len(queued) > ahead:
                engine.wait(queued.popleft())
        elif retiring:
            while queued:
                engine.wait(queued.popleft())
            time.sleep(1e-4)
        elif pending:
            time.sleep(max(0.0, min(pending[0]["arrival"] - (clock() - t0), 0.01)))
    while queued:
        engine.wait(queued.popleft())
    serve_batched.peak_bytes = peak_used[0]
    return records, clock() - t0


def serve_sequential(requests, engine, store="f32", clock=time.perf_counter):
    """One solve at a time in arrival order, FP32, one launch per step."""
    records = []
    t0 = clock()
    for req in sorted(requests, key=lambda r: r["arrival"]):
        now = clock() - t0
        if req["arrival"] > now:
            time.sleep(req["arrival"] - now)
        m, nbytes, q = engine.create(req, store)
        rec = Record(req["rid"], req["arrival"], admitted=clock() - t0, steps=req["steps"],
                     cells=int(np.prod(req["grid"])), lattice=req["lattice"], store=store, q=q)
        engine.run_alone(m, req["steps"])
        rec.finished = clock() - t0
        records.append(rec)
    return records, clock() - t0


def summarize(records, elapsed):
    lat = np.array([r.finished - r.arrival for r in records])
    cell_updates = float(sum(r.cells * r.steps for r in records))
    # algorithmic bytes: every population read once and written once per cell update
    nbytes = float(sum(r.cells * r.steps * 2 * r.q * (4 if r.store == "f32" else 2) for r in records))
    return {
        "solves": len(records),
        "elapsed_s": elapsed,
        "solves_per_s": len(records) / elapsed if elapsed > 0 else float("nan"),
        "latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else float("nan"),
        "latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else float("nan"),
        "mlups": cell_updates / elapsed / 1e6 if elapsed > 0 else float("nan"),
        "algorithmic_gb_per_s": nbytes / elapsed / 1e9 if elapsed > 0 else float("nan"),
    }


def main(argv=None):
    """Serve the seeded request stream (config 5) and print one JSON object with both paths."""
    import argparse
    import json

    from . import autotune
    from . import inputs as I
    ap = argparse.ArgumentParser(description="continuous-batching LB solve server vs the plain FP32 path")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=20.0, help="mean arrivals per second (Poisson)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--tick", type=int, default=64)
    ap.add_argument("--large-step-bytes", type=float, default=5e8,
                    help="requests moving at least this much per step run one at a time (0: no limit)")
    ap.add_argument("--skip-sequential", action="store_true")
    ap.add_argument("--policies", default="f16_dev,as_requested",
                    help="comma-separated storage policies of the batched path")
    a = ap.parse_args(argv)
    reqs = I.serving_requests(a.requests, seed=a.seed, rate_per_s=a.rate)
    tuning = autotune.autotune()
    out = {"requests": a.requests, "rate_per_s": a.rate, "seed": a.seed}
    for policy in a.policies.split(","):
        eng = GpuEngine(tuning=tuning)
        rec_b, t_b = serve_batched(reqs, eng, budget_bytes=a.budget_gb * 1e9, tick=a.tick, store_policy=policy,
                                   large_step_bytes=a.large_step_bytes or None)
        out[f"batched_{policy}"] = dict(summarize(rec_b, t_b), peak_resident_gb=serve_batched.peak_bytes / 1e9,
                                        batched_launches=eng.batch.counters()["launches"])
        eng.close()
    if not a.skip_sequential:
        seq = GpuEngine()
        rec_s, t_s = serve_sequential(reqs, seq, store="f32")
        seq.close()
        out["sequential_fp32"] = summarize(rec_s, t_s)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
