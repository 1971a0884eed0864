"""Host logic of the serving loops (admission, ticks, retirement, accounting) on the CPU with the
fake engine: every request runs exactly its steps, arrivals are admitted in order, the memory
budget and the slot limit hold, and the summary is consistent."""
import numpy as np

from paper_2512_16230_gb300 import inputs as I
from paper_2512_16230_gb300 import serve as S


def _requests(n=40, rate=400.0):
    return I.serving_requests(n, seed=3, rate_per_s=rate, steps=(5, 40), side2d=(8, 32), ny2d=(8, 32),
                              side3d=(8, 16))


def test_request_stream_is_seeded_and_shaped():
    a = I.serving_requests(200, seed=7)
    b = I.serving_requests(200, seed=7)
    assert a == b
    arr = np.array([r["arrival"] for r in a])
    assert np.all(np.diff(arr) > 0)
    assert {r["lattice"] for r in a} <= set(I.SERVING_2D + I.SERVING_3D)
    for r in a:
        assert 200 <= r["steps"] <= 5000
        if len(r["grid"]) == 3:
            assert 32 <= r["grid"][0] <= 160 and r["flow"] == "kolmogorov"
        else:
            assert 32 <= r["grid"][0] <= 1024 and 32 <= r["grid"][1] <= 768


def test_batched_loop_runs_every_step_and_respects_limits():
    reqs = _requests()
    eng = S.FakeEngine(seconds_per_cell_step=2e-9, bytes_per_cell=100)
    budget = 3 * 32 * 32 * 100
    seen = []
    orig_add = eng.add

    def add(m):
        seen.append(len(eng.resident))
        orig_add(m)
    eng.add = add
    recs, elapsed = S.serve_batched(reqs, eng, budget_bytes=budget, max_resident=4, tick=7)
    assert sorted(r.rid for r in recs) == [r["rid"] for r in reqs]
    assert max(seen) <= 4
    largest = max(eng.nbytes(r, "f32") for r in reqs)
    # over-budget requests are only admitted alone (otherwise they would starve)
    assert S.serve_batched.peak_bytes <= max(budget, largest)
    for r in recs:
        assert r.arrival <= r.admitted <= r.finished <= elapsed
    by_rid = {r["rid"]: r for r in reqs}
    # every model ran exactly its requested number of steps
    assert sorted(eng.steps_taken.values()) == sorted(by_rid[r.rid]["steps"] for r in recs)
    # admission follows arrival order
    adm = sorted(recs, key=lambda r: r.admitted)
    assert [r.rid for r in adm] == sorted(r.rid for r in recs)


def test_sequential_loop_and_summary():
    reqs = _requests(n=12)
    eng = S.FakeEngine(seconds_per_cell_step=1e-9)
    recs, elapsed = S.serve_sequential(reqs, eng)
    assert [r.rid for r in recs] == [r["rid"] for r in reqs]
    s = S.summarize(recs, elapsed)
    assert s["solves"] == 12
    assert s["latency_p50_s"] <= s["latency_p99_s"]
    assert s["solves_per_s"] == 12 / elapsed
    cells = sum(np.prod(r["grid"]) * r["steps"] for r in reqs)
    assert abs(s["mlups"] - cells / elapsed / 1e6) < 1e-9 * s["mlups"]


def test_storage_policy():
    """The serving policies: FP32 requests stay FP32 under "as_requested"; under both policies a
    16-bit request is stored as FP16 deviations only while its run is no longer than its class's
    FP16 threshold (F16_MAX_STEPS), FP32 otherwise; any other policy is a storage name."""
    assert len(S.SERVING_CLASSES) == 9 and set(S.F16_MAX_STEPS) == set(S.SERVING_CLASSES)
    for flow, lat in S.SERVING_CLASSES:
        top = S.F16_MAX_STEPS[flow, lat]
        for steps in (max(top, 1), top + 1):
            for store in ("f32", "16bit"):
                req = dict(flow=flow, lattice=lat, store=store, steps=steps)
                f16 = "f16_dev" if steps <= top else "f32"
                assert S.store_for(req, "as_requested") == ("f32" if store == "f32" else f16)
                assert S.store_for(req, "f16_dev") == f16
                assert S.store_for(req, "bf16_dev") == "bf16_dev"


def test_step_work_bound_admits_in_order():
    """With a bound on the resident step work (a request waits while it would exceed the bound,
    unless nothing runs), every request still completes and admission stays in arrival order."""
    reqs = _requests(n=30, rate=1e4)
    eng = S.FakeEngine(seconds_per_cell_step=1e-9)
    bound = max(S.step_bytes(r, "f32") for r in reqs)
    recs, _ = S.serve_batched(reqs, eng, budget_bytes=1e12, tick=5, store_policy="f32", max_step_bytes=bound)
    assert sorted(r.rid for r in recs) == [r["rid"] for r in reqs]
    adm = sorted(recs, key=lambda r: r.admitted)
    assert [r.rid for r in adm] == sorted(r.rid for r in recs)
    assert S.step_bytes(dict(lattice="rD3Q53-cubic", grid=(10, 10, 10)), "f32") == 1000 * 2 * 53 * 4
    assert S.step_bytes(dict(lattice="rD2Q17", grid=(10, 20)), "f16_dev") == 200 * 2 * 17 * 2


def test_large_requests_run_one_at_a_time():
    """With a large-request threshold, at most one large request steps at a time, small requests
    behind a waiting large one are admitted past it, every request completes, and the large ones
    start in their arrival order."""
    reqs = _requests(n=40, rate=1e4)
    sizes = sorted(S.step_bytes(r, "f32") for r in reqs)
    large = sizes[len(sizes) * 3 // 4]
    eng = S.FakeEngine(seconds_per_cell_step=2e-9)
    live, peak = [], [0]
    by_model = {}
    orig_create, orig_finish = eng.create, eng.finish

    def create(req, store, prepared=None, stream=None):     # a solve starts stepping
        m, nb, q = orig_create(req, store, prepared, stream)
        by_model[m] = S.step_bytes(req, store) >= large
        live.append(m)
        peak[0] = max(peak[0], sum(by_model[x] for x in live))
        return m, nb, q

    def finish(m):                                           # ... and stops stepping
        live.remove(m)
        return orig_finish(m)
    eng.create, eng.finish = create, finish
    recs, _ = S.serve_batched(reqs, eng, budget_bytes=1e12, tick=5, store_policy="f32", large_step_bytes=large)
    assert sorted(r.rid for r in recs) == [r["rid"] for r in reqs]
    assert peak[0] == 1
    big = [r for r in sorted(recs, key=lambda r: r.admitted) if S.step_bytes(
        dict(lattice=r.lattice, grid=next(q["grid"] for q in reqs if q["rid"] == r.rid)), "f32") >= large]
    assert [r.rid for r in big] == sorted(r.rid for r in big)
