"""The batched engine (lbm_batch_*, persistent kernel over a tile work-list, CUDA-graph steps)
gives the same solves as the single-solve path and as the oracle, whatever the mix."""
import numpy as np
import pytest

from paper_2512_16230_gb300 import inputs as I
from paper_2512_16230_gb300 import workloads as W

from _harness import gpu_model, oracle_model, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _lib(lbm_lib):
    return lbm_lib


# (lattice, eq, grid, store): several groups, ragged tiles, 2D and 3D, NSE with force and NCDE
MIX = [
    ("rD2Q25", "nse", (37, 29), "f32"),
    ("rD2Q25", "nse", (20, 41), "f32"),
    ("rD2Q17", "ncde", (33, 40), "f32"),
    ("rD2Q21", "nse", (31, 17), "f16_dev"),
    ("rD3Q53-cubic", "nse", (13, 11, 9), "f32"),
    ("rD3Q45", "nse", (12, 10, 8), "f16_dev"),
    ("rD3Q33", "nse", (10, 9, 8), "bf16_dev"),
    ("rD3Q53", "nse", (9, 10, 11), "f32"),
]


def _make(lat_cache, name, eq, n, store, seed):
    from paper_2512_16230_gb300 import lbm
    spec = W.LATTICES[name]
    if name not in lat_cache:
        lat_cache[name] = lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w)
    lat = lat_cache[name]
    s = np.random.default_rng(seed).uniform(0.8, 1.8, spec.R)
    d = spec.d
    kw = {}
    if eq == "nse":
        kw["force"] = (0, d - 1, 2e-4, 1, 0.3)
    else:
        kw["u_const"] = tuple([0.03, 0.02, 0.01][:d])
        kw["nonlin"] = 1.0
    m = gpu_model(spec, eq, n, s, 1.1, store=store, lat=lat, **kw)
    if eq == "nse":
        rho, u = I.random_fields(n, d, seed=seed, rho_amp=0.01, u_amp=0.03)
        m.init_fields(rho, u)
    else:
        m.init_fields(I.gaussian_hill(n, spec.c, max(2.0, n[0] / 6), 1.0, noise=1e-3, seed=seed))
    return m


def _compare(a, b, store):
    ra, ua = a.read_fields()
    rb, ub = b.read_fields()
    tol = 1e-6 if store == "f32" else 2e-3
    assert rel_l2(ra, rb) <= tol
    if ua is not None:
        assert rel_l2(ua, ub) <= tol
    return np.array_equal(ra, rb) and (ua is None or np.array_equal(ua, ub))


def test_batch_solos_equal_single_solve_path():
    """Members above the solo threshold run on the single-solve kernels inside the batch (here a
    low threshold makes the larger half of the mix solos, 16-bit storage with n_x % 8 == 0 on the
    row-staged kernel among them; they step on their own stream beside the groups' streams): every
    member is bitwise the same as the same solve alone, and the step counters count each solo step
    once."""
    from paper_2512_16230_gb300 import lbm
    mix = MIX + [("rD3Q53", "nse", (16, 10, 9), "f16_dev"), ("rD2Q17", "ncde", (24, 20), "bf16_dev")]
    cache = {}
    alone = [_make(cache, *spec, seed=i) for i, spec in enumerate(mix)]
    batched = [_make(cache, *spec, seed=i) for i, spec in enumerate(mix)]
    b = lbm.Batch(64)
    b.set_solo_threshold(1000)
    for m in batched:
        b.add(m)
    b.step(13)
    b.step(11)          # stable membership: the groups from the captured graph, the solos beside them
    b.synchronize()
    for m in alone:
        m.step(24)
    assert [m.counters()[0] for m in batched] == [24] * len(mix)
    exact = [_compare(x, y, spec[3]) for x, y, spec in zip(alone, batched, mix)]
    assert all(exact)
    b.close()


def test_batch_equals_single_solve_path():
    from paper_2512_16230_gb300 import lbm
    cache = {}
    alone = [_make(cache, *spec, seed=i) for i, spec in enumerate(MIX)]
    batched = [_make(cache, *spec, seed=i) for i, spec in enumerate(MIX)]
    b = lbm.Batch(64)
    for m in batched:
        b.add(m)
    b.step(13)          # the call after a change: direct launches (13, odd: the buffers swap)
    b.step(19)          # membership stable: captured graph (one branch per group) twice, then 3 direct
    b.synchronize()
    for m in alone:
        m.step(32)
    c = b.counters()
    assert c["groups"] == len({(name, st) for name, _, _, st in MIX}) and c["steps"] == 32
    exact = [_compare(x, y, spec[3]) for x, y, spec in zip(alone, batched, MIX)]
    assert all(exact)   # the same per-cell code: bitwise the same fields
    # membership changes: drop two solves, add a fresh one, keep stepping
    b.remove(batched[1])
    b.remove(batched[4])
    extra_alone = _make(cache, "rD3Q33", "nse", (8, 8, 8), "f32", seed=99)
    extra_batched = _make(cache, "rD3Q33", "nse", (8, 8, 8), "f32", seed=99)
    b.add(extra_batched)
    b.step(10)
    b.synchronize()
    for i, m in enumerate(alone):
        if i not in (1, 4):
            m.step(10)
    extra_alone.step(10)
    for i, (x, y, spec) in enumerate(zip(alone, batched, MIX)):
        if i not in (1, 4):
            _compare(x, y, spec[3])
    _compare(extra_alone, extra_batched, "f32")
    # the removed members kept their state and can be stepped alone again
    batched[1].step(3)
    alone[1].step(3)
    _compare(alone[1], batched[1], "f32")
    print("bit-identical to the single-solve path:", exact)
    b.close()


def test_model_in_batch_is_advanced_only_by_the_batch():
    from paper_2512_16230_gb300 import lbm
    m = _make({}, "rD2Q13", "nse", (16, 12), "f32", seed=1)
    b = lbm.Batch(4)
    b.add(m)
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        m.step(1)
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        b.add(m)
    b.close()
    m.step(1)


def test_batched_solve_against_the_oracle():
    """A Kolmogorov flow (rD3Q45, forced through M2G) advanced in a batch with other solves,
    against the FP64 oracle: FP32 parity bound 1e-5."""
    from paper_2512_16230_gb300 import lbm
    wl = W.kolmogorov_3d(lattice="rD3Q45", n=(12, 16, 10), steps=40, store="f32")
    om = oracle_model(wl.lattice, wl.eq, wl.n, wl.s, wl.s_high, force=wl.force)
    gm = gpu_model(wl.lattice, wl.eq, wl.n, wl.s, wl.s_high, force=wl.force, store="f32")
    rho, u = wl.fields()
    om.init_fields(rho, u)
    gm.init_fields(rho, u)
    other = _make({}, "rD3Q45", "nse", (9, 9, 9), "f32", seed=5)
    b = lbm.Batch(4)
    b.add(gm)
    b.add(other)
    b.step(wl.steps)
    b.synchronize()
    om.step(wl.steps)
    assert rel_l2(gm.get_populations(), om.f) <= 1e-5
    b.close()


@pytest.mark.parametrize("policy", ["as_requested", "f16_dev"])
def test_serving_results_same_alone_and_in_the_mix(policy):
    """Continuous batching: every request of a small seeded mix, served together with the others
    (admitted and retired while others run, ticks of 16 steps, graph replays), gives bitwise the
    fields of the same request run alone in the storage the policy gives it -- the batched kernel
    runs the single-solve per-cell code, so nothing of the mix may leak into a result."""
    from paper_2512_16230_gb300 import serve as S
    reqs = I.serving_requests(24, seed=11, rate_per_s=2000.0, steps=(20, 90), side2d=(16, 48), ny2d=(16, 40),
                              side3d=(8, 20))
    mixed = S.GpuEngine(keep_results=True)
    recs, _ = S.serve_batched(reqs, mixed, tick=16, store_policy=policy)
    assert len(recs) == len(reqs)
    stores = {r.rid: r.store for r in recs}
    assert all(stores[q["rid"]] == S.store_for(q, policy) for q in reqs)
    alone = S.GpuEngine(keep_results=True)
    for req in reqs:
        m, _, _ = alone.create(req, S.store_for(req, policy))
        alone.run_alone(m, req["steps"])
    for req in reqs:
        a, b = alone.results[req["rid"]], mixed.results[req["rid"]]
        assert np.array_equal(b[0], a[0]), req
        if a[1] is not None:
            assert np.array_equal(b[1], a[1]), req


# (lattice, eq, grid, store, settings): the model settings beyond the base scheme inside a batch
VARIANTS = [
    ("rD2Q13", "ncde", (33, 27), "f32", dict(ncde_mode="rate", a1=-0.3)),
    ("rD2Q25", "ncde", (29, 31), "f32", dict(ncde_mode="cde")),
    ("rD2Q17", "ncde", (30, 26), "f16_dev", dict(ncde_mode="moment", a1=0.4, a2=0.05)),
    ("rD2Q13", "ncde", (25, 24), "f32", dict(ncde_mode="rate", a2=-0.04)),
    ("rD2Q9", "nse", (37, 29), "f32", dict(m2g_aniso=True)),
    ("rD3Q27", "nse", (13, 11, 9), "f16_dev", dict(m2g_aniso=True)),
    ("rD3Q27", "nse", (9, 12, 10), "f32", dict(m2g_aniso=True, s_bulk=0.9)),
    ("rD2Q25", "nse", (27, 22), "f32", dict(s_orders={4: 0.9, 5: 1.3, 6: 1.6})),
    ("rD3Q53", "nse", (11, 9, 10), "f16_dev", dict(s_orders={4: 0.8, 5: 1.35, 6: 1.6, 7: 0.9, 8: 1.25})),
    ("rD2Q13", "ncde", (26, 21), "f32", dict(ncde_mode="rate", s_orders={4: 1.4, 5: 0.7})),
]


def _make_variant(lat_cache, name, eq, n, store, settings, seed):
    from paper_2512_16230_gb300 import lbm
    spec = W.LATTICES[name]
    if name not in lat_cache:
        lat_cache[name] = lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w)
    s = np.random.default_rng(seed).uniform(0.8, 1.8, spec.R)
    d = spec.d
    kw = dict(settings)
    if "a2" in kw:
        kw["psi"] = I.random_scalar(n, seed=seed + 50)
    if eq == "nse":
        kw["force"] = (0, d - 1, 2e-4, 1, 0.3)
    else:
        kw["u_const"] = tuple([0.03, 0.02, 0.01][:d])
        kw["nonlin"] = 0.0 if kw.get("ncde_mode") == "cde" else 1.0
    m = gpu_model(spec, eq, n, s, 1.1, store=store, lat=lat_cache[name], **kw)
    if store != "f64":
        m.set_tensor_cores(0)   # batched solves run on the CUDA cores; compare like with like
    if eq == "nse":
        rho, u = I.random_fields(n, d, seed=seed, rho_amp=0.01, u_amp=0.03)
        m.init_fields(rho, u)
    else:
        m.init_fields(I.gaussian_hill(n, spec.c, max(2.0, n[0] / 6), 1.0, noise=1e-3, seed=seed))
    return m


def test_batch_carries_model_variants():
    """The NCDE variants (per-cell rates, CDE, mixed derivative), the cross-diffusion term, the
    delta4 term of M2G with its density history and per-order rates (their own groups, with the
    higher-row table staged per solve), in one batch: after 13 steps (one graph replay and an odd
    remainder, so the populations and the density history swap) and 9 more, every member equals
    the same model stepped alone; changing a member's per-order rates moves it between groups."""
    from paper_2512_16230_gb300 import lbm
    cache = {}
    alone = [_make_variant(cache, *v, seed=10 + i) for i, v in enumerate(VARIANTS)]
    batched = [_make_variant(cache, *v, seed=10 + i) for i, v in enumerate(VARIANTS)]
    b = lbm.Batch(16)
    for m in batched:
        b.add(m)
    b.step(13)
    b.synchronize()
    for m in alone:
        m.step(13)
    for x, y, v in zip(alone, batched, VARIANTS):
        _compare(x, y, v[3])
    b.step(9)
    b.synchronize()
    for m in alone:
        m.step(9)
    for x, y, v in zip(alone, batched, VARIANTS):
        _compare(x, y, v[3])
    for m in (alone[0], batched[0]):
        m.set_high_rates([1.2, 0.8])
    b.step(5)
    b.synchronize()
    for m in alone:
        m.step(5)
    for x, y, v in zip(alone, batched, VARIANTS):
        _compare(x, y, v[3])
    b.close()


# 16-bit storage, with minimal grids (every x access wraps), the gradient terms and an NCDE
# variant: the single-solve kernel and the batched engine run the same per-cell code
BITWISE = [
    ("rD2Q25", "nse", (38, 29), "f16_dev", {}),
    ("rD2Q25", "nse", (6, 7), "bf16_dev", {}),           # n_x = 2 R_max
    ("rD2Q13", "ncde", (40, 22), "f16_dev", dict(ncde_mode="rate", a2=0.05)),
    ("rD3Q53", "nse", (14, 11, 9), "f16_dev", {}),
    ("rD3Q53", "nse", (4, 5, 6), "bf16_dev", {}),
    ("rD3Q27", "nse", (12, 9, 7), "f16_dev", dict(m2g_aniso=True)),
    ("rD2Q9", "nse", (2, 5), "bf16_dev", dict(m2g_aniso=True)),
]


def test_batch_bitwise_equals_single_solve_16bit():
    """For 16-bit storage the batched engine gives bitwise the populations of the single-solve
    kernel over 7 steps (odd: the buffers swap), with the gradient terms and an NCDE variant."""
    from paper_2512_16230_gb300 import lbm
    cache = {}
    alone = [_make_variant(cache, *v, seed=30 + i) for i, v in enumerate(BITWISE)]
    batched = [_make_variant(cache, *v, seed=30 + i) for i, v in enumerate(BITWISE)]
    b = lbm.Batch(16)
    for m in batched:
        b.add(m)
    b.step(7)
    b.synchronize()
    for m in alone:
        m.step(7)
    for x, y, v in zip(alone, batched, BITWISE):
        assert np.array_equal(x.get_populations(), y.get_populations()), v
    b.close()
