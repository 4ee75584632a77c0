"""Batched and served registrations (execution modes around Algorithm A):
each case's result must be the one cgdir_register gives for it alone, bit for
bit, whether it runs in a batch graph, in a serving slot alone, or among
other requests in flight; and the batched path must still match the FP64
oracle."""
import numpy as np
import pytest

import oracle
import phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1301_0970_gb300 as cg  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def mix(n=6, scale=0.22):
    """Uneven mix of small cases (2-8 masks, four CT shapes shrunk), each
    with its own iteration caps and stopping rule."""
    out = []
    for i, c in enumerate(phantom.batch_mix_cases(n, seed=4100, scale=scale)):
        kw = dict(levels=2, iters=[8 + i, 5 + (i % 3)], lam=c.lam, sign=c.signs,
                  stop_mode=cg.CGDIR_STOP_WINDOW10 if i % 2 else cg.CGDIR_STOP_FIXED, eps=1e-3,
                  contour_level_mask=3 if i % 3 == 0 else 2)
        out.append((c, kw))
    c = phantom.make_case("phantom64", shape=(9, 22, 26))       # a case without masks
    out.append((c, dict(levels=2, iters=[6, 4], lam=[], sign=[], stop_mode=cg.CGDIR_STOP_FIXED)))
    return out


def case_dict(c, kw):
    d = dict(static=dev(c.static), moving=dev(c.moving), **kw)
    if kw.get("lam"):
        d["static_masks"] = [dev(m) for m in c.static_masks]
        d["moving_masks"] = [dev(m) for m in c.moving_masks]
    return d


def single(ctx, c, kw):
    d = case_dict(c, kw)
    return ctx.register(d.pop("static"), d.pop("moving"), d.pop("static_masks", None),
                        d.pop("moving_masks", None), **d)


def submit(ctx, c, kw, **extra):
    d = case_dict(c, kw)
    d.update(extra)
    return ctx.submit(d.pop("static"), d.pop("moving"), d.pop("static_masks", None),
                      d.pop("moving_masks", None), **d)


@pytest.fixture(scope="module")
def cases():
    return mix()


@pytest.fixture(scope="module")
def singles(cases):
    with cg.Context(0) as ctx:
        return [(d.cpu(), st) for d, st in (single(ctx, c, kw) for c, kw in cases)]


@pytest.mark.parametrize("graphs", ["1", "0"])
def test_batch_equals_single_bitwise(cases, singles, graphs, monkeypatch):
    monkeypatch.setenv("CGDIR_GRAPHS", graphs)
    with cg.Context(0) as ctx:
        for _ in range(2):                     # the second call replays the cached batch graph
            res = ctx.register_batch([case_dict(c, kw) for c, kw in cases])
            for (d, st), (d1, st1) in zip(res, singles):
                assert torch.equal(d.cpu(), d1)
                assert st == st1


def test_batch_matches_oracle(cases, singles):
    """The batched results (== the single ones) against the FP64 oracle: DVF
    within 0.05 voxel RMS, the same iteration counts."""
    for (c, kw), (d, st) in list(zip(cases, singles))[:3]:
        ref, rst = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks,
                                   levels=kw["levels"], iters=kw["iters"], lam=kw["lam"], sign=kw["sign"],
                                   contour_mask=kw["contour_level_mask"], stop_mode=kw["stop_mode"],
                                   eps=kw["eps"])
        got = d.numpy().astype(np.float64)
        assert float(np.sqrt(((got - ref) ** 2).sum(axis=0).mean())) <= 0.05
        assert [s["iters_run"] for s in st] == [r["iters_run"] for r in rst]


def test_served_alone_equals_served_in_mix(cases, singles):
    with cg.Context(0) as ctx:
        alone = []
        for c, kw in cases:
            r = submit(ctx, c, kw)
            d, st = ctx.wait(r)
            alone.append((d.cpu(), st))
        ctx.set_max_inflight(len(cases))
        reqs = [submit(ctx, c, kw) for c, kw in cases]
        mixed = [ctx.wait(r) for r in reversed(reqs)][::-1]
        for (a, sa), (m, sm), (s1, ss1) in zip(alone, mixed, singles):
            assert torch.equal(a, s1) and torch.equal(m.cpu(), s1)
            assert sa == sm == ss1


def test_submit_refuses_when_every_slot_is_busy(cases):
    c, kw = cases[0]
    with cg.Context(0) as ctx:
        ctx.set_max_inflight(2)
        a, b = submit(ctx, c, kw), submit(ctx, c, kw)
        with pytest.raises(cg.CgdirError) as e:
            submit(ctx, c, kw)
        assert e.value.status == cg.CGDIR_EBUSY
        da, _ = ctx.wait(a)
        d3 = ctx.wait(submit(ctx, c, kw))[0]      # a slot is free again
        db, _ = ctx.wait(b)
        assert torch.equal(da, db) and torch.equal(da, d3)


def test_wait_timeout_leaves_the_request_in_flight():
    c = phantom.make_case("headneck256", shape=(40, 128, 128))
    kw = dict(levels=1, iters=[150], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED)
    with cg.Context(0) as ctx:
        r = submit(ctx, c, kw)
        with pytest.raises(cg.CgdirError) as e:
            ctx.wait(r, timeout_ms=0)
        assert e.value.status == cg.CGDIR_ETIMEDOUT
        d, st = ctx.wait(r)
        ref, _ = single(ctx, c, kw)
        assert torch.equal(d, ref) and st[0]["iters_run"] == 150


def test_pageable_host_output_is_written_at_collection(cases, singles):
    c, kw = cases[1]
    with cg.Context(0) as ctx:
        out = torch.empty((3,) + tuple(c.static.shape), dtype=torch.float32)       # pageable
        r = submit(ctx, c, kw, dvf_out=out)
        d, _ = ctx.wait(r)
        assert d.data_ptr() == out.data_ptr()
        assert torch.equal(out, singles[1][0])


def test_cancel_frees_the_slot():
    c = phantom.make_case("headneck256", shape=(40, 128, 128))
    kw = dict(levels=1, iters=[400], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED)
    small = dict(levels=1, iters=[5], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED)
    with cg.Context(0) as ctx:
        ctx.set_max_inflight(1)
        r = submit(ctx, c, kw)
        ctx.cancel(r)
        d, st = ctx.wait(submit(ctx, c, small))
        ref, rst = single(ctx, c, small)
        assert torch.equal(d, ref) and st == rst


def test_budget_admission_returns_busy_then_admits(cases):
    c, kw = cases[2]
    with cg.Context(0) as probe:
        probe.wait(submit(probe, c, kw))
        one = probe.mem_in_use()
    with cg.Context(0, mem_budget_bytes=int(one * 1.5)) as ctx:
        a = submit(ctx, c, kw)
        with pytest.raises(cg.CgdirError) as e:
            submit(ctx, c, kw)                   # a second slot's buffers would exceed the budget
        assert e.value.status == cg.CGDIR_EBUSY
        da, _ = ctx.wait(a)
        db, _ = ctx.wait(submit(ctx, c, kw))     # reuses the first slot's buffers
        assert torch.equal(da, db)


def test_autotune_records_every_level_and_keeps_results():
    """The autotuner picks launch geometry only: a registration after tuning
    gives the same DVF, bit for bit, as an untuned context (FIXED stopping)."""
    c = phantom.make_case("headneck256", shape=(24, 96, 96))
    kw = dict(levels=3, iters=[6, 4, 3], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED)
    with cg.Context(0) as plain:
        ref, rst = single(plain, c, kw)
    with cg.Context(0) as ctx:
        tab = ctx.autotune(c.shape, c.k, 3)
        assert len(tab) == 3
        assert {t["shape"] for t in tab} == {(6, 24, 24), (12, 48, 48), (24, 96, 96)}
        for t in tab:
            assert t["smooth"] in ("march", "tile", "split", "fused") and t["force_zchunk"] >= 1
            assert t["smooth_ms"] > 0 and t["force_ms"] > 0
            assert t["smooth_ms"] + t["force_ms"] <= (t["default_smooth_ms"] + t["default_force_ms"]) * 1.0001 + 1e-6
        got, st = single(ctx, c, kw)
        assert torch.equal(got, ref)
        assert [s["iters_run"] for s in st] == [s["iters_run"] for s in rst]


def test_tuning_table_round_trip():
    """A tuning table read from one context (and through JSON) installs in
    another: the same choices, the same DVF bit for bit, no timing run; bad
    entries are refused and install nothing."""
    import json
    c = phantom.make_case("phantom64", shape=(16, 40, 44))
    kw = dict(levels=2, iters=[5, 4], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED)
    with cg.Context(0) as a:
        tab = a.autotune(c.shape, c.k, 2)
        ra, _ = single(a, c, kw)
    tab2 = json.loads(json.dumps(tab))
    with cg.Context(0) as b:
        b.load_tuning(tab2)
        got = b.tuning()
        key = lambda t: (tuple(t["shape"]), t["contour"], t["storage_dtype"])
        choice = lambda t: (key(t), t["smooth"], t["smooth_zchunk"], t["force_zchunk"], t["force_width"])
        assert sorted(choice(t) for t in got) == sorted(choice(t) for t in tab)
        rb, _ = single(b, c, kw)
        assert torch.equal(ra, rb)
        for bad in (dict(tab2[0], force_zchunk=0), dict(tab2[0], force_width=3)):
            with pytest.raises(cg.CgdirError):
                b.load_tuning([bad])
        assert len(b.tuning()) == len(tab)


@pytest.mark.parametrize("smooth, force_width", [("march32", 0), ("march", 2), ("march32", 2), ("tile", 0)])
def test_every_tuned_variant_and_pass2_width_gives_the_same_bits(smooth, force_width):
    """Tables naming the 32 x 16 z-march (at a short z chunk), the two-voxel
    pass 2 or the tile smoothing, installed in a context: the registration
    equals an untuned context's bit for bit (a schedule picks kernels, never
    results)."""
    c = phantom.make_case("headneck256", shape=(20, 48, 64))
    kw = dict(levels=2, iters=[6, 5], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED)
    with cg.Context(0) as a:
        ref, _ = single(a, c, kw)
        tab = a.autotune(c.shape, c.k, 2)
    forced = [dict(t, smooth=smooth, smooth_zchunk=3 if smooth != "tile" else 0, force_width=force_width,
                   force_zchunk=max(1, t["force_zchunk"]))
              for t in tab]
    with cg.Context(0) as b:
        b.load_tuning(forced)
        assert all(t["smooth"] == smooth and t["force_width"] == force_width for t in b.tuning())
        got, _ = single(b, c, kw)
    assert torch.equal(ref, got)


def test_shared_gpu_registrations_take_the_per_step_schedule():
    """Where the fused schedule won the tuning, cgdir_register uses it and a
    batch (whose branches share the GPU) the per-step kernels: more launches
    per iteration, the same DVF bit for bit."""
    c = phantom.make_case("headneck256", shape=(24, 64, 64))
    kw = dict(levels=1, iters=[12], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED, contour_level_mask=1)
    with cg.Context(0) as ctx:
        tab = ctx.autotune(c.shape, c.k, 1, contour_level_mask=1)
        single(ctx, c, kw)                       # capture the graphs first
        ctx.register_batch([case_dict(c, kw)])
        n0 = cg.launch_count()
        a, _ = single(ctx, c, kw)
        n1 = cg.launch_count()
        (b, _), = ctx.register_batch([case_dict(c, kw)])
        n2 = cg.launch_count()
    assert torch.equal(a, b)
    if tab[0]["smooth"] == "fused":
        # per iteration after the first: 3 kernels fused, at least 5 per step
        assert (n2 - n1) - (n1 - n0) >= 2 * (12 - 1)


def test_autotune_on_first_use():
    c = phantom.make_case("phantom64", shape=(16, 40, 44))
    kw = dict(levels=2, iters=[5, 4], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED)
    with cg.Context(0) as ctx:
        ctx.set_autotune(True)
        a, _ = single(ctx, c, kw)
        assert len(ctx.tuning()) == 2
        b, _ = single(ctx, c, kw)
        assert torch.equal(a, b)


def _ctx_with_env(env):
    import os
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return cg.Context(0)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("stop", [cg.CGDIR_STOP_FIXED, cg.CGDIR_STOP_WINDOW10])
def test_cooperative_level_kernel_matches_per_iteration_kernels(stop):
    """Small levels run as one cooperative launch (all iterations, grid
    barriers between phases) with the arithmetic of the per-iteration
    kernels: the same DVF bit for bit, and histories equal to FP32
    summation order."""
    c = phantom.make_case("headneck256", shape=(40, 120, 124))
    kw = dict(levels=3, iters=[30, 20, 4], lam=c.lam, sign=c.signs, stop_mode=stop, eps=1e-3,
              contour_level_mask=3)
    base = _ctx_with_env({})
    coop = _ctx_with_env({"CGDIR_COOP_MAX": str(10 ** 7)})
    try:
        a, sa = single(base, c, kw)
        b, sb = single(coop, c, kw)
        coop.profile([cg.CGDIR_K_LEVEL])
        single(coop, c, kw)
        prof = coop.profile_read()
    finally:
        base.close()
        coop.close()
    assert {p["level"] for p in prof if p["kernel"] == "level"} == {0, 1}
    assert [s["iters_run"] for s in sa] == [s["iters_run"] for s in sb]
    for x, y in zip(sa, sb):
        np.testing.assert_allclose(x["rms_id"], y["rms_id"], rtol=1e-6)
    if stop == cg.CGDIR_STOP_FIXED:
        assert torch.equal(a, b)
    else:
        assert float((a - b).abs().max()) <= 1e-4


@pytest.mark.parametrize("variant", ["split", "tile", "fused", "march32"])
def test_smoothing_variants_give_the_same_registration(variant):
    """Every smoothing variant (incl. the split kernels with the composite
    update in the z pass, the fused schedule: 3-D tiles of G(du) with the
    update, 3-D tiles of G(u') with the next warp, the force's stencil pass
    alone, and the 32 x 16 z-march) gives the same DVF as the wide-tile
    z-march, bit for bit."""
    c = phantom.make_case("headneck256", shape=(24, 72, 80))     # nx % 8 == 0: the wide-tile z-march
    kw = dict(levels=2, iters=[6, 5], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED, contour_level_mask=3)
    a_ctx = _ctx_with_env({"CGDIR_SMOOTH": "march"})
    b_ctx = _ctx_with_env({"CGDIR_SMOOTH": variant})
    try:
        a, _ = single(a_ctx, c, kw)
        b, _ = single(b_ctx, c, kw)
    finally:
        a_ctx.close()
        b_ctx.close()
    assert torch.equal(a, b)


@pytest.mark.parametrize("contour", [True, False])
def test_force_pass_variants_agree_bitwise(contour):
    """Pass 2 with one, two and four voxels per thread, at several z chunks:
    the same du, bit for bit (the per-voxel arithmetic is one function with
    every multiply-add written out); the RMS-ID sums agree to rounding."""
    c = phantom.make_case("headneck256", shape=(20, 48, 64))
    bits = lambda m: dev(np.bitwise_or.reduce([(x.astype(np.uint8) << j) for j, x in enumerate(m)], axis=0))
    I0, T0, mb, sb = dev(c.moving), dev(c.static), bits(c.moving_masks), bits(c.static_masks)
    u = dev((0.5 * c.u_gt).astype(np.float32))
    outs = []
    for env in ({"CGDIR_FORCE_WIDTH": "1", "CGDIR_FORCE_ZCHUNK": "1"}, {"CGDIR_FORCE_WIDTH": "1", "CGDIR_FORCE_ZCHUNK": "5"},
                {"CGDIR_FORCE_WIDTH": "2", "CGDIR_FORCE_ZCHUNK": "1"}, {"CGDIR_FORCE_WIDTH": "2", "CGDIR_FORCE_ZCHUNK": "4"},
                {"CGDIR_FORCE_ZCHUNK": "1"}, {"CGDIR_FORCE_ZCHUNK": "3"}):
        ctx = _ctx_with_env(env)
        try:
            du, st = ctx.force(I0, T0, mb, sb, c.lam, c.signs, u, contour=contour, want_stats=True)
            outs.append((du.cpu(), st))
        finally:
            ctx.close()
    for du, st in outs[1:]:
        assert torch.equal(du, outs[0][0])
        assert st[1] == outs[0][1][1]
        assert abs(st[0] - outs[0][1][0]) <= 1e-9 * outs[0][1][0]


@pytest.mark.parametrize("shape, kw", [
    # odd nx (one voxel per thread in the force pass), ragged 8-voxel tiles in x, y and z
    ((13, 37, 45), dict(levels=2, iters=[7, 5], stop_mode=cg.CGDIR_STOP_WINDOW10, eps=1e-3)),
    # additive update, wider and narrower Gaussians (radii 5 and 2), structure terms at both levels
    ((20, 40, 48), dict(levels=2, iters=[6, 4], compose_mode=cg.CGDIR_ADDITIVE, sigma_fluid=1.6,
                        sigma_diff=0.6, contour_level_mask=3, stop_mode=cg.CGDIR_STOP_FIXED)),
    # 16-bit image storage, three levels down to a 5 x 10 x 12 level
    ((20, 40, 48), dict(levels=3, iters=[8, 5, 3], storage_dtype=cg.CGDIR_F16, stop_mode=cg.CGDIR_STOP_FIXED)),
])
def test_fused_schedule_matches_per_step_kernels(shape, kw):
    """The fused schedule against the per-step kernels (tile smoothing, the
    separate update kernel, the force's warp pass) on awkward shapes and
    parameters: the same DVF and histories, bit for bit."""
    c = phantom.make_case("headneck256", shape=shape)
    kw = dict(kw, lam=c.lam, sign=c.signs)
    a_ctx = _ctx_with_env({"CGDIR_SMOOTH": "tile"})
    b_ctx = _ctx_with_env({"CGDIR_SMOOTH": "fused"})
    try:
        a, sa = single(a_ctx, c, kw)
        b, sb = single(b_ctx, c, kw)
    finally:
        a_ctx.close()
        b_ctx.close()
    assert torch.equal(a, b)
    assert [s["iters_run"] for s in sa] == [s["iters_run"] for s in sb]
    for x, y in zip(sa, sb):
        assert np.array_equal(x["rms_id"], y["rms_id"])


def test_fused_schedule_matches_oracle():
    """A whole registration on the fused schedule against the FP64 oracle:
    the same bar as the per-step path (DVF within 0.05 voxel RMS, the same
    iteration counts)."""
    c = phantom.make_case("headneck256", shape=(14, 30, 34))
    kw = dict(levels=2, iters=[10, 6], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_WINDOW10, eps=1e-3,
              contour_level_mask=3)
    ctx = _ctx_with_env({"CGDIR_SMOOTH": "fused"})
    try:
        got, st = single(ctx, c, kw)
    finally:
        ctx.close()
    ref, rst = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=2, iters=[10, 6],
                               lam=c.lam, sign=c.signs, contour_mask=3, stop_mode=cg.CGDIR_STOP_WINDOW10, eps=1e-3)
    got = got.cpu().numpy().astype(np.float64)
    assert float(np.sqrt(((got - ref) ** 2).sum(axis=0).mean())) <= 0.05
    assert [s["iters_run"] for s in st] == [r["iters_run"] for r in rst]


def test_device_wait_that_runs_out_reports_a_timeout_and_the_context_stays_usable():
    """A kernel waits on a barrier that nothing completes (20 ms limit): the
    call returns ETIMEDOUT, the error word is cleared, and the same context
    then registers a case with the same result as a fresh one."""
    c = phantom.make_case("phantom64", shape=(10, 20, 24))
    kw = dict(levels=2, iters=[4, 3], lam=c.lam, sign=c.signs, stop_mode=cg.CGDIR_STOP_FIXED)
    with cg.Context(0) as fresh:
        ref, _ = single(fresh, c, kw)
    with cg.Context(0) as ctx:
        assert ctx.selftest_wait_timeout(20000) == cg.CGDIR_ETIMEDOUT
        assert ctx.selftest_wait_timeout(0) == cg.CGDIR_EINVAL
        got, _ = single(ctx, c, kw)
        assert torch.equal(got, ref)
        assert ctx.selftest_wait_timeout(1000) == cg.CGDIR_ETIMEDOUT
