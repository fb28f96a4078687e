"""Failure paths of the library and of the serving loop, made on the host: a structure that
outgrows the neighbour list, one beyond the ACE-neighbour limit, and device allocations that
fail through the library's own injection hook (ap_inject_alloc_failures).  None of them faults
the GPU: every device-side limit is a bounded write plus a flag that the next synchronising
call reports."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    ap.build()
    return ap


def _ctx(ap, c, x=None, box=None, region=None):
    return ap.APContext(c["eam"], c["ace"], c["box"] if box is None else box, c["x"] if x is None else x, None, None,
                        region, None, None, c["mass"])


def _scaled(c, s):
    box = dict(c["box"])
    box["h"] = np.asarray(c["box"]["h"], dtype=np.float64) * s
    return c["x"] * s, box


def test_list_capacity_overflow_grows_and_matches_a_fresh_context(apl, orc):
    from paper_2505_12958_gb300._capi import AP_ERR_CAPACITY
    c = synth.configs.w_bulk(ncell=6)
    reg = {"kind": "const", "w": 0.0}
    xc, boxc = _scaled(c, 0.9)            # 64 -> ~112 atoms inside the list radius
    with _ctx(apl, c, region=reg) as ctx:
        cap0, _ = ctx.neighbor_info()
        ctx.set_box(boxc)
        ctx.set_state(xc, None, 0.0)
        ctx.compute_forces()
        with pytest.raises(apl.APError) as e:
            ctx.check()
        assert e.value.status == AP_ERR_CAPACITY
        cap1, _ = ctx.neighbor_info()
        assert cap1 > cap0
        ctx.compute_forces()
        ctx.check()
        F = ctx.forces()
        E = ctx.energy()["e_total"]
    with _ctx(apl, c, x=xc, box=boxc, region=reg) as fresh:
        fresh.compute_forces()
        assert np.array_equal(F, fresh.forces())
        assert E == fresh.energy()["e_total"]
    # the compressed cell's forces reach ~13 eV/A: FP32 pair sums carry ~1e-5 of that
    ref = orc.evaluate(xc, boxc, c["eam"], c["ace"], reg)
    assert np.abs(F - ref["forces"]).max() <= 1e-4 + 2e-5 * np.abs(ref["forces"]).max()


def test_failed_list_growth_reports_oom_then_recovers(apl):
    from paper_2505_12958_gb300._capi import AP_ERR_CAPACITY, AP_ERR_OOM, lib
    c = synth.configs.w_bulk(ncell=6)
    reg = {"kind": "const", "w": 0.0}
    xc, boxc = _scaled(c, 0.9)
    with _ctx(apl, c, region=reg) as ctx:
        ctx.set_box(boxc)
        ctx.set_state(xc, None, 0.0)
        ctx.compute_forces()
        lib().ap_inject_alloc_failures(1)
        try:
            with pytest.raises(apl.APError) as e:
                ctx.check()
        finally:
            lib().ap_inject_alloc_failures(0)
        assert e.value.status == AP_ERR_OOM
        ctx.compute_forces()                 # overflows again with the old capacity
        with pytest.raises(apl.APError) as e:
            ctx.check()
        assert e.value.status == AP_ERR_CAPACITY
        ctx.compute_forces()
        ctx.check()
        F = ctx.forces()
    with _ctx(apl, c, x=xc, box=boxc, region=reg) as fresh:
        fresh.compute_forces()
        assert np.array_equal(F, fresh.forces())


def test_ace_neighbour_limit_is_reported_and_not_retried(apl):
    from paper_2505_12958_gb300._capi import AP_ERR_LIMIT
    # BCC at a = 2.0 A: 136 neighbours inside the 5 A ACE cutoff, above the 128 the build holds
    c = synth.configs.w_bulk(ncell=5, a=2.0, sigma=0.0)
    with _ctx(apl, c, region={"kind": "const", "w": 1.0}) as ctx:
        for _ in range(2):
            ctx.compute_forces()
            with pytest.raises(apl.APError) as e:
                ctx.check()
            assert e.value.status == AP_ERR_LIMIT
            assert "ACE cutoff" in str(e.value)


def test_injected_oom_at_init(apl):
    from paper_2505_12958_gb300._capi import AP_ERR_OOM, lib
    c = synth.configs.w_bulk(ncell=4)
    lib().ap_inject_alloc_failures(1)
    try:
        with pytest.raises(apl.APError) as e:
            _ctx(apl, c)
    finally:
        lib().ap_inject_alloc_failures(0)
    assert e.value.status == AP_ERR_OOM
    with _ctx(apl, c) as ctx:             # the next context is created normally
        ctx.compute_forces()
        ctx.check()


def _requests(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        r = synth.configs.serving_request(k, rng, ("Cu", "W")[k % 2], synth.configs.GEOMETRIES[k % 5],
                                          int(np.exp(rng.uniform(np.log(64), np.log(2000)))))
        r["n_steps"] = int(rng.integers(1, 17))
        r["arrival_s"] = 0.0
        out.append(r)
    return out


def _same(a, b):
    assert a.error is None and b.error is None
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v)
    assert np.array_equal(a.forces, b.forces)
    assert a.energy["e_total"] == b.energy["e_total"]


def test_bound_list_sizing_equals_counted_sizing(apl):
    """ap_init with the density-bound capacity (no synchronisation) gives the same bits as
    the counted capacity: the list holds the same entries in the same order."""
    c = synth.configs.w_slab(ncell=8, nz=6, r_in=7.0, r_sw=3.0, R=9.0, penetration=1.0)
    out = []
    for sizing in ("counted", "bound"):
        with apl.APContext(c["eam"], c["ace"], c["box"], c["x"], c["v"], c["fixed"], c["region"], c["indenter"],
                           c["ind_vel"], c["mass"], list_sizing=sizing) as ctx:
            ctx.step(12, 1.0)
            ctx.check()
            x, v, _ = ctx.get_state()
            out.append((ctx.neighbor_info()[0], x, v, ctx.forces(), ctx.energy()["e_total"], ctx.memory_bytes()))
    (cap_c, xc, vc, fc, ec, mc), (cap_b, xb, vb, fb, eb, mb) = out
    assert cap_b >= cap_c
    assert np.array_equal(xc, xb) and np.array_equal(vc, vb) and np.array_equal(fc, fb) and ec == eb
    assert mb <= apl.footprint_bytes(c["eam"], c["ace"], len(c["x"]), c["mass"])


def test_bound_list_sizing_grows_on_a_denser_structure(apl):
    """A cell compressed beyond the bound's 0.1 atoms / A^3 overflows the bound capacity:
    the first check reports AP_ERR_CAPACITY and grows the list, and the next evaluation
    equals that of a context sized by counting."""
    from paper_2505_12958_gb300._capi import AP_ERR_CAPACITY
    c = synth.configs.w_bulk(ncell=6)
    reg = {"kind": "const", "w": 0.0}
    xc, boxc = _scaled(c, 0.72)           # 0.17 atoms / A^3
    with apl.APContext(c["eam"], c["ace"], boxc, xc, None, None, reg, None, None, c["mass"],
                       list_sizing="bound") as ctx:
        cap0, _ = ctx.neighbor_info()
        ctx.compute_forces()
        with pytest.raises(apl.APError) as e:
            ctx.check()
        assert e.value.status == AP_ERR_CAPACITY
        assert ctx.neighbor_info()[0] > cap0
        ctx.compute_forces()
        ctx.check()
        F = ctx.forces()
        E = ctx.energy()["e_total"]
    with _ctx(apl, c, x=xc, box=boxc, region=reg) as counted:
        counted.compute_forces()
        assert np.array_equal(F, counted.forces())
        assert E == counted.energy()["e_total"]


def test_server_refuses_a_request_whose_context_fails_and_serves_the_rest(apl):
    from paper_2505_12958_gb300._capi import lib
    from paper_2505_12958_gb300.serve import Server
    reqs = _requests(21, 5)
    lib().ap_inject_alloc_failures(1)
    try:
        res = {r.id: r for r in Server(chunk=4).run(reqs, realtime=False)}
    finally:
        lib().ap_inject_alloc_failures(0)
    assert len(res) == len(reqs)
    refused = [r for r in res.values() if r.error is not None]
    assert len(refused) == 1 and "AP_ERR_OOM" in refused[0].error and refused[0].id == reqs[0]["id"]
    for q in reqs[1:]:
        alone = Server(chunk=3).run([q], realtime=False)[0]
        _same(res[q["id"]], alone)


def test_server_retires_a_failing_request_without_disturbing_the_others(apl):
    from paper_2505_12958_gb300.serve import Server
    reqs = _requests(22, 4)
    bad = synth.configs.w_bulk(ncell=5, a=2.0, sigma=0.0)      # beyond the ACE-neighbour limit
    bad.update({"id": 99, "n_steps": 6, "arrival_s": 0.0, "region": {"kind": "const", "w": 1.0}})
    mix = reqs[:2] + [bad] + reqs[2:]
    res = {r.id: r for r in Server(chunk=4).run(mix, realtime=False)}
    assert "AP_ERR_LIMIT" in res[99].error
    for q in reqs:
        alone = Server(chunk=5).run([q], realtime=False)[0]
        _same(res[q["id"]], alone)
