"""Replayed step graphs and batched stepping: a step captured as a CUDA graph on a
non-blocking stream must give the same bits as the plain launch loop on the legacy stream,
and a context stepped inside a batch the same bits as the context stepped alone."""
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


def _ctx(apl, c, stream=None, skin=0.3):
    return apl.APContext(c["eam"], c["ace"], c["box"], c["x"], c["v"], c["fixed"], c["region"],
                         c["indenter"], c["ind_vel"], c["mass"], skin=skin, stream=stream)


def _hot_slab():
    c = synth.configs.w_slab(ncell=10, temperature=2000.0, r_in=8.0, r_sw=3.0, R=12.0)
    return c


def test_graph_replay_matches_plain_loop(apl):
    import torch
    c = _hot_slab()
    s = torch.cuda.Stream()
    with _ctx(apl, c) as a, _ctx(apl, c, stream=s) as b:
        a.step(40, 1.0)
        b.step(40, 1.0)
        b.check()
        xa, va, ta = a.get_state()
        xb, vb, tb = b.get_state()
        assert ta == tb == 40.0
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        assert np.array_equal(a.forces(), b.forces())
        ea, eb = a.energy(), b.energy()
        assert ea["e_total"] == eb["e_total"] and np.array_equal(ea["virial"], eb["virial"])
        # the skin is small: the device-side rebuild decision must have fired inside the graph
        assert a.neighbor_info()[1] > 1 and a.neighbor_info() == b.neighbor_info()
        # a changed dt re-captures; a later set_state invalidates nothing it should not
        a.step(3, 0.5)
        b.step(3, 0.5)
        assert np.array_equal(a.get_state()[0], b.get_state()[0])


def test_timed_step_graph_matches_plain_loop(apl):
    """With only the ACE contraction timed, a step replays a graph whose event-record nodes
    around the contraction get a fresh event pair each time."""
    import torch
    c = _hot_slab()
    s = torch.cuda.Stream()
    with _ctx(apl, c) as a, _ctx(apl, c, stream=s) as b:
        a.step(30, 1.0)
        b.profile(2)
        b.step(30, 1.0)
        prof = b.profile_read()
        b.profile(0)
        b.check()
        assert prof["ace"][1] == 31                      # the initial forces, then one per step
        assert 0.0 < prof["ace"][0] / 31 < 50.0          # ms per contraction of this small slab
        xa, va, _ = a.get_state()
        xb, vb, _ = b.get_state()
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        assert b.neighbor_info()[1] > 1 and a.neighbor_info() == b.neighbor_info()
        # one timed step in eight, then the plain graph path: the same trajectory
        b.profile(3)
        b.step(16, 1.0)
        prof = b.profile_read()
        b.profile(0)
        assert prof["ace"][1] == 2 and prof["ace"][0] > 0.0
        b.step(10, 1.0)
        a.step(26, 1.0)
        b.check()
        assert np.array_equal(a.get_state()[0], b.get_state()[0])
        assert np.array_equal(a.get_state()[1], b.get_state()[1])


def test_step_batch_alone_equals_mixed(apl):
    import torch
    cases = [_hot_slab(),
             synth.configs.cu_bulk(ncell=5, r_in=4.0, r_sw=2.0),
             synth.configs.w_bulk(ncell=4, r_in=3.0, r_sw=2.0)]
    for c in cases[1:]:
        c["v"] = synth.lattice.maxwell_velocities(len(c["x"]), 800.0, c["mass"], 7)
    steps = [25, 40, 10]
    alone = []
    for c, k in zip(cases, steps):
        s = torch.cuda.Stream()
        with _ctx(apl, c, stream=s) as ctx:
            apl.step_batch([ctx], [k], 1.0)
            ctx.check()
            alone.append(ctx.get_state())
    streams = [torch.cuda.Stream() for _ in cases]
    ctxs = [_ctx(apl, c, stream=s) for c, s in zip(cases, streams)]
    try:
        # issued in chunks, as a server does
        left = list(steps)
        while any(left):
            chunk = [min(8, k) for k in left]
            apl.step_batch(ctxs, chunk, 1.0)
            left = [k - q for k, q in zip(left, chunk)]
        for ctx, ref in zip(ctxs, alone):
            ctx.check()
            x, v, t = ctx.get_state()
            assert t == ref[2]
            assert np.array_equal(x, ref[0]) and np.array_equal(v, ref[1])
    finally:
        for ctx in ctxs:
            ctx.close()
