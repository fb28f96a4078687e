"""The serving form: a request served in a mix gives the same bits as the request served
alone; served structures of every geometry match the oracle; the footprint estimate bounds
what a context really holds; a tight memory budget serialises admission without changing
results."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FTOL = 1e-4          # eV/A, max per-atom force error against the FP64 oracle
ETOL = 1e-6          # eV/atom


@pytest.fixture(scope="module")
def apl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    ap.build()
    return ap


def _mix(seed, n, max_atoms=3000, max_steps=24):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        sp = ("Cu", "W")[k % 2]
        geo = synth.configs.GEOMETRIES[k % len(synth.configs.GEOMETRIES)]
        nt = int(np.exp(rng.uniform(np.log(64), np.log(max_atoms))))
        r = synth.configs.serving_request(k, rng, sp, geo, nt)
        r["n_steps"] = int(rng.integers(1, max_steps + 1))
        r["arrival_s"] = 0.0
        out.append(r)
    return out


def _same(a, b):
    assert a.id == b.id
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v)
    assert np.array_equal(a.forces, b.forces)
    assert a.energy["e_total"] == b.energy["e_total"]


def test_mix_equals_alone_bitwise(apl):
    from paper_2505_12958_gb300.serve import Server
    reqs = _mix(11, 12)
    mixed = {r.id: r for r in Server(chunk=5).run(reqs, realtime=False)}
    assert len(mixed) == len(reqs)
    for q in reqs:
        alone = Server(chunk=7).run([q], realtime=False)[0]
        _same(mixed[q.get("id")], alone)
        assert mixed[q["id"]].memory_bytes <= mixed[q["id"]].footprint_bytes


def test_tight_budget_serialises_admission(apl):
    from paper_2505_12958_gb300 import footprint_bytes
    from paper_2505_12958_gb300.serve import Server
    reqs = _mix(12, 6)
    big = max(footprint_bytes(r["eam"], r["ace"], len(r["x"]), r["mass"]) for r in reqs)
    s1 = Server(mem_budget=big)
    tight = {r.id: r for r in s1.run(reqs, realtime=False)}
    s2 = Server()
    loose = {r.id: r for r in s2.run(reqs, realtime=False)}
    assert s2.peak_active == len(reqs) and s1.peak_active < len(reqs)
    for k in tight:
        _same(tight[k], loose[k])


def test_served_geometries_match_oracle(apl, orc):
    from paper_2505_12958_gb300.serve import Server
    reqs = _mix(13, 10, max_atoms=1500)
    for r in reqs:
        r["n_steps"] = 0                     # a single-point evaluation of the submitted structure
    res = {r.id: r for r in Server().run(reqs, realtime=False)}
    for q in reqs:
        ref = orc.evaluate(q["x"], q["box"], q["eam"], q["ace"], q["region"])
        got = res[q["id"]]
        n = len(q["x"])
        assert np.abs(got.forces.astype(np.float64) - ref["forces"]).max() <= FTOL, q["geometry"]
        assert abs(got.energy["e_pot"] - ref["e_total"]) / n <= ETOL, q["geometry"]
        assert got.n_ace == ref["n_ace"]


def test_realtime_arrivals_report_latency(apl):
    from paper_2505_12958_gb300.serve import Server, percentile_ms
    reqs = _mix(14, 16, max_atoms=2000, max_steps=10)
    t = np.cumsum(np.random.default_rng(14).exponential(0.002, size=len(reqs)))
    for r, a in zip(reqs, t):
        r["arrival_s"] = float(a)
    res = Server().run(reqs, realtime=True)
    assert len(res) == len(reqs)
    for r in res:
        assert r.admit_s >= r.arrival_s - 1e-9 and r.done_s >= r.admit_s
    assert 0 < percentile_ms(res, 50) <= percentile_ms(res, 99)


def test_batched_step_equals_single_steps_bitwise(apl):
    """ap_step_batch runs each stage as one launch for all contexts (Cu and W mixed, so the
    batched contraction restages its coefficient tables); every context ends with the same
    bits as the same steps taken alone, including contexts that leave the batch early."""
    import torch
    reqs = _mix(31, 7, max_atoms=2500)
    steps = [int(r["n_steps"]) % 9 + 3 for r in reqs]

    def ctx(r):
        return apl.APContext(r["eam"], r["ace"], r["box"], r["x"], r["v"], r["fixed"], r["region"], None, None,
                             r["mass"], stream=torch.cuda.Stream())

    batch = [ctx(r) for r in reqs]
    apl.step_batch(batch, steps, 1.0, torch.cuda.Stream())
    for r, c, k in zip(reqs, batch, steps):
        alone = ctx(r)
        alone.step(k, 1.0)
        xa, va, ta = alone.get_state()
        xb, vb, tb = c.get_state()
        assert ta == tb == k
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        assert np.array_equal(alone.forces(), c.forces())
        assert alone.energy()["e_total"] == c.energy()["e_total"]
        alone.close()
        c.close()


def test_batched_force_evaluation_equals_single(apl, orc):
    import torch
    reqs = _mix(32, 5, max_atoms=1500)
    ctxs = [apl.APContext(r["eam"], r["ace"], r["box"], r["x"], None, None, r["region"], None, None, r["mass"])
            for r in reqs]
    apl.compute_forces_batch(ctxs, torch.cuda.Stream())
    for r, c in zip(reqs, ctxs):
        ref = orc.evaluate(r["x"], r["box"], r["eam"], r["ace"], r["region"])
        F = c.forces()
        assert np.abs(F.astype(np.float64) - ref["forces"]).max() <= FTOL
        with apl.APContext(r["eam"], r["ace"], r["box"], r["x"], None, None, r["region"], None, None,
                           r["mass"]) as one:
            one.compute_forces()
            assert np.array_equal(one.forces(), F)
        c.close()
