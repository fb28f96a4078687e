"""The Nose-Hoover thermostat on a group of atoms (Appendix A, the NVT part of the slab)
on the GPU: the trajectory against the oracle's thermostatted velocity Verlet, the extended
energy over a long run, and the replayed step graph against the plain launch loop."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

KB = 8.617333262e-5


@pytest.fixture(scope="module")
def apl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    ap.build()
    return ap


def _slab():
    c = synth.configs.w_slab(ncell=8, nz=6, r_in=6.0, r_sw=3.0, R=8.0, penetration=1.0, temperature=900.0)
    z = c["x"][:, 2]
    group = ((z > z.min() + 2.5) & (z < z.max() - 4.0)).astype(np.uint8)     # the middle layers
    return c, group


def _ctx(apl, c, stream=None):
    return apl.APContext(c["eam"], c["ace"], c["box"], c["x"], c["v"], c["fixed"], c["region"], c["indenter"],
                         c["ind_vel"], c["mass"], stream=stream)


def test_thermostatted_md_matches_oracle(apl, orc):
    c, group = _slab()
    nsteps = 20
    xo, vo, ep, ek, et, st = orc.md_nh(c["x"], c["v"], c["box"], c["eam"], c["ace"], c["region"], c["indenter"],
                                       c["ind_vel"], c["fixed"], group, 300.0, 100.0, c["mass"], 1.0, nsteps)
    assert st == 0
    with _ctx(apl, c) as ctx:
        ctx.set_thermostat(300.0, 100.0, group)
        ctx.step(nsteps, 1.0)
        rep = ctx.energy()
        x, v, _ = ctx.get_state()
    L = np.asarray(c["box"]["h"]).reshape(3, 3)
    d = x - xo
    for k in range(2):
        d[:, k] -= np.round(d[:, k] / L[k, k]) * L[k, k]
    n = len(x)
    assert np.abs(d).max() < 1e-6 and np.abs(v - vo).max() < 1e-6
    assert abs(rep["e_pot"] + rep["e_ind"] - ep[-1]) / n < 1e-6
    assert abs(rep["e_kin"] - ek[-1]) / n < 1e-6
    assert abs(rep["e_thermostat"] - et[-1]) / n < 1e-6 and et[-1] != 0.0


def test_extended_energy_is_conserved(apl):
    c = synth.configs.w_bulk(ncell=6, r_in=4.0, r_sw=3.0)
    n = len(c["x"])
    c["v"] = synth.lattice.maxwell_velocities(n, 900.0, c["mass"], 5)
    c["fixed"] = np.zeros(n, np.uint8)
    c["indenter"] = None
    c["ind_vel"] = None
    with _ctx(apl, c) as ctx:
        ctx.set_thermostat(300.0, 50.0)
        e0 = ctx.energy()
        H0 = e0["e_total"] + e0["e_kin"] + e0["e_thermostat"]
        worst, Ts = 0.0, []
        for _ in range(10):
            ctx.step(100, 1.0)
            r = ctx.energy()
            worst = max(worst, abs(r["e_total"] + r["e_kin"] + r["e_thermostat"] - H0))
            Ts.append(2 * r["e_kin"] / (3 * n * KB))
    assert worst / n < 2e-4
    assert abs(np.mean(Ts[3:]) - 300.0) < 60.0          # NVE from 900 K would sit near 450 K


def test_graph_replay_with_thermostat_is_bitwise_equal(apl):
    import torch
    c, group = _slab()
    with _ctx(apl, c) as a, _ctx(apl, c, stream=torch.cuda.Stream()) as b:
        for ctx in (a, b):
            ctx.set_thermostat(300.0, 100.0, group)
            ctx.step(19, 1.0)                            # graph path: two 8-step blocks and 3 single steps
        b.check()
        xa, va, _ = a.get_state()
        xb, vb, _ = b.get_state()
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        assert a.energy()["e_thermostat"] == b.energy()["e_thermostat"]


def test_langevin_md_matches_oracle(apl, orc):
    """Langevin forces from the counter-based generator, momentum zeroing every 5 steps:
    the same trajectory as the oracle's, which draws its normal numbers from its own
    implementation of the same generator."""
    c, group = _slab()
    nsteps = 20
    xo, vo, ep, ek, st = orc.md_langevin(c["x"], c["v"], c["box"], c["eam"], c["ace"], c["region"], c["indenter"],
                                         c["ind_vel"], c["fixed"], group, 300.0, 100.0, 12345678901, 5, c["mass"],
                                         1.0, nsteps)
    assert st == 0
    with _ctx(apl, c) as ctx:
        ctx.set_thermostat(300.0, 100.0, group, kind="langevin", seed=12345678901, zero_every=5)
        ctx.step(nsteps, 1.0)
        rep = ctx.energy()
        x, v, _ = ctx.get_state()
    L = np.asarray(c["box"]["h"]).reshape(3, 3)
    d = x - xo
    for k in range(2):
        d[:, k] -= np.round(d[:, k] / L[k, k]) * L[k, k]
    n = len(x)
    assert np.abs(d).max() < 1e-6 and np.abs(v - vo).max() < 1e-6
    assert abs(rep["e_kin"] - ek[-1]) / n < 1e-6
    free = c["fixed"] == 0
    assert np.abs(v[free].sum(axis=0)).max() < 1e-9        # step 20 zeroed the momentum


def test_langevin_graph_replay_is_bitwise_equal(apl):
    import torch
    c, group = _slab()
    with _ctx(apl, c) as a, _ctx(apl, c, stream=torch.cuda.Stream()) as b:
        for ctx in (a, b):
            ctx.set_thermostat(500.0, 50.0, group, kind="langevin", seed=99, zero_every=3)
            ctx.step(19, 1.0)
        b.check()
        xa, va, _ = a.get_state()
        xb, vb, _ = b.get_state()
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
