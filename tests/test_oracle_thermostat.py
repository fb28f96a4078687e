"""Pins of the oracle's Nose-Hoover thermostat on a group (Appendix A: the central part of
the slab is NVT during the indentation, Nose-Hoover with damping time gamma_T^NH).

The extended energy epot + ekin + Q xi^2/2 + N_f k_B T eta is conserved with an error of
second order in dt; an empty group is plain velocity Verlet bit for bit; an infinitely
slow thermostat (tau -> infinity) becomes NVE; the thermostat pulls a hot group toward
the target temperature."""
import numpy as np

import synth

KB = 8.617333262e-5


def _case(T0=600.0):
    c = synth.configs.w_bulk(ncell=3)
    v = synth.lattice.maxwell_velocities(len(c["x"]), T0, c["mass"], 3)
    return c, v


def test_extended_energy_error_is_second_order(orc):
    c, v = _case()
    g = np.ones(len(c["x"]), np.uint8)
    drift = []
    for dt, n in ((1.0, 200), (0.5, 400)):
        _, _, ep, ek, et, st = orc.md_nh(c["x"], v, c["box"], c["eam"], None, None, None, None, None, g, 300.0, 50.0,
                                         c["mass"], dt, n)
        assert st == 0
        H = ep + ek + et
        drift.append(np.abs(H - H[0]).max())
    assert 3.0 < drift[0] / drift[1] < 5.5, drift


def test_empty_group_is_plain_velocity_verlet(orc):
    c, v = _case()
    g = np.zeros(len(c["x"]), np.uint8)
    x1, v1, ep1, ek1, et, _ = orc.md_nh(c["x"], v, c["box"], c["eam"], None, None, None, None, None, g, 300.0, 100.0,
                                        c["mass"], 1.0, 50)
    x2, v2, ep2, ek2, _ = orc.md(c["x"], v, c["box"], c["eam"], None, None, None, None, None, c["mass"], 1.0, 50)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2) and np.array_equal(ep1, ep2)
    assert np.all(et == 0.0)


def test_slow_thermostat_approaches_nve(orc):
    c, v = _case()
    g = np.ones(len(c["x"]), np.uint8)
    x1, v1, *_ = orc.md_nh(c["x"], v, c["box"], c["eam"], None, None, None, None, None, g, 300.0, 1e9,
                           c["mass"], 1.0, 50)
    x2, v2, *_ = orc.md(c["x"], v, c["box"], c["eam"], None, None, None, None, None, c["mass"], 1.0, 50)
    assert np.abs(x1 - x2).max() < 1e-9 and np.abs(v1 - v2).max() < 1e-10


def test_hot_group_relaxes_toward_the_target(orc):
    c, v = _case(T0=1200.0)
    n = len(c["x"])
    g = np.ones(n, np.uint8)
    _, _, ep, ek, et, _ = orc.md_nh(c["x"], v, c["box"], c["eam"], None, None, None, None, None, g, 300.0, 50.0,
                                    c["mass"], 1.0, 1500)
    T = 2 * ek / (3 * n * KB)
    late = T[500:].mean()
    assert abs(late - 300.0) < 60.0, late           # NVE at this energy would stay near 600 K
