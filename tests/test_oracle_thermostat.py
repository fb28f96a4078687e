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


# ---------------------------------------------------------------------------------------
# Langevin thermostat (Appendix A, equilibration) and its counter-based random numbers
# ---------------------------------------------------------------------------------------
def test_philox_known_answer_vectors(orc):
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")
    for vec in json.load(open(path))["vectors"]:
        ctr = [int(w, 16) for w in vec["ctr"]]
        key = [int(w, 16) for w in vec["key"]]
        assert orc.philox4x32_10(ctr, key) == [int(w, 16) for w in vec["out"]]


def test_langevin_limits_and_momentum_zeroing(orc):
    c, v = _case()
    n = len(c["x"])
    g = np.ones(n, np.uint8)
    # tau -> infinity at T = 0: no drag, no noise: plain velocity Verlet
    x1, v1, *_ = orc.md_langevin(c["x"], v, c["box"], c["eam"], None, None, None, None, None, g, 1e-30, 1e30, 7, 0,
                                 c["mass"], 1.0, 30)
    x2, v2, *_ = orc.md(c["x"], v, c["box"], c["eam"], None, None, None, None, None, c["mass"], 1.0, 30)
    assert np.abs(x1 - x2).max() < 1e-12 and np.abs(v1 - v2).max() < 1e-12
    # momentum zeroing every step: the centre-of-mass velocity vanishes
    _, v3, *_ = orc.md_langevin(c["x"], v, c["box"], c["eam"], None, None, None, None, None, g, 300.0, 100.0, 7, 1,
                                c["mass"], 1.0, 10)
    assert np.abs(v3.sum(axis=0)).max() < 1e-12


def test_langevin_group_reaches_the_target_temperature(orc):
    c, v = _case(T0=50.0)
    n = len(c["x"])
    g = np.ones(n, np.uint8)
    _, _, ep, ek, st = orc.md_langevin(c["x"], v, c["box"], c["eam"], None, None, None, None, None, g, 600.0, 50.0,
                                       11, 100, c["mass"], 1.0, 2000)
    assert st == 0
    T = 2 * ek / (3 * n * KB)
    assert abs(T[600:].mean() - 600.0) < 60.0, T[600:].mean()
