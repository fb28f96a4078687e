"""Pins of the oracle's whole AP evaluation (Eq. energy_hyb with w = 1 - lambda,
Eqs. V_indenter and P_ind), its neighbour search and its velocity Verlet.

Structural identities of the method: w = 0 / w = 1 give pure EAM / pure ACE; the energy is
linear in the weights; rotation, translation and permutation invariance; zero net force
without an external field; forces equal the central-difference gradient including the
weight-gradient term of transition atoms; the virial equals minus the strain derivative;
the indenter matches its closed form; NVE energy is conserved to O(dt^2).
"""
import numpy as np
import pytest

import synth
from synth.lattice import bcc, fcc, random_displacements

rng = np.random.default_rng(3)


def _small(species="W", n=3, sigma=0.06, seed=11):
    lat, a = (bcc, 3.165) if species == "W" else (fcc, 3.615)
    x = lat(a, n, n, n)
    x = x + random_displacements(len(x), sigma, seed)
    L = n * a
    box = {"h": np.diag([L, L, L]).ravel(), "origin": (0, 0, 0), "periodic": (1, 1, 1)}
    return x, box, synth.eam_potential(species), synth.ace_potential(species), L


def test_weight_limits_reduce_to_pure_potentials(orc):
    x, box, eam, ace, L = _small()
    e = orc.evaluate(x, box, eam=eam)
    a = orc.evaluate(x, box, ace=ace, region={"kind": "const", "w": 1.0})
    z = orc.evaluate(x, box, eam=eam, ace=ace, region={"kind": "const", "w": 0.0})
    o = orc.evaluate(x, box, eam=eam, ace=ace, region={"kind": "const", "w": 1.0})
    assert z["e_total"] == e["e_total"] and np.array_equal(z["forces"], e["forces"])
    assert o["e_total"] == a["e_total"] and np.array_equal(o["forces"], a["forces"])
    assert z["n_ace"] == 0 and o["n_ace"] == len(x)


def test_sphere_weight_closed_form_and_compaction(orc):
    """w = (1 + cos(pi (d - r_in)/r_sw))/2 in the shell, 1 inside, 0 outside (Sec. 2.2.3 with the
    cosine transition); checked against sin^2(pi (r_in + r_sw - d)/(2 r_sw)), the same function
    written from the outer radius, and the compaction count w > 0 equals #{d < r_in + r_sw},
    including atoms a nanometre-fraction inside the outer radius."""
    r_in, r_sw = 10.0, 3.0
    ro = r_in + r_sw
    d = np.concatenate([[0.0, 3.0, 9.999], np.linspace(r_in, ro, 31)[1:-1],
                        [ro - 1e-3, ro - 1e-6, ro - 1e-9, ro, ro + 1e-9, 14.0, 20.0]])
    k = np.arange(len(d)) + 0.5
    th, ph = np.arccos(1 - 2 * k / len(d)), np.pi * (1 + 5 ** 0.5) * k
    u = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    c = np.array([50.0, 50.0, 50.0])
    x = c + d[:, None] * u
    box = {"h": np.diag([100.0] * 3).ravel(), "origin": (0, 0, 0), "periodic": (0, 0, 0)}
    reg = {"kind": "sphere", "center": tuple(c), "r_in": r_in, "r_sw": r_sw}
    r = orc.evaluate(x, box, synth.eam_potential("W"), synth.ace_potential("W"), reg)
    dd = np.linalg.norm(x - c, axis=1)
    ref = np.where(dd < r_in, 1.0, np.where(dd >= ro, 0.0, np.sin(0.5 * np.pi * (ro - dd) / r_sw) ** 2))
    shell = (dd >= r_in) & (dd < ro)
    # away from the outer radius: relative agreement; within 1e-6 A of it w ~ 1e-13 and below,
    # where any FP64 evaluation carries the rounding of d itself: positive and tiny
    far = shell & (ro - dd > 1e-6)
    assert np.allclose(r["w"][far], ref[far], rtol=1e-7, atol=0.0)
    edge = shell & ~far
    assert edge.sum() >= 2 and (r["w"][edge] > 0).all() and (r["w"][edge] < 1e-12).all()
    assert np.array_equal(r["w"][~shell], ref[~shell])
    mid = shell & (dd - r_in > 0.1) & (ro - dd > 0.1)
    assert np.allclose(r["w"][mid], 0.5 * (1 + np.cos(np.pi * (dd[mid] - r_in) / r_sw)), rtol=1e-12)
    assert r["n_ace"] == int((dd < ro).sum()) and (r["w"][dd < ro] > 0).all()


def test_energy_and_forces_are_linear_in_constant_weights(orc):
    x, box, eam, ace, L = _small("Cu", 3)
    e = orc.evaluate(x, box, eam=eam)
    a = orc.evaluate(x, box, ace=ace, region={"kind": "const", "w": 1.0})
    w = rng.uniform(0, 1, len(x))
    m = orc.evaluate(x, box, eam=eam, ace=ace, region={"kind": "explicit", "w": w})
    assert abs(m["e_total"] - (w @ a["e_atom"] + (1 - w) @ e["e_atom"])) < 1e-9
    c = orc.evaluate(x, box, eam=eam, ace=ace, region={"kind": "const", "w": 0.3})
    assert np.abs(c["forces"] - (0.3 * a["forces"] + 0.7 * e["forces"])).max() < 1e-11
    assert abs(c["e_total"] - (0.3 * a["e_total"] + 0.7 * e["e_total"])) < 1e-9


def test_translation_permutation_and_net_force(orc):
    x, box, eam, ace, L = _small()
    reg = {"kind": "const", "w": 0.4}
    r0 = orc.evaluate(x, box, eam=eam, ace=ace, region=reg)
    r1 = orc.evaluate(x + np.array([1.3, -7.1, 0.4]), box, eam=eam, ace=ace, region=reg)
    p = rng.permutation(len(x))
    r2 = orc.evaluate(x[p], box, eam=eam, ace=ace, region=reg)
    assert abs(r0["e_total"] - r1["e_total"]) < 1e-9 and np.abs(r0["forces"] - r1["forces"]).max() < 1e-10
    assert abs(r0["e_total"] - r2["e_total"]) < 1e-9 and np.abs(r0["forces"][p] - r2["forces"]).max() < 1e-10
    assert np.abs(r0["forces"].sum(axis=0)).max() < 1e-10


def test_rotation_invariance_of_a_free_cluster(orc):
    x, box, eam, ace, L = _small("W", 4, seed=5)
    c = x[np.linalg.norm(x - L / 2, axis=1) < 7.0]
    fbox = {"h": np.diag([100.0] * 3).ravel(), "origin": (-50, -50, -50), "periodic": (0, 0, 0)}
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    reg = {"kind": "sphere", "center": (0, 0, 0), "r_in": 2.0, "r_sw": 3.0}
    c0 = c - c.mean(axis=0)
    r0 = orc.evaluate(c0, fbox, eam=eam, ace=ace, region=reg)
    r1 = orc.evaluate(c0 @ q.T, fbox, eam=eam, ace=ace, region=reg)
    assert 0 < r0["n_ace"] < len(c0)
    assert abs(r0["e_total"] - r1["e_total"]) < 1e-9
    assert np.abs(r0["forces"] @ q.T - r1["forces"]).max() < 1e-9


@pytest.mark.parametrize("species", ["W", "Cu"])
def test_ap_forces_with_transition_atoms_are_the_energy_gradient(orc, species):
    x, box, eam, ace, L = _small(species, 3, sigma=0.07, seed=21)
    reg = {"kind": "sphere", "center": (L / 2, L / 2, L / 2), "r_in": 2.0, "r_sw": 3.0}
    ind = {"center": (L / 2, L / 2, x[:, 2].max() + 2.5), "R": 4.0, "K": 10.0, "dir": (0, 0, -1)}
    r = orc.evaluate(x, box, eam=eam, ace=ace, region=reg, indenter=ind)
    w = r["w"]
    trans = np.where((w > 0) & (w < 1))[0]
    assert len(trans) > 3 and (w == 1).sum() > 0 and (w == 0).sum() > 0
    d = np.linalg.norm(x - np.array(ind["center"]), axis=1)
    touched = np.where(d < ind["R"])[0]
    assert len(touched) > 0
    h = 1e-5
    for i in list(trans[:4]) + list(touched[:2]) + [int(np.argmin(w))]:
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            ep = orc.evaluate(xp, box, eam=eam, ace=ace, region=reg, indenter=ind)["e_total"]
            em = orc.evaluate(xm, box, eam=eam, ace=ace, region=reg, indenter=ind)["e_total"]
            assert abs(-(ep - em) / (2 * h) - r["forces"][i, k]) < 5e-6, (i, k)


def test_virial_is_minus_the_strain_derivative(orc):
    x, box, eam, ace, L = _small("W", 3, seed=8)
    reg = {"kind": "const", "w": 0.5}
    r = orc.evaluate(x, box, eam=eam, ace=ace, region=reg)
    h = 1e-5
    comps = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for c, (a, b) in enumerate(comps):
        e = np.zeros((3, 3)); e[a, b] = e[b, a] = 1.0 if a == b else 0.5
        def E(s):
            F = np.eye(3) + s * e
            hb = (np.asarray(box["h"]).reshape(3, 3) @ F.T).ravel()
            return orc.evaluate(x @ F.T, {"h": hb, "origin": (0, 0, 0), "periodic": (1, 1, 1)},
                                eam=eam, ace=ace, region=reg)["e_total"]
        dE = (E(h) - E(-h)) / (2 * h)
        # the symmetric strain (e_ab = e_ba = 1/2) gives dE/d(eps_ab) once
        assert abs(-dE - r["virial"][c]) < 1e-5 * max(1.0, abs(dE)), (c, dE, r["virial"][c])


def test_indenter_closed_form(orc):
    # Eq. V_indenter: V = K/3 (R - d)^3, F = K (R - d)^2 rhat; Eq. P_ind: load = F . dir
    box = {"h": np.diag([50.0] * 3).ravel(), "origin": (-25, -25, -25), "periodic": (0, 0, 0)}
    x = np.array([[0.3, -0.2, 1.0], [8.0, 8.0, 8.0]])
    ind = {"center": (0.0, 0.0, 4.0), "R": 4.5, "K": 10.0, "dir": (0, 0, -1)}
    r = orc.evaluate(x, box, indenter=ind)
    d = x[0] - np.array(ind["center"])
    dn = np.linalg.norm(d)
    assert abs(r["e_indenter"] - 10.0 / 3 * (4.5 - dn) ** 3) < 1e-12
    F = 10.0 * (4.5 - dn) ** 2 * d / dn
    assert np.abs(r["forces"][0] - F).max() < 1e-12 and np.all(r["forces"][1] == 0)
    assert abs(r["load"] - (-F[2])) < 1e-12


@pytest.mark.parametrize("case", ["cubic", "small_triclinic", "slab"])
def test_cell_list_equals_brute_force(orc, case):
    if case == "cubic":
        x, box, *_ = _small("W", 4)
    elif case == "small_triclinic":
        c = synth.configs.strained_w_cell(2, seed=4)
        x, box = c["x"], c["box"]
    else:
        c = synth.configs.w_slab(ncell=5, nz=4, r_in=5, R=5)
        x, box = c["x"], c["box"]
    rc = 5.45078
    a = orc.neighbors(x, box, rc, mode=0)
    b = orc.neighbors(x, box, rc, mode=1)
    key = lambda t: sorted(zip(t[0], t[1], *np.round(t[2], 9).T))
    assert len(a[0]) == len(b[0]) and key(a) == key(b)


def test_sampled_centers_give_complete_forces(orc):
    c = synth.configs.cu_bulk(ncell=5, r_in=5.0, r_sw=3.0)
    full = orc.evaluate(c["x"], c["box"], c["eam"], c["ace"], c["region"])
    sample = np.array([0, 17, 250, 499])
    pi, pj, _ = orc.neighbors(c["x"], c["box"], 5.0)
    centers = np.unique(np.concatenate([sample, pj[np.isin(pi, sample)]]))
    part = orc.evaluate(c["x"], c["box"], c["eam"], c["ace"], c["region"], centers=centers)
    assert np.abs(part["forces"][sample] - full["forces"][sample]).max() < 1e-12


def test_nve_energy_is_conserved_to_second_order_in_dt(orc):
    x, box, eam, ace, L = _small("W", 3, sigma=0.0)
    reg = {"kind": "sphere", "center": (L / 2, L / 2, L / 2), "r_in": 2.0, "r_sw": 3.0}
    v = synth.lattice.maxwell_velocities(len(x), 600.0, 183.84, 9)
    spread = []
    for dt, n in ((1.0, 200), (0.5, 400)):
        _, _, ep, ek, st = orc.md(x, v, box, eam, ace, reg, None, None, None, 183.84, dt, n)
        assert st == 0
        et = ep + ek
        spread.append(np.abs(et - et[0]).max() / len(x))
    assert spread[0] < 2e-4
    assert 2.5 < spread[0] / spread[1] < 6.0       # ~4x for a second-order integrator
