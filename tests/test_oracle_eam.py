"""Pins of the oracle's EAM (Sec. 2.2.1 Eq. energy_eam; Appendix B forms and tables).

The strongest pins are the paper's printed properties of its fitted W EAM
(Tab. properties_tungsten_potentials): the oracle's energy, evaluated on homogeneously
strained perfect BCC crystals, must reproduce a0, E_coh, C11, C12, C44 and B.
"""
import json
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import synth
from synth.lattice import bcc, fcc, random_displacements

GOLD = os.path.join(os.path.dirname(__file__), "golden", "w_eam_paper_properties.json")
GPA = 160.21766208  # eV/A^3 -> GPa


def _crystal_energy(orc, p, a, strain, lat=bcc, n=4):
    F = np.eye(3) + strain
    x = lat(a, n, n, n) @ F.T
    h = np.diag([n * a] * 3) @ F.T
    r = orc.evaluate(x, {"h": h.ravel(), "origin": (0, 0, 0), "periodic": (1, 1, 1)}, eam=p)
    assert r["status"] == 0
    return r["e_total"], len(x), abs(np.linalg.det(h))


def test_w_eam_reproduces_paper_bulk_properties(orc):
    gold = json.load(open(GOLD))
    p = synth.eam_potential("W")
    res = minimize_scalar(lambda a: _crystal_energy(orc, p, a, np.zeros((3, 3)))[0],
                          bracket=(3.10, 3.18, 3.25), tol=1e-12)
    a0 = res.x
    e0, n, V = _crystal_energy(orc, p, a0, np.zeros((3, 3)))
    h = 1e-4
    E = lambda s: _crystal_energy(orc, p, a0, s)[0]
    d2 = lambda s: (E(h * s) - 2 * e0 + E(-h * s)) / (h * h)
    exx = np.zeros((3, 3)); exx[0, 0] = 1
    eyy = np.zeros((3, 3)); eyy[1, 1] = 1
    shear = np.zeros((3, 3)); shear[1, 2] = shear[2, 1] = 0.5       # engineering gamma_yz
    C11 = d2(exx) / V * GPA
    C12 = (d2(exx + eyy) - 2 * d2(exx)) / 2 / V * GPA
    C44 = d2(shear) / V * GPA
    B = (C11 + 2 * C12) / 3
    assert abs(a0 - gold["lattice_constant_A"]) < 1e-4
    assert abs(e0 / n - gold["cohesive_energy_eV"]) < 5e-3
    assert abs(C11 - gold["C11_GPa"]) < 1.0
    assert abs(C12 - gold["C12_GPa"]) < 1.0
    assert abs(C44 - gold["C44_GPa"]) < 1.0
    assert abs(B - gold["bulk_modulus_GPa"]) < 1.0


def test_w_density_has_its_maximum_at_the_clamp_radius(orc):
    # Eq. tungsten_rho_up: zeta_0 has its maximum at r_cut^rho, where zeta is clamped.
    p = dict(synth.eam_potential("W"))
    rc = p["rho_rclamp"]
    q = dict(p); q["rho_rclamp"] = 0.0                      # the raw zeta_0
    eps = 1e-6
    f = orc.eam_funcs(q, [rc - eps, rc, rc + eps])
    assert abs(f[1, 3]) < 1e-6                               # zeta_0'(r_cut) = 0
    assert f[1, 2] >= f[0, 2] and f[1, 2] >= f[2, 2]         # a maximum
    g = orc.eam_funcs(p, [1.5, 2.0, rc])
    assert np.allclose(g[:, 2], f[1, 2]) and np.all(g[:, 3] == 0.0)


def test_zbl_screening_length_matches_its_formula():
    # a_ZBL = 0.8854 a_0 / (Z1^0.23 + Z2^0.23), a_0 = 0.529 A, Z = 74 -> ~0.0870 A (Appendix B)
    p = synth.eam_potential("W")
    a = 0.8854 * 0.529 / (2 * 74.0 ** 0.23)
    assert abs(a - 0.0870) < 5e-5
    assert abs(p["zbl_a"] - a) / a < 2e-3
    # 1/(4 pi eps0) with eps0 = 55.26e-4 e^2/(eV A) is the Coulomb constant 14.3996 eV A
    assert abs(1.0 / (4 * np.pi * p["zbl_eps0"]) - 14.3996) < 1e-3


@pytest.mark.parametrize("r0", ["r_lo", "r_hi"])
def test_pair_potential_is_c2_at_the_zbl_bridge(orc, r0):
    # Eq. tungsten_Phi_up: Phi and its first two derivatives are continuous at r_lo, r_hi.
    p = synth.eam_potential("W")
    r = p[r0]
    e = 1e-7
    f = orc.eam_funcs(p, [r - e, r + e, r - 2e-4, r - 1e-4, r + 1e-4, r + 2e-4])
    scale = max(1.0, abs(f[0, 0]))
    assert abs(f[0, 0] - f[1, 0]) < 1e-5 * scale
    assert abs(f[0, 1] - f[1, 1]) < 1e-4 * max(1.0, abs(f[0, 1]))
    d2l = (f[3, 1] - f[2, 1]) / 1e-4
    d2r = (f[5, 1] - f[4, 1]) / 1e-4
    assert abs(d2l - d2r) < 2e-2 * max(1.0, abs(d2l))


def test_pair_potential_is_finite_and_repulsive_at_short_range(orc):
    p = synth.eam_potential("W")
    f = orc.eam_funcs(p, np.linspace(0.5, 2.3, 50))
    assert np.all(np.isfinite(f)) and np.all(f[:, 0] > 0) and np.all(f[:, 1] < 0)


@pytest.mark.parametrize("species", ["W", "Cu"])
def test_eam_forces_are_the_energy_gradient(orc, species):
    # small periodic cell (smaller than 2 rc, so several images of an atom are neighbours)
    lat, a, n = (bcc, 3.165, 3) if species == "W" else (fcc, 3.615, 2)
    x = lat(a, n, n, n) + random_displacements(2 * n ** 3 if species == "W" else 4 * n ** 3, 0.08, 5)
    box = {"h": np.diag([n * a] * 3).ravel(), "origin": (0, 0, 0), "periodic": (1, 1, 1)}
    p = synth.eam_potential(species)
    r = orc.evaluate(x, box, eam=p)
    h = 1e-5
    for i in (0, 3, len(x) - 1):
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            fd = -(orc.evaluate(xp, box, eam=p)["e_total"] - orc.evaluate(xm, box, eam=p)["e_total"]) / (2 * h)
            assert abs(fd - r["forces"][i, k]) < 2e-6, (i, k, fd, r["forces"][i, k])


def test_cu_synthetic_eam_is_stable_at_its_lattice_constant(orc):
    # the stated Cu set: zero pressure and positive elastic constants at a = 3.615 A
    p = synth.eam_potential("Cu")
    h = 1e-4
    E = lambda a: _crystal_energy(orc, p, a, np.zeros((3, 3)), lat=fcc, n=3)[0] / 108
    assert abs(E(3.615 + h) - E(3.615 - h)) / (2 * h) < 1e-4
    assert E(3.615 + h) - 2 * E(3.615) + E(3.615 - h) > 0
