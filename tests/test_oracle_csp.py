"""Pins of the oracle's centro-symmetry parameter (the CSP of the switching function,
Appendix B) and of its CSP-driven weights (the library's stated reading of that function).

CSP: zero on perfect FCC/BCC lattices and under homogeneous strain (every neighbour keeps
its opposite partner); a centre atom displaced by delta gives n_nb/2 * 4 |delta|^2 (each
opposite pair sum becomes -2 delta); surface atoms have fewer than n_nb neighbours within
the shell cutoff (-1); brute force over pairings on a small random cluster.
Weights: a lone seed gives the closed form of the spatial switch; the zone and surface
rules; the hysteresis keeps small changes out."""
import itertools

import numpy as np

from synth.lattice import bcc, fcc


def _box(L, periodic=(1, 1, 1)):
    return {"h": np.diag(L).ravel(), "origin": (0, 0, 0), "periodic": periodic}


def test_csp_zero_on_perfect_and_strained_lattices(orc):
    for lat, a, nnb, rc in ((bcc, 3.165, 14, 3.8), (fcc, 3.615, 12, 3.1)):
        x = lat(a, 4, 4, 4)
        c, co = orc.csp(x, _box([4 * a] * 3), nnb, rc)
        assert np.abs(c).max() < 1e-20 and (co == nnb).all()
        F = np.eye(3) + np.array([[0.01, 0.004, 0.0], [0.004, -0.008, 0.002], [0.0, 0.002, 0.005]])
        c, _ = orc.csp(x @ F.T, {"h": (np.diag([4 * a] * 3) @ F.T).ravel(), "origin": (0, 0, 0),
                                  "periodic": (1, 1, 1)}, nnb, rc)
        assert np.abs(c).max() < 1e-20


def test_csp_of_a_displaced_centre_atom(orc):
    for lat, a, nnb, rc in ((bcc, 3.165, 14, 3.8), (fcc, 3.615, 12, 3.1)):
        x = lat(a, 4, 4, 4)
        delta = np.array([0.04, -0.03, 0.02])
        x[7] += delta
        c, _ = orc.csp(x, _box([4 * a] * 3), nnb, rc)
        assert abs(c[7] - nnb / 2 * 4 * delta @ delta) < 1e-12


def test_csp_marks_surface_atoms(orc):
    x = bcc(3.165, 4, 4, 4)
    c, co = orc.csp(x, _box([4 * 3.165] * 2 + [40.0], (1, 1, 0)), 14, 3.8)
    top = x[:, 2] > x[:, 2].max() - 0.1
    assert (c[top] == -1).all() and (co[top] < 14).all()
    mid = (x[:, 2] > 3.0) & (x[:, 2] < x[:, 2].max() - 3.0)
    assert np.abs(c[mid]).max() < 1e-20


def test_csp_equals_the_smallest_pair_sums_by_brute_force(orc):
    rng = np.random.default_rng(5)
    x = bcc(3.165, 3, 3, 3) + rng.normal(0, 0.15, size=(54, 3))
    L = 3 * 3.165
    c, _ = orc.csp(x, _box([L] * 3), 14, 3.8)
    for i in (0, 13, 40):
        R = x - x[i]
        R -= L * np.round(R / L)
        r = np.linalg.norm(R, axis=1)
        idx = [j for j in np.argsort(r) if j != i][:14]
        sums = sorted(float(np.sum((R[a] + R[b]) ** 2)) for a, b in itertools.combinations(idx, 2))
        assert abs(c[i] - sum(sums[:7])) < 1e-12


def _params(**kw):
    p = {"n_nb": 14, "rc": 3.8, "csp_lo": 1.5, "csp_hi": 1.6, "r_lo": 4.0, "r_hi": 12.0, "dlam_min": 0.01,
         "zone_center": (0.0, 0.0, 0.0), "zone_r": 0.0}
    p.update(kw)
    return p


def test_weights_of_a_lone_seed_follow_the_spatial_switch(orc):
    # a line of atoms 1 A apart (no periodic images within r_hi); atom 0 is the only defect
    x = np.stack([np.arange(20.0), np.zeros(20), np.zeros(20)], axis=1) + 5.0
    box = _box([60.0] * 3, (0, 0, 0))
    csp = np.full(20, 0.5)
    csp[0] = 1.58                                 # w0 = 0.8
    w, w0 = orc.csp_weights(x, box, [csp], _params(), np.zeros(20))
    r = np.arange(20.0)
    T = np.where(r <= 4.0, 1.0, np.cos(0.5 * np.pi * (r - 4.0) / 8.0) ** 2)
    T[r >= 12.0] = 0.0
    assert np.allclose(w0[0], 0.8) and np.all(w0[1:] == 0.0)
    assert np.allclose(w[np.abs(0.8 * T) >= 0.01], (0.8 * T)[np.abs(0.8 * T) >= 0.01], atol=1e-14)
    assert np.all(w[np.abs(0.8 * T) < 0.01] == 0.0)          # below dlam_min: unchanged from 0


def test_zone_surface_and_hysteresis_rules(orc):
    x = np.array([[5.0, 5.0, 5.0], [30.0, 5.0, 5.0], [55.0, 5.0, 5.0]])
    box = _box([80.0] * 3, (0, 0, 0))
    blocks = [np.array([-1.0, -1.0, 1.55]), np.array([-1.0, 2.0, 1.55])]
    p = _params(zone_center=(5.0, 5.0, 5.0), zone_r=1.0)
    w, w0 = orc.csp_weights(x, box, blocks, p, np.array([0.0, 0.0, 0.495]))
    assert w0[0] == 1.0                            # surface-like, but inside the zone
    assert w0[1] == 1.0                            # one of two evaluations is a surface: not a surface
                                                   # atom; the valid average 2.0 A^2 is above csp_hi
    assert abs(w0[2] - 0.5) < 1e-12
    assert w[2] == 0.495                           # |0.5 - 0.495| < dlam_min: unchanged
    blocks = [np.array([-1.0, -1.0, 1.55]), np.array([-1.0, -1.0, 1.55]), np.array([1.0, 2.0, 1.55])]
    _, w0 = orc.csp_weights(x, box, blocks, p, np.zeros(3))
    assert w0[1] == 0.0                            # two of three evaluations: a surface atom
