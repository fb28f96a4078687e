"""The synthetic potentials are dynamically stable at their lattice constants: the
dynamical matrix D(q) = sum_j Phi(j, 0) exp(i q . R_j) of the perfect lattice, from oracle
force constants, is positive definite at every q of an 8^3 grid that is not a reciprocal
lattice vector (where the three acoustic modes vanish).  A dropped force-constant term or
a sign error in the fitted Cu EAM or the fitted ACE coefficients shows as a negative mode.
The paper's W EAM needs no fit and must pass as printed."""
import numpy as np
import pytest

import synth
from synth.params.lattice_dynamics import dynamical, force_constants, q_grid


def _eigs(species, kind):
    if kind == "eam":
        Phi, R, L = force_constants(species, eam=synth.eam_potential(species))
    else:
        Phi, R, L = force_constants(species, ace=synth.ace_potential(species), region={"kind": "const", "w": 1.0})
    D = dynamical(Phi, R, q_grid(L, 8))
    return np.linalg.eigvalsh(0.5 * (D + np.transpose(D, (0, 2, 1)))), Phi


@pytest.mark.parametrize("species,kind", [("Cu", "eam"), ("W", "eam"), ("Cu", "ace"), ("W", "ace")])
def test_perfect_lattice_is_dynamically_stable(orc, species, kind):
    ev, Phi = _eigs(species, kind)
    # translation invariance: the force constants sum to zero (acoustic sum rule)
    assert np.abs(Phi.sum(axis=0)).max() < 1e-5
    acoustic = np.abs(ev).max(axis=1) < 1e-5          # q equivalent to Gamma
    assert acoustic.any() and (~acoustic).sum() > 400
    assert ev[~acoustic].min() > 0.05, ev[~acoustic].min()


def test_cu_eam_zone_boundary_phonons(orc):
    """The fitted Cu EAM reproduces the measured X and L phonons to within 10 %."""
    from synth.params.lattice_dynamics import AMU_THZ2
    p = synth.eam_potential("Cu")
    Phi, R, _ = force_constants("Cu", eam=p)
    a = 3.615
    DX = dynamical(Phi, R, np.array([[2 * np.pi / a, 0, 0]]))[0]
    DL = dynamical(Phi, R, np.array([[np.pi / a] * 3]))[0]
    got = {"XL": DX[0, 0], "XT": DX[1, 1], "LL": DL[0, 0] + 2 * DL[0, 1], "LT": DL[0, 0] - DL[0, 1]}
    thz = {"XL": 7.25, "XT": 5.13, "LL": 7.30, "LT": 3.42}
    for k, nu in thz.items():
        nu_got = np.sqrt(got[k] / (p["mass_amu"] * AMU_THZ2)) / (2 * np.pi)
        assert abs(nu_got - nu) / nu < 0.1, (k, nu_got, nu)


def test_cu_ace_surface_forces_follow_the_eam(orc):
    """The Cu ACE is also fitted to EAM forces on distorted bulk and (001) slabs, so on a
    displaced slab that the fit never saw its pure-ACE forces track the EAM forces: a
    surface that pure ACE pulls apart (the failure that fit prevents) gives errors of the
    order of the forces themselves."""
    from synth.lattice import fcc, random_displacements
    a = 3.615
    x = fcc(a, 5, 5, 4)
    x = x + random_displacements(len(x), 0.1, 909)
    box = {"h": np.diag([5 * a, 5 * a, 4 * a + 20.0]).ravel(), "origin": (0.0, 0.0, -10.0), "periodic": (1, 1, 0)}
    fa = orc.evaluate(x, box, ace=synth.ace_potential("Cu"), region={"kind": "const", "w": 1.0})["forces"]
    fe = orc.evaluate(x, box, eam=synth.eam_potential("Cu"))["forces"]
    rms = lambda f: np.sqrt(np.mean(f ** 2))            # noqa: E731
    assert rms(fa - fe) < 0.3 * rms(fe), (rms(fa - fe), rms(fe))
