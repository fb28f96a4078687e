"""Force constants and dynamical matrices of the perfect lattices, from oracle forces.

Used by the parameter scripts beside it (to fit the synthetic sets for dynamical
stability) and by the tests that pin that stability.  The dynamical matrix of a Bravais
lattice is D_ab(q) = sum_j Phi_ab(j, 0) exp(i q . R_j), with Phi_ab(j, 0) = -dF_a(j)/du_b(0)
taken by central differences of the forces when one atom of a periodic supercell moves.
D(q) / m holds the squared phonon frequencies; the lattice is dynamically stable when D(q)
is positive semi-definite at every q.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))
import oracle  # noqa: E402
from synth.lattice import bcc, fcc  # noqa: E402

LATTICE = {"Cu": (fcc, 3.615), "W": (bcc, 3.165)}
AMU_THZ2 = 1.0364269e-4          # 1 amu * (1 rad/ps)^2 in eV / A^2


def supercell(species, ncell=4):
    lat, a = LATTICE[species]
    x = lat(a, ncell, ncell, ncell)
    L = ncell * a
    box = {"h": np.diag([L] * 3).ravel(), "origin": (0, 0, 0), "periodic": (1, 1, 1)}
    return x, box, a, L


def force_constants(species, eam=None, ace=None, region=None, ncell=4, h=2e-3):
    """Phi[j, a, b] = -dF_a(j)/du_b(i0) for the atom i0 nearest the supercell centre, and the
    minimum-image lattice vectors R_j - R_i0."""
    x, box, a, L = supercell(species, ncell)
    i0 = int(np.argmin(np.linalg.norm(x - x.mean(0), axis=1)))
    cols = []
    for b in range(3):
        yp = x.copy(); yp[i0, b] += h
        ym = x.copy(); ym[i0, b] -= h
        fp = oracle.evaluate(yp, box, eam, ace, region)["forces"]
        fm = oracle.evaluate(ym, box, eam, ace, region)["forces"]
        cols.append(-(fp - fm) / (2 * h))
    Phi = np.stack(cols, axis=2)
    R = x - x[i0]
    R -= L * np.round(R / L)
    return Phi, R, L


def q_grid(L, n=8):
    g = np.arange(n)
    return np.array([[i, j, k] for i in g for j in g for k in g], dtype=np.float64) * (2 * np.pi / L)


def dynamical(Phi, R, q):
    """D(q) for each row of q: (nq, 3, 3), real for these centrosymmetric lattices."""
    ph = np.cos(q @ R.T)
    return np.einsum("qj,jab->qab", ph, Phi)


def min_eigenvalue(Phi, R, L, n=8):
    D = dynamical(Phi, R, q_grid(L, n))
    return float(np.linalg.eigvalsh(0.5 * (D + np.transpose(D, (0, 2, 1)))).min())
