"""Writes cu_eam_synth.json: a stated Cu EAM in the paper's W functional family.

The paper uses Mishin's tabulated Cu EAM (Sec. 2.2.1), whose tables are not printed, so
this set replaces it: xi(x) = a1 sqrt(x) + a2 x^2 (Eq. eam_F_Marinica), cubic-knot pair
potential (Eq. eam_Phi_Marinica) and density (Eq. eam_rho_Marinica), knots <= 5.0 A.
The density knots are fixed; a1, a2 and the pair amplitudes are the least-squares
solution that reproduces a0 = 3.615 A, E_coh = -3.54 eV, C11/C12/C44 = 169/122/75 GPa and
the zone-boundary phonons of Cu measured by inelastic neutron scattering (X: 7.25 / 5.13
THz longitudinal / transverse; L: 7.30 / 3.42 THz).  Elastic constants alone leave the
short-wavelength modes free, and a fit to them only was dynamically unstable (negative
eigenvalues of the dynamical matrix, runaway displacements within ~100 fs of MD).  Every
target is linear in the unknowns, so each column is one oracle evaluation with a single
unit coefficient.  The script calls only the oracle.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))
import oracle  # noqa: E402
from synth.lattice import fcc  # noqa: E402
from synth.params.lattice_dynamics import AMU_THZ2, dynamical, force_constants, min_eigenvalue  # noqa: E402

A0, ECOH, C11, C12, C44 = 3.615, -3.54, 169.0, 122.0, 75.0
GPA = 160.21766208
MASS = 63.546
PHONON_THZ = {"XL": 7.25, "XT": 5.13, "LL": 7.30, "LT": 3.42}
RHO_A, RHO_D = [0.1], [5.0]
PHI_D = [2.8, 3.3, 3.8, 4.4, 5.0]
N = 3   # 3x3x3 conventional cells, 108 atoms, periodic (10.8 A > 2 rc)


def params(coefs):
    a1, a2, phis = coefs[0], coefs[1], coefs[2:]
    return {"phi_a": np.asarray(phis), "phi_d": np.asarray(PHI_D), "rho_a": np.asarray(RHO_A),
            "rho_d": np.asarray(RHO_D), "rho_rclamp": 0.0, "F_a1": a1, "F_a2": a2, "F_dxi": 0.0, "zbl": 0}


def zone_boundary(p):
    """m omega^2 (eV/A^2) of the longitudinal and transverse modes at X = (2 pi/a)(1,0,0) and
    L = (pi/a)(1,1,1): D(X) = diag(L, T, T); D(L) = alpha I + beta (J - I), L = alpha + 2 beta,
    T = alpha - beta."""
    Phi, R, _ = force_constants("Cu", eam=p)
    DX = dynamical(Phi, R, np.array([[2 * np.pi / A0, 0.0, 0.0]]))[0]
    DL = dynamical(Phi, R, np.array([[np.pi / A0] * 3]))[0]
    return {"XL": DX[0, 0], "XT": DX[1, 1], "LL": DL[0, 0] + 2 * DL[0, 1], "LT": DL[0, 0] - DL[0, 1]}


def energy(coefs, strain):
    p = params(coefs)
    F = np.eye(3) + strain
    x = fcc(A0, N, N, N) @ F.T
    h = np.diag([N * A0] * 3) @ F.T
    r = oracle.evaluate(x, {"h": h.ravel(), "origin": (0, 0, 0), "periodic": (1, 1, 1)}, eam=p)
    return r["e_total"], len(x), abs(np.linalg.det(h))


def main():
    nu = 2 + len(PHI_D)
    h = 1e-3
    exx = np.zeros((3, 3)); exx[0, 0] = 1
    eyy = np.zeros((3, 3)); eyy[1, 1] = 1
    eiso = np.eye(3)
    g = np.zeros((3, 3)); g[1, 2] = g[2, 1] = 0.5
    rows = {k: np.zeros(nu) for k in ("E", "P", "C11", "C12", "C44", "XL", "XT", "LL", "LT")}
    for k in range(nu):
        c = np.zeros(nu); c[k] = 1.0
        E = lambda s: energy(c, s)[0]
        e0, n, V = energy(c, np.zeros((3, 3)))
        rows["E"][k] = e0 / n
        rows["P"][k] = (E(h * eiso) - E(-h * eiso)) / (2 * h) / V
        d2 = lambda s: (E(h * s) - 2 * e0 + E(-h * s)) / (h * h)
        rows["C11"][k] = d2(exx) / V * GPA
        rows["C12"][k] = (d2(exx + eyy) - 2 * d2(exx)) / 2 / V * GPA
        rows["C44"][k] = d2(g) / V * GPA
        for key, val in zone_boundary(params(c)).items():
            rows[key][k] = val
    kw = {key: MASS * (2 * np.pi * nu_) ** 2 * AMU_THZ2 for key, nu_ in PHONON_THZ.items()}
    keys = ("XL", "XT", "LL", "LT")
    M = np.array([rows["E"], rows["P"] * 1e4, rows["C11"] / 10, rows["C12"] / 10, rows["C44"] / 10] +
                 [rows[key] for key in keys])
    t = np.array([ECOH, 0.0, C11 / 10, C12 / 10, C44 / 10] + [kw[key] for key in keys])
    lam = 1e-4
    Rg = np.sqrt(lam) * np.eye(nu); Rg[0, 0] = Rg[1, 1] = 0.0
    sol, *_ = np.linalg.lstsq(np.vstack([M, Rg]), np.concatenate([t, np.zeros(nu)]), rcond=None)
    out = {
        "_source": "stated synthetic Cu EAM in the functional family of arXiv 2505.12958 Appendix B "
                   "(Mishin's Cu tables, Sec. 2.2.1, are not printed); written by make_cu_eam.py",
        "species": "Cu", "mass_amu": 63.546,
        "phi_a": [round(float(v), 10) for v in sol[2:]], "phi_d": PHI_D,
        "rho_a": RHO_A, "rho_d": RHO_D, "rho_rclamp": 0.0,
        "F_a1": round(float(sol[0]), 10), "F_a2": round(float(sol[1]), 10), "F_dxi": 0.0, "zbl": 0,
        "targets": {"a0": A0, "E_coh": ECOH, "C11": C11, "C12": C12, "C44": C44,
                    "phonons_THz": PHONON_THZ, "m_omega2_eV_A2": kw},
        "achieved": {k: float(v) for k, v in zip(("E_coh", "P_x1e4", "C11/10", "C12/10", "C44/10") + keys, M @ sol)},
    }
    Phi, R, L = force_constants("Cu", eam=params(sol))
    out["min_dynamical_eigenvalue_eV_A2"] = min_eigenvalue(Phi, R, L)
    with open(os.path.join(HERE, "cu_eam_synth.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
