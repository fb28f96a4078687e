"""Writes ace_synth.json: the stated constants of the synthetic ACE (Eq. energy_ace).

The paper gives no ACE basis or coefficients for this purpose (its Cu and W ACE
parametrisations are not printed), so the synthetic ACE is stated here:
  rc = 5.0 A, n_max = 8 Chebyshev radial functions x cosine cutoff, real Y_lm with
  l_max = 4, up to three A factors (body order 4), seeded N(0, 0.1^2) coefficients;
  A_nlm = (1/nref) sum_j g_n(r_ij) Y_lm(rhat_ij) with nref = 1.5;
  phi2 carries the constant basis function B_0 = 1 with coefficient c2_0 = 2, which keeps
  phi2 >= 1.28 on hot (sigma 0.2 A) and +-3% strained Cu and W lattices;
  phi1 carries B_0 with c1_0 chosen so that E^ACE of the perfect lattice equals E^EAM
  there (the role the energy offset Delta xi plays in Appendix B, Eq. tungsten_F_up),
  which keeps the weight-gradient force -grad w (E^ACE - E^EAM) small.
With every coefficient random the perfect lattices are dynamically unstable (the dynamical
matrix has negative eigenvalues down to -5.5 eV/A^2 for Cu and -0.7 for W; MD runs away
within ~100 fs).  The 188 phi1 coefficients of the one- and two-factor functions (nu <= 2)
are therefore fitted: linear least squares that matches the pure-ACE force constants to
the species' EAM force constants on an 8^3 q-grid (4x4x4 supercell), with a ridge term
pulling each coefficient toward its seeded random value (weight lam = 1, relative to the
design matrix norm).  D(q) is linear in phi1's coefficients, so each column is one force-
constant evaluation with a unit coefficient.  The three-factor coefficients and all of
phi2 stay as drawn.
Force constants alone leave the Cu (001) surface unstable in pure-ACE MD under an indenter
(the top layer collapses within a few hundred steps).  For Cu the same least-squares problem
therefore also matches the pure-ACE forces to the EAM forces on five distorted structures
(thermally displaced bulk at 0, -4 % and +3 % strain, and two displaced (001) slabs with
free surfaces): F(c) is linear in phi1's coefficients too, so each column is one force
evaluation with a unit coefficient.  Both blocks of rows are divided by their Frobenius
norms, the force block carries the weight FORCE_WEIGHT; W, whose pure-ACE surface is stable,
keeps weight 0 and its force-constant-only fit.
The fits and the offset are computed with the oracle only.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))
import oracle  # noqa: E402
import synth  # noqa: E402
from synth.lattice import bcc, fcc  # noqa: E402
from synth.params.lattice_dynamics import dynamical, force_constants, min_eigenvalue, q_grid  # noqa: E402

SPEC = {"Cu": (fcc, 3.615, 4), "W": (bcc, 3.165, 5)}
NREF, C2_0, RC = 1.5, 2.0, 5.0
LAM = 1.0
FORCE_WEIGHT = {"Cu": 1.0, "W": 0.0}
TRAIN = [(0.0, 0.10, False), (-0.04, 0.08, False), (0.03, 0.08, False), (0.0, 0.10, True), (0.0, 0.15, True)]


def training_configs(sp):
    """(x, box) of the force-matching structures: (strain, displacement sigma in A, slab)."""
    lat, a0, n = SPEC[sp]
    out = []
    for k, (strain, sigma, slab) in enumerate(TRAIN):
        a = a0 * (1.0 + strain)
        x = lat(a, n, n, n)
        x = x + np.random.default_rng(500 + k).normal(0.0, sigma, size=x.shape)
        if slab:
            box = {"h": np.diag([n * a, n * a, n * a + 20.0]).ravel(), "origin": (0.0, 0.0, -10.0),
                   "periodic": (1, 1, 0)}
        else:
            box = {"h": np.diag([n * a] * 3).ravel(), "origin": (0.0, 0.0, 0.0), "periodic": (1, 1, 1)}
        out.append((x, box))
    return out


def fit_pair_and_two_factor(sp):
    """phi1 coefficients of the nu <= 2 functions (see the module docstring): rows of
    force constants (scaled by 1/||M_D||), of forces for Cu (FORCE_WEIGHT/||M_F||), and the
    ridge sqrt(LAM/nfit) (c - drawn)."""
    ace = synth.ace_potential(sp)
    reg = {"kind": "const", "w": 1.0}
    nfit = int((ace["idx"][:, 0] <= 2).sum())
    PhiE, R, L = force_constants(sp, eam=synth.eam_potential(sp))
    q = q_grid(L, 8)
    DE = dynamical(PhiE, R, q)
    base = dict(ace, c1=ace["c1"].copy())
    base["c1"][:nfit] = 0.0
    Pb, _, _ = force_constants(sp, ace=base, region=reg)
    Db = dynamical(Pb, R, q)
    cols = []
    for k in range(nfit):
        unit = dict(base, c1=base["c1"].copy())
        unit["c1"][k] = 1.0
        Pk, _, _ = force_constants(sp, ace=unit, region=reg)
        cols.append((dynamical(Pk, R, q) - Db).ravel())
    MD = np.stack(cols, axis=1)
    tD = (DE - Db).ravel()
    drawn = ace["c1"][:nfit]
    alpha = FORCE_WEIGHT[sp]
    sr = np.sqrt(LAM / nfit)
    nD = np.linalg.norm(MD)
    A, b = [MD / nD], [tD / nD]
    if alpha > 0:
        fcols, tF = [], []
        for x, box in training_configs(sp):
            fb = oracle.evaluate(x, box, ace=base, region=reg)["forces"]
            fe = oracle.evaluate(x, box, eam=synth.eam_potential(sp))["forces"]
            tF.append((fe - fb).ravel())
            cf = []
            for k in range(nfit):
                unit = dict(base, c1=base["c1"].copy())
                unit["c1"][k] = 1.0
                cf.append((oracle.evaluate(x, box, ace=unit, region=reg)["forces"] - fb).ravel())
            fcols.append(np.stack(cf, axis=1))
        MF, tF = np.vstack(fcols), np.concatenate(tF)
        nF = np.linalg.norm(MF)
        A.append(alpha * MF / nF)
        b.append(alpha * tF / nF)
    A.append(sr * np.eye(nfit))
    b.append(sr * drawn)
    c, *_ = np.linalg.lstsq(np.vstack(A), np.concatenate(b), rcond=None)
    fitted = dict(base, c1=base["c1"].copy())
    fitted["c1"][:nfit] = c
    Pf, _, _ = force_constants(sp, ace=fitted, region=reg)
    info = {"n_fitted": nfit, "ridge_lam": LAM, "force_weight": alpha,
            "rms_shift_from_drawn": float(np.sqrt(np.mean((c - drawn) ** 2))),
            "min_dynamical_eigenvalue_eV_A2": min_eigenvalue(Pf, R, L),
            "min_dynamical_eigenvalue_drawn_eV_A2": min_eigenvalue(*force_constants(sp, ace=ace, region=reg))}
    return [round(float(v), 12) for v in c], info


def main():
    out = {"_source": __doc__.strip().splitlines()[0] + " (make_ace_synth.py)"}
    base = {sp: {"rc": RC, "nref": NREF, "c1_0": 0.0, "c2_0": C2_0} for sp in SPEC}
    with open(os.path.join(HERE, "ace_synth.json"), "w") as f:
        json.dump(base, f)
    for sp in SPEC:
        base[sp]["c1_fit"], base[sp]["c1_fit_info"] = fit_pair_and_two_factor(sp)
        print(sp, base[sp]["c1_fit_info"], flush=True)
    with open(os.path.join(HERE, "ace_synth.json"), "w") as f:
        json.dump(base, f)
    for sp, (lat, a, n) in SPEC.items():
        x = lat(a, n, n, n)
        box = {"h": np.diag([n * a] * 3).ravel(), "origin": (0, 0, 0), "periodic": (1, 1, 1)}
        ace = synth.ace_potential(sp)
        ra = oracle.evaluate(x, box, ace=ace, region={"kind": "const", "w": 1.0})
        re = oracle.evaluate(x, box, eam=synth.eam_potential(sp))
        off = (re["e_total"] - ra["e_total"]) / len(x)
        out[sp] = {"rc": RC, "nref": NREF, "c1_0": round(off, 8), "c2_0": C2_0, "lattice_a": a,
                   "c1_fit_info": base[sp]["c1_fit_info"], "c1_fit": base[sp]["c1_fit"]}
    with open(os.path.join(HERE, "ace_synth.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
