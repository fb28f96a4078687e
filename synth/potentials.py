"""Potential parameters: loaded from JSON (EAM) or drawn from a seeded generator (ACE).

The ACE basis list states which product functions exist (body order <= 4, i.e. up to
three A factors; n < nmax, l <= lmax; for three factors the sorted (l, n) triples with
an even l-sum that satisfy the triangle rule).  It is the potential's specification,
passed to both sides as an integer table; neither side derives it from the other.
"""
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
PARAMS = os.path.join(_HERE, "params")

ACE_SEEDS = {"Cu": 2001, "W": 2002}


def eam_potential(species):
    """EAM parameter dict for 'W' (the paper's table) or 'Cu' (stated synthetic set)."""
    name = {"W": "w_eam_paper.json", "Cu": "cu_eam_synth.json"}[species]
    with open(os.path.join(PARAMS, name)) as f:
        p = json.load(f)
    for k in ("phi_a", "phi_d", "rho_a", "rho_d", "b"):
        p[k] = np.asarray(p.get(k, [0.0] * 6 if k == "b" else []), dtype=np.float64)
    return p


def ace_basis(nmax=8, lmax=4):
    """Integer table (nfunc, 7): (nu, n1, l1, n2, l2, n3, l3), unused slots -1."""
    rows = []
    for n in range(nmax):
        rows.append((1, n, 0, -1, -1, -1, -1))
    for l in range(lmax + 1):
        for n1 in range(nmax):
            for n2 in range(n1, nmax):
                rows.append((2, n1, l, n2, l, -1, -1))
    keys = sorted((l, n) for n in range(nmax) for l in range(lmax + 1))
    for a in range(len(keys)):
        for b in range(a, len(keys)):
            for c in range(b, len(keys)):
                (l1, n1), (l2, n2), (l3, n3) = keys[a], keys[b], keys[c]
                if (l1 + l2 + l3) % 2 == 0 and abs(l1 - l2) <= l3 <= l1 + l2:
                    rows.append((3, n1, l1, n2, l2, n3, l3))
    return np.asarray(rows, dtype=np.int32)


def ace_potential(species, seed=None, nmax=8, lmax=4, sigma=0.1):
    """Synthetic ACE: stated basis, cutoff and normalisation; seeded N(0, sigma^2) coefficients,
    except the phi1 coefficients of the nu <= 2 functions, which params/ace_synth.json holds
    (fitted so that the perfect lattice is dynamically stable; see make_ace_synth.py)."""
    with open(os.path.join(PARAMS, "ace_synth.json")) as f:
        spec = json.load(f)[species]
    idx = ace_basis(nmax, lmax)
    rng = np.random.default_rng(ACE_SEEDS[species] if seed is None else seed)
    c1 = rng.normal(0.0, sigma, size=len(idx))
    c2 = rng.normal(0.0, sigma, size=len(idx))
    if seed is None and "c1_fit" in spec:
        # the phi1 coefficients of the nu <= 2 functions, fitted for dynamical stability
        fit = np.asarray(spec["c1_fit"], dtype=np.float64)
        c1[:len(fit)] = fit
    return {
        "species": species,
        "rc": float(spec["rc"]),
        "nref": float(spec["nref"]),
        "nmax": nmax,
        "lmax": lmax,
        "idx": idx,
        "c1": c1,
        "c2": c2,
        "c1_0": float(spec["c1_0"]),
        "c2_0": float(spec["c2_0"]),
    }
