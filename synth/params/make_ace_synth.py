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
The offset is computed with the oracle only.
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

SPEC = {"Cu": (fcc, 3.615, 4), "W": (bcc, 3.165, 5)}
NREF, C2_0, RC = 1.5, 2.0, 5.0


def main():
    out = {"_source": __doc__.strip().splitlines()[0] + " (make_ace_synth.py)"}
    base = {sp: {"rc": RC, "nref": NREF, "c1_0": 0.0, "c2_0": C2_0} for sp in SPEC}
    with open(os.path.join(HERE, "ace_synth.json"), "w") as f:
        json.dump(base, f)
    for sp, (lat, a, n) in SPEC.items():
        x = lat(a, n, n, n)
        box = {"h": np.diag([n * a] * 3).ravel(), "origin": (0, 0, 0), "periodic": (1, 1, 1)}
        ace = synth.ace_potential(sp)
        ra = oracle.evaluate(x, box, ace=ace, region={"kind": "const", "w": 1.0})
        re = oracle.evaluate(x, box, eam=synth.eam_potential(sp))
        off = (re["e_total"] - ra["e_total"]) / len(x)
        out[sp] = {"rc": RC, "nref": NREF, "c1_0": round(off, 8), "c2_0": C2_0, "lattice_a": a}
    with open(os.path.join(HERE, "ace_synth.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
