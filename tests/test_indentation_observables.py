"""Indentation observables (Eqs. hertz_fit, contact_radius, p_m): the closed forms on
synthetic series (CPU), and a short indentation of a small W slab on the GPU whose load
matches the oracle's Eq. P_ind at the recorded states."""
import numpy as np
import pytest

import synth
from paper_2505_12958_gb300.indentation import EV_PER_A3_IN_GPA, contact_radius, hardness, hertz_modulus


def test_hertz_fit_recovers_the_modulus_of_an_exact_hertz_curve():
    R, E = 40.0, 300.0 / EV_PER_A3_IN_GPA          # 300 GPa in eV/A^3
    h = np.linspace(0.0, 5.0, 60)
    P = 4.0 / 3.0 * E * np.sqrt(R) * h ** 1.5
    assert abs(hertz_modulus(h, P, R) - 300.0) < 1e-9
    # plastic points beyond h_max do not enter the fit
    P2 = P.copy()
    P2[h > 3.0] *= 0.5
    assert abs(hertz_modulus(h, P2, R, h_max=3.0) - 300.0) < 1e-9


def test_contact_radius_and_hardness():
    R = 60.0
    h = np.array([0.0, 1.0, 30.0, 60.0])
    a = contact_radius(h, R)
    assert np.allclose(a, [0.0, np.sqrt(119.0), np.sqrt(30 * 90.0), 60.0])   # a_c = R at h = R
    p = hardness(h, np.array([0.0, 2.0, 5.0, 9.0]), R)
    assert np.isnan(p[0]) and abs(p[1] - 2.0 / (np.pi * 119.0) * EV_PER_A3_IN_GPA) < 1e-12


@pytest.mark.gpu
def test_recorded_load_matches_the_oracle(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    from paper_2505_12958_gb300.indentation import record_indentation
    ap.build()
    c = synth.configs.w_slab(ncell=12, nz=8, r_in=8.0, r_sw=4.0, R=10.0, penetration=1.0, v_ms=2000.0)
    z_surf = c["x"][:, 2].max()
    with ap.APContext(c["eam"], c["ace"], c["box"], c["x"], c["v"], c["fixed"], c["region"], c["indenter"],
                      c["ind_vel"], c["mass"]) as ctx:
        rec = record_indentation(ctx, c["indenter"], c["ind_vel"], z_surf, 60, 20)
        x, _, t = ctx.get_state()
        # the device history (fixed-point sum in the step's blend) agrees with the energy
        # pass's FP64 load of the same state
        p_end = ctx.energy()["load"]
        assert abs(p_end - rec["load"][-1]) <= 1e-8 * abs(p_end) + 1e-8
        # every step is kept: 30 more steps give 30 entries whose times advance by dt
        ctx.record_load(40)
        ctx.step(30, 1.0)
        th, ph = ctx.load_history()
        assert len(th) == 30 and np.allclose(np.diff(th), 1.0) and abs(th[-1] - (t + 30.0)) < 1e-9
        assert ph[-1] > 0
    assert len(rec["load"]) == 4
    assert np.allclose(np.diff(rec["depth"]), 20 * c["ind_vel"][2])            # the tip advances at v
    assert rec["load"][0] > 0 and rec["load"][-1] > rec["load"][0]              # deeper, harder push
    ind = dict(c["indenter"])
    ind["center"] = tuple(np.asarray(c["indenter"]["center"]) - c["ind_vel"] * t)
    ref = orc.evaluate(x, c["box"], c["eam"], c["ace"], c["region"], ind)
    assert abs(rec["load"][-1] - ref["load"]) <= 1e-4 * max(1.0, abs(ref["load"]))
