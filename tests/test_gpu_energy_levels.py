"""The host-buffer evaluation computes the total energy without the per-atom virial; a later
energy report of the same state must still carry the full virial, bit for bit the same as a
report that follows a device evaluation."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    ap.build()
    return ap


def test_energy_report_after_host_evaluation_has_the_virial(apl):
    c = synth.configs.w_slab(ncell=8, nz=6, r_in=6.0, r_sw=3.0, R=8.0, penetration=1.0)

    def ctx():
        return apl.APContext(c["eam"], c["ace"], c["box"], c["x"], c["v"], c["fixed"], c["region"], c["indenter"],
                             c["ind_vel"], c["mass"])

    with ctx() as a, ctx() as b:
        fa, e_host = a.compute_forces_host(c["x"])
        ra = a.energy()
        b.compute_forces()
        rb = b.energy()
        fb = b.forces()
    assert np.array_equal(fa, fb)
    assert np.array_equal(ra["virial"], rb["virial"]) and np.abs(ra["virial"]).max() > 0.0
    assert ra["e_pot"] == rb["e_pot"] and ra["e_ind"] == rb["e_ind"]
    assert e_host == ra["e_pot"] + ra["e_ind"]
