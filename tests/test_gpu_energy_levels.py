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


def test_host_evaluation_graph_matches_plain_launches(apl):
    """On a non-legacy stream the host-buffer evaluation replays a captured graph; it must
    give the bits of the plain launches on the legacy stream, also when the positions move far
    enough to rebuild the neighbour list (decided on the device inside the graph), and without
    positions (the library-owned ones)."""
    import torch
    c = synth.configs.w_slab(ncell=8, nz=6, r_in=6.0, r_sw=3.0, R=8.0, penetration=1.0)
    rng = np.random.default_rng(3)

    def ctx(stream=None):
        return apl.APContext(c["eam"], c["ace"], c["box"], c["x"], c["v"], c["fixed"], c["region"], c["indenter"],
                             c["ind_vel"], c["mass"], skin=0.5, stream=stream)

    with ctx() as a, ctx(torch.cuda.Stream()) as b:
        x = c["x"].copy()
        for k in range(6):
            x = x + rng.normal(0.0, 0.02 if k != 3 else 0.3, x.shape)     # step 3 rebuilds the list
            fa, ea = a.compute_forces_host(x)
            fb, eb = b.compute_forces_host(x)
            assert np.array_equal(fa, fb) and ea == eb
        fa, ea = a.compute_forces_host(None)
        fb, eb = b.compute_forces_host(None)
        assert np.array_equal(fa, fb) and ea == eb
        b.check()
        assert a.neighbor_info() == b.neighbor_info() and b.neighbor_info()[1] >= 1
        ra, rb = a.energy(), b.energy()
        assert np.array_equal(ra["virial"], rb["virial"]) and ra["e_pot"] == rb["e_pot"]
