"""CSP-driven switching weights on the GPU against the oracle: the centro-symmetry parameter
per atom (bulk W and Cu with thermal noise, a W slab with free surfaces and vacancies), and
the block-averaged weights with the precise zone, the surface rule, the spatial switch and
the hysteresis (the library's stated reading of the paper's switching function)."""
import numpy as np
import pytest

import synth
from synth.lattice import bcc, fcc, random_displacements

pytestmark = pytest.mark.gpu

CSP_TOL = 2e-5          # A^2: FP32 pair vectors of ~3 A, sums of 7 squared norms


@pytest.fixture(scope="module")
def apl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    ap.build()
    return ap


def _ctx(apl, sp, x, box, w=None):
    eam, ace = synth.eam_potential(sp), synth.ace_potential(sp)
    w = np.zeros(len(x)) if w is None else w
    return apl.APContext(eam, ace, box, x, None, None, {"kind": "explicit", "w": w}, None, None, eam["mass_amu"])


def _gpu_csp(apl, ctx, p):
    import torch
    out = torch.empty(ctx.n, dtype=torch.float32, device="cuda")
    ctx.csp_accumulate(p, out)
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", ["w_bulk", "cu_bulk", "w_slab"])
def test_csp_matches_oracle(apl, orc, case):
    if case == "w_bulk":
        sp, x, L, per, nnb, rc = "W", bcc(3.165, 6, 6, 6), [6 * 3.165] * 3, (1, 1, 1), 14, 3.8
    elif case == "cu_bulk":
        sp, x, L, per, nnb, rc = "Cu", fcc(3.615, 5, 5, 5), [5 * 3.615] * 3, (1, 1, 1), 12, 3.1
    else:
        sp, x, L, per, nnb, rc = "W", bcc(3.165, 8, 8, 6), [8 * 3.165, 8 * 3.165, 40.0], (1, 1, 0), 14, 3.8
        x = np.delete(x, [5, 77, 300], axis=0)                     # vacancies
    x = x + random_displacements(len(x), 0.1, 41)
    box = {"h": np.diag(L).ravel(), "origin": (0.0, 0.0, -5.0 if per[2] == 0 else 0.0), "periodic": per}
    ref, _ = orc.csp(x, box, nnb, rc)
    p = {"n_nb": nnb, "rc": rc}
    with _ctx(apl, sp, x, box) as ctx:
        got = _gpu_csp(apl, ctx, p)
    assert np.array_equal(got < 0, ref < 0)
    ok = ref >= 0
    assert np.abs(got[ok] - ref[ok]).max() <= CSP_TOL + 1e-5 * np.abs(ref[ok]).max()
    if case == "w_slab":
        assert (ref < 0).sum() > 100 and (ref[ok] > 1.6).sum() > 10       # surfaces and vacancy shells seen


def test_block_averaged_weights_match_oracle(apl, orc):
    x0 = bcc(3.165, 10, 10, 6)
    x0 = np.delete(x0, [111, 404, 777], axis=0)
    L = [10 * 3.165, 10 * 3.165, 40.0]
    box = {"h": np.diag(L).ravel(), "origin": (0.0, 0.0, -5.0), "periodic": (1, 1, 0)}
    zc = (L[0] / 2, L[1] / 2, x0[:, 2].max())
    p = {"n_nb": 14, "rc": 3.8, "zone_center": zc, "zone_r": 7.0}
    w_init = np.zeros(len(x0))
    w_init[::50] = 0.3                                         # a previous weight field to update
    blocks = []
    with _ctx(apl, "W", x0, box, w_init) as ctx:
        for k in range(3):
            xk = x0 + random_displacements(len(x0), 0.08, 100 + k)
            ctx.set_state(xk)
            blocks.append(orc.csp(xk, box, 14, 3.8)[0])
            ctx.csp_accumulate(p)
        ns = ctx.csp_update_weights(p)
        ctx.compute_forces()                       # the new weights act from the next evaluation
        w = ctx.weights()
        xlast = xk
    pr = dict(p, csp_lo=1.5, csp_hi=1.6, r_lo=4.0, r_hi=12.0, dlam_min=0.01)
    ref, w0 = orc.csp_weights(xlast, box, blocks, pr, w_init)
    assert ns == int((w0 > 0).sum())
    # w0 is linear in the averaged CSP with slope 1/(csp_hi - csp_lo) = 10 A^-2, so the CSP bar
    # carries over times 10; the spatial switch adds FP32 rounding of ~1e-6
    assert np.abs(w - ref).max() < 10 * CSP_TOL + 2e-6
    assert np.array_equal(w > 0, ref > 0)
    assert (ref == 1.0).sum() > 20 and ((ref > 0) & (ref < 1)).sum() > 20


def test_md_with_csp_weights(apl):
    c = synth.configs.w_slab(ncell=12, nz=8, r_in=8.0, r_sw=4.0, R=10.0, penetration=1.5)
    x = c["x"]
    zc = c["region"]["center"]
    p = {"n_nb": 14, "rc": 3.8, "zone_center": zc, "zone_r": 8.0}
    with apl.APContext(c["eam"], c["ace"], c["box"], x, c["v"], c["fixed"], {"kind": "explicit", "w": np.zeros(len(x))},
                       c["indenter"], c["ind_vel"], c["mass"]) as ctx:
        for block in range(3):
            for k in range(5):
                ctx.step(2, 1.0)
                ctx.csp_accumulate(p)
            ctx.csp_update_weights(p)
        ctx.step(5, 1.0)
        ctx.check()
        rep = ctx.energy()
        w = ctx.weights()
    assert rep["n_ace"] == int((w > 0).sum()) and rep["n_ace"] > 100
