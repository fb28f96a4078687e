"""The autograd form: backward of the AP energy against the oracle's analytic forces and
virial and against central finite differences, on strained triclinic W cells with
vacancies and noise (the differentiation workload), for FP64 and FP32 inputs.

The energy is an FP64 total whatever the input dtype, so FP32 and FP64 inputs share the
1e-6 eV/atom bar.  Finite differences of the library energy are noise-limited: each per-atom
ACE energy carries FP32 rounding of ~1e-7 eV and a displacement changes ~60 of them, so the
central difference at h = 1e-4 A (the differentiation workload's step) carries ~5e-3 eV/A of
noise and is held to 2e-2 eV/A, and at h = 1e-3 A ~5e-4 eV/A, held to 2e-3 eV/A; the analytic
checks against the oracle hold the 1e-4 eV/A bar.
"""
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


@pytest.mark.parametrize("ncell,seed,dtype", [(4, 1, "float64"), (5, 2, "float64"), (6, 3, "float32")])
def test_backward_matches_oracle_and_finite_differences(apl, orc, ncell, seed, dtype):
    import torch
    from paper_2505_12958_gb300.autograd import ap_energy
    c = synth.configs.strained_w_cell(ncell, seed=seed)
    reg = {"kind": "const", "w": 0.5}
    ref = orc.evaluate(c["x"], c["box"], c["eam"], c["ace"], reg)
    td = getattr(torch, dtype)
    n = len(c["x"])
    with apl.APContext(c["eam"], c["ace"], c["box"], c["x"], None, None, reg, None, None, c["mass"]) as ctx:
        x = torch.tensor(c["x"], dtype=td, device="cuda", requires_grad=True)
        eps = torch.zeros((3, 3), dtype=td, device="cuda", requires_grad=True)
        E = ap_energy(x, eps, ctx, c["box"])
        E.backward()
        gx = x.grad.double().cpu().numpy()
        gs = eps.grad.double().cpu().numpy()
        # analytic: -dE/dx = oracle forces; -dE/deps = oracle virial
        xr = x.detach().double().cpu().numpy() if dtype == "float32" else c["x"]
        ref = orc.evaluate(xr, c["box"], c["eam"], c["ace"], reg)
        assert np.abs(-gx - ref["forces"]).max() <= 1e-4
        assert E.dtype == torch.float64
        assert abs(E.item() - ref["e_total"]) / n <= 1e-6
        v = ref["virial"]
        W = np.array([[v[0], v[3], v[4]], [v[3], v[1], v[5]], [v[4], v[5], v[2]]])
        assert np.abs(-gs - W).max() <= 2e-5 * np.abs(W).max() + 1e-5 * n
        # central differences of the library energy
        x64 = x.detach().double()
        e64 = eps.detach().double()
        rng = np.random.default_rng(seed)
        for h, tol in ((1e-4, 2e-2), (1e-3, 2e-3)):
            for i in rng.choice(n, size=3, replace=False):
                for k in range(3):
                    xp = x64.clone(); xp[i, k] += h
                    xm = x64.clone(); xm[i, k] -= h
                    e_p = ap_energy(xp, e64, ctx, c["box"]).item()
                    e_m = ap_energy(xm, e64, ctx, c["box"]).item()
                    assert abs((e_p - e_m) / (2 * h) - gx[i, k]) <= tol, (h, i, k)
        # strain differences: E carries ~1e-5-1e-4 eV of FP32 rounding per evaluation, so hs is
        # kept large enough for that noise to stay below ~0.1 eV after the division, while the
        # O(hs^2) truncation (third strain derivative ~1e5 eV) stays at ~1e-2 eV
        hs = 5e-4
        for a, b in ((0, 0), (1, 2)):
            d = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
            d[a, b] = d[b, a] = hs
            e_p = ap_energy(x64, d, ctx, c["box"]).item()
            e_m = ap_energy(x64, -d, ctx, c["box"]).item()
            fd = (e_p - e_m) / (2 * hs)
            an = gs[a, b] + (gs[b, a] if a != b else 0.0)
            assert abs(fd - an) <= 1e-3 * max(1.0, abs(an)) + 0.1


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_strained_cell_sweep_against_oracle(apl, orc, dtype):
    """Nine strained W cells from 4^3 to 12^3 BCC cells (128 - 3456 atoms): backward against the
    oracle's forces and virial at the positions the forward pass saw."""
    import torch
    from paper_2505_12958_gb300.autograd import ap_energy
    td = getattr(torch, dtype)
    reg = {"kind": "const", "w": 0.5}
    for k, ncell in enumerate(range(4, 13)):
        c = synth.configs.strained_w_cell(ncell, seed=500 + k)
        n = len(c["x"])
        with apl.APContext(c["eam"], c["ace"], c["box"], c["x"], None, None, reg, None, None, c["mass"]) as ctx:
            x = torch.tensor(c["x"], dtype=td, device="cuda", requires_grad=True)
            eps = torch.zeros((3, 3), dtype=td, device="cuda", requires_grad=True)
            E = ap_energy(x, eps, ctx, c["box"])
            E.backward()
            xr = x.detach().double().cpu().numpy()
            ref = orc.evaluate(xr, c["box"], c["eam"], c["ace"], reg)
            assert np.abs(-x.grad.double().cpu().numpy() - ref["forces"]).max() <= 1e-4, ncell
            assert abs(E.item() - ref["e_total"]) / n <= 1e-6, ncell
            v = ref["virial"]
            W = np.array([[v[0], v[3], v[4]], [v[3], v[1], v[5]], [v[4], v[5], v[2]]])
            gs = eps.grad.double().cpu().numpy()
            assert np.abs(-gs - W).max() <= 2e-5 * np.abs(W).max() + 1e-5 * n, ncell
