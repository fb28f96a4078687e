"""Precision modes of the atomic-base contraction A_nlm = sum_j g_n Y_lm (tensor cores or
FMA), each against the FP64 oracle on the same AP configuration.

FP32 FMA, 3xTF32 (hi/lo split, FP32-level products) and FP64 accumulation keep the FP32
bar (1e-4 eV/A, 1e-6 eV/atom).  BF16 and FP16 round g and Y to 8- and 11-bit mantissas
(unit roundoff u = 2^-9 and 2^-12): every product g Y and so A carries a relative error
up to ~2u, and the ACE forces and energies inherit it; their bars are 2u times the ACE
force scale (times a safety factor of 10) and 2u times |E^ACE| per atom.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

U = {"bf16": 2.0 ** -9, "fp16": 2.0 ** -12}


@pytest.fixture(scope="module")
def apl():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    ap.build()
    return ap


@pytest.fixture(scope="module")
def case(orc):
    c = synth.configs.cu_bulk(ncell=6, r_in=6.0, r_sw=3.0)
    ref = orc.evaluate(c["x"], c["box"], c["eam"], c["ace"], c["region"])
    ace_only = orc.evaluate(c["x"], c["box"], None, c["ace"], {"kind": "const", "w": 1.0})
    return c, ref, np.abs(ace_only["forces"]).max(), np.abs(ace_only["e_atom"]).max()


@pytest.mark.parametrize("mode", ["fp32", "tf32x3", "fp64", "bf16", "fp16"])
def test_precision_mode_against_oracle(apl, case, mode):
    c, ref, fscale, escale = case
    with apl.APContext(c["eam"], c["ace"], c["box"], c["x"], None, None, c["region"], None, None, c["mass"],
                       precision=mode) as ctx:
        ctx.compute_forces()
        rep = ctx.energy()
        F = ctx.forces().astype(np.float64)
    n = len(c["x"])
    dF = np.abs(F - ref["forces"]).max()
    dE = abs(rep["e_total"] - ref["e_total"]) / n
    print("mode %-7s max|dF| = %.3e eV/A (ACE force scale %.2f)  |dE|/N = %.3e eV" % (mode, dF, fscale, dE))
    if mode in U:
        assert dF <= 10 * 2 * U[mode] * fscale
        assert dE <= 2 * U[mode] * escale
    else:
        assert dF <= 1e-4 and dE <= 1e-6
