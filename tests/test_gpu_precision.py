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


@pytest.fixture(scope="module")
def slab(orc):
    """The 2,000,000-atom Cu (001) indentation slab (5 % ACE), thermal snapshot, with the
    oracle's forces on 1000 seeded atoms: 500 with w > 0 and 500 without."""
    c = synth.configs.cu_slab(sigma=0.066)
    reg = c["region"]
    d = np.linalg.norm(c["x"] - np.asarray(reg["center"]), axis=1)
    rng = np.random.default_rng(3003)
    ace = np.where(d < reg["r_in"] + reg["r_sw"])[0]
    rest = np.where(d >= reg["r_in"] + reg["r_sw"])[0]
    cen = np.concatenate([rng.choice(ace, 500, replace=False), rng.choice(rest, 500, replace=False)])
    # a sampled atom's force needs the energies of every atom within the cutoff of it
    ext = _with_neighbours(c, cen, 5.0 + 1e-6)
    ref = orc.evaluate(c["x"], c["box"], c["eam"], c["ace"], reg, c["indenter"], centers=ext)
    assert ref["status"] == 0
    ext_a = _with_neighbours(c, cen[:500], 5.0 + 1e-6)
    ace_only = orc.evaluate(c["x"], c["box"], None, c["ace"], {"kind": "const", "w": 1.0}, centers=ext_a)
    return c, cen, ref["forces"][cen], np.abs(ace_only["forces"][cen[:500]]).max()


def _with_neighbours(c, idx, rc):
    """idx and every atom within rc of one of them (periodic in x and y, open in z)."""
    from scipy.spatial import cKDTree
    h = np.asarray(c["box"]["h"]).reshape(3, 3)
    L = np.diag(h)
    y = c["x"] - np.asarray(c["box"]["origin"])
    y[:, :2] = np.mod(y[:, :2], L[:2])
    y[:, 2] -= y[:, 2].min()
    tree = cKDTree(y, boxsize=[L[0], L[1], 1e9])
    near = tree.query_ball_point(y[idx], r=rc)
    return np.unique(np.concatenate([np.asarray(idx)] + [np.asarray(v, dtype=np.int64) for v in near]))


@pytest.mark.parametrize("mode", ["fp64", "fp32", "tf32x3", "bf16", "fp16"])
def test_full_size_cu_slab_sampled(apl, slab, mode):
    import torch
    c, cen, fref, fscale = slab
    n = len(c["x"])
    with apl.APContext(c["eam"], c["ace"], c["box"], c["x"], c["v"], c["fixed"], c["region"], c["indenter"],
                       c["ind_vel"], c["mass"], precision=mode) as ctx:
        out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        ctx.compute_forces(None, out)
        ctx.check()
        F = out.cpu().numpy().astype(np.float64)[cen]
    dF = np.abs(F - fref).max()
    print("mode %-7s 2M-atom Cu slab, 1000 sampled atoms: max|dF| = %.3e eV/A (ACE force scale %.2f)"
          % (mode, dF, fscale))
    if mode in U:
        assert dF <= 10 * 2 * U[mode] * fscale
    else:
        assert dF <= 1e-4


@pytest.mark.parametrize("mode", ["fp64", "fp32", "tf32x3", "bf16", "fp16"])
def test_nve_drift_per_precision_mode(apl, mode):
    """NVE energy drift per ps of each A_nlm precision mode: a W (001) slab with the ACE
    hemisphere (geometric weights, so the -grad w force is part of the dynamics), 300 K, no
    indenter, fixed bottom layers, 1000 steps of 1 fs.  The drift is the slope of a
    least-squares line through the total energy sampled every 50 steps.  Velocity Verlet
    keeps the energy of an exact gradient to O(dt^2) without drift; FP32 forces add
    rounding noise (~1e-7 relative), which random-walks the energy by far less than 1e-5
    eV/atom per ps.  BF16 and FP16 round A to 2u relative (u = 2^-9, 2^-12), so their forces
    are not the exact gradient of the energy they report: their bars are 2u times the ACE
    force scale (~1 eV/A) times the ~0.01 A/fs velocity scale times 1000 fs, over 10."""
    c = synth.configs.w_slab(ncell=8, nz=8, r_in=6.0, r_sw=3.0)
    n = len(c["x"])
    with apl.APContext(c["eam"], c["ace"], c["box"], c["x"], c["v"], c["fixed"], c["region"], None, None, c["mass"],
                       precision=mode) as ctx:
        ctx.compute_forces()
        r = ctx.energy()
        ts, es = [0.0], [(r["e_total"] + r["e_kin"]) / n]
        for _ in range(20):
            ctx.step(50, 1.0)
            r = ctx.energy()
            ts.append(r["time_fs"])
            es.append((r["e_total"] + r["e_kin"]) / n)
    slope = np.polyfit(np.asarray(ts) / 1000.0, np.asarray(es), 1)[0]
    dev = np.abs(np.asarray(es) - es[0]).max()
    print("mode %-7s NVE drift %.3e eV/atom/ps, max deviation %.3e eV/atom" % (mode, slope, dev))
    bar = 2 * U[mode] * 1.0 * 0.01 * 1000 / 10 if mode in U else 1e-5
    assert abs(slope) <= bar, (slope, bar)
    assert dev <= max(bar, 2e-4)
