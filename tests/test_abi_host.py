"""CPU checks of the CUDA library's boundary and host logic (no GPU compute).

The library must load, export every function include/ap.h declares, and its host-side
table generators must agree with the oracle's independent routes: the Racah-formula
Gaunt coefficients with the oracle's quadrature, the FP64 re-expanded EAM polynomials
with the oracle's direct evaluation of the Appendix B forms.
"""
import ctypes as C

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def apl():
    import paper_2505_12958_gb300 as ap
    ap.build()
    return ap


def test_library_exports_every_declared_symbol(apl):
    from paper_2505_12958_gb300 import _capi
    names = _capi.header_symbols()
    assert len(names) >= 20
    L = C.CDLL(_capi.LIBPATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert _capi.lib().ap_version() == 1


def test_library_exports_no_undeclared_c_symbols(apl):
    """Every unmangled function the library exports is one include/ap.h declares: the
    library's internal helpers have file or C++ namespace scope and cannot clash with another
    library's symbols."""
    import shutil
    import subprocess
    from paper_2505_12958_gb300 import _capi
    if shutil.which("nm") is None:
        pytest.skip("nm is not installed")
    out = subprocess.run(["nm", "-D", "--defined-only", _capi.LIBPATH], capture_output=True, text=True, check=True).stdout
    exported = {parts[2] for parts in (line.split() for line in out.splitlines())
                if len(parts) == 3 and parts[1] == "T" and not parts[2].startswith("_Z")}
    undeclared = sorted(exported - set(_capi.header_symbols()))
    assert not undeclared, undeclared


def test_gaunt_racah_matches_oracle_quadrature(apl, orc):
    worst = 0.0
    for l1 in range(5):
        for l2 in range(5):
            for l3 in range(5):
                for m1 in range(-l1, l1 + 1):
                    for m2 in range(-l2, l2 + 1):
                        for m3 in range(-l3, l3 + 1):
                            a = apl.gaunt_real(l1, m1, l2, m2, l3, m3)
                            b = orc.gaunt(l1, m1, l2, m2, l3, m3)
                            worst = max(worst, abs(a - b))
    assert worst < 1e-13


@pytest.mark.parametrize("species", ["W", "Cu"])
def test_eam_tables_match_oracle_forms(apl, orc, species):
    eam = synth.eam_potential(species)
    r = np.concatenate([np.linspace(0.5, 6.0, 1500), [2.74451, 2.74456, 2.7445, 2.7446, 2.46396652011306, 1.10002200044,
                                                    2.10004200084, 4.9, 5.45078]])
    ref = orc.eam_funcs(eam, r)
    for k, rr in enumerate(r):
        f, df = apl.eam_table_eval(eam, 0, rr)
        scale = max(1.0, abs(ref[k, 0]))
        assert abs(f - ref[k, 0]) < 1e-10 * scale and abs(df - ref[k, 1]) < 1e-9 * max(1.0, abs(ref[k, 1])), (rr, f, ref[k])
        f, df = apl.eam_table_eval(eam, 1, rr)
        assert abs(f - ref[k, 2]) < 1e-12 and abs(df - ref[k, 3]) < 1e-11, (rr, f, ref[k])


def test_init_rejects_bad_arguments_without_a_gpu(apl):
    # ap_init validates before touching the device: a missing position array is AP_ERR_ARG
    from paper_2505_12958_gb300 import _capi
    c = synth.configs.w_bulk(3)
    p, keep = apl.potential_struct(c["eam"], c["ace"], c["mass"])
    b = _capi.Box()
    h = C.c_void_p()
    st = _capi.lib().ap_init(C.byref(p), C.byref(b), None, None, 10, None, None, None, None, C.byref(h))
    assert st == _capi.AP_ERR_ARG
    p.ace_precision = 7
    x = np.zeros((10, 3))
    st = _capi.lib().ap_init(C.byref(p), C.byref(b), None, None, 10, x.ctypes.data_as(_capi.PD), None, None,
                             None, C.byref(h))
    assert st == _capi.AP_ERR_ARG
    assert len(_capi.lib().ap_last_error(None)) > 0


def test_footprint_estimate_scales_with_atoms(apl):
    from paper_2505_12958_gb300 import _capi
    c = synth.configs.w_bulk(3)
    p, keep = apl.potential_struct(c["eam"], c["ace"], c["mass"])
    a = _capi.lib().ap_footprint_bytes(C.byref(p), 1000, 0.1)
    b = _capi.lib().ap_footprint_bytes(C.byref(p), 2000, 0.1)
    # per atom: the two [25][8] FP32 ACE arrays (1600 B), the list rows and ~300 B of state
    assert 0 < a < b and 2_000_000 < (b - a) < 4_000_000


@pytest.mark.parametrize("species", ["W", "Cu"])
def test_fp32_device_table_lookup_matches_oracle(apl, orc, species):
    """The FP32 table the kernels read, through their own segment lookup (one bin record and
    two compares), on a dense grid and a few ulp either side of every breakpoint."""
    eam = synth.eam_potential(species)
    knots = list(eam["phi_d"]) + list(eam["rho_d"])
    if eam.get("zbl"):
        knots += [eam["r_lo"], eam["r_hi"]]
    if eam.get("rho_rclamp", 0.0) > 0.0:
        knots.append(eam["rho_rclamp"])
    rng = np.random.default_rng(7)
    r = [np.linspace(0.6, 5.5, 4000), rng.uniform(0.6, 5.5, 2000)]
    for d in knots:
        f = np.float32(d)
        r.append(np.array([np.nextafter(f, np.float32(0) if k < 0 else np.float32(10), dtype=np.float32)
                           if k else f for k in (-1, 0, 1)], dtype=np.float64))
    r = np.unique(np.concatenate(r).astype(np.float32).astype(np.float64))
    ref = orc.eam_funcs(eam, r)
    for k, rr in enumerate(r):
        f, df = apl.eam_table_eval(eam, 2, rr)
        assert abs(f - ref[k, 0]) <= 2e-6 * max(1.0, abs(ref[k, 0])), (rr, f, ref[k, 0])
        assert abs(df - ref[k, 1]) <= 2e-5 * max(1.0, abs(ref[k, 1])), (rr, df, ref[k, 1])
        f, df = apl.eam_table_eval(eam, 3, rr)
        assert abs(f - ref[k, 2]) <= 2e-6 * max(1.0, abs(ref[k, 2])), (rr, f, ref[k, 2])
        assert abs(df - ref[k, 3]) <= 2e-5 * max(1.0, abs(ref[k, 3])), (rr, df, ref[k, 3])
