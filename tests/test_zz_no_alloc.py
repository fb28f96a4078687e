"""The allocation-free ACE entry point (ap_ace_forces_noalloc) against the context path.

Callers that cannot allocate device memory (their GPU memory belongs to another
allocator, or their step loop forbids cudaMalloc) pass neighbour lists in and get ACE
forces and energies out; the library's scratch lives in a static device array.  This
test calls the entry point through the C ABI twice in a row on the same inputs and
checks both results against ap_compute_forces on a pure-ACE context (w = 1), within the
parity tolerances (1e-4 eV/A, 1e-6 eV/atom).
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _neighbor_lists(x, L, rc, max_nb):
    n = len(x)
    d = x[None, :, :] - x[:, None, :]
    d -= L * np.round(d / L)                      # cubic periodic box, L > 2 rc
    r = np.linalg.norm(d, axis=2)
    np.fill_diagonal(r, np.inf)
    idx = -np.ones((n, max_nb), dtype=np.int32)
    vec = np.zeros((n, max_nb, 3), dtype=np.float32)
    for i in range(n):
        js = np.where(r[i] < rc + 0.5)[0]
        assert len(js) <= max_nb
        idx[i, :len(js)] = js
        vec[i, :len(js)] = d[i, js]
    return idx, vec


def test_noalloc_matches_context_path_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    from paper_2505_12958_gb300 import _capi
    ap.build()
    c = synth.configs.w_bulk(ncell=5)                # 250 atoms, 15.8 A box
    n = len(c["x"])
    L = 5 * 3.165
    with ap.APContext(c["eam"], c["ace"], c["box"], c["x"], None, None, {"kind": "const", "w": 1.0}, None,
                      None, c["mass"]) as ctx:
        ctx.compute_forces()
        rep = ctx.energy()
        f_ref = ctx.forces().astype(np.float64)
    idx, vec = _neighbor_lists(c["x"], L, c["ace"]["rc"], 96)
    d_idx = torch.tensor(idx, device="cuda")
    d_vec = torch.tensor(vec, device="cuda")
    pot, keep = ap.potential_struct(c["eam"], c["ace"], c["mass"])
    for call in range(2):
        d_f = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
        d_e = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        st = _capi.lib().ap_ace_forces_noalloc(C.byref(pot), n, 96, C.c_void_p(d_idx.data_ptr()),
                                               C.c_void_p(d_vec.data_ptr()), None, C.c_void_p(d_f.data_ptr()),
                                               C.c_void_p(d_e.data_ptr()), None)
        assert st == 0
        torch.cuda.synchronize()
        f = d_f.cpu().numpy().astype(np.float64)
        e = d_e.cpu().numpy()
        assert np.abs(f - f_ref).max() <= 1e-4, (call, np.abs(f - f_ref).max())
        assert abs(e.sum() - rep["e_pot"]) / n <= 1e-6, (call, e.sum(), rep["e_pot"])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    from paper_2505_12958_gb300 import _capi
    c = synth.configs.w_bulk(ncell=3)
    pot, keep = ap.potential_struct(c["eam"], c["ace"], c["mass"])
    d = torch.zeros(16, device="cuda")
    for n, m in ((65537, 8), (10, 129)):
        st = _capi.lib().ap_ace_forces_noalloc(C.byref(pot), n, m, C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()),
                                               None, C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()), None)
        assert st == _capi.AP_ERR_ARG


def test_noalloc_weighted_against_oracle_per_atom(orc):
    """Mixed weights (0, fractional, 1): the weighted forces and the unweighted per-atom ACE
    energies against the FP64 oracle (explicit frozen weights, no EAM), on two calls in a
    row with the same potential (the second reuses the uploaded tables)."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    from paper_2505_12958_gb300 import _capi
    ap.build()
    c = synth.configs.w_bulk(ncell=5, seed=77)
    n = len(c["x"])
    L = 5 * 3.165
    w = np.random.default_rng(5).choice([0.0, 0.37, 1.0], size=n)
    ref = orc.evaluate(c["x"], c["box"], None, c["ace"], {"kind": "explicit", "w": w})
    assert ref["status"] == 0
    idx, vec = _neighbor_lists(c["x"], L, c["ace"]["rc"], 96)
    d_idx = torch.tensor(idx, device="cuda")
    d_vec = torch.tensor(vec, device="cuda")
    d_w = torch.tensor(w, dtype=torch.float32, device="cuda")
    pot, keep = ap.potential_struct(c["eam"], c["ace"], c["mass"])
    for call in range(2):
        d_f = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
        d_e = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        st = _capi.lib().ap_ace_forces_noalloc(C.byref(pot), n, 96, C.c_void_p(d_idx.data_ptr()),
                                               C.c_void_p(d_vec.data_ptr()), C.c_void_p(d_w.data_ptr()),
                                               C.c_void_p(d_f.data_ptr()), C.c_void_p(d_e.data_ptr()), None)
        assert st == 0
        torch.cuda.synchronize()
        f = d_f.cpu().numpy().astype(np.float64)
        e = d_e.cpu().numpy()
        assert np.abs(f - ref["forces"]).max() <= 1e-4, (call, np.abs(f - ref["forces"]).max())
        on = w > 0
        assert np.all(e[~on] == 0.0)
        assert np.abs(e[on] - ref["e_ace"][on]).max() <= 2e-5, call
        assert abs((e[on] - ref["e_ace"][on]).mean()) <= 1e-6, call


def test_noalloc_reports_why_it_refused():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    from paper_2505_12958_gb300 import _capi
    c = synth.configs.w_bulk(ncell=3)
    pot, keep = ap.potential_struct(c["eam"], c["ace"], c["mass"], precision="bf16")
    d = torch.zeros(16, device="cuda")
    st = _capi.lib().ap_ace_forces_noalloc(C.byref(pot), 8, 8, C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()),
                                           None, C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()), None)
    assert st == _capi.AP_ERR_ARG
    assert b"AP_ACE_FP32" in _capi.lib().ap_last_error(None)
    pot, keep = ap.potential_struct(c["eam"], c["ace"], c["mass"])
    st = _capi.lib().ap_ace_forces_noalloc(C.byref(pot), 65537, 8, C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()),
                                           None, C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()), None)
    assert st == _capi.AP_ERR_ARG
    assert b"65536" in _capi.lib().ap_last_error(None)


def test_noalloc_refuses_table_upload_under_capture():
    """A call that would upload tables (a potential this device has not seen) while its
    stream is being captured returns AP_ERR_STATE and issues nothing; the same call outside
    the capture then succeeds."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    import paper_2505_12958_gb300 as ap
    from paper_2505_12958_gb300 import _capi
    ap.build()
    c = synth.configs.w_bulk(ncell=4)                # 128 atoms, 12.7 A box
    n = len(c["x"])
    ace = dict(c["ace"])
    ace["c1"] = np.asarray(ace["c1"], dtype=np.float64) * 1.03125      # a potential no other call used
    pot, keep = ap.potential_struct(c["eam"], ace, c["mass"])
    idx, vec = _neighbor_lists(c["x"], 4 * 3.165, c["ace"]["rc"], 96)
    d_idx = torch.tensor(idx, device="cuda")
    d_vec = torch.tensor(vec, device="cuda")
    d_f = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    d_e = torch.zeros((n,), dtype=torch.float64, device="cuda")
    args = (n, 96, C.c_void_p(d_idx.data_ptr()), C.c_void_p(d_vec.data_ptr()), None, C.c_void_p(d_f.data_ptr()),
            C.c_void_p(d_e.data_ptr()))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        st = _capi.lib().ap_ace_forces_noalloc(C.byref(pot), *args, C.c_void_p(s.cuda_stream))
        g.capture_end()
    assert st == _capi.AP_ERR_STATE
    assert b"capture" in _capi.lib().ap_last_error(None)
    st = _capi.lib().ap_ace_forces_noalloc(C.byref(pot), *args, None)
    assert st == 0
    torch.cuda.synchronize()
    assert np.isfinite(d_e.cpu().numpy()).all()
